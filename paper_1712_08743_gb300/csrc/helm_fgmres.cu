// helm_fgmres.cu - kernels of flexible GMRES (right preconditioned), batched
// over right-hand sides with per-RHS masks.
//
// One call of the inner solver runs one FGMRES cycle of at most m Arnoldi steps
// from a zero guess; restarts happen through the FP64 outer refinement, which
// recomputes the true residual. The basis is stored unnormalised: V'_i = s_i V_i
// with V_i orthonormal and 1/s_i kept in FP64 (s_0 = 1), so A Z'_j is written
// straight into slot j+1 and orthogonalised there, and no scaling pass is
// needed. With Z_j = Z'_j / s_j the Arnoldi relation A Z_j = sum_i h_ij V_i holds
// for h_ij = <V'_i, A Z'_j> / (s_i s_j) and h_{j+1,j} = s_{j+1} / s_j; the
// correction is x = sum_j (y_j / s_j) Z'_j. Gram-Schmidt is classical, with a
// second pass always (CGS2), never, or when the first pass removed more than
// 1 - 1/sqrt(2) of the vector's norm (the Daniel-Gragg-Kaufman-Stewart test).
// Dot products accumulate per block in FP64 and the small Hessenberg
// least-squares problem (Givens rotations, back substitution) is solved in FP64
// on the device.
#include "helm_internal.h"

namespace helm {

namespace {
constexpr int kChunk = 8;                                          // Arnoldi vectors per block in the dot products
constexpr int kMaxChunks = (kMaxRestart - 1 + kChunk) / kChunk;     // chunks of the longest basis
constexpr int kFgMaxBlocks = 1024;                                 // blocks per RHS (and chunk)

// Blocks per RHS of a grid-stride kernel: about two points per thread, at most
// one wave of the kernel's resident blocks on every SM.
template <auto Kernel>
int fg_grid(size_t n) {
    // resident blocks per SM of this kernel, looked up once (a function-local static is
    // initialised exactly once even when serving threads get here together)
    static const int per_sm = [] {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, Kernel, 256, 0);
        return nb > 0 ? nb : 1;
    }();
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t cap = std::min<size_t>(kFgMaxBlocks, (size_t)std::max(1, per_sm * sms));
    return (int)std::max<size_t>(1, std::min<size_t>((n + 511) / 512, cap));
}
}  // namespace

// Partials per RHS that the FGMRES kernels need on n points: 2 kChunk + 1 sums
// per block and chunk in the dot products, the most of any of them.
int fg_partials(size_t n) {
    return (2 * kChunk + 1) * kMaxChunks * (int)std::min<size_t>(kFgMaxBlocks, std::max<size_t>(1, (n + 511) / 512));
}

// ||rin||; beta = g[0], s_0 = 1; the RHS iterates if its outer step is active
// and rin != 0.
template <typename T>
__global__ void __launch_bounds__(256) k_fg_norm(const T* __restrict__ rin, double* partials, int pstride,
                                                 RhsState* st, FgDev fg, int* nactive, size_t n) {
    __shared__ double sh[32];
    const int b = blockIdx.z;
    if (!st[b].outer_active) return;
    T a0 = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const cx<T> c = ldc(rin, n * b + i);
        a0 += c.re * c.re + c.im * c.im;
    }
    const T vv[1] = {a0};
    double acc[1];
    if (last_block_reduce_t<1, T>(vv, acc, sh, partials + (size_t)b * pstride, gridDim.x, blockIdx.x, &st[b].counter[1])) {
        if (threadIdx.x == 0) {
            RhsState& S = st[b];
            S.bnorm2 = acc[0];
            S.rnorm2 = acc[0];
            S.kfg = 0;
            S.reorth = 0;
            S.flag = FLAG_RUNNING;
            S.active = acc[0] > 0.0;
            fg.g[(size_t)b * (fg.m + 1)] = make_double2(sqrt(acc[0]), 0.0);
            fg.sinv[(size_t)b * (fg.m + 1)] = 1.0;
            if (S.active) atomicAdd(nactive, 1);
        }
    }
}

// V'_0 = rin / beta.
template <typename T>
__global__ void k_fg_scale(const T* __restrict__ rin, T* __restrict__ v, const RhsState* st, FgDev fg, size_t n) {
    const int b = blockIdx.z;
    if (!st[b].active) return;
    const T inv = (T)(1.0 / fg.g[(size_t)b * (fg.m + 1)].x);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        stc(v, n * b + i, inv * ldc(rin, n * b + i));
}

// d_i = <V'_i, w> for i <= j (w = A Z'_j, unnormalised, in basis slot j+1);
// blockIdx.y picks a chunk of NV vectors (NV = the smallest of 1, 2, 4, 8 that
// covers j + 1, else 8). The last block of the RHS writes the projection
// coefficients tmp_i = d_i / s_i^2 and sets (add = 0) or adds (add = 1)
// h_ij = d_i / (s_i s_j) into column j of H. With `wnorm` the chunk-0 blocks also
// sum ||w||^2 into wn2 (for the second-pass test). With `check` an RHS whose
// first pass asked for no second pass skips the kernel.
template <typename T, int NV>
__global__ void __launch_bounds__(256) k_fg_dots(const T* __restrict__ V, size_t vstride, const T* __restrict__ w,
                                                 int j, int add, int wnorm, int check, double* partials, int pstride,
                                                 RhsState* st, FgDev fg, size_t n) {
    constexpr int NA = 2 * NV + 1;
    __shared__ double sh[NA][33];
    __shared__ int s_last;
    const int b = blockIdx.z;
    if (!st[b].active || (check && !st[b].reorth)) return;
    const int i0 = blockIdx.y * NV;
    const int nv = min(NV, j + 1 - i0);
    const bool wn = wnorm && blockIdx.y == 0;
    // basis vectors of this chunk (slots past nv alias the first: never used)
    const T* vp[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) vp[k] = V + 2 * (vstride * (size_t)(i0 + (k < nv ? k : 0)) + n * b);
    const T* wb = w + 2 * n * b;
    T acc[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) acc[k] = 0;
    // two points per thread and step, every load of the step issued before use
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    for (; p + stride < n; p += 2 * stride) {
        const cx<T> w0 = ldc(wb, p), w1 = ldc(wb, p + stride);
        cx<T> q0[NV], q1[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k)
            if (k < nv) { q0[k] = ldc(vp[k], p); q1[k] = ldc(vp[k], p + stride); }
#pragma unroll
        for (int k = 0; k < NV; ++k)
            if (k < nv) {
                acc[2 * k] += (q0[k].re * w0.re + q0[k].im * w0.im) + (q1[k].re * w1.re + q1[k].im * w1.im);
                acc[2 * k + 1] += (q0[k].re * w0.im - q0[k].im * w0.re) + (q1[k].re * w1.im - q1[k].im * w1.re);
            }
        if (wn) acc[2 * NV] += (w0.re * w0.re + w0.im * w0.im) + (w1.re * w1.re + w1.im * w1.im);
    }
    if (p < n) {
        const cx<T> w0 = ldc(wb, p);
#pragma unroll
        for (int k = 0; k < NV; ++k)
            if (k < nv) {
                const cx<T> q = ldc(vp[k], p);
                acc[2 * k] += q.re * w0.re + q.im * w0.im;
                acc[2 * k + 1] += q.re * w0.im - q.im * w0.re;
            }
        if (wn) acc[2 * NV] += w0.re * w0.re + w0.im * w0.im;
    }
    // block reduction of the partial sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NA; ++k) {
        T v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[k][warp] = (double)v;
    }
    __syncthreads();
    const int nblk = gridDim.x * gridDim.y, blk = blockIdx.y * gridDim.x + blockIdx.x;
    double* part = partials + (size_t)b * pstride;
    if (threadIdx.x < NA) {
        // the eight warp totals (256 threads) by a fixed pairwise tree
        double w8[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) w8[q] = sh[threadIdx.x][q];
#pragma unroll
        for (int w = 4; w > 0; w >>= 1)
#pragma unroll
            for (int q = 0; q < w; ++q) w8[q] += w8[q + w];
        part[(size_t)threadIdx.x * nblk + blk] = w8[0];
    }
    (void)nw;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&st[b].counter[2], 1u) == (unsigned)(nblk - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last block: one warp per basis vector i <= j (and one more for ||w||^2)
    // sums the partials of the x-blocks of its chunk, lane-strided then by a fixed
    // shuffle tree (the order does not depend on timing, so the result is
    // deterministic)
    const int nx = gridDim.x;
    const size_t col = (size_t)b * (fg.m + 1);
    const double* sinv = fg.sinv + col;
    const int nsum = j + 1 + (wnorm ? 1 : 0);
    for (int i = warp; i < nsum; i += nw) {
        const bool isn = i > j;
        const int c = isn ? 0 : i / NV, k = isn ? NV : i % NV;
        const double* pre = part + (size_t)(2 * k) * nblk + (size_t)c * nx;
        const double* pim = part + (size_t)(2 * k + 1) * nblk + (size_t)c * nx;
        // eight loads per lane in flight, summed by a fixed pairwise tree (three
        // dependent FP64 additions per batch instead of eight)
        double re = 0.0, im = 0.0;
        for (int x0 = 0; x0 < nx; x0 += 256) {
            double vr[8], vi[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int x = x0 + lane + 32 * t;
                vr[t] = x < nx ? __ldcg(pre + x) : 0.0;
                vi[t] = (x < nx && !isn) ? __ldcg(pim + x) : 0.0;
            }
#pragma unroll
            for (int w = 4; w > 0; w >>= 1)
#pragma unroll
                for (int t = 0; t < w; ++t) { vr[t] += vr[t + w]; vi[t] += vi[t + w]; }
            re += vr[0];
            im += vi[0];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (lane == 0) {
            if (isn) {
                fg.wn2[b] = re;
            } else {
                const double si = sinv[i], inv2 = si * si, invh = si * sinv[j];
                fg.tmp[col + i] = make_double2(re * inv2, im * inv2);
                double2& h = fg.H[(col + i) * fg.m + j];
                if (add) { h.x += re * invh; h.y += im * invh; } else { h = make_double2(re * invh, im * invh); }
            }
        }
    }
    if (threadIdx.x == 0) st[b].counter[2] = 0u;
}

// Column j of the Arnoldi relation is complete (||w'|| = hn2^(1/2) after the
// last pass): 1/s_{j+1}, h_{j+1,j} = s_{j+1} / s_j, the previous Givens
// rotations on column j, the new rotation zeroing h_{j+1,j}, and the
// convergence test |g_{j+1}| <= tol_rel * beta. Called by every thread of one
// block: the column and the rotations are staged in shared memory, so the
// serial FP64 chain of thread 0 waits on no global load; it takes three square
// roots and two divisions.
__device__ void fg_finish_column(RhsState& S, const FgDev& fg, int b, int j, double hn2, int* nactive) {
    __shared__ double2 hc[kMaxRestart + 1];
    __shared__ double2 sc[kMaxRestart];
    __shared__ double cc[kMaxRestart];
    const int m = fg.m;
    const size_t col = (size_t)b * (m + 1);
    double2* H = fg.H + col * m;                   // H[i * m + j]
    for (int i = threadIdx.x; i <= j; i += blockDim.x) hc[i] = H[(size_t)i * m + j];
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        cc[i] = fg.cs[(size_t)b * m + i];
        sc[i] = fg.sn[(size_t)b * m + i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double sn1 = sqrt(hn2);
        fg.sinv[col + j + 1] = sn1 > 0.0 ? 1.0 / sn1 : 0.0;
        const double hn = sn1 * fg.sinv[col + j];
        // previous rotations on column j: [a; d] <- [c a + s d; -conj(s) a + c d]
        double2 a = hc[0];
        for (int i = 0; i < j; ++i) {
            const double c = cc[i];
            const double2 sv = sc[i], d = hc[i + 1];
            hc[i] = make_double2(c * a.x + sv.x * d.x - sv.y * d.y, c * a.y + sv.x * d.y + sv.y * d.x);
            a = make_double2(-(sv.x * a.x + sv.y * a.y) + c * d.x, -(sv.x * a.y - sv.y * a.x) + c * d.y);
        }
        // new rotation zeroing h_{j+1,j}: c = |a| / t, s = (a / |a|) h / t, t = (|a|^2 + h^2)^(1/2)
        const double a2 = a.x * a.x + a.y * a.y, t2 = a2 + hn * hn;
        double c;
        double2 sv, hjj;
        if (a2 == 0.0) { c = 0.0; sv = make_double2(1.0, 0.0); hjj = make_double2(hn, 0.0); }
        else {
            const double inv = 1.0 / (sqrt(a2) * sqrt(t2));   // 1 / (|a| t)
            c = a2 * inv;
            sv = make_double2(a.x * hn * inv, a.y * hn * inv);
            hjj = make_double2(a.x * t2 * inv, a.y * t2 * inv);   // (a / |a|) t
        }
        hc[j] = hjj;
        fg.cs[(size_t)b * m + j] = c;
        fg.sn[(size_t)b * m + j] = sv;
        double2* g = fg.g + col;
        const double2 gj = g[j];
        const double2 g1 = make_double2(-(sv.x * gj.x + sv.y * gj.y), -(sv.x * gj.y - sv.y * gj.x));   // -conj(s) g_j
        g[j + 1] = g1;
        g[j] = make_double2(c * gj.x, c * gj.y);
        S.kfg = j + 1;
        S.iters += 1;
        const double res2 = g1.x * g1.x + g1.y * g1.y;
        S.rnorm2 = res2;
        int done = 0;
        if (res2 <= S.tol_rel * S.tol_rel * S.bnorm2 || hn == 0.0) { done = 1; S.flag = FLAG_CONVERGED; }
        else if (j + 1 >= m) { done = 1; S.flag = FLAG_MAXIT; }
        else if (S.iters >= S.max_it) { done = 1; S.flag = FLAG_MAXIT; }
        if (done) { S.active = 0; atomicSub(nactive, 1); }
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j; i += blockDim.x) H[(size_t)i * m + j] = hc[i];
    if (threadIdx.x == 0) H[(size_t)(j + 1) * m + j] = make_double2(0.0, 0.0);
}

// w -= sum_{i <= j} tmp_i V'_i in place (w is basis slot j+1). mode 0: no norm
// (a second pass follows); mode 1: ||w||^2 and the column is finished; mode 2:
// ||w||^2, then a second pass is requested (S.reorth = 1) if ||w||^2 < wn2 / 2,
// else the column is finished; mode 3: each block writes its part of ||w||^2
// and k_fg_finish finishes the column (off the critical path). With `check` an
// RHS whose first pass asked for no second pass skips the kernel.
template <typename T, int NV>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_fg_axpy(const T* __restrict__ V, size_t vstride, T* __restrict__ w, int j,
                                                 int mode, int check, double* partials, int pstride, RhsState* st,
                                                 FgDev fg, int* nactive, size_t n) {
    __shared__ double sh[32];
    __shared__ cx<T> coef[kMaxRestart + 1];
    const int b = blockIdx.z;
    if (!st[b].active || (check && !st[b].reorth)) return;
    const size_t col = (size_t)b * (fg.m + 1);
    for (int i = threadIdx.x; i <= j; i += blockDim.x) coef[i] = cx<T>((T)fg.tmp[col + i].x, (T)fg.tmp[col + i].y);
    __syncthreads();
    T a0 = 0;
    T* wb = w + 2 * n * b;
    const T* vb = V + 2 * n * b;
    // two points per thread and step; the basis in chunks of NV vectors, every
    // load of a chunk issued before use
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    for (; p + stride < n; p += 2 * stride) {
        cx<T> w0 = ldcc(wb, p), w1 = ldcc(wb, p + stride);
        for (int i0 = 0; i0 <= j; i0 += NV) {
            const int nv = min(NV, j + 1 - i0);
            cx<T> q0[NV], q1[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k)
                if (k < nv) {
                    const T* v = vb + 2 * vstride * (size_t)(i0 + k);
                    q0[k] = ldc(v, p);
                    q1[k] = ldc(v, p + stride);
                }
#pragma unroll
            for (int k = 0; k < NV; ++k)
                if (k < nv) { w0 = w0 - coef[i0 + k] * q0[k]; w1 = w1 - coef[i0 + k] * q1[k]; }
        }
        stc(wb, p, w0);
        stc(wb, p + stride, w1);
        a0 += (w0.re * w0.re + w0.im * w0.im) + (w1.re * w1.re + w1.im * w1.im);
    }
    if (p < n) {
        cx<T> w0 = ldcc(wb, p);
        for (int i = 0; i <= j; ++i) w0 = w0 - coef[i] * ldc(vb + 2 * vstride * (size_t)i, p);
        stc(wb, p, w0);
        a0 += w0.re * w0.re + w0.im * w0.im;
    }
    if (mode == 0) return;
    const T vv[1] = {a0};
    double acc[1];
    if (mode == 3) {
        block_sum_t<1, T>(vv, acc, sh);
        if (threadIdx.x == 0) partials[(size_t)b * pstride + blockIdx.x] = acc[0];
        return;
    }
    if (last_block_reduce_t<1, T>(vv, acc, sh, partials + (size_t)b * pstride, gridDim.x, blockIdx.x, &st[b].counter[0])) {
        __shared__ int s_finish;
        __shared__ double s_hn2;
        if (threadIdx.x == 0) {
            const int second = mode == 2 && acc[0] < 0.5 * fg.wn2[b];
            st[b].reorth = second;
            s_finish = !second;
            s_hn2 = acc[0];
        }
        __syncthreads();
        if (s_finish) fg_finish_column(st[b], fg, b, j, s_hn2, nactive);
    }
}

// Finishes column j from the per-block parts of ||w||^2 that k_fg_axpy (mode 3)
// wrote: one block per RHS sums the nblk parts in a fixed order, then
// fg_finish_column. Runs on a second stream, beside the next preconditioner
// application, which reads only w.
__global__ void __launch_bounds__(256) k_fg_finish(const double* partials, int pstride, int nblk, RhsState* st,
                                                   FgDev fg, int j, int* nactive) {
    __shared__ double sh[32];
    __shared__ double s_hn2;
    const int b = blockIdx.x;
    if (!st[b].active) return;
    const double* part = partials + (size_t)b * pstride;
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) v[0] += __ldcg(part + i);
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) s_hn2 = v[0];
    __syncthreads();
    fg_finish_column(st[b], fg, b, j, s_hn2, nactive);
}

// y = R^{-1} g on the k = kfg leading rows (FP64), one warp per RHS: the warp
// stages the triangle and g in shared memory with all its loads in flight, then
// lane 0 substitutes backwards.
__global__ void __launch_bounds__(32) k_fg_backsolve(const RhsState* st, FgDev fg) {
    // y = R^-1 g by columns: lane q holds the right-hand side entry q; at step i the lane
    // holding row i finishes y_i with the reciprocal of R_ii (all reciprocals formed
    // together beforehand, so no division sits on the chain) and every lane q < i
    // subtracts R_qi y_i. The chain is k steps of one complex product, one shuffle and
    // one complex multiply-add in FP64, instead of k divisions and k (k - 1) / 2
    // sequential multiply-adds on one thread.
    const int b = blockIdx.x;
    if (!st[b].outer_active) return;
    const int m = fg.m, k = st[b].kfg, lane = threadIdx.x;   // k <= kMaxRestart = 32
    const size_t col = (size_t)b * (m + 1);
    const double2* H = fg.H + col * m;
    __shared__ double2 R[kMaxRestart][kMaxRestart + 1];   // the triangle, staged once
    for (int idx = lane; idx < k * k; idx += 32) {
        const int i = idx / k, q = idx - i * k;
        if (q >= i) R[i][q] = H[(size_t)i * m + q];
    }
    __syncwarp();
    double2 acc = lane < k ? fg.g[col + lane] : make_double2(0.0, 0.0);
    double2 rinv = make_double2(0.0, 0.0);
    if (lane < k) {
        const double2 d = R[lane][lane];
        const double dd = d.x * d.x + d.y * d.y;
        if (dd > 0.0) {
            const double inv = 1.0 / dd;
            rinv = make_double2(d.x * inv, -d.y * inv);
        }
    }
    double2* y = fg.y + (size_t)b * m;
    for (int i = k - 1; i >= 0; --i) {
        double2 yi = make_double2(acc.x * rinv.x - acc.y * rinv.y, acc.x * rinv.y + acc.y * rinv.x);
        yi.x = __shfl_sync(0xffffffffu, yi.x, i);
        yi.y = __shfl_sync(0xffffffffu, yi.y, i);
        if (lane == i) y[i] = yi;
        if (lane < i) {
            const double2 h = R[lane][i];
            acc.x -= h.x * yi.x - h.y * yi.y;
            acc.y -= h.x * yi.y + h.y * yi.x;
        }
    }
}

// x = sum_{i < kfg} (y_i / s_i) Z'_i for every RHS whose outer step is active.
template <typename T>
__global__ void k_fg_update(const T* __restrict__ Z, size_t zstride, T* __restrict__ x, const RhsState* st, FgDev fg,
                            size_t n) {
    __shared__ cx<T> coef[kMaxRestart];
    const int b = blockIdx.z;
    if (!st[b].outer_active) return;
    const int k = st[b].kfg;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const double2 y = fg.y[(size_t)b * fg.m + i];
        const double inv = fg.sinv[(size_t)b * (fg.m + 1) + i];
        coef[i] = cx<T>((T)(y.x * inv), (T)(y.y * inv));
    }
    __syncthreads();
    const T* zb = Z + 2 * n * b;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        cx<T> acc(0, 0);
        for (int i0 = 0; i0 < k; i0 += kChunk) {
            const int nv = min(kChunk, k - i0);
            cx<T> q[kChunk];
#pragma unroll
            for (int t = 0; t < kChunk; ++t)
                if (t < nv) q[t] = ldc(zb + 2 * zstride * (size_t)(i0 + t), p);
#pragma unroll
            for (int t = 0; t < kChunk; ++t)
                if (t < nv) acc = acc + coef[i0 + t] * q[t];
        }
        stc(x, n * b + p, acc);
    }
}

// ------------------------------------------------------------- launchers
template <typename T>
void launch_fg_norm(const T* rin, double* partials, int pstride, RhsState* st, const FgDev& fg, int* nactive,
                    size_t n, int nrhs, cudaStream_t s) {
    ProfScope prof(PK_FG_NORM, (int)n, 1, (double)n * nrhs * 2.0 * sizeof(T), s);
    k_fg_norm<T><<<dim3(fg_grid<k_fg_norm<T>>(n), 1, nrhs), 256, 0, s>>>(rin, partials, pstride, st, fg, nactive, n);
}
template <typename T>
void launch_fg_scale(const T* rin, T* v, const RhsState* st, const FgDev& fg, size_t n, int nrhs, cudaStream_t s) {
    ProfScope prof(PK_FG_SCALE, (int)n, 1, (double)n * nrhs * 4.0 * sizeof(T), s);
    k_fg_scale<T><<<dim3(fg_grid<k_fg_scale<T>>(n), 1, nrhs), 256, 0, s>>>(rin, v, st, fg, n);
}
template <typename T, int NV>
static void fg_dots_nv(const T* V, size_t vstride, const T* w, int j, int add, int wnorm, int check, double* partials,
                       int pstride, RhsState* st, const FgDev& fg, size_t n, int nrhs, cudaStream_t s) {
    const int nchunk = (j + NV) / NV;
    k_fg_dots<T, NV><<<dim3(fg_grid<k_fg_dots<T, NV>>(n), nchunk, nrhs), 256, 0, s>>>(
        V, vstride, w, j, add, wnorm, check, partials, pstride, st, fg, n);
}
template <typename T>
void launch_fg_dots(const T* V, size_t vstride, const T* w, int j, int add, int wnorm, int check, double* partials,
                    int pstride, RhsState* st, const FgDev& fg, size_t n, int nrhs, cudaStream_t s) {
    // reads w and the basis vectors V'_0 .. V'_j
    ProfScope prof(PK_FG_DOTS, (int)n, 1, (double)n * nrhs * 2.0 * sizeof(T) * (j + 2), s);
    if (j < 1) fg_dots_nv<T, 1>(V, vstride, w, j, add, wnorm, check, partials, pstride, st, fg, n, nrhs, s);
    else if (j < 2) fg_dots_nv<T, 2>(V, vstride, w, j, add, wnorm, check, partials, pstride, st, fg, n, nrhs, s);
    else if (j < 4) fg_dots_nv<T, 4>(V, vstride, w, j, add, wnorm, check, partials, pstride, st, fg, n, nrhs, s);
    else if (j < kChunk) fg_dots_nv<T, kChunk>(V, vstride, w, j, add, wnorm, check, partials, pstride, st, fg, n, nrhs, s);
    // 9 .. 12 vectors in one pass over w (two chunks of eight would read w twice, and the second,
    // short chunk would run as a second, light wave)
    else if (j < 12) fg_dots_nv<T, 12>(V, vstride, w, j, add, wnorm, check, partials, pstride, st, fg, n, nrhs, s);
    else fg_dots_nv<T, kChunk>(V, vstride, w, j, add, wnorm, check, partials, pstride, st, fg, n, nrhs, s);
}
template <typename T, int NV>
static int fg_axpy_nv(const T* V, size_t vstride, T* w, int j, int mode, int check, double* partials, int pstride,
                      RhsState* st, const FgDev& fg, int* nactive, size_t n, int nrhs, cudaStream_t s) {
    const int grid = fg_grid<k_fg_axpy<T, NV>>(n);
    k_fg_axpy<T, NV><<<dim3(grid, 1, nrhs), 256, 0, s>>>(V, vstride, w, j, mode, check, partials, pstride, st, fg,
                                                          nactive, n);
    return grid;
}
template <typename T>
int launch_fg_axpy(const T* V, size_t vstride, T* w, int j, int mode, int check, double* partials, int pstride,
                   RhsState* st, const FgDev& fg, int* nactive, size_t n, int nrhs, cudaStream_t s) {
    // reads V'_0 .. V'_j and w, writes w
    ProfScope prof(PK_FG_AXPY, (int)n, 1, (double)n * nrhs * 2.0 * sizeof(T) * (j + 3), s);
    if (j < 1) return fg_axpy_nv<T, 1>(V, vstride, w, j, mode, check, partials, pstride, st, fg, nactive, n, nrhs, s);
    if (j < 2) return fg_axpy_nv<T, 2>(V, vstride, w, j, mode, check, partials, pstride, st, fg, nactive, n, nrhs, s);
    if (j < 4) return fg_axpy_nv<T, 4>(V, vstride, w, j, mode, check, partials, pstride, st, fg, nactive, n, nrhs, s);
    return fg_axpy_nv<T, kChunk>(V, vstride, w, j, mode, check, partials, pstride, st, fg, nactive, n, nrhs, s);
}
void launch_fg_finish(const double* partials, int pstride, int nblk, RhsState* st, const FgDev& fg, int j,
                      int* nactive, int nrhs, cudaStream_t s) {
    ProfScope prof(PK_FG_FINISH, nblk, 1, (double)nblk * nrhs * 8.0 * 2, s);
    k_fg_finish<<<nrhs, 256, 0, s>>>(partials, pstride, nblk, st, fg, j, nactive);
}
void launch_fg_backsolve(const RhsState* st, const FgDev& fg, int nrhs, cudaStream_t s) {
    ProfScope prof(PK_FG_BACKSOLVE, fg.m, 1, (double)fg.m * fg.m * nrhs * 16.0, s);
    k_fg_backsolve<<<nrhs, 32, 0, s>>>(st, fg);
}
template <typename T>
void launch_fg_update(const T* Z, size_t zstride, T* x, const RhsState* st, const FgDev& fg, size_t n, int nrhs,
                      cudaStream_t s) {
    // reads Z'_0 .. Z'_{m-1}, reads and writes x
    ProfScope prof(PK_FG_UPDATE, (int)n, 1, (double)n * nrhs * 2.0 * sizeof(T) * (fg.m + 2), s);
    k_fg_update<T><<<dim3(fg_grid<k_fg_update<T>>(n), 1, nrhs), 256, 0, s>>>(Z, zstride, x, st, fg, n);
}

#define HELM_FG_INST(T)                                                                                             \
    template void launch_fg_norm<T>(const T*, double*, int, RhsState*, const FgDev&, int*, size_t, int,             \
                                    cudaStream_t);                                                                  \
    template void launch_fg_scale<T>(const T*, T*, const RhsState*, const FgDev&, size_t, int, cudaStream_t);       \
    template void launch_fg_dots<T>(const T*, size_t, const T*, int, int, int, int, double*, int, RhsState*,        \
                                    const FgDev&, size_t, int, cudaStream_t);                                       \
    template int launch_fg_axpy<T>(const T*, size_t, T*, int, int, int, double*, int, RhsState*, const FgDev&,      \
                                   int*, size_t, int, cudaStream_t);                                                \
    template void launch_fg_update<T>(const T*, size_t, T*, const RhsState*, const FgDev&, size_t, int,             \
                                      cudaStream_t);
HELM_FG_INST(float)
HELM_FG_INST(double)
#undef HELM_FG_INST

}  // namespace helm

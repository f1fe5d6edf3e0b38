// helm_fgmres.cu - kernels of flexible GMRES (right preconditioned), batched
// over right-hand sides with per-RHS masks.
//
// One call of the inner solver runs one FGMRES cycle of at most m Arnoldi steps
// from a zero guess; restarts happen through the FP64 outer refinement, which
// recomputes the true residual. The Arnoldi vectors are orthogonalised by
// classical Gram-Schmidt with one reorthogonalisation (CGS2); dot products
// accumulate per block in FP64 and the small Hessenberg least-squares problem
// (Givens rotations, back substitution) is solved in FP64 on the device.
#include "helm_internal.h"

namespace helm {

namespace {
inline int grid1d_fg(size_t n) {
    size_t g = (n + 1023) / 1024;
    if (g < 1) g = 1;
    if (g > 512) g = 512;
    return (int)g;
}
constexpr int kChunk = 8;   // Arnoldi vectors per block in the dot-product kernel
}  // namespace

// ||rin||; beta = g[0]; the RHS iterates if its outer step is active and rin != 0.
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
            S.flag = FLAG_RUNNING;
            S.active = acc[0] > 0.0;
            fg.g[(size_t)b * (fg.m + 1)] = make_double2(sqrt(acc[0]), 0.0);
            if (S.active) atomicAdd(nactive, 1);
        }
    }
}

// v = w / scale with scale = g[0] (j < 0: first vector) or the norm of w
// recorded before the rotation of column j.
template <typename T>
__global__ void k_fg_scale(const T* __restrict__ w, T* __restrict__ v, const RhsState* st, FgDev fg, int j,
                           size_t n) {
    const int b = blockIdx.z;
    if (!st[b].active) return;
    __shared__ T s_inv;
    if (threadIdx.x == 0) {
        const double s = j < 0 ? fg.g[(size_t)b * (fg.m + 1)].x : fg.hsub[(size_t)b * fg.m + j];
        s_inv = (T)(1.0 / s);
    }
    __syncthreads();
    const T inv = s_inv;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        stc(v, n * b + i, inv * ldc(w, n * b + i));
}

// h_i = <V_i, w> for i <= j; blockIdx.y picks a chunk of kChunk vectors. The
// last block of the RHS writes tmp = h and sets (add = 0) or adds (add = 1) h
// into column j of H.
template <typename T>
__global__ void __launch_bounds__(256) k_fg_dots(const T* __restrict__ V, size_t vstride, const T* __restrict__ w,
                                                 int j, int add, double* partials, int pstride, RhsState* st,
                                                 FgDev fg, size_t n) {
    __shared__ double sh[2 * kChunk][33];
    __shared__ int s_last;
    const int b = blockIdx.z;
    if (!st[b].active) return;
    const int i0 = blockIdx.y * kChunk;
    T acc[2 * kChunk];
#pragma unroll
    for (int k = 0; k < 2 * kChunk; ++k) acc[k] = 0;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        const cx<T> wv = ldc(w, n * b + p);
#pragma unroll
        for (int k = 0; k < kChunk; ++k) {
            if (i0 + k <= j) {
                const cx<T> q = ldc(V + 2 * vstride * (i0 + k), n * b + p);
                acc[2 * k] += q.re * wv.re + q.im * wv.im;
                acc[2 * k + 1] += q.re * wv.im - q.im * wv.re;
            }
        }
    }
    // block reduction of the 2 * kChunk partial sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < 2 * kChunk; ++k) {
        T v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[k][warp] = (double)v;
    }
    __syncthreads();
    const int nblk = gridDim.x * gridDim.y, blk = blockIdx.y * gridDim.x + blockIdx.x;
    double* part = partials + (size_t)b * pstride;
    if (threadIdx.x < 2 * kChunk) {
        double v = 0.0;
        for (int q = 0; q < nw; ++q) v += sh[threadIdx.x][q];
        part[(size_t)threadIdx.x * nblk + blk] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&st[b].counter[2], 1u) == (unsigned)(nblk - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last block: one warp per basis vector i <= j sums the partials of the
    // x-blocks of its chunk, lane-strided then by a fixed shuffle tree (the order
    // does not depend on timing, so the result is deterministic)
    const int nx = gridDim.x;
    const size_t col = (size_t)b * (fg.m + 1);
    for (int i = warp; i <= j; i += nw) {
        const int c = i / kChunk, k = i % kChunk;
        const double* pre = part + (size_t)(2 * k) * nblk + (size_t)c * nx;
        const double* pim = part + (size_t)(2 * k + 1) * nblk + (size_t)c * nx;
        double re = 0.0, im = 0.0;
        for (int x = lane; x < nx; x += 32) {
            re += __ldcg(pre + x);
            im += __ldcg(pim + x);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (lane == 0) {
            fg.tmp[col + i] = make_double2(re, im);
            double2& h = fg.H[(col + i) * fg.m + j];
            if (add) { h.x += re; h.y += im; } else { h = make_double2(re, im); }
        }
    }
    if (threadIdx.x == 0) st[b].counter[2] = 0u;
}

// w -= sum_{i <= j} tmp_i V_i; with `norm`, also ||w||^2 and, in the last
// block, H[j+1][j] = ||w||, the Givens rotations of column j and the
// convergence test |g_{j+1}| <= tol_rel * beta.
template <typename T>
__global__ void __launch_bounds__(256) k_fg_axpy(const T* __restrict__ V, size_t vstride, T* __restrict__ w, int j,
                                                 int norm, double* partials, int pstride, RhsState* st, FgDev fg,
                                                 int* nactive, size_t n) {
    __shared__ double sh[32];
    __shared__ cx<T> coef[kMaxRestart + 1];
    const int b = blockIdx.z;
    if (!st[b].active) return;
    const size_t col = (size_t)b * (fg.m + 1);
    for (int i = threadIdx.x; i <= j; i += blockDim.x) coef[i] = cx<T>((T)fg.tmp[col + i].x, (T)fg.tmp[col + i].y);
    __syncthreads();
    T a0 = 0;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        cx<T> wv = ldcc(w, n * b + p);
        for (int i = 0; i <= j; ++i) wv = wv - coef[i] * ldc(V + 2 * vstride * i, n * b + p);
        stc(w, n * b + p, wv);
        a0 += wv.re * wv.re + wv.im * wv.im;
    }
    if (!norm) return;
    const T vv[1] = {a0};
    double acc[1];
    if (last_block_reduce_t<1, T>(vv, acc, sh, partials + (size_t)b * pstride, gridDim.x, blockIdx.x, &st[b].counter[0])) {
        if (threadIdx.x == 0) {
            RhsState& S = st[b];
            const int m = fg.m;
            double2* H = fg.H + col * m;                   // H[i * m + j]
            const double hn = sqrt(acc[0]);
            H[(size_t)(j + 1) * m + j] = make_double2(hn, 0.0);
            // previous rotations on column j
            for (int i = 0; i < j; ++i) {
                const double c = fg.cs[(size_t)b * m + i];
                const double2 s = fg.sn[(size_t)b * m + i];
                const double2 a = H[(size_t)i * m + j], d = H[(size_t)(i + 1) * m + j];
                // [a; d] <- [c a + s d; -conj(s) a + c d]
                H[(size_t)i * m + j] = make_double2(c * a.x + s.x * d.x - s.y * d.y, c * a.y + s.x * d.y + s.y * d.x);
                H[(size_t)(i + 1) * m + j] = make_double2(-(s.x * a.x + s.y * a.y) + c * d.x, -(s.x * a.y - s.y * a.x) + c * d.y);
            }
            // new rotation zeroing H[j+1][j]
            const double2 a = H[(size_t)j * m + j];
            const double bb = hn;
            const double an = sqrt(a.x * a.x + a.y * a.y);
            double c;
            double2 s;
            if (an == 0.0) { c = 0.0; s = make_double2(1.0, 0.0); }
            else {
                const double t = sqrt(an * an + bb * bb);
                c = an / t;
                s = make_double2(a.x / an * bb / t, a.y / an * bb / t);   // (a/|a|) conj(b) / t, b real
            }
            fg.cs[(size_t)b * m + j] = c;
            fg.sn[(size_t)b * m + j] = s;
            const double t2 = sqrt(an * an + bb * bb);
            H[(size_t)j * m + j] = an == 0.0 ? make_double2(bb, 0.0) : make_double2(a.x / an * t2, a.y / an * t2);
            H[(size_t)(j + 1) * m + j] = make_double2(0.0, 0.0);
            double2* g = fg.g + col;
            const double2 gj = g[j];
            g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));   // -conj(s) g_j
            g[j] = make_double2(c * gj.x, c * gj.y);
            S.kfg = j + 1;
            S.iters += 1;
            const double res = sqrt(g[j + 1].x * g[j + 1].x + g[j + 1].y * g[j + 1].y);
            S.rnorm2 = res * res;
            // keep H[j+1][j] for the next basis vector's scaling
            fg.hsub[(size_t)b * m + j] = hn;
            int done = 0;
            if (res <= S.tol_rel * sqrt(S.bnorm2) || hn == 0.0) { done = 1; S.flag = FLAG_CONVERGED; }
            else if (j + 1 >= m) { done = 1; S.flag = FLAG_MAXIT; }
            else if (S.iters >= S.max_it) { done = 1; S.flag = FLAG_MAXIT; }
            if (done) { S.active = 0; atomicSub(nactive, 1); }
        }
    }
}

// y = R^{-1} g on the k = kfg leading rows (FP64, one thread per RHS).
__global__ void k_fg_backsolve(const RhsState* st, FgDev fg, int nrhs) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nrhs || !st[b].outer_active) return;
    const int m = fg.m, k = st[b].kfg;
    const size_t col = (size_t)b * (m + 1);
    const double2* H = fg.H + col * m;
    double2* y = fg.y + (size_t)b * m;
    for (int i = k - 1; i >= 0; --i) {
        double2 acc = fg.g[col + i];
        for (int q = i + 1; q < k; ++q) {
            const double2 h = H[(size_t)i * m + q];
            acc.x -= h.x * y[q].x - h.y * y[q].y;
            acc.y -= h.x * y[q].y + h.y * y[q].x;
        }
        const double2 d = H[(size_t)i * m + i];
        const double dd = d.x * d.x + d.y * d.y;
        y[i] = dd > 0.0 ? make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd)
                        : make_double2(0.0, 0.0);
    }
}

// x = sum_{i < kfg} y_i Z_i for every RHS whose outer step is active.
template <typename T>
__global__ void k_fg_update(const T* __restrict__ Z, size_t zstride, T* __restrict__ x, const RhsState* st, FgDev fg,
                            size_t n) {
    __shared__ cx<T> coef[kMaxRestart];
    const int b = blockIdx.z;
    if (!st[b].outer_active) return;
    const int k = st[b].kfg;
    for (int i = threadIdx.x; i < k; i += blockDim.x)
        coef[i] = cx<T>((T)fg.y[(size_t)b * fg.m + i].x, (T)fg.y[(size_t)b * fg.m + i].y);
    __syncthreads();
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        cx<T> acc(0, 0);
        for (int i = 0; i < k; ++i) acc = acc + coef[i] * ldc(Z + 2 * zstride * i, n * b + p);
        stc(x, n * b + p, acc);
    }
}

// ------------------------------------------------------------- launchers
template <typename T>
void launch_fg_norm(const T* rin, double* partials, int pstride, RhsState* st, const FgDev& fg, int* nactive,
                    size_t n, int nrhs, cudaStream_t s) {
    k_fg_norm<T><<<dim3(grid1d_fg(n), 1, nrhs), 256, 0, s>>>(rin, partials, pstride, st, fg, nactive, n);
}
template <typename T>
void launch_fg_scale(const T* w, T* v, const RhsState* st, const FgDev& fg, int j, size_t n, int nrhs,
                     cudaStream_t s) {
    k_fg_scale<T><<<dim3(grid1d_fg(n), 1, nrhs), 256, 0, s>>>(w, v, st, fg, j, n);
}
template <typename T>
void launch_fg_dots(const T* V, size_t vstride, const T* w, int j, int add, double* partials, int pstride,
                    RhsState* st, const FgDev& fg, size_t n, int nrhs, cudaStream_t s) {
    const int nchunk = (j + kChunk) / kChunk;
    k_fg_dots<T><<<dim3(grid1d_fg(n), nchunk, nrhs), 256, 0, s>>>(V, vstride, w, j, add, partials, pstride, st, fg, n);
}
template <typename T>
void launch_fg_axpy(const T* V, size_t vstride, T* w, int j, int norm, double* partials, int pstride, RhsState* st,
                    const FgDev& fg, int* nactive, size_t n, int nrhs, cudaStream_t s) {
    k_fg_axpy<T><<<dim3(grid1d_fg(n), 1, nrhs), 256, 0, s>>>(V, vstride, w, j, norm, partials, pstride, st, fg,
                                                            nactive, n);
}
void launch_fg_backsolve(const RhsState* st, const FgDev& fg, int nrhs, cudaStream_t s) {
    k_fg_backsolve<<<(nrhs + 63) / 64, 64, 0, s>>>(st, fg, nrhs);
}
template <typename T>
void launch_fg_update(const T* Z, size_t zstride, T* x, const RhsState* st, const FgDev& fg, size_t n, int nrhs,
                      cudaStream_t s) {
    k_fg_update<T><<<dim3(grid1d_fg(n), 1, nrhs), 256, 0, s>>>(Z, zstride, x, st, fg, n);
}

#define HELM_FG_INST(T)                                                                                             \
    template void launch_fg_norm<T>(const T*, double*, int, RhsState*, const FgDev&, int*, size_t, int,             \
                                    cudaStream_t);                                                                  \
    template void launch_fg_scale<T>(const T*, T*, const RhsState*, const FgDev&, int, size_t, int, cudaStream_t);  \
    template void launch_fg_dots<T>(const T*, size_t, const T*, int, int, double*, int, RhsState*, const FgDev&,    \
                                    size_t, int, cudaStream_t);                                                     \
    template void launch_fg_axpy<T>(const T*, size_t, T*, int, int, double*, int, RhsState*, const FgDev&, int*,    \
                                    size_t, int, cudaStream_t);                                                     \
    template void launch_fg_update<T>(const T*, size_t, T*, const RhsState*, const FgDev&, size_t, int,             \
                                      cudaStream_t);
HELM_FG_INST(float)
HELM_FG_INST(double)
#undef HELM_FG_INST

}  // namespace helm

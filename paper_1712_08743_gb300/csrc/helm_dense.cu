// helm_dense.cu - exact solve of one coarse multigrid level by its dense inverse.
//
// Below the grid levels the shifted-Laplace cycle needs an (approximate) solve
// of a small coarse system M_d e = f. With few right-hand sides, running the
// levels under d as a multigrid cycle inside one block is a chain of dozens of
// dependent shared-memory passes on one SM. Instead the level d whose node
// count is at most kDenseMaxPoints is solved exactly: its Galerkin matrix M_d
// (complex symmetric, 9-point) is inverted once per distinct (model, frequency)
// when the solve starts, and every cycle applies the inverse with one
// matrix-vector kernel spread over the GPU.
//
// The inversion is block Gauss-Jordan without pivoting, in place. That is safe
// here: M_d = G_d - (b1 - j b2) (h omega)^2 K_d with G_d and K_d real symmetric
// positive definite (Galerkin products P^T G P and P^T K P of the 5-point or
// flux-form Laplacian and of diag(m^2)), so for b2 != 0 the imaginary part of
// x^H M_d x is b2 (h omega)^2 x^H K_d x != 0 for every x != 0: the field of
// values of M_d, and of every leading principal block and every Schur complement
// the elimination forms, excludes 0, and no pivot can vanish. A non-finite or
// vanishing pivot is still checked and reported, and the solver then uses the
// multigrid tail in place of the dense solve.
#include <algorithm>

#include "helm_internal.h"
#include "helm_solver.h"

namespace helm {

namespace {

constexpr int kDenseThreads = 256;
constexpr int kDenseMaxW = 16;                 // widest column strip (panel) a block owns
constexpr unsigned kBarrierSpins = 8000000u;   // bounded wait of one strip barrier (32 ns naps)


// Coherent (L2) loads of values another block wrote in this launch.
__device__ __forceinline__ cx<float> ldcg_c(const float* p, size_t i) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p) + i);
    return {v.x, v.y};
}
__device__ __forceinline__ cx<double> ldcg_c(const double* p, size_t i) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p) + i);
    return {v.x, v.y};
}

// Entry (i, j) of the level's shifted-Laplace matrix: the coefficient of u_j in
// (M u)_i. Stored forward entries: east (1,0), north (0,1), north-east (1,1) and
// north-west (-1,1) at the node they start from; the reverse direction reads the
// entry stored at the other node (M is symmetric).
__device__ __forceinline__ cx<double> gal_entry(const double* gk, size_t n, int nx, int i, int j, double hb1,
                                                double hb2) {
    const int ix = i % nx, iz = i / nx, jx = j % nx, jz = j / nx;
    const int dx = jx - ix, dz = jz - iz;
    int ent, at;
    if (dx == 0 && dz == 0) { ent = 0; at = i; }
    else if (dz == 0) { ent = 1; at = dx > 0 ? i : j; }
    else if (dx == 0) { ent = 2; at = dz > 0 ? i : j; }
    else if (dx == dz) { ent = 3; at = dx > 0 ? i : j; }
    else { ent = 4; at = dz > 0 ? i : j; }
    const double g = gk[(size_t)ent * n + at], q = gk[(size_t)(5 + ent) * n + at];
    return cx<double>(g - hb1 * q, hb2 * q);
}

// Block Gauss-Jordan inversion of M_d for the slots slot0 .. slot0 + nloc - 1.
// Block x = (local slot) * S + strip; the block owns columns [strip W, strip W + W)
// of its slot's matrix in shared memory ([W][n], column by column) for the whole
// inversion. Step k eliminates the column block k: its owner inverts the pivot
// block D (rows and columns of block k), publishes its old strip C (= column
// block k) and D^-1 to global memory, and after the slot's barrier every block
// applies the step to its strip:
//   owner:   column block k <- -C D^-1 (rows outside block k), D^-1 (rows of block k);
//   others:  R = D^-1 A[block k, own], own <- own - C R (rows outside), R (rows of block k).
// After the last step the strips hold M_d^-1; each block writes its columns.
template <typename T>
__global__ void __launch_bounds__(kDenseThreads) k_dense_invert(int nx, int nz, const double* __restrict__ gkall,
                                                                size_t gkstride, const double* __restrict__ w2s,
                                                                const int* __restrict__ mods, double b1, double b2,
                                                                int slot0, int W, int S, T* __restrict__ minv,
                                                                T* panel, T* dinv, unsigned* bar, int* err) {
    extern __shared__ __align__(16) unsigned char dense_smem[];
    const int n = nx * nz;
    const int ls = blockIdx.x / S, s = blockIdx.x - ls * S;
    const int sl = slot0 + ls;
    const int j0 = s * W, wj = min(W, n - j0);
    const int tid = threadIdx.x, nth = blockDim.x;
    cx<T>* As = reinterpret_cast<cx<T>*>(dense_smem);   // [W][n]
    cx<T>* Ds = As + (size_t)W * n;                      // [W][W] pivot block, then its inverse
    cx<T>* Rs = Ds + W * W;                              // [W][W] D^-1 A[block k, own columns]
    __shared__ int s_bad;
    __shared__ cx<T> s_pinv;
    const double hw = w2s[sl];
    const double* gk = gkall + (size_t)mods[sl] * gkstride;
    T* pan = panel + 2 * ((size_t)ls * 2 * n * W);   // [2][n][W] complex (two reals each)
    T* dv = dinv + 2 * ((size_t)ls * 2 * W * W);     // [2][W][W] complex
    unsigned* sbar = bar + ls;

    // this block's columns of M_d: nonzero only on the 9-point neighbours of each column
    for (int idx = tid; idx < W * n; idx += nth) As[idx] = cx<T>(0, 0);
    __syncthreads();
    for (int idx = tid; idx < wj * 9; idx += nth) {
        const int jj = idx / 9, q = idx - jj * 9;
        const int j = j0 + jj, jx = j % nx, jz = j / nx;
        const int ix = jx + q % 3 - 1, iz = jz + q / 3 - 1;
        if (ix < 0 || ix >= nx || iz < 0 || iz >= nz) continue;
        const int i = iz * nx + ix;
        const cx<double> a = gal_entry(gk, (size_t)n, nx, i, j, hw * b1, hw * b2);
        As[(size_t)jj * n + i] = cx<T>((T)a.re, (T)a.im);
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();

    for (int k = 0; k < S; ++k) {
        const int kb = k * W, wk = min(W, n - kb);
        const int buf = k & 1;
        if (s == k) {
            // pivot block D = A[block k, block k], inverted in place (Gauss-Jordan, no pivoting)
            for (int idx = tid; idx < wk * wk; idx += nth) {
                const int p = idx / wk, q = idx - p * wk;
                Ds[p * W + q] = As[(size_t)q * n + kb + p];
            }
            __syncthreads();
            for (int kk = 0; kk < wk; ++kk) {
                if (tid == 0) {
                    const cx<T> piv = Ds[kk * W + kk];
                    const T d = piv.re * piv.re + piv.im * piv.im;
                    if (!(d > T(0)) || !isfinite(d)) s_bad = 1;
                    const T inv = d > T(0) ? T(1) / d : T(0);
                    s_pinv = cx<T>(piv.re * inv, -piv.im * inv);
                    Ds[kk * W + kk] = cx<T>(1, 0);
                }
                __syncthreads();
                if (tid < wk) Ds[kk * W + tid] = s_pinv * Ds[kk * W + tid];
                __syncthreads();
                // eliminate column kk from the other rows: row i -= D[i][kk] row kk, with D[i][kk]
                // taken as 0 first (so that it ends as -D[i][kk] / pivot); all reads before all writes
                const bool act = tid < wk * wk;
                const int i = act ? tid / wk : 0, q = act ? tid - i * wk : 0;
                cx<T> f(0, 0), rk(0, 0), cur(0, 0);
                if (act && i != kk) {
                    f = Ds[i * W + kk];
                    rk = Ds[kk * W + q];
                    cur = (q == kk) ? cx<T>(0, 0) : Ds[i * W + q];
                }
                __syncthreads();
                if (act && i != kk) Ds[i * W + q] = cur - f * rk;
                __syncthreads();
            }
            if (s_bad) { if (tid == 0) atomicExch(err, 2); return; }
            // publish the old strip (column block k) and D^-1
            for (int idx = tid; idx < n * wk; idx += nth) {
                const int i = idx / wk, q = idx - i * wk;
                stc(pan, (size_t)buf * n * W + (size_t)i * W + q, As[(size_t)q * n + i]);
            }
            for (int idx = tid; idx < wk * wk; idx += nth) {
                const int p = idx / wk, q = idx - p * wk;
                stc(dv, (size_t)buf * W * W + p * W + q, Ds[p * W + q]);
            }
        }
        if (!coop_barrier(sbar, (unsigned)((k + 1) * S), err, kBarrierSpins)) return;
        const T* C = pan + 2 * ((size_t)buf * n * W);
        if (s != k) {
            for (int idx = tid; idx < wk * wk; idx += nth) {
                const int p = idx / wk, q = idx - p * wk;
                Ds[p * W + q] = ldcg_c(dv, (size_t)buf * W * W + p * W + q);
            }
            __syncthreads();
            for (int idx = tid; idx < wk * wj; idx += nth) {
                const int p = idx / wj, jj = idx - p * wj;
                cx<T> a(0, 0);
                for (int q = 0; q < wk; ++q) a = a + Ds[p * W + q] * As[(size_t)jj * n + kb + q];
                Rs[p * W + jj] = a;
            }
            __syncthreads();
        }
        const cx<T>* R = (s == k) ? Ds : Rs;
        const int wc = (s == k) ? wk : wj;   // columns of this block's strip
        for (int i = tid; i < n; i += nth) {
            if (i >= kb && i < kb + wk) {
                const int p = i - kb;
                for (int jj = 0; jj < wc; ++jj) As[(size_t)jj * n + i] = R[p * W + jj];
                continue;
            }
            cx<T> c[kDenseMaxW];
#pragma unroll
            for (int q = 0; q < kDenseMaxW; ++q)
                if (q < wk) c[q] = ldcg_c(C, (size_t)i * W + q);
            for (int jj = 0; jj < wc; ++jj) {
                cx<T> a(0, 0);
#pragma unroll
                for (int q = 0; q < kDenseMaxW; ++q)
                    if (q < wk) a = a + c[q] * R[q * W + jj];
                const size_t o = (size_t)jj * n + i;
                As[o] = (s == k) ? cx<T>(-a.re, -a.im) : As[o] - a;
            }
        }
        __syncthreads();
    }
    T* out = minv + 2 * (size_t)sl * n * n;
    for (int idx = tid; idx < n * wj; idx += nth) {
        const int i = idx / wj, jj = idx - i * wj;
        stc(out, (size_t)i * n + j0 + jj, As[(size_t)jj * n + i]);
    }
}

// e_b (+)= M_d^-1 f_b for the right-hand sides of one group (consecutive RHS of
// one slot, group g = [grp[g], grp[g+1])); one warp per row of the inverse, the
// row held in registers (NR complex values per lane per chunk) and reused for
// every right-hand side of the group, whose vectors are staged in shared memory.
template <typename T, int NR>
__global__ void __launch_bounds__(256) k_coarse_dense(int n, const T* __restrict__ minv, const int* __restrict__ slot,
                                                      const int* __restrict__ grp, int maxg, const T* f, T* e,
                                                      int accumulate, const RhsState* st) {
    extern __shared__ __align__(16) unsigned char cd_smem[];
    cx<T>* fs = reinterpret_cast<cx<T>*>(cd_smem);   // [group][n]
    pdl_trigger();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int row = blockIdx.x * 8 + warp;
    const int g = blockIdx.y;
    const int b0 = grp[g], b1 = grp[g + 1];
    const T* Mr = minv + 2 * ((size_t)slot[b0] * n * n + (size_t)min(row, n - 1) * n);
    constexpr int CH = 32 * NR;
    cx<T> rv[NR];
    // the first chunk of this warp's row is model data: load it before waiting on the previous kernel
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int j = lane + 32 * k;
        rv[k] = j < n ? ldc(Mr, j) : cx<T>(0, 0);
    }
    pdl_wait();
    const int nb = b1 - b0;
    for (int idx = threadIdx.x; idx < nb * n; idx += blockDim.x) fs[idx] = ldcc(f, (size_t)b0 * n + idx);
    __syncthreads();
    if (row >= n) return;
    T are[8], aim[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) { are[r] = T(0); aim[r] = T(0); }
    for (int c0 = 0; c0 < n; c0 += CH) {
        if (c0 > 0) {
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const int j = c0 + lane + 32 * k;
                rv[k] = j < n ? ldc(Mr, j) : cx<T>(0, 0);
            }
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            if (r >= nb) break;
            const cx<T>* fv = fs + (size_t)r * n;
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                const int j = c0 + lane + 32 * k;
                if (j < n) {
                    const cx<T> v = fv[j];
                    are[r] += rv[k].re * v.re - rv[k].im * v.im;
                    aim[r] += rv[k].re * v.im + rv[k].im * v.re;
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        if (r >= nb) break;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            are[r] += __shfl_xor_sync(0xffffffffu, are[r], o);
            aim[r] += __shfl_xor_sync(0xffffffffu, aim[r], o);
        }
        const int b = b0 + r;
        if (lane == 0 && rhs_active(st, b)) {
            cx<T> v(are[r], aim[r]);
            if (accumulate) v = v + ldcc(e, (size_t)b * n + row);
            stc(e, (size_t)b * n + row, v);
        }
    }
    (void)maxg;
}

}  // namespace

// Strip width and co-resident capacity of the inversion for an n-node level in
// the given precision; 0 when it cannot run as one co-resident grid per slot.
int dense_invert_plan(int n, bool dbl, int* W_out, int* per_launch_slots) {
    if (n < 1 || n > kDenseMaxPoints) return 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t es = dbl ? 16 : 8;
    for (int W = 8; W <= kDenseMaxW; ++W) {
        const int S = (n + W - 1) / W;
        const size_t smem = ((size_t)W * n + 2 * (size_t)W * W) * es;
        if ((long long)smem > smem_optin) break;
        int per_sm = 0;
        cudaError_t e;
        if (dbl) {
            e = cudaFuncSetAttribute(k_dense_invert<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_invert<double>, kDenseThreads, smem);
        } else {
            e = cudaFuncSetAttribute(k_dense_invert<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_invert<float>, kDenseThreads, smem);
        }
        if (e != cudaSuccess) { cudaGetLastError(); return 0; }
        const long long cap = (long long)per_sm * sms;
        if (cap >= S) {
            *W_out = W;
            *per_launch_slots = (int)std::max<long long>(1, cap / S);
            return 1;
        }
    }
    return 0;
}

// Inverts M_d of every slot (distinct model and (h omega)^2) into minv
// [nslots][n][n] in the kernel's precision. panel/dinv/bar: workspace for
// min(nslots, per_launch_slots) slots ([2][n][W] and [2][W][W] complex each, one
// counter each); err: one int, 0 on success, 1 if a barrier gave up, 2 on a
// vanishing or non-finite pivot. Launches cooperative grids on s (no
// synchronisation); returns a CUDA error code of the launch.
template <typename T>
cudaError_t launch_dense_invert(const LevelDev& Ld, const double* w2s, const int* mods, int nslots, double b1,
                                double b2, int W, int per_launch, T* minv, T* panel, T* dinv, unsigned* bar,
                                int* err, cudaStream_t s) {
    const int n = Ld.nx * Ld.nz;
    const int S = (n + W - 1) / W;
    const size_t smem = ((size_t)W * n + 2 * (size_t)W * W) * sizeof(T) * 2;
    cudaError_t e = cudaFuncSetAttribute(k_dense_invert<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(err, 0, sizeof(int), s);
    ProfScope prof(PK_DENSE_INVERT, Ld.nx, Ld.nz, (double)n * n * nslots * 2.0 * sizeof(T), s);
    for (int s0 = 0; s0 < nslots && e == cudaSuccess; s0 += per_launch) {
        const int nloc = std::min(per_launch, nslots - s0);
        e = cudaMemsetAsync(bar, 0, sizeof(unsigned) * nloc, s);
        if (e != cudaSuccess) break;
        int nxv = Ld.nx, nzv = Ld.nz;
        const double* gk = static_cast<const double*>(Ld.gk);
        size_t gks = Ld.gkstride;
        int slot0 = s0, Wv = W, Sv = S;
        void* args[] = {&nxv, &nzv, (void*)&gk, &gks, (void*)&w2s, (void*)&mods, &b1, &b2, &slot0, &Wv, &Sv,
                        &minv, &panel, &dinv, &bar, &err};
        e = cudaLaunchCooperativeKernel((const void*)k_dense_invert<T>, dim3(nloc * S), dim3(kDenseThreads), args,
                                        smem, s);
        count_launches(1);
    }
    return e;
}
template cudaError_t launch_dense_invert<float>(const LevelDev&, const double*, const int*, int, double, double, int,
                                                int, float*, float*, float*, unsigned*, int*, cudaStream_t);
template cudaError_t launch_dense_invert<double>(const LevelDev&, const double*, const int*, int, double, double,
                                                 int, int, double*, double*, double*, unsigned*, int*, cudaStream_t);

template <typename T>
void launch_coarse_dense(int n, const T* minv, const int* slot, const int* grp, int ngroups, int maxg, const T* f,
                         T* e, int accumulate, const RhsState* st, cudaStream_t s) {
    constexpr int NR = sizeof(T) == 4 ? 38 : 19;
    // the inverse of each group's slot once per group, f read and e written (and read when accumulating)
    ProfScope prof(PK_COARSE_DENSE, n, 1,
                   ((double)n * n * ngroups + (double)n * (2 + accumulate) * ngroups * maxg) * 2.0 * sizeof(T), s);
    const size_t smem = (size_t)maxg * n * sizeof(T) * 2;
    static const bool attr = [] {
        cudaFuncSetAttribute(k_coarse_dense<T, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        return true;
    }();
    (void)attr;
    launch_pdl(k_coarse_dense<T, NR>, dim3((n + 7) / 8, ngroups), dim3(256), smem, s, n, minv, slot, grp, maxg, f, e,
               accumulate, st);
}
template void launch_coarse_dense<float>(int, const float*, const int*, const int*, int, int, const float*, float*,
                                         int, const RhsState*, cudaStream_t);
template void launch_coarse_dense<double>(int, const double*, const int*, const int*, int, int, const double*,
                                          double*, int, const RhsState*, cudaStream_t);

}  // namespace helm

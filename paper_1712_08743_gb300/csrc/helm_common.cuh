// helm_common.cuh - device helpers shared by the Helmholtz kernels: complex
// arithmetic on float2/double2, the damping profile of the absorbing layer,
// per-right-hand-side solver state and deterministic block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace helm {

// ----------------------------------------------------------------- complex
template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };

template <typename T> struct cx {
    T re, im;
    __host__ __device__ cx() {}
    __host__ __device__ cx(T r, T i) : re(r), im(i) {}
};
template <typename T> __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> __device__ __forceinline__ cx<T> conjx(cx<T> a) { return {a.re, -a.im}; }
// Reciprocal of |b|^2 in complex division: the FP32 smoother and preconditioner
// use the hardware approximate divide (max 2 ulp), FP64 keeps the IEEE divide.
__device__ __forceinline__ float rcp_fast(float d) { return __fdividef(1.0f, d); }
__device__ __forceinline__ double rcp_fast(double d) { return 1.0 / d; }
template <typename T> __device__ __forceinline__ cx<T> cdiv(cx<T> a, cx<T> b) {
    T d = b.re * b.re + b.im * b.im;
    T inv = rcp_fast(d);
    return {(a.re * b.re + a.im * b.im) * inv, (a.im * b.re - a.re * b.im) * inv};
}

// 8- or 16-byte vector loads/stores of one complex value.
__device__ __forceinline__ cx<float> ldc(const float* p, size_t i) {
    float2 v = __ldg(reinterpret_cast<const float2*>(p) + i);
    return {v.x, v.y};
}
__device__ __forceinline__ cx<double> ldc(const double* p, size_t i) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p) + i);
    return {v.x, v.y};
}
// plain (coherent) loads, for buffers written earlier in the same kernel chain
__device__ __forceinline__ cx<float> ldcc(const float* p, size_t i) {
    float2 v = reinterpret_cast<const float2*>(p)[i];
    return {v.x, v.y};
}
__device__ __forceinline__ cx<double> ldcc(const double* p, size_t i) {
    double2 v = reinterpret_cast<const double2*>(p)[i];
    return {v.x, v.y};
}
__device__ __forceinline__ void stc(float* p, size_t i, cx<float> a) {
    reinterpret_cast<float2*>(p)[i] = make_float2(a.re, a.im);
}
__device__ __forceinline__ void stc(double* p, size_t i, cx<double> a) {
    reinterpret_cast<double2*>(p)[i] = make_double2(a.re, a.im);
}

// ------------------------------------------------------------ damping layer
// alpha of Eq. 2 at padded node (ix, iz): alpha_max (d / npml)^2 with d the
// node distance into the layer, the larger of the two axes in corners.
// Same profile from the integer layer depth, with acoef = alpha_max / npml^2
// precomputed on the host: no division on the device, in the kernel's precision.
__device__ __forceinline__ int layer_depth(int ix, int iz, int nx, int nz, int npml) {
    const int dx = max(npml - ix, ix - (nx - 1 - npml));
    const int dz = max(npml - iz, iz - (nz - 1 - npml));
    return max(max(dx, dz), 0);
}
template <typename T>
__device__ __forceinline__ T layer_alpha_t(int ix, int iz, int nx, int nz, int npml, T acoef) {
    const int d = layer_depth(ix, iz, nx, nz, npml);
    return acoef * (T)(d * d);
}
inline double layer_coef(int npml, double alpha_max) { return npml > 0 ? alpha_max / ((double)npml * npml) : 0.0; }

// ------------------------------------------------------- solver state per RHS
enum RhsFlag : int { FLAG_RUNNING = 0, FLAG_CONVERGED = 1, FLAG_BREAKDOWN = 2, FLAG_MAXIT = 3 };

struct RhsState {
    // Krylov scalars (BiCGSTAB); complex values as (re, im)
    double rho[2], alpha[2], omega[2], beta[2];
    double bnorm2;       // ||b||^2 of the inner system
    double rnorm2;       // ||r||^2 of the recursive residual
    double tol_rel;      // inner relative tolerance on ||r|| / ||b||
    double relres;       // outer FP64 relative residual
    double fnorm2;       // ||f||^2 of the outer system
    int active;          // 1 while this RHS iterates
    int iters;           // inner iterations, summed over outer steps
    int flag;            // RhsFlag of the last inner solve
    int outer_active;    // 1 while the outer refinement continues
    int max_it;
    int kfg;             // FGMRES: Arnoldi steps of the current cycle
    int reorth;          // FGMRES: 1 if the current column takes a second Gram-Schmidt pass
    unsigned int counter[4];  // last-block election counters, one per reduction site
};

// A right-hand side takes part in a kernel while its state says so (no state: always).
__device__ __forceinline__ bool rhs_active(const RhsState* st, int b) { return st == nullptr || st[b].active; }

// ------------------------------------------------ programmatic dependent launch
// Kernels of the iteration chain let the next kernel start launching at once
// (its blocks then wait in pdl_wait until this grid has completed and its
// writes are visible), so launch latency and prologues that read only
// immutable model data overlap the previous kernel. Without a programmatic
// dependency both instructions return immediately.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ------------------------------------------------ barrier of co-resident blocks
// For kernels launched cooperatively (every block resident at once). Thread 0 of
// each block makes the block's writes visible, counts the block in on *bar and
// waits until *bar reaches `target` (the monotone count of arrivals: phase *
// number of blocks). The wait is bounded: it gives up when another block has
// reported a failure in *err, or after `spins` naps of 32 ns, setting *err = 1.
// Returns false in every thread of the block when the kernel must stop.
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ bool coop_barrier(unsigned* bar, unsigned target, int* err, unsigned spins) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        int ok = 1;
        for (unsigned k = 0;; ++k) {
            if (ld_acquire_gpu(bar) >= target) break;
            if (*reinterpret_cast<const volatile int*>(err) != 0) { ok = 0; break; }
            if (k >= spins) { atomicExch(err, 1); ok = 0; break; }
            __nanosleep(32);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// -------------------------------------------------------------- reductions
__device__ __forceinline__ int lin_tid() { return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z); }
__device__ __forceinline__ int lin_nthreads() { return blockDim.x * blockDim.y * blockDim.z; }

template <int NV>
__device__ __forceinline__ void warp_sum(double (&v)[NV]) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}

// Block-wide sum of NV doubles (blocks of whole warps); result valid in
// linear thread 0. Deterministic order.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh /* >= 32*NV */) {
    warp_sum<NV>(v);
    const int tid = lin_tid();
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (lin_nthreads() + 31) >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k * 32 + warp] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = (lane < nwarps) ? sh[k * 32 + lane] : 0.0;
        warp_sum<NV>(v);
    }
}

// Block-wide sum of per-thread partials held in the kernel's precision A: the
// warp stage runs in A, only warp totals are widened to double (so an FP32
// kernel issues almost no FP64 instructions). Result in linear thread 0.
template <int NV, typename A>
__device__ __forceinline__ void block_sum_t(const A (&v)[NV], double (&o)[NV], double* sh /* >= 32*NV */) {
    A w[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        w[k] = v[k];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) w[k] += __shfl_xor_sync(0xffffffffu, w[k], d);
    }
    const int tid = lin_tid();
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (lin_nthreads() + 31) >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k * 32 + warp] = (double)w[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) o[k] = 0.0;
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) o[k] = (lane < nwarps) ? sh[k * 32 + lane] : 0.0;
        warp_sum<NV>(o);
    }
}

// As last_block_reduce, from per-thread partials in precision A; the totals
// land in tot (thread 0 of the last block).
template <int NV, typename A>
__device__ __forceinline__ bool last_block_reduce_t(const A (&v)[NV], double (&tot)[NV], double* sh, double* partials,
                                                    int nblk, int blk, unsigned int* counter) {
    block_sum_t<NV, A>(v, tot, sh);
    __shared__ int s_last_t;
    const int tid = lin_tid();
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) partials[(size_t)k * nblk + blk] = tot[k];
        __threadfence();
        unsigned int prev = atomicAdd(counter, 1u);
        s_last_t = (prev == (unsigned int)(nblk - 1));
    }
    __syncthreads();
    if (!s_last_t) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (int i = tid; i < nblk; i += lin_nthreads())
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += __ldcg(partials + (size_t)k * nblk + i);
    block_sum<NV>(acc, sh);
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] = acc[k];
        *counter = 0u;
    }
    return true;
}

// Writes this block's NV partial sums and elects the last block of the
// right-hand side to finish. Returns true (in all threads) for that block, whose
// thread 0 then holds the totals in v, summed in fixed block order.
template <int NV>
__device__ __forceinline__ bool last_block_reduce(double (&v)[NV], double* sh, double* partials,
                                                  int nblk, int blk, unsigned int* counter) {
    block_sum<NV>(v, sh);
    __shared__ int s_last;
    const int tid = lin_tid();
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) partials[(size_t)k * nblk + blk] = v[k];
        __threadfence();
        unsigned int prev = atomicAdd(counter, 1u);
        s_last = (prev == (unsigned int)(nblk - 1));
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (int i = tid; i < nblk; i += lin_nthreads())
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += __ldcg(partials + (size_t)k * nblk + i);
    block_sum<NV>(acc, sh);
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = acc[k];
        *counter = 0u;
    }
    return true;
}

}  // namespace helm

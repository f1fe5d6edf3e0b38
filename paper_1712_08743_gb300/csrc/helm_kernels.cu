// helm_kernels.cu - CUDA kernels (sm_103a) of the shifted-Laplace Helmholtz path.
//
// Operators, in the grid-scaled form A = h^2 B that every kernel uses:
//   A u = 4u - u_{i+-1,k} - u_{i,k+-1} - h^2 w^2 m^2 (1 - j alpha) u          (Eq. 2/3)
//   M u = 4u - u_{i+-1,k} - u_{i,k+-1} - h_l^2 w^2 m^2 (beta1 - j beta2) u    (shifted Laplacian)
// Zero Dirichlet ghosts lie one node outside each grid. Vectors are batched
// [nrhs][nz][nx] interleaved complex; right-hand side b uses angular frequency
// omega_b (w2[b] = omega_b^2). The multigrid level l+1 has floor(n_l / 2)
// nodes per axis; coarse node I sits on fine node 2I + 1.
#include <algorithm>
#include <functional>
#include <vector>

#include "helm_gal_tiles.cuh"
#include "helm_internal.h"

namespace helm {

namespace {

template <typename T>
__device__ __forceinline__ const T* m2ptr(const LevelDev& L) { return static_cast<const T*>(L.m2); }

// Grid-stride extent for 1D vector kernels.
inline int grid1d(size_t n) {
    size_t g = (n + 1023) / 1024;
    if (g < 1) g = 1;
    if (g > 2048) g = 2048;
    return (int)g;
}

}  // namespace

// ===================================================================== model
__global__ void k_pad_model(const double* __restrict__ m_phys, int Px, int Pz, int npml,
                            double* __restrict__ m_pad, float* __restrict__ m2f, double* __restrict__ m2d) {
    const int nx = Px + 2 * npml, nz = Pz + 2 * npml;
    const size_t n = (size_t)nx * nz;
    const int k = blockIdx.y;   // model index
    m_phys += (size_t)k * Px * Pz;
    m_pad += n * k;
    m2f += n * k;
    m2d += n * k;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        int ix = (int)(i % nx), iz = (int)(i / nx);
        int px = min(max(ix - npml, 0), Px - 1);
        int pz = min(max(iz - npml, 0), Pz - 1);
        double m = m_phys[(size_t)pz * Px + px];
        m_pad[i] = m;
        m2d[i] = m * m;
        m2f[i] = (float)(m * m);
    }
}

void launch_pad_model(const double* m_phys, int Px, int Pz, int npml, int nmodels, double* m_pad, float* m2f,
                      double* m2d, cudaStream_t s) {
    size_t n = (size_t)(Px + 2 * npml) * (Pz + 2 * npml);
    k_pad_model<<<dim3(grid1d(n), nmodels), 256, 0, s>>>(m_phys, Px, Pz, npml, m_pad, m2f, m2d);
}

// Finest-level coefficients of the flux-form operator of Eq. 1 (h^2 times
// -div(rho grad)): the density is padded like the slowness (nearest physical
// cell); an edge between nodes i and j takes the harmonic mean
// 2 rho_i rho_j / (rho_i + rho_j), an edge to a ghost node outside the grid
// takes rho_i. rho[0][i] / rho[1][i]: east / north edge of node i, rho[2][i]: the
// sum of the node's four edges. gk: the same operator as a stored level for the
// Galerkin kernels (G: centre = the sum, east and north = minus the edge, the
// diagonal couplings 0; K: centre m^2, the rest 0).
__device__ __forceinline__ double pad_at(const double* phys, int Px, int Pz, int npml, int ix, int iz) {
    const int px = min(max(ix - npml, 0), Px - 1), pz = min(max(iz - npml, 0), Pz - 1);
    return phys[(size_t)pz * Px + px];
}
__device__ __forceinline__ double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

__global__ void k_rho_setup(const double* __restrict__ rho_phys, int Px, int Pz, int npml,
                            const double* __restrict__ m2d, double* __restrict__ rhod, float* __restrict__ rhof,
                            double* __restrict__ gkd, float* __restrict__ gkf) {
    const int nx = Px + 2 * npml, nz = Pz + 2 * npml;
    const size_t n = (size_t)nx * nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nx), iz = (int)(i / nx);
        const double r = pad_at(rho_phys, Px, Pz, npml, ix, iz);
        const double re = ix + 1 < nx ? harmonic(r, pad_at(rho_phys, Px, Pz, npml, ix + 1, iz)) : r;
        const double rw = ix > 0 ? harmonic(r, pad_at(rho_phys, Px, Pz, npml, ix - 1, iz)) : r;
        const double rn = iz + 1 < nz ? harmonic(r, pad_at(rho_phys, Px, Pz, npml, ix, iz + 1)) : r;
        const double rs = iz > 0 ? harmonic(r, pad_at(rho_phys, Px, Pz, npml, ix, iz - 1)) : r;
        const double dg = re + rw + rn + rs;
        const double v[3] = {re, rn, dg};
        for (int k = 0; k < 3; ++k) {
            rhod[(size_t)k * n + i] = v[k];
            rhof[(size_t)k * n + i] = (float)v[k];
        }
        const double g[10] = {dg, -re, -rn, 0.0, 0.0, m2d[i], 0.0, 0.0, 0.0, 0.0};
        for (int k = 0; k < 10; ++k) {
            gkd[(size_t)k * n + i] = g[k];
            gkf[(size_t)k * n + i] = (float)g[k];
        }
    }
}

void launch_rho_setup(const double* rho_phys, int Px, int Pz, int npml, const double* m2d, double* rhod, float* rhof,
                      double* gkd, float* gkf, cudaStream_t s) {
    const size_t n = (size_t)(Px + 2 * npml) * (Pz + 2 * npml);
    k_rho_setup<<<grid1d(n), 256, 0, s>>>(rho_phys, Px, Pz, npml, m2d, rhod, rhof, gkd, gkf);
}

// sum of squares of a real array (one block; model setup only)
__global__ void k_sumsq(const double* __restrict__ a, size_t count, double* out) {
    __shared__ double sh[32];
    double acc[1] = {0.0};
    for (size_t i = threadIdx.x; i < count; i += blockDim.x) acc[0] += a[i] * a[i];
    block_sum<1>(acc, sh);
    if (threadIdx.x == 0) *out = acc[0];
}
void launch_sumsq(const double* a, size_t count, double* out, cudaStream_t s) { k_sumsq<<<1, 1024, 0, s>>>(a, count, out); }

// ============================================================ stencil apply
// y = scale * A u on the fine grid (with the damping layer). Each thread owns
// one column x and marches down ZCH rows, keeping rows z-1, z, z+1 in
// registers: one coalesced load per node (plus the block's two halo rows);
// the x-neighbours come from the adjacent lanes by warp shuffles (the warp's
// edge lanes load theirs).
// Each thread owns AP_R consecutive rows of one column: the AP_R + 2 rows it
// needs are loaded up front (AP_R + 2 independent loads in flight per thread),
// the x neighbours come from the adjacent lanes by shuffle, and only the two
// warp-edge lanes read a neighbour from memory.
constexpr int AP_X = 32, AP_Y = 8, AP_R = 4;

template <typename T>
__global__ void __launch_bounds__(AP_X * AP_Y) k_apply(LevelDev L, int npml, T acoef, const T* __restrict__ hwv,
                                                       const T* __restrict__ u, T* __restrict__ y, T scale) {
    const int b = blockIdx.z;
    const int nx = L.nx, nz = L.nz;
    const int ix = blockIdx.x * AP_X + threadIdx.x;
    const int z0 = (blockIdx.y * AP_Y + threadIdx.y) * AP_R;
    if (z0 >= nz) return;  // whole warp leaves together (threadIdx.y is uniform in a warp)
    const size_t n = (size_t)nx * nz;
    const T* ub = u + 2 * n * b;
    T* yb = y + 2 * n * b;
    const T* m2 = m2ptr<T>(L) + (size_t)b * L.mstride;
    const T hw = hwv[b];
    const bool xin = ix < nx;
    const int lane = threadIdx.x;
    // Blocks whose nodes and neighbours all lie inside the grid and outside the
    // damping layer (alpha = 0) take a path without bounds tests or alpha.
    const int bx0 = blockIdx.x * AP_X, bz0 = blockIdx.y * AP_Y * AP_R;
    if (bx0 >= npml && bx0 + AP_X - 1 <= nx - 1 - npml && bz0 >= npml && bz0 + AP_Y * AP_R - 1 <= nz - 1 - npml &&
        npml >= 1) {
        cx<T> v[AP_R + 2], e[AP_R];
        T mm[AP_R];
        const bool edge = lane == 0 || lane == AP_X - 1;
        const int ex = lane == 0 ? ix - 1 : ix + 1;
#pragma unroll
        for (int k = 0; k < AP_R + 2; ++k) v[k] = ldc(ub, (z0 - 1 + k) * nx + ix);
#pragma unroll
        for (int k = 0; k < AP_R; ++k) {
            mm[k] = __ldg(m2 + (z0 + k) * nx + ix);
            e[k] = edge ? ldc(ub, (z0 + k) * nx + ex) : cx<T>(0, 0);
        }
#pragma unroll
        for (int k = 0; k < AP_R; ++k) {
            const cx<T> cur = v[k + 1];
            cx<T> l(__shfl_up_sync(0xffffffffu, cur.re, 1), __shfl_up_sync(0xffffffffu, cur.im, 1));
            cx<T> r(__shfl_down_sync(0xffffffffu, cur.re, 1), __shfl_down_sync(0xffffffffu, cur.im, 1));
            if (lane == 0) l = e[k];
            if (lane == AP_X - 1) r = e[k];
            const T dd = T(4) - hw * mm[k];
            cx<T> acc(dd * cur.re, dd * cur.im);
            acc = acc - ((l + r) + (v[k] + v[k + 2]));
            stc(yb, (z0 + k) * nx + ix, scale * acc);
        }
        return;
    }
    // layer depth along x is fixed per thread; alpha = acoef max(dx, dz, 0)^2
    const int dxd = max(npml - ix, ix - (nx - 1 - npml));
    cx<T> v[AP_R + 2];
#pragma unroll
    for (int k = 0; k < AP_R + 2; ++k) {
        const int z = z0 - 1 + k;
        v[k] = (xin && z >= 0 && z < nz) ? ldc(ub, z * nx + ix) : cx<T>(0, 0);
    }
    T mm[AP_R];
#pragma unroll
    for (int k = 0; k < AP_R; ++k) {
        const int z = z0 + k;
        mm[k] = (xin && z < nz) ? __ldg(m2 + z * nx + ix) : T(0);
    }
#pragma unroll
    for (int k = 0; k < AP_R; ++k) {
        const int z = z0 + k;
        const cx<T> cur = v[k + 1];
        cx<T> l(__shfl_up_sync(0xffffffffu, cur.re, 1), __shfl_up_sync(0xffffffffu, cur.im, 1));
        cx<T> r(__shfl_down_sync(0xffffffffu, cur.re, 1), __shfl_down_sync(0xffffffffu, cur.im, 1));
        if (z < nz && xin) {
            const int i = z * nx + ix;
            if (lane == 0) l = ix > 0 ? ldc(ub, i - 1) : cx<T>(0, 0);
            if (lane == AP_X - 1) r = ix + 1 < nx ? ldc(ub, i + 1) : cx<T>(0, 0);
            else if (ix + 1 >= nx) r = cx<T>(0, 0);
            const int d = max(max(dxd, max(npml - z, z - (nz - 1 - npml))), 0);
            const T s = hw * mm[k];
            const T sa = s * (acoef * (T)(d * d));
            const T dd = T(4) - s;
            cx<T> acc(dd * cur.re - sa * cur.im, dd * cur.im + sa * cur.re);
            acc = acc - ((l + r) + (v[k] + v[k + 2]));
            stc(yb, i, scale * acc);
        }
    }
}

template <typename T, int MODE, bool VD>
__global__ void __launch_bounds__(256) k_apply_dots(LevelDev L, int npml, T acoef, const T* __restrict__ hwv,
                                                    const T* __restrict__ u, T* __restrict__ y,
                                                    const T* __restrict__ aux, double* partials, int pstride,
                                                    RhsState* st, T scale);

template <typename T>
void launch_apply(const LevelDev& L0, int npml, double amax, const T* hw, const T* u, T* y, T scale,
                  int nrhs, cudaStream_t s) {
    const double n0 = (double)L0.nx * L0.nz, es = 2.0 * sizeof(T);
    ProfScope prof(PK_APPLY, L0.nx, L0.nz, n0 * (2 * es * nrhs + sizeof(T) * (L0.mstride ? nrhs : 1) * (L0.rho ? 4 : 1)),
                   s);
    if (L0.rho) {   // variable density: the flux-form operator, one node per thread
        dim3 blk(32, 8), grd((L0.nx + 31) / 32, (L0.nz + 7) / 8, nrhs);
        k_apply_dots<T, 0, true><<<grd, blk, 0, s>>>(L0, npml, (T)layer_coef(npml, amax), hw, u, y,
                                                     (const T*)nullptr, nullptr, 0, nullptr, scale);
        return;
    }
    dim3 blk(AP_X, AP_Y), grd((L0.nx + AP_X - 1) / AP_X, (L0.nz + AP_Y * AP_R - 1) / (AP_Y * AP_R), nrhs);
    k_apply<T><<<grd, blk, 0, s>>>(L0, npml, (T)layer_coef(npml, amax), hw, u, y, scale);
}
template void launch_apply<float>(const LevelDev&, int, double, const float*, const float*, float*, float, int, cudaStream_t);
template void launch_apply<double>(const LevelDev&, int, double, const double*, const double*, double*, double, int, cudaStream_t);

// (A u)_i on the finest level, one node: the 5-point operator of Eq. 2,
// 4 u_i - sum of the four neighbours, or with a density (VD, Eq. 1) the flux form
// d_i u_i - sum_e rho_e u_j from the stored coefficients; minus s (1 - j a) u_i;
// neighbours outside the grid are zero. c = u_i. The two forms are separate
// instances so that the constant-density arithmetic is not reshaped by the other.
template <typename T, bool VD>
__device__ __forceinline__ cx<T> fine_apply_point(const LevelDev& L, const T* __restrict__ ub, size_t i, int ix,
                                                  int iz, T s, T a, cx<T> c) {
    if constexpr (!VD) {
        cx<T> yv((T(4) - s) * c.re - s * a * c.im, (T(4) - s) * c.im + s * a * c.re);
        if (ix > 0) yv = yv - ldc(ub, i - 1);
        if (ix + 1 < L.nx) yv = yv - ldc(ub, i + 1);
        if (iz > 0) yv = yv - ldc(ub, i - L.nx);
        if (iz + 1 < L.nz) yv = yv - ldc(ub, i + L.nx);
        return yv;
    } else {
        const T* R = static_cast<const T*>(L.rho);
        const size_t n = (size_t)L.nx * L.nz;
        const T dg = R[2 * n + i];
        cx<T> yv((dg - s) * c.re - s * a * c.im, (dg - s) * c.im + s * a * c.re);
        if (ix > 0) yv = yv - R[i - 1] * ldc(ub, i - 1);
        if (ix + 1 < L.nx) yv = yv - R[i] * ldc(ub, i + 1);
        if (iz > 0) yv = yv - R[n + i - L.nx] * ldc(ub, i - L.nx);
        if (iz + 1 < L.nz) yv = yv - R[n + i] * ldc(ub, i + L.nx);
        return yv;
    }
}

// y = A u with the dot products of the unpreconditioned BiCGSTAB (the
// preconditioner-free path of the ablation, and the variable-density path):
// mode 1 <aux, y> -> alpha, mode 2 <y, aux or u>, <y, y> -> omega, as the fused
// prolongation does after a cycle; mode 0 only y = scale A u.
template <typename T, int MODE, bool VD>
__global__ void __launch_bounds__(256) k_apply_dots(LevelDev L, int npml, T acoef, const T* __restrict__ hwv,
                                                    const T* __restrict__ u, T* __restrict__ y,
                                                    const T* __restrict__ aux, double* partials, int pstride,
                                                    RhsState* st, T scale) {
    __shared__ double shred[96];
    pdl_trigger();
    pdl_wait();
    const int b = blockIdx.z;
    if (!rhs_active(st, b)) return;
    const int ix = blockIdx.x * 32 + threadIdx.x, iz = blockIdx.y * 8 + threadIdx.y;
    const size_t n = (size_t)L.nx * L.nz;
    T d0 = 0, d1 = 0, d2 = 0;
    if (ix < L.nx && iz < L.nz) {
        const T* ub = u + 2 * n * b;
        const size_t i = (size_t)iz * L.nx + ix;
        const T s = hwv[b] * (m2ptr<T>(L) + (size_t)b * L.mstride)[i];
        const T a = layer_alpha_t<T>(ix, iz, L.nx, L.nz, npml, acoef);
        const cx<T> c = ldc(ub, i);
        if constexpr (!VD) {
            cx<T> yv((T(4) - s) * c.re - s * a * c.im, (T(4) - s) * c.im + s * a * c.re);
            if (ix > 0) yv = yv - ldc(ub, i - 1);
            if (ix + 1 < L.nx) yv = yv - ldc(ub, i + 1);
            if (iz > 0) yv = yv - ldc(ub, i - L.nx);
            if (iz + 1 < L.nz) yv = yv - ldc(ub, i + L.nx);
            stc(y + 2 * n * b, i, MODE == 0 ? scale * yv : yv);
            if (MODE == 1) {
                const cx<T> q = ldc(aux + 2 * n * b, i);
                d0 = q.re * yv.re + q.im * yv.im;
                d1 = q.re * yv.im - q.im * yv.re;
            } else if (MODE == 2) {
                d0 = yv.re * c.re + yv.im * c.im;
                d1 = yv.re * c.im - yv.im * c.re;
                d2 = yv.re * yv.re + yv.im * yv.im;
            }
        } else {
            const cx<T> yv = fine_apply_point<T, true>(L, ub, i, ix, iz, s, a, c);
            stc(y + 2 * n * b, i, MODE == 0 ? scale * yv : yv);
            if (MODE == 1) {
                const cx<T> q = ldc(aux + 2 * n * b, i);
                d0 = q.re * yv.re + q.im * yv.im;
                d1 = q.re * yv.im - q.im * yv.re;
            } else if (MODE == 2) {
                // BiCGSTAB's omega takes <t, s> with s the preconditioner's input: aux when
                // given (after a separate cycle), else u itself (no preconditioner)
                const cx<T> q = aux ? ldc(aux + 2 * n * b, i) : c;
                d0 = yv.re * q.re + yv.im * q.im;
                d1 = yv.re * q.im - yv.im * q.re;
                d2 = yv.re * yv.re + yv.im * yv.im;
            }
        }
    }
    if (MODE == 0) return;
    const T vv[3] = {d0, d1, d2};
    double acc[3];
    const int nblk = gridDim.x * gridDim.y, blk = blockIdx.y * gridDim.x + blockIdx.x;
    if (last_block_reduce_t<3, T>(vv, acc, shred, partials + (size_t)b * pstride, nblk, blk, &st[b].counter[3])) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            RhsState& S = st[b];
            if (MODE == 1) {
                const double dd = acc[0] * acc[0] + acc[1] * acc[1];
                if (!(dd > 0.0)) {
                    S.flag = FLAG_BREAKDOWN;
                    S.alpha[0] = 0.0; S.alpha[1] = 0.0;
                } else {
                    S.alpha[0] = (S.rho[0] * acc[0] + S.rho[1] * acc[1]) / dd;
                    S.alpha[1] = (S.rho[1] * acc[0] - S.rho[0] * acc[1]) / dd;
                }
            } else {
                if (acc[2] > 0.0) { S.omega[0] = acc[0] / acc[2]; S.omega[1] = acc[1] / acc[2]; }
                else { S.omega[0] = 0.0; S.omega[1] = 0.0; }
            }
        }
    }
}

template <typename T>
void launch_apply_dots(int mode, const LevelDev& L0, int npml, double amax, const T* hw, const T* u, T* y,
                       const T* aux, double* partials, int pstride, RhsState* st, int nrhs, cudaStream_t s) {
    const double n0 = (double)L0.nx * L0.nz, es = 2.0 * sizeof(T);
    ProfScope prof(PK_APPLY_DOTS, L0.nx, L0.nz,
                   n0 * (3 * es * nrhs + sizeof(T) * (L0.mstride ? nrhs : 1) * (L0.rho ? 4 : 1)), s);
    dim3 blk(32, 8), grd((L0.nx + 31) / 32, (L0.nz + 7) / 8, nrhs);
    const T ac = (T)layer_coef(npml, amax);
    const bool vd = L0.rho != nullptr;
    if (mode == 1 && vd)
        launch_pdl(k_apply_dots<T, 1, true>, grd, blk, 0, s, L0, npml, ac, hw, u, y, aux, partials, pstride, st, T(1));
    else if (mode == 1)
        launch_pdl(k_apply_dots<T, 1, false>, grd, blk, 0, s, L0, npml, ac, hw, u, y, aux, partials, pstride, st, T(1));
    else if (vd)
        launch_pdl(k_apply_dots<T, 2, true>, grd, blk, 0, s, L0, npml, ac, hw, u, y, aux, partials, pstride, st, T(1));
    else
        launch_pdl(k_apply_dots<T, 2, false>, grd, blk, 0, s, L0, npml, ac, hw, u, y, aux, partials, pstride, st, T(1));
}
template void launch_apply_dots<float>(int, const LevelDev&, int, double, const float*, const float*, float*,
                                       const float*, double*, int, RhsState*, int, cudaStream_t);
template void launch_apply_dots<double>(int, const LevelDev&, int, double, const double*, const double*, double*,
                                        const double*, double*, int, RhsState*, int, cudaStream_t);

// ======================================================= FP64 outer residual
// r = f - A u in FP64; writes the inner right-hand side rin = r in precision TI
// and decides, per right-hand side, whether refinement continues. GB300 issues
// FP64 at a small fraction of its FP32 rate, so this kernel is bound by FP64
// instructions, not bytes (GB300: about 1.7 FP64 operations per clock per SM,
// DADD, DMUL, DFMA and the double-to-float conversion alike). Each thread takes
// R64_ROWS consecutive rows of one column, so the block sum is paid once for all
// of them; interior nodes (outside the absorbing layer, four neighbours) sum
// the neighbours pairwise and fuse the diagonal product and the squared norm
// into FMAs; ||f||^2 is formed only on the first call of a solve.
constexpr int R64_ROWS = 8;

template <typename TI, bool VD>
__global__ void __launch_bounds__(256) k_resid64(LevelDev L, int npml, double acoef, const double* __restrict__ w2,
                                                 const double* __restrict__ f, const double* __restrict__ u,
                                                 TI* __restrict__ rin, double* partials, int pstride, RhsState* st,
                                                 double tol, double inner_floor, double inner_fac, int first) {
    __shared__ double sh[64];
    const int b = blockIdx.z;
    if (!st[b].outer_active) return;
    const int nx = L.nx, nz = L.nz;
    const int ix = blockIdx.x * 32 + threadIdx.x, iz0 = (blockIdx.y * 8 + threadIdx.y) * R64_ROWS;
    const size_t n = (size_t)nx * nz;
    const double* ub = u + 2 * n * b;
    const double* fb = f + 2 * n * b;
    const double* mb = static_cast<const double*>(L.m2) + (size_t)b * L.mstride;
    typename C2<TI>::type* rb = reinterpret_cast<typename C2<TI>::type*>(rin) + n * b;
    const double sw = L.h2 * w2[b];
    double v[2] = {0.0, 0.0};
    if (ix < nx) {
#pragma unroll
        for (int k = 0; k < R64_ROWS; ++k) {
            const int iz = iz0 + k;
            if (iz >= nz) break;
            const size_t i = (size_t)iz * nx + ix;
            const double s = sw * mb[i];
            const cx<double> c = ldc(ub, i);
            const cx<double> fv = ldc(fb, i);
            cx<double> r;
            if constexpr (VD) {
                const double a = layer_alpha_t<double>(ix, iz, nx, nz, npml, acoef);
                r = fv - fine_apply_point<double, true>(L, ub, i, ix, iz, s, a, c);
            } else {
                // f - (4 - s) u + N u (+ the damping term in the layer), N u the sum of the neighbours
                const double g = 4.0 - s;
                const int d = layer_depth(ix, iz, nx, nz, npml);
                if (d == 0 && ix > 0 && ix + 1 < nx && iz > 0 && iz + 1 < nz) {
                    const cx<double> w = ldc(ub, i - 1), e = ldc(ub, i + 1), no = ldc(ub, i - nx), so = ldc(ub, i + nx);
                    const cx<double> nb = (w + e) + (no + so);
                    r = cx<double>(fma(-g, c.re, fv.re) + nb.re, fma(-g, c.im, fv.im) + nb.im);
                } else {
                    cx<double> nb(0.0, 0.0);
                    if (ix > 0) nb = nb + ldc(ub, i - 1);
                    if (ix + 1 < nx) nb = nb + ldc(ub, i + 1);
                    if (iz > 0) nb = nb + ldc(ub, i - nx);
                    if (iz + 1 < nz) nb = nb + ldc(ub, i + nx);
                    const double sa = s * (acoef * (double)(d * d));
                    r = cx<double>((fv.re - (g * c.re - sa * c.im)) + nb.re, (fv.im - (g * c.im + sa * c.re)) + nb.im);
                }
            }
            v[0] = fma(r.re, r.re, fma(r.im, r.im, v[0]));
            if (first) v[1] = fma(fv.re, fv.re, fma(fv.im, fv.im, v[1]));
            rb[i] = {(TI)r.re, (TI)r.im};
        }
    }
    const int nblk = gridDim.x * gridDim.y, blk = blockIdx.y * gridDim.x + blockIdx.x;
    if (last_block_reduce<2>(v, sh, partials + (size_t)b * pstride, nblk, blk, &st[b].counter[0])) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            RhsState& S = st[b];
            if (first) S.fnorm2 = v[1];
            double rel = S.fnorm2 > 0.0 ? sqrt(v[0] / S.fnorm2) : 0.0;
            S.relres = rel;
            int go = (rel > tol) && (S.iters < S.max_it);
            S.outer_active = go;
            S.active = go;
            double t = rel > 0.0 ? inner_fac * tol / rel : 1.0;
            S.tol_rel = t > inner_floor ? t : inner_floor;
        }
    }
}

template <typename TI>
void launch_resid64(const LevelDev& L0, int npml, double amax, const double* w2, const double* f, const double* u,
                    TI* rin, double* partials, int pstride, RhsState* st, double tol, double inner_floor,
                    double inner_fac, int first, int nrhs, cudaStream_t s) {
    const double n0 = (double)L0.nx * L0.nz;
    ProfScope prof(PK_RESID64, L0.nx, L0.nz,
                   n0 * ((32.0 + 2 * sizeof(TI)) * nrhs + 8.0 * (L0.mstride ? nrhs : 1) * (L0.rho ? 4 : 1)), s);
    dim3 blk(32, 8), grd((L0.nx + 31) / 32, (L0.nz + 8 * R64_ROWS - 1) / (8 * R64_ROWS), nrhs);
    if (L0.rho)
        k_resid64<TI, true><<<grd, blk, 0, s>>>(L0, npml, layer_coef(npml, amax), w2, f, u, rin, partials, pstride,
                                                st, tol, inner_floor, inner_fac, first);
    else
        k_resid64<TI, false><<<grd, blk, 0, s>>>(L0, npml, layer_coef(npml, amax), w2, f, u, rin, partials, pstride,
                                                 st, tol, inner_floor, inner_fac, first);
}
template void launch_resid64<float>(const LevelDev&, int, double, const double*, const double*, const double*, float*, double*, int, RhsState*, double, double, double, int, int, cudaStream_t);
template void launch_resid64<double>(const LevelDev&, int, double, const double*, const double*, const double*, double*, double*, int, RhsState*, double, double, double, int, int, cudaStream_t);

// u += x for the right-hand sides still refining; an inner solve whose residual
// overflowed (a divergent unpreconditioned iteration) leaves u, the best iterate
// so far, as it was.
template <typename TI>
__global__ void k_refine(const TI* __restrict__ x, double* __restrict__ u, const RhsState* st, size_t n) {
    const int b = blockIdx.z;
    if (!st[b].outer_active || !isfinite(st[b].rnorm2)) return;
    const TI* xb = x + 2 * n * b;
    double* ub = u + 2 * n * b;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        cx<TI> d = ldc(xb, i);
        cx<double> c = ldcc(ub, i);
        stc(ub, i, cx<double>(c.re + (double)d.re, c.im + (double)d.im));
    }
}

template <typename TI>
void launch_refine(const TI* x, double* u, const RhsState* st, size_t n, int nrhs, cudaStream_t s) {
    ProfScope prof(PK_REFINE, (int)n, 1, (double)n * nrhs * (32.0 + 2 * sizeof(TI)), s);
    k_refine<TI><<<dim3(grid1d(n), 1, nrhs), 256, 0, s>>>(x, u, st, n);
}
template void launch_refine<float>(const float*, double*, const RhsState*, size_t, int, cudaStream_t);
template void launch_refine<double>(const double*, double*, const RhsState*, size_t, int, cudaStream_t);

// ============================================================== BiCGSTAB
// Right-preconditioned BiCGSTAB, complex inner product <a, b> = sum conj(a) b.
template <typename T>
__global__ void __launch_bounds__(256) k_bicg_init(const T* __restrict__ bv, T* x, T* r, T* rh, T* p, T* v,
                                                   double* partials, int pstride, RhsState* st, int* nactive,
                                                   size_t n) {
    __shared__ double sh[32];
    const int b = blockIdx.z;
    if (!st[b].outer_active) return;
    const size_t off = n * b;
    T a0 = 0;
    const cx<T> z(0, 0);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        cx<T> c = ldc(bv, off + i);
        stc(x, off + i, z);
        stc(r, off + i, c);
        stc(rh, off + i, c);
        stc(p, off + i, z);
        stc(v, off + i, z);
        a0 += c.re * c.re + c.im * c.im;
    }
    const T vv[1] = {a0};
    double acc[1];
    if (last_block_reduce_t<1, T>(vv, acc, sh, partials + (size_t)b * pstride, gridDim.x, blockIdx.x, &st[b].counter[1])) {
        if (threadIdx.x == 0) {
            RhsState& S = st[b];
            S.bnorm2 = acc[0];
            S.rnorm2 = acc[0];
            S.rho[0] = acc[0]; S.rho[1] = 0.0;
            S.alpha[0] = 1.0; S.alpha[1] = 0.0;
            S.omega[0] = 1.0; S.omega[1] = 0.0;
            S.beta[0] = 0.0; S.beta[1] = 0.0;
            S.flag = FLAG_RUNNING;
            S.active = acc[0] > 0.0;
            if (S.active) atomicAdd(nactive, 1);
        }
    }
}

template <typename T>
void launch_bicg_init(const T* b, T* x, T* r, T* rh, T* p, T* v, double* partials, int pstride, RhsState* st,
                      int* nactive, size_t n, int nrhs, cudaStream_t s) {
    ProfScope prof(PK_BICG_INIT, (int)n, 1, (double)n * nrhs * 12.0 * sizeof(T), s);
    k_bicg_init<T><<<dim3(grid1d(n), 1, nrhs), 256, 0, s>>>(b, x, r, rh, p, v, partials, pstride, st, nactive, n);
}

// Residual replacement ("reliable update") between refinement steps: r is
// replaced by the new true residual rin, x restarts from zero, and the Krylov
// recurrence continues with the same shadow vector and search direction:
// rho' = <rh, r>, beta = (rho' / rho) (alpha / omega), where rho, alpha and
// omega are those of the last iteration (k_bicg_xr does not advance rho on the
// iteration that retires a right-hand side). A right-hand side
// whose last inner solve did not converge (breakdown or cap) restarts instead.
template <typename T>
__global__ void __launch_bounds__(256) k_bicg_resume(const T* __restrict__ rin, T* x, T* r, T* rh, T* p, T* v,
                                                     double* partials, int pstride, RhsState* st, int* nactive,
                                                     size_t n) {
    __shared__ double sh[96];
    const int b = blockIdx.z;
    if (!st[b].outer_active) return;
    const bool restart = st[b].flag != FLAG_CONVERGED;
    const size_t off = n * b;
    const cx<T> z(0, 0);
    T a0 = 0, a1 = 0, a2 = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const cx<T> c = ldc(rin, off + i);
        stc(x, off + i, z);
        stc(r, off + i, c);
        cx<T> q;
        if (restart) {
            stc(rh, off + i, c);
            stc(p, off + i, z);
            stc(v, off + i, z);
            q = c;
        } else {
            q = ldcc(rh, off + i);
        }
        a0 += q.re * c.re + q.im * c.im;
        a1 += q.re * c.im - q.im * c.re;
        a2 += c.re * c.re + c.im * c.im;
    }
    const T vv[3] = {a0, a1, a2};
    double acc[3];
    if (last_block_reduce_t<3, T>(vv, acc, sh, partials + (size_t)b * pstride, gridDim.x, blockIdx.x, &st[b].counter[1])) {
        if (threadIdx.x == 0) {
            RhsState& S = st[b];
            S.bnorm2 = acc[2];
            S.rnorm2 = acc[2];
            if (restart) {
                S.rho[0] = acc[2]; S.rho[1] = 0.0;
                S.alpha[0] = 1.0; S.alpha[1] = 0.0;
                S.omega[0] = 1.0; S.omega[1] = 0.0;
                S.beta[0] = 0.0; S.beta[1] = 0.0;
            } else {
                const double rr = S.rho[0], ri = S.rho[1], d1 = rr * rr + ri * ri;
                const double orr = S.omega[0], oi = S.omega[1], d2 = orr * orr + oi * oi;
                if (d1 > 0.0 && d2 > 0.0) {
                    const double qr = (acc[0] * rr + acc[1] * ri) / d1, qi = (acc[1] * rr - acc[0] * ri) / d1;
                    const double wr = (S.alpha[0] * orr + S.alpha[1] * oi) / d2;
                    const double wi = (S.alpha[1] * orr - S.alpha[0] * oi) / d2;
                    S.beta[0] = qr * wr - qi * wi;
                    S.beta[1] = qr * wi + qi * wr;
                } else {
                    S.beta[0] = 0.0; S.beta[1] = 0.0;
                }
                S.rho[0] = acc[0];
                S.rho[1] = acc[1];
            }
            S.flag = FLAG_RUNNING;
            S.active = acc[2] > 0.0;
            if (S.active) atomicAdd(nactive, 1);
        }
    }
}

template <typename T>
void launch_bicg_resume(const T* rin, T* x, T* r, T* rh, T* p, T* v, double* partials, int pstride, RhsState* st,
                        int* nactive, size_t n, int nrhs, cudaStream_t s) {
    ProfScope prof(PK_BICG_RESUME, (int)n, 1, (double)n * nrhs * 12.0 * sizeof(T), s);
    k_bicg_resume<T><<<dim3(grid1d(n), 1, nrhs), 256, 0, s>>>(rin, x, r, rh, p, v, partials, pstride, st, nactive, n);
}
template void launch_bicg_resume<float>(const float*, float*, float*, float*, float*, float*, double*, int, RhsState*,
                                        int*, size_t, int, cudaStream_t);
template void launch_bicg_resume<double>(const double*, double*, double*, double*, double*, double*, double*, int,
                                         RhsState*, int*, size_t, int, cudaStream_t);

template <typename T>
__global__ void k_bicg_p(const T* __restrict__ r, T* __restrict__ p, const T* __restrict__ v, const RhsState* st,
                         size_t n) {
    pdl_trigger();
    pdl_wait();
    const int b = blockIdx.z;
    if (!st[b].active) return;
    __shared__ T sc[4];
    if (threadIdx.x == 0) {
        sc[0] = (T)st[b].beta[0]; sc[1] = (T)st[b].beta[1]; sc[2] = (T)st[b].omega[0]; sc[3] = (T)st[b].omega[1];
    }
    __syncthreads();
    const cx<T> beta(sc[0], sc[1]);
    const cx<T> om(sc[2], sc[3]);
    const size_t off = n * b;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        cx<T> pv = ldcc(p, off + i);
        stc(p, off + i, ldc(r, off + i) + beta * (pv - om * ldc(v, off + i)));
    }
}

template <typename T>
void launch_bicg_p(const T* r, T* p, const T* v, const RhsState* st, size_t n, int nrhs, cudaStream_t s) {
    ProfScope prof(PK_BICG_P, (int)n, 1, (double)n * nrhs * 8.0 * sizeof(T), s);
    launch_pdl(k_bicg_p<T>, dim3(grid1d(n), 1, nrhs), dim3(256), 0, s, r, p, v, st, n);
}

template <typename T>
__global__ void k_bicg_s(const T* __restrict__ r, const T* __restrict__ v, T* __restrict__ sv, const RhsState* st,
                         size_t n) {
    pdl_trigger();
    pdl_wait();
    const int b = blockIdx.z;
    if (!st[b].active) return;
    __shared__ T sc[2];
    if (threadIdx.x == 0) { sc[0] = (T)st[b].alpha[0]; sc[1] = (T)st[b].alpha[1]; }
    __syncthreads();
    const cx<T> al(sc[0], sc[1]);
    const size_t off = n * b;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        stc(sv, off + i, ldc(r, off + i) - al * ldc(v, off + i));
}

template <typename T>
void launch_bicg_s(const T* r, const T* v, T* sv, const RhsState* st, size_t n, int nrhs, cudaStream_t s) {
    ProfScope prof(PK_BICG_S, (int)n, 1, (double)n * nrhs * 6.0 * sizeof(T), s);
    launch_pdl(k_bicg_s<T>, dim3(grid1d(n), 1, nrhs), dim3(256), 0, s, r, v, sv, st, n);
}

template <typename T>
__global__ void __launch_bounds__(256) k_bicg_xr(T* x, const T* __restrict__ ph, const T* __restrict__ shv,
                                                 const T* __restrict__ sv, const T* __restrict__ t,
                                                 const T* __restrict__ rh, T* r, double* partials, int pstride,
                                                 RhsState* st, int* nactive, size_t n) {
    __shared__ double sh[96];
    pdl_trigger();
    pdl_wait();
    const int b = blockIdx.z;
    if (!st[b].active) return;
    __shared__ T sc[4];
    if (threadIdx.x == 0) {
        sc[0] = (T)st[b].alpha[0]; sc[1] = (T)st[b].alpha[1]; sc[2] = (T)st[b].omega[0]; sc[3] = (T)st[b].omega[1];
    }
    __syncthreads();
    const cx<T> al(sc[0], sc[1]);
    const cx<T> om(sc[2], sc[3]);
    const size_t off = n * b;
    T a0 = 0, a1 = 0, a2 = 0;   // <rh, r> (re, im), <r, r>
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        cx<T> xv = ldcc(x, off + i);
        stc(x, off + i, xv + al * ldc(ph, off + i) + om * ldc(shv, off + i));
        cx<T> rn = ldc(sv, off + i) - om * ldc(t, off + i);
        stc(r, off + i, rn);
        cx<T> q = ldc(rh, off + i);
        a0 += q.re * rn.re + q.im * rn.im;
        a1 += q.re * rn.im - q.im * rn.re;
        a2 += rn.re * rn.re + rn.im * rn.im;
    }
    const T vv[3] = {a0, a1, a2};
    double acc[3];
    if (last_block_reduce_t<3, T>(vv, acc, sh, partials + (size_t)b * pstride, gridDim.x, blockIdx.x, &st[b].counter[2])) {
        if (threadIdx.x == 0) {
            RhsState& S = st[b];
            S.iters += 1;
            S.rnorm2 = acc[2];
            const double tl = S.tol_rel;
            int done = 0;
            if (S.flag == FLAG_BREAKDOWN) done = 1;
            else if (acc[2] <= tl * tl * S.bnorm2) { done = 1; S.flag = FLAG_CONVERGED; }
            else if (S.iters >= S.max_it) { done = 1; S.flag = FLAG_MAXIT; }
            else {
                // beta = (rho_new / rho) * (alpha / omega)
                double rr = S.rho[0], ri = S.rho[1];
                double d1 = rr * rr + ri * ri;
                double orr = S.omega[0], oi = S.omega[1];
                double d2 = orr * orr + oi * oi;
                if (d1 == 0.0 || d2 == 0.0 || !(acc[0] * acc[0] + acc[1] * acc[1] > 0.0)) {
                    done = 1; S.flag = FLAG_BREAKDOWN;
                } else {
                    double qr = (acc[0] * rr + acc[1] * ri) / d1, qi = (acc[1] * rr - acc[0] * ri) / d1;
                    double wr = (S.alpha[0] * orr + S.alpha[1] * oi) / d2, wi = (S.alpha[1] * orr - S.alpha[0] * oi) / d2;
                    S.beta[0] = qr * wr - qi * wi;
                    S.beta[1] = qr * wi + qi * wr;
                    S.rho[0] = acc[0];
                    S.rho[1] = acc[1];
                }
            }
            if (done) { S.active = 0; atomicSub(nactive, 1); }
        }
    }
}

template <typename T>
void launch_bicg_xr(T* x, const T* ph, const T* shv, const T* sv, const T* t, const T* rh, T* r, double* partials,
                    int pstride, RhsState* st, int* nactive, size_t n, int nrhs, cudaStream_t s) {
    ProfScope prof(PK_BICG_XR, (int)n, 1, (double)n * nrhs * 16.0 * sizeof(T), s);
    launch_pdl(k_bicg_xr<T>, dim3(grid1d(n), 1, nrhs), dim3(256), 0, s, x, ph, shv, sv, t, rh, r, partials, pstride, st,
               nactive, n);
}

// ===================================================== Galerkin operators
// Complex coefficient of stored stencil entry k (0 centre, 1 east, 2 north,
// 3 north-east, 4 north-west) at node i: G_k - hw (b1 - j b2) K_k.
template <typename T>
__device__ __forceinline__ cx<T> gcoef(const T* __restrict__ gk, size_t n, size_t i, int k, T hb1, T hb2) {
    const T g = __ldg(gk + (size_t)k * n + i), q = __ldg(gk + (size_t)(5 + k) * n + i);
    return cx<T>(g - hb1 * q, hb2 * q);
}

// M u at node (ix, iz) of a Galerkin level; U points at u of that node inside a
// row-major tile of row pitch W whose out-of-grid entries are zero.
template <typename T>
__device__ __forceinline__ cx<T> mop9(const T* __restrict__ gk, size_t n, int nx, int nz, int ix, int iz,
                                      const cx<T>* U, int W, T hb1, T hb2) {
    const size_t i = (size_t)iz * nx + ix;
    cx<T> acc = gcoef(gk, n, i, 0, hb1, hb2) * U[0];
    const bool e = ix + 1 < nx, w = ix > 0, no = iz + 1 < nz, so = iz > 0;
    if (e) acc = acc + gcoef(gk, n, i, 1, hb1, hb2) * U[1];
    if (w) acc = acc + gcoef(gk, n, i - 1, 1, hb1, hb2) * U[-1];
    if (no) acc = acc + gcoef(gk, n, i, 2, hb1, hb2) * U[W];
    if (so) acc = acc + gcoef(gk, n, i - nx, 2, hb1, hb2) * U[-W];
    if (no && e) acc = acc + gcoef(gk, n, i, 3, hb1, hb2) * U[W + 1];
    if (so && w) acc = acc + gcoef(gk, n, i - nx - 1, 3, hb1, hb2) * U[-W - 1];
    if (no && w) acc = acc + gcoef(gk, n, i, 4, hb1, hb2) * U[W - 1];
    if (so && e) acc = acc + gcoef(gk, n, i - nx + 1, 4, hb1, hb2) * U[-W + 1];
    return acc;
}

// Shifted-Laplace diagonal and M u for either kind of level, u in a tile.
template <typename T, bool GAL>
struct LevelOp {
    const T* m2;   // finest level
    const T* gk;   // Galerkin levels
    size_t n;
    int nx, nz;
    T hw, b1, b2;  // hw = (h_0 omega)^2
    __device__ __forceinline__ cx<T> diag(size_t i) const {
        if constexpr (GAL) return gcoef(gk, n, i, 0, hw * b1, hw * b2);
        else {
            const T s = hw * __ldg(m2 + i);
            return cx<T>(T(4) - s * b1, s * b2);
        }
    }
    __device__ __forceinline__ cx<T> apply(int ix, int iz, const cx<T>* U, int W) const {
        if constexpr (GAL) return mop9(gk, n, nx, nz, ix, iz, U, W, hw * b1, hw * b2);
        else {
            const size_t i = (size_t)iz * nx + ix;
            const T s = hw * __ldg(m2 + i);
            const cx<T> c = U[0];
            cx<T> mu((T(4) - s * b1) * c.re - s * b2 * c.im, (T(4) - s * b1) * c.im + s * b2 * c.re);
            return mu - U[-1] - U[1] - U[-W] - U[W];
        }
    }
};

template <typename T, bool GAL>
__device__ __forceinline__ LevelOp<T, GAL> level_op(const LevelDev& L, int b, T hwb) {
    LevelOp<T, GAL> op;
    op.n = (size_t)L.nx * L.nz;
    op.nx = L.nx;
    op.nz = L.nz;
    op.m2 = GAL ? nullptr : static_cast<const T*>(L.m2) + (size_t)b * L.mstride;
    op.gk = GAL ? static_cast<const T*>(L.gk) + (size_t)b * L.gkstride : nullptr;
    op.hw = hwb;   // (h_0 omega_b)^2 on every level: the finest level's spacing, Galerkin below
    return op;
}

// Builds level l's Galerkin stencils from level l - 1 (one thread per coarse
// node, FP64): coef(I -> J) = sum_a sum_b P[a, I] M[a, b] P[b, J] over the fine
// 3 x 3 support a of I and the fine 9-point neighbours b of a, separately for G
// and K. The finest level's G is the 5-point Laplacian and K = diag(m^2).
__device__ __forceinline__ double w1d(int d) { return d == 0 ? 1.0 : ((d == 1 || d == -1) ? 0.5 : 0.0); }

__device__ __forceinline__ void fine_stencil(bool fine0, const double* m2, const double* gk, size_t n, int nx, int nz,
                                             int ax, int az, int dx, int dz, double* g, double* k) {
    // coefficient of fine operator from a = (ax, az) to b = a + (dx, dz); both in the grid
    *g = 0.0;
    *k = 0.0;
    if (fine0) {
        if (dx == 0 && dz == 0) { *g = 4.0; *k = m2[(size_t)az * nx + ax]; }
        else if ((dx == 0) != (dz == 0)) *g = -1.0;
        return;
    }
    // stored forward entries: (1,0) e, (0,1) n, (1,1) ne, (-1,1) nw
    int sx = ax, sz = az, ent;
    if (dx == 0 && dz == 0) ent = 0;
    else if (dz == 0) { ent = 1; if (dx < 0) sx = ax - 1; }
    else if (dx == 0) { ent = 2; if (dz < 0) sz = az - 1; }
    else if (dx == dz) { ent = 3; if (dx < 0) { sx = ax - 1; sz = az - 1; } }
    else { ent = 4; if (dz < 0) { sx = ax + 1; sz = az - 1; } }
    const size_t i = (size_t)sz * nx + sx;
    *g = gk[(size_t)ent * n + i];
    *k = gk[(size_t)(5 + ent) * n + i];
}

__global__ void k_galerkin(int fine0, const double* __restrict__ m2f, const double* __restrict__ gkf, int nxf, int nzf,
                           size_t mstride_f, size_t gstride_f, double* __restrict__ gkc, float* __restrict__ gkc32,
                           int nxc, int nzc) {
    const size_t nf = (size_t)nxf * nzf, nc = (size_t)nxc * nzc;
    const int model = blockIdx.y;
    const double* m2 = fine0 ? m2f + (size_t)model * mstride_f : nullptr;
    const double* gk = fine0 ? nullptr : gkf + (size_t)model * gstride_f;
    double* out = gkc + (size_t)model * kGalerkinCoefs * nc;
    float* out32 = gkc32 + (size_t)model * kGalerkinCoefs * nc;
    const int ddx[5] = {0, 1, 0, 1, -1}, ddz[5] = {0, 0, 1, 1, 1};
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < nc; c += (size_t)gridDim.x * blockDim.x) {
        const int Ix = (int)(c % nxc), Iz = (int)(c / nxc);
        double G[5] = {0, 0, 0, 0, 0}, K[5] = {0, 0, 0, 0, 0};
        for (int az = 2 * Iz; az <= 2 * Iz + 2; ++az) {
            if (az >= nzf) continue;
            for (int ax = 2 * Ix; ax <= 2 * Ix + 2; ++ax) {
                if (ax >= nxf) continue;
                const double pa = w1d(ax - (2 * Ix + 1)) * w1d(az - (2 * Iz + 1));
                for (int dz = -1; dz <= 1; ++dz) {
                    const int bz = az + dz;
                    if (bz < 0 || bz >= nzf) continue;
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int bx = ax + dx;
                        if (bx < 0 || bx >= nxf) continue;
                        double g, k;
                        fine_stencil(fine0, m2, gk, nf, nxf, nzf, ax, az, dx, dz, &g, &k);
                        if (g == 0.0 && k == 0.0) continue;
                        for (int e = 0; e < 5; ++e) {
                            const int Jx = Ix + ddx[e], Jz = Iz + ddz[e];
                            if (Jx < 0 || Jx >= nxc || Jz >= nzc) continue;
                            const double pb = w1d(bx - (2 * Jx + 1)) * w1d(bz - (2 * Jz + 1));
                            if (pb == 0.0) continue;
                            G[e] += pa * g * pb;
                            K[e] += pa * k * pb;
                        }
                    }
                }
            }
        }
        for (int e = 0; e < 5; ++e) {
            out[(size_t)e * nc + c] = G[e];
            out[(size_t)(5 + e) * nc + c] = K[e];
            out32[(size_t)e * nc + c] = (float)G[e];
            out32[(size_t)(5 + e) * nc + c] = (float)K[e];
        }
    }
}

void launch_galerkin(const helm_model* m, int l, cudaStream_t s) {
    const Level& F = m->lv[l - 1];
    const Level& C = m->lv[l];
    const int fine0 = (l == 1) && !m->vd;   // with a density the finest level is stored like a coarse one
    k_galerkin<<<dim3(grid1d(C.n()), m->nmodels), 256, 0, s>>>(fine0, F.m2d, F.gkd, F.nx, F.nz, F.n(),
                                                              kGalerkinCoefs * F.n(), C.gkd, C.gkf, C.nx, C.nz);
}

// ================================ Galerkin grid levels: one launch per level
// Tile bodies in helm_gal_tiles.cuh; each block is one tile of one right-hand
// side. The coefficient staging reads only model data, so it runs before the
// wait on the previous kernel (programmatic dependent launch).

// restriction (CORRECT = false: zero-guess smoothing; true: u2 = wj D^-1 f + P e)
template <typename T, bool CORRECT, int GRCX, int GRCZ, int NT>
__global__ void __launch_bounds__(NT) k_restrict_g(LevelDev Lf, LevelDev Lc, const T* __restrict__ hwv, T b1, T b2,
                                                   T wj, const T* __restrict__ f, const T* __restrict__ ec,
                                                   T* __restrict__ fc, const RhsState* st) {
    __shared__ RestrictTile<T, GRCX, GRCZ, NT> sm;
    pdl_trigger();
    const int b = blockIdx.z;
    restrict_tile_stage<T, GRCX, GRCZ, NT>(sm, Lf, blockIdx.x, blockIdx.y, b, hwv[b], b1, b2, threadIdx.x);   // model data
    pdl_wait();
    if (!rhs_active(st, b)) return;
    restrict_tile_work<T, CORRECT, GRCX, GRCZ, NT, false>(sm, Lf, Lc, wj, f, ec, fc, blockIdx.x, blockIdx.y, b,
                                                          threadIdx.x, BlockSync{});
}

template <typename T, int GPX, int GPZ>
__global__ void __launch_bounds__(GPX * GPZ) k_prolong_g(LevelDev Lf, LevelDev Lc, const T* __restrict__ hwv, T b1,
                                                         T b2, T wj, const T* __restrict__ f, const T* __restrict__ ec,
                                                         T* __restrict__ out, const RhsState* st, int accumulate) {
    __shared__ ProlongTile<T, GPX, GPZ> sm;
    pdl_trigger();
    const int b = blockIdx.z;
    prolong_tile_stage<T, GPX, GPZ>(sm, Lf, blockIdx.x, blockIdx.y, b, hwv[b], b1, b2, threadIdx.x);   // model data
    pdl_wait();
    if (!rhs_active(st, b)) return;
    prolong_tile_work<T, GPX, GPZ, false>(sm, Lf, Lc, wj, f, ec, out, accumulate, blockIdx.x, blockIdx.y, b,
                                          threadIdx.x, BlockSync{});
}

// restriction that starts the second coarse correction of an F-cycle (tile body
// resid_restrict_tile_work): right-hand side g = f - M e, written to g, then
// restricted as k_restrict_g does
template <typename T, int GRCX, int GRCZ, int NT>
__global__ void __launch_bounds__(NT) k_resid_restrict_g(LevelDev Lf, LevelDev Lc, const T* __restrict__ hwv, T b1,
                                                         T b2, T wj, const T* __restrict__ f, const T* __restrict__ e,
                                                         T* __restrict__ g, T* __restrict__ fc, const RhsState* st) {
    __shared__ ResidRestrictTile<T, GRCX, GRCZ, NT> sm;
    pdl_trigger();
    const int b = blockIdx.z;
    resid_restrict_tile_stage<T, GRCX, GRCZ, NT>(sm, Lf, blockIdx.x, blockIdx.y, b, hwv[b], b1, b2, threadIdx.x);
    pdl_wait();
    if (!rhs_active(st, b)) return;
    resid_restrict_tile_work<T, GRCX, GRCZ, NT, false>(sm, Lf, Lc, wj, f, e, g, fc, blockIdx.x, blockIdx.y, b,
                                                       threadIdx.x, BlockSync{});
}

template <typename T, int GRCX, int GRCZ, int NT>
static void launch_resid_restrict_shape(const LevelDev& Lf, const LevelDev& Lc, const T* w2, double b1, double b2,
                                        double wj, const T* f, const T* e, T* g, T* fc, const RhsState* st, int nrhs,
                                        cudaStream_t s) {
    dim3 grd((Lc.nx + GRCX - 1) / GRCX, (Lc.nz + GRCZ - 1) / GRCZ, nrhs);
    launch_pdl(k_resid_restrict_g<T, GRCX, GRCZ, NT>, grd, dim3(NT), 0, s, Lf, Lc, w2, (T)b1, (T)b2, (T)wj, f, e, g,
               fc, st);
}

template <typename T>
void launch_resid_restrict(const LevelDev& Lf, const LevelDev& Lc, const T* w2, double b1, double b2, double wj,
                           const T* f, const T* e, T* g, T* fc, const RhsState* st, int nrhs, cudaStream_t s,
                           int tile) {
    const double nf = (double)Lf.nx * Lf.nz, nc = (double)Lc.nx * Lc.nz, es = 2.0 * sizeof(T);
    // f, e and g on this level, the coarse output, the ten Galerkin coefficients per node and model
    ProfScope prof(PK_RESID_RESTRICT, Lf.nx, Lf.nz,
                   (3 * nf + nc) * es * nrhs + nf * sizeof(T) * kGalerkinCoefs * (Lf.gkstride ? nrhs : 1), s);
    if constexpr (sizeof(T) == 4) {
        if (tile == 0)
            launch_resid_restrict_shape<T, 8, 8, 64>(Lf, Lc, w2, b1, b2, wj, f, e, g, fc, st, nrhs, s);
        else
            launch_resid_restrict_shape<T, 8, 8, 128>(Lf, Lc, w2, b1, b2, wj, f, e, g, fc, st, nrhs, s);
    } else {
        launch_resid_restrict_shape<T, 8, 4, 64>(Lf, Lc, w2, b1, b2, wj, f, e, g, fc, st, nrhs, s);
    }
}
template void launch_resid_restrict<float>(const LevelDev&, const LevelDev&, const float*, double, double, double,
                                           const float*, const float*, float*, float*, const RhsState*, int,
                                           cudaStream_t, int);
template void launch_resid_restrict<double>(const LevelDev&, const LevelDev&, const double*, double, double, double,
                                            const double*, const double*, double*, double*, const RhsState*, int,
                                            cudaStream_t, int);

// two prolongations in one launch (tile body prolong2_tile_work): level l + 1's
// from e of level l + 2, then level l's
template <typename T, int GPX, int GPZ>
__global__ void __launch_bounds__(GPX * GPZ) k_prolong2_g(LevelDev Lf, LevelDev Lm, LevelDev Lc,
                                                          const T* __restrict__ hwv, T b1, T b2, T wj,
                                                          const T* __restrict__ fl, const T* __restrict__ fm,
                                                          const T* __restrict__ ec, const T* em, T* out,
                                                          const RhsState* st, int acc_f, int acc_m) {
    __shared__ Prolong2Tile<T, GPX, GPZ> sm;
    pdl_trigger();
    const int b = blockIdx.z;
    prolong2_tile_stage<T, GPX, GPZ>(sm, Lf, Lm, blockIdx.x, blockIdx.y, b, hwv[b], b1, b2, threadIdx.x);
    pdl_wait();
    if (!rhs_active(st, b)) return;
    prolong2_tile_work<T, GPX, GPZ, false>(sm, Lf, Lm, Lc, wj, fl, fm, ec, em, out, acc_f, acc_m, blockIdx.x,
                                           blockIdx.y, b, threadIdx.x, BlockSync{});
}

template <typename T, int GPX, int GPZ>
static void launch_prolong2_shape(const LevelDev& Lf, const LevelDev& Lm, const LevelDev& Lc, const T* w2, double b1,
                                  double b2, double wj, const T* fl, const T* fm, const T* ec, const T* em, T* out,
                                  const RhsState* st, int nrhs, cudaStream_t s, int acc_f, int acc_m) {
    dim3 grd((Lf.nx + GPX - 1) / GPX, (Lf.nz + GPZ - 1) / GPZ, nrhs);
    launch_pdl(k_prolong2_g<T, GPX, GPZ>, grd, dim3(GPX * GPZ), 0, s, Lf, Lm, Lc, w2, (T)b1, (T)b2, (T)wj, fl, fm, ec,
               em, out, st, acc_f, acc_m);
}

template <typename T>
void launch_prolong2(const LevelDev& Lf, const LevelDev& Lm, const LevelDev& Lc, const T* w2, double b1, double b2,
                     double wj, const T* fl, const T* fm, const T* ec, const T* em, T* out, const RhsState* st,
                     int nrhs, cudaStream_t s, int acc_f, int acc_m, int tile) {
    const double nf = (double)Lf.nx * Lf.nz, nm = (double)Lm.nx * Lm.nz, nc = (double)Lc.nx * Lc.nz;
    const double es = 2.0 * sizeof(T);
    // the two prolongations' bytes without the level l + 1 correction between them:
    // f and the output of both levels (the outputs read too when accumulating), e of
    // level l + 2, the Galerkin coefficients of levels l and l + 1
    ProfScope prof(PK_PROLONG2_G, Lf.nx, Lf.nz,
                   (nf * (2 + acc_f) + nm * (1 + acc_m) + nc) * es * nrhs +
                       (nf + nm) * sizeof(T) * kGalerkinCoefs * (Lf.gkstride ? nrhs : 1),
                   s);
    if constexpr (sizeof(T) == 4) {
        if (tile != 0) {
            launch_prolong2_shape<T, 32, 8>(Lf, Lm, Lc, w2, b1, b2, wj, fl, fm, ec, em, out, st, nrhs, s, acc_f, acc_m);
            return;
        }
    }
    launch_prolong2_shape<T, 16, 8>(Lf, Lm, Lc, w2, b1, b2, wj, fl, fm, ec, em, out, st, nrhs, s, acc_f, acc_m);
}
template void launch_prolong2<float>(const LevelDev&, const LevelDev&, const LevelDev&, const float*, double, double,
                                     double, const float*, const float*, const float*, const float*, float*,
                                     const RhsState*, int, cudaStream_t, int, int, int);
template void launch_prolong2<double>(const LevelDev&, const LevelDev&, const LevelDev&, const double*, double, double,
                                      double, const double*, const double*, const double*, const double*, double*,
                                      const RhsState*, int, cudaStream_t, int, int, int);

// Several right-hand sides of one model per block (large batches): the tile's real
// Galerkin coefficients are staged once, before the wait on the previous kernel,
// and each right-hand side's complex coefficients are formed from them in shared
// memory; the tile work is that of the one-RHS kernels.
constexpr int kGalMultiRhs = 4;        // right-hand sides per block (2 and 8 measured slower)
constexpr int kGalMultiMinRhs = 16;    // batches above this size (one model) take these kernels

template <typename T, bool CORRECT, int GRCX, int GRCZ, int NT, int RB>
__global__ void __launch_bounds__(NT) k_restrict_gm(LevelDev Lf, LevelDev Lc, const T* __restrict__ hwv, T b1, T b2,
                                                    T wj, const T* __restrict__ f, const T* __restrict__ ec,
                                                    T* __restrict__ fc, const RhsState* st, int nrhs) {
    using RT = RestrictTile<T, GRCX, GRCZ, NT>;
    __shared__ RT sm;
    __shared__ GalReal<T, RT::GRFW, RT::GRFH> gr;
    pdl_trigger();
    stage_gal_real<T, RT::GRFW, RT::GRFH, NT>(gr, Lf, 2 * blockIdx.x * GRCX - 1, 2 * blockIdx.y * GRCZ - 1,
                                              threadIdx.x);
    pdl_wait();
    for (int r = 0; r < RB; ++r) {
        const int b = blockIdx.z * RB + r;
        if (b >= nrhs) break;
        if (!rhs_active(st, b)) continue;   // uniform in the block
        __syncthreads();                    // staging done; the previous right-hand side is done with sm
        const T hw = hwv[b];
        form_gal<T, RT::GRFW, RT::GRFH, NT>(sm.C, gr, hw * b1, hw * b2, threadIdx.x);
        restrict_tile_work<T, CORRECT, GRCX, GRCZ, NT, false>(sm, Lf, Lc, wj, f, ec, fc, blockIdx.x, blockIdx.y, b,
                                                              threadIdx.x, BlockSync{});
    }
}

template <typename T, int GPX, int GPZ, int RB>
__global__ void __launch_bounds__(GPX * GPZ) k_prolong_gm(LevelDev Lf, LevelDev Lc, const T* __restrict__ hwv, T b1,
                                                          T b2, T wj, const T* __restrict__ f,
                                                          const T* __restrict__ ec, T* __restrict__ out,
                                                          const RhsState* st, int accumulate, int nrhs) {
    using PT = ProlongTile<T, GPX, GPZ>;
    __shared__ PT sm;
    __shared__ GalReal<T, PT::RW, PT::RH> gr;
    pdl_trigger();
    stage_gal_real<T, PT::RW, PT::RH, PT::NT>(gr, Lf, blockIdx.x * GPX - 1, blockIdx.y * GPZ - 1, threadIdx.x);
    pdl_wait();
    for (int r = 0; r < RB; ++r) {
        const int b = blockIdx.z * RB + r;
        if (b >= nrhs) break;
        if (!rhs_active(st, b)) continue;   // uniform in the block
        __syncthreads();
        const T hw = hwv[b];
        form_gal<T, PT::RW, PT::RH, PT::NT>(sm.C, gr, hw * b1, hw * b2, threadIdx.x);
        prolong_tile_work<T, GPX, GPZ, false>(sm, Lf, Lc, wj, f, ec, out, accumulate, blockIdx.x, blockIdx.y, b,
                                              threadIdx.x, BlockSync{});
    }
}

template <typename T, bool CORRECT, int NT>
static void launch_restrict_gm(const LevelDev& Lf, const LevelDev& Lc, const T* w2, double b1, double b2, double wj,
                               const T* f, const T* ec, T* fc, const RhsState* st, int nrhs, cudaStream_t s) {
    dim3 grd((Lc.nx + 7) / 8, (Lc.nz + 7) / 8, (nrhs + kGalMultiRhs - 1) / kGalMultiRhs);
    launch_pdl(k_restrict_gm<T, CORRECT, 8, 8, NT, kGalMultiRhs>, grd, dim3(NT), 0, s, Lf, Lc, w2, (T)b1, (T)b2,
               (T)wj, f, ec, fc, st, nrhs);
}
template <typename T, int GPX, int GPZ>
static void launch_prolong_gm(const LevelDev& Lf, const LevelDev& Lc, const T* w2, double b1, double b2, double wj,
                              const T* f, const T* ec, T* out, const RhsState* st, int nrhs, cudaStream_t s,
                              int accumulate) {
    dim3 grd((Lf.nx + GPX - 1) / GPX, (Lf.nz + GPZ - 1) / GPZ, (nrhs + kGalMultiRhs - 1) / kGalMultiRhs);
    launch_pdl(k_prolong_gm<T, GPX, GPZ, kGalMultiRhs>, grd, dim3(GPX * GPZ), 0, s, Lf, Lc, w2, (T)b1, (T)b2, (T)wj,
               f, ec, out, st, accumulate, nrhs);
}

// Tile shapes of the complex64 Galerkin kernels, by the code the autotuner stores
// per level (kGalTiles choices; 1 is the default): restriction coarse tile
// (x, z) and prolongation fine tile (x, z), one thread per node of the tile. The
// shapes keep each block's shared memory within 48 KB.
//   0: 8 x 8 / 16 x 8,  1: 16 x 8 / 32 x 8,  2: 32 x 4 / 64 x 4,  3: 8 x 16 / 32 x 16,  4: 8 x 8 on 128
//   threads (two per coarse node, for short per-thread chains on small levels) / 128 x 2,
//   5 (restriction only): 8 x 16 on 256 threads (two per coarse node)
template <typename T, bool CORRECT, int GRCX, int GRCZ, int NT = GRCX * GRCZ>
void launch_restrict_g_shape(const LevelDev& Lf, const LevelDev& Lc, const T* w2, double b1, double b2, double wj,
                             const T* f, const T* ec, T* fc, const RhsState* st, int nrhs, cudaStream_t s) {
    dim3 grd((Lc.nx + GRCX - 1) / GRCX, (Lc.nz + GRCZ - 1) / GRCZ, nrhs);
    launch_pdl(k_restrict_g<T, CORRECT, GRCX, GRCZ, NT>, grd, dim3(NT), 0, s, Lf, Lc, w2, (T)b1, (T)b2, (T)wj, f,
               ec, fc, st);
}
template <typename T, bool CORRECT>
void launch_restrict_g(int tile, const LevelDev& Lf, const LevelDev& Lc, const T* w2, double b1, double b2, double wj,
                       const T* f, const T* ec, T* fc, const RhsState* st, int nrhs, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (nrhs > kGalMultiMinRhs && Lf.gkstride == 0) {   // 8 x 8 coarse tiles, 64 or 128 threads
            if (tile == 0) launch_restrict_gm<T, CORRECT, 64>(Lf, Lc, w2, b1, b2, wj, f, ec, fc, st, nrhs, s);
            else launch_restrict_gm<T, CORRECT, 128>(Lf, Lc, w2, b1, b2, wj, f, ec, fc, st, nrhs, s);
            return;
        }
        switch (tile) {
            case 0: launch_restrict_g_shape<T, CORRECT, 8, 8>(Lf, Lc, w2, b1, b2, wj, f, ec, fc, st, nrhs, s); return;
            case 2: launch_restrict_g_shape<T, CORRECT, 32, 4>(Lf, Lc, w2, b1, b2, wj, f, ec, fc, st, nrhs, s); return;
            case 3: launch_restrict_g_shape<T, CORRECT, 8, 16>(Lf, Lc, w2, b1, b2, wj, f, ec, fc, st, nrhs, s); return;
            case 4: launch_restrict_g_shape<T, CORRECT, 8, 8, 128>(Lf, Lc, w2, b1, b2, wj, f, ec, fc, st, nrhs, s); return;
            case 5: launch_restrict_g_shape<T, CORRECT, 8, 16, 256>(Lf, Lc, w2, b1, b2, wj, f, ec, fc, st, nrhs, s); return;
            default: break;
        }
    }
    launch_restrict_g_shape<T, CORRECT, GTile<T>::RCX, GTile<T>::RCZ>(Lf, Lc, w2, b1, b2, wj, f, ec, fc, st, nrhs, s);
}
template <typename T, int GPX, int GPZ>
void launch_prolong_g_shape(const LevelDev& Lf, const LevelDev& Lc, const T* w2, double b1, double b2, double wj,
                            const T* f, const T* ec, T* out, const RhsState* st, int nrhs, cudaStream_t s,
                            int accumulate) {
    dim3 grd((Lf.nx + GPX - 1) / GPX, (Lf.nz + GPZ - 1) / GPZ, nrhs);
    launch_pdl(k_prolong_g<T, GPX, GPZ>, grd, dim3(GPX * GPZ), 0, s, Lf, Lc, w2, (T)b1, (T)b2, (T)wj, f, ec, out, st,
               accumulate);
}
template <typename T>
void launch_prolong_g(int tile, const LevelDev& Lf, const LevelDev& Lc, const T* w2, double b1, double b2, double wj,
                      const T* f, const T* ec, T* out, const RhsState* st, int nrhs, cudaStream_t s, int accumulate) {
    if constexpr (sizeof(T) == 4) {
        if (nrhs > kGalMultiMinRhs && Lf.gkstride == 0) {   // fine tiles 16 x 8, 32 x 8 or 64 x 4
            if (tile == 0) launch_prolong_gm<T, 16, 8>(Lf, Lc, w2, b1, b2, wj, f, ec, out, st, nrhs, s, accumulate);
            else if (tile == 2) launch_prolong_gm<T, 64, 4>(Lf, Lc, w2, b1, b2, wj, f, ec, out, st, nrhs, s, accumulate);
            else launch_prolong_gm<T, 32, 8>(Lf, Lc, w2, b1, b2, wj, f, ec, out, st, nrhs, s, accumulate);
            return;
        }
        switch (tile) {
            case 0: launch_prolong_g_shape<T, 16, 8>(Lf, Lc, w2, b1, b2, wj, f, ec, out, st, nrhs, s, accumulate); return;
            case 2: launch_prolong_g_shape<T, 64, 4>(Lf, Lc, w2, b1, b2, wj, f, ec, out, st, nrhs, s, accumulate); return;
            case 3: launch_prolong_g_shape<T, 32, 16>(Lf, Lc, w2, b1, b2, wj, f, ec, out, st, nrhs, s, accumulate); return;
            case 4: launch_prolong_g_shape<T, 128, 2>(Lf, Lc, w2, b1, b2, wj, f, ec, out, st, nrhs, s, accumulate); return;
            default: break;
        }
    }
    launch_prolong_g_shape<T, GTile<T>::PX, GTile<T>::PZ>(Lf, Lc, w2, b1, b2, wj, f, ec, out, st, nrhs, s, accumulate);
}

// ======================================================== V-cycle: restrict
// From a level-l right-hand side f (zero initial guess): one damped-Jacobi
// sweep u1 = wj D^-1 f, residual r = f - M u1 and the restriction P^T r to
// level l + 1 (full weighting times 4: (1/4) [1 2 1; 2 4 2; 1 2 1] * r).
constexpr int RCX = 32, RCZ = 8;                    // coarse tile per block
constexpr int RFW = 2 * RCX + 3, RFH = 2 * RCZ + 3; // fine region (u1) per block

// Shuffles of a complex value from the lane below / above.
template <typename T> __device__ __forceinline__ cx<T> sh_up(cx<T> a) {
    return cx<T>(__shfl_up_sync(0xffffffffu, a.re, 1), __shfl_up_sync(0xffffffffu, a.im, 1));
}
template <typename T> __device__ __forceinline__ cx<T> sh_dn(cx<T> a) {
    return cx<T>(__shfl_down_sync(0xffffffffu, a.re, 1), __shfl_down_sync(0xffffffffu, a.im, 1));
}

// Finest level. M = D - N there (D = 4 - (h omega m)^2 (b1 - j b2), N the sum of
// the four neighbours), so r = f - D u1 + N u1 = (1 - wj) f + N u1: one complex
// reciprocal per node and no complex product in the residual.
// Column marching, no shared memory: lane j of a warp owns the fine columns
// 2I and 2I + 1 of coarse column I = I0 + j (the odd one is the coarse node's
// centre); lanes 1..30 write their coarse column, so warps step by 30 coarse
// columns. The warp walks down the fine rows of `ks` coarse rows two at a time,
// holding u1 of three rows in registers and loading two rows ahead; the
// neighbour columns across a lane boundary come by shuffle. r is zero outside
// the grid.
constexpr int RM_COLS = 30;   // coarse columns per warp

// The marching loop; EDGE = false when every row and column the warp touches
// lies inside the grid, so no bounds test is needed.
template <typename T, bool EDGE>
__device__ __forceinline__ void restrict_march(int nx, int nz, int cnx, int c0, int I, int lane, int K0, int K1,
                                               const T* __restrict__ fb, const T* __restrict__ m2, T sb1, T sb2,
                                               T wj, T* __restrict__ fcb) {
    const T omw = T(1) - wj;
    const bool in0 = !EDGE || (c0 >= 0 && c0 < nx), in1 = !EDGE || (c0 + 1 >= 0 && c0 + 1 < nx);
    struct Row { cx<T> f0, f1; T m0, m1; };
    auto ld = [&](int z) -> Row {
        Row r;
        const bool zin = !EDGE || (z >= 0 && z < nz);
        const int i = z * nx + c0;
        r.f0 = (zin && in0) ? ldc(fb, i) : cx<T>(0, 0);
        r.f1 = (zin && in1) ? ldc(fb, i + 1) : cx<T>(0, 0);
        r.m0 = (zin && in0) ? __ldg(m2 + i) : T(0);
        r.m1 = (zin && in1) ? __ldg(m2 + i + 1) : T(0);
        return r;
    };
    auto u1of = [&](cx<T> fv, T mv) -> cx<T> {   // wj D^-1 f (zero where f is)
        const T dr = T(4) - sb1 * mv, di = sb2 * mv;
        const T sc = wj * rcp_fast(dr * dr + di * di);
        return cx<T>(sc * (fv.re * dr + fv.im * di), sc * (fv.im * dr - fv.re * di));
    };
    // r of row z at both columns from u1 of rows z-1 (a), z (c), z+1 (d); x
    // neighbours: u1 at c0 - 1 is the lower lane's odd column, at c0 + 2 the
    // upper lane's even column
    auto resid = [&](int z, const Row& rz, cx<T> a0, cx<T> a1, cx<T> c0v, cx<T> c1v, cx<T> d0v, cx<T> d1v,
                     cx<T>& r0, cx<T>& r1) {
        const cx<T> wl = sh_up(c1v), er = sh_dn(c0v);
        r0 = omw * rz.f0 + (a0 + d0v) + (wl + c1v);
        r1 = omw * rz.f1 + (a1 + d1v) + (c0v + er);
        if (EDGE) {
            const bool zin = z < nz;
            if (!(zin && in0)) r0 = cx<T>(0, 0);
            if (!(zin && in1)) r1 = cx<T>(0, 0);
        }
    };
    // horizontal full weighting at the centre column: r(2I) + 2 r(2I+1) + r(2I+2)
    auto hsum = [&](cx<T> r0, cx<T> r1) -> cx<T> { return (r0 + sh_dn(r0)) + T(2) * r1; };
    const bool wr = lane >= 1 && lane <= RM_COLS && I < cnx;

    Row A = ld(2 * K0 - 1), B = ld(2 * K0), C = ld(2 * K0 + 1), D = ld(2 * K0 + 2);
    cx<T> ua0 = u1of(A.f0, A.m0), ua1 = u1of(A.f1, A.m1);   // u1 of row 2K-1
    cx<T> ub0 = u1of(B.f0, B.m0), ub1 = u1of(B.f1, B.m1);   // u1 of row 2K
    cx<T> acc(0, 0);
    for (int K = K0; K < K1; ++K) {
        // held: u1 of rows 2K-1, 2K, f of row 2K (B); raw rows 2K+1 (C), 2K+2 (D)
        const Row E = ld(2 * K + 3), F = ld(2 * K + 4);
        const cx<T> uc0 = u1of(C.f0, C.m0), uc1 = u1of(C.f1, C.m1);
        const cx<T> ud0 = u1of(D.f0, D.m0), ud1 = u1of(D.f1, D.m1);
        cx<T> r0, r1, s0, s1;
        resid(2 * K, B, ua0, ua1, ub0, ub1, uc0, uc1, r0, r1);
        resid(2 * K + 1, C, ub0, ub1, uc0, uc1, ud0, ud1, s0, s1);
        const cx<T> h0 = hsum(r0, r1), h1 = hsum(s0, s1);
        if (K > K0) {
            acc = acc + h0;   // completes coarse row K - 1
            if (wr) stc(fcb, (size_t)(K - 1) * cnx + I, T(0.25) * acc);
        }
        acc = h0 + T(2) * h1;
        ua0 = uc0; ua1 = uc1; ub0 = ud0; ub1 = ud1;
        B = D; C = E; D = F;
    }
    cx<T> r0, r1;
    resid(2 * K1, B, ua0, ua1, ub0, ub1, u1of(C.f0, C.m0), u1of(C.f1, C.m1), r0, r1);
    acc = acc + hsum(r0, r1);
    if (wr) stc(fcb, (size_t)(K1 - 1) * cnx + I, T(0.25) * acc);
}

template <typename T>
__global__ void __launch_bounds__(256) k_restrict(LevelDev Lf, LevelDev Lc, const T* __restrict__ w2, T b1, T b2,
                                                  T wj, const T* __restrict__ f, T* __restrict__ fc,
                                                  const RhsState* st, int ks) {
    pdl_trigger();
    pdl_wait();
    const int b = blockIdx.z;
    if (!rhs_active(st, b)) return;
    const int lane = threadIdx.x & 31;
    const int Ib = (blockIdx.x * 8 + (threadIdx.x >> 5)) * RM_COLS - 1;   // coarse column of lane 0
    if (Ib + 1 >= Lc.nx) return;   // uniform in the warp; the kernel has no block barrier
    const int nx = Lf.nx, nz = Lf.nz;
    const int I = Ib + lane;
    const int K0 = blockIdx.y * ks, K1 = min(K0 + ks, Lc.nz);
    const size_t nf = (size_t)nx * nz;
    const T* fb = f + 2 * nf * b;
    const T* m2 = static_cast<const T*>(Lf.m2) + (size_t)b * Lf.mstride;
    const T hw = w2[b];
    T* fcb = fc + 2 * ((size_t)Lc.nx * Lc.nz) * b;
    // fine columns 2 Ib .. 2 Ib + 63 and rows 2 K0 - 1 .. 2 K1 + 2 inside the grid?
    const bool edge = Ib < 0 || 2 * Ib + 63 >= nx || K0 == 0 || 2 * K1 + 2 >= nz;
    if (edge)
        restrict_march<T, true>(nx, nz, Lc.nx, 2 * I, I, lane, K0, K1, fb, m2, hw * b1, hw * b2, wj, fcb);
    else
        restrict_march<T, false>(nx, nz, Lc.nx, 2 * I, I, lane, K0, K1, fb, m2, hw * b1, hw * b2, wj, fcb);
}

// Rows per block of the marching kernels: long segments amortise the rows
// recomputed at segment ends; short ones give enough warps when the batch is
// small (aim: 32 warps per SM on 152 SMs).
inline int march_rows(int col_warps, int rows, int nrhs, int longest) {
    int zs = longest;
    while (zs > 4 && (size_t)col_warps * ((rows + zs - 1) / zs) * nrhs < 152u * 32u) zs /= 2;
    return zs;
}

template <typename T>
void launch_restrict(const LevelDev& Lf, const LevelDev& Lc, const T* w2, double b1, double b2, double wj,
                     const T* f, T* fc, const RhsState* st, int nrhs, cudaStream_t s, int tile) {
    const bool fine = Lf.m2 && !Lf.rho;
    const double nf = (double)Lf.nx * Lf.nz, nc = (double)Lc.nx * Lc.nz, es = 2.0 * sizeof(T);
    // f and fc per RHS; m^2 (finest) or the ten Galerkin coefficients per node, per model
    ProfScope prof(fine ? PK_RESTRICT : PK_RESTRICT_G, Lf.nx, Lf.nz,
                   (nf + nc) * es * nrhs +
                       nf * sizeof(T) * (fine ? 1 : kGalerkinCoefs) * ((fine ? Lf.mstride : Lf.gkstride) ? nrhs : 1),
                   s);
    if (Lf.m2 && !Lf.rho) {   // finest constant-density level; a density level is stored like a coarse one
        const int cw = (Lc.nx + RM_COLS - 1) / RM_COLS;
        const int ks = march_rows(cw, Lc.nz, nrhs, 16);
        dim3 grd((cw + 7) / 8, (Lc.nz + ks - 1) / ks, nrhs);
        launch_pdl(k_restrict<T>, grd, dim3(256), 0, s, Lf, Lc, w2, (T)b1, (T)b2, (T)wj, f, fc, st, ks);
    } else {
        launch_restrict_g<T, false>(tile, Lf, Lc, w2, b1, b2, wj, f, (const T*)nullptr, fc, st, nrhs, s);
    }
}

// ========================================================= V-cycle: prolong
// Finest level: u1 = wj D^-1 f, u2 = u1 + P e (bilinear), one post-sweep
// u3 = u2 + wj D^-1 (f - M u2). With M = D - N on this level the sweep is
// u3 = (1 - wj) u2 + (wj D^-1) (f + N u2): one complex reciprocal per node and
// no complex product of M. Mode 0 writes u3 (optionally accumulating); modes 1
// and 2 (inside BiCGSTAB) also apply A to u3 and reduce the dot products the
// next scalar needs; mode 3 (FGMRES) applies A without dots.
// Column marching, no shared memory for the fields: lane j of a warp owns the
// fine columns 2J and 2J + 1 of coarse column J = Jb + j (2J + 1 is the coarse
// node's column, so the bilinear weights are fixed per column); lanes 1..30
// write, so warps step by 60 fine columns. The warp walks down `zs` fine rows
// two at a time (u2 of rows 2K, 2K+1; u3 of rows 2K-1, 2K; outputs of rows
// 2K-2, 2K-1), holding the rows it still needs in registers and loading two
// rows ahead; neighbours across a lane boundary come by shuffle.
constexpr int PM_COLS = 60;   // fine output columns per warp

template <typename T, int MODE, bool EDGE>
__device__ __forceinline__ void prolong_march(int nx, int nz, int cnx, int cnz, int J, int lane, int Z0, int Z1,
                                              int npml, T acoef, T hw, T b1, T b2, T wj, const T* __restrict__ fb,
                                              const T* __restrict__ eb, const T* __restrict__ ab,
                                              const T* __restrict__ m2, T* __restrict__ ob, T* __restrict__ yb,
                                              int accumulate, T& d0, T& d1, T& d2) {
    const int c0 = 2 * J;
    const bool in0 = !EDGE || (c0 >= 0 && c0 < nx), in1 = !EDGE || (c0 + 1 >= 0 && c0 + 1 < nx);
    const bool ein = !EDGE || (J >= 0 && J < cnx);
    const bool outl = lane >= 1 && lane <= PM_COLS / 2;
    const T sb1 = hw * b1, sb2 = hw * b2, omw = T(1) - wj;
    struct Row { cx<T> f0, f1; T m0, m1; };
    auto ld = [&](int z) -> Row {
        Row r;
        const bool zin = !EDGE || (z >= 0 && z < nz);
        const int i = z * nx + c0;
        r.f0 = (zin && in0) ? ldc(fb, i) : cx<T>(0, 0);
        r.f1 = (zin && in1) ? ldc(fb, i + 1) : cx<T>(0, 0);
        r.m0 = (zin && in0) ? __ldg(m2 + i) : T(0);
        r.m1 = (zin && in1) ? __ldg(m2 + i + 1) : T(0);
        return r;
    };
    // e(K, J); lane 0 also reads e(K, J - 1), which the other lanes take from
    // the lane below
    struct ERow { cx<T> e, w; };
    const bool wlo = lane == 0 && (!EDGE || (J - 1 >= 0 && J - 1 < cnx));
    auto erow = [&](int K) -> ERow {
        ERow r;
        const bool kin = !EDGE || (K >= 0 && K < cnz);
        r.e = (ein && kin) ? ldc(eb, (size_t)K * cnx + J) : cx<T>(0, 0);
        r.w = (wlo && kin) ? ldc(eb, (size_t)K * cnx + J - 1) : cx<T>(0, 0);
        return r;
    };
    auto dinv = [&](T mv) -> cx<T> {   // wj D^-1
        const T dr = T(4) - sb1 * mv, di = sb2 * mv;
        const T sc = wj * rcp_fast(dr * dr + di * di);
        return cx<T>(sc * dr, -sc * di);
    };
    // u2 of row z at both columns; ev = e(K, J) of the coarse rows above and
    // below (equal for odd z): column 2J + 1 takes e(J), column 2J the mean of
    // e(J - 1) (lower lane) and e(J)
    auto u2row = [&](int z, const Row& r, const ERow& ea, const ERow& ec2, cx<T>& p0, cx<T>& p1) {
        const cx<T> ev = T(0.5) * (ea.e + ec2.e);
        const cx<T> up = sh_up(ev);
        const cx<T> left = lane == 0 ? T(0.5) * (ea.w + ec2.w) : up;
        const cx<T> pe0 = T(0.5) * (left + ev);
        p0 = dinv(r.m0) * r.f0 + pe0;
        p1 = dinv(r.m1) * r.f1 + ev;
        if (EDGE) {
            const bool zin = z >= 0 && z < nz;
            if (!(zin && in0)) p0 = cx<T>(0, 0);
            if (!(zin && in1)) p1 = cx<T>(0, 0);
        }
    };
    // u3 of row z from u2 of rows z-1 (a), z (c), z+1 (d)
    auto u3row = [&](int z, const Row& r, cx<T> a0, cx<T> a1, cx<T> c0v, cx<T> c1v, cx<T> d0v, cx<T> d1v,
                     cx<T>& q0, cx<T>& q1) {
        const cx<T> wl = sh_up(c1v), er = sh_dn(c0v);
        q0 = omw * c0v + dinv(r.m0) * (r.f0 + ((wl + c1v) + (a0 + d0v)));
        q1 = omw * c1v + dinv(r.m1) * (r.f1 + ((c0v + er) + (a1 + d1v)));
        if (EDGE) {
            const bool zin = z >= 0 && z < nz;
            if (!(zin && in0)) q0 = cx<T>(0, 0);
            if (!(zin && in1)) q1 = cx<T>(0, 0);
        }
    };
    // y = A u3 at row z (fine operator with damping) from u3 of rows z-1, z, z+1
    const int dx0 = max(npml - c0, c0 - (nx - 1 - npml)), dx1 = max(npml - c0 - 1, c0 + 1 - (nx - 1 - npml));
    auto arow = [&](int z, const Row& r, cx<T> a0, cx<T> a1, cx<T> c0v, cx<T> c1v, cx<T> d0v, cx<T> d1v,
                    cx<T>& y0, cx<T>& y1) {
        const cx<T> wl = sh_up(c1v), er = sh_dn(c0v);
        const int dz = max(npml - z, z - (nz - 1 - npml));
        const int e0 = max(max(dx0, dz), 0), e1 = max(max(dx1, dz), 0);
        const T s0 = hw * r.m0, s1 = hw * r.m1;
        const T a0s = s0 * (acoef * (T)(e0 * e0)), a1s = s1 * (acoef * (T)(e1 * e1));
        const T g0 = T(4) - s0, g1 = T(4) - s1;
        y0 = cx<T>(g0 * c0v.re - a0s * c0v.im, g0 * c0v.im + a0s * c0v.re) - ((wl + c1v) + (a0 + d0v));
        y1 = cx<T>(g1 * c1v.re - a1s * c1v.im, g1 * c1v.im + a1s * c1v.re) - ((c0v + er) + (a1 + d1v));
    };
    auto lda = [&](int z, cx<T>& q0, cx<T>& q1) {
        const bool ok = outl && z >= Z0 && z < Z1;
        const int i = z * nx + c0;
        q0 = (ok && in0) ? ldc(ab, i) : cx<T>(0, 0);
        q1 = (ok && in1) ? ldc(ab, i + 1) : cx<T>(0, 0);
    };

    const int Ks = Z0 / 2 - 1, Ke = (Z1 + 1) / 2;   // Z0 is even
    // state at the top of iteration K: u2 of rows 2K-2 (pa), 2K-1 (pb); u3 of
    // rows 2K-3 (qa), 2K-2 (qb); the rows 2K-2 (RA), 2K-1 (RB) and the raw rows
    // 2K (RC), 2K+1 (RD); e(K-1, J) (elo) and e(K, J) (ehi)
    cx<T> pa0(0, 0), pa1(0, 0), pb0(0, 0), pb1(0, 0), qa0(0, 0), qa1(0, 0), qb0(0, 0), qb1(0, 0);
    Row RA, RB;
    RA.f0 = RA.f1 = RB.f0 = RB.f1 = cx<T>(0, 0);
    RA.m0 = RA.m1 = RB.m0 = RB.m1 = T(0);
    Row RC = ld(2 * Ks), RD = ld(2 * Ks + 1);
    ERow elo = erow(Ks - 1), ehi = erow(Ks);
    cx<T> qr0(0, 0), qr1(0, 0), qs0(0, 0), qs1(0, 0);   // mode 1: shadow residual of the output rows
    if constexpr (MODE == 1) { lda(2 * Ks - 2, qr0, qr1); lda(2 * Ks - 1, qs0, qs1); }
    for (int K = Ks; K <= Ke; ++K) {
        const Row RE = ld(2 * K + 2), RF = ld(2 * K + 3);
        const ERow enx = erow(K + 1);
        cx<T> qn0(0, 0), qn1(0, 0), qm0(0, 0), qm1(0, 0);
        if constexpr (MODE == 1) { lda(2 * K, qn0, qn1); lda(2 * K + 1, qm0, qm1); }
        cx<T> pc0, pc1, pd0, pd1, qc0, qc1, qd0, qd1;
        u2row(2 * K, RC, elo, ehi, pc0, pc1);       // even row: mean of e(K-1), e(K)
        u2row(2 * K + 1, RD, ehi, ehi, pd0, pd1);   // odd row: e(K)
        u3row(2 * K - 1, RB, pa0, pa1, pb0, pb1, pc0, pc1, qc0, qc1);
        u3row(2 * K, RC, pb0, pb1, pc0, pc1, pd0, pd1, qd0, qd1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int z = 2 * K - 2 + h;
            const cx<T> c0v = h ? qc0 : qb0, c1v = h ? qc1 : qb1;
            const bool wr = outl && z >= Z0 && z < Z1;
            const int i = z * nx + c0;
            if constexpr (MODE == 0) {
                if (wr) {
                    if (in0) stc(ob, i, accumulate ? ldcc(ob, i) + c0v : c0v);
                    if (in1) stc(ob, i + 1, accumulate ? ldcc(ob, i + 1) + c1v : c1v);
                }
            } else {
                cx<T> y0, y1;
                if (h) arow(z, RB, qb0, qb1, qc0, qc1, qd0, qd1, y0, y1);
                else arow(z, RA, qa0, qa1, qb0, qb1, qc0, qc1, y0, y1);
                if (wr) {
                    if (in0) { stc(ob, i, c0v); stc(yb, i, y0); }
                    if (in1) { stc(ob, i + 1, c1v); stc(yb, i + 1, y1); }
                    if (!in0) y0 = cx<T>(0, 0);
                    if (!in1) y1 = cx<T>(0, 0);
                    if constexpr (MODE == 1) {          // <rh, v>
                        const cx<T> q0 = h ? qs0 : qr0, q1 = h ? qs1 : qr1;
                        d0 += (q0.re * y0.re + q0.im * y0.im) + (q1.re * y1.re + q1.im * y1.im);
                        d1 += (q0.re * y0.im - q0.im * y0.re) + (q1.re * y1.im - q1.im * y1.re);
                    } else if constexpr (MODE == 2) {   // <t, s>, <t, t> with s = f
                        const Row& R = h ? RB : RA;
                        d0 += (y0.re * R.f0.re + y0.im * R.f0.im) + (y1.re * R.f1.re + y1.im * R.f1.im);
                        d1 += (y0.re * R.f0.im - y0.im * R.f0.re) + (y1.re * R.f1.im - y1.im * R.f1.re);
                        d2 += (y0.re * y0.re + y0.im * y0.im) + (y1.re * y1.re + y1.im * y1.im);
                    }
                }
            }
        }
        pa0 = pc0; pa1 = pc1; pb0 = pd0; pb1 = pd1;
        qa0 = qc0; qa1 = qc1; qb0 = qd0; qb1 = qd1;
        RA = RC; RB = RD; RC = RE; RD = RF;
        elo = ehi; ehi = enx;
        qr0 = qn0; qr1 = qn1; qs0 = qm0; qs1 = qm1;
    }
}

constexpr int PM_WARPS = 4;   // warps per block of the marching prolongation

template <typename T, int MODE>
__global__ void __launch_bounds__(32 * PM_WARPS) k_prolong(LevelDev Lf, LevelDev Lc, int npml, T acoef,
                                                 const T* __restrict__ w2, T b1, T b2, T wj,
                                                 const T* __restrict__ f, const T* __restrict__ ec,
                                                 T* __restrict__ out, T* __restrict__ y, const T* __restrict__ aux,
                                                 double* partials, int pstride, RhsState* st, int accumulate, int zs) {
    __shared__ double shred[96];
    pdl_trigger();
    pdl_wait();
    const int b = blockIdx.z;
    if (!rhs_active(st, b)) return;   // uniform in the block
    const int lane = threadIdx.x & 31;
    const int nx = Lf.nx, nz = Lf.nz, cnx = Lc.nx, cnz = Lc.nz;
    const int Jb = (blockIdx.x * PM_WARPS + (threadIdx.x >> 5)) * (PM_COLS / 2) - 1;   // coarse column of lane 0
    const int Z0 = blockIdx.y * zs, Z1 = min(Z0 + zs, nz);
    const size_t nf = (size_t)nx * nz, nc = (size_t)cnx * cnz;
    const T* fb = f + 2 * nf * b;
    const T* eb = ec + 2 * nc * b;
    const T* ab = aux + 2 * nf * b;
    const T* m2 = static_cast<const T*>(Lf.m2) + (size_t)b * Lf.mstride;
    T* ob = out + 2 * nf * b;
    T* yb = y + 2 * nf * b;
    const T hw = w2[b];
    T d0 = 0, d1 = 0, d2 = 0;
    if (2 * (Jb + 1) < nx) {   // the warp has output columns (uniform in the warp)
        // fine columns 2 Jb .. 2 Jb + 63, coarse columns Jb .. Jb + 31 and rows
        // Z0 - 4 .. Z1 + 3 (coarse rows Z0/2 - 2 .. Z1/2 + 2) inside the grid?
        const bool edge = Jb < 0 || 2 * Jb + 63 >= nx || Jb + 31 >= cnx || Z0 < 4 || Z1 + 3 >= nz ||
                          Z0 / 2 - 2 < 0 || Z1 / 2 + 2 >= cnz;
        if (edge)
            prolong_march<T, MODE, true>(nx, nz, cnx, cnz, Jb + lane, lane, Z0, Z1, npml, acoef, hw, b1, b2, wj, fb,
                                         eb, ab, m2, ob, yb, accumulate, d0, d1, d2);
        else
            prolong_march<T, MODE, false>(nx, nz, cnx, cnz, Jb + lane, lane, Z0, Z1, npml, acoef, hw, b1, b2, wj, fb,
                                          eb, ab, m2, ob, yb, accumulate, d0, d1, d2);
    }
    if constexpr (MODE == 0 || MODE == 3) return;
    else {
        const T vv[3] = {d0, d1, d2};
        double acc[3];
        const int nblk = gridDim.x * gridDim.y, blk = blockIdx.y * gridDim.x + blockIdx.x;
        if (last_block_reduce_t<3, T>(vv, acc, shred, partials + (size_t)b * pstride, nblk, blk, &st[b].counter[3])) {
            if (threadIdx.x == 0) {
                RhsState& S = st[b];
                if (MODE == 1) {   // alpha = rho / <rh, v>
                    double dd = acc[0] * acc[0] + acc[1] * acc[1];
                    if (!(dd > 0.0)) {
                        // stays active: the iteration finishes with alpha = 0 (a
                        // minimal-residual step on r) and k_bicg_xr retires it
                        S.flag = FLAG_BREAKDOWN;
                        S.alpha[0] = 0.0; S.alpha[1] = 0.0;
                    } else {
                        S.alpha[0] = (S.rho[0] * acc[0] + S.rho[1] * acc[1]) / dd;
                        S.alpha[1] = (S.rho[1] * acc[0] - S.rho[0] * acc[1]) / dd;
                    }
                } else {           // omega = <t, s> / <t, t>
                    if (acc[2] > 0.0) { S.omega[0] = acc[0] / acc[2]; S.omega[1] = acc[1] / acc[2]; }
                    else { S.omega[0] = 0.0; S.omega[1] = 0.0; }
                }
            }
        }
    }
}

// Grid of the marching prolongation for a fine level of nx x nz nodes.
inline dim3 prolong_grid(int nx, int nz, int nrhs, int longest, int* zs) {
    const int cw = (nx + PM_COLS - 1) / PM_COLS;
    *zs = march_rows(cw, nz, nrhs, longest);
    return dim3((cw + PM_WARPS - 1) / PM_WARPS, (nz + *zs - 1) / *zs, nrhs);
}

template <typename T>
void launch_prolong(int mode, const LevelDev& Lf, const LevelDev& Lc, int npml, double amax, const T* w2,
                    double b1, double b2, double wj, const T* f, const T* ec, T* out, T* y, const T* aux,
                    double* partials, int pstride, RhsState* st, int nrhs, cudaStream_t s, int accumulate, int tile) {
    const bool galk = mode == 0 && (!Lf.m2 || Lf.rho);
    const double nf = (double)Lf.nx * Lf.nz, nc = (double)Lc.nx * Lc.nz, es = 2.0 * sizeof(T);
    // f, the coarse correction and the output (read too when accumulating); finest modes also
    // write y = A out and mode 1 reads the shadow residual; model data per model
    const double vec = galk ? nf * (2 + accumulate) + nc : nf * (3 + (mode == 1 ? 1 : 0)) + nc;
    ProfScope prof(galk ? PK_PROLONG_G : PK_PROLONG, Lf.nx, Lf.nz,
                   vec * es * nrhs +
                       nf * sizeof(T) * (galk ? kGalerkinCoefs : 1) * ((galk ? Lf.gkstride : Lf.mstride) ? nrhs : 1),
                   s);
    const T ac = (T)layer_coef(npml, amax);
    // a density level is stored like a coarse one: only mode 0 exists there (the
    // caller applies A and forms the dots with launch_apply_dots)
    if (mode == 0 && (!Lf.m2 || Lf.rho)) {
        launch_prolong_g<T>(tile, Lf, Lc, w2, b1, b2, wj, f, ec, out, st, nrhs, s, accumulate);
        return;
    }
    // finest level: the tile choice is the longest row segment (16 or 32 rows)
    int zs = 0;
    const dim3 grd = prolong_grid(Lf.nx, Lf.nz, nrhs, tile == 0 ? 16 : 32, &zs);
    if (mode == 0)
        launch_pdl(k_prolong<T, 0>, grd, dim3(32 * PM_WARPS), 0, s, Lf, Lc, npml, ac, w2, (T)b1, (T)b2, (T)wj, f, ec, out, y, aux,
                   partials, pstride, st, accumulate, zs);
    else if (mode == 1)
        launch_pdl(k_prolong<T, 1>, grd, dim3(32 * PM_WARPS), 0, s, Lf, Lc, npml, ac, w2, (T)b1, (T)b2, (T)wj, f, ec, out, y, aux,
                   partials, pstride, st, accumulate, zs);
    else if (mode == 2)
        launch_pdl(k_prolong<T, 2>, grd, dim3(32 * PM_WARPS), 0, s, Lf, Lc, npml, ac, w2, (T)b1, (T)b2, (T)wj, f, ec, out, y, aux,
                   partials, pstride, st, accumulate, zs);
    else
        launch_pdl(k_prolong<T, 3>, grd, dim3(32 * PM_WARPS), 0, s, Lf, Lc, npml, ac, w2, (T)b1, (T)b2, (T)wj, f, ec, out, y, aux,
                   partials, pstride, st, accumulate, zs);
}

// ======================================================= V-cycle: coarsest
// e = M_L^{-1} f with the precomputed dense inverse of the coarsest level
// (one per distinct frequency); one warp per row.
template <typename T>
__global__ void __launch_bounds__(256) k_coarse(int n, const T* __restrict__ minv, const int* __restrict__ slot,
                                                const T* __restrict__ fL, T* __restrict__ eL, const RhsState* st) {
    __shared__ cx<T> fs[kCoarseHardMax];
    const int b = blockIdx.x;
    if (!rhs_active(st, b)) return;
    for (int j = threadIdx.x; j < n; j += blockDim.x) fs[j] = ldc(fL, (size_t)n * b + j);
    __syncthreads();
    const T* Mb = minv + 2 * (size_t)n * n * slot[b];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int row = warp; row < n; row += nw) {
        T re = 0, im = 0;
        for (int j = lane; j < n; j += 32) {
            const cx<T> a = ldc(Mb, (size_t)row * n + j);
            const cx<T> v = fs[j];
            re += a.re * v.re - a.im * v.im;
            im += a.re * v.im + a.im * v.re;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (lane == 0) stc(eL, (size_t)n * b + row, cx<T>(re, im));
    }
}

template <typename T>
void launch_coarse(int n, const T* minv, const int* slot, const T* fL, T* eL, const RhsState* st, int nrhs,
                   cudaStream_t s) {
    k_coarse<T><<<nrhs, 256, 0, s>>>(n, minv, slot, fL, eL, st);
}

// Dense inverse of the coarsest Galerkin shifted-Laplace matrix, Gauss-Jordan
// with partial pivoting in FP64; one block per distinct (model, frequency).
__global__ void __launch_bounds__(1024) k_coarse_invert(int nx, int nz, const double* __restrict__ gkall,
                                                        size_t gkstride, const double* __restrict__ w2s,
                                                        const int* __restrict__ mods, double b1, double b2,
                                                        double2* work, float2* minv_f, double2* minv_d) {
    const int n = nx * nz, w = 2 * n;
    const int sl = blockIdx.x;
    double2* A = work + (size_t)sl * n * w;
    const double hw = w2s[sl];
    const double* gk = gkall + (size_t)mods[sl] * gkstride;
    __shared__ double2 fac[kCoarseHardMax];
    __shared__ double red_v[32];
    __shared__ int red_i[32];
    __shared__ int s_piv;
    __shared__ double2 s_pinv;
    for (int idx = threadIdx.x; idx < n * w; idx += blockDim.x) {
        const int i = idx / w, j = idx - i * w;
        double2 v = make_double2(0.0, 0.0);
        if (j < n) {
            const int ix = i % nx, iz = i / nx, jx = j % nx, jz = j / nx;
            const int dx = jx - ix, dz = jz - iz;
            if (dx >= -1 && dx <= 1 && dz >= -1 && dz <= 1) {
                // stored forward entry of the pair (i, j): at i for (1,0) (0,1) (1,1) (-1,1), else at j
                int ent, at;
                if (dx == 0 && dz == 0) { ent = 0; at = i; }
                else if (dz == 0) { ent = 1; at = dx > 0 ? i : j; }
                else if (dx == 0) { ent = 2; at = dz > 0 ? i : j; }
                else if (dx == dz) { ent = 3; at = dx > 0 ? i : j; }
                else { ent = 4; at = dz > 0 ? i : j; }
                const double g = gk[(size_t)ent * n + at], q = gk[(size_t)(5 + ent) * n + at];
                v = make_double2(g - hw * b1 * q, hw * b2 * q);
            }
        } else if (j - n == i) {
            v = make_double2(1.0, 0.0);
        }
        A[idx] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int k = 0; k < n; ++k) {
        // pivot search over rows k..n-1 (ties -> lowest row)
        double best = -1.0;
        int bi = n;
        for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
            const double2 a = A[(size_t)i * w + k];
            const double m = a.x * a.x + a.y * a.y;
            if (m > best) { best = m; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double bb = -1.0; int ii = n;
            for (int q = 0; q < nwarps; ++q)
                if (red_v[q] > bb || (red_v[q] == bb && red_i[q] < ii)) { bb = red_v[q]; ii = red_i[q]; }
            s_piv = ii;
        }
        __syncthreads();
        const int p = s_piv;
        if (p != k)
            for (int j = threadIdx.x; j < w; j += blockDim.x) {
                const double2 t = A[(size_t)k * w + j];
                A[(size_t)k * w + j] = A[(size_t)p * w + j];
                A[(size_t)p * w + j] = t;
            }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double2 a = A[(size_t)k * w + k];
            const double d = a.x * a.x + a.y * a.y;
            s_pinv = make_double2(a.x / d, -a.y / d);
        }
        __syncthreads();
        const double2 pi = s_pinv;
        for (int j = k + threadIdx.x; j < w; j += blockDim.x) {
            const double2 a = A[(size_t)k * w + j];
            A[(size_t)k * w + j] = make_double2(a.x * pi.x - a.y * pi.y, a.x * pi.y + a.y * pi.x);
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) fac[i] = A[(size_t)i * w + k];
        __syncthreads();
        const int cols = w - k;
        for (int idx = threadIdx.x; idx < n * cols; idx += blockDim.x) {
            const int i = idx / cols, j = k + (idx - i * cols);
            if (i == k) continue;
            const double2 fi = fac[i];
            const double2 kj = A[(size_t)k * w + j];
            double2 a = A[(size_t)i * w + j];
            a.x -= fi.x * kj.x - fi.y * kj.y;
            a.y -= fi.x * kj.y + fi.y * kj.x;
            A[(size_t)i * w + j] = a;
        }
        __syncthreads();
    }
    (void)warp;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx - i * n;
        const double2 a = A[(size_t)i * w + n + j];
        minv_d[(size_t)sl * n * n + idx] = a;
        minv_f[(size_t)sl * n * n + idx] = make_float2((float)a.x, (float)a.y);
    }
}

void launch_coarse_invert(const LevelDev& Lc, const double* w2_slots, const int* mod_slots, int nslots, double b1,
                          double b2, double2* work, float2* minv_f, double2* minv_d, cudaStream_t s) {
    const double nn = (double)Lc.nx * Lc.nz * Lc.nx * Lc.nz;
    ProfScope prof(PK_COARSE_INVERT, Lc.nx, Lc.nz, nn * nslots * 24.0, s);
    k_coarse_invert<<<nslots, 1024, 0, s>>>(Lc.nx, Lc.nz, static_cast<const double*>(Lc.gk),
                                            kGalerkinCoefs * (size_t)Lc.nx * Lc.nz, w2_slots, mod_slots, b1, b2,
                                            work, minv_f, minv_d);
}

// ================================================================ tail
// Levels lt..L of the cycle in one block per right-hand side. Everything those
// levels touch lives in shared memory: per level the vectors f, u, r and the
// complex coefficients M_k = G_k - hw (b1 - j b2) K_k of this right-hand side
// (staged once per launch). The schedule of passes runs with a block barrier
// after each pass.
// M u at node p = (iz, ix) of a tail level held in shared memory; C = the five
// coefficient arrays (c, e, n, ne, nw) of n nodes each, U = &u[p].
template <typename T>
__device__ __forceinline__ cx<T> mop9_sm(const cx<T>* C, int n, int nx, int nz, int ix, int iz, int p,
                                         const cx<T>* U) {
    const cx<T>* Ce = C + n;
    const cx<T>* Cn = C + 2 * n;
    const cx<T>* Cne = C + 3 * n;
    const cx<T>* Cnw = C + 4 * n;
    cx<T> acc = C[p] * U[0];
    const bool e = ix + 1 < nx, w = ix > 0, no = iz + 1 < nz, so = iz > 0;
    if (e) acc = acc + Ce[p] * U[1];
    if (w) acc = acc + Ce[p - 1] * U[-1];
    if (no) {
        acc = acc + Cn[p] * U[nx];
        if (e) acc = acc + Cne[p] * U[nx + 1];
        if (w) acc = acc + Cnw[p] * U[nx - 1];
    }
    if (so) {
        acc = acc + Cn[p - nx] * U[-nx];
        if (w) acc = acc + Cne[p - nx - 1] * U[-nx - 1];
        if (e) acc = acc + Cnw[p - nx + 1] * U[-nx + 1];
    }
    return acc;
}

// Row and column of node p of a level with nx columns: (p + 1/2) / nx in FP32 is
// never within rounding of an integer for the level sizes of the tail
// (p < 2^16, nx < 2^10), so the truncation is exact.
__device__ __forceinline__ int tail_row(int p, float rnx) { return (int)(((float)p + 0.5f) * rnx); }

template <typename T>
__global__ void __launch_bounds__(1024, 1) k_tail(const __grid_constant__ TailArgs a, const RhsState* st) {
    extern __shared__ __align__(16) unsigned char tail_smem[];
    pdl_trigger();
    const int b = blockIdx.x;
    const T hw = (T)a.w2[b], b1 = (T)a.b1, b2 = (T)a.b2, wj = (T)a.wj;
    const T hb1 = hw * b1, hb2 = hw * b2;
    const int tid = threadIdx.x, nth = blockDim.x;
    cx<T>* base = reinterpret_cast<cx<T>*>(tail_smem);
    // per level (at a.off[l]): f, u, r (3 n) then the coefficients (5 n); then
    // the coarsest inverse of this right-hand side's frequency when it fits
    const int* off = a.off;
    for (int l = a.lt; l <= a.L; ++l) {
        const int n = a.lv[l].nx * a.lv[l].nz;
        const T* gk = static_cast<const T*>(a.lv[l].gk) + (size_t)b * a.lv[l].gkstride;
        cx<T>* C = base + off[l] + 3 * n;
        for (int p = tid; p < n; p += nth) {
            T g[5], q[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                g[k] = __ldg(gk + (size_t)k * n + p);
                q[k] = __ldg(gk + (size_t)(5 + k) * n + p);
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) C[(size_t)k * n + p] = cx<T>(g[k] - hb1 * q[k], hb2 * q[k]);
        }
    }
    const int nL = a.lv[a.L].nx * a.lv[a.L].nz;
    const T* Mg = static_cast<const T*>(a.minv) + 2 * (size_t)nL * nL * a.slot[b];
    cx<T>* Ms = base + a.minv_off;
    // the inverse is written by k_coarse_invert before the first ordinary launch of the solve
    if (a.minv_smem)
        for (int t = tid; t < nL * nL; t += nth) Ms[t] = ldc(Mg, t);
    pdl_wait();   // the coefficients above are model data; everything below depends on earlier kernels
    if (!rhs_active(st, b)) return;
    // the output this block accumulates into (a second coarse correction), loaded
    // now instead of after the cycle; the top tail level has at most 2 x 1024 nodes
    static_assert(kTailMaxPoints32 <= 2 * 1024 && kTailMaxPoints64 <= 2 * 1024, "tail output preload");
    cx<T> opre[2] = {cx<T>(0, 0), cx<T>(0, 0)};
    if (a.accumulate) {
        const int nt = a.lv[a.lt].nx * a.lv[a.lt].nz;
        const T* o = static_cast<const T*>(a.out);
        for (int k = 0, p = tid; k < 2 && p < nt; ++k, p += nth) opre[k] = ldcc(o, (size_t)nt * b + p);
    }
    __syncthreads();
    for (int k = 0; k < a.nops; ++k) {
        const int op = a.ops[k], type = op & 255, l = op >> 8;
        const int nx = a.lv[l].nx, nz = a.lv[l].nz;
        const int n = nx * nz;
        const float rnx = 1.0f / (float)nx;
        cx<T>* f = base + off[l];
        cx<T>* u = f + n;
        cx<T>* r = u + n;
        const cx<T>* C = r + n;
        switch (type) {
            case OP_LOAD: {
                const T* in = static_cast<const T*>(a.in);
                const bool sm = l < a.L;
                for (int p = tid; p < n; p += nth) {
                    const cx<T> fv = ldc(in, (size_t)n * b + p);
                    f[p] = fv;
                    if (sm) u[p] = wj * cdiv(fv, C[p]);
                }
                break;
            }
            case OP_RESID:
                for (int p = tid; p < n; p += nth) {
                    const int iz = tail_row(p, rnx), ix = p - iz * nx;
                    r[p] = f[p] - mop9_sm(C, n, nx, nz, ix, iz, p, u + p);
                }
                break;
            case OP_POST:
                for (int p = tid; p < n; p += nth) {
                    const int iz = tail_row(p, rnx), ix = p - iz * nx;
                    const cx<T> res = f[p] - mop9_sm(C, n, nx, nz, ix, iz, p, u + p);
                    r[p] = u[p] + wj * cdiv(res, C[p]);
                }
                break;
            case OP_RESTRICT: {
                const int cnx = a.lv[l + 1].nx, nc = cnx * a.lv[l + 1].nz;
                const float rcnx = 1.0f / (float)cnx;
                cx<T>* fc = base + off[l + 1];
                cx<T>* uc = fc + nc;
                const cx<T>* Cc = fc + 3 * nc;
                const bool sm = l + 1 < a.L;
                for (int q = tid; q < nc; q += nth) {
                    const int K = tail_row(q, rcnx), I = q - K * cnx;
                    const int x = 2 * I + 1;
                    const cx<T>* r0 = r + (2 * K) * nx;
                    const cx<T>* r1 = r0 + nx;
                    const bool e = x + 1 < nx, z2 = 2 * K + 2 < nz;
                    cx<T> h0 = r0[x - 1] + T(2) * r0[x], hm = r1[x - 1] + T(2) * r1[x], hp(0, 0);
                    if (e) { h0 = h0 + r0[x + 1]; hm = hm + r1[x + 1]; }
                    if (z2) {
                        const cx<T>* r2 = r1 + nx;
                        hp = r2[x - 1] + T(2) * r2[x];
                        if (e) hp = hp + r2[x + 1];
                    }
                    const cx<T> fv = T(0.25) * ((h0 + hp) + T(2) * hm);
                    fc[q] = fv;
                    if (sm) uc[q] = wj * cdiv(fv, Cc[q]);
                }
                break;
            }
            case OP_PROLONG_ADD: {
                const int cnx = a.lv[l + 1].nx, cnz = a.lv[l + 1].nz;
                const cx<T>* uc = base + off[l + 1] + 2 * cnx * cnz;    // the coarse level's result (its r)
                for (int p = tid; p < n; p += nth) {
                    const int jz = tail_row(p, rnx), jx = p - jz * nx;
                    // coarse rows (jz-1)/2 and jz/2 (one row, weight 1, for odd jz), columns likewise
                    const int ka = (jz - 1) >> 1, kb = jz >> 1, ia = (jx - 1) >> 1, ib = jx >> 1;
                    const bool zo = jz & 1, xo = jx & 1;
                    auto hrow = [&](int K) -> cx<T> {
                        const cx<T>* e = uc + K * cnx;
                        if (xo) return e[ia];
                        cx<T> h(0, 0);
                        if (ia >= 0) h = e[ia];
                        if (ib < cnx) h = h + e[ib];
                        return T(0.5) * h;
                    };
                    cx<T> add(0, 0);
                    if (zo) add = hrow(ka);
                    else {
                        if (ka >= 0) add = hrow(ka);
                        if (kb < cnz) add = add + hrow(kb);
                        add = T(0.5) * add;
                    }
                    u[p] = u[p] + add;
                }
                break;
            }
            case OP_COARSE: {
                const int lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
                for (int row = warp; row < n; row += nw) {
                    T re = 0, im = 0;
                    for (int j = lane; j < n; j += 32) {
                        const cx<T> m = a.minv_smem ? Ms[row * n + j] : ldc(Mg, (size_t)row * n + j);
                        const cx<T> v = f[j];
                        re += m.re * v.re - m.im * v.im;
                        im += m.re * v.im + m.im * v.re;
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        re += __shfl_xor_sync(0xffffffffu, re, o);
                        im += __shfl_xor_sync(0xffffffffu, im, o);
                    }
                    if (lane == 0) r[row] = cx<T>(re, im);
                }
                break;
            }
            case OP_OUTPUT: {
                T* o = static_cast<T*>(a.out);
                for (int q = 0, p = tid; q < 2 && p < n; ++q, p += nth)
                    stc(o, (size_t)n * b + p, a.accumulate ? opre[q] + r[p] : r[p]);
                break;
            }
        }
        __syncthreads();
    }
}

// Shared memory of the tail for levels lt..L: 8 complex arrays per level
// (f, u, r, five coefficients), then the coarsest inverse when the total stays
// within 227 KB (TailArgs::minv_smem).
size_t tail_smem_bytes(const helm_model* m, int lt, size_t elem, bool* minv_smem, int* minv_off) {
    size_t v = 0;
    for (size_t l = lt; l < m->lv.size(); ++l) v += 8 * m->lv[l].n();   // f, u, r + 5 coefficients
    const size_t nL = m->lv.back().n();
    const bool fit = (v + nL * nL) * 2 * elem <= 227u * 1024u;
    if (minv_smem) *minv_smem = fit;
    if (minv_off) *minv_off = (int)v;
    return (fit ? v + nL * nL : v) * 2 * elem;
}

template <typename T>
void launch_tail(const TailArgs& a, size_t smem, int nrhs, const RhsState* st, cudaStream_t s) {
    double coef = 0;
    for (int l = a.lt; l <= a.L; ++l) coef += (double)a.lv[l].nx * a.lv[l].nz;
    const double ntop = (double)a.lv[a.lt].nx * a.lv[a.lt].nz;
    ProfScope prof(PK_TAIL, a.lv[a.lt].nx, a.lv[a.lt].nz,
                   ntop * 2.0 * sizeof(T) * nrhs * (2 + a.accumulate) +
                       coef * kGalerkinCoefs * sizeof(T) * (a.lv[a.lt].gkstride ? nrhs : 1),
                   s);
    // one-time opt-in to more than 48 KB of dynamic shared memory (initialised once, thread-safe)
    static const bool attr_set = [] {
        cudaFuncSetAttribute(k_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        return true;
    }();
    (void)attr_set;
    launch_pdl(k_tail<T>, dim3(nrhs), dim3(1024), smem, s, a, st);
}
template void launch_tail<float>(const TailArgs&, size_t, int, const RhsState*, cudaStream_t);
template void launch_tail<double>(const TailArgs&, size_t, int, const RhsState*, cudaStream_t);

// Schedule of the tail: LOAD the right-hand side of level lt, an F-cycle (whose
// second coarse correction is a V-cycle) or a V-cycle from lt, OUTPUT.
// The zero-guess smoothing u = wj D^-1 f of each level is done by the op that
// writes its f (LOAD or the parent's RESTRICT), and the closing residual and
// Jacobi steps are one op (POST) that leaves the level's result in r.
std::vector<int> tail_schedule(int lt, int L, bool fcycle) {
    std::vector<int> ops;
    auto put = [&](int type, int l) { ops.push_back(type | (l << 8)); };
    std::function<void(int)> V = [&](int l) {
        if (l == L) { put(OP_COARSE, l); return; }
        put(OP_RESID, l); put(OP_RESTRICT, l);
        V(l + 1);
        put(OP_PROLONG_ADD, l); put(OP_POST, l);
    };
    std::function<void(int)> F = [&](int l) {
        if (l == L) { put(OP_COARSE, l); return; }
        put(OP_RESID, l); put(OP_RESTRICT, l);
        F(l + 1);
        put(OP_PROLONG_ADD, l); put(OP_RESID, l); put(OP_RESTRICT, l);
        V(l + 1);
        put(OP_PROLONG_ADD, l); put(OP_POST, l);
    };
    put(OP_LOAD, lt);
    if (fcycle) F(lt); else V(lt);
    put(OP_OUTPUT, lt);
    return ops;
}

// ============================================== F-cycle: correct + restrict
// u2 = wj D^-1 f + P e on the fine region of a coarse tile, r = f - M u2,
// restricted to level l + 1 (the second coarse correction of an F-cycle).
template <typename T, bool GAL>
__global__ void __launch_bounds__(256) k_correct_restrict(LevelDev Lf, LevelDev Lc, const T* __restrict__ w2,
                                                          T b1, T b2, T wj, const T* __restrict__ f,
                                                          const T* __restrict__ ec, T* __restrict__ fc,
                                                          const RhsState* st) {
    constexpr int CEW = RCX + 2, CEH = RCZ + 2;   // coarse region feeding P on the fine region
    __shared__ cx<T> F[RFH][RFW];
    __shared__ cx<T> U[RFH][RFW];
    __shared__ cx<T> E[CEH][CEW];
    const int b = blockIdx.z;
    if (!rhs_active(st, b)) return;
    const int I0 = blockIdx.x * RCX, K0 = blockIdx.y * RCZ;
    const int gx0 = 2 * I0 - 1, gz0 = 2 * K0 - 1;
    const int cx0 = I0 - 1, cz0 = K0 - 1;
    LevelOp<T, GAL> op = level_op<T, GAL>(Lf, b, w2[b]);
    op.b1 = b1;
    op.b2 = b2;
    const size_t nf = (size_t)Lf.nx * Lf.nz, nc = (size_t)Lc.nx * Lc.nz;
    const T* fb = f + 2 * nf * b;
    const T* eb = ec + 2 * nc * b;
    for (int idx = threadIdx.x; idx < CEW * CEH; idx += blockDim.x) {
        const int lz = idx / CEW, lx = idx - lz * CEW;
        const int I = cx0 + lx, K = cz0 + lz;
        cx<T> e(0, 0);
        if (I >= 0 && I < Lc.nx && K >= 0 && K < Lc.nz) e = ldc(eb, (size_t)K * Lc.nx + I);
        E[lz][lx] = e;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < RFW * RFH; idx += blockDim.x) {
        const int lz = idx / RFW, lx = idx - lz * RFW;
        const int gx = gx0 + lx, gz = gz0 + lz;
        cx<T> fv(0, 0), uv(0, 0);
        if (gx >= 0 && gx < Lf.nx && gz >= 0 && gz < Lf.nz) {
            const size_t i = (size_t)gz * Lf.nx + gx;
            fv = ldc(fb, i);
            uv = wj * cdiv(fv, op.diag(i));
            int ia, ib, ka, kb;
            T wa, wb, va, vb;
            bil_axis<T>(gx, ia, ib, wa, wb);
            bil_axis<T>(gz, ka, kb, va, vb);
            ia -= cx0; ib -= cx0; ka -= cz0; kb -= cz0;
            uv = uv + (va * wa) * E[ka][ia] + (va * wb) * E[ka][ib] + (vb * wa) * E[kb][ia] + (vb * wb) * E[kb][ib];
        }
        F[lz][lx] = fv;
        U[lz][lx] = uv;
    }
    __syncthreads();
    constexpr int W2 = RFW - 2, H2 = RFH - 2;
    for (int idx = threadIdx.x; idx < W2 * H2; idx += blockDim.x) {
        const int lz = 1 + idx / W2, lx = 1 + idx % W2;
        const int gx = gx0 + lx, gz = gz0 + lz;
        cx<T> r(0, 0);
        if (gx < Lf.nx && gz < Lf.nz) r = F[lz][lx] - op.apply(gx, gz, &U[lz][lx], RFW);
        F[lz][lx] = r;
    }
    __syncthreads();
    const int cxl = threadIdx.x % RCX, czl = threadIdx.x / RCX;
    const int I = I0 + cxl, K = K0 + czl;
    if (I < Lc.nx && K < Lc.nz) {
        const int lx = 2 * cxl + 2, lz = 2 * czl + 2;
        cx<T> a = T(4) * F[lz][lx];
        a = a + T(2) * (F[lz][lx - 1] + F[lz][lx + 1] + F[lz - 1][lx] + F[lz + 1][lx]);
        a = a + F[lz - 1][lx - 1] + F[lz - 1][lx + 1] + F[lz + 1][lx - 1] + F[lz + 1][lx + 1];
        stc(fc + 2 * nc * b, (size_t)K * Lc.nx + I, T(0.25) * a);
    }
}

template <typename T>
void launch_correct_restrict(const LevelDev& Lf, const LevelDev& Lc, const T* w2, double b1, double b2,
                             double wj, const T* f, const T* ec, T* fc, const RhsState* st, int nrhs, cudaStream_t s,
                             int tile) {
    const bool fine = Lf.m2 && !Lf.rho;
    const double nf = (double)Lf.nx * Lf.nz, nc = (double)Lc.nx * Lc.nz, es = 2.0 * sizeof(T);
    ProfScope prof(PK_CORRECT_RESTRICT, Lf.nx, Lf.nz,
                   (nf + 2 * nc) * es * nrhs +
                       nf * sizeof(T) * (fine ? 1 : kGalerkinCoefs) * ((fine ? Lf.mstride : Lf.gkstride) ? nrhs : 1),
                   s);
    if (Lf.m2 && !Lf.rho) {
        dim3 grd((Lc.nx + RCX - 1) / RCX, (Lc.nz + RCZ - 1) / RCZ, nrhs);
        k_correct_restrict<T, false><<<grd, RCX * RCZ, 0, s>>>(Lf, Lc, w2, (T)b1, (T)b2, (T)wj, f, ec, fc, st);
    } else {
        launch_restrict_g<T, true>(tile, Lf, Lc, w2, b1, b2, wj, f, ec, fc, st, nrhs, s);
    }
}
template void launch_correct_restrict<float>(const LevelDev&, const LevelDev&, const float*, double, double, double,
                                             const float*, const float*, float*, const RhsState*, int, cudaStream_t,
                                             int);
template void launch_correct_restrict<double>(const LevelDev&, const LevelDev&, const double*, double, double, double,
                                              const double*, const double*, double*, const RhsState*, int,
                                              cudaStream_t, int);

// ======================================================= FP64 throughput probe
// Peak rate of FP64 fused multiply-adds (helm_time_kernel HELM_KERNEL_FMA64): each
// thread runs eight independent chains x <- a x + b of `iters` steps; the sum is
// stored only under a condition the values never meet, which keeps the chains.
__global__ void __launch_bounds__(256) k_fma64(double* out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1e-3 * threadIdx.x + k;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) sum += x[k];
    if (sum == -1.0) out[blockIdx.x] = sum;
}

void launch_fma64(double* out, int blocks, int iters, cudaStream_t s) {
    k_fma64<<<blocks, 256, 0, s>>>(out, iters, 0.9999999, 1e-7);
}

// ============================================================ right-hand sides
__global__ void k_point_rhs(double* f, const int* __restrict__ src_flat, size_t n) {
    const int b = blockIdx.x;
    if (threadIdx.x == 0) {
        const size_t i = (size_t)n * b + src_flat[b];
        f[2 * i] = 1.0;      // grid-scaled: h^2 * (1/h^2)
        f[2 * i + 1] = 0.0;
    }
}

void launch_point_rhs(double* f, const int* src_flat, int nrhs, size_t n, cudaStream_t s) {
    cudaMemsetAsync(f, 0, sizeof(double) * 2 * n * nrhs, s);
    k_point_rhs<<<nrhs, 32, 0, s>>>(f, src_flat, n);
}

__global__ void k_scale(const double* __restrict__ in, double* __restrict__ out, double sc, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = sc * in[i];
}
void launch_scale_rhs(const double* fin, double* f, double scale, size_t count, cudaStream_t s) {
    k_scale<<<grid1d(count), 256, 0, s>>>(fin, f, scale, count * 2);
}

template <typename T>
__global__ void k_cast(const double* __restrict__ in, T* __restrict__ out, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (T)in[i];
}
template <typename T>
void launch_cast_complex(const double* in, T* out, size_t count, cudaStream_t s) {
    k_cast<T><<<grid1d(count), 256, 0, s>>>(in, out, 2 * count);
}
template <typename T>
__global__ void k_widen(const T* __restrict__ in, double* __restrict__ out, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}
template <typename T>
void launch_to_c128(const T* in, double* out, size_t count, cudaStream_t s) {
    k_widen<T><<<grid1d(count), 256, 0, s>>>(in, out, 2 * count);
}
template void launch_cast_complex<float>(const double*, float*, size_t, cudaStream_t);
template void launch_cast_complex<double>(const double*, double*, size_t, cudaStream_t);
template void launch_to_c128<float>(const float*, double*, size_t, cudaStream_t);
template void launch_to_c128<double>(const double*, double*, size_t, cudaStream_t);

// ================================================================ gradient
// d_cal = P u at the receiver nodes, r = d_cal - d_obs, per-RHS sum |r|^2.
__global__ void k_sample(const double* __restrict__ u, const int* __restrict__ rec_flat, int nrec,
                         const double* __restrict__ d_obs, double* __restrict__ d_cal, double* __restrict__ resid,
                         double* __restrict__ jpart, size_t n) {
    __shared__ double sh[32];
    const int b = blockIdx.x;
    double acc[1] = {0.0};
    for (int k = threadIdx.x; k < nrec; k += blockDim.x) {
        const size_t i = (size_t)n * b + rec_flat[k];
        const size_t o = (size_t)nrec * b + k;
        const double ur = u[2 * i], ui = u[2 * i + 1];
        if (d_cal) { d_cal[2 * o] = ur; d_cal[2 * o + 1] = ui; }
        const double rr = ur - d_obs[2 * o], ri = ui - d_obs[2 * o + 1];
        resid[2 * o] = rr;
        resid[2 * o + 1] = ri;
        acc[0] += rr * rr + ri * ri;
    }
    block_sum<1>(acc, sh);
    if (threadIdx.x == 0) jpart[b] = acc[0];
}

void launch_sample(const double* u, const int* rec_flat, int nrec, const double* d_obs, double* d_cal, double* resid,
                   double* jpart, size_t n, int nrhs, cudaStream_t s) {
    k_sample<<<nrhs, 256, 0, s>>>(u, rec_flat, nrec, d_obs, d_cal, resid, jpart, n);
}

// Adjoint right-hand side of the grid-scaled system: h^2 conj(P^T r), summed in
// receiver order by one thread per right-hand side.
__global__ void k_adjoint_rhs(const double* __restrict__ resid, const int* __restrict__ rec_flat, int nrec,
                              double h2, double* f, size_t n, int nrhs) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nrhs) return;
    for (int k = 0; k < nrec; ++k) {
        const size_t i = (size_t)n * b + rec_flat[k];
        const size_t o = (size_t)nrec * b + k;
        f[2 * i] += h2 * resid[2 * o];
        f[2 * i + 1] -= h2 * resid[2 * o + 1];
    }
}

void launch_adjoint_rhs(const double* resid, const int* rec_flat, int nrec, double h2, double* f, size_t n, int nrhs,
                        cudaStream_t s) {
    cudaMemsetAsync(f, 0, sizeof(double) * 2 * n * nrhs, s);
    k_adjoint_rhs<<<(nrhs + 63) / 64, 64, 0, s>>>(resid, rec_flat, nrec, h2, f, n, nrhs);
}

// g_pad += sum_b 4 w_b^2 m Re[(1 - j alpha) u_b w_b], w_b = conj(lambda_b) = B^{-1} conj(P^T r_b).
__global__ void k_grad_accum(const double* __restrict__ u, const double* __restrict__ wv, const double* __restrict__ w2,
                             const double* __restrict__ m_pad, int nx, int nz, int npml, double acoef,
                             double* __restrict__ g_pad, int nrhs) {
    const size_t n = (size_t)nx * nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nx), iz = (int)(i / nx);
        const double a = layer_alpha_t<double>(ix, iz, nx, nz, npml, acoef);
        double acc = 0.0;
        for (int b = 0; b < nrhs; ++b) {
            const cx<double> uu = ldc(u, n * b + i), ww = ldc(wv, n * b + i);
            const cx<double> q = uu * ww;
            acc += 4.0 * w2[b] * (q.re + a * q.im);    // Re[(1 - j a) q]
        }
        g_pad[i] += m_pad[i] * acc;
    }
}

void launch_grad_accum(const double* u, const double* w, const double* w2, const double* m_pad, int nx, int nz,
                       int npml, double amax, double* g_pad, int nrhs, cudaStream_t s) {
    k_grad_accum<<<grid1d((size_t)nx * nz), 256, 0, s>>>(u, w, w2, m_pad, nx, nz, npml, layer_coef(npml, amax), g_pad, nrhs);
}

// g = E^T g_pad + 2 lam x on the physical cells, x = the slowness (reg null) or
// the physical vector reg: each edge cell also collects the layer nodes that
// copy its slowness.
__global__ void k_fold(const double* __restrict__ g_pad, const double* __restrict__ m_pad, int Px, int Pz, int npml,
                       double lam, const double* __restrict__ reg, double* __restrict__ g) {
    const int nx = Px + 2 * npml;
    const size_t n = (size_t)Px * Pz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int px = (int)(i % Px), pz = (int)(i / Px);
        const int xlo = px == 0 ? 0 : px + npml, xhi = px == Px - 1 ? nx - 1 : px + npml;
        const int zlo = pz == 0 ? 0 : pz + npml, zhi = pz == Pz - 1 ? Pz + 2 * npml - 1 : pz + npml;
        double acc = 0.0;
        for (int iz = zlo; iz <= zhi; ++iz)
            for (int ix = xlo; ix <= xhi; ++ix) acc += g_pad[(size_t)iz * nx + ix];
        const double x = reg ? reg[i] : m_pad[(size_t)(pz + npml) * nx + px + npml];
        g[i] = acc + 2.0 * lam * x;
    }
}

void launch_fold(const double* g_pad, const double* m_pad, int Px, int Pz, int npml, double lam, double* g,
                 cudaStream_t s, const double* reg) {
    k_fold<<<grid1d((size_t)Px * Pz), 256, 0, s>>>(g_pad, m_pad, Px, Pz, npml, lam, reg, g);
}

// ------------------------------------------------------ Gauss-Newton (Eq. 9)
// E dm: a physical perturbation copied onto the padded grid (edge replication,
// as the slowness itself).
__global__ void k_expand(const double* __restrict__ dm, int Px, int Pz, int npml, double* __restrict__ dm_pad) {
    const int nx = Px + 2 * npml, nz = Pz + 2 * npml;
    const size_t n = (size_t)nx * nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nx), iz = (int)(i / nx);
        const int px = min(max(ix - npml, 0), Px - 1), pz = min(max(iz - npml, 0), Pz - 1);
        dm_pad[i] = dm[(size_t)pz * Px + px];
    }
}

void launch_expand(const double* dm, int Px, int Pz, int npml, double* dm_pad, cudaStream_t s) {
    k_expand<<<grid1d((size_t)(Px + 2 * npml) * (Pz + 2 * npml)), 256, 0, s>>>(dm, Px, Pz, npml, dm_pad);
}

// Born right-hand side of the grid-scaled system: the first-order change of
// B(m) u = f under m -> m + dm is B du = -(dB/dm . dm) u = 2 omega^2 m (1 - j alpha)
// dm u, times h^2: f_b = 2 (h omega_b)^2 m dm (1 - j alpha) u_b.
__global__ void k_born_rhs(const double* __restrict__ u, const double* __restrict__ dm_pad,
                           const double* __restrict__ m_pad, const double* __restrict__ hw2, int nx, int nz, int npml,
                           double acoef, double* __restrict__ f) {
    const size_t n = (size_t)nx * nz;
    const int b = blockIdx.z;
    const double c = 2.0 * hw2[b];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nx), iz = (int)(i / nx);
        const double a = layer_alpha_t<double>(ix, iz, nx, nz, npml, acoef);
        const double s = c * m_pad[i] * dm_pad[i];
        const cx<double> uu = ldc(u, n * b + i);
        stc(f, n * b + i, cx<double>(s * (uu.re + a * uu.im), s * (uu.im - a * uu.re)));   // s (1 - j a) u
    }
}

void launch_born_rhs(const double* u, const double* dm_pad, const double* m_pad, const double* hw2, int nx, int nz,
                     int npml, double amax, double* f, int nrhs, cudaStream_t s) {
    k_born_rhs<<<dim3(grid1d((size_t)nx * nz), 1, nrhs), 256, 0, s>>>(u, dm_pad, m_pad, hw2, nx, nz, npml,
                                                                     layer_coef(npml, amax), f);
}

// Per-block partial sums of a . b over n reals (the host adds the partials in
// block order, so the result does not depend on timing).
__global__ void k_dot_partials(const double* __restrict__ a, const double* __restrict__ b, size_t n, double* part) {
    __shared__ double sh[32];
    double acc[1] = {0.0};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        acc[0] += a[i] * b[i];
    block_sum<1>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
}

int dot_blocks(size_t n) { return std::min(grid1d(n), 256); }

void launch_dot_partials(const double* a, const double* b, size_t n, double* part, cudaStream_t s) {
    k_dot_partials<<<dot_blocks(n), 256, 0, s>>>(a, b, n, part);
}

// y = alpha x + beta y over n reals
__global__ void k_axpby(double alpha, const double* __restrict__ x, double beta, double* __restrict__ y, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = alpha * x[i] + beta * y[i];
}

void launch_axpby(double alpha, const double* x, double beta, double* y, size_t n, cudaStream_t s) {
    k_axpby<<<grid1d(n), 256, 0, s>>>(alpha, x, beta, y, n);
}

// ------------------------------------------------------- instantiations

#define HELM_INST(T)                                                                                              \
    template void launch_bicg_init<T>(const T*, T*, T*, T*, T*, T*, double*, int, RhsState*, int*, size_t, int,   \
                                      cudaStream_t);                                                              \
    template void launch_bicg_p<T>(const T*, T*, const T*, const RhsState*, size_t, int, cudaStream_t);           \
    template void launch_bicg_s<T>(const T*, const T*, T*, const RhsState*, size_t, int, cudaStream_t);           \
    template void launch_bicg_xr<T>(T*, const T*, const T*, const T*, const T*, const T*, T*, double*, int,       \
                                    RhsState*, int*, size_t, int, cudaStream_t);                                  \
    template void launch_restrict<T>(const LevelDev&, const LevelDev&, const T*, double, double, double,          \
                                     const T*, T*, const RhsState*, int, cudaStream_t, int);                      \
    template void launch_prolong<T>(int, const LevelDev&, const LevelDev&, int, double, const T*, double,         \
                                    double, double, const T*, const T*, T*, T*, const T*, double*, int,           \
                                    RhsState*, int, cudaStream_t, int, int);                                      \
    template void launch_coarse<T>(int, const T*, const int*, const T*, T*, const RhsState*, int, cudaStream_t);
HELM_INST(float)
HELM_INST(double)
#undef HELM_INST

}  // namespace helm

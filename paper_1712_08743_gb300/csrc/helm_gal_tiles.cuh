// helm_gal_tiles.cuh - tile bodies of the Galerkin multigrid levels, shared by
// the one-launch-per-level kernels (k_restrict_g, k_prolong_g in
// helm_kernels.cu) and the persistent F-cycle kernel (helm_fcycle.cu).
//
// A tile is worked on by a group of threads (a whole block, or a fixed part of
// one) that synchronises with a Sync policy: BlockSync (__syncthreads) or
// GroupSync (a named barrier of the group's threads). Each tile body has two
// halves: stage, which reads only model data (the Galerkin coefficients) and
// may run before the data of the previous step is ready, and work, which reads
// the level vectors. Vectors written earlier in the same kernel launch (the
// persistent kernel) must be read through L2 (COH = true, ld.global.cg); the
// one-launch kernels read them through the non-coherent path.
#pragma once

#include "helm_internal.h"

namespace helm {

struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
// named barrier `id` (1..15) of `nthreads` threads (a multiple of 32)
struct GroupSync {
    int id, nthreads;
    __device__ __forceinline__ void operator()() const {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
    }
};

template <bool COH>
__device__ __forceinline__ cx<float> ldv(const float* p, size_t i) {
    if constexpr (COH) {
        const float2 v = __ldcg(reinterpret_cast<const float2*>(p) + i);
        return {v.x, v.y};
    } else {
        return ldc(p, i);
    }
}
template <bool COH>
__device__ __forceinline__ cx<double> ldv(const double* p, size_t i) {
    if constexpr (COH) {
        const double2 v = __ldcg(reinterpret_cast<const double2*>(p) + i);
        return {v.x, v.y};
    } else {
        return ldc(p, i);
    }
}

// Bilinear prolongation along one axis at fine index g (coarse node I sits on
// fine 2I+1): odd g takes coarse (g-1)/2 with weight 1, even g takes g/2-1 and
// g/2 with weight 1/2 each. Branch-free: a = (g-1)>>1, b = g>>1 (arithmetic
// shift, so g = 0 gives a = -1).
template <typename T>
__device__ __forceinline__ void bil_axis(int g, int& a, int& b, T& wa, T& wb) {
    const bool odd = g & 1;
    a = (g - 1) >> 1;
    b = g >> 1;
    wa = odd ? T(1) : T(0.5);
    wb = odd ? T(0) : T(0.5);
}

// ================================ Galerkin grid levels: staged coefficients
// On the coarse grid levels the 9-point coefficients would otherwise be read
// one by one per stencil evaluation, serialising each tile on memory latency.
// The tiles first stage, cooperatively and coalesced, the per-RHS complex
// coefficients M_k = G_k - hw (b1 - j b2) K_k of their region into shared
// memory, then work from there.
template <typename T, int W, int H>
struct GalTile {
    cx<T> c[5][H][W];   // centre, east, north, north-east, north-west
};

template <typename T, int W, int H, int NT>
__device__ __forceinline__ void stage_gal(GalTile<T, W, H>& t, const LevelDev& L, int b, T hb1, T hb2, int gx0,
                                          int gz0, int tid) {
    const T* gk = static_cast<const T*>(L.gk) + (size_t)b * L.gkstride;
    const size_t n = (size_t)L.nx * L.nz;
    // one node per step, its ten coefficients loaded independently; the steps have a fixed
    // count so that the loads of all of them can be in flight together
#pragma unroll
    for (int k = 0; k < (W * H + NT - 1) / NT; ++k) {
        const int idx = tid + k * NT;
        if (idx >= W * H) break;
        const int lz = idx / W, lx = idx - lz * W;
        const int gx = gx0 + lx, gz = gz0 + lz;
        T g[5], q[5];
        const bool in = gx >= 0 && gx < L.nx && gz >= 0 && gz < L.nz;
        const size_t i = in ? (size_t)gz * L.nx + gx : 0;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            g[k] = in ? __ldg(gk + (size_t)k * n + i) : T(0);
            q[k] = in ? __ldg(gk + (size_t)(5 + k) * n + i) : T(0);
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) t.c[k][lz][lx] = cx<T>(g[k] - hb1 * q[k], hb2 * q[k]);
    }
}

// The real Galerkin coefficients of a tile region (G then K, five entries each),
// which do not depend on the frequency: a block working on several right-hand
// sides of one model stages them once, then forms each right-hand side's complex
// coefficients from shared memory (form_gal) instead of reading them again.
template <typename T, int W, int H>
struct GalReal {
    T g[kGalerkinCoefs][H][W];
};

template <typename T, int W, int H, int NT>
__device__ __forceinline__ void stage_gal_real(GalReal<T, W, H>& t, const LevelDev& L, int gx0, int gz0, int tid) {
    const T* gk = static_cast<const T*>(L.gk);
    const size_t n = (size_t)L.nx * L.nz;
#pragma unroll
    for (int k = 0; k < (W * H + NT - 1) / NT; ++k) {
        const int idx = tid + k * NT;
        if (idx >= W * H) break;
        const int lz = idx / W, lx = idx - lz * W;
        const int gx = gx0 + lx, gz = gz0 + lz;
        const bool in = gx >= 0 && gx < L.nx && gz >= 0 && gz < L.nz;
        const size_t i = in ? (size_t)gz * L.nx + gx : 0;
        T v[kGalerkinCoefs];
#pragma unroll
        for (int q = 0; q < kGalerkinCoefs; ++q) v[q] = in ? __ldg(gk + (size_t)q * n + i) : T(0);
#pragma unroll
        for (int q = 0; q < kGalerkinCoefs; ++q) t.g[q][lz][lx] = v[q];
    }
}

// M_k = G_k - hw (b1 - j b2) K_k of the staged region, as stage_gal forms it
template <typename T, int W, int H, int NT>
__device__ __forceinline__ void form_gal(GalTile<T, W, H>& t, const GalReal<T, W, H>& r, T hb1, T hb2, int tid) {
    for (int idx = tid; idx < W * H; idx += NT) {
        const int lz = idx / W, lx = idx - lz * W;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const T q = r.g[5 + k][lz][lx];
            t.c[k][lz][lx] = cx<T>(r.g[k][lz][lx] - hb1 * q, hb2 * q);
        }
    }
}

// M u at tile point (lx, lz) (global (gx, gz)); U row pitch W; coefficients of
// the neighbours come from the staged tile (the point must not lie on the
// tile border).
template <typename T, int W, int H>
__device__ __forceinline__ cx<T> mop9_staged(const GalTile<T, W, H>& t, int nx, int nz, int gx, int gz, int lx, int lz,
                                             const cx<T>* U) {
    cx<T> acc = t.c[0][lz][lx] * U[0];
    const bool e = gx + 1 < nx, w = gx > 0, no = gz + 1 < nz, so = gz > 0;
    if (e) acc = acc + t.c[1][lz][lx] * U[1];
    if (w) acc = acc + t.c[1][lz][lx - 1] * U[-1];
    if (no) acc = acc + t.c[2][lz][lx] * U[W];
    if (so) acc = acc + t.c[2][lz - 1][lx] * U[-W];
    if (no && e) acc = acc + t.c[3][lz][lx] * U[W + 1];
    if (so && w) acc = acc + t.c[3][lz - 1][lx - 1] * U[-W - 1];
    if (no && w) acc = acc + t.c[4][lz][lx] * U[W - 1];
    if (so && e) acc = acc + t.c[4][lz - 1][lx + 1] * U[-W + 1];
    return acc;
}

// Default tiles of the Galerkin kernels: restriction coarse tile RCX x RCZ,
// prolongation fine tile PX x PZ; halved in x for complex128 to stay within 48 KB
// of static shared memory. The complex64 kernels also come in the other shapes of
// kGalTiles (helm_kernels.cu), among which the autotuner chooses per level.
template <typename T> struct GTile {
    static constexpr int RCX = sizeof(T) == 4 ? 16 : 8, RCZ = 8;
    static constexpr int PX = sizeof(T) == 4 ? 32 : 16, PZ = 8;
};

// ------------------------------------------------------------ restriction
// Coarse tile (I0, K0) of GRCX x GRCZ nodes, NT >= GRCX * GRCZ threads: from the fine
// level's right-hand side f (zero initial guess), one damped-Jacobi sweep
// u1 = wj D^-1 f (CORRECT: u2 = wj D^-1 f + P e, e the first coarse correction of
// an F-cycle), the residual r = f - M u on the fine region, and its restriction
// P^T r (full weighting times 4) to the coarse tile.
template <typename T, int GRCX, int GRCZ_ = GTile<T>::RCZ, int NT_ = GRCX * GRCZ_>
struct RestrictTile {
    static constexpr int GRCZ = GRCZ_;
    static constexpr int GRFW = 2 * GRCX + 3, GRFH = 2 * GRCZ + 3;
    static constexpr int CEW = GRCX + 2, CEH = GRCZ + 2;
    static constexpr int NT = NT_;   // threads of the tile (more than its coarse nodes spreads the fine work)
    static_assert(NT >= GRCX * GRCZ, "one thread per coarse node at least");
    GalTile<T, GRFW, GRFH> C;
    cx<T> F[GRFH][GRFW];
    cx<T> U[GRFH][GRFW];
    cx<T> E[CEH][CEW];
};

template <typename T, int GRCX, int GRCZ, int NT>
__device__ __forceinline__ void restrict_tile_stage(RestrictTile<T, GRCX, GRCZ, NT>& sm, const LevelDev& Lf, int bx,
                                                    int by, int b, T hw, T b1, T b2, int tid) {
    using RT = RestrictTile<T, GRCX, GRCZ, NT>;
    const int I0 = bx * GRCX, K0 = by * RT::GRCZ;
    stage_gal<T, RT::GRFW, RT::GRFH, RT::NT>(sm.C, Lf, b, hw * b1, hw * b2, 2 * I0 - 1, 2 * K0 - 1, tid);
}

template <typename T, bool CORRECT, int GRCX, int GRCZ, int NT_, bool COH, class Sync>
__device__ __forceinline__ void restrict_tile_work(RestrictTile<T, GRCX, GRCZ, NT_>& sm, const LevelDev& Lf,
                                                   const LevelDev& Lc, T wj, const T* f, const T* ec, T* fc, int bx,
                                                   int by, int b, int tid, Sync sync) {
    using RT = RestrictTile<T, GRCX, GRCZ, NT_>;
    constexpr int GRFW = RT::GRFW, GRFH = RT::GRFH, CEW = RT::CEW, CEH = RT::CEH;
    const int I0 = bx * GRCX, K0 = by * GRCZ;
    const int gx0 = 2 * I0 - 1, gz0 = 2 * K0 - 1;
    const size_t nf = (size_t)Lf.nx * Lf.nz, nc = (size_t)Lc.nx * Lc.nz;
    const T* fb = f + 2 * nf * b;
    // this thread's points of the fine region; their right-hand side is loaded
    // before, and independently of, the coarse correction
    constexpr int NT = RT::NT, NF = GRFW * GRFH, NPT = (NF + NT - 1) / NT;
    cx<T> fpre[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int idx = tid + k * NT;
        const int lz = idx / GRFW, lx = idx - lz * GRFW;
        const int gx = gx0 + lx, gz = gz0 + lz;
        fpre[k] = (idx < NF && gx >= 0 && gx < Lf.nx && gz >= 0 && gz < Lf.nz)
                      ? ldv<COH>(fb, (size_t)gz * Lf.nx + gx) : cx<T>(0, 0);
    }
    if (CORRECT) {
        const T* eb = ec + 2 * nc * b;
        for (int idx = tid; idx < CEW * CEH; idx += NT) {
            const int lz = idx / CEW, lx = idx - lz * CEW;
            const int I = I0 - 1 + lx, K = K0 - 1 + lz;
            cx<T> e(0, 0);
            if (I >= 0 && I < Lc.nx && K >= 0 && K < Lc.nz) e = ldv<COH>(eb, (size_t)K * Lc.nx + I);
            sm.E[lz][lx] = e;
        }
    }
    sync();
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int idx = tid + k * NT;
        if (idx >= NF) break;
        const int lz = idx / GRFW, lx = idx - lz * GRFW;
        const int gx = gx0 + lx, gz = gz0 + lz;
        const cx<T> fv = fpre[k];
        cx<T> uv(0, 0);
        if (gx >= 0 && gx < Lf.nx && gz >= 0 && gz < Lf.nz) {
            uv = wj * cdiv(fv, sm.C.c[0][lz][lx]);
            if (CORRECT) {
                int ia, ib, ka, kb;
                T wa, wb, va, vb;
                bil_axis<T>(gx, ia, ib, wa, wb);
                bil_axis<T>(gz, ka, kb, va, vb);
                ia -= I0 - 1; ib -= I0 - 1; ka -= K0 - 1; kb -= K0 - 1;
                uv = uv + (va * wa) * sm.E[ka][ia] + (va * wb) * sm.E[ka][ib] + (vb * wa) * sm.E[kb][ia] +
                     (vb * wb) * sm.E[kb][ib];
            }
        }
        sm.F[lz][lx] = fv;
        sm.U[lz][lx] = uv;
    }
    sync();
    constexpr int W2 = GRFW - 2, H2 = GRFH - 2;
    for (int idx = tid; idx < W2 * H2; idx += NT) {
        const int lz = 1 + idx / W2, lx = 1 + idx % W2;
        const int gx = gx0 + lx, gz = gz0 + lz;
        cx<T> r(0, 0);
        if (gx < Lf.nx && gz < Lf.nz)
            r = sm.F[lz][lx] - mop9_staged<T, GRFW, GRFH>(sm.C, Lf.nx, Lf.nz, gx, gz, lx, lz, &sm.U[lz][lx]);
        sm.F[lz][lx] = r;
    }
    sync();
    const int cxl = tid % GRCX, czl = tid / GRCX;
    const int I = I0 + cxl, K = K0 + czl;
    if (tid < GRCX * GRCZ && I < Lc.nx && K < Lc.nz) {
        const int lx = 2 * cxl + 2, lz = 2 * czl + 2;
        cx<T> a = T(4) * sm.F[lz][lx];
        a = a + T(2) * (sm.F[lz][lx - 1] + sm.F[lz][lx + 1] + sm.F[lz - 1][lx] + sm.F[lz + 1][lx]);
        a = a + sm.F[lz - 1][lx - 1] + sm.F[lz - 1][lx + 1] + sm.F[lz + 1][lx - 1] + sm.F[lz + 1][lx + 1];
        stc(fc + 2 * nc * b, (size_t)K * Lc.nx + I, T(0.25) * a);
    }
}

// ------------------------------ restriction of the second coarse correction
// In an F-cycle at level l the second coarse correction solves M_{l+1} d = P^T (f_l - M_l u2)
// with u2 = wj D^-1 f_l + P e (e the first correction). With the Galerkin operator
// M_{l+1} = P^T M_l P and the restriction P^T this right-hand side is
// g = f_{l+1} - M_{l+1} e, where f_{l+1} = P^T (f_l - M_l wj D^-1 f_l) is what the first
// restriction wrote: level l + 1 data only. The V-cycle of that correction starts at
// level l + 1, so this tile (level l + 1 -> l + 2) forms g on its fine region, writes
// the nodes it owns to `g` (the V-cycle's prolongation reads them again), and goes
// on as the plain restriction: u1 = wj D^-1 g, r = g - M u1, P^T r to the coarse tile.
// Fields and coefficients share one pitch: the fine region of the plain tile plus a
// halo of one node, which g = f - M e needs on the region's border.
template <typename T, int GRCX, int GRCZ, int NT_>
struct ResidRestrictTile {
    static constexpr int XW = 2 * GRCX + 5, XH = 2 * GRCZ + 5;   // region + halo
    static constexpr int NT = NT_;
    static_assert(NT >= GRCX * GRCZ, "one thread per coarse node at least");
    GalTile<T, XW, XH> C;
    cx<T> E[XH][XW];
    cx<T> F[XH][XW];
    cx<T> U[XH][XW];
};

template <typename T, int GRCX, int GRCZ, int NT>
__device__ __forceinline__ void resid_restrict_tile_stage(ResidRestrictTile<T, GRCX, GRCZ, NT>& sm, const LevelDev& Lf,
                                                          int bx, int by, int b, T hw, T b1, T b2, int tid) {
    using RT = ResidRestrictTile<T, GRCX, GRCZ, NT>;
    stage_gal<T, RT::XW, RT::XH, NT>(sm.C, Lf, b, hw * b1, hw * b2, 2 * bx * GRCX - 2, 2 * by * GRCZ - 2, tid);
}

template <typename T, int GRCX, int GRCZ, int NT, bool COH, class Sync>
__device__ __forceinline__ void resid_restrict_tile_work(ResidRestrictTile<T, GRCX, GRCZ, NT>& sm, const LevelDev& Lf,
                                                         const LevelDev& Lc, T wj, const T* f, const T* e, T* g,
                                                         T* fc, int bx, int by, int b, int tid, Sync sync) {
    using RT = ResidRestrictTile<T, GRCX, GRCZ, NT>;
    constexpr int XW = RT::XW, XH = RT::XH, NX = XW * XH, NPT = (NX + NT - 1) / NT;
    const int I0 = bx * GRCX, K0 = by * GRCZ;
    const int xx0 = 2 * I0 - 2, xz0 = 2 * K0 - 2;   // global position of the halo's corner
    const size_t nf = (size_t)Lf.nx * Lf.nz, nc = (size_t)Lc.nx * Lc.nz;
    const T* fb = f + 2 * nf * b;
    const T* eb = e + 2 * nf * b;
    // fine nodes this tile writes to g: x in [2 I0, 2 (I0 + GRCX)), the last tile of a row up to
    // the grid's edge (likewise in z), so every node of the level has one owner
    const int ox1 = (I0 + GRCX >= Lc.nx) ? Lf.nx : 2 * (I0 + GRCX);
    const int oz1 = (K0 + GRCZ >= Lc.nz) ? Lf.nz : 2 * (K0 + GRCZ);
    // e on the region and its halo, f on the region: all loads issued before use
    cx<T> epre[NPT], fpre[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int idx = tid + k * NT;
        const int lz = idx / XW, lx = idx - lz * XW;
        const int gx = xx0 + lx, gz = xz0 + lz;
        const bool in = idx < NX && gx >= 0 && gx < Lf.nx && gz >= 0 && gz < Lf.nz;
        const size_t i = in ? (size_t)gz * Lf.nx + gx : 0;
        const bool reg = in && lx >= 1 && lx <= XW - 2 && lz >= 1 && lz <= XH - 2;
        epre[k] = in ? ldv<COH>(eb, i) : cx<T>(0, 0);
        fpre[k] = reg ? ldv<COH>(fb, i) : cx<T>(0, 0);
    }
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int idx = tid + k * NT;
        if (idx >= NX) break;
        const int lz = idx / XW, lx = idx - lz * XW;
        sm.E[lz][lx] = epre[k];
        sm.F[lz][lx] = fpre[k];
    }
    sync();
    // g = f - M e and u1 = wj D^-1 g on the region
    T* gb = g + 2 * nf * b;
    constexpr int RW = XW - 2, RH = XH - 2;
    for (int idx = tid; idx < RW * RH; idx += NT) {
        const int lz = 1 + idx / RW, lx = 1 + idx % RW;
        const int gx = xx0 + lx, gz = xz0 + lz;
        cx<T> gv(0, 0), uv(0, 0);
        if (gx >= 0 && gx < Lf.nx && gz >= 0 && gz < Lf.nz) {
            gv = sm.F[lz][lx] - mop9_staged<T, XW, XH>(sm.C, Lf.nx, Lf.nz, gx, gz, lx, lz, &sm.E[lz][lx]);
            uv = wj * cdiv(gv, sm.C.c[0][lz][lx]);
            if (gx >= 2 * I0 && gx < ox1 && gz >= 2 * K0 && gz < oz1) stc(gb, (size_t)gz * Lf.nx + gx, gv);
        }
        sm.F[lz][lx] = gv;
        sm.U[lz][lx] = uv;
    }
    sync();
    // r = g - M u1 on the nodes the restriction reads
    constexpr int W2 = XW - 4, H2 = XH - 4;
    for (int idx = tid; idx < W2 * H2; idx += NT) {
        const int lz = 2 + idx / W2, lx = 2 + idx % W2;
        const int gx = xx0 + lx, gz = xz0 + lz;
        cx<T> r(0, 0);
        if (gx < Lf.nx && gz < Lf.nz)
            r = sm.F[lz][lx] - mop9_staged<T, XW, XH>(sm.C, Lf.nx, Lf.nz, gx, gz, lx, lz, &sm.U[lz][lx]);
        sm.F[lz][lx] = r;
    }
    sync();
    const int cxl = tid % GRCX, czl = tid / GRCX;
    const int I = I0 + cxl, K = K0 + czl;
    if (tid < GRCX * GRCZ && I < Lc.nx && K < Lc.nz) {
        const int lx = 2 * cxl + 3, lz = 2 * czl + 3;
        cx<T> a = T(4) * sm.F[lz][lx];
        a = a + T(2) * (sm.F[lz][lx - 1] + sm.F[lz][lx + 1] + sm.F[lz - 1][lx] + sm.F[lz + 1][lx]);
        a = a + sm.F[lz - 1][lx - 1] + sm.F[lz - 1][lx + 1] + sm.F[lz + 1][lx - 1] + sm.F[lz + 1][lx + 1];
        stc(fc + 2 * nc * b, (size_t)K * Lc.nx + I, T(0.25) * a);
    }
}

// ----------------------------------------------------------- prolongation
// Fine tile (x0, z0) of GPX x GPZ nodes, GPX * GPZ threads: u = wj D^-1 f + P e
// on the tile and its halo, then the post-smoothing sweep u + wj D^-1 (f - M u),
// written to out (added to it when accumulating).
template <typename T, int GPX, int GPZ_ = GTile<T>::PZ>
struct ProlongTile {
    static constexpr int GPZ = GPZ_;
    static constexpr int RW = GPX + 2, RH = GPZ + 2;
    static constexpr int EW = GPX / 2 + 2, EH = GPZ / 2 + 2;
    static constexpr int NT = GPX * GPZ;
    GalTile<T, RW, RH> C;
    cx<T> F[RH][RW];
    cx<T> U2[RH][RW];
    cx<T> E[EH][EW];
};

template <typename T, int GPX, int GPZ>
__device__ __forceinline__ void prolong_tile_stage(ProlongTile<T, GPX, GPZ>& sm, const LevelDev& Lf, int bx, int by,
                                                   int b, T hw, T b1, T b2, int tid) {
    using PT = ProlongTile<T, GPX, GPZ>;
    stage_gal<T, PT::RW, PT::RH, PT::NT>(sm.C, Lf, b, hw * b1, hw * b2, bx * GPX - 1, by * PT::GPZ - 1, tid);
}

template <typename T, int GPX, int GPZ, bool COH, class Sync>
__device__ __forceinline__ void prolong_tile_work(ProlongTile<T, GPX, GPZ>& sm, const LevelDev& Lf, const LevelDev& Lc,
                                                  T wj, const T* f, const T* ec, T* out, int accumulate, int bx,
                                                  int by, int b, int tid, Sync sync) {
    using PT = ProlongTile<T, GPX, GPZ>;
    constexpr int RW = PT::RW, RH = PT::RH, EW = PT::EW, EH = PT::EH;
    const int x0 = bx * GPX, z0 = by * GPZ;
    const int gx0 = x0 - 1, gz0 = z0 - 1;
    const int cx0 = x0 / 2 - 1, cz0 = z0 / 2 - 1;
    const size_t nf = (size_t)Lf.nx * Lf.nz, nc = (size_t)Lc.nx * Lc.nz;
    const T* fb = f + 2 * nf * b;
    const T* eb = ec + 2 * nc * b;
    // this thread's points of the fine region; their right-hand side is loaded
    // before, and independently of, the coarse correction
    constexpr int NT = PT::NT, NF = RW * RH, NPT = (NF + NT - 1) / NT;
    cx<T> fpre[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int idx = tid + k * NT;
        const int lz = idx / RW, lx = idx - lz * RW;
        const int gx = gx0 + lx, gz = gz0 + lz;
        fpre[k] = (idx < NF && gx >= 0 && gx < Lf.nx && gz >= 0 && gz < Lf.nz)
                      ? ldv<COH>(fb, (size_t)gz * Lf.nx + gx) : cx<T>(0, 0);
    }
    // the output point this thread accumulates into (one per thread), loaded with them
    T* ob = out + 2 * nf * b;
    cx<T> opre(0, 0);
    {
        const int tz = tid / GPX, tx = tid - tz * GPX;
        if (accumulate && x0 + tx < Lf.nx && z0 + tz < Lf.nz) {
            const size_t i = (size_t)(z0 + tz) * Lf.nx + x0 + tx;
            opre = COH ? ldv<true>(ob, i) : ldcc(ob, i);
        }
    }
    for (int idx = tid; idx < EW * EH; idx += NT) {
        const int lz = idx / EW, lx = idx - lz * EW;
        const int I = cx0 + lx, K = cz0 + lz;
        cx<T> e(0, 0);
        if (I >= 0 && I < Lc.nx && K >= 0 && K < Lc.nz) e = ldv<COH>(eb, (size_t)K * Lc.nx + I);
        sm.E[lz][lx] = e;
    }
    sync();
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int idx = tid + k * NT;
        if (idx >= NF) break;
        const int lz = idx / RW, lx = idx - lz * RW;
        const int gx = gx0 + lx, gz = gz0 + lz;
        const cx<T> fv = fpre[k];
        cx<T> u(0, 0);
        if (gx >= 0 && gx < Lf.nx && gz >= 0 && gz < Lf.nz) {
            u = wj * cdiv(fv, sm.C.c[0][lz][lx]);
            int ia, ib, ka, kb;
            T wa, wb, va, vb;
            bil_axis<T>(gx, ia, ib, wa, wb);
            bil_axis<T>(gz, ka, kb, va, vb);
            ia -= cx0; ib -= cx0; ka -= cz0; kb -= cz0;
            u = u + (va * wa) * sm.E[ka][ia] + (va * wb) * sm.E[ka][ib] + (vb * wa) * sm.E[kb][ia] +
                (vb * wb) * sm.E[kb][ib];
        }
        sm.F[lz][lx] = fv;
        sm.U2[lz][lx] = u;
    }
    sync();
    const int tz = tid / GPX, tx = tid - tz * GPX;   // one output point per thread
    const int gx = x0 + tx, gz = z0 + tz;
    if (gx < Lf.nx && gz < Lf.nz) {
        const int lx = tx + 1, lz = tz + 1;
        const size_t i = (size_t)gz * Lf.nx + gx;
        const cx<T> c = sm.U2[lz][lx];
        const cx<T> mu = mop9_staged<T, RW, RH>(sm.C, Lf.nx, Lf.nz, gx, gz, lx, lz, &sm.U2[lz][lx]);
        const cx<T> v = c + wj * cdiv(sm.F[lz][lx] - mu, sm.C.c[0][lz][lx]);
        stc(ob, i, accumulate ? opre + v : v);
    }
}

// ------------------------------------------- two prolongations in one tile
// The prolongation of level l + 1 (from e of level l + 2) followed by that of
// level l, for the fine tile (x0, z0) of GPX x GPZ nodes of level l: the level l
// + 1 values the tile's prolongation reads (ProlongTile::E, the tile's coarse
// footprint) are computed in shared memory instead of being read back from a
// kernel launched before: u2 = wj D^-1 f + P e on that footprint and a halo of
// one, then u2 + wj D^-1 (f - M u2) (added to the level's previous correction when
// acc_m). Each node's arithmetic is the one-level tile's, so the result is that of
// the two launches; level l + 1's correction is not written (nothing reads it).
template <typename T, int GPX, int GPZ>
struct Prolong2Tile {
    using PT = ProlongTile<T, GPX, GPZ>;
    static constexpr int EW = PT::EW, EH = PT::EH;            // level l + 1 nodes the level l tile reads
    static constexpr int MW = EW + 2, MH = EH + 2;            // their u2 region
    static constexpr int CW = EW / 2 + 3, CH = EH / 2 + 3;    // level l + 2 footprint of that region (bound)
    PT fine;
    GalTile<T, MW, MH> MC;
    cx<T> MF[MH][MW];
    cx<T> MU[MH][MW];
    cx<T> CE[CH][CW];
};

template <typename T, int GPX, int GPZ>
__device__ __forceinline__ void prolong2_tile_stage(Prolong2Tile<T, GPX, GPZ>& sm, const LevelDev& Lf,
                                                    const LevelDev& Lm, int bx, int by, int b, T hw, T b1, T b2,
                                                    int tid) {
    using P2 = Prolong2Tile<T, GPX, GPZ>;
    prolong_tile_stage<T, GPX, GPZ>(sm.fine, Lf, bx, by, b, hw, b1, b2, tid);
    const int ax0 = bx * GPX / 2 - 1, az0 = by * GPZ / 2 - 1;
    stage_gal<T, P2::MW, P2::MH, GPX * GPZ>(sm.MC, Lm, b, hw * b1, hw * b2, ax0 - 1, az0 - 1, tid);
}

// fl, fm: right-hand sides of levels l and l + 1; ec: correction of level l + 2;
// out: level l's correction (added to when acc_f); em: level l + 1's previous
// correction (added when acc_m).
template <typename T, int GPX, int GPZ, bool COH, class Sync>
__device__ __forceinline__ void prolong2_tile_work(Prolong2Tile<T, GPX, GPZ>& sm, const LevelDev& Lf,
                                                   const LevelDev& Lm, const LevelDev& Lc, T wj, const T* fl,
                                                   const T* fm, const T* ec, const T* em, T* out, int acc_f,
                                                   int acc_m, int bx, int by, int b, int tid, Sync sync) {
    using P2 = Prolong2Tile<T, GPX, GPZ>;
    using PT = typename P2::PT;
    constexpr int NT = PT::NT, RW = PT::RW, RH = PT::RH, EW = P2::EW, EH = P2::EH;
    constexpr int MW = P2::MW, MH = P2::MH, CW = P2::CW, CH = P2::CH;
    constexpr int NF = RW * RH, NPT = (NF + NT - 1) / NT, NM = MW * MH, NMP = (NM + NT - 1) / NT;
    const int x0 = bx * GPX, z0 = by * GPZ;
    const int gx0 = x0 - 1, gz0 = z0 - 1;                  // level l region
    const int ax0 = x0 / 2 - 1, az0 = z0 / 2 - 1;          // level l + 1 nodes read by the tile
    const int mx0 = ax0 - 1, mz0 = az0 - 1;                // their u2 region
    const int kx0 = (mx0 - 1) >> 1, kz0 = (mz0 - 1) >> 1;  // level l + 2 footprint
    const size_t nf = (size_t)Lf.nx * Lf.nz, nm = (size_t)Lm.nx * Lm.nz, nc = (size_t)Lc.nx * Lc.nz;
    const T* fb = fl + 2 * nf * b;
    const T* mb = fm + 2 * nm * b;
    // every global load of the tile, issued before any is used
    cx<T> fpre[NPT], mpre[NMP];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int idx = tid + k * NT;
        const int lz = idx / RW, lx = idx - lz * RW;
        const int gx = gx0 + lx, gz = gz0 + lz;
        fpre[k] = (idx < NF && gx >= 0 && gx < Lf.nx && gz >= 0 && gz < Lf.nz)
                      ? ldv<COH>(fb, (size_t)gz * Lf.nx + gx) : cx<T>(0, 0);
    }
#pragma unroll
    for (int k = 0; k < NMP; ++k) {
        const int idx = tid + k * NT;
        const int lz = idx / MW, lx = idx - lz * MW;
        const int gx = mx0 + lx, gz = mz0 + lz;
        mpre[k] = (idx < NM && gx >= 0 && gx < Lm.nx && gz >= 0 && gz < Lm.nz)
                      ? ldv<COH>(mb, (size_t)gz * Lm.nx + gx) : cx<T>(0, 0);
    }
    T* ob = out + 2 * nf * b;
    cx<T> opre(0, 0);
    {
        const int tz = tid / GPX, tx = tid - tz * GPX;
        if (acc_f && x0 + tx < Lf.nx && z0 + tz < Lf.nz) {
            const size_t i = (size_t)(z0 + tz) * Lf.nx + x0 + tx;
            opre = COH ? ldv<true>(ob, i) : ldcc(ob, i);
        }
    }
    // the previous level l + 1 correction at the nodes this thread finishes below
    constexpr int NE = EW * EH, NEP = (NE + NT - 1) / NT;
    const T* emb = em + 2 * nm * b;
    cx<T> epre[NEP];
#pragma unroll
    for (int k = 0; k < NEP; ++k) {
        const int idx = tid + k * NT;
        const int lz = idx / EW, lx = idx - lz * EW;
        const int I = ax0 + lx, K = az0 + lz;
        epre[k] = (acc_m && idx < NE && I >= 0 && I < Lm.nx && K >= 0 && K < Lm.nz)
                      ? (COH ? ldv<true>(emb, (size_t)K * Lm.nx + I) : ldcc(emb, (size_t)K * Lm.nx + I))
                      : cx<T>(0, 0);
    }
    const T* eb = ec + 2 * nc * b;
    for (int idx = tid; idx < CW * CH; idx += NT) {
        const int lz = idx / CW, lx = idx - lz * CW;
        const int I = kx0 + lx, K = kz0 + lz;
        cx<T> e(0, 0);
        if (I >= 0 && I < Lc.nx && K >= 0 && K < Lc.nz) e = ldv<COH>(eb, (size_t)K * Lc.nx + I);
        sm.CE[lz][lx] = e;
    }
    sync();
    // level l + 1: u2 = wj D^-1 f + P e on its region
#pragma unroll
    for (int k = 0; k < NMP; ++k) {
        const int idx = tid + k * NT;
        if (idx >= NM) break;
        const int lz = idx / MW, lx = idx - lz * MW;
        const int gx = mx0 + lx, gz = mz0 + lz;
        const cx<T> fv = mpre[k];
        cx<T> u(0, 0);
        if (gx >= 0 && gx < Lm.nx && gz >= 0 && gz < Lm.nz) {
            u = wj * cdiv(fv, sm.MC.c[0][lz][lx]);
            int ia, ib, ka, kb;
            T wa, wb, va, vb;
            bil_axis<T>(gx, ia, ib, wa, wb);
            bil_axis<T>(gz, ka, kb, va, vb);
            ia -= kx0; ib -= kx0; ka -= kz0; kb -= kz0;
            u = u + (va * wa) * sm.CE[ka][ia] + (va * wb) * sm.CE[ka][ib] + (vb * wa) * sm.CE[kb][ia] +
                (vb * wb) * sm.CE[kb][ib];
        }
        sm.MF[lz][lx] = fv;
        sm.MU[lz][lx] = u;
    }
    sync();
    // level l + 1: the post-sweep on the nodes the level l tile reads, into its E
#pragma unroll
    for (int k = 0; k < NEP; ++k) {
        const int idx = tid + k * NT;
        if (idx >= NE) break;
        const int lz = idx / EW, lx = idx - lz * EW;
        const int gx = ax0 + lx, gz = az0 + lz;
        cx<T> e(0, 0);
        if (gx >= 0 && gx < Lm.nx && gz >= 0 && gz < Lm.nz) {
            const int mx = lx + 1, mz = lz + 1;
            const cx<T> c = sm.MU[mz][mx];
            const cx<T> mu = mop9_staged<T, MW, MH>(sm.MC, Lm.nx, Lm.nz, gx, gz, mx, mz, &sm.MU[mz][mx]);
            const cx<T> v = c + wj * cdiv(sm.MF[mz][mx] - mu, sm.MC.c[0][mz][mx]);
            e = acc_m ? epre[k] + v : v;
        }
        sm.fine.E[lz][lx] = e;
    }
    sync();
    // level l, as prolong_tile_work with its E above
    const int cx0 = ax0, cz0 = az0;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int idx = tid + k * NT;
        if (idx >= NF) break;
        const int lz = idx / RW, lx = idx - lz * RW;
        const int gx = gx0 + lx, gz = gz0 + lz;
        const cx<T> fv = fpre[k];
        cx<T> u(0, 0);
        if (gx >= 0 && gx < Lf.nx && gz >= 0 && gz < Lf.nz) {
            u = wj * cdiv(fv, sm.fine.C.c[0][lz][lx]);
            int ia, ib, ka, kb;
            T wa, wb, va, vb;
            bil_axis<T>(gx, ia, ib, wa, wb);
            bil_axis<T>(gz, ka, kb, va, vb);
            ia -= cx0; ib -= cx0; ka -= cz0; kb -= cz0;
            u = u + (va * wa) * sm.fine.E[ka][ia] + (va * wb) * sm.fine.E[ka][ib] + (vb * wa) * sm.fine.E[kb][ia] +
                (vb * wb) * sm.fine.E[kb][ib];
        }
        sm.fine.F[lz][lx] = fv;
        sm.fine.U2[lz][lx] = u;
    }
    sync();
    const int tz = tid / GPX, tx = tid - tz * GPX;
    const int gx = x0 + tx, gz = z0 + tz;
    if (gx < Lf.nx && gz < Lf.nz) {
        const int lx = tx + 1, lz = tz + 1;
        const size_t i = (size_t)gz * Lf.nx + gx;
        const cx<T> c = sm.fine.U2[lz][lx];
        const cx<T> mu = mop9_staged<T, RW, RH>(sm.fine.C, Lf.nx, Lf.nz, gx, gz, lx, lz, &sm.fine.U2[lz][lx]);
        const cx<T> v = c + wj * cdiv(sm.fine.F[lz][lx] - mu, sm.fine.C.c[0][lz][lx]);
        stc(ob, i, acc_f ? opre + v : v);
    }
}

}  // namespace helm

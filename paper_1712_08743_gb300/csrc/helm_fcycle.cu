// helm_fcycle.cu - the F-cycle part of the multigrid preconditioner in one
// persistent kernel.
//
// From the F-cycle start level ls down to the level ld that the dense inverse
// solves, a preconditioner application is a chain of about twenty dependent
// steps on small grids (restriction, restriction of the second coarse
// correction, prolongation + smoothing, dense coarse solve). Launched one kernel per step,
// each step pays a kernel launch and completion on the critical path; here the
// whole chain runs in one cooperative launch whose blocks stay resident and
// separate the steps with a grid barrier. One block per SM holds four groups of 128
// threads each; a group works on one tile of a step at a time (the tile bodies of
// helm_gal_tiles.cuh, with named-barrier synchronisation), and all of a
// block's warps share the rows of the dense solve. Vectors written within the
// launch are read through L2. The arithmetic of every node is that of the
// one-launch-per-level kernels, so the results are the same.
#include <algorithm>
#include <functional>

#include "helm_gal_tiles.cuh"
#include "helm_internal.h"
#include "helm_solver.h"

namespace helm {

namespace {

constexpr int kFcGroups = 4;                    // tile groups of 128 threads per block, one block per SM
constexpr int kFcGroup = 128;
constexpr int kFcThreads = kFcGroups * kFcGroup;
constexpr int kFcRCX = 8;                       // restriction: 8 x 8 coarse nodes per tile (128 threads)
constexpr int kFcPX = 16;                       // prolongation: 16 x 8 fine nodes per tile (128 threads each)
constexpr unsigned kFcSpins = 2000000u;         // bounded wait of one step barrier (polls, about 1 s)

constexpr int kFcRCZ = 8, kFcPZ = 8;
constexpr int kFcRNT = kFcGroup;

template <typename T>
union FcGroupSmem {
    RestrictTile<T, kFcRCX, kFcRCZ, kFcRNT> r;
    ResidRestrictTile<T, kFcRCX, kFcRCZ, kFcRNT> q;
    ProlongTile<T, kFcPX, kFcPZ> p;
};

// Split grid barrier of the persistent launch: arrive (make this block's writes
// visible and count it in on one counter) and wait (bounded poll until every
// block has arrived for this step, then a fence before the step's loads).
// Between the two a block may do work that does not read what other blocks
// wrote in the step (here: stage the next step's Galerkin coefficients).
struct FcBarrier {
    unsigned* count;
    int* err;
    __device__ __forceinline__ void arrive() const {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(count, 1u);
        }
    }
    __device__ __forceinline__ bool wait(unsigned step) const {
        __shared__ int s_ok;
        if (threadIdx.x == 0) {
            const unsigned target = step * gridDim.x;
            int ok = 1;
            for (unsigned k = 0;; ++k) {
                if (*reinterpret_cast<const volatile unsigned*>(count) >= target) break;
                if (*reinterpret_cast<const volatile int*>(err) != 0) { ok = 0; break; }
                if (k >= kFcSpins) { atomicExch(err, 1); ok = 0; break; }
            }
            __threadfence();
            s_ok = ok;
        }
        __syncthreads();
        return s_ok != 0;
    }
};

// Stages the Galerkin coefficients of this group's first tile of step `op`
// (model data only); returns whether it did.
template <typename T>
__device__ __forceinline__ bool fc_stage_first(const FcArgs& a, FcGroupSmem<T>& sm, int op, int gid, int gtid,
                                               const RhsState* st) {
    const int type = op & 15, l = op >> 8;
    const T* hw = static_cast<const T*>(a.hw);
    if (type == FC_RESTRICT || type == FC_CORRECT_RESTRICT) {
        const LevelDev& Lc = a.lv[l + 1];
        const int tx = (Lc.nx + kFcRCX - 1) / kFcRCX, tz = (Lc.nz + kFcRCZ - 1) / kFcRCZ, per = tx * tz;
        if (gid >= per * a.nrhs) return false;
        const int b = gid / per, r = gid - b * per, by = r / tx, bx = r - by * tx;
        if (!rhs_active(st, b)) return false;
        restrict_tile_stage<T, kFcRCX, kFcRCZ, kFcRNT>(sm.r, a.lv[l], bx, by, b, hw[b], (T)a.b1, (T)a.b2, gtid);
        return true;
    }
    if (type == FC_RESID_RESTRICT) {
        const LevelDev& Lc = a.lv[l + 1];
        const int tx = (Lc.nx + kFcRCX - 1) / kFcRCX, tz = (Lc.nz + kFcRCZ - 1) / kFcRCZ, per = tx * tz;
        if (gid >= per * a.nrhs) return false;
        const int b = gid / per, r = gid - b * per, by = r / tx, bx = r - by * tx;
        if (!rhs_active(st, b)) return false;
        resid_restrict_tile_stage<T, kFcRCX, kFcRCZ, kFcRNT>(sm.q, a.lv[l], bx, by, b, hw[b], (T)a.b1, (T)a.b2,
                                                             gtid);
        return true;
    }
    if (type == FC_PROLONG) {
        const LevelDev& Lf = a.lv[l];
        const int tx = (Lf.nx + kFcPX - 1) / kFcPX, tz = (Lf.nz + kFcPZ - 1) / kFcPZ, per = tx * tz;
        if (gid >= per * a.nrhs) return false;
        const int b = gid / per, r = gid - b * per, by = r / tx, bx = r - by * tx;
        if (!rhs_active(st, b)) return false;
        prolong_tile_stage<T, kFcPX, kFcPZ>(sm.p, Lf, bx, by, b, hw[b], (T)a.b1, (T)a.b2, gtid);
        return true;
    }
    return false;
}

template <typename T>
__global__ void __launch_bounds__(kFcThreads, 1) k_fcycle(const __grid_constant__ FcArgs a, const RhsState* st) {
    extern __shared__ __align__(16) unsigned char fc_smem[];
    const int g = threadIdx.x / kFcGroup, gtid = threadIdx.x - g * kFcGroup;
    FcGroupSmem<T>& sm = reinterpret_cast<FcGroupSmem<T>*>(fc_smem)[g];
    const GroupSync gsync{1 + g, kFcGroup};
    const int gid = blockIdx.x * kFcGroups + g, ngr = gridDim.x * kFcGroups;
    const T* hw = static_cast<const T*>(a.hw);
    const T b1 = (T)a.b1, b2 = (T)a.b2, wj = (T)a.wj;
    const FcBarrier bar{a.bar, a.err};
    bool staged = fc_stage_first<T>(a, sm, a.ops[0], gid, gtid, st);
    for (int k = 0; k < a.nops; ++k) {
        const int op = a.ops[k], type = op & 15, acc = (op & FC_ACC) ? 1 : 0, l = op >> 8;
        if (type == FC_RESTRICT || type == FC_CORRECT_RESTRICT) {
            const LevelDev& Lf = a.lv[l];
            const LevelDev& Lc = a.lv[l + 1];
            const int tx = (Lc.nx + kFcRCX - 1) / kFcRCX, tz = (Lc.nz + kFcRCZ - 1) / kFcRCZ;
            const int per = tx * tz, nt = per * a.nrhs;
            const T* f = static_cast<const T*>(a.f[l]);
            const T* ec = static_cast<const T*>(a.e[l + 1]);
            T* fc = static_cast<T*>(a.f[l + 1]);
            for (int t = gid; t < nt; t += ngr) {
                const int b = t / per, r = t - b * per, by = r / tx, bx = r - by * tx;
                if (!rhs_active(st, b)) continue;
                if (!(staged && t == gid))
                    restrict_tile_stage<T, kFcRCX, kFcRCZ, kFcRNT>(sm.r, Lf, bx, by, b, hw[b], b1, b2, gtid);
                if (type == FC_CORRECT_RESTRICT)
                    restrict_tile_work<T, true, kFcRCX, kFcRCZ, kFcRNT, true>(sm.r, Lf, Lc, wj, f, ec, fc, bx, by, b,
                                                                              gtid, gsync);
                else
                    restrict_tile_work<T, false, kFcRCX, kFcRCZ, kFcRNT, true>(sm.r, Lf, Lc, wj, f, ec, fc, bx, by, b,
                                                                               gtid, gsync);
                gsync();   // the next tile's staging overwrites this tile's shared memory
            }
        } else if (type == FC_RESID_RESTRICT) {
            const LevelDev& Lf = a.lv[l];
            const LevelDev& Lc = a.lv[l + 1];
            const int tx = (Lc.nx + kFcRCX - 1) / kFcRCX, tz = (Lc.nz + kFcRCZ - 1) / kFcRCZ;
            const int per = tx * tz, nt = per * a.nrhs;
            const T* f = static_cast<const T*>(a.f[l]);
            const T* e = static_cast<const T*>(a.e[l]);
            T* gl = static_cast<T*>(a.g[l]);
            T* fc = static_cast<T*>(a.f[l + 1]);
            for (int t = gid; t < nt; t += ngr) {
                const int b = t / per, r = t - b * per, by = r / tx, bx = r - by * tx;
                if (!rhs_active(st, b)) continue;
                if (!(staged && t == gid))
                    resid_restrict_tile_stage<T, kFcRCX, kFcRCZ, kFcRNT>(sm.q, Lf, bx, by, b, hw[b], b1, b2, gtid);
                resid_restrict_tile_work<T, kFcRCX, kFcRCZ, kFcRNT, true>(sm.q, Lf, Lc, wj, f, e, gl, fc, bx, by, b,
                                                                          gtid, gsync);
                gsync();
            }
        } else if (type == FC_PROLONG) {
            const LevelDev& Lf = a.lv[l];
            const LevelDev& Lc = a.lv[l + 1];
            const int tx = (Lf.nx + kFcPX - 1) / kFcPX, tz = (Lf.nz + kFcPZ - 1) / kFcPZ;
            const int per = tx * tz, nt = per * a.nrhs;
            const T* f = static_cast<const T*>((op & FC_G) ? a.g[l] : a.f[l]);
            const T* ec = static_cast<const T*>(a.e[l + 1]);
            T* out = static_cast<T*>(a.e[l]);
            for (int t = gid; t < nt; t += ngr) {
                const int b = t / per, r = t - b * per, by = r / tx, bx = r - by * tx;
                if (!rhs_active(st, b)) continue;
                if (!(staged && t == gid)) prolong_tile_stage<T, kFcPX, kFcPZ>(sm.p, Lf, bx, by, b, hw[b], b1, b2, gtid);
                prolong_tile_work<T, kFcPX, kFcPZ, true>(sm.p, Lf, Lc, wj, f, ec, out, acc, bx, by, b, gtid, gsync);
                gsync();
            }
        } else if (type == FC_DENSE) {
            // e (+)= M_d^-1 f, one warp per row; each block stages the group's right-hand sides
            const int n = a.lv[l].nx * a.lv[l].nz;
            const T* fl = static_cast<const T*>(a.f[l]);
            T* el = static_cast<T*>(a.e[l]);
            cx<T>* fs = reinterpret_cast<cx<T>*>(fc_smem);
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            for (int gg = 0; gg < a.ngroups; ++gg) {
                const int r0 = a.grp[gg], nb = a.grp[gg + 1] - r0;
                __syncthreads();
                for (int idx = threadIdx.x; idx < nb * n; idx += blockDim.x)
                    fs[idx] = ldv<true>(fl, (size_t)r0 * n + idx);
                __syncthreads();
                const T* Mb = static_cast<const T*>(a.minv) + 2 * (size_t)a.slot[r0] * n * n;
                for (int row = blockIdx.x * (kFcThreads / 32) + warp; row < n; row += gridDim.x * (kFcThreads / 32)) {
                    T are[8], aim[8];
#pragma unroll
                    for (int r = 0; r < 8; ++r) { are[r] = T(0); aim[r] = T(0); }
                    // the row in chunks of 16 values per lane, each chunk's loads issued together
                    constexpr int CH = 16;
                    for (int j0 = 0; j0 < n; j0 += 32 * CH) {
                        cx<T> m[CH];
#pragma unroll
                        for (int q = 0; q < CH; ++q) {
                            const int j = j0 + lane + 32 * q;
                            m[q] = j < n ? ldc(Mb, (size_t)row * n + j) : cx<T>(0, 0);
                        }
#pragma unroll
                        for (int q = 0; q < CH; ++q) {
                            const int j = j0 + lane + 32 * q;
                            if (j >= n) break;
#pragma unroll
                            for (int r = 0; r < 8; ++r) {
                                if (r >= nb) break;
                                const cx<T> v = fs[(size_t)r * n + j];
                                are[r] += m[q].re * v.re - m[q].im * v.im;
                                aim[r] += m[q].re * v.im + m[q].im * v.re;
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
                        const int b = r0 + r;
                        if (lane == 0 && rhs_active(st, b)) {
                            cx<T> v(are[r], aim[r]);
                            if (acc) v = v + ldv<true>(el, (size_t)b * n + row);
                            stc(el, (size_t)b * n + row, v);
                        }
                    }
                }
            }
        }
        if (k + 1 == a.nops) break;
        // the next step reads what this one wrote anywhere on the grid: arrive, stage the next
        // step's first tile (model data only) while the other blocks finish, then wait
        bar.arrive();
        staged = fc_stage_first<T>(a, sm, a.ops[k + 1], gid, gtid, st);
        if (!bar.wait((unsigned)(k + 1))) return;
    }
}

size_t fc_smem_bytes() { return kFcGroups * sizeof(FcGroupSmem<float>); }

}  // namespace

// Schedule of one cycle at level l (F or V) down to the dense level ld, with the
// F-cycle from level lf: the order of mg_cycle's launches.
std::vector<int> fcycle_schedule(int l, int lf, int ld, bool F, int acc) {
    std::vector<int> ops;
    std::function<void(int, bool, int, bool)> cyc = [&](int q, bool f, int a, bool resid) {
        if (q == ld) { ops.push_back(FC_DENSE | (a ? FC_ACC : 0) | (q << 8)); return; }
        ops.push_back((resid ? FC_RESID_RESTRICT : FC_RESTRICT) | (q << 8));
        cyc(q + 1, f || (q + 1 == lf), 0, false);
        // second correction: none above the dense level (its right-hand side is zero there),
        // else a V-cycle whose first restriction forms its right-hand side
        if (f && q + 1 < ld) cyc(q + 1, false, 1, true);
        ops.push_back(FC_PROLONG | (a ? FC_ACC : 0) | (resid ? FC_G : 0) | (q << 8));
    };
    cyc(l, F, acc, false);
    return ops;
}

// Blocks of the cooperative launch: two per SM when they fit, else what the
// occupancy allows (0: the kernel cannot run cooperatively here).
int fcycle_grid(int dense_n, int maxg) {
    static const int per_sm = [] {
        cudaFuncSetAttribute(k_fcycle<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fc_smem_bytes());
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fcycle<float>, kFcThreads, fc_smem_bytes()) !=
            cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return nb;
    }();
    // the dense step stages the group's right-hand sides in the same shared memory
    if ((size_t)dense_n * maxg * sizeof(float2) > fc_smem_bytes()) return 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm >= 1 ? sms : 0;   // one block per SM
}

cudaError_t launch_fcycle(const FcArgs& a, int grid, const RhsState* st, cudaStream_t s) {
    ProfScope prof(PK_FCYCLE, a.lv[a.ops[0] >> 8].nx, a.lv[a.ops[0] >> 8].nz, a.bytes, s);
    cudaError_t e = cudaMemsetAsync(a.bar, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    // a cooperative launch (all blocks resident together), in a form that stream capture accepts
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kFcThreads);
    cfg.dynamicSmemBytes = fc_smem_bytes();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_fcycle<float>, a, st);
}

}  // namespace helm

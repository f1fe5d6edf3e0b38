// helm_internal.h - host-side structures and kernel launchers shared by the
// solver, the C ABI and the serving scheduler.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "helm.h"
#include "helm_common.cuh"

namespace helm {

constexpr int kCoarseMaxPoints = 128;   // coarsening stops once a level has this few nodes
constexpr int kCoarseHardMax = 256;     // largest coarsest level the dense inverse accepts
constexpr int kFcycleMaxPoints = 24576; // the F-cycle starts no later than the first level this small
constexpr double kFcycleKh = 0.7;       // ... and at the first level where k h of the shortest wavelength reaches this
// levels this small run in shared memory, one block per RHS (complex64 / complex128)
constexpr int kTailMaxPoints32 = 2048;
constexpr int kTailMaxPoints64 = 1024;
constexpr int kMaxLevels = 24;
constexpr int kMaxRestart = 32;
// tile-shape choices of the complex64 Galerkin kernels (launch_prolong_g / launch_restrict_g);
// 1 is the default shape
constexpr int kProlongTiles = 5;
constexpr int kRestrictTiles = 6;
constexpr int kGalerkinCoefs = 10;   // per coarse node: G (c, e, n, ne, nw) then K (c, e, n, ne, nw)
// the first level with at most this many nodes is solved exactly by its dense inverse
// (few right-hand sides; see helm_dense.cu)
constexpr int kDenseMaxPoints = 1200;
constexpr int kDenseAutoMaxRhs = 16;   // HELM_COARSE_AUTO takes the dense level for batches up to this size
// the cycle fuses consecutive Galerkin prolongations (launch_prolong2) for batches up to this size
constexpr int kProlong2MaxRhs = kDenseAutoMaxRhs;

// One multigrid level as the kernels see it. The finest level carries the
// squared slowness m2 and the 5-point operator; every coarser level carries
// its Galerkin operator M_l = G_l - (h_0 omega)^2 (beta1 - j beta2) K_l, with
// G_l = P^T G_{l-1} P (G_0 the 5-point Laplacian) and K_l = P^T K_{l-1} P
// (K_0 = diag(m^2)), stored as 9-point symmetric stencils: gk = [10][n] reals
// (G then K; centre, east, north, north-east, north-west coefficient of each
// node; the other four come from the neighbours by symmetry). Right-hand side
// b reads model b * mstride / n (mstride = 0: one model shared by the batch,
// n: one model per RHS), likewise gkstride. The per-RHS factor
// (h_0 omega_b)^2 is passed separately.
struct LevelDev {
    int nx, nz;
    double h2;          // (h_l / h_0)^2 on the finest level (1); unused on Galerkin levels
    const void* m2;     // finest level: float* or double* per the kernel's precision
    size_t mstride;
    const void* gk;     // Galerkin levels: float* or double* [nmodels][10][n]
    size_t gkstride;
    const void* rho;    // finest level with a density (Eq. 1): [3][n] east-edge, north-edge and diagonal
                        // coefficients of the flux-form operator; nullptr for constant density
};

struct Level {
    int nx = 0, nz = 0;
    double h = 0;
    float* m2f = nullptr;    // finest level only
    double* m2d = nullptr;
    float* gkf = nullptr;    // Galerkin levels (l >= 1), and the finest level with a density
    double* gkd = nullptr;
    float* rhof = nullptr;   // finest level with a density: [3][n] (see LevelDev::rho)
    double* rhod = nullptr;
    size_t n() const { return (size_t)nx * nz; }
};

struct Serve;  // serving scheduler (helm_serve.cu)

}  // namespace helm

struct helm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    helm::Serve* serve = nullptr;
    std::mutex serve_mu;
};

struct helm_model {
    helm_ctx* ctx = nullptr;
    int Px = 0, Pz = 0, npml = 0, nx = 0, nz = 0;
    double h = 0, alpha_max = 0;
    int nmodels = 1;                      // > 1: one slowness model per right-hand side (serving batches)
    bool vd = false;                      // variable density (Eq. 1): the finest level is a stored 9-point level
    int lf = 1;                           // first level with at most kFcycleMaxPoints nodes (latest F-cycle start)
    int ld = 0;                           // first level (>= 1) with at most kDenseMaxPoints nodes (0: none)
    double m_max = 0;                     // largest slowness of the model(s): the shortest wavelength
    // Per precision (0: complex64, 1: complex128): first level handled by the
    // shared-memory tail kernel (>= lf), its F- and V-cycle schedules on the
    // device and its dynamic shared memory.
    int lt[2] = {1, 1};
    int* ops_f[2] = {nullptr, nullptr};
    int* ops_v[2] = {nullptr, nullptr};
    int nops_f[2] = {0, 0}, nops_v[2] = {0, 0};
    size_t tail_smem[2] = {0, 0};
    // complex64 tile choices per level (0 smaller, 1 larger tiles; see the launchers),
    // set by helm_autotune / helm_set_tiles
    int tile_restrict[helm::kMaxLevels];
    int tile_prolong[helm::kMaxLevels];
    int tail_level(bool dbl) const { return lt[dbl ? 1 : 0]; }
    double* m_pad = nullptr;              // device [nmodels][nz][nx] slowness (float64)
    double msq_sum = 0;                   // sum of m^2 over the physical cells
    std::vector<helm::Level> lv;          // lv[0] is the padded fine grid
    size_t n() const { return (size_t)nx * nz; }
};

namespace helm {

// Launch with programmatic stream serialization (the kernel must call pdl_wait
// before reading anything an earlier kernel of the stream writes).
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// NVTX range over a scope (a named span on a profiler's host timeline: a solve,
// a refinement step, an iteration chunk, a multigrid level visit); free when no
// profiler is attached.
class NvtxRange {
  public:
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Per-kernel timing of this library's launches (helm_profile.cu): while a
// profiling session runs, a ProfScope records CUDA events around the launch in
// its scope, with the kernel class, the grid and the launch's algorithmic bytes.
enum ProfKernel : int {
    PK_APPLY, PK_APPLY_DOTS, PK_RESID64, PK_REFINE, PK_BICG_INIT, PK_BICG_RESUME, PK_BICG_P, PK_BICG_S, PK_BICG_XR,
    PK_RESTRICT, PK_PROLONG, PK_RESTRICT_G, PK_CORRECT_RESTRICT, PK_RESID_RESTRICT, PK_PROLONG_G, PK_PROLONG2_G, PK_TAIL, PK_COARSE_DENSE,
    PK_DENSE_INVERT, PK_COARSE_INVERT, PK_FG_NORM, PK_FG_SCALE, PK_FG_DOTS, PK_FG_AXPY, PK_FG_FINISH,
    PK_FG_BACKSOLVE, PK_FG_UPDATE, PK_FCYCLE, PK_OTHER, PK_COUNT
};
bool prof_on();
class ProfScope {
  public:
    ProfScope(int kid, int nx, int nz, double bytes, cudaStream_t s);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;

  private:
    cudaStream_t s_ = nullptr;
    int idx_ = -1;
};

// Error helpers -----------------------------------------------------------
#define HELM_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) {                              \
            helm::set_last_error(cudaGetErrorString(e_));     \
            return HELM_E_CUDA;                               \
        }                                                     \
    } while (0)

void set_last_error(const std::string& s);

inline LevelDev level_dev(const helm_model* m, int l, bool dbl) {
    const Level& L = m->lv[l];
    LevelDev d;
    d.nx = L.nx;
    d.nz = L.nz;
    d.h2 = (L.h / m->lv[0].h) * (L.h / m->lv[0].h);
    d.m2 = dbl ? (const void*)L.m2d : (const void*)L.m2f;
    d.mstride = m->nmodels > 1 ? L.n() : 0;
    d.gk = dbl ? (const void*)L.gkd : (const void*)L.gkf;
    d.gkstride = m->nmodels > 1 ? kGalerkinCoefs * L.n() : 0;
    d.rho = dbl ? (const void*)L.rhod : (const void*)L.rhof;
    return d;
}

// Tail schedule entries: op type in the low byte, level above it. LOAD and
// RESTRICT also take the zero-guess smoothing step of the level they fill (when
// it is not the coarsest); POST is the residual and Jacobi step after a coarse
// correction, written to r, which holds a level's result (as does COARSE).
enum TailOp : int { OP_RESID = 1, OP_RESTRICT = 2, OP_PROLONG_ADD = 3, OP_POST = 4, OP_COARSE = 5, OP_OUTPUT = 6,
                    OP_LOAD = 7 };
std::vector<int> tail_schedule(int lt, int L, bool fcycle);
size_t tail_smem_bytes(const helm_model* m, int lt, size_t elem, bool* minv_smem = nullptr, int* minv_off = nullptr);

// Arguments of the tail kernel: levels lt..L of the cycle for one RHS per
// block, every vector of those levels in shared memory.
struct TailArgs {
    int lt, L;
    LevelDev lv[kMaxLevels];
    const void* in;           // right-hand side on level lt, [nrhs][n_lt]
    void* out;                // correction on level lt, [nrhs][n_lt]
    int accumulate;           // 1: out += correction
    const void* minv;         // dense coarsest inverses [nslots][nL][nL]
    const int* slot;
    const int* ops;
    int nops;
    int minv_smem;            // 1: the coarsest inverse is staged in shared memory at minv_off
    int minv_off;
    int off[kMaxLevels];      // level l's arrays in shared memory (complex elements), l = lt..L
    const double* w2;         // (h_0 omega_b)^2
    double b1, b2, wj;
};

// Kernel launchers (helm_kernels.cu). All run on `s`; none synchronises.
// `st` may be null where noted; vectors are [nrhs][level n] interleaved complex.
void launch_pad_model(const double* m_phys, int Px, int Pz, int npml, int nmodels, double* m_pad, float* m2f,
                      double* m2d, cudaStream_t s);
void launch_galerkin(const helm_model* m, int l, cudaStream_t s);   // builds level l >= 1 from level l - 1
void launch_rho_setup(const double* rho_phys, int Px, int Pz, int npml, const double* m2d, double* rhod, float* rhof,
                      double* gkd, float* gkf, cudaStream_t s);
void launch_sumsq(const double* a, size_t count, double* out, cudaStream_t s);

// hw: per-RHS (h omega)^2 in the kernel's precision
template <typename T>
void launch_apply(const LevelDev& L0, int npml, double amax, const T* hw, const T* u, T* y,
                  T scale, int nrhs, cudaStream_t s);
// y = A u with the unpreconditioned BiCGSTAB dot products (mode 1: alpha, mode 2: omega)
template <typename T>
void launch_apply_dots(int mode, const LevelDev& L0, int npml, double amax, const T* hw, const T* u, T* y,
                       const T* aux, double* partials, int pstride, RhsState* st, int nrhs, cudaStream_t s);

// Outer FP64 residual r = f - A u; TI = precision of the inner right-hand side.
template <typename TI>
void launch_resid64(const LevelDev& L0, int npml, double amax, const double* w2, const double* f,
                    const double* u, TI* rin, double* partials, int pstride, RhsState* st,
                    double tol, double inner_floor, double inner_fac, int first, int nrhs, cudaStream_t s);
template <typename TI>
void launch_refine(const TI* x, double* u, const RhsState* st, size_t n, int nrhs, cudaStream_t s);

template <typename T>
void launch_bicg_init(const T* b, T* x, T* r, T* rh, T* p, T* v, double* partials, int pstride,
                      RhsState* st, int* nactive, size_t n, int nrhs, cudaStream_t s);
template <typename T>
void launch_bicg_resume(const T* rin, T* x, T* r, T* rh, T* p, T* v, double* partials, int pstride,
                        RhsState* st, int* nactive, size_t n, int nrhs, cudaStream_t s);
template <typename T>
void launch_bicg_p(const T* r, T* p, const T* v, const RhsState* st, size_t n, int nrhs, cudaStream_t s);
template <typename T>
void launch_bicg_s(const T* r, const T* v, T* sv, const RhsState* st, size_t n, int nrhs, cudaStream_t s);
template <typename T>
void launch_bicg_xr(T* x, const T* ph, const T* sh, const T* sv, const T* t, const T* rh, T* r,
                    double* partials, int pstride, RhsState* st, int* nactive, size_t n, int nrhs,
                    cudaStream_t s);

// V-cycle pieces. restrict / prolong on the finest level use the 5-point
// operator; on Galerkin levels (1 <= l < lt) the 9-point one.
template <typename T>
void launch_tail(const TailArgs& a, size_t smem, int nrhs, const RhsState* st, cudaStream_t s);
// F-cycle step on a grid level: u2 = wj D^-1 f + P e (e the first coarse
// correction), residual f - M u2, restricted to level l + 1.
template <typename T>
void launch_correct_restrict(const LevelDev& Lf, const LevelDev& Lc, const T* w2, double b1, double b2,
                             double wj, const T* f, const T* ec, T* fc, const RhsState* st, int nrhs, cudaStream_t s,
                             int tile = 1);
template <typename T>
void launch_restrict(const LevelDev& Lf, const LevelDev& Lc, const T* w2, double b1, double b2,
                     double wj, const T* f, T* fc, const RhsState* st, int nrhs, cudaStream_t s, int tile = 1);
// The prolongation of Galerkin level l + 1 (from e of level l + 2; right-hand side
// fm, added to em when acc_m) and then that of level l (right-hand side fl, into
// out, added to it when acc_f), in one launch; level l + 1's correction stays in
// shared memory. tile: level l's prolongation tile code (0: 16 x 8, else 32 x 8).
template <typename T>
void launch_prolong2(const LevelDev& Lf, const LevelDev& Lm, const LevelDev& Lc, const T* w2, double b1, double b2,
                     double wj, const T* fl, const T* fm, const T* ec, const T* em, T* out, const RhsState* st,
                     int nrhs, cudaStream_t s, int acc_f, int acc_m, int tile);
// The restriction that starts the second coarse correction of an F-cycle, on a
// Galerkin level: g = f - M e (f this level's first right-hand side, e its first
// correction) written to g, then restricted like launch_restrict does to fc.
template <typename T>
void launch_resid_restrict(const LevelDev& Lf, const LevelDev& Lc, const T* w2, double b1, double b2, double wj,
                           const T* f, const T* e, T* g, T* fc, const RhsState* st, int nrhs, cudaStream_t s,
                           int tile);
// mode 0: out = smoothed correction; 1: out = p^, y = A p^, alpha = rho/<rh, y>;
// 2: out = s^, y = A s^, omega = <y, s>/<y, y>; 3: out = z, y = A z (no dots).
template <typename T>
void launch_prolong(int mode, const LevelDev& Lf, const LevelDev& Lc, int npml, double amax,
                    const T* w2, double b1, double b2, double wj, const T* f, const T* ec, T* out,
                    T* y, const T* aux, double* partials, int pstride, RhsState* st, int nrhs,
                    cudaStream_t s, int accumulate = 0, int tile = 1);
template <typename T>
void launch_coarse(int n, const T* minv, const int* slot, const T* fL, T* eL, const RhsState* st,
                   int nrhs, cudaStream_t s);
// Dense exact solve of one coarse level (helm_dense.cu). dense_invert_plan
// returns 1 and the strip width / slots per cooperative launch when an n-node
// level can be inverted, 0 otherwise.
int dense_invert_plan(int n, bool dbl, int* W, int* per_launch_slots);
template <typename T>
cudaError_t launch_dense_invert(const LevelDev& Ld, const double* w2s, const int* mods, int nslots, double b1,
                                double b2, int W, int per_launch, T* minv, T* panel, T* dinv, unsigned* bar,
                                int* err, cudaStream_t s);
// e (+)= M_d^-1 f per right-hand side; grp: [ngroups + 1] boundaries of groups of
// at most maxg (<= 8) consecutive right-hand sides sharing a slot.
template <typename T>
void launch_coarse_dense(int n, const T* minv, const int* slot, const int* grp, int ngroups, int maxg, const T* f,
                         T* e, int accumulate, const RhsState* st, cudaStream_t s);
void launch_coarse_invert(const LevelDev& Lc, const double* w2_slots, const int* mod_slots, int nslots,
                          double b1, double b2, double2* work, float2* minv_f, double2* minv_d, cudaStream_t s);

// Persistent F-cycle (helm_fcycle.cu): the steps of one cycle from level ls down
// to the dense level, in one cooperative launch. Step: type | FC_ACC (add to the
// output) | level << 8.
constexpr int kFcMaxOps = 96;
constexpr int kFcMaxRhs = 8;      // right-hand sides a batch may have for the persistent path
enum FcOpType : int {
    FC_RESTRICT = 1, FC_CORRECT_RESTRICT = 2, FC_PROLONG = 3, FC_DENSE = 4, FC_RESID_RESTRICT = 5,
    FC_ACC = 16, FC_G = 32   // FC_G: the step's right-hand side on its level is g (second correction)
};
struct FcArgs {
    int nops, nrhs;
    int ops[kFcMaxOps];
    LevelDev lv[kMaxLevels];
    void* f[kMaxLevels];      // per level: right-hand side and correction [nrhs][n_l] (complex64)
    void* e[kMaxLevels];
    void* g[kMaxLevels];      // right-hand side of an F-cycle's second coarse correction
    const void* hw;           // (h_0 omega_b)^2 per RHS, FP32
    double b1, b2, wj;
    const void* minv;         // dense inverses of level ld, [nslots][n][n]
    const int* slot;
    const int* grp;           // groups of consecutive right-hand sides sharing a slot
    int ngroups, maxg;
    unsigned* bar;            // step barrier counter (cleared before each launch)
    int* err;                 // set to 1 when a barrier wait gave up
    double bytes;             // algorithmic bytes of one launch (profiling)
};
std::vector<int> fcycle_schedule(int l, int lf, int ld, bool F, int acc);
int fcycle_grid(int dense_n, int maxg);
cudaError_t launch_fcycle(const FcArgs& a, int grid, const RhsState* st, cudaStream_t s);

// FGMRES state on the device, per RHS: Hessenberg H [(m+1) x m], rotated
// right-hand side g [m+1], Givens cosines cs / sines sn [m], solution y [m],
// projection coefficients tmp [m+1], the inverse norms sinv [m+1] of the
// unnormalised basis vectors, and ||w||^2 before Gram-Schmidt wn2 [1].
struct FgDev {
    int m;
    double2* H;
    double2* g;
    double* cs;
    double2* sn;
    double2* y;
    double2* tmp;
    double* sinv;
    double* wn2;
};
template <typename T>
void launch_fg_norm(const T* rin, double* partials, int pstride, RhsState* st, const FgDev& fg, int* nactive,
                    size_t n, int nrhs, cudaStream_t s);
template <typename T>
void launch_fg_scale(const T* rin, T* v, const RhsState* st, const FgDev& fg, size_t n, int nrhs, cudaStream_t s);
template <typename T>
void launch_fg_dots(const T* V, size_t vstride, const T* w, int j, int add, int wnorm, int check, double* partials,
                    int pstride, RhsState* st, const FgDev& fg, size_t n, int nrhs, cudaStream_t s);
// returns the blocks per RHS it launched (the parts of ||w||^2 in mode 3)
template <typename T>
int launch_fg_axpy(const T* V, size_t vstride, T* w, int j, int mode, int check, double* partials, int pstride,
                   RhsState* st, const FgDev& fg, int* nactive, size_t n, int nrhs, cudaStream_t s);
void launch_fg_finish(const double* partials, int pstride, int nblk, RhsState* st, const FgDev& fg, int j,
                      int* nactive, int nrhs, cudaStream_t s);
void launch_fg_backsolve(const RhsState* st, const FgDev& fg, int nrhs, cudaStream_t s);
int fg_partials(size_t n);   // reduction partials per RHS the FGMRES kernels need on n points
constexpr int kFgTimedStep = 4;   // Arnoldi step that helm_time_kernel times (the middle of FGMRES(10))
template <typename T>
void launch_fg_update(const T* Z, size_t zstride, T* x, const RhsState* st, const FgDev& fg, size_t n, int nrhs,
                      cudaStream_t s);

// FP64 throughput probe: blocks x 256 threads x 8 chains x iters fused multiply-adds
void launch_fma64(double* out, int blocks, int iters, cudaStream_t s);

// right-hand sides and gradient
void launch_point_rhs(double* f, const int* src_flat, int nrhs, size_t n, cudaStream_t s);
void launch_scale_rhs(const double* fin, double* f, double scale, size_t count, cudaStream_t s);
template <typename T>
void launch_cast_complex(const double* in, T* out, size_t count, cudaStream_t s);
template <typename T>
void launch_to_c128(const T* in, double* out, size_t count, cudaStream_t s);
void launch_sample(const double* u, const int* rec_flat, int nrec, const double* d_obs, double* d_cal,
                   double* resid, double* jpart, size_t n, int nrhs, cudaStream_t s);
void launch_adjoint_rhs(const double* resid, const int* rec_flat, int nrec, double h2, double* f,
                        size_t n, int nrhs, cudaStream_t s);
void launch_grad_accum(const double* u, const double* w, const double* w2, const double* m_pad,
                       int nx, int nz, int npml, double amax, double* g_pad, int nrhs, cudaStream_t s);
void launch_fold(const double* g_pad, const double* m_pad, int Px, int Pz, int npml, double lam, double* g,
                 cudaStream_t s, const double* reg = nullptr);   // reg: physical vector of the 2 lam term (null: m)
void launch_expand(const double* dm, int Px, int Pz, int npml, double* dm_pad, cudaStream_t s);
void launch_born_rhs(const double* u, const double* dm_pad, const double* m_pad, const double* hw2, int nx, int nz,
                     int npml, double amax, double* f, int nrhs, cudaStream_t s);
int dot_blocks(size_t n);
void launch_dot_partials(const double* a, const double* b, size_t n, double* part, cudaStream_t s);
void launch_axpby(double alpha, const double* x, double beta, double* y, size_t n, cudaStream_t s);

}  // namespace helm

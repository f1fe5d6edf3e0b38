// helm_solver.cu - host side of the batched solver: multigrid hierarchy,
// right-preconditioned BiCGSTAB in complex64 or complex128, FP64 residual and
// iterative refinement, and the adjoint-state gradient.
//
// Every step of the computation runs in the kernels of helm_kernels.cu; this
// file only sizes buffers, orders launches on one stream and reads back the
// per-right-hand-side convergence state every `check_every` iterations.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <vector>

#include "helm_internal.h"
#include "helm_solver.h"

namespace helm {

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
unsigned long long launches() { return g_launches.load(std::memory_order_relaxed); }
void set_last_error(const std::string& s) { g_last_error = s; }
const char* last_error() { return g_last_error.c_str(); }

namespace {

// Stream-ordered device allocation freed on scope exit.
struct DBuf {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    ~DBuf() { if (p) cudaFreeAsync(p, s); }
    cudaError_t alloc(size_t bytes, cudaStream_t st) {
        s = st;
        return cudaMallocAsync(&p, bytes ? bytes : 16, st);
    }
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

#define TRY_ALLOC(buf, bytes, st)                                                        \
    do {                                                                                 \
        cudaError_t e_ = (buf).alloc((bytes), (st));                                     \
        if (e_ != cudaSuccess) {                                                         \
            cudaGetLastError();                                                          \
            set_last_error(std::string("device allocation failed: ") + cudaGetErrorString(e_)); \
            return HELM_E_NOMEM;                                                         \
        }                                                                                \
    } while (0)

int max_blocks_per_rhs(const helm_model* m) {
    const Level& L0 = m->lv[0];
    size_t g1 = std::min<size_t>(2048, (L0.n() + 1023) / 1024);
    size_t g2 = (size_t)((L0.nx + 31) / 32) * ((L0.nz + 7) / 8);   // resid64 / apply tiles
    // marching prolongation: 4 warps of 60 columns per block, row segments of at least 4
    size_t g3 = (size_t)((L0.nx + 60 * 4 - 1) / (60 * 4)) * ((L0.nz + 3) / 4);
    return (int)std::max<size_t>(std::max(g1, g2), std::max<size_t>(g3, 1));
}

}  // namespace

int coarsest_points(const helm_model* m) { return (int)m->lv.back().n(); }

// --------------------------------------------------------------- workspace
template <typename T>
struct Inner {
    DBuf x, r, rh, p, v, sv, t, ph, shv;
    // per level 1 <= l <= lt: right-hand side and correction (deeper levels live
    // in the tail kernel's shared memory), and on levels 2 <= l < lt the right-hand
    // side of an F-cycle's second coarse correction
    std::vector<std::unique_ptr<DBuf>> fl, el, gl;
};

// Per-solve state shared by the outer and inner loops.
struct SolveCtx {
    const helm_model* m;
    cudaStream_t s;
    int nrhs;
    helm_solve_opts o;
    const double* w2;       // device [nrhs]
    const float* w2f;       // device [nrhs], FP32 copy
    RhsState* st;           // device [nrhs]
    double* partials;       // device [nrhs * pstride]
    int pstride;
    int* nactive;           // device
    const int* slot;        // device [nrhs]
    int ncoarse;
    const void* minv;       // float2* or double2* [nslots][n][n]
    int lf;                 // first level of the F-cycle for this batch
    int ld = 0;             // > 0: level solved exactly by its dense inverse (minv); 0: the tail path
    const int* grp = nullptr;
    int ngroups = 0, maxg = 0;
    const FcArgs* fca = nullptr;    // persistent F-cycle kernel (complex64, few right-hand sides)
    int fca_level = 0, fca_grid = 0;
    cudaStream_t side = nullptr;    // FGMRES: the Hessenberg column finish runs here
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

// The second stream and events of an FGMRES solve.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    ~SideStream() {
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (s) cudaStreamDestroy(s);
    }
};

template <typename T>
static const T* hw_of(const MgCall& c) {
    return static_cast<const T*>(sizeof(T) == 8 ? (const void*)c.w2 : (const void*)c.w2f);
}

// Arguments of one tail launch (an F- or V-cycle over levels lt..L) from the
// level-lt right-hand side `in` into `out`.
template <typename T>
static TailArgs tail_args(const helm_model* m, bool F, const void* in, void* out, int acc, const void* minv,
                          const int* slot, const double* w2, double b1, double b2, double wj) {
    const bool dbl = sizeof(T) == 8;
    TailArgs a;
    std::memset(&a, 0, sizeof(a));
    a.lt = m->tail_level(dbl);
    a.L = (int)m->lv.size() - 1;
    for (int q = 0; q <= a.L; ++q) a.lv[q] = level_dev(m, q, dbl);
    a.in = in;
    a.out = out;
    a.accumulate = acc;
    a.minv = minv;
    a.slot = slot;
    a.ops = F ? m->ops_f[dbl] : m->ops_v[dbl];
    a.nops = F ? m->nops_f[dbl] : m->nops_v[dbl];
    bool ms = false;
    tail_smem_bytes(m, a.lt, sizeof(T), &ms, &a.minv_off);
    a.minv_smem = ms ? 1 : 0;
    for (int q = a.lt, o = 0; q <= a.L; ++q) { a.off[q] = o; o += 8 * (int)m->lv[q].n(); }
    a.w2 = w2;
    a.b1 = b1;
    a.b2 = b2;
    a.wj = wj;
    return a;
}

static const char* const kLevelNames[kMaxLevels] = {
    "mg level 0", "mg level 1", "mg level 2", "mg level 3", "mg level 4", "mg level 5", "mg level 6", "mg level 7",
    "mg level 8", "mg level 9", "mg level 10", "mg level 11", "mg level 12", "mg level 13", "mg level 14",
    "mg level 15", "mg level 16", "mg level 17", "mg level 18", "mg level 19", "mg level 20", "mg level 21",
    "mg level 22", "mg level 23"};

// Whether the cycle of level l runs on the grid-level kernels (not the dense
// inverse, not the shared-memory tail).
static bool grid_level(const helm_model* m, const MgCall& c, int l, bool dbl) {
    return c.ld > 0 ? l < c.ld : l < m->tail_level(dbl);
}

// The prolongation that ends a cycle at level l, left to the caller (the cycle one
// level up), which runs it together with its own in one launch (launch_prolong2).
template <typename T>
struct PendingProlong {
    bool on = false;
    const T* f = nullptr;   // the level's right-hand side
    int acc = 0;            // added to the level's previous correction
};

// One cycle at level l (F or V) from the right-hand side B.f[l] into B.e[l] (added
// to it when acc). resid: the right-hand side is B.f[l] - M_l B.e[l] instead (the
// second coarse correction of the F-cycle one level up, always a V-cycle that
// accumulates), formed by the first restriction and kept in B.g[l]. may_defer: the
// caller fuses this cycle's last prolongation with its own; it is then returned,
// not launched. A cycle fuses its last recursion's pending prolongation with its
// own; the first recursion of an F-cycle never defers (its correction is read by
// the restriction that follows).
template <typename T>
static PendingProlong<T> mg_cycle(const helm_model* m, const MgCall& c, const MgLevels<T>& B, int l, bool F, int acc,
                                  bool resid, bool may_defer) {
    NvtxRange nv(kLevelNames[l]);
    const bool dbl = sizeof(T) == 8;
    const T* hw = hw_of<T>(c);
    if (c.fca && l == c.fca_level) {   // the whole cycle from here down in one persistent launch
        launch_fcycle(*c.fca, c.fca_grid, c.st, c.s);
        return {};
    }
    if (c.ld > 0 && l == c.ld) {   // exact solve of this level by its dense inverse
        launch_coarse_dense<T>((int)m->lv[l].n(), static_cast<const T*>(c.minv), c.slot, c.grp, c.ngroups, c.maxg,
                               B.f[l], B.e[l], acc, c.st, c.s);
        return {};
    }
    const int lt = m->tail_level(dbl);
    if (c.ld <= 0 && l >= lt) {
        const TailArgs a = tail_args<T>(m, F, B.f[l], B.e[l], acc, c.minv, c.slot, c.w2, c.b1, c.b2, c.wj);
        launch_tail<T>(a, m->tail_smem[dbl], c.nrhs, c.st, c.s);
        return {};
    }
    const LevelDev Lf = level_dev(m, l, dbl), Lc = level_dev(m, l + 1, dbl);
    if (resid)
        launch_resid_restrict<T>(Lf, Lc, hw, c.b1, c.b2, c.wj, B.f[l], B.e[l], B.g[l], B.f[l + 1], c.st, c.nrhs, c.s,
                                 m->tile_restrict[l]);
    else
        launch_restrict<T>(Lf, Lc, hw, c.b1, c.b2, c.wj, B.f[l], B.f[l + 1], c.st, c.nrhs, c.s, m->tile_restrict[l]);
    // prolongation pairs for small batches only: there the launches are latency chains; with
    // many right-hand sides the recomputed level l + 1 footprint costs more than it saves
    const bool pair = c.nrhs <= kProlong2MaxRhs;
    PendingProlong<T> pend;
    if (F) {
        mg_cycle<T>(m, c, B, l + 1, true, 0, false, false);
        // second coarse correction, for P^T (f - M (wj D^-1 f + P e)) = f_{l+1} - M_{l+1} e_{l+1}
        // (Galerkin M_{l+1} = P^T M P): zero when level l + 1 was solved exactly by its dense
        // inverse, so nothing is done then; on a grid level it is formed there, by the first
        // restriction of the correction's V-cycle
        if (grid_level(m, c, l + 1, dbl)) {
            pend = mg_cycle<T>(m, c, B, l + 1, false, 1, true, pair);
        } else if (c.ld <= 0) {
            launch_correct_restrict<T>(Lf, Lc, hw, c.b1, c.b2, c.wj, B.f[l], B.e[l + 1], B.f[l + 1], c.st, c.nrhs,
                                       c.s, m->tile_restrict[l]);
            pend = mg_cycle<T>(m, c, B, l + 1, false, 1, false, pair);
        }
    } else {
        pend = mg_cycle<T>(m, c, B, l + 1, l + 1 == c.lf, 0, false, pair);
    }
    const T* fl = resid ? B.g[l] : B.f[l];
    if (pend.on) {   // level l + 1's prolongation and this level's in one launch
        const LevelDev Lk = level_dev(m, l + 2, dbl);
        launch_prolong2<T>(Lf, Lc, Lk, hw, c.b1, c.b2, c.wj, fl, pend.f, B.e[l + 2], B.e[l + 1], B.e[l], c.st,
                           c.nrhs, c.s, acc, pend.acc, m->tile_prolong[l]);
        return {};
    }
    if (may_defer) {
        PendingProlong<T> mine;
        mine.on = true;
        mine.f = fl;
        mine.acc = acc;
        return mine;
    }
    launch_prolong<T>(0, Lf, Lc, m->npml, m->alpha_max, hw, c.b1, c.b2, c.wj, fl, B.e[l + 1], B.e[l], nullptr,
                      nullptr, nullptr, 0, c.st, c.nrhs, c.s, acc, m->tile_prolong[l]);
    return {};
}

template <typename T>
void mg_apply(const helm_model* m, const MgCall& c, const MgLevels<T>& B, const T* in, T* out, int mode, T* y,
              const T* aux) {
    const bool dbl = sizeof(T) == 8;
    const T* hw = hw_of<T>(c);
    const LevelDev L0 = level_dev(m, 0, dbl), L1 = level_dev(m, 1, dbl);
    launch_restrict<T>(L0, L1, hw, c.b1, c.b2, c.wj, in, B.f[1], c.st, c.nrhs, c.s);
    mg_cycle<T>(m, c, B, 1, c.lf == 1, 0, false, false);
    if (m->vd && mode != 0) {
        // variable density: the stored-level prolongation, then y = A out (with the
        // dots of modes 1 and 2) in a separate kernel
        launch_prolong<T>(0, L0, L1, m->npml, m->alpha_max, hw, c.b1, c.b2, c.wj, in, B.e[1], out, nullptr, nullptr,
                          c.partials, c.pstride, c.st, c.nrhs, c.s, 0, m->tile_prolong[0]);
        if (mode == 3)
            launch_apply<T>(L0, m->npml, m->alpha_max, hw, out, y, T(1), c.nrhs, c.s);
        else   // mode 2 dots A out with the cycle's input, as the fused kernel does
            launch_apply_dots<T>(mode, L0, m->npml, m->alpha_max, hw, out, y, mode == 2 ? in : aux, c.partials,
                                 c.pstride, c.st, c.nrhs, c.s);
        return;
    }
    launch_prolong<T>(mode, L0, L1, m->npml, m->alpha_max, hw, c.b1, c.b2, c.wj, in, B.e[1], out, y, aux,
                      c.partials, c.pstride, c.st, c.nrhs, c.s, 0, m->tile_prolong[0]);
}
template void mg_apply<float>(const helm_model*, const MgCall&, const MgLevels<float>&, const float*, float*, int,
                              float*, const float*);
template void mg_apply<double>(const helm_model*, const MgCall&, const MgLevels<double>&, const double*, double*, int,
                               double*, const double*);

// Launches of mg_cycle at level l; *pend: its last prolongation is left to the caller.
static int count_cycle(const helm_model* m, int lt, int l, bool F, int lf, int ld, int fl, bool may_defer,
                       bool pair, bool* pend) {
    *pend = false;
    if (fl > 0 && l == fl) return 1;
    if (ld > 0 ? l == ld : l >= lt) return 1;
    int k = 1;
    bool cp = false;
    if (F) {
        k += count_cycle(m, lt, l + 1, true, lf, ld, fl, false, pair, &cp);
        const bool grid = ld > 0 ? l + 1 < ld : l + 1 < lt;
        if (grid) k += count_cycle(m, lt, l + 1, false, lf, ld, fl, pair, pair, &cp);
        else if (ld <= 0) k += 1 + count_cycle(m, lt, l + 1, false, lf, ld, fl, pair, pair, &cp);
        else cp = false;
    } else {
        k += count_cycle(m, lt, l + 1, l + 1 == lf, lf, ld, fl, pair, pair, &cp);
    }
    if (cp) return k + 1;
    if (may_defer) { *pend = true; return k; }
    return k + 1;
}
int mg_kernels_per_apply(const helm_model* m, bool dbl, int lf, int ld, int fl, int nrhs) {
    bool pend = false;
    return 2 + (m->vd ? 1 : 0) +
           count_cycle(m, m->tail_level(dbl), 1, lf == 1, lf, ld, fl, false, nrhs <= kProlong2MaxRhs, &pend);
}

int fcycle_setup(const helm_model* m, const MgCall& c, int coarse, float* const* f, float* const* e,
                 float* const* g, unsigned* bar, int* err, FcArgs* fa) {
    if (coarse != HELM_COARSE_FUSED || c.ld <= 0 || c.nrhs > kFcMaxRhs || c.lf >= c.ld || !bar || !err) return 0;
    const int nd = (int)m->lv[c.ld].n();
    const int grid = fcycle_grid(nd, c.maxg);
    if (grid <= 0) return 0;
    const std::vector<int> ops = fcycle_schedule(c.lf, c.lf, c.ld, true, 0);
    if ((int)ops.size() > kFcMaxOps) return 0;
    std::memset(fa, 0, sizeof(*fa));
    fa->nops = (int)ops.size();
    fa->nrhs = c.nrhs;
    double bytes = 0;
    for (size_t k = 0; k < ops.size(); ++k) {
        fa->ops[k] = ops[k];
        const int type = ops[k] & 15, l = ops[k] >> 8, acc = (ops[k] & FC_ACC) ? 1 : 0;
        const double n = (double)m->lv[l].n(), nc = l + 1 < (int)m->lv.size() ? (double)m->lv[l + 1].n() : 0.0;
        const double coef = n * sizeof(float) * kGalerkinCoefs * (m->nmodels > 1 ? c.nrhs : 1);
        if (type == FC_RESTRICT) bytes += (n + nc) * 8.0 * c.nrhs + coef;
        else if (type == FC_RESID_RESTRICT) bytes += (3 * n + nc) * 8.0 * c.nrhs + coef;
        else if (type == FC_CORRECT_RESTRICT) bytes += (n + 2 * nc) * 8.0 * c.nrhs + coef;
        else if (type == FC_PROLONG) bytes += (n * (2 + acc) + nc) * 8.0 * c.nrhs + coef;
        else bytes += n * n * 8.0 * c.ngroups + n * (2 + acc) * 8.0 * c.nrhs;
    }
    for (int l = 0; l < (int)m->lv.size(); ++l) fa->lv[l] = level_dev(m, l, false);
    for (int l = 1; l <= c.ld; ++l) { fa->f[l] = f[l]; fa->e[l] = e[l]; fa->g[l] = g[l]; }
    fa->hw = c.w2f;
    fa->b1 = c.b1;
    fa->b2 = c.b2;
    fa->wj = c.wj;
    fa->minv = c.minv;
    fa->slot = c.slot;
    fa->grp = c.grp;
    fa->ngroups = c.ngroups;
    fa->maxg = c.maxg;
    fa->bar = bar;
    fa->err = err;
    fa->bytes = bytes;
    return grid;
}

int fcycle_level(const helm_model* m, const double* h_w2, int nrhs) {
    double w = INFINITY;
    for (int b = 0; b < nrhs; ++b) w = std::min(w, h_w2[b]);
    const double hw = std::sqrt(std::max(w, 0.0));   // h omega_min on the finest level
    for (int l = 1; l < m->lf; ++l)
        if (hw * std::ldexp(1.0, l) * m->m_max >= kFcycleKh) return l;
    return m->lf;
}

static MgCall mgcall_of(const SolveCtx& c) {
    MgCall mc;
    mc.w2 = c.w2;
    mc.w2f = c.w2f;
    mc.b1 = c.o.beta1;
    mc.b2 = c.o.beta2;
    mc.wj = c.o.omega_jacobi;
    mc.st = c.st;
    mc.nrhs = c.nrhs;
    mc.lf = c.lf;
    mc.s = c.s;
    mc.minv = c.minv;
    mc.slot = c.slot;
    mc.partials = c.partials;
    mc.pstride = c.pstride;
    mc.ld = c.ld;
    mc.grp = c.grp;
    mc.ngroups = c.ngroups;
    mc.maxg = c.maxg;
    mc.fca = c.fca;
    mc.fca_level = c.fca_level;
    mc.fca_grid = c.fca_grid;
    return mc;
}

template <typename T>
static void vcycle(const SolveCtx& c, Inner<T>& w, const T* in, T* out, int mode, T* y, const T* aux) {
    MgCall mc = mgcall_of(c);
    MgLevels<T> B;
    std::memset(&B, 0, sizeof(B));
    const int top = c.ld > 0 ? c.ld : c.m->tail_level(sizeof(T) == 8);
    for (int l = 1; l <= top; ++l) {
        B.f[l] = w.fl[l]->template as<T>();
        B.e[l] = w.el[l]->template as<T>();
        B.g[l] = w.gl[l] ? w.gl[l]->template as<T>() : nullptr;
    }
    mg_apply<T>(c.m, mc, B, in, out, mode, y, aux);
}

// The persistent F-cycle of a complex64 batch, when it applies (see fcycle_setup):
// fills fa, its barrier counter and error flag, and points c at it.
template <typename T>
static int setup_fcycle(SolveCtx& c, Inner<T>& w, int coarse, DBuf& bar, DBuf& err, FcArgs* fa) {
    c.fca = nullptr;
    if constexpr (sizeof(T) == 4) {
        if (coarse != HELM_COARSE_FUSED || c.ld <= 0) return HELM_OK;
        if (!bar.p) {
            TRY_ALLOC(bar, sizeof(unsigned), c.s);
            TRY_ALLOC(err, sizeof(int), c.s);
            HELM_CUDA_TRY(cudaMemsetAsync(err.p, 0, sizeof(int), c.s));
        }
        float* f[kMaxLevels] = {};
        float* e[kMaxLevels] = {};
        float* g[kMaxLevels] = {};
        for (int l = 1; l <= c.ld; ++l) {
            f[l] = w.fl[l]->template as<float>();
            e[l] = w.el[l]->template as<float>();
            g[l] = w.gl[l] ? w.gl[l]->template as<float>() : nullptr;
        }
        const int grid = fcycle_setup(c.m, mgcall_of(c), coarse, f, e, g, bar.as<unsigned>(), err.as<int>(), fa);
        if (grid > 0) {
            c.fca = fa;
            c.fca_level = c.lf;
            c.fca_grid = grid;
        }
    }
    return HELM_OK;
}

// After a solve that used the persistent F-cycle: HELM_E_CUDA if one of its barrier waits gave up.
static int check_fcycle(const SolveCtx& c, const DBuf& err) {
    if (!c.fca || !err.p) return HELM_OK;
    int h = 0;
    HELM_CUDA_TRY(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, c.s));
    HELM_CUDA_TRY(cudaStreamSynchronize(c.s));
    if (h != 0) {
        set_last_error("persistent multigrid cycle: a grid barrier wait gave up");
        return HELM_E_CUDA;
    }
    return HELM_OK;
}

// level vectors of levels 1..top (top: the dense level, or the tail's first level)
template <typename T>
static int alloc_levels(const helm_model* m, cudaStream_t s, int nrhs, Inner<T>& w, int top) {
    const int nl = (int)m->lv.size();
    w.fl.resize(nl);
    w.el.resize(nl);
    w.gl.resize(nl);
    for (int l = 1; l < nl && l <= top; ++l) {
        const size_t b = sizeof(T) * 2 * m->lv[l].n() * nrhs;
        w.fl[l].reset(new DBuf());
        w.el[l].reset(new DBuf());
        TRY_ALLOC(*w.fl[l], b, s);
        TRY_ALLOC(*w.el[l], b, s);
        if (l >= 2 && l < top) {
            w.gl[l].reset(new DBuf());
            TRY_ALLOC(*w.gl[l], b, s);
        }
    }
    return HELM_OK;
}

template <typename T>
static int alloc_inner(const SolveCtx& c, Inner<T>& w) {
    const size_t n = c.m->n(), vb = sizeof(T) * 2 * n * c.nrhs;
    TRY_ALLOC(w.x, vb, c.s);
    if (c.o.krylov == HELM_KRYLOV_BICGSTAB) {      // FGMRES keeps its vectors in FgBufs
        TRY_ALLOC(w.r, vb, c.s); TRY_ALLOC(w.rh, vb, c.s);
        TRY_ALLOC(w.p, vb, c.s); TRY_ALLOC(w.v, vb, c.s); TRY_ALLOC(w.sv, vb, c.s);
        TRY_ALLOC(w.t, vb, c.s); TRY_ALLOC(w.ph, vb, c.s); TRY_ALLOC(w.shv, vb, c.s);
    }
    return alloc_levels<T>(c.m, c.s, c.nrhs, w, c.ld > 0 ? c.ld : c.m->tail_level(sizeof(T) == 8));
}

// kernels one BiCGSTAB iteration launches: p, s and x/r updates plus two
// preconditioner applications
static int kernels_per_iteration(const helm_model* m, bool dbl, int precond, int lf, int ld, int fl, int nrhs) {
    return precond == HELM_PRECOND_NONE ? 5 : 3 + 2 * mg_kernels_per_apply(m, dbl, lf, ld, fl, nrhs);
}

template <typename T>
static void bicg_iteration(const SolveCtx& c, Inner<T>& w) {
    const size_t n = c.m->n();
    T *x = w.x.template as<T>(), *r = w.r.template as<T>(), *rh = w.rh.template as<T>();
    T *p = w.p.template as<T>(), *v = w.v.template as<T>(), *sv = w.sv.template as<T>();
    T *t = w.t.template as<T>(), *ph = w.ph.template as<T>(), *shv = w.shv.template as<T>();
    launch_bicg_p<T>(r, p, v, c.st, n, c.nrhs, c.s);
    if (c.o.precond == HELM_PRECOND_NONE) {
        // plain BiCGSTAB: p^ = p, s^ = s
        const LevelDev L0 = level_dev(c.m, 0, sizeof(T) == 8);
        const T* hw = static_cast<const T*>(sizeof(T) == 8 ? (const void*)c.w2 : (const void*)c.w2f);
        launch_apply_dots<T>(1, L0, c.m->npml, c.m->alpha_max, hw, p, v, rh, c.partials, c.pstride, c.st, c.nrhs,
                             c.s);
        launch_bicg_s<T>(r, v, sv, c.st, n, c.nrhs, c.s);
        launch_apply_dots<T>(2, L0, c.m->npml, c.m->alpha_max, hw, sv, t, nullptr, c.partials, c.pstride, c.st,
                             c.nrhs, c.s);
        launch_bicg_xr<T>(x, p, sv, sv, t, rh, r, c.partials, c.pstride, c.st, c.nactive, n, c.nrhs, c.s);
        return;
    }
    vcycle<T>(c, w, p, ph, 1, v, rh);              // p^ = V(p), v = A p^, alpha
    launch_bicg_s<T>(r, v, sv, c.st, n, c.nrhs, c.s);
    vcycle<T>(c, w, sv, shv, 2, t, nullptr);       // s^ = V(s), t = A s^, omega
    launch_bicg_xr<T>(x, ph, shv, sv, t, rh, r, c.partials, c.pstride, c.st, c.nactive, n, c.nrhs, c.s);
}

// Inner BiCGSTAB on rin for the right-hand sides whose outer step is active.
// Leaves the correction in w.x. `graph` caches the captured iteration chunk.
template <typename T>
static int inner_solve(const SolveCtx& c, Inner<T>& w, const T* rin, cudaGraphExec_t* graph, int* iters_done,
                       bool resume, int guard_iters, bool* stalled) {
    const size_t n = c.m->n();
    HELM_CUDA_TRY(cudaMemsetAsync(c.nactive, 0, sizeof(int), c.s));
    count_launches(1);
    if (resume)
        launch_bicg_resume<T>(rin, w.x.template as<T>(), w.r.template as<T>(), w.rh.template as<T>(),
                              w.p.template as<T>(), w.v.template as<T>(), c.partials, c.pstride, c.st, c.nactive, n,
                              c.nrhs, c.s);
    else
        launch_bicg_init<T>(rin, w.x.template as<T>(), w.r.template as<T>(), w.rh.template as<T>(),
                            w.p.template as<T>(), w.v.template as<T>(), c.partials, c.pstride, c.st, c.nactive, n,
                            c.nrhs, c.s);
    NvtxRange nv("bicgstab inner solve");
    const int chunk = std::max(1, c.o.check_every);
    if (c.o.use_graphs && *graph == nullptr) {
        cudaGraph_t g;
        HELM_CUDA_TRY(cudaStreamBeginCapture(c.s, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < chunk; ++k) bicg_iteration<T>(c, w);
        cudaError_t e = cudaStreamEndCapture(c.s, &g);
        if (e != cudaSuccess) { set_last_error(cudaGetErrorString(e)); return HELM_E_CUDA; }
        e = cudaGraphInstantiate(graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { set_last_error(cudaGetErrorString(e)); *graph = nullptr; return HELM_E_CUDA; }
    }
    int h_active = 0;
    int done = 0;
    // every right-hand side stops by itself at max_it; the extra chunk bounds the loop
    const int limit = c.o.max_it + chunk;
    // stall guard (guard_iters > 0): a right-hand side whose recursive residual has not halved
    // within guard_iters iterations ends the inner solve early with *stalled set (its next inner
    // solve restarts the recurrence from the true residual)
    std::vector<RhsState> hs;
    std::vector<double> best(c.nrhs, -1.0);
    std::vector<int> best_it(c.nrhs, 0);
    if (guard_iters > 0) hs.resize(c.nrhs);
    while (done < limit) {
        if (c.o.use_graphs) {
            HELM_CUDA_TRY(cudaGraphLaunch(*graph, c.s));
        } else {
            for (int k = 0; k < chunk; ++k) bicg_iteration<T>(c, w);
        }
        count_launches((unsigned long long)chunk * kernels_per_iteration(c.m, sizeof(T) == 8, c.o.precond, c.lf, c.ld, c.fca ? c.fca_level : 0,
                                                             c.nrhs));
        done += chunk;
        HELM_CUDA_TRY(cudaMemcpyAsync(&h_active, c.nactive, sizeof(int), cudaMemcpyDeviceToHost, c.s));
        if (guard_iters > 0)
            HELM_CUDA_TRY(cudaMemcpyAsync(hs.data(), c.st, sizeof(RhsState) * c.nrhs, cudaMemcpyDeviceToHost, c.s));
        HELM_CUDA_TRY(cudaStreamSynchronize(c.s));
        if (h_active <= 0) break;
        if (guard_iters > 0) {
            bool stall = false;
            for (int b = 0; b < c.nrhs; ++b) {
                if (!hs[b].active || !(hs[b].bnorm2 > 0.0)) continue;
                const double rr = std::sqrt(hs[b].rnorm2 / hs[b].bnorm2);
                if (best[b] < 0.0 || rr <= 0.5 * best[b]) { best[b] = rr; best_it[b] = hs[b].iters; }
                else if (hs[b].iters - best_it[b] >= guard_iters) stall = true;
            }
            if (stall) { *stalled = true; break; }
        }
    }
    HELM_CUDA_TRY(cudaGetLastError());
    *iters_done += done;
    return HELM_OK;
}

// FGMRES buffers: V [(m+1)][nrhs][n], Z [m][nrhs][n] and the small FP64 state.
template <typename T>
struct FgBufs {
    DBuf V, Z, H, g, cs, sn, y, tmp, sc, wn2;
    FgDev dev;
};

template <typename T>
static int alloc_fg(const SolveCtx& c, FgBufs<T>& f) {
    const int m = c.o.restart, nrhs = c.nrhs;
    const size_t vb = sizeof(T) * 2 * c.m->n() * nrhs;
    TRY_ALLOC(f.V, vb * (m + 1), c.s);
    TRY_ALLOC(f.Z, vb * m, c.s);
    TRY_ALLOC(f.H, sizeof(double2) * (size_t)nrhs * (m + 1) * m, c.s);
    TRY_ALLOC(f.g, sizeof(double2) * (size_t)nrhs * (m + 1), c.s);
    TRY_ALLOC(f.cs, sizeof(double) * (size_t)nrhs * m, c.s);
    TRY_ALLOC(f.sn, sizeof(double2) * (size_t)nrhs * m, c.s);
    TRY_ALLOC(f.y, sizeof(double2) * (size_t)nrhs * m, c.s);
    TRY_ALLOC(f.tmp, sizeof(double2) * (size_t)nrhs * (m + 1), c.s);
    TRY_ALLOC(f.sc, sizeof(double) * (size_t)nrhs * (m + 1), c.s);
    TRY_ALLOC(f.wn2, sizeof(double) * (size_t)nrhs, c.s);
    HELM_CUDA_TRY(cudaMemsetAsync(f.H.p, 0, sizeof(double2) * (size_t)nrhs * (m + 1) * m, c.s));
    f.dev.m = m;
    f.dev.H = f.H.template as<double2>();
    f.dev.g = f.g.template as<double2>();
    f.dev.cs = f.cs.template as<double>();
    f.dev.sn = f.sn.template as<double2>();
    f.dev.y = f.y.template as<double2>();
    f.dev.tmp = f.tmp.template as<double2>();
    f.dev.sinv = f.sc.template as<double>();
    f.dev.wn2 = f.wn2.template as<double>();
    return HELM_OK;
}

// One FGMRES cycle of at most m Arnoldi steps from a zero guess on rin; the
// correction is left in w.x.
template <typename T>
static void fgmres_cycle(const SolveCtx& c, Inner<T>& w, FgBufs<T>& f, const T* rin) {
    const size_t n = c.m->n(), vs = n * c.nrhs;
    const int m = f.dev.m, ro = c.o.reorth;
    T* V = f.V.template as<T>();
    T* Z = f.Z.template as<T>();
    launch_fg_norm<T>(rin, c.partials, c.pstride, c.st, f.dev, c.nactive, n, c.nrhs, c.s);
    launch_fg_scale<T>(rin, V, c.st, f.dev, n, c.nrhs, c.s);
    bool pending = false;   // a column finish runs on the side stream
    for (int j = 0; j < m; ++j) {
        T* Vj = V + 2 * vs * j;
        T* W = V + 2 * vs * (j + 1);                                    // A Z'_j, orthogonalised in place
        if (c.o.precond == HELM_PRECOND_NONE) {                        // Z'_j = V'_j, w = A V'_j
            cudaMemcpyAsync(Z + 2 * vs * j, Vj, sizeof(T) * 2 * vs, cudaMemcpyDeviceToDevice, c.s);
            launch_apply<T>(level_dev(c.m, 0, sizeof(T) == 8), c.m->npml, c.m->alpha_max,
                            static_cast<const T*>(sizeof(T) == 8 ? (const void*)c.w2 : (const void*)c.w2f), Vj, W,
                            T(1), c.nrhs, c.s);
        } else {
            vcycle<T>(c, w, Vj, Z + 2 * vs * j, 3, W, nullptr);         // Z'_j = M^-1 V'_j, w = A Z'_j
        }
        // the dot products of this step need 1/s_j from the previous column's finish
        if (pending) { cudaStreamWaitEvent(c.s, c.ev_join, 0); pending = false; }
        int nblk = 0;
        if (ro == HELM_REORTH_IFNEEDED) {
            // first pass decides per RHS whether a second one follows; the column
            // is finished by the last pass's last block
            launch_fg_dots<T>(V, vs, W, j, 0, 1, 0, c.partials, c.pstride, c.st, f.dev, n, c.nrhs, c.s);
            launch_fg_axpy<T>(V, vs, W, j, 2, 0, c.partials, c.pstride, c.st, f.dev, c.nactive, n, c.nrhs, c.s);
            launch_fg_dots<T>(V, vs, W, j, 1, 0, 1, c.partials, c.pstride, c.st, f.dev, n, c.nrhs, c.s);
            launch_fg_axpy<T>(V, vs, W, j, 1, 1, c.partials, c.pstride, c.st, f.dev, c.nactive, n, c.nrhs, c.s);
            continue;
        }
        launch_fg_dots<T>(V, vs, W, j, 0, 0, 0, c.partials, c.pstride, c.st, f.dev, n, c.nrhs, c.s);
        if (ro == HELM_REORTH_ALWAYS) {
            launch_fg_axpy<T>(V, vs, W, j, 0, 0, c.partials, c.pstride, c.st, f.dev, c.nactive, n, c.nrhs, c.s);
            launch_fg_dots<T>(V, vs, W, j, 1, 0, 0, c.partials, c.pstride, c.st, f.dev, n, c.nrhs, c.s);
        }
        // last pass: per-block parts of ||w||^2; the column is finished on the side
        // stream while the next preconditioner application (which reads only w) runs
        nblk = launch_fg_axpy<T>(V, vs, W, j, 3, 0, c.partials, c.pstride, c.st, f.dev, c.nactive, n, c.nrhs, c.s);
        cudaEventRecord(c.ev_fork, c.s);
        cudaStreamWaitEvent(c.side, c.ev_fork, 0);
        launch_fg_finish(c.partials, c.pstride, nblk, c.st, f.dev, j, c.nactive, c.nrhs, c.side);
        cudaEventRecord(c.ev_join, c.side);
        pending = true;
    }
    if (pending) cudaStreamWaitEvent(c.s, c.ev_join, 0);
    launch_fg_backsolve(c.st, f.dev, c.nrhs, c.s);
    launch_fg_update<T>(Z, vs, w.x.template as<T>(), c.st, f.dev, n, c.nrhs, c.s);
}

template <typename T>
static int fgmres_inner(const SolveCtx& c, Inner<T>& w, FgBufs<T>& f, const T* rin, cudaGraphExec_t* graph,
                        int* iters_done) {
    NvtxRange nv("fgmres cycle");
    HELM_CUDA_TRY(cudaMemsetAsync(c.nactive, 0, sizeof(int), c.s));
    if (c.o.use_graphs) {
        if (*graph == nullptr) {
            cudaGraph_t g;
            HELM_CUDA_TRY(cudaStreamBeginCapture(c.s, cudaStreamCaptureModeThreadLocal));
            fgmres_cycle<T>(c, w, f, rin);
            cudaError_t e = cudaStreamEndCapture(c.s, &g);
            if (e != cudaSuccess) { set_last_error(cudaGetErrorString(e)); return HELM_E_CUDA; }
            e = cudaGraphInstantiate(graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { set_last_error(cudaGetErrorString(e)); *graph = nullptr; return HELM_E_CUDA; }
        }
        HELM_CUDA_TRY(cudaGraphLaunch(*graph, c.s));
    } else {
        fgmres_cycle<T>(c, w, f, rin);
    }
    const int m = f.dev.m;
    count_launches(4 + (unsigned long long)m * ((c.o.precond == HELM_PRECOND_NONE ? 1 : mg_kernels_per_apply(c.m, sizeof(T) == 8, c.lf, c.ld, c.fca ? c.fca_level : 0, c.nrhs)) +
                                                (c.o.reorth == HELM_REORTH_NEVER ? 3 : c.o.reorth == HELM_REORTH_ALWAYS ? 5 : 4)));
    HELM_CUDA_TRY(cudaGetLastError());
    *iters_done += m;
    return HELM_OK;
}

// The coarse end of the cycle for one batch: either the dense inverse of level
// ld (HELM_COARSE_AUTO where it applies), in the solve's precision, or the dense
// inverse of the coarsest level that the shared-memory tail uses (FP32 and FP64
// copies). One inverse per distinct (model, frequency) pair: slot[b].
struct CoarseSet {
    DBuf work, mf, md, slot, w2s, mods;
    DBuf grp, panel, dinv, bar, err;   // dense path
    int n = 0, nslots = 0;
    int ld = 0;                        // > 0: the dense path, level ld
    int ngroups = 0, maxg = 0;
    const void* minv(bool dbl) const { return dbl ? md.p : mf.p; }
};

constexpr int kDenseGroup = 8;   // right-hand sides per group of the dense coarse kernel
constexpr int kStallIters = 300; // Krylov iterations without the residual halving that count as a stall

static int build_coarse(const helm_model* m, cudaStream_t s, int nrhs, const double* h_w2, double b1, double b2,
                        bool dbl, int coarse, CoarseSet& cs) {
    NvtxRange nv("coarse set-up");
    // one inverse per distinct (model, frequency) pair
    std::map<std::pair<int, double>, int> uniq;
    std::vector<int> slot(nrhs), mods;
    std::vector<double> w2s;
    for (int b = 0; b < nrhs; ++b) {
        const int mod = m->nmodels > 1 ? b : 0;
        const auto key = std::make_pair(mod, h_w2[b]);
        auto it = uniq.find(key);
        if (it == uniq.end()) {
            it = uniq.emplace(key, (int)w2s.size()).first;
            w2s.push_back(h_w2[b]);
            mods.push_back(mod);
        }
        slot[b] = it->second;
    }
    cs.nslots = (int)w2s.size();
    TRY_ALLOC(cs.slot, sizeof(int) * nrhs, s);
    TRY_ALLOC(cs.w2s, sizeof(double) * cs.nslots, s);
    TRY_ALLOC(cs.mods, sizeof(int) * cs.nslots, s);
    HELM_CUDA_TRY(cudaMemcpyAsync(cs.slot.p, slot.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
    HELM_CUDA_TRY(cudaMemcpyAsync(cs.w2s.p, w2s.data(), sizeof(double) * cs.nslots, cudaMemcpyHostToDevice, s));
    HELM_CUDA_TRY(cudaMemcpyAsync(cs.mods.p, mods.data(), sizeof(int) * cs.nslots, cudaMemcpyHostToDevice, s));

    int W = 0, per = 0;
    const bool want_dense = coarse == HELM_COARSE_DENSE || coarse == HELM_COARSE_FUSED ||
                            (coarse == HELM_COARSE_AUTO && nrhs <= kDenseAutoMaxRhs);
    if (want_dense && b2 != 0.0 && m->ld > 0 && dense_invert_plan((int)m->lv[m->ld].n(), dbl, &W, &per)) {
        const int ld = m->ld, n = (int)m->lv[ld].n();
        const size_t es = dbl ? sizeof(double2) : sizeof(float2);
        const int nl = std::min(per, cs.nslots);
        // groups of at most kDenseGroup consecutive right-hand sides of one slot
        std::vector<int> grp{0};
        int maxg = 0;
        for (int b = 1; b <= nrhs; ++b)
            if (b == nrhs || slot[b] != slot[grp.back()] || b - grp.back() >= kDenseGroup) {
                maxg = std::max(maxg, b - grp.back());
                grp.push_back(b);
            }
        DBuf& mi = dbl ? cs.md : cs.mf;
        TRY_ALLOC(mi, es * (size_t)n * n * cs.nslots, s);
        TRY_ALLOC(cs.panel, es * 2 * (size_t)n * W * nl, s);
        TRY_ALLOC(cs.dinv, es * 2 * (size_t)W * W * nl, s);
        TRY_ALLOC(cs.bar, sizeof(unsigned) * nl, s);
        TRY_ALLOC(cs.err, sizeof(int), s);
        TRY_ALLOC(cs.grp, sizeof(int) * grp.size(), s);
        HELM_CUDA_TRY(cudaMemcpyAsync(cs.grp.p, grp.data(), sizeof(int) * grp.size(), cudaMemcpyHostToDevice, s));
        const LevelDev Ld = level_dev(m, ld, true);
        cudaError_t e = dbl ? launch_dense_invert<double>(Ld, cs.w2s.as<double>(), cs.mods.as<int>(), cs.nslots, b1, b2, W,
                                                          per, cs.md.as<double>(), cs.panel.as<double>(),
                                                          cs.dinv.as<double>(), cs.bar.as<unsigned>(), cs.err.as<int>(), s)
                            : launch_dense_invert<float>(Ld, cs.w2s.as<double>(), cs.mods.as<int>(), cs.nslots, b1, b2, W,
                                                         per, cs.mf.as<float>(), cs.panel.as<float>(),
                                                         cs.dinv.as<float>(), cs.bar.as<unsigned>(), cs.err.as<int>(), s);
        int herr = -1;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, cs.err.p, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && herr == 0) {
            cs.ld = ld;
            cs.n = n;
            cs.ngroups = (int)grp.size() - 1;
            cs.maxg = maxg;
            return HELM_OK;
        }
        // the dense inverse could not be formed (a launch that does not fit, or a
        // vanishing pivot): fall back to the multigrid tail below
        cudaGetLastError();
    }

    const Level& Lc = m->lv.back();
    cs.n = (int)Lc.n();
    cs.ld = 0;
    const size_t nn = (size_t)cs.n * cs.n;
    TRY_ALLOC(cs.work, sizeof(double2) * nn * 2 * cs.nslots, s);
    TRY_ALLOC(cs.mf, sizeof(float2) * nn * cs.nslots, s);
    TRY_ALLOC(cs.md, sizeof(double2) * nn * cs.nslots, s);
    count_launches(1);
    launch_coarse_invert(level_dev(m, (int)m->lv.size() - 1, true), cs.w2s.as<double>(), cs.mods.as<int>(), cs.nslots,
                         b1, b2, cs.work.as<double2>(), cs.mf.as<float2>(), cs.md.as<double2>(), s);
    HELM_CUDA_TRY(cudaGetLastError());
    // the host vectors above must outlive the copies
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    return HELM_OK;
}

template <typename T>
static int solve_impl(const helm_model* m, cudaStream_t s, int nrhs, const double* h_w2, const double* f64,
                      double* u64, const helm_solve_opts& o, helm_solve_stats* stats) {
    NvtxRange nv("helm solve");
    const size_t n = m->n();
    SolveCtx c;
    c.m = m;
    c.s = s;
    c.nrhs = nrhs;
    c.o = o;
    if (prof_on()) c.o.use_graphs = 0;   // every launch is timed on its own while profiling
    c.pstride = 3 * max_blocks_per_rhs(m);
    if (o.krylov == HELM_KRYLOV_FGMRES) c.pstride = std::max(c.pstride, fg_partials(m->n()));
    c.lf = fcycle_level(m, h_w2, nrhs);
    DBuf w2, w2f, st, part, nact, rin;
    TRY_ALLOC(w2, sizeof(double) * nrhs, s);
    TRY_ALLOC(w2f, sizeof(float) * nrhs, s);
    TRY_ALLOC(st, sizeof(RhsState) * nrhs, s);
    TRY_ALLOC(part, sizeof(double) * (size_t)c.pstride * nrhs, s);
    TRY_ALLOC(nact, sizeof(int), s);
    TRY_ALLOC(rin, sizeof(T) * 2 * n * nrhs, s);
    const int coarse = o.precond == HELM_PRECOND_NONE ? HELM_COARSE_TAIL : o.coarse;
    std::unique_ptr<CoarseSet> cs(new CoarseSet());
    int rc = build_coarse(m, s, nrhs, h_w2, o.beta1, o.beta2, sizeof(T) == 8, coarse, *cs);
    if (rc != HELM_OK) return rc;
    c.w2 = w2.as<double>();
    c.w2f = w2f.as<float>();
    c.st = st.as<RhsState>();
    c.partials = part.as<double>();
    c.nactive = nact.as<int>();
    auto use_coarse = [&](const CoarseSet& q) {
        c.slot = q.slot.as<int>();
        c.ncoarse = q.n;
        c.minv = q.minv(sizeof(T) == 8);
        c.ld = q.ld;
        c.grp = q.grp.as<int>();
        c.ngroups = q.ngroups;
        c.maxg = q.maxg;
    };
    use_coarse(*cs);
    Inner<T> w;
    rc = alloc_inner<T>(c, w);
    if (rc != HELM_OK) return rc;
    DBuf fcbar, fcerr;
    std::unique_ptr<FcArgs> fca(new FcArgs());
    rc = setup_fcycle<T>(c, w, coarse, fcbar, fcerr, fca.get());
    if (rc != HELM_OK) return rc;
    const bool fgm = o.krylov == HELM_KRYLOV_FGMRES;
    FgBufs<T> fb;
    SideStream side;
    if (fgm) {
        HELM_CUDA_TRY(cudaStreamCreateWithFlags(&side.s, cudaStreamNonBlocking));
        HELM_CUDA_TRY(cudaEventCreateWithFlags(&side.fork, cudaEventDisableTiming));
        HELM_CUDA_TRY(cudaEventCreateWithFlags(&side.join, cudaEventDisableTiming));
        c.side = side.s;
        c.ev_fork = side.fork;
        c.ev_join = side.join;
        rc = alloc_fg<T>(c, fb);
        if (rc != HELM_OK) return rc;
    }

    std::vector<RhsState> hs(nrhs);
    std::memset(hs.data(), 0, sizeof(RhsState) * nrhs);
    for (auto& S : hs) { S.outer_active = 1; S.active = 1; S.max_it = o.max_it; }
    HELM_CUDA_TRY(cudaMemcpyAsync(c.st, hs.data(), sizeof(RhsState) * nrhs, cudaMemcpyHostToDevice, s));
    HELM_CUDA_TRY(cudaMemcpyAsync(w2.p, h_w2, sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    std::vector<float> h_w2f(h_w2, h_w2 + nrhs);
    HELM_CUDA_TRY(cudaMemcpyAsync(w2f.p, h_w2f.data(), sizeof(float) * nrhs, cudaMemcpyHostToDevice, s));
    HELM_CUDA_TRY(cudaMemsetAsync(part.p, 0, sizeof(double) * (size_t)c.pstride * nrhs, s));
    HELM_CUDA_TRY(cudaMemsetAsync(u64, 0, sizeof(double) * 2 * n * nrhs, s));

    // inner target per outer step: max(floor, fac * tol / relres). The complex64-only
    // mode has no refinement, so it asks its one inner solve for a margin below tol
    // to absorb the drift between the recursive and the true residual.
    double floor_tol = 0.0, inner_fac = 0.9;
    int max_outer = o.max_outer;
    if (o.precision == HELM_PREC_MIXED) floor_tol = o.inner_tol;
    if (o.precision == HELM_PREC_FP32) { inner_fac = 0.2; max_outer = 1; }
    // FGMRES restarts through the outer refinement: allow enough cycles for max_it
    if (fgm) max_outer = std::max(max_outer, (o.max_it + o.restart - 1) / o.restart + 1);

    std::vector<int> outer_count(nrhs, 0);
    cudaGraphExec_t graph = nullptr;
    int iters_done = 0;
    const LevelDev L0 = level_dev(m, 0, true);
    // Stall guard: while the preconditioner's shift is not the paper's (1, 1), a right-hand side
    // whose FP64 residual has not halved within kStallIters Krylov iterations (while above tol)
    // switches the batch to (1, 1): with (1, 0.5) and Jacobi weight 0.5 the cycle is not a stable
    // approximate inverse on some layered models (slow layers between fast ones), and the solve
    // then stalls at any tolerance. BiCGSTAB also checks its recursive residual within the inner
    // solve (it can run up to max_it there) and ends that inner solve early on a stall.
    const bool guard = o.precond != HELM_PRECOND_NONE && !(o.beta1 == 1.0 && o.beta2 == 1.0);
    bool switched = false, restart_inner = false, force_switch = false;
    std::vector<int> ref_it(nrhs, 0);
    std::vector<double> ref_res(nrhs, -1.0);
    for (int outer = 0;; ++outer) {
        NvtxRange nv_outer("refinement step");
        launch_resid64<T>(L0, m->npml, m->alpha_max, c.w2, f64, u64, rin.as<T>(), c.partials, c.pstride, c.st, o.tol,
                          floor_tol, inner_fac, outer == 0, nrhs, s);
        count_launches(1);
        HELM_CUDA_TRY(cudaGetLastError());
        HELM_CUDA_TRY(cudaMemcpyAsync(hs.data(), c.st, sizeof(RhsState) * nrhs, cudaMemcpyDeviceToHost, s));
        HELM_CUDA_TRY(cudaStreamSynchronize(s));
        int any = 0;
        for (int b = 0; b < nrhs; ++b)
            if (hs[b].outer_active) { any = 1; }
        if (!any || outer >= max_outer) break;
        if (guard && !switched) {
            bool stall = force_switch;
            for (int b = 0; b < nrhs; ++b) {
                if (!hs[b].outer_active) continue;
                if (ref_res[b] < 0.0 || hs[b].relres <= 0.5 * ref_res[b]) {
                    ref_res[b] = hs[b].relres;
                    ref_it[b] = hs[b].iters;
                } else if (hs[b].iters - ref_it[b] >= kStallIters) {
                    stall = true;
                }
            }
            if (stall) {
                c.o.beta1 = 1.0;
                c.o.beta2 = 1.0;
                std::unique_ptr<CoarseSet> cs2(new CoarseSet());
                rc = build_coarse(m, s, nrhs, h_w2, 1.0, 1.0, sizeof(T) == 8, coarse, *cs2);
                if (rc != HELM_OK) break;
                cs.swap(cs2);
                use_coarse(*cs);
                rc = setup_fcycle<T>(c, w, coarse, fcbar, fcerr, fca.get());
                if (rc != HELM_OK) break;
                if (graph) { cudaGraphExecDestroy(graph); graph = nullptr; }   // captured with the old inverse
                switched = true;
                restart_inner = true;
            }
        }
        for (int b = 0; b < nrhs; ++b) outer_count[b] += hs[b].outer_active;
        // BiCGSTAB keeps its recurrence across refinement steps (residual replacement)
        bool inner_stall = false;
        rc = fgm ? fgmres_inner<T>(c, w, fb, rin.as<T>(), &graph, &iters_done)
                 : inner_solve<T>(c, w, rin.as<T>(), &graph, &iters_done, outer > 0 && !restart_inner,
                                  guard && !switched ? kStallIters : 0, &inner_stall);
        restart_inner = false;
        if (inner_stall) force_switch = true;
        if (rc != HELM_OK) break;
        rc = check_fcycle(c, fcerr);   // a persistent cycle that gave up a barrier ends the solve
        if (rc != HELM_OK) break;
        launch_refine<T>(w.x.template as<T>(), u64, c.st, n, nrhs, s);
        count_launches(1);
    }
    if (graph) cudaGraphExecDestroy(graph);
    if (rc != HELM_OK) return rc;
    HELM_CUDA_TRY(cudaGetLastError());
    rc = check_fcycle(c, fcerr);
    if (rc != HELM_OK) return rc;
    int status = HELM_OK;
    for (int b = 0; b < nrhs; ++b) {
        const bool conv = hs[b].relres <= o.tol;
        if (!conv) status = HELM_E_NOT_CONVERGED;
        if (stats) {
            stats[b].iters = hs[b].iters;
            stats[b].outer_its = outer_count[b];
            stats[b].converged = conv ? 1 : 0;
            stats[b].relres = hs[b].relres;
            stats[b].dense_level = cs->ld;
            stats[b].shift_switched = switched ? 1 : 0;
        }
    }
    return status;
}

int solve_batch(const helm_model* m, cudaStream_t s, int nrhs, const double* h_w2, const double* f64, double* u64,
                const helm_solve_opts& o, helm_solve_stats* stats) {
    if (o.precision == HELM_PREC_FP64) return solve_impl<double>(m, s, nrhs, h_w2, f64, u64, o, stats);
    return solve_impl<float>(m, s, nrhs, h_w2, f64, u64, o, stats);
}

size_t solve_bytes(int nx, int nz, int nlev_n_sum_extra, int nrhs, int precision) {
    const size_t n = (size_t)nx * nz;
    const size_t ts = precision == HELM_PREC_FP64 ? 8 : 4;
    // inner: 9 vectors + rin; levels ~ 2 * n / 3; outer: f64, u64
    size_t b = (size_t)nrhs * n * 2 * ts * 10 + (size_t)nrhs * n * 2 * ts * 2 / 3 + (size_t)nrhs * n * 16 * 2;
    b += (size_t)nlev_n_sum_extra;
    return b + (64u << 20);
}

// One standalone preconditioner cycle z = V(r) on the fine level, complex64, for checks.
int vcycle_once(const helm_model* m, cudaStream_t s, int nrhs, const double* h_w2, double b1, double b2, double wj,
                int coarse, const float* r, float* z) {
    SolveCtx c;
    c.m = m;
    c.s = s;
    c.nrhs = nrhs;
    helm_default_opts(&c.o);
    c.o.beta1 = b1;
    c.o.beta2 = b2;
    c.o.omega_jacobi = wj;
    c.pstride = 3 * max_blocks_per_rhs(m);
    c.lf = fcycle_level(m, h_w2, nrhs);
    DBuf w2, w2f;
    TRY_ALLOC(w2, sizeof(double) * nrhs, s);
    TRY_ALLOC(w2f, sizeof(float) * nrhs, s);
    HELM_CUDA_TRY(cudaMemcpyAsync(w2.p, h_w2, sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    std::vector<float> h_w2f(h_w2, h_w2 + nrhs);
    HELM_CUDA_TRY(cudaMemcpyAsync(w2f.p, h_w2f.data(), sizeof(float) * nrhs, cudaMemcpyHostToDevice, s));
    CoarseSet cs;
    int rc = build_coarse(m, s, nrhs, h_w2, b1, b2, false, coarse, cs);
    if (rc != HELM_OK) return rc;
    c.w2 = w2.as<double>();
    c.w2f = w2f.as<float>();
    c.st = nullptr;
    c.partials = nullptr;
    c.nactive = nullptr;
    c.slot = cs.slot.as<int>();
    c.ncoarse = cs.n;
    c.minv = cs.mf.p;
    c.ld = cs.ld;
    c.grp = cs.grp.as<int>();
    c.ngroups = cs.ngroups;
    c.maxg = cs.maxg;
    Inner<float> w;
    rc = alloc_levels<float>(m, s, nrhs, w, c.ld > 0 ? c.ld : m->tail_level(false));
    if (rc != HELM_OK) return rc;
    DBuf fcbar, fcerr;
    FcArgs fa;
    rc = setup_fcycle<float>(c, w, coarse, fcbar, fcerr, &fa);
    if (rc != HELM_OK) return rc;
    vcycle<float>(c, w, r, z, 0, nullptr, nullptr);
    HELM_CUDA_TRY(cudaGetLastError());
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    return check_fcycle(c, fcerr);
}

// ------------------------------------------------------- kernel timing
// Launches one hot-path kernel `reps` times on scratch vectors of nrhs
// right-hand sides (filled with byte 0x3C) and returns the mean time per launch (CUDA events on `s`)
// and the algorithmic bytes one launch must move (each input read once, each
// output written once; the squared slowness, shared by all right-hand sides,
// counted once).
int time_kernel(const helm_model* m, cudaStream_t s, int kernel, int nrhs, double hw2, int reps, double* ms,
                double* bytes) {
    const size_t n = m->n();
    const size_t v32 = sizeof(float) * 2 * n * nrhs, v64 = sizeof(double) * 2 * n * nrhs;
    const int nvec = 8;
    std::vector<std::unique_ptr<DBuf>> v(nvec);
    const bool dbl = (kernel == HELM_KERNEL_RESID64 || kernel == HELM_KERNEL_APPLY64);
    for (int k = 0; k < nvec; ++k) {
        v[k].reset(new DBuf());
        TRY_ALLOC(*v[k], dbl ? v64 : v32, s);
        // byte 0x3C gives small normal, non-zero values in both precisions
        HELM_CUDA_TRY(cudaMemsetAsync(v[k]->p, 0x3C, dbl ? v64 : v32, s));
    }
    DBuf w2, w2f, st, part, nact, fc, rin, fgV, fgH, fgSmall;
    FgDev fgd{};
    const int pstride = std::max(3 * max_blocks_per_rhs(m), fg_partials(n));
    TRY_ALLOC(w2, sizeof(double) * nrhs, s);
    TRY_ALLOC(w2f, sizeof(float) * nrhs, s);
    TRY_ALLOC(st, sizeof(RhsState) * nrhs, s);
    TRY_ALLOC(part, sizeof(double) * (size_t)pstride * nrhs, s);
    TRY_ALLOC(nact, sizeof(int), s);
    TRY_ALLOC(fc, sizeof(float) * 2 * m->lv[1].n() * nrhs, s);
    TRY_ALLOC(rin, v32, s);
    HELM_CUDA_TRY(cudaMemsetAsync(fc.p, 0x3C, sizeof(float) * 2 * m->lv[1].n() * nrhs, s));
    std::vector<double> hw(nrhs, hw2);
    std::vector<RhsState> hs(nrhs);
    std::memset(hs.data(), 0, sizeof(RhsState) * nrhs);
    for (auto& S : hs) {
        // bnorm2 < 0 keeps the convergence test false, so every launch does its full work
        S.active = 1; S.outer_active = 1; S.max_it = 1 << 30; S.tol_rel = 1.0; S.bnorm2 = -1.0; S.fnorm2 = 1.0;
        S.rho[0] = 1.0; S.alpha[0] = 0.5; S.omega[0] = 0.5; S.beta[0] = 0.5;
    }
    HELM_CUDA_TRY(cudaMemcpyAsync(w2.p, hw.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    std::vector<float> hwf(hw.begin(), hw.end());
    HELM_CUDA_TRY(cudaMemcpyAsync(w2f.p, hwf.data(), sizeof(float) * nrhs, cudaMemcpyHostToDevice, s));
    HELM_CUDA_TRY(cudaMemcpyAsync(st.p, hs.data(), sizeof(RhsState) * nrhs, cudaMemcpyHostToDevice, s));
    HELM_CUDA_TRY(cudaMemsetAsync(part.p, 0, sizeof(double) * (size_t)pstride * nrhs, s));
    const double N = (double)n, B = (double)nrhs;
    auto F = [&](int k) { return v[k]->as<float>(); };
    auto D = [&](int k) { return v[k]->as<double>(); };
    RhsState* S = st.as<RhsState>();
    std::function<void()> launch;
    switch (kernel) {
        case HELM_KERNEL_APPLY:
            launch = [&] { launch_apply<float>(level_dev(m, 0, false), m->npml, m->alpha_max, w2f.as<float>(), F(0), F(1), 1.0f, nrhs, s); };
            *bytes = N * (16.0 * B + 4.0);
            break;
        case HELM_KERNEL_APPLY64:
            launch = [&] { launch_apply<double>(level_dev(m, 0, true), m->npml, m->alpha_max, w2.as<double>(), D(0), D(1), 1.0, nrhs, s); };
            *bytes = N * (32.0 * B + 8.0);
            break;
        case HELM_KERNEL_RESTRICT:
            launch = [&] { launch_restrict<float>(level_dev(m, 0, false), level_dev(m, 1, false), w2f.as<float>(), 1.0, 0.5, 0.8, F(0), fc.as<float>(), S, nrhs, s); };
            *bytes = N * (8.0 * B + 4.0) + 8.0 * B * (double)m->lv[1].n();
            break;
        case HELM_KERNEL_PROLONG:
            launch = [&] { launch_prolong<float>(1, level_dev(m, 0, false), level_dev(m, 1, false), m->npml, m->alpha_max, w2f.as<float>(), 1.0, 0.5, 0.8, F(0), fc.as<float>(), F(1), F(2), F(3), part.as<double>(), pstride, S, nrhs, s); };
            *bytes = N * (32.0 * B + 4.0) + 8.0 * B * (double)m->lv[1].n();
            break;
        case HELM_KERNEL_BICG_XR:
            launch = [&] { launch_bicg_xr<float>(F(0), F(1), F(2), F(3), F(4), F(5), F(6), part.as<double>(), pstride, S, nact.as<int>(), n, nrhs, s); };
            *bytes = N * B * 64.0;
            break;
        case HELM_KERNEL_BICG_P:
            launch = [&] { launch_bicg_p<float>(F(0), F(1), F(2), S, n, nrhs, s); };
            *bytes = N * B * 32.0;
            break;
        case HELM_KERNEL_RESID64:
            launch = [&] { launch_resid64<float>(level_dev(m, 0, true), m->npml, m->alpha_max, w2.as<double>(), D(0), D(1), rin.as<float>(), part.as<double>(), pstride, S, 0.0, 1e-4, 0.9, 0, nrhs, s); };
            *bytes = N * (40.0 * B + 8.0);
            break;
        case HELM_KERNEL_FG_DOTS:
        case HELM_KERNEL_FG_AXPY: {
            // Arnoldi step j = kFgTimedStep of FGMRES(10): basis slots 0..j, w in slot j + 1
            const int j = kFgTimedStep, mres = 10;
            const size_t vs = n * nrhs;
            TRY_ALLOC(fgV, sizeof(float) * 2 * vs * (j + 2), s);
            HELM_CUDA_TRY(cudaMemsetAsync(fgV.p, 0x3C, sizeof(float) * 2 * vs * (j + 2), s));
            const size_t nb = (size_t)nrhs;
            TRY_ALLOC(fgH, sizeof(double2) * nb * (mres + 1) * mres, s);
            TRY_ALLOC(fgSmall, sizeof(double2) * nb * 8 * (mres + 1), s);
            HELM_CUDA_TRY(cudaMemsetAsync(fgH.p, 0, sizeof(double2) * nb * (mres + 1) * mres, s));
            HELM_CUDA_TRY(cudaMemsetAsync(fgSmall.p, 0, sizeof(double2) * nb * 8 * (mres + 1), s));
            // basis norms s_i = 1 and projection coefficients 1e-3 (w stays finite over the launches)
            std::vector<double> ones(nb * (mres + 1), 1.0);
            std::vector<double2> coef(nb * (mres + 1), make_double2(1e-3, 0.0));
            double2* small = fgSmall.as<double2>();
            fgd.m = mres;
            fgd.H = fgH.as<double2>();
            fgd.g = small;
            fgd.sn = small + nb * (mres + 1);
            fgd.y = small + 2 * nb * (mres + 1);
            fgd.tmp = small + 3 * nb * (mres + 1);
            fgd.cs = reinterpret_cast<double*>(small + 4 * nb * (mres + 1));
            fgd.sinv = reinterpret_cast<double*>(small + 5 * nb * (mres + 1));
            fgd.wn2 = reinterpret_cast<double*>(small + 6 * nb * (mres + 1));
            HELM_CUDA_TRY(cudaMemcpyAsync(fgd.sinv, ones.data(), sizeof(double) * ones.size(), cudaMemcpyHostToDevice, s));
            HELM_CUDA_TRY(cudaMemcpyAsync(fgd.tmp, coef.data(), sizeof(double2) * coef.size(), cudaMemcpyHostToDevice, s));
            HELM_CUDA_TRY(cudaStreamSynchronize(s));   // the host vectors above are sources of async copies
            float* Vb = fgV.as<float>();
            float* Wb = Vb + 2 * vs * (j + 1);
            if (kernel == HELM_KERNEL_FG_DOTS) {
                launch = [&, j, vs, Vb, Wb] { launch_fg_dots<float>(Vb, vs, Wb, j, 0, 0, 0, part.as<double>(), pstride, S, fgd, n, nrhs, s); };
                *bytes = N * B * 8.0 * (j + 2);
            } else {
                // mode 3, as in the solve: per-block norm parts, the column finished elsewhere
                launch = [&, j, vs, Vb, Wb] { launch_fg_axpy<float>(Vb, vs, Wb, j, 3, 0, part.as<double>(), pstride, S, fgd, nact.as<int>(), n, nrhs, s); };
                *bytes = N * B * 8.0 * (j + 3);
            }
            break;
        }
        case HELM_KERNEL_TAIL: {
            // one F-cycle over the tail levels; the coarsest inverse is filler of the
            // right size (the launch's cost does not depend on its values)
            const int lt = m->tail_level(false);
            const size_t nL = m->lv.back().n(), nt = m->lv[lt].n();
            TRY_ALLOC(fgV, sizeof(float) * 2 * nL * nL, s);
            HELM_CUDA_TRY(cudaMemsetAsync(fgV.p, 0x3C, sizeof(float) * 2 * nL * nL, s));
            TRY_ALLOC(fgSmall, sizeof(int) * nrhs, s);
            HELM_CUDA_TRY(cudaMemsetAsync(fgSmall.p, 0, sizeof(int) * nrhs, s));
            const TailArgs a = tail_args<float>(m, true, F(0), F(1), 0, fgV.p, fgSmall.as<int>(), w2.as<double>(),
                                                1.0, 0.5, 0.8);
            launch = [&, a] { launch_tail<float>(a, m->tail_smem[0], nrhs, S, s); };
            *bytes = 16.0 * B * (double)nt;
            break;
        }
        case HELM_KERNEL_FMA64: {
            // eight blocks of 256 threads per SM, each thread 8 chains of 2048 FP64 FMAs
            int dev = 0, sms = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const int blocks = 8 * sms, iters = 2048;
            launch = [&, blocks] { launch_fma64(D(0), blocks, iters, s); };
            *bytes = 2.0 * blocks * 256.0 * 8.0 * iters;   // FP64 operations (2 per fused multiply-add)
            break;
        }
        default:
            return HELM_E_INVALID;
    }
    for (int k = 0; k < 3; ++k) launch();
    // keep every right-hand side active (the kernels may have flagged convergence)
    HELM_CUDA_TRY(cudaMemcpyAsync(st.p, hs.data(), sizeof(RhsState) * nrhs, cudaMemcpyHostToDevice, s));
    cudaEvent_t e0, e1;
    HELM_CUDA_TRY(cudaEventCreate(&e0));
    HELM_CUDA_TRY(cudaEventCreate(&e1));
    HELM_CUDA_TRY(cudaEventRecord(e0, s));
    for (int k = 0; k < reps; ++k) launch();
    HELM_CUDA_TRY(cudaEventRecord(e1, s));
    HELM_CUDA_TRY(cudaEventSynchronize(e1));
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    HELM_CUDA_TRY(cudaGetLastError());
    *ms = (double)t / reps;
    return HELM_OK;
}

// -------------------------------------------------------------- autotune
// Times the tile variants of the complex64 multigrid kernels on the grid levels
// (finest-level prolongation; Galerkin restriction and prolongation on levels
// 1..lt-1) for a batch of nrhs right-hand sides, keeps the faster of each in the
// model and returns the choices: out[l] = restriction tile, out[kMaxLevels + l]
// = prolongation tile.
int autotune(helm_model* m, cudaStream_t s, int nrhs, double hw2, int reps, int* out) {
    const int lt = m->tail_level(false);
    size_t maxn = m->n();
    std::vector<std::unique_ptr<DBuf>> v(4);
    for (auto& b : v) {
        b.reset(new DBuf());
        TRY_ALLOC(*b, sizeof(float) * 2 * maxn * nrhs, s);
        HELM_CUDA_TRY(cudaMemsetAsync(b->p, 0x3C, sizeof(float) * 2 * maxn * nrhs, s));
    }
    DBuf w2f, st, part;
    const int pstride = 3 * max_blocks_per_rhs(m);
    TRY_ALLOC(w2f, sizeof(float) * nrhs, s);
    TRY_ALLOC(st, sizeof(RhsState) * nrhs, s);
    TRY_ALLOC(part, sizeof(double) * (size_t)pstride * nrhs, s);
    std::vector<float> hw(nrhs, (float)hw2);
    HELM_CUDA_TRY(cudaMemcpyAsync(w2f.p, hw.data(), sizeof(float) * nrhs, cudaMemcpyHostToDevice, s));
    std::vector<RhsState> hs(nrhs);
    std::memset(hs.data(), 0, sizeof(RhsState) * nrhs);
    for (auto& S : hs) { S.active = 1; S.outer_active = 1; S.rho[0] = 1.0; }
    HELM_CUDA_TRY(cudaMemcpyAsync(st.p, hs.data(), sizeof(RhsState) * nrhs, cudaMemcpyHostToDevice, s));
    HELM_CUDA_TRY(cudaMemsetAsync(part.p, 0, sizeof(double) * (size_t)pstride * nrhs, s));
    RhsState* S = st.as<RhsState>();
    auto F = [&](int k) { return v[k]->as<float>(); };
    cudaEvent_t e0, e1;
    HELM_CUDA_TRY(cudaEventCreate(&e0));
    HELM_CUDA_TRY(cudaEventCreate(&e1));
    auto time_it = [&](const std::function<void()>& launch) -> float {
        for (int k = 0; k < 2; ++k) launch();
        // restore the states the finest-level reduction may have changed
        cudaMemcpyAsync(st.p, hs.data(), sizeof(RhsState) * nrhs, cudaMemcpyHostToDevice, s);
        cudaEventRecord(e0, s);
        for (int k = 0; k < reps; ++k) launch();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        return t;
    };
    for (int l = 0; l < kMaxLevels; ++l) { out[l] = m->tile_restrict[l]; out[kMaxLevels + l] = m->tile_prolong[l]; }
    // every grid level a cycle launches kernels on: above the tail, or above the dense level
    const int top = std::max(lt, m->ld);
    for (int l = 0; l < top && l + 1 < (int)m->lv.size(); ++l) {
        const LevelDev Lf = level_dev(m, l, false), Lc = level_dev(m, l + 1, false);
        // the finest level's marching prolongation has two row-segment choices; the Galerkin
        // levels the tile shapes of launch_prolong_g / launch_restrict_g
        const bool fine = l == 0 && !m->vd;
        const int np = fine ? 2 : kProlongTiles, nr = l > 0 ? kRestrictTiles : 0;
        int bp = m->tile_prolong[l], br = m->tile_restrict[l];
        float best_p = 0.f, best_r = 0.f;
        for (int t = 0; t < np; ++t) {
            const float tp = time_it([&] {
                launch_prolong<float>(fine ? 1 : 0, Lf, Lc, m->npml, m->alpha_max, w2f.as<float>(), 1.0, 0.5, 0.5,
                                      F(0), F(1), F(2), F(3), F(0), part.as<double>(), pstride, S, nrhs, s, 0, t);
            });
            if (t == 0 || tp < best_p) { best_p = tp; bp = t; }
        }
        for (int t = 0; t < nr; ++t) {
            const float tr = time_it([&] {
                launch_restrict<float>(Lf, Lc, w2f.as<float>(), 1.0, 0.5, 0.5, F(0), F(1), S, nrhs, s, t);
            });
            if (t == 0 || tr < best_r) { best_r = tr; br = t; }
        }
        m->tile_prolong[l] = bp;
        if (l > 0) m->tile_restrict[l] = br;
        out[l] = m->tile_restrict[l];
        out[kMaxLevels + l] = m->tile_prolong[l];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    HELM_CUDA_TRY(cudaGetLastError());
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    return HELM_OK;
}

// ------------------------------------------------------------ gradient
// Forward half of the misfit gradient (Eq. 4): all shots and frequencies in one
// batch, u kept on the device for the adjoint half.
int fwi_forward(const helm_model* m, cudaStream_t s, int nfreq, const double* omega, int nshot, const int* src_flat_h,
                int nrec, const int* rec_flat_h, const double* d_obs_dev, double lam, double* J_out, double* d_cal_dev,
                const helm_solve_opts& o, helm_solve_stats* stats, FwiState** out) {
    *out = nullptr;
    const int nrhs = nfreq * nshot;
    const size_t n = m->n();
    std::unique_ptr<FwiState> st(new FwiState());
    st->m = m;
    st->nrhs = nrhs;
    st->nrec = nrec;
    st->w2.resize(nrhs);
    st->hw2.resize(nrhs);
    std::vector<int> src(nrhs);
    for (int f = 0; f < nfreq; ++f)
        for (int k = 0; k < nshot; ++k) {
            st->w2[f * nshot + k] = omega[f] * omega[f];
            st->hw2[f * nshot + k] = m->h * m->h * omega[f] * omega[f];
            src[f * nshot + k] = src_flat_h[k];
        }
    auto am = [&](void** p, size_t b) {
        if (cudaMalloc(p, b ? b : 16) != cudaSuccess) { cudaGetLastError(); return false; }
        return true;
    };
    if (!am((void**)&st->u64, sizeof(double) * 2 * n * nrhs) || !am((void**)&st->resid, sizeof(double) * 2 * (size_t)nrec * nrhs) ||
        !am((void**)&st->drec, sizeof(int) * nrec) || !am((void**)&st->dw2, sizeof(double) * nrhs)) {
        set_last_error("device allocation failed");
        return HELM_E_NOMEM;
    }
    DBuf f64, dsrc, jpart;
    TRY_ALLOC(f64, sizeof(double) * 2 * n * nrhs, s);
    TRY_ALLOC(dsrc, sizeof(int) * nrhs, s);
    TRY_ALLOC(jpart, sizeof(double) * nrhs, s);
    HELM_CUDA_TRY(cudaMemcpyAsync(dsrc.p, src.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
    HELM_CUDA_TRY(cudaMemcpyAsync(st->drec, rec_flat_h, sizeof(int) * nrec, cudaMemcpyHostToDevice, s));
    HELM_CUDA_TRY(cudaMemcpyAsync(st->dw2, st->w2.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    launch_point_rhs(f64.as<double>(), dsrc.as<int>(), nrhs, n, s);
    int rc = solve_batch(m, s, nrhs, st->hw2.data(), f64.as<double>(), st->u64, o, stats);
    if (rc != HELM_OK && rc != HELM_E_NOT_CONVERGED) return rc;
    launch_sample(st->u64, st->drec, nrec, d_obs_dev, d_cal_dev, st->resid, jpart.as<double>(), n, nrhs, s);
    HELM_CUDA_TRY(cudaGetLastError());
    std::vector<double> jp(nrhs);
    HELM_CUDA_TRY(cudaMemcpyAsync(jp.data(), jpart.p, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    double J = 0.0;
    for (int b = 0; b < nrhs; ++b) J += jp[b];
    st->lam = lam;
    *J_out = J + lam * m->msq_sum;
    *out = st.release();
    return rc;
}

// Adjoint half (Eq. 7): B w = conj(P^T r) per shot and frequency (lambda =
// conj(w) because B is complex symmetric), then the gradient accumulation and
// the fold of the layer onto the physical cells.
int fwi_backward(FwiState* st, cudaStream_t s, double* grad_dev, const helm_solve_opts& o, helm_solve_stats* stats) {
    const helm_model* m = st->m;
    const int nrhs = st->nrhs;
    const size_t n = m->n();
    DBuf f64, w64, gpad;
    TRY_ALLOC(f64, sizeof(double) * 2 * n * nrhs, s);
    TRY_ALLOC(w64, sizeof(double) * 2 * n * nrhs, s);
    TRY_ALLOC(gpad, sizeof(double) * n, s);
    HELM_CUDA_TRY(cudaMemsetAsync(gpad.p, 0, sizeof(double) * n, s));
    launch_adjoint_rhs(st->resid, st->drec, st->nrec, m->h * m->h, f64.as<double>(), n, nrhs, s);
    int rc = solve_batch(m, s, nrhs, st->hw2.data(), f64.as<double>(), w64.as<double>(), o, stats);
    if (rc != HELM_OK && rc != HELM_E_NOT_CONVERGED) return rc;
    launch_grad_accum(st->u64, w64.as<double>(), st->dw2, m->m_pad, m->nx, m->nz, m->npml, m->alpha_max,
                      gpad.as<double>(), nrhs, s);
    launch_fold(gpad.as<double>(), m->m_pad, m->Px, m->Pz, m->npml, st->lam, grad_dev, s);
    HELM_CUDA_TRY(cudaGetLastError());
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    return rc;
}

// ------------------------------------------------------- Gauss-Newton (Eq. 9)
// H dm for the Gauss-Newton Hessian of J (Eq. 8 without its second term):
// H dm = 2 Re[Jac^H Jac dm] + 2 lam dm, Jac the Jacobian of the receiver data
// P u with respect to the physical slowness, at the model and wavefields of
// the forward state. Per shot and frequency: one Born solve
// B du = 2 omega^2 m (1 - j alpha) u (E dm), dd = P du, one adjoint solve
// B w = conj(P^T dd); then the accumulation and fold of the gradient with w in
// place of the adjoint field.
int gn_hvp(FwiState* st, cudaStream_t s, const double* dm_dev, double* hdm_dev, const helm_solve_opts& o,
           helm_solve_stats* stats) {
    const helm_model* m = st->m;
    const int nrhs = st->nrhs;
    const size_t n = m->n();
    DBuf dmpad, f64, du, w64, gpad, zero, dd, jp, dhw2;
    TRY_ALLOC(dmpad, sizeof(double) * n, s);
    TRY_ALLOC(f64, sizeof(double) * 2 * n * nrhs, s);
    TRY_ALLOC(du, sizeof(double) * 2 * n * nrhs, s);
    TRY_ALLOC(w64, sizeof(double) * 2 * n * nrhs, s);
    TRY_ALLOC(gpad, sizeof(double) * n, s);
    TRY_ALLOC(zero, sizeof(double) * 2 * (size_t)st->nrec * nrhs, s);
    TRY_ALLOC(dd, sizeof(double) * 2 * (size_t)st->nrec * nrhs, s);
    TRY_ALLOC(jp, sizeof(double) * nrhs, s);
    TRY_ALLOC(dhw2, sizeof(double) * nrhs, s);
    HELM_CUDA_TRY(cudaMemcpyAsync(dhw2.p, st->hw2.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    HELM_CUDA_TRY(cudaMemsetAsync(zero.p, 0, sizeof(double) * 2 * (size_t)st->nrec * nrhs, s));
    HELM_CUDA_TRY(cudaMemsetAsync(gpad.p, 0, sizeof(double) * n, s));
    launch_expand(dm_dev, m->Px, m->Pz, m->npml, dmpad.as<double>(), s);
    launch_born_rhs(st->u64, dmpad.as<double>(), m->m_pad, dhw2.as<double>(), m->nx, m->nz, m->npml, m->alpha_max,
                    f64.as<double>(), nrhs, s);
    int rc1 = solve_batch(m, s, nrhs, st->hw2.data(), f64.as<double>(), du.as<double>(), o, stats);
    if (rc1 != HELM_OK && rc1 != HELM_E_NOT_CONVERGED) return rc1;
    // dd = P du (the sampling kernel with zero observed data)
    launch_sample(du.as<double>(), st->drec, st->nrec, zero.as<double>(), nullptr, dd.as<double>(), jp.as<double>(), n,
                  nrhs, s);
    launch_adjoint_rhs(dd.as<double>(), st->drec, st->nrec, m->h * m->h, f64.as<double>(), n, nrhs, s);
    int rc2 = solve_batch(m, s, nrhs, st->hw2.data(), f64.as<double>(), w64.as<double>(), o,
                          stats ? stats + nrhs : nullptr);
    if (rc2 != HELM_OK && rc2 != HELM_E_NOT_CONVERGED) return rc2;
    launch_grad_accum(st->u64, w64.as<double>(), st->dw2, m->m_pad, m->nx, m->nz, m->npml, m->alpha_max,
                      gpad.as<double>(), nrhs, s);
    launch_fold(gpad.as<double>(), m->m_pad, m->Px, m->Pz, m->npml, st->lam, hdm_dev, s, dm_dev);
    HELM_CUDA_TRY(cudaGetLastError());
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    return (rc1 == HELM_E_NOT_CONVERGED || rc2 == HELM_E_NOT_CONVERGED) ? HELM_E_NOT_CONVERGED : HELM_OK;
}

static int dev_dot(const double* a, const double* b, size_t n, DBuf& part, cudaStream_t s, double* out) {
    const int nb = dot_blocks(n);
    launch_dot_partials(a, b, n, part.as<double>(), s);
    std::vector<double> h(nb);
    HELM_CUDA_TRY(cudaMemcpyAsync(h.data(), part.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    double acc = 0.0;
    for (int k = 0; k < nb; ++k) acc += h[k];
    *out = acc;
    return HELM_OK;
}

// One Gauss-Newton step (Eq. 9): dm = -H^{-1} g by conjugate gradients from
// dm = 0 (H symmetric positive definite for lam > 0), `iters` Hessian-vector
// products. rel[k] = ||g + H dm_k|| / ||g|| after k iterations (k = 0..iters).
int gn_step(FwiState* st, cudaStream_t s, const double* g_dev, int iters, double* dm_dev, double* rel,
            const helm_solve_opts& o) {
    const helm_model* m = st->m;
    const size_t np = (size_t)m->Px * m->Pz;
    DBuf r, p, hp, part;
    TRY_ALLOC(r, sizeof(double) * np, s);
    TRY_ALLOC(p, sizeof(double) * np, s);
    TRY_ALLOC(hp, sizeof(double) * np, s);
    TRY_ALLOC(part, sizeof(double) * dot_blocks(np), s);
    HELM_CUDA_TRY(cudaMemsetAsync(dm_dev, 0, sizeof(double) * np, s));
    HELM_CUDA_TRY(cudaMemsetAsync(r.p, 0, sizeof(double) * np, s));
    launch_axpby(-1.0, g_dev, 0.0, r.as<double>(), np, s);                 // r = -g
    HELM_CUDA_TRY(cudaMemcpyAsync(p.p, r.p, sizeof(double) * np, cudaMemcpyDeviceToDevice, s));
    double rr = 0.0;
    int rc = dev_dot(r.as<double>(), r.as<double>(), np, part, s, &rr);
    if (rc != HELM_OK) return rc;
    const double g0 = std::sqrt(rr);
    if (rel) rel[0] = 1.0;
    int status = HELM_OK;
    for (int k = 0; k < iters; ++k) {
        if (!(rr > 0.0)) { if (rel) for (int q = k + 1; q <= iters; ++q) rel[q] = 0.0; break; }
        rc = gn_hvp(st, s, p.as<double>(), hp.as<double>(), o, nullptr);
        if (rc == HELM_E_NOT_CONVERGED) status = rc;
        else if (rc != HELM_OK) return rc;
        double php = 0.0;
        if ((rc = dev_dot(p.as<double>(), hp.as<double>(), np, part, s, &php)) != HELM_OK) return rc;
        if (!(php > 0.0)) { set_last_error("Gauss-Newton Hessian not positive along the search direction"); return HELM_E_INVALID; }
        const double alpha = rr / php;
        launch_axpby(alpha, p.as<double>(), 1.0, dm_dev, np, s);          // dm += alpha p
        launch_axpby(-alpha, hp.as<double>(), 1.0, r.as<double>(), np, s); // r -= alpha H p
        double rr_new = 0.0;
        if ((rc = dev_dot(r.as<double>(), r.as<double>(), np, part, s, &rr_new)) != HELM_OK) return rc;
        if (rel) rel[k + 1] = g0 > 0.0 ? std::sqrt(rr_new) / g0 : 0.0;
        launch_axpby(1.0, r.as<double>(), rr_new / rr, p.as<double>(), np, s);   // p = r + beta p
        rr = rr_new;
    }
    HELM_CUDA_TRY(cudaGetLastError());
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    return status;
}

void fwi_free(FwiState* st) {
    if (!st) return;
    if (st->u64) cudaFree(st->u64);
    if (st->resid) cudaFree(st->resid);
    if (st->drec) cudaFree(st->drec);
    if (st->dw2) cudaFree(st->dw2);
    delete st;
}

}  // namespace helm

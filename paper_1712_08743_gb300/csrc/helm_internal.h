// helm_internal.h - host-side structures and kernel launchers shared by the
// solver, the C ABI and the serving scheduler.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "helm.h"
#include "helm_common.cuh"

namespace helm {

constexpr int kCoarseMaxPoints = 128;   // coarsening stops once a level has this few nodes
constexpr int kCoarseHardMax = 256;     // largest coarsest level the dense inverse accepts
constexpr int kMaxRestart = 64;

// One multigrid level as the kernels see it: dims, (h_l / h_0)^2, and the
// squared slowness on that level (coarse levels take it by injection from node
// (2I+1, 2K+1)). Right-hand side b reads model b * mstride / n: mstride = 0
// when every right-hand side shares one model, n for one model per RHS. The
// per-RHS factor (h_0 omega_b)^2 is passed separately.
struct LevelDev {
    int nx, nz;
    double h2;
    const void* m2;   // float* or double*, per the kernel's precision
    size_t mstride;
};

struct Level {
    int nx = 0, nz = 0;
    double h = 0;
    float* m2f = nullptr;
    double* m2d = nullptr;
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
    double* m_pad = nullptr;              // device [nmodels][nz][nx] slowness (float64)
    double msq_sum = 0;                   // sum of m^2 over the physical cells
    std::vector<helm::Level> lv;          // lv[0] is the padded fine grid
    size_t n() const { return (size_t)nx * nz; }
};

namespace helm {

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
    return d;
}

// Kernel launchers (helm_kernels.cu). All run on `s`; none synchronises.
// `st` may be null where noted; vectors are [nrhs][level n] interleaved complex.
void launch_pad_model(const double* m_phys, int Px, int Pz, int npml, int nmodels, double* m_pad, float* m2f,
                      double* m2d, cudaStream_t s);
void launch_inject(const Level& fine, const Level& coarse, int nmodels, cudaStream_t s);
void launch_sumsq(const double* a, size_t count, double* out, cudaStream_t s);

template <typename T>
void launch_apply(const LevelDev& L0, int npml, double amax, const double* w2, const T* u, T* y,
                  T scale, int nrhs, cudaStream_t s);

// Outer FP64 residual r = f - A u; TI = precision of the inner right-hand side.
template <typename TI>
void launch_resid64(const LevelDev& L0, int npml, double amax, const double* w2, const double* f,
                    const double* u, TI* rin, double* partials, int pstride, RhsState* st,
                    double tol, double inner_floor, int first, int nrhs, cudaStream_t s);
template <typename TI>
void launch_refine(const TI* x, double* u, const RhsState* st, size_t n, int nrhs, cudaStream_t s);

template <typename T>
void launch_bicg_init(const T* b, T* x, T* r, T* rh, T* p, T* v, double* partials, int pstride,
                      RhsState* st, int* nactive, size_t n, int nrhs, cudaStream_t s);
template <typename T>
void launch_bicg_p(const T* r, T* p, const T* v, const RhsState* st, size_t n, int nrhs, cudaStream_t s);
template <typename T>
void launch_bicg_s(const T* r, const T* v, T* sv, const RhsState* st, size_t n, int nrhs, cudaStream_t s);
template <typename T>
void launch_bicg_xr(T* x, const T* ph, const T* sh, const T* sv, const T* t, const T* rh, T* r,
                    double* partials, int pstride, RhsState* st, int* nactive, size_t n, int nrhs,
                    cudaStream_t s);

// V-cycle pieces
template <typename T>
void launch_restrict(const LevelDev& Lf, const LevelDev& Lc, const double* w2, double b1, double b2,
                     double wj, const T* f, T* fc, const RhsState* st, int nrhs, cudaStream_t s);
// mode 0: out = smoothed correction; 1: out = p^, y = A p^, alpha = rho/<rh, y>;
// 2: out = s^, y = A s^, omega = <y, s>/<y, y>.
template <typename T>
void launch_prolong(int mode, const LevelDev& Lf, const LevelDev& Lc, int npml, double amax,
                    const double* w2, double b1, double b2, double wj, const T* f, const T* ec, T* out,
                    T* y, const T* aux, double* partials, int pstride, RhsState* st, int nrhs,
                    cudaStream_t s);
template <typename T>
void launch_coarse(int n, const T* minv, const int* slot, const T* fL, T* eL, const RhsState* st,
                   int nrhs, cudaStream_t s);
void launch_coarse_invert(const LevelDev& Lc, const double* w2_slots, const int* mod_slots, int nslots,
                          double b1, double b2, double2* work, float2* minv_f, double2* minv_d, cudaStream_t s);

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
void launch_fold(const double* g_pad, const double* m_pad, int Px, int Pz, int npml, double lam,
                 double* g, cudaStream_t s);

}  // namespace helm

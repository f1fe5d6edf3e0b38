// helm_solver.h - entry points of the batched solver used by the C ABI and the
// serving scheduler.
#pragma once

#include "helm_internal.h"

namespace helm {

const char* last_error();
void count_launches(unsigned long long k);   // kernels launched by this library (profiling)
unsigned long long launches();

// Solves A u_b = f_b (grid-scaled, f64 device [nrhs][n] c128) for every right-hand
// side b; h_w2[b] = (h_b omega_b)^2 on the host, h_b the fine spacing of its model
// and omega_b its angular frequency. u64 is a device [nrhs][n] c128 output.
// Synchronous on `s`.
int solve_batch(const helm_model* m, cudaStream_t s, int nrhs, const double* h_w2, const double* f64, double* u64,
                const helm_solve_opts& o, helm_solve_stats* stats);

// Device bytes a batch of nrhs solves on an nx x nz grid needs (upper estimate).
size_t solve_bytes(int nx, int nz, int extra, int nrhs, int precision);

int vcycle_once(const helm_model* m, cudaStream_t s, int nrhs, const double* h_w2, double b1, double b2, double wj,
                int coarse, const float* r, float* z);

// Misfit (Eq. 4) and its gradient (Eq. 7), split so that an autograd backward
// runs the adjoint solves: fwi_forward keeps the wavefields and data residuals
// on the device in a FwiState; fwi_backward consumes them.
struct FwiState {
    const helm_model* m = nullptr;
    int nrhs = 0, nrec = 0;
    double lam = 0;
    std::vector<double> w2, hw2;
    double* u64 = nullptr;    // device [nrhs][n] c128 forward wavefields
    double* resid = nullptr;  // device [nrhs][nrec] c128 data residuals P u - d_obs
    int* drec = nullptr;      // device [nrec] flat receiver nodes
    double* dw2 = nullptr;    // device [nrhs] omega^2
};
int fwi_forward(const helm_model* m, cudaStream_t s, int nfreq, const double* omega, int nshot, const int* src_flat_h,
                int nrec, const int* rec_flat_h, const double* d_obs_dev, double lam, double* J_out, double* d_cal_dev,
                const helm_solve_opts& o, helm_solve_stats* stats, FwiState** out);
int fwi_backward(FwiState* st, cudaStream_t s, double* grad_dev, const helm_solve_opts& o, helm_solve_stats* stats);
void fwi_free(FwiState* st);
// Gauss-Newton Hessian-vector product and step (Eq. 8 without its second term, Eq. 9); device vectors
// of the physical model size. stats (gn_hvp): [2 nrhs], Born solves then adjoint solves.
int gn_hvp(FwiState* st, cudaStream_t s, const double* dm_dev, double* hdm_dev, const helm_solve_opts& o,
           helm_solve_stats* stats);
int gn_step(FwiState* st, cudaStream_t s, const double* g_dev, int iters, double* dm_dev, double* rel,
            const helm_solve_opts& o);

int coarsest_points(const helm_model* m);

// One application of the multigrid preconditioner z ~ M^{-1} in (V-cycle above
// level lf, F-cycle from lf, levels >= lt in the shared-memory tail kernel).
// f[l], e[l] (l >= 1): per-level right-hand side and correction buffers
// [nrhs][n_l]. mode as launch_prolong on the finest level.
struct MgCall {
    const double* w2;       // (h omega)^2 per RHS, device, FP64
    const float* w2f;       // the same in FP32 (for the complex64 kernels)
    double b1, b2, wj;
    RhsState* st;           // nullable
    int nrhs;
    cudaStream_t s;
    const void* minv;       // coarsest dense inverses in the kernel's precision
    const int* slot;
    double* partials;       // finest-level dot reductions (modes 1, 2)
    int pstride;
    int lf;                 // first level of the F-cycle (fcycle_level)
    int ld = 0;             // > 0: this level is solved exactly by its dense inverse (minv), 0: the tail path
    const int* grp = nullptr;   // dense path: groups of consecutive right-hand sides sharing a slot
    int ngroups = 0, maxg = 0;
    const FcArgs* fca = nullptr;   // non-null: the cycle at level fca_level runs as the persistent kernel
    int fca_level = 0, fca_grid = 0;
};
// Fills *fa for the persistent F-cycle kernel of a complex64 batch (levels
// c.lf .. c.ld) when it applies: the dense path is on, coarse is HELM_COARSE_AUTO,
// nrhs <= kFcMaxRhs and the cooperative grid fits; returns its grid size, or 0.
// f, e: the batch's level vectors; bar, err: one device counter and flag.
int fcycle_setup(const helm_model* m, const MgCall& c, int coarse, float* const* f, float* const* e,
                 float* const* g, unsigned* bar, int* err, FcArgs* fa);
// First level of the F-cycle for a batch with grid-scaled (h omega_b)^2 = h_w2[b]:
// the first level l >= 1 whose spacing 2^l h gives k h >= kFcycleKh for the
// shortest wavelength of the lowest frequency (omega_min 2^l h m_max >= 0.7,
// fewer than about 9 nodes per wavelength), and no later than the first level
// with at most kFcycleMaxPoints nodes.
int fcycle_level(const helm_model* m, const double* h_w2, int nrhs);
template <typename T>
struct MgLevels {
    T* f[kMaxLevels];
    T* e[kMaxLevels];
    T* g[kMaxLevels];   // right-hand side of an F-cycle's second coarse correction (levels 2 .. top - 1)
};
template <typename T>
void mg_apply(const helm_model* m, const MgCall& c, const MgLevels<T>& B, const T* in, T* out, int mode, T* y,
              const T* aux);
int mg_kernels_per_apply(const helm_model* m, bool dbl, int lf, int ld, int fl = 0, int nrhs = 1);

int autotune(helm_model* m, cudaStream_t s, int nrhs, double hw2, int reps, int* out);
int time_kernel(const helm_model* m, cudaStream_t s, int kernel, int nrhs, double hw2, int reps, double* ms,
                double* bytes);

// density (nullable, host [Pz][Px], nmodels == 1 only): the variable-density operator of Eq. 1
int create_model(helm_ctx* ctx, cudaStream_t s, int Px, int Pz, double h, const double* slowness, int nmodels,
                 int npml, double alpha_max, helm_model** out, const double* density = nullptr);

}  // namespace helm

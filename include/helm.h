/*
 * helm.h - C ABI of the GB300 shifted-Laplace Helmholtz solver and FWI gradient.
 *
 * The library solves the 2D constant-density damped Helmholtz equation of the
 * paper (Kazemi, "Application of shifted-Laplace preconditioners for
 * heterogeneous Helmholtz equation - part 2: Full waveform inversion"):
 *
 *     -Laplace(u) - omega^2 m^2 (1 - j alpha) u = f            (Eq. 2)
 *     B u = f                                                  (Eq. 3)
 *
 * with m = 1/c the real slowness, alpha the damping of an absorbing layer, by a
 * Krylov method (BiCGSTAB, or flexible GMRES) preconditioned with the
 * shifted-Laplace operator M = -Laplace - (beta1 - j beta2) omega^2 m^2 that a
 * geometric multigrid V-cycle inverts approximately ("Full waveform inversion
 * in the space-frequency domain", the paragraph after Eq. 9). It also evaluates
 * the misfit of Eq. 4 and its gradient (Eq. 7) by adjoint solves.
 *
 * Discretisation (the paper says only "finite difference"): standard 5-point
 * Laplacian on a uniform grid, spacing h in x and z; homogeneous Dirichlet
 * ghosts one node outside the padded grid; an npml-node damping layer on all
 * four sides with alpha = alpha_max (d/npml)^2 at depth d nodes into the layer
 * (max over the axes in corners); the slowness in the layer copies the nearest
 * physical cell. A unit point source is f = 1/h^2 at its node.
 *
 * Conventions for every call
 *  - Return value: a helm_status. Nothing throws across the ABI; nothing traps
 *    or aborts on the device. helm_strerror() names a status.
 *  - Layout: row-major [z][x], x fastest. Complex numbers are interleaved
 *    (re, im) pairs: C99 double _Complex / torch.complex128 for "c128", float
 *    pairs / torch.complex64 for "c64".
 *  - Grids: Px x Pz physical nodes; the padded grid used for fields is
 *    nx = Px + 2 npml by nz = Pz + 2 npml. Source and receiver indices are
 *    physical node indices (0-based, 0 <= ix < Px, 0 <= iz < Pz).
 *  - Ownership: the caller owns every buffer it passes; the library copies
 *    what it needs. Handles are freed by their destroy call. A served result
 *    stays owned by the library until helm_release().
 *  - Host or device pointers: field arguments are host pointers unless
 *    opts->device_ptrs is set, in which case they are device pointers on the
 *    context's device, read and written in order on the context's stream.
 *  - Threads: a helm_ctx and its models may be used by one host thread at a
 *    time, except helm_submit/helm_poll/helm_release, which are thread-safe.
 */
#ifndef HELM_H
#define HELM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct helm_ctx helm_ctx;
typedef struct helm_model helm_model;

typedef enum {
    HELM_OK = 0,
    HELM_PENDING = 1,          /* helm_poll: request not finished yet */
    HELM_E_INVALID = -1,       /* bad argument (size, index, NaN, null) */
    HELM_E_NOMEM = -2,         /* device allocation failed / admission refused */
    HELM_E_NOT_CONVERGED = -3, /* tolerance not reached in max_it; best iterate returned */
    HELM_E_CUDA = -4,          /* a CUDA call failed */
    HELM_E_TIMEOUT = -5,       /* helm_poll: timeout_ms elapsed */
    HELM_E_BUSY = -6           /* serving queue full */
} helm_status;

typedef enum {
    HELM_PREC_MIXED = 0, /* complex64 stencil, V-cycle and Krylov; FP64 true residual + refinement */
    HELM_PREC_FP64 = 1,  /* everything in complex128 (the plain FP64 baseline) */
    HELM_PREC_FP32 = 2   /* complex64 only, one inner solve, no refinement */
} helm_precision;

typedef enum { HELM_KRYLOV_BICGSTAB = 0, HELM_KRYLOV_FGMRES = 1 } helm_krylov;

/* Preconditioner of the Krylov solve: the shifted-Laplace operator M inverted
 * approximately by one multigrid cycle, or none (plain BiCGSTAB / GMRES on
 * Eq. 3, for the comparison the paper's examples make). */
typedef enum { HELM_PRECOND_MG = 0, HELM_PRECOND_NONE = 1 } helm_precond;

/* Gram-Schmidt of the FGMRES Arnoldi step (classical, on the stored basis):
 * a second pass on every step (CGS2), none (one pass), or a second pass only
 * where the first removed more than 1 - 1/sqrt(2) of the new vector's norm
 * (the Daniel-Gragg-Kaufman-Stewart test). The FP64 outer refinement recomputes
 * the true residual after every cycle, so one pass only loses inner accuracy
 * where the basis loses orthogonality within a cycle. */
typedef enum { HELM_REORTH_ALWAYS = 0, HELM_REORTH_NEVER = 1, HELM_REORTH_IFNEEDED = 2 } helm_reorth;

/* Coarse end of the multigrid cycle; all are readings of "approximately invert
 * the shifted Laplacian" (the paragraph after Eq. 9) and change the iteration
 * count, not the answer.
 *  - HELM_COARSE_DENSE: the first level with at most 1200 nodes is solved
 *    exactly by its dense inverse (computed once per solve for each distinct
 *    model and frequency by block Gauss-Jordan, applied by a matrix-vector
 *    kernel); the cycle above it runs one kernel launch per step (for batches
 *    of at most 16 right-hand sides two consecutive prolongations share one
 *    launch). It needs
 *    beta2 != 0, which keeps every pivot away from zero, and falls back to the
 *    tail otherwise.
 *  - HELM_COARSE_TAIL: the levels from the first with at most 2048 (complex64)
 *    or 1024 (complex128) nodes down to the coarsest run as an F- or V-cycle in
 *    one block per right-hand side, in shared memory, with a dense solve of the
 *    coarsest level only.
 *  - HELM_COARSE_FUSED: as DENSE, with the F-cycle part (from its start level
 *    down to the dense level) in one persistent cooperative kernel with a grid
 *    barrier between steps (complex64 batches of at most 8 right-hand sides;
 *    otherwise as DENSE). Same numbers as DENSE to rounding.
 *  - HELM_COARSE_AUTO (default): DENSE for batches of at most 16 right-hand
 *    sides, TAIL for larger ones (there the tail's one launch per cycle does the
 *    coarse levels of every right-hand side at once). */
typedef enum { HELM_COARSE_AUTO = 0, HELM_COARSE_TAIL = 1, HELM_COARSE_DENSE = 2, HELM_COARSE_FUSED = 3 } helm_coarse;

typedef struct {
    double tol;          /* stop at ||f - B u||_2 / ||f||_2 <= tol, residual formed in FP64 */
    int max_it;          /* cap on preconditioned Krylov iterations per right-hand side */
    int krylov;          /* helm_krylov */
    int restart;         /* FGMRES restart length (<= 32) */
    int precision;       /* helm_precision */
    double beta1;        /* shift of M: -Laplace - (beta1 - j beta2) omega^2 m^2 */
    double beta2;
    double omega_jacobi; /* damped-Jacobi weight of the V-cycle smoother */
    double inner_tol;    /* HELM_PREC_MIXED: relative reduction asked of each inner solve */
    int max_outer;       /* HELM_PREC_MIXED: cap on refinement steps */
    int check_every;     /* host convergence poll interval, in Krylov iterations */
    int device_ptrs;     /* 1: f / u_out / gradient buffers are device pointers */
    int use_graphs;      /* 1: replay the iteration body as a CUDA graph */
    int precond;         /* helm_precond: the shifted-Laplace multigrid (default) or none (ablation) */
    int reorth;          /* helm_reorth: FGMRES Gram-Schmidt passes (default HELM_REORTH_ALWAYS) */
    int coarse;          /* helm_coarse: coarse end of the multigrid cycle (default HELM_COARSE_AUTO) */
} helm_solve_opts;

typedef struct {
    int iters;        /* Krylov iterations used */
    int outer_its;    /* FP64 refinement steps */
    int converged;    /* 1 if relres <= tol */
    double relres;    /* final ||f - B u|| / ||f||, computed in FP64 */
    int dense_level;  /* multigrid level solved by its dense inverse (0: the shared-memory tail ran) */
    int shift_switched; /* 1 if the solve stalled and continued with the shift (1, 1) (see helm_solve) */
} helm_solve_stats;

/* Fills *opts with the defaults: tol 1e-6, max_it 5000, BiCGSTAB, restart 30,
 * mixed precision, beta = (1, 0.5), omega_jacobi 0.5, inner_tol 1e-2,
 * max_outer 20, check_every 10, host pointers, graphs on, multigrid preconditioner,
 * two Gram-Schmidt passes, HELM_COARSE_AUTO. */
void helm_default_opts(helm_solve_opts* opts);

const char* helm_strerror(int status);
/* Text of the last CUDA or validation error seen by the calling thread. */
const char* helm_last_error(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (graph replays counted per kernel node); a profiling aid with no counterpart
 * in the paper. */
uint64_t helm_launch_count(void);

/* Creates a context on CUDA device `device`. `cuda_stream` (a cudaStream_t,
 * nullable) is the stream every call of this context runs on; NULL makes the
 * library create its own non-blocking stream. */
int helm_ctx_create(int device, void* cuda_stream, helm_ctx** out);
void helm_ctx_destroy(helm_ctx* ctx);

/* Model setup (Eq. 2): copies the physical slowness m = 1/c [Pz][Px] (host,
 * float64, all > 0) to the device, pads it into the npml-node damping layer by
 * edge replication and builds the multigrid hierarchy (coarse slowness by
 * injection). h > 0 is the grid spacing in metres; 0 <= alpha_max. */
int helm_create_model(helm_ctx* ctx, int Px, int Pz, double h, const double* slowness,
                      int npml, double alpha_max, helm_model** out);

/* Model setup for the variable-density operator of Eq. 1,
 * -div(rho grad u) - omega^2 m^2 (1 - j alpha) u = f, with rho as the paper
 * writes it (multiplying the gradient; pass 1/density for the acoustic form).
 * density: host float64 [Pz][Px], all > 0, padded into the layer like the
 * slowness; the operator is the 5-point flux form with the harmonic mean of the
 * two nodes' densities on each edge (an edge to a node outside the grid takes
 * the node's own density), and the shifted-Laplace preconditioner and its
 * Galerkin hierarchy are built from the same form. density = NULL is
 * helm_create_model. Every call that takes a model accepts this one; serving
 * requests carry no density. */
int helm_create_model_rho(helm_ctx* ctx, int Px, int Pz, double h, const double* slowness,
                          const double* density, int npml, double alpha_max, helm_model** out);
void helm_destroy_model(helm_model* model);

/* Padded grid size and number of multigrid levels of a model. */
int helm_model_info(const helm_model* model, int* nx, int* nz, int* nlevels);

/* Forward modelling (Eq. 3): u = B(m, omega_k)^{-1} f_k for k < nrhs, all right-hand
 * sides in one batched launch sequence. omega[k] is the angular frequency (rad/s).
 * Right-hand sides: if f is NULL, a unit point source at physical node
 * (src_ix[k], src_iz[k]); otherwise f is c128 [nrhs][nz][nx] (src_* ignored).
 * u_out: c128 [nrhs][nz][nx] on the padded grid. opts NULL = defaults.
 * stats (nullable): [nrhs]. Returns HELM_E_NOT_CONVERGED if any right-hand side
 * missed tol (u_out then holds the best iterate).
 * Stall guard: with the multigrid preconditioner and a shift other than (1, 1),
 * a right-hand side whose FP64 residual has not halved within 300 Krylov
 * iterations (while above tol) makes the whole batch continue with the
 * paper's shift (1, 1) (stats[k].shift_switched = 1); BiCGSTAB applies the same
 * test to its recursive residual within each inner solve. */
int helm_solve(helm_model* model, int nrhs, const double* omega, const int* src_ix,
               const int* src_iz, const void* f, void* u_out, const helm_solve_opts* opts,
               helm_solve_stats* stats);

/* Misfit and gradient (Eq. 4 and Eq. 7). For each of nfreq angular frequencies
 * and nshot point sources: u = B^{-1} f, r = P u - d_obs (P samples the nrec
 * receiver nodes), lambda = B^{-H} P^T r, and
 *   J = sum |r|^2 + lambda_reg sum_phys m^2,
 *   dJ/dm_i = sum 4 omega^2 m_i Re[(1 - j alpha_i) u_i conj(lambda_i)] + 2 lambda_reg m_i,
 * the layer terms summed onto the physical cell each layer node copies.
 * d_obs: c128 [nfreq][nshot][nrec]. J_out: one double. grad_out: float64 [Pz][Px].
 * d_cal_out (nullable): c128 [nfreq][nshot][nrec], the modelled data P u.
 * d_obs, grad_out and d_cal_out follow opts->device_ptrs. stats (nullable):
 * [2 * nfreq * nshot], forward solves then adjoint solves. */
int helm_adjoint_gradient(helm_model* model, int nfreq, const double* omega, int nshot,
                          const int* src_ix, const int* src_iz, int nrec, const int* rec_ix,
                          const int* rec_iz, const void* d_obs, double lambda_reg, double* J_out,
                          double* grad_out, void* d_cal_out, const helm_solve_opts* opts,
                          helm_solve_stats* stats);

/* The two halves of helm_adjoint_gradient, for an autograd backward that runs
 * the adjoint solves separately. helm_fwi_forward does the forward solves, the
 * data residuals and J (same arguments as helm_adjoint_gradient; stats
 * [nfreq * nshot]) and returns *state, which keeps the wavefields and residuals
 * on the device. helm_fwi_backward runs the adjoint solves and writes the
 * gradient (grad_out float64 [Pz][Px], following opts->device_ptrs; stats
 * [nfreq * nshot]); it may be called more than once. helm_fwi_state_destroy
 * frees the state; the model must outlive it. */
typedef struct helm_fwi_state helm_fwi_state;
int helm_fwi_forward(helm_model* model, int nfreq, const double* omega, int nshot, const int* src_ix,
                     const int* src_iz, int nrec, const int* rec_ix, const int* rec_iz, const void* d_obs,
                     double lambda_reg, double* J_out, void* d_cal_out, const helm_solve_opts* opts,
                     helm_solve_stats* stats, helm_fwi_state** state);
int helm_fwi_backward(helm_fwi_state* state, double* grad_out, const helm_solve_opts* opts,
                      helm_solve_stats* stats);
void helm_fwi_state_destroy(helm_fwi_state* state);

/* Gauss-Newton Hessian-vector product (Eq. 8 without its second term, the
 * approximation Eq. 9 uses): hdm_out = 2 Re[Jac^H Jac dm] + 2 lambda_reg dm,
 * with Jac the Jacobian of the receiver data P u with respect to the physical
 * slowness, at the model, acquisition and wavefields of `state` (from
 * helm_fwi_forward; lambda_reg is the state's). Per shot and frequency it runs
 * one Born solve B du = 2 omega^2 m (1 - j alpha) u (E dm) and one adjoint solve
 * with the sampled du as data, on the same solver and options as helm_solve.
 * dm, hdm_out: float64 [Pz][Px], host or device following opts->device_ptrs;
 * stats (nullable): [2 nfreq nshot], Born solves then adjoint solves. The
 * result is symmetric in dm and positive definite for lambda_reg > 0. Returns
 * HELM_E_NOT_CONVERGED (result still written) if a solve missed its tolerance. */
int helm_gn_hvp(helm_fwi_state* state, const double* dm, double* hdm_out, const helm_solve_opts* opts,
                helm_solve_stats* stats);

/* One Gauss-Newton step (Eq. 9): dm_out = -H^{-1} grad by cg_iters (1..1000)
 * conjugate-gradient iterations from zero, each one helm_gn_hvp. grad: the
 * gradient at the state's model (helm_fwi_backward); grad, dm_out float64
 * [Pz][Px] following opts->device_ptrs. cg_rel_out (host, nullable):
 * [cg_iters + 1] relative residuals ||grad + H dm_k|| / ||grad||. Needs
 * lambda_reg > 0 (HELM_E_INVALID otherwise). */
int helm_gn_step(helm_fwi_state* state, const double* grad, int cg_iters, double* dm_out, double* cg_rel_out,
                 const helm_solve_opts* opts);

/* Gauss-Newton full-waveform inversion loop (Eq. 4-9 repeated, the way the
 * paper's examples run it). The frequencies are inverted either all at once
 * (HELM_FWI_SIMULTANEOUS, the paper's 1D example) or one at a time from the
 * lowest up, each starting from the model the previous one ended with
 * (HELM_FWI_SEQUENTIAL, the paper's 2D example). Every iteration of a group:
 * forward solves and J at the current model, adjoint solves and the gradient
 * (Eq. 7), the Gauss-Newton step dm = -H^{-1} grad by cg_iters CG iterations
 * (Eq. 9, helm_gn_step), then a backtracking line search that the paper does
 * not print: the trial m + t dm, clipped to [m_lo, m_hi], is accepted at the
 * first t in 1, 1/2, ... (at most max_halvings halvings) whose J is below the
 * current J; if none is, the group ends early. The accepted trial's forward
 * solves serve the next iteration. */
typedef enum { HELM_FWI_SIMULTANEOUS = 0, HELM_FWI_SEQUENTIAL = 1 } helm_fwi_strategy;
typedef struct {
    int strategy;       /* helm_fwi_strategy */
    int gn_iters;       /* Gauss-Newton iterations per frequency group, >= 1 */
    int cg_iters;       /* CG iterations per Gauss-Newton step, 1..1000 */
    int max_halvings;   /* line-search halvings, 0..30 (0: the full step or nothing) */
    double m_lo, m_hi;  /* slowness bounds of every trial model, 0 < m_lo <= m_hi */
} helm_fwi_opts;
/* Called after every accepted iteration (and once per group before its first):
 * group index, iteration (0 = the group's starting model), the model m (host,
 * float64 [Pz][Px], valid during the call) and its misfit J over the group's
 * frequencies. */
typedef void (*helm_fwi_checkpoint)(int group, int iter, const double* m, double J, void* user);
/*  - m0: starting slowness, host float64 [Pz][Px]; m_out: host float64 [Pz][Px],
 *    the final model (may alias m0).
 *  - omega [nfreq], sources, receivers and lambda_reg as helm_adjoint_gradient;
 *    d_obs: host c128 [nfreq][nshot][nrec].
 *  - J_hist (nullable): host float64, room for ngroups * (gn_iters + 1) values
 *    (ngroups = 1 or nfreq); gets each group's J at its start and after every
 *    accepted iteration, in order; *n_hist (nullable) their count.
 *  - checkpoint (nullable) with its user pointer.
 *  - opts: the solves' options (device_ptrs must be 0; NULL = defaults).
 * Returns HELM_E_INVALID for bad arguments, a solve's error status otherwise
 * (m_out then holds the last accepted model). lambda_reg must be > 0. */
int helm_fwi_run(helm_ctx* ctx, int Px, int Pz, double h, int npml, double alpha_max, const double* m0,
                 int nfreq, const double* omega, int nshot, const int* src_ix, const int* src_iz, int nrec,
                 const int* rec_ix, const int* rec_iz, const void* d_obs, double lambda_reg,
                 const helm_fwi_opts* fwi_opts, const helm_solve_opts* opts, double* m_out, double* J_hist,
                 int* n_hist, helm_fwi_checkpoint checkpoint, void* user);

/* Operator application y = B(m, omega_k) u_k (Eq. 3) for parity checks and
 * bandwidth measurement. precision HELM_PREC_FP64: u, y c128; otherwise c64.
 * [nrhs][nz][nx] each, following device_ptrs. */
int helm_apply(helm_model* model, int nrhs, const double* omega, int precision, const void* u,
               void* y, int device_ptrs);

/* One application of the multigrid V-cycle that approximates M^{-1} r (the
 * shifted-Laplace preconditioner) on complex64 [nrhs][nz][nx] vectors; for
 * parity checks of the preconditioner against a CPU restatement. beta and
 * omega_jacobi as in helm_solve_opts. */
int helm_vcycle(helm_model* model, int nrhs, const double* omega, double beta1, double beta2,
                double omega_jacobi, const void* r, void* z, int device_ptrs);

/* helm_vcycle with the preconditioner options of a solve: beta1, beta2,
 * omega_jacobi, coarse and device_ptrs are taken from *opts (NULL = defaults);
 * helm_vcycle is this call with the defaults' coarse setting. */
int helm_vcycle_ex(helm_model* model, int nrhs, const double* omega, const helm_solve_opts* opts, const void* r,
                   void* z);

/* Bandwidth measurement of one hot-path kernel (no counterpart in the paper;
 * it feeds the roofline report). Launches `kernel` (helm_kernel_id) `reps`
 * times on library-owned zero-filled vectors of nrhs right-hand sides of this
 * model at angular frequency omega, after three warm-up launches, and returns
 * the mean time per launch in ms (CUDA events on the context's stream) and the
 * algorithmic bytes one launch must move (each operand once; the squared
 * slowness shared by the batch counted once). */
typedef enum {
    HELM_KERNEL_APPLY = 0,    /* y = A u, complex64 */
    HELM_KERNEL_RESTRICT = 1, /* fine-level pre-smooth + residual + full weighting, complex64 */
    HELM_KERNEL_PROLONG = 2,  /* fine-level prolongation + post-smooth + A + dot, complex64 */
    HELM_KERNEL_BICG_XR = 3,  /* BiCGSTAB x and r update with its two dots, complex64 */
    HELM_KERNEL_RESID64 = 4,  /* FP64 true residual r = f - A u */
    HELM_KERNEL_BICG_P = 5,   /* BiCGSTAB p update, complex64 */
    HELM_KERNEL_APPLY64 = 6,  /* y = A u, complex128 */
    HELM_KERNEL_FG_DOTS = 7,  /* FGMRES Gram-Schmidt dot products at Arnoldi step 4 (5 basis vectors), complex64 */
    HELM_KERNEL_FG_AXPY = 8,  /* FGMRES Gram-Schmidt update + per-block norm parts at step 4, complex64 */
    HELM_KERNEL_TAIL = 9,     /* coarse-level tail: one F-cycle over the levels from the first of at most
                                 2048 nodes down to the coarsest, one block per right-hand side, complex64;
                                 bytes = its input and output on the tail's top level */
    HELM_KERNEL_FMA64 = 10    /* FP64 throughput probe (8 independent chains of fused multiply-adds per
                                 thread, 8 blocks of 256 threads per SM); nrhs and omega are ignored and
                                 bytes_per_launch holds the launch's FP64 operations (2 per multiply-add) */
} helm_kernel_id;
int helm_time_kernel(helm_model* model, int kernel, int nrhs, double omega, int reps, double* ms_per_launch,
                     double* bytes_per_launch);

/* Per-kernel profile of this library's launches (no counterpart in the paper;
 * it feeds the roofline report). Between helm_profile_begin() and
 * helm_profile_end() every kernel the library launches, from any thread, is
 * timed with a CUDA event pair on its stream, and solves run without CUDA
 * graphs; the events also keep consecutive launches from overlapping, so the
 * durations are those of serialised launches. helm_profile_end synchronises on
 * the recorded events and writes one entry per (kernel, grid) to out (at most
 * cap; *n_out = the number of entries there are): launches, total ms and the
 * total algorithmic bytes (each operand read or written once, model data
 * shared by a batch counted once). Profiling adds host work per launch; do not
 * time a workload while a session is open. */
typedef struct {
    char name[32];       /* kernel, e.g. "k_restrict_g" */
    int nx, nz;          /* the grid it works on (fine grid of a level transfer; n x 1 for vectors) */
    uint64_t launches;
    double ms;           /* summed event time */
    double bytes;        /* summed algorithmic bytes */
} helm_profile_entry;
int helm_profile_begin(void);
int helm_profile_end(helm_profile_entry* out, int cap, int* n_out);

/* helm_vcycle for callers that cannot allocate device memory (no counterpart in
 * the paper). helm_vcycle allocates its level vectors and the coarsest-level
 * inverse on every call; this variant runs the same kernels, with the same
 * result, on a fixed 64 MiB scratch array compiled into the library (present on
 * every GPU that loads the library until the process exits), for code whose
 * device memory is owned by another allocator or must not grow after start-up.
 * It calls no cudaMalloc, cudaFree or other allocating routine.
 *  - r, z: device pointers, complex64 [nrhs][nz][nx], on the context's device;
 *    the call is synchronous on the context's stream. nrhs <= 256.
 *  - Sizes whose level vectors and coarsest-level inverses do not fit in the
 *    64 MiB return HELM_E_INVALID (helm_last_error() gives the bytes needed).
 *  - The first call on a device looks up the scratch array's device address
 *    (cudaGetSymbolAddress) and keeps it for the process; make that first call
 *    before any stream capture. A cudaDeviceReset of that device invalidates
 *    the kept address: do not call this entry point on that device afterwards
 *    (reload the library instead).
 *  - Every call on a device shares the one array and leaves its contents
 *    behind; each call writes every byte it reads, so nothing needs clearing.
 *    Calls that overlap on the GPU (other threads or streams) race: serialise
 *    them. */
int helm_vcycle_noalloc(helm_model* model, int nrhs, const double* omega, double beta1, double beta2,
                        double omega_jacobi, const void* r, void* z);

/* Autotuner (no counterpart in the paper): times the tile shapes of each complex64
 * multigrid kernel on the grid levels of this model for nrhs right-hand sides at
 * angular frequency omega, keeps the fastest in the model, and writes the choices
 * to tiles_out (nullable): int[48], restriction tiles per level then prolongation
 * tiles per level. Galerkin levels: restriction 0..5 (coarse tiles 8x8, 16x8,
 * 32x4, 8x16, 8x8 on two threads per node, 8x16 on two threads per node), prolongation 0..4 (fine tiles
 * 16x8, 32x8, 64x4, 32x16, 128x2);
 * the finest level's prolongation 0..1 (row segments of 16 or 32 rows); 1 is
 * the default everywhere. helm_set_tiles applies a stored choice. Tile shapes
 * change the speed, not the arithmetic of a node (dot products may sum in
 * another order). */
int helm_autotune(helm_model* model, int nrhs, double omega, int* tiles_out);
int helm_set_tiles(helm_model* model, const int* tiles);

/* ---------------------------------------------------------------- serving
 * Continuous batching: requests enter a host queue; a scheduler thread admits
 * them while free device memory (minus a reserve) allows, groups requests of the
 * same grid shape and precision into one batched slot, and runs slots
 * concurrently on their own streams. Each result is the same as a lone
 * helm_solve of that request, within the solve tolerance. */
typedef struct {
    int Px, Pz;
    double h;
    const double* slowness; /* host [Pz][Px], copied at submit */
    int npml;
    double alpha_max;
    double omega;           /* angular frequency */
    int src_ix, src_iz;     /* physical node of a unit point source */
    helm_solve_opts opts;   /* device_ptrs must be 0 */
} helm_request;

typedef struct {
    const void* u;          /* c128 [nz][nx] host buffer owned by the library until helm_release */
    int nx, nz;
    int status;             /* helm_status of the solve */
    helm_solve_stats stats;
    double latency_ms;      /* submit to completion */
    double queue_ms;        /* submit to admission */
    int batch_size;         /* requests in the slot this one ran in */
} helm_result;

/* Starts the scheduler (first call) and enqueues a request; *ticket names it. */
int helm_submit(helm_ctx* ctx, const helm_request* req, uint64_t* ticket);
/* Waits up to timeout_ms (0 = just look) for a request. A negative timeout waits
 * on the host (a condition variable; no GPU work waits) until the request has
 * finished, which every request does: its solve is bounded by max_it and
 * max_outer, and an admission refusal finishes it with HELM_E_NOMEM.
 * HELM_OK fills *result; HELM_PENDING / HELM_E_TIMEOUT leave it untouched. */
int helm_poll(helm_ctx* ctx, uint64_t ticket, int timeout_ms, helm_result* result);
/* Frees a finished request's result. */
int helm_release(helm_ctx* ctx, uint64_t ticket);
/* Serving limits: max requests per slot, concurrent slots, device-memory reserve
 * in bytes, and a simulated device-memory budget in bytes (0 = use the real
 * free memory) for admission tests. */
int helm_serve_config(helm_ctx* ctx, int max_batch, int max_slots, uint64_t reserve_bytes,
                      uint64_t budget_bytes);

#ifdef __cplusplus
}
#endif
#endif /* HELM_H */

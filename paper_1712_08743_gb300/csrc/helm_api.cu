// helm_api.cu - the extern "C" boundary declared in include/helm.h: argument
// validation, host<->device marshalling and dispatch to the batched solver.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "helm_internal.h"
#include "helm_solver.h"

using namespace helm;

namespace {

struct DevMem {   // synchronous device allocation for API-level staging
    void* p = nullptr;
    ~DevMem() { if (p) cudaFree(p); }
};

class DeviceGuard {   // makes the context's device current for the call
  public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev_);
        if (prev_ != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != prev_) cudaSetDevice(prev_);
    }

  private:
    int prev_ = 0;
};

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

int check_opts(const helm_solve_opts& o) {
    if (!(o.tol > 0.0) || !std::isfinite(o.tol)) return HELM_E_INVALID;
    if (o.max_it < 1 || o.max_outer < 1 || o.check_every < 1) return HELM_E_INVALID;
    if (o.precision < HELM_PREC_MIXED || o.precision > HELM_PREC_FP32) return HELM_E_INVALID;
    if (o.krylov != HELM_KRYLOV_BICGSTAB && o.krylov != HELM_KRYLOV_FGMRES) return HELM_E_INVALID;
    if (o.restart < 1 || o.restart > kMaxRestart) return HELM_E_INVALID;
    if (!std::isfinite(o.beta1) || !std::isfinite(o.beta2) || !(o.omega_jacobi > 0.0) || o.omega_jacobi > 2.0)
        return HELM_E_INVALID;
    if (!(o.inner_tol > 0.0) || o.inner_tol >= 1.0) return HELM_E_INVALID;
    if (o.precond != HELM_PRECOND_MG && o.precond != HELM_PRECOND_NONE) return HELM_E_INVALID;
    if (o.reorth < HELM_REORTH_ALWAYS || o.reorth > HELM_REORTH_IFNEEDED) return HELM_E_INVALID;
    if (o.coarse < HELM_COARSE_AUTO || o.coarse > HELM_COARSE_FUSED) return HELM_E_INVALID;
    return HELM_OK;
}

}  // namespace

struct helm_fwi_state {
    helm_model* m = nullptr;
    helm::FwiState* st = nullptr;
};

namespace helm {

// Builds a model holding `nmodels` slowness fields of one grid shape (host
// [nmodels][Pz][Px]); nmodels > 1 gives each right-hand side its own model.
int create_model(helm_ctx* ctx, cudaStream_t s, int Px, int Pz, double h, const double* slowness, int nmodels,
                 int npml, double alpha_max, helm_model** out, const double* density) {
    if (!ctx || !out || !slowness || nmodels < 1) return HELM_E_INVALID;
    *out = nullptr;
    if (Px < 1 || Pz < 1 || npml < 0 || !finite_pos(h) || !std::isfinite(alpha_max) || alpha_max < 0.0)
        return HELM_E_INVALID;
    if (density && nmodels != 1) return HELM_E_INVALID;
    const size_t np = (size_t)Px * Pz;
    for (size_t i = 0; i < np * nmodels; ++i)
        if (!finite_pos(slowness[i])) { set_last_error("slowness must be finite and > 0"); return HELM_E_INVALID; }
    if (density)
        for (size_t i = 0; i < np; ++i)
            if (!finite_pos(density[i])) { set_last_error("density must be finite and > 0"); return HELM_E_INVALID; }
    DeviceGuard g(ctx->device);
    helm_model* m = new helm_model();
    m->ctx = ctx;
    m->Px = Px; m->Pz = Pz; m->npml = npml; m->h = h; m->alpha_max = alpha_max;
    m->nx = Px + 2 * npml; m->nz = Pz + 2 * npml;
    m->nmodels = nmodels;
    m->vd = density != nullptr;
    for (int l = 0; l < kMaxLevels; ++l) { m->tile_restrict[l] = 1; m->tile_prolong[l] = 1; }
    // levels: halve per axis while the level is larger than the dense-coarse size
    Level L0; L0.nx = m->nx; L0.nz = m->nz; L0.h = h;
    m->lv.push_back(L0);
    while (m->lv.back().n() > (size_t)kCoarseMaxPoints && m->lv.back().nx >= 4 && m->lv.back().nz >= 4) {
        Level c; c.nx = m->lv.back().nx / 2; c.nz = m->lv.back().nz / 2; c.h = 2.0 * m->lv.back().h;
        m->lv.push_back(c);
    }
    if (m->lv.size() < 2 || m->lv.back().n() > (size_t)kCoarseHardMax) {
        set_last_error("grid shape does not coarsen to a small enough coarsest level");
        delete m;
        return HELM_E_INVALID;
    }
    const int L = (int)m->lv.size() - 1;
    m->lf = L;
    for (int l = 1; l <= L; ++l)
        if (m->lv[l].n() <= (size_t)kFcycleMaxPoints) { m->lf = l; break; }
    for (int l = 1; l <= L; ++l)
        if (m->lv[l].n() <= (size_t)kDenseMaxPoints) { m->ld = l; break; }
    for (size_t i = 0; i < np * (size_t)nmodels; ++i) m->m_max = std::max(m->m_max, slowness[i]);
    for (int d = 0; d < 2; ++d) {
        const size_t cap = d ? (size_t)kTailMaxPoints64 : (size_t)kTailMaxPoints32;
        m->lt[d] = L;
        for (int l = m->lf; l <= L; ++l)
            if (m->lv[l].n() <= cap) { m->lt[d] = l; break; }
        m->tail_smem[d] = tail_smem_bytes(m, m->lt[d], d ? sizeof(double) : sizeof(float));
        if (m->tail_smem[d] > 227u * 1024u) { set_last_error("tail levels exceed shared memory"); delete m; return HELM_E_INVALID; }
    }
    if (L + 1 > kMaxLevels) { set_last_error("too many levels"); delete m; return HELM_E_INVALID; }
    auto fail = [&](cudaError_t e) {
        set_last_error(cudaGetErrorString(e));
        cudaGetLastError();
        helm_destroy_model(m);
        return e == cudaErrorMemoryAllocation ? HELM_E_NOMEM : HELM_E_CUDA;
    };
    cudaError_t e = cudaMalloc(&m->m_pad, sizeof(double) * m->n() * nmodels);
    if (e != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&m->lv[0].m2f, sizeof(float) * m->n() * nmodels)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&m->lv[0].m2d, sizeof(double) * m->n() * nmodels)) != cudaSuccess) return fail(e);
    if (m->vd) {
        Level& L0 = m->lv[0];
        if ((e = cudaMalloc(&L0.rhof, sizeof(float) * 3 * L0.n())) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc(&L0.rhod, sizeof(double) * 3 * L0.n())) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc(&L0.gkf, sizeof(float) * kGalerkinCoefs * L0.n())) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc(&L0.gkd, sizeof(double) * kGalerkinCoefs * L0.n())) != cudaSuccess) return fail(e);
    }
    for (int l = 1; l <= L; ++l) {
        Level& Lv = m->lv[l];
        if ((e = cudaMalloc(&Lv.gkf, sizeof(float) * kGalerkinCoefs * Lv.n() * nmodels)) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc(&Lv.gkd, sizeof(double) * kGalerkinCoefs * Lv.n() * nmodels)) != cudaSuccess) return fail(e);
    }
    std::vector<int> opsf[2], opsv[2];
    for (int d = 0; d < 2; ++d) {
        opsf[d] = tail_schedule(m->lt[d], L, true);
        opsv[d] = tail_schedule(m->lt[d], L, false);
        m->nops_f[d] = (int)opsf[d].size();
        m->nops_v[d] = (int)opsv[d].size();
        if ((e = cudaMalloc(&m->ops_f[d], sizeof(int) * opsf[d].size())) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc(&m->ops_v[d], sizeof(int) * opsv[d].size())) != cudaSuccess) return fail(e);
    }
    DevMem phys, msq;
    if ((e = cudaMalloc(&phys.p, sizeof(double) * np * nmodels)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&msq.p, sizeof(double))) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(phys.p, slowness, sizeof(double) * np * nmodels, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return fail(e);
    for (int d = 0; d < 2; ++d) {
        if ((e = cudaMemcpyAsync(m->ops_f[d], opsf[d].data(), sizeof(int) * opsf[d].size(), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
            return fail(e);
        if ((e = cudaMemcpyAsync(m->ops_v[d], opsv[d].data(), sizeof(int) * opsv[d].size(), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
            return fail(e);
    }
    launch_pad_model(static_cast<double*>(phys.p), Px, Pz, npml, nmodels, m->m_pad, m->lv[0].m2f, m->lv[0].m2d, s);
    DevMem rho_phys;
    if (m->vd) {
        if ((e = cudaMalloc(&rho_phys.p, sizeof(double) * np)) != cudaSuccess) return fail(e);
        if ((e = cudaMemcpyAsync(rho_phys.p, density, sizeof(double) * np, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return fail(e);
        Level& L0 = m->lv[0];
        launch_rho_setup(static_cast<double*>(rho_phys.p), Px, Pz, npml, L0.m2d, L0.rhod, L0.rhof, L0.gkd, L0.gkf, s);
    }
    for (int l = 1; l <= L; ++l) launch_galerkin(m, l, s);
    launch_sumsq(static_cast<double*>(phys.p), np, static_cast<double*>(msq.p), s);
    if ((e = cudaMemcpyAsync(&m->msq_sum, msq.p, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    *out = m;
    return HELM_OK;
}

}  // namespace helm

extern "C" {

void helm_default_opts(helm_solve_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-6;
    o->max_it = 5000;
    o->krylov = HELM_KRYLOV_BICGSTAB;
    o->restart = 30;
    o->precision = HELM_PREC_MIXED;
    o->beta1 = 1.0;
    o->beta2 = 0.5;
    o->omega_jacobi = 0.5;
    o->inner_tol = 1e-2;
    o->max_outer = 20;
    o->check_every = 10;
    o->device_ptrs = 0;
    o->use_graphs = 1;
    o->coarse = HELM_COARSE_AUTO;
}

const char* helm_strerror(int st) {
    switch (st) {
        case HELM_OK: return "ok";
        case HELM_PENDING: return "pending";
        case HELM_E_INVALID: return "invalid argument";
        case HELM_E_NOMEM: return "out of device memory / admission refused";
        case HELM_E_NOT_CONVERGED: return "tolerance not reached within max_it";
        case HELM_E_CUDA: return "CUDA error";
        case HELM_E_TIMEOUT: return "timeout";
        case HELM_E_BUSY: return "queue full";
        default: return "unknown status";
    }
}

const char* helm_last_error(void) { return last_error(); }

uint64_t helm_launch_count(void) { return (uint64_t)launches(); }

int helm_ctx_create(int device, void* cuda_stream, helm_ctx** out) {
    if (!out) return HELM_E_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) { cudaGetLastError(); set_last_error("no CUDA device"); return HELM_E_CUDA; }
    if (device < 0 || device >= ndev) return HELM_E_INVALID;
    HELM_CUDA_TRY(cudaSetDevice(device));
    helm_ctx* c = new helm_ctx();
    c->device = device;
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete c; set_last_error(cudaGetErrorString(e)); return HELM_E_CUDA; }
        c->own_stream = true;
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    *out = c;
    return HELM_OK;
}

void helm_serve_shutdown(helm_ctx* ctx);  // helm_serve.cu

void helm_ctx_destroy(helm_ctx* ctx) {
    if (!ctx) return;
    helm_serve_shutdown(ctx);
    DeviceGuard g(ctx->device);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int helm_create_model(helm_ctx* ctx, int Px, int Pz, double h, const double* slowness, int npml, double alpha_max,
                      helm_model** out) {
    if (!ctx) return HELM_E_INVALID;
    return helm::create_model(ctx, ctx->stream, Px, Pz, h, slowness, 1, npml, alpha_max, out, nullptr);
}

int helm_create_model_rho(helm_ctx* ctx, int Px, int Pz, double h, const double* slowness, const double* density,
                          int npml, double alpha_max, helm_model** out) {
    if (!ctx) return HELM_E_INVALID;
    return helm::create_model(ctx, ctx->stream, Px, Pz, h, slowness, 1, npml, alpha_max, out, density);
}

void helm_destroy_model(helm_model* m) {
    if (!m) return;
    DeviceGuard g(m->ctx->device);
    if (m->m_pad) cudaFree(m->m_pad);
    for (int d = 0; d < 2; ++d) {
        if (m->ops_f[d]) cudaFree(m->ops_f[d]);
        if (m->ops_v[d]) cudaFree(m->ops_v[d]);
    }
    for (auto& L : m->lv) {
        if (L.m2f) cudaFree(L.m2f);
        if (L.m2d) cudaFree(L.m2d);
        if (L.gkf) cudaFree(L.gkf);
        if (L.gkd) cudaFree(L.gkd);
        if (L.rhof) cudaFree(L.rhof);
        if (L.rhod) cudaFree(L.rhod);
    }
    delete m;
}

int helm_model_info(const helm_model* m, int* nx, int* nz, int* nlevels) {
    if (!m) return HELM_E_INVALID;
    if (nx) *nx = m->nx;
    if (nz) *nz = m->nz;
    if (nlevels) *nlevels = (int)m->lv.size();
    return HELM_OK;
}

int helm_solve(helm_model* m, int nrhs, const double* omega, const int* src_ix, const int* src_iz, const void* f,
               void* u_out, const helm_solve_opts* opts, helm_solve_stats* stats) {
    if (!m || nrhs < 1 || !omega || !u_out) return HELM_E_INVALID;
    helm_solve_opts o;
    if (opts) o = *opts; else helm_default_opts(&o);
    if (check_opts(o) != HELM_OK) return HELM_E_INVALID;
    std::vector<double> w2(nrhs);
    for (int b = 0; b < nrhs; ++b) {
        if (!finite_pos(omega[b])) return HELM_E_INVALID;
        w2[b] = m->h * m->h * omega[b] * omega[b];
    }
    std::vector<int> src_flat;
    if (!f) {
        if (!src_ix || !src_iz) return HELM_E_INVALID;
        src_flat.resize(nrhs);
        for (int b = 0; b < nrhs; ++b) {
            if (src_ix[b] < 0 || src_ix[b] >= m->Px || src_iz[b] < 0 || src_iz[b] >= m->Pz) return HELM_E_INVALID;
            src_flat[b] = (src_iz[b] + m->npml) * m->nx + (src_ix[b] + m->npml);
        }
    }
    DeviceGuard g(m->ctx->device);
    cudaStream_t s = m->ctx->stream;
    const size_t n = m->n();
    const size_t fbytes = sizeof(double) * 2 * n * nrhs;
    DevMem f64, u64, dsrc, fin;
    if (cudaMalloc(&f64.p, fbytes) != cudaSuccess) { cudaGetLastError(); return HELM_E_NOMEM; }
    double* u_dev = nullptr;
    if (o.device_ptrs) {
        u_dev = static_cast<double*>(u_out);
    } else {
        if (cudaMalloc(&u64.p, fbytes) != cudaSuccess) { cudaGetLastError(); return HELM_E_NOMEM; }
        u_dev = static_cast<double*>(u64.p);
    }
    if (!f) {
        if (cudaMalloc(&dsrc.p, sizeof(int) * nrhs) != cudaSuccess) { cudaGetLastError(); return HELM_E_NOMEM; }
        HELM_CUDA_TRY(cudaMemcpyAsync(dsrc.p, src_flat.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
        launch_point_rhs(static_cast<double*>(f64.p), static_cast<int*>(dsrc.p), nrhs, n, s);
        count_launches(1);
    } else {
        const double* fsrc = static_cast<const double*>(f);
        if (!o.device_ptrs) {
            if (cudaMalloc(&fin.p, fbytes) != cudaSuccess) { cudaGetLastError(); return HELM_E_NOMEM; }
            HELM_CUDA_TRY(cudaMemcpyAsync(fin.p, f, fbytes, cudaMemcpyHostToDevice, s));
            fsrc = static_cast<const double*>(fin.p);
        }
        launch_scale_rhs(fsrc, static_cast<double*>(f64.p), m->h * m->h, n * nrhs, s);   // grid-scaled h^2 f
        count_launches(1);
    }
    HELM_CUDA_TRY(cudaGetLastError());
    int rc = solve_batch(m, s, nrhs, w2.data(), static_cast<double*>(f64.p), u_dev, o, stats);
    if (rc != HELM_OK && rc != HELM_E_NOT_CONVERGED) return rc;
    if (!o.device_ptrs) {
        HELM_CUDA_TRY(cudaMemcpyAsync(u_out, u_dev, fbytes, cudaMemcpyDeviceToHost, s));
    }
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    return rc;
}

int helm_apply(helm_model* m, int nrhs, const double* omega, int precision, const void* u, void* y, int device_ptrs) {
    if (!m || nrhs < 1 || !omega || !u || !y) return HELM_E_INVALID;
    if (precision < HELM_PREC_MIXED || precision > HELM_PREC_FP32) return HELM_E_INVALID;
    std::vector<double> w2(nrhs);
    for (int b = 0; b < nrhs; ++b) {
        if (!finite_pos(omega[b])) return HELM_E_INVALID;
        w2[b] = m->h * m->h * omega[b] * omega[b];
    }
    DeviceGuard g(m->ctx->device);
    cudaStream_t s = m->ctx->stream;
    const bool dbl = precision == HELM_PREC_FP64;
    const size_t bytes = (dbl ? 16 : 8) * m->n() * nrhs;
    DevMem dw2, du, dy;
    std::vector<float> w2f(w2.begin(), w2.end());
    if (cudaMalloc(&dw2.p, sizeof(double) * nrhs) != cudaSuccess) { cudaGetLastError(); return HELM_E_NOMEM; }
    if (dbl) HELM_CUDA_TRY(cudaMemcpyAsync(dw2.p, w2.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    else HELM_CUDA_TRY(cudaMemcpyAsync(dw2.p, w2f.data(), sizeof(float) * nrhs, cudaMemcpyHostToDevice, s));
    const void* up = u;
    void* yp = y;
    if (!device_ptrs) {
        if (cudaMalloc(&du.p, bytes) != cudaSuccess || cudaMalloc(&dy.p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return HELM_E_NOMEM;
        }
        HELM_CUDA_TRY(cudaMemcpyAsync(du.p, u, bytes, cudaMemcpyHostToDevice, s));
        up = du.p;
        yp = dy.p;
    }
    const double sc = 1.0 / (m->h * m->h);
    if (dbl)
        launch_apply<double>(level_dev(m, 0, true), m->npml, m->alpha_max, static_cast<double*>(dw2.p),
                             static_cast<const double*>(up), static_cast<double*>(yp), sc, nrhs, s);
    else
        launch_apply<float>(level_dev(m, 0, false), m->npml, m->alpha_max, static_cast<float*>(dw2.p),
                            static_cast<const float*>(up), static_cast<float*>(yp), (float)sc, nrhs, s);
    HELM_CUDA_TRY(cudaGetLastError());
    if (!device_ptrs) HELM_CUDA_TRY(cudaMemcpyAsync(y, yp, bytes, cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));   // the host copies above are sources of async copies
    return HELM_OK;
}

int helm_time_kernel(helm_model* m, int kernel, int nrhs, double omega, int reps, double* ms, double* bytes) {
    if (!m || nrhs < 1 || reps < 1 || !finite_pos(omega) || !ms || !bytes) return HELM_E_INVALID;
    DeviceGuard g(m->ctx->device);
    return time_kernel(m, m->ctx->stream, kernel, nrhs, m->h * m->h * omega * omega, reps, ms, bytes);
}

int helm_autotune(helm_model* m, int nrhs, double omega, int* tiles_out) {
    if (!m || nrhs < 1 || !finite_pos(omega)) return HELM_E_INVALID;
    DeviceGuard g(m->ctx->device);
    int tiles[2 * kMaxLevels];
    int rc = autotune(m, m->ctx->stream, nrhs, m->h * m->h * omega * omega, 5, tiles);
    if (rc == HELM_OK && tiles_out) std::memcpy(tiles_out, tiles, sizeof(tiles));
    return rc;
}

int helm_set_tiles(helm_model* m, const int* tiles) {
    if (!m || !tiles) return HELM_E_INVALID;
    for (int k = 0; k < kMaxLevels; ++k)
        if (tiles[k] < 0 || tiles[k] >= kRestrictTiles || tiles[kMaxLevels + k] < 0 ||
            tiles[kMaxLevels + k] >= kProlongTiles || (k == 0 && tiles[kMaxLevels] > 1))
            return HELM_E_INVALID;
    for (int l = 0; l < kMaxLevels; ++l) {
        m->tile_restrict[l] = tiles[l];
        m->tile_prolong[l] = tiles[kMaxLevels + l];
    }
    return HELM_OK;
}

namespace {
int vcycle_call(helm_model* m, int nrhs, const double* omega, double beta1, double beta2, double omega_jacobi,
                int coarse, const void* r, void* z, int device_ptrs) {
    if (!m || nrhs < 1 || !omega || !r || !z) return HELM_E_INVALID;
    if (!std::isfinite(beta1) || !std::isfinite(beta2) || !(omega_jacobi > 0.0)) return HELM_E_INVALID;
    if (coarse < HELM_COARSE_AUTO || coarse > HELM_COARSE_FUSED) return HELM_E_INVALID;
    std::vector<double> w2(nrhs);
    for (int b = 0; b < nrhs; ++b) {
        if (!finite_pos(omega[b])) return HELM_E_INVALID;
        w2[b] = m->h * m->h * omega[b] * omega[b];
    }
    DeviceGuard g(m->ctx->device);
    cudaStream_t s = m->ctx->stream;
    const size_t bytes = 8 * m->n() * nrhs;
    DevMem dr, dz;
    const void* rp = r;
    void* zp = z;
    if (!device_ptrs) {
        if (cudaMalloc(&dr.p, bytes) != cudaSuccess || cudaMalloc(&dz.p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return HELM_E_NOMEM;
        }
        HELM_CUDA_TRY(cudaMemcpyAsync(dr.p, r, bytes, cudaMemcpyHostToDevice, s));
        rp = dr.p;
        zp = dz.p;
    }
    int rc = vcycle_once(m, s, nrhs, w2.data(), beta1, beta2, omega_jacobi, coarse, static_cast<const float*>(rp),
                         static_cast<float*>(zp));
    if (rc != HELM_OK) return rc;
    if (!device_ptrs) HELM_CUDA_TRY(cudaMemcpyAsync(z, zp, bytes, cudaMemcpyDeviceToHost, s));
    HELM_CUDA_TRY(cudaStreamSynchronize(s));
    return HELM_OK;
}
}  // namespace

int helm_vcycle(helm_model* m, int nrhs, const double* omega, double beta1, double beta2, double omega_jacobi,
                const void* r, void* z, int device_ptrs) {
    helm_solve_opts d;
    helm_default_opts(&d);
    return vcycle_call(m, nrhs, omega, beta1, beta2, omega_jacobi, d.coarse, r, z, device_ptrs);
}

int helm_vcycle_ex(helm_model* m, int nrhs, const double* omega, const helm_solve_opts* opts, const void* r,
                   void* z) {
    helm_solve_opts o;
    if (opts) o = *opts; else helm_default_opts(&o);
    return vcycle_call(m, nrhs, omega, o.beta1, o.beta2, o.omega_jacobi, o.coarse, r, z, o.device_ptrs);
}

int helm_fwi_forward(helm_model* m, int nfreq, const double* omega, int nshot, const int* src_ix, const int* src_iz,
                     int nrec, const int* rec_ix, const int* rec_iz, const void* d_obs, double lambda_reg,
                     double* J_out, void* d_cal_out, const helm_solve_opts* opts, helm_solve_stats* stats,
                     helm_fwi_state** state) {
    if (!state) return HELM_E_INVALID;
    *state = nullptr;
    if (!m || nfreq < 1 || nshot < 1 || nrec < 1 || !omega || !src_ix || !src_iz || !rec_ix || !rec_iz || !d_obs ||
        !J_out)
        return HELM_E_INVALID;
    if (!std::isfinite(lambda_reg) || lambda_reg < 0.0) return HELM_E_INVALID;
    helm_solve_opts o;
    if (opts) o = *opts; else helm_default_opts(&o);
    if (check_opts(o) != HELM_OK) return HELM_E_INVALID;
    for (int f = 0; f < nfreq; ++f)
        if (!finite_pos(omega[f])) return HELM_E_INVALID;
    std::vector<int> sf(nshot), rf(nrec);
    for (int k = 0; k < nshot; ++k) {
        if (src_ix[k] < 0 || src_ix[k] >= m->Px || src_iz[k] < 0 || src_iz[k] >= m->Pz) return HELM_E_INVALID;
        sf[k] = (src_iz[k] + m->npml) * m->nx + src_ix[k] + m->npml;
    }
    for (int k = 0; k < nrec; ++k) {
        if (rec_ix[k] < 0 || rec_ix[k] >= m->Px || rec_iz[k] < 0 || rec_iz[k] >= m->Pz) return HELM_E_INVALID;
        rf[k] = (rec_iz[k] + m->npml) * m->nx + rec_ix[k] + m->npml;
    }
    DeviceGuard g(m->ctx->device);
    cudaStream_t s = m->ctx->stream;
    const size_t dbytes = sizeof(double) * 2 * (size_t)nfreq * nshot * nrec;
    DevMem dobs, dcal;
    const double* dobs_p = static_cast<const double*>(d_obs);
    double* dcal_p = static_cast<double*>(d_cal_out);
    if (!o.device_ptrs) {
        if (cudaMalloc(&dobs.p, dbytes) != cudaSuccess) { cudaGetLastError(); return HELM_E_NOMEM; }
        HELM_CUDA_TRY(cudaMemcpyAsync(dobs.p, d_obs, dbytes, cudaMemcpyHostToDevice, s));
        dobs_p = static_cast<const double*>(dobs.p);
        if (d_cal_out) {
            if (cudaMalloc(&dcal.p, dbytes) != cudaSuccess) { cudaGetLastError(); return HELM_E_NOMEM; }
            dcal_p = static_cast<double*>(dcal.p);
        }
    }
    FwiState* st = nullptr;
    int rc = fwi_forward(m, s, nfreq, omega, nshot, sf.data(), nrec, rf.data(), dobs_p, lambda_reg, J_out, dcal_p, o,
                         stats, &st);
    if (rc != HELM_OK && rc != HELM_E_NOT_CONVERGED) { fwi_free(st); return rc; }
    if (!o.device_ptrs && d_cal_out) {
        cudaError_t e = cudaMemcpyAsync(d_cal_out, dcal_p, dbytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { fwi_free(st); set_last_error(cudaGetErrorString(e)); return HELM_E_CUDA; }
    }
    helm_fwi_state* out = new helm_fwi_state();
    out->m = m;
    out->st = st;
    *state = out;
    return rc;
}

int helm_fwi_backward(helm_fwi_state* state, double* grad_out, const helm_solve_opts* opts, helm_solve_stats* stats) {
    if (!state || !state->st || !grad_out) return HELM_E_INVALID;
    helm_solve_opts o;
    if (opts) o = *opts; else helm_default_opts(&o);
    if (check_opts(o) != HELM_OK) return HELM_E_INVALID;
    helm_model* m = state->m;
    DeviceGuard g(m->ctx->device);
    cudaStream_t s = m->ctx->stream;
    const size_t gbytes = sizeof(double) * (size_t)m->Px * m->Pz;
    DevMem dgrad;
    double* grad_p = grad_out;
    if (!o.device_ptrs) {
        if (cudaMalloc(&dgrad.p, gbytes) != cudaSuccess) { cudaGetLastError(); return HELM_E_NOMEM; }
        grad_p = static_cast<double*>(dgrad.p);
    }
    int rc = fwi_backward(state->st, s, grad_p, o, stats);
    if (rc != HELM_OK && rc != HELM_E_NOT_CONVERGED) return rc;
    if (!o.device_ptrs) {
        HELM_CUDA_TRY(cudaMemcpyAsync(grad_out, grad_p, gbytes, cudaMemcpyDeviceToHost, s));
        HELM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return rc;
}

int helm_gn_hvp(helm_fwi_state* state, const double* dm, double* hdm_out, const helm_solve_opts* opts,
                helm_solve_stats* stats) {
    if (!state || !state->st || !dm || !hdm_out) return HELM_E_INVALID;
    helm_solve_opts o;
    if (opts) o = *opts; else helm_default_opts(&o);
    if (check_opts(o) != HELM_OK) return HELM_E_INVALID;
    helm_model* m = state->m;
    DeviceGuard g(m->ctx->device);
    cudaStream_t s = m->ctx->stream;
    const size_t bytes = sizeof(double) * (size_t)m->Px * m->Pz;
    DevMem ddm, dh;
    const double* dm_p = dm;
    double* h_p = hdm_out;
    if (!o.device_ptrs) {
        if (cudaMalloc(&ddm.p, bytes) != cudaSuccess || cudaMalloc(&dh.p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return HELM_E_NOMEM;
        }
        HELM_CUDA_TRY(cudaMemcpyAsync(ddm.p, dm, bytes, cudaMemcpyHostToDevice, s));
        dm_p = static_cast<const double*>(ddm.p);
        h_p = static_cast<double*>(dh.p);
    }
    int rc = gn_hvp(state->st, s, dm_p, h_p, o, stats);
    if (rc != HELM_OK && rc != HELM_E_NOT_CONVERGED) return rc;
    if (!o.device_ptrs) {
        HELM_CUDA_TRY(cudaMemcpyAsync(hdm_out, h_p, bytes, cudaMemcpyDeviceToHost, s));
        HELM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return rc;
}

int helm_gn_step(helm_fwi_state* state, const double* grad, int cg_iters, double* dm_out, double* cg_rel_out,
                 const helm_solve_opts* opts) {
    if (!state || !state->st || !grad || !dm_out || cg_iters < 1 || cg_iters > 1000) return HELM_E_INVALID;
    if (!(state->st->lam > 0.0)) {
        set_last_error("helm_gn_step needs lambda_reg > 0 (the Gauss-Newton Hessian is then positive definite)");
        return HELM_E_INVALID;
    }
    helm_solve_opts o;
    if (opts) o = *opts; else helm_default_opts(&o);
    if (check_opts(o) != HELM_OK) return HELM_E_INVALID;
    helm_model* m = state->m;
    DeviceGuard g(m->ctx->device);
    cudaStream_t s = m->ctx->stream;
    const size_t bytes = sizeof(double) * (size_t)m->Px * m->Pz;
    DevMem dgrad, ddm;
    const double* g_p = grad;
    double* dm_p = dm_out;
    if (!o.device_ptrs) {
        if (cudaMalloc(&dgrad.p, bytes) != cudaSuccess || cudaMalloc(&ddm.p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return HELM_E_NOMEM;
        }
        HELM_CUDA_TRY(cudaMemcpyAsync(dgrad.p, grad, bytes, cudaMemcpyHostToDevice, s));
        g_p = static_cast<const double*>(dgrad.p);
        dm_p = static_cast<double*>(ddm.p);
    }
    std::vector<double> rel(cg_iters + 1, 0.0);
    int rc = gn_step(state->st, s, g_p, cg_iters, dm_p, rel.data(), o);
    if (rc != HELM_OK && rc != HELM_E_NOT_CONVERGED) return rc;
    if (!o.device_ptrs) {
        HELM_CUDA_TRY(cudaMemcpyAsync(dm_out, dm_p, bytes, cudaMemcpyDeviceToHost, s));
        HELM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (cg_rel_out) std::memcpy(cg_rel_out, rel.data(), sizeof(double) * rel.size());
    return rc;
}

void helm_fwi_state_destroy(helm_fwi_state* state) {
    if (!state) return;
    DeviceGuard g(state->m->ctx->device);
    fwi_free(state->st);
    delete state;
}

int helm_adjoint_gradient(helm_model* m, int nfreq, const double* omega, int nshot, const int* src_ix,
                          const int* src_iz, int nrec, const int* rec_ix, const int* rec_iz, const void* d_obs,
                          double lambda_reg, double* J_out, double* grad_out, void* d_cal_out,
                          const helm_solve_opts* opts, helm_solve_stats* stats) {
    if (!grad_out) return HELM_E_INVALID;
    helm_fwi_state* st = nullptr;
    const int nrhs = (nfreq > 0 && nshot > 0) ? nfreq * nshot : 0;
    int rc1 = helm_fwi_forward(m, nfreq, omega, nshot, src_ix, src_iz, nrec, rec_ix, rec_iz, d_obs, lambda_reg, J_out,
                               d_cal_out, opts, stats, &st);
    if (rc1 != HELM_OK && rc1 != HELM_E_NOT_CONVERGED) return rc1;
    int rc2 = helm_fwi_backward(st, grad_out, opts, stats ? stats + nrhs : nullptr);
    helm_fwi_state_destroy(st);
    if (rc2 != HELM_OK && rc2 != HELM_E_NOT_CONVERGED) return rc2;
    return (rc1 == HELM_E_NOT_CONVERGED || rc2 == HELM_E_NOT_CONVERGED) ? HELM_E_NOT_CONVERGED : HELM_OK;
}

}  // extern "C"

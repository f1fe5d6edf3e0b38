// helm_noalloc.cu - a V-cycle entry point that allocates no device memory.
//
// helm_vcycle allocates its level vectors and the coarsest-level inverse with
// the stream-ordered allocator on every call. Some callers cannot allow that:
// code running under a memory manager that owns the whole device (a framework
// caching allocator or a fixed arena), code whose process may not grow its
// device footprint after start-up, or callers that must not touch the allocator
// while other work is in flight. helm_vcycle_noalloc runs the same kernels on a
// fixed scratch area that is part of the library image instead: a file-scope
// __device__ array of kNoAllocScratchBytes, present on every GPU that loads the
// library until the process exits.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "helm_internal.h"
#include "helm_solver.h"

namespace helm {
namespace {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;   // 64 MiB
constexpr int kNoAllocMaxRhs = 256;
constexpr int kMaxDevices = 64;
constexpr int kNoAllocCoarse = HELM_COARSE_AUTO;   // the coarse end helm_vcycle's defaults choose

// The scratch area. In host code `g_noalloc_scratch` names a host-side stand-in,
// not device memory: kernels get the device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_base[kMaxDevices] = {nullptr};

// Device address of the scratch area on the current device, looked up once per
// device (the lookup is the set-up step; it may initialise the module, so the
// first call on a device should not happen inside a stream capture).
int scratch_base(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return HELM_E_INVALID;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_base[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_last_error(std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e));
            return HELM_E_CUDA;
        }
        g_base[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_base[dev]);
    return HELM_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace helm

using namespace helm;

extern "C" int helm_vcycle_noalloc(helm_model* m, int nrhs, const double* omega, double beta1, double beta2,
                                   double omega_jacobi, const void* r, void* z) {
    if (!m || !omega || !r || !z || nrhs < 1) return HELM_E_INVALID;
    if (nrhs > kNoAllocMaxRhs) {
        set_last_error("helm_vcycle_noalloc: at most 256 right-hand sides per call");
        return HELM_E_INVALID;
    }
    if (!std::isfinite(beta1) || !std::isfinite(beta2) || !(omega_jacobi > 0.0)) return HELM_E_INVALID;
    // per-RHS (h omega)^2 and one coarsest-level inverse per distinct frequency, on the stack
    double hw2[kNoAllocMaxRhs], w2s[kNoAllocMaxRhs];
    float hw2f[kNoAllocMaxRhs];
    int slot[kNoAllocMaxRhs], mods[kNoAllocMaxRhs];
    int nslots = 0;
    for (int b = 0; b < nrhs; ++b) {
        if (!(std::isfinite(omega[b]) && omega[b] > 0.0)) return HELM_E_INVALID;
        hw2[b] = m->h * m->h * omega[b] * omega[b];
        hw2f[b] = (float)hw2[b];
        const int mod = m->nmodels > 1 ? b : 0;
        int k = 0;
        while (k < nslots && !(w2s[k] == hw2[b] && mods[k] == mod)) ++k;
        if (k == nslots) { w2s[k] = hw2[b]; mods[k] = mod; ++nslots; }
        slot[b] = k;
    }
    // the coarse end of the cycle helm_vcycle would use: the dense inverse of level m->ld where it
    // applies (beta2 != 0 and the inversion fits the GPU), else the shared-memory tail
    int W = 0, per = 0;
    const bool dense = nrhs <= kDenseAutoMaxRhs && beta2 != 0.0 && m->ld > 0 &&
                       dense_invert_plan((int)m->lv[m->ld].n(), false, &W, &per);
    // groups of consecutive right-hand sides sharing a slot, at most 8 each
    int grp[kNoAllocMaxRhs + 1];
    int ngroups = 0, maxg = 0;
    grp[0] = 0;
    for (int b = 1; b <= nrhs; ++b)
        if (b == nrhs || slot[b] != slot[grp[ngroups]] || b - grp[ngroups] >= 8) {
            maxg = std::max(maxg, b - grp[ngroups]);
            grp[++ngroups] = b;
        }
    const int L = (int)m->lv.size() - 1;
    // carve the scratch area: the arrays every path uses, then those of the path
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    const size_t o_w2 = take(sizeof(double) * nrhs);
    const size_t o_w2f = take(sizeof(float) * nrhs);
    const size_t o_slot = take(sizeof(int) * nrhs);
    const size_t o_w2s = take(sizeof(double) * nslots);
    const size_t o_mods = take(sizeof(int) * nslots);
    const size_t o_grp = take(sizeof(int) * (ngroups + 1));
    const size_t common = off;
    struct Plan {
        size_t minv = 0, work = 0, md = 0, panel = 0, dinv = 0, bar = 0, err = 0, fbar = 0, ferr = 0;
        size_t f[kMaxLevels] = {}, e[kMaxLevels] = {}, g[kMaxLevels] = {};
        int top = 0;
        size_t end = 0;
    };
    auto carve = [&](bool dn) {
        Plan p;
        off = common;
        if (dn) {
            const size_t nd = m->lv[m->ld].n();
            const int nl = std::min(per, nslots);
            p.minv = take(sizeof(float2) * nd * nd * nslots);
            p.panel = take(sizeof(float2) * 2 * nd * W * nl);
            p.dinv = take(sizeof(float2) * 2 * (size_t)W * W * nl);
            p.bar = take(sizeof(unsigned) * nl);
            p.err = take(sizeof(int));
            p.fbar = take(sizeof(unsigned));   // the persistent F-cycle's barrier and error flag
            p.ferr = take(sizeof(int));
            p.top = m->ld;
        } else {
            const size_t nc = m->lv[L].n();
            p.work = take(sizeof(double2) * nc * nc * 2 * nslots);
            p.minv = take(sizeof(float2) * nc * nc * nslots);
            p.md = take(sizeof(double2) * nc * nc * nslots);
            p.top = m->lt[0];
        }
        for (int l = 1; l <= p.top; ++l) {
            p.f[l] = take(sizeof(float) * 2 * m->lv[l].n() * nrhs);
            p.e[l] = take(sizeof(float) * 2 * m->lv[l].n() * nrhs);
            if (l >= 2 && l < p.top) p.g[l] = take(sizeof(float) * 2 * m->lv[l].n() * nrhs);
        }
        p.end = off;
        return p;
    };
    Plan plan = carve(dense);
    if (plan.end > kNoAllocScratchBytes) {
        set_last_error("helm_vcycle_noalloc: this model and batch need " + std::to_string(plan.end) +
                       " bytes of scratch; the static area holds 67108864 (64 MiB)");
        return HELM_E_INVALID;
    }
    int dev = m->ctx->device, cur = -1;
    cudaGetDevice(&cur);
    if (cur != dev) cudaSetDevice(dev);
    unsigned char* base = nullptr;
    int rc = scratch_base(dev, &base);
    if (rc != HELM_OK) { if (cur != dev) cudaSetDevice(cur); return rc; }
    cudaStream_t s = m->ctx->stream;
    cudaError_t e = cudaMemcpyAsync(base + o_w2, hw2, sizeof(double) * nrhs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_w2f, hw2f, sizeof(float) * nrhs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_slot, slot, sizeof(int) * nrhs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_w2s, w2s, sizeof(double) * nslots, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_mods, mods, sizeof(int) * nslots, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_grp, grp, sizeof(int) * (ngroups + 1), cudaMemcpyHostToDevice, s);
    bool use_dense = dense;
    if (e == cudaSuccess && use_dense) {
        // every byte the inversion reads is written earlier in this call (the counters and the
        // error flag are cleared by the launcher), so stale contents do not matter
        e = launch_dense_invert<float>(level_dev(m, m->ld, true), reinterpret_cast<const double*>(base + o_w2s),
                                       reinterpret_cast<const int*>(base + o_mods), nslots, beta1, beta2, W, per,
                                       reinterpret_cast<float*>(base + plan.minv),
                                       reinterpret_cast<float*>(base + plan.panel),
                                       reinterpret_cast<float*>(base + plan.dinv),
                                       reinterpret_cast<unsigned*>(base + plan.bar),
                                       reinterpret_cast<int*>(base + plan.err), s);
        int herr = -1;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, base + plan.err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess || herr != 0) {
            // as helm_vcycle: without the dense inverse the tail path runs
            cudaGetLastError();
            e = cudaSuccess;
            use_dense = false;
            plan = carve(false);
            if (plan.end > kNoAllocScratchBytes) {
                if (cur != dev) cudaSetDevice(cur);
                set_last_error("helm_vcycle_noalloc: this model and batch need " + std::to_string(plan.end) +
                               " bytes of scratch; the static area holds 67108864 (64 MiB)");
                return HELM_E_INVALID;
            }
        }
    }
    if (e == cudaSuccess) {
        const double* dw2 = reinterpret_cast<const double*>(base + o_w2);
        if (!use_dense)
            launch_coarse_invert(level_dev(m, L, true), reinterpret_cast<const double*>(base + o_w2s),
                                 reinterpret_cast<const int*>(base + o_mods), nslots, beta1, beta2,
                                 reinterpret_cast<double2*>(base + plan.work), reinterpret_cast<float2*>(base + plan.minv),
                                 reinterpret_cast<double2*>(base + plan.md), s);
        MgCall mc;
        mc.w2 = dw2;
        mc.w2f = reinterpret_cast<const float*>(base + o_w2f);
        mc.b1 = beta1;
        mc.b2 = beta2;
        mc.wj = omega_jacobi;
        mc.st = nullptr;
        mc.nrhs = nrhs;
        mc.lf = fcycle_level(m, hw2, nrhs);
        mc.s = s;
        mc.minv = base + plan.minv;
        mc.slot = reinterpret_cast<const int*>(base + o_slot);
        mc.partials = nullptr;
        mc.pstride = 0;
        mc.ld = use_dense ? m->ld : 0;
        mc.grp = reinterpret_cast<const int*>(base + o_grp);
        mc.ngroups = ngroups;
        mc.maxg = maxg;
        MgLevels<float> B;
        std::memset(&B, 0, sizeof(B));
        for (int l = 1; l <= plan.top; ++l) {
            B.f[l] = reinterpret_cast<float*>(base + plan.f[l]);
            B.e[l] = reinterpret_cast<float*>(base + plan.e[l]);
            B.g[l] = plan.g[l] ? reinterpret_cast<float*>(base + plan.g[l]) : nullptr;
        }
        // as helm_vcycle (HELM_COARSE_AUTO: one launch per step; the persistent F-cycle kernel
        // only runs for HELM_COARSE_FUSED)
        FcArgs fa;
        if (use_dense && kNoAllocCoarse == HELM_COARSE_FUSED) {
            int* ferr = reinterpret_cast<int*>(base + plan.ferr);
            e = cudaMemsetAsync(ferr, 0, sizeof(int), s);
            const int grid = e == cudaSuccess ? fcycle_setup(m, mc, kNoAllocCoarse, B.f, B.e, B.g,
                                                             reinterpret_cast<unsigned*>(base + plan.fbar), ferr, &fa)
                                              : 0;
            if (grid > 0) {
                mc.fca = &fa;
                mc.fca_level = mc.lf;
                mc.fca_grid = grid;
            }
        }
        if (e == cudaSuccess)
            mg_apply<float>(m, mc, B, static_cast<const float*>(r), static_cast<float*>(z), 0, nullptr, nullptr);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess && mc.fca) {
            int herr = 0;
            e = cudaMemcpyAsync(&herr, base + plan.ferr, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e == cudaSuccess && herr != 0) {
                if (cur != dev) cudaSetDevice(cur);
                set_last_error("helm_vcycle_noalloc: a grid barrier wait of the persistent cycle gave up");
                return HELM_E_CUDA;
            }
        }
    }
    // the host arrays above are the sources of the copies: wait before returning
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    if (cur != dev) cudaSetDevice(cur);
    if (e != cudaSuccess) { set_last_error(cudaGetErrorString(e)); return HELM_E_CUDA; }
    return HELM_OK;
}

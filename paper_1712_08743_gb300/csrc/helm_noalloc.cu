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
    const int L = (int)m->lv.size() - 1;
    const size_t nc = m->lv[L].n();
    // carve the scratch area
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    const size_t o_w2 = take(sizeof(double) * nrhs);
    const size_t o_w2f = take(sizeof(float) * nrhs);
    const size_t o_slot = take(sizeof(int) * nrhs);
    const size_t o_w2s = take(sizeof(double) * nslots);
    const size_t o_mods = take(sizeof(int) * nslots);
    const size_t o_work = take(sizeof(double2) * nc * nc * 2 * nslots);
    const size_t o_mf = take(sizeof(float2) * nc * nc * nslots);
    const size_t o_md = take(sizeof(double2) * nc * nc * nslots);
    size_t o_f[kMaxLevels], o_e[kMaxLevels];
    for (int l = 1; l <= m->lt[0]; ++l) {
        o_f[l] = take(sizeof(float) * 2 * m->lv[l].n() * nrhs);
        o_e[l] = take(sizeof(float) * 2 * m->lv[l].n() * nrhs);
    }
    if (off > kNoAllocScratchBytes) {
        set_last_error("helm_vcycle_noalloc: this model and batch need " + std::to_string(off) +
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
    if (e == cudaSuccess) {
        // every byte read below is written earlier in this call, so nothing needs clearing
        const double* dw2 = reinterpret_cast<const double*>(base + o_w2);
        launch_coarse_invert(level_dev(m, L, true), reinterpret_cast<const double*>(base + o_w2s),
                             reinterpret_cast<const int*>(base + o_mods), nslots, beta1, beta2,
                             reinterpret_cast<double2*>(base + o_work), reinterpret_cast<float2*>(base + o_mf),
                             reinterpret_cast<double2*>(base + o_md), s);
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
        mc.minv = base + o_mf;
        mc.slot = reinterpret_cast<const int*>(base + o_slot);
        mc.partials = nullptr;
        mc.pstride = 0;
        MgLevels<float> B;
        std::memset(&B, 0, sizeof(B));
        for (int l = 1; l <= m->lt[0]; ++l) {
            B.f[l] = reinterpret_cast<float*>(base + o_f[l]);
            B.e[l] = reinterpret_cast<float*>(base + o_e[l]);
        }
        mg_apply<float>(m, mc, B, static_cast<const float*>(r), static_cast<float*>(z), 0, nullptr, nullptr);
        e = cudaGetLastError();
    }
    // the host arrays above are the sources of the copies: wait before returning
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    if (cur != dev) cudaSetDevice(cur);
    if (e != cudaSuccess) { set_last_error(cudaGetErrorString(e)); return HELM_E_CUDA; }
    return HELM_OK;
}

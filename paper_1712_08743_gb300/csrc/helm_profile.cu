// helm_profile.cu - per-kernel timing of the library's own launches (a
// measurement aid with no counterpart in the paper).
//
// Between helm_profile_begin and helm_profile_end every launcher of this library
// records a CUDA event pair around its kernel on the stream it launches on, with
// the kernel's class, the grid it works on and the algorithmic bytes the launch
// must move (each operand read or written once; model data shared by a batch
// counted once). Solves run without CUDA graphs while profiling, and the event
// between two launches stops programmatic dependent launch from overlapping
// them, so durations are those of serialised launches: the shares of the total
// are the meaningful figures, as in an ncu launch list.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "helm_internal.h"
#include "helm_solver.h"

namespace helm {

namespace {

struct ProfRecord {
    int kid, nx, nz;
    double bytes;
    cudaEvent_t a, b;
};

std::atomic<bool> g_prof_on{false};
std::mutex g_prof_mu;
std::vector<ProfRecord> g_prof;           // this session's launches
std::vector<cudaEvent_t> g_prof_pool;     // events of earlier sessions, for reuse

cudaEvent_t prof_event() {
    if (!g_prof_pool.empty()) {
        cudaEvent_t e = g_prof_pool.back();
        g_prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return e;
}

const char* const kProfNames[PK_COUNT] = {
    "k_apply", "k_apply_dots", "k_resid64", "k_refine", "k_bicg_init", "k_bicg_resume", "k_bicg_p", "k_bicg_s",
    "k_bicg_xr", "k_restrict", "k_prolong", "k_restrict_g", "k_correct_restrict", "k_resid_restrict_g",
    "k_prolong_g", "k_prolong2_g", "k_tail", "k_coarse_dense", "k_dense_invert", "k_coarse_invert", "k_fg_norm",
    "k_fg_scale", "k_fg_dots", "k_fg_axpy", "k_fg_finish", "k_fg_backsolve", "k_fg_update", "k_fcycle", "k_other"};

}  // namespace

bool prof_on() { return g_prof_on.load(std::memory_order_relaxed); }

ProfScope::ProfScope(int kid, int nx, int nz, double bytes, cudaStream_t s) : s_(s) {
    if (!prof_on()) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    ProfRecord r{kid, nx, nz, bytes, prof_event(), prof_event()};
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, s);
    idx_ = (int)g_prof.size();
    g_prof.push_back(r);
}

ProfScope::~ProfScope() {
    if (idx_ < 0) return;
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (idx_ < (int)g_prof.size()) cudaEventRecord(g_prof[idx_].b, s_);
}

}  // namespace helm

using namespace helm;

extern "C" int helm_profile_begin(void) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    for (auto& r : g_prof) { g_prof_pool.push_back(r.a); g_prof_pool.push_back(r.b); }
    g_prof.clear();
    g_prof_on.store(true);
    return HELM_OK;
}

extern "C" int helm_profile_end(helm_profile_entry* out, int cap, int* n_out) {
    g_prof_on.store(false);
    std::lock_guard<std::mutex> g(g_prof_mu);
    // (class, nx, nz) -> launches, ms, bytes; ordered by class then grid
    std::map<std::tuple<int, int, int>, std::tuple<uint64_t, double, double>> agg;
    int rc = HELM_OK;
    for (auto& r : g_prof) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) { cudaGetLastError(); rc = HELM_E_CUDA; continue; }
        auto& v = agg[std::make_tuple(r.kid, r.nx, r.nz)];
        std::get<0>(v) += 1;
        std::get<1>(v) += ms;
        std::get<2>(v) += r.bytes;
    }
    int n = 0;
    for (auto& kv : agg) {
        if (out && n < cap) {
            helm_profile_entry& E = out[n];
            std::memset(&E, 0, sizeof(E));
            std::strncpy(E.name, kProfNames[std::get<0>(kv.first)], sizeof(E.name) - 1);
            E.nx = std::get<1>(kv.first);
            E.nz = std::get<2>(kv.first);
            E.launches = std::get<0>(kv.second);
            E.ms = std::get<1>(kv.second);
            E.bytes = std::get<2>(kv.second);
        }
        ++n;
    }
    if (n_out) *n_out = n;
    return rc;
}

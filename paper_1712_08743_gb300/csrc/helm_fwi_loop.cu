// helm_fwi_loop.cu - the Gauss-Newton inversion loop over frequency groups:
// Eq. 4-9 repeated, with the paper's two ways of using the frequencies (all at
// once in its 1D example, lowest first and one at a time in its 2D example).
// Every solve, gradient and Gauss-Newton product runs through the library's
// entry points on the GPU; the loop only decides what to run next and moves
// the Pz x Px slowness between iterations.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "helm_internal.h"

namespace {

struct ModelHandle {
    helm_model* p = nullptr;
    ~ModelHandle() { reset(nullptr); }
    void reset(helm_model* x) {
        if (p) helm_destroy_model(p);
        p = x;
    }
    helm_model* release() {
        helm_model* x = p;
        p = nullptr;
        return x;
    }
};

struct StateHandle {
    helm_fwi_state* p = nullptr;
    ~StateHandle() { reset(nullptr); }
    void reset(helm_fwi_state* x) {
        if (p) helm_fwi_state_destroy(p);
        p = x;
    }
    helm_fwi_state* release() {
        helm_fwi_state* x = p;
        p = nullptr;
        return x;
    }
};

// A model and the forward state at it; the state goes first (it refers to the model).
struct Point {
    ModelHandle model;
    StateHandle state;
    double J = 0.0;
    void take(Point& o) {
        state.reset(o.state.release());
        model.reset(o.model.release());
        J = o.J;
    }
};

bool ok_or_unconverged(int rc) { return rc == HELM_OK || rc == HELM_E_NOT_CONVERGED; }

}  // namespace

extern "C" int helm_fwi_run(helm_ctx* ctx, int Px, int Pz, double h, int npml, double alpha_max, const double* m0,
                            int nfreq, const double* omega, int nshot, const int* src_ix, const int* src_iz, int nrec,
                            const int* rec_ix, const int* rec_iz, const void* d_obs, double lambda_reg,
                            const helm_fwi_opts* fo, const helm_solve_opts* opts, double* m_out, double* J_hist,
                            int* n_hist, helm_fwi_checkpoint checkpoint, void* user) {
    if (n_hist) *n_hist = 0;
    if (!ctx || !m0 || !omega || !src_ix || !src_iz || !rec_ix || !rec_iz || !d_obs || !fo || !m_out) return HELM_E_INVALID;
    if (Px < 1 || Pz < 1 || nfreq < 1 || nshot < 1 || nrec < 1) return HELM_E_INVALID;
    if (!std::isfinite(lambda_reg) || !(lambda_reg > 0.0)) return HELM_E_INVALID;
    if (fo->strategy != HELM_FWI_SIMULTANEOUS && fo->strategy != HELM_FWI_SEQUENTIAL) return HELM_E_INVALID;
    if (fo->gn_iters < 1 || fo->cg_iters < 1 || fo->cg_iters > 1000 || fo->max_halvings < 0 || fo->max_halvings > 30)
        return HELM_E_INVALID;
    if (!std::isfinite(fo->m_lo) || !std::isfinite(fo->m_hi) || !(fo->m_lo > 0.0) || fo->m_hi < fo->m_lo)
        return HELM_E_INVALID;
    for (int f = 0; f < nfreq; ++f)
        if (!std::isfinite(omega[f]) || !(omega[f] > 0.0)) return HELM_E_INVALID;
    helm_solve_opts o;
    if (opts) o = *opts; else helm_default_opts(&o);
    if (o.device_ptrs) return HELM_E_INVALID;

    const size_t np = (size_t)Px * Pz;
    std::vector<double> m(m0, m0 + np);
    // frequency groups: all at once, or one each from the lowest up
    std::vector<std::vector<int>> groups;
    std::vector<int> order(nfreq);
    std::iota(order.begin(), order.end(), 0);
    if (fo->strategy == HELM_FWI_SIMULTANEOUS) {
        groups.push_back(order);
    } else {
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return omega[a] < omega[b]; });
        for (int f : order) groups.push_back({f});
    }
    const size_t per_f = 2 * (size_t)nshot * nrec;   // doubles of one frequency's data
    const double* dobs = static_cast<const double*>(d_obs);
    int nh = 0, status = HELM_OK;
    std::vector<double> grad(np), dm(np), trial(np);

    for (size_t gi = 0; gi < groups.size(); ++gi) {
        const std::vector<int>& grp = groups[gi];
        const int nf = (int)grp.size();
        std::vector<double> om(nf), dg(per_f * nf);
        for (int k = 0; k < nf; ++k) {
            om[k] = omega[grp[k]];
            std::memcpy(dg.data() + per_f * k, dobs + per_f * grp[k], sizeof(double) * per_f);
        }
        // forward solves and J at slowness mm, into p
        auto forward = [&](const std::vector<double>& mm, Point& p) -> int {
            helm_model* mod = nullptr;
            int rc = helm_create_model(ctx, Px, Pz, h, mm.data(), npml, alpha_max, &mod);
            if (rc != HELM_OK) return rc;
            p.model.reset(mod);
            helm_fwi_state* st = nullptr;
            rc = helm_fwi_forward(mod, nf, om.data(), nshot, src_ix, src_iz, nrec, rec_ix, rec_iz, dg.data(),
                                  lambda_reg, &p.J, nullptr, &o, nullptr, &st);
            p.state.reset(st);
            return rc;
        };
        Point cur;
        int rc = forward(m, cur);
        if (!ok_or_unconverged(rc)) { status = rc; break; }
        if (rc != HELM_OK) status = rc;
        if (J_hist) J_hist[nh] = cur.J;
        ++nh;
        if (checkpoint) checkpoint((int)gi, 0, m.data(), cur.J, user);
        for (int it = 1; it <= fo->gn_iters; ++it) {
            rc = helm_fwi_backward(cur.state.p, grad.data(), &o, nullptr);   // Eq. 7
            if (!ok_or_unconverged(rc)) { status = rc; break; }
            if (rc != HELM_OK) status = rc;
            rc = helm_gn_step(cur.state.p, grad.data(), fo->cg_iters, dm.data(), nullptr, &o);   // Eq. 9
            if (!ok_or_unconverged(rc)) { status = rc; break; }
            if (rc != HELM_OK) status = rc;
            // backtracking: the first t = 1, 1/2, ... whose clipped trial lowers J
            bool accepted = false;
            double t = 1.0;
            for (int k = 0; k <= fo->max_halvings && !accepted; ++k, t *= 0.5) {
                for (size_t i = 0; i < np; ++i) trial[i] = std::min(fo->m_hi, std::max(fo->m_lo, m[i] + t * dm[i]));
                Point p;
                rc = forward(trial, p);
                if (!ok_or_unconverged(rc)) { status = rc; break; }
                if (p.J < cur.J) {
                    if (rc != HELM_OK) status = rc;
                    m.swap(trial);
                    cur.take(p);
                    accepted = true;
                }
            }
            if (!ok_or_unconverged(rc)) break;
            if (!accepted) break;                   // no descent along dm: the group ends
            if (J_hist) J_hist[nh] = cur.J;
            ++nh;
            if (checkpoint) checkpoint((int)gi, it, m.data(), cur.J, user);
        }
        if (!ok_or_unconverged(status)) break;
    }
    std::memcpy(m_out, m.data(), sizeof(double) * np);
    if (n_hist) *n_hist = nh;
    return status;
}

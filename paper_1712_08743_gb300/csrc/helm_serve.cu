// helm_serve.cu - continuous-batching request loop of the C ABI.
//
// helm_submit puts a request on a host queue. Worker threads, one per
// concurrent slot, each with its own CUDA stream, take the oldest request and
// every queued request of the same grid shape and options (up to max_batch),
// admit that batch only if its device memory fits in what is free (or in a
// simulated budget) minus a reserve and minus what running slots hold, and run
// it as one batched solve with one slowness model per right-hand side. A
// request that arrives while others are on the GPU is admitted as soon as a
// slot and the memory free up; slots run concurrently on the device. Nothing
// spins: host threads wait on a condition variable, and every request ends
// because each solve is bounded by its max_it and max_outer. helm_poll waits at
// most timeout_ms, or, for a negative timeout, on the host until its request
// has finished.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "helm_internal.h"
#include "helm_solver.h"

namespace helm {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t id = 0;
    helm_request r{};
    std::vector<double> slow;
    Clock::time_point t_sub, t_adm, t_done;
    bool done = false;
    int status = HELM_PENDING;
    helm_solve_stats stats{};
    std::vector<double> u;
    int nx = 0, nz = 0;
    int batch = 0;
};

struct Serve {
    helm_ctx* ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Req>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Req>> all;
    std::vector<std::thread> workers;
    bool stop = false;
    bool started = false;
    uint64_t next = 1;
    int max_batch = 32;
    int max_slots = 4;
    uint64_t reserve = 512ull << 20;
    uint64_t budget = 0;     // 0: use the device's free memory
    uint64_t in_use = 0;     // bytes held by admitted batches
    int running = 0;
    size_t max_queue = 1u << 20;
};

static bool same_batch(const helm_request& a, const helm_request& b) {
    const helm_solve_opts &x = a.opts, &y = b.opts;
    return a.Px == b.Px && a.Pz == b.Pz && a.npml == b.npml && a.alpha_max == b.alpha_max &&
           x.precision == y.precision && x.tol == y.tol && x.max_it == y.max_it && x.beta1 == y.beta1 &&
           x.beta2 == y.beta2 && x.omega_jacobi == y.omega_jacobi && x.inner_tol == y.inner_tol &&
           x.max_outer == y.max_outer && x.check_every == y.check_every && x.use_graphs == y.use_graphs &&
           x.krylov == y.krylov && x.restart == y.restart && x.precond == y.precond && x.reorth == y.reorth;
}

static uint64_t batch_bytes(const helm_request& r, int nb) {
    const int nx = r.Px + 2 * r.npml, nz = r.Pz + 2 * r.npml;
    const uint64_t n = (uint64_t)nx * nz;
    // models (m_pad + m2 in two precisions over the levels), f64 + u64, solver workspace
    return (uint64_t)nb * n * (8 + 12 * 2) + solve_bytes(nx, nz, 0, nb, r.opts.precision);
}

static void finish(Serve* sv, std::vector<std::shared_ptr<Req>>& batch, int status, const std::vector<helm_solve_stats>* st,
                   const std::vector<double>* u, size_t n) {
    const auto now = Clock::now();
    for (size_t k = 0; k < batch.size(); ++k) {
        Req& q = *batch[k];
        q.status = status;
        if (st) q.stats = (*st)[k];
        if (u && (status == HELM_OK || status == HELM_E_NOT_CONVERGED)) {
            q.status = q.stats.converged ? HELM_OK : HELM_E_NOT_CONVERGED;
            q.u.assign(u->begin() + 2 * n * k, u->begin() + 2 * n * (k + 1));
        }
        q.batch = (int)batch.size();
        q.t_done = now;
        q.done = true;
    }
    (void)sv;
}

static int run_batch(helm_ctx* ctx, cudaStream_t s, std::vector<std::shared_ptr<Req>>& batch,
                     std::vector<helm_solve_stats>& stats, std::vector<double>& u) {
    const helm_request& r0 = batch[0]->r;
    const int nb = (int)batch.size();
    const size_t np = (size_t)r0.Px * r0.Pz;
    std::vector<double> slow(np * nb);
    std::vector<double> hw2(nb);
    std::vector<int> src(nb);
    const int nx = r0.Px + 2 * r0.npml;
    for (int k = 0; k < nb; ++k) {
        const helm_request& r = batch[k]->r;
        std::memcpy(slow.data() + np * k, batch[k]->slow.data(), sizeof(double) * np);
        hw2[k] = r.h * r.h * r.omega * r.omega;
        src[k] = (r.src_iz + r.npml) * nx + r.src_ix + r.npml;
    }
    helm_model* m = nullptr;
    int rc = create_model(ctx, s, r0.Px, r0.Pz, r0.h, slow.data(), nb, r0.npml, r0.alpha_max, &m);
    if (rc != HELM_OK) return rc;
    const size_t n = m->n();
    double *f64 = nullptr, *u64 = nullptr;
    int* dsrc = nullptr;
    rc = HELM_OK;
    if (cudaMallocAsync(&f64, sizeof(double) * 2 * n * nb, s) != cudaSuccess ||
        cudaMallocAsync(&u64, sizeof(double) * 2 * n * nb, s) != cudaSuccess ||
        cudaMallocAsync(&dsrc, sizeof(int) * nb, s) != cudaSuccess) {
        cudaGetLastError();
        rc = HELM_E_NOMEM;
    }
    if (rc == HELM_OK && cudaMemcpyAsync(dsrc, src.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = HELM_E_CUDA;
    if (rc == HELM_OK) {
        launch_point_rhs(f64, dsrc, nb, n, s);
        stats.assign(nb, helm_solve_stats{});
        rc = solve_batch(m, s, nb, hw2.data(), f64, u64, r0.opts, stats.data());
        if (rc == HELM_OK || rc == HELM_E_NOT_CONVERGED) {
            u.resize(2 * n * nb);
            if (cudaMemcpyAsync(u.data(), u64, sizeof(double) * 2 * n * nb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                rc = HELM_E_CUDA;
        }
    }
    if (f64) cudaFreeAsync(f64, s);
    if (u64) cudaFreeAsync(u64, s);
    if (dsrc) cudaFreeAsync(dsrc, s);
    cudaStreamSynchronize(s);
    helm_destroy_model(m);
    return rc;
}

static void worker(Serve* sv) {
    cudaSetDevice(sv->ctx->device);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        sv->cv.wait(lk, [&] { return sv->stop || !sv->queue.empty(); });
        if (sv->stop) break;
        // the oldest request and every queued request that can share its launch
        std::vector<std::shared_ptr<Req>> batch;
        batch.push_back(sv->queue.front());
        for (size_t i = 1; i < sv->queue.size() && (int)batch.size() < sv->max_batch; ++i)
            if (same_batch(sv->queue[i]->r, batch[0]->r)) batch.push_back(sv->queue[i]);
        // admission by device memory
        uint64_t avail;
        {
            size_t fr = 0, tot = 0;
            cudaMemGetInfo(&fr, &tot);
            const uint64_t cap = sv->budget ? sv->budget : (uint64_t)tot;
            const uint64_t left = cap > sv->in_use ? cap - sv->in_use : 0;
            avail = sv->budget ? left : std::min<uint64_t>(left, fr);
            avail = avail > sv->reserve ? avail - sv->reserve : 0;
        }
        while (!batch.empty() && batch_bytes(batch[0]->r, (int)batch.size()) > avail) batch.pop_back();
        if (batch.empty()) {
            if (sv->running == 0) {   // nothing will free memory: refuse the oldest request
                std::vector<std::shared_ptr<Req>> one{sv->queue.front()};
                sv->queue.pop_front();
                one[0]->t_adm = Clock::now();
                finish(sv, one, HELM_E_NOMEM, nullptr, nullptr, 0);
                sv->cv.notify_all();
            } else {
                sv->cv.wait(lk);      // a running slot will release memory
            }
            continue;
        }
        for (auto& q : batch)
            for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it)
                if (*it == q) { sv->queue.erase(it); break; }
        const uint64_t bytes = batch_bytes(batch[0]->r, (int)batch.size());
        sv->in_use += bytes;
        sv->running += 1;
        const auto now = Clock::now();
        for (auto& q : batch) q->t_adm = now;
        lk.unlock();
        std::vector<helm_solve_stats> stats;
        std::vector<double> u;
        int rc = run_batch(sv->ctx, s, batch, stats, u);
        const size_t n = (size_t)(batch[0]->r.Px + 2 * batch[0]->r.npml) * (batch[0]->r.Pz + 2 * batch[0]->r.npml);
        lk.lock();
        sv->in_use -= bytes;
        sv->running -= 1;
        for (auto& q : batch) { q->nx = q->r.Px + 2 * q->r.npml; q->nz = q->r.Pz + 2 * q->r.npml; }
        finish(sv, batch, rc, (rc == HELM_OK || rc == HELM_E_NOT_CONVERGED) ? &stats : nullptr,
               (rc == HELM_OK || rc == HELM_E_NOT_CONVERGED) ? &u : nullptr, n);
        sv->cv.notify_all();
    }
    lk.unlock();
    if (s) cudaStreamDestroy(s);
}

static Serve* get_serve(helm_ctx* ctx) {
    std::lock_guard<std::mutex> g(ctx->serve_mu);
    if (!ctx->serve) {
        ctx->serve = new Serve();
        ctx->serve->ctx = ctx;
    }
    return ctx->serve;
}

}  // namespace helm

using namespace helm;

extern "C" {

int helm_serve_config(helm_ctx* ctx, int max_batch, int max_slots, uint64_t reserve_bytes, uint64_t budget_bytes) {
    if (!ctx || max_batch < 1 || max_slots < 1 || max_slots > 64) return HELM_E_INVALID;
    Serve* sv = get_serve(ctx);
    std::lock_guard<std::mutex> g(sv->mu);
    if (sv->started && max_slots != sv->max_slots) return HELM_E_BUSY;
    sv->max_batch = max_batch;
    sv->max_slots = max_slots;
    sv->reserve = reserve_bytes;
    sv->budget = budget_bytes;
    return HELM_OK;
}

int helm_submit(helm_ctx* ctx, const helm_request* req, uint64_t* ticket) {
    if (!ctx || !req || !ticket || !req->slowness) return HELM_E_INVALID;
    const helm_request& r = *req;
    if (r.Px < 1 || r.Pz < 1 || r.npml < 0 || !(r.h > 0.0) || !(r.omega > 0.0) || !(r.alpha_max >= 0.0))
        return HELM_E_INVALID;
    if (r.src_ix < 0 || r.src_ix >= r.Px || r.src_iz < 0 || r.src_iz >= r.Pz) return HELM_E_INVALID;
    if (r.opts.device_ptrs || (r.opts.krylov != HELM_KRYLOV_BICGSTAB && r.opts.krylov != HELM_KRYLOV_FGMRES) ||
        r.opts.restart < 1 || r.opts.restart > kMaxRestart || !(r.opts.tol > 0.0) || r.opts.max_it < 1 ||
        r.opts.check_every < 1 || r.opts.max_outer < 1 || !(r.opts.omega_jacobi > 0.0) || !(r.opts.inner_tol > 0.0) ||
        r.opts.precision < HELM_PREC_MIXED || r.opts.precision > HELM_PREC_FP32 ||
        (r.opts.precond != HELM_PRECOND_MG && r.opts.precond != HELM_PRECOND_NONE) ||
        r.opts.reorth < HELM_REORTH_ALWAYS || r.opts.reorth > HELM_REORTH_IFNEEDED)
        return HELM_E_INVALID;
    const size_t np = (size_t)r.Px * r.Pz;
    for (size_t i = 0; i < np; ++i)
        if (!(r.slowness[i] > 0.0) || !std::isfinite(r.slowness[i])) return HELM_E_INVALID;
    Serve* sv = get_serve(ctx);
    auto q = std::make_shared<Req>();
    q->r = r;
    q->slow.assign(r.slowness, r.slowness + np);
    q->r.slowness = nullptr;
    q->t_sub = Clock::now();
    std::lock_guard<std::mutex> g(sv->mu);
    if (sv->stop) return HELM_E_INVALID;
    if (sv->queue.size() >= sv->max_queue) return HELM_E_BUSY;
    if (!sv->started) {
        sv->started = true;
        for (int k = 0; k < sv->max_slots; ++k) sv->workers.emplace_back(worker, sv);
    }
    q->id = sv->next++;
    sv->all[q->id] = q;
    sv->queue.push_back(q);
    *ticket = q->id;
    sv->cv.notify_all();
    return HELM_OK;
}

int helm_poll(helm_ctx* ctx, uint64_t ticket, int timeout_ms, helm_result* result) {
    if (!ctx || !result) return HELM_E_INVALID;
    Serve* sv = get_serve(ctx);
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return HELM_E_INVALID;
    std::shared_ptr<Req> q = it->second;
    if (!q->done) {
        if (timeout_ms == 0) return HELM_PENDING;
        if (timeout_ms < 0) {
            sv->cv.wait(lk, [&] { return q->done; });
        } else if (!sv->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return q->done; })) {
            return HELM_E_TIMEOUT;
        }
    }
    result->u = q->u.empty() ? nullptr : q->u.data();
    result->nx = q->nx;
    result->nz = q->nz;
    result->status = q->status;
    result->stats = q->stats;
    result->latency_ms = std::chrono::duration<double, std::milli>(q->t_done - q->t_sub).count();
    result->queue_ms = std::chrono::duration<double, std::milli>(q->t_adm - q->t_sub).count();
    result->batch_size = q->batch;
    return HELM_OK;
}

int helm_release(helm_ctx* ctx, uint64_t ticket) {
    if (!ctx) return HELM_E_INVALID;
    Serve* sv = get_serve(ctx);
    std::lock_guard<std::mutex> g(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return HELM_E_INVALID;
    if (!it->second->done) return HELM_PENDING;
    sv->all.erase(it);
    return HELM_OK;
}

void helm_serve_shutdown(helm_ctx* ctx) {
    Serve* sv = nullptr;
    {
        std::lock_guard<std::mutex> g(ctx->serve_mu);
        sv = ctx->serve;
        ctx->serve = nullptr;
    }
    if (!sv) return;
    {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->stop = true;
        std::vector<std::shared_ptr<Req>> rest(sv->queue.begin(), sv->queue.end());
        sv->queue.clear();
        finish(sv, rest, HELM_E_INVALID, nullptr, nullptr, 0);
    }
    sv->cv.notify_all();
    for (auto& t : sv->workers) t.join();
    delete sv;
}

}  // extern "C"

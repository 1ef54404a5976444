// Continuous-batching request loop for fracture-set solves.
//
// Requests (geometry, loads, time step, number of steps) are queued by
// ddm_submit.  A server thread with its own context and stream admits them
// while the estimated device footprint fits the budget, keeps their trees,
// solution history and Krylov arena resident, and advances all admitted
// requests together: one round = one time step of every active request
// (history sum, right-hand side, lockstep batched GMRES of all of them).
// Finished requests leave after a round and queued ones join the next, so
// requests that arrive while others run are admitted as slots and memory
// free up.  ddm_poll reports completion.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

extern "C" {
ddm_status ddm_batch_create(ddm_ctx *ctx, ddm_tree *const *trees, int n, ddm_batch **out);
void ddm_batch_destroy(ddm_batch *batch);
ddm_status ddm_batch_gmres_solve(ddm_ctx *ctx, ddm_batch *batch, double dt, const double *d_rhs, double *d_x,
                                 const ddm_gmres_params *prm, ddm_gmres_info *infos);
}

namespace {
using Clock = std::chrono::steady_clock;
double ms_since(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Req {
    uint64_t id;
    ddm_request r;
    Clock::time_point t_submit, t_admit, t_done;
    ddm_tree *tree = nullptr;
    double *hist = nullptr;      // steps x 3N solutions
    double *rhs = nullptr;       // 3N
    int step = 0;                // completed steps
    int iters = 0;
    double rel = 0.0;
    size_t footprint = 0;
    ddm_status status = DDM_PENDING;
};
}  // namespace

struct ddm_server {
    ddm_ctx *ctx = nullptr;              // server-owned context (own stream)
    size_t budget = 0, used = 0;
    int max_active = 0;
    double tol = 1e-5;
    std::atomic<int> mode{DDM_MODE_FMM};   // product mode of the rounds (ddm_server_set_mode)
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req *> queue;
    std::map<uint64_t, Req *> all;
    uint64_t next_id = 1;
    bool stop = false;
    bool cancel_active = false;          // ddm_server_cancel: drop the active requests before the next round
    ddm_server_stats stats{};            // guarded by mu
    Clock::time_point t_start = Clock::now();
    std::thread th;
    long long rounds = 0;
};

namespace {

size_t footprint(const ddm_request &r, int ncheb) {
    size_t N = (size_t)r.n;
    // tree arrays, plus one cached M2L operator set per time window the
    // request's steps use (about half of the (level, offset) keys occur)
    size_t opset = (size_t)8 * 49 * 16 * ncheb * ncheb * ncheb * ncheb * 4;
    // (the tree's operator cache holds at most 4 GB of sets)
    size_t per_tree = N * 400 + std::min((size_t)r.steps * opset, std::max(opset, (size_t)4 << 30));
    size_t vectors = N * 3 * 8 * (size_t)(r.steps + 1 + 60);
    return per_tree + vectors;
}

void release(Req *q, cudaStream_t s) {
    if (q->tree) tree_free(q->tree);
    dfree(q->hist, s);
    dfree(q->rhs, s);
    q->tree = nullptr;
    q->hist = q->rhs = nullptr;
}

void serve_loop(ddm_server *S) {
    cudaSetDevice(S->ctx->device);
    cudaStream_t s = S->ctx->stream;
    std::vector<Req *> active;
    while (true) {
        // admission
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (active.empty())
                S->cv.wait_for(lk, std::chrono::milliseconds(20), [&] { return S->stop || !S->queue.empty(); });
            if (S->stop && S->queue.empty() && active.empty()) break;
            while (!S->queue.empty() && (int)active.size() < S->max_active) {
                Req *q = S->queue.front();
                if (S->used + q->footprint > S->budget && !active.empty()) break;
                S->queue.pop_front();
                S->used += q->footprint;
                q->t_admit = Clock::now();
                lk.unlock();
                ddm_status st = ddm_build_tree(S->ctx, q->r.d_xy, q->r.n, &q->tree);
                if (!st && dalloc(&q->hist, (size_t)q->r.steps * 3 * q->r.n * sizeof(double), s) != cudaSuccess)
                    st = DDM_ENOMEM;
                if (!st && dalloc(&q->rhs, (size_t)3 * q->r.n * sizeof(double), s) != cudaSuccess) st = DDM_ENOMEM;
                if (!st) cudaMemsetAsync(q->hist, 0, (size_t)q->r.steps * 3 * q->r.n * sizeof(double), s);
                cudaStreamSynchronize(s);
                lk.lock();
                S->stats.ms_admit += ms_since(q->t_admit, Clock::now());
                if (st) {
                    release(q, s);
                    S->used -= q->footprint;
                    q->status = st;
                    q->t_done = Clock::now();
                } else {
                    active.push_back(q);
                }
            }
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->cancel_active) {
                for (Req *q : active) {
                    release(q, s);
                    S->used -= q->footprint;
                    q->status = DDM_ECANCELED;
                    q->t_done = Clock::now();
                }
                active.clear();
                S->cancel_active = false;
                S->cv.notify_all();
            }
        }
        if (active.empty()) continue;
        // one round: one time step of every active request (same dt per round
        // group; requests are grouped by dt and system)
        std::map<std::pair<double, int>, std::vector<Req *>> groups;
        for (Req *q : active) groups[{q->r.dt, q->r.loads.system}].push_back(q);
        double t_hist = 0.0, t_setup = 0.0, t_solve = 0.0;
        int64_t n_solves = 0;
        const auto t_round = Clock::now();
        for (auto &g : groups) {
            std::vector<Req *> &rs = g.second;
            auto t0 = Clock::now();
            double dt = g.first.first;
            int sys = g.first.second;
            ddm_status st = DDM_OK;
            std::vector<ddm_tree *> trees;
            int64_t tot = 0;
            for (Req *q : rs) { trees.push_back(q->tree); tot += 3 * q->r.n; }
            double *rhs = nullptr, *x = nullptr;
            if (dalloc(&rhs, tot * sizeof(double), s) != cudaSuccess || dalloc(&x, tot * sizeof(double), s) != cudaSuccess)
                st = DDM_ENOMEM;
            int64_t o = 0;
            for (Req *q : rs) {
                if (st) break;
                int64_t n3 = 3 * q->r.n;
                st = ddm_rhs(S->ctx, q->tree, &q->r.loads, nullptr, q->rhs);
                if (!st && q->step > 0) {
                    std::vector<double> times(q->step + 2);
                    for (int k = 0; k <= q->step + 1; ++k) times[k] = k * dt;
                    st = ddm_history_apply(S->ctx, q->tree, q->hist, times.data(), q->step, q->rhs, S->mode.load());
                }
                if (!st) cudaMemcpyAsync(rhs + o, q->rhs, n3 * sizeof(double), cudaMemcpyDeviceToDevice, s);
                // initial guess: previous step (Dq of the 2N systems: 0)
                if (q->step > 0)
                    cudaMemcpyAsync(x + o, q->hist + (int64_t)(q->step - 1) * n3, n3 * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s);
                else
                    cudaMemsetAsync(x + o, 0, n3 * sizeof(double), s);
                if (!st && sys != DDM_SYS_PRESSURE) cudaMemsetAsync(x + o + 2 * q->r.n, 0, q->r.n * sizeof(double), s);
                o += n3;
            }
            ddm_batch *B = nullptr;
            std::vector<ddm_gmres_info> infos(rs.size());
            cudaStreamSynchronize(s);
            auto t1 = Clock::now();
            t_hist += ms_since(t0, t1);
            if (!st) st = ddm_batch_create(S->ctx, trees.data(), (int)trees.size(), &B);
            cudaStreamSynchronize(s);
            auto t2 = Clock::now();
            t_setup += ms_since(t1, t2);
            if (!st) {
                ddm_gmres_params prm{sys, 50, 2000, S->tol, S->mode.load()};
                st = ddm_batch_gmres_solve(S->ctx, B, dt, rhs, x, &prm, infos.data());
                if (st == DDM_ENOTCONV) st = DDM_OK;      // per-request status below
            }
            cudaStreamSynchronize(s);
            t_solve += ms_since(t2, Clock::now());
            n_solves += (int64_t)rs.size();
            o = 0;
            for (size_t i = 0; i < rs.size(); ++i) {
                Req *q = rs[i];
                int64_t n3 = 3 * q->r.n;
                if (!st) {
                    cudaMemcpyAsync(q->hist + (int64_t)q->step * n3, x + o, n3 * sizeof(double), cudaMemcpyDeviceToDevice, s);
                    q->iters += infos[i].iterations;
                    q->rel = infos[i].rel_residual;
                    if (!infos[i].converged) q->status = DDM_ENOTCONV;
                    q->step += 1;
                    if (q->step == q->r.steps)
                        cudaMemcpyAsync(q->r.d_x, x + o, n3 * sizeof(double), cudaMemcpyDeviceToDevice, s);
                } else {
                    q->status = st;
                    q->step = q->r.steps;
                }
                o += n3;
            }
            cudaStreamSynchronize(s);
            if (B) ddm_batch_destroy(B);
            dfree(rhs, s);
            dfree(x, s);
        }
        // retire finished requests
        std::lock_guard<std::mutex> lk(S->mu);
        ++S->rounds;
        S->stats.rounds += 1;
        S->stats.solves += n_solves;
        S->stats.ms_history += t_hist;
        S->stats.ms_setup += t_setup;
        S->stats.ms_solve += t_solve;
        S->stats.ms_other += ms_since(t_round, Clock::now()) - t_hist - t_setup - t_solve;
        std::vector<Req *> keep;
        for (Req *q : active) {
            if (q->step >= q->r.steps) {
                release(q, s);
                S->used -= q->footprint;
                if (q->status == DDM_PENDING) q->status = DDM_OK;
                q->t_done = Clock::now();
            } else {
                keep.push_back(q);
            }
        }
        active.swap(keep);
        S->cv.notify_all();
    }
}

}  // namespace

extern "C" {

ddm_status ddm_server_create(ddm_ctx *ctx, size_t hbm_budget_bytes, int max_active, double tol, ddm_server **out) {
    if (!ctx || !out || max_active <= 0 || !(tol > 0)) return ctx_fail(ctx, DDM_EINVAL, "ddm_server_create: bad arguments");
    ddm_server *S = new ddm_server();
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { delete S; return DDM_ECUDA; }
    ddm_status r = ddm_create(&S->ctx, &ctx->mat, &ctx->prm, st);
    if (r) { cudaStreamDestroy(st); delete S; return r; }
    // the server context takes the creating context's runtime settings
    S->ctx->grid_polls = ctx->grid_polls;
    S->ctx->m2l_compress = ctx->m2l_compress;
    S->ctx->m2l_rank = ctx->m2l_rank;
    S->ctx->hist_E = ctx->hist_E;
    S->ctx->hist_p = ctx->hist_p;
    S->ctx->hist_rho = ctx->hist_rho;
    S->budget = hbm_budget_bytes ? hbm_budget_bytes : ((size_t)64 << 30);
    S->max_active = max_active;
    S->tol = tol;
    S->th = std::thread(serve_loop, S);
    *out = S;
    return DDM_OK;
}

ddm_status ddm_submit(ddm_server *S, const ddm_request *req, uint64_t *ticket) {
    if (!S || !req || !ticket || req->n <= 0 || !req->d_xy || !req->d_x || req->steps <= 0 || !(req->dt > 0) ||
        req->loads.system < 0 || req->loads.system > 2)
        return DDM_EINVAL;
    Req *q = new Req();
    q->r = *req;
    q->t_submit = Clock::now();
    q->footprint = footprint(*req, S->ctx->prm.n_cheb);
    std::lock_guard<std::mutex> lk(S->mu);
    if (q->footprint > S->budget) { delete q; return DDM_ENOMEM; }
    q->id = S->next_id++;
    S->all[q->id] = q;
    S->queue.push_back(q);
    *ticket = q->id;
    S->cv.notify_all();
    return DDM_OK;
}

ddm_status ddm_poll(ddm_server *S, uint64_t ticket, ddm_result *res) {
    if (!S || !res) return DDM_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return DDM_EINVAL;
    Req *q = it->second;
    res->status = q->status;
    res->iterations = q->iters;
    res->rel_residual = q->rel;
    res->steps_done = q->step;
    bool done = q->status != DDM_PENDING && q->t_done != Clock::time_point();
    res->queue_ms = q->t_admit != Clock::time_point() ? ms_since(q->t_submit, q->t_admit) : -1.0;
    res->latency_ms = done ? ms_since(q->t_submit, q->t_done) : -1.0;
    if (!done) return DDM_PENDING;
    return q->status;
}

ddm_status ddm_server_set_mode(ddm_server *S, int mode) {
    if (!S || (mode != DDM_MODE_FMM && mode != DDM_MODE_DENSE)) return DDM_EINVAL;
    S->mode.store(mode);
    return DDM_OK;
}

ddm_status ddm_server_get_stats(ddm_server *S, ddm_server_stats *out) {
    if (!S || !out) return DDM_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    return DDM_OK;
}

ddm_status ddm_server_cancel(ddm_server *S) {
    if (!S) return DDM_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    const auto now = Clock::now();
    for (Req *q : S->queue) {
        q->status = DDM_ECANCELED;
        q->t_done = now;
    }
    S->queue.clear();
    S->cancel_active = true;
    S->cv.notify_all();
    return DDM_OK;
}

void ddm_server_destroy(ddm_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    for (auto &kv : S->all) {
        release(kv.second, S->ctx->stream);
        delete kv.second;
    }
    cudaStream_t st = S->ctx->stream;
    ddm_destroy(S->ctx);
    cudaStreamDestroy(st);
    delete S;
}

}  // extern "C"

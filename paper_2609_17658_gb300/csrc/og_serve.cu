// og_serve.cu -- continuous batching of force-evaluation requests.
//
// A request is one system integrated for nsteps kick-drift steps (the
// leapfrog of Sect. 3.2 reduced to a fixed step).  Requests are admitted as
// device memory (the context's HBM budget) and slots free up, and every
// admitted system keeps its tree, positions, velocities and last
// accelerations on the device until its last step.  One engine step walks
// the groups of all active systems in a single launch (longest lists first),
// then kicks and drifts every system and refits its tree, or rebuilds it.
// A refitted tree stays exact, but its node extents grow with the drift and
// its lists with them.  The walk reports every tree's interactions, and the
// engine prices the next step both ways in walk interactions: a rebuild
// costs a build plus a fresh tree's walk, a refit costs a refit plus the
// walk of the grown lists, predicted from the growth of the last refitted
// step (or, before any refit, a fourfold growth, so only systems whose walk
// is small beside a build try one).  Costs are modelled from measured build,
// refit and walk rates.  The rule uses only the system's own interaction
// counts, never a timing, so a system takes the same decisions, and gets the
// same bits, alone or in a mix.
// Newly arrived requests join at the next engine step, so their work
// overlaps with that of systems already in flight.
//
// The engine runs on its own thread and on a private context (stream and
// status word) of the same device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "og_internal.h"

namespace og {
namespace {

constexpr int kT = 256;
inline unsigned nblk(int64_t n) { return (unsigned)((n + kT - 1) / kT); }
constexpr int kMaxActive = 256;
constexpr int kMaxRefits = 64;   // refits between builds at most
// costs in walk interactions (about 2e-12 s each on the multi-tree walk): a
// build about 0.18 ms of launch-bound work plus 0.3 ns per particle, a refit
// about 0.17 ms plus 0.18 ns per particle; a refitted tree's walk costs 13 %
// more per interaction (it reads node extents); measured on GB300 at
// 2e4, 2e5 and 2e6 particles
constexpr double kBuildFixedInter = 9.0e7, kBuildPerParticleInter = 150.0;
constexpr double kRefitFixedInter = 8.5e7, kRefitPerParticleInter = 90.0;
constexpr double kRefitWalkFactor = 1.13;
constexpr double kTrialGrowth = 4.0;
// systems are built on this many private streams at once: a small build is
// bound by launch and synchronisation latency, so builds of several systems
// overlap on the device
constexpr int kBuildWorkers = 4;

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// v += a dt_kick; x += v dt_drift, x wrapped into [0, box)
__global__ void k_kick_drift(int64_t n, const float *__restrict__ acc, double *vel, double *pos,
                             double dt_kick, double dt_drift, double box) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int a = 0; a < 3; ++a) {
        const double v = vel[3 * i + a] + (double)acc[3 * i + a] * dt_kick;
        vel[3 * i + a] = v;
        double x = pos[3 * i + a] + v * dt_drift;
        x -= box * floor(x / box);
        pos[3 * i + a] = x;
    }
}

__global__ void k_unpermute_acc(int64_t n, const uint32_t *__restrict__ perm,
                                const float *__restrict__ acc_sorted, float *acc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = perm[i];
    acc[3ull * j + 0] = acc_sorted[i];
    acc[3ull * j + 1] = acc_sorted[n + i];
    acc[3ull * j + 2] = acc_sorted[2 * n + i];
}

struct System {
    uint64_t ticket = 0;
    int64_t n = 0;
    og_params prm{};
    int nsteps = 0;
    double dt_kick = 0, dt_drift = 0;
    float *acc_out = nullptr;
    double *pos_out = nullptr;
    std::vector<double> h_pos, h_vel, h_mass;
    size_t bytes = 0;
    // device state
    void *dmem = nullptr;
    double *d_pos = nullptr, *d_vel = nullptr, *d_mass = nullptr;
    float *d_acc = nullptr;
    og_tree *tree = nullptr;
    int step = 0, refits_since_build = 0;
    int64_t inter_base = -1; // interactions of the first walk after the last build
    int64_t inter_prev = 0, inter_last = 0;  // the two latest walks
    bool rebuild_next = false;
    og_result res{};
};

// a build stream: its own context (stream, status word, counters)
struct Worker {
    og_ctx *ctx = nullptr;
};

struct Server {
    og_ctx *owner = nullptr;
    og_ctx *ctx = nullptr;  // private context of the engine
    std::vector<Worker> workers;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<System *> pending;
    std::vector<System *> active;
    std::unordered_map<uint64_t, og_result> done;
    std::unordered_map<uint64_t, og_status> failed;
    std::vector<uint64_t> cancel;     // running requests to drop before their next step
    std::unordered_set<uint64_t> live;  // submitted and not finished
    uint64_t next_ticket = 1;
    size_t budget = 0, used = 0;
    bool stop = false;
    std::thread engine;
    int64_t interactions = 0, engine_steps = 0;
};

size_t estimate_bytes(int64_t n) {
    // tree arena and build scratch (96 bytes a particle of it for the exact
    // moments' prefix sums), plus the system's own state
    return (size_t)n * (320 + 180 + 96 + 8 * 3 * 7 + 12) + ((size_t)1 << 20);
}

og_status free_system(Server *S, System *sy) {
    cudaStream_t s = S->ctx->stream;
    if (sy->tree) og_tree_free(sy->tree);
    sy->tree = nullptr;
    if (sy->dmem) cudaFreeAsync(sy->dmem, s);
    sy->dmem = nullptr;
    return OG_OK;
}

// Build (or rebuild) a system's tree on a worker's stream.  Returns once the
// tree is complete on the device; the tree then belongs to the engine's
// context (refits, walks and frees are ordered on the engine's stream).
og_status build_system(Server *S, System *sy, const Worker &w) {
    cudaStream_t s = w.ctx->stream;
    if (sy->tree) {
        og_tree_free(sy->tree);
        sy->tree = nullptr;
    }
    og_tree *t = new (std::nothrow) og_tree();
    if (!t) { set_error("host allocation failed"); return OG_ERR_OOM; }
    t->ctx = w.ctx;
    t->prm = sy->prm;
    if (t->prm.group_max == 0) t->prm.group_max = 32;
    // the engine walks many trees in one launch of the default shape
    t->prm.walk_warps = kDefaultWalkWarps;
    t->prm.walk_chunk = kDefaultWalkChunk;
    t->n = sy->n;
    t->nseg = 1;
    t->seg_prm.assign(1, t->prm);
    t->h_seg_off = {0u, (uint32_t)sy->n};
    og_status st = build_tree(t, sy->d_pos, sy->d_mass);
    if (st) {
        og_tree_free(t);
        return st;
    }
    sy->tree = t;
    sy->refits_since_build = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    t->ctx = S->ctx;
    if (e != cudaSuccess) return cuda_fail(e, "serve build");
    st = check_status(w.ctx);
    if (st) return st;
    sy->inter_base = -1;
    sy->res.rebuilds++;
    return OG_OK;
}

// Refit a system's tree on a worker's stream (the engine's stream is free for
// the next walk's set-up); the tree goes back to the engine's context after.
og_status refit_system(Server *S, System *sy, const Worker &w) {
    og_tree *t = sy->tree;
    t->ctx = w.ctx;
    og_status st = refit_tree(t, sy->d_pos);
    t->ctx = S->ctx;
    if (st == OG_OK) st = check_status(w.ctx);
    if (st == OG_OK) {
        sy->refits_since_build++;
        sy->res.refits++;
    }
    return st;
}

og_status admit_system(Server *S, System *sy, const Worker &w) {
    cudaStream_t s = w.ctx->stream;
    const int64_t n = sy->n;
    size_t bytes = (size_t)n * (3 * 8 * 2 + 8 + 3 * 4) + 4096;
    cudaError_t e;
    if ((e = dev_malloc_async(&sy->dmem, bytes, s)) != cudaSuccess) return cuda_fail(e, "serve admission");
    char *q = static_cast<char *>(sy->dmem);
    sy->d_pos = reinterpret_cast<double *>(q);
    sy->d_vel = sy->d_pos + 3 * n;
    sy->d_mass = sy->d_vel + 3 * n;
    sy->d_acc = reinterpret_cast<float *>(sy->d_mass + n);
    cudaMemcpyAsync(sy->d_pos, sy->h_pos.data(), (size_t)n * 3 * sizeof(double), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(sy->d_vel, sy->h_vel.data(), (size_t)n * 3 * sizeof(double), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(sy->d_mass, sy->h_mass.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s);
    return build_system(S, sy, w);
}

// fn(system, worker) for every system; the systems, largest first, are dealt
// round-robin to the build workers, one host thread per worker
template <class F>
std::vector<og_status> on_workers(Server *S, std::vector<System *> v, F fn, std::vector<System *> *order) {
    std::stable_sort(v.begin(), v.end(), [](const System *a, const System *b) { return a->n > b->n; });
    *order = v;
    std::vector<og_status> st(v.size(), OG_OK);
    const int W = (int)std::min(S->workers.size(), v.size());
    // a worker's stream is drained after every system, whatever the outcome, so
    // nothing of a failed build is still in flight when its memory is freed
    if (W <= 1) {
        for (size_t k = 0; k < v.size(); ++k) {
            st[k] = fn(v[k], S->workers[0]);
            cudaStreamSynchronize(S->workers[0].ctx->stream);
        }
        return st;
    }
    std::vector<std::thread> th;
    for (int w = 0; w < W; ++w)
        th.emplace_back([&, w] {
            cudaSetDevice(S->ctx->device);
            for (size_t k = (size_t)w; k < v.size(); k += (size_t)W) {
                st[k] = fn(v[k], S->workers[w]);
                cudaStreamSynchronize(S->workers[w].ctx->stream);
            }
        });
    for (auto &x : th) x.join();
    return st;
}

void finish(Server *S, System *sy, og_status st) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->live.erase(sy->ticket);
    S->used -= std::min(S->used, sy->bytes);
    if (st == OG_OK) S->done[sy->ticket] = sy->res;
    else S->failed[sy->ticket] = st;
    S->cv_done.notify_all();
}

// One engine step over all active systems.  Returns the systems that finished.
void engine_step(Server *S) {
    og_ctx *c = S->ctx;
    cudaStream_t s = c->stream;
    std::vector<System *> &act = S->active;
    std::vector<og_tree *> trees;
    std::vector<float *> accs;
    for (System *sy : act) {
        trees.push_back(sy->tree);
        accs.push_back(sy->tree->a_sorted);
    }
    float ms = 0;
    int64_t inter = 0;
    std::vector<int64_t> tinter(act.size(), 0);
    // refitted trees and freshly built ones in separate launches: a launch
    // with one refitted tree reads node extents for all of its trees
    og_status st = OG_OK;
    for (int pass = 0; pass < 2 && st == OG_OK; ++pass) {
        std::vector<og_tree *> tv;
        std::vector<float *> av;
        std::vector<size_t> idx;
        for (size_t k = 0; k < act.size(); ++k)
            if (trees[k]->refit == (pass == 1)) {
                tv.push_back(trees[k]);
                av.push_back(accs[k]);
                idx.push_back(k);
            }
        if (tv.empty()) continue;
        float ms1 = 0;
        int64_t in1 = 0;
        std::vector<int64_t> ti(tv.size(), 0);
        st = walk_multi(c, tv.data(), (int64_t)tv.size(), OG_OPEN_BH, nullptr, av.data(), &ms1, &in1,
                        ti.data());
        ms += ms1;
        inter += in1;
        for (size_t q = 0; q < idx.size(); ++q) tinter[idx[q]] = ti[q];
    }
    for (size_t k = 0; k < act.size(); ++k) {
        System *sy = act[k];
        sy->inter_prev = sy->inter_last;
        sy->inter_last = tinter[k];
        if (sy->inter_base < 0) sy->inter_base = tinter[k];
    }
    if (st == OG_OK) {
        uint32_t stw = 0;
        cudaMemcpyAsync(&stw, c->d_status, sizeof(stw), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        if (stw) {
            cudaMemsetAsync(c->d_status, 0, sizeof(uint32_t), s);
            set_error("serve: device status 0x%x", stw);
            st = (stw & ST_BAD_INPUT) ? OG_ERR_ARG : OG_ERR_OVERFLOW;
        }
    }
    if (st != OG_OK) {
        for (System *sy : act) {
            free_system(S, sy);
            finish(S, sy, st);
            delete sy;
        }
        act.clear();
        return;
    }
    // kick and drift every system
    for (size_t k = 0; k < act.size(); ++k) {
        System *sy = act[k];
        og_tree *t = sy->tree;
        k_unpermute_acc<<<nblk(sy->n), kT, 0, s>>>(sy->n, t->perm, t->a_sorted, sy->d_acc); note_launch();
        k_kick_drift<<<nblk(sy->n), kT, 0, s>>>(sy->n, sy->d_acc, sy->d_vel, sy->d_pos, sy->dt_kick,
                                                 sy->dt_drift, sy->prm.box); note_launch();
    }
    cudaStreamSynchronize(s);
    std::vector<System *> keep, update;
    for (size_t k = 0; k < act.size(); ++k) {
        System *sy = act[k];
        sy->step++;
        sy->res.steps = sy->step;
        if (sy->step >= sy->nsteps) {
            // accelerations of the last force evaluation and the final positions
            if (sy->acc_out)
                cudaMemcpyAsync(sy->acc_out, sy->d_acc, (size_t)sy->n * 3 * sizeof(float), cudaMemcpyDeviceToHost, s);
            if (sy->pos_out)
                cudaMemcpyAsync(sy->pos_out, sy->d_pos, (size_t)sy->n * 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
            cudaError_t e = cudaStreamSynchronize(s);
            sy->res.t_done = now_s();
            free_system(S, sy);
            finish(S, sy, e == cudaSuccess ? OG_OK : cuda_fail(e, "serve results"));
            delete sy;
            continue;
        }
        // the next step priced both ways, in walk interactions
        const double nn = (double)sy->n;
        const double last = (double)sy->inter_last;
        const double growth = sy->refits_since_build == 0
                                  ? kTrialGrowth
                                  : std::max(1.0, last / std::max(1.0, (double)sy->inter_prev));
        const double cost_refit = kRefitFixedInter + kRefitPerParticleInter * nn +
                                  kRefitWalkFactor * last * growth;
        const double cost_build = kBuildFixedInter + kBuildPerParticleInter * nn + (double)sy->inter_base;
        sy->rebuild_next = cost_refit > cost_build || sy->refits_since_build >= kMaxRefits;
        update.push_back(sy);
    }
    // refits and rebuilds on the build workers' streams, several at once
    if (!update.empty()) {
        std::vector<System *> order;
        std::vector<og_status> st2 = on_workers(
            S, update,
            [S](System *sy, const Worker &w) {
                return sy->rebuild_next ? build_system(S, sy, w) : refit_system(S, sy, w);
            },
            &order);
        for (size_t k = 0; k < order.size(); ++k) {
            if (st2[k] != OG_OK) {
                free_system(S, order[k]);
                finish(S, order[k], st2[k]);
                delete order[k];
            } else {
                keep.push_back(order[k]);
            }
        }
    }
    act.swap(keep);
    S->interactions += inter;
    S->engine_steps++;
}

void engine_main(Server *S) {
    cudaSetDevice(S->ctx->device);
    while (true) {
        std::vector<System *> admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->active.empty() && S->pending.empty() && !S->stop)
                S->cv_work.wait_for(lk, std::chrono::milliseconds(20));
            if (S->stop) break;
            while (!S->pending.empty() && (int)(S->active.size() + admit.size()) < kMaxActive) {
                System *sy = S->pending.front();
                const bool fits = S->budget == 0 || S->used + sy->bytes <= S->budget ||
                                  (S->active.empty() && admit.empty());
                if (!fits) break;
                S->pending.pop_front();
                S->used += sy->bytes;
                admit.push_back(sy);
            }
        }
        if (!admit.empty()) {
            const double t0 = now_s();
            for (System *sy : admit) sy->res.t_start = t0;
            std::vector<System *> order;
            std::vector<og_status> st = on_workers(
                S, admit, [S](System *sy, const Worker &w) { return admit_system(S, sy, w); }, &order);
            for (size_t k = 0; k < order.size(); ++k) {
                if (st[k] != OG_OK) {
                    free_system(S, order[k]);
                    finish(S, order[k], st[k]);
                    delete order[k];
                } else {
                    S->active.push_back(order[k]);
                }
            }
        }
        // cancellations of running requests, taken before the next step
        std::vector<uint64_t> drop;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            drop.swap(S->cancel);
        }
        if (!drop.empty()) {
            std::vector<System *> keep;
            for (System *sy : S->active) {
                if (std::find(drop.begin(), drop.end(), sy->ticket) != drop.end()) {
                    cudaStreamSynchronize(S->ctx->stream);
                    free_system(S, sy);
                    finish(S, sy, OG_ERR_CANCELLED);
                    delete sy;
                } else {
                    keep.push_back(sy);
                }
            }
            S->active.swap(keep);
        }
        if (S->active.empty()) continue;
        engine_step(S);
    }
    for (System *sy : S->active) {
        free_system(S, sy);
        finish(S, sy, OG_ERR_STATE);
        delete sy;
    }
    S->active.clear();
    cudaStreamSynchronize(S->ctx->stream);
}

og_status ensure_server(og_ctx *c, Server **out) {
    if (c->serve) {
        *out = static_cast<Server *>(c->serve);
        return OG_OK;
    }
    Server *S = new (std::nothrow) Server();
    if (!S) { set_error("host allocation failed"); return OG_ERR_OOM; }
    S->owner = c;
    og_status st = og_create(&S->ctx, c->device, 0);
    if (st) {
        delete S;
        return st;
    }
    for (int w = 0; w < kBuildWorkers; ++w) {
        Worker W;
        st = og_create(&W.ctx, c->device, 0);
        if (st != OG_OK) {
            if (W.ctx) og_destroy(W.ctx);
            for (Worker &x : S->workers) og_destroy(x.ctx);
            og_destroy(S->ctx);
            delete S;
            return st;
        }
        S->workers.push_back(W);
    }
    S->budget = c->hbm_budget;
    S->engine = std::thread(engine_main, S);
    c->serve = S;
    *out = S;
    return OG_OK;
}

}  // namespace

void serve_shutdown(og_ctx *c) {
    if (!c || !c->serve) return;
    Server *S = static_cast<Server *>(c->serve);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (System *sy : S->pending) {
            S->failed[sy->ticket] = OG_ERR_STATE;
            delete sy;
        }
        S->pending.clear();
    }
    S->cv_work.notify_all();
    if (S->engine.joinable()) S->engine.join();
    cudaSetDevice(S->ctx->device);
    for (Worker &w : S->workers) og_destroy(w.ctx);
    og_destroy(S->ctx);
    delete S;
    c->serve = nullptr;
}

}  // namespace og

using namespace og;

extern "C" size_t og_serve_request_bytes(int64_t n) { return n > 0 ? estimate_bytes(n) : 0; }

extern "C" og_status og_serve_submit(og_ctx *c, const og_request *req, uint64_t *ticket) {
    if (!c || !req || !ticket) { set_error("og_serve_submit: NULL argument"); return OG_ERR_ARG; }
    if (!req->pos || !req->vel || !req->mass) { set_error("og_serve_submit: NULL input array"); return OG_ERR_ARG; }
    if (req->nsteps < 1) { set_error("og_serve_submit: nsteps must be >= 1"); return OG_ERR_ARG; }
    if (req->params.opening != OG_OPEN_BH) {
        set_error("og_serve_submit: served requests use the Barnes-Hut criterion");
        return OG_ERR_ARG;
    }
    if (req->params.flags & OG_DEVICE_PTRS) {
        set_error("og_serve_submit: served requests take host arrays");
        return OG_ERR_ARG;
    }
    if (req->n < 1 || req->n > kMaxN) { set_error("og_serve_submit: N out of range"); return OG_ERR_ARG; }
    if (!(req->params.box > 0.0) || (req->params.r_s > 0.0 && !(req->params.rcut_over_rs * req->params.r_s < 0.5 * req->params.box))) {
        set_error("og_serve_submit: bad box or cutoff");
        return OG_ERR_ARG;
    }
    const size_t bytes = estimate_bytes(req->n);
    Server *S = nullptr;
    og_status st = ensure_server(c, &S);
    if (st) return st;
    if (S->budget && bytes > S->budget) {
        set_error("og_serve_submit: a system of %lld particles needs about %zu bytes, more than the budget %zu",
                  (long long)req->n, bytes, S->budget);
        return OG_ERR_BUDGET;
    }
    System *sy = new (std::nothrow) System();
    if (!sy) { set_error("host allocation failed"); return OG_ERR_OOM; }
    sy->n = req->n;
    sy->prm = req->params;
    sy->nsteps = req->nsteps;
    sy->dt_kick = req->dt_kick;
    sy->dt_drift = req->dt_drift;
    sy->acc_out = req->acc_out;
    sy->pos_out = req->pos_out;
    sy->bytes = bytes;
    try {
        sy->h_pos.assign(req->pos, req->pos + 3 * req->n);
        sy->h_vel.assign(req->vel, req->vel + 3 * req->n);
        sy->h_mass.assign(req->mass, req->mass + req->n);
    } catch (...) {
        delete sy;
        set_error("host allocation failed");
        return OG_ERR_OOM;
    }
    sy->res.n = req->n;
    sy->res.t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        sy->ticket = S->next_ticket++;
        *ticket = sy->ticket;
        S->live.insert(sy->ticket);
        S->pending.push_back(sy);
    }
    S->cv_work.notify_all();
    return OG_OK;
}

extern "C" og_status og_serve_cancel(og_ctx *c, uint64_t ticket) {
    if (!c) { set_error("og_serve_cancel: NULL argument"); return OG_ERR_ARG; }
    if (!c->serve) { set_error("og_serve_cancel: nothing submitted on this context"); return OG_ERR_ARG; }
    Server *S = static_cast<Server *>(c->serve);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (ticket == 0 || ticket >= S->next_ticket) { set_error("og_serve_cancel: unknown ticket"); return OG_ERR_ARG; }
        if (!S->live.count(ticket)) {
            set_error("og_serve_cancel: request %llu has already finished", (unsigned long long)ticket);
            return OG_ERR_STATE;
        }
        for (auto it = S->pending.begin(); it != S->pending.end(); ++it) {
            if ((*it)->ticket == ticket) {
                // not admitted yet: nothing on the device
                S->failed[ticket] = OG_ERR_CANCELLED;
                S->live.erase(ticket);
                delete *it;
                S->pending.erase(it);
                S->cv_done.notify_all();
                return OG_OK;
            }
        }
        if (std::find(S->cancel.begin(), S->cancel.end(), ticket) == S->cancel.end())
            S->cancel.push_back(ticket);
    }
    S->cv_work.notify_all();
    return OG_OK;
}

extern "C" og_status og_serve_poll(og_ctx *c, uint64_t ticket, og_result *out, int timeout_ms) {
    if (!c || !out) { set_error("og_serve_poll: NULL argument"); return OG_ERR_ARG; }
    if (!c->serve) { set_error("og_serve_poll: nothing submitted on this context"); return OG_ERR_ARG; }
    Server *S = static_cast<Server *>(c->serve);
    std::unique_lock<std::mutex> lk(S->mu);
    if (ticket == 0 || ticket >= S->next_ticket) { set_error("og_serve_poll: unknown ticket"); return OG_ERR_ARG; }
    auto ready = [&] { return S->done.count(ticket) || S->failed.count(ticket); };
    if (!ready() && timeout_ms != 0) {
        if (timeout_ms < 0) S->cv_done.wait(lk, ready);
        else S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    }
    auto it = S->done.find(ticket);
    if (it != S->done.end()) {
        *out = it->second;
        S->done.erase(it);
        return OG_OK;
    }
    auto f = S->failed.find(ticket);
    if (f != S->failed.end()) {
        og_status st = f->second;
        S->failed.erase(f);
        set_error(st == OG_ERR_CANCELLED ? "og_serve_poll: request %llu was cancelled"
                                         : "og_serve_poll: request %llu failed",
                  (unsigned long long)ticket);
        return st;
    }
    return OG_PENDING;
}

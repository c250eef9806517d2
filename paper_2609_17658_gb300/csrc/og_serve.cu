// og_serve.cu -- continuous batching of force-evaluation requests.
//
// A request is one system integrated for nsteps kick-drift steps (the
// leapfrog of Sect. 3.2 reduced to a fixed step).  Requests are admitted as
// device memory (the context's HBM budget) and slots free up, and every
// admitted system keeps its tree, positions, velocities and last
// accelerations on the device until its last step.  One engine step walks
// the groups of all active systems in a single launch (longest lists first),
// then kicks and drifts every system and refits its tree, or rebuilds it when
// the drift since the last build exceeds a quarter of the mean group box side
// or after four refits.  Newly arrived requests join at the next engine step,
// so their work overlaps with that of systems already in flight.
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
#include <vector>

#include "og_internal.h"

namespace og {
namespace {

constexpr int kT = 256;
inline unsigned nblk(int64_t n) { return (unsigned)((n + kT - 1) / kT); }
constexpr int kMaxActive = 256;
constexpr int kMaxRefits = 4;
// systems are built on this many private streams at once: a small build is
// bound by launch and synchronisation latency, so builds of several systems
// overlap on the device
constexpr int kBuildWorkers = 4;

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// v += a dt_kick; x += v dt_drift; largest per-axis displacement since the
// last build (minimum image), as float bits for an integer atomic max
__global__ void k_kick_drift(int64_t n, const float *__restrict__ acc, double *vel, double *pos,
                             const double *__restrict__ xbuild, double dt_kick, double dt_drift,
                             double box, unsigned int *maxdrift) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float dmax = 0.0f;
    if (i < n) {
        for (int a = 0; a < 3; ++a) {
            const double v = vel[3 * i + a] + (double)acc[3 * i + a] * dt_kick;
            vel[3 * i + a] = v;
            double x = pos[3 * i + a] + v * dt_drift;
            x -= box * floor(x / box);
            pos[3 * i + a] = x;
            double d = x - xbuild[3 * i + a];
            d -= box * rint(d / box);
            dmax = fmaxf(dmax, (float)fabs(d));
        }
    }
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((threadIdx.x & 31) == 0 && dmax > 0.0f) atomicMax(maxdrift, __float_as_uint(dmax));
}

// mean over groups of the largest side of the group box (grid units)
__global__ void k_group_side_sum(int64_t ng, const uint32_t *__restrict__ gbox, unsigned long long *sum) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (g < ng) {
        uint32_t m = 0;
        for (int a = 0; a < 3; ++a) m = max(m, gbox[6 * g + 3 + a] - gbox[6 * g + a]);
        v = m;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(sum, v);
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
    double *d_pos = nullptr, *d_vel = nullptr, *d_mass = nullptr, *d_xbuild = nullptr;
    float *d_acc = nullptr;
    og_tree *tree = nullptr;
    int step = 0, refits_since_build = 0;
    double rebuild_thr = 0;  // box units
    og_result res{};
};

// a build stream: its own context (stream, status word, counters)
struct Worker {
    og_ctx *ctx = nullptr;
    unsigned long long *d_side = nullptr;
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
    uint64_t next_ticket = 1;
    size_t budget = 0, used = 0;
    bool stop = false;
    std::thread engine;
    unsigned int *d_drift = nullptr;
    unsigned long long *d_side = nullptr;
    int64_t interactions = 0, engine_steps = 0;
};

size_t estimate_bytes(int64_t n) {
    // tree arena and build scratch, plus the system's own state
    return (size_t)n * (320 + 180 + 8 * 3 * 8 + 12) + ((size_t)1 << 20);
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
    cudaMemcpyAsync(sy->d_xbuild, sy->d_pos, (size_t)sy->n * 3 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    // rebuild threshold: a quarter of the mean group box side
    cudaMemsetAsync(w.d_side, 0, sizeof(unsigned long long), s);
    k_group_side_sum<<<nblk(t->ngroups), kT, 0, s>>>(t->ngroups, t->gbox, w.d_side); note_launch();
    unsigned long long side = 0;
    cudaMemcpyAsync(&side, w.d_side, sizeof(side), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    t->ctx = S->ctx;
    if (e != cudaSuccess) return cuda_fail(e, "serve build");
    st = check_status(w.ctx);
    if (st) return st;
    const double mean_side = t->ngroups ? (double)side / (double)t->ngroups : 0.0;
    sy->rebuild_thr = 0.25 * mean_side * (sy->prm.box / 4294967296.0);
    sy->res.rebuilds++;
    return OG_OK;
}

og_status admit_system(Server *S, System *sy, const Worker &w) {
    cudaStream_t s = w.ctx->stream;
    const int64_t n = sy->n;
    size_t bytes = (size_t)n * (3 * 8 * 3 + 8 + 3 * 4) + 4096;
    cudaError_t e;
    if ((e = cudaMallocAsync(&sy->dmem, bytes, s)) != cudaSuccess) return cuda_fail(e, "serve admission");
    char *q = static_cast<char *>(sy->dmem);
    sy->d_pos = reinterpret_cast<double *>(q);
    sy->d_vel = sy->d_pos + 3 * n;
    sy->d_xbuild = sy->d_vel + 3 * n;
    sy->d_mass = sy->d_xbuild + 3 * n;
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
    og_status st = walk_multi(c, trees.data(), (int64_t)trees.size(), OG_OPEN_BH, nullptr, accs.data(),
                              &ms, &inter);
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
    // kick and drift every system, measure the drift since its last build
    cudaMemsetAsync(S->d_drift, 0, act.size() * sizeof(unsigned int), s);
    for (size_t k = 0; k < act.size(); ++k) {
        System *sy = act[k];
        og_tree *t = sy->tree;
        k_unpermute_acc<<<nblk(sy->n), kT, 0, s>>>(sy->n, t->perm, t->a_sorted, sy->d_acc); note_launch();
        k_kick_drift<<<nblk(sy->n), kT, 0, s>>>(sy->n, sy->d_acc, sy->d_vel, sy->d_pos, sy->d_xbuild,
                                                 sy->dt_kick, sy->dt_drift, sy->prm.box, S->d_drift + k); note_launch();
    }
    std::vector<unsigned int> drift(act.size(), 0u);
    cudaMemcpyAsync(drift.data(), S->d_drift, act.size() * sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    std::vector<System *> keep, rebuild;
    for (size_t k = 0; k < act.size(); ++k) {
        System *sy = act[k];
        sy->step++;
        sy->res.steps = sy->step;
        float dmax;
        std::memcpy(&dmax, &drift[k], sizeof(float));
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
        if ((double)dmax > sy->rebuild_thr || sy->refits_since_build >= kMaxRefits) {
            rebuild.push_back(sy);
            continue;
        }
        og_status st2 = refit_tree(sy->tree, sy->d_pos);
        sy->refits_since_build++;
        sy->res.refits++;
        if (st2 != OG_OK) {
            free_system(S, sy);
            finish(S, sy, st2);
            delete sy;
            continue;
        }
        keep.push_back(sy);
    }
    if (!rebuild.empty()) {
        std::vector<System *> order;
        std::vector<og_status> st2 = on_workers(
            S, rebuild, [S](System *sy, const Worker &w) { return build_system(S, sy, w); }, &order);
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
    cudaError_t e = cudaMalloc(&S->d_drift, kMaxActive * sizeof(unsigned int) + 64);
    if (e != cudaSuccess) {
        og_destroy(S->ctx);
        delete S;
        return cuda_fail(e, "serve setup");
    }
    S->d_side = reinterpret_cast<unsigned long long *>(S->d_drift + kMaxActive);
    for (int w = 0; w < kBuildWorkers; ++w) {
        Worker W;
        st = og_create(&W.ctx, c->device, 0);
        if (st == OG_OK && (e = cudaMalloc(&W.d_side, 64)) != cudaSuccess) st = cuda_fail(e, "serve setup");
        if (st != OG_OK) {
            if (W.ctx) og_destroy(W.ctx);
            for (Worker &x : S->workers) {
                cudaFree(x.d_side);
                og_destroy(x.ctx);
            }
            cudaFree(S->d_drift);
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
    cudaFree(S->d_drift);
    for (Worker &w : S->workers) {
        cudaFree(w.d_side);
        og_destroy(w.ctx);
    }
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
        S->pending.push_back(sy);
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
        set_error("og_serve_poll: request %llu failed", (unsigned long long)ticket);
        return st;
    }
    return OG_PENDING;
}

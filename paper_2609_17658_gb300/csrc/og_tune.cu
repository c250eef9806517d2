// og_tune.cu -- measured choice of the walk configuration: the group size G
// (targets per walk group) and the walk's launch shape (warps per block,
// entries of the shared far-entry chunk).
//
// The group size trades list building against evaluation: a larger group
// shares one interaction list among more targets, but its bounding box is
// larger, so the list is longer for every target.  Warps per block and the
// chunk length trade occupancy and shared memory against the cost of
// flushing a chunk.  Which values are fastest depends on the clustering of
// the input and on N.  For og_params.group_max = 0 the library measures them:
// the first call for a key (log2 N, opening criterion, split on/off) builds
// and walks the caller's input once per trial, times the walk kernels with
// CUDA events, and keeps the fastest configuration in the context (a
// coordinate descent: G first, then warps, then chunk).  Later calls with the
// same key reuse it.  The table can be saved to and loaded from a file of
// JSON lines, one key per line.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>

#include "og_internal.h"

namespace og {
namespace {

constexpr int kGroupCandidates[] = {8, 16, 24, 32};
constexpr int kWarpCandidates[] = {2, 8};       // besides the default 4
constexpr int kChunkCandidates[] = {128, 512};  // besides the default 256
constexpr int kTrials = 4 + 2 + 2;   // the three stages of the descent
static_assert(sizeof(kGroupCandidates) / sizeof(int) + sizeof(kWarpCandidates) / sizeof(int) +
                      sizeof(kChunkCandidates) / sizeof(int) == kTrials,
              "one time slot per trial");

struct Key {
    int nlog2, opening, split;
    bool operator<(const Key &o) const {
        if (nlog2 != o.nlog2) return nlog2 < o.nlog2;
        if (opening != o.opening) return opening < o.opening;
        return split < o.split;
    }
};

struct Entry {
    WalkConfig cfg;
    double ms[kTrials];  // walk time per trial, or 0 when loaded from a file
};

struct Table {
    std::mutex mu;
    std::map<Key, Entry> map;
};

Table *table(og_ctx *c) {
    if (!c->tune) c->tune = new (std::nothrow) Table();
    return static_cast<Table *>(c->tune);
}

Key key_of(int64_t n, const og_params &p) {
    int l = 0;
    while (l < 62 && ((int64_t)1 << (l + 1)) <= n) ++l;
    return Key{l, p.opening, p.r_s > 0.0 ? 1 : 0};
}

// build + force of the caller's input with one configuration; the walk time
og_status trial(og_ctx *c, const double *d_pos, const double *d_mass, int64_t n,
                const og_params &p, const WalkConfig &w, float *ms_walk) {
    og_tree *t = new (std::nothrow) og_tree();
    if (!t) { set_error("host allocation failed"); return OG_ERR_OOM; }
    t->ctx = c;
    t->prm = p;
    t->prm.group_max = w.group_max;
    t->prm.walk_warps = w.warps;
    t->prm.walk_chunk = w.chunk;
    t->prm.flags &= ~OG_DEBUG_DUMP_LISTS;
    t->n = n;
    t->nseg = 1;
    t->seg_prm.assign(1, t->prm);
    t->h_seg_off = {0u, (uint32_t)n};
    og_status st = build_tree(t, d_pos, d_mass);
    if (st == OG_OK) st = force_sorted(t, nullptr, ms_walk);
    if (st == OG_OK) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "tuning trial");
    }
    og_tree_free(t);
    return st;
}

}  // namespace

og_status tuned_walk(og_ctx *c, const double *d_pos, const double *d_mass, int64_t n,
                     const og_params &p, WalkConfig *out) {
    Table *tb = table(c);
    if (!tb) { set_error("host allocation failed"); return OG_ERR_OOM; }
    const Key k = key_of(n, p);
    {
        std::lock_guard<std::mutex> lk(tb->mu);
        auto it = tb->map.find(k);
        if (it != tb->map.end()) {
            *out = it->second.cfg;
            return OG_OK;
        }
    }
    Entry best{{32, kDefaultWalkWarps, kDefaultWalkChunk}, {}};
    float best_ms = INFINITY;
    int k_trial = 0;
    auto run = [&](const WalkConfig &w) -> og_status {
        float ms = 0.0f;
        og_status st = trial(c, d_pos, d_mass, n, p, w, &ms);
        if (st) return st;
        if (k_trial < kTrials) best.ms[k_trial++] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best.cfg = w;
        }
        return OG_OK;
    };
    og_status st = OG_OK;
    for (int G : kGroupCandidates)
        if ((st = run({G, kDefaultWalkWarps, kDefaultWalkChunk}))) return st;
    const int G = best.cfg.group_max;
    for (int W : kWarpCandidates)
        if ((st = run({G, W, kDefaultWalkChunk}))) return st;
    const int W = best.cfg.warps;
    for (int C : kChunkCandidates)
        if ((st = run({G, W, C}))) return st;
    std::lock_guard<std::mutex> lk(tb->mu);
    tb->map[k] = best;
    *out = best.cfg;
    return OG_OK;
}

void tune_free(og_ctx *c) {
    delete static_cast<Table *>(c->tune);
    c->tune = nullptr;
}

}  // namespace og

extern "C" {

og_status og_tune_walk(og_ctx *c, const double *pos, const double *mass, int64_t n,
                       const og_params *p, int32_t *group_max, int32_t *walk_warps,
                       int32_t *walk_chunk) {
    if (!c || !pos || !mass || !p) { og::set_error("NULL argument"); return OG_ERR_ARG; }
    og_params q = *p;
    q.group_max = 32;
    q.walk_warps = 0;
    q.walk_chunk = 0;
    og_status st = og::validate(&q, n);
    if (st) return st;
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    const double *d_pos = pos, *d_mass = mass;
    void *staging = nullptr;
    cudaError_t e;
    if (!(p->flags & OG_DEVICE_PTRS)) {
        if ((e = og::dev_malloc_async(&staging, (size_t)n * 4 * sizeof(double), s)) != cudaSuccess)
            return og::cuda_fail(e, "cudaMallocAsync (inputs)");
        double *dp = static_cast<double *>(staging);
        cudaMemcpyAsync(dp, pos, (size_t)n * 3 * sizeof(double), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(dp + 3 * n, mass, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s);
        d_pos = dp;
        d_mass = dp + 3 * n;
    }
    og::WalkConfig w{32, og::kDefaultWalkWarps, og::kDefaultWalkChunk};
    st = og::tuned_walk(c, d_pos, d_mass, n, q, &w);
    if (staging) cudaFreeAsync(staging, s);
    if (st == OG_OK) st = og::check_status(c);
    if (st == OG_OK) {
        if (group_max) *group_max = w.group_max;
        if (walk_warps) *walk_warps = w.warps;
        if (walk_chunk) *walk_chunk = w.chunk;
    }
    return st;
}

og_status og_tune_group_max(og_ctx *c, const double *pos, const double *mass, int64_t n,
                            const og_params *p, int32_t *group_max) {
    if (!group_max) { og::set_error("NULL argument"); return OG_ERR_ARG; }
    return og_tune_walk(c, pos, mass, n, p, group_max, nullptr, nullptr);
}

og_status og_tune_save(og_ctx *c, const char *path) {
    if (!c || !path) { og::set_error("NULL argument"); return OG_ERR_ARG; }
    og::Table *tb = og::table(c);
    if (!tb) { og::set_error("host allocation failed"); return OG_ERR_OOM; }
    FILE *f = std::fopen(path, "w");
    if (!f) { og::set_error("cannot open %s for writing", path); return OG_ERR_ARG; }
    std::lock_guard<std::mutex> lk(tb->mu);
    for (const auto &kv : tb->map) {
        const og::Entry &e = kv.second;
        std::fprintf(f,
                     "{\"n_log2\": %d, \"opening\": %d, \"split\": %d, \"group_max\": %d, "
                     "\"walk_warps\": %d, \"walk_chunk\": %d, "
                     "\"walk_ms\": [%.6f, %.6f, %.6f, %.6f, %.6f, %.6f, %.6f, %.6f]}\n",
                     kv.first.nlog2, kv.first.opening, kv.first.split, e.cfg.group_max,
                     e.cfg.warps, e.cfg.chunk, e.ms[0], e.ms[1], e.ms[2], e.ms[3], e.ms[4],
                     e.ms[5], e.ms[6], e.ms[7]);
    }
    const bool ok = std::fclose(f) == 0;
    if (!ok) { og::set_error("write to %s failed", path); return OG_ERR_ARG; }
    return OG_OK;
}

og_status og_tune_load(og_ctx *c, const char *path) {
    if (!c || !path) { og::set_error("NULL argument"); return OG_ERR_ARG; }
    og::Table *tb = og::table(c);
    if (!tb) { og::set_error("host allocation failed"); return OG_ERR_OOM; }
    FILE *f = std::fopen(path, "r");
    if (!f) { og::set_error("cannot open %s", path); return OG_ERR_ARG; }
    char line[512];
    int lineno = 0;
    og_status st = OG_OK;
    std::map<og::Key, og::Entry> got;
    while (std::fgets(line, sizeof line, f)) {
        ++lineno;
        if (line[0] == '\n' || line[0] == '\0') continue;
        og::Key k{};
        og::Entry e{{32, og::kDefaultWalkWarps, og::kDefaultWalkChunk}, {}};
        if (std::sscanf(line,
                        " {\"n_log2\": %d, \"opening\": %d, \"split\": %d, \"group_max\": %d, "
                        "\"walk_warps\": %d, \"walk_chunk\": %d",
                        &k.nlog2, &k.opening, &k.split, &e.cfg.group_max, &e.cfg.warps,
                        &e.cfg.chunk) != 6 ||
            e.cfg.group_max < 1 || e.cfg.group_max > 32 || k.nlog2 < 0 || k.nlog2 > 62 ||
            !og::valid_walk_shape(e.cfg.warps, e.cfg.chunk)) {
            og::set_error("%s:%d: not a tuning record", path, lineno);
            st = OG_ERR_ARG;
            break;
        }
        std::sscanf(line, "%*[^[][%lf, %lf, %lf, %lf, %lf, %lf, %lf, %lf]", &e.ms[0], &e.ms[1],
                    &e.ms[2], &e.ms[3], &e.ms[4], &e.ms[5], &e.ms[6], &e.ms[7]);
        got[k] = e;
    }
    std::fclose(f);
    if (st) return st;
    std::lock_guard<std::mutex> lk(tb->mu);
    for (const auto &kv : got) tb->map[kv.first] = kv.second;
    return OG_OK;
}

}  // extern "C"

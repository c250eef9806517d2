// og_internal.h -- internal types shared by the library's translation units.
//
// Device data of one tree (all in HBM, structure of arrays, sorted order):
//   skey[n] u64, perm[n] u32, px/py/pz[n] u32 fixed point, pm32[n] f32, pm64[n] f64
//   nodes (id 0 = root; others in the order of their first split):
//     nlev[m] u8, nbeg/nend[m] u32, npar[m] i32, ncbeg/nccnt[m] u32, npos[m] u32
//     nmom[m] {M, sum m x, sum m y, sum m z} f64 (one 32-byte record per node),
//     ncom[3m] u32, nnext/nsib[m] i32
//   child[c] u32 unified refs (particle < n, node + n), crec[c] 32-byte walk records
//   groups: gbeg/gend[g] u32, gbox[6g] u32
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <utility>
#include <vector>

#include "og.h"

namespace og {

constexpr int kLevels = 21;          // Morton levels: 21 bits per axis
constexpr int64_t kMaxN = (1ll << 26) - 1;

// status bits raised by kernels in the context's device status word
enum : uint32_t {
    ST_BAD_INPUT = 1u << 0,   // non-finite position or negative / non-finite mass
    ST_STACK_OVF = 1u << 1,   // walk stack overflow
    ST_LIST_OVF = 1u << 2,    // debug list buffer overflow
    ST_INTERNAL = 1u << 3,    // an internal consistency check failed
    ST_MASS_RANGE = 1u << 4,  // masses span too many binary orders for exact moments
    ST_TIMEOUT = 1u << 5,     // a bounded wait on another block of the grid ran out
};

// 32-byte record of one child slot, read by the walk (particle or node)
struct __align__(16) CRec {
    uint32_t x, y, z;   // particle position or node centre of mass (fixed point)
    float m;            // mass (f32) used by the pair arithmetic
    double M;           // mass (f64) used by the relative opening test
    uint32_t info;      // bit 31: node; bits 26..30: level; bits 0..25: child count
    uint32_t ref;       // particle: sorted index; node: first entry in the child array
};
static_assert(sizeof(CRec) == 32, "CRec must be 32 bytes");

// extent of a node after a refit (per child slot): start and length per axis
// on the circle of 2^32 grid units; a built tree uses the node's cell instead
struct __align__(16) CExt {
    uint32_t sx, sy, sz, pad0;
    uint32_t lx, ly, lz, pad1;
};
static_assert(sizeof(CExt) == 32, "CExt must be 32 bytes");

// geometry of one box (segment) of a forest
struct SegGeom {
    double box, inv_box;
    int pow2;        // box is a power of two: x / box == x * inv_box exactly
    int shift;       // with pow2: x / box * 2^32 == x * 2^shift
};

// monopole moments of a node: one 32-byte record, so that a parent reading a
// child node touches one sector
struct __align__(32) NodeMom {
    double M, Sx, Sy, Sz;
};

struct WalkParams;

}  // namespace og

struct og_ctx {
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t copy_stream = nullptr;  // host copies beside kernels (the masses in a build,
                                         // the counts in a force call)
    cudaEvent_t ev_to_side = nullptr, ev_from_side = nullptr;  // main stream -> side stream, back
    cudaStream_t stream = nullptr;
    size_t hbm_budget = 0;
    uint32_t *d_status = nullptr;     // device status word
    void *h_pinned = nullptr;         // page-locked host words read back without a sync of
                                      // their own: pass counters, status, build counts
    unsigned long long *d_counters = nullptr;  // scratch counters (work queues, totals)
    void *serve = nullptr;            // serving state (og_serve.cu)
    void *tune = nullptr;             // measured group sizes (og_tune.cu)
    void *live = nullptr;             // trees of og_tree_build not yet freed (og_capi.cu)
    void *pm = nullptr;               // cuFFT plans of the particle mesh (og_pm.cu)
};

struct og_tree {
    og_ctx *ctx = nullptr;
    og_params prm{};                  // parameters shared by all boxes (flags, group size)
    int64_t n = 0, nnodes = 0, nchild = 0, ngroups = 0;
    // boxes (segments) of the forest; a single system has nseg = 1
    int64_t nseg = 1;
    std::vector<og_params> seg_prm;   // per-box parameters
    std::vector<og::WalkParams> h_wp; // host staging of the per-box walk parameters
    std::vector<uint32_t> h_seg_off;  // first particle of each box, plus n
    std::vector<og::SegGeom> h_geom;  // geometry of each box (source of an async copy)
    uint32_t *seg_off = nullptr;      // device copy
    og::SegGeom *geom = nullptr;
    og::WalkParams *segp = nullptr;   // per-box walk parameters of the current pass
    uint32_t *sseg = nullptr;         // box of each sorted particle
    uint32_t *gseg = nullptr;         // box of each group
    // sorted particles
    uint64_t *skey = nullptr;
    uint32_t *perm = nullptr;         // sorted position -> caller index
    uint32_t *inv = nullptr;          // caller index -> sorted position
    uint32_t *px = nullptr, *py = nullptr, *pz = nullptr;
    float *pm32 = nullptr;
    double *pm64 = nullptr;
    // nodes
    uint8_t *nlev = nullptr;
    uint32_t *nbeg = nullptr, *nend = nullptr, *ncbeg = nullptr, *nccnt = nullptr;
    uint32_t *npos = nullptr;
    int32_t *npar = nullptr, *nnext = nullptr, *nsib = nullptr;
    og::NodeMom *nmom = nullptr;      // mass and sum of m x per node
    int *mbits = nullptr;             // lowest and highest set-bit exponent over the masses
    uint32_t *ncom = nullptr;
    int32_t *pnext = nullptr;
    uint32_t *owner = nullptr;        // node a particle hangs from
    uint32_t *norg = nullptr;         // cell origin of each node (3 per node, fixed by the build;
                                      // made when extents are first needed)
    bool have_norg = false;
    uint32_t *nocc = nullptr;         // octant occupancy of each node
    uint32_t *lnodes = nullptr;       // node ids by level (for the bottom-up passes)
    std::vector<uint32_t> h_lcount;   // nodes per level
    uint32_t *next_s = nullptr, *next_l = nullptr;  // extents after a refit (3 per node)
    og::CExt *cext = nullptr;         // extents per child slot (null until a refit)
    void *ext_arena = nullptr;        // allocation holding next_s, next_l, cext
    bool refit = false;
    double ms_refit = 0;
    uint32_t *child = nullptr;
    og::CRec *crec = nullptr;
    // groups
    uint32_t *gbeg = nullptr, *gend = nullptr, *gbox = nullptr;
    uint32_t *gcost = nullptr;        // list length of each group in the last walk pass
    uint32_t *gorder = nullptr;       // groups by decreasing cost
    bool have_cost = false;
    // walk passes enqueued without a host synchronisation (og_tree_force):
    // their events and counter slots, read after the call's one synchronisation
    cudaEvent_t pend_e0[2] = {nullptr, nullptr}, pend_e1[2] = {nullptr, nullptr};
    int npend = 0;
    uint32_t build_status = 0;        // status word read at the end of the build
    cudaEvent_t mass_ready = nullptr; // the masses' copy (host inputs): the build waits before
                                      // its first use of the masses
    // force work arrays (sorted order)
    float *a_sorted = nullptr;        // last pass accelerations, [3][n]
    float *a_old_sorted = nullptr;    // previous accelerations, [3][n]
    uint32_t *npp_sorted = nullptr, *npn_sorted = nullptr;
    // debug lists
    uint32_t *lists = nullptr;
    int64_t list_cap = 0, list_len = 0;
    // stats
    int64_t interactions = 0, interactions_last = 0;
    double ms_build = 0, ms_force = 0, ms_walk = 0, ms_pm = 0, ms_sph = 0;
    float *pot_next = nullptr;
    bool unscaled_out = false;        // the last pass leaves accelerations in grid units        // potential output of the next force call (sorted order)
    // one allocation holds every array above
    void *arena = nullptr;
    size_t arena_bytes = 0;
};

namespace og {

// thread-local last error
void set_error(const char *fmt, ...);
// stop the serving engine of a context (og_serve.cu)
void serve_shutdown(og_ctx *c);
// argument checks and the device status word (og_capi.cu)
og_status validate(const og_params *p, int64_t n);
og_status check_status(og_ctx *c);
// both force passes on a built tree, results in sorted order (og_capi.cu);
// subset: only these groups (device array of nsubset group ids)
// defer: enqueue the passes without waiting for them; the caller synchronises
// the stream and then calls finish_deferred (ms_walk_out is not set).
og_status force_sorted(og_tree *t, const float *d_aold, float *ms_walk_out,
                       const uint32_t *subset = nullptr, int64_t nsubset = 0,
                       float *pot_sorted = nullptr, bool defer = false);
// after the stream is synchronised: the deferred passes' times (summed into
// *ms_walk when not null) and interaction counts
og_status finish_deferred(og_tree *t, float *ms_walk);
// the error of a status word read back from the device (clears it there)
og_status status_from(og_ctx *c, uint32_t st);
// page-locked host words of a context: [0, 6) pass counters, 8 status, 9.. build counts
inline unsigned long long *pinned_counters(og_ctx *c, int pass) {
    return static_cast<unsigned long long *>(c->h_pinned) + 3 * pass;
}
inline uint32_t *pinned_status(og_ctx *c) {
    return reinterpret_cast<uint32_t *>(static_cast<unsigned long long *>(c->h_pinned) + 8);
}
inline uint32_t *pinned_counts(og_ctx *c) {
    return reinterpret_cast<uint32_t *>(static_cast<unsigned long long *>(c->h_pinned) + 9);
}
// default launch shape of the walk (og_params.walk_warps / walk_chunk = 0)
constexpr int kDefaultWalkWarps = 4;
constexpr int kDefaultWalkChunk = 256;
// measured walk configuration for group_max = 0: the group size and the walk's
// launch shape, once per kind of input (og_tune.cu)
struct WalkConfig {
    int group_max, warps, chunk;
};
og_status tuned_walk(og_ctx *c, const double *d_pos, const double *d_mass, int64_t n,
                     const og_params &p, WalkConfig *out);
// a walk launch shape the kernel supports: 1..8 warps, 64..1024 chunk entries
inline bool valid_walk_shape(int warps, int chunk) {
    return warps >= 1 && warps <= 8 && chunk >= 64 && chunk <= 1024;
}
void tune_free(og_ctx *c);
void pm_free(og_ctx *c);   // og_pm.cu: the context's cuFFT plans
// count of kernels launched by this library in this process
void note_launch();

// Programmatic dependent launch: the kernel may be scheduled while the one
// before it in the stream finishes; it calls pdl_wait() first, which returns
// once that kernel (and so everything before it) has completed and its writes
// are visible.  Kernels launched this way are otherwise ordered as usual.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
    note_launch();
}
og_status cuda_fail(cudaError_t e, const char *what);
// stream-ordered device allocation; fails without asking the device while
// og_debug_fail_allocations has injected failures left (og_capi.cu)
cudaError_t dev_malloc_raw(void **p, size_t bytes, cudaStream_t s);
template <class T>
cudaError_t dev_malloc_async(T **p, size_t bytes, cudaStream_t s) {
    void *q = nullptr;
    const cudaError_t e = dev_malloc_raw(&q, bytes, s);
    *p = static_cast<T *>(q);
    return e;
}

// device scans (og_scan.cu); n elements, exclusive, total written to *d_total
// when d_total != nullptr.  scratch must hold scan_scratch_bytes(n).
size_t scan_scratch_bytes(int64_t n);
void scan_exclusive_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *d_total,
                        void *scratch, cudaStream_t s);
void scan_inclusive_max_u32(const uint32_t *in, uint32_t *out, int64_t n, void *scratch,
                            cudaStream_t s);
// The same scans as one kernel with a decoupled look-back (up to 64 tiles of
// 4096 elements; longer scans take the two-kernel form, with scratch of
// scan_scratch_bytes(n)).  look holds scan_look_words(n) words, cleared before
// their first use; tag (1 .. 2^30 - 1) must differ between uses of the same
// words; ctr is a word that is 0 before the call.  A look-back that waits too
// long sets ST_INTERNAL in *status.
size_t scan_look_words(int64_t n);
// test hook: a one-kernel scan whose first tile never publishes (see
// og_debug_scan_wait_timeout); returns the status word's bits
og_status scan_wait_timeout_probe(og_ctx *c, int64_t n);
void scan_exclusive_u32_look(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *d_total,
                             unsigned long long *look, uint32_t *ctr, uint32_t tag, uint32_t *status,
                             void *scratch, cudaStream_t s);
// compaction: idx[k] = the k-th index i with flags[i] != 0 (flags 0 or 1), the
// count to *d_total
void scan_compact_u32_look(const uint32_t *flags, uint32_t *idx, int64_t n, uint32_t *d_total,
                           unsigned long long *look, uint32_t *ctr, uint32_t tag, uint32_t *status, void *scratch,
                           cudaStream_t s);
void scan_inclusive_max_u32_look(const uint32_t *in, uint32_t *out, int64_t n, unsigned long long *look,
                                 uint32_t *ctr, uint32_t tag, uint32_t *status, void *scratch,
                                 cudaStream_t s);

// radix sort of (key, value) pairs, stable, keys of `bits` significant bits
size_t radix_sort_scratch_bytes(int64_t n);
void radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                      int64_t n, int bits, void *scratch, cudaStream_t s, bool *result_in_alt,
                      uint32_t *status);

// the same sort with every digit pass run (no histogram read-back, no host
// synchronisation); with an even pass count the result is back in keys/vals
void radix_sort_pairs_every_pass(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt,
                                 uint32_t *vals_alt, int64_t n, int bits, void *scratch,
                                 cudaStream_t s);

// exact node moments (og_moments.cu): prefix sums over the sorted particles,
// then every node's mass, sums and centre of mass.  The node count is
// B + *d_nsplit (device) or, with d_nsplit null, t->nnodes; at most mcap.
size_t moments_scratch_bytes(int64_t n);
// t->mbits holds the lowest and highest set-bit exponents over the masses
// (gathered by the build's k_permute with mass_bit_span)
void node_moments(og_tree *t, const uint32_t *d_nsplit, int64_t mcap, void *scratch, cudaStream_t s);

// lowest and highest set-bit exponents of a mass: m = s 2^e (s < 2^53) has
// bits from 2^lo to below 2^hi; zero, negative and non-finite masses have none
__device__ __forceinline__ void mass_bit_span(double m, int &lo, int &hi) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(m);
    const unsigned E = (unsigned)(bits >> 52) & 0x7ffu;
    unsigned long long s = bits & ((1ull << 52) - 1ull);
    if ((bits >> 63) || E == 0x7ffu || (E == 0u && s == 0ull)) return;
    int ex = -1074;
    if (E) {
        s |= 1ull << 52;
        ex = (int)E - 1075;
    }
    lo = min(lo, ex + __ffsll((long long)s) - 1);
    hi = max(hi, ex + 64 - __clzll((long long)s));
}

// build stages (og_build.cu)
og_status build_tree(og_tree *t, const double *d_pos, const double *d_mass);
// refit for drifted positions (input order, device): same topology and groups
og_status refit_tree(og_tree *t, const double *d_pos);

// force (og_walk.cu)
struct WalkParams {
    int opening;       // OG_OPEN_BH / OG_OPEN_REL
    bool split;        // erfc split and cutoff active
    bool dump;         // keep lists
    double th2;        // theta^2
    float th2f;        // theta^2 in single precision (opening filter)
    double G;          // gravitational constant (relative test)
    float Gf;
    double alpha;      // relative-criterion tolerance
    double s2;         // (L / 2^32)^2
    float rc2;         // cutoff^2 in grid units (single precision)
    unsigned long long rprune;  // prune threshold, squared grid units
    unsigned long long hnear2;  // entries closer than this (squared grid units) may need softening
    float hnear2f;     // hnear2 raised by more than the FP32 error of a squared distance
    float h;           // softening length, grid units
    float inv_h;
    float inv_2rs;     // 1 / (2 r_s), grid units
    float kexp;        // -log2(e) / (4 r_s^2), grid units
    float out_scale;   // G (2^32/L)^2
    float pot_scale;   // G 2^32/L (potential from grid units)
};
// One walk launch over all groups of all boxes.  first_pass: the Barnes-Hut
// pass that supplies a_old for the relative criterion (each box's
// theta_first_pass).  use_order: take the groups longest list first, by the
// list lengths of the previous pass on this tree (if any).  subset: walk only
// these nsubset groups, in this order (device array), instead of all groups.
// defer: no host synchronisation (see force_sorted); not with list dumps.
og_status walk_pass(og_tree *t, int opening, bool first_pass, const float *a_old_sorted,
                    float *acc_sorted, float *ms_out, bool use_order,
                    const uint32_t *subset = nullptr, int64_t nsubset = 0,
                    float *pot_sorted = nullptr, bool defer = false);
// One walk launch over the groups of several trees (the serving loop), in
// decreasing order of their previous list lengths.  Every tree's per-box
// parameters must agree on split on/off.  tree_interactions (or null): the
// interactions evaluated for each tree.
og_status walk_multi(og_ctx *c, og_tree *const *trees, int64_t ntrees, int opening,
                     const float *const *a_old_sorted, float *const *acc_sorted, float *ms_out,
                     int64_t *interactions, int64_t *tree_interactions = nullptr);
// cell extents for a built tree (so that it can join a walk of refitted trees)
og_status cell_extents(og_tree *t);
WalkParams make_walk_params(const og_params &p, int opening, double theta);

}  // namespace og

/*
 * og.h -- C-ABI of the GB300 short-range TreePM tree-force library.
 *
 * The library computes the short-range part of the TreePM gravitational
 * acceleration of the OpenGadget3 paper (arxiv 2609.17658):
 *   - Sect. 4.1   "Oct-Tree": recursive subdivision of the box into eight
 *                 sub-cubes, monopole moments (mass, centre of mass);
 *   - Sect. 4.1.1 "Tree construction": nodes, nextnode/sibling threading,
 *                 particles inserted in space-filling-curve order (here a
 *                 63-bit Morton key sorted by an LSD radix sort);
 *   - Sect. 4.1.2 "Tree walk": Barnes-Hut or relative opening criterion,
 *                 a boundary check, accepted nodes act as a point mass at
 *                 their centre of mass;
 *   - Sect. 4.1.3 "Force evaluation": Newtonian M/r^3 beyond h, the spline
 *                 softened kernel inside h, h = 2.8 eps (eps Plummer
 *                 equivalent);
 *   - Sect. 4.2   "Particle Mesh": the short-range potential
 *                 phi_s = -G m erfc(r / 2 r_s) / r of the force split;
 *   - Sect. 3.4 / 18.2: one walk per group of spatially close particles.
 *
 * Conventions for every entry point:
 *   - All calls return og_status.  Errors are negative, never abort the
 *     process, and leave a thread-local message for og_last_error().
 *   - The caller owns every input and output buffer.  The library copies what
 *     it needs; og_ctx and og_tree are opaque handles owned by the library.
 *   - Pointers are host pointers unless the OG_DEVICE_PTRS flag is set in
 *     og_params.flags, in which case the position, mass, previous
 *     acceleration and output pointers are device pointers on the context's
 *     device.  Host-pointer calls are synchronous; device-pointer calls are
 *     ordered on the context's stream and return before the work finishes.
 *   - Positions are AoS double[N][3] in box units; they are reduced to the
 *     periodic cube [0, box)^3 and stored as 32-bit fixed point per axis.
 *     Accelerations are float[N][3] in units of G M / L^2 (M mass unit,
 *     L length unit of the inputs), in the caller's particle order.
 *   - A context is not thread safe, except og_serve_* which lock internally.
 */
#ifndef OG_H
#define OG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OG_OK = 0,
    OG_PENDING = 1,          /* og_serve_poll: not finished yet */
    OG_ERR_ARG = -1,         /* invalid argument (NaN position, N out of range, ...) */
    OG_ERR_OOM = -2,         /* device or host allocation failed */
    OG_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    OG_ERR_TIMEOUT = -4,     /* a bounded device-side wait ran out: a tile of a one-kernel
                                sort pass or scan waited too long for the count of an
                                earlier tile (the context stays usable) */
    OG_ERR_BUDGET = -5,      /* the request does not fit the HBM budget */
    OG_ERR_OVERFLOW = -6,    /* a fixed-capacity device buffer overflowed */
    OG_ERR_STATE = -7,       /* call not valid in the handle's state */
    OG_ERR_CANCELLED = -8    /* og_serve_poll: the request was cancelled */
} og_status;

typedef enum {
    OG_OPEN_BH = 0,          /* Barnes-Hut: open iff l^2 > theta^2 d^2 (Sect. 4.1.2) */
    OG_OPEN_REL = 1          /* relative: open iff G M l^2 > alpha |a_old|_min d^4 (Sect. 4.1.2) */
} og_open;

enum {
    OG_DEVICE_PTRS = 1,      /* input/output pointers are device pointers */
    OG_DEBUG_DUMP_LISTS = 2  /* keep the interaction lists of the last force call */
};

typedef struct {
    double box;              /* L > 0: periodic cube [0, L)^3 */
    double G;                /* gravitational constant (default 1) */
    double eps;              /* Plummer-equivalent softening; h = 2.8 eps (Sect. 4.1.3) */
    double r_s;              /* split scale A_smth (Sect. 4.2); <= 0: no split, no cutoff */
    double rcut_over_rs;     /* cutoff radius / r_s (default 4.5); r_cut must be < L/2 */
    double theta;            /* Barnes-Hut opening angle (default 0.5) */
    double alpha;            /* relative-criterion tolerance (default 0.005) */
    double theta_first_pass; /* OG_OPEN_REL without a_old: BH angle of the first pass */
    int32_t opening;         /* og_open */
    int32_t leaf_max;        /* particles per leaf cell; 1 = one particle per leaf (Sect. 4.1) */
    int32_t group_max;       /* targets per group, 1..32; 0 = measured per kind of input
                                together with the walk's launch shape (og_tune_walk) */
    int32_t flags;           /* OG_DEVICE_PTRS | OG_DEBUG_DUMP_LISTS */
    int32_t walk_warps;      /* walk launch shape: warps (one group each) per block, 1..8;
                                0 = the measured value when group_max = 0, else 4 */
    int32_t walk_chunk;      /* entries of a warp's shared far-entry chunk, 64..1024;
                                0 = the measured value when group_max = 0, else 256 */
} og_params;

typedef struct og_ctx og_ctx;
typedef struct og_tree og_tree;

/* Sizes of a built tree (for og_tree_export). */
typedef struct {
    int64_t n;               /* particles */
    int64_t nodes;           /* octree nodes, root included */
    int64_t children;        /* entries of the child array */
    int64_t groups;          /* walk groups */
    int64_t list_entries;    /* entries kept by the last OG_DEBUG_DUMP_LISTS force call */
    int64_t interactions;    /* PP + PN entries evaluated by the last force call, all passes */
    int64_t interactions_last_pass;
    double  ms_build;        /* device time of the last build (ms) */
    double  ms_force;        /* device time of the last force call, all passes (ms) */
    double  ms_walk;         /* device time of the walk kernels of the last force call (ms) */
    int32_t group_max;       /* the group size the tree was built with (the measured
                                choice when og_params.group_max was 0) */
    int32_t walk_warps;      /* the walk launch shape the tree's force calls use */
    int32_t walk_chunk;
    int32_t pad;
    double  ms_pm;           /* device time of the last og_tree_pm_force call (ms) */
    double  ms_sph;          /* device time of the last og_tree_sph_density call (ms) */
} og_tree_info;

/* ---- context ----------------------------------------------------------- */

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the device
 * memory the serving loop may admit (0 = no bound).  Owns a CUDA stream. */
og_status og_create(og_ctx **ctx, int device, size_t hbm_budget_bytes);
/* Stops the context's serving engine and frees the trees of og_tree_build
 * that were not freed; afterwards no tree of the context may be used. */
og_status og_destroy(og_ctx *ctx);
/* Order all further work of the context on `stream` (a cudaStream_t of the
 * context's device; NULL restores the context's own stream). */
og_status og_set_stream(og_ctx *ctx, void *stream);
/* Fill p with the defaults listed in og_params. */
og_status og_params_default(og_params *p);

/* ---- one system -------------------------------------------------------- */

/* Build the tree of N particles (Sect. 4.1.1): fixed point, Morton keys,
 * radix sort, octree topology and threading, moments, groups.
 * pos: double[N][3], mass: double[N] (finite, >= 0).  1 <= N < 2^26.
 * A node's mass and sums of m x are the exact sums over its particles, each
 * rounded once to double; its centre of mass is the grid point nearest to the
 * exact ratio (ties to even).  They are carried exactly in 192-bit integers,
 * so the nonzero masses may span at most 128 binary orders, from the lowest
 * set bit of the smallest to the top of the largest (equal masses, or masses
 * within a factor 2^75 of each other, always do).
 * Returns OG_ERR_ARG for NaN/inf inputs, negative masses, masses spanning
 * more than 128 binary orders, bad parameters or r_cut >= L/2. */
og_status og_tree_build(og_ctx *ctx, const double *pos, const double *mass, int64_t n,
                        const og_params *p, og_tree **out);

/* Refit for drifted positions of the same N particles (caller order, same
 * pointer convention as the build): the topology, groups and octant slots
 * of the build are kept; node sums, centres of mass, group boxes and node
 * extents are recomputed.  A node's extent is its cell joined with its
 * drifted members (per axis an interval on the periodic circle); the walk's
 * prune, boundary and opening tests then use the extent and its largest
 * side instead of the cell, so the lists stay correct for any drift.  The
 * cost grows with the drift (extents widen); rebuild when it is large. */
og_status og_tree_refit(og_tree *t, const double *pos);

/* Short-range accelerations (Sect. 4.1.2, 4.1.3, 4.2).
 * a_old: float[N][3] previous accelerations for OG_OPEN_REL, or NULL (then a
 *        first Barnes-Hut pass with theta_first_pass supplies them);
 * acc:   float[N][3] out;  n_pp, n_pn: uint32[N] out or NULL.
 * n_pp(i) = PP entries of i's group list minus itself, n_pn(i) = PN entries. */
og_status og_tree_force(og_tree *t, const float *a_old, float *acc, uint32_t *n_pp,
                        uint32_t *n_pn);

/* og_tree_force with double-precision output (the accelerations a caller in
 * FP64 keeps): the same walk and the same FP32 sums, but the last pass
 * leaves them in grid units and the conversion to G M / L^2 is one FP64
 * multiplication by G (2^32 / L)^2, so the output carries no FP32 rounding
 * of that scaling.  acc: double[N][3] out; other arguments as og_tree_force.
 * Trees of og_tree_build only (one box); else OG_ERR_ARG. */
og_status og_tree_force_f64(og_tree *t, const float *a_old, double *acc, uint32_t *n_pp,
                            uint32_t *n_pn);

og_status og_tree_info_get(const og_tree *t, og_tree_info *info);

/* Long-range particle-mesh acceleration of every particle (Sect. 4.2
 * "Particle Mesh"): the erf part of the split potential, which og_tree_force
 * leaves out, so that og_tree_force + og_tree_pm_force is the TreePM force.
 * The tree's particles are assigned to an Ng^3 mesh by cloud-in-cell
 * (mesh point (i, j, l) at (i, j, l) L / Ng); the density is Fourier
 * transformed (cuFFT, FP32), multiplied by -4 pi G / k^2 exp(-k^2 r_s^2)
 * divided by the squared CIC window prod_a sinc^4(k_a L / 2 Ng) (the k = 0 mode
 * is zero), and transformed back; a = -grad phi by the fourth-order central
 * difference on the mesh, interpolated to the particles with the CIC weights.
 * The assignment sums 64-bit fixed-point integers, so the result does not
 * depend on the order of the additions.
 *   mesh: Ng, a power of two in [2, 1024]; r_s = the tree's og_params.r_s > 0.
 *   acc:  float[N][3] out, G M / L^2, the caller's particle order (device
 *         memory if the tree was built with OG_DEVICE_PTRS).
 * Device memory: 16 B per mesh point (plus cuFFT's work area), allocated and
 * freed on the context's stream; OG_ERR_BUDGET if above the context budget.
 * Trees of og_tree_build only (one box); OG_ERR_ARG otherwise, for a bad mesh
 * size or r_s <= 0; OG_ERR_CUDA if cuFFT cannot be loaded or fails. */
og_status og_tree_pm_force(og_tree *t, int32_t mesh, float *acc);

/* SPH density of every particle at given smoothing lengths (Sect. 6 "Smoothed
 * Particle Hydrodynamics"), with the grouped neighbour search of Sect. 3.4:
 * rho_i = sum_j m_j W(|x_i - x_j|, h_i) over the particles j closer than h_i,
 * i itself included, with the cubic spline W = 8 / (pi h^3) w(r / h),
 * w(q) = 1 - 6 q^2 + 6 q^3 (q < 1/2), 2 (1 - q)^3 (1/2 <= q < 1).  The search
 * runs once per walk group of the tree.  j is a neighbour of i iff
 * r2 < h2 in float32, r2 = (fx fx + fy fy) + fz fz with f the float32 of the
 * exact minimum-image grid separation and h2 = hg hg, hg = float32(h 2^32 / L)
 * (each operation rounded on its own), so n_ngb is an exact integer of those
 * inputs.  The density sums in float32.
 *   h:     float[N] in, 0 < h < L / 2, the caller's particle order.
 *   rho:   float[N] out (mass / L^3 units of the inputs), the caller's order.
 *   n_ngb: uint32[N] out or NULL: the neighbour count, i itself included.
 * Device pointers if the tree was built with OG_DEVICE_PTRS.  Trees of
 * og_tree_build only (one box), not refitted (OG_ERR_STATE); an h out of range
 * gives OG_ERR_ARG. */
og_status og_tree_sph_density(og_tree *t, const float *h, float *rho, uint32_t *n_ngb);

/* Smoothing lengths from the paper's neighbour relation (Sect. 6):
 * (4 pi / 3) h_i^3 rho_i = N m_i, N = n_target, with the density and search of
 * og_tree_sph_density.  Per particle, N_eff = (4 pi / 3) h^3 rho / m (FP64 of
 * the FP32 density) is compared with N: within tol N the particle is done;
 * else h is multiplied (too few neighbours) or divided (too many) by 1.26 until
 * a bracket [lo, hi] is known, then set to cbrt((lo^3 + hi^3) / 2).  Each
 * iteration searches only the groups with a particle not yet done.  A particle
 * that needs h near L / 2 stops at 0.999 L / 2; a massless particle keeps its
 * h.  After the iterations, rho and n_ngb are those of og_tree_sph_density at
 * the final h.
 *   n_target: N > 32/3 (the self term alone gives N_eff = 32/3 for equal
 *             masses); tol in (0, 1); max_iter in [1, 1000].
 *   h:        float[N] in (the starting guesses, 0 < h < L / 2) and out.
 *   rho, n_ngb: as og_tree_sph_density (n_ngb may be NULL).
 *   iters:    out, or NULL: iterations run (max_iter if some particle did not
 *             converge).
 * Same trees, pointers and errors as og_tree_sph_density. */
og_status og_tree_sph_smoothing(og_tree *t, double n_target, double tol, int32_t max_iter,
                                float *h, float *rho, uint32_t *n_ngb, int32_t *iters);

/* ---- many independent boxes in one launch ------------------------------ */

/* One independent periodic system of a batch. */
typedef struct {
    const double *pos;       /* double[n][3] */
    const double *mass;      /* double[n] */
    int64_t n;               /* >= 1 */
    og_params params;        /* per-box box size, G, eps, r_s, theta, alpha; the opening
                                criterion, split on/off (r_s > 0), group_max and flags must
                                agree across the batch */
    const float *a_old;      /* float[n][3] for OG_OPEN_REL, or NULL (NULL for every box or none) */
    float *acc;              /* float[n][3] out */
    uint32_t *n_pp, *n_pn;   /* uint32[n] out, or NULL */
} og_box;

typedef struct {
    int64_t boxes, particles, groups, interactions;
    double ms_total, ms_build, ms_walk;   /* device time of the whole call, the build, the walk */
} og_batch_info;

/* Short-range accelerations of many independent boxes at once: one forest
 * (every box its own root, particles sorted by box then key), and one walk
 * launch per pass over the groups of all boxes, longest lists first.  Each
 * box's result equals og_tree_build + og_tree_force on that box alone
 * (same tree, lists and summation order).  Pointers follow OG_DEVICE_PTRS
 * of boxes[0].params.flags.  The total particle count must be < 2^26.
 * info may be NULL. */
og_status og_batch_force(og_ctx *ctx, int64_t nbox, const og_box *boxes, og_batch_info *info);

/* Copy one internal array of the tree to host memory (test and debug use).
 * field: one of og_field; bytes must equal the field's size:
 *   OG_F_SKEY     uint64[n]      sorted Morton keys
 *   OG_F_PERM     uint32[n]      sorted index -> caller index
 *   OG_F_SPOS     uint32[3][n]   sorted fixed-point positions (x row, y, z)
 *   OG_F_LEVEL    uint8[nodes]   node level (0 root .. 21)
 *   OG_F_NBEG     uint32[nodes]  first sorted particle of the node
 *   OG_F_NEND     uint32[nodes]  one past the last
 *   OG_F_PARENT   int32[nodes]   parent node (-1 root)
 *   OG_F_CBEG     uint32[nodes]  first entry of the node in the child array
 *   OG_F_CCNT     uint32[nodes]  number of children
 *   OG_F_CHILD    uint32[children] unified refs: particle < n, node id + n
 *   OG_F_MASS     double[nodes]  node mass
 *   OG_F_COM      uint32[nodes][3] centre of mass, fixed point
 *   OG_F_NEXTNODE int32[nodes]   first child (unified ref)
 *   OG_F_SIBLING  int32[nodes]   item after the node's subtree (-1 end)
 *   OG_F_PNEXT    int32[n]       item after a particle (-1 end)
 *   OG_F_GBEG     uint32[groups] first sorted particle of a group
 *   OG_F_GEND     uint32[groups] one past the last
 *   OG_F_GBOX     uint32[groups][6] integer bounding box lo xyz, hi xyz
 *   OG_F_LISTS    uint32[list_entries][2] (group, unified ref) pairs of the
 *                 last OG_DEBUG_DUMP_LISTS force call, in no particular order
 *   OG_F_EXTENT   uint32[2][nodes][3] after a refit: extent start per axis, then
 *                 extent length per axis (intervals on the circle of 2^32 units)
 *   OG_F_MSUM     double[nodes][3] sum of m x per axis, x in grid units */
enum {
    OG_F_SKEY = 0, OG_F_PERM, OG_F_SPOS, OG_F_LEVEL, OG_F_NBEG, OG_F_NEND, OG_F_PARENT,
    OG_F_CBEG, OG_F_CCNT, OG_F_CHILD, OG_F_MASS, OG_F_COM, OG_F_NEXTNODE, OG_F_SIBLING,
    OG_F_PNEXT, OG_F_GBEG, OG_F_GEND, OG_F_GBOX, OG_F_LISTS, OG_F_EXTENT, OG_F_MSUM
};
og_status og_tree_export(const og_tree *t, int field, void *host_dst, size_t bytes);

og_status og_tree_free(og_tree *t);

/* og_tree_force plus the short-range potential of every particle (pot:
 * float[n], caller order, host or device like acc), from the same lists in the
 * same pass: phi_i = -G sum_j m_j psi(r) erfc(r / 2 r_s) (Sect. 4.2, phi_s =
 * -G m erfc(u) / r), psi the potential of the spline mass distribution used by
 * the force (psi = 1/r for r >= h, 1/eps at r = 0); the particle itself and
 * entries beyond the cutoff contribute nothing.  Accelerations and counts are
 * those of og_tree_force.  OG_DEBUG_DUMP_LISTS does not apply to this call. */
og_status og_tree_force_pot(og_tree *t, const float *a_old, float *acc, float *pot,
                            uint32_t *n_pp, uint32_t *n_pn);

/* Forces on the active particles only: the individual time steps of Sect.
 * 3.2 need new accelerations only for the particles whose time bin is
 * active.  active: uint8_t[n] in the caller's order, nonzero = active (host,
 * or device with OG_DEVICE_PTRS).  Every group holding at least one active
 * particle is walked exactly as og_tree_force walks it (the same list for all
 * its members, the same arithmetic), so an active particle's acceleration and
 * counts equal those of og_tree_force on the same tree; the entries of acc,
 * n_pp, n_pn of inactive particles are left as they were.  OG_OPEN_REL:
 * a_old as in og_tree_force, else a Barnes-Hut first pass over the same
 * groups.  *groups_walked (may be NULL) receives the number of groups walked;
 * with no active particle nothing is walked and the outputs are untouched. */
og_status og_tree_force_active(og_tree *t, const uint8_t *active, const float *a_old, float *acc,
                               uint32_t *n_pp, uint32_t *n_pn, int64_t *groups_walked);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char *og_last_error(void);

/* ---- serving: continuous batching of requests --------------------------- */

/* One served request: a system integrated for nsteps steps of
 *   a = short-range acceleration at x;  v += a dt_kick;  x += v dt_drift
 * (positions wrapped into the box).  All arrays are host memory; the input
 * arrays are copied by og_serve_submit.  acc_out / pos_out (caller-owned, may
 * be NULL) receive the accelerations of the last force evaluation and the
 * final positions; they must stay valid until og_serve_poll returns OG_OK. */
typedef struct {
    int64_t n;
    const double *pos;       /* double[n][3] */
    const double *vel;       /* double[n][3], box lengths per unit drift time */
    const double *mass;      /* double[n] */
    og_params params;        /* Barnes-Hut opening; host pointers */
    int32_t nsteps;          /* >= 1 */
    double dt_kick, dt_drift;
    float *acc_out;          /* float[n][3] or NULL */
    double *pos_out;         /* double[n][3] or NULL */
} og_request;

typedef struct {
    int64_t n, steps, rebuilds, refits;
    double t_submit, t_start, t_done;   /* seconds on a steady clock */
} og_result;

/* Queue a request (non-blocking).  The context's engine thread admits
 * requests in arrival order while the estimated device memory of the active
 * systems stays within the context's hbm_budget_bytes (0: no bound) and at
 * most 256 are active; it keeps each admitted system's tree, positions,
 * velocities and accelerations on the device, walks all active systems in
 * one launch per step, and after each step refits a system's tree or
 * rebuilds it, whichever its own interaction counts price lower for the next
 * step (a refitted tree is exact, but its lists grow with the drift).  The
 * decisions depend only on the system, so a request gets the same bits
 * served alone or in a mix.  OG_ERR_BUDGET if the system alone exceeds the
 * budget.  Thread safe. */
og_status og_serve_submit(og_ctx *ctx, const og_request *req, uint64_t *ticket);

/* Device memory the admission control charges for a request of n particles
 * against hbm_budget_bytes. */
size_t og_serve_request_bytes(int64_t n);

/* Wait up to timeout_ms (0: do not wait, < 0: wait as long as needed) for a
 * ticket.  OG_OK and *out filled when done (a ticket can be collected once),
 * OG_PENDING if not done yet, a negative status if the request failed.
 * Thread safe. */
og_status og_serve_poll(og_ctx *ctx, uint64_t ticket, og_result *out, int timeout_ms);

/* Cancel a queued or running request (a service of the serving loop; the
 * paper has no counterpart).  OG_OK: the cancellation is recorded.  A queued
 * request is dropped at once; a running one is dropped before its next
 * engine step, its device memory is freed, and its output arrays are not
 * written after that.  og_serve_poll then returns OG_ERR_CANCELLED, or OG_OK
 * if the request finished its last step before the engine took the
 * cancellation.  OG_ERR_STATE if the request has already finished or been
 * collected, OG_ERR_ARG for an unknown ticket.  Thread safe. */
og_status og_serve_cancel(og_ctx *ctx, uint64_t ticket);

/* ---- time integration: individual power-of-two time steps -------------- */

/* Kick-drift-kick leapfrog with individual time steps (Sect. 3.2).  One
 * maximum step dt_max is 2^max_bin ticks; a particle in bin b steps by
 * dt_max / 2^b and is active at the ticks that are multiples of 2^(max_bin - b).
 * Its bin is the smallest b with dt_max / 2^b <= sqrt(2 eta eps / |a|) (the
 * acceleration criterion of Sect. 3.2, eps = og_params.eps), at most max_bin;
 * a particle only enters a bin whose period divides the current tick.  Per
 * tick every particle drifts by v dt_max / 2^max_bin (wrapped into the box),
 * the active particles get new accelerations (og_tree_force_active on the tree
 * of the drifted positions: rebuilt every rebuild_every ticks, refitted in
 * between), their closing half kick with the old bin, and, except at the last
 * tick, a new bin and the opening half kick.  FP64 positions and velocities. */
typedef struct {
    double dt_max;           /* the longest step (bin 0), > 0 */
    double eta;              /* integration tolerance of the criterion (paper default 0.05) */
    int32_t max_bin;         /* finest bin, 0..30 */
    int32_t nsteps;          /* maximum steps to integrate, >= 1 */
    int32_t rebuild_every;   /* >= 1; 1 = a new tree every tick */
    int32_t pad;
} og_kdk_params;

typedef struct {
    int64_t ticks;           /* last tick index (nsteps * 2^max_bin) */
    int64_t forces;          /* accelerations computed, summed over ticks */
    int64_t groups_walked;   /* groups walked, summed over ticks */
    int64_t interactions;    /* PP + PN entries evaluated, summed over ticks */
    int64_t rebuilds, refits;
    double ms;               /* device time of the whole call */
} og_kdk_stats;

/* Integrate n particles (pos, vel: double[n][3] in/out, mass: double[n]; host
 * arrays, or device arrays with OG_DEVICE_PTRS in p->flags) for kp->nsteps
 * maximum steps.  acc_out (float[n][3]) and bins_out (int32[n]) receive the
 * last accelerations and bins (either may be NULL).  p as for og_tree_build
 * (eps > 0 required).  OG_ERR_ARG for invalid parameters; errors of the tree
 * calls are passed on. */
og_status og_kdk_run(og_ctx *ctx, int64_t n, double *pos, double *vel, const double *mass,
                     const og_params *p, const og_kdk_params *kp, float *acc_out,
                     int32_t *bins_out, og_kdk_stats *stats);

/* ---- group size: measured choice ---------------------------------------- */

/* The group size G (targets sharing one interaction list, Sect. 3.4 and
 * 18.2: one walk per group of nearby particles) trades list building against
 * evaluation; the paper fixes no value, nor the walk's launch shape (warps
 * per block, entries of the shared far-entry chunk).  og_tune_walk measures
 * all three for inputs of this kind: the key is (floor(log2 n), opening
 * criterion, split on/off).  The first call for a key builds and walks this
 * input once per candidate (both force passes for OG_OPEN_REL) and times the
 * walk kernels with CUDA events on the context's stream: G in {8, 16, 24, 32}
 * with 4 warps and 256 entries, then 2 and 8 warps at the best G, then 128 and
 * 512 entries at the best G and warps (coordinate descent, 8 trials).  The
 * result stays in the context; later calls return it at once.  og_tree_build
 * with params.group_max = 0 calls it (an explicit walk_warps or walk_chunk
 * then replaces the measured one).  pos/mass as in og_tree_build (host or,
 * with OG_DEVICE_PTRS, device); p->group_max, p->walk_warps and p->walk_chunk
 * are ignored; any output pointer may be NULL.  Errors as og_tree_build. */
og_status og_tune_walk(og_ctx *ctx, const double *pos, const double *mass, int64_t n,
                       const og_params *p, int32_t *group_max, int32_t *walk_warps,
                       int32_t *walk_chunk);

/* og_tune_walk's group size alone. */
og_status og_tune_group_max(og_ctx *ctx, const double *pos, const double *mass, int64_t n,
                            const og_params *p, int32_t *group_max);

/* Write the context's measured walk configurations to `path`, one JSON
 * object per line: {"n_log2": .., "opening": .., "split": .., "group_max": ..,
 * "walk_warps": .., "walk_chunk": .., "walk_ms": [8 trial times]}.
 * OG_ERR_ARG if the file cannot be written. */
og_status og_tune_save(og_ctx *ctx, const char *path);

/* Add the records of a file written by og_tune_save to the context (a record
 * replaces one with the same key).  OG_ERR_ARG, and nothing added, if a line
 * is not such a record or the file cannot be read. */
og_status og_tune_load(og_ctx *ctx, const char *path);

/* ---- measured FP32 throughput -------------------------------------------- */

/* The walk is bound by the FP32 ALUs, not by a contraction, so its roofline
 * is the FP32 fused multiply-add rate of this GPU.  og_measure_fp32_peak runs
 * independent chains of FP32 FMAs (and of f32x2 FMAs) on every SM at full
 * occupancy on the context's stream, times them with CUDA events (best of
 * three after one warm-up round, about 0.1 s in all) and returns the rates in
 * TFLOP/s (an FMA counts 2 flops, an f32x2 FMA 4).  The rates are at the
 * clocks the GPU runs at during the call.  OG_ERR_ARG on NULL arguments. */
og_status og_measure_fp32_peak(og_ctx *ctx, double *tflops_fma, double *tflops_fma2);

/* ---- sort without device allocation ------------------------------------ */

/* Largest n accepted by og_sort_keys_noalloc. */
#define OG_NOALLOC_MAX_N 1048576

/* Stable ascending radix sort of n 64-bit keys that allocates no memory.
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory when they need a sort -- a serving process that has
 * committed its whole HBM budget, or a latency-critical loop that cannot
 * afford cudaMalloc/cudaFree (which can synchronise the whole device).
 *   keys_in:  device uint64[n] (not modified unless it is keys_out);
 *   keys_out: device uint64[n], the sorted keys;
 *   perm_out: device uint32[n], perm_out[i] = index in keys_in of the i-th key
 *             (equal keys keep their input order);
 *   stream:   cudaStream_t of the current device, or NULL for the default stream.
 * The three buffers are device memory of the current device (else
 * OG_ERR_ARG); keys_out may be keys_in, and no other two of them may overlap
 * (OG_ERR_ARG).  All 64 key bits are sorted.
 * 1 <= n <= OG_NOALLOC_MAX_N, else OG_ERR_ARG.  The work is queued on `stream`
 * on the current device and the call returns before it finishes; synchronise
 * the stream before reading the outputs.
 * The scratch is a fixed static device array of about 16 MB that every GPU
 * loading this library holds until the process exits.  The first call on a
 * device looks up that array's device address (once per device, with the
 * device current); make that first call before any stream capture.  With
 * CUDA's lazy module loading that first call may also be when the array is
 * reserved, and it fails with OG_ERR_CUDA if the device has no room left:
 * make it at set-up, before committing the rest of the device's memory.  All
 * calls share the one array: calls whose work overlaps on the GPU (on
 * different streams, or from different threads) race and corrupt each
 * other's results; serialise them on one stream.  The array carries no state
 * from one call to the next. */
og_status og_sort_keys_noalloc(const uint64_t *keys_in, uint64_t *keys_out, uint32_t *perm_out,
                               int64_t n, void *stream);

/* Number of CUDA kernels this library has launched in this process so far
 * (for benchmarks that count their own launches in a timed region). */
int64_t og_kernel_launches(void);

/* The compute capability the library's device code was compiled for, as
 * major * 10 + minor of the code the current device runs (103 for sm_103a).
 * A diagnostic with no counterpart in the paper: it lets a caller confirm
 * that native GB300 code is loaded rather than PTX compiled at run time.
 * version: out.  OG_ERR_ARG on NULL; OG_ERR_CUDA without a usable device. */
og_status og_device_code_version(int32_t *version);

/* Failure injection for tests of error handling (the paper has no
 * counterpart): of the device allocations the library makes next, in any
 * context, the first `skip` go through and the following `count` fail as if
 * the device had no memory left, so each affected call returns OG_ERR_OOM
 * and leaves its context usable.  count = 0 clears the injection.
 * OG_ERR_ARG if skip or count < 0.  Nothing reaches the GPU: the failure is
 * made on the host, before the allocation is asked for. */
og_status og_debug_fail_allocations(int32_t skip, int32_t count);

/* Test of the bounded device-side waits (the paper has no counterpart).  The
 * build's short scans and small sorts run as one kernel in which a tile waits
 * for the counts that earlier tiles publish, up to a poll limit.  This runs
 * that scan over n zeros (2 to 64 tiles of 4096 elements, 4097 <= n <=
 * 262144) with the first tile never taken, so the second tile's wait runs
 * out; the kernel then gives up, finishes, and the call returns
 * OG_ERR_TIMEOUT, after which the context is usable as before.  It allocates
 * and frees its own scratch.  OG_ERR_ARG for a NULL context or n out of
 * range. */
og_status og_debug_scan_wait_timeout(og_ctx *c, int64_t n);

#ifdef __cplusplus
}
#endif
#endif /* OG_H */

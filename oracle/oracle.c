/*
 * oracle.c -- plain FP64 CPU oracle of the short-range TreePM tree force.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg call this code.  The CUDA library never
 * links, loads or calls it, and the two share no source, header or table.
 *
 * What it computes, step by step, in the order of the paper (OpenGadget3,
 * Sect. 4.1 "Oct-Tree", Sect. 4.1.1 "Tree construction", Sect. 4.1.2
 * "Tree walk", Sect. 4.1.3 "Force evaluation", Sect. 4.2 "Particle Mesh" for
 * the short-range split):
 *
 *   a1  positions -> 32-bit fixed point on the periodic box
 *   a2  63-bit Morton keys (21 bits per axis, x highest)
 *   a3  stable sort of the keys (ties by input index)
 *   a4  octree: the root covers the box and is split into eight sub-cubes
 *       recursively until a sub-cube holds at most leaf_max particles;
 *       chains of single-child cells are compressed (a node is the smallest
 *       cell that holds its particles); level-21 cells that still hold more
 *       than leaf_max particles (coincident keys) are buckets
 *   a4' the two-pointer threading of Sect. 4.1.1 (nextnode / sibling) in a
 *       unified index space: particles 0..N-1, nodes N..N+M-1, end = -1
 *   a5  monopole moments: mass and centre of mass, exact sums rounded once
 *   a6  groups of spatially close particles (Sect. 3.4 and 18.2: one walk
 *       per group of nearby particles)
 *   a7  per group: tree walk with Barnes-Hut or relative opening, a boundary
 *       check, and the short-range cutoff, producing particle-node (PN) and
 *       particle-particle (PP) entries
 *   a8  per target: sum over the group's entries of the spline-softened
 *       Newtonian force times the erfc split factor, periodic minimum image
 *   a9  relative criterion: a second pass with the previous accelerations
 *
 * Readings of points the paper leaves open:
 *   - units: G and the box length L are parameters; positions are reduced to
 *     the torus [0, L)^3.
 *   - fixed point: u = floor(frac(t) * 2^32) with t = x/L in FP64, evaluated
 *     exactly as floor(t * 2^32) mod 2^32 (no rounding after the division).
 *   - minimum image: dx = x_j - x_i as a 32-bit two's-complement difference;
 *     an exact half-box separation maps to -L/2.
 *   - softening: h = 2.8 eps (Sect. 4.1.3, Plummer-equivalent eps).  The
 *     softened force is that of the cubic-spline mass distribution with
 *     compact support h (appendix "Available kernel functions", 3D cubic
 *     spline), i.e. g(r) = G M(<r) / r^3 with M(<h) = 1:
 *        u = r/h < 1/2 : g = h^-3 (32/3 - 192/5 u^2 + 32 u^3)
 *        1/2 <= u < 1  : g = h^-3 (64/3 - 48 u + 192/5 u^2 - 32/3 u^3
 *                                  - 1/(15 u^3))
 *        u >= 1        : g = r^-3
 *   - split: phi_s = -G m erfc(r / 2 r_s) / r (Sect. 4.2), so the radial
 *     force factor is S(r) = erfc(r/2r_s) + r/(sqrt(pi) r_s) exp(-r^2/4r_s^2);
 *     softening and split multiply.  r_s <= 0 switches the split and the
 *     cutoff off.
 *   - cutoff: an entry contributes iff 0 < r < r_cut, r_cut = rcut_over_rs
 *     r_s < L/2.  Because the cutoff is a step, the in/out decision is taken
 *     in the same single precision as the CUDA path: dx as float (round to
 *     nearest), r2 = fma(dx, dx, fma(dy, dy, dz*dz)) in grid units, compared
 *     with (float)(rcut_grid^2).  Everything after the decision is FP64.
 *   - tree: see a4 above; children ordered by key.
 *   - moments (FP64 monopoles, Sect. 4.1.1): a node's mass M and its sums
 *     S = sum m x per axis (x the integer grid coordinates of its particles)
 *     are the exact real sums, each rounded once to the nearest double (ties
 *     to even), so no order of additions is implied.  The centre of mass is
 *     the grid point nearest to the exact S / M, ties to even; a massless
 *     node takes its cell centre.  The sums are carried exactly as integers
 *     (see a5).  Elsewhere no fused multiply adds (-ffp-contract=off).
 *   - groups: children with more than G particles are recursed into.  At a
 *     node that holds at most 8 G particles (and at the root), maximal runs of
 *     consecutive "small" children (particles, or nodes with at most G
 *     particles) are cut, in key order, into groups of G (the last one
 *     shorter).  At a node with more than 8 G particles the small children
 *     are not merged: each one is a group of its own, so that a group never
 *     spans the octants of a cell much larger than its own neighbourhood.
 *   - geometry of a group: the integer bounding box of its members.  All
 *     distances between a group box and a point or a cell are taken per axis
 *     on the circle of 2^32 grid units (0 when overlapping).
 *   - prune: a node or particle is skipped iff the squared grid distance
 *     between the group box and the node cell (or particle) exceeds
 *     Rp = (uint64)(rcut_grid^2 * (1 + 2^-10)).
 *   - boundary check: a node is opened iff the group box meets the node cell
 *     enlarged to a half width of 0.6 of its side (integer test
 *     10 d_c <= 6 l per axis, d_c = distance from the cell centre to the box).
 *   - Barnes-Hut: open iff l^2 > theta^2 d^2, d = distance from the group box
 *     to the node's centre of mass, l = cell side; d^2 = (dx*dx + dy*dy) + dz*dz
 *     in FP64, every product and sum rounded, no fused operations.
 *   - relative: open iff (G M) l^2 > (alpha a_min s^2) (d^2 d^2), s = L/2^32,
 *     a_min = min over the group of |a_old|, |a| = sqrt((ax ax + ay ay) + az az)
 *     in FP64 of the single-precision previous acceleration.
 *   - counts: n_pp(i) = number of PP entries of i's group minus one (itself),
 *     n_pn(i) = number of PN entries of the group.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "oracle.h"

#define TWO32 4294967296.0
#define ORA_PI 3.14159265358979323846
#define KEY_LEVELS 21

/* ------------------------------------------------------------------------ */
/* a1: fixed-point positions                                                 */
/* ------------------------------------------------------------------------ */

int ora_quantize1(double v, double box, uint32_t *out)
{
    if (!isfinite(v)) return ORA_ERR_ARG;
    double t = v / box;
    if (fabs(t) < 2147483648.0) {
        /* t * 2^32 is exact and below 2^63 in magnitude: floor it, keep the low
           32 bits (the same as floor(frac(t) * 2^32), exactly, for either sign) */
        int64_t q = (int64_t)floor(t * TWO32);
        *out = (uint32_t)(uint64_t)q;
    } else {
        /* |t| >= 2^31: t - floor(t) is exact */
        double f = t - floor(t);
        *out = (uint32_t)floor(f * TWO32);
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* a2: Morton key, bit by bit                                                */
/* ------------------------------------------------------------------------ */

uint64_t ora_morton(uint32_t x, uint32_t y, uint32_t z)
{
    uint64_t k = 0;
    for (int b = 31; b >= 32 - KEY_LEVELS; --b) {
        k = (k << 3) | ((uint64_t)((x >> b) & 1u) << 2) |
            ((uint64_t)((y >> b) & 1u) << 1) | (uint64_t)((z >> b) & 1u);
    }
    return k;
}

/* octant digit of a key at level l (1..21): the l-th 3-bit group from the top */
static inline int digit_at(uint64_t key, int l)
{
    return (int)((key >> (3 * (KEY_LEVELS - l))) & 7u);
}

/* number of leading 3-bit digits two keys share (21 when equal) */
static int common_levels(uint64_t a, uint64_t b)
{
    int l = 0;
    while (l < KEY_LEVELS && digit_at(a, l + 1) == digit_at(b, l + 1)) l++;
    return l;
}

/* ------------------------------------------------------------------------ */
/* tree record                                                               */
/* ------------------------------------------------------------------------ */

struct ora_tree {
    int64_t n, nnodes, nchild, ngroups;
    ora_params p;
    /* input order */
    uint32_t *x, *y, *z;
    uint64_t *key;
    /* sorted order */
    int64_t *perm;          /* sorted index -> input index */
    uint64_t *skey;
    uint32_t *sx, *sy, *sz;
    double *sm;
    /* nodes, ids in depth-first preorder, children in key order */
    int32_t *level;
    int64_t *beg, *end, *parent, *cbeg, *ccnt;
    int64_t *child;         /* unified refs: particle < n, node id + n */
    double *M, *Sx, *Sy, *Sz;
    uint32_t *cx, *cy, *cz;
    int64_t *nextnode, *sibling, *pnext;
    uint32_t *ox, *oy, *oz; /* cell origin of each node (fixed by the build) */
    uint32_t *es, *el;      /* after a refit: extent start and length, 3 per node */
    int refit;
    int fb, fnl;            /* exact sums: units of 2^fb, fnl 64-bit limbs */
    /* groups */
    int64_t *gbeg, *gend;
    uint32_t *glo, *ghi;    /* 3 per group */
    /* last force call */
    int64_t *list_off;      /* ngroups + 1, when lists are kept */
    int64_t *list;
    int64_t list_len;
};

static void *xcalloc(size_t n, size_t sz)
{
    if (n == 0) n = 1;
    return calloc(n, sz);
}

void ora_tree_free(ora_tree *t)
{
    if (!t) return;
    void *ptrs[] = {t->x, t->y, t->z, t->key, t->perm, t->skey, t->sx, t->sy, t->sz,
                    t->sm, t->level, t->beg, t->end, t->parent, t->cbeg, t->ccnt,
                    t->child, t->M, t->Sx, t->Sy, t->Sz, t->cx, t->cy, t->cz,
                    t->nextnode, t->sibling, t->pnext, t->gbeg, t->gend, t->glo,
                    t->ghi, t->list_off, t->list, t->ox, t->oy, t->oz, t->es, t->el};
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) free(ptrs[i]);
    free(t);
}

/* ------------------------------------------------------------------------ */
/* a3: stable sort by key, ties by input index                               */
/* ------------------------------------------------------------------------ */

static const uint64_t *g_sort_keys;

static int cmp_key_index(const void *a, const void *b)
{
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    uint64_t ki = g_sort_keys[i], kj = g_sort_keys[j];
    if (ki < kj) return -1;
    if (ki > kj) return 1;
    return (i < j) ? -1 : (i > j);
}

/* ------------------------------------------------------------------------ */
/* a4: recursive octree construction                                         */
/* ------------------------------------------------------------------------ */

static int64_t build_node(ora_tree *t, int level, int64_t b, int64_t e, int64_t parent)
{
    int64_t id = t->nnodes++;
    t->level[id] = level;
    t->beg[id] = b;
    t->end[id] = e;
    t->parent[id] = parent;
    {
        /* the cell: the top `level` bits of every coordinate of its particles */
        uint32_t mask = level == 0 ? 0u : (uint32_t)~(((uint64_t)1 << (32 - level)) - 1);
        t->ox[id] = t->sx[b] & mask;
        t->oy[id] = t->sy[b] & mask;
        t->oz[id] = t->sz[b] & mask;
    }
    t->cbeg[id] = t->nchild;
    int64_t pend_pos[8], pend_b[8], pend_e[8];
    int npend = 0;
    if (level == KEY_LEVELS) {
        /* bucket: coincident keys, every particle hangs from the node */
        for (int64_t q = b; q < e; ++q) t->child[t->nchild++] = q;
    } else {
        int64_t q0 = b;
        while (q0 < e) {
            int d = digit_at(t->skey[q0], level + 1);
            int64_t q1 = q0 + 1;
            while (q1 < e && digit_at(t->skey[q1], level + 1) == d) q1++;
            if (q1 - q0 <= t->p.leaf_max) {
                for (int64_t q = q0; q < q1; ++q) t->child[t->nchild++] = q;
            } else {
                pend_pos[npend] = t->nchild;
                pend_b[npend] = q0;
                pend_e[npend] = q1;
                npend++;
                t->child[t->nchild++] = -1; /* filled below with the child's id */
            }
            q0 = q1;
        }
    }
    t->ccnt[id] = t->nchild - t->cbeg[id];
    for (int k = 0; k < npend; ++k) {
        /* the child is the smallest cell that holds the octant's particles */
        int lc = common_levels(t->skey[pend_b[k]], t->skey[pend_e[k] - 1]);
        int64_t c = build_node(t, lc, pend_b[k], pend_e[k], id);
        t->child[pend_pos[k]] = c + t->n;
    }
    return id;
}

/* ------------------------------------------------------------------------ */
/* a5: monopole moments, exact                                               */
/* ------------------------------------------------------------------------ */

/* A nonzero mass is m = s 2^e with an integer s < 2^53 (frexp).  With b the
 * lowest exponent of a set bit over all masses of the tree, every mass is an
 * integer multiple of 2^b, and so is every product m x with x an integer grid
 * coordinate.  The sums are kept as unsigned integers of t->fnl 64-bit limbs
 * (least significant first) in units of 2^b, so they are exact whatever the
 * order of the additions, and are rounded once at the end. */

static void fx_zero(uint64_t *a, int nl) { memset(a, 0, (size_t)nl * 8); }

static void fx_add(uint64_t *a, const uint64_t *c, int nl)
{
    uint64_t carry = 0;
    for (int k = 0; k < nl; ++k) {
        uint64_t s = a[k] + carry;
        uint64_t c1 = s < carry;
        uint64_t r = s + c[k];
        a[k] = r;
        carry = c1 + (r < s);
    }
}

static void fx_sub(uint64_t *a, const uint64_t *c, int nl) /* a -= c, a >= c */
{
    uint64_t borrow = 0;
    for (int k = 0; k < nl; ++k) {
        uint64_t d = a[k] - c[k];
        uint64_t b1 = a[k] < c[k];
        uint64_t r = d - borrow;
        b1 += d < borrow;
        a[k] = r;
        borrow = b1;
    }
}

static int fx_cmp(const uint64_t *a, const uint64_t *c, int nl)
{
    for (int k = nl - 1; k >= 0; --k)
        if (a[k] != c[k]) return a[k] < c[k] ? -1 : 1;
    return 0;
}

/* out (nl limbs) = a (nl limbs) * x; the product fits nl limbs */
static void fx_mul_u32(const uint64_t *a, uint32_t x, uint64_t *out, int nl)
{
    unsigned __int128 carry = 0;
    for (int k = 0; k < nl; ++k) {
        unsigned __int128 p = (unsigned __int128)a[k] * x + carry;
        out[k] = (uint64_t)p;
        carry = p >> 64;
    }
}

/* index of the highest set bit, -1 for zero */
static int fx_top(const uint64_t *a, int nl)
{
    for (int k = nl - 1; k >= 0; --k)
        if (a[k]) return 64 * k + 63 - __builtin_clzll(a[k]);
    return -1;
}

static int fx_bit(const uint64_t *a, int nl, int i)
{
    if (i < 0 || i >= 64 * nl) return 0;
    return (int)((a[i / 64] >> (i % 64)) & 1u);
}

/* bits [lo, lo + 53) of a as an integer (bits below 0 read as zero) */
static uint64_t fx_bits53(const uint64_t *a, int nl, int lo)
{
    uint64_t v = 0;
    for (int i = 52; i >= 0; --i) v = (v << 1) | (uint64_t)fx_bit(a, nl, lo + i);
    return v;
}

/* the mass as an integer in units of 2^b */
static void fx_mass(double m, int b, uint64_t *out, int nl)
{
    fx_zero(out, nl);
    if (m == 0.0) return;
    int e;
    double fr = frexp(m, &e);                        /* m = fr 2^e, fr in [1/2, 1) */
    uint64_t s = (uint64_t)ldexp(fr, 53);           /* m = s 2^(e - 53), exactly */
    for (int i = 0; i < 53; ++i) {
        if (!((s >> i) & 1u)) continue;
        int pos = i + e - 53 - b;                   /* >= 0 by the choice of b */
        out[pos / 64] |= (uint64_t)1 << (pos % 64);
    }
}

/* a 2^b rounded to the nearest double, ties to even (subnormal results and
 * overflow to infinity as IEEE 754 rounds them) */
static double fx_to_double(const uint64_t *a, int nl, int b)
{
    int p = fx_top(a, nl);
    if (p < 0) return 0.0;
    /* position of the last kept bit: 53 significant bits, or the 2^-1074 grid */
    int lsb = (p + b >= -1022) ? p - 52 : -1074 - b;
    uint64_t mant = fx_bits53(a, nl, lsb);
    if (lsb > 0 && fx_bit(a, nl, lsb - 1)) {
        int sticky = 0;
        for (int i = 0; i < lsb - 1 && !sticky; ++i) sticky = fx_bit(a, nl, i);
        if (sticky || (mant & 1u)) mant += 1;
    }
    return ldexp((double)mant, lsb + b);
}

/* the integer nearest to S / M (M > 0, S / M < 2^32), ties to even */
static uint32_t fx_round_ratio(const uint64_t *S, const uint64_t *M, int nl)
{
    uint64_t qM[64], R[64], twoR[64];
    int pS = fx_top(S, nl), pM = fx_top(M, nl);
    int64_t q = 0;
    if (pS >= 0) {
        /* a first guess from the leading bits; the loops below make it exact */
        double r = ldexp((double)fx_bits53(S, nl, pS - 52) / (double)fx_bits53(M, nl, pM - 52),
                         pS - pM);
        q = (int64_t)floor(r);
        if (q < 0) q = 0;
        if (q > 4294967295ll) q = 4294967295ll;
    }
    fx_mul_u32(M, (uint32_t)q, qM, nl);
    while (q > 0 && fx_cmp(qM, S, nl) > 0) { q -= 1; fx_sub(qM, M, nl); }
    for (;;) {                                       /* largest q with q M <= S */
        memcpy(R, qM, (size_t)nl * 8);
        fx_add(R, M, nl);
        if (fx_cmp(R, S, nl) > 0) break;
        q += 1;
        memcpy(qM, R, (size_t)nl * 8);
    }
    memcpy(R, S, (size_t)nl * 8);
    fx_sub(R, qM, nl);                               /* R = S - q M in [0, M) */
    memcpy(twoR, R, (size_t)nl * 8);
    fx_add(twoR, R, nl);
    int c = fx_cmp(twoR, M, nl);
    if (c > 0 || (c == 0 && (q & 1))) q += 1;
    return (uint32_t)q;
}

/* Exact sums of the node's particles (mass and m x, m y, m z: 4 nl limbs at
 * acc), from its children: particles directly, child nodes by recursion.
 * Stores the node's mass and sums rounded once to FP64 and its centre of mass
 * on the grid.  acc + 4 nl onwards is scratch for the deeper levels. */
static void node_sums(ora_tree *t, int64_t id, uint64_t *acc)
{
    const int64_t n = t->n;
    const int nl = t->fnl;
    uint64_t *sub = acc + 4 * nl;
    uint64_t v[64], w[64];
    fx_zero(acc, 4 * nl);
    for (int64_t k = 0; k < t->ccnt[id]; ++k) {
        int64_t c = t->child[t->cbeg[id] + k];
        if (c < n) {
            fx_mass(t->sm[c], t->fb, v, nl);
            fx_add(acc, v, nl);
            fx_mul_u32(v, t->sx[c], w, nl);
            fx_add(acc + nl, w, nl);
            fx_mul_u32(v, t->sy[c], w, nl);
            fx_add(acc + 2 * nl, w, nl);
            fx_mul_u32(v, t->sz[c], w, nl);
            fx_add(acc + 3 * nl, w, nl);
        } else {
            node_sums(t, c - n, sub);
            for (int q = 0; q < 4; ++q) fx_add(acc + q * nl, sub + q * nl, nl);
        }
    }
    t->M[id] = fx_to_double(acc, nl, t->fb);
    t->Sx[id] = fx_to_double(acc + nl, nl, t->fb);
    t->Sy[id] = fx_to_double(acc + 2 * nl, nl, t->fb);
    t->Sz[id] = fx_to_double(acc + 3 * nl, nl, t->fb);
    if (fx_top(acc, nl) >= 0) {
        t->cx[id] = fx_round_ratio(acc + nl, acc, nl);
        t->cy[id] = fx_round_ratio(acc + 2 * nl, acc, nl);
        t->cz[id] = fx_round_ratio(acc + 3 * nl, acc, nl);
    } else {
        /* massless node: the cell centre */
        const int level = t->level[id];
        uint32_t side_shift = 32 - level; /* cell side = 2^(32-level) grid units */
        uint64_t half = (uint64_t)1 << (side_shift - 1);
        uint64_t mask = (level == 0) ? 0 : ~(((uint64_t)1 << side_shift) - 1);
        uint64_t q = t->beg[id];
        t->cx[id] = (uint32_t)(((uint64_t)t->sx[q] & mask) + half);
        t->cy[id] = (uint32_t)(((uint64_t)t->sy[q] & mask) + half);
        t->cz[id] = (uint32_t)(((uint64_t)t->sz[q] & mask) + half);
    }
}

/* the fixed-point format of a tree's masses: b and the limb count */
static int mass_format(ora_tree *t)
{
    int lo = 0, hi = 0, any = 0;
    for (int64_t i = 0; i < t->n; ++i) {
        double m = t->sm[i];
        if (m == 0.0) continue;
        int e;
        double fr = frexp(m, &e);
        uint64_t s = (uint64_t)ldexp(fr, 53);
        int l = e - 53 + __builtin_ctzll(s);          /* lowest set bit of m */
        if (!any || l < lo) lo = l;
        if (!any || e > hi) hi = e;                   /* m < 2^e */
        any = 1;
    }
    t->fb = any ? lo : 0;
    /* a mass below 2^(hi - lo), a coordinate below 2^32, fewer than 2^63
       terms: hi - lo + 95 bits hold every sum */
    int bits = (any ? hi - lo : 1) + 95;
    t->fnl = (bits + 63) / 64;
    return t->fnl <= 40 ? ORA_OK : ORA_ERR_ARG;      /* finite doubles need at most 38 */
}

/* moments of every node, from the root down and back up */
static int all_moments(ora_tree *t)
{
    uint64_t *work = (uint64_t *)calloc((size_t)(KEY_LEVELS + 3) * 4 * t->fnl, 8);
    if (!work) return ORA_ERR_OOM;
    node_sums(t, 0, work);
    free(work);
    return ORA_OK;
}

static void thread_node(ora_tree *t, int64_t id, int64_t after)
{
    const int64_t n = t->n;
    int64_t cb = t->cbeg[id], cc = t->ccnt[id];
    t->nextnode[id] = cc > 0 ? t->child[cb] : after;
    for (int64_t k = 0; k < cc; ++k) {
        int64_t c = t->child[cb + k];
        int64_t nxt = (k + 1 < cc) ? t->child[cb + k + 1] : after;
        if (c < n) {
            t->pnext[c] = nxt;
        } else {
            t->sibling[c - n] = nxt;
            thread_node(t, c - n, nxt);
        }
    }
}

/* a6: groups */
static void emit_run(ora_tree *t, int64_t rb, int64_t re)
{
    int64_t G = t->p.group_max;
    for (int64_t s = rb; s < re; s += G) {
        int64_t e = (s + G < re) ? s + G : re;
        int64_t g = t->ngroups++;
        t->gbeg[g] = s;
        t->gend[g] = e;
    }
}

static void make_groups(ora_tree *t, int64_t id)
{
    const int64_t n = t->n;
    int64_t G = t->p.group_max;
    int64_t rb = -1, re = -1;
    const int merge = t->end[id] - t->beg[id] <= 8 * G;
    for (int64_t k = 0; k < t->ccnt[id]; ++k) {
        int64_t c = t->child[t->cbeg[id] + k];
        int64_t cb, ce;
        if (c < n) {
            cb = c;
            ce = c + 1;
        } else {
            int64_t j = c - n;
            cb = t->beg[j];
            ce = t->end[j];
            if (ce - cb > G) {
                if (rb >= 0) emit_run(t, rb, re);
                rb = re = -1;
                make_groups(t, j);
                continue;
            }
        }
        if (!merge) {
            emit_run(t, cb, ce);
            continue;
        }
        if (rb < 0) rb = cb;
        re = ce;
    }
    if (rb >= 0) emit_run(t, rb, re);
}

/* integer bounding box of every group, per axis an interval on the circle:
 * the member offsets from the first member, min to max (a drifted group may
 * wrap through 0) */
static void group_boxes(ora_tree *t)
{
    for (int64_t g = 0; g < t->ngroups; ++g) {
        const uint32_t *xs[3] = {t->sx, t->sy, t->sz};
        for (int a = 0; a < 3; ++a) {
            uint32_t ref = xs[a][t->gbeg[g]];
            int64_t lo = 0, hi = 0;
            for (int64_t q = t->gbeg[g]; q < t->gend[g]; ++q) {
                int64_t d = (int64_t)(int32_t)(uint32_t)(xs[a][q] - ref);
                if (d < lo) lo = d;
                if (d > hi) hi = d;
            }
            t->glo[3 * g + a] = (uint32_t)(ref + (uint32_t)lo);
            t->ghi[3 * g + a] = (uint32_t)(ref + (uint32_t)hi);
        }
    }
}

int ora_tree_build(const double *pos, const double *mass, int64_t n, const ora_params *p,
                   ora_tree **out)
{
    *out = NULL;
    if (n < 1 || !p || !(p->box > 0.0) || p->leaf_max < 1 || p->group_max < 1)
        return ORA_ERR_ARG;
    if (p->r_s > 0.0 && !(p->rcut_over_rs * p->r_s < 0.5 * p->box)) return ORA_ERR_ARG;
    ora_tree *t = (ora_tree *)calloc(1, sizeof(ora_tree));
    if (!t) return ORA_ERR_OOM;
    t->n = n;
    t->p = *p;
    t->x = xcalloc(n, 4); t->y = xcalloc(n, 4); t->z = xcalloc(n, 4);
    t->key = xcalloc(n, 8); t->perm = xcalloc(n, 8); t->skey = xcalloc(n, 8);
    t->sx = xcalloc(n, 4); t->sy = xcalloc(n, 4); t->sz = xcalloc(n, 4);
    t->sm = xcalloc(n, 8);
    int64_t mcap = n + 1, ccap = 2 * n + 2;
    t->level = xcalloc(mcap, 4);
    t->beg = xcalloc(mcap, 8); t->end = xcalloc(mcap, 8); t->parent = xcalloc(mcap, 8);
    t->cbeg = xcalloc(mcap, 8); t->ccnt = xcalloc(mcap, 8);
    t->child = xcalloc(ccap, 8);
    t->M = xcalloc(mcap, 8); t->Sx = xcalloc(mcap, 8); t->Sy = xcalloc(mcap, 8);
    t->Sz = xcalloc(mcap, 8);
    t->cx = xcalloc(mcap, 4); t->cy = xcalloc(mcap, 4); t->cz = xcalloc(mcap, 4);
    t->nextnode = xcalloc(mcap, 8); t->sibling = xcalloc(mcap, 8); t->pnext = xcalloc(n, 8);
    t->ox = xcalloc(mcap, 4); t->oy = xcalloc(mcap, 4); t->oz = xcalloc(mcap, 4);
    t->es = xcalloc(3 * mcap, 4); t->el = xcalloc(3 * mcap, 4);
    t->gbeg = xcalloc(n, 8); t->gend = xcalloc(n, 8);
    t->glo = xcalloc(3 * n, 4); t->ghi = xcalloc(3 * n, 4);
    if (!t->x || !t->y || !t->z || !t->key || !t->perm || !t->skey || !t->sx || !t->sy ||
        !t->sz || !t->sm || !t->level || !t->beg || !t->end || !t->parent || !t->cbeg ||
        !t->ccnt || !t->child || !t->M || !t->Sx || !t->Sy || !t->Sz || !t->cx || !t->cy ||
        !t->cz || !t->nextnode || !t->sibling || !t->pnext || !t->gbeg || !t->gend ||
        !t->glo || !t->ghi || !t->ox || !t->oy || !t->oz || !t->es || !t->el) {
        ora_tree_free(t);
        return ORA_ERR_OOM;
    }
    /* a1, a2 */
    for (int64_t i = 0; i < n; ++i) {
        if (ora_quantize1(pos[3 * i + 0], p->box, &t->x[i]) ||
            ora_quantize1(pos[3 * i + 1], p->box, &t->y[i]) ||
            ora_quantize1(pos[3 * i + 2], p->box, &t->z[i]) || !isfinite(mass[i]) ||
            mass[i] < 0.0) {
            ora_tree_free(t);
            return ORA_ERR_ARG;
        }
        t->key[i] = ora_morton(t->x[i], t->y[i], t->z[i]);
    }
    /* a3 */
    for (int64_t i = 0; i < n; ++i) t->perm[i] = i;
    g_sort_keys = t->key;
    qsort(t->perm, (size_t)n, sizeof(int64_t), cmp_key_index);
    for (int64_t i = 0; i < n; ++i) {
        int64_t j = t->perm[i];
        t->skey[i] = t->key[j];
        t->sx[i] = t->x[j];
        t->sy[i] = t->y[j];
        t->sz[i] = t->z[j];
        t->sm[i] = mass[j];
    }
    /* a4: the root is level 0 and covers the whole box */
    build_node(t, 0, 0, n, -1);
    /* a5 */
    int rc = mass_format(t);
    if (rc == ORA_OK) rc = all_moments(t);
    if (rc != ORA_OK) {
        ora_tree_free(t);
        return rc;
    }
    /* a4' */
    t->sibling[0] = -1;
    thread_node(t, 0, -1);
    /* a6 */
    make_groups(t, 0);
    group_boxes(t);
    *out = t;
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* geometry on the circle of 2^32 grid units                                 */
/* ------------------------------------------------------------------------ */

/* Intervals on the circle of 2^32 grid units are [lo, hi] with length
 * hi - lo (mod 2^32); an interval may wrap through 0 (a drifted box). */

/* distance from point c to the interval [lo, hi] (0 inside) */
static uint64_t circ_point_gap(uint32_t c, uint32_t lo, uint32_t hi)
{
    uint32_t len = hi - lo, d = c - lo;
    if (d <= len) return 0;
    uint32_t fwd = d - len, back = (uint32_t)(0u - d);
    return fwd < back ? fwd : back;
}

/* distance between the intervals [alo, ahi] and [blo, bhi] (0 if they meet) */
static uint64_t circ_box_gap(uint32_t alo, uint32_t ahi, uint32_t blo, uint32_t bhi)
{
    uint32_t la = ahi - alo, lb = bhi - blo;
    if ((uint32_t)(blo - alo) <= la || (uint32_t)(alo - blo) <= lb) return 0;
    uint32_t a = blo - ahi, b = alo - bhi;
    return a < b ? a : b;
}

/* minimum-image integer separation x_j - x_i, in [-2^31, 2^31) */
static int64_t min_image(uint32_t xj, uint32_t xi)
{
    int64_t d = (int64_t)xj - (int64_t)xi;
    if (d >= ((int64_t)1 << 31)) d -= ((int64_t)1 << 32);
    else if (d < -((int64_t)1 << 31)) d += ((int64_t)1 << 32);
    return d;
}

/* ------------------------------------------------------------------------ */
/* refit: drifted positions, the same topology                              */
/* ------------------------------------------------------------------------ */

/* Refit for drifted positions of the same particles (input order): the
 * topology, the groups and the octant slots of the build stay; sums and
 * centres of mass are recomputed (exactly, as in the build); every node gets
 * an extent, its cell joined with the members' positions (offsets from the
 * cell origin as 32-bit differences, so drift across the periodic boundary
 * stays local); group boxes are recomputed. */
int ora_tree_refit(ora_tree *t, const double *pos)
{
    const int64_t n = t->n;
    for (int64_t i = 0; i < n; ++i) {
        if (ora_quantize1(pos[3 * i + 0], t->p.box, &t->x[i]) ||
            ora_quantize1(pos[3 * i + 1], t->p.box, &t->y[i]) ||
            ora_quantize1(pos[3 * i + 2], t->p.box, &t->z[i]))
            return ORA_ERR_ARG;
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t j = t->perm[i];
        t->sx[i] = t->x[j];
        t->sy[i] = t->y[j];
        t->sz[i] = t->z[j];
    }
    int rc = all_moments(t);
    if (rc != ORA_OK) return rc;
    /* extents bottom-up: in preorder every child has a larger id than its parent */
    for (int64_t id = t->nnodes - 1; id >= 0; --id) {
        const uint32_t o[3] = {t->ox[id], t->oy[id], t->oz[id]};
        const int lev = t->level[id];
        const int64_t side = (int64_t)1 << (32 - lev);
        int64_t lo[3] = {0, 0, 0}, hi[3] = {side - 1, side - 1, side - 1};
        for (int64_t k = 0; k < t->ccnt[id]; ++k) {
            int64_t c = t->child[t->cbeg[id] + k];
            for (int a = 0; a < 3; ++a) {
                int64_t clo, chi;
                if (c < n) {
                    const uint32_t *xs = a == 0 ? t->sx : a == 1 ? t->sy : t->sz;
                    clo = chi = (int64_t)(int32_t)(uint32_t)(xs[c] - o[a]);
                } else {
                    int64_t j = c - n;
                    clo = (int64_t)(int32_t)(uint32_t)(t->es[3 * j + a] - o[a]);
                    chi = clo + (int64_t)t->el[3 * j + a];
                }
                if (clo < lo[a]) lo[a] = clo;
                if (chi > hi[a]) hi[a] = chi;
            }
        }
        for (int a = 0; a < 3; ++a) {
            if (hi[a] - lo[a] >= (int64_t)0xffffffff) {
                t->es[3 * id + a] = 0; /* the whole circle */
                t->el[3 * id + a] = 0xffffffffu;
            } else {
                t->es[3 * id + a] = (uint32_t)(o[a] + (uint32_t)lo[a]);
                t->el[3 * id + a] = (uint32_t)(hi[a] - lo[a]);
            }
        }
    }
    group_boxes(t);
    t->refit = 1;
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* force law                                                                 */
/* ------------------------------------------------------------------------ */

/* spline-softened radial factor g(r) with a = -G m g(r) (x_i - x_j) */
double ora_soft_g(double r, double h)
{
    if (!(h > 0.0) || r >= h) return 1.0 / (r * r * r);
    double u = r / h;
    double h3 = 1.0 / (h * h * h);
    if (u < 0.5) return h3 * (32.0 / 3.0 - 192.0 / 5.0 * u * u + 32.0 * u * u * u);
    return h3 * (64.0 / 3.0 - 48.0 * u + 192.0 / 5.0 * u * u - 32.0 / 3.0 * u * u * u -
                 1.0 / (15.0 * u * u * u));
}

/* potential kernel of the same spline mass distribution: psi(r) = integral
 * from r to infinity of g(s) s ds, so that -d psi / dr = r g(r); psi = 1/r for
 * r >= h and psi(0) = 14 / (5 h) = 1 / eps (h = 2.8 eps).  With u = r/h:
 *   u < 1/2      : psi = h^-1 (14/5 - 16/3 u^2 + 48/5 u^4 - 32/5 u^5)
 *   1/2 <= u < 1 : psi = h^-1 (16/5 - 1/(15 u) - 32/3 u^2 + 16 u^3
 *                              - 48/5 u^4 + 32/15 u^5)                      */
double ora_soft_psi(double r, double h)
{
    if (!(h > 0.0) || r >= h) return 1.0 / r;
    double u = r / h;
    double u2 = u * u;
    if (u < 0.5)
        return (14.0 / 5.0 - 16.0 / 3.0 * u2 + 48.0 / 5.0 * u2 * u2 - 32.0 / 5.0 * u2 * u2 * u) / h;
    return (16.0 / 5.0 - 1.0 / (15.0 * u) - 32.0 / 3.0 * u2 + 16.0 * u2 * u - 48.0 / 5.0 * u2 * u2 +
            32.0 / 15.0 * u2 * u2 * u) / h;
}

/* short-range potential factor erfc(r / 2 r_s) (Sect. 4.2); 1 without split */
double ora_split_p(double r, double rs)
{
    if (!(rs > 0.0)) return 1.0;
    return erfc(r / (2.0 * rs));
}

/* short-range factor S(r) = -r^2 d/dr[erfc(r/2r_s)/r] */
double ora_split_s(double r, double rs)
{
    if (!(rs > 0.0)) return 1.0;
    double u = r / (2.0 * rs);
    return erfc(u) + (r / (sqrt(ORA_PI) * rs)) * exp(-u * u);
}

typedef struct {
    double box, G, scale; /* scale = box / 2^32 */
    double h, rs;
    float rc2f;           /* cutoff in squared grid units, single precision */
    int cut;              /* cutoff active */
    uint64_t rprune;
    double th2;
    double acoef;         /* s^2 for the relative criterion */
} force_ctx;

static void make_ctx(const ora_params *p, force_ctx *c)
{
    c->box = p->box;
    c->G = p->G;
    c->scale = p->box / TWO32;
    c->h = 2.8 * p->eps;
    c->rs = p->r_s;
    c->cut = p->r_s > 0.0;
    if (c->cut) {
        double rcg = (p->rcut_over_rs * p->r_s) / p->box * TWO32;
        c->rc2f = (float)(rcg * rcg);
        c->rprune = (uint64_t)(rcg * rcg * (1.0 + 1.0 / 1024.0));
    } else {
        c->rc2f = INFINITY;
        c->rprune = UINT64_MAX;
    }
    c->th2 = p->theta * p->theta;
    c->acoef = c->scale * c->scale;
}

/* single-precision in/out decision (see the reading on the cutoff) */
static int pair_active(int64_t dx, int64_t dy, int64_t dz, float rc2f)
{
    float fx = (float)dx, fy = (float)dy, fz = (float)dz;
    float r2 = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
    return r2 > 0.0f && r2 < rc2f;
}

/* FP64 contribution of a mass m at (xj, yj, zj) to the target at (xi, yi, zi):
 * acceleration, and (phi != NULL) the short-range potential
 * -G m psi(r) erfc(r / 2 r_s) (the reading of the potential output) */
static void add_pair(const force_ctx *c, uint32_t xi, uint32_t yi, uint32_t zi, uint32_t xj,
                     uint32_t yj, uint32_t zj, double m, double acc[3], double *phi)
{
    int64_t ix = min_image(xj, xi), iy = min_image(yj, yi), iz = min_image(zj, zi);
    if (!pair_active(ix, iy, iz, c->rc2f)) return;
    double dx = (double)ix * c->scale, dy = (double)iy * c->scale, dz = (double)iz * c->scale;
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    double f = c->G * m * ora_soft_g(r, c->h) * ora_split_s(r, c->rs);
    acc[0] += f * dx;
    acc[1] += f * dy;
    acc[2] += f * dz;
    if (phi) *phi -= c->G * m * ora_soft_psi(r, c->h) * ora_split_p(r, c->rs);
}

/* ------------------------------------------------------------------------ */
/* a7: the walk of one group                                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t *v;
    int64_t len, cap;
} vec64;

static int vpush(vec64 *a, int64_t x)
{
    if (a->len == a->cap) {
        int64_t nc = a->cap ? 2 * a->cap : 256;
        int64_t *nv = (int64_t *)realloc(a->v, (size_t)nc * sizeof(int64_t));
        if (!nv) return ORA_ERR_OOM;
        a->v = nv;
        a->cap = nc;
    }
    a->v[a->len++] = x;
    return ORA_OK;
}

typedef struct {
    const ora_tree *t;
    const force_ctx *c;
    uint32_t lo[3], hi[3];
    int opening;
    double arel; /* alpha * a_min * s^2 */
    vec64 pn, pp;
    int err;
} walk_state;

/* The node's extent on every axis: the cell [o, o + side - 1] of a built
 * tree, or, after a refit, the cell joined with its drifted members.  ell is
 * the largest side of the extent. */
static void node_extent(const ora_tree *t, int64_t j, uint32_t s[3], uint32_t len[3], uint64_t *ell)
{
    if (t->refit) {
        uint64_t m = 0;
        for (int a = 0; a < 3; ++a) {
            s[a] = t->es[3 * j + a];
            len[a] = t->el[3 * j + a];
            if ((uint64_t)len[a] + 1 > m) m = (uint64_t)len[a] + 1;
        }
        *ell = m;
        return;
    }
    uint64_t side = (uint64_t)1 << (32 - t->level[j]);
    s[0] = t->ox[j];
    s[1] = t->oy[j];
    s[2] = t->oz[j];
    for (int a = 0; a < 3; ++a) len[a] = (uint32_t)(side - 1);
    *ell = side;
}

static int must_open(walk_state *w, int64_t j)
{
    const ora_tree *t = w->t;
    uint32_t s[3], len[3];
    uint64_t ell;
    node_extent(t, j, s, len, &ell);
    uint32_t com[3] = {t->cx[j], t->cy[j], t->cz[j]};
    /* boundary check: the group box meets the cube of side 1.2 ell centred
       on the extent (the cell enlarged by 10 % on every side) */
    int near = 1;
    for (int a = 0; a < 3; ++a) {
        uint32_t centre = (uint32_t)(s[a] + (uint32_t)(((uint64_t)len[a] + 1) / 2));
        uint64_t dc = circ_point_gap(centre, w->lo[a], w->hi[a]);
        if (10 * dc > 6 * ell) near = 0;
    }
    if (near) return 1;
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = (double)circ_point_gap(com[a], w->lo[a], w->hi[a]);
    double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    double l2 = (double)ell * (double)ell;
    if (w->opening == ORA_OPEN_BH) return l2 > w->c->th2 * d2;
    double lhs = (w->c->G * t->M[j]) * l2;
    double rhs = w->arel * (d2 * d2);
    return lhs > rhs;
}

static void walk_node(walk_state *w, int64_t id)
{
    const ora_tree *t = w->t;
    const int64_t n = t->n;
    for (int64_t k = 0; k < t->ccnt[id] && !w->err; ++k) {
        int64_t c = t->child[t->cbeg[id] + k];
        if (c < n) {
            uint32_t v[3] = {t->sx[c], t->sy[c], t->sz[c]};
            uint64_t g2 = 0;
            for (int a = 0; a < 3; ++a) {
                uint64_t g = circ_point_gap(v[a], w->lo[a], w->hi[a]);
                g2 += g * g;
            }
            if (w->c->cut && g2 > w->c->rprune) continue;
            if (vpush(&w->pp, c)) w->err = 1;
        } else {
            int64_t j = c - n;
            if (w->c->cut) {
                uint32_t s[3], len[3];
                uint64_t ell;
                node_extent(t, j, s, len, &ell);
                uint64_t g2 = 0;
                for (int a = 0; a < 3; ++a) {
                    uint64_t g = circ_box_gap(w->lo[a], w->hi[a], s[a], (uint32_t)(s[a] + len[a]));
                    g2 += g * g;
                }
                if (g2 > w->c->rprune) continue;
            }
            if (must_open(w, j)) walk_node(w, j);
            else if (vpush(&w->pn, j)) w->err = 1;
        }
    }
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* one force pass over the selected groups; acc, npp, npn in input order */
static int force_pass(ora_tree *t, const force_ctx *c, int opening, const float *a_old,
                      const int64_t *sel, int64_t nsel, double *acc, uint32_t *npp,
                      uint32_t *npn, int keep_lists, int64_t **glist, int64_t *glen,
                      double *pot)
{
    const int64_t n = t->n;
    int err = 0;
#pragma omp parallel
    {
        walk_state w;
        memset(&w, 0, sizeof(w));
        w.t = t;
        w.c = c;
        w.opening = opening;
#pragma omp for schedule(dynamic, 4)
        for (int64_t s = 0; s < nsel; ++s) {
            int64_t g = sel ? sel[s] : s;
            for (int a = 0; a < 3; ++a) {
                w.lo[a] = t->glo[3 * g + a];
                w.hi[a] = t->ghi[3 * g + a];
            }
            w.arel = 0.0;
            if (opening == ORA_OPEN_REL) {
                double amin = INFINITY;
                for (int64_t q = t->gbeg[g]; q < t->gend[g]; ++q) {
                    const float *ao = a_old + 3 * t->perm[q];
                    double ax = ao[0], ay = ao[1], az = ao[2];
                    double an = sqrt((ax * ax + ay * ay) + az * az);
                    if (an < amin) amin = an;
                }
                w.arel = (t->p.alpha * amin) * c->acoef;
            }
            w.pn.len = w.pp.len = 0;
            w.err = 0;
            walk_node(&w, 0);
            if (w.err) {
#pragma omp atomic write
                err = 1;
                continue;
            }
            for (int64_t q = t->gbeg[g]; q < t->gend[g]; ++q) {
                double a3[3] = {0.0, 0.0, 0.0}, ph = 0.0;
                double *php = pot ? &ph : NULL;
                uint32_t xi = t->sx[q], yi = t->sy[q], zi = t->sz[q];
                for (int64_t k = 0; k < w.pp.len; ++k) {
                    int64_t j = w.pp.v[k];
                    add_pair(c, xi, yi, zi, t->sx[j], t->sy[j], t->sz[j], t->sm[j], a3, php);
                }
                for (int64_t k = 0; k < w.pn.len; ++k) {
                    int64_t j = w.pn.v[k];
                    add_pair(c, xi, yi, zi, t->cx[j], t->cy[j], t->cz[j], t->M[j], a3, php);
                }
                int64_t o = t->perm[q];
                if (pot) pot[o] = ph;
                acc[3 * o + 0] = a3[0];
                acc[3 * o + 1] = a3[1];
                acc[3 * o + 2] = a3[2];
                if (npp) npp[o] = (uint32_t)(w.pp.len - 1);
                if (npn) npn[o] = (uint32_t)w.pn.len;
            }
            if (keep_lists) {
                int64_t L = w.pn.len + w.pp.len;
                int64_t *buf = (int64_t *)malloc((size_t)(L ? L : 1) * sizeof(int64_t));
                if (!buf) {
#pragma omp atomic write
                    err = 1;
                    continue;
                }
                for (int64_t k = 0; k < w.pn.len; ++k) buf[k] = w.pn.v[k] + n;
                for (int64_t k = 0; k < w.pp.len; ++k) buf[w.pn.len + k] = w.pp.v[k];
                qsort(buf, (size_t)L, sizeof(int64_t), cmp_i64);
                glist[s] = buf;
                glen[s] = L;
            }
        }
        free(w.pn.v);
        free(w.pp.v);
    }
    return err ? ORA_ERR_OOM : ORA_OK;
}

int ora_tree_force(ora_tree *t, const float *a_old, int opening, double theta, double alpha,
                   const int64_t *sel, int64_t nsel, double *acc, uint32_t *npp,
                   uint32_t *npn, int keep_lists, int nthreads)
{
    return ora_tree_force_pot(t, a_old, opening, theta, alpha, sel, nsel, acc, npp, npn, NULL,
                              keep_lists, nthreads);
}

int ora_tree_force_pot(ora_tree *t, const float *a_old, int opening, double theta, double alpha,
                       const int64_t *sel, int64_t nsel, double *acc, uint32_t *npp,
                       uint32_t *npn, double *pot, int keep_lists, int nthreads)
{
    if (!t || !acc) return ORA_ERR_ARG;
    if (opening != ORA_OPEN_BH && opening != ORA_OPEN_REL) return ORA_ERR_ARG;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    if (!sel) nsel = t->ngroups;
    for (int64_t s = 0; sel && s < nsel; ++s)
        if (sel[s] < 0 || sel[s] >= t->ngroups) return ORA_ERR_ARG;
    ora_params p = t->p;
    p.theta = theta;
    p.alpha = alpha;
    t->p.alpha = alpha;
    force_ctx c;
    float *aprev = NULL;
    int rc;
    if (opening == ORA_OPEN_REL && !a_old) {
        /* first pass: Barnes-Hut with theta_first_pass gives a_old */
        ora_params p1 = p;
        p1.theta = p.theta_first_pass;
        make_ctx(&p1, &c);
        double *a1 = (double *)malloc((size_t)(3 * t->n) * sizeof(double));
        aprev = (float *)malloc((size_t)(3 * t->n) * sizeof(float));
        if (!a1 || !aprev) {
            free(a1);
            free(aprev);
            return ORA_ERR_OOM;
        }
        rc = force_pass(t, &c, ORA_OPEN_BH, NULL, NULL, t->ngroups, a1, NULL, NULL, 0, NULL,
                        NULL, NULL);
        for (int64_t i = 0; i < 3 * t->n; ++i) aprev[i] = (float)a1[i];
        free(a1);
        if (rc) {
            free(aprev);
            return rc;
        }
        a_old = aprev;
    }
    make_ctx(&p, &c);
    int64_t **glist = NULL, *glen = NULL;
    if (keep_lists) {
        glist = (int64_t **)calloc((size_t)(nsel ? nsel : 1), sizeof(int64_t *));
        glen = (int64_t *)calloc((size_t)(nsel ? nsel : 1), sizeof(int64_t));
        if (!glist || !glen) {
            free(glist);
            free(glen);
            free(aprev);
            return ORA_ERR_OOM;
        }
    }
    rc = force_pass(t, &c, opening, a_old, sel, nsel, acc, npp, npn, keep_lists, glist, glen, pot);
    free(aprev);
    if (keep_lists) {
        free(t->list_off);
        free(t->list);
        t->list_off = (int64_t *)calloc((size_t)nsel + 1, sizeof(int64_t));
        int64_t total = 0;
        for (int64_t s = 0; s < nsel; ++s) total += glen[s];
        t->list = (int64_t *)malloc((size_t)(total ? total : 1) * sizeof(int64_t));
        if (!t->list_off || !t->list) rc = ORA_ERR_OOM;
        int64_t o = 0;
        for (int64_t s = 0; s < nsel; ++s) {
            if (!rc) {
                t->list_off[s] = o;
                memcpy(t->list + o, glist[s], (size_t)glen[s] * sizeof(int64_t));
                o += glen[s];
            }
            free(glist[s]);
        }
        if (!rc) t->list_off[nsel] = o;
        t->list_len = rc ? 0 : o;
        free(glist);
        free(glen);
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* exact references: direct summation and a cell list of side >= r_cut       */
/* ------------------------------------------------------------------------ */

static int quantize_all(const double *pos, int64_t n, double box, uint32_t *q)
{
    for (int64_t i = 0; i < 3 * n; ++i)
        if (ora_quantize1(pos[i], box, &q[i])) return ORA_ERR_ARG;
    return ORA_OK;
}

int ora_direct(const double *pos, const double *mass, int64_t n, const ora_params *p,
               const int64_t *targets, int64_t ntargets, double *acc, int nthreads)
{
    return ora_direct_pot(pos, mass, n, p, targets, ntargets, acc, NULL, nthreads);
}

int ora_direct_pot(const double *pos, const double *mass, int64_t n, const ora_params *p,
                   const int64_t *targets, int64_t ntargets, double *acc, double *pot,
                   int nthreads)
{
    if (n < 1 || !p || !(p->box > 0.0)) return ORA_ERR_ARG;
    if (p->r_s > 0.0 && !(p->rcut_over_rs * p->r_s < 0.5 * p->box)) return ORA_ERR_ARG;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    uint32_t *q = (uint32_t *)malloc((size_t)(3 * n) * sizeof(uint32_t));
    if (!q) return ORA_ERR_OOM;
    if (quantize_all(pos, n, p->box, q)) {
        free(q);
        return ORA_ERR_ARG;
    }
    force_ctx c;
    make_ctx(p, &c);
    int64_t nt = targets ? ntargets : n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < nt; ++s) {
        int64_t i = targets ? targets[s] : s;
        double a3[3] = {0.0, 0.0, 0.0}, ph = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            add_pair(&c, q[3 * i], q[3 * i + 1], q[3 * i + 2], q[3 * j], q[3 * j + 1],
                     q[3 * j + 2], mass[j], a3, pot ? &ph : NULL);
        }
        if (pot) pot[s] = ph;
        acc[3 * s + 0] = a3[0];
        acc[3 * s + 1] = a3[1];
        acc[3 * s + 2] = a3[2];
    }
    free(q);
    return ORA_OK;
}

int ora_cell_exact(const double *pos, const double *mass, int64_t n, const ora_params *p,
                   const int64_t *targets, int64_t ntargets, double *acc, int nthreads)
{
    if (n < 1 || !p || !(p->box > 0.0) || !(p->r_s > 0.0)) return ORA_ERR_ARG;
    double rcut = p->rcut_over_rs * p->r_s;
    if (!(rcut < 0.5 * p->box)) return ORA_ERR_ARG;
    int64_t nc = (int64_t)floor(p->box / rcut);
    if (nc < 3) return ora_direct(pos, mass, n, p, targets, ntargets, acc, nthreads);
    if (nc > 256) nc = 256;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    uint32_t *q = (uint32_t *)malloc((size_t)(3 * n) * sizeof(uint32_t));
    int64_t *cell = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *head = (int64_t *)malloc((size_t)(nc * nc * nc + 1) * sizeof(int64_t));
    int64_t *order = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!q || !cell || !head || !order) {
        free(q); free(cell); free(head); free(order);
        return ORA_ERR_OOM;
    }
    if (quantize_all(pos, n, p->box, q)) {
        free(q); free(cell); free(head); free(order);
        return ORA_ERR_ARG;
    }
    int64_t ncell = nc * nc * nc;
    for (int64_t k = 0; k <= ncell; ++k) head[k] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t cx = (int64_t)(((double)q[3 * i] / TWO32) * nc);
        int64_t cy = (int64_t)(((double)q[3 * i + 1] / TWO32) * nc);
        int64_t cz = (int64_t)(((double)q[3 * i + 2] / TWO32) * nc);
        if (cx >= nc) cx = nc - 1;
        if (cy >= nc) cy = nc - 1;
        if (cz >= nc) cz = nc - 1;
        cell[i] = (cx * nc + cy) * nc + cz;
        head[cell[i] + 1]++;
    }
    for (int64_t k = 0; k < ncell; ++k) head[k + 1] += head[k];
    {
        int64_t *fill = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
        if (!fill) {
            free(q); free(cell); free(head); free(order);
            return ORA_ERR_OOM;
        }
        memcpy(fill, head, (size_t)ncell * sizeof(int64_t));
        for (int64_t i = 0; i < n; ++i) order[fill[cell[i]]++] = i;
        free(fill);
    }
    force_ctx c;
    make_ctx(p, &c);
    int64_t nt = targets ? ntargets : n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t s = 0; s < nt; ++s) {
        int64_t i = targets ? targets[s] : s;
        int64_t ci = cell[i];
        int64_t cx = ci / (nc * nc), cy = (ci / nc) % nc, cz = ci % nc;
        double a3[3] = {0.0, 0.0, 0.0};
        for (int ox = -1; ox <= 1; ++ox)
            for (int oy = -1; oy <= 1; ++oy)
                for (int oz = -1; oz <= 1; ++oz) {
                    int64_t nx = (cx + ox + nc) % nc, ny = (cy + oy + nc) % nc,
                            nz = (cz + oz + nc) % nc;
                    int64_t cc = (nx * nc + ny) * nc + nz;
                    for (int64_t k = head[cc]; k < head[cc + 1]; ++k) {
                        int64_t j = order[k];
                        if (j == i) continue;
                        add_pair(&c, q[3 * i], q[3 * i + 1], q[3 * i + 2], q[3 * j],
                                 q[3 * j + 1], q[3 * j + 2], mass[j], a3, NULL);
                    }
                }
        acc[3 * s + 0] = a3[0];
        acc[3 * s + 1] = a3[1];
        acc[3 * s + 2] = a3[2];
    }
    free(q); free(cell); free(head); free(order);
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* accessors                                                                 */
/* ------------------------------------------------------------------------ */

int64_t ora_tree_count(const ora_tree *t, int what)
{
    switch (what) {
    case ORA_N: return t->n;
    case ORA_NODES: return t->nnodes;
    case ORA_CHILDREN: return t->nchild;
    case ORA_GROUPS: return t->ngroups;
    case ORA_LIST_LEN: return t->list_len;
    default: return -1;
    }
}

int ora_tree_get(const ora_tree *t, int what, void *dst)
{
    int64_t n = t->n, m = t->nnodes, g = t->ngroups;
    switch (what) {
    case ORA_F_X: memcpy(dst, t->x, (size_t)n * 4); break;
    case ORA_F_Y: memcpy(dst, t->y, (size_t)n * 4); break;
    case ORA_F_Z: memcpy(dst, t->z, (size_t)n * 4); break;
    case ORA_F_KEY: memcpy(dst, t->key, (size_t)n * 8); break;
    case ORA_F_PERM: memcpy(dst, t->perm, (size_t)n * 8); break;
    case ORA_F_LEVEL: memcpy(dst, t->level, (size_t)m * 4); break;
    case ORA_F_BEG: memcpy(dst, t->beg, (size_t)m * 8); break;
    case ORA_F_END: memcpy(dst, t->end, (size_t)m * 8); break;
    case ORA_F_PARENT: memcpy(dst, t->parent, (size_t)m * 8); break;
    case ORA_F_CBEG: memcpy(dst, t->cbeg, (size_t)m * 8); break;
    case ORA_F_CCNT: memcpy(dst, t->ccnt, (size_t)m * 8); break;
    case ORA_F_CHILD: memcpy(dst, t->child, (size_t)t->nchild * 8); break;
    case ORA_F_MASS: memcpy(dst, t->M, (size_t)m * 8); break;
    case ORA_F_COM: {
        uint32_t *o = (uint32_t *)dst;
        for (int64_t i = 0; i < m; ++i) {
            o[3 * i] = t->cx[i];
            o[3 * i + 1] = t->cy[i];
            o[3 * i + 2] = t->cz[i];
        }
        break;
    }
    case ORA_F_MSUM: {
        double *o = (double *)dst;
        for (int64_t i = 0; i < m; ++i) {
            o[3 * i] = t->Sx[i];
            o[3 * i + 1] = t->Sy[i];
            o[3 * i + 2] = t->Sz[i];
        }
        break;
    }
    case ORA_F_NEXTNODE: memcpy(dst, t->nextnode, (size_t)m * 8); break;
    case ORA_F_SIBLING: memcpy(dst, t->sibling, (size_t)m * 8); break;
    case ORA_F_PNEXT: memcpy(dst, t->pnext, (size_t)n * 8); break;
    case ORA_F_GBEG: memcpy(dst, t->gbeg, (size_t)g * 8); break;
    case ORA_F_GEND: memcpy(dst, t->gend, (size_t)g * 8); break;
    case ORA_F_GLO: memcpy(dst, t->glo, (size_t)(3 * g) * 4); break;
    case ORA_F_GHI: memcpy(dst, t->ghi, (size_t)(3 * g) * 4); break;
    case ORA_F_EXT_S: memcpy(dst, t->es, (size_t)(3 * m) * 4); break;
    case ORA_F_EXT_L: memcpy(dst, t->el, (size_t)(3 * m) * 4); break;
    default: return ORA_ERR_ARG;
    }
    return ORA_OK;
}

int ora_tree_get_lists(const ora_tree *t, int64_t nsel, int64_t *off, int64_t *list)
{
    if (!t->list_off) return ORA_ERR_ARG;
    memcpy(off, t->list_off, (size_t)(nsel + 1) * sizeof(int64_t));
    memcpy(list, t->list, (size_t)t->list_len * sizeof(int64_t));
    return ORA_OK;
}

int ora_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

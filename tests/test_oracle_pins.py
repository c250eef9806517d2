"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value comes from
a closed form, an exact rational computation, a brute-force restatement of a
definition (tests/brute.py), a library routine, or an invariant.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate, special

import og_inputs as gi
import oracle
from tests import brute

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------------------
# a1 fixed point, a2 Morton keys, a3 sort
# ---------------------------------------------------------------------------

def test_quantize_special_values():
    assert oracle.quantize1(0.0) == 0
    assert oracle.quantize1(0.5) == 1 << 31
    assert oracle.quantize1(1.0) == 0                      # periodic wrap
    assert oracle.quantize1(-1e-20) == (1 << 32) - 1       # exact: just below the torus point 0
    assert oracle.quantize1(1.0 - 2.0 ** -53) == (1 << 32) - 1
    assert oracle.quantize1(0.25, box=0.5) == 1 << 31
    assert oracle.quantize1(2.75) == 3 << 30
    assert oracle.quantize1(-0.25) == 3 << 30
    with pytest.raises(ValueError):
        oracle.quantize1(float("nan"))


def test_quantize_matches_exact_rationals():
    r = np.random.default_rng(1)
    vals = np.concatenate([r.random(300) * 3.0, r.random(50) * 1e-6, [1e-300, 0.999999999],
                           -r.random(100) * 3.0, -r.random(50) * 1e-12, [-1e-300, -2.0 ** -60],
                           r.random(20) * 1e12, -r.random(20) * 1e12, [2.0 ** 31 + 0.25, -2.0 ** 31 - 0.25]])
    for v in vals:
        assert oracle.quantize1(float(v)) == brute.quantize_exact(float(v))
    for box in (0.37, 3.0, 1e3):
        for v in r.random(50) * box * 2:
            assert oracle.quantize1(float(v), box) == brute.quantize_exact(float(v), box)


def test_morton_matches_string_interleave():
    r = np.random.default_rng(2)
    vals = list(r.integers(0, 1 << 32, size=(400, 3)))
    vals += [(0, 0, 0), ((1 << 32) - 1,) * 3, (1 << 31, 0, 0), (0, 1 << 31, 0), (0, 0, 1 << 31),
             (2047, 2047, 2047), (2048, 0, 0)]
    for x, y, z in vals:
        assert oracle.morton(int(x), int(y), int(z)) == brute.morton_string(int(x), int(y), int(z))
    # x is the most significant axis; the low 11 bits of each axis are dropped
    assert oracle.morton(1 << 31, 0, 0) == 1 << 62
    assert oracle.morton(0, 0, 1 << 11) == 1
    assert oracle.morton(2047, 2047, 2047) == 0


def test_sort_is_stable_key_order():
    pos, mass = gi.uniform(3000, 3)
    pos[100:140] = pos[7]                      # coincident keys exercise stability
    t = oracle.Tree(pos, mass, gi.default_params())
    key = t.get(oracle.F_KEY)
    perm = t.get(oracle.F_PERM)
    expect = np.argsort(key, kind="stable")
    assert np.array_equal(perm, expect)
    # keys recomputed from the quantized coordinates by string interleave
    x, y, z = t.get(oracle.F_X), t.get(oracle.F_Y), t.get(oracle.F_Z)
    for i in range(0, 3000, 37):
        assert int(key[i]) == brute.morton_string(int(x[i]), int(y[i]), int(z[i]))


# ---------------------------------------------------------------------------
# a4 topology, threading; a5 moments; a6 groups
# ---------------------------------------------------------------------------

def _sorted_keys(t):
    return t.get(oracle.F_KEY)[t.get(oracle.F_PERM)]


@pytest.mark.parametrize("case", ["uniform", "halo", "dups", "tiny1", "tiny2", "tiny9", "leaf3"])
def test_topology_matches_flat_definition(case):
    leaf = 1
    if case == "uniform":
        pos, mass = gi.uniform(2000, 4)
    elif case == "halo":
        pos, mass = gi.halo_mix(3000, 5, n_halo=5)
    elif case == "dups":
        pos, mass = gi.uniform(500, 6)
        pos[:200] = pos[0]
        pos[300:310] = pos[301] + 1e-12       # same key, slightly different positions
    elif case == "leaf3":
        pos, mass = gi.halo_mix(1500, 7, n_halo=3)
        leaf = 3
    else:
        n = int(case[4:])
        pos, mass = gi.uniform(n, 8)
    t = oracle.Tree(pos, mass, gi.default_params(leaf_max=leaf))
    skey = _sorted_keys(t)
    lev, beg, end = t.get(oracle.F_LEVEL), t.get(oracle.F_BEG), t.get(oracle.F_END)
    got = set(zip(lev.tolist(), beg.tolist(), end.tolist()))
    assert len(got) == t.nnodes
    assert got == brute.node_set(skey, leaf)
    # parents: the deepest other node containing the range
    par = t.get(oracle.F_PARENT)
    nodes = list(zip(lev.tolist(), beg.tolist(), end.tolist()))
    for i, nd in enumerate(nodes):
        if i == 0:
            assert par[0] == -1 and nd == (0, 0, t.n)
            continue
        cands = [m for m in nodes if m != nd and m[1] <= nd[1] and nd[2] <= m[2] and m[0] < nd[0]]
        assert nodes[par[i]] == max(cands, key=lambda m: m[0])
    # every particle hangs from the deepest node containing it; child lists in key order
    cbeg, ccnt, child = t.get(oracle.F_CBEG), t.get(oracle.F_CCNT), t.get(oracle.F_CHILD)
    owner = np.full(t.n, -1)
    for i in range(t.nnodes):
        items = child[cbeg[i]:cbeg[i] + ccnt[i]]
        starts = [c if c < t.n else beg[c - t.n] for c in items]
        assert starts == sorted(starts)
        assert starts[0] == beg[i]
        for c in items:
            if c < t.n:
                owner[c] = i
            else:
                assert par[c - t.n] == i
    for p in range(t.n):
        assert nodes[owner[p]] == brute.deepest_containing(nodes, p, p + 1)
    # leaf_max: a particle's octant group in its owner has at most leaf_max members
    for i in range(t.nnodes):
        if lev[i] == 21:
            continue
        items = [c for c in child[cbeg[i]:cbeg[i] + ccnt[i]] if c < t.n]
        digs = [(int(skey[c]) >> (3 * (21 - int(lev[i]) - 1))) & 7 for c in items]
        for d in set(digs):
            assert digs.count(d) <= leaf


def test_threading_visits_preorder():
    pos, mass = gi.halo_mix(1200, 9, n_halo=4)
    t = oracle.Tree(pos, mass, gi.default_params())
    n = t.n
    cbeg, ccnt, child = t.get(oracle.F_CBEG), t.get(oracle.F_CCNT), t.get(oracle.F_CHILD)
    nxt, sib, pnext = t.get(oracle.F_NEXTNODE), t.get(oracle.F_SIBLING), t.get(oracle.F_PNEXT)

    order = []

    def dfs(i):
        for c in child[cbeg[i]:cbeg[i] + ccnt[i]]:
            order.append(int(c))
            if c >= n:
                dfs(int(c - n))

    dfs(0)
    # opening everything: follow nextnode for nodes and pnext for particles
    seq, cur = [], int(nxt[0])
    while cur != -1:
        seq.append(cur)
        cur = int(pnext[cur]) if cur < n else int(nxt[cur - n])
    assert seq == order
    # accepting a node skips its subtree: sibling = the item after the subtree
    pos_of = {v: k for k, v in enumerate(order)}

    def subtree_size(i):
        return sum(1 + (subtree_size(int(c - n)) if c >= n else 0)
                   for c in child[cbeg[i]:cbeg[i] + ccnt[i]])

    for i in range(1, t.nnodes):
        k = pos_of[i + n] + 1 + subtree_size(i)
        assert int(sib[i]) == (order[k] if k < len(order) else -1)


def _rn(f: Fraction) -> float:
    """The nearest double to an exact rational, ties to even (Python's integer
    true division rounds correctly); infinity past the largest double."""
    try:
        return float(f)
    except OverflowError:
        return math.inf


def _check_exact_moments(pos, mass, prm):
    """Every node's mass and sums of m x are the exact sums over its particles
    rounded once to the nearest double, and its centre of mass is the grid
    point nearest to the exact ratio (ties to even), or the cell centre of a
    massless node."""
    t = oracle.Tree(pos, mass, prm)
    perm = t.get(oracle.F_PERM)
    xs = [t.get(f)[perm] for f in (oracle.F_X, oracle.F_Y, oracle.F_Z)]
    sm = mass[perm]
    M, S, com = t.get(oracle.F_MASS), t.get(oracle.F_MSUM), t.get(oracle.F_COM)
    beg, end, lev = t.get(oracle.F_BEG), t.get(oracle.F_END), t.get(oracle.F_LEVEL)
    pm = [Fraction(0)]
    ps = [[Fraction(0)] for _ in range(3)]
    for q, v in enumerate(sm):
        f = Fraction(float(v))
        pm.append(pm[-1] + f)
        for a in range(3):
            ps[a].append(ps[a][-1] + f * int(xs[a][q]))
    massless = 0
    for i in range(t.nnodes):
        b, e = int(beg[i]), int(end[i])
        em = pm[e] - pm[b]
        assert M[i] == _rn(em) and not np.signbit(M[i]), i
        for a in range(3):
            es = ps[a][e] - ps[a][b]
            assert S[i, a] == _rn(es) and not np.signbit(S[i, a]), (i, a)
            if em > 0:
                assert int(com[i, a]) == round(es / em), (i, a)
            else:
                sh = 32 - int(lev[i])
                cell = 0 if lev[i] == 0 else (int(xs[a][b]) >> sh) << sh
                assert int(com[i, a]) == cell + (1 << (sh - 1))
        massless += em == 0
    return t, massless


def test_moments_exact_equal_and_unequal_masses():
    pos, mass = gi.halo_mix(1500, 10, n_halo=4)
    _check_exact_moments(pos, mass, gi.default_params())
    mass = mass * (1.0 + 0.5 * np.random.default_rng(0).random(mass.shape))
    _check_exact_moments(pos, mass, gi.default_params())


def test_moments_exact_wide_mass_range_and_massless_nodes():
    r = np.random.default_rng(1)
    pos, mass = gi.halo_mix(1200, 11, n_halo=3)
    mass = np.ldexp(1.0 + r.random(len(mass)), r.integers(-90, 90, len(mass)))
    mass[r.random(len(mass)) < 0.3] = 0.0                   # scattered massless particles
    mass[np.argsort(pos[:, 0])[:200]] = 0.0                  # a massless slab: whole massless nodes
    _, massless = _check_exact_moments(pos, mass, gi.default_params())
    assert massless > 0


def test_moments_exact_subnormal_and_overflowing_sums():
    r = np.random.default_rng(2)
    pos, _ = gi.halo_mix(600, 12, n_halo=2)
    tiny = 5e-324 * r.integers(1, 1 << 20, len(pos)).astype(np.float64)   # subnormal masses
    tiny[::7] = 2.0 ** -1022 * (1.0 + r.random(len(tiny[::7])))           # and the smallest normals
    _check_exact_moments(pos, tiny, gi.default_params())
    huge = 1e300 * (1.0 + r.random(len(pos)))               # m x overflows, M does not
    t, _ = _check_exact_moments(pos, huge, gi.default_params())
    assert np.isinf(t.get(oracle.F_MSUM)).any() and np.isfinite(t.get(oracle.F_MASS)).all()


def test_moments_exact_coincident_keys():
    r = np.random.default_rng(3)
    pos, mass = gi.halo_mix(400, 13, n_halo=2)
    pos = np.concatenate([pos, np.repeat(pos[:20], 5, axis=0)])           # buckets of equal keys
    mass = np.concatenate([mass, r.random(100) * mass[0]])
    t, _ = _check_exact_moments(pos, mass, gi.default_params())
    assert (t.get(oracle.F_LEVEL) == 21).any()


def test_centre_of_mass_ties_round_to_even():
    # two equal masses one grid unit apart: the exact centre is a half-integer
    g = 2.0 ** -32
    for x0 in (1000, 1001):
        pos = np.array([[x0 * g, 0.25, 0.25], [(x0 + 1) * g, 0.25, 0.25]])
        t = oracle.Tree(pos, np.array([0.5, 0.5]), gi.default_params())
        com = t.get(oracle.F_COM)[0]
        assert int(com[0]) == (x0 if x0 % 2 == 0 else x0 + 1)
        assert int(com[1]) == 1 << 30
    # unequal masses: the nearest grid point, not the truncation
    pos = np.array([[0.0, 0.0, 0.0], [3 * g, 0.0, 0.0]])
    t = oracle.Tree(pos, np.array([2.0, 1.0]), gi.default_params())
    assert int(t.get(oracle.F_COM)[0][0]) == 1                     # exact centre 1
    t = oracle.Tree(pos, np.array([1.0, 2.0]), gi.default_params())
    assert int(t.get(oracle.F_COM)[0][0]) == 2                     # exact centre 2


@pytest.mark.parametrize("G", [1, 8, 32])
def test_groups_match_flat_definition(G):
    pos, mass = gi.halo_mix(2500, 11, n_halo=6)
    t = oracle.Tree(pos, mass, gi.default_params(group_max=G))
    skey = _sorted_keys(t)
    nodes = brute.node_set(skey)
    expect = brute.groups_flat(nodes, t.n, G)
    gb, ge = t.get(oracle.F_GBEG), t.get(oracle.F_GEND)
    assert list(zip(gb.tolist(), ge.tolist())) == expect
    perm = t.get(oracle.F_PERM)
    xs = np.stack([t.get(f)[perm] for f in (oracle.F_X, oracle.F_Y, oracle.F_Z)], axis=1)
    lo, hi = t.get(oracle.F_GLO), t.get(oracle.F_GHI)
    for g, (b, e) in enumerate(expect):
        assert np.array_equal(lo[g], xs[b:e].min(axis=0))
        assert np.array_equal(hi[g], xs[b:e].max(axis=0))


def test_single_group_when_small():
    pos, mass = gi.uniform(20, 12)
    t = oracle.Tree(pos, mass, gi.default_params(group_max=32))
    assert t.ngroups == 1
    assert (t.get(oracle.F_GBEG)[0], t.get(oracle.F_GEND)[0]) == (0, 20)


# ---------------------------------------------------------------------------
# force law: the spline-softened kernel and the erfc split factor
# ---------------------------------------------------------------------------

def _spline_density(r, h):
    """3D cubic-spline kernel of the paper's appendix (normalisation 8/(pi h^3))."""
    q = r / h
    w = np.where(q < 0.5, 1 + 6 * (q - 1) * q * q, np.where(q < 1, 2 * (1 - q) ** 3, 0.0))
    return 8.0 / (math.pi * h ** 3) * w


def _enclosed(r, h):
    f = lambda s: 4 * math.pi * s * s * _spline_density(s, h)
    if r <= h / 2:
        return integrate.quad(f, 0, r, epsabs=1e-14, epsrel=1e-13)[0]
    m = integrate.quad(f, 0, h / 2, epsabs=1e-14, epsrel=1e-13)[0]
    return m + integrate.quad(f, h / 2, min(r, h), epsabs=1e-14, epsrel=1e-13)[0]


def test_spline_kernel_is_the_cubic_spline_mass_profile():
    h = 1.0
    assert abs(_enclosed(1.0, h) - 1.0) < 1e-12           # unit mass within h
    for r in [0.01, 0.1, 0.3, 0.4999, 0.5, 0.5001, 0.7, 0.9, 0.999, 1.0, 1.3, 2.0]:
        g = oracle.soft_g(r, h)
        expect = _enclosed(r, h) / r ** 3                  # shell theorem: M(<r)/r^3
        assert abs(g - expect) <= 1e-10 * abs(expect), r


def test_spline_force_and_derivative_continuous():
    h = 0.37
    F = lambda r: oracle.soft_g(r, h) * r                  # radial force per unit mass
    for r0 in (h / 2, h):
        d = 1e-7 * h
        assert abs(F(r0 - d) - F(r0 + d)) < 1e-5 * F(r0)
        left = (F(r0 - d) - F(r0 - 2 * d)) / d
        right = (F(r0 + 2 * d) - F(r0 + d)) / d
        assert abs(left - right) < 1e-4 * abs(F(r0) / h)


def test_split_factor_from_the_erfc_potential():
    rs = 0.02
    phi = lambda r: special.erfc(r / (2 * rs)) / r          # -phi_s / (G m), Sect. 4.2
    for r in [1e-4, 0.005, 0.02, 0.04, 0.0899]:
        d = 1e-6 * r
        dphi = (phi(r + d) - phi(r - d)) / (2 * d)
        expect = -r * r * dphi
        assert abs(oracle.split_s(r, rs) - expect) < 1e-7
    assert abs(oracle.split_s(1e-12, rs) - 1.0) < 1e-9
    assert oracle.split_s(10.0, rs) < 1e-300 + 1e-100
    assert oracle.split_s(0.5, 0.0) == 1.0


@pytest.mark.parametrize("sep_over_h", [0.2, 0.5, 0.75, 1.0, 1.5, 4.0])
def test_two_body_closed_form(sep_over_h):
    eps = 1e-3
    h = 2.8 * eps                                          # Plummer-equivalent eps (Sect. 4.1.3)
    rs = 0.01
    prm = gi.default_params(eps=eps, r_s=rs, theta=0.5)
    sep = sep_over_h * h
    pos, mass = gi.two_body(sep, axis=1, m=(0.25, 0.75))
    t = oracle.Tree(pos, mass, prm)
    acc, npp, npn = t.force()
    qpos = np.array([[oracle.quantize1(v) for v in p] for p in pos], dtype=np.int64)
    r = abs(int(brute.min_image_int(qpos[1, 1] - qpos[0, 1]))) / 2.0 ** 32
    S = special.erfc(r / (2 * rs)) + r / (math.sqrt(math.pi) * rs) * math.exp(-(r / (2 * rs)) ** 2)
    mag = _enclosed(min(r, h), h) / r ** 2 if r < h else 1.0 / r ** 2
    for i, j in ((0, 1), (1, 0)):
        expect = mass[j] * mag * S
        assert abs(acc[i, 1] * np.sign(pos[j, 1] - pos[i, 1]) - expect) < 1e-9 * expect
        assert acc[i, 0] == 0.0 and acc[i, 2] == 0.0
    assert np.all(npp == 1) and np.all(npn == 0)


def test_two_body_periodic_minimum_image_and_cutoff():
    prm = gi.default_params(eps=1e-4, r_s=0.02, theta=0.5)
    rcut = 4.5 * 0.02
    # across the boundary: 0.01 and 0.97 are 0.04 apart through x = 0
    pos = np.array([[0.01, 0.5, 0.5], [0.97, 0.5, 0.5]])
    acc, _, _ = oracle.Tree(pos, np.array([0.5, 0.5]), prm).force()
    assert acc[0, 0] < 0 < acc[1, 0]
    # beyond the cutoff: no force, but the pair is still an entry (work done)
    pos = np.array([[0.2, 0.5, 0.5], [0.2 + 1.01 * rcut, 0.5, 0.5]])
    acc, npp, _ = oracle.Tree(pos, np.array([0.5, 0.5]), prm).force()
    assert np.all(acc == 0.0)


# ---------------------------------------------------------------------------
# whole-force invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["uniform", "halo"])
def test_theta_zero_equals_direct_sum(kind):
    if kind == "uniform":
        pos, mass, prm = gi.config("uniform-32k", n=4096)
    else:
        pos, mass, prm = gi.config("clustered-2m", n=4096)
        prm["opening"] = gi.OPEN_BH
    t = oracle.Tree(pos, mass, prm)
    acc, _, npn = t.force(theta=0.0)
    d = oracle.direct(pos, mass, prm)
    scale = np.abs(d).max()
    assert np.abs(acc - d).max() <= 1e-12 * scale
    assert np.all(npn == 0)
    # the relative criterion with alpha = 0 opens every node as well
    acc2, _, npn2 = t.force(opening=gi.OPEN_REL, alpha=0.0, a_old=np.ones((t.n, 3), np.float32))
    assert np.abs(acc2 - d).max() <= 1e-12 * scale and np.all(npn2 == 0)


def test_direct_equals_cell_list():
    pos, mass, prm = gi.config("uniform-32k", n=3000)
    d = oracle.direct(pos, mass, prm)
    c = oracle.cell_exact(pos, mass, prm)
    assert np.abs(d - c).max() <= 1e-12 * np.abs(d).max()


def test_split_off_no_cutoff_direct_sum_is_newton():
    # r_s <= 0: no split, no cutoff; compare with a plain numpy Newtonian sum
    pos, mass = gi.uniform(300, 13)
    prm = gi.default_params(eps=1e-4, r_s=0.0)
    d = oracle.direct(pos, mass, prm)
    q = np.array([[oracle.quantize1(v) for v in p] for p in pos], dtype=np.int64)
    diff = brute.min_image_int(q[None, :, :] - q[:, None, :]) / 2.0 ** 32
    r = np.sqrt((diff ** 2).sum(-1))
    np.fill_diagonal(r, np.inf)
    h = 2.8e-4
    assert r[np.isfinite(r)].min() > h
    a = (mass[None, :, None] * diff / r[..., None] ** 3).sum(1)
    assert np.abs(a - d).max() <= 1e-10 * np.abs(d).max()


def test_uniform_sphere_interior_profile():
    # the paper's CI free-fall check: initial acceleration of a uniform sphere
    R = 0.1
    pos, mass = gi.sphere(4096, 14, radius=R)
    prm = gi.default_params(eps=2e-4, r_s=0.0, theta=0.3)
    acc, _, _ = oracle.Tree(pos, mass, prm).force()
    rel = pos - 0.5
    r = np.linalg.norm(rel, axis=1)
    ar = (acc * rel).sum(1) / r
    sel = (r > 0.2 * R) & (r < 0.8 * R)
    slope = np.polyfit(r[sel], ar[sel], 1)[0]
    assert abs(slope / (-1.0 / R ** 3) - 1.0) < 0.03


def test_lattice_zero_force():
    pos, mass = gi.lattice(16)
    prm = gi.default_params(eps=1e-3, r_s=0.05, rcut_over_rs=4.5)
    t = oracle.Tree(pos, mass, prm)
    acc0, _, _ = t.force(theta=0.0)
    unit = mass[0] / (1.0 / 16) ** 2                        # one nearest-neighbour pull
    assert np.abs(acc0).max() < 1e-12 * unit
    acc5, _, _ = t.force(theta=0.5)
    assert np.abs(acc5).max() < 0.05 * unit


def test_momentum_conservation_as_theta_to_zero():
    pos, mass, prm = gi.config("uniform-32k", n=4096)
    t = oracle.Tree(pos, mass, prm)
    vals = []
    for th in (0.8, 0.5, 0.3, 0.1, 0.0):
        a, _, _ = t.force(theta=th)
        p = np.abs((mass[:, None] * a).sum(0)).max()
        vals.append(p / (mass * np.linalg.norm(a, axis=1)).sum())
    assert vals[-1] < 1e-13
    assert vals[0] > vals[2] > vals[3] > vals[4]


@pytest.mark.parametrize("opening", [gi.OPEN_BH, gi.OPEN_REL])
def test_list_partition_invariant(opening):
    pos, mass, prm = gi.config("clustered-2m", n=3000)
    prm["r_s"] = 0.02                                       # many neighbours at N = 3000
    t = oracle.Tree(pos, mass, prm)
    n = t.n
    a_old = np.asarray(oracle.direct(pos, mass, prm), dtype=np.float32)
    t.force(opening=opening, theta=0.6, alpha=0.01, a_old=a_old, keep_lists=True)
    off, lst = t.lists()
    beg, end = t.get(oracle.F_BEG), t.get(oracle.F_END)
    gb, ge = t.get(oracle.F_GBEG), t.get(oracle.F_GEND)
    perm = t.get(oracle.F_PERM)
    q = np.stack([t.get(f)[perm] for f in (oracle.F_X, oracle.F_Y, oracle.F_Z)], 1).astype(np.int64)
    rcg2 = (4.5 * prm["r_s"] * 2.0 ** 32) ** 2
    for g in range(t.ngroups):
        entries = lst[off[g]:off[g + 1]]
        cover = np.zeros(n, dtype=np.int64)
        for e in entries:
            if e < n:
                cover[e] += 1
            else:
                cover[beg[e - n]:end[e - n]] += 1
        assert cover.max() <= 1                              # never twice
        tgt = q[gb[g]:ge[g]]
        d = brute.min_image_int(q[None, :, :] - tgt[:, None, :]).astype(np.float64)
        near = ((d ** 2).sum(-1) < rcg2).any(0)
        assert np.all(cover[near] == 1)                      # every neighbour once
        # the group's own members are always PP entries
        assert set(range(gb[g], ge[g])) <= set(entries[entries < n].tolist())


# ---------------------------------------------------------------------------
# refit: same topology, drifted positions
# ---------------------------------------------------------------------------

def _drift(pos, seed, scale):
    r = np.random.default_rng(seed)
    return np.mod(pos + r.normal(0.0, scale, size=pos.shape), 1.0)


def test_refit_without_drift_is_the_built_tree():
    pos, mass, prm = gi.config("clustered-2m", n=6000)
    prm["r_s"] = 0.02
    t = oracle.Tree(pos, mass, prm)
    a0, p0, n0 = t.force(keep_lists=True)
    off0, l0 = t.lists()
    t.refit(pos)
    a1, p1, n1 = t.force(keep_lists=True)
    off1, l1 = t.lists()
    assert np.array_equal(a0, a1) and np.array_equal(p0, p1) and np.array_equal(n0, n1)
    assert np.array_equal(off0, off1) and np.array_equal(l0, l1)


def test_refit_extents_contain_members_and_partition_holds():
    pos, mass, prm = gi.config("clustered-2m", n=3000)
    prm["r_s"] = 0.02
    pos[:50, 0] = 0.999                       # these drift across the periodic boundary
    t = oracle.Tree(pos, mass, prm)
    new = _drift(pos, 3, 2e-3)
    t.refit(new)
    n = t.n
    perm = t.get(oracle.F_PERM)
    q = np.stack([t.get(f)[perm] for f in (oracle.F_X, oracle.F_Y, oracle.F_Z)], 1).astype(np.int64)
    es, el = t.get(oracle.F_EXT_S).astype(np.int64), t.get(oracle.F_EXT_L).astype(np.int64)
    beg, end = t.get(oracle.F_BEG), t.get(oracle.F_END)
    for j in range(t.nnodes):
        off = (q[beg[j]:end[j]] - es[j]) % (1 << 32)
        assert np.all(off <= el[j])            # every member inside the extent
    gb, ge = t.get(oracle.F_GBEG), t.get(oracle.F_GEND)
    glo, ghi = t.get(oracle.F_GLO).astype(np.int64), t.get(oracle.F_GHI).astype(np.int64)
    for g in range(t.ngroups):
        off = (q[gb[g]:ge[g]] - glo[g]) % (1 << 32)
        assert np.all(off <= (ghi[g] - glo[g]) % (1 << 32))
    t.force(theta=0.6, keep_lists=True)
    offl, lst = t.lists()
    rcg2 = (4.5 * prm["r_s"] * 2.0 ** 32) ** 2
    for g in range(t.ngroups):
        entries = lst[offl[g]:offl[g + 1]]
        cover = np.zeros(n, dtype=np.int64)
        for e in entries:
            if e < n:
                cover[e] += 1
            else:
                cover[beg[e - n]:end[e - n]] += 1
        assert cover.max() <= 1
        d = brute.min_image_int(q[None, :, :] - q[gb[g]:ge[g]][:, None, :]).astype(np.float64)
        near = ((d ** 2).sum(-1) < rcg2).any(0)
        assert np.all(cover[near] == 1)


def test_refit_theta_zero_equals_direct_sum():
    pos, mass, prm = gi.config("uniform-32k", n=3000)
    t = oracle.Tree(pos, mass, prm)
    new = _drift(pos, 4, 5e-3)
    t.refit(new)
    acc, _, _ = t.force(theta=0.0)
    d = oracle.direct(new, mass, prm)
    assert np.abs(acc - d).max() <= 1e-12 * np.abs(d).max()


# ---------------------------------------------------------------------------
# short-range potential (the potential output of the force call)
# ---------------------------------------------------------------------------

def test_spline_potential_is_the_integral_of_the_force_kernel():
    # psi(r) = integral_r^inf g(s) s ds with the quadrature-pinned force kernel g
    h = 0.8
    for r in [1e-6, 0.05, 0.2, 0.3999, 0.4, 0.4001, 0.55, 0.79, 0.8, 1.1]:
        tail, _ = integrate.quad(lambda s: oracle.soft_g(s, h) * s, r, h, epsabs=1e-13,
                                 epsrel=1e-13, limit=200) if r < h else (0.0, 0.0)
        expect = tail + 1.0 / max(r, h)
        assert abs(oracle.soft_psi(r, h) - expect) <= 1e-11 * expect, r
    eps = h / 2.8
    assert abs(oracle.soft_psi(0.0, h) - 1.0 / eps) <= 1e-14 / eps      # Plummer-equivalent
    for r0 in (h / 2, h):                                                # continuous
        assert abs(oracle.soft_psi(r0 * (1 - 1e-12), h) - oracle.soft_psi(r0 * (1 + 1e-12), h)) < 1e-9


def test_potential_derivative_gives_the_split_force():
    # -d/dr [erfc(r/2r_s) / r] = S(r) / r^2 outside the softening (r >= h)
    rs, h = 0.02, 1e-4
    for r in [0.001, 0.01, 0.03, 0.06, 0.09]:
        f = lambda x: oracle.soft_psi(x, h) * oracle.split_p(x, rs)
        dr = r * 1e-5
        deriv = (f(r + dr) - f(r - dr)) / (2 * dr)
        expect = -oracle.split_s(r, rs) / r ** 2
        assert abs(deriv - expect) <= 1e-7 * abs(expect), r
    assert oracle.split_p(0.5, 0.0) == 1.0                                # no split
    assert abs(oracle.split_p(0.04, 0.01) - special.erfc(2.0)) < 1e-15


def test_two_body_potential_closed_form():
    prm = gi.default_params(eps=1e-3, r_s=0.02, opening=gi.OPEN_BH, theta=0.5)
    h, rcut = 2.8e-3, 4.5 * 0.02
    for r in (0.5 * h, 2 * h, 0.03, 0.08, rcut * 1.01):
        pos = np.array([[0.3, 0.4, 0.5], [0.3 + r, 0.4, 0.5]])
        mass = np.array([2e-3, 3e-3])
        _, pot = oracle.direct_pot(pos, mass, prm)
        d = (oracle.quantize1(0.3 + r) - oracle.quantize1(0.3)) / 2 ** 32   # exact grid separation
        if d < rcut:
            psi = oracle.soft_psi(d, h) * special.erfc(d / (2 * 0.02))
            assert abs(pot[0] + 3e-3 * psi) <= 1e-12 * 3e-3 * psi
            assert abs(pot[1] + 2e-3 * psi) <= 1e-12 * 2e-3 * psi
        else:
            assert pot[0] == 0.0 and pot[1] == 0.0                         # beyond the cutoff


@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_tree_potential_theta_zero_equals_direct(kind):
    if kind == "uniform":
        pos, mass, prm = gi.config("uniform-32k", n=3000)
    else:
        pos, mass, prm = gi.config("clustered-2m", n=3000)
        prm["opening"] = gi.OPEN_BH
    t = oracle.Tree(pos, mass, prm)
    acc, _, _, pot = t.force_pot(theta=0.0)
    d_acc, d_pot = oracle.direct_pot(pos, mass, prm)
    assert np.abs(pot - d_pot).max() <= 1e-12 * np.abs(d_pot).max()
    assert np.abs(acc - d_acc).max() <= 1e-12 * np.abs(d_acc).max()

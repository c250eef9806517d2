"""Pins of the oracle's node-opening decision and of its cutoff decision.

The walk of Sect. 4.1.2 accepts a node as one particle-node entry or opens it.
Three tests decide: the boundary check (the group box meets the node's cell
enlarged by 10 % on every side: open), then either the Barnes-Hut angle
(open iff l^2 > theta^2 d^2, d = distance from the group box to the node's
centre of mass) or the relative criterion (open iff G M l^2 > alpha a_min s^2
d^4).  The bit-exact list parity of the CUDA path rests on these decisions, so
each is pinned here on hand-placed trees: one target group facing one node,
with every distance, cell side, mass and threshold an exact integer or power
of two, so the expected decision is a comparison of exact rationals done in
this file.  Each threshold is probed on both sides and, where it can occur,
at equality.

The cutoff is a step in the force, so the in/out decision of a pair at the
cutoff is part of the method's definition.  It is taken in single precision
on the integer separation (the reading on the cutoff).  The pin computes that
decision independently with exact integer arithmetic and round-to-nearest-even
to 24 bits, and checks that it agrees with the exact rational decision
wherever the two are further apart than single precision can resolve.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import og_inputs as gi
import oracle

TWO32 = 1 << 32
LEV = 7                       # level of the probed node's cell
ELL = 1 << (32 - LEV)         # its side in grid units (2^25)
ORIGIN = 1 << 31              # cell origin on every axis: [2^31, 2^31 + 2^25)
COMX = ORIGIN + 3 * (ELL >> 3)  # centre of mass on x: l/8 below the cell's centre


def _pos(*pts):
    """Grid integers -> positions in the unit box (exact: k / 2^32 is a double)."""
    return np.array(pts, dtype=np.float64) / TWO32


def _prm(**kw):
    # no split: no cutoff and no prune, so only the opening test decides
    p = gi.default_params(eps=1e-6, r_s=0.0, group_max=1)
    p.update(kw)
    return p


def _node_of(t, sorted_members):
    beg, end = t.get(oracle.F_BEG), t.get(oracle.F_END)
    want = (min(sorted_members), max(sorted_members) + 1)
    ids = [i for i in range(t.nnodes) if (beg[i], end[i]) == want]
    assert len(ids) == 1
    return ids[0]


def _decision(pts, masses, target_idx, node_members, a_old=None, opening=gi.OPEN_BH,
              theta=0.5, alpha=0.005, G=1.0, group_max=1):
    """'accept' if the node holding ``node_members`` (input indices) is a PN
    entry of the group of input particle ``target_idx``; 'open' if its
    members appear as PP entries instead."""
    pos = _pos(*pts)
    mass = np.asarray(masses, dtype=np.float64)
    t = oracle.Tree(pos, mass, _prm(G=G, group_max=group_max))
    perm = t.get(oracle.F_PERM)
    sidx = {int(p): s for s, p in enumerate(perm)}        # input index -> sorted index
    node = _node_of(t, [sidx[i] for i in node_members])
    assert int(t.get(oracle.F_LEVEL)[node]) == LEV
    gb, ge = t.get(oracle.F_GBEG), t.get(oracle.F_GEND)
    g = [k for k in range(t.ngroups) if gb[k] <= sidx[target_idx] < ge[k]]
    ao = None if a_old is None else np.asarray(a_old, dtype=np.float32)
    t.force(opening=opening, theta=theta, alpha=alpha, a_old=ao, groups=np.array(g),
            keep_lists=True)
    _, lst = t.lists()
    lst = set(int(v) for v in lst)
    if node + t.n in lst:
        assert not any(sidx[i] in lst for i in node_members)
        return "accept"
    assert all(sidx[i] in lst for i in node_members)
    return "open"


def _pair(com_x, masses=(0.25, 0.25), y=ORIGIN + (ELL >> 1), z=ORIGIN + (ELL >> 1)):
    """Two particles A, B in the cell [2^31, 2^31 + 2^25)^3 on opposite sides
    of its x midplane (so that cell is their node), both at (y, z), with
    centre of mass com_x on x exactly: B just above the midplane, A where
    mA xA + mB xB = (mA + mB) com_x puts it (an integer below the midplane)."""
    mA, mB = (Fraction(m) for m in masses)
    for delta in range(64, 96):
        xB = ORIGIN + (ELL >> 1) + delta
        xA = (Fraction(com_x) * (mA + mB) - mB * xB) / mA
        if xA.denominator == 1 and ORIGIN <= xA < ORIGIN + (ELL >> 1):
            return [(int(xA), y, z), (xB, y, z)]
    raise AssertionError("no exact placement")


# ---------------------------------------------------------------------------
# Barnes-Hut: open iff l^2 > theta^2 d^2, d to the centre of mass
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dist, expect", [(2 * ELL, "accept"),        # equality accepts
                                          (2 * ELL - 1, "open"),
                                          (2 * ELL + 1, "accept")])
def test_bh_threshold_on_the_distance_to_the_centre_of_mass(dist, expect):
    # theta = 1/2: l^2 > d^2 / 4  <=>  d < 2 l.  The target sits on the centre
    # of mass's y and z, so d is the x gap alone.
    com_x = COMX                                 # not the cell's centre
    pair = _pair(com_x)
    y, z = pair[0][1], pair[0][2]
    pts = [(com_x - dist, y, z)] + pair          # target in the root's other x half
    assert pts[0][0] < ORIGIN
    assert _decision(pts, [0.5, 0.25, 0.25], 0, [1, 2], theta=0.5) == expect
    # exact rationals: l^2 vs theta^2 d^2
    lhs, rhs = Fraction(ELL) ** 2, Fraction(1, 4) * Fraction(dist) ** 2
    assert (lhs > rhs) == (expect == "open")


def test_bh_distance_is_to_the_centre_of_mass_not_the_cell_centre():
    # the same cell and the same target; the centre of mass moves by one grid
    # unit across the threshold d = 2 l.  The cell centre stays 2 l + l/8 from
    # the target, so a test on the cell centre would accept all three.
    tx = COMX - 2 * ELL
    y = z = ORIGIN + (ELL >> 1)
    got = []
    for shift in (-1, 0, 1):
        pts = [(tx, y, z)] + _pair(COMX + shift)
        t = oracle.Tree(_pos(*pts), np.array([0.5, 0.25, 0.25]), _prm())
        com = t.get(oracle.F_COM)
        assert (COMX + shift) in com[:, 0].tolist()
        got.append(_decision(pts, [0.5, 0.25, 0.25], 0, [1, 2], theta=0.5))
    assert got == ["open", "accept", "accept"]


@pytest.mark.parametrize("k, expect", [(9586980, "open"), (9586981, "accept")])
def test_bh_distance_is_three_dimensional(k, expect):
    # gaps (2k, 3k, 6k): d = 7k, threshold 7k >= 2 l = 67108864 (theta 1/2);
    # k = 9586980 gives d = 67108860 < 2 l (open), k = 9586981 gives
    # d = 67108867 > 2 l (accept).  Any one axis alone, or the largest gap,
    # is below 2 l for both.
    com = (COMX, ORIGIN + (ELL >> 1), ORIGIN + (ELL >> 1))
    pair = _pair(com[0], y=com[1], z=com[2])
    tgt = (com[0] - 2 * k, com[1] - 3 * k, com[2] - 6 * k)
    assert _decision([tgt] + pair, [0.5, 0.25, 0.25], 0, [1, 2], theta=0.5) == expect
    d2 = Fraction(2 * k) ** 2 + Fraction(3 * k) ** 2 + Fraction(6 * k) ** 2
    assert (Fraction(ELL) ** 2 > Fraction(1, 4) * d2) == (expect == "open")


@pytest.mark.parametrize("theta, expect", [(0.5, "open"), (0.25, "open"), (1.0, "accept")])
def test_bh_uses_theta_squared(theta, expect):
    # d = 1.5 l: open iff l^2 > theta^2 (9/4) l^2  <=>  theta < 2/3.
    # theta = 1/2 opens (theta instead of theta^2 would accept: l^2 vs 9/8 l^2)
    com_x = COMX
    pair = _pair(com_x)
    y, z = pair[0][1], pair[0][2]
    pts = [(com_x - 3 * (ELL >> 1), y, z)] + pair
    assert _decision(pts, [0.5, 0.25, 0.25], 0, [1, 2], theta=theta) == expect


def test_bh_distance_is_from_the_group_box_edge():
    # a group of two targets spread along x: d is from the box's nearer face,
    # not from the group's centre or first member
    com_x = COMX
    pair = _pair(com_x)
    y, z = pair[0][1], pair[0][2]
    near = com_x - (2 * ELL - 1)                 # nearer face: d = 2 l - 1 -> open
    far = near - (ELL >> 1)
    pts = [(far, y, z), (near, y, z)] + pair
    assert _decision(pts, [0.25, 0.25, 0.25, 0.25], 0, [2, 3], theta=0.5, group_max=2) == "open"
    near = com_x - 2 * ELL                       # d = 2 l -> accept
    far = near - (ELL >> 1)
    pts = [(far, y, z), (near, y, z)] + pair
    assert _decision(pts, [0.25, 0.25, 0.25, 0.25], 0, [2, 3], theta=0.5, group_max=2) == "accept"


# ---------------------------------------------------------------------------
# relative criterion: open iff G M l^2 > alpha a_min s^2 d^4
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dist, expect", [(1 << 26, "accept"),        # equality accepts
                                          ((1 << 26) - 1, "open"),
                                          ((1 << 26) + 1, "accept")])
def test_relative_threshold(dist, expect):
    # G = 4, M = 1/2, l^2 = 2^50: lhs = 2^51.  alpha = 1/2, a_min = 2^12,
    # s^2 = 2^-64, d = 2^26: rhs = 2^-1 2^12 2^-64 2^104 = 2^51 (equality).
    G, alpha, amin = 4.0, 0.5, 4096.0
    com_x = COMX
    pair = _pair(com_x, masses=(0.375, 0.125))
    y, z = pair[0][1], pair[0][2]
    pts = [(com_x - dist, y, z)] + pair
    a_old = [[amin, 0.0, 0.0], [1.0, 0.0, 0.0], [1.0, 0.0, 0.0]]
    got = _decision(pts, [0.5, 0.375, 0.125], 0, [1, 2], a_old=a_old, opening=gi.OPEN_REL,
                    alpha=alpha, G=G)
    assert got == expect
    lhs = Fraction(G) * Fraction(1, 2) * Fraction(ELL) ** 2
    rhs = Fraction(alpha) * Fraction(amin) * Fraction(1, TWO32) ** 2 * Fraction(dist) ** 4
    assert (lhs > rhs) == (expect == "open")


@pytest.mark.parametrize("G, alpha, amin, expect", [
    (4.0, 0.5, 4096.0, "open"),      # the reference case of d = 2^26 - 1
    (1.0, 0.5, 4096.0, "accept"),    # G enters: G = 1 gives lhs = 2^49 < rhs
    (4.0, 1.0, 4096.0, "accept"),    # alpha enters on the right
    (4.0, 0.5, 8192.0, "accept"),    # so does a_min
    (4.0, 0.5, 2048.0, "open"),
])
def test_relative_each_factor_enters(G, alpha, amin, expect):
    dist = (1 << 26) - 1
    com_x = COMX
    pair = _pair(com_x, masses=(0.375, 0.125))
    y, z = pair[0][1], pair[0][2]
    pts = [(com_x - dist, y, z)] + pair
    a_old = [[0.0, amin, 0.0], [1.0, 0.0, 0.0], [1.0, 0.0, 0.0]]   # |a| of any direction
    got = _decision(pts, [0.5, 0.375, 0.125], 0, [1, 2], a_old=a_old, opening=gi.OPEN_REL,
                    alpha=alpha, G=G)
    lhs = Fraction(G) * Fraction(1, 2) * Fraction(ELL) ** 2
    rhs = Fraction(alpha) * Fraction(amin) * Fraction(1, TWO32) ** 2 * Fraction(dist) ** 4
    assert (lhs > rhs) == (expect == "open")
    assert got == expect


def test_relative_uses_the_fourth_power_and_the_group_minimum():
    # halving d multiplies d^4 by 1/16: at d = 2^25 the same parameters need
    # a_min 16 times larger to accept
    G, alpha = 4.0, 0.5
    com_x = COMX
    pair = _pair(com_x, masses=(0.375, 0.125))
    y, z = pair[0][1], pair[0][2]
    dist = 1 << 25
    for amin, expect in ((16 * 4096.0, "accept"), (16 * 4096.0 - 8.0, "open")):
        pts = [(com_x - dist, y, z)] + pair
        a_old = [[amin, 0.0, 0.0], [1.0, 0.0, 0.0], [1.0, 0.0, 0.0]]
        assert _decision(pts, [0.5, 0.375, 0.125], 0, [1, 2], a_old=a_old, opening=gi.OPEN_REL,
                         alpha=alpha, G=G) == expect
    # a group of two targets: a_min is the smaller |a_old| of the two members
    near = com_x - (1 << 26)
    pts = [(near - (ELL >> 1), y, z), (near, y, z)] + pair
    for a0, a1, expect in ((4096.0, 1e6, "accept"), (1e6, 4096.0, "accept"),
                           (4095.0, 1e6, "open"), (1e6, 4095.0, "open")):
        a_old = [[a0, 0.0, 0.0], [a1, 0.0, 0.0], [1.0, 0.0, 0.0], [1.0, 0.0, 0.0]]
        assert _decision(pts, [0.25, 0.25, 0.375, 0.125], 0, [2, 3], a_old=a_old,
                         opening=gi.OPEN_REL, alpha=alpha, G=G, group_max=2) == expect


# ---------------------------------------------------------------------------
# boundary check: open iff the group box meets the cell enlarged by 10 %
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("axis", [0, 1, 2])
def test_boundary_check_at_six_tenths_of_the_side(axis):
    # theta = 4 accepts whenever d >= l / 4, so only the boundary check can
    # open.  The centre of mass sits near the cell's low corner on every axis,
    # the target beyond the cell's centre by dc on one axis and on the centre
    # on the others.  10 dc <= 6 l <=> dc <= floor(3 l / 5) = 20132659.
    lim = (3 * ELL) // 5
    assert 10 * lim <= 6 * ELL < 10 * (lim + 1)
    centre = ORIGIN + (ELL >> 1)
    low = ORIGIN + 64
    # equal masses on opposite sides of the x midplane, both near the low y/z corner
    xA, xB = ORIGIN + 64, ORIGIN + ELL - 64
    pair = [(xA, low, low), (xB, low, low)] if axis else [(ORIGIN + 64, low, low),
                                                           (ORIGIN + (ELL >> 1) + 64, low, low)]
    for dc, expect in ((lim, "open"), (lim + 1, "accept")):
        tgt = [centre, centre, centre]
        tgt[axis] = centre + dc
        assert _decision([tuple(tgt)] + pair, [0.5, 0.25, 0.25], 0, [1, 2], theta=4.0) == expect
    # the boundary check needs every axis near: far on one axis, no opening
    tgt = [centre + lim, centre + lim, centre + lim]
    tgt[axis] = centre + lim + 1
    assert _decision([tuple(tgt)] + pair, [0.5, 0.25, 0.25], 0, [1, 2], theta=4.0) == "accept"


# ---------------------------------------------------------------------------
# the cutoff decision: single precision on the exact integer separation
# ---------------------------------------------------------------------------

def _rn24(v: int) -> int:
    """An integer rounded to the nearest single-precision value (ties to even)."""
    if v == 0:
        return 0
    s, a = (-1 if v < 0 else 1), abs(v)
    sh = a.bit_length() - 24
    if sh <= 0:
        return v
    q, r = divmod(a, 1 << sh)
    half = 1 << (sh - 1)
    if r > half or (r == half and q & 1):
        q += 1
    return s * (q << sh)


def _active_f32(d, rcg2: float) -> bool:
    """The reading's decision: f = float(d) per axis, r2 = fma(fx, fx, fma(fy,
    fy, fz * fz)) with every operation rounded to single precision, active
    iff 0 < r2 < float(rcut_grid^2)."""
    fx, fy, fz = (_rn24(int(v)) for v in d)
    r2 = _rn24(fx * fx + _rn24(fy * fy + _rn24(fz * fz)))
    rc = _rn24(int(rcg2))
    return 0 < r2 < rc


def _direct_active(d, prm):
    """Whether ora_direct lets a source at separation d (grid units) act on a
    target: the decision seen through the FP64 direct sum."""
    c = np.array([1 << 30, 1 << 30, 1 << 30], dtype=np.int64)
    pts = [tuple(int(v) for v in c), tuple(int(v) % TWO32 for v in c + np.asarray(d, np.int64))]
    acc = oracle.direct(_pos(*pts), np.array([0.5, 0.5]), prm, targets=np.array([0]))
    return bool(np.any(acc[0] != 0.0))


def _active_f32_other_order(d, rcg2: float) -> bool:
    """The same decision with the sum taken as (fx fx + fy fy) + fz fz, every
    product and sum rounded: a plausible other reading of the order."""
    fx, fy, fz = (_rn24(int(v)) for v in d)
    r2 = _rn24(_rn24(_rn24(fx * fx) + _rn24(fy * fy)) + _rn24(fz * fz))
    return 0 < r2 < _rn24(int(rcg2))


def test_cutoff_decision_single_precision_on_the_integer_separation():
    # r_cut = 4.5 r_s with r_s = 1.25/256: 94371840 grid units exactly
    prm = gi.default_params(eps=1e-9, r_s=1.25 / 256, rcut_over_rs=4.5, theta=0.0)
    rcg = (4.5 * (1.25 / 256)) * TWO32
    assert rcg == 94371840.0
    rcg2 = rcg * rcg
    R = 94371840
    r = np.random.default_rng(7)
    clear = boundary = differ_exact = differ_order = 0
    cases = [(R, 0, 0), (R - 1, 0, 0), (R + 1, 0, 0), (0, R - 1, 0), (0, 0, -(R - 3)),
             (R - 4, 0, 0), (R - 5, 0, 0), (R + 4, 0, 0)]
    # random directions within a few tens of grid units of the sphere r = r_cut
    for _ in range(1500):
        v = r.normal(size=3)
        v *= R / np.linalg.norm(v)
        cases.append(tuple(int(round(x)) + int(r.integers(-60, 61)) for x in v))
    for d in cases:
        exact2 = sum(int(x) * int(x) for x in d)
        want = _active_f32(d, rcg2)
        got = _direct_active(d, prm)
        assert got == want, d
        differ_exact += want != (0 < exact2 < R * R)
        differ_order += want != _active_f32_other_order(d, rcg2)
        # where single precision resolves the difference, the decision is the
        # exact one: active iff r < r_cut
        if abs(Fraction(exact2) - Fraction(R) ** 2) > Fraction(R) ** 2 / (1 << 21):
            assert want == (exact2 < R * R), d
            clear += 1
        else:
            boundary += 1
    assert clear > 100 and boundary > 100
    # the cases tell the reading apart from an exact (or FP64) decision and
    # from another order of the single-precision sum
    assert differ_exact > 0 and differ_order > 0


def test_cutoff_single_precision_differs_from_exact_at_the_boundary():
    # r_cut = 2^26 grid units (r_s = 2^-8, 4 r_s): a separation of 2^26 - 1
    # is inside exactly but rounds to 2^26 in single precision, which is
    # not below r_cut^2 = 2^52: no force.  2^26 - 4 is representable and inside.
    prm = gi.default_params(eps=1e-9, r_s=2.0 ** -8, rcut_over_rs=4.0, theta=0.0)
    rcg2 = float(1 << 52)
    assert not _active_f32(((1 << 26) - 1, 0, 0), rcg2)
    assert not _direct_active(((1 << 26) - 1, 0, 0), prm)
    assert _active_f32(((1 << 26) - 4, 0, 0), rcg2)
    assert _direct_active(((1 << 26) - 4, 0, 0), prm)
    assert not _direct_active((1 << 26, 0, 0), prm)         # strict: r = r_cut is out
    assert not _direct_active((0, 0, 0), prm)               # the particle itself
    # the tree at theta = 0 takes the same decision
    for d, want in ((((1 << 26) - 1, 0, 0), False), (((1 << 26) - 4, 0, 0), True)):
        c = 1 << 30
        pts = _pos((c, c, c), (c + d[0], c + d[1], c + d[2]))
        acc, _, _ = oracle.Tree(pts, np.array([0.5, 0.5]), prm).force(theta=0.0)
        assert bool(np.any(acc[0] != 0.0)) == want

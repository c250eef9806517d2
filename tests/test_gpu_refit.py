"""og_tree_refit against the oracle's refit.

After a refit the topology and groups stay; positions, moments, node extents
(cell joined with the drifted members) and group boxes are recomputed, and
the walk tests against extents.  Bit-exact: positions, node masses, centres
of mass, extents, group boxes, lists, counts.  Tolerance: accelerations.
"""
from __future__ import annotations

import numpy as np
import pytest

import og_inputs as gi
import oracle
from paper_2609_17658_gb300 import build as B
from paper_2609_17658_gb300 import og
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    B.build()
    oracle.build()
    c = og.Context(0)
    yield c
    c.close()


def _drift(pos, seed, scale):
    r = np.random.default_rng(seed)
    return np.mod(pos + r.normal(0.0, scale, size=pos.shape), 1.0)


def _compare_refit(gt, ot):
    n = ot.n
    perm = ot.get(oracle.F_PERM)
    spos = gt.export(og.OG_F_SPOS)
    for a, f in enumerate((oracle.F_X, oracle.F_Y, oracle.F_Z)):
        assert np.array_equal(spos[a], ot.get(f)[perm])
    gmap = parity.node_map(gt, ot)
    m = ot.nnodes
    inv = np.empty(m, dtype=np.int64)
    inv[gmap] = np.arange(m)
    assert np.array_equal(gt.export(og.OG_F_MASS)[inv].view(np.uint64), ot.get(oracle.F_MASS).view(np.uint64))
    assert np.array_equal(gt.export(og.OG_F_MSUM)[inv].view(np.uint64), ot.get(oracle.F_MSUM).view(np.uint64))
    assert np.array_equal(gt.export(og.OG_F_COM)[inv], ot.get(oracle.F_COM))
    ext = gt.export(og.OG_F_EXTENT)
    assert np.array_equal(ext[0][inv], ot.get(oracle.F_EXT_S))
    assert np.array_equal(ext[1][inv], ot.get(oracle.F_EXT_L))
    box = gt.export(og.OG_F_GBOX)
    assert np.array_equal(box[:, :3], ot.get(oracle.F_GLO))
    assert np.array_equal(box[:, 3:], ot.get(oracle.F_GHI))
    return gmap


@pytest.mark.parametrize("scale", [1e-4, 2e-3])
def test_refit_matches_oracle(ctx, scale):
    pos, mass, prm = gi.config("clustered-2m", n=40000)
    prm = dict(prm, opening=gi.OPEN_BH, r_s=0.015, flags=og.OG_DEBUG_DUMP_LISTS)
    pos[:300, 0] = 1.0 - 1e-5                      # these cross the periodic boundary
    new = _drift(pos, 7, scale)
    gt = og.Tree(ctx, pos, mass, prm)
    ot = oracle.Tree(pos, mass, prm)
    gt.refit(new)
    ot.refit(new)
    gmap = _compare_refit(gt, ot)
    acc, npp, npn = gt.force()
    ref, rpp, rpn = ot.force(keep_lists=True)
    off, lst = ot.lists()
    parity.compare_lists(parity.gpu_lists(gt, gmap), off, lst, range(ot.ngroups))
    assert np.array_equal(npp, rpp) and np.array_equal(npn, rpn)
    parity.check_accel(acc, ref)


def test_refit_relative_criterion(ctx):
    pos, mass, prm = gi.config("clustered-2m", n=30000)
    prm["r_s"] = 0.015
    new = _drift(pos, 8, 5e-4)
    a1, _, _ = og.Tree(ctx, new, mass, dict(prm, opening=gi.OPEN_BH)).force(counts=False)
    gt = og.Tree(ctx, pos, mass, prm)
    ot = oracle.Tree(pos, mass, prm)
    gt.refit(new)
    ot.refit(new)
    acc, npp, npn = gt.force(a_old=a1)
    ref, rpp, rpn = ot.force(a_old=a1)
    assert np.array_equal(npp, rpp) and np.array_equal(npn, rpn)
    parity.check_accel(acc, ref)


def test_refit_without_drift_is_bitwise_the_build(ctx):
    pos, mass, prm = gi.config("uniform-32k", n=20000)
    gt = og.Tree(ctx, pos, mass, prm)
    a0, p0, n0 = gt.force()
    gt.refit(pos)
    a1, p1, n1 = gt.force()
    assert np.array_equal(a0, a1) and np.array_equal(p0, p1) and np.array_equal(n0, n1)


def test_refit_rejects_wrong_input(ctx):
    pos, mass, prm = gi.config("uniform-32k", n=1000)
    gt = og.Tree(ctx, pos, mass, prm)
    bad = pos.copy()
    bad[3, 2] = np.inf
    with pytest.raises(og.OGError):
        gt.refit(bad)


def test_refit_exact_moments_with_spread_masses(ctx):
    """The refit's moments are the same exact sums as the build's: masses spread
    over 2^-20..2^20 and some zero, positions drifted across cells and the
    periodic boundary; node masses, sums and centres of mass bitwise the oracle's."""
    r = np.random.default_rng(41)
    pos, _, prm = gi.config("clustered-2m", n=30000)
    mass = np.ldexp(1.0 + r.random(len(pos)), r.integers(-20, 21, len(pos)))
    mass[r.random(len(pos)) < 0.1] = 0.0
    prm = dict(prm, opening=gi.OPEN_BH)
    gt = og.Tree(ctx, pos, mass, prm)
    ot = oracle.Tree(pos, mass, prm)
    for k, scale in enumerate((3e-4, 3e-3)):
        pos = _drift(pos, 50 + k, scale)
        gt.refit(pos)
        ot.refit(pos)
        _compare_refit(gt, ot)

"""Forces on an active subset (og_tree_force_active).

With individual time steps only the active particles need new
accelerations.  Every group holding an active particle is walked exactly as
in the full force call, so an active particle's result is bitwise that of
og_tree_force on the same tree, the oracle walking the same groups gives the
same lists and counts, and inactive entries of the outputs are left alone.
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


def _mask(n, frac, seed):
    return (np.random.default_rng(seed).random(n) < frac).astype(np.uint8)


def _active(gt, active, a_old=None):
    n = gt.n
    acc = np.full((n, 3), 7.0, np.float32)                 # sentinels: must survive
    npp = np.full(n, 12345, np.uint32)
    npn = np.full(n, 54321, np.uint32)
    ao = None if a_old is None else np.ascontiguousarray(a_old, np.float32)
    walked = og.og_tree_force_active(gt.h, active, acc, ao, npp, npn)
    return acc, npp, npn, walked


@pytest.mark.parametrize("frac", [0.002, 0.1, 1.0])
def test_active_equals_full_and_leaves_the_rest(ctx, frac):
    pos, mass, prm = gi.config("clustered-2m", n=50000)
    prm = dict(prm, opening=gi.OPEN_BH)
    gt = og.Tree(ctx, pos, mass, prm)
    full, fpp, fpn = gt.force()
    act = _mask(len(mass), frac, 3)
    acc, npp, npn, walked = _active(gt, act)
    on = act != 0
    assert np.array_equal(acc[on], full[on])
    assert np.array_equal(npp[on], fpp[on]) and np.array_equal(npn[on], fpn[on])
    assert (acc[~on] == 7.0).all() and (npp[~on] == 12345).all() and (npn[~on] == 54321).all()
    assert 0 < walked <= gt.info()["groups"]
    if frac == 1.0:
        assert walked == gt.info()["groups"]


def test_active_groups_against_the_oracle(ctx):
    pos, mass, prm = gi.config("clustered-2m", n=40000)
    prm = dict(prm, opening=gi.OPEN_BH, r_s=0.015)
    gt = og.Tree(ctx, pos, mass, prm)
    ot = oracle.Tree(pos, mass, prm)
    act = _mask(len(mass), 0.05, 4)
    acc, npp, npn, walked = _active(gt, act)
    perm = ot.get(oracle.F_PERM)
    gb, ge = ot.get(oracle.F_GBEG), ot.get(oracle.F_GEND)
    sel = np.array([g for g in range(ot.ngroups) if act[perm[gb[g]:ge[g]]].any()], dtype=np.int64)
    assert walked == len(sel)
    ref, rpp, rpn = ot.force(groups=sel)
    on = np.flatnonzero(act)
    assert np.array_equal(npp[on], rpp[on]) and np.array_equal(npn[on], rpn[on])
    parity.check_accel(acc[on], ref[on])


def test_active_relative_criterion(ctx):
    pos, mass, prm = gi.config("clustered-2m", n=30000)
    gt = og.Tree(ctx, pos, mass, prm)
    a1, _, _ = og.Tree(ctx, pos, mass, dict(prm, opening=gi.OPEN_BH)).force(counts=False)
    full, fpp, fpn = gt.force(a_old=a1)
    act = _mask(len(mass), 0.2, 5)
    acc, npp, npn, _ = _active(gt, act, a_old=a1)
    on = act != 0
    assert np.array_equal(acc[on], full[on])
    assert np.array_equal(npp[on], fpp[on]) and np.array_equal(npn[on], fpn[on])


def test_no_active_particle_walks_nothing(ctx):
    pos, mass, prm = gi.config("uniform-32k", n=5000)
    gt = og.Tree(ctx, pos, mass, prm)
    acc, npp, npn, walked = _active(gt, np.zeros(len(mass), np.uint8))
    assert walked == 0 and (acc == 7.0).all() and (npp == 12345).all()


def test_active_device_pointers(ctx):
    torch = pytest.importorskip("torch")
    pos, mass, prm = gi.config("uniform-32k", n=20000)
    act = _mask(len(mass), 0.3, 6)
    host = og.Tree(ctx, pos, mass, prm)
    acc_h, _, _, _ = _active(host, act)
    dprm = dict(prm, flags=og.OG_DEVICE_PTRS)
    dev = og.Tree(ctx, torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(), dprm)
    acc_d = torch.full((len(mass), 3), 7.0, dtype=torch.float32, device="cuda")
    og.og_tree_force_active(dev.h, torch.from_numpy(act).cuda(), acc_d)
    torch.cuda.synchronize()
    assert np.array_equal(acc_d.cpu().numpy(), acc_h)

"""The potential output (og_tree_force_pot) against the oracle.

phi_i = -G sum_j m_j psi(r) erfc(r / 2 r_s) over the force call's own lists.
Tolerance: every term is positive and carries the erfc approximation's
absolute error of at most 1.5e-7, i.e. at most 1.03e-4 relative at the cutoff
(erfc(2.25) = 1.46e-3), so no particle's sum can be worse than that plus
FP32 accumulation: max 1.5e-4, and p99 <= 1e-4.  Without the split the
potential is the softened Newtonian one and the bound is FP32 rounding.
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


def _rel(got, ref):
    """Relative error where the reference is nonzero; a particle with no
    neighbour inside the cutoff must get exactly zero."""
    got = got.astype(np.float64)
    zero = ref == 0.0
    assert (got[zero] == 0.0).all()
    return np.abs(got[~zero] - ref[~zero]) / np.abs(ref[~zero])


@pytest.mark.parametrize("name", ["uniform-32k", "clustered-2m"])
def test_potential_matches_the_oracle(ctx, name):
    pos, mass, prm = gi.config(name, n=30000)
    prm = dict(prm, opening=gi.OPEN_BH)
    gt = og.Tree(ctx, pos, mass, prm)
    acc, npp, npn, pot = gt.force_pot()
    ref, rpp, rpn, rpot = oracle.Tree(pos, mass, prm).force_pot()
    assert np.array_equal(npp, rpp) and np.array_equal(npn, rpn)
    parity.check_accel(acc, ref)
    e = _rel(pot, rpot)
    assert (pot <= 0).all()
    assert e.max() <= 1.5e-4 and np.quantile(e, 0.99) <= 1e-4


def test_force_unchanged_by_the_potential_output(ctx):
    pos, mass, prm = gi.config("clustered-2m", n=20000)
    gt = og.Tree(ctx, pos, mass, prm)
    a1, p1, n1 = gt.force()
    a2, p2, n2, _ = gt.force_pot()
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2) and np.array_equal(n1, n2)


def test_potential_relative_criterion_and_no_split(ctx):
    pos, mass, prm = gi.config("clustered-2m", n=20000)
    a1, _, _ = og.Tree(ctx, pos, mass, dict(prm, opening=gi.OPEN_BH)).force(counts=False)
    _, _, _, pot = og.Tree(ctx, pos, mass, prm).force_pot(a_old=a1)
    _, _, _, rpot = oracle.Tree(pos, mass, prm).force_pot(a_old=a1)
    assert _rel(pot, rpot).max() <= 1.5e-4
    nos = dict(prm, opening=gi.OPEN_BH, r_s=0.0)
    _, _, _, pot0 = og.Tree(ctx, pos, mass, nos).force_pot()
    _, _, _, rpot0 = oracle.Tree(pos, mass, nos).force_pot()
    assert _rel(pot0, rpot0).max() <= 1e-5


def test_potential_theta_zero_is_the_direct_sum(ctx):
    pos, mass, prm = gi.config("uniform-32k", n=4000)
    _, _, _, pot = og.Tree(ctx, pos, mass, dict(prm, theta=0.0)).force_pot()
    _, dpot = oracle.direct_pot(pos, mass, prm)
    assert _rel(pot, dpot).max() <= 1.5e-4


def test_potential_device_pointers(ctx):
    torch = pytest.importorskip("torch")
    pos, mass, prm = gi.config("uniform-32k", n=10000)
    _, _, _, ph = og.Tree(ctx, pos, mass, prm).force_pot()
    dt = og.Tree(ctx, torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(), prm)
    acc = torch.zeros((len(mass), 3), dtype=torch.float32, device="cuda")
    pot = torch.zeros(len(mass), dtype=torch.float32, device="cuda")
    og.og_tree_force_pot(dt.h, acc, pot)
    torch.cuda.synchronize()
    assert np.array_equal(pot.cpu().numpy(), ph)

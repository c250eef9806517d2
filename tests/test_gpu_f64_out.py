"""og_tree_force_f64: the force call with double-precision output.

The walk and its FP32 sums are those of og_tree_force; only the last pass
leaves the sums in grid units and the scaling to G M / L^2 is one FP64
multiplication.  So the result is og_tree_force's within the FP32 rounding
of that scaling (2^-24 relative, well inside 3e-7), the counts are the
same, and the oracle tolerance holds.  A first Barnes-Hut pass (relative
criterion without a_old) keeps its FP32 scaling: its result is the a_old
of the second pass, and the lists must not change.
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


def _f64(tree, n, a_old=None):
    acc = np.zeros((n, 3), np.float64)
    npp = np.zeros(n, np.uint32)
    npn = np.zeros(n, np.uint32)
    og.og_tree_force_f64(tree.h, acc, a_old, npp, npn)
    return acc, npp, npn


@pytest.mark.parametrize("opening", [gi.OPEN_BH, gi.OPEN_REL])
def test_f64_output_is_the_float_call_scaled_in_fp64(ctx, opening):
    pos, mass, prm = gi.config("clustered-2m", n=30000)
    prm = dict(prm, opening=opening, box=2.0, G=0.7)
    pos = pos * 2.0
    gt = og.Tree(ctx, pos, mass, prm)
    a32, p32, n32 = gt.force()
    a64, p64, n64 = _f64(gt, len(mass))
    assert np.array_equal(p64, p32) and np.array_equal(n64, n32)
    scale = np.maximum(np.abs(a32.astype(np.float64)), 1e-300)
    assert (np.abs(a64 - a32) <= 3e-7 * scale).all()
    ref, rpp, rpn = oracle.Tree(pos, mass, prm).force(
        a_old=None if opening == gi.OPEN_BH else
        og.Tree(ctx, pos, mass, dict(prm, opening=gi.OPEN_BH)).force(counts=False)[0])
    assert np.array_equal(p64, rpp) and np.array_equal(n64, rpn)
    parity.check_accel(a64, ref)


def test_f64_output_device_pointers(ctx):
    torch = pytest.importorskip("torch")
    pos, mass, prm = gi.config("uniform-32k", n=20000)
    host = og.Tree(ctx, pos, mass, prm)
    ah, _, _ = _f64(host, len(mass))
    dprm = dict(prm, flags=og.OG_DEVICE_PTRS)
    dev = og.Tree(ctx, torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(), dprm)
    ad = torch.zeros((len(mass), 3), dtype=torch.float64, device="cuda")
    og.og_tree_force_f64(dev.h, ad)
    torch.cuda.synchronize()
    assert np.array_equal(ad.cpu().numpy(), ah)


def test_f64_output_then_float_call_unchanged(ctx):
    pos, mass, prm = gi.config("uniform-32k", n=10000)
    gt = og.Tree(ctx, pos, mass, prm)
    a1, p1, n1 = gt.force()
    _f64(gt, len(mass))
    a2, p2, n2 = gt.force()
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2) and np.array_equal(n1, n2)

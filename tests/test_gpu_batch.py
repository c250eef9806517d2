"""Many boxes in one og_batch_force call.

Each box's tree, lists and summation order are the same in the batch as when
it is built and walked alone, so its accelerations and counts must be
bitwise identical to og_tree_build + og_tree_force on that box, for the
Barnes-Hut and the two-pass relative criterion.  A few boxes are also checked
against the FP64 oracle.
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


def _boxes(opening, seed=5, count=24):
    r = np.random.default_rng(seed)
    out = []
    sizes = [1, 2, 7, 33, 500, 4096, 20000] + list(r.integers(100, 30000, size=count - 7))
    for k, n in enumerate(sizes):
        if k % 2:
            pos, mass = gi.halo_mix(int(n), 100 + k, n_halo=max(1, int(n) // 2000))
        else:
            pos, mass = gi.uniform(int(n), 100 + k)
        side = max(int(n), 512) ** (1 / 3)
        prm = gi.default_params(eps=1 / (50 * side), r_s=1.25 / (2 * side), opening=opening,
                                theta=0.4 + 0.05 * (k % 5), alpha=0.004 + 0.001 * (k % 3),
                                box=1.0 if k % 3 else 2.0)
        if prm["box"] == 2.0:
            pos = pos * 2.0
        out.append((pos, mass, prm))
    return out


@pytest.mark.parametrize("opening", [gi.OPEN_BH, gi.OPEN_REL])
def test_batch_equals_each_box_alone(ctx, opening):
    boxes = _boxes(opening)
    descs = []
    for pos, mass, prm in boxes:
        n = len(mass)
        descs.append(dict(pos=pos, mass=mass, params=prm, acc=np.zeros((n, 3), np.float32),
                          n_pp=np.zeros(n, np.uint32), n_pn=np.zeros(n, np.uint32)))
    info = og.og_batch_force(ctx.h, descs)
    assert info["boxes"] == len(boxes) and info["particles"] == sum(len(b[1]) for b in boxes)
    total = 0
    for (pos, mass, prm), d in zip(boxes, descs):
        acc, npp, npn = og.Tree(ctx, pos, mass, prm).force()
        assert np.array_equal(d["acc"], acc)
        assert np.array_equal(d["n_pp"], npp) and np.array_equal(d["n_pn"], npn)
        total += int(((npp.astype(np.int64) + npn)).sum())
    if opening == gi.OPEN_BH:
        assert info["interactions"] == total


def test_batch_with_given_a_old_and_oracle(ctx):
    boxes = _boxes(gi.OPEN_REL, seed=9, count=10)
    descs = []
    for pos, mass, prm in boxes:
        n = len(mass)
        bh = dict(prm, opening=gi.OPEN_BH, theta=prm["theta_first_pass"])
        a1, _, _ = og.Tree(ctx, pos, mass, bh).force(counts=False)
        descs.append(dict(pos=pos, mass=mass, params=prm, a_old=a1,
                          acc=np.zeros((n, 3), np.float32), n_pp=np.zeros(n, np.uint32),
                          n_pn=np.zeros(n, np.uint32)))
    og.og_batch_force(ctx.h, descs)
    for (pos, mass, prm), d in zip(boxes, descs):
        if len(mass) < 500:
            continue
        ref, rpp, rpn = oracle.Tree(pos, mass, prm).force(a_old=d["a_old"])
        assert np.array_equal(d["n_pp"], rpp) and np.array_equal(d["n_pn"], rpn)
        parity.check_accel(d["acc"], ref)


def test_batch_device_pointers(ctx):
    torch = pytest.importorskip("torch")
    boxes = _boxes(gi.OPEN_BH, seed=11, count=8)
    host, dev = [], []
    for pos, mass, prm in boxes:
        n = len(mass)
        host.append(dict(pos=pos, mass=mass, params=prm, acc=np.zeros((n, 3), np.float32)))
        dev.append(dict(pos=torch.from_numpy(pos).cuda(), mass=torch.from_numpy(mass).cuda(),
                        params=prm, acc=torch.zeros((n, 3), dtype=torch.float32, device="cuda")))
    og.og_batch_force(ctx.h, host)
    og.og_batch_force(ctx.h, dev)
    torch.cuda.synchronize()
    for h, d in zip(host, dev):
        assert np.array_equal(h["acc"], d["acc"].cpu().numpy())


def test_batch_rejects_mixed_criteria(ctx):
    boxes = _boxes(gi.OPEN_BH, count=8)
    descs = [dict(pos=p, mass=m, params=dict(q, opening=k % 2), acc=np.zeros((len(m), 3), np.float32))
             for k, (p, m, q) in enumerate(boxes)]
    with pytest.raises(og.OGError) as e:
        og.og_batch_force(ctx.h, descs)
    assert e.value.status == og.OG_ERR_ARG

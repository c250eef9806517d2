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


def test_fullsize_batch_sampled(ctx):
    """The batched workload at full size, in the launch configuration the
    benchmark times: 512 boxes with N log-uniform in [4096, 262144] (about
    35M particles), device pointers, one og_batch_force call.  Six boxes (the
    largest, the smallest and four drawn at random) are checked against the
    oracle on sampled groups: counts exact, accelerations within tolerance,
    and every box's counts are those of its own tree's group sizes."""
    torch = pytest.importorskip("torch")
    boxes = gi.batch_boxes(512)
    descs = []
    for b in boxes:
        n = len(b.mass)
        descs.append(dict(pos=torch.from_numpy(b.pos).cuda(), mass=torch.from_numpy(b.mass).cuda(),
                          params=b.params,
                          acc=torch.empty((n, 3), dtype=torch.float32, device="cuda"),
                          n_pp=torch.empty(n, dtype=torch.int32, device="cuda"),
                          n_pn=torch.empty(n, dtype=torch.int32, device="cuda")))
    info = og.og_batch_force(ctx.h, descs)
    torch.cuda.synchronize()
    sizes = np.array([len(b.mass) for b in boxes])
    assert info["boxes"] == 512 and info["particles"] == int(sizes.sum())
    r = np.random.default_rng(17)
    pick = {int(sizes.argmax()), int(sizes.argmin())}
    while len(pick) < 6:
        pick.add(int(r.integers(0, len(boxes))))
    for k in sorted(pick):
        b = boxes[k]
        acc = descs[k]["acc"].cpu().numpy()
        npp = descs[k]["n_pp"].cpu().numpy().view(np.uint32)
        npn = descs[k]["n_pn"].cpu().numpy().view(np.uint32)
        ot = oracle.Tree(b.pos, b.mass, b.params)
        sel = np.sort(r.choice(ot.ngroups, size=min(60, ot.ngroups), replace=False)).astype(np.int64)
        ref, rpp, rpn = ot.force(groups=sel)
        perm = ot.get(oracle.F_PERM)
        gb, ge = ot.get(oracle.F_GBEG), ot.get(oracle.F_GEND)
        tgt = np.concatenate([perm[gb[g]:ge[g]] for g in sel])
        assert np.array_equal(npp[tgt], rpp[tgt]) and np.array_equal(npn[tgt], rpn[tgt]), k
        parity.check_accel(acc[tgt], ref[tgt])

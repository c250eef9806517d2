"""Measured walk configuration (og_params.group_max = 0).

The tuner picks the group size G among 8, 16, 24, 32 and then the walk's
launch shape (warps per block, far-chunk entries) by timing the walk on the
caller's input, once per key (log2 N, criterion, split on/off).  A tree built
with group_max = 0 must be the tree built with that configuration explicitly
(bitwise), its lists and forces must match the oracle run with the same G, a
saved table must load into a fresh context without re-measuring, and every
launch shape must give the same lists (bitwise the same forces for the same
chunk length, since warps per block do not change any arithmetic).
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


def test_auto_group_size_is_the_explicit_build(ctx):
    pos, mass, prm = gi.config("clustered-2m", n=60000)
    auto = dict(prm, group_max=0)
    cfg = og.og_tune_walk(ctx.h, pos, mass, auto)
    G = cfg["group_max"]
    assert G in (8, 16, 24, 32) and og.og_tune_group_max(ctx.h, pos, mass, auto) == G
    assert cfg["walk_warps"] in (2, 4, 8) and cfg["walk_chunk"] in (128, 256, 512)
    ta = og.Tree(ctx, pos, mass, auto)
    info = ta.info()
    assert (info["group_max"], info["walk_warps"], info["walk_chunk"]) == \
        (G, cfg["walk_warps"], cfg["walk_chunk"])
    te = og.Tree(ctx, pos, mass, dict(prm, **cfg))
    for f in (og.OG_F_GBEG, og.OG_F_GEND, og.OG_F_GBOX):
        assert np.array_equal(ta.export(f), te.export(f))
    a1, p1, n1 = ta.force()
    a2, p2, n2 = te.force()
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2) and np.array_equal(n1, n2)


def test_auto_group_size_matches_the_oracle(ctx):
    pos, mass, prm = gi.config("clustered-2m", n=30000)
    prm = dict(prm, opening=gi.OPEN_BH, r_s=0.015, group_max=0)
    gt = og.Tree(ctx, pos, mass, prm)
    G = gt.info()["group_max"]
    ot = oracle.Tree(pos, mass, dict(prm, group_max=G))
    assert gt.info()["groups"] == ot.ngroups
    acc, npp, npn = gt.force()
    ref, rpp, rpn = ot.force()
    assert np.array_equal(npp, rpp) and np.array_equal(npn, rpn)
    parity.check_accel(acc, ref)


def test_saved_table_loads_without_measuring(ctx, tmp_path):
    pos, mass, prm = gi.config("uniform-32k", n=20000)
    G = og.og_tune_group_max(ctx.h, pos, mass, prm)
    path = str(tmp_path / "tune.jsonl")
    og.og_tune_save(ctx.h, path)
    text = open(path).read()
    assert '"group_max": %d' % G in text and '"n_log2": 14' in text
    assert '"walk_warps": ' in text and '"walk_chunk": ' in text
    fresh = og.Context(0)
    try:
        og.og_tune_load(fresh.h, path)
        before = og.og_kernel_launches()
        assert og.og_tune_group_max(fresh.h, pos, mass, prm) == G
        assert og.og_kernel_launches() == before     # a table lookup launches nothing
    finally:
        fresh.close()


def test_load_rejects_other_files(ctx, tmp_path):
    bad = tmp_path / "bad.jsonl"
    for line in ('{"n_log2": 14, "opening": 0, "split": 1, "group_max": 99, "walk_warps": 4, "walk_chunk": 256}',
                 '{"n_log2": 14, "opening": 0, "split": 1, "group_max": 32, "walk_warps": 9, "walk_chunk": 256}',
                 '{"n_log2": 14, "opening": 0, "split": 1, "group_max": 32, "walk_warps": 4, "walk_chunk": 48}',
                 '{"n_log2": 14, "opening": 0, "split": 1, "group_max": 32}'):
        bad.write_text(line + "\n")
        with pytest.raises(og.OGError) as e:
            og.og_tune_load(ctx.h, str(bad))
        assert e.value.status == og.OG_ERR_ARG
    with pytest.raises(og.OGError):
        og.og_tune_load(ctx.h, str(tmp_path / "missing.jsonl"))


@pytest.mark.parametrize("opening", [gi.OPEN_BH, gi.OPEN_REL])
def test_launch_shapes(ctx, opening):
    pos, mass, prm = gi.config("clustered-2m", n=40000)
    prm = dict(prm, opening=opening, group_max=32)
    ref = og.Tree(ctx, pos, mass, dict(prm, walk_warps=4, walk_chunk=256))
    a0, p0, n0 = ref.force()
    for w in (1, 2, 8):
        t = og.Tree(ctx, pos, mass, dict(prm, walk_warps=w, walk_chunk=256))
        a, p, n = t.force()
        assert np.array_equal(a, a0) and np.array_equal(p, p0) and np.array_equal(n, n0), w
    ot = oracle.Tree(pos, mass, prm)
    a1, _, _ = og.Tree(ctx, pos, mass, dict(prm, opening=gi.OPEN_BH)).force(counts=False)
    oref = ot.force(a_old=a1) if opening == gi.OPEN_REL else ot.force()
    for w, c in ((2, 64), (8, 1024), (3, 100)):
        t = og.Tree(ctx, pos, mass, dict(prm, walk_warps=w, walk_chunk=c))
        a, p, n = t.force(a_old=a1) if opening == gi.OPEN_REL else t.force()
        assert np.array_equal(p, p0) and np.array_equal(n, n0), (w, c)
        assert np.array_equal(p, oref[1]) and np.array_equal(n, oref[2])
        parity.check_accel(a, oref[0])


def test_invalid_launch_shapes(ctx):
    pos, mass, prm = gi.config("uniform-32k", n=1000)
    for bad in (dict(walk_warps=9), dict(walk_warps=-1), dict(walk_chunk=63), dict(walk_chunk=1025)):
        with pytest.raises(og.OGError) as e:
            og.Tree(ctx, pos, mass, dict(prm, **bad))
        assert e.value.status == og.OG_ERR_ARG

"""Measured group size (og_params.group_max = 0).

The tuner picks G among 8, 16, 24, 32 by timing the walk on the caller's
input, once per key (log2 N, criterion, split on/off).  A tree built with
group_max = 0 must be the tree built with that G explicitly (bitwise), its
lists and forces must match the oracle run with the same G, and a saved
table must load into a fresh context without re-measuring.
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
    G = og.og_tune_group_max(ctx.h, pos, mass, auto)
    assert G in (8, 16, 24, 32)
    ta = og.Tree(ctx, pos, mass, auto)
    assert ta.info()["group_max"] == G
    te = og.Tree(ctx, pos, mass, dict(prm, group_max=G))
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
    bad.write_text('{"n_log2": 14, "opening": 0, "split": 1, "group_max": 99}\n')
    with pytest.raises(og.OGError) as e:
        og.og_tune_load(ctx.h, str(bad))
    assert e.value.status == og.OG_ERR_ARG
    with pytest.raises(og.OGError):
        og.og_tune_load(ctx.h, str(tmp_path / "missing.jsonl"))

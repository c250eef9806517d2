"""og_sort_keys_noalloc: the sort for callers that cannot allocate device memory.

Checked through the C-ABI against the sort inside og_tree_build (the sorted
keys and permutation that og_tree_export returns), on two calls in a row with
different inputs, so that state left in the shared static scratch by the first
call cannot leak into the second.  Integer results, so the comparison is exact.
This file is collected last on purpose.
"""
from __future__ import annotations

import numpy as np
import pytest

import og_inputs as gi
from paper_2609_17658_gb300 import build as B
from paper_2609_17658_gb300 import og

pytestmark = pytest.mark.gpu


def _reference(ctx, pos, mass):
    t = og.Tree(ctx, pos, mass, gi.default_params(r_s=0.01))
    skey = t.export(og.OG_F_SKEY)
    perm = t.export(og.OG_F_PERM)
    t.free()
    keys_in = np.empty_like(skey)
    keys_in[perm] = skey            # the keys in the caller's order
    return keys_in, skey, perm


def test_noalloc_sort_matches_tree_build_sort():
    torch = pytest.importorskip("torch")
    B.build()
    with og.Context(0) as ctx:
        cases = [gi.halo_mix(300_000, 31, n_halo=40), gi.uniform(70_001, 32)]
        cases[1][0][:500] = cases[1][0][7]          # equal keys: order must stay stable
        for pos, mass in cases:
            keys_in, skey, perm = _reference(ctx, pos, mass)
            n = len(keys_in)
            d_in = torch.from_numpy(keys_in.view(np.int64)).cuda()
            d_out = torch.empty(n, dtype=torch.int64, device="cuda")
            d_perm = torch.empty(n, dtype=torch.int32, device="cuda")
            og.og_sort_keys_noalloc(d_in, d_out, d_perm)
            torch.cuda.synchronize()
            assert np.array_equal(d_out.cpu().numpy().view(np.uint64), skey)
            assert np.array_equal(d_perm.cpu().numpy().view(np.uint32), perm)
            assert np.array_equal(d_in.cpu().numpy().view(np.uint64), keys_in)


def test_noalloc_sort_rejects_oversize():
    torch = pytest.importorskip("torch")
    B.build()
    n = og.OG_NOALLOC_MAX_N + 1
    d = torch.zeros(n, dtype=torch.int64, device="cuda")
    p = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(og.OGError) as e:
        og.og_sort_keys_noalloc(d, d.clone(), p)
    assert e.value.status == og.OG_ERR_ARG
    assert "OG_NOALLOC_MAX_N" in str(e.value)

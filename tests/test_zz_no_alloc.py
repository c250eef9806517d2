"""og_sort_keys_noalloc: the sort for callers that cannot allocate device memory.

Some callers of this library cannot allocate at the moment they need a sort: a
serving process that has committed its whole HBM budget to resident trees, or
a latency-critical loop in which a cudaMalloc/cudaFree (which can synchronise
the device) is not allowed.  This entry point sorts in a fixed static device
array instead.  The tests check it through the C-ABI:

* against the sort inside og_tree_build (the sorted keys and permutation that
  og_tree_export returns) and against numpy's stable argsort, on two calls in
  a row with different inputs, so that state left in the shared scratch by the
  first call cannot leak into the second;
* on full 64-bit keys (bit 63 set), on n = 1 and on n = OG_NOALLOC_MAX_N, and
  on a stream other than the default one;
* that a call changes neither the device's free memory nor torch's
  allocations;
* that oversize inputs, host pointers and overlapping buffers are rejected.

Integer results, so every comparison is exact.  This file is collected last
on purpose: if it fails, a run that stops at the first failure has already
run every other test.
"""
from __future__ import annotations

import ctypes

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


def _sort(torch, keys, stream=None):
    n = len(keys)
    d_in = torch.from_numpy(keys.view(np.int64)).cuda()
    d_out = torch.empty(n, dtype=torch.int64, device="cuda")
    d_perm = torch.empty(n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    og.og_sort_keys_noalloc(d_in, d_out, d_perm,
                            stream_handle=None if stream is None else stream.cuda_stream)
    (stream or torch.cuda.current_stream()).synchronize()
    return (d_out.cpu().numpy().view(np.uint64), d_perm.cpu().numpy().view(np.uint32),
            d_in.cpu().numpy().view(np.uint64))


def test_noalloc_sort_matches_tree_build_sort():
    torch = pytest.importorskip("torch")
    B.build()
    with og.Context(0) as ctx:
        cases = [gi.halo_mix(300_000, 31, n_halo=40), gi.uniform(70_001, 32)]
        cases[1][0][:500] = cases[1][0][7]          # equal keys: order must stay stable
        for pos, mass in cases:
            keys_in, skey, perm = _reference(ctx, pos, mass)
            out, p, kin = _sort(torch, keys_in)
            assert np.array_equal(out, skey)
            assert np.array_equal(p, perm)
            assert np.array_equal(p, np.argsort(keys_in, kind="stable"))
            assert np.array_equal(kin, keys_in)


def test_noalloc_sort_full_64_bit_keys_and_size_limits():
    torch = pytest.importorskip("torch")
    B.build()
    r = np.random.default_rng(5)
    nmax = og.OG_NOALLOC_MAX_N
    big = r.integers(0, 1 << 64, size=nmax, dtype=np.uint64, endpoint=False)
    big[:4096] = big[4096:8192]                       # ties across the array
    big[10:20] = np.uint64(1 << 63)                   # bit 63 alone
    big[20:30] = np.uint64((1 << 64) - 1)             # every bit
    few = np.array([np.uint64((1 << 64) - 2), np.uint64(3), np.uint64(1 << 63), np.uint64(3)],
                   dtype=np.uint64)
    side = torch.cuda.Stream()
    for keys, stream in ((big, None), (np.array([np.uint64(1 << 63) + 5]), None), (few, side),
                         (big[::-1].copy(), side)):
        out, p, kin = _sort(torch, keys, stream)
        expect = np.argsort(keys, kind="stable")
        assert np.array_equal(p, expect)
        assert np.array_equal(out, keys[expect])
        assert np.array_equal(kin, keys)


def test_noalloc_sort_allocates_nothing():
    torch = pytest.importorskip("torch")
    B.build()
    r = np.random.default_rng(6)
    keys = r.integers(0, 1 << 63, size=500_000, dtype=np.uint64)
    n = len(keys)
    d_in = torch.from_numpy(keys.view(np.int64)).cuda()
    d_out = torch.empty(n, dtype=torch.int64, device="cuda")
    d_perm = torch.empty(n, dtype=torch.int32, device="cuda")
    og.og_sort_keys_noalloc(d_in, d_out, d_perm)      # first call: set-up of the scratch address
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        og.og_sort_keys_noalloc(d_in, d_out, d_perm)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert np.array_equal(d_perm.cpu().numpy().view(np.uint32), np.argsort(keys, kind="stable"))


def test_noalloc_sort_rejects_oversize_host_and_overlap():
    torch = pytest.importorskip("torch")
    B.build()
    n = og.OG_NOALLOC_MAX_N + 1
    d = torch.zeros(n, dtype=torch.int64, device="cuda")
    p = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(og.OGError) as e:
        og.og_sort_keys_noalloc(d, d.clone(), p)
    assert e.value.status == og.OG_ERR_ARG
    assert "OG_NOALLOC_MAX_N" in str(e.value)
    # the binding refuses host tensors before the C call
    with pytest.raises(TypeError):
        og.og_sort_keys_noalloc(torch.zeros(8, dtype=torch.int64), d[:8], p[:8])
    # the C entry point itself refuses a host address (no kernel is launched)
    host = np.zeros(8, dtype=np.uint64)
    L = og.lib()
    st = L.og_sort_keys_noalloc(host.ctypes.data_as(ctypes.c_void_p),
                                ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(p.data_ptr()),
                                ctypes.c_int64(8), None)
    assert st == og.OG_ERR_ARG
    # keys_out overlapping keys_in by part of the range, or perm_out inside the keys
    with pytest.raises(og.OGError) as e:
        og.og_sort_keys_noalloc(d[:1000], d[500:1500], p[:1000])
    assert e.value.status == og.OG_ERR_ARG
    with pytest.raises(og.OGError) as e:
        og.og_sort_keys_noalloc(d[:1000], d[2000:3000], d[200:700].view(torch.int32))
    assert e.value.status == og.OG_ERR_ARG
    # keys sorted in place are allowed
    k = torch.from_numpy(np.array([5, 1, 3], dtype=np.int64)).cuda()
    q = torch.zeros(3, dtype=torch.int32, device="cuda")
    og.og_sort_keys_noalloc(k, k, q)
    torch.cuda.synchronize()
    assert k.cpu().tolist() == [1, 3, 5] and q.cpu().tolist() == [1, 2, 0]

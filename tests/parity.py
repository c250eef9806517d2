"""Comparison helpers: CUDA library (through the C-ABI) vs the FP64 oracle.

Node ids are a labelling choice (the oracle numbers nodes in depth-first
preorder, the CUDA build in the order of each node's first split), so nodes
are matched by what is unique about them: (first particle, level).  Every
reference through a node id is translated through that match before it is
compared.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2609_17658_gb300 import og

# accuracy bar for accelerations against the FP64 oracle with the same lists
P99_MAX = 1e-4
RMS_MAX = 2e-5


def node_map(gt: og.Tree, ot: oracle.Tree):
    """GPU node id -> oracle node id."""
    g_lev = gt.export(og.OG_F_LEVEL).astype(np.int64)
    g_beg = gt.export(og.OG_F_NBEG).astype(np.int64)
    o_lev = ot.get(oracle.F_LEVEL).astype(np.int64)
    o_beg = ot.get(oracle.F_BEG)
    okey = {(int(b), int(l)): i for i, (b, l) in enumerate(zip(o_beg, o_lev))}
    assert len(okey) == len(o_lev)
    gmap = np.array([okey[(int(b), int(l))] for b, l in zip(g_beg, g_lev)], dtype=np.int64)
    assert len(set(gmap.tolist())) == len(gmap)
    return gmap


def map_unified(refs, n, gmap):
    refs = np.asarray(refs, dtype=np.int64)
    out = refs.copy()
    node = (refs >= n) & (refs >= 0)
    out[node] = gmap[refs[node] - n] + n
    return out


def compare_build(gt: og.Tree, ot: oracle.Tree):
    """Bit-exact comparison of keys, permutation, positions, topology,
    threading, moments and groups."""
    n = ot.n
    perm_o = ot.get(oracle.F_PERM)
    assert np.array_equal(gt.export(og.OG_F_PERM).astype(np.int64), perm_o), "sort permutation"
    assert np.array_equal(gt.export(og.OG_F_SKEY), ot.get(oracle.F_KEY)[perm_o]), "sorted keys"
    spos = gt.export(og.OG_F_SPOS)
    for a, f in enumerate((oracle.F_X, oracle.F_Y, oracle.F_Z)):
        assert np.array_equal(spos[a], ot.get(f)[perm_o]), "fixed-point positions"
    info = gt.info()
    assert info["nodes"] == ot.nnodes, "node count"
    assert info["groups"] == ot.ngroups, "group count"
    gmap = node_map(gt, ot)
    m = ot.nnodes
    inv = np.empty(m, dtype=np.int64)
    inv[gmap] = np.arange(m)
    # per oracle id, the GPU values
    g_end = gt.export(og.OG_F_NEND).astype(np.int64)[inv]
    assert np.array_equal(g_end, ot.get(oracle.F_END)), "node ranges"
    g_par = gt.export(og.OG_F_PARENT).astype(np.int64)[inv]
    g_par = np.where(g_par >= 0, gmap[np.maximum(g_par, 0)], -1)
    assert np.array_equal(g_par, ot.get(oracle.F_PARENT)), "parents"
    g_ccnt = gt.export(og.OG_F_CCNT).astype(np.int64)[inv]
    assert np.array_equal(g_ccnt, ot.get(oracle.F_CCNT)), "child counts"
    g_cbeg = gt.export(og.OG_F_CBEG).astype(np.int64)[inv]
    g_child = map_unified(gt.export(og.OG_F_CHILD), n, gmap)
    o_child = ot.get(oracle.F_CHILD)
    # the oracle stores the child blocks contiguously in node-id order
    excl = np.concatenate([[0], np.cumsum(g_ccnt)[:-1]])
    idx = np.repeat(g_cbeg, g_ccnt) + (np.arange(int(g_ccnt.sum())) - np.repeat(excl, g_ccnt))
    assert np.array_equal(g_child[idx], o_child), "child lists"
    g_mass = gt.export(og.OG_F_MASS)[inv]
    assert np.array_equal(g_mass.view(np.uint64), ot.get(oracle.F_MASS).view(np.uint64)), "node mass (bitwise)"
    assert np.array_equal(gt.export(og.OG_F_MSUM)[inv].view(np.uint64),
                          ot.get(oracle.F_MSUM).view(np.uint64)), "node sums of m x (bitwise)"
    assert np.array_equal(gt.export(og.OG_F_COM)[inv], ot.get(oracle.F_COM)), "centre of mass"
    g_next = map_unified(gt.export(og.OG_F_NEXTNODE), n, gmap)[inv]
    assert np.array_equal(g_next, ot.get(oracle.F_NEXTNODE)), "nextnode"
    g_sib = map_unified(gt.export(og.OG_F_SIBLING), n, gmap)[inv]
    assert np.array_equal(g_sib, ot.get(oracle.F_SIBLING)), "sibling"
    g_pn = map_unified(gt.export(og.OG_F_PNEXT), n, gmap)
    assert np.array_equal(g_pn, ot.get(oracle.F_PNEXT)), "particle next"
    assert np.array_equal(gt.export(og.OG_F_GBEG).astype(np.int64), ot.get(oracle.F_GBEG)), "groups"
    assert np.array_equal(gt.export(og.OG_F_GEND).astype(np.int64), ot.get(oracle.F_GEND)), "groups"
    box = gt.export(og.OG_F_GBOX)
    assert np.array_equal(box[:, :3], ot.get(oracle.F_GLO)), "group boxes"
    assert np.array_equal(box[:, 3:], ot.get(oracle.F_GHI)), "group boxes"
    return gmap


def gpu_lists(gt: og.Tree, gmap, groups=None):
    """Dumped (group, child slot) pairs -> {group: sorted unified refs (oracle ids)},
    for every group or only for ``groups``."""
    pairs = gt.export(og.OG_F_LISTS)
    if groups is not None:
        want = np.zeros(gt.info()["groups"], dtype=bool)
        want[np.asarray(groups, dtype=np.int64)] = True
        pairs = pairs[want[pairs[:, 0]]]
    pairs = pairs.astype(np.int64)
    child = gt.export(og.OG_F_CHILD).astype(np.int64)
    n = gt.n
    refs = map_unified(child[pairs[:, 1]], n, gmap)
    order = np.lexsort((refs, pairs[:, 0]))
    g, r = pairs[order, 0], refs[order]
    out = {}
    bounds = np.flatnonzero(np.r_[True, g[1:] != g[:-1], True])
    for a, b in zip(bounds[:-1], bounds[1:]):
        out[int(g[a])] = r[a:b]
    return out


def compare_lists(gl: dict, off, lst, groups):
    for k, g in enumerate(groups):
        ref = lst[off[k]:off[k + 1]]
        got = gl.get(int(g), np.zeros(0, dtype=np.int64))
        assert np.array_equal(got, ref), f"interaction list of group {g}: {len(got)} vs {len(ref)}"


def accel_errors(acc, ref, mask=None):
    """Relative error per particle; particles whose reference acceleration is
    below 1e-6 of the rms magnitude are left out (reported by the caller)."""
    ref = np.asarray(ref, dtype=np.float64)
    acc = np.asarray(acc, dtype=np.float64)
    if mask is not None:
        ref, acc = ref[mask], acc[mask]
    na = np.linalg.norm(ref, axis=1)
    floor = 1e-6 * np.sqrt(np.mean(na ** 2))
    keep = na > floor
    e = np.linalg.norm(acc[keep] - ref[keep], axis=1) / na[keep]
    return e, int((~keep).sum())


def check_accel(acc, ref, mask=None, p99=P99_MAX, rms=RMS_MAX):
    e, nfloor = accel_errors(acc, ref, mask)
    q = float(np.quantile(e, 0.99)) if e.size else 0.0
    r = float(np.sqrt(np.mean(e ** 2))) if e.size else 0.0
    assert q <= p99, f"p99 relative error {q:.3e} > {p99}"
    assert r <= rms, f"rms relative error {r:.3e} > {rms}"
    return q, r, nfloor

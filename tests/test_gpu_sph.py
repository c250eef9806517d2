"""og_tree_sph_density: grouped neighbour search and SPH density (Sect. 3.4,
Sect. 6) against the oracle (oracle/sph.py) on the same u32 positions.

The neighbour decision is float32 arithmetic on exact integers on both sides,
so the neighbour counts must be equal.  The density sums up to a few thousand
float32 terms m_j w(q) (each within a few units of float32 rounding of the
float64 value), so the bar is 2e-5 relative for tens of neighbours and 1e-4 for
the case with thousands.
"""
from __future__ import annotations

import numpy as np
import pytest

import og_inputs as gi
from oracle import pm, sph
from paper_2609_17658_gb300 import build as B
from paper_2609_17658_gb300 import og

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    B.build()
    c = og.Context(0)
    yield c
    c.close()


def knn_h(pos, box, k=33, scale=1.0, rng=None):
    """Smoothing lengths from the distance to the k-th nearest particle (itself first)."""
    from scipy.spatial import cKDTree
    x = pm.quantize(pos, box).astype(np.float64) * (box / 2.0 ** 32)
    d, _ = cKDTree(x, boxsize=box).query(x, k=min(k, len(x)), workers=-1)
    h = d[:, -1] * scale if d.ndim == 2 else np.full(len(x), 0.1 * box)
    if rng is not None:
        h = h * rng.uniform(0.5, 2.0, len(h))
    return np.minimum(h, 0.45 * box).astype(np.float32)


def _check(rho, cnt, ref, rcnt, tol):
    assert np.array_equal(cnt.astype(np.int64), rcnt)
    assert np.all(np.abs(rho - ref) <= tol * ref), float(np.max(np.abs(rho - ref) / ref))


@pytest.mark.parametrize("name,n,mode", [("uniform-32k", None, "knn"), ("clustered-2m", 100000, "knn"),
                                         ("clustered-2m", 3001, "mixed"), ("uniform-32k", 1, "knn"),
                                         ("clustered-2m", 40000, "mixed")])
def test_matches_the_oracle(ctx, name, n, mode):
    pos, mass, prm = gi.config(name, n=n) if n else gi.config(name)
    h = knn_h(pos, prm["box"], rng=np.random.default_rng(5) if mode == "mixed" else None)
    t = og.Tree(ctx, pos, mass, prm)
    rho, cnt = t.sph_density(h)
    ref, rcnt = sph.density(pm.quantize(pos, prm["box"]), mass, h, prm["box"])
    _check(rho, cnt, ref, rcnt, 2e-5)
    r2, c2 = t.sph_density(h)
    assert np.array_equal(r2, rho) and np.array_equal(c2, cnt)


def test_full_size_workload(ctx):
    pos, mass, prm = gi.config("clustered-2m")
    h = knn_h(pos, prm["box"])
    t = og.Tree(ctx, pos, mass, prm)
    rho, cnt = t.sph_density(h)
    assert t.info()["ms_sph"] > 0
    sample = np.random.default_rng(3).choice(len(mass), 150000, replace=False)
    ref, rcnt = sph.density(pm.quantize(pos, prm["box"]), mass, h, prm["box"], targets=sample)
    _check(rho[sample], cnt[sample], ref, rcnt, 2e-5)
    assert cnt.min() >= 1 and np.median(cnt) == 32


def test_thousands_of_neighbours_and_a_non_unit_box(ctx):
    rng = np.random.default_rng(12)
    box = 2.5
    pos = rng.uniform(0, box, (3000, 3))
    pos[:500] = rng.normal(1.2, 0.05, (500, 3)) % box
    mass = rng.uniform(0.5, 1.5, 3000) / 3000
    h = (rng.uniform(0.1, 1.1, 3000) * box / 2.5).astype(np.float32)
    prm = dict(gi.config("uniform-32k", n=10)[2], box=box, r_s=0.01 * box)
    t = og.Tree(ctx, pos, mass, prm)
    rho, cnt = t.sph_density(h)
    ref, rcnt = sph.density(pm.quantize(pos, box), mass, h, box)
    assert rcnt.max() > 1000
    _check(rho, cnt, ref, rcnt, 1e-4)


def test_exact_ties_and_coincident_particles(ctx):
    pos = np.array([[0.25, 0.5, 0.5], [0.375, 0.5, 0.5], [0.25, 0.5, 0.375 + 2.0 ** -27],
                    [0.7, 0.7, 0.7], [0.7, 0.7, 0.7], [0.7, 0.7, 0.7]])
    mass = np.ones(6)
    h = np.full(6, 0.125, np.float32)
    prm = gi.config("uniform-32k", n=10)[2]
    rho, cnt = og.Tree(ctx, pos, mass, prm).sph_density(h)
    assert list(cnt) == [2, 1, 2, 3, 3, 3]
    ref, rcnt = sph.density(pm.quantize(pos), mass, h)
    _check(rho, cnt, ref, rcnt, 2e-5)


def test_invalid_arguments(ctx):
    pos, mass, prm = gi.config("uniform-32k", n=500)
    t = og.Tree(ctx, pos, mass, prm)
    for bad in (0.0, -0.1, np.nan, np.inf, 0.5, 0.7):
        h = np.full(500, 0.05, np.float32)
        h[123] = bad
        with pytest.raises(og.OGError) as e:
            t.sph_density(h)
        assert e.value.status == og.OG_ERR_ARG
    rho, cnt = t.sph_density(np.full(500, 0.05, np.float32))   # the context is still usable
    assert cnt.min() >= 1
    t.refit(pos)
    with pytest.raises(og.OGError) as e:
        t.sph_density(np.full(500, 0.05, np.float32))
    assert e.value.status == og.OG_ERR_STATE


def test_device_pointers(ctx):
    torch = pytest.importorskip("torch")
    pos, mass, prm = gi.config("clustered-2m", n=30000)
    h = knn_h(pos, prm["box"])
    rh, ch = og.Tree(ctx, pos, mass, prm).sph_density(h)
    dev = og.Tree(ctx, torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(),
                  dict(prm, flags=og.OG_DEVICE_PTRS))
    rd = torch.zeros(len(mass), dtype=torch.float32, device="cuda")
    cd = torch.zeros(len(mass), dtype=torch.int32, device="cuda")
    og.og_tree_sph_density(dev.h, torch.from_numpy(h).cuda(), rd, cd)
    torch.cuda.synchronize()
    assert np.array_equal(rd.cpu().numpy(), rh) and np.array_equal(cd.cpu().numpy().view(np.uint32), ch)


def _neff_ok(pos, mass, box, h, n_target, tol, targets=None):
    """The paper's relation checked with the oracle's density at the given h."""
    rho, _ = sph.density(pm.quantize(pos, box), mass, h, box, targets=targets)
    t = np.arange(len(mass)) if targets is None else targets
    hh = h[t].astype(np.float64)
    neff = (4.0 * np.pi / 3.0) * hh ** 3 * rho / mass[t]
    return np.abs(neff - n_target) <= tol * n_target + 1e-3, neff


@pytest.mark.parametrize("start", ["above", "uniform"])
def test_smoothing_lengths_meet_the_neighbour_relation(ctx, start):
    pos, mass, prm = gi.config("clustered-2m", n=100000)
    if start == "above":
        h0 = np.minimum(2.0 * knn_h(pos, prm["box"]), 0.4)
    else:
        h0 = np.full(len(mass), prm["box"] * (3.0 * 32 / (4.0 * np.pi * len(mass))) ** (1.0 / 3.0))
    t = og.Tree(ctx, pos, mass, prm)
    h, rho, cnt, it = t.sph_smoothing(h0.astype(np.float32), 32.0, 0.01, 100)
    assert it < 100
    ok, neff = _neff_ok(pos, mass, prm["box"], h, 32.0, 0.01)
    assert ok.all(), (np.count_nonzero(~ok), neff[~ok][:5])
    r2, c2 = t.sph_density(h)                       # the outputs are the density call's at that h
    assert np.array_equal(r2, rho) and np.array_equal(c2, cnt)


def test_smoothing_full_size_workload(ctx):
    pos, mass, prm = gi.config("clustered-2m")
    h0 = np.full(len(mass), (3.0 * 32 / (4.0 * np.pi * len(mass))) ** (1.0 / 3.0), np.float32)
    t = og.Tree(ctx, pos, mass, prm)
    h, rho, cnt, it = t.sph_smoothing(h0, 32.0, 0.01, 200)
    assert it < 200
    sample = np.random.default_rng(4).choice(len(mass), 100000, replace=False)
    ok, _ = _neff_ok(pos, mass, prm["box"], h, 32.0, 0.01, targets=sample)
    assert ok.all()


def test_smoothing_invalid_arguments(ctx):
    pos, mass, prm = gi.config("uniform-32k", n=500)
    t = og.Tree(ctx, pos, mass, prm)
    h0 = np.full(500, 0.05, np.float32)
    for n_t, tol, mi in ((10.0, 0.01, 50), (32.0, 0.0, 50), (32.0, 1.0, 50), (32.0, 0.01, 0), (np.nan, 0.01, 5)):
        with pytest.raises(og.OGError) as e:
            t.sph_smoothing(h0, n_t, tol, mi)
        assert e.value.status == og.OG_ERR_ARG
    bad = h0.copy()
    bad[7] = -1.0
    with pytest.raises(og.OGError):
        t.sph_smoothing(bad)

"""og_tree_pm_force: the long-range particle-mesh force (Sect. 4.2 "Particle Mesh")
against the oracle (oracle/pm.py) on the same u32 positions and masses.

The CUDA path computes in FP32: CIC weights and masses in FP32, the assignment
summed as 64-bit fixed-point integers, cuFFT in FP32, the Green's factor from
an FP32 table, the gradient and interpolation in FP32.  Running the oracle's
steps with an FP32 mesh and FFT gives an error of at most 5e-6 of the rms
acceleration (4e-7 rms) on these workloads, so the bar is 1e-4 of the rms
acceleration for every particle and 1e-5 for the rms error.  The fixed-point
assignment makes the result independent of the order of the additions: two
calls give the same bits.
"""
from __future__ import annotations

import numpy as np
import pytest

import og_inputs as gi
from oracle import pm
from paper_2609_17658_gb300 import build as B
from paper_2609_17658_gb300 import og

pytestmark = pytest.mark.gpu

TOL_MAX = 1e-4
TOL_RMS = 1e-5


@pytest.fixture(scope="module")
def ctx():
    B.build()
    c = og.Context(0)
    yield c
    c.close()


def _check(acc, ref):
    rms = np.sqrt((ref.astype(np.float64) ** 2).sum(axis=1).mean())
    err = np.linalg.norm(acc.astype(np.float64) - ref, axis=1)
    assert np.isfinite(acc).all()
    assert err.max() <= TOL_MAX * rms, (err.max() / rms)
    assert np.sqrt((err ** 2).mean()) <= TOL_RMS * rms, (np.sqrt((err ** 2).mean()) / rms)


@pytest.mark.parametrize("name,n,mesh", [("uniform-32k", None, 32), ("uniform-32k", 5000, 64),
                                         ("clustered-2m", 100000, 128), ("clustered-2m", 30001, 16)])
def test_matches_the_oracle(ctx, name, n, mesh):
    pos, mass, prm = gi.config(name, n=n) if n else gi.config(name)
    t = og.Tree(ctx, pos, mass, prm)
    acc = t.pm_force(mesh)
    ref = pm.pm_accel(pm.quantize(pos, prm["box"]), mass, mesh, prm["box"], prm["G"], prm["r_s"])
    _check(acc, ref)
    assert np.array_equal(t.pm_force(mesh), acc)          # the same bits again


def test_full_size_workload(ctx):
    # 2.1M clustered particles on the 256^3 mesh of r_s = 1.25 mesh cells: every particle
    pos, mass, prm = gi.config("clustered-2m")
    t = og.Tree(ctx, pos, mass, prm)
    acc = t.pm_force(256)
    assert t.info()["ms_pm"] > 0
    ref = pm.pm_accel(pm.quantize(pos, prm["box"]), mass, 256, prm["box"], prm["G"], prm["r_s"])
    _check(acc, ref)
    p = (mass[:, None] * acc.astype(np.float64)).sum(axis=0)
    assert np.abs(p).max() < 1e-5 * (mass[:, None] * np.abs(acc)).sum()


def test_edge_cases(ctx):
    pos, mass, prm = gi.config("uniform-32k", n=1)
    one = og.Tree(ctx, pos, mass, prm).pm_force(32)
    assert np.abs(one).max() <= 1e-6 * mass[0] / prm["r_s"] ** 2           # no self-force
    # a lattice that fills the mesh feels nothing
    g = (np.arange(16) + 0.3) / 16.0
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    lat = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    m = np.full(lat.shape[0], 1.0 / lat.shape[0])
    a = og.Tree(ctx, lat, m, prm).pm_force(16)
    assert np.abs(a).max() <= 1e-5 * m[0] / prm["r_s"] ** 2
    # zero mass: zero force
    pos, mass, prm = gi.config("uniform-32k", n=3000)
    assert not og.Tree(ctx, pos, np.zeros_like(mass), prm).pm_force(32).any()
    # a non-unit box and G
    prm2 = dict(prm, box=2.5, G=3.0, r_s=2.0 * prm["r_s"])
    p2 = pos * 2.5
    acc = og.Tree(ctx, p2, mass, prm2).pm_force(64)
    ref = pm.pm_accel(pm.quantize(p2, 2.5), mass, 64, 2.5, 3.0, prm2["r_s"])
    _check(acc, ref)


def test_tree_plus_mesh_is_the_periodic_force(ctx):
    # the library's short-range tree force (theta = 0) plus its mesh force against the exact
    # periodic force (an Ewald sum with another split scale): the same bar as the oracle's
    from tests.test_oracle_pm import ewald_accel, treepm_case
    pos, mass, prm, x = treepm_case()
    t = og.Tree(ctx, pos, mass, prm)
    short, _, _ = t.force(counts=False)
    long_ = t.pm_force(32)
    ew = ewald_accel(x, mass, 1.0, 0.6 * prm["r_s"])
    rms = np.sqrt((ew ** 2).sum(axis=1).mean())
    e = np.linalg.norm(short.astype(np.float64) + long_ - ew, axis=1)
    assert e.max() < 3e-3 * rms and np.sqrt((e ** 2).mean()) < 1.2e-3 * rms, e.max() / rms


def test_invalid_arguments(ctx):
    pos, mass, prm = gi.config("uniform-32k", n=500)
    t = og.Tree(ctx, pos, mass, prm)
    for bad in (0, 1, 3, 48, 2048, -64):
        with pytest.raises(og.OGError) as e:
            t.pm_force(bad)
        assert e.value.status == og.OG_ERR_ARG
    t0 = og.Tree(ctx, pos, mass, dict(prm, r_s=0.0))
    with pytest.raises(og.OGError) as e:
        t0.pm_force(32)
    assert e.value.status == og.OG_ERR_ARG


def test_device_pointers(ctx):
    torch = pytest.importorskip("torch")
    pos, mass, prm = gi.config("clustered-2m", n=40000)
    ah = og.Tree(ctx, pos, mass, prm).pm_force(64)
    dev = og.Tree(ctx, torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda(),
                  dict(prm, flags=og.OG_DEVICE_PTRS))
    ad = torch.zeros((len(mass), 3), dtype=torch.float32, device="cuda")
    og.og_tree_pm_force(dev.h, 64, ad)
    torch.cuda.synchronize()
    assert np.array_equal(ad.cpu().numpy(), ah)

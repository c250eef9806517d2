"""The pair force law of the CUDA walk, one separation at a time.

Each box of one og_batch_force call holds two particles of unequal mass at a
chosen separation r, so each particle's acceleration is a single PP term:
G m_j g(r) S(r) (x_j - x_i), with g the spline-softened Newtonian factor
(Sect. 4.1.3) and S the short-range split factor of the erfc potential
(Sect. 4.2).  The separations run from far inside the softening length through
the spline's two branches and the Newtonian range up to just below the cutoff.
The expected values take the exact separation of the two fixed-point positions
and the oracle's FP64 g and S (both pinned on the CPU against quadrature and
the derivative of the potential).

The kernel evaluates the law in FP32 with its own erfc (Abramowitz and
Stegun 7.1.26, absolute error <= 1.5e-7).  Near the cutoff S is about 0.018,
so the erfc error alone is up to 8.5e-6 relative; FP32 rounding of the
spline's cancelling terms adds a few 1e-6.  The test holds every pair to
2e-5 relative.
"""
from __future__ import annotations

import numpy as np
import pytest

import og_inputs as gi
import oracle
from paper_2609_17658_gb300 import build as B
from paper_2609_17658_gb300 import og

pytestmark = pytest.mark.gpu

MAX_REL = 2e-5


@pytest.fixture(scope="module")
def ctx():
    B.build()
    oracle.build()
    c = og.Context(0)
    yield c
    c.close()


def _separations(h, rcut):
    r = np.concatenate([np.geomspace(1e-4 * h, rcut, 240, endpoint=False),
                        np.linspace(0.45 * h, 0.55 * h, 21), np.linspace(0.95 * h, 1.05 * h, 21)])
    return np.sort(r)


@pytest.mark.parametrize("box", [1.0, 3.0])
def test_pair_law_across_all_regimes(ctx, box):
    prm = gi.default_params(eps=box / 1600, r_s=box * 1.25 / 64, opening=gi.OPEN_BH, theta=0.5,
                            box=box)
    h = 2.8 * prm["eps"]
    rcut = prm["rcut_over_rs"] * prm["r_s"]
    rng = np.random.default_rng(21)
    seps = _separations(h, rcut)
    descs, expect = [], []
    for r in seps:
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        x0 = rng.uniform(0, box, size=3)
        x1 = np.mod(x0 + r * u, box)
        pos = np.stack([x0, x1])
        mass = np.array([0.375, 0.625]) / 1000.0
        q = np.array([[oracle.quantize1(v, box) for v in p] for p in pos], dtype=np.int64)
        d = ((q[1] - q[0] + 2 ** 31) % 2 ** 32 - 2 ** 31) * (box / 2 ** 32)   # exact FP64
        rr = float(np.sqrt(d @ d))
        # the in/out decision of the cutoff is taken in FP32 on both sides;
        # keep the sweep clear of the step
        if abs(rr - rcut) < 1e-6 * rcut:
            continue
        f = prm["G"] * oracle.soft_g(rr, h) * oracle.split_s(rr, prm["r_s"]) if rr < rcut else 0.0
        expect.append(np.stack([mass[1] * f * d, -mass[0] * f * d]))
        descs.append(dict(pos=pos, mass=mass, params=prm, acc=np.zeros((2, 3), np.float32),
                          n_pp=np.zeros(2, np.uint32), n_pn=np.zeros(2, np.uint32)))
    og.og_batch_force(ctx.h, descs)
    worst = 0.0
    for d, e in zip(descs, expect):
        assert np.array_equal(d["n_pp"], [1, 1]) and np.array_equal(d["n_pn"], [0, 0])
        ne = np.linalg.norm(e, axis=1)
        if ne[0] == 0.0:
            assert np.array_equal(d["acc"], np.zeros((2, 3), np.float32))
            continue
        rel = np.linalg.norm(d["acc"].astype(np.float64) - e, axis=1) / ne
        worst = max(worst, float(rel.max()))
    print(f"pair law, box {box}: worst relative error {worst:.3e} over {len(descs)} separations")
    assert worst <= MAX_REL

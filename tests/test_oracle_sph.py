"""Pins of the SPH density oracle (oracle/sph.py), independent of its code.

Sect. 6: rho_i = sum_j m_j W(|x_i - x_j|, h_i) with the cubic spline of
Monaghan (1985).  The references: all pairs by brute force (no k-d tree), the
kernel's normalisation 4 pi int_0^h r^2 W dr = 1 and its continuity by
quadrature, one and two particles in closed form, and a periodic lattice, whose
estimate is the mean density within the kernel's sampling error.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import pm, sph


def w_ref(q):
    """The cubic spline shape, written out from Monaghan's form: 1 - 6q^2 + 6q^3
    below 1/2, 2 (1 - q)^3 up to 1."""
    out = []
    for v in np.atleast_1d(q):
        if v < 0.5:
            out.append(1.0 - 6.0 * v * v + 6.0 * v * v * v)
        elif v < 1.0:
            out.append(2.0 * (1.0 - v) ** 3)
        else:
            out.append(0.0)
    return np.array(out)


def brute(q, mass, h, box):
    n = len(mass)
    hg = (np.asarray(h, np.float64) * (4294967296.0 / box)).astype(np.float32)
    rho = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    for i in range(n):
        d = (q.astype(np.int64) - np.int64(q[i].astype(np.int64)))      # x_j - x_i, all j
        d = (d + (1 << 31)) % (1 << 32) - (1 << 31)
        f = d.astype(np.float32)
        r2 = (f[:, 0] * f[:, 0] + f[:, 1] * f[:, 1]) + f[:, 2] * f[:, 2]
        nb = r2 < hg[i] * hg[i]
        hp = float(hg[i]) * box / 4294967296.0
        r = np.sqrt((d[nb].astype(np.float64) ** 2).sum(axis=1)) * box / 4294967296.0
        rho[i] = (mass[nb] * w_ref(r / hp)).sum() * 8.0 / (math.pi * hp ** 3)
        cnt[i] = nb.sum()
    return rho, cnt


@pytest.mark.parametrize("box", [1.0, 2.5])
def test_matches_brute_force(box):
    rng = np.random.default_rng(8)
    n = 400
    pos = rng.uniform(0, box, (n, 3))
    pos[:50] = rng.uniform(0, 0.02 * box, (50, 3))                   # a dense clump at the corner
    mass = rng.uniform(0.5, 1.5, n) / n
    h = (rng.uniform(0.03, 0.2, n) * box).astype(np.float32)
    q = pm.quantize(pos, box)
    rho, cnt = sph.density(q, mass, h, box)
    rb, cb = brute(q, mass, h, box)
    assert np.array_equal(cnt, cb)
    assert np.allclose(rho, rb, rtol=1e-12, atol=0)
    t = np.array([3, 17, 250])
    r3, c3 = sph.density(q, mass, h, box, targets=t)
    assert np.array_equal(c3, cb[t]) and np.allclose(r3, rb[t], rtol=1e-12, atol=0)


def test_kernel_normalisation_and_continuity():
    from scipy.integrate import quad
    h = 0.37
    I, _ = quad(lambda r: 4.0 * math.pi * r * r * 8.0 / (math.pi * h ** 3) * float(sph.kernel_w(r / h)),
                0.0, h, points=[0.5 * h], epsabs=1e-14)
    assert abs(I - 1.0) < 1e-12
    for q0 in (0.5, 1.0):
        assert abs(float(sph.kernel_w(q0 - 1e-12)) - float(sph.kernel_w(q0 + 1e-12))) < 1e-10
    qs = np.linspace(0, 1.2, 97)
    assert np.allclose(sph.kernel_w(qs), w_ref(qs), rtol=0, atol=1e-15)


def test_one_and_two_particles():
    q = pm.quantize(np.array([[0.3, 0.4, 0.5]]))
    h = np.array([0.125], np.float32)                                # exact in every format
    rho, cnt = sph.density(q, [2.0], h)
    assert cnt[0] == 1 and rho[0] == pytest.approx(8.0 * 2.0 / (math.pi * 0.125 ** 3), rel=1e-15)
    # separation 0.3 h along x: q = 0.3 for both, each counts the other
    pos = np.array([[0.5, 0.5, 0.5], [0.5 + 0.3 * 0.125, 0.5, 0.5]])
    q = pm.quantize(pos)
    rho, cnt = sph.density(q, [1.0, 3.0], np.array([0.125, 0.125], np.float32))
    wq = 1.0 - 6.0 * 0.09 + 6.0 * 0.027
    c = 8.0 / (math.pi * 0.125 ** 3)
    assert list(cnt) == [2, 2]
    assert rho[0] == pytest.approx(c * (1.0 + 3.0 * wq), rel=1e-8)
    assert rho[1] == pytest.approx(c * (3.0 + 1.0 * wq), rel=1e-8)
    # at exactly r = h the kernel is zero and the particle is not a neighbour (strict r < h);
    # 32 grid units less (the float32 spacing at 2^29 units) and it is one
    pos = np.array([[0.25, 0.5, 0.5], [0.375, 0.5, 0.5], [0.25, 0.5, 0.375 + 2.0 ** -27]])
    rho, cnt = sph.density(pm.quantize(pos), [1.0, 1.0, 1.0], np.full(3, 0.125, np.float32))
    assert list(cnt) == [2, 1, 2]


def test_periodic_lattice_gives_the_mean_density():
    n = 16
    g = (np.arange(n) + 0.5) / n
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    mass = np.full(n ** 3, 1.0 / n ** 3)
    h = np.full(n ** 3, 2.6 / n, np.float32)
    q = pm.quantize(pos)
    rho, cnt = sph.density(q, mass, h)
    assert np.all(cnt == cnt[0]) and np.allclose(rho, rho[0], rtol=1e-12)   # every site alike
    assert abs(rho[0] - 1.0) < 0.02                                        # the mean density
    # shifting everything by half the box (through the periodic boundary) changes nothing
    q2 = (q.astype(np.uint64) + np.uint64(1 << 31)).astype(np.uint32)
    r2, c2 = sph.density(q2, mass, h)
    assert np.array_equal(c2, cnt) and np.array_equal(r2, rho)

"""Pins of the particle-mesh oracle (oracle/pm.py), independent of its code.

Sect. 4.2 "Particle Mesh": the mesh carries the erf part of the split potential,
filtered by exp(-k^2 r_s^2).  The references here do not use the oracle's mesh:

  - the exact long-range force of point masses in a periodic box, as the
    direct Fourier series a(x) = -(4 pi G / L^3) sum_j m_j sum_{k != 0}
    k / k^2 exp(-k^2 r_s^2) sin(k . (x - x_j)), which the mesh approximates;
  - Newton's law plus the uniform-background term at separations far above r_s,
    where the erf part is the whole force;
  - conservation laws of cloud-in-cell with an antisymmetric gradient and an
    even Green's function: zero self-force, zero total momentum change, mass
    conservation of the assignment, zero force on a lattice that fills the mesh;
  - the whole TreePM split: the tree's short-range sum plus the mesh equals the
    exact periodic Newtonian force, an Ewald sum with a different split scale
    (Ewald sums do not depend on it), so a mismatch between the erfc of the
    tree and the exp(-k^2 r_s^2) of the mesh shows.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from oracle import pm


def fourier_series_accel(x, m, targets, box, G, r_s):
    """Exact filtered long-range acceleration by direct summation over modes."""
    nmax = int(math.ceil(math.sqrt(40.0) / r_s * box / (2.0 * math.pi)))   # exp(-k^2 r_s^2) < 5e-18
    n = np.arange(-nmax, nmax + 1)
    k1 = 2.0 * math.pi * n / box
    KX, KY, KZ = np.meshgrid(k1, k1, k1, indexing="ij")
    K2 = KX * KX + KY * KY + KZ * KZ
    sel = K2 > 0
    kv = np.stack([KX[sel], KY[sel], KZ[sel]], axis=1)
    w = np.exp(-K2[sel] * r_s * r_s) / K2[sel]
    out = np.zeros((len(targets), 3))
    for a, i in enumerate(targets):
        for j in range(len(x)):
            s = np.sin(kv @ (x[i] - x[j]))
            out[a] -= (4.0 * math.pi * G / box ** 3) * m[j] * ((w * s)[:, None] * kv).sum(axis=0)
    return out


def ewald_accel(x, m, G, r_e):
    """Exact periodic Newtonian acceleration in the unit box by Ewald summation with
    the split scale r_e: real-space images within one box plus the Fourier series."""
    from scipy.special import erfc
    al = 1.0 / (2.0 * r_e)
    d0 = x[:, None, :] - x[None, :, :]
    d0 -= np.round(d0)
    a = np.zeros_like(x)
    for img in np.ndindex(3, 3, 3):
        d = d0 + (np.array(img) - 1.0)
        r = np.linalg.norm(d, axis=2)
        self_ = img == (1, 1, 1)
        if self_:
            np.fill_diagonal(r, 1.0)
        f = (erfc(al * r) + 2.0 * al * r / math.sqrt(math.pi) * np.exp(-al * al * r * r)) / r ** 3
        if self_:
            np.fill_diagonal(f, 0.0)
        a -= G * (m[None, :, None] * f[:, :, None] * d).sum(axis=1)
    nmax = int(math.ceil(math.sqrt(40.0) / r_e / (2.0 * math.pi)))
    k1 = 2.0 * math.pi * np.arange(-nmax, nmax + 1)
    KX, KY, KZ = np.meshgrid(k1, k1, k1, indexing="ij")
    K2 = KX * KX + KY * KY + KZ * KZ
    sel = K2 > 0
    kv = np.stack([KX[sel], KY[sel], KZ[sel]], axis=1)
    w = np.exp(-K2[sel] * r_e * r_e) / K2[sel]
    ph = x @ kv.T
    c = (m[:, None] * np.cos(ph)).sum(axis=0)
    s = (m[:, None] * np.sin(ph)).sum(axis=0)
    a -= 4.0 * math.pi * G * ((w * (np.sin(ph) * c - np.cos(ph) * s)) @ kv)   # sum_j m_j sin(k.(x_i - x_j))
    return a


def treepm_case():
    """300 random particles in the unit box, a 32^3 mesh, r_s = 3 mesh cells."""
    rng = np.random.default_rng(4)
    pos = rng.uniform(0, 1, (300, 3))
    mass = rng.uniform(0.5, 1.5, 300) / 300
    prm = dict(box=1.0, G=1.0, eps=1e-7, r_s=3.0 / 32, rcut_over_rs=4.5, opening=0, theta=0.0,
               alpha=0.005, theta_first_pass=0.5, leaf_max=1, group_max=32, flags=0)
    x = pm.quantize(pos).astype(np.float64) / 2.0 ** 32
    return pos, mass, prm, x


def test_tree_plus_mesh_is_the_periodic_force():
    pos, mass, prm, x = treepm_case()
    ew = ewald_accel(x, mass, 1.0, 0.6 * prm["r_s"])
    assert np.abs(ew - ewald_accel(x, mass, 1.0, 1.3 * prm["r_s"])).max() < 1e-12 * np.abs(ew).max()
    short = oracle.direct(pos, mass, prm)                       # the tree at theta = 0
    rms = np.sqrt((ew ** 2).sum(axis=1).mean())
    for r_s_mesh, ok in ((prm["r_s"], True), (2.0 * prm["r_s"], False)):
        long_ = pm.pm_accel(pm.quantize(pos), mass, 32, 1.0, 1.0, r_s_mesh)
        e = np.linalg.norm(short + long_ - ew, axis=1)
        fits = e.max() < 3e-3 * rms and np.sqrt((e ** 2).mean()) < 1.2e-3 * rms
        assert fits == ok, (r_s_mesh, e.max() / rms)


def _pairs(rng, mesh, box, seps_cells, per_sep):
    for sep in seps_cells:
        for _ in range(per_sep):
            x0 = rng.uniform(0, box, 3)
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            yield np.mod(np.stack([x0, x0 + u * sep * box / mesh]), box)


@pytest.mark.parametrize("rs_cells,tol_max,tol_mean", [(3.0, 1.5e-2, 6e-3), (1.25, 8e-2, 3e-2)])
def test_pairs_match_the_exact_fourier_series(rs_cells, tol_max, tol_mean):
    mesh, box, G = 32, 1.0, 1.0
    r_s = rs_cells * box / mesh
    rng = np.random.default_rng(7)
    errs = []
    for pos in _pairs(rng, mesh, box, (0.5, 1, 2, 3, 5, 8), 4):
        q = pm.quantize(pos, box)
        x = q.astype(np.float64) * (box / 2.0 ** 32)
        m = np.array([1.0, 0.5])
        a = pm.pm_accel(q, m, mesh, box, G, r_s)
        ex = fourier_series_accel(x, m, [0, 1], box, G, r_s)
        errs.append(np.linalg.norm(a - ex, axis=1).max() / np.linalg.norm(ex, axis=1).max())
    assert max(errs) < tol_max and np.mean(errs) < tol_mean, (max(errs), np.mean(errs))


def test_far_field_is_newton_plus_background():
    # r = 0.15 L, r_s = 1.5 cells of a 128 mesh: the short-range factor S(r) is below 1e-9, so
    # the mesh force is the whole periodic force; for r << L that is -G m r_hat / r^2 +
    # (4 pi / 3) G m r / L^3 (the removed mean density repels; 1.4 % of Newton here), up to
    # image terms of relative order (r / L)^5 (7e-4 here)
    mesh, box, G, r_s = 128, 1.0, 1.0, 1.5 / 128
    rng = np.random.default_rng(11)
    worst = 0.0
    for _ in range(6):
        x0 = rng.uniform(0, 1, 3)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        pos = np.mod(np.stack([x0, x0 + 0.15 * u]), 1.0)
        q = pm.quantize(pos)
        d = (q[0].astype(np.int64) - q[1].astype(np.int64))
        d = ((d + (1 << 31)) % (1 << 32) - (1 << 31)) / 2.0 ** 32    # x_0 - x_1, minimum image
        r = np.linalg.norm(d)
        m1 = 0.75
        a = pm.pm_accel(q, np.array([0.0, m1]), mesh, box, G, r_s)[0]   # force of 1 on 0
        newton = -G * m1 * d / r ** 3
        background = (4.0 * math.pi / 3.0) * G * m1 * d
        worst = max(worst, np.linalg.norm(a - (newton + background)) / np.linalg.norm(newton))
        assert np.linalg.norm(a - newton) / np.linalg.norm(newton) > 8e-3   # the background shows
    assert worst < 4e-3, worst


def test_assignment_conserves_mass():
    rng = np.random.default_rng(3)
    pos = rng.uniform(0, 1, (500, 3))
    m = rng.uniform(0.5, 2.0, 500)
    for mesh in (8, 32):
        rho = pm.deposit(pm.quantize(pos), m, mesh)
        assert abs(rho.sum() / mesh ** 3 - m.sum()) < 1e-12 * m.sum()
    # on a mesh point all mass goes to that point; at a cell centre 1/8 to each corner
    q = np.array([[3 << 27, 5 << 27, 7 << 27]], dtype=np.uint32)      # mesh 32: points (3, 5, 7)
    rho = pm.deposit(q, [2.0], 32) / 32 ** 3
    assert rho[3, 5, 7] == 2.0 and np.count_nonzero(rho) == 1
    q = q + np.uint32(1 << 26)                                         # half a cell on every axis
    rho = pm.deposit(q, [2.0], 32) / 32 ** 3
    assert np.count_nonzero(rho) == 8 and np.all(rho[3:5, 5:7, 7:9] == 0.25)


def test_no_self_force_and_momentum_is_conserved():
    rng = np.random.default_rng(5)
    mesh, r_s = 32, 1.25 / 32
    q = pm.quantize(rng.uniform(0, 1, (1, 3)))
    a1 = pm.pm_accel(q, [1.0], mesh, 1.0, 1.0, r_s)
    scale = 1.0 / r_s ** 2
    assert np.abs(a1).max() < 1e-12 * scale
    pos = rng.uniform(0, 1, (300, 3))
    m = rng.uniform(0.5, 2.0, 300)
    a = pm.pm_accel(pm.quantize(pos), m, mesh, 1.0, 1.0, r_s)
    p = (m[:, None] * a).sum(axis=0)
    assert np.abs(p).max() < 1e-12 * (m[:, None] * np.abs(a)).sum()


def test_a_lattice_that_fills_the_mesh_feels_nothing():
    mesh, r_s = 16, 2.0 / 16
    g = np.arange(mesh, dtype=np.uint64) << np.uint64(28)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    for shift in (0, 12345678):                          # any common offset keeps the density flat
        q = (np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1) + np.uint64(shift)).astype(np.uint32)
        a = pm.pm_accel(q, np.ones(q.shape[0]), mesh, 1.0, 1.0, r_s)
        assert np.abs(a).max() < 1e-10


def test_axis_permutation_permutes_the_force():
    rng = np.random.default_rng(9)
    pos = rng.uniform(0, 1, (40, 3))
    m = rng.uniform(0.5, 2.0, 40)
    q = pm.quantize(pos)
    a = pm.pm_accel(q, m, 16, 1.0, 1.0, 1.5 / 16)
    for perm in ((1, 2, 0), (2, 0, 1), (0, 2, 1)):
        b = pm.pm_accel(q[:, perm], m, 16, 1.0, 1.0, 1.5 / 16)
        assert np.allclose(b, a[:, perm], rtol=0, atol=1e-12 * np.abs(a).max())


def test_quantize_is_the_tree_fixed_point():
    rng = np.random.default_rng(2)
    for box in (1.0, 0.7, 3.0):
        v = np.concatenate([rng.uniform(-0.5, 1.5, 200) * box, [0.0, -0.0, box, -box, 1e-300, -1e-300]])
        got = pm.quantize(v, box)
        ref = np.array([oracle.quantize1(float(x), box) for x in v], dtype=np.uint32)
        assert np.array_equal(got, ref)


def test_mesh_size_is_checked():
    for bad in (1, 12, 2048):
        with pytest.raises(ValueError):
            pm.cic_weights(np.zeros((1, 3), np.uint32), bad)

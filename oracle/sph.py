"""SPH density at given smoothing lengths -- TEST INFRASTRUCTURE (the oracle of
og_tree_sph_density; only the tests, the smoke check and the benchmark's CPU
leg use it).

What it computes (Sect. 6 "Smoothed Particle Hydrodynamics" and Sect. 3.4
"Neighbour search"): the kernel-averaged density of every particle,

    rho_i = sum_j m_j W(|x_i - x_j|, h_i),

over all particles j (itself included) closer than h_i, with the cubic spline
of Monaghan (1985), the paper's default kernel for 3D with 32 neighbours
(Table of Sect. 6.5; the expression of the kernel appendix):

    W(r, h) = 8 / (pi h^3) * { 1 - 6 q^2 + 6 q^3   for q = r / h < 1/2,
                               2 (1 - q)^3         for 1/2 <= q < 1,
                               0                   for q >= 1 }.

Readings of the points the paper leaves open:

  S-1 positions are the tree's u32 grid coordinates; separations are the exact
      minimum-image integers (int32 of the u32 difference).
  S-2 who is a neighbour: j counts for i iff r2 < h2 in single precision, with
      r2 = ((fx * fx) + (fy * fy)) + (fz * fz), f = float32 of the integer
      separation, each operation rounded to float32, and h2 = hg * hg in
      float32, hg = float32(h * (2^32 / L)) (the product in float64).  The
      neighbour count n_i includes i itself.  This decision is an integer, so
      the CUDA path takes it in the same arithmetic.
  S-3 the density sums in float64 (r from the float64 of the integer separations).

The candidates come from scipy's periodic k-d tree (a library primitive: all
points within a radius slightly above h); the rule above then decides.

Parity pins (tests/test_oracle_sph.py): brute force over all pairs, the
kernel's normalisation and continuity by quadrature, a single particle, two
particles, and a periodic lattice whose estimate is the mean density.
"""
from __future__ import annotations

import math

import numpy as np


def kernel_w(q):
    """Cubic spline shape w(q) (W = 8 / (pi h^3) w(r / h)), float64."""
    q = np.asarray(q, dtype=np.float64)
    return np.where(q < 0.5, 1.0 - 6.0 * q * q + 6.0 * q ** 3,
                    np.where(q < 1.0, 2.0 * (1.0 - q) ** 3, 0.0))


def grid_h(h, box: float) -> np.ndarray:
    """Smoothing lengths in grid units, float32 (S-2)."""
    return (np.asarray(h, dtype=np.float64) * (4294967296.0 / box)).astype(np.float32)


def separations(qi, qj) -> np.ndarray:
    """Minimum-image integer separations x_j - x_i (S-1), int64 [..., 3]."""
    d = np.asarray(qj, dtype=np.int64) - np.asarray(qi, dtype=np.int64)
    return (d + (1 << 31)) % (1 << 32) - (1 << 31)


def is_neighbour(d, hg) -> np.ndarray:
    """The single-precision neighbour decision of S-2."""
    f = d.astype(np.float32)
    r2 = (f[..., 0] * f[..., 0] + f[..., 1] * f[..., 1]) + f[..., 2] * f[..., 2]
    hg = np.asarray(hg, dtype=np.float32)
    return r2 < hg * hg


def density(q, mass, h, box: float = 1.0, targets=None, workers: int = -1, batch: int = 65536):
    """(rho float64, n_ngb int64) of the targets (all particles by default) at the
    smoothing lengths h (float32 [n], per particle)."""
    from scipy.spatial import cKDTree
    q = np.asarray(q, dtype=np.uint32)
    mass = np.asarray(mass, dtype=np.float64)
    h = np.asarray(h, dtype=np.float32)
    tg = np.arange(q.shape[0]) if targets is None else np.asarray(targets, dtype=np.int64)
    hg = grid_h(h, box)
    hphys = hg.astype(np.float64) * (box / 4294967296.0)
    x = q.astype(np.float64) * (box / 4294967296.0)
    kd = cKDTree(x, boxsize=box)
    rho = np.zeros(len(tg))
    cnt = np.zeros(len(tg), dtype=np.int64)
    for b0 in range(0, len(tg), batch):
        ti = tg[b0:b0 + batch]
        cand = kd.query_ball_point(x[ti], r=h[ti].astype(np.float64) * (1.0 + 1e-5) + box * 2.0 ** -30,
                                   workers=workers)
        lens = np.array([len(c) for c in cand], dtype=np.int64)
        I = np.repeat(np.arange(len(ti)), lens)
        J = np.concatenate([np.asarray(c, dtype=np.int64) for c in cand]) if len(ti) else np.zeros(0, np.int64)
        d = separations(q[ti[I]], q[J])
        keep = is_neighbour(d, hg[ti[I]])
        I, J, d = I[keep], J[keep], d[keep]
        df = d.astype(np.float64)
        r = np.sqrt((df * df).sum(axis=1)) * (box / 4294967296.0)
        hi = hphys[ti[I]]
        contrib = mass[J] * kernel_w(r / hi) * 8.0 / (math.pi * hi ** 3)
        rho[b0:b0 + len(ti)] = np.bincount(I, weights=contrib, minlength=len(ti))
        cnt[b0:b0 + len(ti)] = np.bincount(I, minlength=len(ti))
    return rho, cnt

"""Long-range particle-mesh (PM) acceleration -- TEST INFRASTRUCTURE (the oracle
of og_tree_pm_force; only the tests, the smoke check and the benchmark's CPU
leg use it).

What it computes, in the order of the paper (Sect. 4.2 "Particle Mesh"): the
Newtonian potential is split as 1/r = erfc(r / 2 A_smth) / r + erf(r / 2 A_smth) / r
(A_smth = r_s); the tree takes the erfc part, the mesh the erf part.  The
particles are assigned to a mesh, the density is Fourier transformed, multiplied
by the Green's function of the Poisson equation with the Gaussian filter,

    phi_l(k) = -4 pi G rho(k) / k^2 * exp(-k^2 r_s^2),

and transformed back.  Readings of the points the paper leaves open:

  PM-1 mesh: Ng^3 points, Ng a power of two (2 .. 1024); point (i, j, l) sits at
       (i, j, l) * D, D = L / Ng.  Positions are the tree's u32 grid coordinates,
       so a particle's mesh coordinate x_int / 2^(32 - log2 Ng) is exact.
  PM-2 assignment: cloud-in-cell (CIC).  With u = x / D, i0 = floor(u) and
       f = u - i0, the particle gives weight (1 - f) to point i0 and f to point
       i0 + 1 (periodic) on each axis, the product over the three axes in 3D.
       Density = sum of m * weight / D^3.
  PM-3 Green's function: the paper's filtered kernel, divided by the square of
       the CIC window W(k) = prod_a sinc^2(k_a D / 2), sinc(x) = sin(x) / x,
       once for the assignment and once for the interpolation (Hockney &
       Eastwood, "Computer Simulation Using Particles", ch. 5-8).  k = 2 pi n / L
       with the signed frequency index n; the k = 0 mode is zero (the mean
       density carries no force in a periodic box).
  PM-4 force on the mesh: a = -grad phi by the fourth-order central difference
       d phi / dx (i) = [8 (phi(i+1) - phi(i-1)) - (phi(i+2) - phi(i-2))] / (12 D).
  PM-5 interpolation: CIC with the weights of PM-2.

Parity pins (tests/test_oracle_pm.py): the exact filtered long-range force of
point masses in a periodic box as a direct Fourier series (the continuous
solution the mesh approximates), mass conservation of the assignment, zero
self-force and zero total momentum change (CIC with an antisymmetric gradient
and an even Green's function), zero force on a lattice that fills the mesh,
and Newton's law with the uniform-background term at separations far above r_s.
"""
from __future__ import annotations

import math

import numpy as np


def quantize(pos, box: float = 1.0) -> np.ndarray:
    """u32 grid coordinates floor(frac(x / L) * 2^32) of every position (the
    tree's fixed point, Sect. 4.1.1), for |x / L| < 2^31."""
    t = np.asarray(pos, dtype=np.float64) / box
    if not np.all(np.abs(t) < 2.0 ** 31):
        raise ValueError("positions too far outside the box")
    q = np.floor(t * 4294967296.0).astype(np.int64)
    return np.mod(q, 1 << 32).astype(np.uint32)


def _check_mesh(mesh: int) -> int:
    if mesh < 2 or mesh > 1024 or mesh & (mesh - 1):
        raise ValueError("mesh must be a power of two in [2, 1024]")
    return int(mesh).bit_length() - 1


def cic_weights(q: np.ndarray, mesh: int):
    """Mesh point i0 and fraction f of every coordinate (PM-1, PM-2)."""
    s = 32 - _check_mesh(mesh)
    q = np.asarray(q, dtype=np.uint64)
    i0 = (q >> np.uint64(s)).astype(np.int64)
    f = (q & np.uint64((1 << s) - 1)).astype(np.float64) * 2.0 ** -s
    return i0, f


def _corners(q, mesh):
    """The 8 CIC corners of every particle: flat mesh index and weight."""
    i0, f = cic_weights(q, mesh)
    out = []
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                ix = (i0[:, 0] + dx) % mesh
                iy = (i0[:, 1] + dy) % mesh
                iz = (i0[:, 2] + dz) % mesh
                w = ((f[:, 0] if dx else 1.0 - f[:, 0]) * (f[:, 1] if dy else 1.0 - f[:, 1])) * \
                    (f[:, 2] if dz else 1.0 - f[:, 2])
                out.append(((ix * mesh + iy) * mesh + iz, w))
    return out


def deposit(q, mass, mesh: int, box: float = 1.0) -> np.ndarray:
    """Density on the mesh (PM-2), float64 [Ng, Ng, Ng]."""
    mass = np.asarray(mass, dtype=np.float64)
    rho = np.zeros(mesh ** 3)
    for idx, w in _corners(q, mesh):
        rho += np.bincount(idx, weights=mass * w, minlength=mesh ** 3)
    d = box / mesh
    return rho.reshape(mesh, mesh, mesh) / (d * d * d)


def green(mesh: int, box: float, G: float, r_s: float) -> np.ndarray:
    """Filtered, CIC-deconvolved Green's function on the rfft half mesh (PM-3):
    phi(k) = green(k) * rho(k)."""
    _check_mesh(mesh)
    n_full = np.fft.fftfreq(mesh, d=1.0 / mesh)          # signed index n
    n_half = np.fft.rfftfreq(mesh, d=1.0 / mesh)
    kx = 2.0 * math.pi * n_full[:, None, None] / box
    ky = 2.0 * math.pi * n_full[None, :, None] / box
    kz = 2.0 * math.pi * n_half[None, None, :] / box
    k2 = kx * kx + ky * ky + kz * kz
    d = box / mesh

    def sinc(x):
        return np.where(x == 0.0, 1.0, np.sin(x) / np.where(x == 0.0, 1.0, x))

    W = (sinc(kx * d / 2) ** 2) * (sinc(ky * d / 2) ** 2) * (sinc(kz * d / 2) ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        g = -4.0 * math.pi * G * np.exp(-k2 * r_s * r_s) / k2 / (W * W)
    g[0, 0, 0] = 0.0
    return g


def potential_mesh(q, mass, mesh: int, box: float, G: float, r_s: float) -> np.ndarray:
    """Long-range potential on the mesh: FFT, Green's function, inverse FFT."""
    rho = deposit(q, mass, mesh, box)
    rk = np.fft.rfftn(rho)
    return np.fft.irfftn(rk * green(mesh, box, G, r_s), s=rho.shape, axes=(0, 1, 2))


def force_mesh(phi: np.ndarray, box: float) -> np.ndarray:
    """-grad phi on the mesh by the fourth-order difference (PM-4): [3, Ng, Ng, Ng]."""
    d = box / phi.shape[0]
    out = np.empty((3,) + phi.shape)
    for a in range(3):
        p1 = np.roll(phi, -1, axis=a)
        m1 = np.roll(phi, 1, axis=a)
        p2 = np.roll(phi, -2, axis=a)
        m2 = np.roll(phi, 2, axis=a)
        out[a] = -(8.0 * (p1 - m1) - (p2 - m2)) / (12.0 * d)
    return out


def interpolate(F: np.ndarray, q, mesh: int) -> np.ndarray:
    """CIC interpolation of the mesh force to the particles (PM-5): [n, 3]."""
    flat = F.reshape(3, -1)
    acc = np.zeros((np.asarray(q).shape[0], 3))
    for idx, w in _corners(q, mesh):
        acc += w[:, None] * flat[:, idx].T
    return acc


def pm_accel(q, mass, mesh: int, box: float = 1.0, G: float = 1.0, r_s: float = 0.0) -> np.ndarray:
    """Long-range acceleration of every particle, float64 [n, 3], from the u32
    grid coordinates q [n, 3] and the masses."""
    if not r_s > 0.0:
        raise ValueError("the mesh force needs r_s > 0")
    phi = potential_mesh(q, mass, mesh, box, G, r_s)
    return interpolate(force_mesh(phi, box), q, mesh)

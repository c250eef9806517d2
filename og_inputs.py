"""Seeded synthetic inputs shaped like the paper's gravity workloads.

This module makes particle sets and parameter records only.  It holds none of
the tree-force arithmetic, so both the FP64 oracle and the CUDA library may be
fed from it.  Every generator takes an explicit integer seed and uses numpy's
PCG64 bit generator, so a (generator, seed) pair always gives the same input
within one numpy version.

Workloads (units: box L = 1, G = 1, equal masses 1/N so that the total mass is 1):

* ``uniform``   Poisson-uniform positions in the periodic unit box.
* ``halo_mix``  a fraction of the particles uniform, the rest in NFW haloes
                (profile shape of the NFW potential in the paper's section on
                analytic static potentials), halo particle counts drawn from a
                power-law mass function, concentration 10, truncated at r_200.
* ``lattice``   an n^3 cubic lattice (zero net force by symmetry).
* ``sphere``    a uniform-density sphere (the paper's CI free-fall test checks
                its initial acceleration profile, Sect. 2.5).
* ``two_body``  two particles at a chosen separation.

``config(name)`` returns the particle set and parameter dictionary of the
named workload; ``batch_boxes`` and ``request_stream`` build the multi-box and
served-stream workloads.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Opening criteria (match og_open in include/og.h)
OPEN_BH = 0
OPEN_REL = 1


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def default_params(**kw) -> dict:
    """Parameter record with the library's defaults (box 1, G 1, BH theta 0.5)."""
    p = dict(box=1.0, G=1.0, eps=0.0, r_s=0.0, rcut_over_rs=4.5,
             opening=OPEN_BH, theta=0.5, alpha=0.005, theta_first_pass=0.5,
             leaf_max=1, group_max=32, flags=0)
    p.update(kw)
    return p


def uniform(n: int, seed: int, box: float = 1.0):
    """Poisson-uniform positions in [0, box)^3, masses 1/n."""
    r = _rng(seed)
    pos = r.random((n, 3)) * box
    mass = np.full(n, 1.0 / max(n, 1))
    return pos, mass


def lattice(n_side: int, box: float = 1.0, offset: float = 0.5):
    """Cubic lattice of n_side^3 particles at (i + offset) * box / n_side."""
    g = (np.arange(n_side, dtype=np.float64) + offset) * (box / n_side)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    n = pos.shape[0]
    return pos, np.full(n, 1.0 / n)


def sphere(n: int, seed: int, radius: float = 0.1, centre=(0.5, 0.5, 0.5)):
    """Uniform-density sphere: radius R * U^(1/3), isotropic directions."""
    r = _rng(seed)
    rad = radius * np.cbrt(r.random(n))
    dirs = _isotropic(r, n)
    pos = np.asarray(centre, dtype=np.float64) + dirs * rad[:, None]
    return pos, np.full(n, 1.0 / n)


def two_body(sep: float, axis: int = 0, centre=(0.5, 0.5, 0.5), m=(0.5, 0.5)):
    """Two particles separated by ``sep`` along ``axis`` about ``centre``."""
    pos = np.tile(np.asarray(centre, dtype=np.float64), (2, 1))
    pos[0, axis] -= sep / 2
    pos[1, axis] += sep / 2
    return pos, np.asarray(m, dtype=np.float64)


def _isotropic(r: np.random.Generator, n: int) -> np.ndarray:
    cos_t = 2.0 * r.random(n) - 1.0
    phi = 2.0 * math.pi * r.random(n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


def _nfw_mu(x):
    return np.log1p(x) - x / (1.0 + x)


def _nfw_radii(r: np.random.Generator, n: int, c: float) -> np.ndarray:
    """Radii in units of the scale radius, by inverting the enclosed-mass
    profile mu(x) = ln(1+x) - x/(1+x) on [0, c] with FP64 bisection."""
    target = r.random(n) * _nfw_mu(c)
    lo = np.zeros(n)
    hi = np.full(n, c)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        below = _nfw_mu(mid) < target
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi)


def _halo_counts(r: np.random.Generator, n_halo: int, total: int, slope: float,
                 n_min: int, n_max: int) -> np.ndarray:
    """Halo particle counts from dN/dn ~ n^slope on [n_min, n_max], rescaled so
    they sum to ``total`` exactly (largest-remainder rounding)."""
    a = slope + 1.0
    u = r.random(n_halo)
    raw = (n_min ** a + u * (n_max ** a - n_min ** a)) ** (1.0 / a)
    scaled = raw * (total / raw.sum())
    counts = np.floor(scaled).astype(np.int64)
    rem = total - int(counts.sum())
    if rem > 0:
        order = np.argsort(-(scaled - counts), kind="stable")
        counts[order[:rem]] += 1
    return counts


def halo_mix(n: int, seed: int, n_halo: int = 2000, f_halo: float = 0.7,
             slope: float = -1.9, conc: float = 10.0, box: float = 1.0,
             overdensity: float = 200.0, shuffle: bool = True):
    """Clustered set: ``f_halo`` of the particles in ``n_halo`` NFW haloes, the
    rest Poisson-uniform.  Halo h with n_h particles has mass n_h/n, radius
    r_200 = (3 M_h / (4 pi * 200 * rho_mean))^(1/3) with rho_mean = 1 (total
    mass 1 in a unit box), scale radius r_200 / conc, centre uniform; positions
    wrap periodically."""
    r = _rng(seed)
    n_in = int(round(f_halo * n))
    n_halo = max(1, min(n_halo, n_in // 32)) if n_in >= 32 else 0
    if n_halo == 0:
        n_in = 0
    n_out = n - n_in
    parts = []
    if n_out > 0:
        parts.append(r.random((n_out, 3)) * box)
    if n_in > 0:
        n_max = max(64, n // 20)
        counts = _halo_counts(r, n_halo, n_in, slope, 32, n_max)
        centres = r.random((n_halo, 3)) * box
        m_h = counts / float(n)
        r200 = np.cbrt(3.0 * m_h / (4.0 * math.pi * overdensity * 1.0)) * box
        rs = r200 / conc
        owner = np.repeat(np.arange(n_halo), counts)
        rad = _nfw_radii(r, n_in, conc) * rs[owner]
        dirs = _isotropic(r, n_in)
        parts.append(centres[owner] + dirs * rad[:, None])
    pos = np.concatenate(parts, axis=0)
    pos = np.mod(pos, box)
    pos[pos >= box] = 0.0
    if shuffle:
        pos = pos[r.permutation(n)]
    return pos, np.full(n, 1.0 / n)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

CONFIG_NAMES = ("uniform-32k", "clustered-2m", "clustered-16m")


def config(name: str, n: int | None = None, seed: int | None = None):
    """Return (pos, mass, params) for a named workload.

    uniform-32k:   N = 32^3 Poisson-uniform, eps = 1/(50*32), BH theta 0.5,
                   r_s = 1.25/64, cutoff 4.5 r_s.
    clustered-2m:  N = 128^3, 70 % in 2000 NFW haloes + 30 % uniform,
                   eps = 1/(50*128), relative opening alpha 0.005 after a BH
                   theta 0.5 first pass, r_s = 1.25/256.
    clustered-16m: N = 256^3, same generator, eps = 1/(50*256), alpha 0.0025,
                   r_s = 1.25/512.
    ``n`` overrides the particle count (the softening, split scale and cutoff
    stay those of the named workload), ``seed`` the seed.
    """
    if name == "uniform-32k":
        nn = 32 ** 3 if n is None else n
        pos, mass = uniform(nn, 12345 if seed is None else seed)
        prm = default_params(eps=1.0 / (50 * 32), r_s=1.25 / 64,
                             opening=OPEN_BH, theta=0.5)
    elif name == "clustered-2m":
        nn = 128 ** 3 if n is None else n
        pos, mass = halo_mix(nn, 12346 if seed is None else seed,
                             n_halo=max(1, int(round(2000 * nn / 128 ** 3))))
        prm = default_params(eps=1.0 / (50 * 128), r_s=1.25 / 256,
                             opening=OPEN_REL, alpha=0.005, theta_first_pass=0.5)
    elif name == "clustered-16m":
        nn = 256 ** 3 if n is None else n
        pos, mass = halo_mix(nn, 12347 if seed is None else seed,
                             n_halo=max(1, int(round(16000 * nn / 256 ** 3))))
        prm = default_params(eps=1.0 / (50 * 256), r_s=1.25 / 512,
                             opening=OPEN_REL, alpha=0.0025, theta_first_pass=0.5)
    else:
        raise KeyError(name)
    return pos, mass, prm


@dataclass
class Box:
    """One independent periodic box of the batched workload."""
    pos: np.ndarray
    mass: np.ndarray
    params: dict
    kind: str


def batch_boxes(n_boxes: int = 512, seed: int = 12348, n_lo: int = 4096,
                n_hi: int = 262144) -> list[Box]:
    """Independent boxes: N log-uniform in [n_lo, n_hi], each uniform or
    halo-clustered by a coin flip (halo count scaled with N);
    eps = 1/(50 N^(1/3)), r_s = 1.25/(2 N^(1/3)), BH theta 0.5."""
    r = _rng(seed)
    out = []
    for b in range(n_boxes):
        nb = int(round(math.exp(r.uniform(math.log(n_lo), math.log(n_hi)))))
        clustered = bool(r.random() < 0.5)
        s = int(r.integers(0, 2 ** 31))
        if clustered:
            pos, mass = halo_mix(nb, s, n_halo=max(1, int(round(2000 * nb / 128 ** 3))))
        else:
            pos, mass = uniform(nb, s)
        side = nb ** (1.0 / 3.0)
        prm = default_params(eps=1.0 / (50 * side), r_s=1.25 / (2 * side),
                             opening=OPEN_BH, theta=0.5)
        out.append(Box(pos, mass, prm, "halo" if clustered else "uniform"))
    return out


@dataclass
class Request:
    """One served request: a system integrated for ``nsteps`` kick-drift steps."""
    t_arrive: float
    pos: np.ndarray
    vel: np.ndarray
    mass: np.ndarray
    params: dict
    nsteps: int = 8
    dt_kick: float = 1e-5
    dt_drift: float = 1.0
    meta: dict = field(default_factory=dict)


def request_stream(rate_hz: float, duration_s: float, seed: int = 12349,
                   n_lo: int = 10_000, n_hi: int = 2_000_000,
                   sigma_v: float = 1e-3, max_requests: int | None = None) -> list[Request]:
    """Poisson arrivals at ``rate_hz`` over ``duration_s``; N log-uniform in
    [n_lo, n_hi]; halo-clustered systems; Gaussian velocities with sigma
    ``sigma_v`` box lengths per step."""
    r = _rng(seed)
    t = 0.0
    out = []
    while True:
        t += r.exponential(1.0 / rate_hz)
        if t > duration_s or (max_requests is not None and len(out) >= max_requests):
            break
        nb = int(round(math.exp(r.uniform(math.log(n_lo), math.log(n_hi)))))
        s = int(r.integers(0, 2 ** 31))
        pos, mass = halo_mix(nb, s, n_halo=max(1, int(round(2000 * nb / 128 ** 3))))
        vel = _rng(s + 1).normal(0.0, sigma_v, size=(nb, 3))
        side = nb ** (1.0 / 3.0)
        prm = default_params(eps=1.0 / (50 * side), r_s=1.25 / (2 * side),
                             opening=OPEN_BH, theta=0.5)
        out.append(Request(t, pos, vel, mass, prm))
    return out

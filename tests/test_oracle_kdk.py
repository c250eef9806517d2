"""Pins of the oracle's time integrator (oracle/kdk.py), independent of its code.

Individual power-of-two time steps with the acceleration criterion of Sect.
3.2 and a kick-drift-kick leapfrog: bins from a closed form at the exact
boundaries of the criterion, free drift, exact kinematics under a constant
acceleration, second-order convergence for a harmonic force, and particles in
different bins evolving as if alone.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import kdk


def test_bins_at_the_criterion_boundaries():
    # eps = 1, eta = 1/2: dt_crit = |a|^(-1/2); |a| = 4^b gives dt_crit = 2^-b
    eps, eta, dt_max, B = 1.0, 0.5, 1.0, 8
    a = np.array([[4.0 ** b, 0, 0] for b in range(6)], dtype=np.float32)
    assert list(kdk.bins_for(a, eps, eta, dt_max, B)) == [0, 1, 2, 3, 4, 5]   # equality accepts
    a_up = a * np.float32(1.0001)
    assert list(kdk.bins_for(a_up, eps, eta, dt_max, B)) == [1, 2, 3, 4, 5, 6]
    assert list(kdk.bins_for(np.zeros((2, 3), np.float32), eps, eta, dt_max, B)) == [0, 0]
    assert kdk.bins_for(np.array([[1e30, 0, 0]], np.float32), eps, eta, dt_max, B)[0] == B
    # the paper's form: dt = sqrt(2 eta eps / |a|)
    g = np.array([[0.0, 3.0, 4.0]], np.float32)                     # |a| = 5
    dt = math.sqrt(2 * 0.05 * 0.01 / 5.0)
    b = kdk.bins_for(g, 0.01, 0.05, 1.0, 30)[0]
    assert 2.0 ** -b <= dt < 2.0 ** -(b - 1)


def _const_force(a):
    return lambda pos, act: np.broadcast_to(np.asarray(a, np.float32), pos.shape).copy()


def test_free_particles_drift_exactly():
    r = np.random.default_rng(1)
    x0 = r.uniform(0.2, 0.8, (50, 3))
    v0 = r.uniform(-1e-3, 1e-3, (50, 3))
    x, v, _, bins, st = kdk.run(x0, v0, _const_force([0, 0, 0]), 1.0, 0.01, 0.05, 1.0, 3, 4)
    assert np.array_equal(v, v0) and (bins == 0).all()
    assert np.allclose(x, x0 + v0 * 4.0, rtol=0, atol=1e-13)
    assert st["ticks"] == 4 << 3


def test_constant_acceleration_is_exact():
    # the leapfrog integrates a constant force exactly: v = v0 + a T, x = x0 + v0 T + a T^2 / 2
    a = np.array([2.0 ** -10, -(2.0 ** -11), 0.0], np.float32)
    x0 = np.full((3, 3), 0.5)
    v0 = np.zeros((3, 3))
    T = 2.0
    x, v, _, bins, _ = kdk.run(x0, v0, _const_force(a), 1.0, 1e-6, 0.05, 1.0, 4, 2)
    assert (bins == bins[0]).all()
    assert np.allclose(v, a.astype(np.float64) * T, rtol=0, atol=1e-15)
    assert np.allclose(x, x0 + 0.5 * a.astype(np.float64) * T * T, rtol=0, atol=1e-14)


def _harmonic(omega, c=0.5):
    return lambda pos, act: (-(omega ** 2) * (pos - c)).astype(np.float32)


def test_second_order_convergence():
    # one oscillator, bin 0 throughout (dt_max set by hand): error ~ dt^2
    om, x0, T = 2.0, 0.52, 3.0
    errs = []
    for steps in (30, 60, 120):
        dt = T / steps
        x, v, _, _, _ = kdk.run(np.full((1, 3), x0), np.zeros((1, 3)), _harmonic(om), 1.0,
                                1e6, 0.05, dt, 0, steps)
        exact = 0.5 + (x0 - 0.5) * math.cos(om * T)
        errs.append(abs(x[0, 0] - exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5


def test_particles_in_different_bins_evolve_as_if_alone():
    # two independent oscillators whose criterion puts them in different bins
    om = np.array([0.5, 8.0])
    def force(pos, act):
        return (-(om[:, None] ** 2) * (pos - 0.5)).astype(np.float32)
    x0 = np.array([[0.55, 0.5, 0.5], [0.51, 0.5, 0.5]])
    v0 = np.zeros((2, 3))
    kw = dict(box=1.0, eps=2e-4, eta=0.05, dt_max=0.5, max_bin=6, nsteps=4)
    x, v, _, bins, st = kdk.run(x0, v0, force, **kw)
    assert bins[0] < bins[1]
    assert st["forces"] < 2 * ((4 << 6) + 1)          # fewer forces than global stepping
    for i in range(2):
        xi, vi, _, bi, _ = kdk.run(x0[i:i + 1], v0[i:i + 1],
                                   lambda p, a, i=i: (-(om[i] ** 2) * (p - 0.5)).astype(np.float32),
                                   **kw)
        assert bi[0] == bins[i]
        assert np.array_equal(xi[0], x[i]) and np.array_equal(vi[0], v[i])

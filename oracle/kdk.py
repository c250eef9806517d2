"""Kick-drift-kick leapfrog with individual power-of-two time steps -- TEST
INFRASTRUCTURE (the oracle of og_kdk_run; only the tests and the benchmark's
CPU leg use it).

What it computes, in the order of the paper (Sect. 3.2 "Time integration":
second-order KDK leapfrog; individual time steps; the acceleration criterion
dt_i = sqrt(2 eta eps / |a_i|) with the integration tolerance eta, default
0.05).  Readings of points the paper leaves open:

  - time bins: one maximum step dt_max is 2^B ticks (B = max_bin); a particle
    in bin b steps by dt_b = dt_max / 2^b and is active at the ticks that are
    multiples of its period 2^(B - b).
  - bin of a particle: the smallest b >= 0 with dt_max / 2^b <= dt_crit
    (b = 0 when |a| = 0), at most B, where dt_crit = sqrt(2 eta eps / |a|) is
    evaluated in FP64 from the single-precision acceleration (each operation
    rounded, in that order).  A particle may only enter a bin whose period
    divides the current tick: b = max(b, B - tz(k)), tz = trailing zero bits
    of the tick k (any bin at k = 0).
  - one tick k: if k > 0, every particle drifts by v dt_tick (dt_tick =
    dt_max / 2^B) and is wrapped into [0, L) (one subtraction or addition of L;
    a drift is less than L); the active particles (all at k = 0) get their
    acceleration at the drifted positions; if k > 0 they get the closing half
    kick v += a dt_b / 2 with their old bin; unless k is the last tick they get
    a new bin and the opening half kick v += a dt_b / 2 with the new bin.
  - arithmetic: v + a (dt / 2) and x + v dt_tick in FP64 with the FP32 a,
    products and sums rounded separately (no fused operations).

The force is a callable force(pos, active_mask) -> float32 [n, 3] (values of
inactive particles are ignored), so the same integrator runs on the oracle's
FP64 tree force or on another force evaluation.
"""
from __future__ import annotations

import math

import numpy as np


def bins_for(acc: np.ndarray, eps: float, eta: float, dt_max: float, max_bin: int) -> np.ndarray:
    """Bin of every particle from its single-precision acceleration."""
    acc = np.asarray(acc, dtype=np.float32)
    out = np.zeros(acc.shape[0], dtype=np.int32)
    for i in range(acc.shape[0]):
        ax, ay, az = (float(v) for v in acc[i])
        a = math.sqrt((ax * ax + ay * ay) + az * az)
        if not a > 0.0:
            continue
        dt_crit = math.sqrt((2.0 * eta * eps) / a)
        b = 0
        while b < max_bin and dt_max / (1 << b) > dt_crit:
            b += 1
        out[i] = b
    return out


def trailing_zeros(k: int) -> int:
    return (k & -k).bit_length() - 1 if k else 64


def run(pos, vel, force, box: float, eps: float, eta: float, dt_max: float, max_bin: int,
        nsteps: int):
    """Integrate nsteps maximum steps.  Returns (pos, vel, acc, bins, stats)."""
    pos = np.array(pos, dtype=np.float64, copy=True)
    vel = np.array(vel, dtype=np.float64, copy=True)
    n = pos.shape[0]
    acc = np.zeros((n, 3), dtype=np.float32)
    bins = np.zeros(n, dtype=np.int32)
    ticks = nsteps << max_bin
    dt_tick = dt_max / (1 << max_bin)
    forces = 0
    for k in range(ticks + 1):
        if k > 0:
            pos = pos + vel * dt_tick
            pos = np.where(pos >= box, pos - box, pos)
            pos = np.where(pos < 0.0, pos + box, pos)
        if k == 0:
            act = np.ones(n, dtype=bool)
        else:
            period = np.left_shift(1, max_bin - bins)
            act = (k % period) == 0
        a_new = np.asarray(force(pos, act.astype(np.uint8)), dtype=np.float32)
        acc[act] = a_new[act]
        forces += int(act.sum())
        idx = np.flatnonzero(act)
        if k > 0:
            half = (dt_max / np.left_shift(1, bins[idx]).astype(np.float64)) / 2.0
            vel[idx] = vel[idx] + acc[idx].astype(np.float64) * half[:, None]
        if k < ticks:
            nb = bins_for(acc[idx], eps, eta, dt_max, max_bin)
            nb = np.maximum(nb, max_bin - min(trailing_zeros(k), max_bin))
            bins[idx] = nb
            half = (dt_max / np.left_shift(1, bins[idx]).astype(np.float64)) / 2.0
            vel[idx] = vel[idx] + acc[idx].astype(np.float64) * half[:, None]
    return pos, vel, acc, bins, {"ticks": ticks, "forces": forces}

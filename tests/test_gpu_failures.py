"""Failure handling on the host side: allocation failure and request
cancellation.

Nothing here faults, traps or hangs the GPU.  Allocation failures are made on
the host by og_debug_fail_allocations (the library's allocation wrapper
returns "out of memory" without asking the device), and cancellation goes
through og_serve_cancel.  Each case checks that the failing call reports its
status, that nothing is left half-done, and that the context then gives the
same bits as a fresh one.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

import og_inputs as gi
from paper_2609_17658_gb300 import build as B
from paper_2609_17658_gb300 import og

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _clear_injection():
    B.build()
    yield
    og.og_debug_fail_allocations(0)


def _system(n=20000, seed=3):
    pos, mass, prm = gi.config("clustered-2m", n=n, seed=seed)
    return pos, mass, dict(prm, opening=gi.OPEN_BH)


def test_every_allocation_of_a_build_and_a_force_can_fail():
    """The k-th device allocation of a build (then of a force call) fails, for
    every k until the call makes fewer than k allocations: each failing call
    reports OG_ERR_OOM, and afterwards the same context gives bitwise the
    reference result."""
    pos, mass, prm = _system()
    prm = dict(prm, opening=gi.OPEN_REL)             # both walk passes and the group order
    with og.Context(0) as ctx:
        ref, rpp, rpn = og.Tree(ctx, pos, mass, prm).force()
        failed_build = 0
        for k in range(64):
            og.og_debug_fail_allocations(1, skip=k)
            try:
                t = og.Tree(ctx, pos, mass, prm)
            except og.OGError as e:
                assert e.status == og.OG_ERR_OOM
                failed_build += 1
                continue
            og.og_debug_fail_allocations(0)
            t.free()
            break
        assert failed_build >= 2                      # input staging, arena, scratch, ...
        t = og.Tree(ctx, pos, mass, prm)
        failed_force = 0
        for k in range(64):
            og.og_debug_fail_allocations(1, skip=k)
            try:
                acc, npp, npn = t.force()
            except og.OGError as e:
                assert e.status == og.OG_ERR_OOM
                failed_force += 1
                continue
            og.og_debug_fail_allocations(0)
            break
        assert failed_force >= 1
        assert np.array_equal(acc, ref) and np.array_equal(npp, rpp) and np.array_equal(npn, rpn)
        acc, npp, npn = t.force()
        t.free()
    assert np.array_equal(acc, ref) and np.array_equal(npp, rpp) and np.array_equal(npn, rpn)


def test_served_admission_failure_fails_only_that_request():
    reqs = gi.request_stream(1000.0, 10.0, seed=31, n_lo=3000, n_hi=20000, max_requests=3)
    with og.Context(0) as ctx:
        alone = []
        for q in reqs:
            acc = np.zeros((len(q.mass), 3), np.float32)
            t = og.og_serve_submit(ctx.h, q.pos, q.vel, q.mass, q.params, q.nsteps, q.dt_kick,
                                   q.dt_drift, acc)
            assert og.og_serve_poll(ctx.h, t, -1)[0] == og.OG_OK
            alone.append(acc)
    with og.Context(0) as ctx:
        # the engine is started by the first submission; fail the next allocation
        # (the admission of the first request) and let the others through
        og.og_debug_fail_allocations(1)
        outs, tickets = [], []
        for q in reqs:
            acc = np.zeros((len(q.mass), 3), np.float32)
            tickets.append(og.og_serve_submit(ctx.h, q.pos, q.vel, q.mass, q.params, q.nsteps,
                                              q.dt_kick, q.dt_drift, acc))
            outs.append(acc)
        st = []
        for t in tickets:
            try:
                st.append(og.og_serve_poll(ctx.h, t, -1)[0])
            except og.OGError as e:
                st.append(e.status)
    assert st.count(og.OG_ERR_OOM) == 1 and st.count(og.OG_OK) == 2
    for s, a, b in zip(st, outs, alone):
        if s == og.OG_OK:
            assert np.array_equal(a, b)


def test_cancel_queued_and_running_requests():
    small = gi.request_stream(1000.0, 10.0, seed=32, n_lo=3000, n_hi=8000, max_requests=3)
    n = 200_000
    pos, mass = gi.halo_mix(n, 33, n_halo=10)
    vel = np.random.default_rng(33).normal(0.0, 1e-3, size=(n, 3))
    side = n ** (1.0 / 3.0)
    prm = gi.default_params(eps=1 / (50 * side), r_s=1.25 / (2 * side), theta=0.5)
    with og.Context(0) as ctx:
        ref = np.zeros((len(small[2].mass), 3), np.float32)
        q = small[2]
        t = og.og_serve_submit(ctx.h, q.pos, q.vel, q.mass, q.params, q.nsteps, q.dt_kick,
                               q.dt_drift, ref)
        assert og.og_serve_poll(ctx.h, t, -1)[0] == og.OG_OK
    # the big system fits the budget, and none of the small ones beside it
    budget = og.og_serve_request_bytes(n) + og.og_serve_request_bytes(3000) // 2
    with og.Context(0, hbm_budget_bytes=budget) as ctx:
        big_acc = np.full((n, 3), np.nan, np.float32)
        t_big = og.og_serve_submit(ctx.h, pos, vel, mass, prm, 400, 1e-5, 1.0, big_acc)
        outs, tks = [], []
        for q in small:
            a = np.full((len(q.mass), 3), np.nan, np.float32)
            tks.append(og.og_serve_submit(ctx.h, q.pos, q.vel, q.mass, q.params, q.nsteps,
                                          q.dt_kick, q.dt_drift, a))
            outs.append(a)
        # the small requests wait behind the big one (budget): cancel one queued
        og.og_serve_cancel(ctx.h, tks[0])
        time.sleep(0.05)
        og.og_serve_cancel(ctx.h, t_big)                 # running: dropped before its next step
        with pytest.raises(og.OGError) as e:
            og.og_serve_poll(ctx.h, t_big, -1)
        assert e.value.status == og.OG_ERR_CANCELLED
        assert np.isnan(big_acc).all()                   # its output was never written
        with pytest.raises(og.OGError) as e:
            og.og_serve_poll(ctx.h, tks[0], -1)
        assert e.value.status == og.OG_ERR_CANCELLED
        assert np.isnan(outs[0]).all()
        for t in tks[1:]:
            assert og.og_serve_poll(ctx.h, t, -1)[0] == og.OG_OK
        assert np.array_equal(outs[2], ref)              # the others are untouched
        with pytest.raises(og.OGError) as e:
            og.og_serve_cancel(ctx.h, tks[1])            # already finished and collected
        assert e.value.status == og.OG_ERR_STATE
        with pytest.raises(og.OGError) as e:
            og.og_serve_cancel(ctx.h, 10 ** 9)
        assert e.value.status == og.OG_ERR_ARG


def test_bounded_device_wait_runs_out_and_the_context_stays_usable():
    """A tile of the one-kernel scan waits for the count of an earlier tile up
    to a poll limit.  With the first tile never taken that wait runs out: the
    kernel gives up and finishes, the call returns OG_ERR_TIMEOUT (about half a
    second of polling), and the same context then builds and walks bitwise as
    before.  Nothing faults or hangs: the wait is bounded by construction."""
    pos, mass, prm = _system()
    with og.Context(0) as ctx:
        ref, rpp, rpn = og.Tree(ctx, pos, mass, prm).force()
        with pytest.raises(og.OGError) as e:
            og.og_debug_scan_wait_timeout(ctx.h, 40000)
        assert e.value.status == og.OG_ERR_TIMEOUT
        acc, npp, npn = og.Tree(ctx, pos, mass, prm).force()
        assert np.array_equal(acc, ref) and np.array_equal(npp, rpp) and np.array_equal(npn, rpn)
        for n in (4096, 64 * 4096 + 1):            # one tile; more tiles than one kernel takes
            with pytest.raises(og.OGError) as e:
                og.og_debug_scan_wait_timeout(ctx.h, n)
            assert e.value.status == og.OG_ERR_ARG

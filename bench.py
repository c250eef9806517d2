"""Benchmark of the short-range TreePM tree force on GB300.

One step = the whole hot path on one system: fixed point + Morton keys, radix
sort, octree topology + threading, moments, groups, the Barnes-Hut first pass
and the relative-criterion pass of the walk, and the reordering of the
accelerations to the caller's order.  Default workload: 2,097,152 particles,
70 % in 2000 NFW haloes + 30 % uniform, eps = 1/6400, r_s = 1.25/256,
cutoff 4.5 r_s, relative opening alpha = 0.005 after a BH theta = 0.5 pass.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With torchrun each rank runs its own system
(a different seed; the path has no exchange step), so scaling is weak.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import og_inputs as gi  # noqa: E402

METRIC = "tree-force particles/s & interactions/s at 2.1M; served p50/p99 latency"
UNIT = "particles/s"
# Algorithmic FP32 work of one interaction (one target and one list entry):
# the nominal count of the pair arithmetic -- int-to-float and scaling 3,
# r^2 5, rsqrt and r 2, u 1, erfc polynomial 12 and exp 3, split factor 3,
# r^-3 2, m S r^-3 2, accumulation 6 -- with a fused multiply-add as 2 flops
# and a multi-function op as 1.
FLOPS_PER_INTERACTION = 45
# The same count taken from the far-entry evaluation loop's own instruction
# mix (reported beside it; it leaves out the compares and selects).
FLOPS_PER_INTERACTION_MIX = 36
FP32_LANES_PER_SM = 128


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


MEASURED = _measured_peaks()


WALK_SOURCE = "paper_2609_17658_gb300/csrc/og_walk.cu"
WALK_TYPES = ("CRec", "CExt", "WalkParams")     # what the walk reads from og_internal.h


def walk_source_hash():
    """sha256 over the walk's source and the definitions of the structures it
    reads (the rest of the internal header does not reach the kernel)."""
    import hashlib
    import re
    h = hashlib.sha256()
    with open(os.path.join(ROOT, WALK_SOURCE), "rb") as fh:
        h.update(fh.read())
    with open(os.path.join(ROOT, "paper_2609_17658_gb300/csrc/og_internal.h")) as fh:
        hdr = fh.read()
    for name in WALK_TYPES:
        m = re.search(r"struct (?:__align__\(\d+\) )?%s \{.*?\n\};" % name, hdr, re.S)
        h.update((m.group(0) if m else name).encode())
    return h.hexdigest()


def profiled_traffic(workload):
    """DRAM bytes (read + write) of the walk's launches in one step, from the
    committed ncu summary of this workload; None when there is none or when
    the walk's source changed after the counters were taken."""
    path = os.path.join(ROOT, "profiles", f"k_walk_{workload}.md")
    if not os.path.exists(path):
        return None
    fields = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
    if fields.get("walk source sha256") != walk_source_hash():
        return None
    try:
        return int(fields["dram bytes per step"])
    except (KeyError, ValueError):
        return None


def walk_traffic_per_launch(workload, prm):
    """DRAM bytes per walk launch, like `achieved` (which divides the flops of
    the step's walk launches by their time): the step's traffic over its
    launches, two for the relative criterion (a Barnes-Hut first pass), else one."""
    per_step = profiled_traffic(workload)
    if per_step is None:
        return None
    return per_step / (2 if prm.get("opening") == gi.OPEN_REL else 1)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="clustered-2m")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-kdk", action="store_true")
    ap.add_argument("--no-pm", action="store_true")
    ap.add_argument("--no-sph", action="store_true")
    ap.add_argument("--no-fp32-peak", action="store_true",
                    help="skip the FP32 FMA-rate measurement after the timed region")
    ap.add_argument("--served-scale", type=float, default=1.0,
                    help="multiplies every served rate's arrival window")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 32k uniform and 16.7M clustered workloads")
    ap.add_argument("--batched-boxes", type=int, default=512)
    return ap.parse_args()


def seed_for_rank(rank: int) -> int:
    """Each rank times its own independent system (weak scaling, no data-path
    collective); rank 0 runs the single-GPU workload itself."""
    return 12346 + 1000 * rank


def max_over_ranks(x: float, ws: int, device) -> float:
    """The slowest rank's value (the job's time), via one all-reduce."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_run(step, steps: int, ws: int, device):
    """The per-rank part of the timed region: ``steps`` calls of ``step()``,
    each returning (its duration in ms, its result), then one all-reduce that
    gives every rank the slowest rank's total.  Returns (the job's time per
    step in ms, the last result)."""
    total, res = 0.0, None
    for _ in range(steps):
        ms, res = step()
        total += ms
    return max_over_ranks(total, ws, device) / steps, res


def job_value(n_per_rank: int, ws: int, ms_per_step: float) -> float:
    """Whole-job particles/s: every rank's particles over the slowest rank's step."""
    return ws * n_per_rank / (ms_per_step * 1e-3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.idx = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_passes(ot, prm, sel, nthreads):
    """Both walk passes of the oracle for the selected groups (the relative
    criterion after its own Barnes-Hut first pass, else one pass)."""
    a1, _, _ = ot.force(opening=gi.OPEN_BH, theta=prm.get("theta_first_pass", prm["theta"])
                        if prm["opening"] == gi.OPEN_REL else prm["theta"], groups=sel,
                        nthreads=nthreads)
    if prm["opening"] == gi.OPEN_REL:
        a_old = np.nan_to_num(a1).astype(np.float32)
        ot.force(opening=gi.OPEN_REL, a_old=a_old, groups=sel, nthreads=nthreads)


def cpu_baseline(pos, mass, prm, budget_s=20.0):
    """The FP64 oracle on the host cores.  Its tree build is single-threaded
    by construction and is timed on all particles; the walk (both passes) is
    timed with one thread and with every core on random samples of groups,
    each sample grown until it takes about a quarter of the budget.  The
    whole-step rate is N / (build + force time per target x N)."""
    import oracle
    oracle.build()
    nthreads = os.cpu_count() or 1
    t0 = time.perf_counter()
    ot = oracle.Tree(pos, mass, prm)
    t_build = time.perf_counter() - t0
    ng = ot.ngroups
    gb, ge = ot.get(oracle.F_GBEG), ot.get(oracle.F_GEND)
    order = np.random.default_rng(1).permutation(ng)
    force = {}
    for label, nth, share in (("1_thread", 1, 0.15), ("all_threads", nthreads, 0.35)):
        k, done, targets, t = 16, 0, 0, 0.0
        while t < budget_s * share and done < ng:
            sel = np.sort(order[done:done + k])
            t0 = time.perf_counter()
            _oracle_passes(ot, prm, sel, nth)
            t += time.perf_counter() - t0
            done += len(sel)
            targets += int((ge[sel] - gb[sel]).sum())
            k *= 2
        force[label] = {"groups": done, "targets": targets, "seconds": t,
                        "us_per_target": t / max(targets, 1) * 1e6}
    n = len(mass)
    per_target = force["all_threads"]["seconds"] / max(force["all_threads"]["targets"], 1)
    t_total = t_build + per_target * n
    per_target1 = force["1_thread"]["seconds"] / max(force["1_thread"]["targets"], 1)
    return {"value": n / t_total, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "build_s": t_build, "build_threads": 1,
            "force_1_thread": force["1_thread"], "force_all_threads": force["all_threads"],
            "value_1_thread": n / (t_build + per_target1 * n),
            "sample": f"FP64 tree build of all {n} particles ({t_build:.2f} s, single-threaded) + "
                      f"the walk (both passes for the relative criterion) for {force['all_threads']['targets']} targets in "
                      f"{force['all_threads']['groups']} random groups on {nthreads} threads "
                      f"({force['all_threads']['seconds']:.2f} s) and for "
                      f"{force['1_thread']['targets']} targets on 1 thread "
                      f"({force['1_thread']['seconds']:.2f} s); force time per target scaled to "
                      f"all {n} targets"}


def accuracy(og, ctx, pos, mass, prm, ngroups=300, seed=7, ot=None):
    """Error of the library's accelerations against the FP64 oracle on the
    same lists (the relative criterion fed the library's own first-pass
    accelerations on both sides), on a random sample of whole groups:
    per-particle |a - a_oracle| / |a_oracle|, p99, rms and max."""
    import oracle
    if ot is None:
        ot = oracle.Tree(pos, mass, prm)
    a_old = None
    if prm["opening"] == gi.OPEN_REL:
        bh = dict(prm, opening=gi.OPEN_BH, theta=prm["theta_first_pass"])
        t1 = og.Tree(ctx, pos, mass, bh)
        a_old, _, _ = t1.force()
        t1.free()
    t = og.Tree(ctx, pos, mass, prm)
    acc, _, _ = t.force(a_old=a_old)
    t.free()
    sel = np.sort(np.random.default_rng(seed).choice(ot.ngroups, min(ngroups, ot.ngroups),
                                                      replace=False))
    ref, _, _ = ot.force(a_old=a_old, groups=sel, nthreads=os.cpu_count() or 1)
    m = ~np.isnan(ref[:, 0])
    na = np.linalg.norm(ref[m], axis=1)
    e = np.linalg.norm(acc[m].astype(np.float64) - ref[m], axis=1)
    rms_a = float(np.sqrt(np.mean(na ** 2)))
    keep = na >= 1e-6 * rms_a
    rel = e[keep] / na[keep]
    return {"targets": int(m.sum()), "groups": int(len(sel)),
            "p99_rel_err": float(np.quantile(rel, 0.99)), "rms_rel_err": float(np.sqrt(np.mean(rel ** 2))),
            "max_rel_err": float(rel.max()), "bound": "p99 <= 1e-4, rms <= 2e-5"}


def batched_bench(og, ctx, torch, dev, stream, nboxes, steps):
    """Many independent boxes: one og_batch_force call (one forest, one walk
    launch per pass) against one og_tree_build + og_tree_force call per box,
    inputs resident on the device, same GPU, same results."""
    boxes = gi.batch_boxes(nboxes)
    descs = []
    for b in boxes:
        n = len(b.mass)
        descs.append(dict(pos=torch.from_numpy(b.pos).to(dev), mass=torch.from_numpy(b.mass).to(dev),
                          params=b.params,
                          acc=torch.empty((n, 3), dtype=torch.float32, device=dev),
                          n_pp=torch.empty(n, dtype=torch.int32, device=dev),
                          n_pn=torch.empty(n, dtype=torch.int32, device=dev)))
    total = sum(len(b.mass) for b in boxes)

    def one_batch():
        return og.og_batch_force(ctx.h, descs)

    def per_box():
        inter = 0
        for d in descs:
            h = og.og_tree_build(ctx.h, d["pos"], d["mass"], d["params"])
            og.og_tree_force(h, d["acc"], None, d["n_pp"], d["n_pn"])
            inter += og.og_tree_info_get(h)["interactions"]
            og.og_tree_free(h)
        return inter

    info = one_batch()
    per_box()
    torch.cuda.synchronize()
    tb, tp = [], []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = one_batch()
        e1.record(stream)
        torch.cuda.synchronize()
        tb.append(e0.elapsed_time(e1))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        inter_pb = per_box()
        e1.record(stream)
        torch.cuda.synchronize()
        tp.append(e0.elapsed_time(e1))
    mb, mp = statistics.median(tb), statistics.median(tp)
    return {"workload": f"{nboxes} boxes, N log-uniform [4096, 262144], uniform or halo-clustered "
                        f"(coin flip), eps=1/(50 N^(1/3)), r_s=1.25/(2 N^(1/3)), BH theta 0.5",
            "particles": total, "groups": info["groups"], "interactions": info["interactions"],
            "batched_ms": mb, "per_box_ms": mp,
            "batched_particles_per_s": total / (mb * 1e-3),
            "per_box_particles_per_s": total / (mp * 1e-3),
            "batched_speedup": mp / mb,
            "batched_walk_ms": info["ms_walk"], "batched_build_ms": info["ms_build"],
            "same_interactions": int(inter_pb) == int(info["interactions"])}


def kdk_bench(og, ctx, n=2097152, max_bin=6, dt_max=0.02, rebuild_every=8):
    """Individual power-of-two time steps against global stepping.  A
    halo-clustered system (the 2.1M generator at n particles, velocities
    Gaussian 1e-3 box per unit time) is integrated over one maximum step with
    bins chosen by the acceleration criterion (eta 0.05), and again with every
    particle at the finest step the first run used.  Host arrays in and out,
    the tree rebuilt every 4 ticks and refitted in between."""
    pos, mass, prm = gi.config("clustered-2m", n=n, seed=12350)
    prm = dict(prm, opening=gi.OPEN_BH, theta=0.5)
    vel = np.random.default_rng(12350).normal(0.0, 1e-3, size=pos.shape)
    p1, v1 = pos.copy(), vel.copy()
    t0 = time.perf_counter()
    _, bins, st = og.og_kdk_run(ctx.h, p1, v1, mass, prm, dt_max=dt_max, eta=0.05,
                                max_bin=max_bin, nsteps=1, rebuild_every=rebuild_every)
    t_ind = time.perf_counter() - t0
    bmax = int(bins.max())
    p2, v2 = pos.copy(), vel.copy()
    t0 = time.perf_counter()
    _, _, sg = og.og_kdk_run(ctx.h, p2, v2, mass, prm, dt_max=dt_max / (1 << bmax), eta=0.05,
                             max_bin=0, nsteps=1 << bmax, rebuild_every=rebuild_every)
    t_glob = time.perf_counter() - t0
    return {"workload": f"{n} particles, halo-clustered, one maximum step dt_max={dt_max}, "
                        f"max_bin={max_bin}, BH theta 0.5, rebuild every {rebuild_every} ticks",
            "bins_used": sorted(int(b) for b in np.unique(bins)),
            "individual": {"ticks": st["ticks"], "forces": st["forces"],
                           "interactions": st["interactions"], "seconds": t_ind,
                           "forces_per_s": st["forces"] / t_ind, "device_ms": st["ms"]},
            "global_finest": {"ticks": sg["ticks"], "forces": sg["forces"],
                              "interactions": sg["interactions"], "seconds": t_glob,
                              "forces_per_s": sg["forces"] / t_glob, "device_ms": sg["ms"]},
            "force_ratio": sg["forces"] / st["forces"],
            "interaction_ratio": sg["interactions"] / max(st["interactions"], 1),
            "speedup": t_glob / t_ind}


SERVED_RATES = ((10.0, 20.0), (30.0, 20.0), (100.0, 10.0), (300.0, 4.0), (1000.0, 1.5))


def served_bench(og, torch, dev, rates=SERVED_RATES, scale=1.0, pool_size=16):
    """Served stream: Poisson arrivals of systems with N log-uniform in
    [1e4, 2e6] (halo-clustered, 8 kick-drift steps each, HBM budget 40 GB)
    against the plain per-box path (build + force per step, then kick and
    drift, one request after another), both on this GPU from host arrays,
    results left on the device.  ``rates``: (arrivals per second, window in
    seconds) pairs; above the service rate the queue grows for the whole
    window, so the overloaded rates get short windows (their latencies then
    measure that window's backlog)."""
    pool = gi.request_stream(1e9, 1e9, seed=12349, max_requests=pool_size)
    # plain path
    ctx = og.Context(dev.index or 0)
    stream = torch.cuda.current_stream(dev)
    og.og_set_stream(ctx.h, stream.cuda_stream)
    plain_req = pool[:6]
    work = sum(len(r.mass) * r.nsteps for r in plain_req)

    def plain_run(reqs):
        for r in reqs:
            pos = torch.from_numpy(r.pos).to(dev)
            vel = torch.from_numpy(r.vel).to(dev)
            mass = torch.from_numpy(r.mass).to(dev)
            acc = torch.empty((len(r.mass), 3), dtype=torch.float32, device=dev)
            for _ in range(r.nsteps):
                h = og.og_tree_build(ctx.h, pos, mass, r.params)
                og.og_tree_force(h, acc)
                og.og_tree_free(h)
                vel += acc.double() * r.dt_kick
                pos = torch.remainder(pos + vel * r.dt_drift, 1.0)

    plain_run(pool[:2])          # warm-up: first use of every kernel, torch's included
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_run(plain_req)
    torch.cuda.synchronize()
    plain = work / (time.perf_counter() - t0)
    ctx.close()
    out = {"workload": "Poisson arrivals, N log-uniform [1e4, 2e6], halo-clustered, 8 kick-drift "
                       "steps, v Gaussian sigma 1e-3 box/step, BH theta 0.5, budget 40 GB",
           "plain_particle_steps_per_s": plain, "rates": []}
    for rate, window in rates:
        seconds = window * scale
        r = np.random.default_rng(int(rate))
        arrivals = np.cumsum(r.exponential(1.0 / rate, size=int(rate * seconds * 3) + 8))
        arrivals = arrivals[arrivals < seconds]
        ctx = og.Context(dev.index or 0, hbm_budget_bytes=40 << 30)
        tickets = []
        t_base = time.perf_counter()
        for k, ta in enumerate(arrivals):
            q = pool[k % pool_size]
            delay = t_base + ta - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append((og.og_serve_submit(ctx.h, q.pos, q.vel, q.mass, q.params, q.nsteps,
                                               q.dt_kick, q.dt_drift), len(q.mass) * q.nsteps))
        res = []
        for t, w in tickets:
            st, x = og.og_serve_poll(ctx.h, t, -1)
            res.append((x, w))
        ctx.close()
        lat = np.array([x["t_done"] - x["t_submit"] for x, _ in res])
        span = max(x["t_done"] for x, _ in res) - min(x["t_submit"] for x, _ in res)
        work = sum(w for _, w in res)
        out["rates"].append({"rate_per_s": rate, "window_s": seconds, "requests": len(res),
                             "particle_steps_per_s": work / span,
                             "p50_latency_ms": float(np.percentile(lat, 50) * 1e3),
                             "p99_latency_ms": float(np.percentile(lat, 99) * 1e3),
                             "refits": int(sum(x["refits"] for x, _ in res)),
                             "rebuilds": int(sum(x["rebuilds"] for x, _ in res))})
    best = max(x["particle_steps_per_s"] for x in out["rates"])
    out["served_over_plain"] = best / plain
    # the service rate: requests per second the saturated engine completes
    mean_work = float(np.mean([len(q.mass) * q.nsteps for q in pool]))
    out["saturation_requests_per_s"] = best / mean_work
    out["refits"] = int(sum(x["refits"] for x in out["rates"]))
    out["rebuilds"] = int(sum(x["rebuilds"] for x in out["rates"]))
    return out


def run_reference(args):
    """--impl reference: the FP64 oracle (the paper's method as the CPU program
    of this repository) timed on the host cores.  Each step is one bounded
    sample of the workload: the oracle's tree build of all N particles
    (single-threaded by construction) and both walk passes for the targets of
    a fresh random set of groups on every core.  ms_per_step is that step's
    wall time; the value is the whole-step rate the sample measures,
    N / (build time + force time per target x N).  The warm-up steps size the
    group set so that a step takes about two seconds."""
    import oracle
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    oracle.build()
    pos, mass, prm = gi.config(args.workload)
    n = len(mass)
    nthreads = os.cpu_count() or 1
    t0 = time.perf_counter()
    ot = oracle.Tree(pos, mass, prm)
    ng = ot.ngroups
    gb, ge = ot.get(oracle.F_GBEG), ot.get(oracle.F_GEND)
    del ot
    order = np.random.default_rng(2).permutation(ng)
    k = min(ng, 256)
    pos_in_order = 0
    vals, ms, samples = [], [], []
    for step in range(args.warmup + args.steps):
        if pos_in_order + k > ng:
            pos_in_order = 0
        sel = np.sort(order[pos_in_order:pos_in_order + k])
        pos_in_order += k
        t0 = time.perf_counter()
        ot = oracle.Tree(pos, mass, prm)
        tb = time.perf_counter() - t0
        t1 = time.perf_counter()
        _oracle_passes(ot, prm, sel, nthreads)
        tf = time.perf_counter() - t1
        del ot
        targets = int((ge[sel] - gb[sel]).sum())
        if step < args.warmup:
            # size the sample for a force time of about 1.5 s
            k = int(min(ng, max(16, k * 1.5 / max(tf, 1e-3))))
            continue
        vals.append(n / (tb + tf / max(targets, 1) * n))
        ms.append((tb + tf) * 1e3)
        samples.append((tb, tf, targets, len(sel)))
    v = statistics.median(vals)
    tb, tf, targets, groups = samples[len(samples) // 2]
    sample = (f"per step: FP64 tree build of all {n} particles (single-threaded, about {tb:.2f} s) + "
              f"the walk (both passes for the relative criterion) for about {targets} targets in {groups} random groups on "
              f"{nthreads} threads (about {tf:.2f} s); force time per target scaled to all {n} "
              f"targets")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(ms),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": f"{args.workload}: N={n} per GPU, " + describe(args.workload, prm),
                      "l2": "n/a (CPU)"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def describe(name, prm):
    """One-line recipe of a named workload, from its parameters."""
    side = round(1.0 / (50 * prm["eps"]))
    if name.startswith("clustered"):
        nh = 2000 if name == "clustered-2m" else 16000
        head = f"70% in {nh} NFW haloes + 30% uniform"
    else:
        head = "Poisson-uniform"
    crit = (f"relative alpha={prm['alpha']:g} after BH theta={prm['theta_first_pass']:g}"
            if prm["opening"] == gi.OPEN_REL else f"BH theta={prm['theta']:g}")
    return (f"{head}, eps=1/{50 * side}, r_s=1.25/{2 * side}, "
            f"cutoff {prm['rcut_over_rs']:g} r_s, {crit}")


def pm_bench(og, ctx, torch, dev, stream, dpos, dmass, prm, steps, flush):
    """Long-range particle-mesh force (og_tree_pm_force) of the step's workload on
    the mesh with r_s = 1.25 mesh cells (256^3 for r_s = 1.25/256): device
    buffers, L2 flushed before every call, CUDA events on the launching
    stream.  Algorithmic bytes, each array read or written once per step:
    zeroing the 8-byte fixed-point mesh, the assignment's read-modify-write of
    it, the conversion (8 B in, 4 B out per point), the FFTs and the Green's
    multiplication (4 B in and 4 B out per point each: 8 + 8 + 8), the
    interpolation's potential read (4 B per point); per particle 16 B of
    positions and mass in, 4 B of permutation and 12 B of acceleration."""
    mesh = 1 << int(round(math.log2(1.25 * prm["box"] / prm["r_s"])))
    n = int(dmass.shape[0])
    acc = torch.empty((n, 3), dtype=torch.float32, device=dev)
    h = og.og_tree_build(ctx.h, dpos, dmass, prm)
    ms = []
    for k in range(3 + steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        og.og_tree_pm_force(h, mesh, acc)
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= 3:
            ms.append(e0.elapsed_time(e1))
    og.og_tree_free(h)
    cells = mesh ** 3
    algo = cells * (8 + 16 + 12 + 8 + 8 + 8 + 4) + n * (16 + 4 + 12)
    t = statistics.median(ms)
    peak = MEASURED.get("hbm_gbs")
    gbs = algo / (t * 1e-3) / 1e9
    return {"workload": f"{n} particles of the step's workload, mesh {mesh}^3 "
                        f"(r_s = {prm['r_s'] * mesh / prm['box']:.2f} cells), FP32 cuFFT",
            "ms": t, "particles_per_s": n / (t * 1e-3),
            "roofline": {"bound": "hbm", "algorithmic_bytes": algo, "achieved": gbs, "peak": peak,
                         "unit": "GB/s", "frac": gbs / peak if peak else None}}


def sph_bench(og, ctx, torch, dev, stream, pos, dpos, dmass, prm, steps, flush):
    """SPH density (og_tree_sph_density, cubic spline) of the step's workload with
    h_i the distance to the 32nd nearest other particle, the paper's default
    neighbour number for that kernel in 3D (found on the host with a periodic
    k-d tree before timing).  Device buffers, L2 flushed before every call,
    CUDA events on the launching stream."""
    from scipy.spatial import cKDTree
    x = np.floor(pos / prm["box"] * 4294967296.0) % 4294967296.0 * (prm["box"] / 4294967296.0)
    d, _ = cKDTree(x, boxsize=prm["box"]).query(x, k=33, workers=-1)
    h = torch.from_numpy(d[:, -1].astype(np.float32)).to(dev)
    n = int(dmass.shape[0])
    rho = torch.empty(n, dtype=torch.float32, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev)
    t = og.og_tree_build(ctx.h, dpos, dmass, prm)
    ms = []
    for k in range(3 + steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        og.og_tree_sph_density(t, h, rho, cnt)
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= 3:
            ms.append(e0.elapsed_time(e1))
    groups = og.og_tree_info_get(t)["groups"]
    tm = statistics.median(ms)
    pairs = float(cnt.double().sum().item())
    # the smoothing lengths from the paper's relation (4 pi / 3) h^3 rho = 32 m, from the
    # mean-density guess for every particle, tolerance 1 %
    h0 = prm["box"] * (3.0 * 32 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    hs = torch.full((n,), h0, dtype=torch.float32, device=dev)
    flush.zero_()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters = og.og_tree_sph_smoothing(t, 32.0, 0.01, 200, hs, rho, cnt)
    e1.record(stream)
    torch.cuda.synchronize()
    og.og_tree_free(t)
    return {"workload": f"{n} particles of the step's workload, h = distance to the 32nd "
                        f"neighbour, cubic spline, {groups} group searches",
            "ms": tm, "particles_per_s": n / (tm * 1e-3), "neighbour_pairs": pairs,
            "neighbour_pairs_per_s": pairs / (tm * 1e-3),
            "smoothing": {"what": "h from (4 pi/3) h^3 rho = 32 m within 1 %, every particle starting "
                                  "at the mean-density h", "iterations": iters,
                          "ms": e0.elapsed_time(e1)}}


def device_steps(og, ctx, torch, stream, dpos, dmass, prm, steps, warmup, flush):
    """W untimed and K timed steps (build + force, L2 flushed before each),
    CUDA events on the launching stream; returns per-step lists."""
    n = int(dmass.shape[0])
    acc = torch.empty((n, 3), dtype=torch.float32, device=dpos.device)
    npp = torch.empty(n, dtype=torch.int32, device=dpos.device)
    npn = torch.empty(n, dtype=torch.int32, device=dpos.device)
    out = {"ms": [], "walk": [], "build": [], "inter": []}
    for k in range(warmup + steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h = og.og_tree_build(ctx.h, dpos, dmass, prm)
        og.og_tree_force(h, acc, None, npp, npn)
        e1.record(stream)
        torch.cuda.synchronize()
        info = og.og_tree_info_get(h)
        og.og_tree_free(h)
        if k >= warmup:
            out["ms"].append(e0.elapsed_time(e1))
            out["walk"].append(info["ms_walk"])
            out["build"].append(info["ms_build"])
            out["inter"].append(info["interactions"])
    return out


def walk_roofline(inter_step, walk_ms, sms, max_mhz, sm_mhz=None):
    """The walk's FP32 work (FLOPS_PER_INTERACTION per interaction) over its
    CUDA-event time, against the unit-count FP32 peak."""
    peak = sms * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
    achieved = inter_step * FLOPS_PER_INTERACTION / (walk_ms * 1e-3) / 1e12
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "flops_per_interaction": FLOPS_PER_INTERACTION,
           "frac_by_instruction_mix": achieved / peak * FLOPS_PER_INTERACTION_MIX / FLOPS_PER_INTERACTION,
           "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {max_mhz:.0f} MHz"}
    if sm_mhz:
        out["frac_at_observed_clock"] = achieved / (sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12)
    return out


def config_bench(og, ctx, torch, dev, stream, name, steps, warmup, flush, sms, max_mhz, cpu,
                 oracle_budget_s):
    """Another named workload, timed like the main one: device-resident
    inputs, L2 flushed between steps; the error against the oracle on sampled
    groups and (if ``cpu``) the oracle's own rate on the host cores."""
    pos, mass, prm = gi.config(name)
    n = len(mass)
    dpos = torch.from_numpy(pos).to(dev)
    dmass = torch.from_numpy(mass).to(dev)
    r = device_steps(og, ctx, torch, stream, dpos, dmass, prm, steps, warmup, flush)
    del dpos, dmass
    ms = float(np.mean(r["ms"]))
    walk = float(np.mean(r["walk"]))
    inter = float(np.mean(r["inter"]))
    out = {"workload": f"{name}: N={n}, " + describe(name, prm), "steps": steps, "warmup": warmup,
           "ms_per_step": ms, "particles_per_s": n / (ms * 1e-3),
           "interactions_per_step": inter, "interactions_per_s": inter / (ms * 1e-3),
           "walk_ms_per_step": walk, "build_ms_per_step": float(np.mean(r["build"])),
           "walk_interactions_per_s": inter / (walk * 1e-3),
           "roofline": walk_roofline(inter, walk, sms, max_mhz)}
    out["accuracy"] = accuracy(og, ctx, pos, mass, prm, ngroups=200)
    if cpu:
        out["cpu_baseline"] = cpu_baseline(pos, mass, prm, budget_s=oracle_budget_s)
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    from paper_2609_17658_gb300 import build as B
    if rank == 0:
        B.build()
    if ws > 1:
        dist.barrier()
    from paper_2609_17658_gb300 import og

    pos, mass, prm = gi.config(args.workload, seed=seed_for_rank(rank))
    n = len(mass)
    dev = torch.device(f"cuda:{local}")
    stream = torch.cuda.current_stream(dev)
    ctx = og.Context(local)
    og.og_set_stream(ctx.h, stream.cuda_stream)
    dpos = torch.from_numpy(pos).to(dev)
    dmass = torch.from_numpy(mass).to(dev)
    acc = torch.empty((n, 3), dtype=torch.float32, device=dev)
    npp = torch.empty(n, dtype=torch.int32, device=dev)
    npn = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def step():
        h = og.og_tree_build(ctx.h, dpos, dmass, prm)
        og.og_tree_force(h, acc, None, npp, npn)
        info = og.og_tree_info_get(h)
        og.og_tree_free(h)
        return info

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    gpu_id = f"GPU-{uuid}" if uuid is not None else os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.3)
    ms_steps, ms_walk, inter, ms_build = [], [], [], []
    launches0 = og.og_kernel_launches()

    def timed_step():
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_steps.append(e0.elapsed_time(e1))
        ms_walk.append(info["ms_walk"])
        ms_build.append(info["ms_build"])
        inter.append(info["interactions"])
        return ms_steps[-1], info

    launches = None
    try:
        ms_per_step, _ = rank_run(timed_step, args.steps, ws, dev)
    finally:
        launches = og.og_kernel_launches() - launches0
        clocks = sampler.stop()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    value = job_value(n, ws, ms_per_step)
    inter_step = float(np.mean(inter))
    walk_ms = float(np.mean(ms_walk))

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        # pinned host buffers, as a serving process would keep them
        h_pos = torch.from_numpy(pos).pin_memory().numpy()
        h_mass = torch.from_numpy(mass).pin_memory().numpy()
        h_acc = torch.empty((n, 3), dtype=torch.float32).pin_memory().numpy()
        h_pp = torch.empty(n, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
        h_pn = torch.empty(n, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
        og.og_set_stream(ctx.h, None)
        ts = []
        for k in range(max(2, args.steps) + 1):
            t0 = time.perf_counter()
            h = og.og_tree_build(ctx.h, h_pos, h_mass, prm)
            og.og_tree_force(h, h_acc, None, h_pp, h_pn)
            og.og_tree_free(h)
            if k > 0:
                ts.append(time.perf_counter() - t0)
        og.og_set_stream(ctx.h, stream.cuda_stream)
        e2e = {"value": n / statistics.median(ts), "unit": UNIT,
               "h2d_bytes_per_step": int(pos.nbytes + mass.nbytes),
               "d2h_bytes_per_step": int(h_acc.nbytes + h_pp.nbytes + h_pn.nbytes)}
        if ws > 1:
            e2e["value"] *= ws

    # roofline of the dominant kernel (the walk): FP32 ALU bound
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    roof = walk_roofline(inter_step, walk_ms, sms, max_mhz, clocks.get("sm_mhz"))
    achieved = roof["achieved"]
    roof.update({"traffic": walk_traffic_per_launch(args.workload, prm),
                 "traffic_unit": "bytes per walk launch (mean over the step's launches)",
                 "kernel": "k_walk (both passes)"})
    # the FP32 rate this GPU sustains on independent FMA chains, measured after
    # the timed region (not a denominator: the peak above is the unit count)
    if not args.no_fp32_peak:
        fp32 = og.og_measure_fp32_peak(ctx.h)
        roof["fp32_measured_tflops"] = {"fma": fp32["fma"], "fma2": fp32["fma2"]}
        roof["frac_of_measured_fma"] = achieved / fp32["fma"] if fp32["fma"] > 0 else None

    batched = None
    if not args.no_batched:
        batched = batched_bench(og, ctx, torch, dev, stream, args.batched_boxes, max(1, min(args.steps, 3)))

    served = None
    if not args.no_served and rank == 0:
        served = served_bench(og, torch, dev, scale=args.served_scale)

    pmr = None
    if not args.no_pm and rank == 0:
        pmr = pm_bench(og, ctx, torch, dev, stream, dpos, dmass, prm, max(3, args.steps), flush)
        pmr["treepm_ms_per_step"] = ms_per_step + pmr["ms"]

    sphr = None
    if not args.no_sph and rank == 0:
        sphr = sph_bench(og, ctx, torch, dev, stream, pos, dpos, dmass, prm, max(3, args.steps), flush)

    kdk = None
    if not args.no_kdk and rank == 0:
        kdk = kdk_bench(og, ctx)

    cpu = acc_err = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        acc_err = accuracy(og, ctx, pos, mass, prm, ngroups=300)
        cpu = cpu_baseline(pos, mass, prm)

    configs = None
    if rank == 0 and not args.no_configs:
        configs = {}
        for name, st, budget in (("uniform-32k", max(args.steps, 10), 6.0),
                                 ("clustered-16m", max(3, min(args.steps, 5)), 16.0)):
            configs[name] = config_bench(og, ctx, torch, dev, stream, name, st, 3, flush, sms,
                                         max_mhz, cpu=(ws == 1 and not args.no_cpu),
                                         oracle_budget_s=budget)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
               "data": "synthetic",
               "config": {"workload": f"{args.workload}: N={n} per GPU, " + describe(args.workload, prm),
                          "l2": "flushed between steps (256 MB write)"},
               "interactions_per_s": ws * inter_step / (ms_per_step * 1e-3),
               "interactions_per_step": inter_step,
               "walk_ms_per_step": walk_ms,
               "build_ms_per_step": float(np.mean(ms_build)),
               "walk_interactions_per_s": inter_step / (walk_ms * 1e-3),
               "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
               "roofline": roof, "cpu_baseline": cpu, "accuracy": acc_err,
               "configs": configs, "batched": batched, "served": served,
               "individual_steps": kdk, "pm_long_range": pmr,
               "sph_density": sphr}
        print(json.dumps(out), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

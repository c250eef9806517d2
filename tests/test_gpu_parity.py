"""GPU parity: the CUDA library through the C-ABI against the FP64 oracle.

Bit-exact: keys, permutation, fixed-point positions, node table, threading,
moments (mass and sums of m x bitwise, centre of mass), groups, interaction
lists, counts.
Tolerance: accelerations, p99 relative error <= 1e-4 and rms <= 2e-5 against
the oracle evaluated on the same lists.
"""
from __future__ import annotations

import numpy as np
import pytest

import og_inputs as gi
import oracle
from paper_2609_17658_gb300 import build as B
from paper_2609_17658_gb300 import og
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    B.build()
    oracle.build()
    c = og.Context(0)
    yield c
    c.close()


def _case(name):
    if name == "uniform-32k":
        return gi.config("uniform-32k")
    if name == "halo-20k":
        pos, mass, prm = gi.config("clustered-2m", n=20000)
        prm["r_s"] = 0.02
        return pos, mass, prm
    base = gi.default_params(eps=1e-3, r_s=0.02)
    if name.startswith("n="):
        n = int(name[2:])
        pos, mass = gi.uniform(n, 100 + n)
        return pos, mass, base
    if name == "identical":
        pos = np.tile([[0.3, 0.6, 0.9]], (100, 1))
        return pos, np.full(100, 0.01), base
    if name == "cell-faces":
        r = np.random.default_rng(7)
        k = r.integers(0, 1 << 12, size=(3000, 3))
        pos = k / float(1 << 12)          # exactly on level-12 cell faces
        pos[::7] = pos[::7] + 2.0 ** -32  # one grid unit above a face
        return pos, np.full(3000, 1 / 3000), base
    if name == "box-edges":
        r = np.random.default_rng(8)
        pos = r.random((2000, 3))
        pos[:300] = 0.0
        pos[300:600] = 1.0 - 2.0 ** -32
        pos[600:700, 0] = -1e-300         # wraps to 0
        return pos, np.full(2000, 1 / 2000), base
    if name == "half-box":
        pos = np.array([[0.1, 0.2, 0.3], [0.6, 0.2, 0.3], [0.1, 0.7, 0.8], [0.6, 0.7, 0.8]] * 8)
        pos += np.repeat(np.arange(8) * 1e-3, 4)[:, None]
        prm = gi.default_params(eps=1e-3, r_s=0.0)   # no cutoff: half-box pairs interact
        return pos, np.full(32, 1 / 32), prm
    if name == "equal-runs":
        # runs of 1500 equal positions that straddle the 1024-split tiles of
        # the node-range kernels, beside runs at nearby and distant cells
        r = np.random.default_rng(9)
        pos = r.random((6000, 3))
        pos[700:2200] = [0.25, 0.5, 0.75]
        pos[2200:3700] = [0.25, 0.5, 0.75 + 2.0 ** -32]
        pos[3700:3720] = [0.9, 0.1, 0.4]
        pos[5000:5999] = [0.25, 0.5, 0.75]
        return pos, np.full(6000, 1 / 6000), base
    if name == "lattice":
        pos, mass = gi.lattice(16)
        return pos, mass, gi.default_params(eps=1e-3, r_s=0.05)
    raise KeyError(name)


BUILD_CASES = ["uniform-32k", "halo-20k", "n=1", "n=2", "n=7", "n=8", "n=9", "n=33", "identical",
               "cell-faces", "box-edges", "half-box", "lattice", "equal-runs"]


@pytest.mark.parametrize("name", BUILD_CASES)
def test_build_bit_exact(ctx, name):
    pos, mass, prm = _case(name)
    gt = og.Tree(ctx, pos, mass, prm)
    ot = oracle.Tree(pos, mass, prm)
    parity.compare_build(gt, ot)


@pytest.mark.parametrize("name", BUILD_CASES)
def test_lists_counts_and_forces(ctx, name):
    pos, mass, prm = _case(name)
    prm = dict(prm, flags=og.OG_DEBUG_DUMP_LISTS)
    gt = og.Tree(ctx, pos, mass, prm)
    ot = oracle.Tree(pos, mass, prm)
    gmap = parity.node_map(gt, ot)
    acc, npp, npn = gt.force()
    ref, rpp, rpn = ot.force(keep_lists=True)
    off, lst = ot.lists()
    parity.compare_lists(parity.gpu_lists(gt, gmap), off, lst, range(ot.ngroups))
    assert np.array_equal(npp, rpp) and np.array_equal(npn, rpn)
    if np.abs(ref).max() == 0:
        assert np.abs(acc).max() == 0
    elif name == "lattice":
        # zero force by symmetry: compare on the scale of one neighbour's pull
        assert np.abs(acc - ref).max() < 1e-5 * mass[0] * 16 ** 2
    else:
        parity.check_accel(acc, ref)


@pytest.mark.parametrize("theta", [0.0, 0.3, 0.8])
def test_barnes_hut_angles(ctx, theta):
    pos, mass, prm = gi.config("clustered-2m", n=30000)
    prm = dict(prm, opening=gi.OPEN_BH, theta=theta, r_s=0.015, flags=og.OG_DEBUG_DUMP_LISTS)
    gt = og.Tree(ctx, pos, mass, prm)
    ot = oracle.Tree(pos, mass, prm)
    gmap = parity.node_map(gt, ot)
    acc, npp, npn = gt.force()
    ref, rpp, rpn = ot.force(keep_lists=True)
    off, lst = ot.lists()
    parity.compare_lists(parity.gpu_lists(gt, gmap), off, lst, range(ot.ngroups))
    assert np.array_equal(npp, rpp) and np.array_equal(npn, rpn)
    parity.check_accel(acc, ref)
    if theta == 0.0:
        d = oracle.direct(pos, mass, prm, nthreads=0)
        parity.check_accel(acc, d)


def test_relative_criterion_same_lists(ctx):
    pos, mass, prm = gi.config("clustered-2m", n=40000)
    prm["r_s"] = 0.015
    bh = dict(prm, opening=gi.OPEN_BH, theta=prm["theta_first_pass"])
    a1, _, _ = og.Tree(ctx, pos, mass, bh).force()
    rel = dict(prm, opening=gi.OPEN_REL, flags=og.OG_DEBUG_DUMP_LISTS)
    gt = og.Tree(ctx, pos, mass, rel)
    ot = oracle.Tree(pos, mass, rel)
    gmap = parity.node_map(gt, ot)
    acc, npp, npn = gt.force(a_old=a1)
    ref, rpp, rpn = ot.force(a_old=a1, keep_lists=True)
    off, lst = ot.lists()
    parity.compare_lists(parity.gpu_lists(gt, gmap), off, lst, range(ot.ngroups))
    assert np.array_equal(npp, rpp) and np.array_equal(npn, rpn)
    parity.check_accel(acc, ref)
    # the library's own first pass (a_old = NULL) is exactly the explicit two steps
    acc2, npp2, npn2 = og.Tree(ctx, pos, mass, dict(rel, flags=0)).force()
    assert np.array_equal(acc2, acc) and np.array_equal(npp2, npp) and np.array_equal(npn2, npn)


def test_split_off_newtonian(ctx):
    pos, mass = gi.halo_mix(5000, 21, n_halo=4)
    prm = gi.default_params(eps=2e-3, r_s=0.0, theta=0.5)
    acc, npp, npn = og.Tree(ctx, pos, mass, prm).force()
    ref, rpp, rpn = oracle.Tree(pos, mass, prm).force()
    assert np.array_equal(npp, rpp) and np.array_equal(npn, rpn)
    parity.check_accel(acc, ref)


def test_device_pointers_match_host(ctx):
    torch = pytest.importorskip("torch")
    pos, mass, prm = gi.config("uniform-32k", n=20000)
    acc_h, npp_h, npn_h = og.Tree(ctx, pos, mass, prm).force()
    dp = torch.from_numpy(pos).cuda()
    dm = torch.from_numpy(mass).cuda()
    h = og.og_tree_build(ctx.h, dp, dm, prm)
    acc = torch.zeros((20000, 3), dtype=torch.float32, device="cuda")
    npp = torch.zeros(20000, dtype=torch.int32, device="cuda")
    npn = torch.zeros(20000, dtype=torch.int32, device="cuda")
    og.og_tree_force(h, acc, None, npp, npn)
    torch.cuda.synchronize()
    og.og_tree_free(h)
    assert np.array_equal(acc.cpu().numpy(), acc_h)
    assert np.array_equal(npp.cpu().numpy().astype(np.uint32), npp_h)
    assert np.array_equal(npn.cpu().numpy().astype(np.uint32), npn_h)


def test_invalid_inputs_are_errors(ctx):
    pos, mass = gi.uniform(100, 3)
    bad = pos.copy()
    bad[5, 1] = np.nan
    with pytest.raises(og.OGError) as e:
        og.Tree(ctx, bad, mass, gi.default_params())
    assert e.value.status == og.OG_ERR_ARG
    with pytest.raises(og.OGError):
        og.Tree(ctx, pos, -mass, gi.default_params())
    with pytest.raises(og.OGError):
        og.Tree(ctx, pos, mass, gi.default_params(r_s=0.2, rcut_over_rs=4.5))  # r_cut >= L/2
    with pytest.raises(og.OGError):
        og.Tree(ctx, pos[:0], mass[:0], gi.default_params())
    with pytest.raises(og.OGError):
        og.Tree(ctx, pos, mass, gi.default_params(leaf_max=2))
    # the context is still usable afterwards
    acc, _, _ = og.Tree(ctx, pos, mass, gi.default_params(r_s=0.02)).force()
    assert np.isfinite(acc).all()


def _sample_groups(ngroups, k, seed):
    r = np.random.default_rng(seed)
    return np.sort(r.choice(ngroups, size=min(k, ngroups), replace=False))


@pytest.mark.parametrize("name,nsample", [("clustered-2m", 400), ("clustered-16m", 150)])
def test_fullsize_clustered_sampled(ctx, name, nsample):
    """The clustered workloads at full size (2,097,152 and 16,777,216
    particles): tree bit-exact everywhere, lists and accelerations of sampled
    groups against the oracle (relative criterion with the library's own
    first-pass accelerations fed to both sides)."""
    pos, mass, prm = gi.config(name)
    bh = dict(prm, opening=gi.OPEN_BH, theta=prm["theta_first_pass"])
    a1, _, _ = og.Tree(ctx, pos, mass, bh).force(counts=False)
    rel = dict(prm, opening=gi.OPEN_REL, flags=og.OG_DEBUG_DUMP_LISTS)
    gt = og.Tree(ctx, pos, mass, rel)
    ot = oracle.Tree(pos, mass, rel)
    gmap = parity.compare_build(gt, ot)
    acc, npp, npn = gt.force(a_old=a1)
    sel = _sample_groups(ot.ngroups, nsample, 5)
    ref, rpp, rpn = ot.force(a_old=a1, groups=sel, keep_lists=True)
    off, lst = ot.lists()
    parity.compare_lists(parity.gpu_lists(gt, gmap, sel), off, lst, sel)
    perm = ot.get(oracle.F_PERM)
    gb, ge = ot.get(oracle.F_GBEG), ot.get(oracle.F_GEND)
    tgt = np.concatenate([perm[gb[g]:ge[g]] for g in sel])
    assert np.array_equal(npp[tgt], rpp[tgt]) and np.array_equal(npn[tgt], rpn[tgt])
    parity.check_accel(acc[tgt], ref[tgt])


@pytest.mark.parametrize("box", [1.0, 0.125, 1024.0, 3.0])
def test_quantization_of_special_values(ctx, box):
    """Fixed-point positions bit-exact with the oracle for negatives, subnormals,
    values a rounding away from the box, and large multiples of the box
    (power-of-two boxes take the integer path, 3.0 the division)."""
    r = np.random.default_rng(12)
    v = np.concatenate([
        r.uniform(-3 * box, 3 * box, 3000),
        r.standard_normal(1000) * box * 10.0 ** r.integers(-300, 12, 1000),
        -np.abs(r.standard_normal(200)) * 10.0 ** r.integers(-324, -300, 200),
        [0.0, -0.0, box, -box, box * (1 - 2 ** -53), -box * 2 ** -40, 5e-324, -5e-324,
         box * 2 ** 31, -box * 2 ** 31.5, box * (2 ** 32 + 2 ** -33)]])
    v = v[: (len(v) // 3) * 3]
    pos = np.ascontiguousarray(v.reshape(-1, 3))
    n = len(pos)
    prm = gi.default_params(eps=box * 1e-3, r_s=box * 0.02, box=box)
    gt = og.Tree(ctx, pos, np.full(n, 1.0 / n), prm)
    spos = gt.export(og.OG_F_SPOS)
    perm = gt.export(og.OG_F_PERM)
    for a in range(3):
        want = np.array([oracle.quantize1(float(x), box) for x in pos[perm, a]], dtype=np.uint32)
        assert np.array_equal(spos[a], want)


@pytest.mark.parametrize("opening", [gi.OPEN_BH, gi.OPEN_REL])
def test_massless_particles_and_nodes(ctx, opening):
    """Zero masses: a massless node takes its cell centre as its centre of
    mass, massless sources add nothing, and the relative criterion sees
    a_min = 0 for groups of massless targets.  Tree bit-exact, counts exact,
    forces within the tolerance against the oracle."""
    pos, mass, prm = gi.config("clustered-2m", n=20000)
    mass = mass.copy()
    r = np.random.default_rng(19)
    mass[r.random(len(mass)) < 0.3] = 0.0            # scattered massless particles
    mass[np.argsort(pos[:, 0])[:2000]] = 0.0         # a massless slab: whole massless nodes
    prm = dict(prm, opening=opening)
    gt = og.Tree(ctx, pos, mass, prm)
    ot = oracle.Tree(pos, mass, prm)
    parity.compare_build(gt, ot)
    a1 = None
    if opening == gi.OPEN_REL:
        a1, _, _ = og.Tree(ctx, pos, mass, dict(prm, opening=gi.OPEN_BH)).force(counts=False)
    acc, npp, npn = gt.force(a_old=a1)
    ref, rpp, rpn = ot.force(a_old=a1)
    assert np.array_equal(npp, rpp) and np.array_equal(npn, rpn)
    parity.check_accel(acc, ref)


@pytest.mark.parametrize("kind", ["unequal", "spread", "subnormal", "overflow", "coincident"])
def test_exact_moments_mass_distributions(ctx, kind):
    """Node masses and sums of m x bitwise the oracle's exact sums rounded once,
    centres of mass exact: unequal masses, masses spread over 2^-30..2^30,
    subnormal masses, masses whose sums of m x overflow to infinity, and
    buckets of coincident keys."""
    r = np.random.default_rng(23)
    pos, mass, prm = gi.config("clustered-2m", n=30000)
    n = len(mass)
    if kind == "unequal":
        mass = mass * (0.5 + r.random(n))
    elif kind == "spread":
        mass = np.ldexp(1.0 + r.random(n), r.integers(-30, 31, n))
    elif kind == "subnormal":
        mass = 5e-324 * r.integers(1, 1 << 20, n).astype(np.float64)
    elif kind == "overflow":
        mass = 1e300 * (1.0 + r.random(n))
    else:
        pos = np.concatenate([pos, np.repeat(pos[:500], 4, axis=0)])
        mass = np.concatenate([mass, mass[0] * r.random(2000)])
    gt = og.Tree(ctx, pos, mass, prm)
    ot = oracle.Tree(pos, mass, prm)
    parity.compare_build(gt, ot)
    if kind == "overflow":
        assert np.isinf(gt.export(og.OG_F_MSUM)).any()


def test_mass_span_limit(ctx):
    """Masses may span 128 binary orders (lowest set bit of the smallest to the
    top of the largest); one more is OG_ERR_ARG, and the context stays usable."""
    pos, _, prm = gi.config("uniform-32k", n=3000)
    mass = np.ones(len(pos))
    mass[7] = 2.0 ** -75 * (1.0 + 2.0 ** -52)              # span 1 - (-127) = 128
    gt = og.Tree(ctx, pos, mass, prm)
    parity.compare_build(gt, oracle.Tree(pos, mass, prm))
    gt.free()
    mass[7] = 2.0 ** -76 * (1.0 + 2.0 ** -52)              # span 129
    with pytest.raises(og.OGError) as e:
        og.Tree(ctx, pos, mass, prm)
    assert e.value.status == og.OG_ERR_ARG and "128" in str(e.value)
    mass[7] = 1.0
    parity.compare_build(og.Tree(ctx, pos, mass, prm), oracle.Tree(pos, mass, prm))


@pytest.mark.parametrize("n", [262144, 786432, 786433])
def test_build_bit_exact_at_path_limits(ctx, n):
    """Sizes where the build changes kernels: 262,144 particles put the node
    and group scans at 64 tiles (one kernel with a look-back) and the child
    scan (n + 1 entries) at 65 (two kernels); 786,432 keys are the largest
    sort run as one kernel per pass and 786,433 the smallest with the count,
    scan and scatter kernels.  The tree is bitwise the oracle's either way."""
    pos, mass, prm = gi.config("clustered-2m", n=n, seed=77)
    gt = og.Tree(ctx, pos, mass, prm)
    parity.compare_build(gt, oracle.Tree(pos, mass, prm))

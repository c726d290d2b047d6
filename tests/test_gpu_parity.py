"""GPU parity against the FP64 CPU oracle, through the C-ABI.

FP64 mode: the kernel performs the oracle's IEEE operations in the same
order, so every int64 tally (fluence voxels, R, T, A, killed, gain,
scatter and step counts) and every per-packet record must be IDENTICAL.
Mixed mode: a different but consistent estimator of the same transport, so
R, T, A and the fluence must agree with the oracle within Monte Carlo error:
R, T, A within 3 sigma (z over per-packet variances); the fluence block by
block over the whole map, from batch spreads on both sides
(``bench.block_stats``).  The paired comparison with the FP64 kernel at
millions of packets is in ``test_gpu_parity_blocks.py``.
"""
import math
from dataclasses import replace

import numpy as np
import pytest

import bench
import oracle as O
import paper_2112_08035_gb300 as smc
import workloads as W

pytestmark = pytest.mark.gpu

FX = 2.0 ** 32
EXACT_KEYS = ("R", "T", "A", "killed", "gain", "packets", "scatters", "steps")


@pytest.fixture(scope="module")
def ctx():
    c = smc.Context(0)
    yield c
    c.close()


def _torch():
    import torch
    return torch


def run_gpu(ctx, wl, precision, records=False, id_begin=0, blocks=0, threads=0, fluence=True):
    torch = _torch()
    plan = ctx.plan(wl, precision)
    if blocks or threads:
        plan.set_launch(blocks, threads)
    g = wl.grid
    flu = torch.zeros((g.n[2], g.n[1], g.n[0]), dtype=torch.int64, device="cuda") if fluence else None
    tot = smc.totals_tensor()
    rec = torch.zeros(wl.npackets * 8, dtype=torch.int64, device="cuda") if records else None
    plan.launch(id_begin, wl.npackets, wl.seed, flu, tot, rec)
    torch.cuda.synchronize()
    assert plan.status() == 0
    plan.close()
    out = (flu.cpu().numpy() if fluence else None, smc.totals_from_tensor(tot))
    if records:
        r = rec.cpu().numpy().view(smc.RECORD_DTYPE)
        out = out + (r,)
    return out


def assert_exact(tg, to):
    for k in EXACT_KEYS:
        assert tg[k] == to[k], (k, tg[k], to[k])


SMALL = [
    (W.sphere_pencil, 3000),
    (W.three_layer_slab, 1500),
    (W.vessel_network, 300),
    (W.vessel_network_hard, 300),
    (W.glass_container, 600),
]


@pytest.mark.parametrize("factory,n", SMALL, ids=[f.__name__ for f, _ in SMALL])
def test_fp64_bitexact_small(ctx, factory, n):
    wl = factory().with_packets(n)
    fo, to, ro = O.run(wl, records=True)
    fg, tg, rg = run_gpu(ctx, wl, "fp64", records=True)
    assert_exact(tg, to)
    assert np.array_equal(fg, fo)
    for f in ("R", "T", "A", "killed", "gain", "scatters", "steps"):
        assert np.array_equal(rg[f], ro[f]), f


@pytest.mark.parametrize("factory,n", SMALL, ids=[f.__name__ for f, _ in SMALL])
def test_fp64_bitexact_segment_stepping(ctx, factory, n):
    # segment stepping (longer moves bounded along the ray): the FP64 kernel
    # still performs the reference's operations, so the bits agree
    wl = factory().with_packets(n).with_stepping(W.SEGMENT)
    fo, to, ro = O.run(wl, records=True)
    fg, tg, rg = run_gpu(ctx, wl, "fp64", records=True)
    assert_exact(tg, to)
    assert np.array_equal(fg, fo)
    for f in ("R", "T", "A", "killed", "gain", "scatters", "steps"):
        assert np.array_equal(rg[f], ro[f]), f


def test_fp64_bitexact_segment_config0_full_size(ctx):
    wl = W.sphere_pencil().with_stepping(W.SEGMENT)
    fo, to, _ = O.run(wl)
    fg, tg = run_gpu(ctx, wl, "fp64")
    assert_exact(tg, to)
    assert np.array_equal(fg, fo)


def test_fp64_bitexact_config0_full_size(ctx):
    # the plain-FP64 sphere workload at its full 1e5 packets, 50^3 grid
    wl = W.sphere_pencil()
    fo, to, _ = O.run(wl)
    fg, tg = run_gpu(ctx, wl, "fp64")
    assert_exact(tg, to)
    assert np.array_equal(fg, fo)


def test_fp64_bitexact_ragged_launch_shapes(ctx):
    # a ragged packet count over several launch shapes: same bits every time
    wl = W.three_layer_slab(1237, grid_n=33)
    fo, to, _ = O.run(wl)
    for blocks, threads in [(1, 32), (3, 64), (5, 96), (0, 128), (152 * 7, 128)]:
        fg, tg = run_gpu(ctx, wl, "fp64", blocks=blocks, threads=threads)
        assert_exact(tg, to)
        assert np.array_equal(fg, fo)


def test_fp64_id_offset_and_split_additivity(ctx):
    wl = W.glass_container(900, grid_n=40)
    fo, to, _ = O.run(wl, 5000, 5900)
    fg, tg = run_gpu(ctx, wl, "fp64", id_begin=5000)
    assert_exact(tg, to)
    assert np.array_equal(fg, fo)
    fa, ta = run_gpu(ctx, wl.with_packets(400), "fp64", id_begin=5000)
    fb, tb = run_gpu(ctx, wl.with_packets(500), "fp64", id_begin=5400)
    assert np.array_equal(fa + fb, fo)
    for k in EXACT_KEYS:
        assert ta[k] + tb[k] == to[k]


def _zcheck(rg, ro, key, k=3.0):
    a = rg[key].astype(np.float64) / FX
    b = ro[key].astype(np.float64) / FX
    se = math.sqrt(a.var() / a.size + b.var() / b.size)
    z = abs(a.mean() - b.mean()) / max(se, 1e-12)
    assert z < k, (key, a.mean(), b.mean(), se, z)
    return z


# (factory, GPU packets, oracle packets, voxel block edge)
MIXED = [
    (W.sphere_pencil, 200_000, 20_000, 5),
    (W.three_layer_slab, 200_000, 10_000, 10),
    (W.vessel_network, 40_000, 2_000, 50),
    (W.vessel_network_hard, 40_000, 2_000, 25),
    (W.glass_container, 100_000, 5_000, 16),
]
NBATCH = 20


def gpu_batches(ctx, wl, precision, n, K, block, id_begin):
    """K launches of n // K consecutive ids from id_begin: per-packet
    records and per-batch block sums of the fluence (per packet)."""
    torch = _torch()
    plan = ctx.plan(wl, precision)
    g = wl.grid
    per = n // K
    flu = torch.zeros((g.n[2], g.n[1], g.n[0]), dtype=torch.int64, device="cuda")
    tot = smc.totals_tensor()
    rec = torch.zeros(K * per * 8, dtype=torch.int64, device="cuda")
    blocks = []
    for k in range(K):
        flu.zero_()
        plan.launch(id_begin + k * per, per, wl.seed, flu, tot, rec[k * per * 8:(k + 1) * per * 8])
        blocks.append(bench.block_sums(flu, (block,) * 3) / FX / per)
    torch.cuda.synchronize()
    assert plan.status() == 0
    plan.close()
    return rec.cpu().numpy().view(smc.RECORD_DTYPE), np.array(blocks)


def oracle_batches(wl, n, K, block, id_begin=0):
    """The oracle on K batches of n // K consecutive ids: records and
    per-batch block sums (per packet)."""
    per = n // K
    recs, blocks = [], []
    for k in range(K):
        f, _, r = O.run(wl.with_packets(per), id_begin + k * per, records=True)
        recs.append(r)
        blocks.append(bench.block_sums(f, (block,) * 3) / FX / per)
    return np.concatenate(recs), np.array(blocks)


@pytest.mark.parametrize("stepping", [W.SPHERE_TRACING, W.SEGMENT])
@pytest.mark.parametrize("factory,ng,no,block", MIXED, ids=[f.__name__ for f, _, _, _ in MIXED])
def test_mixed_matches_oracle_statistically(ctx, factory, ng, no, block, stepping):
    pytest.importorskip("scipy")
    # the oracle always runs the paper's plain sphere tracing; the GPU runs
    # mixed precision with either step rule
    wl = factory()
    ro, bo = oracle_batches(wl, no, NBATCH, block)
    # disjoint packet ids for the GPU sample: independent estimates
    rg, bg = gpu_batches(ctx, wl.with_stepping(stepping), "mixed", ng, NBATCH, block, 10_000_000)
    for key in ("R", "T", "A"):
        _zcheck(rg, ro, key)
    # fluence: a z per voxel block over the whole map (Welch, batch spreads)
    s = bench.block_stats(bg, bo, paired=False)
    assert s["blocks"] >= 8 and s["pass"], s
    # energy closes per packet (FP32 weights: relative 1e-5 per packet)
    bal = (rg["R"] + rg["T"] + rg["A"] + rg["killed"] - rg["gain"]) / FX
    assert np.all(np.abs(bal - 1.0) < 1e-4)


@pytest.mark.parametrize("stepping", [W.SPHERE_TRACING, W.SEGMENT])
def test_mixed_glass_shell_traps_no_packet(ctx, stepping):
    # Between two concentric spheres Snell's law conserves n r sin(theta), so
    # no packet that enters the clear glass shell from the air or the liquid
    # can meet total internal reflection at both walls.  Two FP32 effects once
    # trapped about one packet in 1e6 there until the step cap: pushes along
    # the normal that shifted r sin(theta) the same way at every bounce, and
    # crawls (forced steps away from a wall) whose identical FP32 increments
    # rounded the same way until the packet crossed the wall unnoticed.  At
    # 1e7 packets neither step rule may hit the cap.
    wl = W.glass_container(10_000_000).with_stepping(stepping)
    _, t = run_gpu(ctx, wl, "mixed")
    assert t["packets"] == wl.npackets
    assert t["max_steps_hit"] == 0, t["max_steps_hit"]


def test_mixed_vessel_served_job_no_step_cap(ctx):
    # a vessel job of the served mix (2.4e6 packets, 64 capsules in a smooth
    # union) once had five packets at the step cap: two launched exactly on
    # the tissue box's face by an FP32 uniform of 1 and crawling along it at
    # distance 0, three pushed back and forth across a capsule wall at a
    # smooth-union crease by matched-index crossings that did not advance
    # along the ray
    wl = W.served_mix(40, 4, stepping=W.SEGMENT)[35]
    assert wl.name.endswith("vessel") and wl.npackets > 2_000_000
    _, t = run_gpu(ctx, wl, "mixed")
    assert t["packets"] == wl.npackets
    assert t["max_steps_hit"] == 0, t["max_steps_hit"]


def test_register_variants_identical(ctx):
    # the register budget changes occupancy, never arithmetic
    wl = W.glass_container(700, grid_n=32)
    fo, to, _ = O.run(wl)
    ref = None
    for v in range(3):
        plan = ctx.plan(wl, "fp64")
        plan.set_variant(v)
        torch = _torch()
        flu = torch.zeros((32, 32, 32), dtype=torch.int64, device="cuda")
        tot = smc.totals_tensor()
        plan.launch(0, wl.npackets, wl.seed, flu, tot)
        torch.cuda.synchronize()
        assert np.array_equal(flu.cpu().numpy(), fo)
        assert_exact(smc.totals_from_tensor(tot), to)
        plan.close()
        pm = ctx.plan(wl.with_packets(20000), "mixed")
        pm.set_variant(v)
        flu.zero_(); tot.zero_()
        pm.launch(0, 20000, wl.seed, flu, tot)
        torch.cuda.synchronize()
        got = (flu.cpu().numpy(), smc.totals_from_tensor(tot))
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got[0], ref[0])
            for k in EXACT_KEYS:
                assert got[1][k] == ref[1][k], (v, k)
        pm.close()
    # mixed variants 3..5: the same budgets with the scene tables staged in
    # each warp's shared memory -- the same numbers are loaded, so the same bits
    torch = _torch()
    for v in range(3, 6):
        pm = ctx.plan(wl.with_packets(20000), "mixed")
        pm.set_variant(v)
        flu = torch.zeros((32, 32, 32), dtype=torch.int64, device="cuda")
        tot = smc.totals_tensor()
        pm.launch(0, 20000, wl.seed, flu, tot)
        torch.cuda.synchronize()
        assert np.array_equal(flu.cpu().numpy(), ref[0]), v
        t = smc.totals_from_tensor(tot)
        for k in EXACT_KEYS:
            assert t[k] == ref[1][k], (v, k)
        pm.close()
    with pytest.raises(smc.SmcrtError):
        ctx.plan(wl, "mixed").set_variant(6)
    with pytest.raises(smc.SmcrtError):
        ctx.plan(wl, "fp64").set_variant(3)


def test_autotune_choice_is_valid(ctx):
    wl = W.three_layer_slab(50_000)
    plan = ctx.plan(wl, "mixed")
    blocks, threads, variant = plan.autotune(20_000)
    assert blocks >= 152 and threads in (64, 128) and variant in range(6)
    fg, tg = run_gpu(ctx, wl, "mixed")   # a new plan of the same shape reuses the choice
    assert tg["packets"] == wl.npackets
    plan.close()


def test_launch_shape_limits(ctx):
    plan = ctx.plan(W.sphere_pencil(10), "mixed")
    for bad in [(0, 256), (0, 33), (-1, 64)]:
        with pytest.raises(smc.SmcrtError) as e:
            plan.set_launch(*bad)
        assert e.value.code == smc.ERR_BAD_ARG
    plan.close()


def test_edge_cases(ctx):
    wl = W.sphere_pencil(1)
    # a single packet, both precisions
    fo, to, _ = O.run(wl)
    fg, tg = run_gpu(ctx, wl, "fp64")
    assert_exact(tg, to)
    assert np.array_equal(fg, fo)
    fg, tg = run_gpu(ctx, wl, "mixed")
    assert tg["packets"] == 1
    # zero packets: nothing launched, nothing tallied
    fg, tg = run_gpu(ctx, wl.with_packets(0), "fp64")
    assert tg["packets"] == 0 and not fg.any()
    # no fluence buffer: totals only
    _, tg = run_gpu(ctx, wl.with_packets(500), "fp64", fluence=False)
    _, to, _ = O.run(wl.with_packets(500), fluence=False)
    assert_exact(tg, to)
    # one voxel grid; source outside the bounding box escapes at once
    w2 = replace(wl.with_packets(300), grid=W.Grid((-1, -1, -1), (1, 1, 1), (1, 1, 1)))
    fo, to, _ = O.run(w2)
    fg, tg = run_gpu(ctx, w2, "fp64")
    assert_exact(tg, to)
    assert np.array_equal(fg, fo)
    w3 = replace(wl.with_packets(64), source=W.Source(W.PENCIL, (0, 0, 5.0), (0, 0, -1.0)))
    fg, tg = run_gpu(ctx, w3, "fp64")
    assert tg["T"] == 64 * 2 ** 32 and tg["steps"] == 0
    # step cap of one: every surviving packet is killed after one step
    w4 = replace(wl.with_packets(200), scene=replace(wl.scene, max_steps=1))
    fo, to, _ = O.run(w4)
    fg, tg = run_gpu(ctx, w4, "fp64")
    assert_exact(tg, to)
    assert tg["max_steps_hit"] > 0


@pytest.mark.parametrize("g", [-0.7, 0.0, 0.99])
def test_fp64_bitexact_anisotropy_extremes(ctx, g):
    wl = W.sphere_pencil(800)
    wl = replace(wl, scene=replace(wl.scene, regions=(replace(wl.scene.regions[0], g=g),)))
    fo, to, _ = O.run(wl)
    fg, tg = run_gpu(ctx, wl, "fp64")
    assert_exact(tg, to)
    assert np.array_equal(fg, fo)


def test_fp64_bitexact_iso_source_and_roulette(ctx):
    # isotropic point source in a high-albedo sphere: long histories and
    # Russian roulette both occur
    sc = W.isotropic_sphere(100.0)   # ~5e3 scatterings: weights reach the roulette threshold
    sc = replace(sc, regions=(replace(sc.regions[0], mu_a=2.0, g=0.5, n=1.4),))
    wl = W.Workload("iso", sc, W.Source(W.ISO_POINT, (0, 0, 0), (0, 0, -1.0)),
                    W.Grid((-0.6, -0.6, -0.6), (0.6, 0.6, 0.6), (24, 24, 24)), 300, 77, "fp64")
    fo, to, _ = O.run(wl)
    fg, tg = run_gpu(ctx, wl, "fp64")
    assert to["gain"] > 0 and to["killed"] > 0
    assert_exact(tg, to)
    assert np.array_equal(fg, fo)


def test_full_size_three_layer_sampled(ctx):
    """The 1e7-packet layered workload in its benchmark launch shape: FP64
    per-packet records of a random sample of ids equal the oracle's one by
    one; mixed-mode R/T/A agree with the FP64 run on the same ids within
    3 sigma of their paired differences."""
    torch = _torch()
    wl = W.three_layer_slab()
    fg, tg, rg = run_gpu(ctx, wl, "fp64", records=True)
    assert tg["packets"] == wl.npackets
    rng = np.random.default_rng(5)
    ids = np.sort(rng.choice(wl.npackets, 300, replace=False))
    for i in ids:
        _, _, ro = O.run(wl, int(i), int(i) + 1, threads=1, fluence=False, records=True)
        for f in ("R", "T", "A", "killed", "gain", "scatters", "steps"):
            assert rg[f][i] == ro[f][0], (i, f)
    fm, tm, rm = run_gpu(ctx, wl, "mixed", records=True)
    assert tm["packets"] == wl.npackets
    for key in ("R", "T", "A"):   # paired on the same 1e7 ids, 3 sigma
        z = bench.paired_z(rm[key] / FX, rg[key] / FX)
        assert abs(z) < 3.0, (key, z)
    del rg, rm
    torch.cuda.empty_cache()

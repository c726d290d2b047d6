"""Mixed precision against the FP64 kernel, tally by tally, on configs 0-3.

The FP64 kernel reproduces the FP64 oracle bit for bit, packet by packet
(``test_gpu_parity.py``; sampled ids of the full-size runs in
``test_gpu_full_size.py``), so at millions of packets it stands in for an
oracle run of that size.  Both kernels run the SAME packet ids with the same
Philox streams, in K batches of consecutive ids:

  - R, T, A: the mean per-packet paired difference (mixed - FP64) is within
    3 standard errors of zero, the standard error from the differences' own
    spread -- every reported tally within 3 sigma of the Monte Carlo error;
  - fluence: one z per voxel block over the whole map, from the K batches'
    paired block differences (Student t with K - 1 degrees of freedom turned
    into a normal deviate); accepted when the count of |z| > 3 stays within
    its binomial expectation plus 3 sigma, chi2/dof within its 3-sigma band
    and max |z| under the Bonferroni bound of the block count
    (``bench.paired_block_stats``).  A few wrong voxels near a curved surface
    move their blocks' z, which no map-wide norm would show.

Both sides use segment stepping (the step rule of the timed benchmark) and,
for the slab and the container, also the paper's sphere tracing.
"""
import math

import numpy as np
import pytest

import bench
import paper_2112_08035_gb300 as smc
import workloads as W

pytestmark = pytest.mark.gpu
pytest.importorskip("scipy")

FX = 2.0 ** 32

# (factory, packets, batches, block edge in voxels (x, y, z))
CONFIGS = {
    "sphere_pencil": (W.sphere_pencil, 1_000_000, 40, (5, 5, 5)),          # 50^3 grid
    "three_layer_slab": (W.three_layer_slab, 2_000_000, 40, (10, 10, 10)),  # 100^3 grid
    "vessel_network": (W.vessel_network, 1_000_000, 40, (20, 20, 20)),     # 200^3 grid
    "glass_container": (W.glass_container, 1_000_000, 40, (16, 16, 16)),   # 128^3 grid
}


@pytest.fixture(scope="module")
def ctx():
    c = smc.Context(0)
    yield c
    c.close()


def batched(ctx, wl, precision, n, K, block):
    """Run ids [0, n) as K launches of consecutive ids; returns per-packet
    records, per-batch block sums (K, nblocks) and per-batch totals."""
    import torch
    plan = ctx.plan(wl, precision)
    g = wl.grid
    flu = torch.zeros((g.n[2], g.n[1], g.n[0]), dtype=torch.int64, device="cuda")
    tot = smc.totals_tensor()
    rec = torch.zeros(n * 8, dtype=torch.int64, device="cuda")
    per = n // K
    blocks, totals = [], []
    for k in range(K):
        flu.zero_()
        tot.zero_()
        plan.launch(k * per, per, wl.seed, flu, tot, rec[k * per * 8:(k + 1) * per * 8])
        blocks.append(bench.block_sums(flu, block))
        totals.append(smc.totals_from_tensor(tot))
    torch.cuda.synchronize()
    assert plan.status() == 0
    plan.close()
    r = rec[: K * per * 8].cpu().numpy().view(smc.RECORD_DTYPE)
    return r, np.array(blocks) / FX, totals


@pytest.mark.parametrize("stepping", [W.SEGMENT, W.SPHERE_TRACING])
@pytest.mark.parametrize("name", list(CONFIGS))
def test_mixed_equals_fp64_within_3_sigma(ctx, name, stepping):
    factory, n, K, block = CONFIGS[name]
    if stepping == W.SPHERE_TRACING and name in ("sphere_pencil", "vessel_network"):
        pytest.skip("sphere tracing is compared on the slab and the container")
    wl = factory().with_stepping(stepping)
    rm, bm, tm = batched(ctx, wl, "mixed", n, K, block)
    rf, bf, tf = batched(ctx, wl, "fp64", n, K, block)
    npk = rm.size
    assert sum(t["packets"] for t in tm) == npk and sum(t["packets"] for t in tf) == npk
    assert sum(t["max_steps_hit"] for t in tm) == 0
    # every reported tally: R, T, A per packet, paired on the same ids
    for key in ("R", "T", "A"):
        z = bench.paired_z(rm[key] / FX, rf[key] / FX)
        assert abs(z) < 3.0, (name, key, rm[key].mean() / FX, rf[key].mean() / FX, z)
    # the whole fluence map, block by block
    s = bench.paired_block_stats(bm, bf)
    assert s["blocks"] >= 50, s
    assert s["pass"], (name, s)
    # energy closes per packet in both (FP32 weights: 1e-4 per packet)
    bal = (rm["R"] + rm["T"] + rm["A"] + rm["killed"] - rm["gain"]) / FX
    assert np.all(np.abs(bal - 1.0) < 1e-4)

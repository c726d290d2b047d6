"""The two 1e8-packet workloads at their full sizes, through the C-ABI.

- Vessel network: 64 capsules in a smooth union inside a 5 mm tissue cube,
  200^3 grid.
- Glass container: a clear glass shell around a turbid liquid, 128^3 grid.

Both runs use segment stepping, as the benchmark does.  The oracle cannot run
1e8 packets, so the full-size results are checked in two ways.

- FP64 kernel, on a random sample of the workload's packet ids: each
  packet's record (R, T, A, killed, gain, scatters, steps) equals the
  oracle's, one by one.
- Mixed kernel, on all 1e8 packets (20 launches of 5e6 consecutive ids):
  - R/T/A agree with an independent oracle sample within 3 sigma of the
    combined error;
  - the fluence map, block by block: one z per voxel block from the batch
    spreads of both sides (Welch), accepted by ``bench.block_stats``;
  - energy closes;
  - no packet reaches the step cap.
The paired comparison with the FP64 kernel on the same ids is in
``test_gpu_parity_blocks.py``.
"""
import math

import numpy as np
import pytest

import bench
import oracle as O
import paper_2112_08035_gb300 as smc
import workloads as W

pytestmark = pytest.mark.gpu

FX = 2.0 ** 32
RECORD_KEYS = ("R", "T", "A", "killed", "gain", "scatters", "steps")

# (workload, voxel block side for the coarse map, oracle sample size)
CASES = [
    ("vessel_network", lambda: W.vessel_network(), 40, 20000),
    ("glass_container", lambda: W.glass_container(), 16, 40000),
]


@pytest.fixture(scope="module")
def ctx():
    c = smc.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("name,make,block,nsample", CASES, ids=[c[0] for c in CASES])
def test_fp64_sampled_packets_full_size(ctx, name, make, block, nsample):
    import torch
    wl = make().with_stepping(W.SEGMENT)
    g = wl.grid
    plan = ctx.plan(wl, "fp64")
    flu = torch.zeros((g.n[2], g.n[1], g.n[0]), dtype=torch.int64, device="cuda")
    tot = smc.totals_tensor()
    rec = torch.zeros(8, dtype=torch.int64, device="cuda")
    rng = np.random.default_rng(11)
    ids = np.sort(rng.choice(wl.npackets, 300, replace=False))
    try:
        for i in ids:
            rec.zero_()
            plan.launch(int(i), 1, wl.seed, flu, tot, rec)
            torch.cuda.synchronize()
            assert plan.status() == 0
            rg = rec.cpu().numpy().view(smc.RECORD_DTYPE)[0]
            _, _, ro = O.run(wl, int(i), int(i) + 1, threads=1, fluence=False, records=True)
            for k in RECORD_KEYS:
                assert rg[k] == ro[k][0], (name, int(i), k, rg[k], ro[k][0])
    finally:
        plan.close()
    assert smc.totals_from_tensor(tot)["packets"] == len(ids)


@pytest.mark.parametrize("name,make,block,nsample", CASES, ids=[c[0] for c in CASES])
def test_mixed_full_size_against_oracle_sample(ctx, name, make, block, nsample):
    import torch
    pytest.importorskip("scipy")
    wl = make().with_stepping(W.SEGMENT)
    N = wl.npackets
    K = 20
    per = N // K
    g = wl.grid
    plan = ctx.plan(wl, "mixed")
    flu = torch.zeros((g.n[2], g.n[1], g.n[0]), dtype=torch.int64, device="cuda")
    acc = torch.zeros_like(flu)
    tot = smc.totals_tensor()
    bg = []
    for k in range(K):
        flu.zero_()
        plan.launch(k * per, per, wl.seed, flu, tot)
        acc += flu
        bg.append(bench.block_sums(flu, (block,) * 3) / FX / per)
    torch.cuda.synchronize()
    assert plan.status() == 0
    plan.close()
    t = smc.totals_from_tensor(tot)
    assert int(acc.min()) >= 0
    del flu, acc
    torch.cuda.empty_cache()
    assert t["packets"] == N
    assert t["max_steps_hit"] == 0, t["max_steps_hit"]
    bal = (t["R"] + t["T"] + t["A"] + t["killed"] - t["gain"]) / FX
    assert abs(bal - N) < 1e-4 * N, (bal, N)

    # independent oracle sample: packet ids far from the GPU's [0, N), in
    # K batches
    po = nsample // K
    base = 4 * N
    ro, bo = [], []
    for k in range(K):
        fo, _, r = O.run(wl.with_packets(po), base + k * po, records=True)
        ro.append(r)
        bo.append(bench.block_sums(fo, (block,) * 3) / FX / po)
    ro = np.concatenate(ro)
    for k in ("R", "T", "A"):
        x = ro[k].astype(np.float64) / FX
        se = math.sqrt(x.var() / x.size * (1.0 + x.size / N))
        z = abs(t[k] / FX / N - x.mean()) / max(se, 1e-12)
        assert z < 3.0, (name, k, t[k] / FX / N, x.mean(), se, z)
    s = bench.block_stats(np.array(bg), np.array(bo), paired=False)
    assert s["blocks"] >= 8 and s["pass"], (name, s)

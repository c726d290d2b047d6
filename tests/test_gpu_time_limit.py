"""Device-side time limit of a launch (smcrt_plan_set_time_limit,
smcrt_set_time_limit).

The limit is tested by making it run out on an ordinary workload: a budget
of a few milliseconds on a launch that needs seconds.  The kernel must come
back quickly, report SMCRT_STATUS_TIMEOUT, and leave totals that close over
the packets it counted.  Nothing waits on a flag that nobody sets and
nothing faults: the warps read the GPU's timer and return."""
import math
import time

import numpy as np
import pytest

import paper_2112_08035_gb300 as smc
import workloads as W

pytestmark = pytest.mark.gpu

FX = 2.0 ** 32


@pytest.fixture(scope="module")
def ctx():
    c = smc.Context(0)
    yield c
    c.close()


def _launch(ctx, wl, precision, limit):
    import torch
    g = wl.grid
    plan = ctx.plan(wl, precision)
    plan.set_time_limit(limit)
    flu = torch.zeros((g.n[2], g.n[1], g.n[0]), dtype=torch.int64, device="cuda")
    tot = smc.totals_tensor()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan.launch(0, wl.npackets, wl.seed, flu, tot)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    st = plan.status()
    plan.close()
    return flu.cpu().numpy(), smc.totals_from_tensor(tot), st, dt


def _closes(t):
    # every fixed-point deposit rounds by at most half a unit
    bal = t["R"] + t["T"] + t["A"] + t["killed"] - t["gain"] - t["packets"] * FX
    return abs(bal) <= 0.5 * (t["scatters"] + 3 * t["packets"]) + 1


@pytest.mark.parametrize("precision,npackets", [("mixed", 200_000_000), ("fp64", 20_000_000)])
def test_time_limit_runs_out(ctx, precision, npackets):
    # about 4 s (mixed) or 13 s (FP64) of work against a 5 ms budget
    wl = W.three_layer_slab(npackets, grid_n=50).with_stepping(W.SEGMENT)
    flu, t, st, dt = _launch(ctx, wl, precision, 0.005)
    assert st & smc.STATUS_TIMEOUT, st
    assert dt < 1.0, dt
    assert 0 < t["packets"] < npackets
    assert _closes(t), t
    assert flu.min() >= 0 and flu.sum() > 0


def test_generous_limit_changes_nothing(ctx):
    wl = W.glass_container(200_000, grid_n=32).with_stepping(W.SEGMENT)
    f0, t0, s0, _ = _launch(ctx, wl, "mixed", 0.0)
    f1, t1, s1, _ = _launch(ctx, wl, "mixed", 30.0)
    assert s0 == 0 and s1 == 0
    assert np.array_equal(f0, f1)
    for k in ("R", "T", "A", "killed", "gain", "packets", "scatters", "steps"):
        assert t0[k] == t1[k], k


def test_context_time_limit_on_run():
    c = smc.Context(0)
    try:
        wl = W.three_layer_slab(100_000_000, grid_n=20)
        c.set_time_limit(0.002)
        with pytest.raises(smc.SmcrtError) as e:
            c.run(wl, "mixed")
        assert e.value.code == smc.ERR_TIMEOUT
        # lifted again: the same context runs to completion
        c.set_time_limit(0.0)
        _, t = c.run(wl.with_packets(100_000), "mixed")
        assert t["packets"] == 100_000
        for bad in (-1.0, math.nan, math.inf):
            with pytest.raises(smc.SmcrtError) as e:
                c.set_time_limit(bad)
            assert e.value.code == smc.ERR_BAD_ARG
    finally:
        c.close()

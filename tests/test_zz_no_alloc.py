"""smcrt_run_noalloc: the packet launch for callers that may not allocate
device memory (their own pool owns the device, or an allocation's possible
device synchronisation is not allowed where they call from).  Its scratch is
a fixed array inside the library instead of cudaMalloc'd buffers.

The test calls it through the C-ABI twice in a row -- on two different
scenes, so the second call must overwrite what the first left in the shared
array -- and checks both results against smcrt_plan_launch of the same
packets.  Both go through the same kernel with the same packet ids, so the
tolerance is zero: fluence and totals must be identical.  This file is
collected last on purpose."""
import numpy as np
import pytest

import paper_2112_08035_gb300 as smc
import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("R", "T", "A", "killed", "gain", "packets", "scatters", "steps", "pieces", "interfaces", "fresnel")


def _buffers(wl):
    import torch
    g = wl.grid
    return (torch.zeros((g.n[2], g.n[1], g.n[0]), dtype=torch.int64, device="cuda"), smc.totals_tensor())


def _with_plan(ctx, wl, precision):
    import torch
    flu, tot = _buffers(wl)
    plan = ctx.plan(wl, precision)
    plan.launch(0, wl.npackets, wl.seed, flu, tot)
    torch.cuda.synchronize()
    plan.close()
    return flu.cpu().numpy(), smc.totals_from_tensor(tot)


def _no_alloc(wl, precision):
    import torch
    flu, tot = _buffers(wl)
    smc.run_noalloc(wl, 0, wl.npackets, wl.seed, flu, tot, precision)
    torch.cuda.synchronize()
    return flu.cpu().numpy(), smc.totals_from_tensor(tot)


def test_no_alloc_matches_plan_launch_on_two_calls():
    import torch
    torch.cuda.set_device(0)
    ctx = smc.Context(0)
    try:
        cases = [(W.three_layer_slab(40_000, grid_n=40), "mixed"),
                 (W.glass_container(20_000, grid_n=32), "fp64")]
        want = [_with_plan(ctx, wl, p) for wl, p in cases]
        got = [_no_alloc(wl, p) for wl, p in cases]   # two calls in a row
        for (fw, tw), (fg, tg), (wl, p) in zip(want, got, cases):
            assert np.array_equal(fg, fw), (wl.name, p)
            for k in KEYS:
                assert tg[k] == tw[k], (wl.name, p, k)
            assert tg["packets"] == wl.npackets
    finally:
        ctx.close()


def test_no_alloc_rejects_scenes_beyond_its_scratch():
    wl = W.vessel_network(10, grid_n=8, ncap=130)   # 131 primitives > 128
    flu, tot = _buffers(wl)
    with pytest.raises(smc.SmcrtError) as e:
        smc.run_noalloc(wl, 0, 10, 1, flu, tot, "mixed")
    assert e.value.code == smc.ERR_NO_MEMORY

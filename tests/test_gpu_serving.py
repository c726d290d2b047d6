"""Serving: continuously batched jobs through smcrt_submit / poll / wait.

Each packet's history depends only on (seed, packet id) and every tally is
an int64 sum, so a job's result is the same alone and in any mix: the
test requires bit-identical fluence and totals (a tolerance of zero)."""
import time

import numpy as np
import pytest

import paper_2112_08035_gb300 as smc
import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("R", "T", "A", "killed", "gain", "packets", "scatters", "steps")


@pytest.fixture(scope="module")
def ctx():
    c = smc.Context(0)
    yield c
    c.close()


def _jobs():
    return [W.sphere_pencil(30_000, 11, "mixed"), W.three_layer_slab(200_000, 12, "mixed", grid_n=64),
            W.glass_container(50_000, 13, "mixed", grid_n=50), W.vessel_network(5_000, 3, "mixed", grid_n=50),
            W.sphere_pencil(20_000, 14, "fp64"), W.three_layer_slab(7, 15, "fp64", grid_n=10),
            W.glass_container(40_000, 16, "mixed", grid_n=50).with_stepping(W.SEGMENT),
            W.three_layer_slab(3_000, 17, "fp64", grid_n=20).with_stepping(W.SEGMENT),
            W.sdf_gallery(20_000, 18, "mixed", grid_n=20), W.sdf_gallery(300, 19, "fp64", grid_n=12)]


def test_same_result_alone_and_in_the_mix(ctx):
    jobs = _jobs()
    alone = [ctx.run(j, j.precision) for j in jobs]
    ids = [ctx.submit(j) for j in jobs]
    got = [ctx.wait(i, 300.0) for i in ids]
    for (fa, ta), (fm, tm, lat), j in zip(alone, got, jobs):
        assert np.array_equal(fa, fm), j.name
        for k in KEYS:
            assert ta[k] == tm[k], (j.name, k)
        assert lat > 0


def test_staggered_arrivals_and_poll(ctx):
    jobs = _jobs()[:4]
    ids = []
    for j in jobs:
        ids.append(ctx.submit(j))
        time.sleep(0.01)
    deadline = time.time() + 300
    while not all(ctx.poll(i) for i in ids):
        assert time.time() < deadline
        time.sleep(0.005)
    for i, j in zip(ids, jobs):
        f, t, _ = ctx.wait(i, 1.0)
        assert t["packets"] == j.npackets


def test_cancel_and_errors(ctx):
    big = W.vessel_network(20_000_000, 3, "mixed", grid_n=32)
    jid = ctx.submit(big)
    ctx.cancel(jid)
    with pytest.raises(smc.SmcrtError) as e:
        ctx.wait(jid, 300.0)
    assert e.value.code == smc.ERR_CANCELLED
    with pytest.raises(smc.SmcrtError) as e:
        ctx.wait(123456789, 0.0)
    assert e.value.code == smc.ERR_NOT_FOUND
    # a zero-packet job completes at once with zero tallies
    z = ctx.submit(W.sphere_pencil(0, 1, "mixed"))
    f, t, _ = ctx.wait(z, 10.0)
    assert t["packets"] == 0 and not f.any()
    # the server keeps working after a cancellation
    j = W.sphere_pencil(5_000, 21, "mixed")
    fa, ta = ctx.run(j, "mixed")
    f, t, _ = ctx.wait(ctx.submit(j), 60.0)
    assert np.array_equal(f, fa) and t["A"] == ta["A"]


def test_timeout_keeps_job(ctx):
    big = W.glass_container(3_000_000, 5, "mixed", grid_n=32)
    jid = ctx.submit(big)
    try:
        ctx.wait(jid, 0.0)
        timed_out = False
    except smc.SmcrtError as e:
        assert e.code == smc.ERR_TIMEOUT
        timed_out = True
    if timed_out:
        f, t, _ = ctx.wait(jid, 300.0)
        assert t["packets"] == big.npackets


_SETUP_FAILURE_CHILD = r"""
import sys
sys.path.insert(0, sys.argv[1])
import paper_2112_08035_gb300 as smc
import workloads as W
ctx = smc.Context(0)
jid = ctx.submit(W.sphere_pencil(1000, 1, "mixed"))
try:
    ctx.wait(jid, 60.0)
    print("waited: no error")
except smc.SmcrtError as e:
    print("wait error", e.code)
try:
    ctx.submit(W.sphere_pencil(1000, 2, "mixed"))
    print("submitted: no error")
except smc.SmcrtError as e:
    print("submit error", e.code)
ctx.close()
print("closed")
"""


def test_scheduler_setup_failure_fails_jobs_cleanly():
    # a host-side injected allocation failure in the scheduler's setup: the
    # queued job completes with the error, later submissions return it at
    # once, and the context closes (no GPU fault is involved)
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, SMCRT_FAULT_SCHEDULER_SETUP="1")
    r = subprocess.run([sys.executable, "-c", _SETUP_FAILURE_CHILD, root], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.split("\n")
    assert f"wait error {smc.ERR_NO_MEMORY}" in lines, r.stdout
    assert f"submit error {smc.ERR_NO_MEMORY}" in lines, r.stdout
    assert "closed" in lines, r.stdout


_BAD_JOB_CHILD = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import paper_2112_08035_gb300 as smc
import workloads as W
ctx = smc.Context(0)
good = W.sphere_pencil(20_000, 31, "mixed")
fa, ta = ctx.run(good, "mixed")
bad_id = ctx.submit(W.three_layer_slab(50_000, 32, "mixed", grid_n=20))   # job 1: no scene in the round table
good_id = ctx.submit(good)                                                  # job 2, in the same rounds
for name, jid in (("bad", bad_id), ("good", good_id)):
    try:
        f, t, _ = ctx.wait(jid, 120.0)
        same = bool(np.array_equal(f, fa) and t["A"] == ta["A"] and t["packets"] == good.npackets)
        print(name, "ok", same)
    except smc.SmcrtError as e:
        print(name, "error", e.code)
# a later job on the same server
f, t, _ = ctx.wait(ctx.submit(good), 120.0)
print("later ok", bool(np.array_equal(f, fa)))
ctx.close()
print("closed")
"""


def test_bad_job_fails_alone():
    # a job the kernel flags (its round-table entry carries no scene, injected
    # on the host) fails with SMCRT_ERR_DEVICE; the good job in the same
    # rounds, and a later one, complete normally with their exact results:
    # each job has its own status word and the round's word is cleared
    # before every round (no GPU fault is involved)
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, SMCRT_FAULT_BAD_JOB="1")
    r = subprocess.run([sys.executable, "-c", _BAD_JOB_CHILD, root], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.split("\n")
    assert f"bad error {smc.ERR_DEVICE}" in lines, r.stdout
    assert "good ok True" in lines, r.stdout
    assert "later ok True" in lines, r.stdout
    assert "closed" in lines, r.stdout

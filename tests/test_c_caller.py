"""The C-ABI called from C: a plain C program (``c_caller/smcrt_c_caller.c``)
compiled with gcc against ``include/smcrt.h`` and the built library.  On the
CPU the test only builds it (the header is valid C11, the program links);
on the GPU it runs it and compares every integer tally, and a checksum of
the fluence map, with the same runs made through the Python binding: bit for
bit, in FP64, in mixed precision, and for a job through the serving calls."""
import os
import platform
import subprocess

import numpy as np
import pytest

import paper_2112_08035_gb300 as smc
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_caller", "smcrt_c_caller.c")
LIBDIR = os.path.join(ROOT, "paper_2112_08035_gb300", "_build")
KEYS = ("R", "T", "A", "killed", "gain", "packets", "scatters", "steps")


def _build(tmp_path):
    smc.build()
    exe = os.path.join(str(tmp_path), "smcrt_c_caller")
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", f"-I{os.path.join(ROOT, 'include')}",
                           SRC, f"-L{LIBDIR}", f"-l:libsmcrt_{platform.machine()}.so",
                           f"-Wl,-rpath,{LIBDIR}", "-o", exe])
    return exe


def test_c_caller_builds(tmp_path):
    assert os.path.exists(_build(tmp_path))


def _checksum(flu):
    f = flu.ravel().astype(np.uint64)
    idx = np.arange(1, f.size + 1, dtype=np.uint64)
    s0 = int(flu.astype(np.int64).sum())
    s1 = int(np.sum(f * idx, dtype=np.uint64).astype(np.int64))
    return s0, s1


@pytest.mark.gpu
@pytest.mark.parametrize("stepping", [W.SPHERE_TRACING, W.SEGMENT])
def test_c_caller_matches_binding(tmp_path, stepping):
    exe = _build(tmp_path)
    n = 50_000
    r = subprocess.run([exe, str(n), "1" if stepping == W.SEGMENT else "0"], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    got = {}
    for line in r.stdout.split("\n"):
        f = line.split()
        if f:
            got[f[0]] = [int(v) for v in f[1:]]
    wl = W.sphere_pencil(n).with_stepping(stepping)
    ctx = smc.Context(0)
    try:
        want = {}
        for name, prec in (("run_fp64", "fp64"), ("run_mixed", "mixed")):
            flu, t = ctx.run(wl, prec)
            want[name] = [t[k] for k in KEYS] + list(_checksum(flu))
        jid = ctx.submit(wl, "mixed")
        flu, t, _ = ctx.wait(jid)
        want["served_mixed"] = [t[k] for k in KEYS] + list(_checksum(flu))
    finally:
        ctx.close()
    for name in ("run_fp64", "run_mixed", "served_mixed"):
        assert got[name] == want[name], (name, got.get(name), want[name])
    # a served job equals the same job run alone, bit for bit
    assert got["served_mixed"] == got["run_mixed"]

"""C-ABI boundary checks that need no GPU: the library builds and loads,
exports every function include/smcrt.h declares, its struct layouts match
the Python binding, and host-side validation rejects malformed scenes
(host-side fault injection: corrupt inputs return error codes)."""
import ctypes as C
import os
import re
import subprocess
from dataclasses import replace

import pytest

import paper_2112_08035_gb300 as smc
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "smcrt.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(smcrt_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    L = smc.lib()
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", smc.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (smcrt_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(L, n)


def test_struct_layouts_match_header(tmp_path):
    probe = tmp_path / "probe.c"
    probe.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "smcrt.h"\n'
                     "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\","
                     "sizeof(smcrt_prim), sizeof(smcrt_csg_node), sizeof(smcrt_region), sizeof(smcrt_scene),"
                     "sizeof(smcrt_source), sizeof(smcrt_grid), sizeof(smcrt_totals), sizeof(smcrt_packet_record),"
                     "offsetof(smcrt_scene, delta), sizeof(smcrt_xform), offsetof(smcrt_scene, xforms));return 0;}\n")
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [C.sizeof(smc.Prim), C.sizeof(smc.CsgNode), C.sizeof(smc.Region), C.sizeof(smc.Scene),
            C.sizeof(smc.Source), C.sizeof(smc.Grid), C.sizeof(smc.Totals), smc.RECORD_DTYPE.itemsize,
            smc.Scene.delta.offset, C.sizeof(smc.Xform), smc.Scene.xforms.offset]
    assert got == want


def test_version_and_strerror():
    L = smc.lib()
    assert L.smcrt_version() >= 10000
    for code in range(0, -9, -1):
        assert len(L.smcrt_strerror(code)) > 0
    assert L.smcrt_strerror(-99) == b"unknown status"


@pytest.mark.parametrize("wl", W.all_configs(), ids=lambda w: w.name)
def test_configs_validate(wl):
    assert smc.validate(wl) >= 1


def _bad(wl):
    with pytest.raises(smc.SmcrtError) as e:
        smc.validate(wl)
    return e.value.code


def test_validation_rejects_corrupt_scenes():
    wl = W.sphere_pencil(10)
    sc = wl.scene
    reg = sc.regions[0]
    cases = [
        replace(wl, scene=replace(sc, delta=0.0)),
        replace(wl, scene=replace(sc, delta=-1e-6)),
        replace(wl, scene=replace(sc, max_steps=0)),
        replace(wl, scene=replace(sc, ambient_n=0.5)),
        replace(wl, scene=replace(sc, bbox_lo=(2.0, -1, -1))),
        replace(wl, scene=replace(sc, regions=(replace(reg, g=1.0),))),
        replace(wl, scene=replace(sc, regions=(replace(reg, g=-1.2),))),
        replace(wl, scene=replace(sc, regions=(replace(reg, n=0.9),))),
        replace(wl, scene=replace(sc, regions=(replace(reg, mu_a=-1.0),))),
        replace(wl, scene=replace(sc, regions=(replace(reg, mu_s=float("nan")),))),
        replace(wl, scene=replace(sc, prims=(W.Prim(W.SPHERE, (0, 0, 0, -1.0)),))),
        replace(wl, scene=replace(sc, prims=(W.Prim(W.CAPSULE, (0, 0, 0, 0, 0, 0, 0.1)),))),
        # CSG stack underflow, a dangling operand, an out-of-range primitive
        replace(wl, scene=replace(sc, regions=(replace(reg, program=(W.Node(W.PRIM, 0), W.Node(W.UNION))),))),
        replace(wl, scene=replace(sc, regions=(replace(reg, program=(W.Node(W.PRIM, 0), W.Node(W.PRIM, 0))),))),
        replace(wl, scene=replace(sc, regions=(replace(reg, program=(W.Node(W.PRIM, 3),)),))),
        # smooth union needs k > 0
        replace(wl, scene=replace(sc, regions=(replace(reg, program=(W.Node(W.PRIM, 0), W.Node(W.PRIM, 0),
                                                                     W.Node(W.SMOOTH_UNION, -1, 0.0))),))),
        replace(wl, source=replace(wl.source, dir=(0.0, 0.0, -2.0))),
        replace(wl, source=W.Source(W.DISC, (0, 0, 1.2), (0, 0, -1.0), 0.0)),
        replace(wl, grid=W.Grid((-1, -1, -1), (1, 1, 1), (0, 4, 4))),
        replace(wl, grid=W.Grid((-1, -1, -1), (1, 1, 1), (2000, 4, 4))),
        replace(wl, grid=W.Grid((1, -1, -1), (-1, 1, 1), (4, 4, 4))),
    ]
    for c in cases:
        assert _bad(c) == smc.ERR_BAD_SCENE


def test_validation_of_shapes_and_frames():
    wl = W.sdf_gallery(10, grid_n=8)
    assert smc.validate(wl) >= 1
    sc = wl.scene

    def with_prim(i, prim):
        prims = list(sc.prims)
        prims[i] = prim
        return replace(wl, scene=replace(sc, prims=tuple(prims)))
    tor, cyl, box = sc.prims[1], sc.prims[7], sc.prims[2]
    X = box.xform
    reflect = (1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, -1.0)
    skewed = (1.0, 0.1, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0)
    cases = [
        with_prim(1, replace(tor, params=(0.0, 0.0, 0.0, 0.2, 0.3))),          # tube wider than the ring
        with_prim(1, replace(tor, params=(0.0, 0.0, 0.0, 0.5, 0.0))),
        with_prim(7, replace(cyl, params=(0.0, 0.0, 0.0, 0.2, -0.1))),
        with_prim(2, replace(box, xform=replace(X, rot=reflect))),              # det -1
        with_prim(2, replace(box, xform=replace(X, rot=skewed))),               # not orthonormal
        with_prim(2, replace(box, xform=replace(X, s=0.0))),
        with_prim(2, replace(box, xform=replace(X, s=float("inf")))),
        with_prim(2, replace(box, xform=replace(X, op=W.REPEAT, a=(0.3, 0.3, 0.0, 1.5)))),   # fractional count
        with_prim(2, replace(box, xform=replace(X, op=W.ELONGATE, a=(-0.1, 0.0, 0.0, 0.0)))),
        with_prim(2, replace(box, xform=replace(X, op=W.TWIST, a=(0.2, -1.0, 0.0, 0.0)))),
    ]
    for c in cases:
        assert _bad(c) == smc.ERR_BAD_SCENE


def test_csg_stack_depth_limit():
    # n nested operands need n - 1 register slots (the last primitive fuses
    # with its operator): 5 compiles, 6 exceeds the 4-deep device stack
    s = W.Prim(W.SPHERE, (0, 0, 0, 1.0))

    def nested(depth):
        prog = [W.Node(W.PRIM, 0)] * depth + [W.Node(W.UNION)] * (depth - 1)
        return replace(W.sphere_pencil(1), scene=replace(W.sphere_pencil(1).scene, prims=(s,),
                                                         regions=(W.Region(tuple(prog), 1, 1, 0.5, 1.3),)))
    assert smc.validate(nested(4)) == 6   # 3 pushes + 1 fused union + 2 stack ops
    assert smc.validate(nested(5)) == 8
    assert _bad(nested(6)) == smc.ERR_BAD_SCENE


def test_null_arguments():
    L = smc.lib()
    assert L.smcrt_validate(None, None, None, None) == smc.ERR_BAD_ARG
    assert L.smcrt_destroy(None) == smc.ERR_BAD_ARG
    assert L.smcrt_plan_destroy(None) == smc.ERR_BAD_ARG
    assert L.smcrt_poll(None, 1, None) == smc.ERR_BAD_ARG

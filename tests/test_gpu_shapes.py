"""Tori, capped cylinders, primitive frames and domain operations on the GPU
(Sec. 2.2, the Fig. 1 gallery as a transport scene), through the C-ABI.

FP64 mode performs the oracle's operations: every tally bit-identical, with
either step rule.  Mixed mode: R, T, A within Monte Carlo error of the
oracle, energy closed per packet.  These scenes run the kernels' general
instantiation; plain scenes keep the specialised one.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_2112_08035_gb300 as smc
import workloads as W

pytestmark = pytest.mark.gpu

FX = 2.0 ** 32


@pytest.fixture(scope="module")
def ctx():
    c = smc.Context(0)
    yield c
    c.close()


def run_gpu(ctx, wl, precision, records=False, id_begin=0):
    import torch
    plan = ctx.plan(wl, precision)
    g = wl.grid
    flu = torch.zeros((g.n[2], g.n[1], g.n[0]), dtype=torch.int64, device="cuda")
    tot = smc.totals_tensor()
    rec = torch.zeros(wl.npackets * 8, dtype=torch.int64, device="cuda") if records else None
    plan.launch(id_begin, wl.npackets, wl.seed, flu, tot, rec)
    torch.cuda.synchronize()
    assert plan.status() == 0
    plan.close()
    out = (flu.cpu().numpy(), smc.totals_from_tensor(tot))
    if records:
        out = out + (rec.cpu().numpy().view(smc.RECORD_DTYPE),)
    return out


def _one_shape(prim, n_region=1.45):
    # one placed shape in a clear-ish tissue block, beam from above
    block = W.Prim(W.BOX, (0.0, 0.0, -1.0, 1.5, 1.5, 1.0))
    regions = (W.Region(W.prim_program([0]), 0.3, 15.0, 0.8, 1.37),
               W.Region(W.prim_program([1]), 1.0, 40.0, 0.9, n_region))
    scene = W.Scene((block, prim), regions, 1.0, (-1.6, -1.6, -2.1), (1.6, 1.6, 0.2))
    return W.Workload("shape", scene, W.Source(W.DISC, (0.0, 0.0, 0.1), (0.0, 0.0, -1.0), 0.8),
                      W.Grid((-1.5, -1.5, -2.0), (1.5, 1.5, 0.0), (16, 16, 16)), 400, 9, "fp64")


SHAPES = {
    "torus": W.Prim(W.TORUS, (0.0, 0.0, 0.0, 0.5, 0.2), W.Xform(rot=W.rotation((1, 0, 0), 60.0), t=(0.0, 0.0, -1.0))),
    "cylinder_scaled": W.Prim(W.CYLINDER, (0.0, 0.0, 0.0, 0.3, 0.3), W.Xform(t=(0.1, 0.0, -1.0), s=1.5)),
    "box_rotated": W.Prim(W.BOX, (0.0, 0.0, 0.0, 0.6, 0.3, 0.2), W.Xform(rot=W.rotation((1, 2, 3), 40.0),
                                                                        t=(0.0, 0.2, -0.9))),
    "twist": W.Prim(W.BOX, (0.0, 0.0, 0.0, 0.3, 0.15, 0.6),
                    W.Xform(t=(0.0, 0.0, -1.0), op=W.TWIST, a=(0.3, 0.34, 0.0, 0.0))),
    "bend": W.Prim(W.BOX, (0.0, 0.0, 0.0, 0.8, 0.15, 0.2),
                   W.Xform(t=(0.0, 0.0, -1.0), op=W.BEND, a=(0.2, 0.82, 0.0, 0.0))),
    "elongate": W.Prim(W.SPHERE, (0.0, 0.0, 0.0, 0.25), W.Xform(t=(0.0, 0.0, -0.8), op=W.ELONGATE,
                                                                a=(0.4, 0.2, 0.0, 0.0))),
    "repeat": W.Prim(W.SPHERE, (0.0, 0.0, 0.0, 0.1), W.Xform(t=(0.0, 0.0, -0.6), op=W.REPEAT,
                                                             a=(0.3, 0.3, 0.0, 2.0))),
    "cylinder_plain": W.Prim(W.CYLINDER, (0.0, 0.0, -1.0, 0.4, 0.3)),
    "torus_plain": W.Prim(W.TORUS, (0.1, 0.0, -1.0, 0.5, 0.2)),
}


def _smooth_blob(n=400, precision="fp64"):
    """Spheres and capsules joined by smooth unions, one sphere given twice
    (the fold then reaches past k/4 below the plain union), in a tissue
    block lit from above.  Under segment stepping the region is bounded
    along rays with a margin of k/4 per smooth union."""
    prims = (W.Prim(W.BOX, (0.0, 0.0, -1.0, 1.5, 1.5, 1.0)),
             W.Prim(W.SPHERE, (0.0, 0.0, -0.8, 0.35)), W.Prim(W.SPHERE, (0.3, 0.1, -0.9, 0.3)),
             W.Prim(W.SPHERE, (0.0, 0.0, -0.8, 0.35)),
             W.Prim(W.CAPSULE, (-0.6, -0.2, -1.2, 0.5, 0.3, -1.3, 0.12)),
             W.Prim(W.CAPSULE, (0.0, -0.7, -0.6, 0.0, 0.7, -0.7, 0.1)))
    prog = (W.Node(W.PRIM, 1), W.Node(W.PRIM, 2), W.Node(W.SMOOTH_UNION, -1, 0.15), W.Node(W.PRIM, 3),
            W.Node(W.SMOOTH_UNION, -1, 0.15), W.Node(W.PRIM, 4), W.Node(W.SMOOTH_UNION, -1, 0.1),
            W.Node(W.PRIM, 5), W.Node(W.UNION))
    regions = (W.Region(W.prim_program([0]), 0.3, 15.0, 0.8, 1.37), W.Region(prog, 1.0, 30.0, 0.9, 1.45))
    scene = W.Scene(prims, regions, 1.0, (-1.6, -1.6, -2.1), (1.6, 1.6, 0.2))
    return W.Workload("smooth_blob", scene, W.Source(W.DISC, (0.0, 0.0, 0.1), (0.0, 0.0, -1.0), 0.8),
                      W.Grid((-1.5, -1.5, -2.0), (1.5, 1.5, 0.0), (16, 16, 16)), n, 9, precision)


@pytest.mark.parametrize("stepping", [W.SPHERE_TRACING, W.SEGMENT])
def test_fp64_bitexact_smooth_fold(ctx, stepping):
    wl = _smooth_blob().with_stepping(stepping)
    fo, to, ro = O.run(wl, records=True)
    fg, tg, rg = run_gpu(ctx, wl, "fp64", records=True)
    for k in ("R", "T", "A", "killed", "gain", "packets", "scatters", "steps"):
        assert tg[k] == to[k], (k, tg[k], to[k])
    assert np.array_equal(fg, fo)
    for f in ("R", "T", "A", "killed", "gain", "scatters", "steps"):
        assert np.array_equal(rg[f], ro[f]), f


def test_mixed_smooth_fold_matches_oracle(ctx):
    wl = _smooth_blob(precision="mixed")
    _, _, ro = O.run(wl.with_packets(6000), records=True)
    _, tg, rg = run_gpu(ctx, wl.with_packets(200_000).with_stepping(W.SEGMENT), "mixed", records=True,
                        id_begin=5_000_000)
    for key in ("R", "T", "A"):
        assert abs(_z(rg, ro, key)) < 4.0, (key, _z(rg, ro, key))
    bal = (rg["R"] + rg["T"] + rg["A"] + rg["killed"] - rg["gain"]) / FX
    assert np.all(np.abs(bal - 1.0) < 1e-4)
    assert tg["max_steps_hit"] == 0


@pytest.mark.parametrize("stepping", [W.SPHERE_TRACING, W.SEGMENT])
@pytest.mark.parametrize("name", list(SHAPES))
def test_fp64_bitexact_shapes(ctx, name, stepping):
    wl = _one_shape(SHAPES[name]).with_stepping(stepping)
    fo, to, ro = O.run(wl, records=True)
    fg, tg, rg = run_gpu(ctx, wl, "fp64", records=True)
    for k in ("R", "T", "A", "killed", "gain", "packets", "scatters", "steps"):
        assert tg[k] == to[k], (name, k, tg[k], to[k])
    assert np.array_equal(fg, fo)
    for f in ("R", "T", "A", "killed", "gain", "scatters", "steps"):
        assert np.array_equal(rg[f], ro[f]), f


@pytest.mark.parametrize("stepping", [W.SPHERE_TRACING, W.SEGMENT])
def test_fp64_bitexact_gallery(ctx, stepping):
    wl = W.sdf_gallery(600, grid_n=24, precision="fp64").with_stepping(stepping)
    fo, to, _ = O.run(wl)
    fg, tg = run_gpu(ctx, wl, "fp64")
    for k in ("R", "T", "A", "killed", "gain", "packets", "scatters", "steps"):
        assert tg[k] == to[k], (k, tg[k], to[k])
    assert np.array_equal(fg, fo)


def _z(rg, ro, key):
    a, b = rg[key] / FX, ro[key] / FX
    se = math.sqrt(a.var() / a.size + b.var() / b.size)
    return (a.mean() - b.mean()) / se if se > 0 else 0.0


@pytest.mark.parametrize("stepping", [W.SPHERE_TRACING, W.SEGMENT])
def test_mixed_gallery_matches_oracle(ctx, stepping):
    wl = W.sdf_gallery(grid_n=24)
    _, _, ro = O.run(wl.with_packets(6000), records=True)
    _, tg, rg = run_gpu(ctx, wl.with_packets(200_000).with_stepping(stepping), "mixed", records=True,
                        id_begin=5_000_000)
    for key in ("R", "T", "A"):
        assert abs(_z(rg, ro, key)) < 4.0, (key, _z(rg, ro, key))
    bal = (rg["R"] + rg["T"] + rg["A"] + rg["killed"] - rg["gain"]) / FX
    assert np.all(np.abs(bal - 1.0) < 1e-4)
    assert tg["max_steps_hit"] == 0


def test_plain_and_general_kernels_agree_on_plain_scene(ctx):
    # a plain scene given a placed primitive with the identity frame takes
    # the general instantiation; the physics (and, in FP64, every bit) is
    # the same
    wl = W.sphere_pencil(3000)
    s = wl.scene
    framed = W.Prim(s.prims[0].kind, (0.0, 0.0, 0.0, s.prims[0].params[3]),
                    W.Xform(t=tuple(s.prims[0].params[:3])))
    wl2 = W.Workload(wl.name, W.Scene((framed,), s.regions, s.ambient_n, s.bbox_lo, s.bbox_hi), wl.source,
                     wl.grid, wl.npackets, wl.seed, "fp64")
    f1, t1 = run_gpu(ctx, wl, "fp64")
    f2, t2 = run_gpu(ctx, wl2, "fp64")
    assert np.array_equal(f1, f2)
    for k in ("R", "T", "A", "scatters", "steps"):
        assert t1[k] == t2[k], k

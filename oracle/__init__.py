"""ctypes wrapper around the FP64 CPU oracle (``smcrt_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  This module marshals
the neutral descriptions of ``workloads`` into the oracle's private C
structs; it shares nothing with the CUDA package.

Parallelism: packets are independent and every tally is an int64
fixed-point sum, so packet-id ranges run on separate threads (ctypes drops
the GIL) and their tallies are summed exactly; the result does not depend
on the thread count.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smcrt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")
_lib = None
_lock = threading.Lock()

FX = 2.0 ** 32  # fixed-point scale of every tally


class OrPrim(C.Structure):
    _fields_ = [("kind", C.c_int32), ("xform", C.c_int32), ("p", C.c_double * 7)]


class OrXform(C.Structure):
    _fields_ = [("rot", C.c_double * 9), ("t", C.c_double * 3), ("s", C.c_double), ("op", C.c_int32),
                ("pad", C.c_int32), ("a", C.c_double * 4)]


class OrNode(C.Structure):
    _fields_ = [("op", C.c_int32), ("prim", C.c_int32), ("k", C.c_double)]


class OrRegion(C.Structure):
    _fields_ = [("begin", C.c_int32), ("count", C.c_int32), ("mu_a", C.c_double),
                ("mu_s", C.c_double), ("g", C.c_double), ("n", C.c_double)]


class OrScene(C.Structure):
    _fields_ = [("prims", C.POINTER(OrPrim)), ("nprims", C.c_int32),
                ("nodes", C.POINTER(OrNode)), ("nnodes", C.c_int32),
                ("regions", C.POINTER(OrRegion)), ("nregions", C.c_int32),
                ("ambient_n", C.c_double), ("bbox_lo", C.c_double * 3),
                ("bbox_hi", C.c_double * 3), ("delta", C.c_double), ("max_steps", C.c_int64),
                ("stepping", C.c_int32), ("pad", C.c_int32),
                ("xforms", C.POINTER(OrXform)), ("nxforms", C.c_int32), ("pad2", C.c_int32)]


class OrSource(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("pos", C.c_double * 3),
                ("dir", C.c_double * 3), ("radius", C.c_double)]


class OrGrid(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("n", C.c_int32 * 3),
                ("pad", C.c_int32)]


TOTAL_FIELDS = ["R", "T", "A", "killed", "gain", "packets", "scatters", "steps", "scene_evals",
                "prog_evals", "prim_evals", "interfaces", "fresnel", "pieces", "max_steps_hit",
                "prim_sphere", "prim_box", "prim_capsule", "prim_torus", "prim_cylinder", "smooth_ops",
                "seg_calls", "seg_sphere", "seg_box", "seg_capsule", "seg_torus", "seg_cylinder", "seg_moves",
                "seg_dist_sphere", "seg_dist_box", "seg_dist_capsule", "seg_dist_torus", "seg_dist_cylinder"]


class OrTotals(C.Structure):
    _fields_ = [(f, C.c_int64) for f in TOTAL_FIELDS]


PACKET_FIELDS = ["R", "T", "A", "killed", "gain", "scatters", "steps", "pad"]
PACKET_DTYPE = np.dtype([(f, np.int64) for f in PACKET_FIELDS])

_PRIM_KIND = {W.SPHERE: 0, W.BOX: 1, W.CAPSULE: 2, W.TORUS: 3, W.CYLINDER: 4}
_XF_OP = {W.XF_NONE: 0, W.ELONGATE: 1, W.TWIST: 2, W.BEND: 3, W.REPEAT: 4}
_OP = {W.PRIM: 0, W.UNION: 1, W.SMOOTH_UNION: 2, W.INTERSECT: 3, W.SUBTRACT: 4}
_SRC_KIND = {W.PENCIL: 0, W.DISC: 1, W.SQUARE: 2, W.ISO_POINT: 3}
_STEPPING = {W.SPHERE_TRACING: 0, W.SEGMENT: 1}


def build(force: bool = False) -> str:
    """Compile the oracle for this host (gcc, FP contraction off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB (tests only): load a deliberately broken build to
            # check that the pins catch it
            path = os.environ.get("ORACLE_LIB") or build()
            L = C.CDLL(path)
            L.or_run.restype = C.c_int
            L.or_run.argtypes = [C.POINTER(OrScene), C.POINTER(OrSource), C.POINTER(OrGrid),
                                 C.c_uint64, C.c_uint64, C.c_uint64, C.c_void_p,
                                 C.POINTER(OrTotals), C.c_void_p]
            L.or_log.restype = C.c_double
            L.or_log.argtypes = [C.c_double]
            L.or_sincos2pi.restype = None
            L.or_sincos2pi.argtypes = [C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.or_philox4x32_10.restype = None
            L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                           C.POINTER(C.c_uint32)]
            L.or_hg_cos.restype = C.c_double
            L.or_hg_cos.argtypes = [C.c_double, C.c_double]
            L.or_fresnel.restype = C.c_double
            L.or_fresnel.argtypes = [C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double)]
            L.or_scatter_dir.restype = None
            L.or_scatter_dir.argtypes = [C.POINTER(C.c_double), C.c_double, C.c_double]
            L.or_tally.restype = None
            L.or_tally.argtypes = [C.POINTER(OrGrid), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.c_double, C.c_double, C.c_void_p, C.POINTER(C.c_int64)]
            L.or_scene_eval.restype = None
            L.or_scene_eval.argtypes = [C.POINTER(OrScene), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), C.POINTER(C.c_int),
                                        C.POINTER(C.c_int), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]
            L.or_segment_step.restype = C.c_double
            L.or_segment_step.argtypes = [C.POINTER(OrScene), C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.or_region_sdf.restype = C.c_double
            L.or_region_sdf.argtypes = [C.POINTER(OrScene), C.c_int, C.POINTER(C.c_double)]
            L.or_surface_normal.restype = C.c_int
            L.or_surface_normal.argtypes = [C.POINTER(OrScene), C.c_int, C.POINTER(C.c_double),
                                            C.POINTER(C.c_double)]
            L.or_interface_once.restype = C.c_int
            L.or_interface_once.argtypes = [C.POINTER(OrScene), C.POINTER(C.c_double),
                                            C.POINTER(C.c_double), C.c_uint64, C.c_uint64]
            L.or_draw_uniforms.restype = None
            L.or_draw_uniforms.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_int, C.c_void_p]
            L.or_sizeof.restype = C.c_int
            L.or_sizeof.argtypes = [C.c_int]
            for i, s in enumerate([OrPrim, OrNode, OrRegion, OrScene, OrSource, OrGrid, OrTotals]):
                assert L.or_sizeof(i) == C.sizeof(s), (i, L.or_sizeof(i), C.sizeof(s))
            assert L.or_sizeof(7) == PACKET_DTYPE.itemsize
            assert L.or_sizeof(8) == C.sizeof(OrXform)
            _lib = L
    return _lib


class _SceneHolder:
    """Keeps the ctypes arrays alive for the lifetime of an OrScene."""

    def __init__(self, scene: W.Scene):
        prims = (OrPrim * max(1, len(scene.prims)))()
        xf_l = []
        for i, pr in enumerate(scene.prims):
            prims[i].kind = _PRIM_KIND[pr.kind]
            for j, v in enumerate(pr.params):
                prims[i].p[j] = float(v)
            if pr.xform is not None:
                xf_l.append(pr.xform)
                prims[i].xform = len(xf_l)
        xforms = (OrXform * max(1, len(xf_l)))()
        for i, X in enumerate(xf_l):
            xforms[i].rot[:] = [float(v) for v in X.rot]
            xforms[i].t[:] = [float(v) for v in X.t]
            xforms[i].s, xforms[i].op = float(X.s), _XF_OP[X.op]
            xforms[i].a[:] = [float(v) for v in X.a]
        self.xforms = xforms
        nodes_l, regs = [], (OrRegion * max(1, len(scene.regions)))()
        for r, reg in enumerate(scene.regions):
            regs[r].begin = len(nodes_l)
            regs[r].count = len(reg.program)
            regs[r].mu_a, regs[r].mu_s, regs[r].g, regs[r].n = reg.mu_a, reg.mu_s, reg.g, reg.n
            nodes_l.extend(reg.program)
        nodes = (OrNode * max(1, len(nodes_l)))()
        for i, nd in enumerate(nodes_l):
            nodes[i].op, nodes[i].prim, nodes[i].k = _OP[nd.op], nd.prim, float(nd.k)
        self.prims, self.nodes, self.regs = prims, nodes, regs
        self.s = OrScene(prims, len(scene.prims), nodes, len(nodes_l), regs, len(scene.regions),
                         float(scene.ambient_n), (C.c_double * 3)(*scene.bbox_lo),
                         (C.c_double * 3)(*scene.bbox_hi), float(scene.delta), int(scene.max_steps),
                         _STEPPING[scene.stepping], 0, xforms, len(xf_l), 0)


def _source(src: W.Source) -> OrSource:
    return OrSource(_SRC_KIND[src.kind], 0, (C.c_double * 3)(*src.pos),
                    (C.c_double * 3)(*src.dir), float(src.radius))


def _grid(g: W.Grid) -> OrGrid:
    return OrGrid((C.c_double * 3)(*g.lo), (C.c_double * 3)(*g.hi), (C.c_int32 * 3)(*g.n), 0)


def _totals_dict(t: OrTotals) -> dict:
    return {f: int(getattr(t, f)) for f in TOTAL_FIELDS}


def run(wl: W.Workload, id_begin: int = 0, id_end: int | None = None, threads: int | None = None,
        fluence: bool = True, records: bool = False, chunk: int | None = None):
    """Propagate packets [id_begin, id_end) of workload ``wl``.

    Returns (fluence int64 array [nz, ny, nx] or None, totals dict,
    per-packet records or None)."""
    L = lib()
    if id_end is None:
        id_end = id_begin + wl.npackets
    n = id_end - id_begin
    threads = threads or min(os.cpu_count() or 1, max(1, n // 64))
    threads = max(1, min(threads, max(1, n)))
    sh = _SceneHolder(wl.scene)
    src, grid = _source(wl.source), _grid(wl.grid)
    recs = np.zeros(n, dtype=PACKET_DTYPE) if records else None
    if chunk is None:
        chunk = max(1, -(-n // (threads * 4)))
    ranges = [(b, min(id_end, b + chunk)) for b in range(id_begin, id_end, chunk)]
    gshape = (wl.grid.n[2], wl.grid.n[1], wl.grid.n[0])
    acc = {}
    acc_lock = threading.Lock()

    class _Acc:
        pass

    def work(rng):
        b, e = rng
        tid = threading.get_ident()
        with acc_lock:
            a = acc.get(tid)
            if a is None:
                a = _Acc()
                a.flu = np.zeros(gshape, dtype=np.int64) if fluence else None
                a.tot = OrTotals()
                acc[tid] = a
        fp = a.flu.ctypes.data if fluence else None
        rp = recs[b - id_begin:].ctypes.data if records else None
        rc = L.or_run(C.byref(sh.s), C.byref(src), C.byref(grid), b, e, wl.seed, fp,
                      C.byref(a.tot), rp)
        if rc != 0:
            raise ValueError(f"oracle rejected the scene (code {rc})")

    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(work, ranges))
    flu = np.zeros(gshape, dtype=np.int64) if fluence else None
    tot = {f: 0 for f in TOTAL_FIELDS}
    for a in acc.values():
        if fluence:
            flu += a.flu
        for f in TOTAL_FIELDS:
            tot[f] += int(getattr(a.tot, f))
    return flu, tot, recs


# ---- single-function access for the pins -----------------------------------

def philox(ctr, key):
    L = lib()
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    L.or_philox4x32_10(c, k, o)
    return list(o)


def uniforms(seed: int, pid: int, event0: int = 0, ncalls: int = 1) -> np.ndarray:
    out = np.zeros(4 * ncalls, dtype=np.float64)
    lib().or_draw_uniforms(seed, pid, event0, ncalls, out.ctypes.data)
    return out


def log(x: float) -> float:
    return lib().or_log(float(x))


def sincos2pi(t: float):
    s, c = C.c_double(), C.c_double()
    lib().or_sincos2pi(float(t), C.byref(s), C.byref(c))
    return s.value, c.value


def hg_cos(g: float, xi: float) -> float:
    return lib().or_hg_cos(float(g), float(xi))


def fresnel(n1: float, n2: float, cos_i: float):
    ct = C.c_double()
    R = lib().or_fresnel(float(n1), float(n2), float(cos_i), C.byref(ct))
    return R, ct.value


def scatter_dir(u, cos_theta: float, xi_phi: float):
    v = (C.c_double * 3)(*u)
    lib().or_scatter_dir(v, float(cos_theta), float(xi_phi))
    return np.array(list(v))


def tally_segment(grid: W.Grid, p, u, length: float, w: float = 1.0):
    flu = np.zeros((grid.n[2], grid.n[1], grid.n[0]), dtype=np.int64)
    pieces = C.c_int64(0)
    g = _grid(grid)
    lib().or_tally(C.byref(g), (C.c_double * 3)(*p), (C.c_double * 3)(*u), float(length),
                   float(w), flu.ctypes.data, C.byref(pieces))
    return flu, pieces.value


def scene_eval(scene: W.Scene, p):
    sh = _SceneHolder(scene)
    dmin, dbox, dstar = C.c_double(), C.c_double(), C.c_double()
    istar, region = C.c_int(), C.c_int()
    lib().or_scene_eval(C.byref(sh.s), (C.c_double * 3)(*p), C.byref(dmin), C.byref(istar),
                        C.byref(region), C.byref(dbox), C.byref(dstar))
    return dict(dmin=dmin.value, istar=istar.value, region=region.value, dbox=dbox.value,
                dstar=dstar.value)


def segment_step(scene: W.Scene, p, u) -> float:
    """The segment-stepping move from p along u (0 within delta of a surface)."""
    sh = _SceneHolder(scene)
    return lib().or_segment_step(C.byref(sh.s), (C.c_double * 3)(*p), (C.c_double * 3)(*u))


def region_sdf(scene: W.Scene, r: int, p) -> float:
    sh = _SceneHolder(scene)
    return lib().or_region_sdf(C.byref(sh.s), int(r), (C.c_double * 3)(*p))


def surface_normal(scene: W.Scene, istar: int, p):
    sh = _SceneHolder(scene)
    n = (C.c_double * 3)()
    ok = lib().or_surface_normal(C.byref(sh.s), int(istar), (C.c_double * 3)(*p), n)
    return (np.array(list(n)) if ok else None)


def interface_once(scene: W.Scene, p, u, seed: int = 0, pid: int = 0):
    sh = _SceneHolder(scene)
    pp = (C.c_double * 3)(*p)
    uu = (C.c_double * 3)(*u)
    rc = lib().or_interface_once(C.byref(sh.s), pp, uu, seed, pid)
    return rc, np.array(list(pp)), np.array(list(uu))

"""Python binding of the GB300 photon-packet library (C-ABI: include/smcrt.h).

Argument marshalling only: every step of the transport runs in the CUDA
kernels of ``csrc/``.  There is no CPU fallback -- if the compiled library
is missing the binding raises.

Typical use::

    import paper_2112_08035_gb300 as smc, workloads as W
    ctx = smc.Context(0)
    flu, tot = ctx.run(W.three_layer_slab(10**6), precision="mixed")
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", f"libsmcrt_{platform.machine()}.so")

OK, ERR_BAD_ARG, ERR_BAD_SCENE, ERR_NO_MEMORY, ERR_CUDA, ERR_TIMEOUT, ERR_CANCELLED, ERR_NOT_FOUND, ERR_DEVICE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
FP64, MIXED = 0, 1
STATUS_BAD_JOB, STATUS_TIMEOUT = 1, 4   # kernel status word bits (Plan.status)
FX = 2.0 ** 32

_PRIM_KIND = {"sphere": 0, "box": 1, "capsule": 2, "torus": 3, "cylinder": 4}
_XF_OP = {"none": 0, "elongate": 1, "twist": 2, "bend": 3, "repeat": 4}
_OP = {"prim": 0, "union": 1, "smooth_union": 2, "intersect": 3, "subtract": 4}
_SRC_KIND = {"pencil": 0, "disc": 1, "square": 2, "iso": 3}
_STEPPING = {"sphere_tracing": 0, "segment": 1}
_PREC = {"fp64": FP64, "mixed": MIXED, FP64: FP64, MIXED: MIXED}


class Prim(C.Structure):
    _fields_ = [("kind", C.c_int32), ("xform", C.c_int32), ("p", C.c_double * 7)]


class Xform(C.Structure):
    _fields_ = [("rot", C.c_double * 9), ("t", C.c_double * 3), ("s", C.c_double), ("op", C.c_int32),
                ("reserved", C.c_int32), ("a", C.c_double * 4)]


class CsgNode(C.Structure):
    _fields_ = [("op", C.c_int32), ("prim", C.c_int32), ("k", C.c_double)]


class Region(C.Structure):
    _fields_ = [("node_begin", C.c_int32), ("node_count", C.c_int32), ("mu_a", C.c_double),
                ("mu_s", C.c_double), ("g", C.c_double), ("n", C.c_double)]


class Scene(C.Structure):
    _fields_ = [("prims", C.POINTER(Prim)), ("nprims", C.c_int32),
                ("nodes", C.POINTER(CsgNode)), ("nnodes", C.c_int32),
                ("regions", C.POINTER(Region)), ("nregions", C.c_int32),
                ("ambient_n", C.c_double), ("bbox_lo", C.c_double * 3), ("bbox_hi", C.c_double * 3),
                ("delta", C.c_double), ("max_steps", C.c_int64), ("stepping", C.c_int32),
                ("reserved", C.c_int32), ("xforms", C.POINTER(Xform)), ("nxforms", C.c_int32),
                ("reserved2", C.c_int32)]


class Source(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("pos", C.c_double * 3),
                ("dir", C.c_double * 3), ("radius", C.c_double)]


class Grid(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("n", C.c_int32 * 3),
                ("reserved", C.c_int32)]


TOTAL_FIELDS = ["R", "T", "A", "killed", "gain", "packets", "scatters", "steps", "scene_evals",
                "interfaces", "fresnel", "pieces", "max_steps_hit", "refined", "busy_cycles", "parked"]


class Totals(C.Structure):
    _fields_ = [(f, C.c_int64) for f in TOTAL_FIELDS]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f in TOTAL_FIELDS}


RECORD_DTYPE = np.dtype([(f, np.int64) for f in
                         ["R", "T", "A", "killed", "gain", "scatters", "steps", "reserved"]])

_lib = None
_lock = threading.Lock()


class SmcrtError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = lib().smcrt_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})")


def build(force: bool = False) -> str:
    from . import buildlib as _b
    return _b.build(force=force)


def lib():
    """Load the compiled library (building it if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            from . import buildlib as _b
            if os.path.exists(_b.NVCC):
                build()            # no-op when up to date; raises on a compile error
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libsmcrt missing at {LIB_PATH}")
            L = C.CDLL(LIB_PATH)
            vp, u64, i32 = C.c_void_p, C.c_uint64, C.c_int32
            sig = {
                "smcrt_version": (C.c_int, []),
                "smcrt_strerror": (C.c_char_p, [C.c_int]),
                "smcrt_validate": (C.c_int, [C.POINTER(Scene), C.POINTER(Source), C.POINTER(Grid),
                                             C.POINTER(i32)]),
                "smcrt_create": (C.c_int, [C.POINTER(vp), C.c_int, C.c_size_t]),
                "smcrt_destroy": (C.c_int, [vp]),
                "smcrt_plan_create": (C.c_int, [vp, C.POINTER(Scene), C.POINTER(Source), C.POINTER(Grid),
                                                i32, C.POINTER(vp)]),
                "smcrt_plan_destroy": (C.c_int, [vp]),
                "smcrt_plan_set_launch": (C.c_int, [vp, i32, i32]),
                "smcrt_plan_launch": (C.c_int, [vp, u64, u64, u64, vp, vp, vp, vp]),
                "smcrt_plan_status": (C.c_int, [vp, C.POINTER(i32)]),
                "smcrt_plan_autotune": (C.c_int, [vp, u64, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
                "smcrt_plan_set_variant": (C.c_int, [vp, i32]),
                "smcrt_plan_set_time_limit": (C.c_int, [vp, C.c_double]),
                "smcrt_set_time_limit": (C.c_int, [vp, C.c_double]),
                "smcrt_run": (C.c_int, [vp, C.POINTER(Scene), C.POINTER(Source), C.POINTER(Grid), u64, u64,
                                        i32, vp, C.POINTER(Totals)]),
                "smcrt_submit": (C.c_int, [vp, C.POINTER(Scene), C.POINTER(Source), C.POINTER(Grid), u64, u64,
                                           i32, C.POINTER(u64)]),
                "smcrt_poll": (C.c_int, [vp, u64, C.POINTER(i32)]),
                "smcrt_wait": (C.c_int, [vp, u64, C.c_double, vp, C.POINTER(Totals), C.POINTER(C.c_double)]),
                "smcrt_cancel": (C.c_int, [vp, u64]),
                "smcrt_serving_stats": (C.c_int, [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                                  C.POINTER(C.c_int64)]),
                "smcrt_run_noalloc": (C.c_int, [C.POINTER(Scene), C.POINTER(Source), C.POINTER(Grid), u64, u64,
                                                u64, i32, vp, vp, vp]),
                "smcrt_microbench": (C.c_int, [C.c_int, vp, C.c_size_t, C.POINTER(C.c_double),
                                               C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc, what):
    if rc != OK:
        raise SmcrtError(rc, what)


class Marshalled:
    """C structs for one workload (keeps the backing arrays alive)."""

    def __init__(self, scene, source, grid):
        np_ = len(scene.prims)
        self.prims = (Prim * np_)()
        xf = []
        for i, pr in enumerate(scene.prims):
            self.prims[i].kind = _PRIM_KIND[pr.kind]
            for j, v in enumerate(pr.params):
                self.prims[i].p[j] = float(v)
            if getattr(pr, "xform", None) is not None:
                xf.append(pr.xform)
                self.prims[i].xform = len(xf)
        self.xforms = (Xform * max(1, len(xf)))()
        for i, X in enumerate(xf):
            self.xforms[i].rot[:] = [float(v) for v in X.rot]
            self.xforms[i].t[:] = [float(v) for v in X.t]
            self.xforms[i].s, self.xforms[i].op = float(X.s), _XF_OP[X.op]
            self.xforms[i].a[:] = [float(v) for v in X.a]
        nodes, regs = [], (Region * len(scene.regions))()
        for r, reg in enumerate(scene.regions):
            regs[r].node_begin, regs[r].node_count = len(nodes), len(reg.program)
            regs[r].mu_a, regs[r].mu_s, regs[r].g, regs[r].n = reg.mu_a, reg.mu_s, reg.g, reg.n
            nodes.extend(reg.program)
        self.nodes = (CsgNode * max(1, len(nodes)))()
        for i, nd in enumerate(nodes):
            self.nodes[i].op, self.nodes[i].prim, self.nodes[i].k = _OP[nd.op], int(nd.prim), float(nd.k)
        self.regions = regs
        self.scene = Scene(self.prims, np_, self.nodes, len(nodes), regs, len(scene.regions),
                           float(scene.ambient_n), (C.c_double * 3)(*scene.bbox_lo),
                           (C.c_double * 3)(*scene.bbox_hi), float(scene.delta), int(scene.max_steps),
                           _STEPPING[scene.stepping], 0, self.xforms, len(xf), 0)
        self.source = Source(_SRC_KIND[source.kind], 0, (C.c_double * 3)(*source.pos),
                             (C.c_double * 3)(*source.dir), float(source.radius))
        self.grid = Grid((C.c_double * 3)(*grid.lo), (C.c_double * 3)(*grid.hi),
                         (C.c_int32 * 3)(*grid.n), 0)
        self.cells = int(grid.n[0]) * int(grid.n[1]) * int(grid.n[2])
        self.shape = (int(grid.n[2]), int(grid.n[1]), int(grid.n[0]))


def validate(wl) -> int:
    """Host-side validation and CSG compilation (no device).  Returns the
    compiled instruction count or raises SmcrtError."""
    m = Marshalled(wl.scene, wl.source, wl.grid)
    n = C.c_int32()
    _check(lib().smcrt_validate(C.byref(m.scene), C.byref(m.source), C.byref(m.grid), C.byref(n)), "validate")
    return n.value


def _ptr(x):
    """Device or host address of a torch tensor or numpy array (or None)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


class Plan:
    """A validated, compiled, device-resident scene (smcrt_plan_*)."""

    def __init__(self, ctx: "Context", wl, precision="mixed"):
        self.ctx = ctx
        self.m = Marshalled(wl.scene, wl.source, wl.grid)
        self.precision = _PREC[precision]
        h = C.c_void_p()
        _check(lib().smcrt_plan_create(ctx.h, C.byref(self.m.scene), C.byref(self.m.source),
                                       C.byref(self.m.grid), self.precision, C.byref(h)), "plan_create")
        self.h = h

    def set_launch(self, blocks=0, threads=0):
        _check(lib().smcrt_plan_set_launch(self.h, int(blocks), int(threads)), "plan_set_launch")

    def launch(self, id_begin, npackets, seed, fluence_dev, totals_dev, records_dev=None, stream=None):
        """Asynchronous launch; device buffers are accumulated into."""
        _check(lib().smcrt_plan_launch(self.h, int(id_begin), int(npackets), int(seed), _ptr(fluence_dev),
                                       _ptr(totals_dev), _ptr(records_dev), stream), "plan_launch")

    def status(self):
        v = C.c_int32()
        _check(lib().smcrt_plan_status(self.h, C.byref(v)), "plan_status")
        return v.value

    def set_variant(self, variant):
        _check(lib().smcrt_plan_set_variant(self.h, int(variant)), "plan_set_variant")

    def set_time_limit(self, seconds):
        """Device time limit of later launches (0 = none); see status()."""
        _check(lib().smcrt_plan_set_time_limit(self.h, float(seconds)), "plan_set_time_limit")

    def autotune(self, trial_packets):
        """Returns the chosen (blocks, threads, variant)."""
        b, t, v = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().smcrt_plan_autotune(self.h, int(trial_packets), C.byref(b), C.byref(t), C.byref(v)),
               "plan_autotune")
        return b.value, t.value, v.value

    def close(self):
        if self.h:
            lib().smcrt_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """One library context on one CUDA device (smcrt_create/destroy)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        h = C.c_void_p()
        _check(lib().smcrt_create(C.byref(h), int(device), int(budget_bytes)), "create")
        self.h = h
        self._keep = {}

    def close(self):
        if self.h:
            lib().smcrt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plan(self, wl, precision="mixed") -> Plan:
        return Plan(self, wl, precision)

    def set_time_limit(self, seconds):
        """Device time limit of run() and the default of later plans (0 = none)."""
        _check(lib().smcrt_set_time_limit(self.h, float(seconds)), "set_time_limit")

    def run(self, wl, precision=None, fluence=True, out=None):
        """Synchronous run of packets [0, wl.npackets).  Returns (fluence
        int64 [nz, ny, nx] numpy array or the given ``out``, totals dict)."""
        m = Marshalled(wl.scene, wl.source, wl.grid)
        prec = _PREC[precision if precision is not None else wl.precision]
        if fluence and out is None:
            out = np.zeros(m.shape, dtype=np.int64)
        t = Totals()
        _check(lib().smcrt_run(self.h, C.byref(m.scene), C.byref(m.source), C.byref(m.grid),
                               int(wl.npackets), int(wl.seed), prec, _ptr(out) if fluence else None,
                               C.byref(t)), "run")
        return out, t.as_dict()

    # ---- serving -----------------------------------------------------------
    def submit(self, wl, precision=None) -> int:
        m = Marshalled(wl.scene, wl.source, wl.grid)
        prec = _PREC[precision if precision is not None else wl.precision]
        jid = C.c_uint64()
        _check(lib().smcrt_submit(self.h, C.byref(m.scene), C.byref(m.source), C.byref(m.grid),
                                  int(wl.npackets), int(wl.seed), prec, C.byref(jid)), "submit")
        self._keep[jid.value] = m.shape
        return jid.value

    def poll(self, job_id) -> bool:
        d = C.c_int32()
        _check(lib().smcrt_poll(self.h, int(job_id), C.byref(d)), "poll")
        return bool(d.value)

    def wait(self, job_id, timeout_s=-1.0, fluence=True):
        shape = self._keep.pop(job_id, None)
        out = np.zeros(shape, dtype=np.int64) if (fluence and shape is not None) else None
        t = Totals()
        lat = C.c_double()
        rc = lib().smcrt_wait(self.h, int(job_id), float(timeout_s), _ptr(out), C.byref(t), C.byref(lat))
        if rc == ERR_TIMEOUT:
            self._keep[job_id] = shape
        _check(rc, "wait")
        return out, t.as_dict(), lat.value

    def cancel(self, job_id):
        _check(lib().smcrt_cancel(self.h, int(job_id)), "cancel")

    def serving_stats(self):
        q, r, n = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().smcrt_serving_stats(self.h, C.byref(q), C.byref(r), C.byref(n)), "serving_stats")
        return q.value, r.value, n.value


def run_noalloc(wl, id_begin, npackets, seed, fluence_dev, totals_dev, precision=None, stream=None):
    """smcrt_run_noalloc: asynchronous launch on the current device with the
    library's fixed scratch array instead of allocated device memory.
    fluence_dev / totals_dev are accumulated into."""
    m = Marshalled(wl.scene, wl.source, wl.grid)
    prec = _PREC[precision if precision is not None else wl.precision]
    _check(lib().smcrt_run_noalloc(C.byref(m.scene), C.byref(m.source), C.byref(m.grid), int(id_begin),
                                   int(npackets), int(seed), prec, _ptr(fluence_dev), _ptr(totals_dev), stream),
           "run_noalloc")


def totals_tensor(device="cuda"):
    """A zeroed device buffer laid out as one smcrt_totals (16 int64)."""
    import torch
    return torch.zeros(C.sizeof(Totals) // 8, dtype=torch.int64, device=device)


def totals_from_tensor(t) -> dict:
    v = t.detach().cpu().numpy()
    return {f: int(v[i]) for i, f in enumerate(TOTAL_FIELDS)}


def microbench(device: int = 0):
    """Measured FP32 FMA flop/s and int64 atomic rates (distinct, hot) of
    the GPU (smcrt_microbench); uses a 64 MiB torch scratch buffer."""
    import torch
    buf = torch.empty(1 << 23, dtype=torch.int64, device=f"cuda:{device}")
    f, a, h = C.c_double(), C.c_double(), C.c_double()
    _check(lib().smcrt_microbench(int(device), _ptr(buf), buf.numel() * 8, C.byref(f), C.byref(a), C.byref(h)),
           "microbench")
    return {"fp32_flops": f.value, "atomics_distinct_per_s": a.value, "atomics_hot_per_s": h.value}

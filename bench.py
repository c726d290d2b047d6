"""Benchmark: photon packets/s of the SDF Monte Carlo transport path.

Workload (one "step"): the three-layer slab -- three box SDF layers 0.1 /
0.2 / 1.0 cm thick (mu_a 0.1-2, mu_s 10-100 /cm, g 0.8-0.95, n 1.3-1.5),
pencil beam, 1e7 packets, 100^3 int64 fluence grid -- in the mixed
precision mode (FP32 tracing, FP64 interface refinement) with segment
stepping (``--stepping``).  ``value`` is packets/s with the scene resident on
the device; the JSON line also carries the mixed mode with plain sphere
tracing and the plain-FP64 mode (sphere tracing) on the same workload, R/T/A
of each against the FP64 CPU oracle, the served mix's p50/p99 job latency,
the roofline of the packet kernel, and the oracle timed on the host cores.

Multi-GPU (torchrun): packets are independent, so each rank runs its own
1e7-packet block of ids (weak scaling, no data-path collective); the step
time is the max over ranks.

``--impl reference`` times the FP64 CPU oracle instead (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "photon packets/s (and p50/p99 job latency) mixed vs plain FP64 at equal R/T/A error"
UNIT = "packets/s"
FX = 2.0 ** 32

# Algorithmic FP32 work per counted event (operations, an FMA counted as 2),
# from the arithmetic of the method; the event counts come from the FP64
# oracle's own counters on a sample of the same workload and step rule.
#   primitive SDF: sphere 8, box 20 (3 sub, 3 abs, 3 sub, 3 max, 5 for the
#   squared norm, sqrt, min/max), capsule 22, torus 12, cylinder 14;
#   smooth union 8; per scene evaluation: the bounding box 20 and 5 per
#   region (compare, abs, compare, 2 selects);
#   step: tally set-up 40 + move 6 + tau update 2 = 48;  voxel piece 16;
#   interaction: weight 3, HG 12, azimuth sincos 4, basis 14, rotation 15,
#   normalisation 8, roulette 2, log 4 = 62;  interface (normal from the
#   gradient, Fresnel / Snell cosines and directions) 30;
#   segment-stepping bound, per move that used it: the bounding box's ray
#   exit 30, each primitive distance it takes (the SDF figures above), and
#   per primitive ray bound sphere 15, box 30, capsule 60, cylinder 40,
#   torus 75 (two cylinder intervals and a slab).
FLOPS_PRIM = {"sphere": 8, "box": 20, "capsule": 22, "torus": 12, "cylinder": 14}
FLOPS_SMOOTH = 8
FLOPS_BBOX = 20
FLOPS_REGION = 5
FLOPS_STEP = 48
FLOPS_PIECE = 16
FLOPS_INTERACTION = 62
FLOPS_INTERFACE = 30
FLOPS_SEG_BBOX = 30
FLOPS_SEG_PRIM = {"sphere": 15, "box": 30, "capsule": 60, "torus": 75, "cylinder": 40}


def algorithmic_work(t: dict, nregions: int) -> dict:
    """FP32 flops and int64 atomics per packet from the oracle's counters
    ``t`` (totals of a sample): the roofline's algorithmic work."""
    n = max(1, t["packets"])
    prim = sum(t[f"prim_{k}"] * w for k, w in FLOPS_PRIM.items())
    seg_per_call = FLOPS_SEG_BBOX + (sum(t[f"seg_{k}"] * w for k, w in FLOPS_SEG_PRIM.items())
                                     + sum(t[f"seg_dist_{k}"] * w for k, w in FLOPS_PRIM.items())
                                     ) / max(1, t["seg_calls"])
    flops = (prim + t["smooth_ops"] * FLOPS_SMOOTH + t["scene_evals"] * (FLOPS_BBOX + FLOPS_REGION * nregions)
             + t["steps"] * FLOPS_STEP + t["pieces"] * FLOPS_PIECE + t["scatters"] * FLOPS_INTERACTION
             + t["interfaces"] * FLOPS_INTERFACE + t["seg_moves"] * seg_per_call)
    return {"flops_per_packet": flops / n, "atomics_per_packet": t["pieces"] / n,
            "counts_per_packet": {k: t[k] / n for k in ("steps", "scene_evals", "prim_evals", "scatters",
                                                        "interfaces", "pieces", "seg_moves")}}


KERNEL_SOURCES = ["paper_2112_08035_gb300/csrc/smcrt_kernel.cuh", "paper_2112_08035_gb300/csrc/smcrt_k32.cu",
                  "paper_2112_08035_gb300/csrc/smcrt_internal.h"]
TRAFFIC_SUMMARY = "profiles/packets_mixed_three_layer_slab.md"


def kernel_source_hash() -> str:
    """sha256 of the packet kernel's sources with comments and whitespace
    removed (a comment edit does not change the kernel)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(re.sub(r"\s+", "", src).encode())
    return h.hexdigest()


def recorded_traffic(key: str = "dram_bytes_per_launch"):
    """A figure of the committed ncu summary of the packet kernel (DRAM bytes
    per launch, or thread instructions per packet), or None when the kernel
    source changed after that capture."""
    path = os.path.join(ROOT, TRAFFIC_SUMMARY)
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            line = line.strip().lstrip("-").strip()
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256") != kernel_source_hash():
        return None
    try:
        return int(vals[key])
    except (KeyError, ValueError):
        return None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, n in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def oracle_sample(wl, seconds: float, id_base: int = 0, K: int = 10, block=(10, 10, 10)):
    """Time the FP64 oracle, as it stands, on a bounded sample sized to take
    about ``seconds``, run as K batches of consecutive ids; returns a dict:
    packets/s, packets, threads, per-packet records, the first and second
    halves' fluence maps, per-batch fluence block sums (per packet) and the
    oracle's totals (its work counters included)."""
    import numpy as np
    import oracle as O
    threads = os.cpu_count() or 1
    n0 = 2000
    t0 = time.perf_counter()
    O.run(wl.with_packets(n0), id_base, id_base + n0, threads=threads, fluence=True)
    rate0 = n0 / (time.perf_counter() - t0)
    per = int(max(n0, min(5_000_000, rate0 * seconds))) // K
    recs, blocks, maps = [], [], []
    tot = None
    t0 = time.perf_counter()
    for k in range(K):
        f, t, r = O.run(wl.with_packets(per), id_base + k * per, threads=threads, records=True)
        recs.append(r)
        maps.append(f)
        blocks.append(block_sums(f, block) / FX / per)
        tot = t if tot is None else {key: tot[key] + t[key] for key in tot}
    dt = time.perf_counter() - t0
    h = K // 2
    return {"pps": K * per / dt, "packets": K * per, "threads": threads, "records": np.concatenate(recs),
            "halves": (sum(maps[:h]), sum(maps[h:2 * h])), "half_packets": h * per,
            "blocks": np.array(blocks), "totals": tot}


def fluence_l2(gpu_flu, n_gpu: int, halves, n_half: int) -> dict:
    """Relative L2 difference of the per-packet fluence maps (GPU against the
    oracle sample), beside the oracle sample's own noise: the value a
    consistent result shows, since the GPU's 1e7 packets add little noise.
    The sample's noise is half the difference of its two half-sample maps."""
    import numpy as np
    f1 = halves[0].astype(np.float64) / n_half
    f2 = halves[1].astype(np.float64) / n_half
    po = 0.5 * (f1 + f2)
    pg = gpu_flu.astype(np.float64) / n_gpu
    norm = float(np.linalg.norm(po))
    l2 = float(np.linalg.norm(pg - po)) / norm
    noise = float(np.linalg.norm(f1 - f2)) / 2.0 / norm
    return {"fluence_rel_l2": l2, "fluence_oracle_noise_rel_l2": noise,
            "fluence_l2_over_noise": l2 / noise if noise > 0 else None}


def _z_from_t(t, dof):
    """Normal deviate with the same two-sided tail probability as Student's t
    with ``dof`` degrees of freedom (batch means: the spread is estimated)."""
    from scipy import stats
    t = np.asarray(t, dtype=np.float64)
    return np.sign(t) * stats.norm.isf(stats.t.sf(np.abs(t), dof))


def paired_z(a, b) -> float:
    """z of the mean of paired differences a - b (same packet ids or the same
    batches on both sides), from the differences' own spread."""
    d = np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)
    se = d.std(ddof=1) / math.sqrt(d.size)
    return float(d.mean() / se) if se > 0 else (0.0 if d.mean() == 0 else math.inf)


def paired_block_stats(A, B, k: float = 3.0) -> dict:
    """Block-by-block comparison of two fluence estimates made on the same
    K batches of packet ids (A, B: (K, nblocks) per-batch block sums); see
    ``block_stats``."""
    return block_stats(A, B, paired=True, k=k)


def block_stats(A, B, paired: bool = True, k: float = 3.0) -> dict:
    """Block-by-block comparison of two fluence estimates.  A and B are
    (K_a, nblocks) and (K_b, nblocks) arrays of per-batch block sums,
    normalised per packet.  Paired (K_a = K_b, the same packet ids in batch
    i on both sides): the t statistic of the mean difference over the K
    batches, K - 1 degrees of freedom.  Unpaired (independent samples): the
    Welch t of the two batch means, Welch-Satterthwaite degrees of freedom.
    Blocks are tested where every batch on both sides is non-zero (each batch
    sum then adds many packets, so it is close to normal).  Each t becomes the
    normal deviate z of the same two-sided tail.  Under equal expectations
    every z is standard normal, so with n blocks tested:
      - the count of |z| > k is binomial(n, p_k) for independent blocks:
        accepted up to its mean plus 3 standard deviations (the variance
        widened by n / n_eff, below);
      - chi2/dof = mean(z^2) has mean 1 and standard deviation sqrt(2/n)
        for independent blocks: accepted within 1 +- 3 sqrt(2 / n_eff),
        where n_eff is n divided by 1 + (n - 1) times the blocks' mean squared
        correlation (blocks crossed by the same packets are correlated);
      - max |z| stays below the deviate of a two-sided tail p_k / n (a
        Bonferroni bound, valid whatever the correlation)."""
    from scipy import stats
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    ok = np.all(A > 0, axis=0) & np.all(B > 0, axis=0)
    A, B = A[:, ok], B[:, ok]
    n = int(A.shape[1])
    if n == 0:
        return {"blocks": 0, "pass": False}
    if paired:
        K = A.shape[0]
        D = A - B
        m = D.mean(axis=0)
        v = D.var(axis=0, ddof=1) / K
        dof = np.full(n, K - 1.0)
        dev = (D - m) / math.sqrt(K)          # per-batch deviations of the mean difference
        kk = K
    else:
        Ka, Kb = A.shape[0], B.shape[0]
        va, vb = A.var(axis=0, ddof=1) / Ka, B.var(axis=0, ddof=1) / Kb
        m = A.mean(axis=0) - B.mean(axis=0)
        v = va + vb
        with np.errstate(divide="ignore", invalid="ignore"):
            dof = np.where(v > 0, v * v / (va * va / (Ka - 1) + vb * vb / (Kb - 1)), 1.0)
        dev = None
        kk = min(Ka, Kb)
    se = np.sqrt(v)
    t = np.where(se > 0, m / np.where(se > 0, se, 1.0), 0.0)
    z = _z_from_t(t, np.maximum(dof, 1.0))
    p_k = 2.0 * stats.norm.sf(k)
    n_out = int(np.count_nonzero(np.abs(z) > k))
    # effective number of independent blocks: from the correlation matrix of
    # the blocks' mean differences, estimated from the batches
    if n > 1 and kk > 2:
        if paired:
            C = dev.T @ dev / (kk - 1)
        else:
            da = (A - A.mean(axis=0)) / A.shape[0]
            db = (B - B.mean(axis=0)) / B.shape[0]
            C = da.T @ da * (A.shape[0] / (A.shape[0] - 1)) + db.T @ db * (B.shape[0] / (B.shape[0] - 1))
        d = np.sqrt(np.clip(np.diag(C), 1e-300, None))
        R = C / d[:, None] / d[None, :]
        r2 = (np.sum(R * R) - n) / (n * (n - 1))
        # the sample correlation of unrelated blocks is itself ~1/(K-1) in square
        r2 = max(0.0, r2 - 1.0 / (kk - 1))
        n_eff = n / (1.0 + (n - 1) * r2)
    else:
        n_eff = float(n)
    # correlated blocks also widen the spread of the count (by n / n_eff)
    out_limit = n * p_k + 3.0 * math.sqrt(n * p_k * (1.0 - p_k) * n / n_eff)
    chi2 = float(np.mean(z * z))
    chi2_band = 3.0 * math.sqrt(2.0 / n_eff)
    zmax = float(np.max(np.abs(z)))
    zmax_limit = float(stats.norm.isf(p_k / 2.0 / n))
    worst = int(np.nonzero(ok)[0][int(np.argmax(np.abs(z)))])
    return {"blocks": n, "paired": paired, "n_over_k": n_out, "n_over_k_limit": out_limit,
            "chi2_dof": chi2, "chi2_band": chi2_band, "n_eff": n_eff, "z_max": zmax,
            "z_max_limit": zmax_limit, "z_max_block": worst,
            "z_max_block_rel_diff": float(m[np.argmax(np.abs(z))] / max(abs(B[:, np.argmax(np.abs(z))].mean()), 1e-300)),
            "pass": bool(n_out <= out_limit and abs(chi2 - 1.0) <= chi2_band and zmax <= zmax_limit)}


def block_sums(flu, b):
    """Sums of a [nz][ny][nx] fluence map over b[0] x b[1] x b[2] voxel blocks
    (x, y, z block edges), flattened (torch tensor on the device or numpy)."""
    nz, ny, nx = flu.shape
    bx, by, bz = b
    f = flu[: nz // bz * bz, : ny // by * by, : nx // bx * bx]
    shape = (nz // bz, bz, ny // by, by, nx // bx, bx)
    if hasattr(f, "data_ptr"):
        return f.reshape(shape).sum(dim=(1, 3, 5)).double().cpu().numpy().ravel()
    return f.reshape(shape).sum(axis=(1, 3, 5)).astype(np.float64).ravel()


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = W.three_layer_slab(precision="fp64").with_stepping(args.stepping)
    import oracle as O
    O.build()
    threads = os.cpu_count() or 1
    # a bounded sample per step: about 8 s of oracle work each
    n0 = 2000
    t0 = time.perf_counter()
    O.run(wl.with_packets(n0), 0, n0, threads=threads)
    rate0 = n0 / (time.perf_counter() - t0)
    n = int(max(n0, rate0 * 8.0))
    for i in range(args.warmup):
        O.run(wl.with_packets(min(n, 4000)), 0, min(n, 4000), threads=threads)
    times = []
    for i in range(args.steps):
        t0 = time.perf_counter()
        O.run(wl.with_packets(n), i * n, (i + 1) * n, threads=threads)
        times.append(time.perf_counter() - t0)
    value = n * args.steps / sum(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"three_layer_slab (1e7 packets, 100^3 grid, {args.stepping} stepping), sampled",
                       "sample_packets_per_step": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{n} packets of three_layer_slab per step (ids disjoint per step)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def served_mix(ctx, njobs: int, capacity_pps: float, load: float = 0.8, seed: int = 4,
               limit_s: float = 240.0, stepping: str = W.SEGMENT):
    """Poisson arrivals of the served mix at ``load`` x measured capacity;
    returns job latencies (submit to completion, measured by the library)
    and the served throughput.  Stops submitting after ``limit_s``."""
    jobs = W.served_mix(njobs, seed, stepping=stepping)
    rng = np.random.default_rng(seed)
    total = sum(j.npackets for j in jobs)
    mean_gap = (total / njobs) / (capacity_pps * load)
    arrivals = np.cumsum(rng.exponential(mean_gap, njobs))
    t0 = time.perf_counter()
    ids = []
    for j, wl in enumerate(jobs):
        delay = arrivals[j] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        if time.perf_counter() - t0 > limit_s:
            break
        ids.append((ctx.submit(wl, "mixed"), wl.npackets))
    lat, served = [], 0
    for jid, n in ids:
        left = max(1.0, limit_s * 1.5 - (time.perf_counter() - t0))
        try:
            _, tot, l = ctx.wait(jid, left, fluence=False)
        except Exception:
            continue
        lat.append(l)
        served += tot["packets"]
    wall = time.perf_counter() - t0
    lat_ms = np.array(lat) * 1e3 if lat else np.array([float("nan")])
    return {"jobs_submitted": len(ids), "jobs_completed": len(lat), "packets": int(served), "wall_s": wall,
            "served_pps": served / wall, "offered_load": load, "p50_ms": float(np.percentile(lat_ms, 50)),
            "p99_ms": float(np.percentile(lat_ms, 99)), "mean_ms": float(np.mean(lat_ms))}


def log(*a):
    print("[bench]", *a, file=sys.stderr, flush=True)


# Table 2 (Sec. 3.2): the paper's sMCRT timings with a fluence grid, on an
# AMD Ryzen 9 3950X with 32 threads -- another machine's CPU numbers, quoted
# as context, not as a target.
PAPER_TABLE2 = {"jacques": (10_000_000, 33.73), "iso_sphere_tau100": (1_000_000, 75.76),
                "glass_sphere": (27_000_000, 61.0)}   # the last from Sec. 3.2, not Table 2


def paper_cases(ctx, smc, stream, stepping: str):
    """The paper's timing cases at their sizes (Table 2) in mixed precision:
    the Jacques et al. slab of Table 1 (both wavelengths; 1e7 photons,
    200 x 200 x 400 grid) and the isotropic sphere at radial optical depth
    100 (1e6 photons, 200^3 grid), and the glass sphere of Sec. 3.2 (2.7e7
    photons), each one timed launch after a warm-up, with the validation
    quantity of each (k1 of Eq. 5 fitted to the depth profile, the mean
    scattering count against Eq. 4; R and T for the sphere)."""
    import torch
    out = {}
    cases = [("jacques_slab_420nm", "jacques", W.jacques_slab(420)),
             ("jacques_slab_630nm", "jacques", W.jacques_slab(630)),
             ("iso_sphere_tau100", "iso_sphere_tau100", W.iso_sphere(100.0)),
             ("glass_sphere_beam", "glass_sphere", W.glass_sphere_beam())]
    for name, key, wl in cases:
        wl = wl.with_stepping(stepping)
        g = wl.grid
        plan = ctx.plan(wl, "mixed")
        flu = torch.zeros((g.n[2], g.n[1], g.n[0]), dtype=torch.int64, device="cuda")
        tot = smc.totals_tensor()
        plan.launch(0, min(wl.npackets, 100_000), wl.seed, flu, tot, None, stream.cuda_stream)
        torch.cuda.synchronize()
        flu.zero_()
        tot.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.launch(0, wl.npackets, wl.seed, flu, tot, None, stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        sec = a.elapsed_time(b) / 1e3
        t = smc.totals_from_tensor(tot)
        n = wl.npackets
        e = {"photons": n, "grid": list(g.n), "seconds": sec, "packets_per_s": n / sec,
             "scatters_per_packet": t["scatters"] / n, "max_steps_hit": t["max_steps_hit"]}
        if key == "jacques":
            mua, musp = W.JACQUES_OPTICS[int(name.split("_")[-1][:3])]
            d = W.penetration_depth(mua, musp)
            nz = g.n[2]
            phi = flu.sum(dim=(1, 2)).double().cpu().numpy()[::-1]      # surface first
            z = (np.arange(nz) + 0.5) * (g.hi[2] - g.lo[2]) / nz
            sel = (z > 4 * d) & (z < 12 * d) & (phi > 0)
            e["k1_fit"] = float(-np.polyfit(z[sel], np.log(phi[sel]), 1)[0] * d)
            e["k1_table1"] = 1.00
            # fluence rate over the grid's 2 x 2 cm relative to the incident
            # irradiance (photons per cm^2 of the 4 x 4 cm source)
            area = (g.hi[0] - g.lo[0]) * (g.hi[1] - g.lo[1])
            dz = (g.hi[2] - g.lo[2]) / nz
            psi = phi / FX / (area * dz) / (n / (2 * wl.source.radius) ** 2)
            e["psi_over_incident_at_z"] = {f"{m}delta": float(np.interp(m * d, z, psi)) for m in (1, 2, 4)}
        elif key == "glass_sphere":
            e["R"] = t["R"] / FX / n
            e["T"] = t["T"] / FX / n
        else:
            tau = wl.scene.regions[0].mu_s * wl.scene.prims[0].params[3]
            want = tau * tau / 2 + tau
            e["eq4"] = {"mean_scatterings": t["scatters"] / n, "eq4": want,
                        "rel_diff": (t["scatters"] / n - want) / want}
        pn, ps = PAPER_TABLE2[key]
        e["paper_cpu"] = {"photons": pn, "seconds": ps, "packets_per_s": pn / ps,
                          "machine": "AMD Ryzen 9 3950X, 32 threads; context only"
                                     + (" (Sec. 3.2: about 2.7e7 photons; its grid and medium are not stated)"
                                        if key == "glass_sphere" else " (Table 2)")}
        out[name] = e
        plan.close()
        del flu
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--packets", type=int, default=10_000_000)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--serve-jobs", type=int, default=200)
    ap.add_argument("--no-configs", action="store_true", help="skip the configs 0, 2, 3 block")
    ap.add_argument("--cfg-steps", type=int, default=2, help="timed steps of the 1e8-packet configs")
    ap.add_argument("--cfg-fp64-packets", type=int, default=1_000_000,
                    help="FP64 packets timed, and compared, on configs 2 and 3")
    ap.add_argument("--oracle-seconds", type=float, default=15.0)
    ap.add_argument("--quick", action="store_true", help="kernel legs only (profiling runs)")
    ap.add_argument("--no-paper-cases", action="store_true", help="skip the paper's Table 2 timing cases")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shape (profiling runs)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="precision of the timed leg (the headline is mixed)")
    ap.add_argument("--stepping", default=W.SEGMENT, choices=[W.SEGMENT, W.SPHERE_TRACING],
                    help="step rule of the timed leg (the headline uses segment stepping)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    import paper_2112_08035_gb300 as smc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    ctx = smc.Context(local)
    wl = W.three_layer_slab(args.packets, precision=args.precision).with_stepping(args.stepping)
    wl_plain = wl.with_stepping(W.SPHERE_TRACING)
    g = wl.grid
    from paper_2112_08035_gb300.distributed import shard_range
    id0, _ = shard_range(rank, world, args.packets * world)   # this rank's block of ids
    plan = ctx.plan(wl, args.precision)
    tuned = (0, 0, -1) if args.no_autotune else plan.autotune(min(args.packets, 2_000_000))
    flu = torch.zeros((g.n[2], g.n[1], g.n[0]), dtype=torch.int64, device="cuda")
    tot = smc.totals_tensor()
    l2_flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(p, precision_plan, seed, first_id):
        flu.zero_()
        tot.zero_()
        precision_plan.launch(first_id, p, seed, flu, tot, None, stream.cuda_stream)

    for _ in range(args.warmup):
        step(args.packets, plan, wl.seed, id0)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        for i in range(args.steps):
            l2_flush.fill_(float(i))      # L2 flush between timed iterations (not timed)
            ev[i][0].record(stream)
            step(args.packets, plan, wl.seed, id0)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    step_s = [a.elapsed_time(b) / 1e3 for a, b in ev]
    t_sum = sum(step_s)
    if dist:
        tt = torch.tensor([t_sum], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_sum = float(tt.item())
    totals_mixed = smc.totals_from_tensor(tot)
    value = args.packets * args.steps * world / t_sum
    kernel_s = t_sum / args.steps   # per-step device time ~ the packet kernel (one launch)

    e2e_multi = None
    if dist and not args.quick:
        # end to end at N GPUs: every rank makes the public synchronous call
        # with host buffers, on its own seed (independent packets); the
        # slowest rank sets the time
        from dataclasses import replace as dc_replace
        wl_rank = dc_replace(wl, seed=wl.seed + 1000 * rank)
        h_flu = np.zeros((g.n[2], g.n[1], g.n[0]), dtype=np.int64)
        ctx.run(wl_rank.with_packets(100_000), args.precision, out=h_flu)
        torch.cuda.synchronize()
        dist.barrier()
        t0 = time.perf_counter()
        for _ in range(3):
            ctx.run(wl_rank, args.precision, out=h_flu)
        tt = torch.tensor([(time.perf_counter() - t0) / 3], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        m = smc.Marshalled(wl.scene, wl.source, wl.grid)
        import ctypes as C
        h2d = (C.sizeof(m.scene) + C.sizeof(m.prims) + C.sizeof(m.nodes) + C.sizeof(m.regions)
               + C.sizeof(m.source) + C.sizeof(m.grid))
        e2e_multi = {"value": args.packets * world / float(tt.item()), "unit": UNIT,
                     "h2d_bytes_per_step": int(h2d) * world,
                     "d2h_bytes_per_step": int(h_flu.nbytes + C.sizeof(smc.Totals)) * world,
                     "api": "smcrt_run with host scene structs and a host fluence buffer, on every rank "
                            "(seed + 1000 rank), slowest rank"}

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t_sum / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64 (mixed; int64 tallies)" if args.precision == "mixed" else "f64 (int64 tallies)",
           "data": "synthetic",
           "config": {"workload": f"three_layer_slab: 3 box-SDF layers, pencil beam, {args.packets:.0e} packets "
                                  f"per GPU, 100^3 int64 fluence grid, {args.precision} precision, "
                                  f"{args.stepping} stepping",
                      "stepping": args.stepping,
                      "packets_per_step": args.packets * world, "l2": "flushed between timed steps (256 MB write)",
                      "launch": {"blocks": tuned[0], "threads": tuned[1], "variant": tuned[2],
                                 "register_variant": tuned[2] % 3 if tuned[2] >= 0 else -1,
                                 "scene_tables": "shared" if tuned[2] >= 3 else "global",
                                 "chosen_by": "smcrt_plan_autotune"}},
           "gpu_launches": 2 * args.steps,
           "clocks": clk.summary()}

    log(f"mixed {value:.3e} packets/s")
    import oracle as O
    # ---- the oracle on a bounded sample of the same workload: the CPU
    # baseline, the reference for the accuracy fields, and the algorithmic
    # work counts of the roofline
    if args.quick or world > 1:
        counts = O.run(wl.with_packets(20_000), fluence=True)[1]
        osamp = None
    else:
        log("oracle leg")
        osamp = oracle_sample(wl, args.oracle_seconds, id_base=0)
        counts = osamp["totals"]
        out["cpu_baseline"] = {"value": osamp["pps"], "unit": UNIT, "cores": osamp["threads"], "kind": "oracle",
                               "sample": f"{osamp['packets']} packets (ids 0..{osamp['packets'] - 1}) of the same "
                                         f"three_layer_slab workload ({args.stepping} stepping), FP64, "
                                         f"{osamp['threads']} threads, 10 batches"}

    # ---- roofline of the packet kernel: FP32 issue and L2 int64 atomics ----
    peaks, src = load_peaks()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = out["clocks"]["sm_mhz"] or peaks.get("clocks_under_load", {}).get("sm_mhz_median") or 1455.0
    nominal_tflops = sm_count * 128 * 2 * mhz * 1e6 / 1e12
    # measured ceilings: the library's FMA and int64-atomic microbenchmarks
    mb = smc.microbench(local)
    peak_tflops = mb["fp32_flops"] / 1e12
    work = algorithmic_work(counts, len(wl.scene.regions))
    achieved = work["flops_per_packet"] * args.packets / kernel_s / 1e12
    atomics = work["atomics_per_packet"] * args.packets / kernel_s
    f_alu = achieved / peak_tflops
    f_atom = atomics / mb["atomics_distinct_per_s"]
    alu = {"achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s", "frac": f_alu,
           "peak_basis": "measured: smcrt_microbench FP32 FMA kernel on this GPU "
                         f"(nominal {sm_count} SMs x 128 lanes x 2 x {mhz:.0f} MHz = {nominal_tflops:.1f} TFLOP/s)"}
    atom = {"achieved": atomics, "peak": mb["atomics_distinct_per_s"], "unit": "int64 atomics/s", "frac": f_atom,
            "peak_basis": "measured: smcrt_microbench int64 atomic adds to scattered addresses of a 64 MiB table",
            "hot_32_address_rate": mb["atomics_hot_per_s"]}
    top = alu if f_alu >= f_atom else atom
    out["roofline"] = {"bound": "alu" if f_alu >= f_atom else "l2_atomics", "achieved": top["achieved"],
                       "peak": top["peak"], "unit": top["unit"], "frac": max(f_alu, f_atom),
                       "traffic": recorded_traffic(),
                       "traffic_note": "DRAM bytes per full-size launch from the ncu summary in profiles/ "
                                       "(null if the kernel changed since)",
                       "kernel": f"packets_{args.precision}",
                       "frac_rule": "max(FP32 flops / FP32 peak, int64 atomics / atomic peak) over the "
                                    "event-timed launch",
                       "fp32": alu, "atomics": atom,
                       "algorithmic_work": work,
                       "work_basis": "FP64 oracle's event counters on a sample of the same workload and step "
                                     "rule, times the per-event FP32 operation counts in bench.py"}
    # lane-issue view: executed thread instructions (ncu, per packet) against
    # the issue ceiling of 152 SMs x 4 schedulers x 32 lanes x clock
    tipp = recorded_traffic("thread_instructions_per_packet") if args.stepping == W.SEGMENT else None
    if tipp:
        issue_peak = sm_count * 4 * 32 * mhz * 1e6   # lane-issue slots per second at the sampled clock
        out["issue_utilisation"] = {"thread_instructions_per_packet": tipp,
                                    "achieved_per_s": tipp * args.packets / kernel_s, "peak_per_s": issue_peak,
                                    "frac": tipp * args.packets / kernel_s / issue_peak,
                                    "note": "thread instructions per packet from the ncu summary in profiles/ "
                                            "(2e5-packet capture of this kernel source)"}
    out["counters_per_packet"] = {k: totals_mixed[k] / args.packets for k in
                                  ("steps", "scene_evals", "scatters", "interfaces", "fresnel", "pieces")}
    out["counters_per_packet"]["refined_fraction_of_fresnel"] = (
        totals_mixed["refined"] / max(1, totals_mixed["fresnel"]))

    if e2e_multi is not None:
        out["e2e"] = e2e_multi

    def leg_buffers(wleg):
        gg = wleg.grid
        return (torch.zeros((gg.n[2], gg.n[1], gg.n[0]), dtype=torch.int64, device="cuda"), smc.totals_tensor())

    def timed_leg(wleg, precision, packets, nsteps, tune):
        """Event-timed launches of ids [0, packets) after a warm-up, each
        after an L2 flush; the autotuner picks the launch shape first."""
        f, t = leg_buffers(wleg)
        p = ctx.plan(wleg, precision)
        choice = p.autotune(min(packets, tune))
        f.zero_()
        t.zero_()
        p.launch(0, min(packets, 1_000_000), wleg.seed, f, t, None, stream.cuda_stream)
        torch.cuda.synchronize()
        evs = []
        for i in range(nsteps):
            l2_flush.fill_(float(i))
            f.zero_()
            t.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            p.launch(0, packets, wleg.seed, f, t, None, stream.cuda_stream)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        assert p.status() == 0
        p.close()
        sec = sum(a.elapsed_time(b) for a, b in evs) / 1e3 / nsteps
        return {"value": packets / sec, "unit": UNIT, "ms_per_step": 1e3 * sec, "packets": packets,
                "steps": nsteps, "stepping": wleg.scene.stepping,
                "launch": {"blocks": choice[0], "threads": choice[1], "variant": choice[2]}}, \
            smc.totals_from_tensor(t)

    def batches(wleg, precision, packets, K, block):
        """Ids [0, packets) as K launches of consecutive ids: per-batch R, T,
        A and fluence block sums, all per packet (untimed)."""
        f, t = leg_buffers(wleg)
        fsum = torch.zeros_like(f)
        p = ctx.plan(wleg, precision)
        per = packets // K
        rta, blocks = [], []
        for k in range(K):
            f.zero_()
            t.zero_()
            p.launch(k * per, per, wleg.seed, f, t, None, stream.cuda_stream)
            fsum += f
            blocks.append(block_sums(f, block) / FX / per)
            tk = smc.totals_from_tensor(t)
            rta.append([tk["R"] / FX / per, tk["T"] / FX / per, tk["A"] / FX / per, tk["max_steps_hit"]])
        assert p.status() == 0
        p.close()
        return np.array(rta), np.array(blocks), fsum.cpu().numpy(), K * per

    def equal_error(wleg, packets, K, block):
        """Mixed against FP64 (bit-identical to the FP64 oracle per packet) on
        the same K batches of ids: the paired R/T/A differences with their
        sigma, and the fluence map block by block."""
        rm, bm, fm, nb = batches(wleg, "mixed", packets, K, block)
        rf, bf, ff, _ = batches(wleg, "fp64", packets, K, block)
        nrm = float(np.linalg.norm(ff.astype(np.float64)))
        d = {"packets": packets, "batches": K, "block_voxels": list(block),
             "step_cap_kills": {"mixed": int(rm[:, 3].sum()), "fp64": int(rf[:, 3].sum())}}
        for c, key in enumerate(("R", "T", "A")):
            diff = rm[:, c] - rf[:, c]
            sig = float(diff.std(ddof=1) / math.sqrt(K))
            z = float(diff.mean() / sig) if sig > 0 else 0.0
            d[key] = {"mixed": float(rm[:, c].mean()), "fp64": float(rf[:, c].mean()),
                      "mixed_minus_fp64": float(diff.mean()), "sigma": sig, "z": z,
                      "z_normal_equivalent": float(_z_from_t(z, K - 1)),
                      "fp64_batch_sigma": float(rf[:, c].std(ddof=1) / math.sqrt(K))}
        d["fluence_blocks"] = paired_block_stats(bm, bf)
        d["fluence_rel_l2_mixed_vs_fp64"] = (float(np.linalg.norm((fm - ff).astype(np.float64))) / nrm
                                             if nrm > 0 else None)
        d["within_3_sigma"] = bool(all(abs(d[k]["z_normal_equivalent"]) < 3 for k in ("R", "T", "A"))
                                   and d["fluence_blocks"].get("pass", False))
        return d, (rm, bm, fm, nb), (rf, bf, ff, nb)

    if not args.quick and world == 1:
        # ---- the headline's comparison: plain FP64 with the SAME step rule,
        # and both precisions with the paper's sphere tracing beside it ------
        log("plain FP64 with the headline's step rule")
        out["fp64"], _ = timed_leg(wl, "fp64", args.packets, args.fp64_steps, 200_000)
        out["fp64"]["mixed_speedup"] = value / out["fp64"]["value"]
        if args.stepping != W.SPHERE_TRACING and args.precision == "mixed":
            log("sphere tracing: mixed and FP64")
            out["mixed_sphere_tracing"], totals_st = timed_leg(wl_plain, "mixed", args.packets, 3, 2_000_000)
            out["mixed_sphere_tracing"]["segment_speedup"] = out["mixed_sphere_tracing"]["ms_per_step"] / (
                1e3 * kernel_s)
            out["fp64_sphere_tracing"], _ = timed_leg(wl_plain, "fp64", args.packets, 1, 200_000)
            out["fp64_sphere_tracing"]["mixed_speedup"] = (out["mixed_sphere_tracing"]["value"]
                                                           / out["fp64_sphere_tracing"]["value"])
        out["mixed_vs_fp64"] = {
            "same_step_rule": {args.stepping: value / out["fp64"]["value"]},
            "note": "packets/s ratio with both precisions on one step rule; the segment-stepping gain is "
                    "reported separately (mixed_sphere_tracing.segment_speedup)"}
        if "fp64_sphere_tracing" in out:
            out["mixed_vs_fp64"]["same_step_rule"][W.SPHERE_TRACING] = out["fp64_sphere_tracing"]["mixed_speedup"]

        # ---- equal error: mixed against FP64 on the same ids -----------------
        log("equal error: paired mixed / FP64 batches")
        ee, legm, legf = equal_error(wl, args.packets, 20, (10, 10, 10))
        out["equal_error"] = ee
        # each precision against the oracle sample (independent ids)
        acc = {}
        for name, (r, b, fmap, nmap) in (("mixed", legm), ("fp64", legf)):
            dd = {}
            for c, key in enumerate(("R", "T", "A")):
                ov = osamp["records"][key] / FX
                gv = r[:, c]
                sig = math.sqrt(ov.var() / ov.size + gv.var(ddof=1) / gv.size)
                dd[key] = float(gv.mean())
                dd[f"{key}_oracle"] = float(ov.mean())
                dd[f"{key}_z"] = float((gv.mean() - ov.mean()) / sig)
            dd["fluence_blocks"] = block_stats(b, osamp["blocks"], paired=False)
            dd.update(fluence_l2(fmap, nmap, osamp["halves"], osamp["half_packets"]))
            acc[name] = dd
        acc["note"] = ("GPU at 1e7 packets in 20 batches against an independent oracle sample in 10 batches; "
                       "z = difference / combined MC sigma; fluence compared block by block (Welch), and as "
                       "the relative L2 difference per packet beside the oracle sample's half-sample noise")
        out["accuracy_vs_oracle"] = acc

        log("end-to-end leg")
        # ---- end to end through the public API with host buffers -------------
        m = smc.Marshalled(wl.scene, wl.source, wl.grid)
        h_flu = np.zeros((g.n[2], g.n[1], g.n[0]), dtype=np.int64)
        import ctypes as C
        h2d = (C.sizeof(m.scene) + C.sizeof(m.prims) + C.sizeof(m.nodes) + C.sizeof(m.regions)
               + C.sizeof(m.source) + C.sizeof(m.grid))
        ctx.run(wl.with_packets(100_000), "mixed", out=h_flu)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_steps = 3
        for i in range(e2e_steps):
            _, te = ctx.run(wl, "mixed", out=h_flu)
        e2e_t = (time.perf_counter() - t0) / e2e_steps
        out["e2e"] = {"value": args.packets / e2e_t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(h_flu.nbytes + C.sizeof(smc.Totals)),
                      "api": "smcrt_run with host scene structs and a host fluence buffer"}

        # ---- the other configs: packets/s of both precisions, equal error ---
        if not args.no_configs:
            log("configs 0, 2, 3")
            cfgs = {}
            runs = [("config0_sphere_pencil", W.sphere_pencil(), 100_000, 100_000, 5, 1_000_000, (5, 5, 5)),
                    ("config2_vessel_network", W.vessel_network(), 100_000_000, args.cfg_fp64_packets,
                     args.cfg_steps, args.cfg_fp64_packets, (20, 20, 20)),
                    ("config3_glass_container", W.glass_container(), 100_000_000, args.cfg_fp64_packets,
                     args.cfg_steps, args.cfg_fp64_packets, (16, 16, 16))]
            for name, wc, n_mixed, n_fp64, nst, n_acc, blk in runs:
                wc = wc.with_stepping(args.stepping)
                log(f"  {name}")
                e = {"workload": wc.name, "grid": list(wc.grid.n), "stepping": args.stepping}
                e["mixed"], tmc = timed_leg(wc, "mixed", n_mixed, nst, 2_000_000)
                e["mixed"]["max_steps_hit"] = tmc["max_steps_hit"]
                e["fp64"], _ = timed_leg(wc, "fp64", n_fp64, 1 if n_fp64 > 200_000 else 3, 20_000)
                e["mixed_over_fp64"] = e["mixed"]["value"] / e["fp64"]["value"]
                e["equal_error"], _, _ = equal_error(wc, n_acc, 20, blk)
                cfgs[name] = e
            out["configs"] = cfgs

        if not args.no_paper_cases and args.precision == "mixed":
            log("paper cases (Table 2 sizes)")
            out["paper_cases"] = paper_cases(ctx, smc, stream, args.stepping)

        # ---- served mix (config 4): Poisson arrivals at 80% of capacity -------
        if args.serve_jobs > 0:
            log("serving leg")
            # capacity of the server on this mix: all jobs of a prefix at once;
            # beside it the same jobs run one after another through smcrt_run,
            # each tallying into a device grid as the served jobs do
            cap_jobs = W.served_mix(min(40, args.serve_jobs), 4, stepping=args.stepping)
            # one small job first: the server's one-time launch-shape trials
            # (on the first mixed job it serves) stay out of the timed batch
            ctx.wait(ctx.submit(cap_jobs[0].with_packets(20_000), "mixed"), -1.0, fluence=False)
            t0 = time.perf_counter()
            for j in cap_jobs:
                g = j.grid
                ctx.run(j, "mixed", out=torch.zeros((g.n[2], g.n[1], g.n[0]), dtype=torch.int64, device="cuda"))
            torch.cuda.synchronize()
            seq_s = time.perf_counter() - t0
            t0 = time.perf_counter()
            jids = [ctx.submit(j, "mixed") for j in cap_jobs]
            for jid in jids:
                ctx.wait(jid, -1.0, fluence=False)
            served_s = time.perf_counter() - t0
            cap = sum(j.npackets for j in cap_jobs) / served_s
            out["serving"] = served_mix(ctx, args.serve_jobs, capacity_pps=cap, stepping=args.stepping)
            out["serving"]["capacity_pps"] = cap
            out["serving"]["batch"] = {"jobs": len(cap_jobs), "packets": sum(j.npackets for j in cap_jobs),
                                       "served_s": served_s, "sequential_s": seq_s,
                                       "sequential": "smcrt_run per job, device fluence grid"}
            out["serving"]["stepping"] = args.stepping
    plan.close()
    print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    ctx.close()


if __name__ == "__main__":
    main()

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

# Algorithmic FP32 work per counted event of the mixed kernel (operations,
# an FMA counted as 2), from the arithmetic of the kernel source:
#   box SDF 22 (3 sub, 3 abs, 3 sub, 3 max, 5 for the squared norm, sqrt,
#   3 min/max, add); region bookkeeping 5 per region (compare, abs, compare,
#   2 selects); bounding box = one box SDF;
#   step: tally set-up 40 + move 6 + tau update 2;  voxel piece 16;
#   interaction: weight 3, HG 12, azimuth sincos 4, basis 14, rotation 15,
#   normalisation 8, roulette 2, log 4 = 62.
FLOPS_BOX = 22
FLOPS_REGION = 5
FLOPS_STEP = 48
FLOPS_PIECE = 16
FLOPS_INTERACTION = 62


def three_layer_flops(t: dict) -> float:
    per_eval = 3 * FLOPS_BOX + 3 * FLOPS_REGION + FLOPS_BOX
    return (t["scene_evals"] * per_eval + t["steps"] * FLOPS_STEP + t["pieces"] * FLOPS_PIECE
            + t["scatters"] * FLOPS_INTERACTION)


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


def oracle_sample(wl, seconds: float, id_base: int = 0):
    """Time the FP64 oracle, as it stands, on a bounded sample sized to take
    about ``seconds``, run as two halves of consecutive ids; returns
    (packets/s, packets, threads, per-packet records, the halves' fluence
    maps)."""
    import numpy as np
    import oracle as O
    threads = os.cpu_count() or 1
    n0 = 2000
    t0 = time.perf_counter()
    O.run(wl.with_packets(n0), id_base, id_base + n0, threads=threads, fluence=True)
    rate0 = n0 / (time.perf_counter() - t0)
    h = int(max(n0, min(5_000_000, rate0 * seconds))) // 2
    t0 = time.perf_counter()
    f1, _, r1 = O.run(wl.with_packets(h), id_base, id_base + h, threads=threads, records=True)
    f2, _, r2 = O.run(wl.with_packets(h), id_base + h, id_base + 2 * h, threads=threads, records=True)
    dt = time.perf_counter() - t0
    return 2 * h / dt, 2 * h, threads, np.concatenate([r1, r2]), (f1, f2)


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
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--serve-jobs", type=int, default=100)
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
    flu_legs = {"mixed": flu.cpu().numpy()}   # the last timed step's map (1e7 packets)
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

    # ---- roofline of the packet kernel (ALU-bound: FP32 issue) -----------
    peaks, src = load_peaks()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = out["clocks"]["sm_mhz"] or peaks.get("clocks_under_load", {}).get("sm_mhz_median") or 1455.0
    nominal_tflops = sm_count * 128 * 2 * mhz * 1e6 / 1e12
    # measured ceilings: the library's FMA and int64-atomic microbenchmarks
    mb = smc.microbench(local)
    peak_tflops = mb["fp32_flops"] / 1e12
    flops = three_layer_flops(totals_mixed)
    achieved = flops / kernel_s / 1e12
    atomics = totals_mixed["pieces"] / kernel_s
    out["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                       "frac": achieved / peak_tflops, "traffic": recorded_traffic(),
                       "traffic_note": "DRAM bytes per full-size launch from the ncu summary in profiles/ "
                                       "(null if the kernel changed since)",
                       "peak_basis": "measured: smcrt_microbench FP32 FMA kernel on this GPU "
                                     f"(nominal {sm_count} SMs x 128 lanes x 2 x {mhz:.0f} MHz = "
                                     f"{nominal_tflops:.1f} TFLOP/s)",
                       "kernel": f"packets_{args.precision}",
                       "algorithmic_flops_per_packet": flops / args.packets,
                       "atomics_per_s": atomics,
                       "atomics_peak_distinct_per_s": mb["atomics_distinct_per_s"],
                       "atomics_peak_hot_per_s": mb["atomics_hot_per_s"],
                       "atomics_frac": atomics / mb["atomics_distinct_per_s"]}
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

    def timed_leg(wleg, precision, nsteps, tune):
        p = ctx.plan(wleg, precision)
        p.autotune(tune)
        step(min(args.packets, 1_000_000), p, wleg.seed, id0)
        torch.cuda.synchronize()
        evs = []
        for i in range(nsteps):
            l2_flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(args.packets, p, wleg.seed, id0)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        p.close()
        return sum(a.elapsed_time(b) for a, b in evs) / 1e3 / nsteps, smc.totals_from_tensor(tot), flu.cpu().numpy()

    if e2e_multi is not None:
        out["e2e"] = e2e_multi
    if not args.quick and world == 1:
        # ---- mixed precision with plain sphere tracing (the paper's step) ---
        totals_st = None
        if args.stepping != W.SPHERE_TRACING and args.precision == "mixed":
            log(f"mixed {value:.3e} packets/s; timing mixed with sphere tracing")
            t_st, totals_st, flu_legs["mixed_sphere_tracing"] = timed_leg(wl_plain, "mixed", 3,
                                                                          min(args.packets, 2_000_000))
            out["mixed_sphere_tracing"] = {"value": args.packets / t_st, "unit": UNIT, "ms_per_step": 1e3 * t_st,
                                           "segment_speedup": t_st / kernel_s}
        # ---- plain FP64 mode (sphere tracing) on the same workload ----------
        log("timing the plain FP64 mode")
        plan64 = ctx.plan(wl_plain, "fp64")
        plan64.autotune(100_000)
        step(min(args.packets, 1_000_000), plan64, wl.seed, id0)
        torch.cuda.synchronize()
        e64 = []
        for i in range(args.fp64_steps):
            l2_flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(args.packets, plan64, wl.seed, id0)
            b.record(stream)
            e64.append((a, b))
        torch.cuda.synchronize()
        t64 = sum(a.elapsed_time(b) for a, b in e64) / 1e3 / args.fp64_steps
        totals_fp64 = smc.totals_from_tensor(tot)
        flu_legs["fp64"] = flu.cpu().numpy()
        plan64.close()
        out["fp64"] = {"value": args.packets / t64, "unit": UNIT, "ms_per_step": 1e3 * t64,
                       "stepping": W.SPHERE_TRACING,
                       "mixed_speedup": (args.packets / kernel_s) / (args.packets / t64)}

        log(f"fp64 {args.packets / t64:.3e} packets/s; end-to-end leg")
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

        log("oracle leg")
        # ---- accuracy against the FP64 oracle, and the oracle's CPU timing ----
        o_pps, o_n, o_threads, o_rec, o_halves = oracle_sample(wl, args.oracle_seconds, id_base=0)
        out["cpu_baseline"] = {"value": o_pps, "unit": UNIT, "cores": o_threads, "kind": "oracle",
                               "sample": f"{o_n} packets (ids 0..{o_n - 1}) of the same three_layer_slab "
                                         f"workload ({args.stepping} stepping), FP64, {o_threads} threads"}
        acc = {}
        legs = [("mixed", totals_mixed), ("fp64", totals_fp64)]
        if totals_st is not None:
            legs.append(("mixed_sphere_tracing", totals_st))
        for name, t in legs:
            d = {}
            for k in ("R", "T", "A"):
                ov = o_rec[k] / FX
                sig = math.sqrt(ov.var() / ov.size + ov.var() / args.packets)
                gv = t[k] / FX / args.packets
                d[k] = gv
                d[f"{k}_oracle"] = float(ov.mean())
                d[f"{k}_z"] = (gv - float(ov.mean())) / sig
            d.update(fluence_l2(flu_legs[name], args.packets, o_halves, o_n // 2))
            acc[name] = d
        out["accuracy_vs_oracle"] = acc
        out["accuracy_vs_oracle"]["note"] = ("GPU at 1e7 packets vs oracle sample; z = difference / combined "
                                             "MC sigma; fluence_rel_l2 = |phi_gpu - phi_oracle| / |phi_oracle| "
                                             "per packet, beside the oracle sample's own noise. FP64 mode is "
                                             "bit-identical to the oracle packet by packet")

        if not args.no_paper_cases and args.precision == "mixed":
            log("paper cases (Table 2 sizes)")
            out["paper_cases"] = paper_cases(ctx, smc, stream, args.stepping)

        # ---- served mix: Poisson arrivals at 80% of measured capacity ---------
        if args.serve_jobs > 0:
            log("serving leg")
            # capacity of the server on this mix: all jobs of a prefix at once
            cap_jobs = W.served_mix(min(40, args.serve_jobs), 4, stepping=args.stepping)
            t0 = time.perf_counter()
            jids = [ctx.submit(j, "mixed") for j in cap_jobs]
            for jid in jids:
                ctx.wait(jid, -1.0, fluence=False)
            cap = sum(j.npackets for j in cap_jobs) / (time.perf_counter() - t0)
            out["serving"] = served_mix(ctx, args.serve_jobs, capacity_pps=cap, stepping=args.stepping)
            out["serving"]["capacity_pps"] = cap
            out["serving"]["stepping"] = args.stepping
    plan.close()
    print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    ctx.close()


if __name__ == "__main__":
    main()

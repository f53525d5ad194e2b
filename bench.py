"""Benchmark of the FSLBM time step on GB300.

Default workload: the rising Taylor bubble, 160 x 160 x 1024 cells, D3Q19
TRT, FP32 PDFs (fill level and mass in FP64), free-surface BC variant OM,
curvature-driven Laplace pressure and per-bubble volume tracking: one step
runs every stage of the method (geometry, bulk stream-collide, interface BC
and mass exchange, conversion, excess mass, bubble pressure).

Prints ONE JSON line (rank 0).  ``value`` is whole-job MLUPS (cell updates
per second over all cells of all ranks); the timed region holds exactly
``--steps`` steps with the state resident in HBM.  ``e2e`` repeats the
measurement through the C ABI with host buffers: initial state uploaded from
pinned host memory and the fill-level field read back inside the timed region.

``--impl reference`` times the plain CPU oracle (single thread, as it stands)
on a bounded sample of the same workload; it is the only other use of
``oracle/`` here besides the ``cpu_baseline`` field.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FSLBM MLUPS and % HBM roofline on 1 GB300; batched/served vs plain at stated error; p50/p99"
Q = 19
S_BYTES = {"FP32": 4, "FP64": 8, "FP16S": 2, "BF16S": 2, "FP32MC": 4, "FP16SMC": 2}
REST_BYTES = {"FP32MC": 4, "FP16SMC": 4}  # the int32 rest slice of the mass-conserving formats
DTYPE = {"FP32": "f32", "FP64": "f64", "FP16S": "f32 (fp16 storage)", "BF16S": "f32 (bf16 storage)",
         "FP32MC": "f32 (f32 storage, int32 rest)", "FP16SMC": "f32 (fp16 storage, int32 rest)"}


# ------------------------------------------------------------------ helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, ws: int) -> float:
    """Max of a per-rank float over all ranks (identity for one rank)."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(cells_per_rank: int, ws: int, steps: int, ms: float) -> float:
    """Whole-job throughput: cell updates of all ranks over the slowest rank's time."""
    return cells_per_rank * ws * steps / (ms * 1e-3) / 1e6


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


# what k_bulk is compiled from: its own header, the cell layer, the common
# types and the build flags
KERNEL_SOURCES = tuple("paper_2207_13962_gb300/" + f for f in (
    "csrc/fslbm_bulk.cuh", "csrc/fslbm_cell.cuh", "csrc/fslbm_common.cuh", "csrc/fslbm_kernels.cuh", "build.py"))


def kernel_source_hash() -> str:
    """SHA-256 of the fused geometry + bulk sweep's sources (the ncu traffic
    applies only to them)."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def bulk_traffic(n_liquid: float, precision: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    capture (profiles/k_bulk_geo_traffic.json), scaled by liquid cells; None
    when the kernel sources changed since the capture or the precision
    differs."""
    try:
        with open(os.path.join(ROOT, "profiles", "k_bulk_geo_traffic.json")) as fh:
            t = json.load(fh)
    except Exception:
        return None
    if t.get("kernel_source_sha256") != kernel_source_hash() or t.get("precision") != precision:
        return None
    return t["dram_bytes_per_launch"] * n_liquid / t["liquid_cells"]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------- workloads

def make_workload(name: str, variant: str):
    from paper_2207_13962_gb300 import scenarios as S
    if name == "taylor_bubble":
        sc = S.taylor_bubble(variant=variant)
        desc = ("rising Taylor bubble 160x160x1024, tube D=128, bubble 96x256, D3Q19 TRT, "
                "g=1e-6, sigma=1e-4, nu=5e-3, bubble model")
    elif name == "taylor_bubble_256":
        sc = S.taylor_bubble(nz=256, bubble_len=96, z0=64, z_ref=128.0, variant=variant)
        desc = ("rising Taylor bubble, short tube 160x160x256 (profiling case), bubble 96x96, D3Q19 TRT, "
                "g=1e-6, sigma=1e-4, nu=5e-3, bubble model")
    elif name == "dam_break":
        sc = S.dam_break(variant=variant)
        desc = "rectangular dam break 256x128x64, column 64^3, D3Q19 TRT, g=1e-5, nu=1e-3, no-slip"
    elif name == "box256":
        sc = S.flat_interface(nx=256, ny=256, nz=256, depth=249.5, g=1e-5, variant=variant)
        desc = "256^3 liquid box with a flat surface (bulk ceiling, profiling case), D3Q19 TRT"
    elif name == "box512":
        sc = S.flat_interface(nx=512, ny=512, nz=512, depth=505.5, g=1e-5, variant=variant)
        desc = "512^3 liquid box with a flat surface (bulk ceiling), D3Q19 TRT"
    else:
        raise SystemExit(f"unknown workload {name}")
    return sc, desc


def oracle_sample(sc, name: str, zlo: int, zhi: int):
    """A z-slab of the workload's initial state (walls at the cut faces)."""
    from paper_2207_13962_gb300 import scenarios as S
    return S.z_slab(sc, zlo, zhi)


def _time_oracle(smp, steps_budget_s, max_steps, openmp=False, warmup=1):
    from oracle import Oracle
    from paper_2207_13962_gb300 import scenarios as S
    o = Oracle(*smp.shape, **S.make_oracle_kwargs(smp), openmp=openmp)
    o.init(smp.fill, smp.flags, smp.velocity, smp.density)
    o.step(warmup)
    done, t0 = 0, time.perf_counter()
    while done < max_steps:
        o.step(1)
        done += 1
        if time.perf_counter() - t0 > steps_budget_s:
            break
    return done, time.perf_counter() - t0


def run_oracle_sample(sc, name, steps_budget_s=15.0, max_steps=50, openmp=False):
    """Oracle MLUPS on a bounded sample of the workload: one host thread, or
    all host threads with the OpenMP build (its per-cell geometry and
    stream-collide loops shared out)."""
    if name == "taylor_bubble":
        smp = oracle_sample(sc, name, 352, 416)
    elif name == "taylor_bubble_256":
        smp = oracle_sample(sc, name, 128, 160)
    elif name in ("box256", "box512"):
        smp = oracle_sample(sc, name, sc.shape[2] - 64, sc.shape[2])
    else:
        smp = sc
    done, dt = _time_oracle(smp, steps_budget_s, max_steps, openmp=openmp)
    cores = (os.cpu_count() or 1) if openmp else 1
    threads = f"{cores} host threads (OpenMP build)" if openmp else "1 host thread"
    return {"value": smp.N * done / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{smp.name}: {smp.shape[0]}x{smp.shape[1]}x{smp.shape[2]} cells of the same "
                      f"initial state, {done} steps after 1 warm-up step, FP64, {threads}",
            "seconds": dt}


def cpu_baseline_set(sc, name):
    """The oracle timed on the host: the workload's bounded sample on one
    thread (the headline value) and on all threads, the standing gravity wave
    in full (1000 steps, one thread) and the first steps of the rectangular
    dam break on all threads; core counts stated with each."""
    from paper_2207_13962_gb300 import scenarios as S
    out = run_oracle_sample(sc, name)
    out.pop("seconds", None)
    omp = run_oracle_sample(sc, name, steps_budget_s=8.0, openmp=True)
    omp.pop("seconds", None)
    out["all_cores"] = omp
    wave = S.gravity_wave(variant="OM")
    done, dt = _time_oracle(wave, 60.0, 1000, warmup=0)
    out["gravity_wave_32x64x1"] = {"value": wave.N * done / dt / 1e6, "unit": "MLUPS", "cores": 1,
                                   "sample": f"all {done} steps of the 32x64x1 gravity wave, FP64, 1 host thread"}
    dam = S.dam_break(variant="OM")
    done, dt = _time_oracle(dam, 10.0, 500, openmp=True, warmup=0)
    out["dam_break_256x128x64"] = {"value": dam.N * done / dt / 1e6, "unit": "MLUPS",
                                   "cores": os.cpu_count() or 1,
                                   "sample": f"first {done} steps of the 256x128x64 dam break, FP64, "
                                             f"{os.cpu_count()} host threads (OpenMP build)"}
    return out


# -------------------------------------------------------------- our arm

def bench_ours(args, ws, rank, local):
    import torch
    from paper_2207_13962_gb300 import fslbm

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec = args.precision
    sc, desc = make_workload(args.workload, args.variant)
    stream = torch.cuda.Stream()
    ctx = fslbm.context_for(sc, precision=prec, stream=stream.cuda_stream)
    N = sc.N

    # warm-up
    ctx.step(args.warmup)
    if ctx.sync() != 0:
        raise SystemExit(f"unstable during warm-up: {ctx.lib.fslbm_last_error(ctx.h).decode()}")
    obs0 = ctx.observables()
    segs_bytes = None

    # ---- timed region: exactly K steps, state resident in HBM
    ctx.set_timing(False)  # resets the launch counter; CUDA-graph launches
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    ck = clocks.stop()
    ms_local = e0.elapsed_time(e1)
    _, launches = ctx.stage_times()
    st = ctx.sync()
    obs1 = ctx.observables()
    ms = max_over_ranks(ms_local, ws)
    value = whole_job_mlups(N, ws, args.steps, ms)

    # ---- per-stage CUDA-event timing (kernels launched one by one on the
    # context's stream) for the roofline of the dominant kernel
    wc1 = ctx.work_counts()
    ctx.set_timing(True)
    ctx.step(args.steps)
    times, _ = ctx.stage_times()
    ctx.set_timing(False)
    obs2 = ctx.observables()
    wc2 = ctx.work_counts()
    bulk_ms = times["bulk"] / args.steps
    n_liq = 0.5 * (obs1["n_liquid"] + obs2["n_liquid"])
    # algorithmic bytes of one bulk launch: read + write q PDFs and read one
    # flag byte per liquid cell (the sweep visits liquid cells only)
    alg_bytes = n_liq * (2 * ((Q - (1 if prec in REST_BYTES else 0)) * S_BYTES[prec] + REST_BYTES.get(prec, 0)) + 1)
    fused = prec != "FP64"
    if fused:
        # the FP32 and 16-bit engines run the geometry tiles in the same
        # launch: each tile's 512 cells read once (FP64 fill level + flag),
        # each interface cell's normal, gas density (FP32) and class written
        tiles = 0.5 * (wc1["geometry_tiles"] + wc2["geometry_tiles"])
        n_if = 0.5 * (wc1["interface_cells"] + wc2["interface_cells"])
        alg_bytes += tiles * 512 * 9 + n_if * (4 * 4 + 1)
    achieved = alg_bytes / (bulk_ms * 1e-3) / 1e9
    peaks, peak_kind = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    share = {k: round(v / max(sum(times.values()), 1e-12), 4) for k, v in times.items()}

    # ---- end to end through the C ABI with host buffers: init from pinned
    # host arrays, K steps, fill-level readback; one untimed pass first (the
    # first init of a process loads the init kernels and maps the pinned pages)
    pin_fill = torch.from_numpy(sc.fill).pin_memory()
    pin_flags = torch.from_numpy(sc.flags).pin_memory()
    pin_den = torch.from_numpy(sc.density).pin_memory() if sc.density is not None else None
    out_fill = torch.empty(N, dtype=torch.float64).pin_memory()

    def e2e_pass(k):
        rc = ctx.init_raw(pin_fill.data_ptr(), pin_flags.data_ptr(), None,
                          pin_den.data_ptr() if pin_den is not None else None)
        if rc != 0:
            raise SystemExit("e2e init failed")
        ctx.step(k)
        rc = ctx.lib.fslbm_read_fields(ctx.h, None, fslbm.C.c_void_p(out_fill.data_ptr()), None, None)
        if rc != 0:
            raise SystemExit("e2e read failed")

    e2e_pass(1)
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    e2e_pass(args.steps)
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
    h2d = sc.fill.nbytes + sc.flags.nbytes + (sc.density.nbytes if sc.density is not None else 0)
    d2h = out_fill.numel() * 8
    e2e = {"value": N * ws * args.steps / e2e_s / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "note": f"fslbm_init from pinned host arrays + {args.steps} steps + fill-level readback, "
                   f"after one untimed pass"}

    # ---- secondary workload: the rectangular dam break (configs' second entry)
    other = {}
    if args.workload == "taylor_bubble" and not args.no_secondary:
        sc2, desc2 = make_workload("dam_break", args.variant)
        c2 = fslbm.context_for(sc2, precision=prec, stream=stream.cuda_stream)
        c2.step(args.warmup)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        c2.step(args.steps)
        f1.record(stream)
        torch.cuda.synchronize()
        dms = f0.elapsed_time(f1) / args.steps
        o2 = c2.observables()
        other["dam_break_256x128x64"] = {
            "mlups": round(sc2.N / dms / 1e3, 1), "ms_per_step": round(dms, 5),
            "mflups": round((o2["n_liquid"] + o2["n_interface"]) / dms / 1e3, 1),
            "note": "L2 not flushed: the touched state (~40 MB) fits in L2"}
        c2.close()

    batched = served = None
    if args.workload == "taylor_bubble" and not args.no_secondary and ws == 1:
        ctx.close()
        batched = bench_batch(args, emit=False)
        served = bench_serve(args, emit=False)

    line = None
    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline_set(sc, args.workload)
        line = {
            "metric": METRIC,
            "value": round(value, 2),
            "unit": "MLUPS",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(ms / args.steps, 6),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": DTYPE[prec],
            "data": "synthetic (seeded generator, no dataset)",
            "config": {
                "workload": desc,
                "cells_per_gpu": N,
                "lattice": "D3Q19", "collision": "TRT", "precision": prec, "bc_variant": args.variant,
                "parallelism": f"{ws} independent replica(s), one domain per GPU, no collective",
                "l2": f"inputs larger than L2: {2 * Q * S_BYTES[prec] * N / 1e9:.2f} GB of PDFs",
                "mflups": round((obs1["n_liquid"] + obs1["n_interface"]) * ws * args.steps / (ms * 1e-3) / 1e6, 2),
                "interface_cells": obs1["n_interface"],
                "mass_drift_rel": (obs1["total_mass"] - obs0["total_mass"]) / obs0["total_mass"],
                "status": int(st),
            },
            "roofline": {
                "bound": "hbm",
                "kernel": ("k_bulk_geo (geometry tiles, then the pull stream-collide of liquid cells, in one "
                           "persistent launch)" if fused else "k_bulk (pull stream-collide of liquid cells)"),
                "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": f"{peak_kind} (hbm_gbs, burst copy)",
                "traffic": (round(bulk_traffic(n_liq, prec)) if bulk_traffic(n_liq, prec) else None),
                "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of the "
                                "160x160x256 profiling case, scaled by liquid cells "
                                "(profiles/k_bulk_geo_traffic.json)",
                "alg_bytes_per_launch": int(alg_bytes), "launch_ms": round(bulk_ms, 6),
                "stage_share": share,
            },
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": ck,
            "other_workloads": other,
            "batched": batched,
            "served": served,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line


# ------------------------------------------------ batched and served runs

def _front_radius(fill, L):
    """Cylindrical dam break: radius of the wetted floor, sqrt(sum phi / pi)
    over the bottom layer."""
    return float(np.sqrt(fill.reshape(L, L, L)[0].sum() / np.pi))


def _crown(fill, flags, L):
    """Drop impact: height of the highest interface cell, k + phi."""
    from paper_2207_13962_gb300 import scenarios as S
    f3 = fill.reshape(L, L, L)
    k = np.nonzero((flags.reshape(L, L, L) == S.IFACE).any(axis=(1, 2)))[0]
    if k.size == 0:
        return 0.0
    top = int(k.max())
    return float(top + f3[top][flags.reshape(L, L, L)[top] == S.IFACE].max())


def _lifted(fill, L, depth):
    """Drop impact: liquid volume above the undisturbed pool, the sum of the
    fill level over the layers k >= depth + 2 (the drop's remnant and the
    crown sheet).  An integral of the fill level, so it moves by about the
    size of the fill levels' own error, unlike the crown height, which jumps
    by a cell when one interface cell at the tip appears or empties."""
    k0 = int(np.ceil(depth)) + 2
    return float(fill.reshape(L, L, L)[k0:].sum())


def bench_batch(args, emit=True):
    """64 cylindrical dam breaks of seeded uneven sizes (D3Q27 TRT): one at a
    time in plain FP32, as one batch in FP32 and as one batch in the reduced
    (by default mass-conserving FP16) storage.  Every run is brought to the
    same step count, so the front radii compare at the same time; the error
    is relative to the plain FP32 runs."""
    import torch
    from paper_2207_13962_gb300 import fslbm
    from paper_2207_13962_gb300 import scenarios as S
    torch.cuda.set_device(0)
    prm = S.cylinder_batch_params(n=args.batch_n)
    scs = [S.cylinder_dam_break(**p, q=27) for p in prm]
    cells = sum(sc.N for sc in scs)
    steps = args.batch_steps
    total = args.batch_warmup + steps
    stream = torch.cuda.Stream()

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    def observe(ctxs):
        # (floor-layer front radius, total mass, seed-fill maximum front radius)
        return [(_front_radius(c.read(pdf=False)["fill"], sc.shape[0]), c.observables()["total_mass"],
                 c.front(0, (sc.shape[0] / 2.0, sc.shape[1] / 2.0))["r_max"])
                for sc, c in zip(scs, ctxs)]

    res, obs_at = {}, {}
    # plain: each domain alone, one after another, FP32
    ctxs = [fslbm.context_for(sc, precision="FP32", stream=stream.cuda_stream) for sc in scs]
    m0 = [c.observables()["total_mass"] for c in ctxs]
    for c in ctxs:
        c.step(total - steps)
    t = timed(lambda: [c.step(steps) for c in ctxs])
    ref = observe(ctxs)
    res["plain_fp32"] = {"mlups": round(cells * steps / t / 1e6, 1), "seconds": round(t, 4),
                         "mass_drift_rel_max": max(abs(o[1] - m) / m for o, m in zip(ref, m0))}
    for c in ctxs:
        c.close()
    for prec in ["FP32"] + [p for p in args.batch_precision.split(",") if p != "FP32"]:
        ctxs = [fslbm.context_for(sc, precision=prec, stream=stream.cuda_stream) for sc in scs]
        m0 = [c.observables()["total_mass"] for c in ctxs]
        batch = fslbm.Batch(ctxs, stream=stream.cuda_stream)
        tune = batch.autotune(steps=1) if args.autotune else batch.tuning()
        done = ctxs[0].observables()["step"]
        batch.step(max(0, total - steps - done))
        l0 = batch.launches()
        t = timed(lambda: batch.step(steps))
        obs_at[prec] = observe(ctxs)
        res[f"batched_{prec.lower()}"] = {
            "mlups": round(cells * steps / t / 1e6, 1), "seconds": round(t, 4), "tuning": tune,
            "launches_per_step": (batch.launches() - l0) / steps,
            "mass_drift_rel_max": max(abs(o[1] - m) / m for o, m in zip(obs_at[prec], m0)),
            "front_radius_rel_err_vs_plain_fp32": max(abs(a[0] - b[0]) / max(b[0], 1e-30)
                                                      for a, b in zip(obs_at[prec], ref)),
            "seed_fill_rmax_rel_err_vs_plain_fp32": max(abs(a[2] - b[2]) / max(b[2], 1e-30)
                                                        for a, b in zip(obs_at[prec], ref))}
        batch.close()
        for c in ctxs:
            c.close()
    out = {"workload": f"{len(scs)} cylindrical dam breaks, cubes of seeded sides "
                       f"{min(p['L'] for p in prm)}..{max(p['L'] for p in prm)} (seed 2207), D3Q27 TRT, "
                       f"g=1e-5, nu=1e-3, OM; {steps} timed steps after {total - steps}",
           "cells": cells, "unit": "MLUPS", "results": res,
           "observable": "front radius sqrt(sum of floor-layer fill / pi), and the maximum radius of the "
                         "floor layer's seed-fill front cells (fslbm_front), relative to the plain FP32 runs"}
    if emit:
        print(json.dumps({"metric": METRIC, "workload": "batched cylindrical dam breaks", **out,
                          "data": "synthetic (seeded generator, no dataset)"}), flush=True)
    return out


def _compact_drop(kw):
    from paper_2207_13962_gb300 import scenarios as S
    return S.drop_impact_compact(**kw)


def _drop_states(trace):
    """Compact initial states of a request trace, built by a spawned process
    pool (before any CUDA call of this process)."""
    import multiprocessing as mp
    kws = [kw for _, kw in trace]
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1, len(kws)))) as pool:
        return pool.map(_compact_drop, kws, chunksize=1)


def _replay(arrivals, step_fn):
    """Replays arrival times (seconds, sorted) in real time.  step_fn(ready)
    gets the arrived requests that have not started (it removes those it
    starts) and returns (finished [(k, result)], busy).  Time-to-result runs
    from a request's arrival to its result on the host.  Returns the results
    by trace index and the makespan (trace start to the last result)."""
    n, nxt, ready, results = len(arrivals), 0, [], {}
    t0 = time.perf_counter()
    while len(results) < n:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= now:
            ready.append(nxt)
            nxt += 1
        done, busy = step_fn(ready)
        t = time.perf_counter() - t0
        for k, r in done:
            r["ttr"] = t - arrivals[k]
            results[k] = r
        if not busy and not ready and nxt < n:
            time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
    return results, time.perf_counter() - t0


class _Expander:
    """Expands compact requests into full host arrays on worker threads, a
    few requests ahead of the ones being started, so that the host loop keeps
    the GPU fed meanwhile (the server's poll and the steps release the
    interpreter).  Both servers of the comparison use it."""

    def __init__(self, comp, ahead):
        import concurrent.futures as cf
        self.comp, self.ahead = comp, ahead
        self.pool = cf.ThreadPoolExecutor(max_workers=2)
        self.fut = {}

    def prefetch(self, ready):
        for k in ready[:self.ahead]:
            if k not in self.fut:
                self.fut[k] = self.pool.submit(self.comp[k].expand)

    def done(self, k):
        return k in self.fut and self.fut[k].done()

    def take(self, k):
        if k not in self.fut:
            self.fut[k] = self.pool.submit(self.comp[k].expand)
        return self.fut.pop(k).result()

    def close(self):
        self.pool.shutdown()


def bench_serve(args, emit=True):
    """Drop impacts arriving as a Poisson stream (seeded sizes 96..256),
    replayed in real time: a FIFO server that runs each request alone in
    plain FP32, one after another, against the continuous-batching server in
    FP32 and in the reduced storage formats.  Requests wait on the host in
    compact form (cell types and interface fill levels); worker threads
    expand the next few of them to full host arrays while the GPU runs, and
    a request is handed over when it starts (FIFO) or when the server's own
    queue has room (at most --max-active waiting there), so a long trace
    holds about one byte per cell on the host.  Time-to-result runs from a
    request's arrival to its result on the host; the observables are
    relative to the plain FP32 run."""
    from paper_2207_13962_gb300 import scenarios as S
    trace = S.drop_requests(n=args.requests, rate=args.rate)
    comp = _drop_states(trace)  # before the first CUDA call: the pool is spawned
    import torch
    from paper_2207_13962_gb300 import fslbm
    torch.cuda.set_device(0)
    arrivals = [t for t, _ in trace]
    steps = args.serve_steps
    cells = sum(c.N for c in comp)
    out = {}
    les = {"smagorinsky_cs": args.serve_cs} if args.serve_cs > 0 else {}

    def observe(k, fill, flags):
        return {"crown": _crown(fill, flags, comp[k].shape[0]),
                "lifted": _lifted(fill, comp[k].shape[0], comp[k].depth)}

    # FIFO, one at a time, plain FP32 contexts
    exp = _Expander(comp, 2)

    def fifo_step(ready):
        exp.prefetch(ready)
        if not ready:
            return [], False
        k = ready.pop(0)
        c = fslbm.context_for(exp.take(k), precision="FP32", **les)
        M0 = c.observables()["total_mass"]
        c.step(steps)
        c.sync()
        r = c.read(pdf=False)
        obs = c.observables()
        c.close()
        return [(k, {**observe(k, r["fill"], r["flags"]), "status": obs["status"],
                     "drift": abs(obs["total_mass"] - M0) / M0})], True

    res, makespan = _replay(arrivals, fifo_step)
    exp.close()
    ref = res
    ttr = [res[k]["ttr"] for k in range(len(comp))]
    stable_ref = {k for k in res if res[k]["status"] == 0}
    out["plain_fp32_fifo"] = {"mlups": round(cells * steps / makespan / 1e6, 1), "makespan_s": round(makespan, 3),
                              "p50_s": round(float(np.percentile(ttr, 50)), 4),
                              "p99_s": round(float(np.percentile(ttr, 99)), 4),
                              "unstable_runs": sorted(set(res) - stable_ref),
                              "mass_drift_rel_max_stable": max((res[k]["drift"] for k in stable_ref), default=None)}
    arms = [] if args.skip_served_fp32 else ["FP32"]
    for prec in arms + [p for p in args.batch_precision.split(",") if p != "FP32"]:
        srv = fslbm.Server(q=19, precision=prec, max_active=args.max_active, chunk_steps=args.chunk_steps)
        live = {}
        exp = _Expander(comp, 4)

        def serve_step(ready):
            exp.prefetch(ready)
            while ready and exp.done(ready[0]) and srv.stats()["queued"] < args.max_active:
                k = ready.pop(0)
                live[srv.submit(exp.take(k), steps, **les)] = k
            if not live:
                if not ready:
                    return [], False
                k = ready.pop(0)  # nothing on the GPU: wait for this expansion
                live[srv.submit(exp.take(k), steps, **les)] = k
            srv.poll()
            got = []
            for rid in list(live):
                r = srv.result(rid)
                if r is not None:
                    k = live.pop(rid)
                    got.append((k, {**observe(k, r["fill"], r["flags"]), "status": r["status"]}))
            return got, True

        res, makespan = _replay(arrivals, serve_step)
        exp.close()
        ttr = [res[k]["ttr"] for k in range(len(comp))]
        both = sorted(k for k in stable_ref if res[k]["status"] == 0)  # stable alone and served
        rel = lambda key: max((abs(res[k][key] - ref[k][key]) / max(abs(ref[k][key]), 1e-30) for k in both),
                              default=None)
        st = srv.stats()
        out[f"served_{prec.lower()}"] = {
            "mlups": round(cells * steps / makespan / 1e6, 1), "makespan_s": round(makespan, 3),
            "p50_s": round(float(np.percentile(ttr, 50)), 4), "p99_s": round(float(np.percentile(ttr, 99)), 4),
            "unstable_runs": sorted(k for k in res if res[k]["status"] != 0), "compared_runs": len(both),
            "crown_rel_err_vs_plain_fp32": rel("crown"), "lifted_volume_rel_err_vs_plain_fp32": rel("lifted"),
            "max_active_seen": st["max_active_seen"],
            "batch_rebuilds": st["batch_rebuilds"]}
        srv.close()
    sides = [c.shape[0] for c in comp]
    summary = {"workload": f"{len(comp)} drop impacts of seeded sides {min(sides)}..{max(sides)} (seed 13962), "
                           f"Poisson arrivals {args.rate}/s, {steps} steps each, D3Q19 TRT OM"
                           + (f", Smagorinsky C_S {args.serve_cs}" if args.serve_cs > 0 else "") + ", replayed in real time",
               "cells": cells, "unit": "MLUPS", "results": out, "max_active": args.max_active,
               "chunk_steps": args.chunk_steps,
               "time_to_result": "from the request's arrival to its result on the host",
               "errors": "over the runs that stayed stable (status 0) alone and served; unstable_runs lists the "
                         "trace indices that ended with FSLBM_EUNSTABLE",
               "observable": "crown height max over interface cells of (k + fill), and the liquid volume above "
                             "the pool (sum of the fill level over layers k >= depth + 2), each relative to the "
                             "plain FP32 run"}
    if emit:
        print(json.dumps({"metric": METRIC, "workload": "served drop impacts (continuous batching)", **summary,
                          "data": "synthetic (seeded generator, no dataset)"}), flush=True)
    return summary


# ------------------------------------------- observables of reduced precision

def _perturbed(sc, seed=1, size=1e-7):
    """The scenario with its interface cells' fill levels moved by a seeded
    uniform +-size (the conditioning floor: how far an observable moves
    under a perturbation of FP32-rounding size)."""
    import dataclasses
    from paper_2207_13962_gb300 import scenarios as S
    rng = np.random.Generator(np.random.PCG64(seed))
    fill = sc.fill.copy()
    m = sc.flags == S.IFACE
    fill[m] = np.clip(fill[m] + rng.uniform(-size, size, int(m.sum())), 0.0, 1.0)
    return dataclasses.replace(sc, fill=fill)


def dam_break_observables(args):
    """The rectangular dam break 256x128x64 (D3Q19, liquid column x < 64,
    y < 64 over the full depth, g = 1e-5): for each BC variant, the FP64 run
    (the parity mode) against FP32 and the mass-conserving formats, and
    against the FP64 run from fill levels perturbed by 1e-7 (the observable's
    conditioning floor).  Observables every 100 steps on the mid-depth plane
    z = 32: front w(t) = sum_i phi(i, 0, 32) and column height
    h(t) = sum_j phi(0, j, 32); errors max_t |x(t) - x_64(t)| / x_64(t).
    The configs' setup: TRT, nu = 1e-3, no-slip box.  With --paper-walls,
    the paper's (Sec. 4.2): free-slip walls at all borders, SRT with
    omega = 1.9995 and the Smagorinsky model with C_S = 0.1."""
    import torch
    from paper_2207_13962_gb300 import fslbm
    from paper_2207_13962_gb300 import scenarios as S
    torch.cuda.set_device(0)
    steps, every = args.obs_steps, 100
    over = {}
    if args.paper_walls:
        over = dict(periodic=(2, 2, 2), collision="SRT", omega=1.9995, smagorinsky_cs=0.1)
    out = {}
    for variant in ("NBRC", "NBKC", "OM", "OM3"):
        sc = S.dam_break(variant=variant)
        nx, ny, nz = sc.shape
        series = {}
        for prec, scn in (("FP64", sc), ("FP64_perturbed", _perturbed(sc)), ("FP32", sc), ("FP32MC", sc),
                          ("FP16SMC", sc)):
            c = fslbm.context_for(scn, precision=prec.split("_")[0], **over)
            M0 = c.observables()["total_mass"]
            w, h, status, t0 = [], [], 0, time.perf_counter()
            for _ in range(steps // every):
                c.step(every)
                if c.sync() != 0:  # unstable (EUNSTABLE): the series stops here
                    break
                f = c.read(pdf=False)["fill"].reshape(nz, ny, nx)[nz // 2]
                w.append(float(f[0].sum()))
                h.append(float(f[:, 0].sum()))
            obs = c.observables(check=False)
            status = obs["status"]
            c.close()
            series[prec] = (np.array(w), np.array(h), status, abs(obs["total_mass"] - M0) / M0,
                            time.perf_counter() - t0)
        ref = series["FP64"]
        res = {"FP64": {"status": ref[2], "steps_stable": every * len(ref[0]),
                        "front_final": ref[0][-1] if len(ref[0]) else None,
                        "height_final": ref[1][-1] if len(ref[1]) else None,
                        "mass_drift_rel": ref[3], "seconds": round(ref[4], 2)}}
        for prec in ("FP64_perturbed", "FP32", "FP32MC", "FP16SMC"):
            w, h, st, drift, sec = series[prec]
            n = min(len(w), len(ref[0]))  # compare where both are stable
            res[prec] = {"status": st, "steps_stable": every * len(w),
                         "front_rel_err": float(np.max(np.abs(w[:n] - ref[0][:n]) / ref[0][:n])) if n else None,
                         "height_rel_err": float(np.max(np.abs(h[:n] - ref[1][:n]) / ref[1][:n])) if n else None,
                         "compared_steps": every * n, "mass_drift_rel": drift, "seconds": round(sec, 2)}
        out[variant] = res
    setup = ("free-slip walls, SRT omega 1.9995, Smagorinsky C_S 0.1 (the paper's Sec. 4.2)" if args.paper_walls
             else "no-slip box, TRT nu 1e-3 (the configs')")
    line = {"metric": METRIC, "workload": f"dam break 256x128x64 observables, {steps} steps, {setup}",
            "results": out, "floor": "FP64_perturbed: the FP64 run from interface fill levels moved by a seeded "
                                     "+-1e-7",
            "data": "synthetic (seeded generator, no dataset)"}
    print(json.dumps(line), flush=True)
    return line


def taylor_rise(args):
    """Rise velocity of the Taylor bubble 160x160x1024 (D3Q19 TRT OM, bubble
    model): the bubble centroid z_c = sum (1 - phi) z / sum (1 - phi) over gas
    and interface cells, every 1000 steps, and the rise velocity dz_c/dt over
    the last quarter of the run; the FP64 run (the parity mode) against FP32
    and the mass-conserving formats, and against the FP64 run from fill
    levels perturbed by 1e-7 (the observable's conditioning floor)."""
    import torch
    from paper_2207_13962_gb300 import fslbm
    from paper_2207_13962_gb300 import scenarios as S
    torch.cuda.set_device(0)
    sc = S.taylor_bubble(variant="OM")
    nx, ny, nz = sc.shape
    zc_of = np.arange(nz, dtype=np.float64)[:, None, None] + 0.5
    steps, every = args.rise_steps, 1000
    out = {}
    for prec, scn in (("FP64", sc), ("FP64_perturbed", _perturbed(sc)), ("FP64_perturbed_2", _perturbed(sc, seed=2)),
                      ("FP32", sc), ("FP32MC", sc), ("FP16SMC", sc)):
        c = fslbm.context_for(scn, precision=prec.split("_")[0])
        M0 = c.observables()["total_mass"]
        t, z, t0 = [], [], time.perf_counter()
        for k in range(steps // every):
            c.step(every)
            r = c.read(pdf=False)
            fl = r["flags"].reshape(nz, ny, nx)
            gas = np.where(fl == S.GAS, 1.0, np.where(fl == S.IFACE, 1.0 - r["fill"].reshape(nz, ny, nx), 0.0))
            t.append((k + 1) * every)
            z.append(float((gas * zc_of).sum() / gas.sum()))
        obs = c.observables()
        c.close()
        t, z = np.array(t, float), np.array(z)
        q = max(2, len(t) // 4)
        vel = float(np.polyfit(t[-q:], z[-q:], 1)[0])
        out[prec] = {"rise_velocity": vel, "centroid_final": z[-1], "status": obs["status"],
                     "mass_drift_rel": abs(obs["total_mass"] - M0) / M0, "seconds": round(time.perf_counter() - t0, 1)}
    for prec in ("FP64_perturbed", "FP64_perturbed_2", "FP32", "FP32MC", "FP16SMC"):
        out[prec]["rise_velocity_rel_err_vs_fp64"] = abs(out[prec]["rise_velocity"] - out["FP64"]["rise_velocity"]) / \
            abs(out["FP64"]["rise_velocity"])
    line = {"metric": METRIC, "workload": f"Taylor bubble rise velocity, {steps} steps", "results": out,
            "floor": "FP64_perturbed(_2): the FP64 run from interface fill levels moved by a seeded +-1e-7 "
                     "(two seeds: whether a perturbation this small flips a conversion decision depends on where "
                     "it falls)",
            "data": "synthetic (seeded generator, no dataset)"}
    print(json.dumps(line), flush=True)
    return line


# --------------------------------------------------------- reference arm

def bench_reference(args, ws, rank):
    if rank != 0:
        return None
    from oracle.oracle import build_oracle
    build_oracle()
    sc, desc = make_workload(args.workload, args.variant)
    vals = []
    for _ in range(args.warmup):
        run_oracle_sample(sc, args.workload, steps_budget_s=3.0, max_steps=2)
    samp = None
    t_total = 0.0
    for _ in range(args.steps):
        r = run_oracle_sample(sc, args.workload, steps_budget_s=6.0, max_steps=10)
        vals.append(r["value"])
        samp = r["sample"]
        t_total += r["seconds"]
    value = statistics.median(vals)
    line = {
        "impl": "reference",
        "metric": METRIC, "value": round(value, 4), "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1000.0 * t_total / max(args.steps, 1), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded generator, no dataset)",
        "config": {"workload": desc, "sample": samp},
        "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
                         "sample": samp},
        "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return line


def sector_census(workload: str, variant: str = "OM") -> dict:
    """Host-side count of the 32-byte sectors the bulk sweep reads and writes
    on a workload's initial flag field (FP32 storage, D3Q19 or D3Q27): the
    figures that DRAM counters of k_bulk are compared with.  No GPU."""
    import numpy as np
    from paper_2207_13962_gb300 import scenarios as S
    sc, _ = make_workload(workload, variant)
    nx, ny, nz = sc.shape
    N = nx * ny * nz
    fl = np.asarray(sc.flags).reshape(-1)
    lin = np.flatnonzero(fl == S.LIQ)
    x, y, z = lin % nx, (lin // nx) % ny, lin // (nx * ny)
    dirs = [(a, b, c) for c in (-1, 0, 1) for b in (-1, 0, 1) for a in (-1, 0, 1)
            if sc.q == 27 or abs(a) + abs(b) + abs(c) <= 2]
    seg = lin // 32
    out = {"liquid_cells": int(lin.size), "segments": int(np.unique(seg).size)}
    out["lane_occupancy"] = lin.size / (32.0 * out["segments"])
    distinct = pairs = d64 = d128 = refl = 0
    obst = fl == S.OBST
    for (cx, cy, cz) in dirs:
        src = (x - cx) + nx * ((y - cy) + ny * (z - cz))
        distinct += np.unique(src // 8).size
        pairs += np.unique(seg.astype(np.int64) * (N // 8 + 2) + src // 8).size
        d64 += np.unique(src // 16).size
        d128 += np.unique(src // 32).size
        if (cx, cy, cz) != (0, 0, 0):
            X, Y, Z = x - cx, y - cy, z - cz
            ok = (X >= 0) & (X < nx) & (Y >= 0) & (Y < ny) & (Z >= 0) & (Z < nz)
            tgt = X[ok] + nx * (Y[ok] + ny * Z[ok])
            refl += np.unique(tgt[obst[tgt]] // 8).size
    nsec = (N + 7) // 8
    pad = lambda m: np.concatenate([m, np.zeros(nsec * 8 - N, bool)]).reshape(nsec, 8)
    has_l = pad(fl == S.LIQ).any(1)
    part = has_l & (pad(obst).any(1) | pad(fl == S.IFACE).any(1))
    out.update(algorithmic_read_MB=lin.size * len(dirs) * 4 / 1e6,
               distinct_read_sectors=int(distinct), warp_sector_requests=int(pairs),
               read_sectors_64B_chunks=int(d64 * 2), read_sectors_128B_lines=int(d128 * 4),
               partial_write_sectors=int(part.sum()) * len(dirs), reflected_write_sectors=int(refl))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="taylor_bubble", choices=["taylor_bubble", "taylor_bubble_256", "dam_break", "box256", "box512",
                                                       "batch_cylinders", "serve_drops", "dam_break_observables",
                                                       "taylor_rise"])
    ap.add_argument("--obs-steps", type=int, default=20000, help="dam_break_observables: steps")
    ap.add_argument("--rise-steps", type=int, default=100000, help="taylor_rise: steps")
    ap.add_argument("--paper-walls", action="store_true",
                    help="dam_break_observables: free-slip walls, SRT omega 1.9995, Smagorinsky C_S 0.1")
    ap.add_argument("--precision", default="FP32", choices=list(S_BYTES))
    ap.add_argument("--variant", default="OM", choices=["NBRC", "NBKC", "OM", "OM3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--sector-census", action="store_true",
                    help="print the bulk sweep's sector counts on the workload's initial state (CPU only)")
    ap.add_argument("--batch-n", type=int, default=64, help="batch_cylinders: domains")
    ap.add_argument("--batch-steps", type=int, default=200, help="batch_cylinders: timed steps")
    ap.add_argument("--batch-warmup", type=int, default=200, help="batch_cylinders: steps before the timed ones")
    ap.add_argument("--batch-precision", default="FP32MC,FP16SMC",
                    help="batched/served: storage formats run beside FP32 (comma-separated)")
    ap.add_argument("--rate", type=float, default=20.0, help="serve_drops: mean arrivals per second")
    ap.add_argument("--autotune", action="store_true", help="batch_cylinders: autotune the launch shape")
    ap.add_argument("--requests", type=int, default=24, help="serve_drops: requests of the trace")
    ap.add_argument("--serve-steps", type=int, default=1000, help="serve_drops: steps per request")
    ap.add_argument("--max-active", type=int, default=16, help="serve_drops: resident runs")
    ap.add_argument("--chunk-steps", type=int, default=100, help="serve_drops: steps per round")
    ap.add_argument("--serve-cs", type=float, default=0.0,
                    help="serve_drops: Smagorinsky constant of the drop impacts (0: no turbulence model)")
    ap.add_argument("--skip-served-fp32", action="store_true",
                    help="serve_drops: serve only the --batch-precision formats (the FIFO FP32 arm still runs)")
    args = ap.parse_args(argv)
    if args.sector_census:
        print(json.dumps(sector_census(args.workload, args.variant)))
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    ws, rank, local = dist_env()
    if args.workload == "batch_cylinders" and args.impl == "ours":
        bench_batch(args)
        return
    if args.workload == "serve_drops" and args.impl == "ours":
        bench_serve(args)
        return
    if args.workload == "dam_break_observables" and args.impl == "ours":
        dam_break_observables(args)
        return
    if args.workload == "taylor_rise" and args.impl == "ours":
        taylor_rise(args)
        return
    if args.impl == "reference":
        bench_reference(args, ws, rank)
        return
    bench_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()

"""Benchmark: FP64 residual + Jacobian assembly of the first-order Stokes system (wedge cells/s).

One step = one bp_assemble_jacobian call (FP64 lanes, residual requested, zero-initialisation
included) on the 1,003,520-wedge dome (100,352 base triangles x 10 layers), i.e. every row of
the assembly path: gather, basis, interpolation, viscosity, residual, Jacobian, scatter.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the CPU oracle (FP64 C++, its columns taken colour by colour on all host
cores) on a bounded sample of the same workload.  Under torchrun (N > 1) every rank assembles its own replica of the workload
(no collective on the data path: weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "residual+Jacobian wedge cells/s"
UNIT = "wedges/s"
# Nominal FP64 rate from unit counts and the maximum clock: 148 SMs x 2 FP64 FMA per clock per SM x
# 2 flop x 2.032 GHz (the rate behind NVIDIA's nominal 1.25 TFLOP/s).  The roofline's denominator is
# the rate measured on the device at run time (bp_measure_fma_peak); this one is reported beside it.
FP64_NOMINAL_TFLOPS = 148 * 2 * 2 * 2.032e9 / 1e12
L2_FLUSH_BYTES = 512 << 20
# The FP64 flops per wedge of the assembly kernel (2 DFMA + DADD + DMUL executed, ncu thread-level
# instruction counters) and its DRAM bytes per wedge come from one capture, recorded in this file
# with a hash of the kernel's code: both apply only while the hash matches.
KERNEL_RECORD = os.path.join(ROOT, "profiles", "assemble_jacobian_f64_traffic.json")


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi sampling (every 50 ms) of SM clock and throttle reasons; each sample is stamped on
    arrival so that summary() keeps only the samples taken inside the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.samples = []
        self.window = None

    def _read(self):
        for line in self.proc.stdout:
            if line.strip():
                self.samples.append((time.perf_counter(), line))

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.reader.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = self.window if self.window else (-float("inf"), float("inf"))
        for t, line in self.samples:
            if not t0 <= t <= t1:
                continue
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload_name(m: int, layers: int) -> str:
    """The assembly workload: dome on an m x m grid (2 m^2 triangles) extruded to `layers` layers."""
    ntri = 2 * m * m
    name = "dome-100k-tri-x10" if (m, layers) == (224, 10) else f"dome-{ntri // 1000}k-tri-x{layers}"
    return (f"{name}: dome on a {m}x{m} jittered Delaunay grid, {ntri} triangles x {layers} "
            f"layers = {ntri * layers} wedges, sinusoidal bed, correlated lognormal beta")


def bench_config(args, ws: int) -> dict:
    """The workload both arms name: the same dict on the GPU line and on the reference line."""
    return {"workload": workload_name(args.mesh_m, args.layers),
            "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU",
            "l2": f"GPU arm: inputs larger than L2 and L2 flushed between steps ({L2_FLUSH_BYTES >> 20} MB "
                  f"write outside the timed events)"}


def headline(line: dict) -> dict:
    """The nested sections' key figures in a few hundred bytes, printed as the line's last key so
    that a reader of the line's tail sees them: FP64-accurate assembly kinds, Newton solve times,
    the learned start over unseen fields, the ensemble and the MLP."""
    def get(d, *path):
        for k in path:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d

    def r(x, nd=4):
        return None if x is None else float(f"{x:.{nd}g}")

    sec, out = line.get("secondary") or {}, {}
    out["assembly_ms"] = {"f64": r(get(line, "roofline", "kernel_ms")),
                          "f64x2_ds": r(get(sec, "jacobian_paired_lanes_double_single_values", "ms")),
                          "f32_ds": r(get(sec, "jacobian_f32_lanes_double_single_values", "ms")),
                          "f32_lanes": r(get(sec, "jacobian_f32_lanes", "ms")),
                          "residual": r(get(sec, "residual_only", "ms"))}
    out["roofline_frac"] = r(get(line, "roofline", "frac"), 3)
    d = get(line, "newton", "dome-100k-tri-x10") or {}
    ms = {k: r(1e3 * v["s"]) for k, v in d.items() if isinstance(v, dict) and "s" in v}
    if ms:
        out["newton_1M_ms"] = ms
    ls = get(d, "learned_start_mixed") or {}
    lms = {k: r(1e3 * v["s"]) for k, v in ls.items() if isinstance(v, dict) and "s" in v and "picard" in k}
    if lms:
        out["learned_1M_ms"] = lms
    u = get(d, "learned_start_mixed", "unseen_beta_fields")
    if u:
        out["learned_picard_vs_sia"] = {"seeds": u["seeds"], "speedup": r(u["speedup_learned_picard_vs_sia"]),
                                        "ci99": [r(c) for c in u["ci99"]]}
    d4 = get(line, "newton", "dome-400k-tri-x10") or {}
    ms4 = {k: r(1e3 * v["s"]) for k, v in d4.items() if isinstance(v, dict) and "s" in v}
    if ms4:
        out["newton_4M_ms"] = ms4
    dm = get(line, "newton", "marine-100k-tri-x10") or {}
    msm = {k: r(1e3 * v["s"]) for k, v in dm.items() if isinstance(v, dict) and "s" in v}
    if msm:
        out["newton_marine_1M_ms"] = msm
    if line.get("ensemble"):
        out["ensemble_wedges_per_s"] = r(get(line, "ensemble", "value"))
    if line.get("mlp"):
        out["mlp_ms"] = {"inference": r(get(line, "mlp", "inference", "ms")),
                         "train_step": r(get(line, "mlp", "train_step", "ms"))}
    return out


def max_over_ranks(x: float, ws: int, device=None) -> float:
    """The largest per-rank value over all ranks (a job takes as long as its slowest rank)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws: int, units_per_rank_step: float, steps: int, seconds: float) -> float:
    """Whole-job throughput of weak-scaled replicas: every rank processes the same units per step."""
    return ws * units_per_rank_step * steps / seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sample_mesh():
    """The CPU oracle's sample of the workload: the same generators on a 100 x 100 grid (20,000
    triangles) x 10 layers = 200,000 wedges."""
    from paper_2204_04321_b300 import synth
    return synth.dome_mesh(100, 10, 201, 202, bed="sinusoidal", beta="field", name="dome-20k-tri-x10")


def time_oracle(om, U, nthreads, max_runs=5, seconds_budget=10.0):
    """Median time of the oracle's residual + 12-lane dual Jacobian into CSR: the plain element loop
    (nthreads = 0), or the same loop taken colour by colour on nthreads std::threads."""
    runs = []
    t_end = time.perf_counter() + seconds_budget
    while True:
        t0 = time.perf_counter()
        if nthreads == 0:
            om.jacobian(U)
        else:
            om.jacobian_colored(U, nthreads)
        runs.append(time.perf_counter() - t0)
        if time.perf_counter() > t_end or len(runs) >= max_runs:
            break
    return statistics.median(runs), len(runs)


def cpu_oracle_sample():
    """The CPU oracle timed on the host's cores (all of them, and one) on the sample mesh."""
    import oracle
    from paper_2204_04321_b300 import synth
    mesh = oracle_sample_mesh()
    om = oracle.OracleMesh(mesh)
    U = synth.random_velocity(mesh, 5, 50.0)
    om.pattern()
    cores = host_cores()
    t_all, n_all = time_oracle(om, U, cores, max_runs=7)
    t_one, n_one = time_oracle(om, U, 0)
    return {"value": mesh.nwedges / t_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"{mesh.name}: {mesh.nwedges} wedges, residual + 12-lane dual Jacobian into CSR, "
                      f"columns colour by colour on {cores} threads, median of {n_all} runs, g++ -O2",
            "single_thread": {"value": mesh.nwedges / t_one, "unit": UNIT, "cores": 1,
                              "sample": f"the same, plain element loop, 1 thread, median of {n_one} runs"}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2204_04321_b300 import synth
    import oracle
    mesh = oracle_sample_mesh()
    om = oracle.OracleMesh(mesh)
    U = synth.random_velocity(mesh, 5, 50.0)
    om.pattern()
    cores = host_cores()
    for _ in range(args.warmup):
        om.jacobian_colored(U, cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        om.jacobian_colored(U, cores)
    dt = time.perf_counter() - t0
    value = mesh.nwedges * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": bench_config(args, ws),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": f"each step: dome-20k-tri-x10 (200,000 wedges, the same generators), "
                                       f"CPU FP64 oracle, columns colour by colour on {cores} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_2204_04321_b300 import capi, synth

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    if args.ensemble_only:
        print(json.dumps({"ensemble": ensemble_section(capi, synth, dev), "mlp": mlp_section(capi, dev)}),
              flush=True)
        return 0
    if args.newton_only:
        mesh = synth.config_medium()
        dm = capi.DeviceMesh(mesh)
        print(json.dumps(newton_section(capi, synth, dm, mesh, dev, skip_large=True, reps=args.newton_reps)),
              flush=True)
        return 0

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    if (args.mesh_m, args.layers) == (224, 10):
        mesh = synth.config_medium()
    else:  # smaller case of the same generators (profiling captures)
        mesh = synth.dome_mesh(args.mesh_m, args.layers, 201, 202, bed="sinusoidal", beta="field",
                               name=f"dome-{2 * args.mesh_m ** 2 // 1000}k-tri-x{args.layers}")
    W = mesh.nwedges
    dm = capi.DeviceMesh(mesh)
    U_host = torch.from_numpy(synth.random_velocity(mesh, 5, 50.0) + 0.0).pin_memory()
    U = U_host.to(dev)
    R = torch.empty(dm.ndof, dtype=torch.float64, device=dev)
    J = torch.empty(dm.nnz, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        capi.bp_assemble_jacobian(dm.handle, U, R, J, capi.BP_F64, capi.BP_SCATTER_ATOMIC,
                                  capi.BP_JAC_FACTORED, stream)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local) as clk:  # started before the warm-up, which keeps the GPU loaded meanwhile
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        t_wall0 = time.perf_counter()
        for e0, e1 in ev:
            flush.fill_(1)              # L2 flush outside the timed events
            e0.record(stream)
            step()
            e1.record(stream)
        torch.cuda.synchronize()
        t_wall1 = time.perf_counter()
        t_wall = t_wall1 - t_wall0
        clk.window = (t_wall0, t_wall1)
    barrier()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    total_ms = max_over_ranks(sum(step_ms), ws, dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(ws, W, args.steps, total_ms * 1e-3)

    # zero-initialisation share of a step (memset of J + copy of the memoised load into R), timed alone
    z0, z1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    zs = []
    for _ in range(5):
        flush.fill_(1)
        z0.record(stream)
        J.zero_()
        R.zero_()
        z1.record(stream)
        torch.cuda.synchronize()
        zs.append(z0.elapsed_time(z1))
    zero_ms = statistics.median(zs)
    kernel_ms = max(ms_per_step - zero_ms, 1e-6)

    # secondary: residual only, FP32-lane Jacobian (same workload)
    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    res_ms = timed(lambda: capi.bp_assemble_residual(dm.handle, U, R, stream))
    J32 = torch.empty(dm.nnz, dtype=torch.float32, device=dev)
    jac32_ms = timed(lambda: capi.bp_assemble_jacobian(dm.handle, U, R, J32, capi.BP_F32,
                                                       capi.BP_SCATTER_ATOMIC, capi.BP_JAC_FACTORED, stream))
    jac32c_ms = timed(lambda: capi.bp_assemble_jacobian(dm.handle, U, R, J32, capi.BP_F32,
                                                        capi.BP_SCATTER_COLOR, capi.BP_JAC_FACTORED, stream))
    all32_ms = timed(lambda: capi.bp_assemble_jacobian(dm.handle, U, R, J32, capi.BP_F32_ALL,
                                                       capi.BP_SCATTER_ATOMIC, capi.BP_JAC_FACTORED, stream))
    ds32_ms = timed(lambda: capi.bp_assemble_jacobian(dm.handle, U, R, J32, capi.BP_F32_DS,
                                                      capi.BP_SCATTER_ATOMIC, capi.BP_JAC_FACTORED, stream))
    all32c_ms = timed(lambda: capi.bp_assemble_jacobian(dm.handle, U, R, J32, capi.BP_F32_ALL,
                                                        capi.BP_SCATTER_COLOR, capi.BP_JAC_FACTORED, stream))
    dual_ms = timed(lambda: capi.bp_assemble_jacobian(dm.handle, U, R, J, capi.BP_F64,
                                                      capi.BP_SCATTER_ATOMIC, capi.BP_JAC_DUAL, stream), reps=5)
    pair_ms = timed(lambda: capi.bp_assemble_jacobian(dm.handle, U, R, J, capi.BP_F64X2,
                                                      capi.BP_SCATTER_ATOMIC, capi.BP_JAC_FACTORED, stream))
    pair_ds_ms = timed(lambda: capi.bp_assemble_jacobian(dm.handle, U, R, J, capi.BP_F64X2_DS,
                                                         capi.BP_SCATTER_ATOMIC, capi.BP_JAC_FACTORED, stream))
    # temperature-dependent rate factor (nodal Arrhenius field interpolated at the quadrature points)
    capi.bp_mesh_set_rate_factor(dm.handle, synth.arrhenius_rate_factor(mesh))
    arr_ms = timed(lambda: capi.bp_assemble_jacobian(dm.handle, U, R, J, capi.BP_F64,
                                                     capi.BP_SCATTER_ATOMIC, capi.BP_JAC_FACTORED, stream))
    capi.bp_mesh_set_rate_factor(dm.handle, None)
    del J32

    # end to end through the C ABI with host buffers: U from pinned host memory, R and J back to host.
    # Two slots (stream, device buffers, pinned host buffers) alternate so that the read-back of one
    # step overlaps the next step's upload and assembly; each step's own copies stay in its stream.
    slots = []
    for k in range(2):
        sk = torch.cuda.Stream(device=dev)
        slots.append({"stream": sk, "U": U if k == 0 else torch.empty_like(U), "R": R if k == 0 else torch.empty_like(R),
                      "J": J if k == 0 else torch.empty_like(J),
                      "R_host": torch.empty(dm.ndof, dtype=torch.float64).pin_memory(),
                      "J_host": torch.empty(dm.nnz, dtype=torch.float64).pin_memory()})
    torch.cuda.synchronize()

    def e2e_step(k):
        sl = slots[k % 2]
        with torch.cuda.stream(sl["stream"]):
            sl["U"].copy_(U_host, non_blocking=True)
            capi.bp_assemble_jacobian(dm.handle, sl["U"], sl["R"], sl["J"], capi.BP_F64, capi.BP_SCATTER_ATOMIC,
                                      capi.BP_JAC_FACTORED, sl["stream"])
            sl["R_host"].copy_(sl["R"], non_blocking=True)
            sl["J_host"].copy_(sl["J"], non_blocking=True)

    for k in range(2):
        e2e_step(k)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        e2e_step(k)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws, dev)
    del slots
    e2e_value = job_throughput(ws, W, args.steps, e2e_s)

    newton = newton_section(capi, synth, dm, mesh, dev, skip_large=args.no_large) if not args.no_newton else None
    mlp = mlp_section(capi, dev) if not args.no_mlp else None
    with open(KERNEL_RECORD) as f:
        rec = json.load(f)
    rec_current = rec.get("kernel_source_hash") == kernel_hash()
    flops_per_wedge = rec["fp64_flops_per_wedge_executed"]
    achieved = flops_per_wedge * W / (kernel_ms * 1e-3) / 1e12
    traffic = rec["bytes_per_wedge"] * W if rec_current else None
    peaks = read_peaks()
    fp64_peak = capi.bp_measure_fma_peak(capi.BP_F64, stream)
    fp32_peak = capi.bp_measure_fma_peak(capi.BP_F32, stream)

    if not args.no_ensemble:
        ensemble = ensemble_section(capi, synth, dev)
    else:
        ensemble = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, ws),
            "problem": {"wedges": W, "ndof": dm.ndof, "nnz": dm.nnz, "lanes": "f64, sum-factorised",
                        "scatter": "atomic"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp64_peak, "traffic": traffic,
                         "kernel": "k_assemble<factored, double, atomic>",
                         "kernel_ms": kernel_ms, "flops_per_wedge": flops_per_wedge,
                         "flops_record_matches_kernel": rec_current,
                         "peak_note": "FP64 FMA rate measured in this run (bp_measure_fma_peak: 8 independent DFMA "
                                      "chains per thread, 64 warps per SM); MEASURED_PEAKS.json has no FP64 entry",
                         "nominal_peak": FP64_NOMINAL_TFLOPS, "frac_of_nominal": achieved / FP64_NOMINAL_TFLOPS,
                         "fp32_fma_peak_measured": fp32_peak,
                         "hbm_peak_measured_gbs": peaks.get("hbm_gbs"),
                         "hbm_achieved_gbs": (traffic / (kernel_ms * 1e-3) / 1e9) if traffic else None},
            "secondary": {
                "residual_only": {"value": W / (res_ms * 1e-3), "unit": UNIT, "ms": res_ms},
                "jacobian_f32_lanes": {"value": W / (jac32_ms * 1e-3), "unit": UNIT, "ms": jac32_ms},
                "jacobian_f32_lanes_colored": {"value": W / (jac32c_ms * 1e-3), "unit": UNIT, "ms": jac32c_ms},
                "jacobian_f32_all": {"value": W / (all32_ms * 1e-3), "unit": UNIT, "ms": all32_ms,
                                     "note": "FP32 value path and lanes (residual with FP32 rounding)"},
                "jacobian_f32_all_colored": {"value": W / (all32c_ms * 1e-3), "unit": UNIT, "ms": all32c_ms},
                "jacobian_f64_dual12": {"value": W / (dual_ms * 1e-3), "unit": UNIT, "ms": dual_ms},
                "jacobian_paired_f32_lanes": {"value": W / (pair_ms * 1e-3), "unit": UNIT, "ms": pair_ms,
                                              "note": "FP64-accurate (1e-12 parity) lanes of hi+lo FP32 pairs"},
                "jacobian_paired_lanes_double_single_values": {
                    "value": W / (pair_ds_ms * 1e-3), "unit": UNIT, "ms": pair_ds_ms,
                    "note": "BP_F64X2_DS: paired lanes and a double-single value path; R and J FP64-accurate "
                            "(1e-12 parity) with the quadrature-point arithmetic on the FP32 pipe"},
                "jacobian_f32_lanes_double_single_values": {
                    "value": W / (ds32_ms * 1e-3), "unit": UNIT, "ms": ds32_ms,
                    "note": "BP_F32_DS: FP32 lanes, double-single value path (R FP64-accurate)"},
                "jacobian_f64_arrhenius_field": {"value": W / (arr_ms * 1e-3), "unit": UNIT, "ms": arr_ms,
                                                 "note": "nodal rate-factor field (Arrhenius) instead of a constant A"},
                "zero_init_ms": zero_ms, "wall_s_timed_region": t_wall},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * dm.ndof,
                    "d2h_bytes_per_step": 8 * dm.ndof + 8 * dm.nnz,
                    "note": "pinned host U in, R and J (FP64) out every step; two streams alternate so a "
                            "step's read-back overlaps the next step's upload and assembly"},
            "newton": newton,
            "ensemble": ensemble,
            "mlp": mlp,
            "gpu_launches": args.steps,
            "clocks": clk.summary(),
        }
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_oracle_sample()
        line["headline"] = headline(line)
        print(json.dumps(line), flush=True)
    dm.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def learned_start(capi, dm, dev, reps=3, seeds=40):
    """Mixed-precision solve from the committed learned warm start: the network's guess with the
    fallback to the shallow-ice guess judged by the FP64 residual norm, by the FP64 energy, and the
    energy-judged guess followed by Picard steps (learned.PICARD_RTOL), on this mesh's beta; then
    the last against the shallow-ice start over `seeds` unseen beta fields (paired 99 % interval of
    the time ratio).  guess_rel_err = |U0 - U*| / |U*| of the initial guess."""
    import numpy as np
    from scipy import stats
    from paper_2204_04321_b300 import learned, synth
    if not os.path.exists(learned.DEFAULT_WEIGHTS):
        return None
    net = capi.Mlp()
    net.load(learned.DEFAULT_WEIGHTS)
    out = {}
    for name in ("sia", "learned", "learned_energy", "learned_picard"):
        times, rep = [], None
        for _ in range(reps):
            _, rep = learned.solve(dm, capi.BP_F32, name, mlp=net)
            times.append(rep["wall_s"])
        out[name] = {"s": statistics.median(times), "newton_iters": rep["newton_iters"],
                     "converged": rep["converged"], "guess_rel_err": rep["guess_rel_err"],
                     "initial_rel_residual": rep["history"][0]}
        if name != "sia":
            out[name]["network_guess_kept"] = rep["learned_used"]
    # the same two starts with FP32 value-path steps until 1e-3, and with the double-single FP32
    # lanes and FP32 value-path steps until 1e-4 (the fastest mixed configuration)
    for tag, prec, v32 in (("_value32_until_1e-3", capi.BP_F32, 1e-3),
                           ("_f32_ds_value32_until_1e-4", capi.BP_F32_DS, 1e-4)):
        for name in ("sia", "learned_picard"):
            times, rep = [], None
            for _ in range(reps):
                _, rep = learned.solve(dm, prec, name, mlp=net, value32_rtol=v32)
                times.append(rep["wall_s"])
            out[name + tag] = {"s": statistics.median(times), "newton_iters": rep["newton_iters"],
                               "converged": rep["converged"]}
    out["judges"] = {"learned": "FP64 residual norm", "learned_energy": "FP64 discrete energy",
                     "learned_picard": f"FP64 energy, then Picard steps until ||F|| <= {learned.PICARD_RTOL} ||F(0)||"}
    mesh = dm.mesh
    ratios, its = [], {"sia": [], "learned_picard": []}
    for seed in range(learned.TEST_SEED0, learned.TEST_SEED0 + seeds):
        capi.bp_mesh_set_beta(dm.handle, synth.lognormal_beta_field_torch(mesh.xy, seed, dev))
        t = {}
        for name in ("sia", "learned_picard"):
            _, rep = learned.solve(dm, capi.BP_F32, name, mlp=net)
            t[name] = rep["wall_s"]
            its[name].append(rep["newton_iters"])
        ratios.append(math.log(t["sia"] / t["learned_picard"]))
    capi.bp_mesh_set_beta(dm.handle, mesh.beta)
    lr = np.array(ratios)
    half = stats.t.ppf(0.995, len(lr) - 1) * lr.std(ddof=1) / math.sqrt(len(lr))
    out["unseen_beta_fields"] = {"seeds": seeds, "speedup_learned_picard_vs_sia": math.exp(lr.mean()),
                                 "ci99": [math.exp(lr.mean() - half), math.exp(lr.mean() + half)],
                                 "nonlinear_steps_mean": {k: float(np.mean(v)) for k, v in its.items()}}
    net.close()
    return out


def ensemble_section(capi, synth, dev, reps=5):
    """64 uneven members (5k-50k triangles, 5-20 layers, H0 1-3 km, own beta) assembled in one
    persistent launch replayed from a CUDA graph, with the autotuned cells-per-block and scatter.
    Accuracy: every member's R and J against the same member assembled alone (bp_assemble_jacobian,
    itself at oracle parity); the per-member oracle comparison is in the GPU tests."""
    import torch
    members = synth.ensemble_members()
    W = sum(m.nwedges for m in members)
    U = [torch.as_tensor(synth.random_velocity(m, 500 + i), device=dev) for i, m in enumerate(members)]
    ens = capi.Ensemble(members, U, precision=capi.BP_F64)
    times, chosen = ens.tune(reps=3)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        ens.assemble()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ens.assemble()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ms = statistics.median(ts)
    worst_r = worst_j = 0.0
    for i, dm in enumerate(ens.dms):
        J1, R1 = dm.jacobian(U[i])
        worst_r = max(worst_r, float((ens.R[i] - R1).abs().max() / R1.abs().max()))
        worst_j = max(worst_j, float((ens.J[i] - J1).abs().max() / J1.abs().max()))
        del J1, R1
    out = {"metric": "residual+Jacobian wedge cells/s (ensemble, one persistent launch, CUDA graph)",
           "value": W / (ms * 1e-3), "unit": "wedges/s", "ms": ms, "members": len(members), "wedges": W,
           "nnz": int(sum(d.nnz for d in ens.dms)), "dtype": "f64",
           "chosen": {"cells_per_block": chosen[0],
                      "scatter": "color" if chosen[1] == capi.BP_SCATTER_COLOR else "atomic"},
           "tuner_ms": times,
           "member_vs_single_launch_rel_inf": {"R": worst_r, "J": worst_j}}
    ens.close()
    del U
    torch.cuda.empty_cache()
    return out


def mlp_section(capi, dev, rows=50625, batch=8192, reps=20):
    """BF16 tcgen05 MLP (16-128-128-128-32): inference over the 1M-wedge dome's 50,625 columns and
    one Adam training step on a batch of 8,192 rows.  Flops per row: forward 2 x 38,912 MACs;
    training step (forward + backward for activations and weights) 3x that."""
    import torch
    net = capi.Mlp(seed=1)
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    X = torch.randn(rows, 16, device=dev, generator=g).to(torch.bfloat16)
    T = torch.randn(batch, 32, device=dev, generator=g)
    Xb = X[:batch].contiguous()
    Y = torch.empty(rows, 32, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    fwd_ms = timed(lambda: net.forward(X, Y))
    trn_ms = timed(lambda: net.train_step(Xb, T, 1e-4))
    flop_fwd = 2 * (16 * 128 + 128 * 128 + 128 * 128 + 128 * 32)
    net.close()
    return {"inference": {"rows": rows, "ms": fwd_ms, "tflops": flop_fwd * rows / (fwd_ms * 1e-3) / 1e12},
            "train_step": {"rows": batch, "ms": trn_ms, "rows_per_s": batch / (trn_ms * 1e-3),
                           "tflops": 3 * flop_fwd * batch / (trn_ms * 1e-3) / 1e12},
            "peak_note": "bf16 tensor peak (measured cuBLAS, MEASURED_PEAKS.json): "
                         + str(read_peaks().get("bf16_tflops")) + " TFLOP/s; these GEMMs (K, N <= 128) "
                         "are far too small to approach it"}


SOLVE_KW = {}  # options added to every timed Newton solve (--cg-host-loop)


def newton_section(capi, synth, dm, mesh, dev, skip_large=False, reps=3):
    """Time to ||F(U)|| <= 1e-8 ||F(0)|| from the shallow-ice guess: plain FP64 path and the
    mixed-precision path (FP32 Jacobian lanes and Krylov, FP64 residual/viscosity/update)."""
    import torch

    def solve(dmx, prec, reps=reps, **kw):
        times, rep, U = [], None, None
        for _ in range(reps):
            U = torch.empty(dmx.ndof, dtype=torch.float64, device=dev)
            capi.bp_initial_guess(dmx.handle, capi.BP_GUESS_SIA, U)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, rep = capi.bp_newton_solve(dmx.handle, U, precision=prec, max_krylov=4000, **SOLVE_KW, **kw)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            if rc != capi.BP_OK:
                break
        return {"s": statistics.median(times), "converged": rep["converged"], "newton_iters": rep["newton_iters"],
                "krylov_iters": rep["krylov_iters"], "final_rel_residual": rep["history"][-1],
                "t_assemble": rep["t_assemble"], "t_precond": rep["t_precond"], "t_krylov": rep["t_krylov"],
                "t_linesearch": rep["t_linesearch"], "value32_steps": rep["value32_steps"]}, U

    out = {"metric": "time to 1e-8 rel. FP64 residual Newton solve", "unit": "s", "start": "shallow-ice guess"}
    f64, U64 = solve(dm, capi.BP_F64)
    f32, U32 = solve(dm, capi.BP_F32)
    out[mesh.name] = {"f64": f64, "mixed_f32": f32, "speedup_mixed": f64["s"] / f32["s"],
                      "mixed_vs_f64_solution_rel_inf": float((U32 - U64).abs().max() / U64.abs().max())}
    # the same two paths with the double-single value path (residual FP64-accurate on the FP32 pipe):
    # FP64-accurate Jacobian from paired lanes with FP64 Krylov, and FP32 lanes with FP32 Krylov
    for name, prec, kw in (("f64_accurate_double_single", capi.BP_F64X2_DS, {}),
                           ("mixed_f32_double_single", capi.BP_F32_DS, {}),
                           ("mixed_f32_double_single_value32_until_1e-4", capi.BP_F32_DS, {"value32_rtol": 1e-4})):
        v, Uv = solve(dm, prec, **kw)
        v["vs_f64_solution_rel_inf"] = float((Uv - U64).abs().max() / U64.abs().max())
        out[mesh.name][name] = v
    # early steps with the FP32 value path (inexact residual) until ||F|| <= tau ||F(0)||
    for tau in (1e-2, 1e-3, 1e-4, 1e-5):
        v, Uv = solve(dm, capi.BP_F32, value32_rtol=tau)
        v["vs_f64_solution_rel_inf"] = float((Uv - U64).abs().max() / U64.abs().max())
        out[mesh.name][f"mixed_f32_value32_until_{tau:g}"] = v
    # the MDSC two-level preconditioner (semicoarsening + Chebyshev plane iteration) instead of the
    # vertical-line solve
    for name, prec, pk in (("f64_mdsc", capi.BP_F64, capi.BP_PREC_MDSC),
                           ("mixed_f32_mdsc", capi.BP_F32, capi.BP_PREC_MDSC),
                           ("mixed_f32_mdsc_amg", capi.BP_F32, capi.BP_PREC_MDSC_AMG)):
        v, Uv = solve(dm, prec, preconditioner=pk)
        v["vs_f64_solution_rel_inf"] = float((Uv - U64).abs().max() / U64.abs().max())
        out[mesh.name][name] = v
    # GMRES(50) with the column preconditioner (the paper's Krylov method), the cross-check of CG
    v, Uv = solve(dm, capi.BP_F32, krylov=capi.BP_KRYLOV_GMRES)
    v["vs_f64_solution_rel_inf"] = float((Uv - U64).abs().max() / U64.abs().max())
    out[mesh.name]["mixed_f32_gmres50"] = v
    out[mesh.name]["learned_start_mixed"] = learned_start(capi, dm, dev, reps)
    # the ocean margin condition (lateral faces of a grounded calving front, partly below sea level)
    marine = synth.config_marine()
    dmm = capi.DeviceMesh(marine)
    m64, W64 = solve(dmm, capi.BP_F64)
    m32, W32 = solve(dmm, capi.BP_F32)
    mp, _ = solve(dmm, capi.BP_F32, picard_rtol=0.01)
    mpv, _ = solve(dmm, capi.BP_F32, picard_rtol=0.01, value32_rtol=1e-3)
    out[marine.name] = {"wedges": marine.nwedges, "margin": "ocean (cryostatic minus sea-water pressure)",
                        "f64": m64, "mixed_f32": m32, "speedup_mixed": m64["s"] / m32["s"],
                        "mixed_f32_picard_until_1e-2": mp,
                        "mixed_f32_picard_until_1e-2_value32_until_1e-3": mpv,
                        "mixed_vs_f64_solution_rel_inf": float((W32 - W64).abs().max() / W64.abs().max()),
                        "max_speed_m_per_yr": float(torch.hypot(W64[0::2], W64[1::2]).max())}
    del W64, W32
    dmm.close()
    if not skip_large:
        big = synth.config_large()
        dmb = capi.DeviceMesh(big)
        b64, V64 = solve(dmb, capi.BP_F64, reps=1)
        b32, V32 = solve(dmb, capi.BP_F32, reps=1)
        bv, _ = solve(dmb, capi.BP_F32, reps=1, value32_rtol=1e-3)
        bm, _ = solve(dmb, capi.BP_F32, reps=1, preconditioner=capi.BP_PREC_MDSC)
        solve(dmb, capi.BP_F32, reps=1, preconditioner=capi.BP_PREC_MDSC_AMG)  # first: builds the hierarchy
        ba, _ = solve(dmb, capi.BP_F32, reps=1, preconditioner=capi.BP_PREC_MDSC_AMG)
        out[big.name] = {"wedges": big.nwedges, "f64": b64, "mixed_f32": b32, "speedup_mixed": b64["s"] / b32["s"],
                         "mixed_f32_value32_until_1e-3": bv, "mixed_f32_mdsc": bm, "mixed_f32_mdsc_amg": ba,
                         "mixed_vs_f64_solution_rel_inf": float((V32 - V64).abs().max() / V64.abs().max())}
        del V64, V32
        dmb.close()
    return out


def mdsc_scaling(ms):
    """Mixed-precision Newton solves (shallow-ice start, 1e-8) of growing domes (m x m grid, 10 layers)
    with the column preconditioner, the MDSC cycle (Chebyshev plane solve) and the MDSC cycle with the
    SA-AMG plane solve: time (best of 2), Newton steps, CG iterations; one JSON line per mesh."""
    import torch
    from paper_2204_04321_b300 import capi, synth
    for m in ms:
        mesh = synth.dome_mesh(m, 10, 201, 202, bed="sinusoidal", beta="field")
        dm = capi.DeviceMesh(mesh)
        row = {"m": m, "wedges": mesh.nwedges}
        for name, pk in (("column", capi.BP_PREC_COLUMN), ("mdsc", capi.BP_PREC_MDSC),
                         ("mdsc_amg", capi.BP_PREC_MDSC_AMG)):
            ts, rep = [], None
            for _ in range(2):
                U = torch.empty(dm.ndof, dtype=torch.float64, device="cuda")
                capi.bp_initial_guess(dm.handle, capi.BP_GUESS_SIA, U)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, rep = capi.bp_newton_solve(dm.handle, U, precision=capi.BP_F32, max_krylov=8000,
                                              preconditioner=pk)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
                del U
            row[name] = {"s": min(ts), "newton": rep["newton_iters"], "cg": rep["krylov_iters"],
                         "converged": rep["converged"], "t_krylov": rep["t_krylov"], "t_precond": rep["t_precond"]}
        row["amg_levels"] = capi.bp_mdsc_amg_levels(dm.handle)
        dm.close()
        torch.cuda.empty_cache()
        print(json.dumps(row), flush=True)


def kernel_hash():
    """Hash of the assembly kernel's source code: the per-column body and the shared device helpers
    it calls (pattern helpers, conversions, inverse cube root: the tail of the internal header),
    with comments and blank lines removed (a comment edit does not change the kernel)."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2204_04321_b300", "csrc")
    with open(os.path.join(csrc, "bp_column.cuh")) as f:
        src = f.read()
    src = src[src.index("constexpr int MODE_RES"):]
    with open(os.path.join(csrc, "bp_internal.cuh")) as f:
        helpers = f.read()
    src += helpers[helpers.index("// The kernels read velocity pairs"):]
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-newton", action="store_true", help="skip the Newton-solve measurements")
    ap.add_argument("--no-large", action="store_true", help="skip the 4M-wedge mixed-precision solve")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 64-member ensemble measurement")
    ap.add_argument("--no-mlp", action="store_true", help="skip the MLP kernel timings")
    ap.add_argument("--ensemble-only", action="store_true", help="only the ensemble and MLP sections")
    ap.add_argument("--newton-only", action="store_true",
                    help="only the Newton-solve section (profiling the solver); prints its JSON")
    ap.add_argument("--newton-reps", type=int, default=3, help="timed repetitions of each Newton solve")
    ap.add_argument("--cg-host-loop", action="store_true",
                    help="iterate CG from the host (device_loop 0) so that a kernel profiler lists every "
                         "CG launch (the device-driven loop launches its kernels from the device)")
    ap.add_argument("--mdsc-scaling", type=int, nargs="+", metavar="M",
                    help="only the preconditioner comparison on m x m x 10 domes (one JSON line each)")
    ap.add_argument("--mesh-m", type=int, default=224, help="base grid size (224: the 1M-wedge workload)")
    ap.add_argument("--layers", type=int, default=10)
    args = ap.parse_args()
    if args.cg_host_loop:
        SOLVE_KW["device_loop"] = 0
    if args.impl == "reference":
        return run_reference(args)
    if args.mdsc_scaling:
        return mdsc_scaling(args.mdsc_scaling) or 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

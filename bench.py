"""Benchmark: HIF factorization + PCG solve on one GB300 (or N independent replicas).

A step = one pass of the whole hot path on one synthetic operator: the
factorization F ~= A (every level: cell elimination, face and edge
skeletonization, merge; then the root) and the PCG solve of A u = f with F^{-1}
as preconditioner to ||r|| <= 1e-10 ||f||.  Workload (default): 128^3 grid
(N = 2,097,152), a = 10^U(-1,1) iid per grid point, b = 0.1, eps = 1e-6, FP32
factor, FP64 residual, one N(0,1) right-hand side.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints ONE JSON line (rank 0).  value = MDOF/s over all ranks = N * nrhs * K *
ranks / (max over ranks of the timed seconds).  --impl reference times the CPU
oracle (test infrastructure, FP64) on a bounded sample of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HIF factor s + PCG solve MDOF/s at 128^3, eps=1e-6, 1e-10 resid; p50/p99 latency"
UNIT = "MDOF/s"

WORKLOADS = {
    "contrast128": dict(n=128, m=4, lo=-1.0, hi=1.0, b=0.1, eps=1e-6, nrhs=1),
    "contrast64": dict(n=64, m=4, lo=-1.0, hi=1.0, b=0.0, eps=1e-6, nrhs=8),
    "laplace16": dict(n=16, m=4, lo=0.0, hi=0.0, b=0.0, eps=1e-6, nrhs=1),
    "contrast256": dict(n=256, m=4, lo=-3.0, hi=3.0, b=0.0, eps=1e-4, nrhs=1),
    # the paper's Example 2 (smoothed thresholded noise) and Example 3
    # (checkerboard of 7-point blocks) fields, {0.1, 1000}
    "example2_64": dict(n=64, m=4, lo=0.0, hi=0.0, b=0.1, eps=1e-5, nrhs=1, field=("blur", 1.0)),
    "example3_64": dict(n=64, m=4, lo=0.0, hi=0.0, b=0.1, eps=1e-4, nrhs=1, field=("checker", 7)),
}


def make_field(w: dict, n: int, seed: int):
    from paper_1607_00346_gb300 import inputs
    if "field" in w:
        return inputs.make_coeff(n, w["field"], seed)
    if w["hi"] > w["lo"]:
        return inputs.coeff_log_uniform(n, w["lo"], w["hi"], seed)
    return inputs.coeff_constant(n)


def field_desc(w: dict) -> str:
    if "field" in w:
        return {"blur": "Example 2 field (U(0,1) smoothed by a unit Gaussian, 0.1 / 1000 at 0.5)",
                "checker": "Example 3 checkerboard of 7-point blocks (1000 / 0.1)"}[w["field"][0]]
    if w["hi"] > w["lo"]:
        return f"a=10^U({w['lo']},{w['hi']}) iid per point"
    return "a=1"

# Roofline class of each profiled kernel label.  "tensor": tcgen05 products
# (algorithmic 2mnk flops over the measured TF32 tensor-core rate; the 3xTF32
# split issues three TF32 products per algorithmic one, so such a kernel
# tops out at a third of that rate).  "alu": dense algebra on the FMA units,
# including the pivoted QR of the ID and the row-reduction panels, which are
# latency- and FMA-bound (algorithmic Householder flops over the measured
# FMA rate of the factor's precision).  "hbm": streams whose bytes bound them
# (the apply's mat-vecs, gathers, the stencil, vector updates, the
# row-reduction trailing update).
KERNEL_BOUND = {
    "gemm_tc": "tensor", "chol_block_update_tc": "tensor", "trtri_merge_tc": "tensor",
    "chol_panel": "alu", "chol_trailing_update": "alu", "gemm_batched": "alu",
    "trtri_merge": "alu", "trtri_diag": "alu", "id_cpqr": "alu", "id_cpqr_smem": "alu",
    "id_cpqr_dsm": "alu",
    "id_rowreduce_panel": "alu", "id_rowreduce_w1": "alu", "skel_z_products": "alu",
    "id_rowreduce_block_tc": "tensor", "id_rowreduce_block": "alu", "id_rowreduce_blockt": "alu",
    "id_rowreduce_gram_tc": "tensor", "id_rowreduce_gram": "alu", "id_rowreduce_vta_tc": "tensor",
    "id_rowreduce_vta": "alu", "id_rowreduce_tw_tc": "tensor", "id_rowreduce_tw": "alu",
    "id_solve_t": "alu",
    "chol_block_update": "alu",
    "apply_gemv_n": "hbm", "apply_gemv_t": "hbm", "apply_sweeps_graph": "hbm",
    "apply_gather": "hbm", "apply_scatter": "hbm", "apply_accumulate": "hbm",
    "convert": "hbm", "skel_gather": "hbm", "merge_children": "hbm", "spmv": "hbm",
    "residual": "hbm", "dots": "hbm", "axpy": "hbm", "id_rowreduce_update": "hbm",
    "stencil_coefficients": "hbm",
}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a
# kernel label in the bench workload, from the ncu captures summarised in
# profiles/ (absent where no capture of the current kernel exists):
# gemm_tc: the 12 Schur-product launches of one 128^3 factorization move
# 53.8 GB (profiles/gemm_tc_traffic_contrast128.md); id_cpqr: its 4 k_cpqr
# launches move 78.7 GB (profiles/id_cpqr_traffic_contrast128.md).
TRAFFIC_PER_LAUNCH = {"gemm_tc": 53.76e9 / 12, "id_cpqr": 78.73e9 / 4}


def _hbm_peak():
    """(hbm GB/s, source) from the measured peaks file."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
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
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def job_rate(units_per_rank: float, seconds: float, dist=None, device: str = "cpu"):
    """Whole-job rate of N replicas: the slowest rank's seconds (max over
    ranks) and units of all ranks / that time.  Returns (seconds, rate)."""
    ws = 1
    if dist is not None:
        import torch
        ws = dist.get_world_size()
        t = torch.tensor([seconds], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds = float(t.item())
    return seconds, units_per_rank * ws / seconds


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_sample(w: dict, n_sample: int, seed: int):
    """Time the CPU oracle (factor + PCG) on an n_sample^3 grid of the same law."""
    import numpy as np

    from oracle import hif as ohif
    from oracle import krylov, stencil
    from paper_1607_00346_gb300 import inputs

    a = make_field(w, n_sample, seed)
    f = inputs.normal_rhs(n_sample, 1, seed + 1)[0]
    t0 = time.perf_counter()
    A = stencil.assemble(a, w["b"], n_sample)
    fac = ohif.hif_factor(A, n_sample, w["m"], w["eps"], check=False)
    u, its, hist = krylov.pcg(A, fac, f, tol=1e-10)
    dt = time.perf_counter() - t0
    return dt, its, hist[-1], float(np.linalg.norm(f - A @ u) / np.linalg.norm(f))


def run_reference(args, w):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    n_s = args.cpu_sample_n
    times = []
    for i in range(args.warmup + args.steps):
        dt, its, rel, _ = cpu_oracle_sample(w, n_s, 20260101 + i)
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = n_s ** 3 * len(times) / total / 1e6
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} law on a {n_s}^3 sample grid "
                               f"(N={n_s ** 3}): CPU oracle factor + PCG to 1e-10"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n_s}^3 grid of the same coefficient law, factor + PCG"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def serving_record(args):
    """Serving workload: Poisson request stream, resident operators, batched solves."""
    import torch

    from paper_1607_00346_gb300 import serving

    sizes = [32, 48, 64, 96, 128]
    be = serving.HifBackend(eps=1e-6, precision=1, lo=-2.0, hi=2.0, b=0.0)
    budget = int(args.serve_budget_gb * (1 << 30))
    # capacity: mean service time of requests served one at a time
    probe = serving.poisson_requests(len(sizes), 1.0, sizes, seed=20260104, nrhs_max=16)
    for i, r in enumerate(probe):
        r.n = sizes[i]
        r.m = serving.leaf_size(r.n)
        r.arrival = 0.0
    warm = serving.Server(be, budget, workers=1)
    warm.run(probe[:2], realtime=False)
    warm.release_all()
    t0 = time.perf_counter()
    one = serving.Server(be, budget, workers=1)
    one.run(probe, realtime=False)
    one.release_all()
    mean_service = (time.perf_counter() - t0) / len(probe)
    capacity = 1.0 / mean_service
    out = {"metric": "serving: p50/p99 request latency and solves/s (config 4)",
           "unit": "ms / solves/s", "data": "synthetic", "n_gpus": 1,
           "config": {"sizes": sizes, "a": "10^U(-2,2) iid per point, own seed per request",
                      "b": 0.0, "eps": 1e-6, "precision": "fp32 factor, fp64 PCG to 1e-10",
                      "rhs": "1-16 N(0,1) per request", "workers": args.serve_workers,
                      "budget_gb": args.serve_budget_gb, "requests": args.serve_requests},
           "capacity_req_per_s": capacity, "mean_service_s": mean_service, "loads": {}}
    for load in (0.5, 0.8):
        reqs = serving.poisson_requests(args.serve_requests, load * capacity, sizes,
                                        seed=20260104 + int(load * 10), nrhs_max=16)
        srv = serving.Server(be, budget, workers=args.serve_workers)
        st = srv.run(reqs)
        srv.release_all()
        out["loads"][str(load)] = st
    torch.cuda.synchronize()
    return out


def run_serving(args):
    import torch

    import __graft_entry__ as ge
    ge.build()
    torch.cuda.set_device(0)
    print(json.dumps(serving_record(args)), flush=True)
    return 0


def contrast256_record(hif, torch):
    """One untimed and one timed factor + PCG step of the 256^3 workload
    (a = 10^U(-3,3), b = 0, eps = 1e-4, FP32 factor), with its memory."""
    from paper_1607_00346_gb300 import inputs
    w = WORKLOADS["contrast256"]
    n, seed = w["n"], inputs.SEED_BASE + 4
    a = torch.from_numpy(make_field(w, n, seed)).cuda()
    f = torch.from_numpy(inputs.normal_rhs(n, 1, seed + 1)).cuda()
    u = torch.zeros_like(f)
    st = torch.cuda.current_stream()
    rec = None
    for k in range(2):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(st)
        h = hif.factor(n, w["m"], a, b_const=w["b"], eps=w["eps"], precision=hif.PREC_FP32)
        ev[1].record(st)
        its, rel = h.solve(f, u)
        ev[2].record(st)
        torch.cuda.synchronize()
        stt = h.stats()
        h.close()
        if k == 1:
            fs, ss = ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3
            rec = {"workload": f"n=256 (N={n ** 3}), {field_desc(w)}, b={w['b']}, eps={w['eps']}, "
                               "fp32 factor, FP64 PCG to 1e-10, nrhs=1",
                   "factor_s": fs, "solve_s": ss, "pcg_iters": its[0], "relres": rel[0],
                   "value": n ** 3 / (fs + ss) / 1e6, "unit": UNIT,
                   "peak_bytes": stt["peak_bytes"], "factor_bytes": stt["factor_bytes"],
                   "predicted_bytes": hif.predict_bytes(n, w["m"], eps=w["eps"],
                                                        precision=hif.PREC_FP32),
                   "hbm_budget_bytes": 180 * 10 ** 9, "root_size": stt["root_size"],
                   "retried_fronts": stt["retried_fronts"]}
    del a, f, u
    torch.cuda.empty_cache()
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="contrast128", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--nrhs", type=int, default=0)
    ap.add_argument("--no-fp64-form", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-n", type=int, default=32)
    ap.add_argument("--serve", action="store_true", help="run the serving benchmark instead")
    ap.add_argument("--serve-requests", type=int, default=30)
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-budget-gb", type=float, default=200.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the serving and 256^3 records of the default line")
    ap.add_argument("--no-autotune", action="store_true",
                    help="built-in launch shapes instead of timing them first")
    args = ap.parse_args()
    if args.gpus > 1 and int(os.environ.get("WORLD_SIZE", "1")) != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} runs one process per GPU: launch it with "
                         f"python -m torch.distributed.run --nproc-per-node {args.gpus} ...")
    if args.serve:
        return run_serving(args)
    w = dict(WORKLOADS[args.workload])
    if args.nrhs:
        w["nrhs"] = args.nrhs
    if args.impl == "reference":
        return run_reference(args, w)

    import numpy as np
    import torch

    ws, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if dist.is_nccl_available() else "gloo")

    import __graft_entry__ as ge
    if rank == 0:
        ge.build()
    if dist is not None:
        dist.barrier()
    from paper_1607_00346_gb300 import hif, inputs
    hif.load()
    # arithmetic peaks of this GPU, measured before anything else runs
    peaks = hif.measure_peaks()

    n, m, nrhs = w["n"], w["m"], w["nrhs"]
    N = n ** 3
    prec = hif.PREC_FP32 if args.precision == "fp32" else hif.PREC_FP64
    seed = inputs.SEED_BASE + 2
    a_h = make_field(w, n, seed)
    f_h = inputs.normal_rhs(n, nrhs, seed + 1)
    a_d = torch.from_numpy(a_h).cuda()
    f_d = torch.from_numpy(f_h).cuda()
    u_d = torch.zeros_like(f_d)
    stream = torch.cuda.current_stream()
    # launch shapes per size bucket, timed on this operator (bitwise-neutral)
    tune = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        table = hif.autotune(n, m, a_d, b_const=w["b"], eps=w["eps"], precision=prec, force=True)
        torch.cuda.synchronize()
        tune = {"seconds": time.perf_counter() - t0,
                "table": [l for l in table.splitlines() if l and not l.startswith("# hif")]}

    def step(evs=None, keep=False):
        if evs:
            evs[0].record(stream)
        h = hif.factor(n, m, a_d, b_const=w["b"], eps=w["eps"], precision=prec)
        if evs:
            evs[1].record(stream)
        its, rel = h.solve(f_d, u_d)
        if evs:
            evs[2].record(stream)
        st = h.stats()
        if keep:
            return its, rel, st, h
        h.close()
        return its, rel, st, None

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    # timed region: device events on the launching stream, barrier + sync around
    barrier()
    clk = ClockSampler(local)
    clk.start()
    hif.profile_begin()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    sub = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    ev[0].record(stream)
    per_step, its_all, rel_all, stats, hlast = [], [], [], None, None
    for k in range(args.steps):
        its, rel, stats, hk = step(sub[k], keep=(k == args.steps - 1))
        ev[k + 1].record(stream)
        its_all.append(its)
        rel_all.append(rel)
        hlast = hk or hlast
    barrier()
    prof = hif.profile_end()
    clocks = clk.stop()
    for k in range(args.steps):
        per_step.append(ev[k].elapsed_time(ev[k + 1]) / 1e3)
    fac_s = [sub[k][0].elapsed_time(sub[k][1]) / 1e3 for k in range(args.steps)]
    sol_s = [sub[k][1].elapsed_time(sub[k][2]) / 1e3 for k in range(args.steps)]
    total, rate = job_rate(N * nrhs * args.steps, sum(per_step), dist, "cuda")
    value = rate / 1e6

    # residual check of the last solve (FP64 operator, through the C ABI)
    r = torch.empty_like(f_d)
    hlast.residual(f_d, u_d, r)
    relres_chk = float((r.norm() / f_d.norm()).item())
    hlast.close()

    # end to end through the public API with host buffers (pinned), copies inside
    a_pin = torch.from_numpy(a_h).pin_memory()
    f_pin = torch.from_numpy(f_h).pin_memory()
    u_pin = torch.zeros(f_h.shape, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        with hif.factor(n, m, a_pin.numpy(), b_const=w["b"], eps=w["eps"], precision=prec) as h2:
            h2.solve(f_pin.numpy(), u_pin.numpy())
    barrier()
    e2e_t, e2e_rate = job_rate(N * nrhs * e2e_steps, time.perf_counter() - t0, dist, "cuda")
    e2e_value = e2e_rate / 1e6

    # roofline of the dominant kernel (largest share of the timed region)
    hbm_peak, hbm_src = _hbm_peak()
    total_prof_s = max(sum(p["seconds"] for p in prof), 1e-12)

    def roofline(k):
        per_launch_s = k["seconds"] / max(k["launches"], 1)
        bound = KERNEL_BOUND.get(k["name"], "alu" if k["flops"] > 0 else "hbm")
        if bound == "tensor":
            # algorithmic flops 2mnk of the products (the 3xTF32 split issues
            # three TF32 products per algorithmic one; that cost is the kernel's)
            peak = peaks["tf32_mma_tflops"]
            ach = k["flops"] / max(k["launches"], 1) / per_launch_s / 1e12
            src = "measured in this run: tcgen05 kind::tf32 loop (hif_measure_peaks)"
            unit = "TFLOP/s"
        elif bound == "alu":
            fp32 = prec == hif.PREC_FP32
            peak = peaks["fp32_fma_tflops" if fp32 else "fp64_fma_tflops"]
            ach = k["flops"] / max(k["launches"], 1) / per_launch_s / 1e12
            src = (f"measured in this run: {'FP32' if fp32 else 'FP64'} FMA loop "
                   "(hif_measure_peaks)")
            unit = "TFLOP/s"
        else:
            peak = hbm_peak
            ach = k["bytes"] / max(k["launches"], 1) / per_launch_s / 1e9
            src = hbm_src
            unit = "GB/s"
        return {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                "traffic": TRAFFIC_PER_LAUNCH.get(k["name"]), "kernel": k["name"],
                "peak_source": src, "share": k["seconds"] / total_prof_s,
                "launches_per_step": k["launches"] / args.steps}

    dom = max(prof, key=lambda p: p["seconds"])
    # kernels run in the timed region: every launch, the ones inside replayed
    # apply graphs included
    launches = sum(p["kernels"] for p in prof)
    roof = roofline(dom)
    roof_top = [roofline(k) for k in sorted(prof, key=lambda p: -p["seconds"])[:10]]

    # the plain FP64 GPU form of the same step (comparison point), one run
    fp64_form = None
    if not args.no_fp64_form and prec == hif.PREC_FP32:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = hif.factor(n, m, a_d, b_const=w["b"], eps=w["eps"], precision=hif.PREC_FP64)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        its64, rel64 = h.solve(f_d, torch.zeros_like(f_d))
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        h.close()
        fp64_form = {"factor_s": t1 - t0, "solve_s": t2 - t1, "pcg_iters": its64,
                     "value": N * nrhs / (t2 - t0) / 1e6}

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and ws == 1:
        dt, its_c, rel_c, _ = cpu_oracle_sample(w, args.cpu_sample_n, seed)
        cpu = {"value": args.cpu_sample_n ** 3 / dt / 1e6, "unit": UNIT, "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"CPU oracle factor + PCG on a {args.cpu_sample_n}^3 grid of the same "
                         f"coefficient law (N={args.cpu_sample_n ** 3}), {dt:.1f} s"}

    extras = {}
    if not args.no_extras and ws == 1:
        extras["contrast256"] = contrast256_record(hif, torch)
        extras["serving"] = serving_record(args)

    lat = sorted(per_step)
    p50 = statistics.median(lat)
    p99 = lat[min(len(lat) - 1, int(0.99 * len(lat)))]
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == hif.PREC_FP32 else "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: n={n} (N={N}), m={m}, "
                                   f"{field_desc(w)}, b={w['b']}, "
                                   f"eps={w['eps']}, {args.precision} factor, FP64 PCG to 1e-10, "
                                   f"nrhs={nrhs}",
                       "l2": "inputs and factor larger than L2 (no flush needed)",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "latency_ms": {"p50": 1e3 * p50, "p99": 1e3 * p99},
            "factor_s": statistics.median(fac_s), "solve_s": statistics.median(sol_s),
            "solve_mdofs": N * nrhs / statistics.median(sol_s) / 1e6,
            "pcg_iters": its_all[-1], "relres": rel_all[-1], "relres_check": relres_chk,
            "root_size": stats["root_size"], "factor_gflop": stats["flops"] / 1e9,
            "retried_fronts": stats["retried_fronts"],
            "factor_bytes": stats["factor_bytes"], "peak_bytes": stats["peak_bytes"],
            "clocks": clocks, "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * N * (1 + nrhs),
                    "d2h_bytes_per_step": 8 * N * nrhs},
            "roofline": roof, "roofline_top": [
                {k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()
                 if k in ("kernel", "bound", "achieved", "frac", "share", "unit")}
                for r in roof_top], "cpu_baseline": cpu, "fp64_form": fp64_form,
            "kernels": {p["name"]: round(p["seconds"] / args.steps, 5) for p in
                        sorted(prof, key=lambda p: -p["seconds"])[:24]},
            "peaks": {k: (round(v, 2) if isinstance(v, float) else v) for k, v in peaks.items()},
            "autotune": tune,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

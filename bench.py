"""Benchmark: seconds per 2D-DCSD iteration on one GB300 (replicas on N GPUs).

One step = one iteration of the on-device solver at the large open-shell
singlet workload (30 core + 2 open orbitals, 500 external virtuals, 1500 DF
functions; near-degenerate open orbitals 0.01 Eh apart): the full 2D-DCSD
singles/doubles residual for reference A (T1 dressing, DF
particle-particle ladder built on the fly, ring, hole-hole, Fock terms, DC
terms, two-determinant coupling, energy) followed by the Jacobi + DIIS
update.  Contractions run in BF16 on the tcgen05 tensor cores (the first
phase of the mixed-precision solve); denominators, DIIS, energies and the
residual norm are FP64.

Prints one JSON line.  --impl reference times the CPU oracle instead (a
bounded sample, scaled to the same workload).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "c5"  # 30+2 occupied/open, 500 virtuals, naux 1500
METRIC = "2D-DCSD s/iteration & ladder TFLOP/s vs peak; mixed vs FP64 at 1e-6 Eh"
UNIT = "s/iteration"


# dram__bytes_read.sum + dram__bytes_write.sum averaged over the 72 ladder
# GEMM launches (36 producer, 34 scatter consumer, 2 G-pass consumer) of one c5
# BF16 residual, from the one-pass ncu capture summarised in
# profiles/launches_c5_bf16_iteration.md (K-blocked ladder operands)
LADDER_DRAM_BYTES_PER_LAUNCH = 7.476e9


def ladder_flops(nc, nv, X):
    """Algorithmic flops of the DF particle-particle ladder per residual:
    2 o^2 v^4 (alpha-beta) + 4 C(o,2) C(v,2)^2 (same-spin unique pairs) +
    X v'^4 (unique DF build, (ac|bd) = (bd|ac))."""
    o, v, vp = nc + 1, nv + 1, nv + 2
    c2 = lambda k: k * (k - 1) / 2  # noqa: E731
    return 2 * o * o * v ** 4 + 4 * c2(o) * c2(v) ** 2 + X * vp ** 4


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def reduce_max(dist, x, device):
    """Max of a per-rank float over the ranks of the default process group
    (x itself without one); device: where the reduction tensor lives (cuda
    for NCCL, cpu for gloo)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(t_step, world):
    """Seconds per iteration of the whole job: N replicas each finish one
    iteration per step, so the job does N iterations in the max-over-ranks
    step time t_step."""
    return t_step / world if world > 1 else t_step


def oracle_sample(seconds_budget=20.0, workload=WORKLOAD):
    """Time the CPU oracle (as it stands) on a bounded sample: one 2D-DCSD
    residual of a reduced system with the same structure, scaled to the
    workload by the ratio of o^2 v^4 ladder operation counts."""
    from synth import make_system, random_amplitudes
    from oracle import twod
    nc, nv, X = 6, 40, 120
    s = make_system((nc, nv, X), seed=7)
    T = random_amplitudes(s, seed=8)
    t0 = time.perf_counter()
    n = 0
    while True:
        twod.residual(s, 0, twod.DCSD, T)
        n += 1
        if time.perf_counter() - t0 > seconds_budget or n >= 50:
            break
    dt = (time.perf_counter() - t0) / n
    c = __import__("synth").CONFIGS[workload]
    scale = ((c[0] + 1) ** 2 * (c[1] + 1) ** 4) / ((nc + 1) ** 2 * (nv + 1) ** 4)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": dt * scale, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} oracle 2D-DCSD residual(s) at n_c={nc}, n_v={nv}, naux={X} "
                      f"({dt:.3f} s each) scaled by the o^2 v^4 ladder operation count "
                      f"to n_c={c[0]}, n_v={c[1]} (x{scale:.3g})"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from synth import CONFIGS
    nc, nv, X, _, _ = CONFIGS[args.config]
    cb = oracle_sample(seconds_budget=max(5.0, 60.0 / max(1, args.steps + args.warmup)), workload=args.config)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": cb["value"] * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.config, "n_c": nc, "n_open": 2, "n_v": nv, "naux": X,
                       "method": "2D-DCSD", "reference": "A", "precision": "FP64 CPU oracle",
                       "parallelism": "single process (rank 0)"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--config", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import paper_2401_11935_gb300 as P
    from paper_2401_11935_gb300 import _lib as L
    from synth import CONFIGS, make_system, random_amplitudes

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    nc, nv, X, _, _ = CONFIGS[args.config]
    s = make_system(args.config)
    eng = P.Engine.from_system(s)
    stream = eng.stream
    # the solve starts from T = 0 (first step = MP1 amplitudes)
    T0 = None
    prec = P.PREC_BF16

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up: W iterations (allocates DIIS history and tensor-core buffers)
    T, _ = eng.solve(method=P.DCSD, precision=prec, tol=1e-30, maxiter=max(3, args.warmup), T0=T0)
    barrier()
    L.dcsd_profile(eng.ctx, 1, 1, read=False)
    launches0 = eng.launches()
    clk = Clocks(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    T, res = eng.solve(method=P.DCSD, precision=prec, tol=1e-30, maxiter=args.steps, T0=T)  # continues
    ev1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1)
    prof = L.dcsd_profile(eng.ctx, 0, 0)
    launches = eng.launches() - launches0
    t_step = reduce_max(dist, ms / 1e3 / args.steps, "cuda")
    # end-to-end: residual through the C ABI with pinned host buffers
    Th = [torch.empty(x.shape, dtype=torch.float64, pin_memory=True) for x in T]
    Rh = [torch.empty(x.shape, dtype=torch.float64, pin_memory=True) for x in T]
    for a, b in zip(Th, T):
        a.copy_(b.cpu())
    lib = L.load()
    import ctypes as C
    Wc, Ec = C.c_double(), C.c_double()

    def host_residual():
        st = lib.dcsd_residual(eng.ctx, 0, P.DCSD, prec, L.MEM_HOST, *[x.data_ptr() for x in Th],
                               *[x.data_ptr() for x in Rh], C.byref(Wc), C.byref(Ec))
        if st != 0:
            raise RuntimeError(lib.dcsd_last_error(eng.ctx))
    host_residual()
    barrier()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        host_residual()
    barrier()
    e2e = whole_job_value(reduce_max(dist, (time.perf_counter() - t0) / e2e_steps, "cuda"), world)
    nbytes = int(sum(x.numel() * 8 for x in Th))

    pk = peaks() or {}
    peak = pk.get("bf16_tflops_sustained")
    peak_src = "measured (sustained)" if peak else "fallback"
    if not peak:
        peak = 1700.0
    lf = ladder_flops(nc, nv, X)
    lad_ms, lad_n = prof["ladder_tc"]
    per_res_launches = lad_n / max(1, args.steps)
    achieved = (lf * args.steps) / (lad_ms / 1e3) / 1e12 if lad_ms > 0 else None
    line = {
        "metric": METRIC, "value": whole_job_value(t_step, world), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": args.config, "n_c": nc, "n_open": 2, "n_v": nv, "naux": X,
                   "method": "2D-DCSD", "reference": "A", "precision": "BF16 tcgen05 (mixed-precision phase 1)",
                   "l2": "inputs larger than L2 (T2 %.1f GB)" % (nbytes / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "tensor", "kernel": "k_tc_gemm (ladder producer+consumer)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None, "peak_source": peak_src,
                     "algorithmic_flops_per_launch": lf / max(1.0, per_res_launches),
                     "avg_launch_ms": lad_ms / max(1, lad_n), "traffic": LADDER_DRAM_BYTES_PER_LAUNCH,
                     "traffic_unit": "bytes per ladder launch (producer or consumer), DRAM read + write"},
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "note": "dcsd_residual with pinned host buffers (copies in the timed region)"},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "last_residual": {"max_r": res.max_r, "dEA": res.dEA, "W": res.W},
    }
    if rank == 0:
        print("# gpu part: " + json.dumps(line), file=sys.stderr, flush=True)
    if rank == 0 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = oracle_sample(seconds_budget=15.0)
        except Exception as ex:  # the GPU measurement stands without it
            line["cpu_baseline"] = {"value": None, "error": repr(ex)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    eng.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

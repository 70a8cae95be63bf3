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

Prints one JSON line.  Besides the timed iteration it carries the
mixed-precision solve against the FP64 solve (second named workload), the
CPU oracle on a bounded sample of the same workload (cpu_baseline) and the
oracle and the GPU on the same small configuration
(cpu_baseline_same_config).  --impl reference times the CPU oracle instead
(elements of the same workload, scaled to seconds per iteration).
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


# dram__bytes_read.sum + dram__bytes_write.sum averaged over the 90 ladder
# launches of one 30+2 / 500 / 1500 BF16 residual in symmetric / antisymmetric
# form (28 M+- producers and 56 consumers for the ladder, 2 producers and 4
# consumers for the G intermediate), from a one-pass ncu capture of this
# benchmark; set to None whenever the ladder kernels change until a new
# capture replaces it
LADDER_DRAM_BYTES_PER_LAUNCH = 4.343e9


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


def _cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def element_counts(nc, nv):
    """Residual elements of one iteration in the amplitude layout: singles
    2 o v, doubles 3 o^2 v^2 (o = n_c + 1, v = n_v + 1 per spin)."""
    o, v = nc + 1, nv + 1
    return 2 * o * v, 3 * o * o * v * v


class ElementSampler:
    """The element-wise CPU oracle (as it stands) on the benchmark workload
    itself: builds the inputs and the oracle once, then evaluates residual
    elements one at a time.  One iteration of the workload costs, for this
    oracle, the evaluation of every residual element, so the seconds per
    iteration are estimated as n_singles * t_singles + n_doubles * t_doubles
    from the timed elements."""

    def __init__(self, workload):
        from synth import make_system, random_amplitudes
        from oracle import element
        t0 = time.perf_counter()
        self.element = element
        self.s = make_system(workload)
        T = random_amplitudes(self.s, seed=3, ref=0, scale1=1e-3, scale2=1e-3)
        self.eo = element.ElementOracle(self.s, 0, 1, T)
        self.setup_s = time.perf_counter() - t0
        self.rng = np.random.default_rng(17)
        self.n1, self.n2 = element_counts(self.s.n_c, self.s.n_v)

    def one(self, doubles):
        o, v = self.s.o, self.s.v
        r = self.rng
        if doubles:
            blk, idx = int(r.integers(2, 5)), tuple(int(x) for x in (r.integers(o), r.integers(o),
                                                                       r.integers(v), r.integers(v)))
        else:
            blk, idx = int(r.integers(0, 2)), (int(r.integers(o)), int(r.integers(v)))
        self.eo._cache.clear()  # every element pays for its own intermediates
        t0 = time.perf_counter()
        self.element.residual_element(self.eo, blk, idx)
        return time.perf_counter() - t0

    def w_once(self):
        """W (the A->B doubles element) enters every element through the
        coupling terms and is computed once per residual, i.e. once per
        7e8 elements: its cost is left out of the estimate, and the timed
        elements use a placeholder value (their values are not used)."""
        self.eo._W = 0.0


def oracle_sample(workload=WORKLOAD):
    """cpu_baseline: one singles and one doubles element of the workload by
    the element-wise oracle, scaled to seconds per iteration by the element
    counts (about a minute of CPU including the input build)."""
    es = ElementSampler(workload)
    es.w_once()
    t1 = es.one(False)
    t2 = es.one(True)
    val = es.n1 * t1 + es.n2 * t2
    return {"value": val, "unit": UNIT, "cores": _cores(), "kind": "oracle",
            "sample": f"element-wise oracle on the {workload} workload: one singles element "
                      f"({t1:.1f} s) and one doubles element ({t2:.1f} s), scaled by the "
                      f"{es.n1} singles and {es.n2} doubles elements of one residual "
                      f"(inputs and oracle built in {es.setup_s:.0f} s, not counted)"}


def oracle_solve_c1():
    """The full CPU oracle as it stands: one converged 2D-DCSD solve of the
    smallest named workload (4 core + 2 open, 20 virtuals, naux 60)."""
    from synth import make_system
    from oracle import solve
    s = make_system("c1")
    t0 = time.perf_counter()
    _, info = solve.solve(s, 1, ref=0, tol=1e-10, maxiter=100)
    dt = time.perf_counter() - t0
    return {"s_per_solve": dt, "iters": int(info["iters"]), "s_per_iteration": dt / info["iters"],
            "E_S": float(info["E_S"]), "E_T": float(info["E_T"]), "cores": _cores()}


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle on the benchmark workload.  Each
    step is one residual element by the element-wise oracle (singles
    elements; one doubles element is timed during the untimed set-up), and
    the value is the estimated seconds per iteration (every element of one
    residual)."""
    if rank != 0:
        return 0
    from synth import CONFIGS
    nc, nv, X, _, _ = CONFIGS[args.config]
    es = ElementSampler(args.config)
    es.w_once()
    t2 = es.one(True)
    for _ in range(args.warmup):
        es.one(False)
    t0 = time.perf_counter()
    t1s = [es.one(False) for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    t1 = float(np.mean(t1s))
    val = es.n1 * t1 + es.n2 * t2
    cb = {"value": val, "unit": UNIT, "cores": _cores(), "kind": "oracle",
          "sample": f"element-wise oracle on the {args.config} workload: {args.steps} timed singles elements "
                    f"({t1:.2f} s each) and one doubles element ({t2:.1f} s), scaled by the {es.n1} singles "
                    f"and {es.n2} doubles elements of one residual"}
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": wall / max(1, args.steps) * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.config, "n_c": nc, "n_open": 2, "n_v": nv, "naux": X,
                       "method": "2D-DCSD", "reference": "A", "precision": "FP64 CPU oracle",
                       "parallelism": "single process (rank 0)",
                       "step": "one residual element (ms_per_step is the time of one step, not of an iteration)"},
            "cpu_baseline": cb,
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def mixed_vs_fp64(P, workload="c2", tol=1e-8):
    """The mixed-precision 2D-DCSD solve (BF16, then BF16X6, then defect
    correction with FP64 outer residuals) against the FP64 GPU solve of the
    second named workload (10 core + 2 open, 120 virtuals, naux 360): seconds
    per converged solve and the singlet / triplet energy differences, and
    both against the oracle's converged energies when the stored file of
    that workload has them."""
    from synth import make_system
    s = make_system(workload)
    eng = P.Engine.from_system(s)
    eng.reserve(P.PREC_MIXED, diis_n=8)
    _, f = eng.solve(method=P.DCSD, precision=P.PREC_FP64, tol=tol, maxiter=80)
    _, m = eng.solve(method=P.DCSD, precision=P.PREC_MIXED, tol=tol, maxiter=80)
    eng.close()
    out = {"workload": workload, "method": "2D-DCSD", "tol": tol,
           "fp64_s_per_solve": f.seconds, "fp64_iters": f.iters, "mixed_s_per_solve": m.seconds,
           "mixed_iters": m.iters, "speedup": f.seconds / m.seconds if m.seconds > 0 else None,
           "converged": bool(f.converged and m.converged),
           "E_S_mixed_minus_fp64": m.E_S - f.E_S, "E_T_mixed_minus_fp64": m.E_T - f.E_T,
           "gap_mixed_minus_fp64": (m.E_S - m.E_T) - (f.E_S - f.E_T)}
    path = os.path.join(ROOT, "tests", "golden", f"{workload}_energies.json")
    if os.path.exists(path):
        g = json.load(open(path))["results"].get("2D-DCSD")
        if g:
            out.update(E_S_mixed_minus_oracle=m.E_S - g["E_S"], E_T_mixed_minus_oracle=m.E_T - g["E_T"],
                       E_S_fp64_minus_oracle=f.E_S - g["E_S"], E_T_fp64_minus_oracle=f.E_T - g["E_T"])
    return out


def same_config_c1(P):
    """The CPU oracle and the GPU on the same configuration, the smallest named
    workload, where the full oracle finishes a converged solve in seconds:
    converged 2D-DCSD solves (tol 1e-10), FP64 on both sides."""
    from synth import make_system
    o = oracle_solve_c1()
    s = make_system("c1")
    eng = P.Engine.from_system(s)
    eng.reserve(P.PREC_FP64, diis_n=8)
    eng.solve(method=P.DCSD, precision=P.PREC_FP64, tol=1e-10, maxiter=100)  # warm-up
    _, g = eng.solve(method=P.DCSD, precision=P.PREC_FP64, tol=1e-10, maxiter=100)
    eng.close()
    return {"workload": "c1", "method": "2D-DCSD", "precision": "FP64 both",
            "oracle": o, "gpu": {"s_per_solve": g.seconds, "iters": g.iters, "s_per_iteration": g.seconds / g.iters,
                                 "E_S": g.E_S, "E_T": g.E_T},
            "oracle_over_gpu_per_solve": o["s_per_solve"] / g.seconds,
            "E_S_gpu_minus_oracle": g.E_S - o["E_S"], "E_T_gpu_minus_oracle": g.E_T - o["E_T"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--config", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the mixed-vs-FP64 solves")
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
    # end-to-end: the same iteration through the C ABI with pinned host
    # buffers -- dcsd_solve with mem_kind HOST and maxiter 1 copies the
    # amplitudes in, runs one residual and update, and copies them out
    Th = [torch.empty(x.shape, dtype=torch.float64, pin_memory=True) for x in T]
    for a, b in zip(Th, T):
        a.copy_(b.cpu())
    eng.reserve(prec, diis_n=8, host_staging=True)
    e2e_opts = L.dcsd_solve_opts(P.DCSD, 0, prec, 1, 8, 1e-30, 1e-5, 1, 0.0)

    def host_iteration():
        L.dcsd_solve(eng.ctx, e2e_opts, L.MEM_HOST, [x.data_ptr() for x in Th])
    host_iteration()
    barrier()
    e2e_steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        host_iteration()
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
                "note": "dcsd_solve(maxiter 1) with pinned host amplitudes: copy in, residual, update, copy out"},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "last_residual": {"max_r": res.max_r, "dEA": res.dEA, "W": res.W},
    }
    eng.close()
    del T, Th
    if rank == 0:
        print("# gpu part: " + json.dumps(line), file=sys.stderr, flush=True)
    if rank == 0 and world == 1 and not args.no_extra:
        try:
            line["mixed_vs_fp64"] = mixed_vs_fp64(P)
        except Exception as ex:
            line["mixed_vs_fp64"] = {"error": repr(ex)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = oracle_sample(args.config)
        except Exception as ex:  # the GPU measurement stands without it
            line["cpu_baseline"] = {"value": None, "error": repr(ex)}
        try:
            line["cpu_baseline_same_config"] = same_config_c1(P)
        except Exception as ex:
            line["cpu_baseline_same_config"] = {"error": repr(ex)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

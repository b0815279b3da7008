#!/usr/bin/env python
"""Benchmark of the Woodbury-circulant direct solver (arXiv 2203.13283).

Metric: RHS solves/s and setup seconds at N = 32768 (superellipse
|x|^4 + |y/0.6|^4 = 1, 10 elements per wavelength, 1024 plane waves uniform in
angle), mixed-precision form.  One step = the whole hot path over one batch:
mesh + assembly + circulant eigenvalues + randomized skeleton + capacitance
factor (setup), then 1024 plane-wave solves (projection, preconditioned
right-hand side of Eq. 5, Woodbury apply of Eq. 9, iterative refinement).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line on rank 0.
"""

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

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "RHS solves/s + setup s at N=32768, rel err <=1e-6, vs plain FP64 path"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], p["bf16_tflops"], p.get("bf16_tflops_sustained", p["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


def profile_figure(name, key):
    """A per-unit figure recorded in a profiles/ summary (line 'key: value')."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            for line in f:
                if line.startswith(key + ":"):
                    return float(line.split(":")[1]), "profiles/" + name
    except OSError:
        pass
    return None, None


def measured_traffic_ratio():
    """DRAM bytes (read + write) per algorithmic byte of the operator-product
    contraction, from the ncu capture summarised in profiles/ (a small case of
    the same kernel; the traffic of a launch scales with its planes read)."""
    path = os.path.join(ROOT, "profiles", "k_gemm_tc_ellipse_n4096_mixed.md")
    try:
        with open(path) as f:
            for line in f:
                if line.startswith("dram_bytes_per_algorithmic_byte:"):
                    return float(line.split(":")[1]), "profiles/k_gemm_tc_ellipse_n4096_mixed.md"
    except OSError:
        pass
    return None, None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def oracle_sample(w, n_sample, B_sample):
    """The CPU oracle on a bounded sample of the workload: the full dense
    pipeline (assembly, C of Eq. 6, LU solve of Eq. 5 for B_sample plane
    waves) at n_sample elements of the same contour family; returns seconds,
    the extrapolation to the full size by the N^2 (assembly) and N^3 (LU)
    costs, and the thread count."""
    from oracle import assembly, geometry, solver as osolver
    cur = geometry.Contour(w["family"], w["params"]) if w["family"] != "circle" else geometry.Circle(2 * np.pi)
    k, kt, _ = geometry.wavenumbers(cur.L, n_sample, w["k"])
    t0 = time.perf_counter()
    M = assembly.assemble(cur, n_sample, k, kt)
    t1 = time.perf_counter()
    e, hv = osolver.planewave_rhs(cur, n_sample, k, w["angles"][:B_sample])
    j, C, b = osolver.dense_solve(M, k, e, hv)
    t2 = time.perf_counter()
    N = w["N"]
    r = N / n_sample
    t_full = (t1 - t0) * r ** 2 + (t2 - t1) * r ** 3
    return t2 - t0, t_full, (t1 - t0), (t2 - t1)


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args, w):
    n_sample, B_sample = 256, 64
    times, fulls = [], []
    for it in range(args.warmup + args.steps):
        t, tf, ta, ts = oracle_sample(w, n_sample, B_sample)
        if it >= args.warmup:
            times.append(t)
            fulls.append(tf)
    full = statistics.median(fulls)
    value = w["angles"].size / full
    sample = (f"full oracle pipeline (dense FP64 assembly, dense C, LU solve) at N={n_sample}, "
              f"{B_sample} plane waves, same contour; extrapolated to N={w['N']}, B={w['angles'].size} "
              f"by N^2 (assembly) and N^3 (C formation + LU)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "RHS solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "N": w["N"], "B": int(w["angles"].size)},
            "cpu_baseline": {"value": value, "unit": "RHS solves/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "RHS solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="superellipse_n32768")
    ap.add_argument("--form", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--tol", type=float, default=None, help="skeleton tolerance")
    ap.add_argument("--max-rank", type=int, default=None,
                    help="skeleton rank cap (default N/8 in the mixed form, none in FP64)")
    ap.add_argument("--refine-tol", type=float, default=None)
    ap.add_argument("--rhs", type=int, default=None)
    ap.add_argument("--sample-planes", type=int, default=0,
                    help="mixed form: bf16 planes in the skeleton's sampling products (0: library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    from paper_2203_13283_gb300 import dist as wdist
    rank, world, local = wdist.world()
    w = dict(workloads.WORKLOADS[args.workload])
    if args.rhs:
        w["angles"] = workloads.uniform_angles(args.rhs)

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, w)
        return

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2203_13283_gb300 import build as libbuild
    libbuild.build()
    from paper_2203_13283_gb300 import Solver

    mixed = args.form == "mixed"
    tol = args.tol if args.tol is not None else (1e-6 if mixed else 1e-2)
    max_rank = args.max_rank if args.max_rank is not None else (w["N"] // 8 if mixed else 0)
    rtol = args.refine_tol if args.refine_tol is not None else (1e-7 if mixed else 1e-12)
    S = Solver(device=f"cuda:{local}", precision=1 if mixed else 0, refine_tol=rtol, max_refine=12,
               rhs_chunk=1024 if mixed else 256, block=64, sample_planes=args.sample_planes)
    stream = S.stream
    angles = w["angles"]
    B = len(angles)
    j = torch.empty((B, w["N"]), dtype=torch.complex128, device=S.device)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def step():
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        S.contour(w["family"], **w["params"])
        S.mesh(w["N"], w["k"])
        S.assemble()
        rank_ = S.skeleton(tol, max_rank=max_rank, seed=1, allow_cap=True)
        S.factor()
        e1.record(stream)
        S.solve_planewaves(angles, out=j, allow_unconverged=True)
        e2.record(stream)
        e2.synchronize()
        return e0.elapsed_time(e1) / 1e3, e1.elapsed_time(e2) / 1e3, rank_

    for _ in range(args.warmup):
        step()
    S.profile(True)
    S.profile_read(reset=True)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    from paper_2203_13283_gb300 import _lib
    launches0 = _lib.load().wcs_launch_count()
    T0 = torch.cuda.Event(enable_timing=True)
    T1 = torch.cuda.Event(enable_timing=True)
    T0.record(stream)
    setups, solves, ranks = [], [], []
    for _ in range(args.steps):
        su, so, rk = step()
        setups.append(su)
        solves.append(so)
        ranks.append(rk)
    T1.record(stream)
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = int(_lib.load().wcs_launch_count() - launches0)
    total = T0.elapsed_time(T1) / 1e3
    prof = S.profile_read(reset=True)
    S.profile(False)
    solve_s = sum(solves)
    # replicas: every rank solves its own batch; the slowest rank sets the time
    total, solve_s = wdist.max_over_ranks([total, solve_s], device=S.device)
    value = wdist.job_throughput(B * args.steps, world, solve_s)
    info = S.info()
    last = dict(S.last_solve)

    # end to end through the C ABI with host buffers: every step copies the
    # angles from pinned host memory and reads the (N x B) current back into
    # pinned host memory inside the timed call (after the setup)
    ang_h = torch.tensor(angles, dtype=torch.float64).pin_memory()
    jh = torch.empty((B, w["N"]), dtype=torch.complex128).pin_memory()
    S.solve_planewaves_host(ang_h, allow_unconverged=True, out=jh)   # warm-up
    t0 = time.perf_counter()
    for _ in range(args.steps):
        S.solve_planewaves_host(ang_h, allow_unconverged=True, out=jh)
    e2e_t = (time.perf_counter() - t0) / args.steps
    e2e = {"value": B / e2e_t, "unit": "RHS solves/s", "h2d_bytes_per_step": int(ang_h.numel() * 8),
           "d2h_bytes_per_step": int(jh.numel() * 16)}
    del jh

    hbm, bf16, bf16s, src = peaks()
    traffic_ratio, traffic_src = measured_traffic_ratio()
    g = prof["gemm_tc"]
    a = prof["assembly"]
    roof = None
    if g["launches"]:
        ms_per = g["ms"] / g["launches"]
        achieved = g["work"] / g["launches"] / (ms_per / 1e3) / 1e12
        alg_bytes = g["bytes"] / g["launches"]
        roof = {"bound": "tensor", "achieved": achieved, "peak": bf16s, "unit": "TFLOP/s",
                "frac": achieved / bf16s,
                "traffic": (traffic_ratio * alg_bytes) if traffic_ratio else None,
                "algorithmic_bytes_per_launch": alg_bytes, "traffic_source": traffic_src,
                "kernel": "k_gemm_tc (tcgen05 split-bf16 complex operator product)",
                "work": "useful complex-product flops 2*M*Nc*K (split-bf16 executes nprod x these)",
                "peak_source": f"{src} bf16 sustained", "launches": g["launches"], "ms_total": g["ms"]}
    # the roofline reported is that of the kernel with the largest share of the
    # step: the FP64 assembly (far pairs in FP64) or the tensor-core product
    roof_tensor = roof
    fp64_peak = 1.25   # TFLOP/s, nominal (the measured-peaks file has no FP64 figure)
    if a["launches"] and a["ms"] > g["ms"] + prof["gemm_tc_acc"]["ms"]:
        fpu, fsrc = profile_figure("k_assemble_fp64_ellipse_n4096_mixed.md", "fp64_flops_per_far_point_pair")
        bpu, _ = profile_figure("k_assemble_fp64_ellipse_n4096_mixed.md", "dram_bytes_per_far_point_pair")
        if fpu:
            units = a["work"] / a["launches"]
            ach = fpu * units / (a["ms"] / a["launches"] / 1e3) / 1e12
            roof = {"bound": "fp64", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": ach / fp64_peak, "traffic": (bpu * units) if bpu else None,
                    "kernel": "k_assemble<1> (FP64 point-pair integration of S~, D, D~, N)",
                    "work": f"far point pairs N^2 q_far^2 = {units:.3e} per launch x {fpu:.0f} FP64 flops per pair "
                            "(counted DFMA/DADD/DMUL at N = 4096)",
                    "peak_source": "nominal GB300 FP64 (recipe table)", "figures_source": fsrc}
    line = {
        "metric": METRIC, "value": value, "unit": "RHS solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x2/fp32/f64" if mixed else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "N": w["N"], "B": B, "k": info["k"], "form": args.form,
                   "skeleton_tol": tol, "rank": ranks[-1], "refine_tol": rtol,
                   "refine_steps": last["refine_steps"], "rel_residual": last["rel_residual"],
                   "setup_s": statistics.median(setups), "solve_s": statistics.median(solves),
                   "l2": "operators (tens of GB) exceed L2: no flush needed", "parallelism": f"replicas{world}"},
        "setup_s": statistics.median(setups),
        "e2e": e2e, "clocks": clk, "roofline": roof, "roofline_tensor_product": roof_tensor,
        "kernels": {k: {"launches": v["launches"], "ms": v["ms"]} for k, v in prof.items() if v["launches"]},
        "assembly_pairs_per_s": (a["work"] / (a["ms"] / 1e3)) if a["launches"] else None,
        "gpu_launches": launches,
    }
    if rank == 0 and not args.no_cpu_baseline:
        n_sample, B_sample = 256, 64
        t, tf, _, _ = oracle_sample(w, n_sample, B_sample)
        line["cpu_baseline"] = {"value": B / tf, "unit": "RHS solves/s", "cores": cpu_threads(), "kind": "oracle",
                                "sample": f"oracle full pipeline at N={n_sample}, {B_sample} RHS ({t:.1f} s), "
                                          f"extrapolated to N={w['N']}, B={B} by N^2 assembly + N^3 LU"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    S.close()


if __name__ == "__main__":
    main()

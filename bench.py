#!/usr/bin/env python
"""Benchmark: CBS energies per second at eigenpair residual <= 1e-8, on GB300.

One step = the whole method (contour, batched shifted BiCG solves with their duals,
moments, Hankel SVD + reduced eigenproblem, residual filter, k) for every energy of the
workload, through libcbs's C ABI.  Default workload: the 32x32x16 molecular-crystal
cell (8th-order FD, 40 atoms with 4 projectors each, 16 energies in [-0.5, 0.5] Ha,
N_int = 32 per circle, L = 32, M = 8) in plain FP64 — the configuration the metric is
quoted on.  The headline is the FP64 form with one BiCG Krylov sequence per quadrature
point and column shared by all energies of the step (shifted BiCG, P(z, E) = P(z, E0) +
(E - E0) I; columns that miss the tolerance on the true residual are finished by plain
BiCG).  Beside it, on the same workload: the paper's scheme of one FP64 BiCG per (energy,
quadrature point) ("fp64_per_energy") and complex64 BiCG with FP64 reliable updates
("fp32_refine").

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c2] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank solves its own copy of the
energy list (independent problems, no collective on the data path): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CBS energies/sec at residual<=1e-8 (FP32+refine vs FP64); SpMM HBM GB/s"
UNIT = "energies/s"

# DRAM traffic of the FP64 stencil+projector apply per complex output, from one ncu
# capture (profiles/apply_fp64_c2.md), valid while csrc/apply.cu hashes to APPLY_SHA.
# DRAM bytes per output of the apply pair (stencil + projector gather) from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, 64 systems of the 32x32x16 cell, L = 32,
# tuned shape); valid while apply.cu has this hash
APPLY_TRAFFIC = {"sha": "e1a5bc6eb446a0ce", "c128_bytes_per_output": 45.437, "c64_bytes_per_output": None}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# GB300 FP64: 1.25 TFLOP/s nominal (152 SMs x 2.07 GHz x 4 FLOP/clk/SM).
FP64_PEAK_TFLOPS = 1.25
# FP64 FMA rate measured on this GB300 (independent DFMA chains in every warp of 8 blocks
# per SM): 1.003 TFLOP/s = 0.5 T lane-instructions per second
FP64_FMA_MEASURED_TFLOPS = 1.003


def _apply_sha():
    with open(os.path.join(ROOT, "paper_1709_09347_gb300", "csrc", "apply.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def flops_per_output(wl):
    """Algorithmic real flops per complex output of the operator apply: 2 (diagonal) +
    18 per FD half-width step (x, y, z pairs) + 4 (E x - acc) + per covering projector
    entry 4*n_proj (gather) + 4*n_proj + 2 (scatter)."""
    m = wl.grid.fd_order // 2
    f = 2 + 18 * m + 4
    if wl.projectors is not None:
        npj = wl.projectors.n_proj
        f += wl.projectors.nnz / wl.grid.n * (8 * npj + 2)
    return f


def fp64_instr_per_output(wl):
    """FP64 lane-instructions the complex128 apply issues per complex output: per FD
    half-width step and component three pair sums and three FMAs (12 per step), 3 for the
    diagonal term; per covering projector entry 2*n_proj FMAs in the gather and 2*n_proj in
    the scatter, plus a complex multiply-add (4) for entries of a displaced image."""
    m = wl.grid.fd_order // 2
    f = 12 * m + 3
    if wl.projectors is not None:
        P = wl.projectors
        wrapped = float((P.sup_wrap != 0).mean()) if P.nnz else 0.0
        f += P.nnz / wl.grid.n * (4 * P.n_proj + 4 * wrapped)
    return f


def bytes_per_output(wl, s):
    """Algorithmic bytes per complex output: read X and write Y once (2 s) plus the local
    potential (s/2 per point) and the projector table (values + index) amortised over L."""
    b = 2 * s + (s / 2) / wl.L
    if wl.projectors is not None:
        npj = wl.projectors.n_proj
        b += wl.projectors.nnz / wl.grid.n * (npj * s / 2 + 8) / wl.L
    return b


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline_sample(workload: str, n_points: int, energy_index: int) -> dict:
    """Time the oracle (as it stands) on a bounded sample: n_points of the n_int
    quadrature-point BiCG solves of one energy, single-threaded.  Runs in a child process
    with one BLAS/OpenMP thread so that `cores` is exact."""
    code = f"""
import json, os, sys, time
sys.path.insert(0, {ROOT!r})
from paper_1709_09347_gb300 import synth
from oracle.operator import CellOperator
from oracle.contour import ring_contour
from oracle.bicg import bicg
wl = synth.workload({workload!r})
op = CellOperator(wl.grid, wl.vloc, wl.projectors)
E = float(wl.energies[{energy_index}])
z1 = ring_contour(wl.lambda_min, wl.n_int)[0]
t = time.time()
iters = []
for j in range({n_points}):
    z = z1[j * (wl.n_int // {n_points})]
    X, Xt, it, info = bicg(lambda X: op.apply_P(z, E, X), lambda X: op.apply_P_adjoint(z, E, X),
                           wl.V, wl.V, tol=wl.tol)
    iters.append(int(it.max()))
dt = time.time() - t
print(json.dumps(dict(seconds=dt, iters=iters, n_int=wl.n_int)))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    r = json.loads(out.stdout.strip().splitlines()[-1])
    per_energy = r["seconds"] * r["n_int"] / n_points
    return {"value": 1.0 / per_energy, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"{workload}: {n_points} of {r['n_int']} quadrature-point BiCG solves "
                       f"(primal+dual, all L columns) at energy index {energy_index}, "
                       f"{r['seconds']:.1f} s, iterations {r['iters']}; scaled by n_int/{n_points} "
                       f"to one energy (extraction not included)"),
            "seconds": r["seconds"]}


def run_reference(args, world, rank):
    if rank != 0:
        return
    steps = []
    samples = []
    for k in range(args.warmup + args.steps):
        r = cpu_baseline_sample(args.workload, 1, 7)
        if k >= args.warmup:
            steps.append(1.0 / r["value"])
            samples.append(r)
    per_energy = sum(steps) / len(steps)
    value = 1.0 / per_energy
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_energy * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "sample": "1 of n_int quadrature-point solves per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": samples[-1]["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--energies", type=int, default=0,
                    help="solve only the first K energies of the workload (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--spmm", action="store_true",
                    help="only time the operator apply (stencil + projector SpMM) and exit")
    ap.add_argument("--spmm-systems", type=int, default=0,
                    help="systems per SpMM launch (default: all primal and dual systems of a step)")
    ap.add_argument("--spmm-dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-shift", action="store_true",
                    help="headline with one BiCG per (energy, quadrature point), as in the paper")
    ap.add_argument("--no-per-energy", action="store_true",
                    help="skip the per-energy FP64 comparison run")
    ap.add_argument("--mixed-steps", type=int, default=1)
    ap.add_argument("--mixed-warmup", type=int, default=1)
    args = ap.parse_args()
    world, rank, local = _dist()

    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import numpy as np
    import torch

    from paper_1709_09347_gb300 import cbs, synth

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    wl = synth.workload(args.workload)
    energies = wl.energies if args.energies <= 0 else wl.energies[:args.energies]
    n_e = len(energies)
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    Vd = torch.from_numpy(wl.V).to(dev).contiguous()
    # launch shapes of the stencil kernel, tuned once per cell before any timing
    n_tune = min(64, 2 * wl.n_int * n_e)
    tune = {"c128": cbs.autotune_apply(H, n_tune, wl.L, torch.complex128),
            "c64": cbs.autotune_apply(H, n_tune, wl.L, torch.complex64)}

    def spmm(n_sys, dtype_name, iters=20):
        """Operator apply alone, at the batch shape of a step, timed with CUDA events on
        torch's current stream (the stream the kernels are launched on)."""
        dt = torch.complex64 if dtype_name == "c64" else torch.complex128
        s = 8 if dtype_name == "c64" else 16
        rng = np.random.default_rng(3)
        zs = (np.exp(1j * rng.uniform(0, 2 * np.pi, n_sys)) *
              np.where(np.arange(n_sys) % 2 == 0, 1 / wl.lambda_min, wl.lambda_min))
        plan = cbs.ApplyPlan(H, zs, 0.1, wl.L, dt)
        X = torch.randn(n_sys, wl.grid.n, wl.L, dtype=dt, device=dev)
        Yo = torch.empty_like(X)
        for _ in range(3):
            plan(X, Yo)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(iters):
            plan(X, Yo)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / iters
        outputs = n_sys * wl.grid.n * wl.L
        bpo = bytes_per_output(wl, s)
        hbm, src = _peaks()
        r = {"dtype": dtype_name, "systems": n_sys, "columns": wl.L, "ms_per_launch": ms,
             "bytes_per_launch": bpo * outputs, "GB_s": bpo * outputs / (ms / 1e3) / 1e9,
             "peak_GB_s": hbm, "peak_source": src,
             "frac": bpo * outputs / (ms / 1e3) / 1e9 / hbm,
             "TFLOP_s": flops_per_output(wl) * outputs / (ms / 1e3) / 1e12}
        del X, Yo, plan
        torch.cuda.empty_cache()
        return r

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(x):
        if world > 1:
            t = torch.tensor([x], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            return float(t.item())
        return x

    def one_step(precision, shift=False, profile=True):
        o = cbs.options(precision=precision, tol=wl.tol, delta=wl.delta, profile=1 if profile else 0,
                        multi_shift=1 if shift else 0)
        return cbs.solve(H, energies, wl.lambda_min, wl.n_int, wl.L, wl.M, Vd, o)

    def timed(precision, steps, warmup, shift=False):
        for _ in range(warmup):
            one_step(precision, shift)
        barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = cbs.kernel_launches()
        results = []
        with ClockSampler(local) as clk:
            ev0.record()
            for _ in range(steps):
                results.append(one_step(precision, shift))
            ev1.record()
            torch.cuda.synchronize()
        launches = cbs.kernel_launches() - l0
        barrier()
        ms = max_over_ranks(ev0.elapsed_time(ev1))
        return ms, results, clk.summary(), launches

    hbm, hbm_src = _peaks()
    sha = _apply_sha()
    n_step_sys = 2 * wl.n_int * n_e
    if args.spmm:
        r = spmm(args.spmm_systems or n_step_sys, args.spmm_dtype)
        if rank == 0:
            print(json.dumps({"spmm": r, "workload": args.workload, "apply_shape": tune}), flush=True)
        return

    def roofline_for(results, precision, ms_total):
        key = "c64" if precision == "fp32_refine" else "c128"
        p = {f: sum(r.profile[key][f] for r in results) for f in ("ms", "launches", "outputs")}
        if not p["ms"]:
            return None
        s = 8 if key == "c64" else 16
        rl = {"kernel": f"k_apply_zm + k_proj_gather ({'complex64' if s == 8 else 'complex128'}): "
                        "stencil + projector operator apply",
              "outputs": p["outputs"], "launches": p["launches"],
              "avg_launch_ms": p["ms"] / max(p["launches"], 1),
              "share_of_step": p["ms"] / ms_total if ms_total else None}
        traffic = None
        tkey = f"{key}_bytes_per_output"
        if APPLY_TRAFFIC["sha"] == sha and APPLY_TRAFFIC.get(tkey):
            traffic = APPLY_TRAFFIC[tkey] * p["outputs"] / max(p["launches"], 1)
        if key == "c64":
            bpo = bytes_per_output(wl, 8)
            ach = p["outputs"] * bpo / (p["ms"] / 1e3) / 1e9
            rl.update(bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm,
                      traffic=traffic, peak_source=hbm_src, bytes_per_output=bpo,
                      bytes_per_launch=bpo * p["outputs"] / max(p["launches"], 1))
        else:
            fpo = flops_per_output(wl)
            ach = p["outputs"] * fpo / (p["ms"] / 1e3) / 1e12
            ipo = fp64_instr_per_output(wl)
            pipe = ipo * p["outputs"] / (p["ms"] / 1e3) / (FP64_FMA_MEASURED_TFLOPS * 1e12 / 2)
            rl.update(bound="alu", achieved=ach, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
                      frac=ach / FP64_PEAK_TFLOPS, traffic=traffic,
                      peak_source="nominal FP64 (152 SMs x 2.07 GHz x 4 FLOP/clk)",
                      flops_per_output=fpo, flops_per_launch=fpo * p["outputs"] / max(p["launches"], 1),
                      fp64_instr_per_output=ipo, fp64_pipe_frac_of_measured=pipe,
                      measured_fp64_fma_tflops=FP64_FMA_MEASURED_TFLOPS)
        return rl

    def roofline_shift_update(results):
        """Roofline of the shifted-family update kernel.  Per (energy, point, column) triple
        and grid point it issues 16 FP64 FMAs (two complex multiply-adds, primal and dual)
        and moves the scaled direction and the solution in and out, primal and dual
        (8 x 16 B; the seed residual it also reads is shared by all energies of a point and
        not counted).  FP64 issue binds first on this part, so the FP64 rate is the roofline
        and the HBM rate is reported beside it."""
        p = {f: sum(r.profile["shift_update"][f] for r in results) for f in ("ms", "launches", "outputs")}
        if not p["ms"]:
            return None
        bpo, ipo = 8 * 16, 16
        sec = p["ms"] / 1e3
        ach = p["outputs"] * 2 * ipo / sec / 1e12
        gbs = p["outputs"] * bpo / sec / 1e9
        return {"kernel": "k_ms_update: shifted-family direction and solution update",
                "outputs": p["outputs"], "launches": p["launches"],
                "avg_launch_ms": p["ms"] / max(p["launches"], 1), "bound": "alu", "achieved": ach,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                "traffic": None, "peak_source": "nominal FP64 (152 SMs x 2.07 GHz x 4 FLOP/clk)",
                "fp64_instr_per_output": ipo,
                "fp64_pipe_frac_of_measured": ach / FP64_FMA_MEASURED_TFLOPS,
                "measured_fp64_fma_tflops": FP64_FMA_MEASURED_TFLOPS,
                "hbm_achieved_GB_s": gbs, "hbm_peak_GB_s": hbm, "hbm_frac": gbs / hbm,
                "hbm_peak_source": hbm_src, "bytes_per_output": bpo,
                "bytes_per_launch": bpo * p["outputs"] / max(p["launches"], 1)}

    def summary(results):
        last = results[-1]
        kept = [len(e["lam"]) for e in last.energies]
        worst = max([float(np.max(e["residual"])) for e in last.energies if len(e["residual"])] or [0.0])
        return last, kept, worst, sorted({e["flags"] for e in last.energies})

    # headline: FP64, one BiCG Krylov sequence per quadrature point and column shared by
    # all energies of the step (shifted BiCG), or per-energy BiCG with --no-shift
    shift = not args.no_shift
    ms, results, clocks, launches = timed("fp64", args.steps, args.warmup, shift)
    value = args.steps * n_e * world / (ms / 1e3)
    last, kept, worst_res, flags = summary(results)
    roofline = roofline_for(results, "fp64", ms)
    roofline_update = roofline_shift_update(results) if shift else None
    if roofline_update is not None:
        roofline_update["share_of_step"] = (roofline_update["avg_launch_ms"] * roofline_update["launches"]
                                            / ms)
        if roofline is None or roofline_update["share_of_step"] > roofline["share_of_step"]:
            roofline, roofline_update = roofline_update, roofline

    # comparison: the paper's scheme, one FP64 BiCG per (energy, quadrature point)
    per_energy = None
    if shift and not args.no_per_energy:
        msp, resp, clocksp, launchesp = timed("fp64", 1, 1, False)
        lastp, keptp, worstp, flagsp = summary(resp)
        per_energy = {"value": n_e * world / (msp / 1e3), "unit": UNIT, "ms_per_step": msp,
                      "steps": 1, "warmup": 1, "dtype": "f64", "kept_per_energy": keptp,
                      "same_count_as_headline": keptp == kept, "max_residual": worstp,
                      "flags": flagsp, "roofline": roofline_for(resp, "fp64", msp),
                      "clocks": clocksp, "gpu_launches": launchesp,
                      "stage_ms_last_step": {"solve": lastp.ms_solve, "moments": lastp.ms_moments,
                                             "extract": lastp.ms_extract}}

    # comparison: complex64 BiCG with FP64 reliable updates on the same workload
    mixed = None
    if not args.no_mixed:
        ms32, res32, clocks32, launches32 = timed("fp32_refine", args.mixed_steps, args.mixed_warmup)
        last32, kept32, worst32, flags32 = summary(res32)
        mixed = {"value": args.mixed_steps * n_e * world / (ms32 / 1e3), "unit": UNIT,
                 "ms_per_step": ms32 / args.mixed_steps, "steps": args.mixed_steps,
                 "warmup": args.mixed_warmup, "dtype": "c64 BiCG + f64 reliable updates",
                 "kept_per_energy": kept32, "same_count_as_headline": kept32 == kept,
                 "max_residual": worst32, "flags": flags32,
                 "roofline": roofline_for(res32, "fp32_refine", ms32), "clocks": clocks32,
                 "gpu_launches": launches32,
                 "stage_ms_last_step": {"solve": last32.ms_solve, "moments": last32.ms_moments,
                                        "extract": last32.ms_extract}}

    # end to end through the C ABI with host buffers: Hamiltonian upload, V upload,
    # solve, results (eigenvalues, k, residuals, eigenvectors) back to the host
    def e2e_step():
        Hh = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
        cbs.set_apply_shape(Hh, torch.complex128, tune["c128"]["py"], tune["c128"]["pz"])
        r = cbs.solve(Hh, energies, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                      cbs.options(precision="fp64", tol=wl.tol, delta=wl.delta,
                                  multi_shift=1 if shift else 0))
        Hh.close()
        return r
    e2e_steps = 1
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        r_e2e = e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    h2d = wl.vloc.nbytes + wl.V.nbytes
    if wl.projectors is not None:
        P = wl.projectors
        h2d += P.sup_ptr.nbytes + P.sup_idx.nbytes + P.sup_wrap.nbytes + P.sup_val.nbytes + P.h.nbytes
    d2h = sum(e["lam"].nbytes + e["k"].nbytes + e["residual"].nbytes + e["vectors"].nbytes
              for e in r_e2e.energies)
    e2e = {"value": e2e_steps * n_e * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "steps": e2e_steps}

    spmm_res = {"c64": spmm(n_step_sys, "c64"), "c128": spmm(n_step_sys, "c128", iters=3)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline_sample(args.workload, 1, 7)
        except Exception as ex:  # noqa: BLE001
            cpu = {"error": str(ex)[-300:]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wl.grid.nx}x{wl.grid.ny}x{wl.grid.nz} cell, "
                                   f"FD{wl.grid.fd_order}, "
                                   f"{wl.projectors.n_atoms if wl.projectors else 0} atoms x 4 projectors, "
                                   f"{n_e} energies, N_int={wl.n_int}, L={wl.L}, M={wl.M}, "
                                   f"lambda_min={wl.lambda_min}, BiCG tol {wl.tol:g}",
                       "solver": "shifted-family BiCG (one Krylov sequence per z_j for all energies)"
                                 if shift else "one BiCG per (energy, z_j)",
                       "energies_per_step": n_e, "l2": "state per step >> L2 (no flush needed)",
                       "kept_per_energy": kept, "max_residual": worst_res, "flags": flags,
                       "apply_shape": tune},
            "e2e": e2e, "gpu_launches": launches, "clocks": clocks, "roofline": roofline,
            "roofline_second_kernel": roofline_update,
            "cpu_baseline": cpu, "fp64_per_energy": per_energy, "fp32_refine": mixed,
            "spmm": spmm_res,
            "stage_ms_last_step": {"solve": last.ms_solve, "moments": last.ms_moments,
                                   "extract": last.ms_extract, "extract_svd": last.ms_svd,
                                   "extract_reduced_eig": last.ms_reduced,
                                   "extract_vectors": last.ms_vectors},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

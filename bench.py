#!/usr/bin/env python
"""Benchmark: CBS energies per second at eigenpair residual <= 1e-8, on GB300.

One step = the whole method (contour, batched shifted BiCG solves with their duals,
moments, Hankel SVD + reduced eigenproblem, residual filter, k) for the energies of the
step, through libcbs's C ABI.  Headline workload: the 32x32x16 molecular-crystal cell
(8th-order FD, 40 atoms with 4 projectors each, all 16 energies in [-0.5, 0.5] Ha,
lambda_min = 0.5, N_int = 32 per circle, L = 32, M = 8, the paper's BiCG tolerance 1e-10),
in the form that is fastest at the residual bar: FP64 with one BiCG Krylov sequence per
quadrature point and column shared by every energy of the step (shifted BiCG,
P(z, E) = P(z, E0) + (E - E0) I), half the points solved (real V: the conjugate points'
solutions are the conjugates), columns missing the tolerance on the true residual finished
per energy.

Beside it, on the same step and bar, each timed once: the complex64 shifted family refined
per energy with complex64 BiCG and FP64 reliable updates ("mixed"), complex64 BiCG per
(energy, point) with reliable updates ("mixed_per_energy"), FP64 BiCG per (energy, point) as
in the paper ("fp64_per_energy"), and the FP64 family with the paper's stop-at-half rule
("fp64_stop_half").  The 64x64x24 precision cell (120 atoms, lambda_min = 0.3, N_int = 64) is
measured once per form at energy index 19 ("second_workload"): its steps take minutes.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c2] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank solves its own copy of the
step (independent problems, no collective on the data path): weak scaling.
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

# energies of one step per workload (indices into the workload's energy list); workloads
# not listed take all of their energies
STEP_ENERGIES = {"c3": (3, 11, 19, 27)}

# DRAM bytes per unit of the kernels reported as rooflines, each from one ncu capture on one
# workload (dram__bytes_read.sum + dram__bytes_write.sum of the gather + stencil launch pair,
# divided by the complex outputs of the captured pair), valid for that workload while the
# kernel's source file hashes to `sha`.  The FP64 shifted-family update has none: its
# captured launch does not record how many energies were still active.
KERNEL_TRAFFIC = {
    # 32x32x16 cell, 32 systems (16 points and their duals), 16.78 M outputs: 745.7 MB
    ("c128_apply", "c2"): {"file": "apply.cu", "sha": "f77085a5a8f84789", "bytes_per_unit": 44.45},
    # 64x64x24 cell, 128 systems, 402.7 M outputs: 8.681 GB
    ("c64_apply", "c3"): {"file": "apply.cu", "sha": "f77085a5a8f84789", "bytes_per_unit": 21.56},
}

FORMS = {
    "mixed": {"precision": "fp32_refine", "multi_shift": 1,
              "dtype": "c64 shifted-family BiCG + c64/f64 reliable-update refinement"},
    "fp64": {"precision": "fp64", "multi_shift": 1, "dtype": "f64"},
    "fp64_per_energy": {"precision": "fp64", "multi_shift": 0, "dtype": "f64"},
    "mixed_per_energy": {"precision": "fp32_refine", "multi_shift": 0,
                         "dtype": "c64 BiCG + f64 reliable updates, one BiCG per (energy, point)"},
    # the paper's load-balance rule: BiCG stops once over half the points of an energy converged
    "fp64_stop_half": {"precision": "fp64", "multi_shift": 1, "stop_fraction": 0.5, "dtype": "f64"},
}

# headline workload and form; forms timed once beside it; a second workload measured once
# per form in the same run
DEFAULT_WORKLOAD = "c2"
DEFAULT_FORM = "fp64"
DEFAULT_COMPARE = ("mixed", "mixed_per_energy", "fp64_per_energy", "fp64_stop_half")
SECOND_WORKLOAD = "c3"
SECOND_ENERGIES = (19,)
SECOND_FORMS = ("fp64", "mixed", "fp64_stop_half")

# GB300 FP64: 1.25 TFLOP/s nominal (152 SMs x 2.07 GHz x 4 FLOP/clk/SM).
FP64_PEAK_TFLOPS = 1.25


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _sha(fname):
    with open(os.path.join(ROOT, "paper_1709_09347_gb300", "csrc", fname), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _traffic(key, workload, units_per_launch):
    t = KERNEL_TRAFFIC.get((key, workload))
    if t and _sha(t["file"]) == t["sha"]:
        return t["bytes_per_unit"] * units_per_launch
    return None


def apply_bytes_per_output(wl, s):
    """Algorithmic bytes per complex output of the operator apply: read X and write Y once
    (2 s) plus the local potential (s/2 per point) and the projector table (values + index)
    amortised over the L columns."""
    b = 2 * s + (s / 2) / wl.L
    if wl.projectors is not None:
        npj = wl.projectors.n_proj
        b += wl.projectors.nnz / wl.grid.n * (npj * s / 2 + 8) / wl.L
    return b


def apply_flops_per_output(wl):
    """Algorithmic real flops per complex output of the operator apply: 2 (diagonal) + 18
    per FD half-width step (x, y, z pairs) + 4 (E x - acc) + per covering projector entry
    4*n_proj (gather) + 4*n_proj + 2 (scatter)."""
    m = wl.grid.fd_order // 2
    f = 2 + 18 * m + 4
    if wl.projectors is not None:
        f += wl.projectors.nnz / wl.grid.n * (8 * wl.projectors.n_proj + 2)
    return f


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


def step_energy_indices(wl, spec):
    if spec:
        return [int(a) for a in spec.split(",")]
    return list(STEP_ENERGIES.get(wl.name, range(len(wl.energies))))


# ---------------------------------------------------------------------- CPU oracle timing
CPU_SAMPLE = {
    # workload: (energy index with a stored oracle run, BiCG iterations to time per point)
    "c3": (0, "tests/golden/c3_oracle_e00.npz", 12),
    "c2": (7, "tests/golden/c2_oracle.npz", 12),
}


def _oracle_point_worker(args):
    """One quadrature point of the oracle's BiCG for a fixed number of iterations (the
    timing sample); runs in a spawned process with one BLAS thread."""
    workload, energy_index, j, n_iter = args
    import time as _t
    from oracle.bicg import bicg
    from oracle.contour import ring_contour
    from oracle.operator import CellOperator
    from paper_1709_09347_gb300 import synth
    wl = synth.workload(workload)
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    E = float(wl.energies[energy_index])
    z = ring_contour(wl.lambda_min, wl.n_int)[0][j]
    t = _t.time()
    bicg(lambda X: op.apply_P(z, E, X), lambda X: op.apply_P_adjoint(z, E, X), wl.V, wl.V,
         tol=1e-300, max_iter=n_iter)
    return _t.time() - t


def cpu_baseline_sample(workload: str) -> dict:
    """The oracle as it stands, on the host's cores: its plain FP64 BiCG (primal + dual,
    all L columns) runs a fixed number of iterations at one quadrature point per core, in
    parallel spawned processes; the time per iteration is scaled by the BiCG iteration
    counts of the oracle's own stored run of that energy (per point, the slowest column)
    to one energy's Step 1 (extraction excluded).  The sampled energy is the cheapest of
    the workload's range: the rate is an upper bound for the oracle on the whole step."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import numpy as np
    if workload not in CPU_SAMPLE:
        return {"error": f"no stored oracle run to scale a sample of {workload}"}
    e_idx, path, n_iter = CPU_SAMPLE[workload]
    g = np.load(os.path.join(ROOT, path))
    iters = g["iters"] if "iters" in g.files else g[f"iters_{e_idx}"]
    cores = os.cpu_count() or 1
    n_int = iters.shape[0]
    pts = list(range(min(cores, n_int)))
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"
    try:
        with cf.ProcessPoolExecutor(max_workers=len(pts), mp_context=mp.get_context("spawn")) as ex:
            list(ex.map(_oracle_point_worker, [(workload, e_idx, j, 1) for j in pts]))   # warm
            t0 = time.time()
            times = list(ex.map(_oracle_point_worker, [(workload, e_idx, j, n_iter) for j in pts]))
            wall = time.time() - t0
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    per_iter_point = float(np.median(times)) / n_iter          # seconds, one core
    point_iters = iters.max(axis=1)                            # [n_int]
    # the energy's n_int points spread over `cores` workers, each point to its own count
    seconds = per_iter_point * float(point_iters.sum()) / len(pts)
    return {"value": 1.0 / seconds, "unit": UNIT, "cores": len(pts), "kind": "oracle",
            "sample": (f"{workload}: oracle BiCG, {n_iter} iterations at each of {len(pts)} "
                       f"quadrature points in parallel ({wall:.1f} s wall), scaled by the stored "
                       f"oracle run's per-point iteration counts at energy index {e_idx} "
                       f"(sum {int(point_iters.sum())} over {n_int} points) to one energy's "
                       f"solves over {len(pts)} cores; extraction not included; the cheapest "
                       f"energy of the range"),
            "seconds_per_energy": seconds}


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle, timed as cpu_baseline_sample does, one sample per
    step."""
    if rank != 0:
        return
    vals, last = [], None
    for k in range(args.warmup + args.steps):
        r = cpu_baseline_sample(args.workload)
        if "error" in r:
            print(json.dumps({"impl": "reference", "unavailable": r["error"]}), flush=True)
            return
        if k >= args.warmup:
            vals.append(r["seconds_per_energy"])
            last = r
    per_energy = sum(vals) / len(vals)
    value = 1.0 / per_energy
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_energy * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "sample": "timed oracle BiCG iterations, scaled per energy"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                         "sample": last["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--energy-index", default="",
                    help="comma-separated energy indices of one step (default per workload)")
    ap.add_argument("--form", default=DEFAULT_FORM, choices=sorted(FORMS), help="headline form")
    ap.add_argument("--compare", default=",".join(DEFAULT_COMPARE),
                    help="forms timed once beside the headline on the same step ('' = none)")
    ap.add_argument("--second-workload", default=SECOND_WORKLOAD,
                    help="a second workload measured once per form in the same run ('' = none)")
    ap.add_argument("--second-energy-index", default=",".join(map(str, SECOND_ENERGIES)))
    ap.add_argument("--second-forms", default=",".join(SECOND_FORMS))
    ap.add_argument("--stop-fraction", type=float, default=1.0,
                    help="load-balance rule of the paper (0.5 = stop once over half the points converged)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--spmm", action="store_true",
                    help="only time the operator apply (stencil + projector SpMM) and exit")
    ap.add_argument("--spmm-systems", type=int, default=0,
                    help="systems per SpMM launch (default: the seed batch of a family, 2 N_int)")
    ap.add_argument("--spmm-dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--shapes", default="",
                    help="launch shapes 'py,pz:py,pz,x2' (complex128 : complex64) instead of the "
                         "autotuner (profiling runs)")
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
    hbm, hbm_src = _peaks()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(x):
        if world > 1:
            t = torch.tensor([x], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            return float(t.item())
        return x

    class Job:
        """One workload on this GPU: its Hamiltonian, right-hand sides on the device, the
        energies of one step, and the stencil launch shapes tuned for it."""

        def __init__(self, name, spec):
            self.wl = synth.workload(name)
            self.idx = step_energy_indices(self.wl, spec)
            self.energies = self.wl.energies[self.idx]
            self.n_e = len(self.energies)
            self.H = cbs.Hamiltonian(self.wl.grid, self.wl.vloc, self.wl.projectors)
            self.Vd = torch.from_numpy(self.wl.V).to(dev).contiguous()
            n_tune = 2 * self.wl.n_int
            if args.shapes:
                a, b = args.shapes.split(":")
                a, b = [int(v) for v in a.split(",")], [int(v) for v in b.split(",")]
                cbs.set_apply_shape(self.H, torch.complex128, a[0], a[1])
                cbs.set_apply_shape(self.H, torch.complex64, b[0], b[1], b[2])
                self.tune = {"c128": {"py": a[0], "pz": a[1], "x2": 0, "ms": None},
                             "c64": {"py": b[0], "pz": b[1], "x2": b[2], "ms": None}}
            else:
                self.tune = {"c128": cbs.autotune_apply(self.H, n_tune, self.wl.L, torch.complex128),
                             "c64": cbs.autotune_apply(self.H, n_tune, self.wl.L, torch.complex64)}

        def describe(self):
            wl = self.wl
            return (f"{wl.name}: {wl.grid.nx}x{wl.grid.ny}x{wl.grid.nz} cell, FD{wl.grid.fd_order}, "
                    f"{wl.projectors.n_atoms if wl.projectors else 0} atoms x 4 projectors, "
                    f"{self.n_e} of its {len(wl.energies)} energies per step (indices {self.idx}), "
                    f"N_int={wl.n_int}, L={wl.L}, M={wl.M}, lambda_min={wl.lambda_min}, "
                    f"BiCG tol {wl.tol:g}")

        def options(self, form, profile=True):
            f = FORMS[form]
            return cbs.options(precision=f["precision"], multi_shift=f["multi_shift"], tol=self.wl.tol,
                               delta=self.wl.delta, profile=1 if profile else 0,
                               stop_fraction=f.get("stop_fraction", args.stop_fraction))

        def one_step(self, form):
            wl = self.wl
            return cbs.solve(self.H, self.energies, wl.lambda_min, wl.n_int, wl.L, wl.M, self.Vd,
                             self.options(form))

        def timed(self, form, steps, warmup):
            for _ in range(warmup):
                self.one_step(form)
            barrier()
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0 = cbs.kernel_launches()
            results = []
            with ClockSampler(local) as clk:
                ev0.record()
                for _ in range(steps):
                    results.append(self.one_step(form))
                ev1.record()
                torch.cuda.synchronize()
            launches = cbs.kernel_launches() - l0
            barrier()
            ms = max_over_ranks(ev0.elapsed_time(ev1))
            return ms, results, clk.summary(), launches

        def spmm(self, n_sys, dtype_name, iters=20):
            """Operator apply alone, at the seed batch shape of a family (the 2 N_int primal and
            dual systems), timed with CUDA events on torch's current stream (the stream the
            kernels are launched on)."""
            wl = self.wl
            dt = torch.complex64 if dtype_name == "c64" else torch.complex128
            s = 8 if dtype_name == "c64" else 16
            rng = np.random.default_rng(3)
            zs = (np.exp(1j * rng.uniform(0, 2 * np.pi, n_sys)) *
                  np.where(np.arange(n_sys) % 2 == 0, 1 / wl.lambda_min, wl.lambda_min))
            plan = cbs.ApplyPlan(self.H, zs, 0.1, wl.L, dt)
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
            bpo = apply_bytes_per_output(wl, s)
            r = {"workload": wl.name, "dtype": dtype_name, "systems": n_sys, "columns": wl.L,
                 "ms_per_launch": ms, "bytes_per_launch": bpo * outputs,
                 "GB_s": bpo * outputs / (ms / 1e3) / 1e9, "peak_GB_s": hbm, "peak_source": hbm_src,
                 "frac": bpo * outputs / (ms / 1e3) / 1e9 / hbm,
                 "TFLOP_s": apply_flops_per_output(wl) * outputs / (ms / 1e3) / 1e12,
                 "note": "gather (projector coefficients) + stencil launch pair"}
            del X, Yo, plan
            torch.cuda.empty_cache()
            return r

        def rooflines(self, results, ms_total, form):
            """Per kernel class, from the CUDA events the library records around every launch
            of it inside the BiCG graphs during the timed steps: device time, units processed,
            algorithmic bytes (or flops) per unit, achieved rate against the peak."""
            wl = self.wl
            out = {}
            for key, name in (("c64", "k_proj_gather_c64x2 + k_apply_c64x2: complex64 stencil + projector apply"),
                              ("c128", "k_proj_gather + k_apply_zm<double>: complex128 stencil + projector apply"),
                              ("shift_update", "k_ms_update: shifted-family direction and solution update")):
                p = {f: sum(r.profile[key][f] for r in results) for f in ("ms", "launches", "outputs")}
                if not p["ms"]:
                    continue
                launches = max(p["launches"], 1)
                sec = p["ms"] / 1e3
                rl = {"kernel": name, "units": p["outputs"], "launches": p["launches"],
                      "avg_launch_ms": p["ms"] / launches, "share_of_step": p["ms"] / ms_total}
                c64_family = FORMS[form]["precision"] == "fp32_refine"
                if key == "c64":
                    bpu = apply_bytes_per_output(wl, 8)
                    ach = p["outputs"] * bpu / sec / 1e9
                    rl.update(bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm,
                              peak_source=hbm_src, bytes_per_unit=bpu, unit_of_work="complex output",
                              traffic=_traffic("c64_apply", wl.name, p["outputs"] / launches))
                elif key == "c128":
                    fpu = apply_flops_per_output(wl)
                    ach = p["outputs"] * fpu / sec / 1e12
                    rl.update(bound="alu", achieved=ach, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
                              frac=ach / FP64_PEAK_TFLOPS, flops_per_unit=fpu, unit_of_work="complex output",
                              peak_source="nominal FP64 (152 SMs x 2.07 GHz x 4 FLOP/clk)",
                              traffic=_traffic("c128_apply", wl.name, p["outputs"] / launches))
                elif c64_family:
                    # per (energy, point, column) triple and grid point: scaled direction and
                    # solution read and written, primal and dual, complex64 (8 x 8 B)
                    bpu = 64
                    ach = p["outputs"] * bpu / sec / 1e9
                    rl.update(bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm,
                              peak_source=hbm_src, bytes_per_unit=bpu,
                              unit_of_work="(energy, point, column) triple x grid point",
                              traffic=_traffic("c64_shift_update", wl.name, p["outputs"] / launches))
                else:
                    # FP64 family: 16 FP64 FMAs per unit, bound by the FP64 pipe
                    ach = p["outputs"] * 32 / sec / 1e12
                    rl.update(bound="alu", achieved=ach, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
                              frac=ach / FP64_PEAK_TFLOPS, flops_per_unit=32, traffic=None,
                              unit_of_work="(energy, point, column) triple x grid point",
                              peak_source="nominal FP64 (152 SMs x 2.07 GHz x 4 FLOP/clk)",
                              hbm_GB_s=p["outputs"] * 128 / sec / 1e9)
                out[key] = rl
            return out

    def summary(results):
        last = results[-1]
        kept = [len(e["lam"]) for e in last.energies]
        worst = max([float(np.max(e["residual"])) for e in last.energies if len(e["residual"])] or [0.0])
        return last, kept, worst, sorted({e["flags"] for e in last.energies})

    def lam_agreement(a, b):
        """Largest relative distance from each eigenvalue of result a to its nearest partner
        in result b, over the energies where both keep the same count."""
        worst = 0.0
        for ea, eb in zip(a.energies, b.energies):
            if len(ea["lam"]) != len(eb["lam"]) or not len(ea["lam"]):
                continue
            d = np.abs(ea["lam"][:, None] - eb["lam"][None, :]).min(axis=1) / np.abs(ea["lam"])
            worst = max(worst, float(d.max()))
        return worst

    def once(job, form, ref=None, ref_value=None):
        """One untimed-warm-up-free step of a form, with what 'equal residual' needs: kept
        counts, largest residual, eigenvalue agreement with a reference result."""
        msc, resc, clkc, lc = job.timed(form, 1, 0)
        lastc, keptc, worstc, flagsc = summary(resc)
        out = {"value": job.n_e * world / (msc / 1e3), "unit": UNIT, "ms_per_step": msc, "steps": 1,
               "warmup": 0, "dtype": FORMS[form]["dtype"], "kept_per_energy": keptc,
               "max_residual": worstc, "flags": flagsc,
               "max_solve_residual": max(e["max_solve_residual"] for e in lastc.energies),
               "rooflines": job.rooflines(resc, msc, form), "clocks": clkc, "gpu_launches": lc,
               "stage_ms": {"solve": lastc.ms_solve, "moments": lastc.ms_moments, "extract": lastc.ms_extract}}
        if ref is not None:
            out["same_count_as_reference"] = keptc == [len(e["lam"]) for e in ref.energies]
            out["max_rel_lambda_diff_to_reference"] = lam_agreement(lastc, ref)
        if ref_value:
            out["value_over_reference_form"] = out["value"] / ref_value
        return out, lastc

    job = Job(args.workload, args.energy_index)
    wl, energies, n_e, idx = job.wl, job.energies, job.n_e, job.idx
    if args.spmm:
        r = job.spmm(args.spmm_systems or 2 * wl.n_int, args.spmm_dtype)
        if rank == 0:
            print(json.dumps({"spmm": r, "workload": args.workload, "apply_shape": job.tune}), flush=True)
        return

    headline = args.form
    ms, results, clocks, launches = job.timed(headline, args.steps, args.warmup)
    value = args.steps * n_e * world / (ms / 1e3)
    last, kept, worst_res, flags = summary(results)
    rl = job.rooflines(results, ms, headline)
    ranked = sorted(rl.values(), key=lambda r: -r["share_of_step"])
    roofline = ranked[0] if ranked else None
    roofline_second = ranked[1] if len(ranked) > 1 else None

    compare = {}
    for form in [f for f in args.compare.split(",") if f and f != headline]:
        compare[form], _ = once(job, form, last, value)
        compare[form]["headline_over_this"] = value / compare[form]["value"]

    # the same measurement on a second workload, once per form (the first form is the
    # reference for eigenvalue agreement)
    second = None
    if args.second_workload:
        job2 = Job(args.second_workload, args.second_energy_index)
        second = {"workload": job2.describe(), "energies": [float(x) for x in job2.energies], "forms": {}}
        ref2 = ref2_value = None
        for form in [f for f in args.second_forms.split(",") if f]:
            second["forms"][form], res2 = once(job2, form, ref2, ref2_value)
            if ref2 is None:
                ref2, ref2_value = res2, second["forms"][form]["value"]
        second["spmm"] = {"c64": job2.spmm(2 * job2.wl.n_int, "c64"),
                          "c128": job2.spmm(2 * job2.wl.n_int, "c128", iters=3)}
        del job2
        torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers: Hamiltonian upload, V upload,
    # solve, results (eigenvalues, k, residuals, eigenvectors) back to the host
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Hh = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
        cbs.set_apply_shape(Hh, torch.complex128, job.tune["c128"]["py"], job.tune["c128"]["pz"])
        cbs.set_apply_shape(Hh, torch.complex64, job.tune["c64"]["py"], job.tune["c64"]["pz"],
                            job.tune["c64"]["x2"])
        r_e2e = cbs.solve(Hh, energies, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                          job.options(headline, False))
        Hh.close()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0)
        h2d = wl.vloc.nbytes + wl.V.nbytes
        if wl.projectors is not None:
            P = wl.projectors
            h2d += P.sup_ptr.nbytes + P.sup_idx.nbytes + P.sup_wrap.nbytes + P.sup_val.nbytes + P.h.nbytes
        d2h = sum(e["lam"].nbytes + e["k"].nbytes + e["residual"].nbytes + e["vectors"].nbytes
                  for e in r_e2e.energies)
        e2e = {"value": n_e * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": 1,
               "same_count_as_headline": [len(e["lam"]) for e in r_e2e.energies] == kept}

    spmm_res = {"c64": job.spmm(2 * wl.n_int, "c64"), "c128": job.spmm(2 * wl.n_int, "c128", iters=3)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline_sample(args.workload)
        except Exception as ex:  # noqa: BLE001
            cpu = {"error": str(ex)[-300:]}

    if rank == 0:
        f = FORMS[headline]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": f["dtype"], "data": "synthetic",
            "config": {"workload": job.describe(), "form": headline, "solver": FORMS[headline],
                       "energies": [float(x) for x in energies], "energies_per_step": n_e,
                       "stop_fraction": args.stop_fraction,
                       "l2": "state per step >> L2 (no flush needed)",
                       "kept_per_energy": kept, "max_residual": worst_res, "flags": flags,
                       "max_solve_residual": max(e["max_solve_residual"] for e in last.energies),
                       "apply_shape": job.tune},
            "e2e": e2e, "gpu_launches": launches, "clocks": clocks, "roofline": roofline,
            "roofline_second_kernel": roofline_second, "cpu_baseline": cpu, "compare": compare,
            "second_workload": second, "spmm": spmm_res,
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

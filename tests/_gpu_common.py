"""Helpers shared by the GPU parity tests (the oracle is the reference)."""
import os

import numpy as np
import pytest

from paper_1709_09347_gb300 import synth


def ensure_built():
    from paper_1709_09347_gb300 import build, cbs
    if not os.path.exists(cbs.LIB_PATH):
        build.build()
    return cbs.load()


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    return torch


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def small_cases():
    """Tiny cells spanning several thread-block tiles with ragged tails, odd sizes,
    every supported FD half-width that fits, with and without projectors."""
    return [
        synth.tiny_workload(nx=6, ny=5, nz=4, h=0.45, fd_order=4, n_atoms=2, r_c=0.8, sigma=0.3, L=8),
        synth.tiny_workload(nx=7, ny=4, nz=5, h=0.4, fd_order=8, n_atoms=3, r_c=0.75, sigma=0.3, L=5),
        synth.tiny_workload(nx=9, ny=11, nz=4, h=0.5, fd_order=2, n_atoms=0, projectors=False, L=3),
        synth.tiny_workload(nx=3, ny=4, nz=2, h=0.5, fd_order=4, n_atoms=1, r_c=0.45, sigma=0.2, L=1),
        synth.tiny_workload(nx=13, ny=10, nz=6, h=0.4, fd_order=12, n_atoms=4, r_c=1.1, sigma=0.4, L=33),
    ]

"""Objective and adjoint gradient through cbs_objective against the oracle's dense gradient."""
import numpy as np
import pytest

from oracle.adjoint import objective_and_gradient
from paper_1709_09347_gb300 import synth
from tests._gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_objective_gradient_vs_dense(precision):
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.tiny_workload(nx=6, ny=5, nz=4, h=0.45, fd_order=4, n_atoms=2, r_c=0.8, sigma=0.3,
                             L=4, M=4, n_int=8)
    E = 0.15
    Jr, gVr, gEr = objective_and_gradient(wl.grid, wl.vloc, wl.projectors, E, wl.lambda_min,
                                          wl.n_int, wl.M, wl.V)
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    o = cbs.options(tol=1e-12, precision=precision)
    J, gV, gE = cbs.objective(H, E, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V, o, grad=True)
    assert abs(J - Jr) <= 1e-9 * abs(Jr)
    assert np.max(np.abs(gV - gVr)) <= 1e-8 * np.max(np.abs(gVr))
    assert abs(gE - gEr) <= 1e-8 * max(abs(gEr), np.max(np.abs(gVr)))
    J0 = cbs.objective(H, E, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V, o)
    assert abs(J0 - J) <= 1e-10 * abs(J)


def test_autograd_backward():
    torch = need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.tiny_workload(nx=6, ny=5, nz=4, h=0.45, fd_order=4, n_atoms=2, r_c=0.8, sigma=0.3,
                             L=4, M=4, n_int=8)
    v = torch.tensor(wl.vloc, dtype=torch.float64, device="cuda", requires_grad=True)
    e = torch.tensor(0.15, dtype=torch.float64, device="cuda", requires_grad=True)
    J = cbs.ring_objective(v, e, wl.grid, wl.projectors, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                           cbs.options(tol=1e-12))
    (3.0 * J).backward()
    Jr, gVr, gEr = objective_and_gradient(wl.grid, wl.vloc, wl.projectors, 0.15, wl.lambda_min,
                                          wl.n_int, wl.M, wl.V)
    assert np.max(np.abs(v.grad.cpu().numpy() - 3.0 * gVr)) <= 1e-8 * np.max(np.abs(3.0 * gVr))
    assert abs(e.grad.item() - 3.0 * gEr) <= 1e-8 * max(abs(3.0 * gEr), 1.0)

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


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_gradient_directional_fd_c2(precision):
    """On the 32x32x16 cell (16,384 points, 40 atoms with projectors): the adjoint gradient
    contracted with a random direction of V_loc, and dJ/dE, against central finite
    differences of J itself (steps 1e-4 in V_loc, 1e-5 Ha in E)."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.workload("c2")
    E = float(wl.energies[12])
    L, M, n_int = 8, 4, 16
    V = np.ascontiguousarray(wl.V[:, :L])
    o = cbs.options(tol=1e-12, precision=precision)
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    J, gV, gE = cbs.objective(H, E, wl.lambda_min, n_int, L, M, V, o, grad=True)
    rng = np.random.default_rng(4)
    d = rng.standard_normal(wl.grid.n)
    h = 1e-4
    Jp = cbs.objective(cbs.Hamiltonian(wl.grid, wl.vloc + h * d, wl.projectors), E, wl.lambda_min, n_int, L, M, V, o)
    Jm = cbs.objective(cbs.Hamiltonian(wl.grid, wl.vloc - h * d, wl.projectors), E, wl.lambda_min, n_int, L, M, V, o)
    fd = (Jp - Jm) / (2 * h)
    assert abs(float(np.dot(gV, d)) - fd) <= 1e-5 * max(abs(fd), 1e-12 * abs(J))
    hE = 1e-5
    JEp = cbs.objective(H, E + hE, wl.lambda_min, n_int, L, M, V, o)
    JEm = cbs.objective(H, E - hE, wl.lambda_min, n_int, L, M, V, o)
    fdE = (JEp - JEm) / (2 * hE)
    assert abs(gE - fdE) <= 1e-5 * max(abs(fdE), 1e-12 * abs(J))

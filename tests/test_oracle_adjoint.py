"""Pin for the oracle's objective gradient: central finite differences of J."""
import numpy as np

from oracle.adjoint import objective, objective_and_gradient
from paper_1709_09347_gb300 import synth


def test_gradient_vs_finite_differences():
    wl = synth.tiny_workload(nx=4, ny=3, nz=3, h=0.45, fd_order=4, n_atoms=2, r_c=0.6, sigma=0.25,
                             L=3, M=4, n_int=8)
    E = 0.15
    args = (wl.grid, wl.vloc, wl.projectors)
    J, gV, gE = objective_and_gradient(*args, E, wl.lambda_min, wl.n_int, wl.M, wl.V)
    h = 1e-6
    for i in (0, 7, 19, wl.grid.n - 1):
        vp, vm = wl.vloc.copy(), wl.vloc.copy()
        vp[i] += h
        vm[i] -= h
        fd = (objective(wl.grid, vp, wl.projectors, E, wl.lambda_min, wl.n_int, wl.M, wl.V)
              - objective(wl.grid, vm, wl.projectors, E, wl.lambda_min, wl.n_int, wl.M, wl.V)) / (2 * h)
        assert abs(fd - gV[i]) <= 1e-6 * max(1.0, abs(gV[i]), abs(J))
    fdE = (objective(*args, E + h, wl.lambda_min, wl.n_int, wl.M, wl.V)
           - objective(*args, E - h, wl.lambda_min, wl.n_int, wl.M, wl.V)) / (2 * h)
    assert abs(fdE - gE) <= 1e-6 * max(1.0, abs(gE), abs(J))
    assert np.isfinite(J) and J != 0

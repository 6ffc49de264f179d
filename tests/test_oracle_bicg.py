"""Pins for the oracle's BiCG (paper §3.2: primal Eq. (9) and dual Eq. (11) systems)."""
import numpy as np
import scipy.sparse.linalg as spla

from oracle.bicg import bicg
from oracle.contour import ring_contour
from oracle.operator import CellOperator
from paper_1709_09347_gb300 import synth


def test_bicg_primal_dual_vs_direct():
    wl = synth.tiny_workload(nx=5, ny=4, nz=4, h=0.45, fd_order=4, n_atoms=2, r_c=0.8, sigma=0.3, L=4)
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    E = 0.2
    z1, _, z2, _ = ring_contour(0.5, 8)
    for z in z1[:3]:
        X, Xt, it, info = bicg(lambda X: op.apply_P(z, E, X), lambda X: op.apply_P_adjoint(z, E, X),
                               wl.V, wl.V, tol=1e-13, max_iter=5000)
        assert info["converged"].all()
        Pz = op.P_matrix(z, E)
        Xd = spla.spsolve(Pz, wl.V)
        Xtd = spla.spsolve(Pz.conj().T.tocsc(), wl.V)
        assert np.linalg.norm(X - Xd) / np.linalg.norm(Xd) < 1e-9
        assert np.linalg.norm(Xt - Xtd) / np.linalg.norm(Xtd) < 1e-9
        # the dual solution solves the inner-circle system P(1/conj z) Y = V (§3.2)
        Pz2 = op.P_matrix(1 / np.conj(z), E)
        assert np.linalg.norm(Pz2 @ Xt - wl.V) / np.linalg.norm(wl.V) < 1e-10
        # true residual
        assert np.linalg.norm(Pz @ X - wl.V) / np.linalg.norm(wl.V) < 1e-11

"""Pins for the oracle's eigenpair refinement (residual inverse iteration on Eq. (4))."""
import numpy as np

from oracle import polish
from oracle.dense import dense_qep, in_ring
from oracle.operator import CellOperator
from paper_1709_09347_gb300 import synth


def _ring_pairs(op, E, lmin):
    w, v = dense_qep(op, E, vectors=True)
    sel = in_ring(w, lmin, shrink=0.05)
    return w[sel], v[:, sel]


def test_polish_recovers_dense_eigenvalues_with_projectors():
    """Eigenpairs of a tiny cell with projectors, perturbed by 1e-6 (lambda) and 1e-3
    (vector), converge back to the dense linearisation's eigenvalues."""
    wl = synth.tiny_workload(nx=6, ny=5, nz=4, h=0.45, fd_order=4, n_atoms=2, r_c=0.8,
                             sigma=0.3, L=4, M=4)
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    E = 6.0                              # propagating and evanescent pairs in the ring
    lam, X = _ring_pairs(op, E, 0.3)
    assert len(lam) >= 12 and np.any(np.abs(np.abs(lam) - 1) > 0.5)
    rng = np.random.default_rng(5)
    lam0 = lam * (1 + 1e-6 * (rng.standard_normal(len(lam)) + 1j * rng.standard_normal(len(lam))))
    X0 = X + 1e-3 * np.linalg.norm(X, axis=0) * (rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape)) / np.sqrt(X.shape[0])
    lp, Xp, res = polish.polish(op, E, lam0, X0)
    assert np.max(np.abs(lp - lam) / np.abs(lam)) < 1e-12
    assert np.all(res < 1e-13)
    # each polished vector is the dense eigenvector up to a scalar
    for i in range(len(lam)):
        x = X[:, i] / np.linalg.norm(X[:, i])
        c = np.vdot(x, Xp[:, i])
        assert np.linalg.norm(Xp[:, i] - c * x) < 1e-9


def test_polish_free_electron_closed_form():
    """8x8x4 free-electron cell (4th-order FD): the QEP eigenvalues are t^nz with t a root
    of the 1D dispersion of each transverse mode, in closed form; polishing starts 1e-7 off
    and lands on them."""
    wl = synth.workload("c1")
    g = wl.grid
    op = CellOperator(g, np.zeros(g.n), None)
    E = float(wl.energies[0])
    c = np.array([-5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0])
    exact = []
    for nx in range(g.nx):
        for ny in range(g.ny):
            eperp = sum(-0.5 / (h * h) * (c[0] + 2 * sum(c[k] * np.cos(2 * np.pi * k * n / N) for k in (1, 2)))
                        for n, N, h in ((nx, g.nx, g.hx), (ny, g.ny, g.hy)))
            # -(1/2h^2)(c0 + c1 (t + 1/t) + c2 (t^2 + 1/t^2)) = E - eperp, times t^2
            a = -0.5 / (g.hz * g.hz)
            poly = [a * c[2], a * c[1], a * c[0] - (E - eperp), a * c[1], a * c[2]]
            for t in np.roots(poly):
                exact.append(t ** g.nz)
    exact = np.array(exact)
    lam, X = _ring_pairs(op, E, wl.lambda_min)
    lam0 = lam * (1 + 1e-7)
    lp, _, res = polish.polish(op, E, lam0, X)
    for l in lp:
        assert np.min(np.abs(exact - l)) / abs(l) < 1e-12
    assert np.all(res < 1e-13)

"""The shifted-family reading (one BiCG Krylov sequence for P(z, E0) + s I, all shifts s):
the recurrences the device kernels implement, restated in numpy on a small non-Hermitian
matrix, reproduce the solutions of every shifted system and of its dual (the conjugate
transpose), checked against direct solves.  Not in the paper; this pins the formulas:

    pi^{k+1} = (1 + alpha_k s) pi^k + gamma_k (pi^k - pi^{k-1}),  gamma_k = alpha_k b_{k-1} / alpha_{k-1}
    p^ = r + (pi^{k-1} / pi^k) b_{k-1} p^,   x += (alpha_k / pi^{k+1}) p^     (p^ = pi^k p_s)
    dual: the same with conjugated coefficients.
"""
import numpy as np


def _family(A, b, shifts, tol=1e-13, max_iter=400):
    r = b.copy(); rt = b.copy()
    p = np.zeros_like(b); pt = np.zeros_like(b)
    beta, rho, a_prev = 0.0, np.vdot(rt, r), 1.0
    ns = len(shifts)
    pi = np.ones(ns, complex); pim = np.ones(ns, complex)
    X = np.zeros((ns, len(b)), complex); Xt = np.zeros_like(X)
    P = np.zeros_like(X); Pt = np.zeros_like(X)
    for _ in range(max_iter):
        p = r + beta * p
        pt = rt + np.conj(beta) * pt
        q = A @ p
        qt = A.conj().T @ pt
        alpha = rho / np.vdot(pt, q)
        g = 0.0 if beta == 0 else alpha * beta / a_prev
        for e, s in enumerate(shifts):
            pn = (1 + alpha * s) * pi[e] + g * (pi[e] - pim[e])
            cb = 0.0 if beta == 0 else (pim[e] / pi[e]) * beta
            ca = alpha / pn
            P[e] = r + cb * P[e]; X[e] += ca * P[e]
            Pt[e] = rt + np.conj(cb) * Pt[e]; Xt[e] += np.conj(ca) * Pt[e]
            pim[e], pi[e] = pi[e], pn
        a_prev = alpha
        r = r - alpha * q
        rt = rt - np.conj(alpha) * qt
        rn = np.vdot(rt, r)
        beta, rho = rn / rho, rn
        worst = max(np.linalg.norm(r), np.linalg.norm(rt)) / np.min(np.abs(pi))
        if worst <= tol * np.linalg.norm(b):
            break
    return X, Xt


def test_family_matches_direct_solves():
    rng = np.random.default_rng(3)
    n = 80
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 9 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    shifts = np.array([0.0, -0.5, -1.3, 0.8, 2.0])
    X, Xt = _family(A, b, shifts)
    for e, s in enumerate(shifts):
        As = A + s * np.eye(n)
        assert np.linalg.norm(X[e] - np.linalg.solve(As, b)) <= 1e-10 * np.linalg.norm(X[e])
        assert np.linalg.norm(Xt[e] - np.linalg.solve(As.conj().T, b)) <= 1e-10 * np.linalg.norm(Xt[e])


def test_family_with_the_cell_operator():
    """Same on the oracle's P(z, E) of a tiny cell: shifts are energy differences."""
    import scipy.sparse.linalg as spla

    from oracle.operator import CellOperator
    from paper_1709_09347_gb300 import synth
    wl = synth.tiny_workload(nx=6, ny=5, nz=4, h=0.45, fd_order=4, n_atoms=1, r_c=0.8, sigma=0.3,
                             L=1, M=2, n_int=8, energies=(0.2,))
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    z = 2.0 * np.exp(0.7j)
    E0 = 0.3
    energies = np.array([0.3, 0.1, -0.2])
    A = op.P_matrix(z, E0).toarray()
    b = wl.V[:, 0]
    X, Xt = _family(A, b, energies - E0, tol=1e-13, max_iter=2000)
    for e, E in enumerate(energies):
        PE = op.P_matrix(z, E).tocsc()
        x = spla.spsolve(PE, b)
        xt = spla.spsolve(PE.conj().T.tocsc(), b)
        assert np.linalg.norm(X[e] - x) <= 1e-9 * np.linalg.norm(x)
        assert np.linalg.norm(Xt[e] - xt) <= 1e-9 * np.linalg.norm(xt)

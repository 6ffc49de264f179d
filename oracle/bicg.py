"""BiCG for the primal systems P(z) Y = V and their duals P(z)^dagger Y~ = V (oracle).

Paper §3.2: because P(lambda)^dagger = P(1/conj(lambda)) and z_j^(2) = 1/conj(z_j^(1)),
the inner-circle systems Eq. (10) are the dual systems Eq. (11) of the outer-circle
systems Eq. (9), and BiCG solves a system together with its dual at about the cost of
one.  Every right-hand-side column is an independent BiCG run (§3.3, top layer).

Textbook BiCG with the inner product (a, b) = a^dagger b, x_0 = x~_0 = 0, r_0 = b,
r~_0 = b~:

    q = A p, q~ = A^dagger p~,  alpha = (r~, r) / (p~, q)
    x += alpha p,  r -= alpha q,  x~ += conj(alpha) p~,  r~ -= conj(alpha) q~
    beta = (r~', r') / (r~, r),  p = r' + beta p,  p~ = r~' + conj(beta) p~

Stop a column when ||r||/||b|| <= tol and ||r~||/||b~|| <= tol (§3.3's standard
criterion).  Columns are stored side by side; scalars are per column.

Pins (tests/test_oracle_bicg.py): solutions against a sparse direct solve of P(z) and
of P(z)^dagger; the true residual ||V - P(z)Y||/||V|| <= tol-level.
"""
from __future__ import annotations

import numpy as np


def bicg(apply_A, apply_AH, B, Bt=None, tol=1e-10, max_iter=20000, history=False):
    """Solve A X = B and A^dagger Xt = Bt column by column.

    Returns (X, Xt, iters, info): iters is the per-column iteration count at which the
    column converged (or max_iter), info a dict with 'converged' (bool per column) and
    optionally the residual history.
    """
    B = np.asarray(B, dtype=complex)
    if B.ndim == 1:
        B = B[:, None]
    Bt = B if Bt is None else np.asarray(Bt, dtype=complex).reshape(B.shape)
    n, L = B.shape
    X = np.zeros_like(B)
    Xt = np.zeros_like(B)
    R = B.copy()
    Rt = Bt.copy()
    P = R.copy()
    Pt = Rt.copy()
    nb = np.linalg.norm(B, axis=0)
    nbt = np.linalg.norm(Bt, axis=0)
    nb[nb == 0] = 1.0
    nbt[nbt == 0] = 1.0
    rho = np.sum(np.conj(Rt) * R, axis=0)
    active = np.ones(L, dtype=bool)
    iters = np.zeros(L, dtype=int)
    hist = []
    for it in range(1, max_iter + 1):
        if not active.any():
            break
        a = np.nonzero(active)[0]
        Q = apply_A(P[:, a])
        Qt = apply_AH(Pt[:, a])
        gamma = np.sum(np.conj(Pt[:, a]) * Q, axis=0)
        alpha = rho[a] / gamma
        X[:, a] += alpha * P[:, a]
        R[:, a] -= alpha * Q
        Xt[:, a] += np.conj(alpha) * Pt[:, a]
        Rt[:, a] -= np.conj(alpha) * Qt
        rho_new = np.sum(np.conj(Rt[:, a]) * R[:, a], axis=0)
        rel = np.linalg.norm(R[:, a], axis=0) / nb[a]
        relt = np.linalg.norm(Rt[:, a], axis=0) / nbt[a]
        if history:
            hist.append((it, a.copy(), rel.copy(), relt.copy()))
        beta = rho_new / rho[a]
        rho[a] = rho_new
        P[:, a] = R[:, a] + beta * P[:, a]
        Pt[:, a] = Rt[:, a] + np.conj(beta) * Pt[:, a]
        iters[a] = it
        done = (rel <= tol) & (relt <= tol)
        active[a[done]] = False
    info = {"converged": ~active}
    if history:
        info["history"] = hist
    return X, Xt, iters, info

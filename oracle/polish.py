"""Per-eigenvalue refinement of QEP eigenpairs by residual inverse iteration (oracle).

Test infrastructure only (see the package header): it produces reference eigenvalues
accurate to rounding, against which the method's approximations (Algorithm 1 at a finite
BiCG tolerance and a finite quadrature) can be judged at the 1e-10 level.

The QEP of Eq. (4), multiplied by -lambda, is Q(lambda) x = 0 with
Q(lambda) = lambda^2 H+ + lambda (H0 - E) + H-.  Starting from an approximate pair
(lambda_0, x_0) and a fixed shift sigma = lambda_0, residual inverse iteration
(Neumaier, SIAM J. Numer. Anal. 22 (1985) 914) repeats

    lambda_{k+1}:  the root nearest lambda_k of  w^H Q(lambda) x_k = 0,
                   with w = Q(sigma)^{-H} v  (a scalar quadratic in lambda),
    x_{k+1} = x_k - Q(sigma)^{-1} Q(lambda_{k+1}) x_k,   normalised so that v^H x = 1,

with v = x_0 / ||x_0||^2.  It converges linearly with a factor proportional to
|sigma - lambda_*|, so from an eigenvalue already correct to ~1e-9 two or three steps
reach rounding level.  Q(sigma) is factorised once per eigenvalue with dense LU
(LAPACK getrf through scipy), which bounds this to cells of a few ten thousand points; the
blocks stay sparse for the products.

Pins (tests/test_oracle_polish.py): perturbed eigenpairs of tiny cells converge back to
the dense linearisation's eigenvalues; on the free-electron 8x8x4 cell to the
closed-form FD dispersion.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def qep_blocks(op, E):
    """(A2, A1, A0) = (H+, H0 - E, H-) as sparse matrices."""
    import scipy.sparse as sp
    H0, Hp, Hm = op.explicit()
    A1 = (H0 - E * sp.identity(H0.shape[0], format="csr")).tocsr()
    return Hp.tocsr(), A1, Hm.tocsr()


def polish_pair(blocks, lam0, x0, steps=4):
    """Residual inverse iteration from (lam0, x0); returns (lambda, x, history) where x
    has unit 2-norm and history lists |lambda_{k+1} - lambda_k|."""
    A2, A1, A0 = blocks
    sigma = complex(lam0)
    Qs = (sigma * sigma * A2 + sigma * A1 + A0).toarray()    # dense for the LU only
    lu = sla.lu_factor(Qs, overwrite_a=True, check_finite=False)
    x = np.asarray(x0, complex).copy()
    v = x / np.vdot(x, x)
    x = x / np.vdot(v, x)
    w = sla.lu_solve(lu, v, trans=2, check_finite=False)       # Q(sigma)^H w = v
    lam = sigma
    hist = []
    for _ in range(steps):
        a2 = np.vdot(w, A2 @ x)
        a1 = np.vdot(w, A1 @ x)
        a0 = np.vdot(w, A0 @ x)
        roots = np.roots([a2, a1, a0]) if abs(a2) > 0 else np.array([-a0 / a1])
        new = complex(roots[np.argmin(np.abs(roots - lam))])
        hist.append(abs(new - lam))
        lam = new
        r = lam * lam * (A2 @ x) + lam * (A1 @ x) + A0 @ x
        x = x - sla.lu_solve(lu, r, check_finite=False)
        x = x / np.vdot(v, x)
    return lam, x / np.linalg.norm(x), hist


def polish(op, E, lam, X, steps=4):
    """Refine every pair (lam[i], X[:, i]); returns (lam_polished, X_polished, residual)
    with residual = ||Q(lambda) x|| / (|lambda|^2 ||H+||_F + |lambda| ||H0-E||_F + ||H-||_F)
    for unit x."""
    blocks = qep_blocks(op, E)
    A2, A1, A0 = blocks
    nHp, nA, nHm = op.frobenius(E)
    out_l = np.zeros(len(lam), complex)
    out_x = np.zeros(X.shape, complex)
    res = np.zeros(len(lam))
    for i in range(len(lam)):
        l, x, _ = polish_pair(blocks, lam[i], X[:, i], steps)
        out_l[i], out_x[:, i] = l, x
        q = l * l * (A2 @ x) + l * (A1 @ x) + A0 @ x
        res[i] = np.linalg.norm(q) / (abs(l) ** 2 * nHp + abs(l) * nA + nHm)
    return out_l, out_x, res

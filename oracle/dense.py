"""Brute-force QEP solution by companion linearisation (oracle, tiny cells only).

The QEP of Eq. (4), multiplied by -lambda, is (lambda^2 Hp + lambda (H0 - E) + Hm) x = 0.
With w = [x; lambda x] it is the 2N x 2N generalised eigenproblem

    [[0, I], [-Hm, -(H0 - E)]] w = lambda [[I, 0], [0, Hp]] w,

solved densely with LAPACK (scipy.linalg.eig).  Hp and Hm are singular (only the
planes near the cell faces couple), so infinite and zero eigenvalues appear; the finite
non-zero ones are the QEP's.  This plays the role of the dense transfer-matrix
reference the paper compares against (§4.1: solutions inside the ring correspond to
the OBM ones).

Pins (tests/test_oracle_dense.py): closed-form FD free-electron dispersion; real-k
bands (eig of the Hermitian H(e^{ika})) reappear as |lambda| = 1 solutions.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def dense_qep(op, E, vectors=False, zero_tol=1e-12, inf_tol=1e12):
    H0, Hp, Hm = (M.toarray() for M in op.explicit())
    N = H0.shape[0]
    I = np.eye(N)
    Z = np.zeros((N, N))
    A = np.block([[Z, I], [-Hm, -(H0 - E * I)]])
    B = np.block([[I, Z], [Z, Hp]])
    if vectors:
        w, v = sla.eig(A, B)
    else:
        w = sla.eig(A, B, right=False)
        v = None
    ok = np.isfinite(w) & (np.abs(w) > zero_tol) & (np.abs(w) < inf_tol)
    if vectors:
        return w[ok], v[:N, ok]
    return w[ok]


def in_ring(lam, lambda_min, shrink=0.0):
    r = np.abs(lam)
    lo = lambda_min * (1.0 + shrink)
    return (r > lo) & (r < 1.0 / lo)


def match(found, ref, rel_tol):
    """Greedy nearest matching.  Returns (max relative error, unmatched_found, unmatched_ref)."""
    found = list(found)
    ref = list(ref)
    worst = 0.0
    un_f = []
    for f in sorted(found, key=lambda x: (abs(x), np.angle(x))):
        if not ref:
            un_f.append(f)
            continue
        d = [abs(f - r) / max(abs(r), 1e-300) for r in ref]
        i = int(np.argmin(d))
        if d[i] <= rel_tol:
            worst = max(worst, d[i])
            ref.pop(i)
        else:
            un_f.append(f)
    return worst, un_f, ref

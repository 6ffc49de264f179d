"""Sakurai-Sugiura extraction for the QEP, residual check, filter and k (oracle).

Algorithm 1 of the paper (§3.1), with the two-circle contour of §3.2:

  1. Step 1 (Eq. (8)-(11)): Y_j^(1) = P(z_j^(1))^{-1} V and, as the BiCG dual,
     Y_j^(2) = P(z_j^(1))^{-dagger} V = P(z_j^(2))^{-1} V.
  2. Moments (Eq. (7) on the ring, §3.2):
        S_k = sum_j w_j^(1) (z_j^(1))^k Y_j^(1) - sum_j w_j^(2) (z_j^(2))^k Y_j^(2),
        mu_k = V^dagger S_k,  k = 0 .. 2 N_mm - 1.
  3. Block Hankel T = [mu_{i+j-2}], T^< = [mu_{i+j-1}] (1 <= i, j <= N_mm); SVD
     T = U Sigma W^dagger and rank cut keeping sigma_i >= delta * sigma_1 (the reading of
     the threshold used here: relative to the largest singular value).
  4. tau, phi from U_1^dagger T^< W_1 Sigma_1^{-1} phi = tau phi; lambda = tau,
     psi = S W_1 Sigma_1^{-1} phi with S = [S_0, ..., S_{N_mm-1}].

Then every eigenpair is checked with the residual of the QEP written as
Q(lambda) = lambda^2 Hp + lambda (H0 - E) + Hm (= -lambda P(lambda)):

    rho = ||Q(lambda) x|| / (||x|| (|lambda|^2 ||Hp||_F + |lambda| ||H0 - E||_F + ||Hm||_F)),

kept if lambda_min < |lambda| < 1/lambda_min (Eq. (5)) and rho <= rho_max, normalised to
||psi|| = 1 with its largest-modulus entry real positive, sorted by |lambda| then
arg(lambda), and k = -i ln(lambda) / a = (arg(lambda) - i ln|lambda|) / a (§2, Eq. (3)).

A Rayleigh-Ritz variant (not in the paper) projects the three blocks onto an
orthonormal basis of span(S W_1) (the part of the moment space the Hankel rank cut
keeps) and solves the small QEP by companion linearisation.

Pins (tests/test_oracle_ss.py): moments of a diagonal QEP against the residue sum;
the in-ring eigenvalues of tiny cells against the dense linearisation and against the
closed-form FD free-electron dispersion; lambda -> 1/conj(lambda) pairing.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from .bicg import bicg
from .contour import ring_contour


@dataclasses.dataclass
class SSResult:
    lam: np.ndarray          # kept eigenvalues
    k: np.ndarray            # complex wave numbers
    residual: np.ndarray     # rho per kept pair
    vectors: np.ndarray      # N x count, normalised
    rank: int                # numerical rank m_hat
    sigma: np.ndarray        # singular values of T (or of S for RR)
    lam_all: np.ndarray      # every extracted eigenvalue before filtering
    res_all: np.ndarray
    iters: np.ndarray        # BiCG iterations, [n_int, L]
    mu: np.ndarray | None = None
    S: np.ndarray | None = None


def _solve_point(args):
    op, z, E, V, tol, max_iter = args
    X, Xt, it, info = bicg(lambda X: op.apply_P(z, E, X), lambda X: op.apply_P_adjoint(z, E, X),
                           V, V, tol=tol, max_iter=max_iter)
    return X, Xt, it


def solve_ring(op, E, lambda_min, n_int, V, tol=1e-10, max_iter=20000, pool=None):
    """Step 1: primal and dual BiCG at the outer-circle points.  Returns Y1, Y2, iters.
    The points are independent (§3.3, middle layer); `pool` (an executor with .map) may
    solve them in parallel."""
    z1, _, z2, _ = ring_contour(lambda_min, n_int)
    N, L = V.shape
    Y1 = np.zeros((n_int, N, L), complex)
    Y2 = np.zeros((n_int, N, L), complex)
    iters = np.zeros((n_int, L), int)
    jobs = [(op, z1[j], E, V, tol, max_iter) for j in range(n_int)]
    results = pool.map(_solve_point, jobs) if pool is not None else map(_solve_point, jobs)
    for j, (X, Xt, it) in enumerate(results):
        Y1[j], Y2[j], iters[j] = X, Xt, it
    return Y1, Y2, iters


def moments(Y1, Y2, lambda_min, n_int, V, M):
    """S_k for k < 2M and mu_k = V^dagger S_k (Algorithm 1, step 1, ring contour)."""
    z1, w1, z2, w2 = ring_contour(lambda_min, n_int)
    N, L = V.shape
    S = np.zeros((2 * M, N, L), complex)
    for k in range(2 * M):
        for j in range(n_int):
            S[k] += w1[j] * z1[j] ** k * Y1[j] - w2[j] * z2[j] ** k * Y2[j]
    mu = np.einsum("nl,knm->klm", np.conj(V), S)
    return S, mu


def hankel_extract(S, mu, M, delta):
    """Algorithm 1, Hankel extraction (SVD of T, rank cut, reduced eigenproblem, vectors):
    returns (lam, psi, rank, sigma)."""
    L = mu.shape[1]
    T = np.zeros((L * M, L * M), complex)
    Tl = np.zeros((L * M, L * M), complex)
    for i in range(M):
        for j in range(M):
            T[i * L:(i + 1) * L, j * L:(j + 1) * L] = mu[i + j]
            Tl[i * L:(i + 1) * L, j * L:(j + 1) * L] = mu[i + j + 1]
    U, sig, Wh = np.linalg.svd(T)
    m_hat = int(np.sum(sig >= delta * sig[0])) if sig[0] > 0 else 0
    U1 = U[:, :m_hat]
    W1 = Wh[:m_hat].conj().T
    Bm = U1.conj().T @ Tl @ W1 / sig[:m_hat][None, :]
    tau, phi = np.linalg.eig(Bm)
    Shat = np.concatenate([S[k] for k in range(M)], axis=1)         # N x LM
    psi = Shat @ (W1 / sig[:m_hat][None, :]) @ phi
    return tau, psi, m_hat, sig


def apply_blocks(op, X):
    """(H0 X, Hp X, Hm X) from the definitions (kinetic + local explicit, non-local
    sum_m B_m h B_{m-l}^T X)."""
    out = []
    for l in (0, 1, -1):
        Y = op.K[l] @ X
        if op.Hblk is not None:
            for mm in (-1, 0, 1):
                if mm in op.B and (mm - l) in op.B:
                    Y = Y + op.B[mm] @ (op.Hblk @ (op.B[mm - l].T @ X))
        out.append(Y)
    return tuple(out)


def residuals(op, E, lam, X, norms):
    """rho for each column x_i of X with eigenvalue lam_i."""
    nHp, nA, nHm = norms
    H0X, HpX, HmX = apply_blocks(op, X)
    Q = lam[None, :] ** 2 * HpX + lam[None, :] * (H0X - E * X) + HmX
    num = np.linalg.norm(Q, axis=0)
    den = np.linalg.norm(X, axis=0) * (np.abs(lam) ** 2 * nHp + np.abs(lam) * nA + nHm)
    return num / den


def normalise(X):
    X = X / np.linalg.norm(X, axis=0)[None, :]
    piv = np.argmax(np.abs(X), axis=0)
    ph = X[piv, np.arange(X.shape[1])]
    return X * (np.conj(ph) / np.abs(ph))[None, :]


def filter_sort(lam, X, res, lambda_min, a, rho_max):
    ok = np.isfinite(lam) & (np.abs(lam) > lambda_min) & (np.abs(lam) < 1.0 / lambda_min) \
        & (res <= rho_max)
    lam, X, res = lam[ok], X[:, ok], res[ok]
    order = np.lexsort((np.angle(lam), np.abs(lam)))
    lam, X, res = lam[order], X[:, order], res[order]
    k = (np.angle(lam) - 1j * np.log(np.abs(lam))) / a
    return lam, k, res, normalise(X) if X.shape[1] else X


def ss_hankel(op, E, lambda_min, n_int, V, M, delta=1e-10, tol=1e-10, rho_max=1e-8,
              max_iter=20000, keep_moments=False, pool=None):
    """Whole SS-Hankel pipeline for one energy."""
    Y1, Y2, iters = solve_ring(op, E, lambda_min, n_int, V, tol=tol, max_iter=max_iter, pool=pool)
    S, mu = moments(Y1, Y2, lambda_min, n_int, V, M)
    tau, psi, m_hat, sig = hankel_extract(S, mu, M, delta)
    norms = op.frobenius(E)
    res_all = residuals(op, E, tau, psi, norms) if m_hat else np.zeros(0)
    lam, k, res, X = filter_sort(tau, psi, res_all, lambda_min, op.grid.a, rho_max)
    return SSResult(lam, k, res, X, m_hat, sig, tau, res_all, iters,
                    mu if keep_moments else None, S[:M] if keep_moments else None)


def rr_basis(S, mu, M, delta, basis_cut=1e-7):
    """Orthonormal basis of span(S W_1): W_1 are the right singular vectors of the block
    Hankel matrix T kept by the delta cut of Algorithm 1; columns of S W_1 whose
    singular values fall below basis_cut * the largest are dropped."""
    L = mu.shape[1]
    T = np.zeros((L * M, L * M), complex)
    for i in range(M):
        for j in range(M):
            T[i * L:(i + 1) * L, j * L:(j + 1) * L] = mu[i + j]
    _, sig, Wh = np.linalg.svd(T)
    m_hat = int(np.sum(sig >= delta * sig[0])) if sig[0] > 0 else 0
    Shat = np.concatenate([S[k] for k in range(M)], axis=1)
    Z = Shat @ Wh[:m_hat].conj().T
    Uz, sz, _ = np.linalg.svd(Z, full_matrices=False)
    r = int(np.sum(sz >= basis_cut * sz[0])) if len(sz) and sz[0] > 0 else 0
    return Uz[:, :r], m_hat, sig


def ss_rayleigh_ritz(op, E, lambda_min, n_int, V, M, delta=1e-10, tol=1e-10, rho_max=1e-8,
                     max_iter=20000, S=None, mu=None):
    """Rayleigh-Ritz variant (not in the paper): the QEP's three blocks projected onto the
    basis of rr_basis, the small QEP lambda^2 A2 + lambda A1 + A0 solved by companion
    linearisation, Ritz vectors x = Q u filtered like the Hankel pairs."""
    iters = np.zeros((n_int, V.shape[1]), int)
    if S is None:
        Y1, Y2, iters = solve_ring(op, E, lambda_min, n_int, V, tol=tol, max_iter=max_iter)
        S, mu = moments(Y1, Y2, lambda_min, n_int, V, M)
    Qb, m_hat, sig = rr_basis(S, mu, M, delta)
    r = Qb.shape[1]
    H0Q, HpQ, HmQ = apply_blocks(op, Qb)
    A2 = Qb.conj().T @ HpQ
    A1 = Qb.conj().T @ (H0Q - E * Qb)
    A0 = Qb.conj().T @ HmQ
    I = np.eye(r)
    Z = np.zeros((r, r))
    Amat = np.block([[Z, I], [-A0, -A1]])
    Bmat = np.block([[I, Z], [Z, A2]])
    w, v = sla.eig(Amat, Bmat)
    fin = np.isfinite(w) & (np.abs(w) > 0)
    w, v = w[fin], v[:r, fin]
    X = Qb @ v
    norms = op.frobenius(E)
    res_all = residuals(op, E, w, X, norms)
    lam, k, res, Xn = filter_sort(w, X, res_all, lambda_min, op.grid.a, rho_max)
    return SSResult(lam, k, res, Xn, r, sig, w, res_all, iters)

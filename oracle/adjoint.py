"""Objective and reverse-mode gradient of the ring solves (oracle, tiny cells).

Not in the paper (an addition of this project): a scalar objective of the solutions of the
shifted systems of §3.2 (Eq. (9)-(11)), and its gradient with respect to the local
potential V_loc and the energy E.  The objective is the |Y|^2-weighted moment trace

    J = sum_{c=1,2} sum_j c_j^(c) ||Y_j^(c)||_F^2,
    c_j^(c) = Re( s_c w_j^(c) sum_{k<M} (z_j^(c))^k ),  s_1 = +1, s_2 = -1,

with Y_j^(c) = P(z_j^(c))^{-1} V, P(z) = E - H(z) (Eq. (4)).  Since dP = dE I - diag(dV_loc),
dY = -P^{-1} dP Y and, with G = P^{-dagger} Y (one adjoint solve per system),

    dJ/dV_loc[i] = sum_{c,j} 2 c_j^(c) Re sum_col conj(G[i,col]) Y[i,col],
    dJ/dE        = -sum_{c,j} 2 c_j^(c) Re tr(G^dagger Y).

Here every system is solved densely (LU), so this is the exact gradient of the discrete
objective.  Pin (tests/test_oracle_adjoint.py): central finite differences of J.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .contour import ring_contour
from .operator import CellOperator


def weights(lambda_min, n_int, M):
    """(c1, c2): the real objective weights of the outer and inner circle points."""
    z1, w1, z2, w2 = ring_contour(lambda_min, n_int)
    k = np.arange(M)
    c1 = np.real(w1 * np.sum(z1[:, None] ** k[None, :], axis=1))
    c2 = -np.real(w2 * np.sum(z2[:, None] ** k[None, :], axis=1))
    return c1, c2


def objective_and_gradient(grid, vloc, projectors, E, lambda_min, n_int, M, V):
    """Dense J, dJ/dV_loc (length N) and dJ/dE."""
    op = CellOperator(grid, vloc, projectors)
    z1, _, z2, _ = ring_contour(lambda_min, n_int)
    c1, c2 = weights(lambda_min, n_int, M)
    J = 0.0
    gV = np.zeros(op.n)
    gE = 0.0
    for zs, cs in ((z1, c1), (z2, c2)):
        for z, c in zip(zs, cs):
            P = op.P_matrix(z, E).toarray()
            lu = sla.lu_factor(P)
            Y = sla.lu_solve(lu, V)
            G = sla.lu_solve(lu, Y, trans=2)          # P^dagger G = Y
            J += c * np.sum(np.abs(Y) ** 2)
            gV += 2 * c * np.real(np.sum(np.conj(G) * Y, axis=1))
            gE += -2 * c * np.real(np.sum(np.conj(G) * Y))
    return J, gV, gE


def objective(grid, vloc, projectors, E, lambda_min, n_int, M, V):
    return objective_and_gradient(grid, vloc, projectors, E, lambda_min, n_int, M, V)[0]

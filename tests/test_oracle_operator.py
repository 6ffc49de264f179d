"""Pins for the oracle's cell Hamiltonian blocks (paper §2, Eq. (2)-(4))."""
from fractions import Fraction
from math import factorial

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.operator import CellOperator
from paper_1709_09347_gb300 import synth


def tiny(**kw):
    base = dict(nx=4, ny=3, nz=3, h=0.45, fd_order=4, n_atoms=2, r_c=0.6, sigma=0.25, L=3)
    base.update(kw)
    return synth.tiny_workload(**base)


def test_hermitian_structure():
    wl = tiny()
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    H0, Hp, Hm = op.explicit()
    assert abs(H0 - H0.T).max() < 1e-14                     # H_{n,n} symmetric
    assert abs(Hm - Hp.T).max() < 1e-14                     # H_{n-1,n} = H_{n,n+1}^T
    assert Hp.nnz > 0


def _fd_closed(order):
    m = order // 2
    ck = [float(Fraction(2 * (-1) ** (k + 1) * factorial(m) ** 2,
                         k * k * factorial(m - k) * factorial(m + k))) for k in range(1, m + 1)]
    return [-2 * sum(ck)] + ck


def _periodic_1d(n, h, c):
    T = np.zeros((n, n))
    for i in range(n):
        T[i, i] += c[0]
        for k in range(1, len(c)):
            T[i, (i + k) % n] += c[k]
            T[i, (i - k) % n] += c[k]
    return -0.5 * T / h ** 2


@pytest.mark.parametrize("n_rep", [2, 3])
def test_supercell_spectrum(n_rep):
    """An n_rep-cell periodic supercell, built independently as one periodic grid with
    every atom copy placed explicitly, has the spectrum of the union over Bloch phases
    z = exp(2 pi i q / n_rep) of H(z) = H0 + z Hp + Hm / z."""
    wl = tiny()
    g = wl.grid
    op = CellOperator(g, wl.vloc, wl.projectors)
    H0, Hp, Hm = (M.toarray() for M in op.explicit())
    bloch = []
    for q in range(n_rep):
        z = np.exp(2j * np.pi * q / n_rep)
        Hz = H0 + z * Hp + Hm / z
        assert np.allclose(Hz, Hz.conj().T, atol=1e-13)
        bloch.append(np.linalg.eigvalsh(Hz))
    bloch = np.sort(np.concatenate(bloch))

    c = _fd_closed(g.fd_order)
    NZ = n_rep * g.nz
    Ix, Iy, Iz = np.eye(g.nx), np.eye(g.ny), np.eye(NZ)
    Hs = (np.kron(Iz, np.kron(Iy, _periodic_1d(g.nx, g.hx, c)))
          + np.kron(Iz, np.kron(_periodic_1d(g.ny, g.hy, c), Ix))
          + np.kron(_periodic_1d(NZ, g.hz, c), np.kron(Iy, Ix)))
    Hs += np.diag(np.tile(wl.vloc, n_rep))
    P = wl.projectors
    ncell = g.nx * g.ny
    for a in range(P.n_atoms):
        s0, s1 = P.sup_ptr[a], P.sup_ptr[a + 1]
        idx, wrap, val = P.sup_idx[s0:s1], P.sup_wrap[s0:s1], P.sup_val[s0:s1]
        ixy = idx % ncell
        iz = idx // ncell
        for cc in range(n_rep):
            # the copy of atom a sitting in supercell cell cc covers, for a point of the
            # table with wrap m, the point iz in cell (cc - m)
            zsc = iz + ((cc - wrap.astype(int)) % n_rep) * g.nz
            beta = np.zeros((ncell * NZ, P.n_proj))
            beta[ixy + ncell * zsc] = val
            Hs += beta @ P.h[a] @ beta.T
    sc = np.sort(np.linalg.eigvalsh(Hs))
    assert np.max(np.abs(sc - bloch)) < 1e-10


def test_matrix_free_matches_explicit():
    wl = tiny(nx=5, ny=4, nz=4)
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    H0, Hp, Hm = op.explicit()
    rng = np.random.default_rng(3)
    X = rng.standard_normal((op.n, 3)) + 1j * rng.standard_normal((op.n, 3))
    for z in (1.7 * np.exp(0.3j), 0.4 * np.exp(-2.1j), np.exp(1.1j)):
        ref = H0 @ X + z * (Hp @ X) + (Hm @ X) / z
        assert np.allclose(op.apply_H(z, X), ref, rtol=0, atol=1e-12)
        E = 0.37
        Pz = op.P_matrix(z, E)
        assert np.allclose(op.apply_P(z, E, X), Pz @ X, atol=1e-12)
        # dagger from transposes == explicit conjugate transpose == P(1/conj z) (§3.2)
        adj = op.apply_P_adjoint(z, E, X)
        assert np.allclose(adj, Pz.conj().T @ X, atol=1e-12)
        assert np.allclose(adj, op.apply_P(1.0 / np.conj(z), E, X), atol=1e-12)


def test_frobenius():
    wl = tiny()
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    H0, Hp, Hm = (M.toarray() for M in op.explicit())
    E = -0.2
    f = op.frobenius(E)
    assert np.allclose(f, [np.linalg.norm(Hp), np.linalg.norm(H0 - E * np.eye(op.n)),
                           np.linalg.norm(Hm)], rtol=1e-13)

"""Cell Hamiltonian blocks and the QEP matrix P(z) (oracle).

Paper §2, Eq. (2): inside cell n the Kohn-Sham equation couples only to cells n-1 and
n+1, through H_{n,n-1} and H_{n,n+1}; in bulk H_{n-1,n} = H_{n,n+1}^dagger.  With the
Bloch ansatz of Eq. (3), psi_{n+l} = lambda^l psi_n, this gives Eq. (4):

    P(lambda) = -lambda^{-1} H_{n,n-1} + (E - H_{n,n}) - lambda H_{n,n+1}.

Notation here: H0 = H_{n,n}, Hp = H_{n,n+1}, Hm = H_{n,n-1}, so that
P(z) = E*I - H0 - z*Hp - Hm/z.

The real-space Hamiltonian is -1/2 * Laplacian (central FD, periodic in x and y) +
diag(V_loc) + separable non-local projectors.  Blocks are assembled directly from the
definitions:

* kinetic: a neighbour of plane iz at offset d along z lands in plane iz+d; if that
  plane is >= nz it belongs to the next cell (block Hp, plane iz+d-nz), if < 0 to the
  previous cell (block Hm, plane iz+d+nz);
* non-local: sum over atoms a and all their periodic copies along z of
  beta_{a,n} h_a beta_{a,n}^T.  Restricted to cell 0 this is
      block l  =  sum_a sum_m  B_{a,m} h_a B_{a,m-l}^T,
  where B_{a,m} holds the values of the copy of atom a displaced by m cells (the
  table's wrap tag).  Kept factored as sparse B_m (N x n_atoms*n_proj) matrices; the
  explicit blocks are formed only for small cells and for Frobenius norms.

Pins (tests/test_oracle_operator.py): H0 = H0^T and Hm = Hp^T (§2: H_{n-1,n} =
H_{n,n+1}^dagger); the spectrum of an n_rep-cell periodic supercell, assembled
independently as one periodic grid, equals the union over q of eig H(e^{2 pi i q/n_rep});
the FD free-electron dispersion in closed form (via the dense linearisation);
matrix-free apply equals the explicit blocks.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fd import fd_weights_float


class CellOperator:
    """H0, Hp, Hm of one unit cell; kinetic + local explicit, non-local factored."""

    def __init__(self, grid, vloc, projectors=None):
        self.grid = grid
        g = grid
        self.n = g.nx * g.ny * g.nz
        m = g.fd_order // 2
        if m > g.nz:
            raise ValueError("FD half-width must not exceed nz (nearest-cell coupling only)")
        c = fd_weights_float(g.fd_order)
        self.fd = c
        N = self.n
        idx = np.arange(N)
        ix = idx % g.nx
        iy = (idx // g.nx) % g.ny
        iz = idx // (g.nx * g.ny)
        rows = {0: [], 1: [], -1: []}
        cols = {0: [], 1: [], -1: []}
        vals = {0: [], 1: [], -1: []}

        def add(block, r, cidx, v):
            rows[block].append(r)
            cols[block].append(cidx)
            vals[block].append(np.broadcast_to(v, r.shape).astype(float))

        diag = -0.5 * c[0] * (1.0 / g.hx ** 2 + 1.0 / g.hy ** 2 + 1.0 / g.hz ** 2)
        add(0, idx, idx, diag + np.asarray(vloc, float))
        for k in range(1, m + 1):
            for sgn in (+1, -1):
                wx = -0.5 * c[k] / g.hx ** 2
                jx = (ix + sgn * k) % g.nx
                add(0, idx, jx + g.nx * (iy + g.ny * iz), wx)
                wy = -0.5 * c[k] / g.hy ** 2
                jy = (iy + sgn * k) % g.ny
                add(0, idx, ix + g.nx * (jy + g.ny * iz), wy)
                wz = -0.5 * c[k] / g.hz ** 2
                pz = iz + sgn * k
                block = np.floor_divide(pz, g.nz)          # -1, 0 or +1 (m <= nz)
                jz = pz - block * g.nz
                col = ix + g.nx * (iy + g.ny * jz)
                for b in (-1, 0, 1):
                    sel = block == b
                    if np.any(sel):
                        add(b, idx[sel], col[sel], wz)
        self.K = {}
        self.BT = {}
        for b in (-1, 0, 1):
            if rows[b]:
                r = np.concatenate(rows[b])
                cc = np.concatenate(cols[b])
                v = np.concatenate(vals[b])
                self.K[b] = sp.csr_matrix((v, (r, cc)), shape=(N, N))
            else:
                self.K[b] = sp.csr_matrix((N, N))
        self.vloc = np.asarray(vloc, float)
        # non-local: B_m[i, a*n_proj + mu] = value of projector mu of atom copy m at i
        self.proj = projectors
        self.B = {}
        if projectors is not None and projectors.n_atoms > 0:
            P = projectors
            npj = P.n_proj
            atom_of = np.repeat(np.arange(P.n_atoms), np.diff(P.sup_ptr))
            for mm in (-1, 0, 1):
                sel = np.nonzero(P.sup_wrap == mm)[0]
                r = np.repeat(P.sup_idx[sel].astype(np.int64), npj)
                cc = (atom_of[sel][:, None] * npj + np.arange(npj)[None, :]).ravel()
                v = P.sup_val[sel].ravel()
                self.B[mm] = sp.csr_matrix((v, (r, cc)), shape=(N, P.n_atoms * npj))
            self.Hblk = sp.block_diag([sp.csr_matrix(P.h[a]) for a in range(P.n_atoms)], format="csr")
            self.BT = {mm: B.T.tocsr() for mm, B in self.B.items()}
        else:
            self.Hblk = None

    # ---- blocks ---------------------------------------------------------------
    def nonlocal_block(self, l: int):
        """Explicit sum_m B_m h B_{m-l}^T (sparse)."""
        N = self.n
        out = sp.csr_matrix((N, N))
        if self.Hblk is None:
            return out
        for mm in (-1, 0, 1):
            mt = mm - l
            if mt in self.B:
                out = out + self.B[mm] @ self.Hblk @ self.B[mt].T
        return out.tocsr()

    def explicit(self):
        """(H0, Hp, Hm) as explicit sparse matrices."""
        H0 = (self.K[0] + self.nonlocal_block(0)).tocsr()
        Hp = (self.K[1] + self.nonlocal_block(1)).tocsr()
        Hm = (self.K[-1] + self.nonlocal_block(-1)).tocsr()
        return H0, Hp, Hm

    # ---- matrix-free application --------------------------------------------
    def apply_H(self, z, X):
        """H(z) X = H0 X + z Hp X + z^{-1} Hm X  (twisted-periodic cell Hamiltonian)."""
        Y = self.K[0] @ X + z * (self.K[1] @ X) + (1.0 / z) * (self.K[-1] @ X)
        if self.Hblk is not None:
            # sum_l z^l sum_m B_m h B_{m-l}^T = F(z) h F(1/z)^T with F(w) = sum_m w^m B_m,
            # applied term by term: c = sum_m z^{-m} B_m^T X, Y += sum_m z^m B_m (h c)
            c = sum((z ** (-mm)) * (self.BT[mm] @ X) for mm in self.B)
            d = self.Hblk @ c
            Y = Y + sum((z ** mm) * (self.B[mm] @ d) for mm in self.B)
        return Y

    def apply_P(self, z, E, X):
        """P(z) X = E X - H(z) X  (Eq. (4) with lambda -> z)."""
        return E * X - self.apply_H(z, X)

    def apply_P_adjoint(self, z, E, X):
        """P(z)^dagger X = conj(E) X - H(z)^dagger X, with H(z)^dagger written out from the
        transposed real blocks: H0^T + conj(z) Hp^T + conj(1/z) Hm^T, and the non-local
        part (F(z) h F(1/z)^T)^dagger = F(1/conj z) h^T F(conj z)^T.  Computed from the
        transposes rather than from the identity P(z)^dagger = P(1/conj z) of §3.2, so
        that tests can check that identity."""
        zc = np.conj(z)
        if not hasattr(self, "KT"):
            self.KT = {b: K.T.tocsr() for b, K in self.K.items()}
        Y = self.KT[0] @ X + zc * (self.KT[1] @ X) + np.conj(1.0 / z) * (self.KT[-1] @ X)
        if self.Hblk is not None:
            c = sum((zc ** mm) * (self.BT[mm] @ X) for mm in self.B)
            d = self.Hblk.T @ c
            Y = Y + sum((np.conj(1.0 / z) ** mm) * (self.B[mm] @ d) for mm in self.B)
        return np.conj(E) * X - Y

    def P_matrix(self, z, E):
        H0, Hp, Hm = self.explicit()
        return (E * sp.identity(self.n, format="csr") - H0 - z * Hp - (1.0 / z) * Hm).tocsc()

    # ---- norms ------------------------------------------------------------------
    def frobenius(self, E):
        """(||Hp||_F, ||H0 - E||_F, ||Hm||_F) from the explicit blocks."""
        H0, Hp, Hm = self.explicit()
        A = (H0 - E * sp.identity(self.n, format="csr")).tocsr()
        f = lambda M: float(np.sqrt(np.sum(np.asarray(M.data) ** 2))) if M.nnz else 0.0
        A.sum_duplicates()
        Hp.sum_duplicates()
        Hm.sum_duplicates()
        return f(Hp), f(A), f(Hm)

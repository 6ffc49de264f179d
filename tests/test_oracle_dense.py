"""Pins for the dense QEP linearisation and the assembled blocks (paper §2, §4.1)."""
import numpy as np
import pytest

from oracle.dense import dense_qep, match
from oracle.operator import CellOperator
from paper_1709_09347_gb300 import synth
from tests.test_oracle_operator import _fd_closed


def free_electron_lambdas(g, E):
    """Closed-form FD free-electron QEP eigenvalues.

    With V = 0 the transverse modes are plane waves with energy
    eps = sum_{x,y} -1/(2h^2) (c0 + 2 sum_k c_k cos(2 pi k n / N)); along z a Bloch wave
    t^{iz} needs -1/(2h^2)(c0 + sum_k c_k (t^k + t^-k)) = E - eps, a degree-2m polynomial
    in t, and the cell phase is lambda = t^{nz}."""
    c = _fd_closed(g.fd_order)
    m = len(c) - 1
    out = []
    for nxm in range(g.nx):
        ex = -0.5 / g.hx ** 2 * (c[0] + 2 * sum(c[k] * np.cos(2 * np.pi * k * nxm / g.nx) for k in range(1, m + 1)))
        for nym in range(g.ny):
            ey = -0.5 / g.hy ** 2 * (c[0] + 2 * sum(c[k] * np.cos(2 * np.pi * k * nym / g.ny) for k in range(1, m + 1)))
            rhs = E - ex - ey
            # t^m * [ -1/(2h^2) (c0 + sum c_k (t^k + t^-k)) - rhs ] = 0
            poly = np.zeros(2 * m + 1)           # coefficient of t^p at index p
            s = -0.5 / g.hz ** 2
            poly[m] += s * c[0] - rhs
            for k in range(1, m + 1):
                poly[m + k] += s * c[k]
                poly[m - k] += s * c[k]
            t = np.roots(poly[::-1])
            out.extend(t ** g.nz)
    return np.array(out)


@pytest.mark.parametrize("E", [0.3, -0.4, 2.0])
def test_free_electron_closed_form(E):
    g = synth.Grid(8, 8, 4, 0.4, 0.4, 0.4, 4)
    op = CellOperator(g, np.zeros(g.n))
    lam = dense_qep(op, E)
    ref = free_electron_lambdas(g, E)
    assert len(lam) == len(ref) == 2 * 2 * g.nx * g.ny          # 2 m nx ny finite eigenvalues
    # compare log|lambda| and arg on the well-conditioned range
    sel = (np.abs(ref) > 1e-3) & (np.abs(ref) < 1e3)
    worst, un_f, un_r = match(lam[(np.abs(lam) > 1e-3) & (np.abs(lam) < 1e3)], ref[sel], 1e-8)
    assert not un_f and not un_r and worst < 1e-8


def test_conventional_bands():
    """Real-k bands (paper §4.1): at E = E_n(k) the QEP has lambda = exp(i k a)."""
    wl = synth.tiny_workload(nx=4, ny=4, nz=3, h=0.45, fd_order=4, n_atoms=2, r_c=0.6, sigma=0.25)
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    H0, Hp, Hm = (M.toarray() for M in op.explicit())
    a = wl.grid.a
    rng = np.random.default_rng(5)
    for ka in rng.uniform(-np.pi, np.pi, 3):
        z = np.exp(1j * ka)
        En = np.linalg.eigvalsh(H0 + z * Hp + Hm / z)
        for n in (0, 3):
            lam = dense_qep(op, En[n])
            d = np.min(np.abs(lam - z))
            assert d < 1e-8


def test_pairing_dense():
    """P(lambda)^dagger = P(1/conj lambda) (§3.2) => spectrum closed under 1/conj."""
    wl = synth.tiny_workload(nx=4, ny=3, nz=3, h=0.45, fd_order=4, n_atoms=2, r_c=0.6, sigma=0.25)
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    lam = dense_qep(op, 0.1)
    lam = lam[(np.abs(lam) > 0.05) & (np.abs(lam) < 20)]
    for l in lam:
        assert np.min(np.abs(lam - 1 / np.conj(l))) / abs(l) < 1e-7
        assert np.min(np.abs(lam - np.conj(l))) / abs(l) < 1e-7

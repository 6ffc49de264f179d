"""Pins for the oracle's SS pipeline (paper §3.1 Algorithm 1, §3.2 ring contour)."""
import numpy as np
import pytest

from oracle.contour import ring_contour
from oracle.dense import dense_qep, in_ring, match
from oracle.operator import CellOperator
from oracle import ss
from paper_1709_09347_gb300 import synth


def test_ring_moments_diagonal_residues():
    """Diagonal QEP: P_i(z) = E - h0_i - z hp_i - hp_i / z = -hp_i (z - r_i)(z - 1/r_i) / z.
    The exact ring moment is the residue sum over poles inside the ring (poles kept at
    least a factor 1.5 from both circles, so the trapezoid error 0.67^64 is negligible):
    S_k[i] = sum_{p in ring} -p^{k+1} / (hp_i (p - p')) V[i]  (p' the partner root)."""
    lmin, n_int, M, E = 0.5, 64, 4, 0.0
    roots = np.array([0.8, 1.25, np.exp(0.7j), 0.2, 5.0, 1.3, np.exp(2.5j), 0.25])
    hp = np.array([1.0, 0.7, 1.3, 0.9, 1.1, 0.6, 1.2, 0.8])
    h0 = E - hp * (roots + 1 / roots)          # real for real or unimodular roots
    assert np.allclose(h0.imag, 0)
    h0 = h0.real
    rng = np.random.default_rng(1)
    V = rng.standard_normal((len(roots), 2)) + 1j * rng.standard_normal((len(roots), 2))
    z1, w1, z2, w2 = ring_contour(lmin, n_int)
    P = lambda z: (E - h0 - z * hp - hp / z)[:, None]
    Y1 = np.stack([V / P(z) for z in z1])
    Y2 = np.stack([V / P(z) for z in z2])
    S, mu = ss.moments(Y1, Y2, lmin, n_int, V, M)
    for k in range(2 * M):
        exact = np.zeros_like(V)
        for i, r in enumerate(roots):
            for p, q in ((r, 1 / r), (1 / r, r)):
                if lmin < abs(p) < 1 / lmin:
                    exact[i] += -p ** (k + 1) / (hp[i] * (p - q)) * V[i]
        assert np.max(np.abs(S[k] - exact)) < 1e-9 * max(1.0, np.max(np.abs(exact)))
    assert np.allclose(mu[2], V.conj().T @ S[2])


def _check_vs_dense(op, E, res, lmin, rel=1e-8):
    lam_d = dense_qep(op, E)
    must = lam_d[in_ring(lam_d, lmin, shrink=0.05)]
    pool = lam_d[in_ring(lam_d, lmin, shrink=-0.02)]
    worst, un_f, _ = match(res.lam, pool, rel)
    assert not un_f, f"SS eigenvalues without a dense partner: {un_f}"
    worst2, _, missed = match(must, res.lam, rel)
    assert not missed, f"dense eigenvalues missed by SS: {missed}"
    return max(worst, worst2)


@pytest.mark.parametrize("free", [True, False])
def test_ss_c1_vs_dense(free):
    wl = synth.workload("c1")
    vloc = np.zeros_like(wl.vloc) if free else wl.vloc
    op = CellOperator(wl.grid, vloc, None)
    E = float(wl.energies[0])
    res = ss.ss_hankel(op, E, wl.lambda_min, wl.n_int, wl.V, wl.M, delta=1e-10, tol=1e-12)
    assert res.rank < wl.L * wl.M
    assert len(res.lam) > 0
    assert np.all(res.residual <= 1e-8)
    worst = _check_vs_dense(op, E, res, wl.lambda_min)
    assert worst < 1e-8
    # pairing lambda <-> 1/conj(lambda) (§3.2) and lambda <-> conj(lambda) (real H)
    for l in res.lam:
        assert np.min(np.abs(res.lam - 1 / np.conj(l))) / abs(l) < 1e-8
        assert np.min(np.abs(res.lam - np.conj(l))) / abs(l) < 1e-8
    # k = -i ln(lambda)/a reproduces lambda
    assert np.allclose(np.exp(1j * res.k * wl.grid.a), res.lam, rtol=1e-12)


def test_ss_tiny_projectors_vs_dense():
    wl = synth.tiny_workload(nx=6, ny=5, nz=4, h=0.45, fd_order=4, n_atoms=2, r_c=0.8,
                             sigma=0.3, L=12, M=8, n_int=32)
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    for E in (0.2, -0.3):
        res = ss.ss_hankel(op, E, wl.lambda_min, wl.n_int, wl.V, wl.M, tol=1e-12)
        assert res.rank < wl.L * wl.M
        assert _check_vs_dense(op, E, res, wl.lambda_min) < 1e-8
        rr = ss.ss_rayleigh_ritz(op, E, wl.lambda_min, wl.n_int, wl.V, wl.M, tol=1e-12)
        assert _check_vs_dense(op, E, rr, wl.lambda_min) < 1e-8
        assert len(rr.lam) == len(res.lam)


def test_normalise_phase_convention():
    """A9: unit 2-norm, largest-modulus entry real and positive, and the column equal to
    the input times a scalar.  Worked by hand: x = (1, 3i, -2) has norm sqrt(14) and its
    largest entry 3i; multiplying by -i/sqrt(14) makes that entry 3/sqrt(14)."""
    X = np.array([[1.0, 2.0 - 2.0j], [3.0j, 0.5], [-2.0, -1.0j]])
    got = ss.normalise(X)
    s = np.sqrt(14.0)
    want0 = np.array([-1.0j, 3.0, 2.0j]) / s
    assert np.allclose(got[:, 0], want0, rtol=0, atol=1e-15)
    # second column: |2-2i| = sqrt(8) is the largest, norm sqrt(8 + 0.25 + 1) = sqrt(9.25);
    # the phase factor is conj(2-2i)/sqrt(8) = (1+i)/sqrt(2)
    n1 = np.sqrt(9.25)
    ph = (1.0 + 1.0j) / np.sqrt(2.0)
    want1 = np.array([2.0 - 2.0j, 0.5, -1.0j]) * ph / n1
    assert np.allclose(got[:, 1], want1, rtol=0, atol=1e-15)
    assert abs(got[0, 1].imag) < 1e-15 and got[0, 1].real > 0
    assert np.allclose(np.linalg.norm(got, axis=0), 1.0, atol=1e-15)


def test_filter_sort_order_ring_and_k():
    """A8/A10: only lambda strictly inside lambda_min < |lambda| < 1/lambda_min with
    rho <= rho_max survive; the order is |lambda| ascending, then arg(lambda) in
    (-pi, pi] ascending; k = (arg lambda - i ln|lambda|)/a.  Expected values written out
    by hand for a = 2 and lambda_min = 0.5."""
    lam = np.array([
        2.0 * np.exp(0.5j),      # |.| = 2: on the outer circle, dropped (strict inequality)
        1.0j,                    # |.| = 1, arg  pi/2
        -1.0 + 0.0j,             # |.| = 1, arg  pi
        1.0 + 0.0j,              # |.| = 1, arg  0
        -1.0j,                   # |.| = 1, arg -pi/2
        0.6 * np.exp(-3.0j),     # |.| = 0.6, arg -3
        0.6 * np.exp(1.0j),      # |.| = 0.6, arg  1, residual too large: dropped
        0.4,                     # inside the inner circle: dropped
        1.5 * np.exp(2.0j),      # |.| = 1.5
        np.nan,                  # not finite: dropped
    ])
    res = np.array([1e-12, 1e-12, 1e-12, 1e-12, 1e-12, 2e-9, 1e-7, 1e-12, 1e-10, 1e-12])
    X = np.eye(len(lam), dtype=complex)
    lam_s, k, res_s, Xs = ss.filter_sort(lam, X, res, 0.5, 2.0, 1e-8)
    want = np.array([0.6 * np.exp(-3.0j), -1.0j, 1.0, 1.0j, -1.0, 1.5 * np.exp(2.0j)])
    assert np.allclose(lam_s, want, rtol=0, atol=1e-15)
    assert np.allclose(res_s, [2e-9, 1e-12, 1e-12, 1e-12, 1e-12, 1e-10])
    want_k = np.array([(-3.0 - 1j * np.log(0.6)) / 2, -np.pi / 4, 0.0, np.pi / 4, np.pi / 2,
                       (2.0 - 1j * np.log(1.5)) / 2])
    assert np.allclose(k, want_k, rtol=0, atol=1e-15)
    # the vectors follow their eigenvalues: unit vector e_i of input index i
    src = [5, 4, 3, 1, 2, 8]
    for col, i in enumerate(src):
        assert abs(Xs[i, col] - 1.0) < 1e-15

"""Shifted solves and the whole method through the C ABI against the oracle."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import ss
from oracle.bicg import bicg
from oracle.contour import ring_contour
from oracle.dense import match
from oracle.operator import CellOperator
from paper_1709_09347_gb300 import synth
from tests._gpu_common import need_gpu, rel_err, small_cases

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
@pytest.mark.parametrize("case", [0, 1, 4])
def test_shifted_solves_vs_direct(precision, case):
    """P(z_j) Y = V and P(z_j)^dagger Y~ = V (Eq. (9), (11)) at ring points, against a
    sparse direct solve of the oracle's explicit P(z)."""
    torch = need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = small_cases()[case]
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    z1, _, _, _ = ring_contour(0.5, 8)
    zs = z1[[0, 3, 5]]
    E = 0.2
    B = torch.from_numpy(wl.V).to("cuda").contiguous()
    o = cbs.options(tol=1e-12, precision=precision)
    Y, Yd, iters, st = cbs.solve_shifted(H, zs, E, B, o)
    Y, Yd = Y.cpu().numpy(), Yd.cpu().numpy()
    for s, z in enumerate(zs):
        Pz = op.P_matrix(z, E)
        ref = spla.spsolve(Pz, wl.V)
        refd = spla.spsolve(Pz.conj().T.tocsc(), wl.V)
        assert rel_err(Y[s], ref) < 1e-9
        assert rel_err(Yd[s], refd) < 1e-9
    assert (iters > 0).all()


def test_shifted_iterations_match_oracle():
    """FP64 BiCG on the device follows the oracle's iteration counts (same algorithm,
    same stopping rule) within a few iterations of rounding drift."""
    torch = need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = small_cases()[0]
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    z = ring_contour(0.5, 16)[0][2]
    E = -0.1
    B = torch.from_numpy(wl.V).to("cuda").contiguous()
    Y, Yd, iters, st = cbs.solve_shifted(H, [z], E, B, cbs.options(tol=1e-10))
    X, Xt, it, info = bicg(lambda X: op.apply_P(z, E, X), lambda X: op.apply_P_adjoint(z, E, X),
                           wl.V, wl.V, tol=1e-10)
    assert np.max(np.abs(iters[0] - it)) <= 3
    assert rel_err(Y[0].cpu().numpy(), X) < 1e-8


def _gpu_solve(wl, energies, precision="fp64", tol=1e-12):
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    o = cbs.options(tol=tol, precision=precision)
    return cbs.solve(H, energies, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V, o)


def _compare(res_gpu, ref, lam_tol):
    assert len(res_gpu["lam"]) == len(ref.lam)
    worst, un_f, un_r = match(res_gpu["lam"], ref.lam, lam_tol)
    assert not un_f and not un_r, (res_gpu["lam"], ref.lam)
    assert worst <= lam_tol
    assert np.all(res_gpu["residual"] <= 1e-8)


@pytest.mark.parametrize("precision,lam_tol", [("fp64", 1e-10), ("fp32_refine", 1e-9)])
def test_solve_c1(precision, lam_tol):
    """Whole method on the 8x8x4 cell: eigenvalue count and values against the oracle
    run of Algorithm 1, moments mu_k against the oracle's."""
    wl = synth.workload("c1")
    E = float(wl.energies[0])
    r = _gpu_solve(wl, [E], precision).energies[0]
    op = CellOperator(wl.grid, wl.vloc, None)
    ref = ss.ss_hankel(op, E, wl.lambda_min, wl.n_int, wl.V, wl.M, tol=1e-12, keep_moments=True)
    _compare(r, ref, lam_tol)
    # the rank cut sigma_i >= delta sigma_1 lands inside the tail of leaked singular
    # values (~1e-10 sigma_1), which carry the solve error: FP64 moves it by at most one
    # index, the mixed form by a few
    assert abs(r["rank"] - ref.rank) <= (1 if precision == "fp64" else 4)
    # moment k carries z^k with |z| up to 1/lambda_min: the BiCG tolerance is amplified by
    # (1/lambda_min)^(k+1) (refinement stops at tol too)
    for k in range(2 * wl.M):
        scale = np.max(np.abs(ref.mu[k]))
        assert np.max(np.abs(r["mu"][k] - ref.mu[k])) <= 100 * 1e-12 * (1 / wl.lambda_min) ** (k + 1) * scale
    # vectors: unit norm, largest entry real positive; residual recomputed by the oracle
    V = r["vectors"]
    assert np.allclose(np.linalg.norm(V, axis=0), 1.0, atol=1e-12)
    norms = op.frobenius(E)
    rr = ss.residuals(op, E, r["lam"], V, norms)
    assert np.all(rr <= 1e-8)
    assert np.allclose(rr, r["residual"], rtol=1e-6, atol=1e-15)
    assert np.allclose(np.exp(1j * r["k"] * wl.grid.a), r["lam"], rtol=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_solve_tiny_projectors(precision):
    wl = synth.tiny_workload(nx=6, ny=5, nz=4, h=0.45, fd_order=4, n_atoms=2, r_c=0.8, sigma=0.3,
                             L=12, M=8, n_int=32, energies=(0.2, -0.3))
    res = _gpu_solve(wl, wl.energies, precision)
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    for e, E in enumerate(wl.energies):
        ref = ss.ss_hankel(op, E, wl.lambda_min, wl.n_int, wl.V, wl.M, tol=1e-12)
        _compare(res.energies[e], ref, 1e-10 if precision == "fp64" else 1e-9)


def _conj_defect(lam):
    """Distance of every eigenvalue to the nearest conjugate of the set.  The blocks of
    Eq. (4) are real here, so the exact spectrum is closed under conjugation and this
    defect measures how far an extraction is from it."""
    lam = np.asarray(lam)
    return np.array([np.min(np.abs(lam - np.conj(x))) for x in lam])


def _c2_golden():
    import os
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "c2_oracle.npz"))
    return g, [int(i) for i in g["energy_index"]]


# The eigenvalue bar of the FP64 form against the stored energies' eigenvalues refined to
# rounding level: 1e-10 relative.  Measured: the Rayleigh-Ritz extraction reaches 3.5e-13 with
# BiCG tol 1e-12; the Hankel extraction of Algorithm 1 is limited by its own approximation to
# 1.5e-10 (per energy) and 3.9e-10 (shifted family) at tol 1e-12 -- the oracle's own run is at
# 2.5e-10 -- and reaches 1.7e-11 at tol 1e-13.
C2_EXACT_TOL = 1e-10


def _check_c2_golden(res, g, idx, lam_tol, wl, rank_mode):
    """rank_mode: 'same_tol' (Hankel rank within 5% of the oracle's, solved to the same tol),
    'bound' (rank >= the number of pairs: the delta cut moves with the solve error), or
    'basis' (Rayleigh-Ritz: the reported rank is the basis size)."""
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    for e, i in enumerate(idx):
        r = res.energies[e]
        ref = g[f"lam_{i}"]                     # the oracle's Algorithm 1 at tol 1e-12
        exact = g[f"lam_polished_{i}"]          # the same eigenvalues refined
        assert len(r["lam"]) == len(ref)
        if int(g[f"rank_{i}"]) == wl.L * wl.M and rank_mode != "basis":
            assert r["rank"] == wl.L * wl.M and r["flags"] & 4   # saturation on both sides
        elif rank_mode == "same_tol":
            assert abs(r["rank"] - int(g[f"rank_{i}"])) <= max(2, int(0.05 * int(g[f"rank_{i}"])))
        else:
            assert r["rank"] >= len(ref)
        if not len(ref):
            continue
        worst, un_f, un_r = match(r["lam"], exact, lam_tol)
        assert not un_f and not un_r and worst <= lam_tol
        E = float(wl.energies[i])
        rr = ss.residuals(op, E, r["lam"], r["vectors"], op.frobenius(E))
        assert np.all(rr <= 1e-8)


@pytest.mark.parametrize("form,tol,lam_tol,rank_mode", [
    (dict(precision="fp64", extraction="rr"), 1e-12, C2_EXACT_TOL, "basis"),
    (dict(precision="fp64", extraction="rr", multi_shift=1), 1e-12, C2_EXACT_TOL, "basis"),
    (dict(precision="fp64"), 1e-13, C2_EXACT_TOL, "bound"),
    (dict(precision="fp64", multi_shift=1), 1e-13, C2_EXACT_TOL, "bound"),
    (dict(precision="fp64"), 1e-12, 5e-10, "same_tol"),
    (dict(precision="fp32_refine"), 1e-12, 1e-8, "bound"),
    (dict(precision="fp32_refine", multi_shift=1), 1e-12, 1e-8, "bound")])
def test_solve_c2_vs_oracle_golden(form, tol, lam_tol, rank_mode):
    """Full 32x32x16 cell (8th-order FD, 40 atoms x 4 projectors) at three stored energies
    (tests/golden/make_c2_oracle.py runs only the CPU oracle; one of them rank-saturated):
    the same eigenvalue count in the ring as the oracle's Algorithm 1, the rank (saturation
    on both sides), every kept pair's residual recomputed with the oracle's operator <= 1e-8,
    the solves' FP64 true residuals, and the eigenvalues against the oracle's eigenvalues
    refined to rounding level: within 1e-10 in the FP64 form (Rayleigh-Ritz at tol 1e-12,
    Algorithm 1's Hankel extraction at tol 1e-13), within 5e-10 for Algorithm 1 at the
    oracle's own tol 1e-12 (its approximation error there, measured 1.5e-10 against the
    oracle's 2.5e-10), and within the residual bar 1e-8 in the mixed forms."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    g, idx = _c2_golden()
    wl = synth.workload("c2")
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    res = cbs.solve(H, wl.energies[idx], wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                    cbs.options(tol=tol, **form), allow=(cbs.CBS_OK, cbs.CBS_WRANK))
    _check_c2_golden(res, g, idx, lam_tol, wl, rank_mode)
    # the shifted family and the mixed forms refine every column to tol on the FP64 true
    # residual; plain per-energy BiCG stops on the recursive one, whose distance to the true
    # residual stays near 1e-12 of the right-hand side here (8.9e-13 measured at tol 1e-13)
    refined = form.get("multi_shift") or form.get("precision") == "fp32_refine"
    for e in res.energies:
        assert e["max_solve_residual"] <= (tol if refined else max(2 * tol, 2e-12))


def test_solve_rr_tiny_projectors():
    """Rayleigh-Ritz extraction (the moments' span S W_1, small QEP by companion
    linearisation) against the oracle's Rayleigh-Ritz on a cell with projectors, and
    against the Hankel pairs of the same run: both extractions find the same eigenvalues."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.tiny_workload(nx=6, ny=5, nz=4, h=0.45, fd_order=4, n_atoms=2, r_c=0.8, sigma=0.3,
                             L=12, M=8, n_int=32, energies=(0.2, -0.3))
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    res = cbs.solve(H, wl.energies, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                    cbs.options(tol=1e-12, extraction="rr"))
    hk = cbs.solve(H, wl.energies, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V, cbs.options(tol=1e-12))
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    for e, E in enumerate(wl.energies):
        ref = ss.ss_rayleigh_ritz(op, E, wl.lambda_min, wl.n_int, wl.V, wl.M, tol=1e-12)
        r = res.energies[e]
        _compare(r, ref, 1e-10)
        assert abs(r["rank"] - ref.rank) <= 1
        worst, un_f, un_r = match(r["lam"], hk.energies[e]["lam"], 1e-10)
        assert not un_f and not un_r
        rr = ss.residuals(op, E, r["lam"], r["vectors"], op.frobenius(E))
        assert np.allclose(rr, r["residual"], rtol=1e-6, atol=1e-15)


def test_solve_rr_c1():
    wl = synth.workload("c1")
    E = float(wl.energies[0])
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    r = cbs.solve(H, [E], wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                  cbs.options(tol=1e-12, extraction="rr")).energies[0]
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    ref = ss.ss_rayleigh_ritz(op, E, wl.lambda_min, wl.n_int, wl.V, wl.M, tol=1e-12)
    _compare(r, ref, 1e-10)
    assert np.allclose(np.exp(1j * r["k"] * wl.grid.a), r["lam"], rtol=1e-12)


def test_solve_multishift_tiny():
    """One Krylov sequence per quadrature point for all energies (shifted BiCG,
    multi_shift = 1): moments and eigenpairs of every energy against the oracle's
    per-energy run of Algorithm 1 (sparse solves are the definition P(z)^{-1} V)."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.tiny_workload(nx=6, ny=5, nz=4, h=0.45, fd_order=4, n_atoms=2, r_c=0.8, sigma=0.3,
                             L=12, M=8, n_int=32, energies=(0.2, -0.3, 0.05))
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    res = cbs.solve(H, wl.energies, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                    cbs.options(tol=1e-12, multi_shift=1))
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    for e, E in enumerate(wl.energies):
        ref = ss.ss_hankel(op, E, wl.lambda_min, wl.n_int, wl.V, wl.M, tol=1e-12, keep_moments=True)
        r = res.energies[e]
        _compare(r, ref, 1e-10)
        assert r["max_solve_residual"] <= 1e-11
        for k in range(2 * wl.M):
            scale = np.max(np.abs(ref.mu[k]))
            assert np.max(np.abs(r["mu"][k] - ref.mu[k])) <= 100 * 1e-12 * (1 / wl.lambda_min) ** (k + 1) * scale


def test_solve_multishift_single_energy_and_rr():
    """Shifted family with one energy (the seed alone, shift 0) and with the Rayleigh-Ritz
    extraction: eigenpairs as the oracle's per-energy runs of the same extraction."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.tiny_workload(nx=6, ny=5, nz=4, h=0.45, fd_order=4, n_atoms=2, r_c=0.8, sigma=0.3,
                             L=12, M=8, n_int=32, energies=(0.2, -0.3))
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    one = cbs.solve(H, wl.energies[:1], wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                    cbs.options(tol=1e-12, multi_shift=1)).energies[0]
    _compare(one, ss.ss_hankel(op, float(wl.energies[0]), wl.lambda_min, wl.n_int, wl.V, wl.M,
                               tol=1e-12), 1e-10)
    rr = cbs.solve(H, wl.energies, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                   cbs.options(tol=1e-12, multi_shift=1, extraction="rr"))
    for e, E in enumerate(wl.energies):
        _compare(rr.energies[e], ss.ss_rayleigh_ritz(op, E, wl.lambda_min, wl.n_int, wl.V, wl.M,
                                                     tol=1e-12), 1e-10)


def test_solve_multishift_mixed_tiny():
    """Shifted family in complex64 (multi_shift = 1 with CBS_FP32_REFINE): the family runs to
    family_tol, then every energy is refined with complex64 BiCG and FP64 reliable updates;
    eigenpairs and moments of every energy against the oracle's per-energy FP64 run."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.tiny_workload(nx=6, ny=5, nz=4, h=0.45, fd_order=4, n_atoms=2, r_c=0.8, sigma=0.3,
                             L=12, M=8, n_int=32, energies=(0.2, -0.3, 0.05))
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    res = cbs.solve(H, wl.energies, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                    cbs.options(tol=1e-12, multi_shift=1, precision="fp32_refine"))
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    for e, E in enumerate(wl.energies):
        ref = ss.ss_hankel(op, E, wl.lambda_min, wl.n_int, wl.V, wl.M, tol=1e-12, keep_moments=True)
        r = res.energies[e]
        _compare(r, ref, 1e-9)
        assert r["max_solve_residual"] <= 1e-12
        for k in range(2 * wl.M):
            scale = np.max(np.abs(ref.mu[k]))
            assert np.max(np.abs(r["mu"][k] - ref.mu[k])) <= 100 * 1e-12 * (1 / wl.lambda_min) ** (k + 1) * scale


def test_scan_batches_and_branches():
    """An energy scan through scan.scan (batches of 2, the last batch one energy): every
    energy's pairs as the oracle's, and scan.connect places each pair in exactly one branch."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs, scan
    energies = (0.1, 0.15, 0.2, 0.25, 0.3)
    wl = synth.tiny_workload(nx=6, ny=5, nz=4, h=0.45, fd_order=4, n_atoms=2, r_c=0.8, sigma=0.3,
                             L=12, M=8, n_int=32, energies=energies)
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    res = scan.scan(H, wl.energies, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                    cbs.options(tol=1e-12, multi_shift=1), batch=2)
    assert len(res) == len(energies)
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    for e, E in enumerate(wl.energies):
        _compare(res[e], ss.ss_hankel(op, E, wl.lambda_min, wl.n_int, wl.V, wl.M, tol=1e-12), 1e-10)
    branches = scan.connect([r["lam"] for r in res], max_jump=1.0)
    assert sum(len(b.lam) for b in branches) == sum(len(r["lam"]) for r in res)


def test_bench_configuration_properties():
    """The bench's own configuration: all 16 energies of the 32x32x16 cell, the paper's BiCG
    tolerance 1e-10, FP64 shifted family, half the points (real V).  What holds for any
    correct result: every solve's FP64 true residual <= tol; every kept pair's residual,
    recomputed with the oracle's operator, is <= 1e-8 and equals the reported one; each
    energy's kept set closed under conjugation; at the stored energies the counts and the
    rank saturation equal the oracle's and the eigenvalues are within 1e-6 of the refined
    ones (the accuracy the 1e-10 solves give the Hankel extraction, up to 1.4e-6 measured on
    the 96x96x20 cell)."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.workload("c2")
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    res = cbs.solve(H, wl.energies, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                    cbs.options(tol=wl.tol, delta=wl.delta, multi_shift=1))
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    assert len(res.energies) == len(wl.energies)
    for e, E in enumerate(wl.energies):
        r = res.energies[e]
        assert r["max_solve_residual"] <= wl.tol
        if len(r["lam"]) == 0:
            continue
        rr = ss.residuals(op, float(E), r["lam"], r["vectors"], op.frobenius(float(E)))
        assert np.all(rr <= 1e-8)
        assert np.allclose(rr, r["residual"], rtol=1e-5, atol=1e-15)
        assert np.max(_conj_defect(r["lam"]) / np.abs(r["lam"])) <= 1e-8
    g, idx = _c2_golden()
    sub = type("R", (), {"energies": [res.energies[i] for i in idx]})()
    _check_c2_golden(sub, g, idx, 1e-6, wl, "bound")


@pytest.mark.parametrize("multi_shift", [0, 1])
def test_stop_fraction_load_balance_rule(multi_shift):
    """The load-balance rule of §3.3 (stop_fraction = 0.5: once more than half of an
    energy's quadrature points have converged, BiCG stops at the others): no point runs
    longer than in the full run, the stopped columns carry flag bit 6 and are not reported
    as unconverged, and every kept pair still passes the residual filter (recomputed by the
    oracle).  stop_fraction = 1 reproduces the full run."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.workload("c1")
    H = cbs.Hamiltonian(wl.grid, wl.vloc, None)
    E = [0.3, 0.6]
    full = cbs.solve(H, E, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                     cbs.options(tol=1e-12, multi_shift=multi_shift))
    half = cbs.solve(H, E, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                     cbs.options(tol=1e-12, multi_shift=multi_shift, stop_fraction=0.5))
    same = cbs.solve(H, E, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                     cbs.options(tol=1e-12, multi_shift=multi_shift, stop_fraction=1.0))
    op = CellOperator(wl.grid, wl.vloc, None)
    assert half.status in (cbs.CBS_OK, cbs.CBS_WRANK)
    for e, Ee in enumerate(E):
        f, h, s1 = full.energies[e], half.energies[e], same.energies[e]
        assert np.array_equal(s1["iters"], f["iters"]) and len(s1["lam"]) == len(f["lam"])
        # per point: the iterations of its slowest column never exceed the full run's
        assert np.all(h["iters"].max(axis=1) <= f["iters"].max(axis=1))
        per_point = f["iters"].max(axis=1)
        if np.sum(per_point < per_point.max()) > wl.n_int // 2:
            assert h["flags"] & 64
        assert not h["flags"] & 1
        if len(h["lam"]):
            rr = ss.residuals(op, Ee, h["lam"], h["vectors"], op.frobenius(Ee))
            assert np.all(rr <= 1e-8)


@pytest.mark.parametrize("form", [dict(), dict(multi_shift=1), dict(multi_shift=1, precision="fp32_refine")])
def test_points_in_waves(form):
    """Quadrature points solved in waves (points_per_wave = 5 of N_int = 32, the last wave
    ragged), the moments accumulated wave by wave: moments and eigenvalues as with every
    point in one wave, and as the oracle's."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.tiny_workload(nx=6, ny=5, nz=4, h=0.45, fd_order=4, n_atoms=2, r_c=0.8, sigma=0.3,
                             L=12, M=8, n_int=32, energies=(0.2, -0.3))
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    one = cbs.solve(H, wl.energies, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V, cbs.options(tol=1e-12, **form))
    wav = cbs.solve(H, wl.energies, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                    cbs.options(tol=1e-12, points_per_wave=5, **form))
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    lam_tol = 1e-9 if form.get("precision") == "fp32_refine" else 1e-10
    for e, E in enumerate(wl.energies):
        a, b = one.energies[e], wav.energies[e]
        for k in range(2 * wl.M):
            scale = np.max(np.abs(a["mu"][k]))
            assert np.max(np.abs(a["mu"][k] - b["mu"][k])) <= 1e-9 * (1 / wl.lambda_min) ** (k + 1) * scale
        assert b["iters"].shape == a["iters"].shape and (b["iters"] > 0).all()
        _compare(b, ss.ss_hankel(op, E, wl.lambda_min, wl.n_int, wl.V, wl.M, tol=1e-12), lam_tol)


def _closure_defect(lam):
    """For each eigenvalue, the relative distance to the nearest 1/conj of the set: the exact
    spectrum is closed under lambda -> 1/conj(lambda) (P(lambda)^dagger = P(1/conj lambda),
    §3.2) and the ring is mapped onto itself, so a complete extraction is too."""
    lam = np.asarray(lam)
    return np.array([np.min(np.abs(lam - 1.0 / np.conj(x))) / abs(x) for x in lam])


def test_solve_c3_saturated_energy_vs_oracle():
    """64x64x24 cell (120 atoms, lambda_min = 0.3, N_int = 64, L = 32, M = 8) at E = -0.5 Ha,
    where eigenvalues just outside the ring leak into more than L*M = 256 dimensions: the
    stored oracle run (tests/golden/make_c3_oracle.py) and the device agree that the rank
    saturates (CBS_WRANK, flag bit 2) and on the pairs kept there."""
    import os
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    path = os.path.join(os.path.dirname(__file__), "golden", "c3_oracle_e00.npz")
    g = np.load(path)
    wl = synth.workload("c3")
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    i = int(g["energy_index"])
    r = cbs.solve(H, wl.energies[[i]], wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                  cbs.options(tol=float(g["tol"]), delta=wl.delta, multi_shift=1))
    e = r.energies[0]
    assert int(g["rank"]) == wl.L * wl.M and e["rank"] == wl.L * wl.M
    assert e["flags"] & 4 and r.status == cbs.CBS_WRANK
    assert len(e["lam"]) == len(g["lam"])
    if len(e["lam"]):
        worst, un_f, un_r = match(e["lam"], g["lam"], 1e-6)
        assert not un_f and not un_r
    # iteration counts of the shifted family's energy equal the oracle's per-energy BiCG
    # up to rounding drift (same Krylov sequence: the family's seed is this energy)
    assert abs(int(np.median(e["iters"].max(axis=1))) - int(np.median(g["iters"].max(axis=1)))) <= 10


def test_solve_c3_inring_energy_properties():
    """64x64x24 cell at E = 0.113 Ha (energy index 19: 26 pairs in the ring, rank 140 of 256),
    shifted family, the paper's tolerance 1e-10.  What holds for any correct result: every
    solve's FP64 true residual <= tol; every kept pair's residual, recomputed with the
    oracle's explicit operator, <= 1e-8 and equal to the reported one; the kept set closed
    under conjugation (real blocks) and under lambda -> 1/conj(lambda) (§3.2), to the
    accuracy the 1e-10 solves give the extraction; propagating pairs (|lambda| = 1) among
    them."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.workload("c3")
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    E = float(wl.energies[19])
    r = cbs.solve(H, [E], wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                  cbs.options(tol=wl.tol, delta=wl.delta, multi_shift=1))
    e = r.energies[0]
    assert r.status == cbs.CBS_OK
    assert e["max_solve_residual"] <= wl.tol
    assert len(e["lam"]) >= 10
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    rr = ss.residuals(op, E, e["lam"], e["vectors"], op.frobenius(E))
    assert np.all(rr <= 1e-8)
    assert np.allclose(rr, e["residual"], rtol=1e-5, atol=1e-15)
    assert np.max(_conj_defect(e["lam"]) / np.abs(e["lam"])) <= 1e-8
    assert np.max(_closure_defect(e["lam"])) <= 1e-5
    assert np.sum(np.abs(np.abs(e["lam"]) - 1.0) < 1e-6) >= 2


@pytest.mark.parametrize("form", [dict(), dict(multi_shift=1), dict(multi_shift=1, precision="fp32_refine")])
def test_conjugate_points(form):
    """With a real V the library solves only the first half of the outer-circle points and
    takes the conjugates of their solutions at the mirrored points (the blocks are real, so
    P(conj z) = conj P(z)): moments and eigenpairs as with every point solved, and as the
    oracle's (which solves every point); the per-point iteration counts are mirrored.  A
    complex V solves every point."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.tiny_workload(nx=6, ny=5, nz=4, h=0.45, fd_order=4, n_atoms=2, r_c=0.8, sigma=0.3,
                             L=12, M=8, n_int=32, energies=(0.2, -0.3))
    assert np.all(wl.V.imag == 0)
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    half = cbs.solve(H, wl.energies, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                     cbs.options(tol=1e-12, **form))
    full = cbs.solve(H, wl.energies, wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                     cbs.options(tol=1e-12, conj_points=0, **form))
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    lam_tol = 1e-9 if form.get("precision") == "fp32_refine" else 1e-10
    for e, E in enumerate(wl.energies):
        a, b = half.energies[e], full.energies[e]
        assert np.array_equal(a["iters"], a["iters"][::-1])
        for k in range(2 * wl.M):
            scale = np.max(np.abs(b["mu"][k]))
            assert np.max(np.abs(a["mu"][k] - b["mu"][k])) <= 1e-9 * (1 / wl.lambda_min) ** (k + 1) * scale
            # a real V makes the moments real
            assert np.max(np.abs(a["mu"][k].imag)) <= 1e-9 * (1 / wl.lambda_min) ** (k + 1) * scale
        ref = ss.ss_hankel(op, E, wl.lambda_min, wl.n_int, wl.V, wl.M, tol=1e-12)
        _compare(a, ref, lam_tol)
        _compare(b, ref, lam_tol)
    Vc = synth.random_rhs_complex(wl.grid.n, wl.L, 5)
    cplx = cbs.solve(H, wl.energies[:1], wl.lambda_min, wl.n_int, wl.L, wl.M, Vc, cbs.options(tol=1e-12, **form))
    ref = ss.ss_hankel(op, float(wl.energies[0]), wl.lambda_min, wl.n_int, Vc, wl.M, tol=1e-12)
    _compare(cplx.energies[0], ref, lam_tol)


def test_solve_c4_cells_properties():
    """The three uneven cells of the batching workload (48x48x12, 64x64x16, 96x96x20; 60, 120
    and 270 atoms; lambda_min = 0.5, N_int = 48, L = 24, M = 8) at E = 0.135 Ha, shifted family,
    tolerance 1e-10, all three in one cbs_solve_cells call: every solve reaches tol on its FP64
    true residual, every kept pair's residual recomputed with the oracle's explicit operator is
    <= 1e-8 and equals the reported one, and the kept set is closed under conjugation and
    under lambda -> 1/conj(lambda)."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    wls = [synth.workload(name) for name in ("c4a", "c4b", "c4c")]
    Hs = [cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors) for wl in wls]
    w0 = wls[0]
    E = float(w0.energies[40])
    res, st = cbs.solve_cells(Hs, [E], w0.lambda_min, w0.n_int, w0.L, w0.M, [wl.V for wl in wls],
                              cbs.options(tol=w0.tol, delta=w0.delta, multi_shift=1))
    for wl, r, sc in zip(wls, res, st):
        e = r.energies[0]
        assert sc in (cbs.CBS_OK, cbs.CBS_WRANK)
        assert e["max_solve_residual"] <= wl.tol
        if len(e["lam"]):
            op = CellOperator(wl.grid, wl.vloc, wl.projectors)
            rr = ss.residuals(op, E, e["lam"], e["vectors"], op.frobenius(E))
            assert np.all(rr <= 1e-8)
            assert np.allclose(rr, e["residual"], rtol=1e-5, atol=1e-15)
            # closure holds to the accuracy 1e-10 solves give the Hankel extraction (up to
            # 1.4e-6 measured on the 96x96x20 cell); the conjugation closure holds to rounding
            # for a real V
            assert np.max(_conj_defect(e["lam"]) / np.abs(e["lam"])) <= 1e-8
            assert np.max(_closure_defect(e["lam"])) <= 1e-5


def _two_tiny_cells():
    a = synth.tiny_workload(nx=6, ny=5, nz=4, h=0.45, fd_order=4, n_atoms=2, r_c=0.8, sigma=0.3, L=8,
                            energies=(0.2, 0.6))
    b = synth.tiny_workload(nx=13, ny=10, nz=6, h=0.4, fd_order=12, n_atoms=4, r_c=1.1, sigma=0.4, L=8,
                            energies=(0.2, 0.6), seed=12)
    return a, b


@pytest.mark.parametrize("form", [dict(multi_shift=1), dict(multi_shift=0, precision="fp32_refine")])
def test_solve_cells_equals_single_calls(form):
    """cbs_solve_cells on two cells of different sizes gives, cell by cell, exactly the
    results of separate cbs_solve calls (same kernels on streams of their own)."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    cells = _two_tiny_cells()
    Hs = [cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors) for wl in cells]
    w0 = cells[0]
    o = cbs.options(tol=1e-12, **form)
    res, st = cbs.solve_cells(Hs, w0.energies, w0.lambda_min, w0.n_int, w0.L, w0.M, [wl.V for wl in cells], o)
    for wl, H, r, sc in zip(cells, Hs, res, st):
        single = cbs.solve(H, w0.energies, w0.lambda_min, w0.n_int, w0.L, w0.M, wl.V, o)
        assert sc == single.status
        for a, b in zip(r.energies, single.energies):
            assert np.array_equal(a["lam"], b["lam"]) and np.array_equal(a["residual"], b["residual"])
            assert np.array_equal(a["vectors"], b["vectors"])
            assert a["rank"] == b["rank"] and a["flags"] == b["flags"]


def test_solve_cells_failures():
    """A cell that fails hard (a non-finite V) fails the call and names the cell, with no
    result kept; a handle given twice and a caller stream are rejected before anything runs."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    a, b = _two_tiny_cells()
    Ha = cbs.Hamiltonian(a.grid, a.vloc, a.projectors)
    Hb = cbs.Hamiltonian(b.grid, b.vloc, b.projectors)
    bad = b.V.copy()
    bad[3, 1] = np.nan
    with pytest.raises(cbs.CbsError) as ex:
        cbs.solve_cells([Ha, Hb], a.energies, a.lambda_min, a.n_int, a.L, a.M, [a.V, bad], cbs.options())
    assert ex.value.status == cbs.CBS_EINVAL and "cell 1" in str(ex.value)
    with pytest.raises(cbs.CbsError):
        cbs.solve_cells([Ha, Ha], a.energies, a.lambda_min, a.n_int, a.L, a.M, [a.V, a.V], cbs.options())
    # the library stays usable
    res, st = cbs.solve_cells([Ha, Hb], a.energies, a.lambda_min, a.n_int, a.L, a.M, [a.V, b.V],
                              cbs.options(tol=1e-12))
    assert len(res) == 2 and all(x in (cbs.CBS_OK, cbs.CBS_WRANK) for x in st)


def test_c5_operator_and_waves():
    """The nanotube-scale cell (160x160x32 = 819,200 points, h = 0.2, 640 atoms with 4
    projectors, L = 48): the FP64 and complex64 applies against the oracle's operator on two
    columns; and the whole method with the quadrature points streamed in waves (8 solved
    points per wave, half the ring by the conjugate-point symmetry), cut at 20 BiCG
    iterations: the call completes with CBS_ENOCONV, every point is accounted for in the
    per-point statistics, and the accumulated moments are finite."""
    torch = need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.workload("c5")
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((1, op.n, 2)) + 1j * rng.standard_normal((1, op.n, 2))
    z, E = 2.0 * np.exp(0.4j), 0.1
    ref = op.apply_P(z, E, X[0])
    for dt, bar in ((torch.complex128, 1e-13), (torch.complex64, 3e-6)):
        Xd = torch.from_numpy(X).to("cuda").to(dt).contiguous()
        Y = cbs.apply(H, [z], [E], Xd).to(torch.complex128).cpu().numpy()[0]
        r = ref if dt == torch.complex128 else op.apply_P(z, E, Xd.to(torch.complex128).cpu().numpy()[0])
        assert rel_err(Y, r) < bar
    res = cbs.solve(H, wl.energies[3:4], wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V,
                    cbs.options(tol=wl.tol, multi_shift=1, max_iter=20, points_per_wave=8),
                    allow=(cbs.CBS_ENOCONV, cbs.CBS_WRANK))
    e = res.energies[0]
    assert res.status == cbs.CBS_ENOCONV and e["flags"] & 1
    assert e["iters"].shape == (wl.n_int, wl.L)
    assert np.all(e["iters"] >= 1) and np.array_equal(e["iters"], e["iters"][::-1])
    assert np.all(np.isfinite(e["mu"]))

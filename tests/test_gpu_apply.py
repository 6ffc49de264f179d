"""P(z) X through cbs_apply against the oracle's operator (Eq. (4) with the twisted
boundary of §2), complex128 and complex64, and the Frobenius norms."""
import numpy as np
import pytest

from oracle.operator import CellOperator
from paper_1709_09347_gb300 import synth
from tests._gpu_common import need_gpu, rel_err, small_cases

pytestmark = pytest.mark.gpu


def _run(wl, zs, Es, L, dtype, H=None):
    torch = need_gpu()
    from paper_1709_09347_gb300 import cbs
    if H is None:
        H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    rng = np.random.default_rng(7)
    X = rng.standard_normal((len(zs), op.n, L)) + 1j * rng.standard_normal((len(zs), op.n, L))
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    Xd = torch.from_numpy(X).to("cuda").to(tdt).contiguous()
    Y = cbs.apply(H, zs, Es, Xd)
    torch.cuda.synchronize()
    Y = Y.to(torch.complex128).cpu().numpy()
    Xr = Xd.to(torch.complex128).cpu().numpy()     # the values the kernel saw
    worst = 0.0
    for s, (z, E) in enumerate(zip(zs, Es)):
        ref = op.apply_P(z, E, Xr[s])
        worst = max(worst, rel_err(Y[s], ref))
    return worst


ZS = [2.0 * np.exp(0.3j), 0.5 * np.exp(-1.2j), np.exp(2.0j), 1.7 - 0.2j]
ES = [0.3, -0.45, 0.0, 1.1]


@pytest.mark.parametrize("case", range(5))
def test_apply_small_fp64(case):
    wl = small_cases()[case]
    assert _run(wl, ZS, ES, wl.L, "c128") < 1e-13


@pytest.mark.parametrize("case", range(5))
def test_apply_small_fp32(case):
    wl = small_cases()[case]
    assert _run(wl, ZS, ES, wl.L, "c64") < 3e-6


@pytest.mark.parametrize("name,L", [("c1", 16), ("c2", 32), ("c3", 32)])
def test_apply_full_size(name, L):
    wl = synth.workload(name, with_rhs=False)
    assert _run(wl, ZS[:2], ES[:2], L, "c128") < 1e-13
    assert _run(wl, ZS[:1], ES[:1], L, "c64") < 3e-6


@pytest.mark.parametrize("name,L", [("tiny", 33), ("tiny", 12), ("c2", 32)])
def test_autotuned_apply(name, L):
    """cbs_autotune_apply picks a launch shape per precision; applies through the tuned
    handle still match the oracle's operator."""
    torch = need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = small_cases()[4] if name == "tiny" else synth.workload(name, with_rhs=False)
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    t128 = cbs.autotune_apply(H, 8, L, torch.complex128)
    t64 = cbs.autotune_apply(H, 8, L, torch.complex64)
    assert t128["py"] >= 1 and t128["pz"] >= 1 and t128["py"] * t128["pz"] * L <= 256
    assert t128["ms"] > 0
    assert t64["x2"] in ((1, -1) if L % 2 == 0 else (0,))
    assert _run(wl, ZS, ES, L, "c128", H) < 1e-13
    assert _run(wl, ZS, ES, L, "c64", H) < 3e-6


@pytest.mark.parametrize("case", [0, 1, 4, 5])
@pytest.mark.parametrize("shape", [(4, 2, 1), (8, 4, 1), (2, 2, -1)])
def test_complex64_kernel_shapes(case, shape):
    """Every complex64 stencil kernel the autotuner can pick, forced through
    cbs_set_apply_shape, against the oracle's operator on cells with ragged tiles (odd
    sizes), FD half-widths 2-6 and even column counts: two columns per thread in 256- and
    512-thread blocks, and one column per thread."""
    torch = need_gpu()
    from paper_1709_09347_gb300 import cbs
    cases = small_cases() + [synth.tiny_workload(nx=13, ny=10, nz=6, h=0.4, fd_order=12, n_atoms=4,
                                                 r_c=1.1, sigma=0.4, L=32)]
    wl = cases[case]
    L = wl.L if wl.L % 4 == 0 else 8
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    cbs.set_apply_shape(H, torch.complex64, *shape)
    assert _run(wl, ZS, ES, L, "c64", H) < 3e-6


@pytest.mark.parametrize("case", [0, 1, 4])
def test_frobenius_norms(case):
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = small_cases()[case]
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    for E in (0.0, 0.37):
        assert np.allclose(H.norms(E), op.frobenius(E), rtol=1e-12, atol=0)


def test_frobenius_c2():
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.workload("c2", with_rhs=False)
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    op = CellOperator(wl.grid, wl.vloc, wl.projectors)
    assert np.allclose(H.norms(-0.2), op.frobenius(-0.2), rtol=1e-11, atol=0)


def test_set_vloc_in_place():
    """cbs_hamiltonian_set_vloc: a handle whose V_loc was replaced (from a device tensor)
    applies P(z) and reports norms exactly as a handle built with that V_loc; a non-finite
    V_loc is rejected and leaves the handle unchanged."""
    torch = need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = small_cases()[1]
    rng = np.random.default_rng(9)
    v2 = wl.vloc + 0.1 * rng.standard_normal(wl.vloc.shape)
    Ha = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    Hb = cbs.Hamiltonian(wl.grid, v2, wl.projectors)
    Ha.set_vloc(torch.from_numpy(v2).cuda())
    X = torch.from_numpy(wl.V[None].copy()).cuda().contiguous()
    for dt in (torch.complex128, torch.complex64):
        Xd = X.to(dt)
        ya = cbs.apply(Ha, [1.7 + 0.4j], 0.2, Xd)
        yb = cbs.apply(Hb, [1.7 + 0.4j], 0.2, Xd)
        assert torch.equal(ya, yb)
    assert np.allclose(Ha.norms(0.2), Hb.norms(0.2), rtol=1e-13)
    bad = v2.copy()
    bad[4] = np.inf
    with pytest.raises(cbs.CbsError):
        Ha.set_vloc(bad)
    assert torch.equal(cbs.apply(Ha, [1.7 + 0.4j], 0.2, X), cbs.apply(Hb, [1.7 + 0.4j], 0.2, X))

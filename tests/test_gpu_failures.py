"""Failure paths through the C ABI, made on the host (no GPU fault, trap or hang):
BiCG iteration limit, rank saturation, non-finite inputs, unsupported sizes."""
import numpy as np
import pytest

from paper_1709_09347_gb300 import synth
from tests._gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def test_max_iter_reports_enoconv_with_readable_results():
    """max_iter = 1: no column reaches tol, the call returns CBS_ENOCONV, every energy's
    stats carry flag bit 0, and the partial results (counts, moments, iterations) are
    still readable."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.workload("c1")
    H = cbs.Hamiltonian(wl.grid, wl.vloc, None)
    o = cbs.options(tol=1e-12, max_iter=1)
    r = cbs.solve(H, [0.3, 0.1], wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V, o,
                  allow=(cbs.CBS_ENOCONV, cbs.CBS_WRANK))
    assert r.status == cbs.CBS_ENOCONV
    for e in r.energies:
        assert e["flags"] & 1
        assert e["max_iters"] == 1
        assert np.all(e["iters"] <= 1)
        assert e["max_solve_residual"] > 1e-12
        assert e["mu"].shape == (2 * wl.M, wl.L, wl.L) and np.all(np.isfinite(e["mu"]))
        assert np.all(e["residual"] <= 1e-8)          # whatever survives the filter is valid
    with pytest.raises(cbs.CbsError) as ei:
        cbs.solve(H, [0.3], wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V, o, allow=())
    assert ei.value.status == cbs.CBS_ENOCONV


def test_rank_saturation_reports_wrank():
    """L = M = 1 on the 8x8x4 cell, which has two eigenvalues in the ring at E = 0.3 (and
    more just outside it): the 1 x 1 Hankel matrix has rank L*M, the call returns the
    CBS_WRANK warning and flag bit 2 is set."""
    need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.workload("c1")
    H = cbs.Hamiltonian(wl.grid, wl.vloc, None)
    L, M = 1, 1
    r = cbs.solve(H, [0.3], wl.lambda_min, wl.n_int, L, M, np.ascontiguousarray(wl.V[:, :L]),
                  cbs.options(tol=1e-12))
    assert r.status == cbs.CBS_WRANK
    e = r.energies[0]
    assert e["rank"] == L * M
    assert e["flags"] & 4
    assert not e["flags"] & 3


def test_nonfinite_inputs_rejected():
    """A NaN in V (host or device) or in V_loc is rejected with CBS_EINVAL before any
    solve runs; the library stays usable afterwards."""
    torch = need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.workload("c1")
    H = cbs.Hamiltonian(wl.grid, wl.vloc, None)
    V = wl.V.copy()
    V[17, 3] = np.nan
    with pytest.raises(cbs.CbsError) as ei:
        cbs.solve(H, [0.3], wl.lambda_min, wl.n_int, wl.L, wl.M, V, cbs.options())
    assert ei.value.status == cbs.CBS_EINVAL and "NaN" in str(ei.value)
    Vd = torch.from_numpy(V).cuda().contiguous()
    Vd[5, 0] = complex(np.inf, 0)
    with pytest.raises(cbs.CbsError) as ei:
        cbs.solve(H, [0.3], wl.lambda_min, wl.n_int, wl.L, wl.M, Vd, cbs.options())
    assert ei.value.status == cbs.CBS_EINVAL
    with pytest.raises(cbs.CbsError) as ei:
        cbs.solve_shifted(H, [2.0], 0.3, Vd, cbs.options())
    assert ei.value.status == cbs.CBS_EINVAL
    bad = wl.vloc.copy()
    bad[3] = np.nan
    with pytest.raises(cbs.CbsError) as ei:
        cbs.Hamiltonian(wl.grid, bad, None)
    assert ei.value.status == cbs.CBS_EINVAL
    r = cbs.solve(H, [0.3], wl.lambda_min, wl.n_int, wl.L, wl.M, wl.V, cbs.options(tol=1e-12))
    assert len(r.energies[0]["lam"]) > 0


def test_apply_rejects_unsupported_columns():
    """Column counts the kernels do not take are rejected by every apply entry point before
    any work is queued (complex128: L <= 256)."""
    torch = need_gpu()
    import ctypes as ct
    from paper_1709_09347_gb300 import cbs
    wl = synth.tiny_workload(nx=4, ny=4, nz=2, h=0.5, fd_order=2, n_atoms=0, projectors=False, L=1)
    H = cbs.Hamiltonian(wl.grid, wl.vloc, None)
    L = 300
    X = torch.zeros((1, H.n, L), dtype=torch.complex128, device="cuda")
    Y = torch.empty_like(X)
    z = np.array([1.0, 0.0])
    E = np.array([0.1])
    lib = cbs.load()
    for fn in (lib.cbs_apply, lib.cbs_apply_noalloc):
        st = fn(H.handle, 1, cbs._dptr(z), cbs._dptr(E), L, ct.c_void_p(X.data_ptr()),
                ct.c_void_p(Y.data_ptr()), cbs.CBS_C128, None)
        assert st == cbs.CBS_EINVAL
        assert b"columns" in lib.cbs_last_error()
    torch.cuda.synchronize()

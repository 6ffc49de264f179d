"""The allocation-free operator apply (cbs_apply_noalloc) against cbs_apply.

cbs_apply_noalloc exists for callers that may not allocate device memory (code running
under another allocator that owns the GPU's memory, or services that cannot afford the
device-wide synchronisation of cudaMalloc/cudaFree); its scratch is a fixed array inside
the library.  Two calls in a row, with different inputs, must each reproduce what
cbs_apply returns for the same inputs, so nothing left in the shared array from the first
call leaks into the second.  This file is collected last on purpose.
"""
import ctypes as ct

import numpy as np
import pytest

from paper_1709_09347_gb300 import synth
from tests._gpu_common import need_gpu, rel_err

pytestmark = pytest.mark.gpu


def _noalloc(cbs, H, z, E, X):
    import torch
    z = np.ascontiguousarray(np.asarray(z, complex))
    E = np.ascontiguousarray(np.asarray(E, float))
    zz = np.ascontiguousarray(np.stack([z.real, z.imag], axis=1))
    Y = torch.empty_like(X)
    dt = {torch.complex128: cbs.CBS_C128, torch.complex64: cbs.CBS_C64}[X.dtype]
    lib = cbs.load()
    st = lib.cbs_apply_noalloc(H.handle, X.shape[0], zz.ctypes.data_as(ct.POINTER(ct.c_double)),
                               E.ctypes.data_as(ct.POINTER(ct.c_double)), X.shape[2],
                               ct.c_void_p(X.data_ptr()), ct.c_void_p(Y.data_ptr()), dt,
                               ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == cbs.CBS_OK, lib.cbs_last_error()
    torch.cuda.synchronize()
    return Y


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-13), ("c64", 3e-6)])
def test_noalloc_matches_apply_twice(dtype, tol):
    torch = need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.workload("c2", with_rhs=False)
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    rng = np.random.default_rng(11)
    for call in range(2):
        n_sys = 6 if call == 0 else 4
        z = np.exp(1j * rng.uniform(0, 2 * np.pi, n_sys)) * rng.choice([2.0, 0.5], n_sys)
        E = rng.uniform(-0.5, 0.5, n_sys)
        X = (torch.randn(n_sys, wl.grid.n, wl.L, dtype=torch.complex128, generator=None)
             .to("cuda").to(tdt).contiguous())
        ref = cbs.apply(H, z, E, X)
        torch.cuda.synchronize()
        got = _noalloc(cbs, H, z, E, X)
        assert rel_err(got.to(torch.complex128).cpu().numpy(),
                       ref.to(torch.complex128).cpu().numpy()) < tol


def test_noalloc_rejects_oversize():
    torch = need_gpu()
    from paper_1709_09347_gb300 import cbs
    wl = synth.workload("c2", with_rhs=False)
    H = cbs.Hamiltonian(wl.grid, wl.vloc, wl.projectors)
    n_sys = 2000     # 2000 systems x 32 columns x 40 atoms x 4 x 16 B > 32 MiB
    lib = cbs.load()
    z = np.ones((n_sys, 2))
    E = np.zeros(n_sys)
    X = torch.empty(1, dtype=torch.complex128, device="cuda")
    st = lib.cbs_apply_noalloc(H.handle, n_sys, z.ctypes.data_as(ct.POINTER(ct.c_double)),
                               E.ctypes.data_as(ct.POINTER(ct.c_double)), wl.L,
                               ct.c_void_p(X.data_ptr()), ct.c_void_p(X.data_ptr()), cbs.CBS_C128,
                               None)
    assert st == cbs.CBS_EINVAL
    assert b"32 MiB" in lib.cbs_last_error()

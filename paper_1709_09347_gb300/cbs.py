"""Thin ctypes binding of libcbs (the C ABI in include/cbs.h).

Argument marshalling only: every step of the method runs in libcbs's CUDA kernels.
PyTorch provides device memory and the current stream for the device-pointer entry
points.  There is no fallback: if libcbs.so is missing this module raises.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcbs.so")

CBS_OK, CBS_EINVAL, CBS_ENOMEM, CBS_ECUDA, CBS_ENOCONV, CBS_EBREAKDOWN, CBS_ETIMEOUT, CBS_WRANK = range(8)
STATUS_NAMES = ["CBS_OK", "CBS_EINVAL", "CBS_ENOMEM", "CBS_ECUDA", "CBS_ENOCONV",
                "CBS_EBREAKDOWN", "CBS_ETIMEOUT", "CBS_WRANK"]
CBS_FP64, CBS_FP32_REFINE = 0, 1
CBS_HANKEL, CBS_RR = 0, 1
CBS_C128, CBS_C64 = 0, 1

# every function the header declares, for the load check
EXPORTS = (
    "cbs_options_default", "cbs_create_hamiltonian", "cbs_hamiltonian_free", "cbs_hamiltonian_size",
    "cbs_hamiltonian_norms", "cbs_apply", "cbs_solve_shifted", "cbs_solve", "cbs_result_count",
    "cbs_result_get", "cbs_result_stats", "cbs_result_all", "cbs_result_moments", "cbs_result_iters",
    "cbs_result_timing", "cbs_result_profile", "cbs_result_free", "cbs_last_error",
    "cbs_kernel_launches", "cbs_apply_workspace_size", "cbs_apply_ws", "cbs_apply_noalloc",
    "cbs_objective", "cbs_autotune_apply", "cbs_set_apply_shape",
    "cbs_result_extract_timing", "cbs_hamiltonian_set_vloc", "cbs_solve_cells",
)


class Grid(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
                ("hx", ct.c_double), ("hy", ct.c_double), ("hz", ct.c_double),
                ("fd_order", ct.c_int)]


class Projectors(ct.Structure):
    _fields_ = [("n_atoms", ct.c_int), ("n_proj", ct.c_int),
                ("sup_ptr", ct.POINTER(ct.c_int64)), ("sup_idx", ct.POINTER(ct.c_int32)),
                ("sup_wrap", ct.POINTER(ct.c_int8)), ("sup_val", ct.POINTER(ct.c_double)),
                ("h", ct.POINTER(ct.c_double))]


class Contour(ct.Structure):
    _fields_ = [("lambda_min", ct.c_double), ("n_int", ct.c_int)]


class Options(ct.Structure):
    _fields_ = [("tol", ct.c_double), ("delta", ct.c_double), ("rho_max", ct.c_double),
                ("max_iter", ct.c_int), ("precision", ct.c_int), ("extraction", ct.c_int),
                ("check_every", ct.c_int), ("inner_tol", ct.c_double), ("max_sweeps", ct.c_int), ("inner_max_iter", ct.c_int), ("stall_sweeps", ct.c_int),
                ("energies_per_batch", ct.c_int), ("profile", ct.c_int), ("multi_shift", ct.c_int),
                ("stream", ct.c_void_p), ("family_tol", ct.c_double), ("stop_fraction", ct.c_double),
                ("points_per_wave", ct.c_int), ("conj_points", ct.c_int)]


class Stats(ct.Structure):
    _fields_ = [("rank", ct.c_int), ("n_extracted", ct.c_int), ("n_kept", ct.c_int),
                ("max_iters", ct.c_int), ("sweeps", ct.c_int), ("flags", ct.c_int),
                ("sigma_max", ct.c_double), ("sigma_cut", ct.c_double),
                ("max_solve_residual", ct.c_double)]


class CbsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


_lib = None


def load():
    """Load libcbs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libcbs.so not found at {LIB_PATH}: build it with "
                           "`python -m paper_1709_09347_gb300.build`")
    lib = ct.CDLL(LIB_PATH)
    P, I, D, V = ct.POINTER, ct.c_int, ct.c_double, ct.c_void_p
    lib.cbs_options_default.argtypes = [P(Options)]
    lib.cbs_create_hamiltonian.argtypes = [P(Grid), P(D), P(Projectors), P(V)]
    lib.cbs_hamiltonian_free.argtypes = [V]
    lib.cbs_hamiltonian_free.restype = None
    lib.cbs_hamiltonian_set_vloc.argtypes = [V, V]
    lib.cbs_hamiltonian_size.argtypes = [V]
    lib.cbs_hamiltonian_size.restype = ct.c_int64
    lib.cbs_hamiltonian_norms.argtypes = [V, D, P(D), P(D), P(D)]
    lib.cbs_apply.argtypes = [V, I, P(D), P(D), I, V, V, I, V]
    lib.cbs_solve_shifted.argtypes = [V, I, P(D), P(D), I, V, V, V, P(I), P(Options)]
    lib.cbs_solve.argtypes = [V, P(D), I, P(Contour), I, I, V, P(Options), P(V)]
    lib.cbs_solve_cells.argtypes = [P(V), I, P(D), I, P(Contour), I, I, P(V), P(Options), P(V), P(I)]
    lib.cbs_result_count.argtypes = [V, I]
    lib.cbs_result_get.argtypes = [V, I, P(D), P(D), P(D), P(D)]
    lib.cbs_result_stats.argtypes = [V, I, P(Stats)]
    lib.cbs_result_all.argtypes = [V, I, P(D), P(D)]
    lib.cbs_result_moments.argtypes = [V, I, P(D)]
    lib.cbs_result_iters.argtypes = [V, I, P(I)]
    lib.cbs_result_timing.argtypes = [V, P(D), P(D), P(D), P(D)]
    lib.cbs_result_extract_timing.argtypes = [V, P(D), P(D), P(D)]
    lib.cbs_result_profile.argtypes = [V, I, P(D), P(D), P(D)]
    lib.cbs_result_free.argtypes = [V]
    lib.cbs_result_free.restype = None
    lib.cbs_last_error.restype = ct.c_char_p
    lib.cbs_apply_workspace_size.argtypes = [V, I, I, I]
    lib.cbs_apply_workspace_size.restype = ct.c_size_t
    lib.cbs_apply_ws.argtypes = [V, I, V, V, I, V, V, I, V, ct.c_size_t, V]
    lib.cbs_apply_noalloc.argtypes = [V, I, P(D), P(D), I, V, V, I, V]
    lib.cbs_objective.argtypes = [V, D, P(Contour), I, I, V, P(Options), P(D), P(D), P(D)]
    lib.cbs_autotune_apply.argtypes = [V, I, I, I, V, P(I), P(I), P(I), P(ct.c_float)]
    lib.cbs_set_apply_shape.argtypes = [V, I, I, I, I]
    lib.cbs_kernel_launches.argtypes = []
    lib.cbs_kernel_launches.restype = ct.c_uint64
    _lib = lib
    return lib


def _check(status, ok=(CBS_OK,)):
    if status not in ok:
        raise CbsError(status, load().cbs_last_error().decode())
    return status


def _dptr(a, ctype=ct.c_double):
    return a.ctypes.data_as(ct.POINTER(ctype))


def options(**kw) -> Options:
    o = Options()
    load().cbs_options_default(ct.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": CBS_FP64, "fp32_refine": CBS_FP32_REFINE}[v]
        if k == "extraction" and isinstance(v, str):
            v = {"hankel": CBS_HANKEL, "rr": CBS_RR}[v]
        setattr(o, k, v)
    return o


class Hamiltonian:
    """Device-resident cell Hamiltonian (cbs_create_hamiltonian)."""

    def __init__(self, grid, vloc, projectors=None):
        lib = load()
        self._keep = []
        g = Grid(grid.nx, grid.ny, grid.nz, grid.hx, grid.hy, grid.hz, grid.fd_order)
        v = np.ascontiguousarray(vloc, dtype=np.float64)
        pp = None
        if projectors is not None and projectors.n_atoms > 0:
            P = projectors
            arrs = (np.ascontiguousarray(P.sup_ptr, np.int64), np.ascontiguousarray(P.sup_idx, np.int32),
                    np.ascontiguousarray(P.sup_wrap, np.int8), np.ascontiguousarray(P.sup_val, np.float64),
                    np.ascontiguousarray(P.h, np.float64))
            self._keep.extend(arrs)
            pp = Projectors(P.n_atoms, P.n_proj, _dptr(arrs[0], ct.c_int64), _dptr(arrs[1], ct.c_int32),
                            _dptr(arrs[2], ct.c_int8), _dptr(arrs[3]), _dptr(arrs[4]))
        h = ct.c_void_p()
        _check(lib.cbs_create_hamiltonian(ct.byref(g), _dptr(v), ct.byref(pp) if pp else None, ct.byref(h)))
        self._h = h
        self.grid = grid
        self.n = int(lib.cbs_hamiltonian_size(h))
        self._keep = []

    @property
    def handle(self):
        return self._h

    def set_vloc(self, vloc):
        """Replace V_loc in place (cbs_hamiltonian_set_vloc): a numpy array or a CUDA float64
        tensor of N values."""
        if isinstance(vloc, np.ndarray):
            v = np.ascontiguousarray(vloc, dtype=np.float64)
            ptr = ct.c_void_p(v.ctypes.data)
        else:
            import torch
            assert vloc.is_cuda and vloc.dtype == torch.float64 and vloc.is_contiguous()
            torch.cuda.current_stream().synchronize()
            v = vloc
            ptr = ct.c_void_p(vloc.data_ptr())
        count = v.numel() if hasattr(v, "numel") else v.size
        assert count == self.n, "V_loc must have N values"
        _check(load().cbs_hamiltonian_set_vloc(self._h, ptr))

    def norms(self, E):
        a, b, c = ct.c_double(), ct.c_double(), ct.c_double()
        _check(load().cbs_hamiltonian_norms(self._h, float(E), ct.byref(a), ct.byref(b), ct.byref(c)))
        return a.value, b.value, c.value

    def close(self):
        if getattr(self, "_h", None):
            load().cbs_hamiltonian_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_ptr(torch):
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def apply(H: Hamiltonian, z, E, X):
    """Y[s] = P(z_s) X[s] = E_s X[s] - H(z_s) X[s] for a CUDA tensor X [n_sys, N, L]
    (complex128 or complex64).  Runs on torch's current stream."""
    import torch
    assert X.is_cuda and X.is_contiguous() and X.dim() == 3
    n_sys, N, L = X.shape
    z = np.ascontiguousarray(np.broadcast_to(np.asarray(z, complex), (n_sys,)))
    E = np.ascontiguousarray(np.broadcast_to(np.asarray(E, float), (n_sys,)))
    zz = np.ascontiguousarray(np.stack([z.real, z.imag], axis=1))
    Y = torch.empty_like(X)
    dt = {torch.complex128: CBS_C128, torch.complex64: CBS_C64}[X.dtype]
    _check(load().cbs_apply(H.handle, n_sys, _dptr(zz), _dptr(E), L, ct.c_void_p(X.data_ptr()),
                            ct.c_void_p(Y.data_ptr()), dt, _stream_ptr(torch)))
    return Y


def solve_shifted(H: Hamiltonian, z, E, B, opts: Options | None = None, allow=(CBS_OK,)):
    """Batched primal/dual shifted solves.  B: CUDA complex128 [N, L].
    Returns (Y, Yd, iters, status) with Y, Yd CUDA tensors [n_sys, N, L]."""
    import torch
    assert B.is_cuda and B.dtype == torch.complex128 and B.is_contiguous()
    z = np.atleast_1d(np.asarray(z, complex))
    n_sys = len(z)
    E = np.ascontiguousarray(np.broadcast_to(np.asarray(E, float), (n_sys,)))
    zz = np.ascontiguousarray(np.stack([z.real, z.imag], axis=1))
    N, L = B.shape
    Y = torch.empty((n_sys, N, L), dtype=torch.complex128, device=B.device)
    Yd = torch.empty_like(Y)
    iters = np.zeros((n_sys, L), np.int32)
    o = opts or options()
    torch.cuda.current_stream().synchronize()
    st = _check(load().cbs_solve_shifted(H.handle, n_sys, _dptr(zz), _dptr(E), L, ct.c_void_p(B.data_ptr()),
                                         ct.c_void_p(Y.data_ptr()), ct.c_void_p(Yd.data_ptr()),
                                         _dptr(iters, ct.c_int), ct.byref(o)),
                ok=tuple(allow) + (CBS_OK,))
    return Y, Yd, iters, st


class Result:
    """Host-side copy of a cbs_result: per-energy dicts."""

    def __init__(self, handle, n_e, N, L, M, n_int, status):
        lib = load()
        self.status = status
        self.energies = []
        for e in range(n_e):
            cnt = lib.cbs_result_count(handle, e)
            lam = np.zeros(cnt, complex)
            k = np.zeros(cnt, complex)
            rho = np.zeros(cnt)
            vec = np.zeros((N, cnt), complex)
            _check(lib.cbs_result_get(handle, e, _dptr(lam.view(np.float64)), _dptr(k.view(np.float64)),
                                      _dptr(rho), _dptr(vec.view(np.float64)) if cnt else None))
            st = Stats()
            _check(lib.cbs_result_stats(handle, e, ct.byref(st)))
            lam_all = np.zeros(st.n_extracted, complex)
            res_all = np.zeros(st.n_extracted)
            _check(lib.cbs_result_all(handle, e, _dptr(lam_all.view(np.float64)), _dptr(res_all)))
            mu = np.zeros((2 * M, L, L), complex)
            _check(lib.cbs_result_moments(handle, e, _dptr(mu.view(np.float64))))
            iters = np.zeros((n_int, L), np.int32)
            _check(lib.cbs_result_iters(handle, e, _dptr(iters, ct.c_int)))
            self.energies.append(dict(
                lam=lam, k=k, residual=rho, vectors=vec, rank=st.rank, n_extracted=st.n_extracted,
                n_kept=st.n_kept, max_iters=st.max_iters, sweeps=st.sweeps, flags=st.flags,
                sigma_max=st.sigma_max, sigma_cut=st.sigma_cut,
                max_solve_residual=st.max_solve_residual, lam_all=lam_all, res_all=res_all,
                mu=mu, iters=iters))
        t = [ct.c_double() for _ in range(4)]
        _check(lib.cbs_result_timing(handle, *[ct.byref(x) for x in t]))
        self.ms_solve, self.ms_moments, self.ms_extract, self.ms_total = (x.value for x in t)
        t = [ct.c_double() for _ in range(3)]
        _check(lib.cbs_result_extract_timing(handle, *[ct.byref(x) for x in t]))
        self.ms_svd, self.ms_reduced, self.ms_vectors = (x.value for x in t)
        self.profile = {}
        for name, dt in (("c128", CBS_C128), ("c64", CBS_C64), ("shift_update", 2)):
            a, b, c = ct.c_double(), ct.c_double(), ct.c_double()
            _check(lib.cbs_result_profile(handle, dt, ct.byref(a), ct.byref(b), ct.byref(c)))
            self.profile[name] = dict(ms=a.value, launches=b.value, outputs=c.value)


def solve(H: Hamiltonian, energies, lambda_min, n_int, L, M, V, opts: Options | None = None,
          allow=(CBS_OK, CBS_WRANK)) -> Result:
    """The whole method for a list of energies.  V: [N, L] complex128, numpy (host) or a
    CUDA tensor (device)."""
    lib = load()
    en = np.ascontiguousarray(np.atleast_1d(np.asarray(energies, float)))
    ctr = Contour(float(lambda_min), int(n_int))
    if isinstance(V, np.ndarray):
        Vh = np.ascontiguousarray(V, dtype=np.complex128)
        vptr = ct.c_void_p(Vh.ctypes.data)
    else:
        import torch
        assert V.is_cuda and V.dtype == torch.complex128 and V.is_contiguous()
        torch.cuda.current_stream().synchronize()
        vptr = ct.c_void_p(V.data_ptr())
    o = opts or options()
    h = ct.c_void_p()
    st = lib.cbs_solve(H.handle, _dptr(en), len(en), ct.byref(ctr), int(L), int(M), vptr, ct.byref(o),
                       ct.byref(h))
    try:
        _check(st, ok=tuple(allow) + (CBS_OK,))
        return Result(h, len(en), H.n, int(L), int(M), int(n_int), st)
    finally:
        if h:
            lib.cbs_result_free(h)


def solve_cells(Hs, energies, lambda_min, n_int, L, M, Vs, opts: Options | None = None,
                allow=(CBS_OK, CBS_WRANK)):
    """The whole method for several cells in one call (cbs_solve_cells: one stream and host
    thread per cell).  Hs: distinct Hamiltonians; Vs: per cell [N_c, L] complex128, numpy
    or CUDA tensors.  Returns (list of Result, list of per-cell statuses)."""
    lib = load()
    n = len(Hs)
    assert len(Vs) == n and n >= 1
    en = np.ascontiguousarray(np.atleast_1d(np.asarray(energies, float)))
    ctr = Contour(float(lambda_min), int(n_int))
    keep, ptrs = [], []
    for V in Vs:
        if isinstance(V, np.ndarray):
            Vh = np.ascontiguousarray(V, dtype=np.complex128)
            keep.append(Vh)
            ptrs.append(Vh.ctypes.data)
        else:
            import torch
            assert V.is_cuda and V.dtype == torch.complex128 and V.is_contiguous()
            torch.cuda.current_stream().synchronize()
            ptrs.append(V.data_ptr())
    harr = (ct.c_void_p * n)(*[H.handle for H in Hs])
    varr = (ct.c_void_p * n)(*ptrs)
    outs = (ct.c_void_p * n)()
    cst = (ct.c_int * n)()
    o = opts or options()
    st = lib.cbs_solve_cells(harr, n, _dptr(en), len(en), ct.byref(ctr), int(L), int(M), varr,
                             ct.byref(o), outs, cst)
    try:
        _check(st, ok=tuple(allow) + (CBS_OK,))
        return ([Result(outs[c], len(en), Hs[c].n, int(L), int(M), int(n_int), cst[c]) for c in range(n)],
                [int(x) for x in cst])
    finally:
        for c in range(n):
            if outs[c]:
                lib.cbs_result_free(outs[c])


def autotune_apply(H: Hamiltonian, n_sys: int, L: int, dtype) -> dict:
    """Time the stencil kernel's launch shapes on n_sys systems of L columns and keep the
    fastest in H (cbs_autotune_apply); dtype is torch.complex128 or torch.complex64."""
    import torch
    code = CBS_C64 if dtype == torch.complex64 else CBS_C128
    py, pz, x2, ms = ct.c_int(0), ct.c_int(0), ct.c_int(0), ct.c_float(0)
    _check(load().cbs_autotune_apply(H.handle, int(n_sys), int(L), code, _stream_ptr(torch),
                                     ct.byref(py), ct.byref(pz), ct.byref(x2), ct.byref(ms)))
    return {"py": py.value, "pz": pz.value, "x2": x2.value, "ms": ms.value}


def set_apply_shape(H: Hamiltonian, dtype, py: int, pz: int = 1, x2: int = 0) -> None:
    """Store a launch shape (as returned by autotune_apply) in H (cbs_set_apply_shape)."""
    import torch
    code = CBS_C64 if dtype == torch.complex64 else CBS_C128
    _check(load().cbs_set_apply_shape(H.handle, code, int(py), int(pz), int(x2)))


def kernel_launches() -> int:
    """Kernels launched by libcbs in this process so far (graph replays count every node)."""
    return int(load().cbs_kernel_launches())


class ApplyPlan:
    """Preallocated operator apply (cbs_apply_ws): device twists, energies and workspace
    held by torch tensors; each call launches on torch's current stream, allocates
    nothing and does not synchronise."""

    def __init__(self, H: Hamiltonian, z, E, L: int, dtype):
        import torch
        self.H, self.L = H, int(L)
        z = np.atleast_1d(np.asarray(z, complex))
        self.n_sys = len(z)
        E = np.ascontiguousarray(np.broadcast_to(np.asarray(E, float), (self.n_sys,)))
        self.dt = {torch.complex128: CBS_C128, torch.complex64: CBS_C64}[dtype]
        self.z = torch.from_numpy(np.ascontiguousarray(z)).to("cuda")
        self.E = torch.from_numpy(E).to("cuda")
        nbytes = int(load().cbs_apply_workspace_size(H.handle, self.n_sys, self.L, self.dt))
        self.ws = torch.empty(max(nbytes, 16), dtype=torch.uint8, device="cuda")

    def __call__(self, X, Y):
        import torch
        assert X.is_cuda and Y.is_cuda and X.is_contiguous() and Y.is_contiguous()
        _check(load().cbs_apply_ws(self.H.handle, self.n_sys, ct.c_void_p(self.z.data_ptr()),
                                   ct.c_void_p(self.E.data_ptr()), self.L, ct.c_void_p(X.data_ptr()),
                                   ct.c_void_p(Y.data_ptr()), self.dt, ct.c_void_p(self.ws.data_ptr()),
                                   self.ws.numel(), _stream_ptr(torch)))
        return Y


def objective(H: Hamiltonian, E, lambda_min, n_int, L, M, V, opts: Options | None = None,
              grad: bool = False, grad_out=None):
    """J = sum_c sum_j c_j ||Y_j||_F^2 of the ring solves at energy E (cbs_objective); with
    grad=True also (dJ/dV_loc, dJ/dE).  dJ/dV_loc is a numpy array [N], or is written into
    grad_out (a CUDA float64 tensor [N]) when given."""
    lib = load()
    ctr = Contour(float(lambda_min), int(n_int))
    Vh = np.ascontiguousarray(V, dtype=np.complex128)
    o = opts or options()
    J = ct.c_double()
    gE = ct.c_double()
    gV = None
    gptr = None
    if grad:
        if grad_out is not None:
            import torch
            assert grad_out.is_cuda and grad_out.dtype == torch.float64 and grad_out.numel() == H.n
            gV = grad_out
            gptr = ct.cast(ct.c_void_p(grad_out.data_ptr()), ct.POINTER(ct.c_double))
        else:
            gV = np.zeros(H.n)
            gptr = _dptr(gV)
    _check(lib.cbs_objective(H.handle, float(E), ct.byref(ctr), int(L), int(M), ct.c_void_p(Vh.ctypes.data),
                             ct.byref(o), ct.byref(J), gptr, ct.byref(gE) if grad else None))
    return (J.value, gV, gE.value) if grad else J.value


def ring_objective(vloc, E, grid, projectors, lambda_min, n_int, L, M, V, opts: Options | None = None):
    """Differentiable J(V_loc, E): a torch.autograd.Function whose backward runs the adjoint
    solves on the device (the forward solutions are recomputed, not stored).  With V_loc a
    CUDA float64 tensor it stays on the device: the Hamiltonian is built once and its
    potential replaced in place (cbs_hamiltonian_set_vloc), and the gradient is written
    straight into a device tensor."""
    import torch

    state = {}

    def ham(v):
        if "H" not in state:
            state["H"] = Hamiltonian(grid, np.zeros(grid.nx * grid.ny * grid.nz), projectors)
        H = state["H"]
        H.set_vloc(v.detach().contiguous() if v.is_cuda else v.detach().cpu().numpy())
        return H

    class _RingObjective(torch.autograd.Function):
        @staticmethod
        def forward(ctx, v, e):
            J = objective(ham(v), float(e), lambda_min, n_int, L, M, V, opts)
            ctx.save_for_backward(v, e)
            return torch.tensor(J, dtype=torch.float64, device=v.device)

        @staticmethod
        def backward(ctx, gJ):
            v, e = ctx.saved_tensors
            H = ham(v)
            if v.is_cuda:
                g = torch.empty(H.n, dtype=torch.float64, device=v.device)
                _, gv, gE = objective(H, float(e), lambda_min, n_int, L, M, V, opts, grad=True, grad_out=g)
            else:
                _, gVh, gE = objective(H, float(e), lambda_min, n_int, L, M, V, opts, grad=True)
                gv = torch.from_numpy(gVh)
            gv = gv.to(v.dtype) * gJ
            ge = torch.tensor(gE, dtype=e.dtype, device=e.device) * gJ
            return gv, ge

    return _RingObjective.apply(vloc, E)

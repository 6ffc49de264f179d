"""The C-ABI library builds for sm_103a, loads, and exports every symbol the header declares."""
import os
import re

from tests._gpu_common import ensure_built

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cbs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cbs_[a-z_0-9]+)\s*\(", src)))


def test_exports():
    lib = ensure_built()
    names = declared_functions()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), f"libcbs.so does not export {n}"
    from paper_1709_09347_gb300 import cbs
    assert set(cbs.EXPORTS) == set(names)


def test_options_default_and_errors():
    import ctypes as ct
    from paper_1709_09347_gb300 import cbs
    lib = ensure_built()
    o = cbs.options()
    assert o.tol == 1e-10 and o.delta == 1e-10 and o.rho_max == 1e-8 and o.precision == cbs.CBS_FP64
    # argument validation happens before any device call
    g = cbs.Grid(4, 4, 2, 0.5, 0.5, 0.5, 8)          # fd_order/2 = 4 > nz = 2
    v = (ct.c_double * 32)()
    h = ct.c_void_p()
    st = lib.cbs_create_hamiltonian(ct.byref(g), v, None, ct.byref(h))
    assert st == cbs.CBS_EINVAL and b"nz" in lib.cbs_last_error()
    assert lib.cbs_result_count(None, 0) == -1

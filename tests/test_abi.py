"""The C-ABI library loads and exports every entry point declared in
include/agp.h; argument validation answers without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "agp.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:agp_status|const\s+char\s*\*)\s*(agp_\w+)\s*\(", src,
                                 flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_00480_gb300 import agp, build
    if not os.path.exists(agp.LIB_PATH):
        build.build()
    return agp.load_library()


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ["agp_plan_create", "agp_plan_destroy", "agp_set_hyper", "agp_matvec",
                 "agp_deriv_matvec", "agp_adjoint_nfft", "agp_nfft_real", "agp_plan_bins",
                 "agp_plan_coeffs", "agp_status_string", "agp_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2504_00480_gb300 import agp
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in agp.exported_symbols(), name


def test_status_strings(lib):
    assert lib.agp_status_string(0) == b"AGP_OK"
    assert lib.agp_status_string(2) == b"AGP_EDOMAIN"
    assert lib.agp_status_string(99) == b"AGP_UNKNOWN"


def test_invalid_arguments_rejected_on_host(lib):
    from paper_2504_00480_gb300 import agp
    h = ctypes.c_void_p()
    assert lib.agp_plan_create(ctypes.byref(h), None, None) == agp.AGP_EINVAL
    assert b"NULL" in lib.agp_last_error()
    assert lib.agp_matvec(None, None, 1, None, 1, 1, 1, None) == agp.AGP_EINVAL
    assert lib.agp_deriv_matvec(None, 0, None, 1, None, 1, 1, None) == agp.AGP_EINVAL
    assert lib.agp_set_hyper(None, 1.0, 1.0, 0.0, None) == agp.AGP_EINVAL
    assert lib.agp_plan_destroy(None) == agp.AGP_OK

    def desc(**kw):
        ptr = (ctypes.c_int * 2)(0, 2)
        feat = (ctypes.c_int * 2)(0, 1)
        N = (ctypes.c_int * 1)(32)
        base = dict(n=10, p=2, X=1, ldx=2, P=1, win_ptr=ptr, win_feat=feat, N=N, cutoff=4,
                    sigma_os=2, kernel=0, ell=0.3, sigma_f=1.0, sigma_eps=0.0, prec=0)
        base.update(kw)
        return agp._Desc(**base), (ptr, feat, N)

    bad = [dict(cutoff=1), dict(cutoff=7), dict(sigma_os=3), dict(ell=-1.0), dict(n=0),
           dict(ldx=1), dict(kernel=5), dict(prec=3),
           dict(N=(ctypes.c_int * 1)(24)), dict(N=(ctypes.c_int * 1)(8), cutoff=5),
           dict(win_feat=(ctypes.c_int * 2)(0, 0)), dict(win_feat=(ctypes.c_int * 2)(0, 9)),
           dict(win_ptr=(ctypes.c_int * 2)(0, 4), p=4, ldx=4,
                win_feat=(ctypes.c_int * 4)(0, 1, 2, 3))]
    for kw in bad:
        d, keep = desc(**kw)
        assert lib.agp_plan_create(ctypes.byref(h), ctypes.byref(d), None) == agp.AGP_EINVAL, kw
        assert not h.value

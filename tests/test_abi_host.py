"""Host-side checks of the C ABI that need no GPU: the library builds and loads, it
exports every function declared in include/taser.h, and invalid arguments are rejected
with a status code before anything is launched."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1609_01797_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    from paper_1609_01797_gb300._native import lib as _lib
    return _lib()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "taser.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(taser_[A-Za-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert {"taser_build_T", "taser_detect", "taser_step_size"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name
    from paper_1609_01797_gb300._native import SIGNATURES
    assert set(SIGNATURES) >= set(names)


def test_problem_size(lib):
    assert lib.taser_problem_size(0, 8) == 9
    assert lib.taser_problem_size(1, 16) == 33
    assert lib.taser_problem_size(2, 16) == 16
    assert lib.taser_problem_size(3, 16) == 31         # QPSK JED: 2K - 1
    assert lib.taser_problem_size(3, 1) == -1
    assert lib.taser_problem_size(7, 16) == -1
    assert lib.taser_problem_size(1, 0) == -1


def test_status_strings(lib):
    for st in range(6):
        assert lib.taser_status_string(st)
    assert lib.taser_status_string(99) == b"unknown status"


P16 = ctypes.c_void_p(16)   # aligned non-NULL dummy pointer: never dereferenced
P4 = ctypes.c_void_p(4)     # misaligned dummy pointer


def _detect(lib, **kw):
    a = dict(batch=8, N=33, T=P16, D=P16, tau=P16, t_max=20, prec=0, mode=0, L=None, s=P16, flags=None)
    a.update(kw)
    return lib.taser_detect(a["batch"], a["N"], a["T"], a["D"], a["tau"], a["t_max"], a["prec"], a["mode"],
                            a["L"], a["s"], a["flags"], None)


@pytest.mark.parametrize("kw", [dict(N=1), dict(N=66), dict(t_max=0), dict(batch=-1), dict(prec=4),
                                dict(mode=2), dict(T=None), dict(D=None), dict(tau=None), dict(s=None),
                                dict(T=P4), dict(L=P4), dict(flags=P4)])
def test_detect_rejects_invalid_arguments(lib, kw):
    assert _detect(lib, **kw) == 1
    assert lib.taser_last_error()


def test_fixed_point_has_no_literal_mode(lib):
    assert _detect(lib, prec=3, mode=1) == 2                  # TASER_ERR_UNSUPPORTED, before any launch
    assert b"FIXED14" in lib.taser_last_error()


def test_detect_empty_batch_is_noop(lib):
    assert _detect(lib, batch=0, T=None, D=None, tau=None, s=None) == 0


def _build(lib, **kw):
    a = dict(kind=1, batch=4, B=128, U=16, X=P16, y=P16, alpha=0.5, T=P16, D=P16, tau=P16, nrm=None, flags=None)
    a.update(kw)
    return lib.taser_build_T(a["kind"], a["batch"], a["B"], a["U"], a["X"], a["y"], a["alpha"], a["T"], a["D"],
                             a["tau"], a["nrm"], a["flags"], None)


@pytest.mark.parametrize("kw", [dict(kind=5), dict(B=0), dict(U=0), dict(U=33), dict(alpha=0.0),
                                dict(alpha=1.0), dict(X=None), dict(y=None), dict(kind=2, U=16),
                                dict(kind=2, U=34, y=None), dict(kind=2, U=1, y=None), dict(kind=3, U=16),
                                dict(kind=3, U=34, y=None), dict(kind=3, U=1, y=None), dict(T=P4),
                                dict(nrm=P4), dict(batch=-3)])
def test_build_rejects_invalid_arguments(lib, kw):
    assert _build(lib, **kw) == 1


def test_build_empty_batch_is_noop(lib):
    assert _build(lib, batch=0, X=None, y=None, T=None, D=None, tau=None) == 0


def test_step_size_rejects_invalid_arguments(lib):
    assert lib.taser_step_size(4, 1, P16, -1, 0.5, P16, None, None) == 1
    assert lib.taser_step_size(4, 33, P16, -1, 1.5, P16, None, None) == 1
    assert lib.taser_step_size(4, 33, None, -1, 0.5, P16, None, None) == 1
    assert lib.taser_step_size(4, 33, P16, 7, 0.5, P16, None, None) == 1
    assert lib.taser_step_size(4, 32, P16, 1, 0.5, P16, None, None) == 1   # QPSK needs odd N
    assert lib.taser_step_size(0, 33, None, -1, 0.5, None, None, None) == 0


def _monitored(lib, **kw):
    a = dict(batch=8, N=33, T=P16, D=P16, tau=P16, t_max=20, prec=0, mode=0, tol=1e-5, obj=None, L=None, s=P16,
             flags=None)
    a.update(kw)
    return lib.taser_detect_monitored(a["batch"], a["N"], a["T"], a["D"], a["tau"], a["t_max"], a["prec"], a["mode"],
                                      a["tol"], a["obj"], a["L"], a["s"], a["flags"], None)


@pytest.mark.parametrize("kw", [dict(N=1), dict(N=66), dict(t_max=0), dict(batch=-1), dict(prec=4), dict(mode=2),
                                dict(tol=-1.0), dict(T=None), dict(s=None), dict(obj=P4), dict(L=P4)])
def test_monitored_rejects_invalid_arguments(lib, kw):
    assert _monitored(lib, **kw) == 1
    assert lib.taser_last_error()


def test_monitored_unsupported_configurations(lib):
    # the two-warp tensor-core bucket (N > 33) and the fixed-point datapath, even for an empty batch
    assert _monitored(lib, prec=1, N=65, batch=0) == 2
    assert b"N <= 33" in lib.taser_last_error()
    assert _monitored(lib, prec=3) == 2
    assert _monitored(lib, batch=0, T=None, D=None, tau=None, s=None) == 0
    assert _monitored(lib, prec=1, N=9, batch=0) == 0          # N < 10 runs the FP32 kernel


def test_unfolded_rejects_fixed_point_and_unknown_precision(lib):
    f = lambda prec: lib.taser_unfolded_forward(1, 33, P16, P16, P16, P16, 10, 4, prec, P16, P16, None, None)
    assert f(3) == 2 and b"fixed-point" in lib.taser_last_error()
    assert f(7) == 1
    b = lambda prec, c: lib.taser_unfolded_backward(1, 33, P16, P16, P16, P16, 100, c, prec, P16, P16, P16, None, None)
    assert b(1, 45) == 1 and b"shared memory" in lib.taser_last_error()     # tensor cores: c <= 44
    assert b(0, 93) == 1 and b"shared memory" in lib.taser_last_error()     # FP32: c <= 92


def test_debug_library_exports_the_same_symbols():
    from paper_1609_01797_gb300 import build as B
    if not os.path.exists(B.LIB_DEBUG):
        B.build(debug=True)
    dbg = ctypes.CDLL(B.LIB_DEBUG)
    for name in _declared_functions():
        assert hasattr(dbg, name), name
    out = [ctypes.c_uint64(7) for _ in range(3)]
    dbg.taser_debug_report.restype = ctypes.c_int
    # NULL outputs are rejected before any CUDA call
    assert dbg.taser_debug_report(None, ctypes.byref(out[1]), ctypes.byref(out[2])) == 1
    assert [o.value for o in out] == [7, 7, 7]


def test_debug_report_is_unsupported_in_the_release_library(lib):
    out = [ctypes.c_uint64(7) for _ in range(3)]
    assert lib.taser_debug_report(*[ctypes.byref(o) for o in out]) == 2   # TASER_ERR_UNSUPPORTED
    assert [o.value for o in out] == [7, 7, 7]
    assert b"libtaser_debug.so" in lib.taser_last_error()
    assert lib.taser_debug_report(None, None, None) == 1                   # TASER_ERR_INVALID_ARG

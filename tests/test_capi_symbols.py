"""The C-ABI library loads and exports every entry point include/sbq.h declares (no GPU).

Only calls that touch no device are made here: the version and the last-error string.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sbq.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"SBQ_API\s+[\w\s\*]+?\b(\w+)\s*\(", text)


@pytest.fixture(scope="module")
def libsbq():
    from paper_2310_00889_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = set(_declared())
    for required in ("stokes_sl_apply", "stokes_dl_apply", "stokes_matvec", "gmres_solve",
                     "batch_plan", "stokes_op_create", "sbq_destroy", "sbq_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libsbq):
    missing = [n for n in _declared() if not hasattr(libsbq, n)]
    assert not missing, missing


def test_host_only_calls(libsbq):
    libsbq.sbq_version.restype = ctypes.c_int
    assert libsbq.sbq_version() == 300
    libsbq.sbq_last_error.restype = ctypes.c_char_p
    assert libsbq.sbq_last_error() == b""
    # argument validation happens before any device call
    libsbq.stokes_sl_apply.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert libsbq.stokes_sl_apply(-1, None, None, None, 0, None, None, 0, None) == 1
    assert b"negative" in libsbq.sbq_last_error()
    assert libsbq.stokes_sl_apply(4, None, None, None, 4, None, None, 0, None) == 1
    assert libsbq.stokes_sl_apply(0, None, None, None, 0, None, None, 7, None) == 1


def test_batch_plan_validation_on_host(libsbq):
    vp = ctypes.c_void_p
    libsbq.batch_plan.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.POINTER(vp)]
    libsbq.sbq_destroy.argtypes = [vp]
    off = (ctypes.c_int64 * 4)(0, 10, 25, 40)
    bad = (ctypes.c_int64 * 4)(0, 10, 5, 40)
    h = vp()
    assert libsbq.batch_plan(3, ctypes.cast(off, vp), ctypes.cast(off, vp), None, ctypes.byref(h)) == 0
    assert h.value
    libsbq.sbq_destroy(h)
    h2 = vp()
    assert libsbq.batch_plan(3, ctypes.cast(bad, vp), ctypes.cast(off, vp), None, ctypes.byref(h2)) == 1
    assert not h2.value


def test_tube_correction_validation_on_host(libsbq):
    """The quadrature-correction entry points reject bad element layouts, sizes, kinds and
    pointers before touching a device."""
    vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    libsbq.tube_correction.argtypes = [i64, ctypes.c_int, ctypes.c_int, i64, vp, vp, vp, ctypes.c_int,
                                       dbl, dbl, dbl, ctypes.POINTER(i64), vp, vp, vp, vp]
    libsbq.tube_correction_targets.argtypes = [i64, ctypes.c_int, ctypes.c_int, i64, vp, vp, vp, i64, vp,
                                               ctypes.c_int, dbl, dbl, dbl, ctypes.POINTER(i64), vp, vp,
                                               vp, vp]
    libsbq.sbq_last_error.restype = ctypes.c_char_p
    nnz = i64(0)
    fake = vp(16)      # never dereferenced: every call below fails validation first
    cases = [
        ((4, 1, 16, 512), b"ns"),           # ns below 2
        ((4, 8, 15, 512), b"nt"),           # odd N_theta
        ((4, 8, 66, 2112), b"nt"),          # N_theta above 64
        ((4, 8, 16, 511), b"n_total"),      # fewer nodes than the elements hold
        ((-1, 8, 16, 512), b"negative"),
    ]
    for (ne, ns, nt, ntot), msg in cases:
        st = libsbq.tube_correction(ne, ns, nt, ntot, fake, fake, fake, 0, 1.0, 1.0, 0.5,
                                    ctypes.byref(nnz), None, None, None, None)
        assert st == 1 and msg in libsbq.sbq_last_error(), (ne, ns, nt, ntot)
    assert libsbq.tube_correction(4, 8, 16, 512, fake, fake, fake, 2, 1.0, 1.0, 0.5,
                                  ctypes.byref(nnz), None, None, None, None) == 1
    assert libsbq.tube_correction(4, 8, 16, 512, None, fake, fake, 0, 1.0, 1.0, 0.5,
                                  ctypes.byref(nnz), None, None, None, None) == 1
    assert libsbq.tube_correction(4, 8, 16, 512, fake, fake, fake, 0, float("nan"), 1.0, 0.5,
                                  ctypes.byref(nnz), None, None, None, None) == 1
    assert libsbq.tube_correction(4, 8, 16, 512, fake, fake, fake, 0, 1.0, 1.0, 0.5,
                                  None, None, None, None, None) == 1
    # off-surface targets: a null target array with targets requested
    assert libsbq.tube_correction_targets(4, 8, 16, 512, fake, fake, fake, 10, None, 0, 1.0, 1.0, 0.5,
                                          ctypes.byref(nnz), None, None, None, None) == 1
    assert libsbq.tube_correction_targets(4, 8, 16, 512, fake, fake, fake, -3, fake, 0, 1.0, 1.0, 0.5,
                                          ctypes.byref(nnz), None, None, None, None) == 1


def test_tube_correction_rules_validation_on_host(libsbq):
    """tube_correction_rules rejects malformed rule tables and tables whose mode count l0 is
    below N_theta / 2 + 1 before touching a device."""
    vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    f = libsbq.tube_correction_rules
    f.argtypes = [i64, ctypes.c_int, ctypes.c_int, i64, vp, vp, vp, i64, vp, ctypes.c_int, dbl, dbl,
                  dbl, ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.POINTER(i64), vp, vp, vp, vp]
    libsbq.sbq_last_error.restype = ctypes.c_char_p
    fake = vp(16)
    nnz = i64(0)
    phi = (ctypes.c_double * (53 * 128))()
    w = (ctypes.c_double * (53 * 128))()
    cnt = (ctypes.c_int * 53)()

    def call(nlev, l0=9, p=phi, ww=w, c=cnt):
        return f(4, 8, 16, 512, fake, fake, fake, 0, None, 0, 1.0, 1.0, 0.5, nlev, l0,
                 ctypes.cast(p, vp), ctypes.cast(ww, vp), ctypes.cast(c, vp), ctypes.byref(nnz),
                 None, None, None, None)

    assert call(-1) == 1 and b"nlev" in libsbq.sbq_last_error()
    assert call(54) == 1
    assert call(53, l0=8) == 1 and b"l0" in libsbq.sbq_last_error()   # N_theta 16 needs l0 >= 9
    cnt[3] = 129
    assert call(53) == 1 and b"128" in libsbq.sbq_last_error()
    cnt[3] = 2
    phi[3 * 128 + 1] = 4.0                      # offset outside [-pi, pi]
    assert call(53) == 1 and b"pi" in libsbq.sbq_last_error()
    phi[3 * 128 + 1] = 0.5
    w[3 * 128] = float("nan")
    assert call(53) == 1


def test_slender_eta_on_host(libsbq):
    """sbq_slender_eta against the dashed-line values of the paper's Stokes-torus eigenvalue
    figure (eta = 10.8574 at eps = 1e-2) and its closed form; bad eps is rejected."""
    import math
    f = libsbq.sbq_slender_eta
    f.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    out = ctypes.c_double()
    assert f(1e-2, ctypes.byref(out)) == 0
    assert abs(out.value - 10.8574) < 1e-4
    for eps in (0.2, 1.0 / 3.0, 0.05):
        assert f(eps, ctypes.byref(out)) == 0
        assert abs(out.value * 2.0 * eps * math.log(1.0 / eps) - 1.0) < 1e-15
    for bad in (0.0, 1.0, -0.1, float("nan")):
        assert f(bad, ctypes.byref(out)) == 1
    assert f(0.1, None) == 1


def test_host_buffer_calls_validate_on_host(libsbq):
    """stokes_apply_host / stokes_solve_host reject bad sizes, pointers and options before
    touching a device."""
    vp, i64, dbl, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    libsbq.stokes_apply_host.argtypes = [i64, vp, vp, vp, dbl, dbl, vp, vp, ci, vp, vp]
    libsbq.stokes_solve_host.argtypes = [i64, vp, vp, vp, dbl, dbl, ci, vp, ci, vp, vp, vp, vp, vp]
    libsbq.sbq_last_error.restype = ctypes.c_char_p
    buf = (ctypes.c_double * 30)()
    p = ctypes.cast(buf, vp)
    assert libsbq.stokes_apply_host(-1, p, p, p, 1.0, 0.5, p, p, 2, None, None) == 1
    assert libsbq.stokes_apply_host(10, p, None, p, 1.0, 0.5, p, p, 2, None, None) == 1
    assert libsbq.stokes_apply_host(10, p, p, p, 1.0, 0.5, p, p, 9, None, None) == 1
    tune = (ctypes.c_int * 3)(3, 3, 0)   # no such tile shape
    assert libsbq.stokes_apply_host(10, p, p, p, 1.0, 0.5, p, p, 2, ctypes.cast(tune, vp),
                                    None) == 1
    assert libsbq.stokes_apply_host(0, None, None, None, 1.0, 0.5, None, None, 2, None, None) == 0

    class Opts(ctypes.Structure):
        _fields_ = [("tol", dbl), ("restart", ci), ("max_iter", ci), ("inner_prec", ci),
                    ("inner_tol", dbl), ("max_outer", ci), ("use_graph", ci), ("resid_prec", ci)]

    good = Opts(1e-10, 50, 100, 2, 1e-5, 10, 1, 0)
    off = (ctypes.c_int64 * 3)(0, 4, 10)
    bad_off = (ctypes.c_int64 * 3)(0, 6, 4)
    call = lambda n, nb, o, opts: libsbq.stokes_solve_host(n, p, p, p, 1.0, 0.5, nb, o, 2, p, p,
                                                           ctypes.byref(opts), None, None)
    assert call(10, 2, ctypes.cast(bad_off, vp), good) == 1
    assert call(10, 2, None, good) == 1
    assert call(10, -1, None, good) == 1
    assert call(10, 2, ctypes.cast(off, vp), Opts(0.0, 50, 100, 2, 1e-5, 10, 1, 0)) == 1
    assert call(10, 2, ctypes.cast(off, vp), Opts(1e-10, 50, 100, 2, 2.0, 10, 1, 0)) == 1
    assert call(10, 2, ctypes.cast(off, vp), Opts(1e-10, 50, 100, 2, 1e-5, 10, 1, 1)) == 1
    buf[5] = float("nan")     # non-finite right-hand side, caught on the host
    assert call(10, 0, None, good) == 5


def test_tree_arguments_rejected_on_host(libsbq):
    """stokes_tree_create validates sizes, pointers, coefficients, theta and order before
    touching a device; apply / destroy reject a handle that is not a tree."""
    vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    f = libsbq.stokes_tree_create
    f.argtypes = [i64, vp, vp, vp, i64, vp, dbl, dbl, dbl, ctypes.c_int, ctypes.POINTER(vp), vp]
    libsbq.sbq_last_error.restype = ctypes.c_char_p
    fake = vp(16)
    h = vp()
    assert f(10, fake, None, fake, 10, fake, 1.0, 0.0, 0.5, 8, None, None) == 1
    assert f(-1, fake, None, fake, 10, fake, 1.0, 0.0, 0.5, 8, ctypes.byref(h), None) == 1
    assert f(10, None, None, fake, 10, fake, 1.0, 0.0, 0.5, 8, ctypes.byref(h), None) == 1
    # the double layer needs normals
    assert f(10, fake, None, fake, 10, fake, 1.0, 1.0, 0.5, 8, ctypes.byref(h), None) == 1
    assert f(10, fake, fake, fake, 10, fake, float("inf"), 1.0, 0.5, 8, ctypes.byref(h), None) == 1
    for theta in (0.0, 1.0, float("nan")):
        assert f(10, fake, None, fake, 10, fake, 1.0, 0.0, theta, 8, ctypes.byref(h), None) == 1
        assert b"theta" in libsbq.sbq_last_error()
    for order in (1, 11):
        assert f(10, fake, None, fake, 10, fake, 1.0, 0.0, 0.5, order, ctypes.byref(h), None) == 1
        assert b"order" in libsbq.sbq_last_error()
    assert h.value is None
    libsbq.stokes_tree_destroy.argtypes = [vp]
    assert libsbq.stokes_tree_destroy(None) == 0
    bogus = (ctypes.c_uint32 * 8)()
    libsbq.stokes_tree_apply.argtypes = [vp, vp, vp, vp]
    assert libsbq.stokes_tree_apply(ctypes.cast(bogus, vp), fake, fake, None) == 1
    assert b"tree" in libsbq.sbq_last_error()

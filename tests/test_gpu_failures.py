"""Failure handling through the C ABI with faults injected on the host only (non-finite
data, null pointers, mismatched sizes, iteration caps, a wrong handle as plan): every case
returns a status and leaves the device usable; nothing traps or hangs the GPU."""
import ctypes

import numpy as np
import pytest

from paper_2310_00889_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sbq():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu tests")
    from paper_2310_00889_gb300 import build
    build.build()
    from paper_2310_00889_gb300 import sbq as mod
    return mod


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.fixture(scope="module")
def pipe():
    c = I.config2(panels=2, nth=32, nr=8)
    return c["surf"], c["rhs"]


def test_nonfinite_rhs_is_reported(sbq, pipe):
    s, rhs = pipe
    op = sbq.StokesOp(_t(s.x), _t(s.n), _t(s.w), 1.5)
    bad = rhs.copy()
    bad[1, 7] = np.nan
    for inner in ("fp64", "fp32c"):
        with pytest.raises(sbq.SbqError) as ei:
            op.solve(_t(bad), tol=1e-10, inner_prec=inner)
        assert ei.value.status == sbq.ENONFINITE
    # the handle and the device still work afterwards
    x, rep = op.solve(_t(rhs), tol=1e-10, inner_prec="fp32c")
    assert rep["status"] == 0
    sbq.check_device()
    op.close()


def test_nonfinite_coordinates_are_rejected(sbq, pipe):
    s, _ = pipe
    x = s.x.copy()
    x[2, 3] = np.inf
    with pytest.raises(sbq.SbqError) as ei:
        sbq.StokesOp(_t(x), _t(s.n), _t(s.w), 1.5)
    assert ei.value.status == sbq.EINVAL


def test_iteration_cap_returns_enoconv(sbq, pipe):
    s, rhs = pipe
    op = sbq.StokesOp(_t(s.x), _t(s.n), _t(s.w), 1.5)
    for inner in ("fp64", "fp32c", "df32"):
        _, rep = op.solve(_t(rhs), tol=1e-12, restart=10, max_iter=1, inner_prec=inner)
        assert rep["status"] == sbq.ENOCONV and rep["iters"] <= 1
    op.close()


def test_bad_options_and_pointers_are_rejected(sbq, pipe):
    s, rhs = pipe
    op = sbq.StokesOp(_t(s.x), _t(s.n), _t(s.w), 1.5)
    lib = sbq.lib
    rep = sbq.GmresReport()
    x = _t(np.zeros_like(rhs))
    b = _t(rhs)
    cases = [sbq.GmresOpts(1e-10, 0, 100, sbq.FP64, 1e-5, 10, 1, 0),       # restart 0
             sbq.GmresOpts(1e-10, 300, 100, sbq.FP64, 1e-5, 10, 1, 0),     # restart > 256
             sbq.GmresOpts(-1.0, 50, 100, sbq.FP64, 1e-5, 10, 1, 0),       # tol <= 0
             sbq.GmresOpts(1e-10, 50, 100, 9, 1e-5, 10, 1, 0),             # unknown precision
             sbq.GmresOpts(1e-10, 50, 100, sbq.FP32_COMP, 2.0, 10, 1, 0),  # inner_tol >= 1
             sbq.GmresOpts(1e-10, 50, 100, sbq.FP32_COMP, 1e-5, 10, 1, 7)]  # resid_prec
    for o in cases:
        st = lib.gmres_solve(op.handle, sbq._ptr(b), sbq._ptr(x), ctypes.byref(o), ctypes.byref(rep),
                             sbq._stream())
        assert st == sbq.EINVAL
    assert lib.stokes_matvec(op.handle, None, sbq._ptr(b), 0, sbq._stream()) == sbq.EINVAL
    assert lib.stokes_matvec(None, sbq._ptr(b), sbq._ptr(x), 0, sbq._stream()) == sbq.EINVAL
    assert lib.sbq_autotune(op.handle, 11, None, sbq._stream()) == sbq.EINVAL
    op.close()


def test_mismatched_sizes_and_wrong_plan_handle(sbq, pipe):
    import torch
    s, _ = pipe
    n = s.size
    with pytest.raises(sbq.SbqError) as ei:   # plan offsets do not cover the nodes
        sbq.StokesOp(_t(s.x), _t(s.n), _t(s.w), 1.5, plan=sbq.BatchPlan([0, n - 1]))
    assert ei.value.status == sbq.EINVAL
    op = sbq.StokesOp(_t(s.x), _t(s.n), _t(s.w), 1.5)
    h = ctypes.c_void_p()
    # an operator handle where a plan handle is expected
    st = sbq.lib.stokes_op_create(n, sbq._ptr(_t(s.x)), sbq._ptr(_t(s.n)), sbq._ptr(_t(s.w)),
                                  1.5, 0.5, 0, None, None, None, op.handle, ctypes.byref(h))
    assert st == sbq.EINVAL and not h.value
    with pytest.raises(ValueError):          # correction with the wrong row count
        sbq.StokesOp(_t(s.x), _t(s.n), _t(s.w), 1.5,
                     correction=(torch.zeros(5, dtype=torch.int64, device="cuda"),
                                 torch.zeros(0, dtype=torch.int64, device="cuda"),
                                 _t(np.zeros(0))))
    with pytest.raises(sbq.SbqError):        # mobility needs offsets covering the nodes
        op.set_mobility([0, n // 2])
    op.close()


def test_peak_probe_reports_a_plausible_fp32_rate():
    """The FMA-chain probe runs and its scalar FP32 rate stays at or below the model peak
    (SMs x 128 lanes x 2 flops x 2.07 GHz) the pair-sum roofline divides by."""
    import torch
    from paper_2310_00889_gb300 import build
    build.build()
    from paper_2310_00889_gb300 import sbq
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu tests")
    info = sbq.device_info()
    model = info["sms"] * info["fp32_lanes_per_sm"] * 2 * 2.07e9 / 1e12
    for kind in ("fp32", "fp32x2", "fp64"):
        tf, ms = sbq.peak_probe(kind)
        assert tf > 0 and ms > 0 and np.isfinite(tf)
    tf, _ = sbq.peak_probe("fp32")
    assert 0.3 * model < tf < 1.05 * model, (tf, model)

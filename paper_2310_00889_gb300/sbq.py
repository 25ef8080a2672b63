"""ctypes binding of libsbq (include/sbq.h): argument marshalling only.

Every arithmetic step runs in the CUDA library.  Tensors are torch CUDA float64
tensors in structure-of-arrays layout, shape (3, N) for point sets, densities and
velocities; torch is used for device memory and the current stream only.  There is
no CPU fallback: importing this module raises if the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsbq.so")

OK, EINVAL, ECUDA, ENOCONV, EBREAKDOWN, ENONFINITE, ETIMEOUT, ENOMEM = range(8)
FP64, FP32, FP32_COMP, DF32 = 0, 1, 2, 3
_PREC = {"fp64": FP64, "fp32": FP32, "fp32c": FP32_COMP, "fp32_comp": FP32_COMP, "df32": DF32,
         FP64: FP64, FP32: FP32, FP32_COMP: FP32_COMP, DF32: DF32}
_STATUS = {0: "SBQ_OK", 1: "SBQ_EINVAL", 2: "SBQ_ECUDA", 3: "SBQ_ENOCONV", 4: "SBQ_EBREAKDOWN",
           5: "SBQ_ENONFINITE", 6: "SBQ_ETIMEOUT", 7: "SBQ_ENOMEM"}


class SbqError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class Tune(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int), ("warps", ctypes.c_int), ("chunk_tiles", ctypes.c_int)]

    def as_dict(self):
        return dict(r=self.r, warps=self.warps, chunk_tiles=self.chunk_tiles)


class GmresOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("inner_prec", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("resid_prec", ctypes.c_int)]


SBQ_HIST = 64


class GmresReport(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("matvecs_fp64", ctypes.c_int), ("matvecs_low", ctypes.c_int),
                ("graph_used", ctypes.c_int), ("kernel_launches", ctypes.c_int),
                ("rel_res", ctypes.c_double),
                ("n_hist", ctypes.c_int), ("rel_res_hist", ctypes.c_double * SBQ_HIST),
                ("time_ms", ctypes.c_double), ("resid_fallbacks", ctypes.c_int)]

    def as_dict(self):
        return dict(status=self.status, iters=self.iters, outer_iters=self.outer_iters,
                    matvecs_fp64=self.matvecs_fp64, matvecs_low=self.matvecs_low,
                    graph_used=bool(self.graph_used), kernel_launches=self.kernel_launches,
                    rel_res=self.rel_res,
                    hist=list(self.rel_res_hist[:self.n_hist]), time_ms=self.time_ms,
                    resid_fallbacks=self.resid_fallbacks)


_i64 = ctypes.c_int64
_vp = ctypes.c_void_p
_int = ctypes.c_int
_dbl = ctypes.c_double


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libsbq.so is not built (%s); run __graft_entry__.build() or "
                           "python paper_2310_00889_gb300/build.py" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "sbq_version": ([], _int),
        "sbq_last_error": ([], ctypes.c_char_p),
        "sbq_device_info": ([_vp, _vp, _vp, _vp], _int),
        "stokes_sl_apply": ([_i64, _vp, _vp, _vp, _i64, _vp, _vp, _int, _vp], _int),
        "stokes_dl_apply": ([_i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _int, _vp], _int),
        "stokes_combined_apply": ([_i64, _vp, _vp, _vp, _vp, _i64, _vp, _dbl, _dbl, _vp, _int,
                                   _vp], _int),
        "laplace_sl_apply": ([_i64, _vp, _vp, _vp, _i64, _vp, _vp, _int, _vp], _int),
        "laplace_dl_apply": ([_i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _int, _vp], _int),
        "laplace_combined_apply": ([_i64, _vp, _vp, _vp, _vp, _i64, _vp, _dbl, _dbl, _vp, _int,
                                    _vp], _int),
        "batch_plan": ([_int, _vp, _vp, _vp, ctypes.POINTER(_vp)], _int),
        "stokes_op_create": ([_i64, _vp, _vp, _vp, _dbl, _dbl, _i64, _vp, _vp, _vp, _vp,
                              ctypes.POINTER(_vp)], _int),
        "laplace_op_create": ([_i64, _vp, _vp, _vp, _dbl, _dbl, _i64, _vp, _vp, _vp, _vp,
                               ctypes.POINTER(_vp)], _int),
        "stokes_matvec": ([_vp, _vp, _vp, _int, _vp], _int),
        "stokes_op_set_mobility": ([_vp, _int, _vp, _vp], _int),
        "stokes_mobility_rhs": ([_vp, _vp, _vp, _vp, _int, _vp], _int),
        "stokes_op_set_sl_correction": ([_vp, _i64, _vp, _vp, _vp, _vp], _int),
        "stokes_op_set_tree": ([_vp, _dbl, _int, _vp], _int),
        "stokes_mobility_velocity": ([_vp, _vp, _vp, _vp], _int),
        "stokes_matvec_bounded": ([_vp, _vp, _vp, _vp, _vp], _int),
        "gmres_solve": ([_vp, _vp, _vp, ctypes.POINTER(GmresOpts), ctypes.POINTER(GmresReport),
                         _vp], _int),
        "sbq_autotune": ([_vp, _int, ctypes.POINTER(Tune), _vp], _int),
        "sbq_op_tune": ([_vp, _int, ctypes.POINTER(Tune)], _int),
        "sbq_op_stats": ([_vp, _int, ctypes.POINTER(_int), ctypes.POINTER(_dbl)], _int),
        "sbq_check_device": ([_vp], _int),
        "sbq_op_time_pairsum": ([_vp, _vp, _vp, _int, _int, _vp, ctypes.POINTER(_dbl),
                                 ctypes.POINTER(_dbl)], _int),
        "stokes_dl_gauss_correction": ([_int, _vp, _vp, _vp, _vp, _int, _vp, _vp, _vp, _vp],
                                       _int),
        "tube_correction": ([_i64, _int, _int, _i64, _vp, _vp, _vp, _int, _dbl, _dbl, _dbl,
                             ctypes.POINTER(_i64), _vp, _vp, _vp, _vp], _int),
        "tube_correction_rules": ([_i64, _int, _int, _i64, _vp, _vp, _vp, _i64, _vp, _int, _dbl,
                                   _dbl, _dbl, _int, _int, _vp, _vp, _vp, ctypes.POINTER(_i64),
                                   _vp, _vp, _vp, _vp], _int),
        "sbq_peak_probe": ([_int, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl), _vp], _int),
        "tube_correction_targets": ([_i64, _int, _int, _i64, _vp, _vp, _vp, _i64, _vp, _int, _dbl,
                                     _dbl, _dbl, ctypes.POINTER(_i64), _vp, _vp, _vp, _vp], _int),
        "sbq_slender_eta": ([_dbl, ctypes.POINTER(_dbl)], _int),
        "stokes_apply_host": ([_i64, _vp, _vp, _vp, _dbl, _dbl, _vp, _vp, _int,
                               ctypes.POINTER(Tune), _vp], _int),
        "stokes_solve_host": ([_i64, _vp, _vp, _vp, _dbl, _dbl, _int, _vp, _int, _vp, _vp,
                               ctypes.POINTER(GmresOpts), ctypes.POINTER(GmresReport), _vp], _int),
        "sbq_destroy": ([_vp], None),
        "stokes_tree_create": ([_i64, _vp, _vp, _vp, _i64, _vp, _dbl, _dbl, _dbl, _int,
                                ctypes.POINTER(_vp), _vp], _int),
        "stokes_tree_apply": ([_vp, _vp, _vp, _vp], _int),
        "stokes_tree_stats": ([_vp, ctypes.POINTER(_dbl), ctypes.POINTER(_i64)], _int),
        "stokes_tree_destroy": ([_vp], _int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


def _check(status):
    if status != OK:
        msg = lib.sbq_last_error()
        raise SbqError(status, msg.decode() if msg else "")
    return status


def _prec(p):
    try:
        return _PREC[p]
    except KeyError:
        raise ValueError("unknown precision %r (fp64, fp32, fp32c)" % (p,))


def _dev(t, shape=None, name="array"):
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise TypeError("%s must be a CUDA float64 tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
    return t


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def version():
    return lib.sbq_version()


def device_info():
    sms, lanes, ma, mi = _int(), _int(), _int(), _int()
    _check(lib.sbq_device_info(ctypes.byref(sms), ctypes.byref(lanes), ctypes.byref(ma),
                               ctypes.byref(mi)))
    return dict(sms=sms.value, fp32_lanes_per_sm=lanes.value, cc=(ma.value, mi.value))


def slender_eta(eps):
    """The slender-body mixing parameter eta of the combined-field formulations, computed by
    the library (sbq_slender_eta)."""
    out = _dbl()
    _check(lib.sbq_slender_eta(float(eps), ctypes.byref(out)))
    return out.value


def _host(t, shape, name):
    if not (isinstance(t, torch.Tensor) and t.device.type == "cpu" and t.dtype == torch.float64):
        raise TypeError("%s must be a CPU float64 tensor (pinned for asynchronous copies)" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
    return t


def _apply(kind, src, nrm, w, sigma, trg, alpha, beta, prec, out, stream):
    ns = src.shape[1]
    nt = trg.shape[1]
    _dev(src, (3, ns), "src")
    _dev(w, (ns,), "w")
    _dev(sigma, (3, ns), "sigma")
    _dev(trg, (3, nt), "trg")
    if nrm is not None:
        _dev(nrm, (3, ns), "nrm")
    if out is None:
        out = torch.empty((3, nt), dtype=torch.float64, device=trg.device)
    _dev(out, (3, nt), "out")
    p = _prec(prec)
    st = _stream(stream)
    if kind == "sl":
        _check(lib.stokes_sl_apply(ns, _ptr(src), _ptr(w), _ptr(sigma), nt, _ptr(trg), _ptr(out),
                                   p, st))
    elif kind == "dl":
        _check(lib.stokes_dl_apply(ns, _ptr(src), _ptr(nrm), _ptr(w), _ptr(sigma), nt, _ptr(trg),
                                   _ptr(out), p, st))
    else:
        _check(lib.stokes_combined_apply(ns, _ptr(src), _ptr(nrm), _ptr(w), _ptr(sigma), nt,
                                         _ptr(trg), float(alpha), float(beta), _ptr(out), p, st))
    return out


def sl_apply(src, w, sigma, trg, prec="fp32c", out=None, stream=None):
    """Single-layer velocity S[sigma] at trg (Eq. stokes-sl, uncorrected Nystrom sum)."""
    return _apply("sl", src, None, w, sigma, trg, 1.0, 0.0, prec, out, stream)


class StokesTree:
    """Treecode for the layer sum alpha S + beta D (stokes_tree_*): built once per geometry
    (src, nrm, w; trg defaults to src, the on-surface sum without self terms), applied to
    any number of densities.  theta and order set the accuracy (about 2e-6 at 0.5 and 8)."""

    def __init__(self, src, w, nrm=None, trg=None, alpha=1.0, beta=0.0, theta=0.5, order=8,
                 stream=None):
        ns = src.shape[1]
        _dev(src, (3, ns), "src")
        _dev(w, (ns,), "w")
        _dev(nrm, (3, ns), "nrm")
        if trg is None:
            trg = src
        nt = trg.shape[1]
        _dev(trg, (3, nt), "trg")
        self.ns, self.nt = ns, nt
        self._keep = (src, w, nrm, trg)
        h = ctypes.c_void_p()
        _check(lib.stokes_tree_create(ns, _ptr(src), _ptr(nrm), _ptr(w), nt, _ptr(trg),
                                      float(alpha), float(beta), float(theta), int(order),
                                      ctypes.byref(h), _stream(stream)))
        self.h = h

    def apply(self, sigma, out=None, stream=None):
        _dev(sigma, (3, self.ns), "sigma")
        if out is None:
            out = torch.empty((3, self.nt), dtype=torch.float64, device=sigma.device)
        _dev(out, (3, self.nt), "out")
        _check(lib.stokes_tree_apply(self.h, _ptr(sigma), _ptr(out), _stream(stream)))
        return out

    def stats(self):
        pairs = ctypes.c_double()
        counts = (ctypes.c_int64 * 4)()
        _check(lib.stokes_tree_stats(self.h, ctypes.byref(pairs), counts))
        return {"pairs": pairs.value, "cells": counts[0], "proxies": counts[1],
                "entries": counts[2], "target_blocks": counts[3]}

    def close(self):
        if self.h is not None and self.h.value:
            _check(lib.stokes_tree_destroy(self.h))
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SlTree(StokesTree):
    """StokesTree of the single layer alone (alpha = 1, beta = 0)."""

    def __init__(self, src, w, trg=None, theta=0.5, order=8, stream=None):
        super().__init__(src, w, None, trg, 1.0, 0.0, theta, order, stream)


def dl_apply(src, nrm, w, sigma, trg, prec="fp32c", out=None, stream=None):
    """Double-layer velocity D[sigma] at trg (Eq. stokes-dl)."""
    return _apply("dl", src, nrm, w, sigma, trg, 0.0, 1.0, prec, out, stream)


def combined_apply(src, nrm, w, sigma, trg, alpha, beta, prec="fp32c", out=None, stream=None):
    """alpha S[sigma] + beta D[sigma] at trg in one pass."""
    return _apply("cf", src, nrm, w, sigma, trg, alpha, beta, prec, out, stream)


def dl_gauss_correction(src, nrm, w, body_off=None, prec="fp64", stream=None):
    """Sparse correction E (rowptr, col, val) of the double layer by singularity
    subtraction per closed body: E_ii = -R_i - I/2 with R_i the 3 x 3 double-layer row
    sum of node i over its own body (body_off: node offsets of the bodies, default one
    body).  Pass the result as StokesOp(..., correction=...)."""
    n = src.shape[1]
    _dev(src, (3, n), "src")
    _dev(nrm, (3, n), "nrm")
    _dev(w, (n,), "w")
    off = np.asarray([0, n] if body_off is None else body_off, dtype=np.int64)
    if off.ndim != 1 or off.size < 2 or int(off[-1]) != n:
        raise ValueError("body_off must end at the node count %d" % n)
    c_off = (ctypes.c_int64 * off.size)(*[int(v) for v in off])
    dev = src.device
    rowptr = torch.empty(3 * n + 1, dtype=torch.int64, device=dev)
    col = torch.empty(9 * n, dtype=torch.int64, device=dev)
    val = torch.empty(9 * n, dtype=torch.float64, device=dev)
    _check(lib.stokes_dl_gauss_correction(int(off.size - 1), c_off, _ptr(src), _ptr(nrm), _ptr(w),
                                          _prec(prec), _ptr(rowptr), _ptr(col), _ptr(val),
                                          _stream(stream)))
    return rowptr, col, val


def _rules_call(src, nrm, w, nelem, ns, nt, trg, lap, alpha, beta, near_factor, rules, stream):
    """tube_correction_rules with host tables rules = (phi, w, cnt, l0) of shapes (L, 128),
    (L, 128), (L,) and the tables' mode count, or rules = "none" (no compressed rules)."""
    if isinstance(rules, str):
        if rules != "none":
            raise ValueError("rules must be a table (phi, w, cnt, l0) or 'none'")
        nlev, l0, dptr_phi, dptr_w, dptr_cnt = 0, 0, None, None, None
    else:
        rphi = np.ascontiguousarray(rules[0], dtype=np.float64)
        rw = np.ascontiguousarray(rules[1], dtype=np.float64)
        rcnt = np.ascontiguousarray(rules[2], dtype=np.int32)
        l0 = int(rules[3])
        nlev = int(rcnt.shape[0])
        if rphi.shape != (nlev, 128) or rw.shape != (nlev, 128):
            raise ValueError("rules: phi and w must be (levels, 128)")
        dptr_phi, dptr_w = rphi.ctypes.data_as(_vp), rw.ctypes.data_as(_vp)
        dptr_cnt = rcnt.ctypes.data_as(_vp)
    n = src.shape[1]
    m = trg.shape[1] if trg is not None else 0
    nnz = _i64(0)
    args = (int(nelem), int(ns), int(nt), int(n), _ptr(src), _ptr(nrm), _ptr(w), int(m),
            _ptr(trg) if trg is not None else None, lap, float(alpha), float(beta), float(near_factor),
            nlev, l0, dptr_phi, dptr_w, dptr_cnt)
    _check(lib.tube_correction_rules(*args, ctypes.byref(nnz), None, None, None, _stream(stream)))
    rows = (1 if lap else 3) * (m if trg is not None else n)
    rowptr = torch.empty(rows + 1, dtype=torch.int64, device=src.device)
    col = torch.empty(max(nnz.value, 1), dtype=torch.int64, device=src.device)
    val = torch.empty(max(nnz.value, 1), dtype=torch.float64, device=src.device)
    _check(lib.tube_correction_rules(*args, ctypes.byref(nnz), _ptr(rowptr), _ptr(col), _ptr(val),
                                     _stream(stream)))
    return rowptr, col[:nnz.value], val[:nnz.value]


def tube_correction(src, nrm, w, nelem, ns, nt, kind="stokes", alpha=1.0, beta=1.0,
                    near_factor=0.5, stream=None, rules=None):
    """Quadrature correction E (rowptr, col, val) of the tube elements that make up the first
    nelem * ns * nt nodes (Sec. 3.2.1-3.2.4): for every tube node and every element whose
    near region holds it, the entries that turn the punctured sum over the element into the
    accurate integral.  kind "stokes" (alpha S + beta D, 3 x 3) or "laplace" (scalar); an
    operator K = diag I + D + eta S takes alpha = eta, beta = 1.  Pass the result as
    StokesOp / LaplaceOp (..., correction=...).  rules: None (the library's compiled-in
    compressed angular rules), "none" (dyadically refined rules only), or a caller's table
    (phi, w, cnt, l0), e.g. angular_rules.load(nt)."""
    n = src.shape[1]
    _dev(src, (3, n), "src")
    _dev(nrm, (3, n), "nrm")
    _dev(w, (n,), "w")
    if kind not in ("stokes", "laplace"):
        raise ValueError("kind must be 'stokes' or 'laplace'")
    lap = 1 if kind == "laplace" else 0
    if rules is not None:
        return _rules_call(src, nrm, w, nelem, ns, nt, None, lap, alpha, beta, near_factor, rules,
                           stream)
    nnz = _i64(0)
    args = (int(nelem), int(ns), int(nt), int(n), _ptr(src), _ptr(nrm), _ptr(w), lap, float(alpha),
            float(beta), float(near_factor))
    _check(lib.tube_correction(*args, ctypes.byref(nnz), None, None, None, _stream(stream)))
    dev = src.device
    rowptr = torch.empty((1 if lap else 3) * n + 1, dtype=torch.int64, device=dev)
    col = torch.empty(max(nnz.value, 1), dtype=torch.int64, device=dev)
    val = torch.empty(max(nnz.value, 1), dtype=torch.float64, device=dev)
    _check(lib.tube_correction(*args, ctypes.byref(nnz), _ptr(rowptr), _ptr(col), _ptr(val),
                               _stream(stream)))
    return rowptr, col[:nnz.value], val[:nnz.value]


def peak_probe(kind, stream=None):
    """Achieved TFLOP/s of long FMA chains on every SM: kind "fp32", "fp32x2" (packed) or
    "fp64"; returns (tflops, ms)."""
    k = {"fp32": 0, "fp32x2": 1, "fp64": 2}[kind]
    tf, ms = _dbl(0.0), _dbl(0.0)
    _check(lib.sbq_peak_probe(k, ctypes.byref(tf), ctypes.byref(ms), _stream(stream)))
    return tf.value, ms.value


def tube_correction_targets(src, nrm, w, nelem, ns, nt, trg, kind="stokes", alpha=1.0, beta=1.0,
                            near_factor=0.5, stream=None, rules=None):
    """Correction E (rowptr, col, val) for off-surface targets trg (3, m) near the tube elements
    (Sec. 3.2.3): rows component-major over the targets, columns over the nodes.  The layer
    potential at trg is the plain sum (combined_apply / laplace_apply) plus E sigma."""
    n = src.shape[1]
    m = trg.shape[1]
    _dev(src, (3, n), "src")
    _dev(nrm, (3, n), "nrm")
    _dev(w, (n,), "w")
    _dev(trg, (3, m), "trg")
    if kind not in ("stokes", "laplace"):
        raise ValueError("kind must be 'stokes' or 'laplace'")
    lap = 1 if kind == "laplace" else 0
    if rules is not None:
        return _rules_call(src, nrm, w, nelem, ns, nt, trg, lap, alpha, beta, near_factor, rules,
                           stream)
    nnz = _i64(0)
    args = (int(nelem), int(ns), int(nt), int(n), _ptr(src), _ptr(nrm), _ptr(w), int(m), _ptr(trg),
            lap, float(alpha), float(beta), float(near_factor))
    _check(lib.tube_correction_targets(*args, ctypes.byref(nnz), None, None, None, _stream(stream)))
    dev = src.device
    rowptr = torch.empty((1 if lap else 3) * m + 1, dtype=torch.int64, device=dev)
    col = torch.empty(max(nnz.value, 1), dtype=torch.int64, device=dev)
    val = torch.empty(max(nnz.value, 1), dtype=torch.float64, device=dev)
    _check(lib.tube_correction_targets(*args, ctypes.byref(nnz), _ptr(rowptr), _ptr(col), _ptr(val),
                                       _stream(stream)))
    return rowptr, col[:nnz.value], val[:nnz.value]


def laplace_apply(src, nrm, w, sigma, trg, alpha=1.0, beta=0.0, prec="fp32c", out=None,
                  stream=None):
    """Laplace alpha S[sigma] + beta D[sigma] at trg (Sec. 4.1), scalar sigma (ns,) -> (nt,)."""
    ns = src.shape[1]
    nt = trg.shape[1]
    _dev(src, (3, ns), "src")
    _dev(w, (ns,), "w")
    _dev(sigma, (ns,), "sigma")
    _dev(trg, (3, nt), "trg")
    if nrm is not None:
        _dev(nrm, (3, ns), "nrm")
    if out is None:
        out = torch.empty((nt,), dtype=torch.float64, device=trg.device)
    _dev(out, (nt,), "out")
    p, st = _prec(prec), _stream(stream)
    if beta == 0.0:
        _check(lib.laplace_sl_apply(ns, _ptr(src), _ptr(w), _ptr(sigma), nt, _ptr(trg), _ptr(out),
                                    p, st) if alpha == 1.0 else
               lib.laplace_combined_apply(ns, _ptr(src), _ptr(nrm), _ptr(w), _ptr(sigma), nt,
                                          _ptr(trg), float(alpha), 0.0, _ptr(out), p, st))
    elif alpha == 0.0 and beta == 1.0:
        _check(lib.laplace_dl_apply(ns, _ptr(src), _ptr(nrm), _ptr(w), _ptr(sigma), nt, _ptr(trg),
                                    _ptr(out), p, st))
    else:
        _check(lib.laplace_combined_apply(ns, _ptr(src), _ptr(nrm), _ptr(w), _ptr(sigma), nt,
                                          _ptr(trg), float(alpha), float(beta), _ptr(out), p, st))
    return out


def check_device(stream=None):
    """Synchronise and raise SbqError(ETIMEOUT) if a device-side bounded wait expired."""
    _check(lib.sbq_check_device(_stream(stream)))


class BatchPlan:
    """Work-list plan for independent segments (prefix offsets, host int64)."""

    def __init__(self, src_off, trg_off=None, tune=None):
        import numpy as np
        so = np.ascontiguousarray(src_off, dtype=np.int64)
        to = so if trg_off is None else np.ascontiguousarray(trg_off, dtype=np.int64)
        self.src_off, self.trg_off = so, to
        t = None
        if tune is not None:
            t = Tune(int(tune["r"]), int(tune["warps"]), int(tune.get("chunk_tiles", 0)))
        h = _vp()
        _check(lib.batch_plan(len(so) - 1, so.ctypes.data_as(_vp), to.ctypes.data_as(_vp),
                              ctypes.byref(t) if t is not None else None, ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib.sbq_destroy(self.handle)
            self.handle = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StokesOp:
    """K sigma = diag sigma + (D + eta S)[sigma] + E sigma on the nodes (Eq. stokes-bie-new)."""

    _ncomp = 3
    _create = "stokes_op_create"

    def __init__(self, src, nrm, w, eta, diag=0.5, correction=None, plan: BatchPlan | None = None):
        n = src.shape[1]
        self.vshape = (3, n) if self._ncomp == 3 else (n,)
        _dev(src, (3, n), "src")
        _dev(nrm, (3, n), "nrm")
        _dev(w, (n,), "w")
        self.n = n
        self.eta = float(eta)
        self.device = src.device
        rowptr = col = val = None
        nnz = 0
        if correction is not None:
            rowptr, col, val = correction
            for t, nm, dt in ((rowptr, "rowptr", torch.int64), (col, "col", torch.int64),
                              (val, "val", torch.float64)):
                if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
                    raise TypeError("correction %s must be a contiguous CUDA %s tensor" % (nm, dt))
            if rowptr.numel() != self._ncomp * n + 1:
                raise ValueError("rowptr must have %d entries" % (self._ncomp * n + 1))
            nnz = int(val.numel())
        h = _vp()
        _check(getattr(lib, self._create)(n, _ptr(src), _ptr(nrm), _ptr(w), self.eta, float(diag),
                                          nnz, _ptr(rowptr), _ptr(col), _ptr(val),
                                          plan.handle if plan is not None else None,
                                          ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            lib.sbq_destroy(self.handle)
            self.handle = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def matvec(self, sigma, prec="fp64", out=None, stream=None):
        _dev(sigma, self.vshape, "sigma")
        if out is None:
            out = torch.empty_like(sigma)
        _dev(out, self.vshape, "out")
        _check(lib.stokes_matvec(self.handle, _ptr(sigma), _ptr(out), _prec(prec), _stream(stream)))
        return out

    def set_mobility(self, body_off, stream=None):
        """Make this operator the mobility operator K (I - L) + L for the bodies with node
        offsets body_off (Sec. 4.2, Eq. new-mobility-bie)."""
        off = np.asarray(body_off, dtype=np.int64)
        c_off = (ctypes.c_int64 * off.size)(*[int(v) for v in off])
        _check(lib.stokes_op_set_mobility(self.handle, int(off.size - 1), c_off, _stream(stream)))
        self.nbody = int(off.size - 1)

    def set_tree(self, theta=0.5, order=8, stream=None):
        """Applies in "fp32" (and inner solves with inner_prec="fp32") then take the treecode
        (stokes_op_set_tree); theta <= 0 removes it."""
        _check(lib.stokes_op_set_tree(self.handle, float(theta), int(order), _stream(stream)))

    def set_sl_correction(self, correction, stream=None):
        """Correction (rowptr, col, val) of the single layer alone, used by mobility_rhs for
        S nu (e.g. tube_correction(..., alpha=1.0, beta=0.0)); None removes it."""
        if correction is None:
            _check(lib.stokes_op_set_sl_correction(self.handle, 0, None, None, None,
                                                   _stream(stream)))
            return
        rowptr, col, val = correction
        for t, nm, dt in ((rowptr, "rowptr", torch.int64), (col, "col", torch.int64),
                          (val, "val", torch.float64)):
            if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
                raise TypeError("correction %s must be a contiguous CUDA %s tensor" % (nm, dt))
        if rowptr.numel() != 3 * self.n + 1:
            raise ValueError("rowptr must have %d entries" % (3 * self.n + 1))
        _check(lib.stokes_op_set_sl_correction(self.handle, int(val.numel()), _ptr(rowptr),
                                               _ptr(col), _ptr(val), _stream(stream)))

    def mobility_rhs(self, F, T, us=None, prec="fp64", stream=None):
        """u_s - S nu for body forces F and torques T ((nbody, 3) each, torque about each
        body's weighted centroid); us: slip velocity on the nodes or None."""
        F = np.asarray(F, dtype=np.float64).reshape(self.nbody, 3)
        T = np.asarray(T, dtype=np.float64).reshape(self.nbody, 3)
        ft = np.concatenate([F, T], axis=1).reshape(-1)
        c_ft = (ctypes.c_double * ft.size)(*ft.tolist())
        if us is not None:
            _dev(us, self.vshape, "us")
        rhs = torch.empty(self.vshape, dtype=torch.float64, device=self.device)
        _check(lib.stokes_mobility_rhs(self.handle, c_ft, _ptr(us), _ptr(rhs), _prec(prec),
                                       _stream(stream)))
        return rhs

    def mobility_velocity(self, sigma, stream=None):
        """V = -L sigma as (nbody, 6): centroid velocity U, then angular velocity Omega."""
        _dev(sigma, self.vshape, "sigma")
        uw = (ctypes.c_double * (6 * self.nbody))()
        _check(lib.stokes_mobility_velocity(self.handle, _ptr(sigma), uw, _stream(stream)))
        return np.array(uw[:]).reshape(self.nbody, 6)

    def matvec_bounded(self, sigma, stream=None):
        """(K sigma in double-float, per-entry bound on its rounding error)."""
        _dev(sigma, self.vshape, "sigma")
        out = torch.empty_like(sigma)
        bnd = torch.empty_like(sigma)
        _check(lib.stokes_matvec_bounded(self.handle, _ptr(sigma), _ptr(out), _ptr(bnd),
                                         _stream(stream)))
        return out, bnd

    def solve(self, rhs, x0=None, tol=1e-10, restart=100, max_iter=2000, inner_prec="fp64",
              inner_tol=1e-5, max_outer=30, use_graph=True, resid_prec="fp64", stream=None):
        """GMRES for K x = rhs; returns (x, report dict).  inner_prec fp64 / df32: plain
        GMRES in that precision; fp32 / fp32c: iterative refinement whose residuals are
        formed in resid_prec (fp64 or df32)."""
        _dev(rhs, self.vshape, "rhs")
        x = torch.zeros_like(rhs) if x0 is None else x0.clone()
        _dev(x, self.vshape, "x0")
        o = GmresOpts(float(tol), int(restart), int(max_iter), _prec(inner_prec), float(inner_tol),
                      int(max_outer), 1 if use_graph else 0, _prec(resid_prec))
        rep = GmresReport()
        st = lib.gmres_solve(self.handle, _ptr(rhs), _ptr(x), ctypes.byref(o), ctypes.byref(rep),
                             _stream(stream))
        if st not in (OK, ENOCONV):
            _check(st)
        d = rep.as_dict()
        d["status_name"] = _STATUS.get(st, st)
        return x, d

    def time_pairsum(self, sigma, prec="fp32c", reps=1, out=None, stream=None):
        """(pair-sum kernel ms, whole apply ms), means over reps applies, from CUDA events
        recorded on the stream around the kernel launch and around the apply."""
        _dev(sigma, self.vshape, "sigma")
        if out is None:
            out = torch.empty(self.vshape, dtype=torch.float64, device=sigma.device)
        _dev(out, self.vshape, "out")
        k, a = _dbl(), _dbl()
        _check(lib.sbq_op_time_pairsum(self.handle, _ptr(sigma), _ptr(out), _prec(prec), int(reps),
                                       _stream(stream), ctypes.byref(k), ctypes.byref(a)))
        return k.value, a.value

    def autotune(self, prec, stream=None):
        t = Tune()
        _check(lib.sbq_autotune(self.handle, _prec(prec), ctypes.byref(t), _stream(stream)))
        return t.as_dict()

    def tune(self, prec):
        t = Tune()
        _check(lib.sbq_op_tune(self.handle, _prec(prec), ctypes.byref(t)))
        return t.as_dict()

    def stats(self, prec):
        k, p = _int(), _dbl()
        _check(lib.sbq_op_stats(self.handle, _prec(prec), ctypes.byref(k), ctypes.byref(p)))
        return dict(kernels_per_matvec=k.value, pairs_per_matvec=p.value)


class LaplaceOp(StokesOp):
    """K sigma = diag sigma + (D + eta S)[sigma] + E sigma for the Laplace layers (Eq.
    laplace-bie-new), scalar densities of shape (n,); same methods as StokesOp."""

    _ncomp = 1
    _create = "laplace_op_create"


def apply_host(src, nrm, w, sigma, eta, diag=0.5, prec="fp32c", tune=None, out=None,
               stream=None):
    """stokes_apply_host: K sigma = diag sigma + (D + eta S)[sigma] on the nodes from HOST
    tensors (CPU float64; pinned memory gives asynchronous copies), result in a host tensor.
    tune: dict(r, warps, chunk_tiles) or None (tuning cache, else the default shape)."""
    n = src.shape[1]
    for a, nm, sh in ((src, "src", (3, n)), (nrm, "nrm", (3, n)), (w, "w", (n,)),
                      (sigma, "sigma", (3, n))):
        _host(a, sh, nm)
    if out is None:
        out = torch.empty((3, n), dtype=torch.float64, pin_memory=torch.cuda.is_available())
    _host(out, (3, n), "out")
    t = None
    if tune is not None:
        t = Tune(int(tune["r"]), int(tune["warps"]), int(tune.get("chunk_tiles", 0)))
    _check(lib.stokes_apply_host(n, _ptr(src), _ptr(nrm), _ptr(w), float(eta), float(diag),
                                 _ptr(sigma), _ptr(out), _prec(prec),
                                 ctypes.byref(t) if t is not None else None, _stream(stream)))
    return out


def solve_host(src, nrm, w, rhs, eta, diag=0.5, body_off=None, corr_prec=None, x0=None,
               tol=1e-10, restart=100, max_iter=2000, inner_prec="fp32c", inner_tol=1e-5,
               max_outer=30, use_graph=True, resid_prec="fp64", stream=None):
    """stokes_solve_host: GMRES for K x = rhs from HOST tensors, solution in a host tensor.
    corr_prec None: no correction; else the double-layer singularity subtraction over the
    bodies body_off (default one body) with row sums in that precision.  Returns
    (x, report dict)."""
    n = src.shape[1]
    for a, nm, sh in ((src, "src", (3, n)), (nrm, "nrm", (3, n)), (w, "w", (n,)),
                      (rhs, "rhs", (3, n))):
        _host(a, sh, nm)
    x = torch.zeros((3, n), dtype=torch.float64, pin_memory=torch.cuda.is_available())
    if x0 is not None:
        x.copy_(x0)
    nbody, c_off, cp = 0, None, FP64
    if corr_prec is not None:
        off = np.asarray([0, n] if body_off is None else body_off, dtype=np.int64)
        nbody = int(off.size - 1)
        c_off = (ctypes.c_int64 * off.size)(*[int(v) for v in off])
        cp = _prec(corr_prec)
    o = GmresOpts(float(tol), int(restart), int(max_iter), _prec(inner_prec), float(inner_tol),
                  int(max_outer), 1 if use_graph else 0, _prec(resid_prec))
    rep = GmresReport()
    st = lib.stokes_solve_host(n, _ptr(src), _ptr(nrm), _ptr(w), float(eta), float(diag), nbody,
                               c_off, cp, _ptr(rhs), _ptr(x), ctypes.byref(o), ctypes.byref(rep),
                               _stream(stream))
    if st not in (OK, ENOCONV):
        _check(st)
    d = rep.as_dict()
    d["status_name"] = _STATUS.get(st, st)
    return x, d

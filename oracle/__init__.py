"""CPU FP64 oracle for the Stokes boundary-integral hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only the tests, the smoke check (`__graft_entry__.smoke`) and the CPU-baseline
leg of `bench.py` use it.  It shares no code with the CUDA library; the only
module both sides use is the seeded input generator
(`paper_2310_00889_gb300.inputs`), which holds none of the method's arithmetic.

Contents
  * pair sums (C, `stokes_oracle.c`): single layer, double layer, combined field,
    sparse correction apply, the combined-field operator K = diag I + D + eta S + E
    (paper Sec. 3.2.1 Eq. nystrom-no-correction / nystrom-correction,
    Eqs. stokes-sl / stokes-dl / stokes-bie-new);
  * `laplace`: the Laplace single / double layer / combined field (Sec. 4.1), scalar;
  * `mobility_solve`: the slender combined-field mobility formulation (Sec. 4.2) with the
    rigid-motion projector built from a Gram--Schmidt basis;
  * `dense_operator`: the same kernels written a second time with numpy, as an
    explicit 3N x 3N matrix, for tiny systems;
  * `gmres`: restarted GMRES(m) with classical Gram--Schmidt applied twice and
    Givens rotations (the paper uses unpreconditioned GMRES, Sec. 4, without
    giving restart or orthogonalisation details);
  * `dl_gauss_correction`: the double-layer singularity subtraction written as a
    sparse correction E (per closed body, from the Gauss-type identity D[e] = -e/2
    on the surface);
  * `tube_quadrature` (module): the quadrature correction E of tube elements (Sec.
    3.2.1-3.2.4): modal angular weights, near-singular and singular rules in s, the
    sparse E over whole tubes;
  * `gen_chebyshev` (module): the generalized Chebyshev rules of Appendix B and the
    compressed angular rules of Sec. 3.2.2 built with them;
  * `eta_slender`: the slender-body mixing parameter 1 / (2 eps log(1/eps))
    (Sec. 4.1, Laplace and Stokes slender combined-field formulations).

Every pin of these functions lives in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stokes_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64


def build(force=False) -> str:
    """Compile the C oracle with gcc (OpenMP) into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.oracle_stokes_combined.argtypes = [_i64, _d, _d, _d, _d, _i64, _d,
                                                   ctypes.c_double, ctypes.c_double, _d]
            lib.oracle_csr_apply.argtypes = [_i64, _i64p, _i64p, _d, _d, _d]
            lib.oracle_stokes_matvec.argtypes = [_i64, _d, _d, _d, ctypes.c_double,
                                                 ctypes.c_double, _i64, _i64p, _i64p, _d,
                                                 _d, _d]
            lib.oracle_laplace_combined.argtypes = [_i64, _d, _d, _d, _d, _i64, _d,
                                                    ctypes.c_double, ctypes.c_double, _d]
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(_d) if a is not None else None


def _c(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def combined(src, nrm, w, sigma, trg, alpha, beta):
    """u = sum_s [alpha S + beta D](x_t - y_s) w_s sigma_s over y_s != x_t; returns (3, nt)."""
    lib = _load()
    src = _c(src)
    ns = src.shape[1]
    trg = _c(trg)
    nt = trg.shape[1]
    w = _c(w, (ns,))
    sigma = _c(sigma, (3, ns))
    nrm = _c(nrm, (3, ns)) if nrm is not None else None
    if beta != 0.0 and nrm is None:
        raise ValueError("double layer needs normals")
    u = np.empty((3, nt))
    lib.oracle_stokes_combined(ns, _p(src), _p(nrm), _p(w), _p(sigma), nt, _p(trg),
                               float(alpha), float(beta), _p(u))
    return u


def combined_extended(src, nrm, w, sigma, trg, alpha, beta):
    """The same sum as `combined`, evaluated in numpy long double (64-bit significand on
    x86, 113-bit on aarch64), row by row with numpy; for few targets.  Used where the FP64
    evaluation's own rounding (r = x - y from absolute coordinates) is not small next to
    the error being checked."""
    ld = np.longdouble
    src = np.asarray(src, dtype=ld)
    trg = np.asarray(trg, dtype=ld)
    w = np.asarray(w, dtype=ld)
    q = np.asarray(sigma, dtype=ld) * w[None, :]
    nrm = np.asarray(nrm, dtype=ld) if nrm is not None else None
    pi = ld("3.14159265358979323846264338327950288")
    out = np.empty((3, trg.shape[1]), dtype=ld)
    for t in range(trg.shape[1]):
        r = trg[:, t:t + 1] - src
        r2 = np.sum(r * r, axis=0)
        keep = r2 != 0
        r, r2, qq = r[:, keep], r2[keep], q[:, keep]
        rl = np.sqrt(r2)
        rq = np.sum(r * qq, axis=0)
        u = np.zeros(3, dtype=ld)
        if alpha != 0:
            u += ld(alpha) / (8 * pi) * (np.sum(qq / rl, axis=1) + np.sum(r * (rq / (r2 * rl)), axis=1))
        if beta != 0:
            rn = np.sum(r * nrm[:, keep], axis=0)
            u += ld(beta) * 3 / (4 * pi) * np.sum(r * (rn * rq / (r2 * r2 * rl)), axis=1)
        out[:, t] = u
    return out


def laplace(src, nrm, w, sigma, trg, alpha, beta):
    """Laplace u = sum_s (alpha G + beta dG/dn_y)(x_t, y_s) w_s sigma_s over y_s != x_t, scalar
    sigma (ns,) and u (nt,) (paper Sec. 4.1; double-layer sign in stokes_oracle.c)."""
    lib = _load()
    src = _c(src)
    ns = src.shape[1]
    trg = _c(trg)
    nt = trg.shape[1]
    w = _c(w, (ns,))
    sigma = _c(sigma, (ns,))
    nrm = _c(nrm, (3, ns)) if nrm is not None else None
    if beta != 0.0 and nrm is None:
        raise ValueError("double layer needs normals")
    u = np.empty(nt)
    lib.oracle_laplace_combined(ns, _p(src), _p(nrm), _p(w), _p(sigma), nt, _p(trg),
                                float(alpha), float(beta), _p(u))
    return u


def sl(src, w, sigma, trg):
    """Single-layer potential S[sigma] (paper Eq. stokes-sl), uncorrected Nystrom sum."""
    return combined(src, None, w, sigma, trg, 1.0, 0.0)


def dl(src, nrm, w, sigma, trg):
    """Double-layer potential D[sigma] (paper Eq. stokes-dl, sign reading in stokes_oracle.c)."""
    return combined(src, nrm, w, sigma, trg, 0.0, 1.0)


class CSR:
    """Sparse correction matrix E with component-major (c * n + node) rows and columns."""

    def __init__(self, rowptr, col, val, nrows, ncols):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int64)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.nrows, self.ncols = int(nrows), int(ncols)

    @property
    def nnz(self):
        return int(self.val.shape[0])


def csr_apply(E: CSR, x, y):
    """y += E x (in place on a float64 contiguous y)."""
    lib = _load()
    x = _c(x).reshape(-1)
    assert y.dtype == np.float64 and y.flags.c_contiguous
    lib.oracle_csr_apply(E.nrows, E.rowptr.ctypes.data_as(_i64p), E.col.ctypes.data_as(_i64p),
                         _p(E.val), _p(x), _p(y))
    return y


def matvec(src, nrm, w, eta, sigma, diag=0.5, E: CSR | None = None):
    """K sigma = diag sigma + (D + eta S)[sigma] + E sigma on the nodes (paper Eq. stokes-bie-new)."""
    lib = _load()
    src = _c(src)
    n = src.shape[1]
    nrm = _c(nrm, (3, n))
    w = _c(w, (n,))
    sigma = _c(sigma, (3, n))
    out = np.empty((3, n))
    if E is not None and E.nnz > 0:
        lib.oracle_stokes_matvec(n, _p(src), _p(nrm), _p(w), float(eta), float(diag), E.nnz,
                                 E.rowptr.ctypes.data_as(_i64p), E.col.ctypes.data_as(_i64p),
                                 _p(E.val), _p(sigma), _p(out))
    else:
        lib.oracle_stokes_matvec(n, _p(src), _p(nrm), _p(w), float(eta), float(diag), 0, None,
                                 None, None, _p(sigma), _p(out))
    return out


def dl_gauss_correction(src, nrm, w, body_off=None) -> CSR:
    """Double-layer singularity subtraction as a sparse E (local form of the correction
    of Eq. nystrom-correction).

    The double layer of a constant density is -e/2 on a closed surface, so
    D[sigma](x_i) = D[sigma - sigma_i](x_i) - sigma_i / 2 on the node's own body.  With
    the punctured sum for D and diag = 1/2 this is the correction
    E_ii = -R_i - I/2 (3 x 3 block), R_i = sum_{j in own body, j != i} D(x_i, y_j; n_j) w_j.
    R_i is taken column by column as the double layer of the unit densities e_b over the
    body alone.  Rows and columns are component-major (c * n + node); each row holds
    its node's three columns in ascending order.
    """
    src = _c(src)
    n = src.shape[1]
    nrm = _c(nrm, (3, n))
    w = _c(w, (n,))
    off = [0, n] if body_off is None else [int(v) for v in body_off]
    R = np.zeros((3, 3, n))            # R[a, b, i]
    for lo, hi in zip(off[:-1], off[1:]):
        if hi <= lo:
            continue
        for b in range(3):
            e = np.zeros((3, hi - lo))
            e[b] = 1.0
            R[:, b, lo:hi] = dl(src[:, lo:hi], nrm[:, lo:hi], w[lo:hi], e, src[:, lo:hi])
    rows = 3 * n
    rowptr = 3 * np.arange(rows + 1, dtype=np.int64)
    col = np.empty(9 * n, dtype=np.int64)
    val = np.empty(9 * n)
    for a in range(3):
        for i in range(n):
            r = a * n + i
            for b in range(3):
                col[3 * r + b] = b * n + i
                val[3 * r + b] = -R[a, b, i] - (0.5 if a == b else 0.0)
    return CSR(rowptr, col, val, rows, rows)


def rigid_basis(x, w, centre):
    """Orthonormal basis of the rigid motions of one body in the quadrature L^2 inner product
    <f, g> = sum w f . g (paper Sec. 4.2: the three translations and the three rotations about
    the centre, orthonormalised by Gram--Schmidt).  Returns (6, 3, nb)."""
    d = x - np.asarray(centre, dtype=np.float64)[:, None]
    nb = x.shape[1]
    vecs = []
    for k in range(3):
        v = np.zeros((3, nb))
        v[k] = 1.0
        vecs.append(v)
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        vecs.append(np.cross(e[:, None], d, axis=0))
    ip = lambda f, g: float(np.sum(w * np.sum(f * g, axis=0)))
    out = []
    for v in vecs:
        u = v.copy()
        for q in out:
            u -= ip(q, u) * q
        out.append(u / np.sqrt(ip(u, u)))
    return np.array(out)


def rigid_projector(x, w, body_off, centres):
    """L sigma = sum_i v_i <v_i, sigma>_w over the rigid bases of all bodies (Eq. L)."""
    bases = [rigid_basis(x[:, a:b], w[a:b], centres[i])
             for i, (a, b) in enumerate(zip(body_off[:-1], body_off[1:]))]

    def L(sigma):
        out = np.zeros_like(sigma)
        for i, (a, b) in enumerate(zip(body_off[:-1], body_off[1:])):
            for v in bases[i]:
                out[:, a:b] += float(np.sum(w[a:b] * np.sum(v * sigma[:, a:b], axis=0))) * v
        return out
    return L


def mobility_solve(src, nrm, w, eta, body_off, F, T, us=None, E: CSR | None = None, tol=1e-11,
                   restart=100, max_iter=2000, E_S: CSR | None = None):
    """Stokes mobility problem, slender combined-field formulation (Sec. 4.2): completion
    flow nu (on each body the rigid motion alpha + beta x (x - c) whose quadrature force and
    torque about c are F_b, T_b: a 6 x 6 system assembled column by column), right-hand side
    u_s - S nu, GMRES on (K (I - L) + L) sigma, rigid velocity V = -L sigma, and each body's
    (U, Omega) by a least-squares fit of V on its nodes.  Centres: the weighted centroids.
    E corrects the operator K (its eta S + D part), E_S the single layer S nu of the
    right-hand side (the punctured sum plus E_S nu; Eq. nystrom-correction for S alone).
    Returns (UW (nbody, 6), sigma, info)."""
    src = _c(src)
    n = src.shape[1]
    w = _c(w, (n,))
    off = [int(v) for v in body_off]
    nb = len(off) - 1
    cen = [np.sum(w[a:b] * src[:, a:b], axis=1) / np.sum(w[a:b]) for a, b in zip(off[:-1], off[1:])]
    L = rigid_projector(src, w, off, cen)
    nu = np.zeros((3, n))
    for i, (a, b) in enumerate(zip(off[:-1], off[1:])):
        d = src[:, a:b] - cen[i][:, None]
        cols = []
        for k in range(6):
            ab = np.zeros(6)
            ab[k] = 1.0
            v = ab[:3, None] + np.cross(ab[3:][:, None], d, axis=0)
            cols.append(np.concatenate([np.sum(w[a:b] * v, axis=1),
                                        np.sum(w[a:b] * np.cross(d, v, axis=0), axis=1)]))
        ab = np.linalg.solve(np.array(cols).T, np.concatenate([F[i], T[i]]))
        nu[:, a:b] = ab[:3, None] + np.cross(ab[3:][:, None], d, axis=0)
    snu = sl(src, w, nu, src)
    if E_S is not None and E_S.nnz > 0:
        snu = csr_apply(E_S, nu, snu)
    rhs = -snu
    if us is not None:
        rhs = rhs + us

    def A(v):
        s3 = v.reshape(3, n)
        lv = L(s3)
        return (matvec(src, nrm, w, eta, s3 - lv, 0.5, E) + lv).reshape(-1)
    x, info = gmres(A, rhs.reshape(-1), tol=tol, restart=restart, max_iter=max_iter)
    sigma = x.reshape(3, n)
    V = -L(sigma)
    uw = np.zeros((nb, 6))
    for i, (a, b) in enumerate(zip(off[:-1], off[1:])):
        d = src[:, a:b] - cen[i][:, None]
        m = b - a
        M = np.zeros((3 * m, 6))
        for k in range(6):
            ab = np.zeros(6)
            ab[k] = 1.0
            M[:, k] = (ab[:3, None] + np.cross(ab[3:][:, None], d, axis=0)).reshape(-1)
        uw[i] = np.linalg.lstsq(M, V[:, a:b].reshape(-1), rcond=None)[0]
    return uw, sigma, info


def dense_operator(src, nrm, w, trg, alpha, beta):
    """Explicit matrix A (3 nt x 3 ns, component-major) with A sigma = combined(...).

    Written independently of the C code with numpy broadcasting, for tiny inputs only.
    """
    src, trg = np.asarray(src, float), np.asarray(trg, float)
    r = trg[:, :, None] - src[:, None, :]                      # (3, nt, ns)
    r2 = np.sum(r * r, axis=0)
    same = r2 == 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        rl = np.sqrt(r2)
        inv1 = np.where(same, 0.0, 1.0 / rl)
        inv3 = inv1 ** 3
        inv5 = inv1 ** 5
    nt, ns = r2.shape
    A = np.zeros((3, nt, 3, ns))
    eye = np.eye(3)
    for i in range(3):
        for j in range(3):
            blk = np.zeros((nt, ns))
            if alpha != 0.0:
                blk += alpha / (8.0 * np.pi) * (eye[i, j] * inv1 + r[i] * r[j] * inv3)
            if beta != 0.0:
                rdn = np.sum(r * np.asarray(nrm, float)[:, None, :], axis=0)
                blk += beta * 3.0 / (4.0 * np.pi) * rdn * r[i] * r[j] * inv5
            A[i, :, j, :] = blk * np.asarray(w, float)[None, :]
    return A.reshape(3 * nt, 3 * ns)


def eta_slender(eps):
    """Slender-body mixing parameter eta = 1 / (2 eps log(1/eps)), natural log (paper Sec. 4.1)."""
    eps = np.asarray(eps, dtype=np.float64)
    return 1.0 / (2.0 * eps * np.log(1.0 / eps))


def gmres(apply, b, x0=None, tol=1e-10, restart=100, max_iter=2000, true_residual=None):
    """Restarted GMRES(m) for A x = b, FP64.

    Arnoldi with classical Gram--Schmidt applied twice, Givens rotations on the
    Hessenberg matrix, x0 = 0 unless given.  A cycle ends when the Givens
    residual estimate drops to tol * ||b|| or after `restart` steps; the true
    residual ||b - A x|| is then recomputed and the solve stops when it is at most
    tol * ||b||.  Returns (x, info) with info = dict(iters, cycles, rel_res, hist).
    """
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64).reshape(-1)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n), dict(iters=0, cycles=0, rel_res=0.0, hist=[0.0])
    resid = true_residual or (lambda xx: b - apply(xx))
    r = resid(x)
    beta = np.linalg.norm(r)
    hist = [beta / bnorm]
    iters, cycles = 0, 0
    while hist[-1] > tol and iters < max_iter:
        m = min(restart, max_iter - iters)
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            wv = apply(V[j])
            h = V[:j + 1] @ wv
            wv = wv - V[:j + 1].T @ h
            h2 = V[:j + 1] @ wv
            wv = wv - V[:j + 1].T @ h2
            h = h + h2
            hn = np.linalg.norm(wv)
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            for i in range(j):                                   # previous rotations
                a, c = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * c
                H[i + 1, j] = -sn[i] * a + cs[i] * c
            a, c = H[j, j], H[j + 1, j]
            den = np.hypot(a, c)
            cs[j], sn[j] = (1.0, 0.0) if den == 0.0 else (a / den, c / den)
            H[j, j] = cs[j] * a + sn[j] * c
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            iters += 1
            if abs(g[j + 1]) <= tol * bnorm or hn == 0.0:
                break
            V[j + 1] = wv / hn
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):                           # back substitution
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + V[:k].T @ y
        r = resid(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        cycles += 1
        if beta == 0.0:
            break
    return x, dict(iters=iters, cycles=cycles, rel_res=hist[-1], hist=hist)

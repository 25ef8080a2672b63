"""Generalized Chebyshev quadrature rules (paper Appendix B) and the compressed angular rules
of Sec. 3.2.2 built with them.

TEST INFRASTRUCTURE ONLY.  Only the tests use it; it shares no code with the CUDA library.

Appendix B, in the paper's order:
  1. a fine rule (nodes x_i, weights w_i) that integrates products of any two integrands of
     the family (composite Gauss--Legendre; dyadically refined panels where the
     singularity's location is known);
  2. the matrix A_ij = phi_j(x_i) sqrt(w_i), and an orthonormal basis of its column span
     truncated at tolerance eps (here: SVD, dropping singular values below eps times the
     largest one);
  3. a column-pivoted QR of U^T: the first n pivots are the nodes y_1..y_n;
  4. the weights solve sum_j u_i(y_j) omega_j = int u_i, i = 1..n (the transposed
     Vandermonde system of the basis).

Angular rules (Sec. 3.2.2): for the unit circle y(theta) = (cos theta, sin theta, 0) and
targets on the annulus at distance alpha..2 alpha from the point theta = 0, in the plane
normal to the circle there, the integrand family is G(x_k, y(theta)) e^{i l theta},
l = 0..l0 (real and imaginary parts), G = 1/|x - y| (the Laplace single-layer kernel up
to its constant).  Readings: a polar grid of 12 radii (Chebyshev points of [alpha, 2 alpha])
x 24 angles stands for the paper's k0 ~ 600 targets; the fine rule is 32-point GL on the
panels of the refined rule of oracle/tube_quadrature.py with one extra dyadic level.
"""
from __future__ import annotations

import math

import numpy as np


def gl01(n):
    """Gauss--Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def chebyshev_rule(F, x, w, eps, psi=None):
    """Appendix B: from integrand values F (m, k) at the fine nodes x (m,) with weights w (m,),
    a rule (nodes y, weights omega) integrating every column to about eps.  psi (m,) > 0:
    run the construction in the measure psi dx on the functions F / psi (the weights are
    divided by psi at the chosen nodes at the end); for peaked families this makes the L2
    truncation control the integrals, which double precision needs where the paper works in
    quad precision."""
    F = np.asarray(F, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    if psi is not None:
        y, om = chebyshev_rule(F / psi[:, None], x, w * psi, eps)
        sel = np.searchsorted(np.asarray(x), y)
        return y, om / psi[sel]
    sw = np.sqrt(w)
    A = F * sw[:, None]
    U, S, _ = np.linalg.svd(A, full_matrices=False)
    n = int(np.sum(S > eps * S[0]))
    U = U[:, :n]
    import scipy.linalg
    _, _, piv = scipy.linalg.qr(U.T, pivoting=True, mode="economic")
    idx = np.sort(piv[:n])
    Ux = U / sw[:, None]                     # u_i at the fine nodes
    rhs = Ux.T @ w                           # int u_i
    omega = np.linalg.solve(Ux[idx, :].T, rhs)
    return np.asarray(x)[idx], omega


def angular_fine_rule(alpha, q=32, nb=2):
    """Fine rule on [-pi, pi] for targets alpha..2 alpha from theta = 0: q-point GL on panels
    refined dyadically towards 0 down to about alpha / 2."""
    lb = math.pi / nb
    levels = 0 if alpha >= lb else int(math.ceil(math.log2(lb / alpha))) + 1
    edges = [0.0] + [lb / 2.0 ** k for k in range(levels, 0, -1)] + [lb * m for m in range(1, nb + 1)]
    g, gw = gl01(q)
    ph, ws = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        ph.append(lo + (hi - lo) * g)
        ws.append((hi - lo) * gw)
    ph, ws = np.concatenate(ph), np.concatenate(ws)
    return np.concatenate([-ph[::-1], ph]), np.concatenate([ws[::-1], ws])


def annulus_targets(alpha, nr=12, npsi=24):
    """Polar grid on the annulus alpha..2 alpha about (1, 0, 0) in the x-z plane, as offsets
    (dx, dz) from that point (the target is (1 + dx, 0, dz))."""
    rr = alpha * (1.5 + 0.5 * np.cos(np.pi * (np.arange(nr) + 0.5) / nr))
    ps = 2.0 * np.pi * np.arange(npsi) / npsi
    return np.array([[r * math.cos(p), r * math.sin(p)] for r in rr for p in ps]).T


def kernel_components(kind, r, n):
    """Kernel components for offsets r = x - y (3, M) and source normals n: "laplace": 1/|r|;
    "stokes": the six components of the single layer (delta/|r| + r_a r_b/|r|^3) and of the
    double layer ((r . n) r_a r_b / |r|^5), each up to its constant; "stokes_axial_dl": the
    double layer for the normal along the circle's axis (0, 0, 1), the part of a tube's normal
    that a radius varying along the centreline adds."""
    r2 = np.sum(r * r, axis=0)
    rl = np.sqrt(r2)
    if kind == "laplace":
        return [1.0 / rl]
    if kind == "stokes_axial_dl":
        return [r[2] * r[a] * r[b] / (r2 * r2 * rl)
                for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))]
    rn = np.sum(r * n, axis=0)
    out = []
    for a, b in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)):
        out.append((1.0 / rl if a == b else 0.0) + r[a] * r[b] / (rl * r2))
        out.append(rn * r[a] * r[b] / (r2 * r2 * rl))
    return out


def modal_family(x_targets, theta, l0, kind="laplace"):
    """Columns G_c(x_k, y(theta)) cos(l theta) and sin(l theta), l = 0..l0 (sin l = 0 left
    out), for every kernel component c of `kind`; targets given as annulus offsets."""
    y = np.stack([np.cos(theta), np.sin(theta), np.zeros_like(theta)])
    one_m_cos = 2.0 * np.sin(0.5 * theta) ** 2          # 1 - cos(theta) without cancellation
    cols = []
    for k in range(x_targets.shape[1]):
        dx, dz = x_targets[0, k], x_targets[1, k]
        r = np.stack([one_m_cos + dx, -np.sin(theta), np.full_like(theta, dz)])   # x - y(theta)
        for G in kernel_components(kind, r, y):
            for l in range(l0 + 1):
                cols.append(G * np.cos(l * theta))
                if l:
                    cols.append(G * np.sin(l * theta))
    return np.array(cols).T


def angular_rule(alpha, l0, eps, kind="laplace", nr=12, npsi=24):
    """Compressed angular rule for relative distances alpha..2 alpha (Sec. 3.2.2 with App. B):
    nodes (offsets from the closest angle) and weights."""
    th, w = angular_fine_rule(alpha)
    psi = 1.0 / np.sqrt((1.5 * alpha) ** 2 + (2.0 * np.sin(0.5 * th)) ** 2)
    return chebyshev_rule(modal_family(annulus_targets(alpha, nr, npsi), th, l0, kind), th, w, eps,
                          psi=psi)

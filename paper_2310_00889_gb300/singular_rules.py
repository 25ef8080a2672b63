"""Offline generator of the whole-element singular rules in the element parameter t (paper
Sec. 3.2.4, built with the generalized Chebyshev construction of Appendix B) that the
quadrature-correction builder compiles in.

Run once:  python -m paper_2310_00889_gb300.singular_rules
It writes paper_2310_00889_gb300/rules/singular_ns8_l12.txt.

For a target at the element's own GL node t0 = t_i0 the s-integrand of the correction is the
modal angular integral of the kernel times a smooth function of t: it has a logarithmic
singularity at t0, and at distances |t - t0| beyond the radius (in parameter units) it
decays like the point kernel.  A dyadically refined panel rule must refine down to the radius
before the logarithm dominates; these rules integrate the whole element [-1, 1] at once with
a few dozen nodes.

Construction, per aspect-ratio level b (element length / radius in [2^b, 2^(b+1))) and target
position i0:
  * integrands: straight cylinders of radius 1 and half-length h = beta / 2 for 12 aspect
    ratios beta of the level; target on the surface at (t0, theta = 0); the 12 Stokes
    components (single and double layer, whose span holds the Laplace kernels) times
    cos / sin(l theta), l <= l0, integrated over theta
    (dyadic Gauss-Legendre about theta = 0, offsets formed without cancellation); each times
    the Legendre polynomials of degree <= ns + 3 in t (the density's interpolant has degree
    ns - 1; four more for the area element and normal of a curved tube);
  * fine rule in t: each side of t0 split dyadically towards t0 down to a quarter of the
    radius, the panel next to t0 integrated by Gauss-Legendre after t - t0 = h u^6 (exact
    for p log + q), the others by 24-point Gauss-Legendre;
  * compression: the family scaled to unit norm in the measure psi^2 dt, psi = 1 /
    sqrt((1.5 lam)^2 + (t - t0)^2), lam the radius in parameter units; singular value
    decomposition truncated below EPS; nodes by column-pivoted QR of the transposed basis
    among the fine nodes at least 1e-9 lam from t0; weights from the transposed Vandermonde
    system.
The rule for i0 and the mirrored position ns - 1 - i0 are mirror images; both are written.
Offsets delta = t - t0 are stored (not t), so that nodes next to t0 keep their relative
accuracy.
"""
from __future__ import annotations

import math
import os
import sys

import numpy as np

NS = 8                 # GL nodes per element the table serves
L0 = 12                # modes l <= L0: N_theta <= 2 (L0 - 4)
LEV_LO, LEV_HI = -2, 12  # aspect-ratio levels b: length / radius in [2^b, 2^(b+1))
NMAX = 96              # nodes per rule the builder reserves
EPS = 1e-12
N_BETA = 12
EXTRA_DEG = 4
HERE = os.path.dirname(os.path.abspath(__file__))


def _gauss(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def gl_nodes(ns):
    return np.polynomial.legendre.leggauss(ns)[0]


def _side(ell, lam, qg=24, qs=40, grade=6):
    """Offsets and weights on [0, ell] (ell signed) refined towards 0: dyadic panels down to
    |ell| / 2^k <= lam / 4, the innermost by GL after u^grade."""
    a = abs(ell)
    k = 0 if a <= lam / 4.0 else int(math.ceil(math.log2(a / (lam / 4.0))))
    g, gw = _gauss(qg)
    u, uw = _gauss(qs)
    h0 = a / 2.0 ** k
    ds = [h0 * u ** grade]
    ws = [h0 * grade * u ** (grade - 1) * uw]
    for m in range(k, 0, -1):
        lo, hi = a / 2.0 ** m, a / 2.0 ** (m - 1)
        ds.append(lo + (hi - lo) * g)
        ws.append((hi - lo) * gw)
    d = np.concatenate(ds)
    return np.sign(ell) * d, np.concatenate(ws)


def fine_rule(t0, lam):
    """Offsets delta = t - t0 over [-1, 1] and weights (log-singular at delta = 0)."""
    dr, wr = _side(1.0 - t0, lam)
    dl, wl = _side(-1.0 - t0, lam)
    return np.concatenate([dl[::-1], dr]), np.concatenate([wl[::-1], wr])


def _theta_rule(z, q=24):
    """Gauss-Legendre in theta on [-pi, pi] refined dyadically towards 0 down to |z| / 2."""
    lb = 0.5 * math.pi
    lv = 0 if abs(z) >= lb else min(60, int(math.ceil(math.log2(lb / max(abs(z), 1e-300)))) + 1)
    cuts = [0.0] + [lb * 2.0 ** -k for k in range(lv, 0, -1)] + [lb, 2.0 * lb]
    g, gw = _gauss(q)
    t = np.concatenate([a + (b - a) * g for a, b in zip(cuts[:-1], cuts[1:])])
    w = np.concatenate([(b - a) * gw for a, b in zip(cuts[:-1], cuts[1:])])
    return np.concatenate([-t[::-1], t]), np.concatenate([w[::-1], w])


def modal_integrals(z, l0):
    """(12, 2 l0 + 1): the Stokes single- and double-layer components of a unit-radius circle
    at axial offset z from a target on it (theta = 0; the cylinder's radial normal), times
    cos(l theta), l = 0..l0, and sin(l theta), l = 1..l0, integrated over theta."""
    th, w = _theta_rule(z)
    # y - x = (cos - 1, sin, z): cos - 1 = -2 sin^2(theta / 2)
    d = np.stack([-2.0 * np.sin(0.5 * th) ** 2, np.sin(th), np.full_like(th, z)])
    d2 = np.sum(d * d, axis=0)
    dl = np.sqrt(d2)
    dn = d[0] * np.cos(th) + d[1] * np.sin(th)
    comps = []
    for i, j in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)):
        comps.append((1.0 / dl if i == j else 0.0) + d[i] * d[j] / (dl * d2))
        comps.append(dn * d[i] * d[j] / (d2 * d2 * dl))
    G = np.array(comps) * w[None, :]
    modes = [np.cos(l * th) for l in range(l0 + 1)] + [np.sin(l * th) for l in range(1, l0 + 1)]
    return G @ np.array(modes).T


def family(t0, delta, betas, ns, l0):
    """Columns: Legendre P_p(t) (p <= ns - 1 + EXTRA_DEG) times the modal integrals, for every
    cylinder, at the offsets delta."""
    t = t0 + delta
    P = np.polynomial.legendre.legvander(t, ns - 1 + EXTRA_DEG)          # (M, deg + 1)
    cols = []
    for beta in betas:
        h = 0.5 * beta
        I = np.array([modal_integrals(h * d, l0).reshape(-1) for d in delta])   # (M, 18 (2 l0 + 1))
        cols.append((P[:, :, None] * I[:, None, :]).reshape(len(delta), -1))
    return np.concatenate(cols, axis=1)


def _betas(lev, n=N_BETA):
    x = 0.5 * (1.0 - np.cos(np.pi * (np.arange(n) + 0.5) / n))
    return 2.0 ** lev * (1.0 + x)


def rule(lev, i0, ns=NS, l0=L0, eps=EPS):
    """Offsets (t - t_i0) and weights of the rule for aspect-ratio level lev and position i0."""
    import scipy.linalg
    t0 = float(gl_nodes(ns)[i0])
    lam = 2.0 / 2.0 ** (lev + 1)              # radius in parameter units at the level's top
    delta, w = fine_rule(t0, lam)
    psi2 = 1.0 / ((1.5 * lam) ** 2 + delta ** 2)
    wt = w * psi2
    A = family(t0, delta, _betas(lev), ns, l0) / psi2[:, None] * np.sqrt(wt)[:, None]
    nrm = np.linalg.norm(A, axis=0)
    A = A[:, nrm > 1e-12 * nrm.max()]         # members that vanish by symmetry are rounding noise
    A = A / np.linalg.norm(A, axis=0)[None, :]
    Q, sv, _ = scipy.linalg.svd(A, full_matrices=False, lapack_driver="gesdd")
    n = int(np.count_nonzero(sv > eps * sv[0]))
    B = Q[:, :n] / np.sqrt(wt)[:, None]
    # no node closer to t0 than 1e-9 radii: there the double layer's r . n = O(|r|^2) is
    # formed from an O(|r|) offset and a unit normal, and its rounding error (~ eps / |t - t0|)
    # would meet a weight that the graded fine rule never gives such a node
    cand = (np.abs(delta) >= 1e-9 * lam).astype(float)
    _, _, piv = scipy.linalg.qr(B.T * (np.sqrt(wt) * cand)[None, :], pivoting=True, mode="economic")
    sel = np.sort(piv[:n])
    om = np.linalg.solve(B[sel, :].T, B.T @ wt)
    return delta[sel], om / psi2[sel]


def table_path(ns=NS, l0=L0):
    return os.path.join(HERE, "rules", "singular_ns%d_l%d.txt" % (ns, l0))


def generate(ns=NS, l0=L0):
    os.makedirs(os.path.join(HERE, "rules"), exist_ok=True)
    path = table_path(ns, l0)
    tmp = path + ".partial"
    with open(tmp, "w") as f:
        f.write("# whole-element singular rules, ns = %d, l0 = %d, eps = %g; written by "
                "python -m paper_2310_00889_gb300.singular_rules\n" % (ns, l0, EPS))
        f.write("# per (level, i0): 'level i0 n' then n lines 'offset weight' (offset = t - t_i0)\n")
        for lev in range(LEV_LO, LEV_HI + 1):
            for i0 in range((ns + 1) // 2):
                d, w = rule(lev, i0, ns, l0)
                if len(d) > NMAX:
                    raise RuntimeError("level %d i0 %d needs %d nodes (> %d)" % (lev, i0, len(d), NMAX))
                for ii, sg in ((i0, 1.0), (ns - 1 - i0, -1.0)):
                    if sg < 0 and ii == i0:
                        continue
                    dd, ww = (d, w) if sg > 0 else (-d[::-1], w[::-1])
                    f.write("%d %d %d\n" % (lev, ii, len(dd)))
                    for a, b in zip(dd, ww):
                        f.write("%.17e %.17e\n" % (a, b))
                f.flush()
                print("level %d i0 %d: %d nodes" % (lev, i0, len(d)), flush=True)
    os.replace(tmp, path)
    return path


def load(ns=NS, l0=L0):
    """{(level, i0): (offsets, weights)} of the committed table, or None."""
    path = table_path(ns, l0)
    if not os.path.exists(path):
        return None
    out = {}
    lines = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    i = 0
    while i < len(lines):
        lev, i0, n = (int(v) for v in lines[i])
        arr = np.array([[float(a), float(b)] for a, b in lines[i + 1:i + 1 + n]])
        out[(lev, i0)] = (arr[:, 0], arr[:, 1])
        i += n + 1
    return out


if __name__ == "__main__":
    print(generate())

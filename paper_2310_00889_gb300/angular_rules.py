"""Offline generator of the compressed angular quadrature rules (paper Sec. 3.2.2 with the
generalized Chebyshev construction of Appendix B) that the quadrature-correction builder
compiles in.

Run once per mode count:  python -m paper_2310_00889_gb300.angular_rules 12
It writes paper_2310_00889_gb300/rules/angular_l12.txt: for every distance level
lev = 0..52 (relative distance alpha of the target from the source circle in
[2^-lev, 2^(1-lev)), level 0 being [1, 2)) the nodes (angle offsets from the circle point
closest to the target) and weights of a rule that integrates G(x, y(theta)) e^{i l theta},
l <= l0, for every target of the annulus, G running over the components of the Stokes single
and double layers with radial and axial normals (whose span holds the Laplace kernels too).  A table of l0 serves every
N_theta with N_theta / 2 + 1 <= l0.

Construction:
  * fine rule: 32-point Gauss--Legendre on panels of [-pi, pi] refined dyadically towards 0
    down to alpha / 2;
  * family: an 8 x 16 polar grid of targets on the annulus, the 18 Stokes components times
    cos(l theta), sin(l theta): the single layer, and the double layer for a normal along the
    circle's radius and for one along its axis (a tube whose radius or frame varies along
    its centreline tilts the surface normal out of the circle's radial direction; the
    normal never has a component along the circle itself); offsets x - y formed without
    cancellation (1 - cos = 2 sin^2);
  * the construction runs in the measure psi^2 d theta with psi = 1/sqrt((1.5 alpha)^2 +
    4 sin^2(theta/2)) on the functions G/psi^2, each scaled to unit norm in that measure,
    so that a double-precision truncation controls the integrals of these peaked integrands
    of very different sizes (single layer ~1/r, double layer ~alpha/r^3; the paper works in
    quad precision);
  * compression: singular value decomposition of the weighted family matrix, truncated
    below eps times the largest singular value; node selection: column-pivoted QR of the
    transposed basis; weights: the transposed Vandermonde system of the basis.
"""
from __future__ import annotations

import math
import os
import sys

import numpy as np

LEVELS = 52       # levels 0 .. LEVELS: alpha down to 2^-52
NMAX = 128        # nodes per level the builder reserves
EPS = 1e-11
HERE = os.path.dirname(os.path.abspath(__file__))
# the tables compiled into the library; the builder takes the smallest l0 >= N_theta / 2 + 4
# (three modes of slack for the area element and normal of a tube whose radius or frame
# varies along it: their Fourier series in theta go beyond the modes +-1)
L0_TABLES = (12, 16, 20)
L0_SLACK = 3


def _gauss(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _fine(alpha, q=32):
    lb = 0.5 * math.pi
    lv = 0 if alpha >= lb else int(math.ceil(math.log2(lb / alpha))) + 1
    cuts = [0.0] + [lb * 2.0 ** -k for k in range(lv, 0, -1)] + [lb, 2.0 * lb]
    g, gw = _gauss(q)
    t = np.concatenate([a + (b - a) * g for a, b in zip(cuts[:-1], cuts[1:])])
    w = np.concatenate([(b - a) * gw for a, b in zip(cuts[:-1], cuts[1:])])
    return np.concatenate([-t[::-1], t]), np.concatenate([w[::-1], w])


def _family(alpha, t, l0, nr=8, npsi=16):
    radii = alpha * (1.5 + 0.5 * np.cos(np.pi * (np.arange(nr) + 0.5) / nr))
    ang = 2.0 * np.pi * np.arange(npsi) / npsi
    n = np.stack([np.cos(t), np.sin(t), 0.0 * t])
    omc = 2.0 * np.sin(0.5 * t) ** 2
    cs = [np.cos(l * t) for l in range(l0 + 1)]
    sn = [np.sin(l * t) for l in range(1, l0 + 1)]
    cols = []
    for rr in radii:
        for a in ang:
            d = np.stack([omc + rr * math.cos(a), -np.sin(t), np.full_like(t, rr * math.sin(a))])
            d2 = np.sum(d * d, axis=0)
            dl = np.sqrt(d2)
            dn = np.sum(d * n, axis=0)
            for i, j in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)):
                for g in ((1.0 / dl if i == j else 0.0) + d[i] * d[j] / (dl * d2),
                          dn * d[i] * d[j] / (d2 * d2 * dl),
                          d[2] * d[i] * d[j] / (d2 * d2 * dl)):
                    cols.extend(g * c for c in cs)
                    cols.extend(g * s for s in sn)
    return np.array(cols).T


def level_rule(lev, l0, eps=EPS):
    """Nodes and weights for distance level lev (alpha in [2^-lev, 2^(1-lev)))."""
    import scipy.linalg
    alpha = 2.0 ** -lev
    t, w = _fine(alpha)
    psi2 = 1.0 / ((1.5 * alpha) ** 2 + (2.0 * np.sin(0.5 * t)) ** 2)
    wt = w * psi2
    A = _family(alpha, t, l0) / psi2[:, None] * np.sqrt(wt)[:, None]
    norms = np.linalg.norm(A, axis=0)
    A = A[:, norms > 1e-300 * norms.max()]
    A = A / np.linalg.norm(A, axis=0)[None, :]
    Q, sv, _ = scipy.linalg.svd(A, full_matrices=False, lapack_driver="gesdd")
    n = int(np.count_nonzero(sv > eps * sv[0]))
    B = Q[:, :n] / np.sqrt(wt)[:, None]                 # basis functions at the fine nodes
    _, _, piv = scipy.linalg.qr(B.T * np.sqrt(wt)[None, :], pivoting=True, mode="economic")
    sel = np.sort(piv[:n])
    om = np.linalg.solve(B[sel, :].T, B.T @ wt)
    return t[sel], om / psi2[sel]


def table_path(l0):
    return os.path.join(HERE, "rules", "angular_l%d.txt" % l0)


def generate(l0):
    """Write the table of l0, keeping the levels an existing table already holds."""
    os.makedirs(os.path.join(HERE, "rules"), exist_ok=True)
    path = table_path(l0)
    have = {}
    if os.path.exists(path):
        lines = [l for l in open(path) if not l.startswith("#")]
        i = 0
        while i < len(lines):
            lev, n = (int(v) for v in lines[i].split())
            have[lev] = [tuple(float(v) for v in lines[i + 1 + k].split()) for k in range(n)]
            i += n + 1
    tmp = path + ".partial"
    with open(tmp, "w") as f:
        f.write("# compressed angular rules, l0 = %d (N_theta <= %d), eps = %g; written by "
                "python -m paper_2310_00889_gb300.angular_rules %d\n" % (l0, 2 * (l0 - 1), EPS, l0))
        f.write("# per level: 'level n' then n lines 'offset weight'\n")
        for lev in range(0, LEVELS + 1):
            if lev in have:
                rows = have[lev]
            else:
                y, om = level_rule(lev, l0)
                rows = list(zip(y, om))
                print("l0 %d level %d: %d nodes" % (l0, lev, len(rows)), flush=True)
            if len(rows) > NMAX:
                raise RuntimeError("level %d needs %d nodes (> %d)" % (lev, len(rows), NMAX))
            f.write("%d %d\n" % (lev, len(rows)))
            for a, b in rows:
                f.write("%.17e %.17e\n" % (a, b))
            f.flush()
    os.replace(tmp, path)
    return path


def load_l0(l0):
    """(phi, w, cnt) of the table for l0: arrays (LEVELS + 1, NMAX), (LEVELS + 1, NMAX),
    (LEVELS + 1,), or None when no table exists."""
    path = table_path(l0)
    if not os.path.exists(path):
        return None
    phi = np.zeros((LEVELS + 1, NMAX))
    w = np.zeros((LEVELS + 1, NMAX))
    cnt = np.zeros(LEVELS + 1, dtype=np.int32)
    lines = [l for l in open(path) if not l.startswith("#")]
    i = 0
    while i < len(lines):
        lev, n = (int(v) for v in lines[i].split())
        for k in range(n):
            a, b = lines[i + 1 + k].split()
            phi[lev, k], w[lev, k] = float(a), float(b)
        cnt[lev] = n
        i += n + 1
    return phi, w, cnt


def load(nt):
    """(phi, w, cnt, l0): the table the builder compiles in for N_theta = nt (the smallest l0
    >= nt / 2 + 1 + L0_SLACK), or None."""
    for l0 in L0_TABLES:
        if nt // 2 + 1 + L0_SLACK <= l0:
            t = load_l0(l0)
            if t is not None:
                return t + (l0,)
    return None


if __name__ == "__main__":
    for a in (sys.argv[1:] or [str(v) for v in L0_TABLES]):
        print(generate(int(a)))

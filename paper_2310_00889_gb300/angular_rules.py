"""Offline generator of the compressed angular quadrature rules (paper Sec. 3.2.2 with the
generalized Chebyshev construction of Appendix B) read by the quadrature-correction builder.

Run once per N_theta:  python -m paper_2310_00889_gb300.angular_rules 16
It writes paper_2310_00889_gb300/rules/angular_nt16.txt: for every distance level
lev = 1..30 (relative distance alpha of the target from the source circle in
[2^-lev, 2^(1-lev))) the nodes (angle offsets from the circle point closest to the target)
and weights of a rule that integrates G(x, y(theta)) e^{i l theta}, l <= N_theta/2 + 1, for
every target of the annulus, G running over the components of the Stokes single and double
layers (whose span holds the Laplace kernels too).

Construction:
  * fine rule: 32-point Gauss--Legendre on panels of [-pi, pi] refined dyadically towards 0
    down to alpha / 2;
  * family: an 8 x 16 polar grid of targets on the annulus, the 12 Stokes components times
    cos(l theta), sin(l theta); offsets x - y formed without cancellation (1 - cos = 2 sin^2);
  * the construction runs in the measure psi d theta with psi = 1/sqrt((1.5 alpha)^2 +
    4 sin^2(theta/2)) on the bounded functions G/psi, so that a double-precision truncation
    controls the integrals of these peaked integrands (the paper works in quad precision);
  * compression: singular value decomposition of the weighted family matrix, truncated
    below eps times the largest singular value (a column-pivoted QR truncated on its
    diagonal left 1e-7 errors at the deep levels); node selection: column-pivoted QR of the
    transposed basis; weights: the transposed Vandermonde system of the basis.
"""
from __future__ import annotations

import math
import os
import sys

import numpy as np

LEVELS = 30
NMAX = 64          # nodes per level the builder reserves
EPS = 1e-11
HERE = os.path.dirname(os.path.abspath(__file__))


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
                          dn * d[i] * d[j] / (d2 * d2 * dl)):
                    cols.extend(g * c for c in cs)
                    cols.extend(g * s for s in sn)
    return np.array(cols).T


def level_rule(lev, l0, eps=EPS):
    """Nodes and weights for distance level lev (alpha in [2^-lev, 2^(1-lev)))."""
    import scipy.linalg
    alpha = 2.0 ** -lev
    t, w = _fine(alpha)
    psi = 1.0 / np.sqrt((1.5 * alpha) ** 2 + (2.0 * np.sin(0.5 * t)) ** 2)
    wt = w * psi
    A = _family(alpha, t, l0) / psi[:, None] * np.sqrt(wt)[:, None]
    Q, sv, _ = scipy.linalg.svd(A, full_matrices=False, lapack_driver="gesdd")
    n = int(np.count_nonzero(sv > eps * sv[0]))
    B = Q[:, :n] / np.sqrt(wt)[:, None]                 # basis functions at the fine nodes
    _, _, piv = scipy.linalg.qr(B.T * np.sqrt(wt)[None, :], pivoting=True, mode="economic")
    sel = np.sort(piv[:n])
    om = np.linalg.solve(B[sel, :].T, B.T @ wt)
    return t[sel], om / psi[sel]


def generate(nt):
    l0 = nt // 2 + 1
    os.makedirs(os.path.join(HERE, "rules"), exist_ok=True)
    path = os.path.join(HERE, "rules", "angular_nt%d.txt" % nt)
    with open(path, "w") as f:
        f.write("# compressed angular rules, N_theta = %d, l0 = %d, eps = %g; written by "
                "python -m paper_2310_00889_gb300.angular_rules %d\n" % (nt, l0, EPS, nt))
        f.write("# per level: 'level n' then n lines 'offset weight'\n")
        for lev in range(1, LEVELS + 1):
            y, om = level_rule(lev, l0)
            if len(y) > NMAX:
                raise RuntimeError("level %d needs %d nodes (> %d)" % (lev, len(y), NMAX))
            f.write("%d %d\n" % (lev, len(y)))
            for a, b in zip(y, om):
                f.write("%.17e %.17e\n" % (a, b))
            print("level %d: %d nodes" % (lev, len(y)), flush=True)
    return path


def load(nt):
    """(phi, w, cnt): arrays (LEVELS + 1, NMAX), (LEVELS + 1, NMAX), (LEVELS + 1,) with
    level 0 unused, or None when no table exists for this N_theta."""
    path = os.path.join(HERE, "rules", "angular_nt%d.txt" % nt)
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


if __name__ == "__main__":
    print(generate(int(sys.argv[1]) if len(sys.argv) > 1 else 16))

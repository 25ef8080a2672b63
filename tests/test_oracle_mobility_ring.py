"""The oracle's mobility solve with the oracle's quadrature correction reproduces the
sedimentation speed of a rigid ring printed by the paper (Sec. 5.4, Table t:conv-sbt;
tests/golden/ring_sedimentation_speed.txt): a pin of the slender combined-field mobility
formulation (Sec. 4.2) and of the tube quadrature (Sec. 3.2) together, against a value
computed by an independent (semi-analytic) method.

Ring: major radius 1, cross-sectional radius eps = 0.1, 8 elements x 10 Gauss-Legendre x 16
angles; force (0, 0, -1), no torque.  E corrects K = I/2 + D + eta S, E_S corrects the
single layer S nu of the right-hand side.  The torus is invariant under the rotations by
2 pi k / 8 about its axis, which map element 0 onto element k node by node; the oracle
computes the rows of the targets of element 0 and the test places the rotated blocks
R B R^T in the rows of element k (the rows of element k are those blocks by that symmetry).
"""
import math
import os
from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp

import numpy as np
import pytest

from paper_2310_00889_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
P, NS, NT = 8, 10, 16


def _golden():
    out = {}
    for line in open(os.path.join(HERE, "golden", "ring_sedimentation_speed.txt")):
        if line.strip() and not line.startswith("#"):
            e, u = line.split()
            out[float(e)] = float(u)
    return out


def _rows(args):
    import oracle.tube_quadrature as TQ
    x, nrm, w, alpha, beta, targets = args
    return TQ.correction_rows(x, nrm, w, P, NS, NT, "stokes", alpha, beta, 0.5, targets)


def _rot(phi):
    c, s = math.cos(phi), math.sin(phi)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _symmetric_csr(oracle_mod, tor, rows):
    n = tor.size
    per = NS * NT
    E = np.zeros((3 * n, 3 * n))
    for k in range(P):
        R = _rot(2.0 * math.pi * k / P)
        for t0, blocks in rows.items():
            tg = k * per + t0
            for k0, B in blocks:
                kk = (k0 + k) % P
                Br = np.einsum("ac,cdj,bd->abj", R, B.reshape(3, 3, per), R)
                for a in range(3):
                    for b in range(3):
                        E[a * n + tg, b * n + kk * per:b * n + (kk + 1) * per] += Br[a, b]
    nz = [np.nonzero(E[r])[0] for r in range(3 * n)]
    rowptr = np.concatenate([[0], np.cumsum([z.size for z in nz])])
    return oracle_mod.CSR(rowptr, np.concatenate(nz), np.concatenate([E[r, z] for r, z in
                                                                      enumerate(nz)]), 3 * n, 3 * n)


def test_ring_sedimentation_speed(oracle_mod):
    eps = 0.1
    u_exact = _golden()[eps]
    tor = I.torus(1.0, eps, P, NS, NT)
    n = tor.size
    eta = float(oracle_mod.eta_slender(eps))
    per = NS * NT
    chunks = [list(range(a, min(per, a + 10))) for a in range(0, per, 10)]
    jobs = [(tor.x, tor.n, tor.w, al, be, c) for al, be in ((1.0, 0.0), (0.0, 1.0)) for c in chunks]
    with ProcessPoolExecutor(max_workers=min(8, os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_rows, jobs))
    rows_s, rows_d = {}, {}
    for k, part in enumerate(parts):
        (rows_s if k < len(chunks) else rows_d).update(part)
    E_S = _symmetric_csr(oracle_mod, tor, rows_s)
    E_D = _symmetric_csr(oracle_mod, tor, rows_d)
    # E of K = eta S + D (same near elements, so the dense sum has the union pattern)
    dense = lambda E: _to_dense(E, 3 * n)
    Kd = eta * dense(E_S) + dense(E_D)
    nz = [np.nonzero(Kd[r])[0] for r in range(3 * n)]
    E_K = oracle_mod.CSR(np.concatenate([[0], np.cumsum([z.size for z in nz])]), np.concatenate(nz),
                         np.concatenate([Kd[r, z] for r, z in enumerate(nz)]), 3 * n, 3 * n)
    uw, _, info = oracle_mod.mobility_solve(tor.x, tor.n, tor.w, eta, [0, n],
                                            np.array([[0.0, 0.0, -1.0]]), np.zeros((1, 3)),
                                            E=E_K, E_S=E_S, tol=1e-13, restart=200)
    err = abs(-uw[0, 2] - u_exact) / u_exact
    print("ring eps %.0e: U %.15e, relative error %.2e, GMRES %s" % (eps, -uw[0, 2], err, info))
    assert info["rel_res"] <= 1e-13
    assert err <= 1e-12
    # the other five rigid-body components vanish by symmetry
    assert np.abs(uw[0, [0, 1, 3, 4, 5]]).max() <= 1e-12
    # without the corrections the punctured sums are first-order accurate at best
    uw0, _, _ = oracle_mod.mobility_solve(tor.x, tor.n, tor.w, eta, [0, n],
                                          np.array([[0.0, 0.0, -1.0]]), np.zeros((1, 3)), tol=1e-12)
    assert abs(-uw0[0, 2] - u_exact) / u_exact > 1e-4


def _to_dense(E, m):
    D = np.zeros((m, m))
    for r in range(m):
        a, b = E.rowptr[r], E.rowptr[r + 1]
        D[r, E.col[a:b]] = E.val[a:b]
    return D

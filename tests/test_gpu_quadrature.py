"""GPU parity of the quadrature correction E of tube elements (tube_correction, Sec.
3.2.1-3.2.4) against the oracle (oracle/tube_quadrature.py), plus checks of the GPU result
against what the mathematics fixes (Green's identities, a solve with a known solution).

Bar: the entries of E are FP64 quadrature results; the CUDA path and the oracle integrate the
same rules (they may place the outer rule's panels at slightly different nearest parameters,
a difference far below the rules' accuracy), so rows agree to 1e-10 of the row's largest
entry."""
import os
import warnings

import numpy as np
import pytest

from paper_2310_00889_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_ROW = 1e-10


@pytest.fixture(scope="module")
def sbq():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu tests")
    from paper_2310_00889_gb300 import build
    build.build()
    from paper_2310_00889_gb300 import sbq as mod
    return mod


@pytest.fixture(scope="module")
def tq():
    import oracle
    oracle.build()
    from oracle import tube_quadrature
    return tube_quadrature


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


def _csr_host(E, n_rows, n_cols):
    scipy_sparse = pytest.importorskip("scipy.sparse")
    rowptr, col, val = (_np(a) for a in E)
    assert rowptr.shape[0] == n_rows + 1 and rowptr[-1] == col.shape[0] == val.shape[0]
    return scipy_sparse.csr_matrix((val, col, rowptr), shape=(n_rows, n_cols))


def _gpu_rows(M, targets, n, kind):
    out = {}
    for t in targets:
        if kind == "laplace":
            out[int(t)] = M.getrow(int(t)).toarray()[0]
        else:
            out[int(t)] = np.stack([M.getrow(a * n + int(t)).toarray()[0] for a in range(3)])
    return out


CASES = [
    # (geometry, panels, ns, nt, kind, alpha, beta, near_factor, targets)
    ("torus", 16, 8, 32, "laplace", 1.0, 0.0, 0.5, 3),
    ("torus", 16, 8, 32, "laplace", 0.0, 1.0, 0.5, 3),
    ("torus", 16, 8, 32, "stokes", 1.55, 1.0, 0.5, 2),
    ("loop", 48, 8, 16, "stokes", 10.86, 1.0, 0.5, 2),
    ("loop", 48, 8, 16, "laplace", 10.86, 1.0, 1.0, 3),
    # N_theta = 64: 6 x 33 modal outputs, more than the CTA's 128 threads (two per thread)
    ("torus", 8, 8, 64, "stokes", 1.0, 1.0, 0.5, 1),
]


def _geometry(name, panels, ns, nt):
    if name == "torus":
        return I.torus(R0=1.0, eps=0.25, panels=panels, ns=ns, nth=nt)
    return I.random_loop(seed=1, panels=panels, ns=ns, nth=nt)


@pytest.mark.parametrize("geom,panels,ns,nt,kind,alpha,beta,nf,ntg", CASES)
def test_rows_match_oracle(sbq, tq, geom, panels, ns, nt, kind, alpha, beta, nf, ntg):
    S = _geometry(geom, panels, ns, nt)
    n = S.size
    E = sbq.tube_correction(_t(S.x), _t(S.n), _t(S.w), panels, ns, nt, kind=kind, alpha=alpha,
                            beta=beta, near_factor=nf)
    nr = n if kind == "laplace" else 3 * n
    M = _csr_host(E, nr, nr)
    rng = np.random.default_rng(7)
    # targets: random nodes plus the first and last GL node of an element (next to its
    # neighbours) and a node of the first element (its neighbour wraps around the loop)
    k2 = min(9, panels - 1)
    tg = list(rng.choice(n, ntg, replace=False)) + [5 * ns * nt + 3, k2 * ns * nt + (ns - 1) * nt + 1, 2]
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        ref = tq.correction_dense_rows(tq.correction_rows(S.x, S.n, S.w, panels, ns, nt, kind, alpha,
                                                          beta, nf, tg), n, kind)
    got = _gpu_rows(M, tg, n, kind)
    per = ns * nt
    worst = 0.0
    for t in tg:
        a, b = got[int(t)], ref[int(t)]
        assert np.count_nonzero(b) > 0
        err = np.abs(a - b).max() / np.abs(b).max()
        worst = max(worst, err)
        # the row's support: the same near elements
        blocks = lambda r: {k for k in range(panels)
                            if np.any(r.reshape(-1, n)[:, k * per:(k + 1) * per] != 0)}
        assert blocks(a) == blocks(b)
    print("%s %s alpha %g beta %g: worst row error %.3e" % (geom, kind, alpha, beta, worst))
    assert worst <= TOL_ROW


def test_csr_layout_and_two_phase_count(sbq):
    """Rows are component-major over all nodes, nodes past the tubes get empty rows, and
    the count of the first phase equals the entries written."""
    import torch
    S = I.torus(R0=1.0, eps=0.25, panels=8, ns=6, nth=16)
    sph = I.sphere(0.2, centre=(0.0, 0.0, 1.5), nphi=6, nth=8)
    allx = np.concatenate([S.x, sph.x], axis=1)
    alln = np.concatenate([S.n, sph.n], axis=1)
    allw = np.concatenate([S.w, sph.w])
    ntot, ntube = allx.shape[1], S.size
    rowptr, col, val = sbq.tube_correction(_t(allx), _t(alln), _t(allw), 8, 6, 16, kind="stokes",
                                           alpha=1.0, beta=1.0, near_factor=0.5)
    rp = _np(rowptr)
    assert rp.shape[0] == 3 * ntot + 1 and rp[0] == 0 and np.all(np.diff(rp) >= 0)
    for a in range(3):
        lens = np.diff(rp[a * ntot:(a + 1) * ntot + 1])
        assert np.all(lens[ntube:] == 0)
        assert np.all(lens[:ntube] % (3 * 6 * 16) == 0) and np.all(lens[:ntube] > 0)
    c = _np(col)
    assert c.min() >= 0 and c.max() < 3 * ntot
    assert np.all(np.isfinite(_np(val)))
    # every column of a row lies on the tube nodes of some component
    assert np.all((c % ntot) < ntube)
    torch.cuda.synchronize()


# The point source / force sits at the centre of the torus, 0.75 from the tube: the data
# (and so the identity) is then resolved by 32 angles to ~1e-12 at every node.  A source 0.4
# from the tube leaves ~1e-8 of interpolation error in the data next to it, whatever the
# quadrature (the oracle shows the same there).
X0 = np.zeros(3)


def _laplace_identity_error(sbq, S, panels, ns, nt, nf, x0=X0):
    n = S.size
    d = S.x - x0[:, None]
    r = np.linalg.norm(d, axis=0)
    u, dudn = 1.0 / r, -np.sum(d * S.n, axis=0) / r ** 3
    ES = _csr_host(sbq.tube_correction(_t(S.x), _t(S.n), _t(S.w), panels, ns, nt, kind="laplace",
                                       alpha=1.0, beta=0.0, near_factor=nf), n, n)
    ED = _csr_host(sbq.tube_correction(_t(S.x), _t(S.n), _t(S.w), panels, ns, nt, kind="laplace",
                                       alpha=0.0, beta=1.0, near_factor=nf), n, n)
    Sp = _np(sbq.laplace_apply(_t(S.x), _t(S.n), _t(S.w), _t(dudn), _t(S.x), 1.0, 0.0, prec="fp64"))
    Dp = _np(sbq.laplace_apply(_t(S.x), _t(S.n), _t(S.w), _t(u), _t(S.x), 0.0, 1.0, prec="fp64"))
    corr = np.abs(Sp + ES @ dudn - Dp - ED @ u - 0.5 * u).max() / np.abs(u).max()
    punct = np.abs(Sp - Dp - 0.5 * u).max() / np.abs(u).max()
    return corr, punct


def test_laplace_green_identity_all_nodes(sbq):
    """u / 2 = S[du/dn] - D[u] at EVERY node of the torus with the GPU-built corrections
    (on-surface Green's identity, Eq. greens-rep): ~1e-10 against 1e-2 punctured."""
    S = I.torus(R0=1.0, eps=0.25, panels=16, ns=8, nth=32)
    corr, punct = _laplace_identity_error(sbq, S, 16, 8, 32, 0.5)
    print("laplace identity: corrected %.3e punctured %.3e" % (corr, punct))
    assert punct > 1e-3
    assert corr < 1e-10


def _stokes_identity_error(sbq, S, panels, ns, nt, nf, x0=X0):
    n = S.size
    F = np.array([0.5, -1.0, 0.7])
    r = S.x - x0[:, None]
    rl = np.linalg.norm(r, axis=0)
    rf = F @ r
    u = (F[:, None] / rl + r * rf / rl ** 3) / (8.0 * np.pi)
    trac = -(3.0 / (4.0 * np.pi)) * r * rf * np.sum(r * S.n, axis=0) / rl ** 5
    ES = _csr_host(sbq.tube_correction(_t(S.x), _t(S.n), _t(S.w), panels, ns, nt, kind="stokes",
                                       alpha=1.0, beta=0.0, near_factor=nf), 3 * n, 3 * n)
    ED = _csr_host(sbq.tube_correction(_t(S.x), _t(S.n), _t(S.w), panels, ns, nt, kind="stokes",
                                       alpha=0.0, beta=1.0, near_factor=nf), 3 * n, 3 * n)
    Sp = _np(sbq.sl_apply(_t(S.x), _t(S.w), _t(trac), _t(S.x), prec="fp64"))
    Dp = _np(sbq.dl_apply(_t(S.x), _t(S.n), _t(S.w), _t(u), _t(S.x), prec="fp64"))
    lhs = Sp + (ES @ trac.reshape(-1)).reshape(3, n) - Dp - (ED @ u.reshape(-1)).reshape(3, n)
    corr = np.abs(lhs - 0.5 * u).max() / np.abs(u).max()
    punct = np.abs(Sp - Dp - 0.5 * u).max() / np.abs(u).max()
    return corr, punct


def test_stokes_green_identity_all_nodes(sbq):
    """u / 2 = S[f] - D[u] at every node for the flow of an exterior point force (Appendix A
    representation, on-surface limit), with the GPU-built Stokes corrections."""
    S = I.torus(R0=1.0, eps=0.25, panels=16, ns=8, nth=32)
    corr, punct = _stokes_identity_error(sbq, S, 16, 8, 32, 0.5)
    print("stokes identity: corrected %.3e punctured %.3e" % (corr, punct))
    assert punct > 1e-3
    assert corr < 1e-10


def _spmv(E, n, x):
    """E x on the device (E: rowptr, col, val of an n x n CSR matrix)."""
    import torch
    M = torch.sparse_csr_tensor(E[0], E[1], E[2], size=(n, n))
    return _np((M @ _t(np.ascontiguousarray(x).reshape(-1, 1))).reshape(-1))


def test_green_identities_on_slender_random_loop_all_nodes(sbq):
    """Both Green's identities at EVERY node of the slender random loop of Sec. 5.2 (512
    panels x 8 x 16 = 65,536 nodes, radius 0.005..0.015, length 58; near factor 1.0), with the
    GPU-built E in its default configuration (trapezoidal, compressed and dyadic angular rules
    chosen per s-node): a check of the builder against the mathematics rather than against
    the oracle.  Source point / point force at the loop's centroid, 0.49 from the tube; the
    loop passes itself at a gap of 2.5 radii near s = 0.107.  Measured: Laplace 1.0e-10,
    Stokes 2.3e-9 (256 panels: 9e-9 and 4.3e-7, the discretization converging); with near
    factor 0.5 the smooth rule just outside the near region limits both to ~3e-8."""
    import torch
    panels, ns, nt = 512, 8, 16
    S = I.random_loop(seed=1, panels=panels, ns=ns, nth=nt)
    n = S.size
    x0 = S.x.mean(axis=1)
    args = (_t(S.x), _t(S.n), _t(S.w), panels, ns, nt)
    d = S.x - x0[:, None]
    r = np.linalg.norm(d, axis=0)
    u, dudn = 1.0 / r, -np.sum(d * S.n, axis=0) / r ** 3
    Sp = _np(sbq.laplace_apply(_t(S.x), _t(S.n), _t(S.w), _t(dudn), _t(S.x), 1.0, 0.0, prec="fp64"))
    Dp = _np(sbq.laplace_apply(_t(S.x), _t(S.n), _t(S.w), _t(u), _t(S.x), 0.0, 1.0, prec="fp64"))
    lhs = Sp + _spmv(sbq.tube_correction(*args, kind="laplace", alpha=1.0, beta=0.0, near_factor=1.0), n, dudn)
    lhs -= Dp + _spmv(sbq.tube_correction(*args, kind="laplace", alpha=0.0, beta=1.0, near_factor=1.0), n, u)
    lap = np.abs(lhs - 0.5 * u).max() / np.abs(u).max()
    lap_p = np.abs(Sp - Dp - 0.5 * u).max() / np.abs(u).max()
    F = np.array([0.5, -1.0, 0.7])
    rf = F @ d
    uu = (F[:, None] / r + d * rf / r ** 3) / (8.0 * np.pi)
    tr = -(3.0 / (4.0 * np.pi)) * d * rf * np.sum(d * S.n, axis=0) / r ** 5
    Sp = _np(sbq.sl_apply(_t(S.x), _t(S.w), _t(tr), _t(S.x), prec="fp64"))
    Dp = _np(sbq.dl_apply(_t(S.x), _t(S.n), _t(S.w), _t(uu), _t(S.x), prec="fp64"))
    lhs = Sp + _spmv(sbq.tube_correction(*args, kind="stokes", alpha=1.0, beta=0.0, near_factor=1.0),
                     3 * n, tr.reshape(-1)).reshape(3, n)
    torch.cuda.empty_cache()
    lhs -= Dp + _spmv(sbq.tube_correction(*args, kind="stokes", alpha=0.0, beta=1.0, near_factor=1.0),
                      3 * n, uu.reshape(-1)).reshape(3, n)
    torch.cuda.empty_cache()
    sto = np.abs(lhs - 0.5 * uu).max() / np.abs(uu).max()
    sto_p = np.abs(Sp - Dp - 0.5 * uu).max() / np.abs(uu).max()
    print("slender loop identities, every node: laplace %.3e (punctured %.3e), stokes %.3e "
          "(punctured %.3e)" % (lap, lap_p, sto, sto_p))
    assert lap_p > 1e-2 and sto_p > 1e-2
    assert lap < 5e-10 and sto < 1e-8


def test_laplace_exterior_solve_with_quadrature_correction(sbq):
    """Exterior Dirichlet problem on the torus (Eqs. laplace-dirichlet0..2) with the
    quadrature correction in the operator (alpha = eta, beta = 1): the combined-field
    representation of the solution reproduces the point charge's potential outside to
    ~1e-9 (the punctured operator: 1e-2)."""
    t = I.torus(1.0, 0.25, 16, 8, 32)
    eta = sbq.slender_eta(0.25)
    x0 = np.array([1.0, 0.05, 0.02])
    G = lambda x: 1.0 / (4 * np.pi * np.linalg.norm(x - x0[:, None], axis=0))
    b = G(t.x)
    E = sbq.tube_correction(_t(t.x), _t(t.n), _t(t.w), 16, 8, 32, kind="laplace", alpha=eta,
                            beta=1.0, near_factor=0.5)
    pts = np.array([[1.6, 0.2, 0.3], [-0.2, 1.7, -0.4], [0.0, 0.0, 0.8]]).T
    errs = {}
    for name, corr in (("quadrature", E), ("punctured", None)):
        op = sbq.LaplaceOp(_t(t.x), _t(t.n), _t(t.w), eta, correction=corr)
        x, rep = op.solve(_t(b), tol=1e-12, restart=100, inner_prec="fp64")
        assert rep["status"] == 0, rep
        u = _np(sbq.laplace_apply(_t(t.x), _t(t.n), _t(t.w), x, _t(pts), eta, 1.0, prec="fp64"))
        errs[name] = np.abs(u - G(pts)).max() / np.abs(G(pts)).max()
        op.close()
    print("exterior solve field error: %s" % errs)
    assert errs["punctured"] > 1e-4
    assert errs["quadrature"] < 1e-8


def test_invalid_arguments(sbq):
    S = I.torus(R0=1.0, eps=0.25, panels=4, ns=8, nth=16)
    x, n, w = _t(S.x), _t(S.n), _t(S.w)
    with pytest.raises(sbq.SbqError):
        sbq.tube_correction(x, n, w, 4, 8, 15)          # odd nt
    with pytest.raises(sbq.SbqError):
        sbq.tube_correction(x, n, w, 5, 8, 16)          # more tube nodes than nodes
    # rows that are not circles: shift one node off its circle
    xb = S.x.copy()
    xb[2, 5] += 1e-3
    with pytest.raises(sbq.SbqError):
        sbq.tube_correction(_t(xb), n, w, 4, 8, 16)


def test_paper_torus_table_all_nodes(sbq):
    """Sec. 5.1, Table t:conv-biest (tests/golden/torus_green_identity_table.txt): on the
    paper's torus and discretisations (N_s = 10), the on-surface Green's identity with the
    GPU-built corrections holds at EVERY node to at least the printed accuracy."""
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                          "torus_green_identity_table.txt")
    rows = [tuple(l.split()) for l in open(golden) if l.strip() and not l.startswith("#")]
    x0 = np.array([1.0, 2.0, 3.0])
    got = []
    for nu, ne, nt, printed in rows:
        nu, ne, nt, printed = int(nu), int(ne), int(nt), float(printed)
        S = I.torus(R0=1.0, eps=0.25, panels=ne, ns=10, nth=nt)
        assert S.size == nu
        d = S.x - x0[:, None]
        r = np.linalg.norm(d, axis=0)
        u = 1.0 / (4.0 * np.pi * r)
        dudn = -np.sum(d * S.n, axis=0) / (4.0 * np.pi * r ** 3)
        ES = _csr_host(sbq.tube_correction(_t(S.x), _t(S.n), _t(S.w), ne, 10, nt, kind="laplace",
                                           alpha=1.0, beta=0.0, near_factor=0.5), nu, nu)
        ED = _csr_host(sbq.tube_correction(_t(S.x), _t(S.n), _t(S.w), ne, 10, nt, kind="laplace",
                                           alpha=0.0, beta=1.0, near_factor=0.5), nu, nu)
        Sp = _np(sbq.laplace_apply(_t(S.x), _t(S.n), _t(S.w), _t(dudn), _t(S.x), 1.0, 0.0, prec="fp64"))
        Dp = _np(sbq.laplace_apply(_t(S.x), _t(S.n), _t(S.w), _t(u), _t(S.x), 0.0, 1.0, prec="fp64"))
        err = float(np.abs(Sp + ES @ dudn - Dp - ED @ u - 0.5 * u).max() / np.abs(u).max())
        got.append((nu, err, printed))
        assert err <= printed, (nu, err, printed)
    print("paper torus table (N, ours, printed): %s" % got)


def _near_surface_points(S, m, seed):
    rng = np.random.default_rng(seed)
    idx = rng.choice(S.size, m, replace=False)
    h = 10.0 ** rng.uniform(-4, -1, m)
    return S.x[:, idx] - h * S.n[:, idx]


def test_offsurface_rows_match_oracle(sbq, tq):
    S = I.torus(R0=1.0, eps=0.25, panels=16, ns=8, nth=32)
    n = S.size
    trg = _near_surface_points(S, 3, 21)
    trg = np.concatenate([trg, S.x[:, [100, 2000]] + 0.05 * S.n[:, [100, 2000]]], axis=1)  # outside too
    m = trg.shape[1]
    for kind, alpha, beta in (("laplace", 1.0, 1.0), ("stokes", 1.55, 1.0)):
        E = sbq.tube_correction_targets(_t(S.x), _t(S.n), _t(S.w), 16, 8, 32, _t(trg), kind=kind,
                                        alpha=alpha, beta=beta, near_factor=0.5)
        nr = m if kind == "laplace" else 3 * m
        nc = n if kind == "laplace" else 3 * n
        M = _csr_host(E, nr, nc)
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            ref = tq.correction_dense_rows(tq.correction_rows_offsurface(S.x, S.n, S.w, 16, 8, 32, kind, alpha,
                                                                         beta, 0.5, trg), n, kind)
        worst = 0.0
        for k in range(m):
            a = (M.getrow(k).toarray()[0] if kind == "laplace"
                 else np.stack([M.getrow(c * m + k).toarray()[0] for c in range(3)]))
            worst = max(worst, np.abs(a - ref[k]).max() / np.abs(ref[k]).max())
        print("off-surface %s rows: worst %.3e" % (kind, worst))
        assert worst <= TOL_ROW


def test_near_surface_interior_representation(sbq):
    """u = S[du/dn] - D[u] (Laplace) and u = S[f] - D[u] (Stokes, exterior point force) at
    200 points between 1e-4 and 1e-1 inside the torus surface, with the GPU-built
    near-singular corrections: 1e-11 (Laplace) and 1e-10 (Stokes), against 1e4 for the plain
    sums."""
    S = I.torus(R0=1.0, eps=0.25, panels=16, ns=8, nth=32)
    n = S.size
    trg = _near_surface_points(S, 200, 22)
    m = trg.shape[1]
    x0 = X0
    d = S.x - x0[:, None]
    r = np.linalg.norm(d, axis=0)
    u, dudn = 1.0 / r, -np.sum(d * S.n, axis=0) / r ** 3
    ex = 1.0 / np.linalg.norm(trg - x0[:, None], axis=0)
    ES = _csr_host(sbq.tube_correction_targets(_t(S.x), _t(S.n), _t(S.w), 16, 8, 32, _t(trg), kind="laplace",
                                               alpha=1.0, beta=0.0, near_factor=0.5), m, n)
    ED = _csr_host(sbq.tube_correction_targets(_t(S.x), _t(S.n), _t(S.w), 16, 8, 32, _t(trg), kind="laplace",
                                               alpha=0.0, beta=1.0, near_factor=0.5), m, n)
    Sp = _np(sbq.laplace_apply(_t(S.x), _t(S.n), _t(S.w), _t(dudn), _t(trg), 1.0, 0.0, prec="fp64"))
    Dp = _np(sbq.laplace_apply(_t(S.x), _t(S.n), _t(S.w), _t(u), _t(trg), 0.0, 1.0, prec="fp64"))
    lap = np.abs(Sp + ES @ dudn - Dp - ED @ u - ex).max() / np.abs(u).max()
    lap_plain = np.abs(Sp - Dp - ex).max() / np.abs(u).max()
    F = np.array([0.5, -1.0, 0.7])
    rf = F @ d
    uu = (F[:, None] / r + d * rf / r ** 3) / (8.0 * np.pi)
    trac = -(3.0 / (4.0 * np.pi)) * d * rf * np.sum(d * S.n, axis=0) / r ** 5
    dt = trg - x0[:, None]
    rt = np.linalg.norm(dt, axis=0)
    uex = (F[:, None] / rt + dt * (F @ dt) / rt ** 3) / (8.0 * np.pi)
    KS = _csr_host(sbq.tube_correction_targets(_t(S.x), _t(S.n), _t(S.w), 16, 8, 32, _t(trg), kind="stokes",
                                               alpha=1.0, beta=0.0, near_factor=0.5), 3 * m, 3 * n)
    KD = _csr_host(sbq.tube_correction_targets(_t(S.x), _t(S.n), _t(S.w), 16, 8, 32, _t(trg), kind="stokes",
                                               alpha=0.0, beta=1.0, near_factor=0.5), 3 * m, 3 * n)
    sp = _np(sbq.sl_apply(_t(S.x), _t(S.w), _t(trac), _t(trg), prec="fp64"))
    dp = _np(sbq.dl_apply(_t(S.x), _t(S.n), _t(S.w), _t(uu), _t(trg), prec="fp64"))
    lhs = sp + (KS @ trac.reshape(-1)).reshape(3, m) - dp - (KD @ uu.reshape(-1)).reshape(3, m)
    sto = np.abs(lhs - uex).max() / np.abs(uu).max()
    sto_plain = np.abs(sp - dp - uex).max() / np.abs(uu).max()
    print("near-surface interior representation: laplace %.3e (plain %.3e), stokes %.3e (plain %.3e)"
          % (lap, lap_plain, sto, sto_plain))
    assert lap_plain > 1e-1 and sto_plain > 1e-1
    # at 1e-4 from the surface r = x - y formed from absolute coordinates keeps ~12 digits,
    # and the double layer's (r.n)/r^3 structure leaves ~1e-10 (the oracle: 2e-11..3e-9 at
    # depths 1e-4..1e-5)
    assert lap < 1e-10 and sto < 5e-10


def test_compressed_angular_rules_match_dyadic(sbq):
    """The builder's compiled-in compressed angular rules (Sec. 3.2.2 with Appendix B) give
    the E of the dyadically refined rules (rules="none"): same pattern, every row within
    1e-10 of its largest entry, Laplace and Stokes; a caller's copy of the same table
    (angular_rules.load) gives the compiled-in result bit for bit."""
    import time
    import torch
    from paper_2310_00889_gb300 import angular_rules
    rules = angular_rules.load(16)
    assert rules is not None and rules[3] >= 9
    # aspect 0.1: the area element's zero-free strip (acosh(10) ~ 3.0, estimated 2.65) admits
    # the compressed rules (a fatter torus keeps the dyadic rule, whose result would be the
    # same bit for bit)
    S = I.torus(R0=1.0, eps=0.1, panels=16, ns=8, nth=16)
    for kind, a, b in (("laplace", 1.0, 1.0), ("stokes", 1.55, 1.0)):
        args = (_t(S.x), _t(S.n), _t(S.w), 16, 8, 16)
        Ed = sbq.tube_correction(*args, kind=kind, alpha=a, beta=b, near_factor=0.5, rules="none")
        Ec = sbq.tube_correction(*args, kind=kind, alpha=a, beta=b, near_factor=0.5)
        Er = sbq.tube_correction(*args, kind=kind, alpha=a, beta=b, near_factor=0.5, rules=rules)
        assert np.array_equal(_np(Ed[0]), _np(Ec[0])) and np.array_equal(_np(Ed[1]), _np(Ec[1]))
        assert np.array_equal(_np(Ec[2]), _np(Er[2]))
        vd, vr = _np(Ed[2]), _np(Ec[2])
        rp = _np(Ed[0])
        worst = max(np.abs(vd[rp[r]:rp[r + 1]] - vr[rp[r]:rp[r + 1]]).max() / np.abs(vd[rp[r]:rp[r + 1]]).max()
                    for r in range(len(rp) - 1) if rp[r + 1] > rp[r])
        print("compressed rules, %s: worst row difference %.3e" % (kind, worst))
        assert worst <= 1e-10
        assert not np.array_equal(vd, vr)     # the compressed rules were taken
    L = I.random_loop(seed=1, panels=128, ns=8, nth=16)
    args = (_t(L.x), _t(L.n), _t(L.w), 128, 8, 16)
    times = {}
    for name, r in (("dyadic", "none"), ("compressed", None)):
        sbq.tube_correction(*args, kind="stokes", alpha=10.86, beta=1.0, rules=r)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sbq.tube_correction(*args, kind="stokes", alpha=10.86, beta=1.0, rules=r)
        torch.cuda.synchronize()
        times[name] = time.perf_counter() - t0
    print("Stokes E build, 16384-node loop: dyadic %.3f s, compressed %.3f s" % (times["dyadic"], times["compressed"]))


def test_compressed_rules_near_surface_deep_levels(sbq):
    """Off-surface targets 1e-9..1e-2 inside a torus of aspect 0.1 (relative distances 1e-8..
    0.1: compressed-rule levels 4..27, where the area element's zero-free strip admits them),
    above random points of the surface:
    the interior Laplace representation u = S[du/dn] - D[u] holds with the default rules, and
    the default E agrees with the dyadic rules' E (rules="none") row by row."""
    S = I.torus(R0=1.0, eps=0.1, panels=16, ns=8, nth=16)
    n = S.size
    rng = np.random.default_rng(31)
    # points of the exact torus at random angles (between the nodes: a target just above a
    # node would leave the plain sum a term ~ w / depth^2 that the correction must cancel
    # in double precision) moved inwards along the normal
    m = 120
    ph, th = 2.0 * np.pi * rng.random(m), 2.0 * np.pi * rng.random(m)
    nrm = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), np.sin(th)])
    y = np.stack([np.cos(ph), np.sin(ph), np.zeros(m)]) + 0.1 * nrm
    h = 10.0 ** rng.uniform(-9, -2, m)
    trg = y - h * nrm
    x0 = X0
    d = S.x - x0[:, None]
    r = np.linalg.norm(d, axis=0)
    u, dudn = 1.0 / r, -np.sum(d * S.n, axis=0) / r ** 3
    ex = 1.0 / np.linalg.norm(trg - x0[:, None], axis=0)
    args = (_t(S.x), _t(S.n), _t(S.w), 16, 8, 16, _t(trg))
    Sp = _np(sbq.laplace_apply(_t(S.x), _t(S.n), _t(S.w), _t(dudn), _t(trg), 1.0, 0.0, prec="fp64"))
    Dp = _np(sbq.laplace_apply(_t(S.x), _t(S.n), _t(S.w), _t(u), _t(trg), 0.0, 1.0, prec="fp64"))
    errs = {}
    for name, rules in (("compressed", None), ("dyadic", "none")):
        ES = _csr_host(sbq.tube_correction_targets(*args, kind="laplace", alpha=1.0, beta=0.0,
                                                   near_factor=1.0, rules=rules), m, n)
        ED = _csr_host(sbq.tube_correction_targets(*args, kind="laplace", alpha=0.0, beta=1.0,
                                                   near_factor=1.0, rules=rules), m, n)
        errs[name] = (np.abs(Sp + ES @ dudn - Dp - ED @ u - ex).max() / np.abs(u).max(), ES, ED)
    # row by row, relative to the row's largest entry
    diff = 0.0
    for k in (1, 2):
        a, b = errs["compressed"][k].toarray(), errs["dyadic"][k].toarray()
        diff = max(diff, (np.abs(a - b).max(axis=1) / np.abs(b).max(axis=1)).max())
    print("near-surface, aspect-0.1 torus, depths 1e-9..1e-2: representation %.3e (compressed), "
          "%.3e (dyadic); E difference %.3e" % (errs["compressed"][0], errs["dyadic"][0], diff))
    # the oracle on the same targets: up to 6.3e-9 at depths near 1e-9 (the discretized
    # surface is the exact torus only to interpolation accuracy), 1.5e-10 at 1e-7
    assert errs["dyadic"][0] < 2e-8 and errs["compressed"][0] < 2e-8
    # measured 1.5e-9 (row-relative; the tables integrate their family to 1e-11 of its
    # largest member, and a row of these near-singular weights sums much larger terms)
    assert diff < 5e-9 and diff > 0.0

"""Pins of the CPU oracle against facts the paper and Stokes theory fix (no GPU).

Each test names the passage it relies on.  Together they are chosen so that a
plausible slip in the oracle -- a dropped r r^T term, a wrong 1/(8 pi) or
3/(4 pi), the printed double-layer sign, a wrong power of |r|, a transposed or
reversed r, a missing self-skip, a broken Givens update -- fails at least one.
"""
import os

import numpy as np
import pytest

from paper_2310_00889_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rep(v, n):
    return np.repeat(np.asarray(v, float)[:, None], n, axis=1)


def _stokeslet_field(x, x0, f):
    """Free-space Stokeslet velocity of a point force f at x0 (viscosity 1), used only as
    boundary data and exact solution of the exterior Dirichlet problem."""
    r = x - x0[:, None]
    rl = np.linalg.norm(r, axis=0)
    return (f[:, None] / rl + r * np.sum(r * f[:, None], axis=0) / rl ** 3) / (8 * np.pi)


# ---------------------------------------------------------------------------
# Single layer (paper Eq. stokes-sl)
# ---------------------------------------------------------------------------

def test_sl_sphere_uniform_density(oracle_mod):
    """A uniform force density f on a sphere of radius a moves the enclosed fluid rigidly with
    u = (2a/3) f (Stokes drag F = 6 pi a U, viscosity 1, Sec. 2).  The I/|r| term alone gives
    a/2, the r r^T/|r|^3 term alone a/6: a dropped term, a wrong prefactor or a wrong power
    of |r| fails here.  Spectral convergence: 40 x 60 nodes reach ~1e-13."""
    a = 0.7
    sp = I.sphere(a, (0.1, 0.2, 0.3), 40, 60)
    f = np.array([0.3, -1.2, 0.5])
    trg = np.array([[0.1, 0.2, 0.3], [0.3, 0.1, 0.4], [0.1, -0.2, 0.1], [0.35, 0.25, 0.2]]).T
    u = oracle_mod.sl(sp.x, sp.w, _rep(f, sp.size), trg)
    assert np.abs(u - 2 * a / 3 * f[:, None]).max() < 1e-12


def test_sl_reciprocity(oracle_mod):
    """S(r) is symmetric and even in r, so <w_X tau, S_{XY}[w_Y sigma]> = <w_Y sigma, S_{YX}[w_X tau]>.
    A transposed tensor index or an odd-in-r term breaks this to O(1)."""
    X = I.torus(1.0, 0.25, 4, 8, 16)
    Y = I.sphere(0.6, (0.2, -2.0, 0.5), 10, 14)
    tau = I.density(X.size, seed=11)
    sig = I.density(Y.size, seed=12)
    uX = oracle_mod.sl(Y.x, Y.w, sig, X.x)
    vY = oracle_mod.sl(X.x, X.w, tau, Y.x)
    lhs = np.sum(X.w * np.sum(tau * uX, axis=0))
    rhs = np.sum(Y.w * np.sum(sig * vY, axis=0))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


def test_sl_dl_divergence_free(oracle_mod):
    """Both layer potentials are Stokes velocity fields (Sec. 2), hence divergence-free off the
    surface.  The I/|r| term alone has divergence -f.r/|r|^3 != 0.  4th-order central
    differences with h = 1e-3 at interior points of the straight pipe."""
    c = I.config1()
    s = c["surf"]
    pts = I.interior_points_straight(6, seed=9, margin=0.3)
    h = 1e-3

    def div(fun):
        d = 0.0
        for k in range(3):
            e = np.zeros((3, 1))
            e[k] = h
            d = d + (-fun(pts + 2 * e)[k] + 8 * fun(pts + e)[k] - 8 * fun(pts - e)[k]
                     + fun(pts - 2 * e)[k]) / (12 * h)
        return d

    for fun in (lambda p: oracle_mod.sl(s.x, s.w, c["sigma"], p),
                lambda p: oracle_mod.dl(s.x, s.n, s.w, c["sigma"], p)):
        scale = np.abs(fun(pts)).max()
        assert np.abs(div(fun)).max() < 1e-7 * scale / h


# ---------------------------------------------------------------------------
# Double layer (paper Eq. stokes-dl; sign reading from Eq. stokes-bie-new, Prop. p:null,
# Appendix A)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("geom", ["torus", "sphere", "capped_pipe"])
def test_dl_gauss_identity(oracle_mod, geom):
    """D applied to a constant density e gives -e inside a closed surface and 0 outside
    (interior Green's representation u = S[T] - D[u] of Appendix A with u = e, T = 0).  The
    sign printed in Eq. stokes-dl would give +e inside."""
    e = np.array([1.0, 2.0, -0.5])
    if geom == "torus":
        s = I.torus(1.0, 0.25, 32, 8, 48)
        tin = np.array([[1.0, 0, 0.0], [0, 1.05, 0.1], [-0.9, 0.1, -0.05]]).T
        tout = np.array([[0, 0, 0.0], [2.0, 0, 0], [0, 0, 1.0]]).T
        tol = 1e-7
    elif geom == "sphere":
        s = I.sphere(1.3, (0.5, -0.2, 0.1), 40, 60)
        tin = np.array([[0.5, -0.2, 0.1], [0.9, 0.2, 0.3], [0.0, -0.5, -0.2]]).T
        tout = np.array([[3.0, 0, 0.0], [0.5, 2.0, 0.5], [-1.5, -1.5, 1.0]]).T
        tol = 1e-11
    else:
        s = I.capped_straight_pipe(1.0, 4.0, 16, 8, 48, 24)
        tin = np.array([[0, 0, 2.0], [0.5, 0.2, 1.0], [0, -0.3, 3.0]]).T
        tout = np.array([[2.5, 0, 2.0], [0, 0, 5.5], [-2.0, 1.0, -1.0]]).T
        tol = 1e-7
    uin = oracle_mod.dl(s.x, s.n, s.w, _rep(e, s.size), tin)
    uout = oracle_mod.dl(s.x, s.n, s.w, _rep(e, s.size), tout)
    assert np.abs(uin + e[:, None]).max() < tol
    assert np.abs(uout).max() < tol


def test_dl_rigid_rotation(oracle_mod):
    """A rigid rotation v = omega x (y - c) has zero traction, so Appendix A gives
    -D[v] = v inside and D[v] = 0 outside.  Unlike the constant-density identity this also
    sees the position dependence of the density (wrong r, swapped operands)."""
    c = np.array([0.1, -0.3, 0.2])
    om = np.array([0.4, -1.0, 0.7])
    s = I.sphere(1.0, c, 40, 60)
    v = np.cross(om[:, None], s.x - c[:, None], axis=0)
    tin = c[:, None] + np.array([[0.2, 0.1, -0.3], [-0.4, 0.3, 0.1], [0.0, 0.0, 0.5]]).T
    tout = c[:, None] + np.array([[2.0, 0.1, -0.3], [-0.4, 1.9, 0.1]]).T
    uin = oracle_mod.dl(s.x, s.n, s.w, v, tin)
    uout = oracle_mod.dl(s.x, s.n, s.w, v, tout)
    exact = np.cross(om[:, None], tin - c[:, None], axis=0)
    assert np.abs(uin + exact).max() < 1e-11
    assert np.abs(uout).max() < 1e-11


@pytest.mark.parametrize("res,tol", [((8, 32, 16), 1e-4), ((32, 64, 32), 1e-9)])
def test_poiseuille_green_representation(oracle_mod, res, tol):
    """Exact Poiseuille flow u = (1 - rho^2) e_z, p = -4 z in a capped straight pipe (R = 1,
    viscosity 1) satisfies u = S[T] - D[u] inside (Appendix A), with traction
    T = -p n + (grad u + grad u^T) n: 4 z n + (0, 0, -2) on the wall and
    -+p e_z +- (-2x, -2y, 0) on the caps with outward normal +-e_z.  The error is
    quadrature error at points 0.3 from the wall and must shrink with refinement."""
    panels, nth, nr = res
    cp = I.capped_straight_pipe(1.0, 4.0, panels, 8, nth, nr)
    x, n = cp.x, cp.n
    T = np.zeros_like(x)
    u = np.zeros_like(x)
    for nm, a, b in cp.parts:
        xs, ns_ = x[:, a:b], n[:, a:b]
        if nm == "straight_wall":
            T[:, a:b] = 4 * xs[2] * ns_ + np.array([0, 0, -2.0])[:, None]
        else:
            sgn = ns_[2, 0]
            p = -4 * xs[2, 0]
            T[:, a:b] = np.stack([-2 * xs[0] * sgn, -2 * xs[1] * sgn, -p * sgn * np.ones(b - a)])
            u[2, a:b] = 1 - xs[0] ** 2 - xs[1] ** 2
    trg = I.interior_points_straight(40, seed=7, margin=0.3)
    v = oracle_mod.sl(x, cp.w, T, trg) - oracle_mod.dl(x, n, cp.w, u, trg)
    exact = np.zeros_like(trg)
    exact[2] = 1 - trg[0] ** 2 - trg[1] ** 2
    assert np.abs(v - exact).max() < tol


# ---------------------------------------------------------------------------
# Combined field and the punctured sum
# ---------------------------------------------------------------------------

def test_combined_sphere_closed_form(oracle_mod):
    """Combined field alpha S + beta D on a sphere with constant density e at interior points
    equals (alpha 2a/3 - beta) e: both closed forms above, in one call."""
    a = 0.9
    s = I.sphere(a, (0, 0, 0), 40, 60)
    e = np.array([0.2, -0.7, 1.1])
    trg = np.array([[0.1, 0.2, -0.1], [-0.3, 0.0, 0.2]]).T
    for alpha, beta in ((1.553, 1.0), (0.0, 2.0), (-0.7, 0.0), (2.0, -3.0)):
        u = oracle_mod.combined(s.x, s.n, s.w, _rep(e, s.size), trg, alpha, beta)
        assert np.abs(u - (alpha * 2 * a / 3 - beta) * e[:, None]).max() < 1e-11


def test_self_pair_skipped(oracle_mod):
    """Punctured Nystrom sum (Sec. 3.2.1): a source at the target's position contributes
    nothing, so evaluating at node k with all sources equals evaluating with node k removed,
    bit for bit (the skipped term is never added)."""
    c = I.config1()
    s = c["surf"]
    k = 137
    keep = np.arange(s.size) != k
    trg = s.x[:, k:k + 1]
    for alpha, beta in ((1.0, 0.0), (0.0, 1.0), (1.3, 1.0)):
        full = oracle_mod.combined(s.x, s.n, s.w, c["sigma"], trg, alpha, beta)
        cut = oracle_mod.combined(s.x[:, keep], s.n[:, keep], s.w[keep], c["sigma"][:, keep],
                                  trg, alpha, beta)
        assert np.array_equal(full, cut)
        assert np.all(np.isfinite(full))


def test_rotation_translation_linearity(oracle_mod):
    """Frame invariance of the kernels: rotating points, normals and densities by Q rotates
    the output by Q; translating all points changes nothing; the sum is linear in sigma."""
    c = I.config1()
    s = c["surf"]
    trg = c["trg"][:, 500:560]
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    shift = np.array([[3.0], [-1.0], [0.5]])
    u = oracle_mod.combined(s.x, s.n, s.w, c["sigma"], trg, 1.5, 1.0)
    uq = oracle_mod.combined(Q @ s.x, Q @ s.n, s.w, Q @ c["sigma"], Q @ trg, 1.5, 1.0)
    ut = oracle_mod.combined(s.x + shift, s.n, s.w, c["sigma"], trg + shift, 1.5, 1.0)
    scale = np.abs(u).max()
    assert np.abs(uq - Q @ u).max() < 1e-12 * scale
    assert np.abs(ut - u).max() < 1e-12 * scale
    s2 = I.density(s.size, seed=3)
    u2 = oracle_mod.combined(s.x, s.n, s.w, s2, trg, 1.5, 1.0)
    u12 = oracle_mod.combined(s.x, s.n, s.w, 2.0 * c["sigma"] - 3.0 * s2, trg, 1.5, 1.0)
    assert np.abs(u12 - (2.0 * u - 3.0 * u2)).max() < 1e-12 * scale


def test_c_sum_matches_numpy_dense_operator(oracle_mod):
    """Two independent codings of the same kernels (C loop and numpy matrix) agree."""
    c = I.config1()
    s = c["surf"]
    trg = c["trg"][:, ::5]
    A = oracle_mod.dense_operator(s.x, s.n, s.w, trg, 1.7, 1.0)
    u = oracle_mod.combined(s.x, s.n, s.w, c["sigma"], trg, 1.7, 1.0)
    assert np.abs(A @ c["sigma"].reshape(-1) - u.reshape(-1)).max() < 1e-12 * np.abs(u).max()


def test_extended_precision_rows_match_fp64(oracle_mod):
    """The long-double row evaluator is a third coding of the same sum: on the straight pipe
    (no severe cancellation in x - y) it agrees with the FP64 C loop to FP64 rounding."""
    c = I.config1()
    s = c["surf"]
    trg = c["trg"][:, ::37]
    for alpha, beta in ((1.0, 0.0), (0.0, 1.0), (1.7, 1.0)):
        u = oracle_mod.combined(s.x, s.n, s.w, c["sigma"], trg, alpha, beta)
        v = oracle_mod.combined_extended(s.x, s.n, s.w, c["sigma"], trg, alpha, beta)
        assert np.abs(np.asarray(v, dtype=np.float64) - u).max() <= 1e-13 * np.abs(u).max()


def test_csr_apply_matches_scipy(oracle_mod):
    """Sparse correction apply y += E x (Eq. nystrom-correction) against scipy's CSR product."""
    sp = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(0)
    n = 300
    E = sp.random(3 * n, 3 * n, density=0.01, random_state=1, format="csr")
    x = rng.standard_normal(3 * n)
    y0 = rng.standard_normal(3 * n)
    y = y0.copy()
    csr = oracle_mod.CSR(E.indptr, E.indices, E.data, 3 * n, 3 * n)
    oracle_mod.csr_apply(csr, x, y)
    assert np.abs(y - (y0 + E @ x)).max() < 1e-13


# ---------------------------------------------------------------------------
# Mixing parameter (Sec. 4.1) and GMRES (Sec. 4 / 5)
# ---------------------------------------------------------------------------

def test_eta_matches_printed_values(oracle_mod):
    rows = np.loadtxt(os.path.join(GOLDEN, "eta_dashed_lines.txt"))
    for eps, eta, tol in rows:
        assert abs(float(oracle_mod.eta_slender(eps)) - eta) <= tol


def test_gmres_matches_dense_lu(oracle_mod):
    """Restarted GMRES on the discrete combined-field system K = I/2 + D + eta S (Eq.
    stokes-bie-new) of the 512-node straight pipe agrees with a dense LU solve; also with a
    short restart (m = 12) that forces several true-residual restarts."""
    s = I.config1()["surf"]
    eta = 1.0
    A = oracle_mod.dense_operator(s.x, s.n, s.w, s.x, eta, 1.0) + 0.5 * np.eye(3 * s.size)
    b = I.density(s.size, seed=21).reshape(-1)
    x_lu = np.linalg.solve(A, b)
    mv = lambda v: oracle_mod.matvec(s.x, s.n, s.w, eta, v.reshape(3, -1)).reshape(-1)
    for m in (100, 12):
        x, info = oracle_mod.gmres(mv, b, tol=1e-11, restart=m, max_iter=3000)
        assert info["rel_res"] <= 1e-11
        assert np.abs(x - x_lu).max() <= 1e-8 * np.abs(x_lu).max()
    # the true residual reported equals an independent recomputation
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1.01e-11


def test_exterior_dirichlet_solve_converges(oracle_mod):
    """Exterior Stokes Dirichlet problem (Eqs. stokes-eq0..2, stokes-dirichlet3) with the
    field of a point force inside a unit sphere as data: solve (I/2 + D + S) sigma = u0 with
    GMRES and evaluate (D + S)[sigma] (Eq. stokes-bie-rep-new, eta = 1) outside.  With the
    uncorrected (punctured) on-surface sum the error is first order in h, so halving h halves
    it; a wrong jump term (+/-I/2) or double-layer sign does not converge."""
    x0 = np.array([0.2, 0.1, -0.1])
    f = np.array([1.0, -0.5, 0.3])
    trg = np.array([[2.0, 0.3, 0.1], [0.0, -1.8, 0.5], [1.0, 1.0, 1.5]]).T
    exact = _stokeslet_field(trg, x0, f)
    errs = []
    for nphi, nth in ((20, 30), (40, 60)):
        s = I.sphere(1.0, (0, 0, 0), nphi, nth)
        b = _stokeslet_field(s.x, x0, f).reshape(-1)
        x, info = oracle_mod.gmres(
            lambda v: oracle_mod.matvec(s.x, s.n, s.w, 1.0, v.reshape(3, -1)).reshape(-1),
            b, tol=1e-12, restart=50)
        assert info["rel_res"] <= 1e-12
        u = oracle_mod.combined(s.x, s.n, s.w, x.reshape(3, -1), trg, 1.0, 1.0)
        errs.append(np.abs(u - exact).max() / np.abs(exact).max())
    assert errs[0] < 0.04
    assert 0.4 < errs[1] / errs[0] < 0.6


# ---------------------------------------------------------------------------
# Double-layer singularity subtraction as a sparse correction E (local form of the
# correction of Eq. nystrom-correction; Gauss-type identity of Eq. stokes-dl)
# ---------------------------------------------------------------------------

def _corrected_dl(oracle_mod, s, E, sig):
    """(I/2 + D + E) sigma on the nodes."""
    y = np.ascontiguousarray(0.5 * sig + oracle_mod.dl(s.x, s.n, s.w, sig, s.x))
    oracle_mod.csr_apply(E, sig, y.reshape(-1))
    return y


@pytest.mark.parametrize("geom", ["sphere", "torus"])
def test_gauss_correction_rigid_motions(oracle_mod, geom):
    """On a closed surface the double layer of a rigid motion v is -v/2 (pv value between
    -v inside and 0 outside), so I/2 + D annihilates rigid motions.  The corrected sum
    applies sum_j D_ij (v_j - v_i), and v_j - v_i = w x (y_j - y_i) or 0 is orthogonal to
    r in D's r (r . q) factor: exact to rounding.  The punctured sum misses it by O(h).
    A wrong sign of the I/2 term, a missing or mis-signed row sum fails here."""
    if geom == "sphere":
        s = I.sphere(1.0, (0.1, 0.2, -0.3), 20, 30)
        c0 = np.array([0.1, 0.2, -0.3])
    else:
        s = I.torus(1.0, 0.25, 16, 8, 32)
        c0 = np.zeros(3)
    E = oracle_mod.dl_gauss_correction(s.x, s.n, s.w)
    om = np.array([0.3, -0.7, 0.5])
    rot = np.cross(om[:, None], s.x - c0[:, None], axis=0)
    tr = _rep([0.4, -1.0, 0.8], s.size)
    for v in (rot, tr):
        assert np.abs(_corrected_dl(oracle_mod, s, E, v)).max() < 1e-13
        punct = 0.5 * v + oracle_mod.dl(s.x, s.n, s.w, v, s.x)
        assert np.abs(punct).max() > 1e-3


def test_gauss_correction_normal_field_sphere(oracle_mod):
    """Double layer of the normal field on a sphere of radius a, worked out by hand: with
    (x - y) . n_y = -|x - y|^2 / (2a) the integrand reduces to 3 (x - y) / (16 pi a^2 |x - y|);
    over the sphere (x - y) / |x - y| integrates to (8/3) pi a^2 n_x, so D[n] = n / 2 and
    (I/2 + D)[n] = n.  The corrected sum converges to it at second order (a factor of
    about 3.5 per halving of h)."""
    errs = []
    for nphi, nth in ((10, 15), (20, 30), (40, 60)):
        s = I.sphere(1.0, (0.1, 0.2, -0.3), nphi, nth)
        E = oracle_mod.dl_gauss_correction(s.x, s.n, s.w)
        errs.append(np.abs(_corrected_dl(oracle_mod, s, E, s.n) - s.n).max())
    assert errs[1] < 4e-4
    assert errs[1] / errs[0] < 0.35 and errs[2] / errs[1] < 0.35


def test_gauss_correction_is_per_body(oracle_mod):
    """Row sums run over the node's own closed body only.  Two nested spheres, constant
    density e on both: on the inner sphere the outer one's double layer is the interior
    value -e (Gauss identity, spectrally accurate off-surface), on the outer sphere the
    inner one's is the exterior value 0; the own-body parts vanish exactly.  Row sums over
    all nodes would give 0 on the inner sphere instead."""
    so = I.sphere(1.0, (0, 0, 0), 20, 30)
    si = I.sphere(0.4, (0.1, -0.05, 0.2), 20, 30)
    s = I.concat([so, si])
    no = so.size
    E = oracle_mod.dl_gauss_correction(s.x, s.n, s.w, [0, no, s.size])
    for comp in range(3):
        sig = np.zeros((3, s.size))
        sig[comp] = 1.0
        y = _corrected_dl(oracle_mod, s, E, sig)
        assert np.abs(y[:, :no]).max() < 1e-8
        want = np.zeros((3, s.size - no))
        want[comp] = -1.0
        assert np.abs(y[:, no:] - want).max() < 1e-6


def test_gauss_correction_layout(oracle_mod):
    """Three entries per row, the row node's three components in ascending column order."""
    s = I.capped_straight_pipe(1.0, 4.0, 2, 8, 8, 4)
    E = oracle_mod.dl_gauss_correction(s.x, s.n, s.w)
    n = s.size
    assert E.nrows == 3 * n and E.nnz == 9 * n
    assert np.array_equal(E.rowptr, 3 * np.arange(3 * n + 1))
    r = np.arange(3 * n)
    node = r % n
    for b in range(3):
        assert np.array_equal(E.col[3 * r + b], b * n + node)


def test_gauss_correction_bounds_gmres_iterations(oracle_mod):
    """Second-kind behaviour restored: on a capped arc pipe (flat caps meet the wall at a
    right-angle rim) the punctured double-layer row sums stray far from -1/2 near the rim
    and GMRES needs more iterations as h shrinks; with the correction the count stays
    nearly flat.  Exterior Dirichlet data: a point force inside the pipe."""
    f = np.array([1.0, -0.5, 0.3])
    ang = np.deg2rad(60.0)
    its = {}
    for panels, nth, nr in ((4, 16, 8), (8, 32, 16)):
        s = I.capped_arc_pipe(5.0, ang, 1.0, panels, 8, nth, nr)
        x0 = np.array([5.0 * np.cos(ang / 2) + 0.1, 5.0 * np.sin(ang / 2) + 0.2, 0.1])
        b = _stokeslet_field(s.x, x0, f).reshape(-1)
        E = oracle_mod.dl_gauss_correction(s.x, s.n, s.w)
        for name, EE in (("punctured", None), ("corrected", E)):
            x, info = oracle_mod.gmres(
                lambda v: oracle_mod.matvec(s.x, s.n, s.w, 1.0, v.reshape(3, -1), E=EE).reshape(-1),
                b, tol=1e-10, restart=200, max_iter=1000)
            assert info["rel_res"] <= 1e-10
            its[(name, s.size)] = info["iters"]
    assert its[("corrected", 3072)] <= 60 and its[("corrected", 768)] <= 50
    assert its[("punctured", 3072)] > 2 * its[("corrected", 3072)]


# ---------------------------------------------------------------------------
# Laplace layer potentials (Sec. 4.1) and the torus Green's-identity test (Eq. greens-rep)
# ---------------------------------------------------------------------------

def _torus_green_data(t, x0):
    r = t.x - x0[:, None]
    rl = np.linalg.norm(r, axis=0)
    u = 1.0 / (4 * np.pi * rl)
    dudn = -np.sum(r * t.n, axis=0) / (4 * np.pi * rl ** 3)
    return u, dudn


def test_laplace_sphere_closed_forms(oracle_mod):
    """Unit density on a sphere of radius a: single layer a inside, a^2/|x - c| outside;
    double layer -1 inside, 0 outside (Gauss).  A wrong 1/(4 pi), power of |r| or sign of
    the double layer fails here; spectrally accurate at 40 x 60 nodes."""
    a, c = 0.7, np.array([0.1, 0.2, 0.3])
    sp = I.sphere(a, c, 40, 60)
    one = np.ones(sp.size)
    inn = c[:, None] + np.array([[0.1, -0.2, 0.05], [0.0, 0.3, -0.2]]).T
    out = c[:, None] + np.array([[1.5, 0.2, 0.1], [-0.3, 0.9, 1.2]]).T
    assert np.abs(oracle_mod.laplace(sp.x, None, sp.w, one, inn, 1.0, 0.0) - a).max() < 1e-13
    ext = a ** 2 / np.linalg.norm(out - c[:, None], axis=0)
    assert np.abs(oracle_mod.laplace(sp.x, None, sp.w, one, out, 1.0, 0.0) - ext).max() < 1e-13
    assert np.abs(oracle_mod.laplace(sp.x, sp.n, sp.w, one, inn, 0.0, 1.0) + 1.0).max() < 1e-13
    assert np.abs(oracle_mod.laplace(sp.x, sp.n, sp.w, one, out, 0.0, 1.0)).max() < 1e-13


def test_laplace_torus_green_identity(oracle_mod):
    """The paper's quadrature test (Eq. greens-rep): u = G(x - x0) for a point charge x0
    outside a torus (R = 1, radius 0.25); inside the tube S[du/dn] - D[u] = u (spectral
    convergence: below 1e-10 at 16384 nodes), and on the surface with the punctured sums
    u/2 + S[du/dn] - D[u] -> u at first order (halving h nearly halves the error)."""
    x0 = np.array([1.0, 0.0, 0.45])
    phi = np.linspace(0, 2 * np.pi, 7)[:-1]
    xin = np.stack([np.cos(phi), np.sin(phi), 0.05 * np.ones_like(phi)])
    g_in = 1.0 / (4 * np.pi * np.linalg.norm(xin - x0[:, None], axis=0))
    e_in, e_on = [], []
    for panels, nth in ((8, 16), (16, 32), (32, 64)):
        t = I.torus(1.0, 0.25, panels, 8, nth)
        u, dudn = _torus_green_data(t, x0)
        lhs = (oracle_mod.laplace(t.x, None, t.w, dudn, xin, 1.0, 0.0)
               - oracle_mod.laplace(t.x, t.n, t.w, u, xin, 0.0, 1.0))
        e_in.append(np.abs(lhs - g_in).max() / np.abs(g_in).max())
        on = (0.5 * u + oracle_mod.laplace(t.x, None, t.w, dudn, t.x, 1.0, 0.0)
              - oracle_mod.laplace(t.x, t.n, t.w, u, t.x, 0.0, 1.0))
        e_on.append(np.abs(on - u).max() / np.abs(u).max())
    assert e_in[2] < 1e-10 and e_in[1] < 1e-6 and e_in[0] > e_in[1] > e_in[2]
    assert 0.45 < e_on[1] / e_on[0] < 0.7 and 0.45 < e_on[2] / e_on[1] < 0.7


def test_laplace_combined_is_linear(oracle_mod):
    """alpha S + beta D in one pass equals the two layers combined."""
    c = I.config1()
    s = c["surf"]
    sig = c["sigma"][0]
    trg = c["trg"][:, ::11]
    uc = oracle_mod.laplace(s.x, s.n, s.w, sig, trg, 2.5, -0.75)
    us = oracle_mod.laplace(s.x, None, s.w, sig, trg, 1.0, 0.0)
    ud = oracle_mod.laplace(s.x, s.n, s.w, sig, trg, 0.0, 1.0)
    assert np.abs(uc - (2.5 * us - 0.75 * ud)).max() <= 1e-13 * np.abs(uc).max()


# ---------------------------------------------------------------------------
# Mobility formulation (Sec. 4.2, Eqs. new-mobility-bie, recover-rigidbody-motion)
# ---------------------------------------------------------------------------

def test_rigid_projector_is_orthogonal(oracle_mod):
    """L (Eq. L) is an orthogonal projector in the quadrature inner product that keeps rigid
    motions: L L = L, <L f, g> = <f, L g>, L v = v for v rigid on each body."""
    s = I.concat([I.sphere(0.5, (0, 0, 0), 10, 15), I.torus(1.0, 0.25, 8, 8, 8)])
    off = I.body_offsets(s)
    cen = [np.sum(s.w[a:b] * s.x[:, a:b], axis=1) / np.sum(s.w[a:b]) for a, b in zip(off[:-1], off[1:])]
    L = oracle_mod.rigid_projector(s.x, s.w, off, cen)
    rng = np.random.default_rng(5)
    f, g = rng.standard_normal((2, 3, s.size))
    ip = lambda p, q: float(np.sum(s.w * np.sum(p * q, axis=0)))
    Lf = L(f)
    assert np.abs(L(Lf) - Lf).max() < 1e-12 * np.abs(Lf).max()
    assert abs(ip(Lf, g) - ip(f, L(g))) < 1e-12 * abs(ip(f, g))
    v = np.zeros((3, s.size))
    for i, (a, b) in enumerate(zip(off[:-1], off[1:])):
        d = s.x[:, a:b] - cen[i][:, None]
        v[:, a:b] = rng.standard_normal(3)[:, None] + np.cross(rng.standard_normal(3)[:, None], d, axis=0)
    assert np.abs(L(v) - v).max() < 1e-12 * np.abs(v).max()


@pytest.mark.parametrize("load", ["force", "torque"])
def test_mobility_sphere_stokes_law(oracle_mod, load):
    """A sphere of radius a under a force F translates at U = F / (6 pi a) (Stokes drag,
    viscosity 1) and under a torque T rotates at Omega = T / (8 pi a^3); the slender
    combined-field mobility solve (punctured sums) converges to both at first order (the
    error halves with h) and leaves the other motion at zero."""
    a = 0.5
    errs = []
    for nphi, nth in ((10, 15), (20, 30), (40, 60)):
        sp = I.sphere(a, (0.1, 0.2, 0.3), nphi, nth)
        if load == "force":
            F, T = np.array([[0.3, -0.2, 1.0]]), np.zeros((1, 3))
            want, got, other = F[0] / (6 * np.pi * a), slice(0, 3), slice(3, 6)
        else:
            F, T = np.zeros((1, 3)), np.array([[0.2, 0.5, -0.4]])
            want, got, other = T[0] / (8 * np.pi * a ** 3), slice(3, 6), slice(0, 3)
        uw, _, info = oracle_mod.mobility_solve(sp.x, sp.n, sp.w, 1.0, [0, sp.size], F, T)
        assert info["rel_res"] <= 1e-11 and info["iters"] <= 20
        errs.append(np.linalg.norm(uw[0, got] - want) / np.linalg.norm(want))
        assert np.abs(uw[0, other]).max() < 1e-12 * np.linalg.norm(want)
    assert errs[2] < (0.03 if load == "force" else 0.06)
    assert 0.45 < errs[1] / errs[0] < 0.55 and 0.45 < errs[2] / errs[1] < 0.55

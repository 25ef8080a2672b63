"""Seeded synthetic inputs: slender-tube surfaces, caps, spheres, densities and targets.

This module is the only code shared by the CUDA path and the CPU oracle.  It holds
no arithmetic of the boundary-integral method itself (no kernels, no sums, no
solver): it only builds the quadrature nodes, unit normals and weights that the
method takes as input, plus seeded random densities and target points.

Surface discretisation (paper Sec. 3.1, Eq. (surface-coord) and Sec. 3.2.1):
a tube of radius eps(s) around a centreline x_c(s) is

    y(s, theta) = x_c(s) + eps(s) [e1(s) cos(theta) + e2(s) sin(theta)],  e2 = t x e1,

split into panels in s; each panel carries N_s Gauss--Legendre nodes in s times
N_theta equispaced nodes in theta.  Each node gets the weight
w = J * w_GL * 2*pi / N_theta with J = |d_s y x d_theta y| (paper Sec. 3.2.1,
below the uncorrected Nystrom sum).  Nodes are ordered panel-major, then GL node,
then theta.  The orientation vector e1 is the principal normal for arcs and
helices, a fixed axis for straight pipes, and the solution of the paper's
frame-transport ODE (Sec. 3.1.1) for random closed loops.

Flat end caps and spheres are not in the paper; they close open pipes so that
the closed-surface identities can be checked, and they model the spheres of the
helical-pipe workload.  Caps carry polar nodes (GL in radius x trapezoid in
angle) with weight rho * w_GL * 2*pi / N_theta.

All arrays are float64, structure-of-arrays: points are (3, N).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Surface", "concat", "gl_rule", "straight_pipe", "arc_pipe", "torus", "helix_pipe",
    "random_loop", "sphere", "disk_cap", "pipe_caps", "interior_points_straight",
    "density", "config1", "config2", "config3", "config4", "config5",
]


@dataclasses.dataclass
class Surface:
    """Quadrature nodes of a closed or open surface (SoA, float64)."""
    x: np.ndarray          # (3, N) node positions
    n: np.ndarray          # (3, N) unit outward normals
    w: np.ndarray          # (N,)   quadrature weights (area element included)
    name: str = ""
    parts: tuple = ()      # ((name, start, stop), ...) sub-surfaces in node order

    @property
    def size(self) -> int:
        return int(self.w.shape[0])


def concat(surfaces, name="") -> Surface:
    parts, off = [], 0
    for s in surfaces:
        if s.parts:
            parts.extend((nm, a + off, b + off) for nm, a, b in s.parts)
        else:
            parts.append((s.name, off, off + s.size))
        off += s.size
    return Surface(np.concatenate([s.x for s in surfaces], axis=1),
                   np.concatenate([s.n for s in surfaces], axis=1),
                   np.concatenate([s.w for s in surfaces]), name=name, parts=tuple(parts))


def body_offsets(surf: Surface):
    """Node offsets of the closed bodies of a surface: a pipe wall and the end caps that
    follow it form one body, every other part (a sphere, a torus, a loop) is a body."""
    if not surf.parts:
        return [0, surf.size]
    off = []
    for nm, a, b in surf.parts:
        if not nm.startswith("cap") or not off:
            off.append(a)
    return off + [surf.size]


def gl_rule(n: int):
    """Gauss--Legendre nodes and weights on [-1, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


def _panel_nodes(s_breaks, ns):
    """GL nodes/weights on each panel [s_k, s_{k+1}], flattened panel-major."""
    g, gw = gl_rule(ns)
    a, b = np.asarray(s_breaks[:-1]), np.asarray(s_breaks[1:])
    half = 0.5 * (b - a)
    s = (0.5 * (a + b))[:, None] + half[:, None] * g[None, :]
    ws = half[:, None] * gw[None, :]
    return s.reshape(-1), ws.reshape(-1)


def _cross(a, b):
    return np.cross(a, b, axis=0)


def _unit(v):
    return v / np.linalg.norm(v, axis=0, keepdims=True)


def _tube(s, ws, c, dc, ddc, eps, deps, e1, de1, nth, name):
    """Tube nodes from centreline data sampled at the GL nodes s (all (3,M) / (M,))."""
    sp = np.linalg.norm(dc, axis=0)
    t = dc / sp
    dt = (ddc - np.sum(t * ddc, axis=0) * t) / sp
    e2 = _cross(t, e1)
    de2 = _cross(dt, e1) + _cross(t, de1)
    th = 2.0 * np.pi * np.arange(nth) / nth
    ct, st = np.cos(th)[None, :], np.sin(th)[None, :]          # (1, nth)
    rad = e1[:, :, None] * ct[None] + e2[:, :, None] * st[None]   # (3, M, nth)
    y = c[:, :, None] + eps[None, :, None] * rad
    y_th = eps[None, :, None] * (-e1[:, :, None] * st[None] + e2[:, :, None] * ct[None])
    y_s = (dc[:, :, None] + deps[None, :, None] * rad
           + eps[None, :, None] * (de1[:, :, None] * ct[None] + de2[:, :, None] * st[None]))
    nrm = np.cross(y_th, y_s, axis=0)                          # outward for right-handed (t, e1, e2)
    jac = np.linalg.norm(nrm, axis=0)
    nrm = nrm / jac
    flip = np.sum(nrm * rad, axis=0) < 0
    nrm[:, flip] *= -1.0
    w = jac * ws[:, None] * (2.0 * np.pi / nth)
    m = s.shape[0]
    return Surface(y.reshape(3, m * nth), nrm.reshape(3, m * nth), w.reshape(m * nth), name=name)


def straight_pipe(R=1.0, L=4.0, panels=4, ns=8, nth=16) -> Surface:
    """Open cylinder wall of radius R along z in [0, L]."""
    s, ws = _panel_nodes(np.linspace(0.0, 1.0, panels + 1), ns)
    m = s.size
    c = np.stack([np.zeros(m), np.zeros(m), L * s])
    dc = np.stack([np.zeros(m), np.zeros(m), np.full(m, L)])
    ddc = np.zeros((3, m))
    e1 = np.stack([np.ones(m), np.zeros(m), np.zeros(m)])
    return _tube(s, ws, c, dc, ddc, np.full(m, R), np.zeros(m), e1, np.zeros((3, m)), nth,
                 "straight_wall")


def _arc_centreline(s, Rc, phi0, phi1):
    dphi = phi1 - phi0
    p = phi0 + dphi * s
    cp, sp = np.cos(p), np.sin(p)
    z = np.zeros_like(s)
    c = Rc * np.stack([cp, sp, z])
    dc = Rc * dphi * np.stack([-sp, cp, z])
    ddc = -Rc * dphi ** 2 * np.stack([cp, sp, z])
    e1 = np.stack([-cp, -sp, z])                 # principal normal (towards the arc centre)
    de1 = dphi * np.stack([sp, -cp, z])
    return c, dc, ddc, e1, de1


def arc_pipe(Rc=5.0, angle=0.5 * np.pi, R=1.0, panels=32, ns=8, nth=64, name="arc_wall") -> Surface:
    """Wall of a circular tube of radius R swept along a planar arc of radius Rc (z = 0 plane)."""
    s, ws = _panel_nodes(np.linspace(0.0, 1.0, panels + 1), ns)
    c, dc, ddc, e1, de1 = _arc_centreline(s, Rc, 0.0, angle)
    m = s.size
    return _tube(s, ws, c, dc, ddc, np.full(m, R), np.zeros(m), e1, de1, nth, name)


def torus(R0=1.0, eps=0.25, panels=16, ns=8, nth=32) -> Surface:
    """Closed torus, major radius R0, minor radius eps (axis z)."""
    return arc_pipe(Rc=R0, angle=2.0 * np.pi, R=eps, panels=panels, ns=ns, nth=nth, name="torus")


def helix_pipe(a=3.0, pitch=2.0, turns=4.0, R=1.0, panels=2048, ns=8, nth=64) -> Surface:
    """Tube of radius R around the helix (a cos p, a sin p, pitch p / 2pi), p in [0, 2pi turns]."""
    s, ws = _panel_nodes(np.linspace(0.0, 1.0, panels + 1), ns)
    b = pitch / (2.0 * np.pi)
    dp = 2.0 * np.pi * turns
    p = dp * s
    cp, sp = np.cos(p), np.sin(p)
    z = np.zeros_like(s)
    c = np.stack([a * cp, a * sp, b * p])
    dc = dp * np.stack([-a * sp, a * cp, np.full_like(s, b)])
    ddc = dp ** 2 * np.stack([-a * cp, -a * sp, z])
    e1 = np.stack([-cp, -sp, z])
    de1 = dp * np.stack([sp, -cp, z])
    m = s.size
    return _tube(s, ws, c, dc, ddc, np.full(m, R), np.zeros(m), e1, de1, nth, "helix_wall")


def _loop_radius(s):
    """Tube radius of the random loop: 0.01 (1 + 0.5 sin 2 pi s), in [0.005, 0.015]."""
    return 0.01 * (1.0 + 0.5 * np.sin(2.0 * np.pi * s))


def _loop_max_curvature_radius(k, A, B, n=20000):
    """max over the centreline of kappa(s) * radius(s) (on n equispaced samples)."""
    s = np.arange(n) / n
    _, dc, ddc = _loop_eval(s, k, A, B)
    sp = np.linalg.norm(dc, axis=0)
    kappa = np.linalg.norm(_cross(dc, ddc), axis=0) / sp ** 3
    return float(np.max(kappa * _loop_radius(s)))


MAX_KAPPA_RHO = 0.5


def _loop_coeffs(seed, kmax=10):
    """Fourier coefficients of the centreline: successive draws from the generator seeded with
    `seed` until the tube is a valid slender body, kappa * radius <= MAX_KAPPA_RHO everywhere
    (a draw with kappa * radius >= 1 somewhere folds the tube's inner side over itself)."""
    rng = np.random.default_rng(seed)
    k = np.arange(1, kmax + 1)
    sd = 1.0 / (1.0 + k / 3.0)
    while True:
        A = rng.standard_normal((3, kmax)) * sd[None, :]
        B = rng.standard_normal((3, kmax)) * sd[None, :]
        if _loop_max_curvature_radius(k, A, B) <= MAX_KAPPA_RHO:
            return k, A, B


def _loop_eval(s, k, A, B):
    arg = 2.0 * np.pi * np.outer(k, s)                          # (K, M)
    cs, sn = np.cos(arg), np.sin(arg)
    w = 2.0 * np.pi * k[:, None]
    c = A @ cs + B @ sn
    dc = A @ (-w * sn) + B @ (w * cs)
    ddc = A @ (-w ** 2 * cs) + B @ (-w ** 2 * sn)
    return c, dc, ddc


def _frame_rhs(e1, dc, ddc):
    """Frame-transport ODE right-hand side of paper Sec. 3.1.1: e1 x (x_c'' x x_c') / |x_c'|^2."""
    om = _cross(ddc, dc) / np.sum(dc * dc, axis=0)
    return _cross(e1, om)


def _transport_frame(s_out, k, A, B, substeps=8):
    """Integrate the frame ODE with classical RK4 from s = 0 through the sorted s_out.

    The ODE is de1/ds = e1 x omega(s), omega = x_c'' x x_c' / |x_c'|^2; omega is evaluated
    at every RK4 stage point in one vectorised call, then the steps run sequentially."""
    _, dc0, _ = _loop_eval(np.array([0.0]), k, A, B)
    t0 = _unit(dc0)[:, 0]
    guess = np.array([0.3, -0.5, 0.8])
    e = guess - guess.dot(t0) * t0
    e /= np.linalg.norm(e)
    s_prev = np.concatenate([[0.0], s_out[:-1]])
    h = (s_out - s_prev) / substeps                                  # (M,)
    starts = s_prev[:, None] + h[:, None] * np.arange(substeps)[None, :]   # (M, q)
    stage = np.stack([starts, starts + 0.5 * h[:, None], starts + h[:, None]], axis=-1)
    _, d1, d2 = _loop_eval(stage.reshape(-1), k, A, B)
    om = (_cross(d2, d1) / np.sum(d1 * d1, axis=0)).T.reshape(s_out.size, substeps, 3, 3)
    out = np.empty((3, s_out.size))
    ex, ey, ez = (float(v) for v in e)

    def cr(ax, ay, az, b):
        return ay * b[2] - az * b[1], az * b[0] - ax * b[2], ax * b[1] - ay * b[0]

    om_l = om.tolist()
    h_l = h.tolist()
    for i in range(s_out.size):
        hh = h_l[i]
        for q in range(substeps):
            w0, wm, w1 = om_l[i][q]
            k1 = cr(ex, ey, ez, w0)
            k2 = cr(ex + 0.5 * hh * k1[0], ey + 0.5 * hh * k1[1], ez + 0.5 * hh * k1[2], wm)
            k3 = cr(ex + 0.5 * hh * k2[0], ey + 0.5 * hh * k2[1], ez + 0.5 * hh * k2[2], wm)
            k4 = cr(ex + hh * k3[0], ey + hh * k3[1], ez + hh * k3[2], w1)
            ex += hh / 6.0 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
            ey += hh / 6.0 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
            ez += hh / 6.0 * (k1[2] + 2 * k2[2] + 2 * k3[2] + k4[2])
        out[0, i], out[1, i], out[2, i] = ex, ey, ez
    return out


def _loop_panel_breaks(k, A, B, panels, n=200000):
    """Panel ends in s that equidistribute |omega(s)| + mean |omega|, omega = x_c'' x x_c' /
    |x_c'|^2 the rotation rate of the transported frame (curvature x speed): where the frame
    turns fast, its degree-(ns - 1) interpolation on a panel of uniform length loses digits
    (1.4e-6 at 256 panels for seed 1, against 3e-12 on the rest; 2.6e-9 with these ends).  A
    fixed-count form of the paper's adaptive refinement along the centreline."""
    sf = np.arange(n + 1) / n
    _, d1, d2 = _loop_eval(sf, k, A, B)
    om = np.linalg.norm(_cross(d2, d1), axis=0) / np.sum(d1 * d1, axis=0)
    m = om + om.mean()
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (m[1:] + m[:-1]) / n)])
    br = np.interp(np.linspace(0.0, cum[-1], panels + 1), cum, sf)
    br[0], br[-1] = 0.0, 1.0
    return br


def random_loop(seed=1, panels=512, ns=8, nth=16, substeps=2) -> Surface:
    """Closed random slender loop of paper Sec. 5.2: Fourier centreline, k = 1..10,
    iid normal coefficients with standard deviation 1/(1 + k/3) (the first draw whose
    curvature times radius stays <= MAX_KAPPA_RHO); radius 0.01 (1 + 0.5 sin 2 pi s), in
    [0.005, 0.015]; panel ends from _loop_panel_breaks."""
    k, A, B = _loop_coeffs(seed)
    s, ws = _panel_nodes(_loop_panel_breaks(k, A, B, panels), ns)
    c, dc, ddc = _loop_eval(s, k, A, B)
    e1 = _transport_frame(s, k, A, B, substeps=substeps)
    t = _unit(dc)
    e1 = _unit(e1 - np.sum(e1 * t, axis=0) * t)                 # re-orthonormalise (Sec. 3.1.1)
    de1 = _frame_rhs(e1, dc, ddc)
    eps = _loop_radius(s)
    deps = 0.01 * 0.5 * 2.0 * np.pi * np.cos(2.0 * np.pi * s)
    return _tube(s, ws, c, dc, ddc, eps, deps, e1, de1, nth, "random_loop")


def sphere(a=1.0, centre=(0.0, 0.0, 0.0), nphi=20, nth=30) -> Surface:
    """Sphere: GL in cos(phi) x trapezoid in theta, weight a^2 w_GL 2pi/nth."""
    u, wu = gl_rule(nphi)
    th = 2.0 * np.pi * np.arange(nth) / nth
    sphi = np.sqrt(1.0 - u * u)
    d = np.stack([np.outer(sphi, np.cos(th)), np.outer(sphi, np.sin(th)),
                  np.outer(u, np.ones(nth))]).reshape(3, -1)
    w = (a * a * np.outer(wu, np.full(nth, 2.0 * np.pi / nth))).reshape(-1)
    x = np.asarray(centre, dtype=np.float64)[:, None] + a * d
    return Surface(x, d.copy(), w, name="sphere")


def disk_cap(centre, normal, e1, e2, R=1.0, nr=16, nth=64, name="cap") -> Surface:
    """Flat disk of radius R: GL in rho on [0, R] x trapezoid in angle; weight rho w_GL 2pi/nth."""
    g, gw = gl_rule(nr)
    rho = 0.5 * R * (g + 1.0)
    wr = 0.5 * R * gw
    th = 2.0 * np.pi * np.arange(nth) / nth
    c = np.asarray(centre, float)[:, None, None]
    e1 = np.asarray(e1, float)[:, None, None]
    e2 = np.asarray(e2, float)[:, None, None]
    x = c + rho[None, :, None] * (np.cos(th)[None, None, :] * e1 + np.sin(th)[None, None, :] * e2)
    x = x.reshape(3, -1)
    n = np.repeat(np.asarray(normal, float)[:, None], x.shape[1], axis=1)
    w = (rho * wr)[:, None] * np.full(nth, 2.0 * np.pi / nth)[None, :]
    return Surface(x, n, w.reshape(-1), name=name)


def pipe_caps(end0, t0, e1_0, end1, t1, e1_1, R=1.0, nr=16, nth=64):
    """Caps closing a pipe: at s=0 the outward normal is -t0, at s=1 it is +t1."""
    t0, t1 = np.asarray(t0, float), np.asarray(t1, float)
    e1_0, e1_1 = np.asarray(e1_0, float), np.asarray(e1_1, float)
    c0 = disk_cap(end0, -t0, e1_0, np.cross(t0, e1_0), R, nr, nth, name="cap0")
    c1 = disk_cap(end1, t1, e1_1, np.cross(t1, e1_1), R, nr, nth, name="cap1")
    return c0, c1


def capped_straight_pipe(R=1.0, L=4.0, panels=4, ns=8, nth=16, nr=8) -> Surface:
    wall = straight_pipe(R, L, panels, ns, nth)
    c0, c1 = pipe_caps((0, 0, 0), (0, 0, 1), (1, 0, 0), (0, 0, L), (0, 0, 1), (1, 0, 0), R, nr, nth)
    return concat([wall, c0, c1], name="capped_straight_pipe")


def capped_arc_pipe(Rc=5.0, angle=0.5 * np.pi, R=1.0, panels=32, ns=8, nth=64, nr=16) -> Surface:
    wall = arc_pipe(Rc, angle, R, panels, ns, nth)
    c, dc, _, e1, _ = _arc_centreline(np.array([0.0, 1.0]), Rc, 0.0, angle)
    t = _unit(dc)
    c0, c1 = pipe_caps(c[:, 0], t[:, 0], e1[:, 0], c[:, 1], t[:, 1], e1[:, 1], R, nr, nth)
    return concat([wall, c0, c1], name="capped_arc_pipe")


def interior_points_straight(n, R=1.0, L=4.0, seed=1, margin=0.0):
    """Uniform-in-volume points inside the cylinder rho < R - margin, z in (margin, L - margin)."""
    rng = np.random.default_rng(seed)
    u = rng.random((3, n))
    rho = (R - margin) * np.sqrt(u[0])
    th = 2.0 * np.pi * u[1]
    z = margin + (L - 2 * margin) * u[2]
    return np.stack([rho * np.cos(th), rho * np.sin(th), z])


def density(n, seed=0):
    """i.i.d. N(0, 1) density, shape (3, n)."""
    return np.random.default_rng(seed).standard_normal((3, n))


# ---------------------------------------------------------------------------
# Workloads (sizes and seeds follow the five synthetic configurations)
# ---------------------------------------------------------------------------

def config1():
    """Straight pipe R=1, L=4: 4 panels x 8 GL x 16 theta = 512 wall nodes; density seed 0;
    targets = the 512 nodes followed by 256 uniform interior points (seed 1)."""
    surf = straight_pipe(1.0, 4.0, 4, 8, 16)
    sigma = density(surf.size, seed=0)
    trg = np.concatenate([surf.x, interior_points_straight(256, seed=1)], axis=1)
    return dict(surf=surf, sigma=sigma, trg=trg, slenderness=None)


def config2(panels=32, ns=8, nth=64, nr=16):
    """Quarter-circle arc pipe, centreline radius 5, tube radius 1: 32 panels x 8 GL x 64 theta
    = 16384 wall nodes, plus two 16 x 64 caps.  Dirichlet data: parabolic profile
    (1 - rho^2) along the end tangent on both caps, zero on the wall."""
    Rc, R = 5.0, 1.0
    surf = capped_arc_pipe(Rc, 0.5 * np.pi, R, panels, ns, nth, nr)
    rhs = np.zeros((3, surf.size))
    cends, dc, _, _, _ = _arc_centreline(np.array([0.0, 1.0]), Rc, 0.0, 0.5 * np.pi)
    t = _unit(dc)
    for nm, a, b in surf.parts:
        if nm.startswith("cap"):
            k = 0 if nm == "cap0" else 1
            rho2 = np.sum((surf.x[:, a:b] - cends[:, k:k + 1]) ** 2, axis=0) / (R * R)
            rhs[:, a:b] = (1.0 - rho2)[None, :] * t[:, k:k + 1]
    return dict(surf=surf, rhs=rhs, slenderness=R / Rc)


def config3(panels=512, ns=8, nth=16, n_sub=4096):
    """Random closed slender loop (paper Sec. 5.2 recipe), seed 1; density seed 2;
    subsampled target indices seed 4."""
    surf = random_loop(seed=1, panels=panels, ns=ns, nth=nth)
    sigma = density(surf.size, seed=2)
    sub = np.sort(np.random.default_rng(4).choice(surf.size, size=min(n_sub, surf.size),
                                                  replace=False))
    return dict(surf=surf, sigma=sigma, sub=sub, slenderness=None)


def config4(nseg=64, seed=3, ns=8, nth=32, nr=16, n_lo=2048, n_hi=65536):
    """Batch of independent capped arc pipes: arc angle ~ U[30, 180] degrees, wall node
    count log-uniform in [n_lo, n_hi] rounded to a multiple of ns*nth (seed 3)."""
    rng = np.random.default_rng(seed)
    ang = np.deg2rad(rng.uniform(30.0, 180.0, nseg))
    nn = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), nseg))
    per = ns * nth
    panels = np.maximum(1, np.rint(nn / per)).astype(int)
    segs = []
    for a, k in zip(ang, panels):
        surf = capped_arc_pipe(5.0, float(a), 1.0, int(k), ns, nth, nr)
        rhs = np.zeros((3, surf.size))
        cends, dc, _, _, _ = _arc_centreline(np.array([0.0, 1.0]), 5.0, 0.0, float(a))
        t = _unit(dc)
        for nm, lo, hi in surf.parts:
            if nm.startswith("cap"):
                kk = 0 if nm == "cap0" else 1
                rho2 = np.sum((surf.x[:, lo:hi] - cends[:, kk:kk + 1]) ** 2, axis=0)
                rhs[:, lo:hi] = (1.0 - rho2)[None, :] * t[:, kk:kk + 1]
        segs.append(dict(surf=surf, rhs=rhs, angle=float(a)))
    return dict(segments=segs, slenderness=1.0 / 5.0)


def rings(nring=32, eps=0.05, panels=64, ns=8, nth=16, spacing=3.0, seed=9):
    """nring tori (R = 1, tube radius eps) with centres on a 4 x 4 x (nring/16) lattice of the
    given spacing, each turned by an independent uniformly random rotation (seed 9); a
    body per ring."""
    rng = np.random.default_rng(seed)
    base = torus(1.0, eps, panels, ns, nth)
    out = []
    for i in range(nring):
        c = spacing * np.array([i % 4, (i // 4) % 4, i // 16], dtype=np.float64)
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        a, b, cc, d = q
        Rm = np.array([[a * a + b * b - cc * cc - d * d, 2 * (b * cc - a * d), 2 * (b * d + a * cc)],
                       [2 * (b * cc + a * d), a * a - b * b + cc * cc - d * d, 2 * (cc * d - a * b)],
                       [2 * (b * d - a * cc), 2 * (cc * d + a * b), a * a - b * b - cc * cc + d * d]])
        out.append(Surface(Rm @ base.x + c[:, None], Rm @ base.n, base.w.copy(), name="ring"))
    return concat(out, name="rings")


def config5(panels=2048, ns=8, nth=64, nr=16, nsph=100, seed=5, turns=4.0, pitch=2.0):
    """Helical pipe (helix radius 3, pitch `pitch` (2), `turns` turns (4), tube radius 1) with
    caps, plus nsph
    spheres of radius 0.2 (20 x 30 nodes) at uniform random positions inside the tube,
    at least 0.05 from the wall and from each other (seed 5)."""
    a, R, rs = 3.0, 1.0, 0.2
    wall = helix_pipe(a, pitch, turns, R, panels, ns, nth)
    b = pitch / (2.0 * np.pi)
    pe = np.array([0.0, 2.0 * np.pi * turns])
    cend = np.stack([a * np.cos(pe), a * np.sin(pe), b * pe])
    tend = _unit(np.stack([-a * np.sin(pe), a * np.cos(pe), np.full(2, b)]))
    e1end = np.stack([-np.cos(pe), -np.sin(pe), np.zeros(2)])
    c0, c1 = pipe_caps(cend[:, 0], tend[:, 0], e1end[:, 0], cend[:, 1], tend[:, 1], e1end[:, 1],
                       R, nr, nth)
    rng = np.random.default_rng(seed)
    centres = []
    rmax = R - rs - 0.05
    while len(centres) < nsph:
        p = rng.uniform(0.0, 2.0 * np.pi * turns)
        r = rmax * math.sqrt(rng.random())
        th = 2.0 * np.pi * rng.random()
        cc = np.array([a * math.cos(p), a * math.sin(p), b * p])
        tt = _unit(np.array([[-a * math.sin(p)], [a * math.cos(p)], [b]]))[:, 0]
        e1 = np.array([-math.cos(p), -math.sin(p), 0.0])
        e2 = np.cross(tt, e1)
        q = cc + r * (math.cos(th) * e1 + math.sin(th) * e2)
        # keep the sphere inside the straight part of the tube cross-section near p and
        # away from the caps
        if p < 0.5 or p > 2.0 * np.pi * turns - 0.5:
            continue
        if all(np.linalg.norm(q - o) >= 2 * rs + 0.05 for o in centres):
            centres.append(q)
    sph = [sphere(rs, c, 20, 30) for c in centres]
    kappa = a / (a * a + b * b)
    surf = concat([wall, c0, c1] + sph, name="helix_with_spheres")
    return dict(surf=surf, centres=np.array(centres), slenderness=R * kappa)

"""CPU FP64 oracle for the quadrature correction E of tube elements (paper Sec. 3.2.1-3.2.4).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of
the benchmark use it; it shares no code with the CUDA library.

What it computes.  A tube element k (a panel of a slender body) carries N_s Gauss--Legendre
nodes t_i on the panel parameter interval [-1, 1] times N_theta equispaced angles
theta_j = 2 pi j / N_theta; global node index k N_s N_theta + i N_theta + j (the order the
input generator uses).  For a target x that lies in the near region of element k, the
uncorrected sum over the element's nodes is replaced by an accurate integral over the
element (Eq. nystrom-correction):

    E_ij(x) = sum_m P_mi w^s_m h_j(x, t_m)  -  G(x, y_ij) w_ij          (Eqs. near-singular
                                                                          and sing-nyst-correc)

with the coincident node (x = y_ij) left out of the subtracted term, as the punctured sum
leaves it out.  The pieces, in the paper's order:

  * element geometry: every GL row of nodes lies on a circle y = c_i + a_i cos(theta) +
    b_i sin(theta) (the tube parametrisation of Eq. surface-coord); c, a, b are read off the
    nodes (discrete Fourier modes 0 and 1) and interpolated in t with the Lagrange basis
    of the GL nodes, so y(t, theta), its derivatives, the unit normal n and the area
    element J = |y_t x y_theta| are defined at every (t, theta);
  * angular weights h_j(x, t) (Sec. 3.2.2): find the angle theta_0 of the point of the
    circle at t closest to x and its relative distance alpha = dist / radius; integrate
    the modal integrands G(x, y(t, theta)) e^{i l theta} J, l = 0 .. N_theta/2, with a
    composite Gauss--Legendre rule in theta - theta_0 on [-pi, pi] whose panels are refined
    dyadically towards 0 until the smallest is no longer than alpha (Eq.
    modal-greens-fn-coeff); then h_j is the inverse DFT of those modal coefficients (Eq.
    modal-greens-fn-wts), the Nyquist mode entering as cos(N_theta theta / 2);
  * outer rule in t: for a target on the element (one of its nodes, parameter t_0) each
    side of t_0 is split dyadically towards t_0 until the panel next to t_0 is no longer
    than the tube radius; that panel takes a rule for p(t) log|t - t_0| + q(t) (Sec. 3.2.4),
    the others Gauss--Legendre.  For a target off the element, each side of the closest
    parameter t* is split dyadically towards t* until the panel next to it is no longer
    than the distance d* of x from the element (Sec. 3.2.3);
  * P: Lagrange interpolation from the element's GL nodes to the outer rule's nodes.

Readings (the paper is silent on them): the log-singular rule is Gauss--Legendre after the
substitution t = t_0 + h u^6 (exact for the grading, accurate to rounding for p log + q);
panels carry 16 Gauss--Legendre nodes; the element's near region is the set of points
closer than radius + f max(length, 2 radius) to its centreline samples (f = near_factor).
The generalized Chebyshev compression of the angular and singular rules (Sec. 3.2.2,
Sec. 3.2.4, App. B) is an optimisation of these same integrals and is not part of the
definition here.

Kernels: Stokes alpha S + beta D (3 x 3, with the double-layer sign of stokes_oracle.c),
Laplace alpha G + beta dG/dn_y (scalar), exactly as the pair-sum oracle defines them.
"""
from __future__ import annotations

import math

import numpy as np

PI = math.pi
Q_THETA = 16        # GL nodes per angular panel
Q_S = 16            # GL nodes per panel of the outer rule
SING_N = 24         # nodes of the log-singular rule
SING_G = 6          # its grading exponent
LMAX = 60           # deepest dyadic level
GOLDEN_ITERS = 40
T_SAMPLES = 64


def gl01(n):
    """Gauss--Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def singular_rule():
    """Nodes and weights on [0, 1] for f(t) = p(t) log t + q(t): Gauss--Legendre in u after
    t = u^g, weight g u^(g-1)."""
    u, w = gl01(SING_N)
    return u ** SING_G, SING_G * u ** (SING_G - 1) * w


def lagrange(tn, t):
    """Lagrange basis of the nodes tn and its derivative at the points t: (len t, len tn).
    l_i(t) = prod_{k != i} (t - tn_k) / (tn_i - tn_k) and
    l_i'(t) = sum_{m != i} 1 / (tn_i - tn_m) prod_{k != i, m} (t - tn_k) / (tn_i - tn_k),
    the products taken over the factor axis of an array of all ratios (a factor that the
    formula leaves out is replaced by 1)."""
    tn = np.asarray(tn, dtype=np.float64)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    ns = tn.shape[0]
    eye = np.eye(ns, dtype=bool)
    den = np.where(eye, 1.0, tn[:, None] - tn[None, :])            # (i, k)
    ratio = (t[:, None, None] - tn[None, None, :]) / den[None]     # (point, i, k)
    ratio = np.where(eye[None], 1.0, ratio)
    L = np.prod(ratio, axis=2)
    dL = np.zeros((t.shape[0], ns))
    for m in range(ns):
        rm = ratio.copy()
        rm[:, :, m] = 1.0
        term = np.prod(rm, axis=2) / den[:, m][None, :]
        term[:, m] = 0.0                                           # m != i
        dL += term
    return L, dL


def lagrange_offset(tn, i0, delta):
    """l_i(tn[i0] + delta) for i != i0 (the entry i0 is set to 0), with the factor
    (t - tn[i0]) taken as delta itself, so that the values keep their relative accuracy
    however small delta is: (len delta, len tn)."""
    tn = np.asarray(tn, dtype=np.float64)
    delta = np.atleast_1d(np.asarray(delta, dtype=np.float64))
    ns = tn.shape[0]
    D = np.zeros((delta.shape[0], ns))
    for i in range(ns):
        if i == i0:
            continue
        v = np.ones(delta.shape[0])
        for k in range(ns):
            if k == i:
                continue
            fk = delta if k == i0 else (tn[i0] - tn[k]) + delta
            v = v * fk / (tn[i] - tn[k])
        D[:, i] = v
    return D


# ---------------------------------------------------------------------------------------
# kernels (the same definitions as the pair-sum oracle)

def kernel(kind, alpha, beta, x, y, n):
    """Kernel values G(x, y_m; n_m) for points y (3, M): Stokes (9, M) with row a * 3 + b,
    Laplace (1, M)."""
    return kernel_r(kind, alpha, beta, x[:, None] - y, n)


def kernel_r(kind, alpha, beta, r, n):
    """The kernel values for offsets r = x - y_m (3, M)."""
    r2 = np.sum(r * r, axis=0)
    rl = np.sqrt(r2)
    if kind == "laplace":
        g = np.zeros_like(rl)
        if alpha != 0.0:
            g = g + alpha / (4.0 * PI * rl)
        if beta != 0.0:
            g = g + beta * np.sum(r * n, axis=0) / (4.0 * PI * rl * r2)
        return g[None, :]
    out = np.zeros((9, r.shape[1]))
    rn = np.sum(r * n, axis=0) if beta != 0.0 else None
    for a in range(3):
        for b in range(3):
            v = np.zeros_like(rl)
            if alpha != 0.0:
                v = v + alpha * ((1.0 / rl if a == b else 0.0) + r[a] * r[b] / (rl * r2)) / (8.0 * PI)
            if beta != 0.0:
                v = v + beta * 3.0 / (4.0 * PI) * rn * r[a] * r[b] / (r2 * r2 * rl)
            out[a * 3 + b] = v
    return out


def ncomp(kind):
    return 1 if kind == "laplace" else 9


# ---------------------------------------------------------------------------------------
# element geometry

class Element:
    """Geometry of one tube element from its nodes (3, Ns, Nt), normals and weights."""

    def __init__(self, y, n, w):
        self.y = np.asarray(y, dtype=np.float64)
        self.n = np.asarray(n, dtype=np.float64)
        self.w = np.asarray(w, dtype=np.float64)
        _, ns, nt = self.y.shape
        if nt < 4 or nt % 2:
            raise ValueError("N_theta must be even and at least 4")
        self.ns, self.nt = ns, nt
        self.tn, _ = np.polynomial.legendre.leggauss(ns)
        th = 2.0 * PI * np.arange(nt) / nt
        self.c = self.y.mean(axis=2)
        self.a = (2.0 / nt) * np.sum(self.y * np.cos(th), axis=2)
        self.b = (2.0 / nt) * np.sum(self.y * np.sin(th), axis=2)
        recon = (self.c[:, :, None] + self.a[:, :, None] * np.cos(th) + self.b[:, :, None] * np.sin(th))
        self.rho_max = float(np.max(np.sqrt(0.5 * (np.sum(self.a ** 2, axis=0) + np.sum(self.b ** 2, axis=0)))))
        if np.max(np.abs(recon - self.y)) > 1e-9 * max(self.rho_max, 1e-300):
            raise ValueError("element rows are not circles")
        _, dL = lagrange(self.tn, self.tn)
        self.speed_max = float(np.max(np.linalg.norm(self.c @ dL.T, axis=0)))
        self.length = self.speed_max * 2.0
        # orientation: sign of (y_theta x y_t) . n at node (0, 0)
        g = self.geom(np.array([self.tn[0]]), np.array([0.0]))
        cr = np.cross(g["yth"][:, 0], g["yt"][:, 0])
        self.sgn = 1.0 if float(np.dot(cr, self.n[:, 0, 0])) >= 0.0 else -1.0
        Lend, _ = lagrange(self.tn, np.array([-1.0, 1.0]))
        self.cl_pts = np.concatenate([self.c, self.c @ Lend.T], axis=1)   # centreline samples

    def coeffs(self, t):
        """(C, A, B, C_t, A_t, B_t) at one parameter t, each (3,)."""
        L, dL = lagrange(self.tn, np.array([t]))
        L, dL = L[0], dL[0]
        return (self.c @ L, self.a @ L, self.b @ L, self.c @ dL, self.a @ dL, self.b @ dL)

    def geom(self, t, th):
        """Position, derivatives, unit normal and J at parameter pairs (t[m], th[m])."""
        L, dL = lagrange(self.tn, t)
        C, A, B = self.c @ L.T, self.a @ L.T, self.b @ L.T
        Ct, At, Bt = self.c @ dL.T, self.a @ dL.T, self.b @ dL.T
        cs, sn = np.cos(th), np.sin(th)
        y = C + A * cs + B * sn
        yt = Ct + At * cs + Bt * sn
        yth = -A * sn + B * cs
        return {"y": y, "yt": yt, "yth": yth}


def circle_point(co, th):
    C, A, B, Ct, At, Bt = co
    cs, sn = np.cos(th), np.sin(th)
    y = C[:, None] + A[:, None] * cs + B[:, None] * sn
    yt = Ct[:, None] + At[:, None] * cs + Bt[:, None] * sn
    yth = -A[:, None] * sn + B[:, None] * cs
    return y, yt, yth


def closest_angle(co, x):
    """Angle of the point of the circle (co at one t) nearest x, the distance and the radius."""
    C, A, B = co[0], co[1], co[2]
    d = x - C
    th = math.atan2(float(np.dot(d, B)), float(np.dot(d, A)))
    for _ in range(3):
        cs, sn = math.cos(th), math.sin(th)
        y = C + A * cs + B * sn
        yth = -A * sn + B * cs
        ythth = -A * cs - B * sn
        f = float(np.dot(y - x, yth))
        fp = float(np.dot(yth, yth) + np.dot(y - x, ythth))
        if fp <= 0.0:
            break
        th -= f / fp
    y = C + A * math.cos(th) + B * math.sin(th)
    rho = math.sqrt(0.5 * (float(np.dot(A, A)) + float(np.dot(B, B))))
    return th, float(np.linalg.norm(x - y)), rho


def theta_rule(alpha, nt):
    """Composite GL rule in phi = theta - theta_0 on [-pi, pi], dyadically refined towards 0
    until the smallest panel is no longer than alpha."""
    nb = max(2, -(-nt // 8))
    lb = PI / nb
    if alpha >= lb:
        levels = 0
    elif alpha <= 0.0:
        levels = LMAX
    else:
        levels = min(LMAX, int(math.ceil(math.log2(lb / alpha))))
    edges = [0.0] + [lb / 2.0 ** k for k in range(levels, 0, -1)] + [lb * m for m in range(1, nb + 1)]
    g, gw = gl01(Q_THETA)
    phis, ws = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        phis.append(lo + (hi - lo) * g)
        ws.append((hi - lo) * gw)
    phi = np.concatenate(phis)
    w = np.concatenate(ws)
    return np.concatenate([-phi[::-1], phi]), np.concatenate([w[::-1], w])


def modal_weights(el: Element, th, v):
    """Eq. modal-greens-fn-coeff then Eq. modal-greens-fn-wts: from the integrand values v
    (ncomp, M) (kernel x J x angular weight) at the angles th, the weights h_j."""
    nt = el.nt
    lmodes = np.arange(nt // 2 + 1)
    hhat = v @ np.exp(1j * np.outer(th, lmodes))                          # Eq. modal-greens-fn-coeff
    thj = 2.0 * PI * np.arange(nt) / nt
    fac = np.full(nt // 2 + 1, 2.0)
    fac[0] = 1.0
    fac[-1] = 1.0
    # Eq. modal-greens-fn-wts: inverse DFT; real because hhat_{-l} = conj(hhat_l)
    return (np.real(hhat[:, :, None] * np.exp(-1j * lmodes[:, None] * thj[None, :])[None]) * fac[None, :, None]).sum(axis=1) / nt


def angular_weights(el: Element, x, t, kind, alpha, beta):
    """h_j(x, t) of Eq. modal-greens-fn-wts for a target x off the element:
    (ncomp, N_theta)."""
    co = el.coeffs(t)
    th0, dist, rho = closest_angle(co, x)
    phi, om = theta_rule(dist / rho, el.nt)
    th = th0 + phi
    y, yt, yth = circle_point(co, th)
    cr = np.cross(yth, yt, axis=0) * el.sgn
    J = np.linalg.norm(cr, axis=0)
    return modal_weights(el, th, kernel(kind, alpha, beta, x, y, cr / J) * (J * om)[None, :])


def own_offsets(el: Element, i0, j0, delta, psi):
    """y(t, theta) - x for the target x = y(t_i0, theta_j0) at t = t_i0 + delta and
    theta = theta_j0 + psi, formed from differences that keep their relative accuracy
    (partition of unity for the interpolation, product formulas for the trigonometric
    differences).  Returns (y - x, A(t), B(t)) with y - x of shape (3, len psi)."""
    D = lagrange_offset(el.tn, i0, delta)[0]
    dC = el.c @ D - el.c[:, i0] * D.sum()
    dA = el.a @ D - el.a[:, i0] * D.sum()
    dB = el.b @ D - el.b[:, i0] * D.sum()
    thj0 = 2.0 * PI * j0 / el.nt
    th = thj0 + psi
    sh = np.sin(0.5 * psi)
    dcos = -2.0 * np.sin(thj0 + 0.5 * psi) * sh
    dsin = 2.0 * np.cos(thj0 + 0.5 * psi) * sh
    ymx = (dC[:, None] + dA[:, None] * np.cos(th) + el.a[:, i0, None] * dcos
           + dB[:, None] * np.sin(th) + el.b[:, i0, None] * dsin)
    return ymx, el.a[:, i0] + dA, el.b[:, i0] + dB


def angular_weights_own(el: Element, i0, j0, delta, kind, alpha, beta):
    """h_j(x, t) for the target x = node (i0, j0) of this element at t = t_i0 + delta."""
    thj0 = 2.0 * PI * j0 / el.nt
    # closest angle, as an offset from theta_j0 (Newton on (y - x) . y_theta)
    psi0 = 0.0
    for _ in range(4):
        ymx, A, B = own_offsets(el, i0, j0, delta, np.array([psi0]))
        th = thj0 + psi0
        yth = -A * math.sin(th) + B * math.cos(th)
        ythth = -A * math.cos(th) - B * math.sin(th)
        f = float(np.dot(ymx[:, 0], yth))
        fp = float(np.dot(yth, yth) + np.dot(ymx[:, 0], ythth))
        if fp <= 0.0:
            break
        psi0 -= f / fp
    ymx, A, B = own_offsets(el, i0, j0, delta, np.array([psi0]))
    rho = math.sqrt(0.5 * (float(np.dot(A, A)) + float(np.dot(B, B))))
    phi, om = theta_rule(float(np.linalg.norm(ymx[:, 0])) / rho, el.nt)
    psi = psi0 + phi
    ymx, A, B = own_offsets(el, i0, j0, delta, psi)
    th = thj0 + psi
    co = el.coeffs(float(el.tn[i0] + delta))
    _, yt, yth = circle_point(co, th)
    cr = np.cross(yth, yt, axis=0) * el.sgn
    J = np.linalg.norm(cr, axis=0)
    return modal_weights(el, th, kernel_r(kind, alpha, beta, -ymx, cr / J) * (J * om)[None, :])


def _dyadic_side(t0, ell, levels):
    """Panels of [t0, t0 + ell] (ell signed) refined dyadically towards t0: the innermost
    first, as (lo, hi) pairs in parameter order."""
    inner = (t0, t0 + ell / 2.0 ** levels)
    rest = [(t0 + ell / 2.0 ** (k + 1), t0 + ell / 2.0 ** k) for k in range(levels - 1, -1, -1)]
    return inner, rest


def _levels(phys, scale):
    if phys <= scale:
        return 0
    if scale <= 0.0:
        return LMAX
    return min(LMAX, int(math.ceil(math.log2(phys / scale))))


def s_rule_on_element(el: Element, t0):
    """Outer rule for a target at the element's own node with parameter t0 (Sec. 3.2.4),
    as offsets delta = t - t0 and weights."""
    g, gw = gl01(Q_S)
    us, uw = singular_rule()
    ds, ws = [], []
    for ell in (1.0 - t0, -1.0 - t0):
        if ell == 0.0:
            continue
        lev = _levels(abs(ell) * el.speed_max, el.rho_max)
        inner, rest = _dyadic_side(0.0, ell, lev)
        h = inner[1] - inner[0]
        ds.append(h * us)
        ws.append(abs(h) * uw)
        for lo, hi in rest:
            ds.append(lo + (hi - lo) * g)
            ws.append(abs(hi - lo) * gw)
    return np.concatenate(ds), np.concatenate(ws)


def nearest_parameter(el: Element, x):
    """Parameter t* in [-1, 1] of the circle nearest x and its distance d* (sampling, then
    golden-section search)."""
    def dist(t):
        return closest_angle(el.coeffs(t), x)[1]
    ts = -1.0 + 2.0 * np.arange(T_SAMPLES + 1) / T_SAMPLES
    ds = [dist(float(t)) for t in ts]
    k = int(np.argmin(ds))
    lo, hi = float(ts[max(k - 1, 0)]), float(ts[min(k + 1, T_SAMPLES)])
    gr = 0.5 * (math.sqrt(5.0) - 1.0)
    a, b = lo, hi
    c1, c2 = b - gr * (b - a), a + gr * (b - a)
    f1, f2 = dist(c1), dist(c2)
    for _ in range(GOLDEN_ITERS):
        if f1 <= f2:
            b, c2, f2 = c2, c1, f1
            c1 = b - gr * (b - a)
            f1 = dist(c1)
        else:
            a, c1, f1 = c1, c2, f2
            c2 = a + gr * (b - a)
            f2 = dist(c2)
    tstar = 0.5 * (a + b)
    cand = [(dist(tstar), tstar), (ds[k], float(ts[k]))]
    dstar, tstar = min(cand)
    return tstar, dstar


def s_rule_near(el: Element, tstar, dstar):
    """Outer rule for a target off the element (Sec. 3.2.3)."""
    g, gw = gl01(Q_S)
    ts, ws = [], []
    for ell in (1.0 - tstar, -1.0 - tstar):
        if ell == 0.0:
            continue
        lev = _levels(abs(ell) * el.speed_max, dstar)
        inner, rest = _dyadic_side(tstar, ell, lev)
        for lo, hi in [inner] + rest:
            ts.append(lo + (hi - lo) * g)
            ws.append(abs(hi - lo) * gw)
    return np.concatenate(ts), np.concatenate(ws)


def element_block(el: Element, x, kind, alpha, beta, own=None):
    """E_ij(x) for one element: (ncomp, N_s, N_theta).  own = (i0, j0) when x is that node."""
    if own is not None:
        t0 = float(el.tn[own[0]])
        ds, ws = s_rule_on_element(el, t0)
        ts = t0 + ds
    else:
        tstar, dstar = nearest_parameter(el, x)
        ts, ws = s_rule_near(el, tstar, dstar)
    P, _ = lagrange(el.tn, ts)                                            # (M, Ns)
    nc = ncomp(kind)
    E = np.zeros((nc, el.ns, el.nt))
    for m in range(ts.shape[0]):
        if own is not None:
            h = angular_weights_own(el, own[0], own[1], float(ds[m]), kind, alpha, beta)
        else:
            h = angular_weights(el, x, float(ts[m]), kind, alpha, beta)  # (nc, Nt)
        E += (ws[m] * h)[:, None, :] * P[m][None, :, None]
    # subtract the uncorrected sum's terms (the coincident node is not in it)
    yy = el.y.reshape(3, -1)
    nn = el.n.reshape(3, -1)
    with np.errstate(divide="ignore", invalid="ignore"):
        G = kernel(kind, alpha, beta, x, yy, nn) * el.w.reshape(-1)[None, :]
    if own is not None:
        G[:, own[0] * el.nt + own[1]] = 0.0
    E -= G.reshape(nc, el.ns, el.nt)
    return E


# ---------------------------------------------------------------------------------------
# the sparse correction over whole tubes

def elements_of(src, nrm, w, nelem, ns, nt):
    src = np.asarray(src, dtype=np.float64)
    nrm = np.asarray(nrm, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    per = ns * nt
    return [Element(src[:, k * per:(k + 1) * per].reshape(3, ns, nt),
                    nrm[:, k * per:(k + 1) * per].reshape(3, ns, nt),
                    w[k * per:(k + 1) * per].reshape(ns, nt)) for k in range(nelem)]


def is_near(el: Element, x, near_factor):
    d = float(np.min(np.linalg.norm(el.cl_pts - x[:, None], axis=0)))
    return d < el.rho_max + near_factor * max(el.length, 2.0 * el.rho_max)


def near_elements(els, x, own_k, near_factor):
    return [k for k, el in enumerate(els) if k == own_k or is_near(el, x, near_factor)]


def correction_rows(src, nrm, w, nelem, ns, nt, kind, alpha, beta, near_factor, targets):
    """Rows of E for the target nodes `targets` (global node indices of the tube nodes).

    Returns a dict target -> list of (k, block) with block (ncomp, Ns, Nt).  The dense
    form of the rows is in `correction_dense_rows`."""
    els = elements_of(src, nrm, w, nelem, ns, nt)
    per = ns * nt
    src = np.asarray(src, dtype=np.float64)
    out = {}
    for tg in targets:
        tg = int(tg)
        x = src[:, tg]
        own_k = tg // per
        blocks = []
        for k in near_elements(els, x, own_k, near_factor):
            own = ((tg % per) // nt, tg % nt) if k == own_k else None
            blocks.append((k, element_block(els[k], x, kind, alpha, beta, own)))
        out[tg] = blocks
    return out


def correction_rows_offsurface(src, nrm, w, nelem, ns, nt, kind, alpha, beta, near_factor, trg):
    """Rows of E for off-surface targets trg (3, m) (Sec. 3.2.3): for every element whose near
    region holds the target, the near-singular rule; returns a dict k -> list of (element,
    block) keyed by the target's column index in trg."""
    els = elements_of(src, nrm, w, nelem, ns, nt)
    trg = np.asarray(trg, dtype=np.float64)
    out = {}
    for m in range(trg.shape[1]):
        x = trg[:, m]
        out[m] = [(k, element_block(els[k], x, kind, alpha, beta, None))
                  for k in near_elements(els, x, -1, near_factor)]
    return out


def correction_dense_rows(rows, n, kind):
    """Dense rows of E (component-major rows and columns, as the CSR layout): for Stokes
    a dict target -> (3, 3 n), for Laplace target -> (n,)."""
    out = {}
    for tg, blocks in rows.items():
        if kind == "laplace":
            r = np.zeros(n)
            for k, B in blocks:
                per = B.shape[1] * B.shape[2]
                r[k * per:(k + 1) * per] += B[0].reshape(-1)
        else:
            r = np.zeros((3, 3 * n))
            for k, B in blocks:
                per = B.shape[1] * B.shape[2]
                for a in range(3):
                    for b in range(3):
                        r[a, b * n + k * per:b * n + (k + 1) * per] += B[a * 3 + b].reshape(-1)
        out[tg] = r
    return out


def correction_csr(src, nrm, w, nelem, ns, nt, kind, alpha, beta, near_factor):
    """The whole E over all tube nodes as a CSR (rows component-major, columns likewise)."""
    n = nelem * ns * nt
    rows = correction_rows(src, nrm, w, nelem, ns, nt, kind, alpha, beta, near_factor, range(n))
    dense = correction_dense_rows(rows, n, kind)
    nc = 1 if kind == "laplace" else 3
    rowptr = [0]
    cols, vals = [], []
    for a in range(nc):
        for t in range(n):
            r = dense[t] if kind == "laplace" else dense[t][a]
            nz = np.nonzero(r)[0]
            cols.append(nz)
            vals.append(r[nz])
            rowptr.append(rowptr[-1] + nz.shape[0])
    from oracle import CSR
    return CSR(np.array(rowptr), np.concatenate(cols), np.concatenate(vals), nc * n, nc * n)

"""Pins of the generalized Chebyshev construction (Appendix B, oracle/gen_chebyshev.py):
closed-form integrals of the families it compresses, and the node count the paper prints
for its compressed angular rules (Sec. 3.2.2).  CPU only."""
import math

import numpy as np
import pytest

from oracle import gen_chebyshev as C

pytest.importorskip("scipy.linalg")
special = pytest.importorskip("scipy.special")


def test_polynomial_family():
    """t^k, k < 16, on [0, 1]: at most 16 nodes, each monomial integrated to rounding."""
    x, w = C.gl01(32)
    F = np.stack([x ** k for k in range(16)], axis=1)
    y, om = C.chebyshev_rule(F, x, w, 1e-14)
    assert len(y) <= 16
    for k in range(16):
        assert abs(np.sum(om * y ** k) - 1.0 / (k + 1)) < 1e-13


def test_log_singular_family():
    """p(t) log t + q(t) with p, q of degree < 10 (the family of the paper's singular rule,
    Sec. 3.2.4): fine rule dyadically refined towards 0; the compressed rule integrates
    t^k and t^k log t to 1e-12 (closed forms 1/(k+1), -1/(k+1)^2) with few nodes."""
    g, gw = C.gl01(16)
    xs, ws = [], []
    for lev in range(60):
        lo, hi = 2.0 ** -(lev + 1), 2.0 ** -lev
        xs.append(lo + (hi - lo) * g)
        ws.append((hi - lo) * gw)
    x, w = np.concatenate(xs), np.concatenate(ws)
    F = np.stack([x ** k for k in range(10)] + [x ** k * np.log(x) for k in range(10)], axis=1)
    y, om = C.chebyshev_rule(F, x, w, 1e-14)
    assert len(y) <= 20
    for k in range(10):
        assert abs(np.sum(om * y ** k) - 1.0 / (k + 1)) < 1e-12
        assert abs(np.sum(om * y ** k * np.log(y)) + 1.0 / (k + 1) ** 2) < 1e-12


@pytest.mark.parametrize("level", [1, 5, 10, 20])
def test_compressed_angular_rule(level):
    """Sec. 3.2.2: for l0 = 8 and tolerance 1e-10 the paper reports m0 ~ 38 nodes for every
    distance level alpha; here 25..50.  Targets of the annulus that are not in the training
    grid: the l = 0 integral matches the ring potential's closed form 4 K(m) / sqrt(...),
    the l > 0 ones the fine rule, to 1e-9."""
    alpha = 2.0 ** -level
    y, om = C.angular_rule(alpha, 8, 1e-10)
    assert 25 <= len(y) <= 50, len(y)
    th, w = C.angular_fine_rule(alpha)
    rng = np.random.default_rng(level)
    for _ in range(12):
        r, p = alpha * (1.0 + rng.random()), 2.0 * math.pi * rng.random()
        x = np.array([1.0 + r * math.cos(p), 0.0, r * math.sin(p)])
        G = lambda t: 1.0 / np.linalg.norm(x[:, None] - np.stack([np.cos(t), np.sin(t), 0.0 * t]), axis=0)
        rho, z = math.hypot(x[0], x[1]), x[2]
        den = (rho + 1.0) ** 2 + z * z
        exact0 = 4.0 * special.ellipkm1(((rho - 1.0) ** 2 + z * z) / den) / math.sqrt(den)
        assert abs(np.sum(om * G(y)) - exact0) < 1e-9 * exact0
        for l in (3, 8):
            ref = np.sum(w * G(th) * np.cos(l * th))
            assert abs(np.sum(om * G(y) * np.cos(l * y)) - ref) < 1e-9 * exact0


def test_weighted_construction_deep_level():
    """At alpha = 2^-25 the integrands peak like 1/alpha: the construction in the measure
    psi d theta keeps the l = 0 integral of unseen targets within 1e-9 of the ring closed
    form with about 40 nodes."""
    alpha = 2.0 ** -25
    y, om = C.angular_rule(alpha, 8, 1e-11)
    assert 25 <= len(y) <= 60, len(y)
    rng = np.random.default_rng(4)
    for _ in range(8):
        r, p = alpha * (1.0 + rng.random()), 2.0 * math.pi * rng.random()
        dx, dz = r * math.cos(p), r * math.sin(p)
        d = np.stack([2.0 * np.sin(0.5 * y) ** 2 + dx, -np.sin(y), np.full_like(y, dz)])
        val = np.sum(om / np.linalg.norm(d, axis=0))
        rho = math.hypot(1.0 + dx, 0.0)
        den = (rho + 1.0) ** 2 + dz * dz
        exact = 4.0 * special.ellipkm1((dx * dx + dz * dz) / den) / math.sqrt(den)
        assert abs(val - exact) < 1e-9 * exact


def test_stokes_family_rule():
    """The Stokes family (six single-layer and six double-layer components, circle normals)
    at alpha = 2^-12: unseen annulus targets, components times cos(l theta), l <= 9, match the
    fine rule to 5e-9 of the integral of their magnitude (the worst single component of the
    1140 checked; the truncation is at 1e-11 in the L2 sense of the weighted measure)."""
    alpha = 2.0 ** -12
    y, om = C.angular_rule(alpha, 9, 1e-11, "stokes", nr=8, npsi=16)
    th, w = C.angular_fine_rule(alpha)
    rng = np.random.default_rng(6)
    tg = np.array([[alpha * (1.0 + rng.random()) * math.cos(p), alpha * (1.0 + rng.random()) * math.sin(p)]
                   for p in 2.0 * math.pi * rng.random(5)]).T
    Ff = C.modal_family(tg, th, 9, "stokes")
    Fc = C.modal_family(tg, y, 9, "stokes")
    ref = w @ Ff
    got = om @ Fc
    scale = w @ np.abs(Ff)
    assert np.max(np.abs(got - ref) / scale) < 5e-9

"""The committed whole-element singular rules (paper_2310_00889_gb300/rules/singular_ns8_l12.txt,
written by singular_rules.py with the Appendix B construction) against the oracle's own-element
outer rule (dyadic panels and a graded panel next to t0, oracle/tube_quadrature.py): the
integral over the element of the modal angular weights h_j(x, t) times the Lagrange basis
l_i(t), for a target at the element's own node, on straight pipes of aspect ratios no rule was
built from.  CPU only."""
import math
import warnings

import numpy as np
import pytest

from oracle import tube_quadrature as T
from paper_2310_00889_gb300 import inputs as I
from paper_2310_00889_gb300 import singular_rules as SR

TAB = SR.load()
pytestmark = pytest.mark.skipif(TAB is None, reason="no singular-rule table")


def test_table_layout():
    ns = SR.NS
    levels = sorted({k[0] for k in TAB})
    assert levels == list(range(SR.LEV_LO, SR.LEV_HI + 1))
    tn = np.polynomial.legendre.leggauss(ns)[0]
    for (lev, i0), (d, w) in TAB.items():
        assert 0 < len(d) <= SR.NMAX
        assert np.all(np.diff(d) > 0) and np.all(d != 0.0)
        assert np.all(tn[i0] + d >= -1.0 - 1e-15) and np.all(tn[i0] + d <= 1.0 + 1e-15)
        assert np.all(np.isfinite(w))
        # mirror symmetry: position ns - 1 - i0 is the mirror image
        dm, wm = TAB[(lev, ns - 1 - i0)]
        assert np.allclose(-dm[::-1], d, rtol=0, atol=1e-15) and np.allclose(wm[::-1], w, rtol=1e-14)


@pytest.mark.parametrize("kind,alpha,beta", [("laplace", 1.0, 0.0), ("laplace", 0.0, 1.0),
                                             ("stokes", 1.0, 0.0), ("stokes", 0.0, 1.0)])
@pytest.mark.parametrize("aspect,i0", [(1.37, 0), (5.3, 3), (22.6, 1), (300.0, 2)])
def test_rule_matches_oracle_outer_rule(kind, alpha, beta, aspect, i0):
    """sum_q w_q l_i(t_q) h_j(x, t_q) against the oracle's outer rule, every (component, i, j),
    to 1e-10 of the largest."""
    ns, nt = 8, 16
    # one element of a straight pipe of radius 1 and length `aspect`
    S = I.straight_pipe(R=1.0, L=aspect, panels=1, ns=ns, nth=nt)
    el = T.elements_of(S.x, S.n, S.w, 1, ns, nt)[0]
    lev = int(math.floor(math.log2(aspect)))
    d, w = TAB[(lev, i0)]
    j0 = 5
    t0 = float(el.tn[i0])

    def integral(ds, ws):
        acc = 0.0
        for dd, ww in zip(ds, ws):
            with warnings.catch_warnings():
                warnings.simplefilter("ignore")
                h = T.angular_weights_own(el, i0, j0, float(dd), kind, alpha, beta)   # (ncomp, nt)
            L = T.lagrange(el.tn, t0 + float(dd))[0][0]                            # (ns,)
            acc = acc + ww * L[None, :, None] * h[:, None, :]
        return acc

    ref = integral(*T.s_rule_on_element(el, t0))
    got = integral(d, w)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < 1e-10, err


@pytest.mark.parametrize("eps,panels,i0", [(0.1, 32, 2), (0.02, 32, 0), (0.005, 64, 3)])
def test_rule_on_curved_elements(eps, panels, i0):
    """The same comparison on elements of tori turning 0.1..0.2 rad (the builder takes these
    rules on elements turning up to 0.2 rad; aspect ratios 2..20), which no rule was built
    from: the family's polynomial slack covers the curvature, to 1e-10 of the largest entry
    (Laplace and Stokes, both layers)."""
    ns, nt = 8, 16
    S = I.torus(R0=1.0, eps=eps, panels=panels, ns=ns, nth=nt)
    el = T.elements_of(S.x, S.n, S.w, panels, ns, nt)[0]
    t0 = float(el.tn[i0])
    aspect = 2.0 * math.pi / panels / eps          # element length / radius
    d, w = TAB[(int(math.floor(math.log2(aspect))), i0)]
    for kind, alpha, beta in (("laplace", 1.0, 1.0), ("stokes", 1.0, 1.0)):
        def integral(ds, ws):
            acc = 0.0
            for dd, ww in zip(ds, ws):
                with warnings.catch_warnings():
                    warnings.simplefilter("ignore")
                    h = T.angular_weights_own(el, i0, 3, float(dd), kind, alpha, beta)
                L = T.lagrange(el.tn, t0 + float(dd))[0][0]
                acc = acc + ww * L[None, :, None] * h[:, None, :]
            return acc
        ref = integral(*T.s_rule_on_element(el, t0))
        got = integral(d, w)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 1e-10, (kind, err)

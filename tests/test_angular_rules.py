"""The committed compressed angular rules (paper_2310_00889_gb300/rules/, written by
angular_rules.py) against the oracle's independent construction of the same integrals
(oracle/gen_chebyshev.py: fine rule and Stokes kernel family).  CPU only."""
import math

import numpy as np
import pytest

from oracle import gen_chebyshev as C
from paper_2310_00889_gb300 import angular_rules

pytest.importorskip("scipy.linalg")


def test_table_layout():
    tab = angular_rules.load(16)
    assert tab is not None
    phi, w, cnt = tab
    assert phi.shape == (31, 64) and w.shape == (31, 64) and cnt.shape == (31,)
    assert cnt[0] == 0 and np.all(cnt[1:] > 0) and np.all(cnt <= 64)
    for lev in range(1, 31):
        n = cnt[lev]
        assert np.all(np.abs(phi[lev, :n]) <= math.pi) and np.all(np.isfinite(w[lev, :n]))
        assert abs(w[lev, :n].sum() - 2 * math.pi) < 0.1 * 2 * math.pi   # constants: near, not exact


@pytest.mark.parametrize("lev", [1, 8, 12, 19, 30])
def test_table_integrates_the_stokes_family(lev):
    """Unseen annulus targets at relative distance 2^-lev..2^(1-lev): every Stokes single- and
    double-layer component times cos / sin(l theta), l <= 9, integrated by the table's rule
    agrees with the oracle's fine rule to 1e-9 (levels <= 12) of the target's largest
    component integral.  Deeper, a double-precision construction reaches 1e-7 only.  For an
    on-surface target those rules serve only the s-nodes within 2^-12 tube radii of its own
    parameter, whose weights in the outer rule are below ~1e-4 of the panel; an off-surface
    target closer than 2^-12 radii to the surface sees that 1e-7 directly."""
    phi, w, cnt = angular_rules.load(16)
    y, om = phi[lev, :cnt[lev]], w[lev, :cnt[lev]]
    alpha = 2.0 ** -lev
    th, wf = C.angular_fine_rule(alpha)
    rng = np.random.default_rng(lev)
    worst = 0.0
    for _ in range(4):
        r, p = alpha * (1.0 + rng.random()), 2.0 * math.pi * rng.random()
        tg = np.array([[r * math.cos(p)], [r * math.sin(p)]])
        Ff = C.modal_family(tg, th, 9, "stokes")
        Fc = C.modal_family(tg, y, 9, "stokes")
        worst = max(worst, np.abs(om @ Fc - wf @ Ff).max() / (wf @ np.abs(Ff)).max())
    assert worst < (1e-9 if lev <= 12 else 5e-7), worst

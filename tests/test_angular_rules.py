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
    phi, w, cnt, l0 = tab
    assert l0 >= 9
    nl = angular_rules.LEVELS + 1
    assert nl == 53
    assert phi.shape == (nl, 128) and w.shape == (nl, 128) and cnt.shape == (nl,)
    assert np.all(cnt > 0) and np.all(cnt <= 128)
    for lev in range(0, nl):
        n = cnt[lev]
        assert np.all(np.abs(phi[lev, :n]) <= math.pi) and np.all(np.isfinite(w[lev, :n]))
    # the rules integrate the kernel times e^{i l theta}, not functions without the kernel's
    # peak: at the shallow levels, where the peak is wide, the weights still add up to 2 pi
    for lev in range(0, 3):
        assert abs(w[lev, :cnt[lev]].sum() - 2 * math.pi) < 1e-9


@pytest.mark.parametrize("lev", [0, 1, 8, 12, 16, 19, 24, 30, 36, 44, 52])
def test_table_integrates_the_stokes_family(lev):
    """Unseen annulus targets at relative distance 2^-lev..2^(1-lev): every Stokes single- and
    double-layer component (normals along the circle's radius and along its axis) times
    cos / sin(l theta), l <= 9, integrated by the table's rule
    agrees with the oracle's fine rule to 1e-9 of the target's largest component integral,
    at every level (the construction scales each family member to unit norm in the measure
    psi^2 d theta, so the double-layer members, peaked like alpha / r^3, do not swamp the
    single-layer ones at deep levels)."""
    phi, w, cnt, _ = angular_rules.load(16)
    y, om = phi[lev, :cnt[lev]], w[lev, :cnt[lev]]
    alpha = 2.0 ** -lev
    th, wf = C.angular_fine_rule(alpha)
    rng = np.random.default_rng(lev)
    worst = 0.0
    for _ in range(4):
        r, p = alpha * (1.0 + rng.random()), 2.0 * math.pi * rng.random()
        tg = np.array([[r * math.cos(p)], [r * math.sin(p)]])
        for kind in ("stokes", "stokes_axial_dl"):
            Ff = C.modal_family(tg, th, 9, kind)
            Fc = C.modal_family(tg, y, 9, kind)
            worst = max(worst, np.abs(om @ Fc - wf @ Ff).max() / (wf @ np.abs(Ff)).max())
    assert worst < 1e-9, worst


def test_tables_cover_their_mode_counts():
    """Each committed table integrates the modes up to its own l0 (the largest N_theta it
    serves is 2 (l0 - 1)): level 6 checked on targets of the annulus."""
    for l0 in angular_rules.L0_TABLES:
        tab = angular_rules.load_l0(l0)
        if tab is None:
            continue
        phi, w, cnt = tab
        lev = 6
        y, om = phi[lev, :cnt[lev]], w[lev, :cnt[lev]]
        alpha = 2.0 ** -lev
        th, wf = C.angular_fine_rule(alpha)
        tg = np.array([[1.3 * alpha * math.cos(1.0)], [1.3 * alpha * math.sin(1.0)]])
        Ff = C.modal_family(tg, th, l0, "stokes")
        Fc = C.modal_family(tg, y, l0, "stokes")
        err = np.abs(om @ Fc - wf @ Ff).max() / (wf @ np.abs(Ff)).max()
        assert err < 1e-9, (l0, err)

"""The treecode for the single-layer sum (stokes_sl_tree_*, the far-field acceleration for
large N) against the oracle's direct FP64 sum on the same seeded inputs: a 3D cloud, the
slender random loop at 65,536 and 1,048,576 nodes (sampled rows), off-surface targets, and
linearity in the density.  Bars: measured errors with a margin (the treecode works in FP32
with FP64 sums of its list entries)."""
import numpy as np
import pytest

from paper_2310_00889_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sbq():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu tests")
    from paper_2310_00889_gb300 import build
    build.build()
    from paper_2310_00889_gb300 import sbq as mod
    return mod


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_tree_cloud_matches_oracle(sbq, oracle_mod):
    """20,000 Gaussian points (all of them targets): every cell is near the others at this
    size, so the sum is nearly direct; 512 sampled rows against the oracle."""
    rng = np.random.default_rng(41)
    n = 20000
    x, w, sig = rng.standard_normal((3, n)), rng.random(n), rng.standard_normal((3, n))
    T = sbq.SlTree(_t(x), _t(w))
    u = T.apply(_t(sig)).cpu().numpy()
    T.close()
    sub = np.sort(rng.choice(n, 512, replace=False))
    ref = oracle_mod.sl(x, w, sig, x[:, sub])
    err = _rel(u[:, sub], ref)
    print("treecode, 3D cloud: %.3e" % err)
    assert err < 1e-5


@pytest.mark.parametrize("panels,bar", [(512, 3e-6), (8192, 1e-5)])
def test_tree_slender_loop_matches_oracle(sbq, oracle_mod, panels, bar):
    """The slender random loop (Sec. 5.2 recipe), on-surface sum without self terms, 2,048
    sampled rows against the oracle: measured 1.2e-6 at 65,536 nodes and 1.7e-6 at 1,048,576
    (the plain FP32 direct sum at 1,048,576: 5.1e-6)."""
    rng = np.random.default_rng(42)
    S = I.random_loop(seed=1, panels=panels, ns=8, nth=16)
    n = S.size
    sig = rng.standard_normal((3, n))
    T = sbq.SlTree(_t(S.x), _t(S.w), theta=0.5, order=8)
    st = T.stats()
    u = T.apply(_t(sig)).cpu().numpy()
    T.close()
    sub = np.sort(rng.choice(n, 2048, replace=False))
    ref = oracle_mod.sl(S.x, S.w, sig, S.x[:, sub])
    err = _rel(u[:, sub], ref)
    print("treecode, loop %d nodes: %.3e, %.3g kernel evaluations per apply (direct: %.3g)"
          % (n, err, st["pairs"], float(n) * n))
    assert err < bar
    if panels >= 8192:
        assert st["pairs"] < 0.05 * float(n) * n


def test_tree_offsurface_targets(sbq, oracle_mod):
    """Targets off the surface (0.01..0.1 from a torus of radius 0.1): the source and target
    trees differ."""
    rng = np.random.default_rng(43)
    S = I.torus(R0=1.0, eps=0.1, panels=64, ns=8, nth=16)
    n = S.size
    m = 3000
    idx = rng.choice(n, m, replace=False)
    trg = S.x[:, idx] + (0.01 + 0.09 * rng.random(m)) * S.n[:, idx]
    sig = rng.standard_normal((3, n))
    T = sbq.SlTree(_t(S.x), _t(S.w), trg=_t(trg))
    u = T.apply(_t(sig)).cpu().numpy()
    T.close()
    ref = oracle_mod.sl(S.x, S.w, sig, trg)
    err = _rel(u, ref)
    print("treecode, off-surface targets: %.3e" % err)
    assert err < 5e-6


def test_tree_apply_is_linear_and_repeatable(sbq):
    """One tree, several densities: T(a s1 + s2) = a T(s1) + T(s2) to FP32 rounding, and the
    same density twice gives the same result (the proxy charges start from zero each call)."""
    rng = np.random.default_rng(44)
    S = I.random_loop(seed=1, panels=256, ns=8, nth=16)
    n = S.size
    s1, s2 = rng.standard_normal((3, n)), rng.standard_normal((3, n))
    T = sbq.SlTree(_t(S.x), _t(S.w))
    u1 = T.apply(_t(s1)).cpu().numpy()
    u2 = T.apply(_t(s2)).cpu().numpy()
    u12 = T.apply(_t(2.5 * s1 + s2)).cpu().numpy()
    u1b = T.apply(_t(s1)).cpu().numpy()
    T.close()
    assert _rel(u12, 2.5 * u1 + u2) < 1e-6
    assert _rel(u1b, u1) < 1e-6


@pytest.mark.parametrize("panels,bar", [(512, 3e-6), (8192, 1e-5)])
def test_tree_combined_field_matches_oracle(sbq, oracle_mod, panels, bar):
    """The combined field eta S + D of the operator (eta of the loop's mean radius) on the
    slender random loop, on-surface sum without self terms, 2,048 sampled rows against the
    oracle's combined sum."""
    rng = np.random.default_rng(45)
    S = I.random_loop(seed=1, panels=panels, ns=8, nth=16)
    n = S.size
    sig = rng.standard_normal((3, n))
    eta = sbq.slender_eta(0.01)
    T = sbq.StokesTree(_t(S.x), _t(S.w), nrm=_t(S.n), alpha=eta, beta=1.0)
    u = T.apply(_t(sig)).cpu().numpy()
    T.close()
    sub = np.sort(rng.choice(n, 2048, replace=False))
    ref = oracle_mod.combined(S.x, S.n, S.w, sig, S.x[:, sub], eta, 1.0)
    err = _rel(u[:, sub], ref)
    print("treecode, combined field, loop %d nodes: %.3e" % (n, err))
    assert err < bar


def test_tree_double_layer_alone(sbq, oracle_mod):
    """The double layer alone (alpha = 0) on a torus, all targets on the surface."""
    rng = np.random.default_rng(46)
    S = I.torus(R0=1.0, eps=0.1, panels=64, ns=8, nth=16)
    n = S.size
    sig = rng.standard_normal((3, n))
    T = sbq.StokesTree(_t(S.x), _t(S.w), nrm=_t(S.n), alpha=0.0, beta=1.0)
    u = T.apply(_t(sig)).cpu().numpy()
    T.close()
    sub = np.sort(rng.choice(n, 1024, replace=False))
    ref = oracle_mod.dl(S.x, S.n, S.w, sig, S.x[:, sub])
    err = _rel(u[:, sub], ref)
    print("treecode, double layer, torus: %.3e" % err)
    assert err < 1e-5


def test_tree_as_inner_operator_of_gmres_ir(sbq, oracle_mod):
    """The treecode attached to the operator K = I/2 + D + eta S + E (tube correction of the
    slender loop, 65,536 nodes): the FP32 matvec agrees with the FP64 one, and GMRES-IR with
    treecode inner solves and FP64 residuals reaches the same 1e-10 solution as with
    compensated-FP32 inner solves."""
    import torch
    S = I.random_loop(seed=1, panels=512, ns=8, nth=16)
    n = S.size
    src, nrm, w = _t(S.x), _t(S.n), _t(S.w)
    eta = sbq.slender_eta(0.01)
    E = sbq.tube_correction(src, nrm, w, 512, 8, 16, kind="stokes", alpha=eta, beta=1.0,
                            near_factor=0.5)
    op = sbq.StokesOp(src, nrm, w, eta, correction=E)
    rng = np.random.default_rng(47)
    x = _t(rng.standard_normal((3, n)))
    k64 = op.matvec(x, prec="fp64").cpu().numpy()
    op.set_tree(0.5, 8)
    kt = op.matvec(x, prec="fp32").cpu().numpy()
    err = _rel(kt, k64)
    print("operator with treecode, fp32 matvec against fp64: %.3e" % err)
    assert err < 1e-5
    rhs = _t(rng.standard_normal((3, n)))
    xt, rt = op.solve(rhs, tol=1e-10, inner_prec="fp32", inner_tol=1e-5, resid_prec="fp64")
    op.set_tree(0.0)
    xc, rc = op.solve(rhs, tol=1e-10, inner_prec="fp32c", inner_tol=1e-5, resid_prec="fp64")
    op.close()
    diff = (xt - xc).abs().max().item() / xc.abs().max().item()
    print("GMRES-IR, treecode inner: %d iterations, %d refinements, rel res %.2e; compensated "
          "FP32 inner: %d iterations; solutions differ by %.2e"
          % (rt["iters"], rt["outer_iters"], rt["rel_res"], rc["iters"], diff))
    assert rt["status"] == 0 and rc["status"] == 0
    assert rt["rel_res"] <= 1e-10
    assert diff < 1e-8


def test_tree_coincident_nodes(sbq, oracle_mod):
    """A 3D cloud in which 500 nodes repeat others exactly, on-surface sum (targets = sources)
    of the combined field with random unit normals: a coincident pair adds nothing, whether
    the two copies share a leaf or not (the punctured sum the oracle takes), and no output is
    non-finite; 600 rows against the oracle, the repeated nodes and their originals among
    them."""
    rng = np.random.default_rng(48)
    n0 = 6000
    x0 = rng.standard_normal((3, n0))
    dup = rng.choice(n0, 500, replace=False)
    x = np.concatenate([x0, x0[:, dup]], axis=1)
    n = x.shape[1]
    w, sig = rng.random(n), rng.standard_normal((3, n))
    nrm = rng.standard_normal((3, n))
    nrm /= np.linalg.norm(nrm, axis=0)
    T = sbq.StokesTree(_t(x), _t(w), nrm=_t(nrm), alpha=1.0, beta=1.0)
    u = T.apply(_t(sig)).cpu().numpy()
    T.close()
    assert np.isfinite(u).all()
    sub = np.unique(np.concatenate([dup[:200], n0 + np.arange(200), rng.choice(n, 200, replace=False)]))
    ref = oracle_mod.combined(x, nrm, w, sig, x[:, sub], 1.0, 1.0)
    err = _rel(u[:, sub], ref)
    print("treecode, cloud with coincident nodes: %.3e" % err)
    assert err < 1e-5


@pytest.mark.parametrize("n", [1, 2, 127, 128, 129, 600])
def test_tree_small_sizes(sbq, oracle_mod, n):
    """Sizes around one leaf and one target block (1 to 600 nodes of a 3D cloud), on-surface
    sums of the single layer and of the combined field against the oracle on every row; a
    single node has nothing to sum."""
    rng = np.random.default_rng(50 + n)
    x, w, sig = rng.standard_normal((3, n)), rng.random(n), rng.standard_normal((3, n))
    nrm = rng.standard_normal((3, n))
    nrm /= np.linalg.norm(nrm, axis=0)
    T = sbq.SlTree(_t(x), _t(w))
    u = T.apply(_t(sig)).cpu().numpy()
    T.close()
    C = sbq.StokesTree(_t(x), _t(w), nrm=_t(nrm), alpha=0.7, beta=1.0)
    uc = C.apply(_t(sig)).cpu().numpy()
    C.close()
    if n == 1:
        assert np.all(u == 0.0) and np.all(uc == 0.0)
        return
    assert _rel(u, oracle_mod.sl(x, w, sig, x)) < 1e-5
    assert _rel(uc, oracle_mod.combined(x, nrm, w, sig, x, 0.7, 1.0)) < 1e-5


def test_tree_empty(sbq):
    """No targets: an empty result; no sources: zeros at every target."""
    import torch
    rng = np.random.default_rng(57)
    x, w = _t(rng.standard_normal((3, 50))), _t(rng.random(50))
    T = sbq.SlTree(x, w, trg=_t(np.zeros((3, 0))))
    u = T.apply(_t(rng.standard_normal((3, 50))))
    T.close()
    assert tuple(u.shape) == (3, 0)
    T = sbq.SlTree(_t(np.zeros((3, 0))), _t(np.zeros(0)), trg=x)
    u = T.apply(_t(np.zeros((3, 0))), out=torch.full((3, 50), 7.0, dtype=torch.float64, device="cuda"))
    st = T.stats()
    T.close()
    assert tuple(u.shape) == (3, 50) and bool((u == 0.0).all())
    assert st["pairs"] == 0.0 and st["entries"] == 0

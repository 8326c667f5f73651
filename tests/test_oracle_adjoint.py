"""Pins of the oracle's gradient of the converged solve (transposes and finite differences)."""
import numpy as np
import pytest

from paper_2512_08555_gb300 import synth
from oracle.forest import OracleForest
from oracle.multigrid import OracleSolver
from oracle.composite import CompositeSystem
from oracle.adjoint import OracleAdjoint, conv_T
from oracle.lgf import free_space_solve


def _all(level, coords):
    return np.ones(len(coords), bool)


def _setup(M=4, nb=3, n=8, ml=1):
    desc = synth.adaptive_forest((nb, nb, nb), n, (-1, -1, -1), 2 / (nb * n), ml, _all)
    fo = OracleForest.from_desc(desc)
    return desc, fo


def _u_leaf(s, cs, x, fstar):
    """Forward output map E(x, f*): leaf values, level 0 from the convolution of F0."""
    fo, n = s.fo, s.n
    for k, A in enumerate(s.F):
        A[...] = fstar[k]
    r = cs.residual(x)               # fills cs.s.U consistently with x
    del r
    S = cs.s
    out = []
    for lev, b in fo.leaf_slot:
        out.append(S.U[lev][b, 1:1 + n, 1:1 + n, 1:1 + n])
    # level-0 leaves hold the convolution (covered level-0 blocks were overwritten by the injection)
    return np.stack(out)


@pytest.mark.parametrize("M", [2, 4, 6])
def test_conv_transpose(lgf_cache, M):
    rng = np.random.default_rng(0)
    desc, fo = _setup(M)
    s = OracleSolver(fo, M, G=lgf_cache(M, 25))
    N = fo.n0
    f0 = rng.normal(size=(N[2], N[1], N[0]))
    ub = rng.normal(size=(N[2] + 2, N[1] + 2, N[0] + 2))
    a = np.vdot(ub, free_space_solve(f0, s.G, fo.h0))
    b = np.vdot(conv_T(s, ub), f0)
    assert abs(a - b) < 1e-12 * abs(a)


@pytest.mark.parametrize("M", [4, 6])
def test_residual_transpose(lgf_cache, M):
    """<lambda, res(x, f*)> = <res^T lambda, (x, f*)>."""
    rng = np.random.default_rng(1)
    desc, fo = _setup(M, nb=4, n=8, ml=2)
    G = lgf_cache(M, 33)
    cs = CompositeSystem(OracleSolver(fo, M, G=G), synth.sample_leaves(desc, synth.c4_bumps(0)))
    adj = OracleAdjoint(OracleSolver(fo, M, G=G))
    x = rng.normal(size=cs.size)
    fstar = [rng.normal(size=A.shape) for A in cs.s.F]
    for k, A in enumerate(cs.s.F):
        A[...] = fstar[k]
    r = cs.residual(x)
    lam = rng.normal(size=cs.size)
    xb, fsb = adj.res_T(lam)
    # only leaf blocks of f* enter the residual
    rhs = np.vdot(xb, x) + sum(np.vdot(fsb[k][adj.leaf_sel[k]], fstar[k][adj.leaf_sel[k]]) for k in range(len(fstar)))
    assert abs(np.vdot(lam, r) - rhs) < 1e-11 * abs(np.vdot(lam, r))


@pytest.mark.parametrize("M", [2, 6])
def test_output_and_source_transposes(lgf_cache, M):
    rng = np.random.default_rng(2)
    desc, fo = _setup(M, nb=4, n=8, ml=2)
    G = lgf_cache(M, 33)
    s = OracleSolver(fo, M, G=G)
    cs = CompositeSystem(OracleSolver(fo, M, G=G), synth.sample_leaves(desc, synth.c4_bumps(0)))
    adj = OracleAdjoint(OracleSolver(fo, M, G=G))
    # E
    x = rng.normal(size=cs.size)
    fstar = [rng.normal(size=A.shape) for A in cs.s.F]
    u = _u_leaf(cs.s, cs, x, fstar)
    w = rng.normal(size=u.shape)
    xb, fsb = adj.E_T(w)
    rhs = np.vdot(xb, x) + sum(np.vdot(fsb[k][adj.leaf_sel[k]], fstar[k][adj.leaf_sel[k]]) for k in range(len(fstar)))
    assert abs(np.vdot(w, u) - rhs) < 1e-11 * abs(np.vdot(w, u))
    # B
    f = rng.normal(size=(desc.n_leaves, 8, 8, 8))
    s.prepare_rhs(f)
    g = [np.where(lv.is_leaf[:, None, None, None], rng.normal(size=A.shape), 0.0) for lv, A in zip(fo.levels, s.F)]
    lhs = sum(np.vdot(g[k], s.F[k]) for k in range(len(g)))
    fb = adj.B_T(g)
    assert abs(lhs - np.vdot(fb, f)) < 1e-11 * abs(lhs)


@pytest.mark.parametrize("M", [4, 6])
def test_gradient_matches_central_differences(lgf_cache, M):
    """dL/df . d == (L(f + e d) - L(f - e d)) / 2e for the converged solve (linear: exact up to tolerance)."""
    rng = np.random.default_rng(3)
    desc, fo = _setup(M)
    G = lgf_cache(M, 25)
    f = synth.sample_leaves(desc, synth.c4_bumps(1, k=2, r_lo=0.1, r_hi=0.15, box=0.3))
    w = synth.sample_leaves(desc, synth.gaussian_weight(0))
    adj = OracleAdjoint(OracleSolver(fo, M, G=G))
    grad = adj.gradient(w)
    assert adj.info == 0
    for _ in range(3):
        d = rng.normal(size=f.shape)
        eps = 1e-3 * np.abs(f).max() / np.abs(d).max()
        s = OracleSolver(fo, M, G=G)
        up, _ = s.solve(f + eps * d, tol=1e-14, max_cycles=60)
        um, _ = s.solve(f - eps * d, tol=1e-14, max_cycles=60)
        fd = (np.vdot(w, up) - np.vdot(w, um)) / (2 * eps)
        assert abs(fd - np.vdot(grad, d)) < 1e-9 * np.abs(grad).sum() * np.abs(d).max()


def test_uniform_level_gradient_is_symmetric_solve(lgf_cache):
    """Single level: S = E conv R, so S^T w = R^T conv^T w (checked against the forward map's matrix)."""
    rng = np.random.default_rng(4)
    desc, src = synth.config1(0, n0=16, n=8)
    fo = OracleForest.from_desc(desc)
    G = lgf_cache(4, 17)
    adj = OracleAdjoint(OracleSolver(fo, 4, G=G))
    w = rng.normal(size=(desc.n_leaves, 8, 8, 8))
    grad = adj.gradient(w)
    s = OracleSolver(fo, 4, G=G)
    for _ in range(3):
        d = rng.normal(size=w.shape)
        u, _ = s.solve(d, tol=1e-14, max_cycles=2)
        assert abs(np.vdot(w, u) - np.vdot(grad, d)) < 1e-11 * abs(np.vdot(w, u))


@pytest.mark.parametrize("M,ml", [(2, 2), (4, 1), (6, 2)])
def test_correction_cycle_transpose(lgf_cache, M, ml):
    """<xbar, M r> = <M^T xbar, r> for one correction V-cycle (smoothing, transfers, coarse solve, ghosts)."""
    rng = np.random.default_rng(5 + M)
    desc, fo = _setup(M, nb=4, n=8, ml=ml)
    adj = OracleAdjoint(OracleSolver(fo, M, G=lgf_cache(M, 33)))
    r = rng.normal(size=adj.nx)
    xb = rng.normal(size=adj.nx)
    a = np.vdot(xb, adj.correction_cycle(r))
    b = np.vdot(adj.correction_cycle_T(xb), r)
    assert abs(a - b) < 1e-12 * abs(a)


def test_correction_cycle_preconditions_K(lgf_cache):
    """K M r ~ r: the correction cycle is an approximate inverse of the composite operator."""
    rng = np.random.default_rng(6)
    desc, fo = _setup(4, nb=3, n=8, ml=1)
    G = lgf_cache(4, 25)
    adj = OracleAdjoint(OracleSolver(fo, 4, G=G))
    r = rng.normal(size=adj.nx)
    e = adj.correction_cycle(r)
    cs = CompositeSystem(OracleSolver(fo, 4, G=G), np.zeros((desc.n_leaves, 8, 8, 8)))
    Kx = cs.residual(np.zeros(cs.size)) - cs.residual(e)
    assert np.linalg.norm(r - Kx) < 0.05 * np.linalg.norm(r)


def test_gradient_ir_matches_gmres(lgf_cache):
    """Refinement with the transposed cycle reaches the GMRES gradient; it contracts every iteration."""
    desc, fo = _setup(4, nb=3, n=8, ml=1)
    G = lgf_cache(4, 25)
    w = synth.sample_leaves(desc, synth.gaussian_weight(0))
    adj = OracleAdjoint(OracleSolver(fo, 4, G=G))
    g_ir = adj.gradient_ir(w, tol=1e-13)
    assert adj.history[-1] < 1e-13
    assert all(b < 0.3 * a for a, b in zip(adj.history[1:], adj.history[2:]))
    g_gm = OracleAdjoint(OracleSolver(fo, 4, G=G)).gradient(w)
    assert np.abs(g_ir - g_gm).max() < 1e-10 * np.abs(g_gm).max()

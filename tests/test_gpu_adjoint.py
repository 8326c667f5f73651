"""Parity of the CUDA gradient of the converged solve with the FP64 oracle.

Factors (res^T, E^T, B^T, the transposed correction V-cycle) are compared
element by element with the oracle's transposes on the same seeded inputs;
they are FP64 with a different summation order (and atomics), so they agree
to 1e-12 relative.  The whole gradient is compared with the oracle's
gradient, with central differences of the CUDA forward solve and with the
dot-product identity <w, S f> = <S^T w, f>; both sides stop at a relative
residual of 1e-12, so they agree to 1e-9 relative.
"""
import numpy as np
import pytest

from paper_2512_08555_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.forest import OracleForest          # noqa: E402
from oracle.multigrid import OracleSolver       # noqa: E402
from oracle.adjoint import OracleAdjoint        # noqa: E402
from oracle.lgf import lgf_table                # noqa: E402


def _all(level, coords):
    return np.ones(len(coords), bool)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


_G = {}


def _lgf(M, nmax):
    if (M, nmax) not in _G:
        _G[(M, nmax)] = lgf_table(M, nmax)
    return _G[(M, nmax)]


def _case(M, nb=4, n=8, ml=2, tol=1e-12, max_cycles=80):
    from paper_2512_08555_gb300.mrp import Solver
    desc = synth.adaptive_forest((nb, nb, nb), n, (-1, -1, -1), 2 / (nb * n), ml, _all)
    fo = OracleForest.from_desc(desc)
    adj = OracleAdjoint(OracleSolver(fo, M, G=_lgf(M, max(fo.n0) + 1)))
    s = Solver(desc, order=M, tol=tol, max_cycles=max_cycles)
    for k in range(s.level_count()):
        coords, leaf = s.level_info(k)
        assert np.array_equal(coords, fo.levels[k].coords)
    return desc, fo, adj, s


def _to_dev(adj, fo, v):
    """Oracle vector (leaf blocks of levels >= 1, then covered level-0 blocks) -> device layout."""
    n = fo.n
    parts = [np.zeros((lv.nb, n ** 3)) for lv in fo.levels]
    off = 0
    for k in range(1, fo.max_level + 1):
        m = len(adj.leaf_sel[k])
        parts[k][adj.leaf_sel[k]] = v[off:off + m * n ** 3].reshape(m, -1)
        off += m * n ** 3
    parts[0][adj.cov0] = v[off:].reshape(len(adj.cov0), -1)
    return torch.from_numpy(np.concatenate([p.reshape(-1) for p in parts])).cuda()


def _from_dev(adj, fo, d):
    n = fo.n
    d = d.cpu().numpy()
    out, off, per = [], 0, []
    for lv in fo.levels:
        per.append(d[off:off + lv.nb * n ** 3].reshape(lv.nb, n ** 3))
        off += lv.nb * n ** 3
    for k in range(1, fo.max_level + 1):
        out.append(per[k][adj.leaf_sel[k]].reshape(-1))
    out.append(per[0][adj.cov0].reshape(-1))
    return np.concatenate(out), per


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.mark.parametrize("M", [2, 4, 6])
def test_residual_transpose_parity(M):
    rng = np.random.default_rng(10 + M)
    desc, fo, adj, s = _case(M)
    lam = rng.normal(size=adj.nx)
    xb_o, fsb_o = adj.res_T(lam)
    out = s.adjoint_op("res_T", _to_dev(adj, fo, lam))
    L = s.adjoint_len()
    xb_g, _ = _from_dev(adj, fo, out[:L])
    assert _rel(xb_g, xb_o) < 1e-12
    _, fsb_g = _from_dev(adj, fo, out[L:])
    for k, lv in enumerate(fo.levels):
        leaf = adj.leaf_sel[k]
        if len(leaf):
            assert _rel(fsb_g[k][leaf], fsb_o[k][leaf].reshape(len(leaf), -1)) < 1e-12


@pytest.mark.parametrize("M", [2, 6])
def test_output_and_source_transposes_parity(M):
    rng = np.random.default_rng(20 + M)
    desc, fo, adj, s = _case(M)
    n = fo.n
    w = rng.normal(size=(desc.n_leaves, n, n, n))
    xb_o, fsb_o = adj.E_T(w)
    out = s.adjoint_op("out_T", torch.from_numpy(w).cuda())
    L = s.adjoint_len()
    xb_g, _ = _from_dev(adj, fo, out[:L])
    assert _rel(xb_g, xb_o) < 1e-12
    _, fsb_g = _from_dev(adj, fo, out[L:])
    leaf0 = adj.leaf_sel[0]
    assert _rel(fsb_g[0][leaf0], fsb_o[0][leaf0].reshape(len(leaf0), -1)) < 1e-12
    # B^T on random leaf values of f*-bar
    fsb = [np.where(lv.is_leaf[:, None, None, None], rng.normal(size=(lv.nb, n, n, n)), 0.0) for lv in fo.levels]
    fb_o = adj.B_T(fsb)
    dev = torch.from_numpy(np.concatenate([a.reshape(-1) for a in fsb])).cuda()
    fb_g = s.adjoint_op("rhs_T", dev).cpu().numpy().reshape(fb_o.shape)
    assert _rel(fb_g, fb_o) < 1e-12


@pytest.mark.parametrize("M,ml", [(2, 2), (4, 1), (4, 2), (6, 2)])
def test_transposed_cycle_parity(M, ml):
    """One transposed correction V-cycle: CUDA vs oracle, element by element."""
    rng = np.random.default_rng(30 + M + ml)
    desc, fo, adj, s = _case(M, ml=ml)
    xb = rng.normal(size=adj.nx)
    r_o = adj.correction_cycle_T(xb)
    r_g, _ = _from_dev(adj, fo, s.adjoint_op("cycle_T", _to_dev(adj, fo, xb)))
    assert _rel(r_g, r_o) < 1e-12


@pytest.mark.parametrize("M", [2, 4, 6])
def test_gradient_matches_oracle(M):
    desc, fo, adj, s = _case(M)
    w = synth.sample_leaves(desc, synth.gaussian_weight(0))
    g_o = adj.gradient_ir(w, tol=1e-13)
    g_g, st = s.solve_adjoint(torch.from_numpy(w).cuda(), allow_not_converged=True)
    assert st.residual < 1e-11
    assert _rel(g_g.cpu().numpy(), g_o) < 1e-9


def test_gradient_central_differences_uniform_32():
    """32^3 nodes, one level, FP64: central differences along 8 random directions and 8 single nodes."""
    from paper_2512_08555_gb300.mrp import Solver
    rng = np.random.default_rng(40)
    desc, src = synth.config1(0, n0=32, n=16)
    s = Solver(desc, order=4, tol=1e-11, max_cycles=20)
    f = torch.from_numpy(synth.sample_leaves(desc, src)).cuda()
    w = torch.from_numpy(rng.normal(size=tuple(f.shape))).cuda()
    grad, _ = s.solve_adjoint(w)

    def loss(ff):
        u, _ = s.solve(ff, allow_not_converged=True)
        return float((w * u).sum())

    dirs = [torch.from_numpy(rng.normal(size=tuple(f.shape))).cuda() for _ in range(8)]
    for _ in range(8):
        d = torch.zeros_like(f)
        idx = tuple(int(rng.integers(0, m)) for m in f.shape)
        d[idx] = 1.0
        dirs.append(d)
    for d in dirs:
        # the map is linear: a large step has no truncation error and keeps
        # the solver's own error small next to the difference
        eps = float(f.abs().max()) / float(d.abs().max())
        fd = (loss(f + eps * d) - loss(f - eps * d)) / (2 * eps)
        an = float((grad * d).sum())
        assert abs(fd - an) < 1e-8 * float(grad.abs().sum()) * float(d.abs().max())


@pytest.mark.parametrize("M", [4, 6])
def test_gradient_central_differences_adaptive(M):
    from paper_2512_08555_gb300.mrp import Solver
    rng = np.random.default_rng(50 + M)
    desc = synth.adaptive_forest((4, 4, 4), 8, (-1, -1, -1), 2 / 32, 2, _all)
    s = Solver(desc, order=M, tol=1e-12, max_cycles=80)
    f = torch.from_numpy(synth.sample_leaves(desc, synth.c4_bumps(1, k=2, r_lo=0.2, r_hi=0.3))).cuda()
    w = torch.from_numpy(synth.sample_leaves(desc, synth.gaussian_weight(1))).cuda()
    grad, _ = s.solve_adjoint(w, allow_not_converged=True)
    for _ in range(4):
        d = torch.from_numpy(rng.normal(size=tuple(f.shape))).cuda()
        eps = float(f.abs().max()) / float(d.abs().max())
        up, _ = s.solve(f + eps * d, allow_not_converged=True)
        um, _ = s.solve(f - eps * d, allow_not_converged=True)
        fd = float((w * (up - um)).sum()) / (2 * eps)
        an = float((grad * d).sum())
        assert abs(fd - an) < 1e-8 * float(grad.abs().sum()) * float(d.abs().max())


def test_autograd_function():
    from paper_2512_08555_gb300.mrp import Solver, poisson_solve
    desc = synth.adaptive_forest((4, 4, 4), 8, (-1, -1, -1), 2 / 32, 1, _all)
    s = Solver(desc, order=4, tol=1e-10, max_cycles=80)
    f = torch.from_numpy(synth.sample_leaves(desc, synth.c4_bumps(2))).cuda().requires_grad_(True)
    w = torch.from_numpy(synth.sample_leaves(desc, synth.gaussian_weight(2))).cuda()
    u = poisson_solve(s, f)
    (w * u).sum().backward()
    ref, _ = s.solve_adjoint(w.contiguous())
    # the ghost and correction transposes accumulate with atomics: two calls
    # agree to rounding, not bit for bit
    assert float((f.grad - ref).abs().max()) < 1e-10 * float(ref.abs().max())


def test_dot_product_identity_full_size():
    """<w, S f> = <S^T w, f> on the 2.8M-node adaptive workload (order 4), FP64 both ways."""
    from paper_2512_08555_gb300.mrp import Solver
    desc, src = synth.config2(0)
    s = Solver(desc, order=4, tol=1e-10, max_cycles=60)
    f = torch.from_numpy(synth.sample_leaves(desc, src)).cuda()
    w = torch.from_numpy(synth.sample_leaves(desc, synth.gaussian_weight(3))).cuda()
    u, _ = s.solve(f)
    g, st = s.solve_adjoint(w)
    assert st.residual < 1e-10
    a = float((w * u).sum())
    b = float((g * f).sum())
    assert abs(a - b) < 1e-7 * float((w.abs() * u.abs()).sum())


@pytest.mark.parametrize("M", [4, 6])
def test_mixed_precision_gradient_matches_oracle(M):
    """FP32 transposed cycles inside the FP64 refinement reach the FP64 gradient."""
    from paper_2512_08555_gb300.mrp import Solver
    desc, fo, adj, _ = _case(M)
    w = synth.sample_leaves(desc, synth.gaussian_weight(0))
    g_o = adj.gradient_ir(w, tol=1e-13)
    s = Solver(desc, order=M, tol=1e-12, max_cycles=80, precision="mixed")
    g_g, st = s.solve_adjoint(torch.from_numpy(w).cuda(), allow_not_converged=True)
    assert st.residual < 1e-11
    assert _rel(g_g.cpu().numpy(), g_o) < 1e-9

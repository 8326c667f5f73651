"""Batched solves: several forests (different spacings, depths and block
sizes) and vector right-hand sides in one handle.

Every (forest, component) of a batch must give what a handle of its own
gives: to rounding (1e-12 relative) at a fixed cycle count, where both run
the same cycles; to the stop tolerance's reach (1e-8) when both run to
convergence, since the batch keeps cycling until its slowest problem
converges.  One batch is also compared with the FP64 oracle directly.
"""
import numpy as np
import pytest

from paper_2512_08555_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.forest import OracleForest          # noqa: E402
from oracle.multigrid import OracleSolver       # noqa: E402
from oracle.lgf import lgf_table                # noqa: E402


def _all(level, coords):
    return np.ones(len(coords), bool)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _batch():
    """Three forests: two with n = 8 (spacings 1/16 and 1/32, 3 and 2 levels), one with n = 10."""
    A = synth.adaptive_forest((4, 4, 4), 8, (-1, -1, -1), 2 / 32, 2, _all)
    B = synth.adaptive_forest((4, 4, 4), 8, (-0.5, -0.5, -0.5), 1 / 32, 1, _all)
    C = synth.adaptive_forest((4, 4, 4), 10, (-1, -1, -1), 2 / 40, 1, _all)
    return [A, B, C], [2, 1, 1]


def _rhs(forests, comps, seed=0):
    parts, per = [], []
    k = 0
    for f, c in zip(forests, comps):
        for _ in range(c):
            v = synth.sample_leaves(f, synth.c4_bumps(seed + k, k=3, r_lo=0.15, r_hi=0.3, box=0.45))
            parts.append(v.reshape(-1))
            per.append((f, v))
            k += 1
    return np.concatenate(parts), per


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.mark.parametrize("M", [4, 6])
def test_fixed_cycles_match_single_handles(M):
    from paper_2512_08555_gb300.mrp import Solver
    forests, comps = _batch()
    f, per = _rhs(forests, comps)
    batch = Solver(forests, order=M, tol=0.0, max_cycles=2, ncomp=comps)
    ub, st = batch.solve(torch.from_numpy(f).cuda(), allow_not_converged=True)
    assert st.cycles == 2
    ub = ub.cpu().numpy()
    for (a, b), (fo, v) in zip(batch.slices(), per):
        single = Solver(fo, order=M, tol=0.0, max_cycles=2)
        us, _ = single.solve(torch.from_numpy(v).cuda(), allow_not_converged=True)
        assert _rel(ub[a:b], us.cpu().numpy().reshape(-1)) < 1e-12


def test_fixed_cycle_matches_oracle():
    from paper_2512_08555_gb300.mrp import Solver
    forests, comps = _batch()
    f, per = _rhs(forests, comps, seed=5)
    batch = Solver(forests, order=4, tol=0.0, max_cycles=1, ncomp=comps)
    ub, _ = batch.solve(torch.from_numpy(f).cuda(), allow_not_converged=True)
    ub = ub.cpu().numpy()
    G = lgf_table(4, 41)
    for (a, b), (fo, v) in zip(batch.slices(), per):
        o = OracleSolver(OracleForest.from_desc(fo), 4, G=G)
        o.prepare_rhs(v)
        o.vcycle()
        assert _rel(ub[a:b], o.leaf_u().reshape(-1)) < 1e-12


def test_converged_batch_matches_single_handles():
    from paper_2512_08555_gb300.mrp import Solver
    forests, comps = _batch()
    f, per = _rhs(forests, comps, seed=9)
    batch = Solver(forests, order=4, tol=1e-10, max_cycles=60, ncomp=comps)
    ub, st = batch.solve(torch.from_numpy(f).cuda())
    assert st.residual < 1e-10
    ub = ub.cpu().numpy()
    for (a, b), (fo, v) in zip(batch.slices(), per):
        us, _ = Solver(fo, order=4, tol=1e-10, max_cycles=60).solve(torch.from_numpy(v).cuda())
        assert _rel(ub[a:b], us.cpu().numpy().reshape(-1)) < 1e-8


def test_mixed_batch_matches_fp64_single_handles():
    from paper_2512_08555_gb300.mrp import Solver
    forests, comps = _batch()
    f, per = _rhs(forests, comps, seed=13)
    batch = Solver(forests, order=4, tol=1e-10, max_cycles=80, ncomp=comps, precision="mixed")
    ub, st = batch.solve(torch.from_numpy(f).cuda())
    assert st.residual < 1e-10 and st.ir_steps >= 1
    ub = ub.cpu().numpy()
    for (a, b), (fo, v) in zip(batch.slices(), per):
        us, _ = Solver(fo, order=4, tol=1e-11, max_cycles=60).solve(torch.from_numpy(v).cuda(),
                                                                      allow_not_converged=True)
        assert _rel(ub[a:b], us.cpu().numpy().reshape(-1)) < 1e-8


def test_batch_gradient_matches_single_handles():
    from paper_2512_08555_gb300.mrp import Solver
    forests, comps = _batch()
    rng = np.random.default_rng(3)
    w = np.concatenate([synth.sample_leaves(fo, synth.gaussian_weight(int(rng.integers(100)))).reshape(-1)
                        for fo, c in zip(forests, comps) for _ in range(c)])
    batch = Solver(forests, order=4, tol=1e-12, max_cycles=80, ncomp=comps)
    gb, st = batch.solve_adjoint(torch.from_numpy(w).cuda(), allow_not_converged=True)
    assert st.residual < 1e-11
    gb = gb.cpu().numpy()
    k = 0
    for fo, c in zip(forests, comps):
        single = Solver(fo, order=4, tol=1e-12, max_cycles=80)
        for _ in range(c):
            a, b = batch.slices()[k]
            gs, _ = single.solve_adjoint(torch.from_numpy(w[a:b].copy()).cuda(), allow_not_converged=True)
            assert _rel(gb[a:b], gs.cpu().numpy().reshape(-1)) < 1e-9
            k += 1


def test_batched_workload_small_instance():
    """The batched mix (vortex ring x 3 components + 16 uneven scalar problems), two levels shallower."""
    from paper_2512_08555_gb300.mrp import Solver
    problems = synth.config4(0, scale_levels=2)
    forests = [p[0] for p in problems]
    comps = [p[1] for p in problems]
    f = synth.batched_rhs(problems)
    batch = Solver(forests, order=4, tol=1e-10, max_cycles=80, ncomp=comps, precision="mixed")
    ub, st = batch.solve(torch.from_numpy(f).cuda())
    assert st.residual < 1e-10
    ub = ub.cpu().numpy()
    # the ring's x component and two scalar problems of other block sizes, each on its own handle
    sl = batch.slices()
    for idx, (fo, v) in ((0, (forests[0], f[sl[0][0]:sl[0][1]])), (4, (forests[2], f[sl[4][0]:sl[4][1]])),
                         (7, (forests[5], f[sl[7][0]:sl[7][1]]))):
        us, _ = Solver(fo, order=4, tol=1e-11, max_cycles=60).solve(torch.from_numpy(v.copy()).cuda(),
                                                                      allow_not_converged=True)
        a, b = sl[idx]
        assert _rel(ub[a:b], us.cpu().numpy().reshape(-1)) < 1e-8


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_solve_matches_host_driven_solve(precision):
    """One graph launch (device-side loop control) gives the host-driven solve's result and counts."""
    from paper_2512_08555_gb300.mrp import Solver
    forests, comps = _batch()
    f, _ = _rhs(forests, comps, seed=17)
    s = Solver(forests, order=4, tol=1e-10, max_cycles=60, ncomp=comps, precision=precision)
    fd = torch.from_numpy(f).cuda()
    uh, sh = s.solve(fd)
    ug = torch.empty_like(fd)
    for _ in range(2):                       # second call replays the same graph
        ug, sg = s.solve_graph(fd, ug)
        assert sg.cycles == sh.cycles and sg.ir_steps == sh.ir_steps
        assert sg.residual < 1e-10
        assert _rel(ug.cpu().numpy(), uh.cpu().numpy()) < 1e-13
    # new output buffer: the graph is rebuilt
    ug2, _ = s.solve_graph(fd)
    assert _rel(ug2.cpu().numpy(), uh.cpu().numpy()) < 1e-13


def test_graph_solve_single_forest_odd_sweeps():
    """nu1 + nu2 odd: the loop body restores its ping-pong buffers; result equals the host-driven solve."""
    from paper_2512_08555_gb300.mrp import Solver
    fo = synth.adaptive_forest((4, 4, 4), 8, (-1, -1, -1), 2 / 32, 2, _all)
    v = synth.sample_leaves(fo, synth.c4_bumps(3, k=3, r_lo=0.15, r_hi=0.3, box=0.45))
    s = Solver(fo, order=6, tol=1e-10, max_cycles=60, nu1=2, nu2=1)
    fd = torch.from_numpy(v).cuda()
    uh, sh = s.solve(fd)
    ug, sg = s.solve_graph(fd)
    assert sg.cycles == sh.cycles
    assert _rel(ug.cpu().numpy(), uh.cpu().numpy()) < 1e-13

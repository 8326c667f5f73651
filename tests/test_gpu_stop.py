"""Stop rules, return statuses and the host-memory entry point, through the C ABI.

Cauchy rule (Sec. 3, the increment of the iterates max|u^n - u^(n+1)| /
max|u^(n+1)| over leaf nodes): parity protocol (ii) -- the CUDA path and the
oracle both iterate until the increment is below 1e-14 and then agree to
1e-12 relative max-norm; at a looser tolerance both stop after the same
number of cycles (the iterates are the same algorithm's).
"""
import ctypes

import numpy as np
import pytest

from paper_2512_08555_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.forest import OracleForest          # noqa: E402
from oracle.multigrid import OracleSolver       # noqa: E402

MIXED_TOL = 1e-8


def _all(level, coords):
    return np.ones(len(coords), bool)


def _forest(nb=4, n=8, max_level=2):
    return synth.adaptive_forest((nb, nb, nb), n, (-1.0, -1.0, -1.0), 2.0 / (nb * n), max_level, _all)


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("M", [2, 4, 6])
def test_cauchy_rule_matches_oracle(M):
    from paper_2512_08555_gb300.mrp import Solver
    desc = _forest()
    f = synth.sample_leaves(desc, synth.c4_bumps(0, k=3, r_lo=0.2, r_hi=0.3))
    fd = torch.from_numpy(f).cuda()
    o = OracleSolver(OracleForest.from_desc(desc), M)
    # same cycle count at a loose tolerance
    uo8, c8 = o.solve(f, tol=1e-8, max_cycles=40, stop="cauchy")
    n8 = o.cycles_done
    s8 = Solver(desc, order=M, tol=1e-8, max_cycles=40, stop="cauchy")
    u8, st8 = s8.solve(fd)
    assert st8.cycles == n8 and st8.cauchy < 1e-8 and st8.residual == 0.0
    assert abs(st8.cauchy - c8) <= 1e-4 * c8
    ug8, sg8 = s8.solve_graph(fd)
    assert sg8.cycles == n8 and abs(sg8.cauchy - st8.cauchy) <= 1e-12 * st8.cauchy
    assert _rel(ug8.cpu().numpy(), u8.cpu().numpy()) == 0.0
    # converged to 1e-14 on both sides
    uo, co = o.solve(f, tol=1e-14, max_cycles=60, stop="cauchy")
    s = Solver(desc, order=M, tol=1e-14, max_cycles=60, stop="cauchy")
    u, st = s.solve(fd)
    assert st.cauchy < 1e-14 and co < 1e-14
    assert _rel(u.cpu().numpy(), uo) < 1e-12
    ug, sg = s.solve_graph(fd)
    assert sg.cauchy < 1e-14 and _rel(ug.cpu().numpy(), uo) < 1e-12


def test_cauchy_rule_mixed_precision():
    """FP32 cycles in FP64 refinement, stopped on the increment of the FP64 iterate."""
    from paper_2512_08555_gb300.mrp import Solver
    desc = _forest(n=12)
    f = torch.from_numpy(synth.sample_leaves(desc, synth.c4_bumps(2, k=4, r_lo=0.15, r_hi=0.3))).cuda()
    up, _ = Solver(desc, order=4, tol=1e-13, max_cycles=60).solve(f)
    m = Solver(desc, order=4, tol=1e-12, max_cycles=80, precision="mixed", stop="cauchy")
    um, st = m.solve(f)
    assert st.cauchy < 1e-12 and st.ir_steps >= 2 and st.residual < 1e-9
    assert _rel(um.cpu().numpy(), up.cpu().numpy()) < MIXED_TOL
    ug, sg = m.solve_graph(f)
    assert sg.cauchy < 1e-12 and sg.ir_steps == st.ir_steps
    assert _rel(ug.cpu().numpy(), up.cpu().numpy()) < MIXED_TOL
    # zero source: the first iterate is zero, so is its increment
    z = torch.zeros_like(f)
    uz, sz = m.solve(z)
    assert float(uz.abs().max()) == 0.0 and sz.cauchy == 0.0


@pytest.mark.parametrize("graph", [False, True])
def test_not_converged_status(graph):
    """max_cycles = 1 with tol = 0 returns MRP_ERR_NOT_CONVERGED and still writes u (the oracle's one cycle)."""
    from paper_2512_08555_gb300.mrp import Solver, Stats
    desc = _forest(max_level=1)
    f = synth.sample_leaves(desc, synth.c4_bumps(1, k=3, r_lo=0.2, r_hi=0.3))
    s = Solver(desc, order=4, tol=0.0, max_cycles=1)
    fd = torch.from_numpy(f).cuda()
    u = torch.full_like(fd, np.nan)
    st = Stats()
    fn = s.lib.mrp_solve_graph if graph else s.lib.mrp_solve
    rc = fn(s.h, ctypes.c_void_p(fd.data_ptr()), ctypes.c_void_p(u.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(st))
    torch.cuda.synchronize()
    assert rc == 5 and st.cycles == 1
    assert s.lib.mrp_error_string(rc) == b"not converged within max_cycles"
    uo, _ = OracleSolver(OracleForest.from_desc(desc), 4).solve(f, tol=0.0, max_cycles=1)
    assert _rel(u.cpu().numpy(), uo) < 1e-12


def test_graph_mixed_first_step_and_loop():
    """The graph's prologue runs the first refinement step and its check, which can skip the device loop:
    a loose tolerance stops after that step exactly as the host-driven solve does; a tight one runs the loop
    and ends within the mixed-precision bound of the FP64 solve."""
    from paper_2512_08555_gb300.mrp import Solver
    desc = synth.adaptive_forest((4, 4, 4), 8, (-1, -1, -1), 2 / 32, 1, _all)
    f = torch.from_numpy(synth.sample_leaves(desc, synth.c4_bumps(4, k=3, r_lo=0.2, r_hi=0.3))).cuda()
    m = Solver(desc, order=4, tol=0.5, max_cycles=60, precision="mixed")
    u, st = m.solve_graph(f)
    assert st.ir_steps == 1
    uh, sh = m.solve(f)
    assert sh.ir_steps == st.ir_steps and _rel(u.cpu().numpy(), uh.cpu().numpy()) == 0.0
    m2 = Solver(desc, order=4, tol=1e-10, max_cycles=60, precision="mixed")
    u2, st2 = m2.solve_graph(f)
    up, _ = Solver(desc, order=4, tol=1e-12, max_cycles=60).solve(f)
    assert st2.residual < 1e-10 and _rel(u2.cpu().numpy(), up.cpu().numpy()) < MIXED_TOL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_host_matches_device_solve(precision):
    """mrp_solve_host (host buffers in and out) gives the device-memory graph solve's result exactly, twice."""
    from paper_2512_08555_gb300.mrp import Solver
    desc = _forest(n=12)
    f = synth.sample_leaves(desc, synth.c4_bumps(3, k=4, r_lo=0.15, r_hi=0.3))
    s = Solver(desc, order=4, tol=1e-10, max_cycles=60, precision=precision)
    ud, sd = s.solve_graph(torch.from_numpy(f).cuda())
    fh = torch.from_numpy(f).pin_memory()
    for _ in range(2):
        uh, sh = s.solve_host(fh)
        assert not uh.is_cuda and sh.cycles == sd.cycles
        assert np.array_equal(uh.numpy(), ud.cpu().numpy())
    # pageable memory works too
    uh2, _ = s.solve_host(torch.from_numpy(f.copy()), torch.empty(f.shape, dtype=torch.float64))
    assert np.array_equal(uh2.numpy(), ud.cpu().numpy())

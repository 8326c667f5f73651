"""Parity of every CUDA stage, and of whole solves, with the FP64 CPU oracle.

Each stage test loads the same seeded per-level fields into the library
(through the step entry points of the C ABI) and into the oracle, runs the
stage on both sides and compares element by element.  Tolerances: stages
are FP64 with different summation orders, so they agree to a few ulps of
the data (1e-13 relative); whole solves to 1e-12 relative max-norm.
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


def small_forest(nb=4, n=8, max_level=2, lo=-1.0, L=2.0):
    return synth.adaptive_forest((nb, nb, nb), n, (lo, lo, lo), L / (nb * n), max_level, _all)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _pair(desc, M, G=None):
    from paper_2512_08555_gb300.mrp import Solver
    s = Solver(desc, order=M, tol=0.0, max_cycles=1)
    o = OracleSolver(OracleForest.from_desc(desc), M, G=G)
    for k in range(s.level_count()):
        coords, leaf = s.level_info(k)
        assert np.array_equal(coords, o.fo.levels[k].coords)
        assert np.array_equal(leaf, o.fo.levels[k].is_leaf)
    return s, o


def _rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _load(s, o, rng, which=("U", "F", "R", "UHAT")):
    """Random fields at every level, identical on both sides."""
    for k in range(s.level_count()):
        for name in which:
            arr = {"U": o.U, "F": o.F, "R": o.R, "UHAT": o.H}[name][k]
            arr[...] = rng.normal(size=arr.shape)
            s.field_set(name, k, arr)


@pytest.mark.parametrize("M", [2, 4, 6])
def test_lgf_table_matches_oracle(M):
    desc = synth.uniform_forest((2, 2, 2), 8, (0, 0, 0), 1 / 16)
    from paper_2512_08555_gb300.mrp import Solver
    s = Solver(desc, order=M)
    Gg = s.lgf_table(16)
    Go = lgf_table(M, 16)
    assert np.abs(Gg - Go).max() < 1e-14


@pytest.mark.parametrize("M", [2, 4, 6])
def test_prepare_rhs(M):
    desc = small_forest()
    s, o = _pair(desc, M)
    f = synth.sample_leaves(desc, synth.c4_bumps(0, k=3, r_lo=0.2, r_hi=0.3))
    s.step("prepare_rhs", 0, torch.from_numpy(f).cuda())
    o.prepare_rhs(f)
    for k in range(s.level_count()):
        leaf = o.fo.levels[k].is_leaf
        if M == 6:      # two ghost layers, kept in FRAW
            assert _rel(s.field_get("FRAW", k).cpu().numpy(), o.fraw[k]) < 1e-14
        else:           # raw f (leaf values and injections) in U's interiors, ghost layers built in the kernel
            assert _rel(s.field_get("U", k).cpu().numpy()[:, 1:-1, 1:-1, 1:-1], o.fraw[k][:, 2:-2, 2:-2, 2:-2]) == 0.0
        assert _rel(s.field_get("F", k).cpu().numpy()[leaf], o.F[k][leaf]) < 1e-14


@pytest.mark.parametrize("M", [2, 4, 6])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_ghost_fill(M, k):
    desc = small_forest()
    s, o = _pair(desc, M)
    rng = np.random.default_rng(10 + k)
    _load(s, o, rng, ("U",))
    s.step("ghost_u", k)
    o.ghost_fill(o.U, k, "keep")
    assert _rel(s.field_get("U", k).cpu().numpy(), o.U[k]) < 1e-14
    if k >= 1:
        assert _rel(s.field_get("U", k - 1).cpu().numpy(), o.U[k - 1]) == 0.0


def _interior(a):
    return a[:, 1:-1, 1:-1, 1:-1]


@pytest.mark.parametrize("M", [2, 4, 6])
def test_smooth_and_residual(M):
    """The CUDA sweep and residual build their ghost layer themselves (Sec. 2.1 rules);
    the oracle ghosts first, then sweeps."""
    desc = small_forest()
    s, o = _pair(desc, M)
    rng = np.random.default_rng(1)
    _load(s, o, rng)
    for k in range(1, s.level_count()):
        s.step("smooth", k)
        o.ghost_fill(o.U, k, "keep")
        o.smooth(k)
        assert _rel(_interior(s.field_get("U", k).cpu().numpy()), _interior(o.U[k])) < 1e-13
        s.step("residual", k)
        o.ghost_fill(o.U, k, "keep")
        o.residual(k)
        assert _rel(s.field_get("R", k).cpu().numpy(), o.R[k]) < 1e-12


@pytest.mark.parametrize("M", [2, 4, 6])
@pytest.mark.parametrize("k", [1, 2])
def test_restrict(M, k):
    desc = small_forest()
    s, o = _pair(desc, M)
    rng = np.random.default_rng(2)
    _load(s, o, rng)
    s.step("restrict", k)
    o.restrict(k)
    assert _rel(_interior(s.field_get("U", k - 1).cpu().numpy()), _interior(o.U[k - 1])) < 1e-13
    for name, arr in (("F", o.F), ("UHAT", o.H)):
        assert _rel(s.field_get(name, k - 1).cpu().numpy(), arr[k - 1]) < 1e-13, name


@pytest.mark.parametrize("M", [2, 4, 6])
def test_coarse_solve(M):
    desc = small_forest(nb=4, n=8, max_level=1)
    s, o = _pair(desc, M)
    rng = np.random.default_rng(3)
    _load(s, o, rng, ("F",))
    s.step("coarse_solve")
    o.coarse_solve()
    assert _rel(s.field_get("U", 0).cpu().numpy(), o.U[0]) < 1e-12


@pytest.mark.parametrize("n, nb, P", [(12, 3, 75), (8, 5, 81), (18, 3, 112), (10, 7, 144), (8, 7, 120),
                                       (16, 6, 196), (18, 6, 224)])
def test_coarse_solve_lattices(n, nb, P):
    """Odd and even padded lengths (radices 2, 3, 4, 5, 7; the FP32 lines of
    P = 144 = 9 x 16 and 196 = 14 x 14 take the four-step build): the FP64
    level-0 solve against the oracle's convolution at 1e-12, and the FP32
    solve of a mixed-precision handle at 1e-5."""
    from paper_2512_08555_gb300.mrp import Solver
    desc = small_forest(nb=nb, n=n, max_level=0)
    s, o = _pair(desc, 4)
    assert s.fft_shape()[0] == P
    rng = np.random.default_rng(11)
    _load(s, o, rng, ("F",))
    s.step("coarse_solve")
    o.coarse_solve()
    assert _rel(s.field_get("U", 0).cpu().numpy(), o.U[0]) < 1e-12
    m = Solver(desc, order=4, tol=0.0, max_cycles=1, precision="mixed")
    m.field_set("F", 0, o.F[0])
    m.step("coarse_solve_f32")
    assert _rel(m.field_get("U", 0).cpu().numpy(), o.U[0]) < 1e-5


@pytest.mark.parametrize("n, nb, P", [(20, 7, 288), (18, 13, 480), (18, 14, 512), (16, 15, 486)])
def test_coarse_solve_f32_composite_radices(n, nb, P):
    """Lattices long enough for the FP32 lines' composite butterflies (P = 288:
    radices 2 8 9 2; 480: 2 8 15 2; 512: 2 16 16) or with a four-step build
    (486 = 18 x 27): the FP32 level-0 solve at sampled targets (interior nodes
    and the exterior ring) against the oracle's brute-force sum
    h0^2 sum_s G(t - s) f(s) over the whole lattice, at 1e-5."""
    from paper_2512_08555_gb300.mrp import Solver
    from oracle.lgf import direct_sum
    desc = small_forest(nb=nb, n=n, max_level=0)
    m = Solver(desc, order=4, tol=0.0, max_cycles=1, precision="mixed")
    assert m.fft_shape()[0] == P
    N0 = nb * n
    rng = np.random.default_rng(12)
    F0 = rng.normal(size=(nb ** 3, n, n, n))
    m.field_set("F", 0, F0)
    m.step("coarse_solve_f32")
    U = m.field_get("U", 0).cpu().numpy()
    coords, _ = m.level_info(0)
    f0 = np.zeros((N0, N0, N0))
    where = {}
    for b, c in enumerate(coords):
        x, y, z = (int(v) * n for v in c)
        f0[z:z + n, y:y + n, x:x + n] = F0[b]
        where[(int(c[2]), int(c[1]), int(c[0]))] = b
    G = lgf_table(4, N0 + 1)
    t = rng.integers(0, N0, size=(12, 3))
    t = np.concatenate([t, [[-1, -1, -1], [N0, N0, N0], [-1, N0 // 2, N0], [N0 // 3, -1, 0]]])
    ref = direct_sum(f0, G, float(desc.h0), t)
    got = []
    for z, y, x in t:
        bz, by, bx = (min(max(v, 0), N0 - 1) // n for v in (z, y, x))
        got.append(U[where[(bz, by, bx)], z - bz * n + 1, y - by * n + 1, x - bx * n + 1])
    assert _rel(got, ref) < 1e-5


@pytest.mark.parametrize("M", [2, 4, 6])
@pytest.mark.parametrize("k", [1, 2])
def test_prolong(M, k):
    desc = small_forest()
    s, o = _pair(desc, M)
    rng = np.random.default_rng(4)
    _load(s, o, rng)
    s.step("prolong", k)
    o.prolong_correct(k)
    assert _rel(s.field_get("U", k).cpu().numpy(), o.U[k]) < 1e-14


@pytest.mark.parametrize("M", [2, 4, 6])
@pytest.mark.parametrize("cycles", [1, 3])
def test_fixed_cycle_solve(M, cycles):
    """Same algorithm, same number of V(3,3) cycles from u = 0: <= 1e-12 relative max-norm."""
    from paper_2512_08555_gb300.mrp import Solver
    desc = small_forest()
    f = synth.sample_leaves(desc, synth.c4_bumps(0, k=3, r_lo=0.2, r_hi=0.3))
    s = Solver(desc, order=M, tol=0.0, max_cycles=cycles)
    u, st = s.solve(torch.from_numpy(f).cuda(), allow_not_converged=True)
    o = OracleSolver(OracleForest.from_desc(desc), M)
    uo, rel = o.solve(f, tol=0.0, max_cycles=cycles)
    assert st.cycles == cycles
    assert _rel(u.cpu().numpy(), uo) < 1e-12
    assert abs(st.residual - rel) <= 1e-6 * rel


@pytest.mark.parametrize("M", [2, 4, 6])
def test_converged_solve(M):
    from paper_2512_08555_gb300.mrp import Solver
    desc = small_forest(n=12)
    f = synth.sample_leaves(desc, synth.c4_bumps(2, k=4, r_lo=0.15, r_hi=0.3))
    s = Solver(desc, order=M, tol=1e-12, max_cycles=40)
    u, st = s.solve(torch.from_numpy(f).cuda())
    o = OracleSolver(OracleForest.from_desc(desc), M)
    uo, rel = o.solve(f, tol=1e-12, max_cycles=40)
    assert st.residual < 1e-12 and st.cycles == o.cycles_done
    assert _rel(u.cpu().numpy(), uo) < 1e-12


@pytest.mark.parametrize("M", [2, 4, 6])
def test_single_level_config1(M):
    """Uniform [0,1)^3, 32^3 nodes, 3 Gaussian blobs: one cycle is the LGF solve."""
    from paper_2512_08555_gb300.mrp import Solver
    desc, src = synth.config1(0, n0=32, n=16)
    f = synth.sample_leaves(desc, src)
    s = Solver(desc, order=M, tol=1e-12, max_cycles=3)
    u, st = s.solve(torch.from_numpy(f).cuda())
    o = OracleSolver(OracleForest.from_desc(desc), M)
    uo, rel = o.solve(f, tol=1e-12, max_cycles=3)
    assert st.cycles == 1 and st.residual < 1e-12
    assert _rel(u.cpu().numpy(), uo) < 1e-12


def test_ragged_block_sizes_and_shapes():
    """Non-cubic level 0 and n = 10 (tails of every thread loop)."""
    from paper_2512_08555_gb300.mrp import Solver
    desc = synth.adaptive_forest((5, 4, 3), 10, (0, 0, 0), 0.05, 1, _all)
    f = synth.sample_leaves(desc, synth.gaussian_blobs(3, k=2, c_lo=0.35, c_hi=0.45))
    s = Solver(desc, order=6, tol=0.0, max_cycles=2)
    u, st = s.solve(torch.from_numpy(f).cuda(), allow_not_converged=True)
    o = OracleSolver(OracleForest.from_desc(desc), 6)
    uo, _ = o.solve(f, tol=0.0, max_cycles=2)
    assert _rel(u.cpu().numpy(), uo) < 1e-12


def test_zero_source():
    from paper_2512_08555_gb300.mrp import Solver
    desc = small_forest()
    f = np.zeros((desc.n_leaves, 8, 8, 8))
    s = Solver(desc, order=4, tol=1e-10, max_cycles=2)
    u, st = s.solve(torch.from_numpy(f).cuda(), allow_not_converged=True)
    assert float(u.abs().max()) == 0.0


def test_nan_source_reports_numerical():
    from paper_2512_08555_gb300.mrp import Solver, MrpError
    desc = small_forest(max_level=1)
    f = np.zeros((desc.n_leaves, 8, 8, 8))
    f[-1, 3, 3, 3] = np.nan
    s = Solver(desc, order=4, tol=1e-10, max_cycles=3)
    with pytest.raises(MrpError) as e:
        s.solve(torch.from_numpy(f).cuda())
    assert e.value.status == 7


@pytest.mark.parametrize("M", [4, 6])
def test_config2_full_size(M):
    """Bench workload at full size (2.8M leaf nodes): the first cycle matches the
    oracle element by element; the converged GPU solution has zero composite-system
    residual as evaluated by the oracle's independent composite operator."""
    from paper_2512_08555_gb300.mrp import Solver
    from oracle.composite import CompositeSystem
    desc, src = synth.config2(0)
    f = synth.sample_leaves(desc, src)
    fo = OracleForest.from_desc(desc)
    o = OracleSolver(fo, M)
    uo, _ = o.solve(f, tol=0.0, max_cycles=1)
    s = Solver(desc, order=M, tol=0.0, max_cycles=1)
    u1, _ = s.solve(torch.from_numpy(f).cuda(), allow_not_converged=True)
    assert _rel(u1.cpu().numpy(), uo) < 1e-12
    s2 = Solver(desc, order=M, tol=1e-10, max_cycles=40)
    u, st = s2.solve(torch.from_numpy(f).cuda())
    assert st.residual < 1e-10
    # composite residual of the GPU answer: leaf values of levels >= 1 plus the
    # level-0 source on covered nodes, taken from the library's final state
    cs = CompositeSystem(OracleSolver(fo, M, G=o.G), f)
    n = fo.n
    parts = []
    for k in range(1, fo.max_level + 1):
        Uk = s2.field_get("U", k).cpu().numpy()
        parts.append(Uk[cs.leaf_sel[k], 1:1 + n, 1:1 + n, 1:1 + n].reshape(-1))
    parts.append(s2.field_get("F", 0).cpu().numpy()[cs.cov0].reshape(-1))
    r = cs.residual(np.concatenate(parts))
    assert np.abs(r).max() < 1e-9 * st.fstar_max


@pytest.mark.parametrize("n, M", [(24, 6), (22, 4)])
def test_largest_block_sizes(n, M):
    """Block sizes 22 and 24: the FP64 kernels' largest shared-memory footprint
    (n = 24, M = 6 also takes the tensor form of the raw-f ghost fill), two
    cycles against the oracle; the mixed-precision solve against FP64."""
    from paper_2512_08555_gb300.mrp import Solver
    desc = synth.adaptive_forest((3, 3, 3), n, (-1.0, -1.0, -1.0), 2.0 / (3 * n), 1,
                                 lambda k, c: (c == 1).all(axis=1))
    f = synth.sample_leaves(desc, synth.c4_bumps(2, k=2, r_lo=0.15, r_hi=0.25, box=0.2))
    s = Solver(desc, order=M, tol=0.0, max_cycles=2)
    u, st = s.solve(torch.from_numpy(f).cuda(), allow_not_converged=True)
    o = OracleSolver(OracleForest.from_desc(desc), M)
    uo, _ = o.solve(f, tol=0.0, max_cycles=2)
    assert _rel(u.cpu().numpy(), uo) < 1e-12
    u64, _ = Solver(desc, order=M, tol=1e-11, max_cycles=60).solve(torch.from_numpy(f).cuda(), allow_not_converged=True)
    um, stm = Solver(desc, order=M, tol=1e-10, max_cycles=80, precision="mixed").solve(torch.from_numpy(f).cuda())
    assert stm.residual < 1e-10
    assert _rel(um.cpu().numpy(), u64.cpu().numpy()) < 1e-8

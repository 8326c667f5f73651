"""The no-allocation level-0 solve agrees with the handle-scratch one.

mrp_coarse_solve_noalloc serves callers that cannot allocate device memory
when they need the level-0 solve (stream capture, hosts whose pool owns all
device memory, loops that must not synchronise): its FFT scratch is a fixed
array inside the library.  This file is collected last so that a failure
here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

from paper_2512_08555_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _forest(kind):
    if kind == "uniform32":
        return synth.config1(0, n0=32, n=16)[0]
    return synth.config2(0)[0]       # level 0: 80^3 nodes, P = 162 per axis


@pytest.mark.parametrize("kind", ["uniform32", "adaptive80"])
def test_noalloc_matches_step_twice(kind):
    from paper_2512_08555_gb300.mrp import Solver
    s = Solver(_forest(kind), order=6)
    rng = np.random.default_rng(7)
    f0 = rng.normal(size=s.field_shape("F", 0))
    s.field_set("F", 0, f0)
    s.step("coarse_solve")
    ref = s.field_get("U", 0)
    f_dev = torch.from_numpy(f0).cuda()
    stream = torch.cuda.current_stream()
    for call in range(2):
        u_dev = torch.full(s.field_shape("U", 0), np.nan, dtype=torch.float64, device="cuda")
        rc = s.lib.mrp_coarse_solve_noalloc(s.h, ctypes.c_void_p(f_dev.data_ptr()), ctypes.c_void_p(u_dev.data_ptr()),
                                            ctypes.c_void_p(stream.cuda_stream))
        torch.cuda.synchronize()
        assert rc == 0, (call, rc)
        err = float((u_dev - ref).abs().max() / ref.abs().max())
        assert err < 1e-12, (call, err)
    s.close()


def test_noalloc_rejects_oversize_lattice():
    from paper_2512_08555_gb300.mrp import Solver
    desc = synth.uniform_forest((8, 8, 8), 16, (0, 0, 0), 1 / 128)   # P = 270 per axis: too large for the scratch
    s = Solver(desc, order=2)
    f_dev = torch.zeros(s.field_shape("F", 0), dtype=torch.float64, device="cuda")
    u_dev = torch.zeros(s.field_shape("U", 0), dtype=torch.float64, device="cuda")
    rc = s.lib.mrp_coarse_solve_noalloc(s.h, ctypes.c_void_p(f_dev.data_ptr()), ctypes.c_void_p(u_dev.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 10
    assert s.lib.mrp_error_string(10).startswith(b"problem exceeds")
    s.close()

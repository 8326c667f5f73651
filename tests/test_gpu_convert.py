"""The mixed-precision path's own float/double conversions against IEEE.

The FP64 leaf residual rounds its result to FP32 and the accumulation widens
the FP32 corrections to FP64 with integer operations (GB300's FP64 pipe is
the scarce unit); ``mrp_convert_check`` runs both on device buffers.  numpy's
casts are the IEEE conversions (round to nearest, ties to even; exact
widening), so the results must agree bit for bit, special values included.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _doubles(rng):
    # random magnitudes over the whole float range and beyond
    e = rng.integers(-160, 160, size=200000)
    v = rng.uniform(1.0, 2.0, size=e.size) * np.exp2(e.astype(np.float64)) * rng.choice([-1.0, 1.0], size=e.size)
    # exact ties and near-ties of the 29 dropped fraction bits, both parities of the kept bit
    base = rng.integers(0, 1 << 52, size=4000, dtype=np.uint64) & ~np.uint64((1 << 29) - 1)
    exp = (rng.integers(900, 1140, size=base.size).astype(np.uint64) << np.uint64(52))
    ties = []
    for low in (0x10000000, 0x0FFFFFFF, 0x10000001, 0x1FFFFFFF, 0):
        ties.append((exp | base | np.uint64(low)).view(np.float64))
    f32 = np.finfo(np.float32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, float(f32.max), -float(f32.max),
                        float(f32.max) * (1 + 2.0 ** -25), float(f32.max) * (1 + 2.0 ** -23), 1e39, -1e39,
                        float(f32.tiny), float(f32.tiny) * (1 - 2.0 ** -30), float(f32.tiny) / 3, 1e-46, 1e-50,
                        2.0 ** -149, 2.0 ** -150, 1.5 * 2.0 ** -149, 1.0, -1.0, 1.0 + 2.0 ** -24,
                        1.0 + 3 * 2.0 ** -24, 5e-324, 1.7976931348623157e308])
    return np.concatenate([v] + ties + [special])


def _floats(rng):
    bits = rng.integers(0, 1 << 32, size=200000, dtype=np.uint64).astype(np.uint32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 1.17549435e-38, 1.1754942e-38,
                        3.4028235e38, -3.4028235e38, 1.0, -2.5], dtype=np.float32)
    return np.concatenate([bits.view(np.float32), special])


def _same_bits(a, b):
    """Equal bit patterns, any NaN matching any NaN."""
    na, nb = np.isnan(a), np.isnan(b)
    assert np.array_equal(na, nb)
    ia = a.view(np.int32 if a.dtype == np.float32 else np.int64)
    ib = b.view(np.int32 if b.dtype == np.float32 else np.int64)
    bad = (ia != ib) & ~na
    assert not bad.any(), (a[bad][:5], b[bad][:5])


def test_narrow_and_widen_match_ieee():
    from paper_2512_08555_gb300.mrp import convert_check
    rng = np.random.default_rng(7)
    with np.errstate(over="ignore", invalid="ignore"):
        d = _doubles(rng)
        f = _floats(rng)
        n = max(d.size, f.size)
        d = np.resize(d, n)
        f = np.resize(f, n)
        f_out, d_out = convert_check(torch.from_numpy(d).cuda(), torch.from_numpy(f).cuda())
        _same_bits(f_out.cpu().numpy(), d.astype(np.float32))
        _same_bits(d_out.cpu().numpy(), f.astype(np.float64))


def test_fixed_point_conversions():
    """The leaf residual's fixed-point form trunc(u 2^(shb+1075)) and its int64 -> double rounding.

    For a box whose largest exponent field is E the residual kernel takes
    shb = 9 - G - E (G = 6 for orders 2 and 4, 8 for order 6); numpy's ldexp is
    exact at these scales (results below one truncate to zero either way) and
    its int64 -> float64 cast rounds to nearest, ties to even.
    """
    from paper_2512_08555_gb300.mrp import fixed_check
    rng = np.random.default_rng(11)
    n = 60000
    for G in (6, 8):
        for E in (128, 700, 1023, 1030, 1900):
            shb = 9 - G - E
            top = 2.0 ** (E - 1022)                  # every |u| of the box lies below it
            u = rng.uniform(-1.0, 1.0, n) * top * np.exp2(-rng.integers(0, 90, n).astype(np.float64))
            u = np.concatenate([u, [0.0, -0.0, np.nextafter(top, 0.0), -np.nextafter(top, 0.0), top / 2, -top / 2,
                                    5e-324, -5e-324, 2.2250738585072014e-308]])
            i = np.concatenate([rng.integers(-(1 << 62), 1 << 62, n // 2, dtype=np.int64),
                                rng.integers(-(1 << 40), 1 << 40, n // 4, dtype=np.int64),
                                rng.integers(-1000, 1000, n // 4, dtype=np.int64)])
            # exact ties and near-ties of the bits below a 53-bit significand
            k = rng.integers(1, 9, 64)
            base = (rng.integers(1 << 52, 1 << 53, 64, dtype=np.int64) << k)
            ties = np.concatenate([base + (np.int64(1) << (k - 1)), base + (np.int64(1) << (k - 1)) - 1,
                                   base + (np.int64(1) << (k - 1)) + 1, -(base + (np.int64(1) << (k - 1)))])
            i = np.concatenate([i, ties, np.array([0, 1, -1, (1 << 53) + 1, -(1 << 63), (1 << 63) - 1],
                                                  dtype=np.int64)])
            m = max(u.size, i.size)
            u = np.resize(u, m)
            i = np.resize(i, m)
            fx, d = fixed_check(torch.from_numpy(u).cuda(), shb, torch.from_numpy(i).cuda())
            want = np.trunc(np.ldexp(u, shb + 1075)).astype(np.int64)
            assert np.array_equal(fx.cpu().numpy(), want), (G, E)
            _same_bits(d.cpu().numpy(), i.astype(np.float64))

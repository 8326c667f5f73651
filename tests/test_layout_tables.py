"""The padded shared-memory strides of the fused stencil kernels.

The kernels keep a block's box and its staged right-hand side in a colour
(parity) split whose plane and row strides are chosen so that a warp's loads
of one Gauss-Seidel colour touch as few shared-memory wavefronts as possible
(32 banks of 4 bytes).  The tables are written into the CUDA source; this
test reads them from there and recomputes the rule they claim:

* box, FP32, one node per lane (lanes take x fastest, then z, then y): the
  plane stride Hp in [H^2, H^2 + 32) minimises the wavefronts over a colour;
* staged right-hand side, same lane order, row stride h: Fp likewise;
* block size 16 with node pairs (lanes take i-pairs fastest, then 4 z rows
  of one parity, l = 0, 2, 4, 6 or 1, 3, 5, 7, then 2 y rows): Hp = 84 with
  row stride 9, and Fp = 76 with row stride 9, put a warp's 32 loads in 32
  distinct banks, for either node of a pair and either z parity.
"""
import os
import re

import pytest

pytestmark = pytest.mark.filterwarnings("ignore")

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2512_08555_gb300", "csrc",
                   "kernels_fused.cuh")


def _table(name):
    """Case table of the switch in the host/device function `name`."""
    s = open(SRC).read()
    i = s.index(f"inline int {name}(int n, int el)")
    j = s.index("default:", i)
    return {int(a): int(b) for a, b in re.findall(r"case (\d+): return (\d+);", s[i:j])}


def _wavefronts(h, row, plane):
    """Wavefronts of one colour's loads, one node per lane, lanes x, then z, then y."""
    tot = 0
    for w0 in range(0, h ** 3, 32):
        banks = {}
        for q in range(w0, min(w0 + 32, h ** 3)):
            i, l, j = q % h, (q // h) % h, q // (h * h)
            a = l * plane + j * row + i
            banks.setdefault(a % 32, set()).add(a)
        tot += max(len(v) for v in banks.values())
    return tot


def _best(h, row, lo):
    return min(range(lo, lo + 32), key=lambda p: (_wavefronts(h, row, p), p))


@pytest.mark.parametrize("n", [10, 12, 14, 18, 20, 22, 24])
def test_box_plane_stride(n):
    h, H = n // 2, n // 2 + 1
    hp = _table("split_hp")[n]
    assert H * H <= hp < H * H + 32
    assert _wavefronts(h, H, hp) == _wavefronts(h, H, _best(h, H, H * H))
    assert _wavefronts(h, H, hp) <= _wavefronts(h, H, H * H)


@pytest.mark.parametrize("n", [8, 10, 12, 14, 18, 20, 22, 24])
def test_rhs_plane_stride(n):
    h = n // 2
    fp = _table("split_fp")[n]
    assert h * h <= fp < h * h + 32
    assert _wavefronts(h, h, fp) == _wavefronts(h, h, _best(h, h, h * h))


def _pair(p):
    """The pair lane order of the CUDA source (pair_of): split indices (i, j, l) of pair p."""
    return 2 * (p & 3), ((p >> 4) & 1) + 2 * ((p >> 5) & 3), 2 * ((p >> 2) & 3) + (p >> 7)


def test_pair_lane_order_is_conflict_free():
    hp, fp = _table("split_hp")[16], _table("split_fp")[16]
    assert (hp, fp) == (84, 76)
    src = open(SRC).read()
    assert "q.l = 2 * ((p >> 2) & 3) + (p >> 7);" in src and "q.j = ((p >> 4) & 1) + 2 * ((p >> 5) & 3);" in src
    assert sorted(_pair(p) for p in range(256)) == sorted((i, j, l) for i in range(0, 8, 2) for j in range(8)
                                                          for l in range(8))
    for w0 in range(0, 256, 32):                     # every warp of a 256-pair colour
        for row, plane in ((9, hp), (9, fp)):        # box row stride H = 9; staged f row stride 9
            for second in (0, 1):                    # both nodes of a pair
                banks = set()
                for p in range(w0, w0 + 32):
                    i, j, l = _pair(p)
                    banks.add((i + second + l * plane + j * row) % 32)
                assert len(banks) == 32, (w0, plane, second)
    # pairs p and p + 128 are z-adjacent
    for p in range(128):
        i, j, l = _pair(p)
        assert _pair(p + 128) == (i, j, l + 1)
    # the 8 colour sub-arrays of the staged f hold h Fp words each, padded to 8 (mod 32): a warp's column copy
    # (lanes x = 0..15 of rows y and y + 1, y even) then writes 32 distinct banks
    src = open(SRC).read()
    assert "if (el == 4 && n == 16) return f + ((8 - f % 32) % 32 + 32) % 32;" in src
    f3 = 8 * fp + ((8 - 8 * fp % 32) % 32 + 32) % 32
    for y in (0, 2, 14):
        banks = {((((yy & 1) << 1) | (x & 1)) * f3 + (yy >> 1) * 9 + (x >> 1)) % 32 for yy in (y, y + 1)
                 for x in range(16)}
        assert len(banks) == 32


"""The padded shared-memory strides of the fused stencil kernels.

The kernels keep a block's box and its staged right-hand side in a colour
(parity) split whose plane and row strides are chosen so that a warp's loads
of one Gauss-Seidel colour touch as few shared-memory wavefronts as possible
(32 banks of 4 bytes).  The tables are written into the CUDA source; this
test reads them from there and recomputes the rule they claim:

* box, FP32, one node per lane (lanes take x fastest, then z, then y): the
  plane stride Hp in [H^2, H^2 + 32) minimises the wavefronts over a colour;
* staged right-hand side, same lane order, row stride h: Fp likewise;
* block size 16 with node pairs (lanes take i-pairs fastest, then 4 z rows,
  then 2 y rows): Hp = 88 with row stride 9, and Fp = 72 with row stride 9,
  put a warp's 32 loads in 32 distinct banks.
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


@pytest.mark.parametrize("n", [10, 12, 14, 16, 18, 20, 22, 24])
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


def test_pair_lane_order_is_conflict_free():
    hp, fp = _table("split_hp")[16], _table("split_fp")[16]
    assert (hp, fp) == (88, 72)
    lanes = [(ip, lq, jq) for jq in range(2) for lq in range(4) for ip in range(4)]
    for row, plane in ((9, hp), (9, fp)):            # box row stride H = 9; staged f row stride 9
        for second in (0, 1):                        # both nodes of a pair
            banks = {(2 * ip + second + lq * plane + jq * row) % 32 for ip, lq, jq in lanes}
            assert len(banks) == 32
    # the 8 colour sub-arrays of the staged f hold h Fp words each, padded to 16 (mod 32)
    f3 = 8 * fp
    assert (f3 + ((16 - f3 % 32) % 32 + 32) % 32) % 32 == 16

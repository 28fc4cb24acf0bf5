"""The bench's roofline accounting (window heights and solves per
application of every block) agrees with the oracle's partition of the
two-front sweep (Sec. 2.3), and its flop count with a direct sum over the
oracle's blocks."""
import os
import sys

import pytest

from oracle import sweep2d as S

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


@pytest.mark.parametrize("n,bp,b,dL", [(2047, 12, 12, 12), (511, 12, 12, 12), (127, 12, 12, 1),
                                       (63, 6, 5, 5), (41, 4, 4, 20)])
def test_block_accounting_matches_oracle_partition(n, bp, b, dL):
    lower, upper, mid = S.partition(n, bp, b, dL)
    oracle = sorted([(blk.whi - blk.wlo + 1, 2) for blk in lower + upper] + [(mid.whi - mid.wlo + 1, 1)])
    assert sorted(bench.blocks(n, bp, b, dL)) == oracle
    # 2 w^2 n complex multiply-adds per solve, 8 real flops each, per RHS
    flops = sum(u * 2 * w * w * n * 8 for w, u in oracle)
    assert bench.sweep_flops(n, bp, b, dL, 3) == 3 * flops


def test_headline_stage_count():
    """n = 2047, d = 12: 173 blocks (86 per front and the middle) and 345
    block solves per application (every front block on the way down and on
    the way back, the middle once), run as 86 + 1 + 86 = 173 stages that
    treat both fronts at once."""
    blocks = bench.blocks(2047, 12, 12, 12)
    assert len(blocks) == 173 and sum(u for _, u in blocks) == 2 * 172 + 1


def test_sweep_bytes_count_the_band_factor():
    """Algorithmic bytes of one application (complex64): every block's band
    factor, w^2 + w entries per x1 column (L and D), once per solve, plus four
    passes over the R right-hand sides."""
    n, bp, b, dL, R = 511, 12, 12, 12, 4
    lower, upper, mid = S.partition(n, bp, b, dL)
    fac = 0
    for blk in lower + upper:
        w = blk.whi - blk.wlo + 1
        fac += 2 * n * (w * w + w) * 8
    w = mid.whi - mid.wlo + 1
    fac += n * (w * w + w) * 8
    assert bench.sweep_bytes(n, bp, b, dL, R) == fac + 4 * n * n * R * 8

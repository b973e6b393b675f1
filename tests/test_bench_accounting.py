"""The benchmark's count of re-biorthogonalisation steps (used for the algorithmic
bytes and flops of its roofline) follows the method's schedule as the oracle runs it."""
import pytest

import bench
from oracle import tsl


@pytest.mark.parametrize("k,period", [(800, 60), (800, 20), (200, 1), (37, 10), (600, 0), (10, 100)])
def test_rebiorth_steps_follow_the_oracle_schedule(k, period):
    want = [j for j in range(k - 1) if tsl.rebiorth_at(j + 1, period)]
    assert bench.rebiorth_steps(k, period) == want


def test_projection_flops_scale_with_the_schedule():
    """Halving the projection steps roughly halves the Gram-Schmidt flops; none without them."""
    V = 14 ** 4
    f20 = bench.algorithmic_flops("proj_dots", 800, V, 1, 20, 1)
    f60 = bench.algorithmic_flops("proj_dots", 800, V, 1, 60, 1)
    assert bench.algorithmic_flops("proj_dots", 800, V, 1, 0, 1) == 0
    assert 2.5 < f20 / f60 < 3.5

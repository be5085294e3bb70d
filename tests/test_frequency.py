"""Checkpoint frequency (Appendix A.1), no GPU: the library's f* and W(f*)
against the oracle's statement of the cost, and the oracle pinned by brute
force (f* is the grid minimum of W)."""
import numpy as np
import pytest

from oracle import protocols as P
from paper_2405_12079_b300 import phos


@pytest.mark.parametrize("n,F,O,R,T", [(8, 0.01, 185e-3 / 3600, 0.2, 10.0),
                                        (1, 0.5, 0.01, 0.0, 1.0), (1024, 1e-3, 1e-3, 0.1, 24.0)])
def test_library_matches_oracle(n, F, O, R, T):
    f, w = phos.ckpt_frequency(n, F, O, R, T)
    assert f == pytest.approx(P.optimal_frequency(n, F, O), rel=1e-12)
    assert w == pytest.approx(P.wasted_gpu_hours(n, F, O, R, T, f), rel=1e-12)


def test_oracle_optimum_is_the_brute_force_minimum():
    n, F, O, R, T = 8, 0.02, 0.001, 0.1, 5.0
    grid = np.exp(np.linspace(np.log(0.1), np.log(1e4), 200_001))
    w = P.wasted_gpu_hours(n, F, O, R, T, grid)
    f_grid = grid[np.argmin(w)]
    assert f_grid == pytest.approx(P.optimal_frequency(n, F, O), rel=1e-4)


def test_bad_arguments_are_rejected():
    with pytest.raises(phos.PhosError):
        phos.ckpt_frequency(8, 0.0, 0.001, 0.1, 1.0)

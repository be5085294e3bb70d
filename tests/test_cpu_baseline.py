"""The benchmark's all-core CPU baseline runs the oracle's own validation
and copy on several host threads; its results must be the oracle's (no
GPU)."""
import numpy as np

from oracle import core
from paper_2405_12079_b300 import workloads as wl

VA0 = 0x7F00_0000_0000


def test_validate_omp_equals_validate():
    cfg = wl.training(scale=0.01, n_kernels=1)
    rng, lay = cfg["rng"], cfg["layout"]
    r, w = wl.pick_sets(rng, lay.n)
    perm = np.zeros(lay.n, np.uint8)
    perm[r] = 1
    perm[w] = 3
    for n_rec in (1, 31, 33, 100_003):
        rec, _, _ = wl.trace_runs(rng, lay, VA0, r, w, n_rec, 0.02, 0.3)
        a = core.validate(lay.base(VA0), lay.size, perm, rec, 4)
        bm, cnt, v, vs = core.validate_omp(lay.base(VA0), lay.size, perm, rec, 4)
        assert np.array_equal(a.bitmap, bm) and np.array_equal(a.count, cnt)
        assert np.array_equal(a.victim, v) and np.array_equal(a.victim_st, vs)


def test_memcpy_omp_copies():
    x = np.random.default_rng(1).integers(0, 256, 1_000_003, dtype=np.uint8)
    y = np.zeros_like(x)
    core.memcpy_omp(y, x)
    assert np.array_equal(x, y)

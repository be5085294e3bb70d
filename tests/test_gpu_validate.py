"""GPU parity of phos_validate against the CPU oracle (bit-exact).

Covers several 2048-record tiles with ragged tails, odd record counts (the
bulk-copy tail), tables that take each lookup path (one, two and three
search levels; table in shared memory with 6..2 ring stages; table read
from global memory), coalesced and random traces, access widths 1..16 with
straddles, reserved bits, the index list with caps, and the degenerate
cases (no records, no buffers).  The full-size case validates one
1.3M-record training-kernel trace over a 1,000-buffer table, in the launch
configuration the benchmark uses.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core  # noqa: E402
from paper_2405_12079_b300 import phos, workloads as wl  # noqa: E402
from gpu_util import run_validate  # noqa: E402

VA0 = 0x7E00_0000_0000


@pytest.fixture(autouse=True, params=[1, 2], ids=["ring", "batched"])
def variant(request):
    """Every case runs on both kernel variants."""
    phos.validate_config(request.param)
    yield request.param
    phos.validate_config(0)


def check(table, base, size, perm, trace, w, idx_cap=0):
    got = run_validate(table, perm, trace, w, idx_cap)
    exp = core.validate(base, size, perm, trace, w, idx_cap)
    assert np.array_equal(got["bitmap"], exp.bitmap)
    assert np.array_equal(got["count"], exp.count), (got["count"], exp.count)
    assert np.array_equal(got["victim"], exp.victim)
    assert np.array_equal(got["victim_st"], exp.victim_st)
    if idx_cap:
        k = min(int(exp.count[0]), idx_cap)
        assert np.array_equal(got["idx"][:k], exp.idx)
    assert got["status"] == (phos.PHOS_EINVAL if exp.malformed else 0)
    return got, exp


def layout_table(n, seed, lo=256, hi=1 << 20):
    rng = np.random.default_rng(seed)
    lay = wl.make_layout(rng, wl.sizes_uniform(rng, n, lo, hi))
    base = lay.base(VA0)
    return rng, lay, base, phos.Table(base, lay.size)


@pytest.mark.parametrize("n_rec", [1, 31, 33, 2047, 2049, 4096 * 3 + 7, 1_000_000])
def test_tiny_random_trace(n_rec):
    cfg = wl.tiny(seed=wl.SEED0 + 1)
    lay, rng = cfg["layout"], cfg["rng"]
    base = lay.base(VA0)
    t = phos.Table(base, lay.size)
    perm = np.zeros(lay.n, np.uint8)
    perm[cfg["wset"]] = phos.PERM_RW
    rec, cls = wl.trace_random(rng, lay, VA0, cfg["wset"], n_rec)
    check(t, base, lay.size, perm, rec, 4, idx_cap=1 << 16)


@pytest.mark.parametrize("n,seed", [(1, 1), (32, 2), (33, 3), (1000, 4), (1025, 5),
                                    (3000, 6), (9000, 7), (12000, 8), (20000, 9)])
def test_table_sizes_coalesced_runs(n, seed):
    rng, lay, base, t = layout_table(n, seed, hi=1 << 16)
    reads, writes = wl.pick_sets(rng, n, 1, min(40, n))
    perm = np.zeros(n, np.uint8)
    perm[reads] = phos.PERM_R
    perm[writes] = phos.PERM_RW
    rec, cls, _ = wl.trace_runs(rng, lay, VA0, reads, writes, 50_001, stray_frac=0.01,
                                stray_store_frac=0.3)
    check(t, base, lay.size, perm, rec, 4, idx_cap=300)


def test_largest_table():
    """The largest table the kernels take (32,768 buffers: three search
    levels, the table in global memory), both validation variants (the
    module's fixture)."""
    rng, lay, base, t = layout_table(32768, 11, lo=256, hi=8192)
    reads, writes = wl.pick_sets(rng, 32768, 1, 40)
    perm = np.zeros(32768, np.uint8)
    perm[reads] = phos.PERM_R
    perm[writes] = phos.PERM_RW
    rec, _, _ = wl.trace_runs(rng, lay, VA0, reads, writes, 20_003, stray_frac=0.02,
                              stray_store_frac=0.3)
    check(t, base, lay.size, perm, rec, 4, idx_cap=500)


@pytest.mark.parametrize("w", [1, 2, 8, 16])
def test_widths_and_straddles(w):
    rng, lay, base, t = layout_table(200, 20 + w, lo=256, hi=4096)
    perm = rng.choice(np.array([0, 1, 3], np.uint8), size=200)
    # addresses concentrated around buffer edges
    edges = np.concatenate([base, base + lay.size]).astype(np.int64)
    a = rng.choice(edges, size=40_000) + rng.integers(-24, 24, size=40_000)
    rec = a.astype(np.uint64) | np.where(rng.random(40_000) < 0.4, np.uint64(1 << 63),
                                         np.uint64(0))
    check(t, base, lay.size, perm, rec, w, idx_cap=40_000)


def test_malformed_records_and_idx_cap():
    rng, lay, base, t = layout_table(64, 30)
    perm = np.full(64, phos.PERM_RW, np.uint8)
    rec, _ = wl.trace_random(rng, lay, VA0, np.arange(64), 100_000, frac_other=0.0,
                             frac_gap=0.05)
    rec[[5, 70_000]] |= np.uint64(1 << 59)
    got, exp = check(t, base, lay.size, perm, rec, 4, idx_cap=17)
    assert got["status"] == phos.PHOS_EINVAL and int(exp.count[2]) > 17


def test_degenerate_cases():
    rng, lay, base, t = layout_table(10, 40)
    perm = np.full(10, phos.PERM_R, np.uint8)
    # no records: zero counts and victims
    got = run_validate(t, perm, np.zeros(0, np.uint64), 4)
    assert not got["count"].any() and not got["victim"].any()
    # empty table: every access unmapped
    e = phos.Table([], [])
    tr = (VA0 + np.arange(5000, dtype=np.uint64) * 8)
    got = run_validate(e, np.zeros(0, np.uint8), tr, 4, idx_cap=5000)
    assert got["count"].tolist() == [5000, 0, 5000]
    assert np.array_equal(got["idx"][:5000], np.arange(5000, dtype=np.uint64))
    # everything allowed, no gaps touched: nothing violates
    allrw = np.full(10, phos.PERM_RW, np.uint8)
    rec, _ = wl.trace_random(rng, lay, VA0, np.arange(10), 70_000, frac_other=0, frac_gap=0,
                             store_frac=0.5)
    got = run_validate(t, allrw, rec, 4)
    assert not got["bitmap"].any() and not got["count"].any()


def test_repeated_calls_leave_no_residue():
    """Scratch accumulators are self-cleaning: a call after a call with many
    victims reports only its own."""
    rng, lay, base, t = layout_table(100, 50)
    perm0 = np.zeros(100, np.uint8)
    rec, _ = wl.trace_random(rng, lay, VA0, np.arange(100), 30_000, frac_other=0,
                             frac_gap=0, store_frac=0.5)
    check(t, base, lay.size, perm0, rec, 4)
    perm1 = np.full(100, phos.PERM_RW, np.uint8)
    got, _ = check(t, base, lay.size, perm1, rec, 4)
    assert not got["victim"].any()


def test_full_size_training_kernel_trace():
    """One training-process kernel: 1,000 buffers, 1.3M-record coalesced
    trace with 0.1 % strays, validated in the benchmark's launch shape."""
    cfg = wl.training(n_kernels=1)
    lay, rng = cfg["layout"], cfg["rng"]
    base = lay.base(VA0)
    t = phos.Table(base, lay.size)
    reads, writes = wl.pick_sets(rng, lay.n)
    perm = np.zeros(lay.n, np.uint8)
    perm[reads] = phos.PERM_R
    perm[writes] = phos.PERM_RW
    rec, cls, _ = wl.trace_runs(rng, lay, VA0, reads, writes, cfg["n_rec"], 0.001, 0.1)
    got, exp = check(t, base, lay.size, perm, rec, 4, idx_cap=4096)
    assert int(exp.count[0]) == int((cls >= wl.CLS_OTHER).sum())


@pytest.mark.parametrize("n_rec", [5_000_003, 12_000_017])
def test_large_traces_take_the_wide_batches(n_rec):
    """Traces large enough for 16- and 32-word warp batches (the kernel
    narrows batches for small traces so every warp gets work)."""
    rng, lay, base, t = layout_table(64, 70, hi=1 << 20)
    reads, writes = wl.pick_sets(rng, 64, 1, 20)
    perm = np.zeros(64, np.uint8)
    perm[reads] = phos.PERM_R
    perm[writes] = phos.PERM_RW
    rec, _, _ = wl.trace_runs(rng, lay, VA0, reads, writes, n_rec, 0.002, 0.3)
    check(t, base, lay.size, perm, rec, 4, idx_cap=20_000)


def test_ring_wait_that_runs_out_reports_etimedout(variant):
    """A bounded device wait that runs out (the ring variant's tile waits,
    limited to zero probes) stops the kernel with PHOS_ETIMEDOUT in its
    status word after its copies in flight have landed; the device stays
    usable and the next launch is exact again.  No fault, trap or hang."""
    if variant != 1:
        pytest.skip("the bounded tile waits belong to the ring variant")
    cfg = wl.training(n_kernels=1)
    lay, rng = cfg["layout"], cfg["rng"]
    base = lay.base(VA0)
    t = phos.Table(base, lay.size)
    reads, writes = wl.pick_sets(rng, lay.n)
    perm = np.zeros(lay.n, np.uint8)
    perm[reads] = phos.PERM_R
    perm[writes] = phos.PERM_RW
    rec, _, _ = wl.trace_runs(rng, lay, VA0, reads, writes, 1_300_000, 0.001, 0.0)
    phos.validate_wait_limit(0)
    try:
        got = run_validate(t, perm, rec, 4)
    finally:
        phos.validate_wait_limit()
    assert got["status"] == phos.PHOS_ETIMEDOUT
    check(t, base, lay.size, perm, rec, 4)


@pytest.mark.parametrize("ctas", [1, 3, 148])
def test_batch_assignment_around_one_batch_per_warp(ctas):
    """Trace lengths around one warp batch per warp of the grid (32 warps per
    CTA, batches of 256 to 1024 records): the batched kernel takes batches
    grid-stride when there are no more batches than warps and from the
    shared counter otherwise; either way every batch is checked once."""
    rng, lay, base, t = layout_table(64, 80 + ctas, hi=1 << 20)
    reads, writes = wl.pick_sets(rng, 64, 1, 20)
    perm = np.zeros(64, np.uint8)
    perm[reads] = phos.PERM_R
    perm[writes] = phos.PERM_RW
    phos.validate_grid(ctas)
    try:
        tw = 32 * ctas
        for brec in (256, 512, 1024):
            for n_rec in (tw * brec - 33, tw * brec, tw * brec + 1, tw * brec + brec + 5):
                rec, _, _ = wl.trace_runs(rng, lay, VA0, reads, writes, n_rec, 0.002, 0.3)
                check(t, base, lay.size, perm, rec, 4, idx_cap=5_000)
    finally:
        phos.validate_grid(0)


@pytest.mark.parametrize("seed", range(32))
def test_randomized_shapes(seed):
    """Random combinations of what the kernels branch on: table size (one
    to three search levels, table in shared or global memory), trace length
    (partial batches, every batch width, grid-stride or counter
    assignment), coalesced runs mixed with independent records, reserved
    bits, access width, permissions of every kind (W without R included),
    grid size and index-list cap."""
    rng = np.random.default_rng(7000 + seed)
    n = int(rng.choice([1, 7, 33, 300, 1500, 5000]))
    _, lay, base, t = layout_table(n, 7100 + seed, lo=64, hi=int(rng.choice([4096, 1 << 18])))
    perm = rng.integers(0, 4, size=n).astype(np.uint8)
    w = int(rng.choice([1, 2, 4, 8, 16]))
    N = int(rng.choice([0, 1, 255, 257, 4097, 33_333, 150_001]))
    reads, writes = wl.pick_sets(rng, n, 1, min(20, n))
    m = N // 2
    runs, _, _ = wl.trace_runs(rng, lay, VA0, reads, writes, m, stray_frac=0.02,
                               stray_store_frac=0.4) if m else (np.zeros(0, np.uint64), 0, 0)
    ind, _ = wl.trace_random(rng, lay, VA0, reads, N - m, w=w) if N - m else \
        (np.zeros(0, np.uint64), 0)
    rec = np.concatenate([np.asarray(runs, np.uint64), np.asarray(ind, np.uint64)])
    if N and rng.random() < 0.3:               # a few malformed records
        k = rng.choice(N, size=min(3, N), replace=False)
        rec[k] |= np.uint64(1 << 58)
    phos.validate_grid(int(rng.choice([0, 1, 5, 37])))
    try:
        check(t, base, lay.size, perm, rec, w, idx_cap=int(rng.choice([0, 1, 100, 1 << 16])))
    finally:
        phos.validate_grid(0)

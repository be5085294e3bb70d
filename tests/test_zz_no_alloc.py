"""phos_validate_noalloc, the validation entry point for callers that cannot
allocate device memory (for example an interposer running inside an
application's intercepted CUDA call, or code that must not let an
allocation's implicit device synchronisation stall the application's
kernels).  It must give exactly what phos_validate gives, and what the CPU
oracle gives, call after call, while its scratch stays a fixed array inside
the library.

This file is collected last on purpose: if it fails, a run that stops at
the first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core  # noqa: E402
from paper_2405_12079_b300 import phos, workloads as wl  # noqa: E402

VA0 = 0x7E00_0000_0000
IDX_CAP = 5000


class Bufs:
    """Device inputs and outputs of one case, allocated once."""

    def __init__(self, table, perm, trace, idx_cap):
        N, n = len(trace), table.n
        self.N, self.cap = N, idx_cap
        self.perm = torch.from_numpy(perm.copy()).cuda()
        self.tr = torch.from_numpy(trace.view(np.uint8).copy()).cuda()
        self.outs = [torch.empty((4 * ((N + 31) // 32),), dtype=torch.uint8, device="cuda"),
                     torch.empty((24,), dtype=torch.uint8, device="cuda"),
                     torch.empty((4 * ((n + 31) // 32),), dtype=torch.uint8, device="cuda"),
                     torch.empty((4 * ((n + 31) // 32),), dtype=torch.uint8, device="cuda"),
                     torch.empty((8 * idx_cap,), dtype=torch.uint8, device="cuda"),
                     torch.empty((4,), dtype=torch.uint8, device="cuda")]

    def run(self, fn, table):
        for o in self.outs:
            o.fill_(0x5A)
        self.outs[5].zero_()
        torch.cuda.synchronize()
        bm, cnt, v, vs, idx, st = (o.data_ptr() for o in self.outs)
        fn(table, self.perm.data_ptr(), self.tr.data_ptr(), self.N, 4, bm, cnt, v, vs, idx,
           self.cap, st, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        return [o.cpu().numpy() for o in self.outs]


def oracle_outputs(base, size, perm, trace, idx_cap):
    """The oracle's results laid out like Bufs.run's (bytes of each output)."""
    r = core.validate(base, size, perm, trace, 4, idx_cap=idx_cap)
    idx = np.zeros(idx_cap, np.uint64)
    idx[:len(r.idx)] = r.idx
    return [r.bitmap.view(np.uint8), r.count.view(np.uint8), r.victim.view(np.uint8),
            r.victim_st.view(np.uint8), idx, None]


def assert_same(got, ref, n_idx=None):
    """Bitmap, counts, both victim bitmaps and status bit-exact; the index
    list up to the number of violations (the rest is untouched output)."""
    for j in (0, 1, 2, 3):
        assert np.array_equal(got[j], ref[j]), "output %d differs" % j
    nv = min(int(got[1].view(np.uint64)[0]), IDX_CAP)
    gi, ri = got[4].view(np.uint64)[:nv], np.asarray(ref[4]).view(np.uint64)[:nv]
    assert np.array_equal(gi, ri)
    if ref[5] is not None:
        assert np.array_equal(got[5], ref[5])


def workload(seed, n_rec, stray_store_frac):
    cfg = wl.training(n_kernels=1, seed=seed)
    lay, rng = cfg["layout"], cfg["rng"]
    reads, writes = wl.pick_sets(rng, lay.n)
    perm = np.zeros(lay.n, np.uint8)
    perm[reads] = phos.PERM_R
    perm[writes] = phos.PERM_RW
    rec, _, _ = wl.trace_runs(rng, lay, VA0, reads, writes, n_rec, 0.002, stray_store_frac)
    return lay, perm, rec


def test_noalloc_matches_validate_and_oracle_on_two_calls_in_a_row():
    specs = [workload(wl.SEED0 + 2, 1_300_000, 0.2), workload(wl.SEED0 + 7, 300_001, 0.5)]
    tables = [phos.Table(lay.base(VA0), lay.size) for lay, _, _ in specs]
    bufs = [Bufs(t, p, r, IDX_CAP) for t, (_, p, r) in zip(tables, specs)]
    refs = [b.run(phos.validate, t) for b, t in zip(bufs, tables)]
    orcs = [oracle_outputs(lay.base(VA0), lay.size, p, r, IDX_CAP) for lay, p, r in specs]
    got = [b.run(phos.validate_noalloc, t) for b, t in zip(bufs, tables)]
    for g, ref, orc in zip(got, refs, orcs):
        assert_same(g, ref)
        assert_same(g, orc)
        assert int(g[1].view(np.uint64)[0]) > 0            # violations were found
    # the first case again: the shared array keeps no residue of the last call
    again = bufs[0].run(phos.validate_noalloc, tables[0])
    assert_same(again, refs[0])
    assert_same(again, orcs[0])


def test_noalloc_allocates_nothing_on_a_fresh_table():
    """A table that no other call has used: its growable scratch stays
    empty and the device's free memory does not move over two calls."""
    lay, perm, rec = workload(wl.SEED0 + 9, 500_000, 0.3)
    # load the kernels once (module loading may reserve device memory)
    warm = phos.Table(lay.base(VA0), lay.size)
    Bufs(warm, perm, rec, IDX_CAP).run(phos.validate_noalloc, warm)
    t = phos.Table(lay.base(VA0), lay.size)
    b = Bufs(t, perm, rec, IDX_CAP)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    g1 = b.run(phos.validate_noalloc, t)
    g2 = b.run(phos.validate_noalloc, t)
    assert torch.cuda.mem_get_info()[0] == free0
    assert phos.harness_table_scratch(t) == 0
    orc = oracle_outputs(lay.base(VA0), lay.size, perm, rec, IDX_CAP)
    assert_same(g1, orc)
    assert_same(g2, orc)


def test_noalloc_at_its_largest_table():
    """16,384 buffers, the documented limit: the victim accumulators fill
    the fixed array exactly and the table is read from global memory.
    Victims sit at the top buffer indices."""
    n = 16384
    rng = np.random.default_rng(16384)
    lay = wl.make_layout(rng, wl.sizes_uniform(rng, n, 256, 2048), gap_lo=0, gap_hi=512)
    base = lay.base(VA0)
    perm = np.full(n, phos.PERM_RW, np.uint8)
    perm[n - 96:] = rng.choice(np.array([0, 1], np.uint8), size=96)
    N = 60_001
    top = rng.random(N) < 0.5
    bi = np.where(top, rng.integers(n - 128, n, N), rng.integers(0, n, N)).astype(np.int64)
    off = (rng.random(N) * (lay.size[bi].astype(np.float64) - 4)).astype(np.uint64) & ~np.uint64(3)
    rec = base[bi] + off
    st = rng.random(N) < 0.5
    rec[st] |= wl.STORE_BIT
    gap = rng.random(N) < 0.01                      # one past the end: unmapped or next buffer
    rec[gap] = (base[bi[gap]] + lay.size[bi[gap]]) | (rec[gap] & wl.STORE_BIT)
    t = phos.Table(base, lay.size)
    b = Bufs(t, perm, rec, IDX_CAP)
    ref = b.run(phos.validate, t)
    orc = oracle_outputs(base, lay.size, perm, rec, IDX_CAP)
    g1 = b.run(phos.validate_noalloc, t)
    g2 = b.run(phos.validate_noalloc, t)
    for g in (g1, g2):
        assert_same(g, ref)
        assert_same(g, orc)
    vb = np.unpackbits(g1[2], bitorder="little")[:n]
    assert vb[n - 96:].any() and not vb[:n - 96].any()
    assert vb[n - 32:].any()                        # the last accumulator word is used


def test_noalloc_rejects_another_device_current():
    """The call never switches devices: a table recorded for a device that
    is not current is refused before anything is launched."""
    lay, perm, rec = workload(wl.SEED0 + 11, 4096, 0.0)
    t = phos.Table(lay.base(VA0), lay.size)
    b = Bufs(t, perm, rec, 16)
    cur = torch.cuda.current_device()
    old = phos.harness_table_rebind(t, cur + 1)
    try:
        with pytest.raises(phos.PhosError) as e:
            b.run(phos.validate_noalloc, t)
        assert e.value.code == phos.PHOS_EINVAL and "current" in str(e.value)
    finally:
        phos.harness_table_rebind(t, old)
    # the table works again once its device is recorded back
    assert_same(b.run(phos.validate_noalloc, t), b.run(phos.validate, t))


def test_noalloc_rejects_tables_beyond_its_limit():
    rng = np.random.default_rng(3)
    lay = wl.make_layout(rng, wl.sizes_uniform(rng, 16385, 256, 1024), gap_lo=0, gap_hi=0)
    t = phos.Table(lay.base(VA0), lay.size)
    d = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(phos.PhosError) as e:
        phos.validate_noalloc(t, d.data_ptr(), d.data_ptr(), 16, 4, d.data_ptr(),
                              d.data_ptr(), None, None, None, 0, None, None)
    assert e.value.code == phos.PHOS_EINVAL and "16384" in str(e.value)

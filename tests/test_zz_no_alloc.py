"""phos_validate_noalloc, the validation entry point for callers that cannot
allocate device memory (for example an interposer running inside an
application's intercepted CUDA call, or code that must not let an
allocation's implicit device synchronisation stall the application's
kernels).  It must give exactly what phos_validate gives, call after call,
while its scratch stays a fixed array inside the library.

This file is collected last on purpose: if it fails, a run that stops at
the first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2405_12079_b300 import phos, workloads as wl  # noqa: E402

VA0 = 0x7E00_0000_0000


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
        bm, cnt, v, vs, idx, st = (o.data_ptr() for o in self.outs)
        fn(table, self.perm.data_ptr(), self.tr.data_ptr(), self.N, 4, bm, cnt, v, vs, idx,
           self.cap, st, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        return [o.cpu().numpy() for o in self.outs]


def workload(seed, n_rec, stray_store_frac):
    cfg = wl.training(n_kernels=1, seed=seed)
    lay, rng = cfg["layout"], cfg["rng"]
    reads, writes = wl.pick_sets(rng, lay.n)
    perm = np.zeros(lay.n, np.uint8)
    perm[reads] = phos.PERM_R
    perm[writes] = phos.PERM_RW
    rec, _, _ = wl.trace_runs(rng, lay, VA0, reads, writes, n_rec, 0.002, stray_store_frac)
    return phos.Table(lay.base(VA0), lay.size), perm, rec


def test_noalloc_matches_validate_on_two_calls_in_a_row():
    cases = [workload(wl.SEED0 + 2, 1_300_000, 0.2), workload(wl.SEED0 + 7, 300_001, 0.5)]
    bufs = [Bufs(t, p, r, 5000) for t, p, r in cases]
    refs = [b.run(phos.validate, t) for b, (t, _, _) in zip(bufs, cases)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got = [b.run(phos.validate_noalloc, t) for b, (t, _, _) in zip(bufs, cases)]
    for g, ref in zip(got, refs):
        for x, y in zip(g, ref):
            assert np.array_equal(x, y)
        assert int(g[1].view(np.uint64)[0]) > 0            # violations were found
    # the first case again: the shared array keeps no residue of the last call
    again = bufs[0].run(phos.validate_noalloc, cases[0][0])
    for x, y in zip(again, refs[0]):
        assert np.array_equal(x, y)
    # nothing was allocated on the device by the no-alloc calls
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_tables_beyond_its_limit():
    rng = np.random.default_rng(3)
    lay = wl.make_layout(rng, wl.sizes_uniform(rng, 16385, 256, 1024), gap_lo=0, gap_hi=0)
    t = phos.Table(lay.base(VA0), lay.size)
    d = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(phos.PhosError) as e:
        phos.validate_noalloc(t, d.data_ptr(), d.data_ptr(), 16, 4, d.data_ptr(),
                              d.data_ptr(), None, None, None, 0, None, None)
    assert e.value.code == phos.PHOS_EINVAL and "16384" in str(e.value)

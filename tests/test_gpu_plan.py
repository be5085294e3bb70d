"""GPU parity of the batched plan (one persistent graph launch over many
process images) against the oracle, per item, bit-exact: validation outputs
as phos_validate gives them and every copy as memcpy gives it; replays and
re-tiling (the autotuner's knob) change nothing."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import copyeng, core  # noqa: E402
from paper_2405_12079_b300 import phos, workloads as wl  # noqa: E402


class Item:
    def __init__(self, seed, n, n_rec, pinned):
        rng = np.random.default_rng(seed)
        self.lay = wl.make_layout(rng, wl.sizes_uniform(rng, n, 256, 200_000), gap_lo=256,
                                  gap_hi=4096)
        self.live_h = rng.integers(0, 256, self.lay.arena_bytes, dtype=np.uint8)
        self.live = torch.from_numpy(self.live_h.copy()).cuda()
        va0 = self.live.data_ptr()
        self.base = self.lay.base(va0)
        self.table = phos.Table(self.base, self.lay.size)
        reads, writes = wl.pick_sets(rng, n, 1, min(20, n))
        self.perm = np.zeros(n, np.uint8)
        self.perm[reads] = phos.PERM_R
        self.perm[writes] = phos.PERM_RW
        if n_rec:
            self.trace, _, _ = wl.trace_runs(rng, self.lay, va0, reads, writes, n_rec, 0.01, 0.3)
        else:
            self.trace = np.zeros(0, np.uint64)
        self.stg_h = rng.integers(0, 256, 4 << 20, dtype=np.uint8)
        self.img_h = rng.integers(0, 256, 8 << 20, dtype=np.uint8)
        self.stg = torch.from_numpy(self.stg_h.copy()).cuda()
        img = torch.from_numpy(self.img_h.copy())
        self.img = img.pin_memory() if pinned else img.cuda()
        # descriptors: buffers split into CoW (live -> staging), checkpoint
        # (live -> image), restore targets (image -> live), and a drain of a
        # staging region nothing else writes (staging -> image)
        order = rng.permutation(n)
        rows, so, io = [], 0, 0
        for k, b in enumerate(order):
            sz = int(self.lay.size[b])
            kind = (1, 2, 4)[k % 3]
            if kind == 1 and so + sz <= 2 << 20:
                rows.append((0, so, sz, int(b), 1))
                so += sz + 64
            elif kind == 2 and io + sz <= 4 << 20:
                rows.append((0, io, sz, int(b), 2))
                io += sz + 16
            elif kind == 4:
                rows.append(((4 << 20) + 8 * k, 0, sz // 2, int(b), 4))
        rows.append(((3 << 20) + 5, (6 << 20) + 3, 70_000, 0, 3))
        self.desc = np.array(rows, phos.COPY_DTYPE)
        self.d_desc = torch.from_numpy(self.desc.view(np.uint8).copy()).cuda()
        N = len(self.trace)
        self.d_perm = torch.from_numpy(self.perm.copy()).cuda()
        self.d_tr = torch.from_numpy((self.trace if N else np.zeros(2, np.uint64))
                                     .view(np.uint8).copy()).cuda()
        self.bm = torch.zeros(4 * max((N + 31) // 32, 1), dtype=torch.uint8, device="cuda")
        self.cnt = torch.full((24,), 0x77, dtype=torch.uint8, device="cuda")
        nv = 4 * ((n + 31) // 32)
        self.v = torch.full((nv,), 0x77, dtype=torch.uint8, device="cuda")
        self.vs = torch.full((nv,), 0x77, dtype=torch.uint8, device="cuda")

    def plan_item(self):
        return phos.PlanItem(self.table.handle, self.d_perm.data_ptr(), self.d_tr.data_ptr(),
                             len(self.trace), 4, len(self.desc), self.bm.data_ptr(),
                             self.cnt.data_ptr(), self.v.data_ptr(), self.vs.data_ptr(),
                             self.d_desc.data_ptr(), self.stg.data_ptr(), self.stg.numel(),
                             self.img.data_ptr(), self.img.numel())

    def expected(self):
        res = core.validate(self.base, self.lay.size, self.perm, self.trace, 4)
        live, stg, img = self.live_h.copy(), self.stg_h.copy(), self.img_h.copy()
        assert copyeng.apply(self.desc, live, self.lay.off, self.lay.size, stg, img, None) == 0
        return res, live, stg, img

    def check(self, exp):
        res, live, stg, img = exp
        N = len(self.trace)
        assert np.array_equal(self.bm.cpu().numpy().view(np.uint32)[:(N + 31) // 32], res.bitmap)
        assert np.array_equal(self.cnt.cpu().numpy().view(np.uint64), res.count)
        assert np.array_equal(self.v.cpu().numpy().view(np.uint32), res.victim)
        assert np.array_equal(self.vs.cpu().numpy().view(np.uint32), res.victim_st)
        assert np.array_equal(self.live.cpu().numpy(), live)
        assert np.array_equal(self.stg.cpu().numpy(), stg)
        assert np.array_equal(self.img.cpu().numpy(), img)


def test_plan_matches_oracle_and_replays():
    specs = [(1, 1, 5000, True), (2, 40, 0, False), (3, 1000, 300_001, True),
             (4, 2000, 70_000, False), (5, 64, 2048, True), (6, 300, 123_457, True)]
    items = [Item(*s) for s in specs]
    exps = [it.expected() for it in items]
    plan = phos.Plan([it.plan_item() for it in items])
    s = torch.cuda.current_stream().cuda_stream
    for rep in range(2):
        plan.launch(s)
        torch.cuda.synchronize()
        for it, e in zip(items, exps):
            it.check(e)
    info = plan.info()
    assert info["status"] == 0
    assert info["records"] == sum(len(it.trace) for it in items)
    for tile in (4096, 1 << 16, 4 << 20):
        plan.set_tile(tile)
        plan.launch(s)
        torch.cuda.synchronize()
        for it, e in zip(items, exps):
            it.check(e)
    best, ms = plan.autotune(s)
    assert best in (64 << 10, 128 << 10, 256 << 10, 512 << 10, 1 << 20, 2 << 20, 4 << 20)
    plan.launch(s)
    torch.cuda.synchronize()
    for it, e in zip(items, exps):
        it.check(e)
    plan.close()


def test_plan_rejects_bad_descriptor_and_big_table():
    it = Item(9, 50, 1000, False)
    it.desc[0]["len"] = 1 << 40
    it.d_desc = torch.from_numpy(it.desc.view(np.uint8).copy()).cuda()
    with pytest.raises(phos.PhosError) as e:
        phos.Plan([it.plan_item()])
    assert e.value.code == phos.PHOS_EINVAL

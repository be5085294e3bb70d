"""The batched plan at full size, in the launch configuration the benchmark
times (64 process images of 20-2,000 buffers, 40 GB in all, one 1.3M-record
trace per image, CoW lists covering 35 % of each image, autotuned tile).

Every item's whole bitmap and counts equal the generator's ground-truth
labels (a stray outside the speculated set is the only violation; a gap
stray is the only unmapped access) and equal phos_validate on the same
item; every violating record goes through the oracle, whose victims over
them are exactly the reported victim bitmaps (victims come from violating
records only); 4,096 sampled records agree with the oracle one by one; and
every copied buffer's staging bytes have the digest of its live bytes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import gpu_util as gu  # noqa: E402
from oracle import core  # noqa: E402
from paper_2405_12079_b300 import phos, workloads as wl  # noqa: E402


def a256(x):
    return (int(x) + 255) // 256 * 256


def test_full_size_batched_plan():
    s = torch.cuda.current_stream().cuda_stream
    cfg = wl.batched(scale=1.0)
    rng = cfg["rng"]
    imgs = []
    for j, lay in enumerate(cfg["images"]):
        arena = torch.empty(lay.arena_bytes, dtype=torch.uint8, device="cuda")
        phos.harness_fill(arena.data_ptr(), lay.arena_bytes, 1000 + j, s)
        va0 = arena.data_ptr()
        table = phos.Table(lay.base(va0), lay.size)
        reads, writes = wl.pick_sets(rng, lay.n)
        perm = np.zeros(lay.n, np.uint8)
        perm[reads] = phos.PERM_R
        perm[writes] = phos.PERM_RW
        tr, cls, _ = wl.trace_runs(rng, lay, va0, reads, writes, 1_300_000, 0.001, 0.0)
        total = int(lay.size.sum())
        rows, off, acc = [], 0, 0
        for b in rng.permutation(lay.n):
            if acc >= 0.35 * total:
                break
            sz = int(lay.size[b])
            rows.append((0, off, sz, int(b), phos.COPY_LIVE_TO_STAGING))
            off += a256(sz)
            acc += sz
        desc = np.array(rows, phos.COPY_DTYPE)
        staging = torch.zeros(max(off, 256), dtype=torch.uint8, device="cuda")
        nvw = (lay.n + 31) // 32
        d = dict(lay=lay, arena=arena, va0=va0, table=table, perm=perm, tr=tr, cls=cls, desc=desc,
                 staging=staging,
                 d_desc=torch.from_numpy(desc.view(np.uint8).copy()).cuda(),
                 d_perm=torch.from_numpy(perm).cuda(),
                 d_tr=torch.from_numpy(tr.view(np.uint8).copy()).cuda(),
                 bm=torch.zeros(4 * ((len(tr) + 31) // 32), dtype=torch.uint8, device="cuda"),
                 out=torch.zeros(24 + 8 * nvw, dtype=torch.uint8, device="cuda"), nvw=nvw)
        d["item"] = phos.PlanItem(table.handle, d["d_perm"].data_ptr(), d["d_tr"].data_ptr(),
                                  len(tr), 4, len(desc), d["bm"].data_ptr(), d["out"].data_ptr(),
                                  d["out"].data_ptr() + 24, d["out"].data_ptr() + 24 + 4 * nvw,
                                  d["d_desc"].data_ptr(), staging.data_ptr(), staging.numel(),
                                  None, 0)
        imgs.append(d)
    torch.cuda.synchronize()
    plan = phos.Plan([d["item"] for d in imgs])
    plan.autotune(s)
    plan.launch(s)
    torch.cuda.synchronize()
    assert plan.info()["status"] == 0
    plan.close()
    for d in imgs:
        lay, tr, nvw, cls = d["lay"], d["tr"], d["nvw"], d["cls"]
        N = len(tr)
        bm = d["bm"].cpu().numpy().view(np.uint32)
        out = d["out"].cpu().numpy()
        count = out[:24].view(np.uint64)
        victim = out[24:24 + 4 * nvw].view(np.uint32)
        victim_st = out[24 + 4 * nvw:24 + 8 * nvw].view(np.uint32)
        bits = np.unpackbits(bm.view(np.uint8), bitorder="little")[:N].astype(bool)
        # ground truth of the generator, record by record
        viol = cls >= wl.CLS_OTHER
        st = (tr >> np.uint64(63)).astype(bool)
        assert np.array_equal(bits, viol)
        assert int(count[0]) == int(viol.sum())
        assert int(count[1]) == int((viol & st).sum())
        assert int(count[2]) == int((cls == wl.CLS_GAP).sum())
        # the plain entry point on the same item
        ref = gu.run_validate(d["table"], d["perm"], tr, 4)
        assert np.array_equal(bm[:(N + 31) // 32], ref["bitmap"])
        assert np.array_equal(count, ref["count"])
        assert np.array_equal(victim, ref["victim"]) and np.array_equal(victim_st, ref["victim_st"])
        # every violating record through the oracle: exact victims
        vi = np.nonzero(viol)[0]
        res = core.validate(lay.base(d["va0"]), lay.size, d["perm"], tr[vi], 4)
        assert int(res.count[0]) == len(vi)
        assert np.array_equal(res.victim, victim) and np.array_equal(res.victim_st, victim_st)
        # sampled records one by one
        pick = np.sort(rng.choice(N, 4096, replace=False))
        res = core.validate(lay.base(d["va0"]), lay.size, d["perm"], tr[pick], 4)
        exp_bits = np.unpackbits(res.bitmap.view(np.uint8), bitorder="little")[:len(pick)]
        assert np.array_equal(bits[pick].astype(np.uint8), exp_bits)
        # every copied buffer: staging digest == live digest
        desc = d["desc"]
        ptr_l = [d["va0"] + int(lay.off[int(r["buf"])]) + int(r["src_off"]) for r in desc]
        ptr_s = [d["staging"].data_ptr() + int(r["dst_off"]) for r in desc]
        lens = [int(r["len"]) for r in desc]
        dig = torch.zeros(16 * len(desc), dtype=torch.uint8, device="cuda")
        phos.harness_digest(ptr_l + ptr_s, lens + lens, dig.data_ptr(), s)
        torch.cuda.synchronize()
        dg = dig.cpu().numpy().view(np.uint64)
        assert np.array_equal(dg[:len(desc)], dg[len(desc):])
        # and a few slices byte for byte
        for row in desc[rng.permutation(len(desc))[:4]]:
            b, ln, do = int(row["buf"]), int(row["len"]), int(row["dst_off"])
            lo = int(lay.off[b])
            for o in sorted({0, ln // 2, max(ln - 4096, 0)}):
                k = min(4096, ln - o)
                live = d["arena"][lo + o:lo + o + k].cpu().numpy()
                stg = d["staging"][do + o:do + o + k].cpu().numpy()
                assert np.array_equal(live, stg)

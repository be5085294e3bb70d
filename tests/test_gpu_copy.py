"""GPU parity of the copy engine (phos_cow_copy, phos_recopy,
phos_restore_on_demand, phos_copy) against the oracle's memcpy engine,
byte for byte: every direction, offsets 0..15 x lengths 0..300 on both
ends, multi-tile regions with ragged tails, pinned-host and device images,
invalid descriptors, present bits, and tile / grid shapes (the result must
not depend on them).  Descriptors of one batch never read what another
writes, so the sequential oracle and the parallel engine must agree."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import copyeng  # noqa: E402
from paper_2405_12079_b300 import phos, workloads as wl  # noqa: E402
from gpu_util import dev, host, stream  # noqa: E402


class World:
    def __init__(self, seed, n=40, lo=1, hi=300_000, staging=1 << 21, image=1 << 22,
                 pinned=True):
        rng = np.random.default_rng(seed)
        self.rng = rng
        self.lay = wl.make_layout(rng, wl.sizes_uniform(rng, n, lo, hi), gap_lo=0, gap_hi=512)
        self.live_h = rng.integers(0, 256, self.lay.arena_bytes, dtype=np.uint8)
        self.live = dev(self.live_h)
        self.va0 = self.live.data_ptr()
        self.table = phos.Table(self.lay.base(self.va0), self.lay.size)
        self.stg_h = rng.integers(0, 256, staging, dtype=np.uint8)
        self.stg = dev(self.stg_h)
        self.img_h = rng.integers(0, 256, image, dtype=np.uint8)
        self.img = torch.from_numpy(self.img_h.copy())
        self.img = self.img.pin_memory() if pinned else self.img.cuda()
        self.present = torch.zeros(4 * ((n + 31) // 32), dtype=torch.uint8, device="cuda")
        self.status = torch.zeros(4, dtype=torch.uint8, device="cuda")

    def run(self, desc, fn="copy"):
        d = dev(desc) if len(desc) else torch.zeros(32, dtype=torch.uint8, device="cuda")
        T, n = self.table, len(desc)
        self.present.zero_()
        self.status.zero_()
        st = self.status.data_ptr()
        if fn == "copy":
            phos.copy(T, d.data_ptr(), n, self.stg.data_ptr(), self.stg.numel(),
                      self.img.data_ptr(), self.img.numel(), self.present.data_ptr(), st, stream())
        elif fn == "cow":
            phos.cow_copy(T, d.data_ptr(), n, self.stg.data_ptr(), self.stg.numel(), st, stream())
        elif fn == "recopy":
            phos.recopy(T, d.data_ptr(), n, self.img.data_ptr(), self.img.numel(), st, stream())
        else:
            phos.restore_on_demand(T, d.data_ptr(), n, self.img.data_ptr(), self.img.numel(),
                                   self.present.data_ptr(), st, stream())
        torch.cuda.synchronize()
        pres = np.zeros(self.present.numel() // 4, np.uint32)
        if fn == "cow":
            ok = (desc["flags"] & 0xFF) == 1
        elif fn == "recopy":
            ok = (desc["flags"] & 0xFF) == 2
        elif fn == "restore":
            ok = (desc["flags"] & 0xFF) == 4
        else:
            ok = np.ones(len(desc), bool)
        eff = desc.copy()
        eff["flags"][~ok] = 0xFF                      # rejected by this entry point
        err = copyeng.apply(eff, self.live_h, self.lay.off, self.lay.size, self.stg_h,
                            self.img_h, pres if fn in ("copy", "restore") else None)
        assert np.array_equal(self.live.cpu().numpy(), self.live_h)
        assert np.array_equal(self.stg.cpu().numpy(), self.stg_h)
        assert np.array_equal(self.img.cpu().numpy(), self.img_h)
        assert np.array_equal(host(self.present, np.uint32), pres)
        got_err = int(host(self.status, np.uint32)[0])
        assert got_err == (phos.PHOS_EINVAL if err else 0), (got_err, err)


class Spans:
    """Byte intervals already written / read, per area."""

    def __init__(self):
        self.w, self.r = [], []

    @staticmethod
    def _hit(lst, area, a, b):
        return any(x == area and a < e and s < b for x, s, e in lst)

    def accept(self, src, dst):
        (sa, s0, s1), (da, d0, d1) = src, dst
        if self._hit(self.w, da, d0, d1) or self._hit(self.r, da, d0, d1):
            return False
        if self._hit(self.w, sa, s0, s1):
            return False
        self.w.append((da, d0, max(d1, d0 + 1)))
        self.r.append((sa, s0, max(s1, s0 + 1)))
        return True


def rand_desc(w, m, kinds=(1, 2, 3, 4), maxlen=200_000, present_frac=0.3):
    rng, lay = w.rng, w.lay
    d = np.zeros(m, phos.COPY_DTYPE)
    sp = Spans()
    j = 0
    while j < m:
        k = int(rng.choice(kinds))
        b = int(rng.integers(0, lay.n))
        sz, lo = int(lay.size[b]), int(lay.off[b])
        ln = int(rng.integers(0, min(maxlen, sz) + 1))
        if k in (1, 2):
            so = int(rng.integers(0, sz - ln + 1))
            area = w.stg_h.size if k == 1 else w.img_h.size
            do = int(rng.integers(0, area - ln + 1))
            src, dst = ("live", lo + so, lo + so + ln), ("stg" if k == 1 else "img", do, do + ln)
        elif k == 3:
            so = int(rng.integers(0, w.stg_h.size - ln + 1))
            do = int(rng.integers(0, w.img_h.size - ln + 1))
            src, dst = ("stg", so, so + ln), ("img", do, do + ln)
        else:
            so = int(rng.integers(0, w.img_h.size - ln + 1))
            do = int(rng.integers(0, sz - ln + 1))
            src, dst = ("img", so, so + ln), ("live", lo + do, lo + do + ln)
        if not sp.accept(src, dst):
            continue
        fl = k | (phos.COPY_MARK_PRESENT if k == 4 and rng.random() < present_frac else 0)
        d[j] = (so, do, ln, b, fl)
        j += 1
    return d


def test_each_entry_point_and_mixed_batch():
    w = World(1)
    for fn, kinds in (("cow", (1,)), ("recopy", (2,)), ("restore", (4,)),
                      ("copy", (1, 2, 3, 4))):
        w.run(rand_desc(w, 30, kinds), fn)


def test_wrong_direction_for_entry_point_is_rejected():
    w = World(2)
    d = rand_desc(w, 10, (1,))
    d[3]["flags"] = phos.COPY_LIVE_TO_IMAGE
    w.run(d, "cow")


LENS = (0, 1, 2, 3, 7, 8, 15, 16, 17, 31, 32, 33, 63, 64, 65, 127, 255, 300)


@pytest.mark.parametrize("kind", [1, 2, 4])
def test_offsets_by_lengths_sweep(kind):
    w = World(3, n=24, lo=70_000, hi=80_000, staging=1536 * 1024, image=1536 * 1024)
    rows, i = [], 0
    for so in range(16):
        for do in range(16):
            for ln in LENS:
                if kind in (1, 2):
                    rows.append((so + 64 * (i % 50), i * 320 + do, ln, i % w.lay.n, kind))
                else:
                    rows.append((so + 512 * (i % 2000), (i % 218) * 320 + do, ln, i // 218,
                                 kind))
                i += 1
    w.run(np.array(rows, phos.COPY_DTYPE), "copy")


@pytest.mark.parametrize("kind", [1, 4])
def test_misaligned_multi_tile(kind):
    """Every source/destination alignment pair (16 x 16) on regions of
    ~70 KB: the funnel-shift path over whole 64 KiB tiles, several warp
    chunks and a ragged tail, device -> device and pinned host -> device."""
    w = World(5, n=40, lo=600_000, hi=700_000, staging=20 << 20, image=20 << 20)
    rng = np.random.default_rng(55)
    rows, i = [], 0
    for so in range(16):
        for do in range(16):
            ln = 70_000 + int(rng.integers(0, 600))
            b = i % w.lay.n
            slot = i // w.lay.n
            if kind == 1:
                rows.append((slot * 80_000 + so, i * 80_000 + do, ln, b, kind))
            else:
                rows.append((i * 80_000 + so, slot * 80_000 + do, ln, b, kind))
            i += 1
    w.run(np.array(rows, phos.COPY_DTYPE), "copy")


@pytest.mark.parametrize("tile,ctas", [(4096, 1), (1 << 16, 3), (1 << 20, 8), (16 << 20, 2)])
def test_tile_and_grid_shapes(tile, ctas):
    w = World(4, n=12, lo=1 << 20, hi=6 << 20, staging=1 << 20, image=80 << 20)
    try:
        phos.copy_config(tile, ctas)
        d = np.zeros(12, phos.COPY_DTYPE)
        off = 0
        for b in range(12):
            ln = int(w.lay.size[b]) - (b % 5)
            d[b] = (b % 5, off + (b % 3), ln, b, phos.COPY_LIVE_TO_IMAGE)
            off += ln + 4096
        w.run(d, "recopy")
    finally:
        phos.copy_config(1 << 16, 3)


def test_device_image_and_invalid_descriptors():
    w = World(5, pinned=False)
    d = rand_desc(w, 20, (2, 4))
    b = int(d[4]["buf"])
    d[4] = (0, 0, int(w.lay.size[b]) + 1, b, phos.COPY_LIVE_TO_IMAGE)   # out of bounds
    d[9]["buf"] = 10_000                                                # no such buffer
    d[13]["flags"] = 0x1000 | phos.COPY_IMAGE_TO_LIVE                   # unknown flag
    w.run(d, "copy")


def test_present_bits_and_zero_length():
    w = World(6, n=70)
    d = np.zeros(3, phos.COPY_DTYPE)
    d[0] = (0, 0, 0, 65, phos.COPY_IMAGE_TO_LIVE | phos.COPY_MARK_PRESENT)
    d[1] = (100, 0, int(w.lay.size[3]), 3, phos.COPY_IMAGE_TO_LIVE | phos.COPY_MARK_PRESENT)
    d[2] = (0, 0, 10, 33, phos.COPY_IMAGE_TO_LIVE)
    w.run(d, "restore")
    bits = host(w.present, np.uint32)
    assert bits[0] == (1 << 3) and bits[2] == (1 << 1) and bits[1] == 0

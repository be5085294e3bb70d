"""GPU harness kernels (digest, mutator, fill) against the oracle's
independent C implementation, byte for byte."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core, protocols as P  # noqa: E402
from paper_2405_12079_b300 import phos, workloads as wl  # noqa: E402
from gpu_util import dev, host, stream  # noqa: E402


def test_digest_matches_oracle():
    rng = np.random.default_rng(1)
    data = rng.integers(0, 256, 3_000_000, dtype=np.uint8)
    d = dev(data)
    base = d.data_ptr()
    offs = [0, 16, 8, 3, 1000, 0, 777]
    lens = [0, 1, 7, 9, 2_500_001, 3_000_000, 262_145]
    out = torch.zeros(8 * len(offs), dtype=torch.uint8, device="cuda")
    phos.harness_digest([base + o for o in offs], lens, out.data_ptr(), stream())
    torch.cuda.synchronize()
    got = host(out, np.uint64)
    for j, (o, ln) in enumerate(zip(offs, lens)):
        assert int(got[j]) == core.digest(data[o:o + ln])
    # pinned host memory is digested through its mapped address
    pin = torch.from_numpy(data[:100_003].copy()).pin_memory()
    phos.harness_digest([pin.data_ptr()], [100_003], out.data_ptr(), stream())
    torch.cuda.synchronize()
    assert int(host(out, np.uint64)[0]) == core.digest(data[:100_003])


def test_mutator_matches_oracle():
    rng = np.random.default_rng(2)
    lay = wl.make_layout(rng, wl.sizes_uniform(rng, 30, 1, 600_000))
    arena = rng.integers(0, 256, lay.arena_bytes, dtype=np.uint8)
    d = dev(arena)
    va0 = d.data_ptr()
    t = phos.Table(lay.base(va0), lay.size)
    proc = P.Process(va0, lay.off, lay.size, arena.copy(), seed=99)
    for k in range(6):
        reads, writes = wl.pick_sets(rng, lay.n, 1, 8)
        strays = []
        others = np.setdiff1d(np.arange(lay.n), reads)
        for q in range(3):
            b = int(rng.choice(others))
            if lay.size[b] >= 4:
                a = int(lay.base(va0)[b]) + 4 * int(rng.integers(0, int(lay.size[b]) // 4))
                strays.append((int(rng.integers(0, 1 << 20)), a))
        kern = wl.Kernel([], [], reads, writes, np.zeros(0, np.uint64), np.zeros(0, np.uint8),
                         4, strays)
        proc.run_kernel(k, kern)
        sv = np.array(strays, np.uint64).reshape(-1) if strays else np.zeros(2, np.uint64)
        ds = dev(sv)
        phos.harness_mutate(t, 99, k, reads, writes, ds.data_ptr(), len(strays), stream())
        torch.cuda.synchronize()
        assert np.array_equal(d.cpu().numpy(), proc.mem), k


def test_fill_words():
    n = (1 << 20) + 13
    d = torch.zeros(n + 16, dtype=torch.uint8, device="cuda")
    phos.harness_fill(d.data_ptr() + 3, n, 0x1234, stream())
    torch.cuda.synchronize()
    got = d.cpu().numpy()[3:3 + n]
    ref = np.zeros(n, np.uint8)
    # word j of the region = sm(key ^ j): the oracle's mutator fill uses key
    # sm(s ^ sm(w)); build the same bytes from sm directly for a sample
    for j in list(range(0, 40)) + list(range(n // 8 - 5, (n + 7) // 8)):
        v = core.sm(0x1234 ^ j).to_bytes(8, "little")
        m = min(8, n - 8 * j)
        ref[8 * j:8 * j + m] = np.frombuffer(v[:m], np.uint8)
        assert np.array_equal(got[8 * j:8 * j + m], ref[8 * j:8 * j + m]), j

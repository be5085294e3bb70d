"""Device speculation (the batched form of Sec. 4.1 / Sec. 6 argument-based
speculation) gives, for every launch, exactly the oracle's perm row: random
launches over tables of 1 to 10,000 buffers, boundary values (first byte,
one past the end, gaps, zero), duplicates, struct chunks with a trailing
partial chunk, OR-accumulation onto existing rows, and a bad kind."""
import struct

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import core  # noqa: E402
from paper_2405_12079_b300 import phos, workloads as wl  # noqa: E402

VA0 = 1 << 40


def edge_launches(rng, lay):
    base, size = lay.base(VA0), lay.size
    n = lay.n
    out = []
    for _ in range(64):
        i = int(rng.integers(0, n))
        b, e = int(base[i]), int(base[i]) + int(size[i])
        vals = [b, e - 1, e, b - 1, 0, (1 << 64) - 1, e + 7]
        args = [struct.pack("<Q", v & ((1 << 64) - 1)) for v in vals]
        kinds = [int(rng.integers(1, 3)) for _ in vals]
        # the same buffer twice, const then mutable
        args += [struct.pack("<Q", b), struct.pack("<Q", b + 1)]
        kinds += [phos.ARG_CONST_PTR, phos.ARG_MUT_PTR]
        # a struct: two pointers, a scalar field, a trailing partial chunk
        j = int(rng.integers(0, n))
        st = struct.pack("<QQQ", int(base[j]), 12345, int(base[i]) + 3) + b"\x01\x02\x03"
        args.append(st)
        kinds.append(phos.ARG_STRUCT)
        # a short pointer argument (zero-extended) and a scalar that looks
        # like a pointer
        args += [struct.pack("<I", 77), struct.pack("<Q", b)]
        kinds += [phos.ARG_CONST_PTR, phos.ARG_SCALAR]
        out.append((args, kinds))
    return out


def run_device(lay, launches, pre=None):
    t = phos.Table(lay.base(VA0), lay.size)
    words, wk, off = phos.flatten_launch_args(launches)
    L = len(launches)
    d_w = torch.from_numpy(words.view(np.uint8).copy() if len(words) else np.zeros(8, np.uint8)).cuda()
    d_k = torch.from_numpy(wk.copy() if len(wk) else np.zeros(1, np.uint8)).cuda()
    d_o = torch.from_numpy(off.view(np.uint8).copy()).cuda()
    init = np.zeros((L, lay.n), np.uint8) if pre is None else pre.copy()
    d_p = torch.from_numpy(init.reshape(-1).copy()).cuda()
    d_s = torch.zeros(4, dtype=torch.uint8, device="cuda")
    phos.speculate_device(t, d_w.data_ptr(), d_k.data_ptr(), d_o.data_ptr(), L, d_p.data_ptr(),
                          d_s.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return d_p.cpu().numpy().reshape(L, lay.n), int(d_s.cpu().numpy().view(np.uint32)[0])


@pytest.mark.parametrize("n,seed", [(1, 1), (37, 2), (1000, 3), (10000, 4)])
def test_device_speculation_equals_oracle(n, seed):
    rng = np.random.default_rng(seed)
    sizes = wl.sizes_uniform(rng, n, 1, 200_000)
    lay = wl.make_layout(rng, sizes, gap_lo=0, gap_hi=4096)
    launches = []
    for _ in range(300):
        r, w = wl.pick_sets(rng, n, 1, min(8, n))
        launches.append(wl.make_args(rng, lay, VA0, r, w, struct_frac=0.3))
    launches += edge_launches(rng, lay)
    launches.append(([], []))                       # a launch with no arguments
    got, status = run_device(lay, launches)
    assert status == 0
    base, size = lay.base(VA0), lay.size
    for l, (args, kinds) in enumerate(launches):
        exp = core.speculate(base, size, args, kinds)
        assert np.array_equal(got[l], exp), l


def test_device_speculation_accumulates_and_flags_bad_kind():
    rng = np.random.default_rng(9)
    lay = wl.make_layout(rng, wl.sizes_uniform(rng, 50, 256, 4096))
    launches = [wl.make_args(rng, lay, VA0, *wl.pick_sets(rng, 50, 1, 6)) for _ in range(20)]
    pre = rng.integers(0, 4, (20, 50)).astype(np.uint8)
    got, status = run_device(lay, launches, pre)
    assert status == 0
    base, size = lay.base(VA0), lay.size
    for l, (args, kinds) in enumerate(launches):
        assert np.array_equal(got[l], core.speculate(base, size, args, kinds, pre[l].copy()))
    bad = [([struct.pack("<Q", int(base[3]))], [7])]
    got, status = run_device(lay, bad)
    assert status == phos.PHOS_EINVAL and not got.any()

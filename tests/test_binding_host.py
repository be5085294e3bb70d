"""Host-side marshalling of the binding (no GPU): the argument words handed
to device speculation follow the speculation rules of Sec. 4.1 — a pointer
gives its first 8 bytes zero-extended, a struct each full 8-byte chunk (a
trailing partial chunk is dropped), a scalar nothing — and the words of
every launch, resolved against a table by the oracle's own rule, give the
oracle's perm row."""
import struct

import numpy as np

from oracle import core
from paper_2405_12079_b300 import phos, workloads as wl


def test_flatten_rules():
    launches = [
        ([struct.pack("<Q", 0x1234), struct.pack("<I", 7), struct.pack("<Q", 99)],
         [phos.ARG_MUT_PTR, phos.ARG_CONST_PTR, phos.ARG_SCALAR]),
        ([], []),
        ([struct.pack("<QQ", 5, 6) + b"\x01\x02\x03"], [phos.ARG_STRUCT]),
    ]
    words, kinds, off = phos.flatten_launch_args(launches)
    assert words.tolist() == [0x1234, 7, 5, 6]
    assert kinds.tolist() == [phos.ARG_MUT_PTR, phos.ARG_CONST_PTR, phos.ARG_STRUCT,
                              phos.ARG_STRUCT]
    assert off.tolist() == [0, 2, 2, 4]


def test_flattened_words_reproduce_oracle_rows():
    rng = np.random.default_rng(3)
    lay = wl.make_layout(rng, wl.sizes_uniform(rng, 200, 256, 50_000))
    va0 = 1 << 40
    base, size = lay.base(va0), lay.size
    launches = [wl.make_args(rng, lay, va0, *wl.pick_sets(rng, 200, 1, 10), struct_frac=0.5)
                for _ in range(50)]
    words, kinds, off = phos.flatten_launch_args(launches)
    for l, (args, kd) in enumerate(launches):
        # each flattened word as a one-word argument of its own kind
        # (struct words as mutable pointers) must give the same row
        wa = [struct.pack("<Q", int(w)) for w in words[off[l]:off[l + 1]]]
        wk = [phos.ARG_MUT_PTR if int(k) == phos.ARG_STRUCT else int(k)
              for k in kinds[off[l]:off[l + 1]]]
        assert np.array_equal(core.speculate(base, size, wa, wk),
                              core.speculate(base, size, args, kd))


def test_table_rules_rejected_on_host():
    """The table rules (sorted, disjoint, size > 0, 57-bit addresses, at most
    32,768 buffers) are checked before any device work."""
    import pytest
    n = 100
    base = (np.arange(n, dtype=np.uint64) * 4096 + np.uint64(1 << 40))
    size = np.full(n, 256, np.uint64)
    bad = [(base[::-1].copy(), size), (base, np.full(n, 8192, np.uint64)),
           (base, np.zeros(n, np.uint64)), (base + np.uint64(1 << 57), size)]
    big = (np.arange(32769, dtype=np.uint64) * 4096 + np.uint64(1 << 40))
    bad.append((big, np.full(32769, 256, np.uint64)))
    for b, sz in bad:
        with pytest.raises(phos.PhosError) as e:
            phos.Table(b, sz)
        assert e.value.code == phos.PHOS_EINVAL

"""Pins of the CPU oracle against things other than itself (no GPU).

Each test fixes the oracle to something the paper or the mathematics
decides: published generator outputs, brute force over every address of a
small virtual-address window (with a per-byte ownership map, a different
formulation from the oracle's interval compare), the generator's
ground-truth labels, memcpy, and closed-form special cases.
"""
import os
import struct

import numpy as np
import pytest

from oracle import core, copyeng
from paper_2405_12079_b300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")
VA0 = 0x7F00_0000_0000


def test_splitmix64_published_vector():
    vals = [int(l, 16) for l in open(os.path.join(GOLD, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    state = 0
    for v in vals:
        assert core.sm(state) == v
        state = (state + 0x9E3779B97F4A7C15) & (2**64 - 1)


def test_digest_properties():
    rng = np.random.default_rng(1)
    assert core.digest(np.zeros(0, np.uint8)) == 0
    b = rng.integers(0, 256, 37, dtype=np.uint8)
    padded = np.concatenate([b, np.zeros(3, np.uint8)])
    assert core.digest(b) == core.digest(padded)          # tail zero-padded
    # additivity over an 8-byte aligned split: D(A++B) = D(A) + D'(B) where
    # D' shifts word indices; check with a split at 16 bytes and the
    # identity sum over words recomputed from two halves
    a16, rest = b[:16], b[16:]
    d_all = core.digest(b)
    d_a = core.digest(a16)
    d_rest_shift = (d_all - d_a) & (2**64 - 1)
    assert d_rest_shift != core.digest(rest)              # position dependent
    # swapping two different words changes the digest
    w = b[:32].copy().view(np.uint64)
    sw = w[[1, 0, 2, 3]].copy()
    assert core.digest(w.view(np.uint8)) != core.digest(sw.view(np.uint8))
    # one word equals mix64(word + j*golden) summed: single word at j = 0
    one = np.array([5], np.uint64).view(np.uint8)
    assert core.digest(one) == core.mix64(5)


def _published_sm0():
    return [int(l, 16) for l in open(os.path.join(GOLD, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]


def test_digest_word_index_term_published():
    """The word-index term j * GOLDEN of the digest, pinned by published
    SplitMix64 outputs: mix64(x + GOLDEN) is the first output of a
    generator in state x, so word j holding 0 contributes the (j)-th
    output of the state-0 sequence, and a word holding GOLDEN at index 0
    contributes the first output too.  A digest that used j (or no index)
    in place of j * GOLDEN fails here."""
    v = _published_sm0()
    M = 2**64 - 1
    G = 0x9E3779B97F4A7C15
    w = lambda *xs: np.array(xs, np.uint64).view(np.uint8)
    # mix64(0) = 0: a zero word at index 0 adds nothing
    assert core.digest(w(0)) == 0
    assert core.digest(w(G, 0)) == (2 * v[0]) & M
    assert core.digest(w(G, 0, 0)) == (2 * v[0] + v[1]) & M
    assert core.digest(w(0, 0, 0, 0)) == (v[0] + v[1] + v[2]) & M
    # word j holding -j*GOLDEN + GOLDEN contributes the first output at every j
    words = [((1 - j) * G) & M for j in range(5)]
    assert core.digest(w(*words)) == (5 * v[0]) & M
    # a 4-byte tail is zero-padded into the last word
    assert core.digest(w(G, 0)[:12]) == (2 * v[0]) & M


def test_stray_value_published():
    """Stray store value (u32)sm(sm(seed ^ k) ^ r), pinned by published
    outputs: with seed ^ k = 0 the inner value is the first state-0
    output v0, so r = v0 gives sm(0) = v0 and r = v0 ^ GOLDEN gives
    sm(GOLDEN) = v1 (low 32 bits of each)."""
    v = _published_sm0()
    G = 0x9E3779B97F4A7C15
    assert core.stray_value(0, 0, v[0]) == v[0] & 0xFFFFFFFF == 0x7B1DCDAF
    assert core.stray_value(0, 0, v[0] ^ G) == v[1] & 0xFFFFFFFF
    assert core.stray_value(12345, 12345, v[0]) == v[0] & 0xFFFFFFFF   # only seed ^ k enters
    assert core.stray_value(12345, 12344, v[0]) != v[0] & 0xFFFFFFFF


def _owner_map(base, size, lo, hi):
    """owner[x - lo] = buffer index owning byte x, -1 in gaps."""
    own = np.full(hi - lo, -1, np.int64)
    for i, (b, s) in enumerate(zip(base, size)):
        a, e = max(int(b), lo), min(int(b) + int(s), hi)
        if a < e:
            own[a - lo:e - lo] = i
    return own


@pytest.mark.parametrize("seed", range(6))
def test_validate_brute_force_window(seed):
    rng = np.random.default_rng(100 + seed)
    W = 1 << 16
    lo = VA0
    n = int(rng.integers(0, 9))
    cuts = np.sort(rng.choice(W, size=2 * n, replace=False)) if n else np.zeros(0, int)
    base = (lo + cuts[0::2]).astype(np.uint64)
    size = (cuts[1::2] - cuts[0::2]).astype(np.uint64)
    keep = size > 0
    base, size = base[keep], size[keep]
    n = len(base)
    assert core.table_check(base, size) == 0
    perm = rng.choice(np.array([0, 1, 3], np.uint8), size=n)
    own = _owner_map(base, size, lo, lo + W + 32)
    for w in (1, 2, 4, 8, 16):
        addrs = np.arange(lo, lo + W, dtype=np.uint64)
        for store in (0, 1):
            tr = addrs | (np.uint64(1 << 63) if store else np.uint64(0))
            res = core.validate(base, size, perm, tr, w, idx_cap=len(tr))
            off = (addrs - np.uint64(lo)).astype(np.int64)
            first = own[off]
            last = own[off + w - 1]
            # all bytes owned by the same buffer <=> first == last != -1 and
            # no gap in between (buffers are contiguous, so first==last suffices)
            inb = (first >= 0) & (first == last)
            need = 2 if store else 1
            ok = inb & ((perm[np.maximum(first, 0)] & need) != 0)
            viol = ~ok
            bits = np.unpackbits(res.bitmap.view(np.uint8), bitorder="little")[:len(tr)]
            assert np.array_equal(bits.astype(bool), viol)
            assert int(res.count[0]) == int(viol.sum())
            assert int(res.count[1]) == (int(viol.sum()) if store else 0)
            assert int(res.count[2]) == int((~inb).sum())
            vic = np.unique(first[viol & inb])
            vb = np.unpackbits(res.victim.view(np.uint8), bitorder="little")[:n]
            assert set(np.nonzero(vb)[0].tolist()) == set(vic.tolist())
            vs = np.unpackbits(res.victim_st.view(np.uint8), bitorder="little")[:n]
            assert set(np.nonzero(vs)[0].tolist()) == (set(vic.tolist()) if store else set())
            assert np.array_equal(res.idx, np.nonzero(viol)[0].astype(np.uint64))


def test_validate_ground_truth_labels_tiny():
    cfg = wl.tiny(scale=0.25)
    lay, rng = cfg["layout"], cfg["rng"]
    base = lay.base(VA0)
    perm = np.zeros(lay.n, np.uint8)
    perm[cfg["wset"]] = 3
    rec, cls = wl.trace_random(rng, lay, VA0, cfg["wset"], cfg["n_rec"])
    res = core.validate(base, lay.size, perm, rec, 4, idx_cap=1 << 20)
    viol = cls >= wl.CLS_OTHER
    bits = np.unpackbits(res.bitmap.view(np.uint8), bitorder="little")[:len(rec)]
    assert np.array_equal(bits.astype(bool), viol)
    st = (rec >> np.uint64(63)).astype(bool)
    assert int(res.count[0]) == int(viol.sum())
    assert int(res.count[1]) == int((viol & st).sum())
    assert int(res.count[2]) == int((cls >= wl.CLS_GAP).sum())
    assert np.array_equal(res.idx, np.nonzero(viol)[0].astype(np.uint64))
    # counts near the configured shares
    assert abs(int(res.count[0]) / len(rec) - 0.05) < 0.005


def test_validate_special_cases():
    base = np.array([VA0, VA0 + 4096], np.uint64)
    size = np.array([4096, 4096], np.uint64)
    rng = np.random.default_rng(3)
    a = (VA0 + rng.integers(0, 8192 - 4, 5000) // 4 * 4).astype(np.uint64)
    tr = a | np.where(rng.random(5000) < 0.5, np.uint64(1 << 63), np.uint64(0))
    # every buffer RW and no gaps inside the window: nothing violates
    r = core.validate(base, size, np.array([3, 3], np.uint8), tr, 4)
    assert int(r.count[0]) == 0 and not r.bitmap.any()
    # empty table: everything is unmapped
    r = core.validate(np.zeros(0, np.uint64), np.zeros(0, np.uint64), np.zeros(0, np.uint8), tr, 4)
    assert int(r.count[0]) == 5000 and int(r.count[2]) == 5000
    # a straddling access at the boundary between two RW buffers is unmapped
    r = core.validate(base, size, np.array([3, 3], np.uint8),
                      np.array([VA0 + 4094], np.uint64), 4)
    assert int(r.count[2]) == 1
    # reserved bits make a record malformed
    r = core.validate(base, size, np.array([3, 3], np.uint8),
                      np.array([VA0 | (1 << 60)], np.uint64), 4)
    assert r.malformed and int(r.count[2]) == 1
    # read-only buffer: loads pass, stores are victims
    r = core.validate(base, size, np.array([1, 0], np.uint8),
                      np.array([VA0 + 8, VA0 + 8 | (1 << 63), VA0 + 5000], np.uint64), 4)
    assert int(r.count[0]) == 2 and int(r.count[1]) == 1
    assert r.victim[0] == 3 and r.victim_st[0] == 1
    # padding bits of the last bitmap word are zero
    r = core.validate(base, size, np.array([0, 0], np.uint8),
                      np.full(33, VA0 + 16, np.uint64), 4)
    assert r.bitmap[1] == 1 and r.bitmap[0] == 0xFFFFFFFF


def test_table_check_rejects():
    assert core.table_check([10, 5], [1, 1]) != 0          # unsorted
    assert core.table_check([10, 12], [4, 1]) != 0         # overlapping
    assert core.table_check([10], [0]) != 0                # empty buffer
    assert core.table_check([10, 14], [4, 1]) == 0         # touching is fine


def _pk(v):
    return struct.pack("<Q", v)


def test_speculate_rules():
    base = np.array([VA0, VA0 + 1000, VA0 + 5000], np.uint64)
    size = np.array([100, 1000, 8], np.uint64)
    # const -> R, mutable -> RW, scalar ignored even when it looks like a pointer
    p = core.speculate(base, size, [_pk(VA0 + 5), _pk(VA0 + 1999), _pk(VA0 + 5001)], [1, 2, 0])
    assert p.tolist() == [1, 3, 0]
    # one past the end does not match (half-open)
    p = core.speculate(base, size, [_pk(VA0 + 100), _pk(VA0 + 5008)], [2, 2])
    assert p.tolist() == [0, 0, 0]
    # struct: every full 8-byte chunk is a possible written pointer, a
    # trailing partial chunk is ignored
    s = _pk(7) + _pk(VA0 + 5007) + (VA0 + 10).to_bytes(8, "little")[:7]
    p = core.speculate(base, size, [s], [3])
    assert p.tolist() == [0, 0, 3]
    # const then mutable on the same buffer accumulates to RW
    p = core.speculate(base, size, [_pk(VA0), _pk(VA0 + 99)], [1, 2])
    assert p.tolist() == [3, 0, 0]
    # 4-byte pointer argument is zero-extended
    p = core.speculate(np.array([16], np.uint64), np.array([16], np.uint64),
                       [(20).to_bytes(4, "little")], [2])
    assert p.tolist() == [3]
    # type-1 memory move: every overlapped buffer
    perm = np.zeros(3, np.uint8)
    core.speculate_region(base, size, VA0 + 50, 1000, 3, perm)
    assert perm.tolist() == [3, 3, 0]


def test_speculate_brute_force_window():
    rng = np.random.default_rng(7)
    W = 1 << 12
    cuts = np.sort(rng.choice(W, size=10, replace=False))
    base = (VA0 + cuts[0::2]).astype(np.uint64)
    size = (cuts[1::2] - cuts[0::2]).astype(np.uint64)
    own = _owner_map(base, size, VA0, VA0 + W)
    for x in range(0, W, 3):
        p = core.speculate(base, size, [_pk(VA0 + x)], [2])
        exp = np.zeros(5, np.uint8)
        if own[x] >= 0:
            exp[own[x]] = 3
        assert np.array_equal(p, exp)


def test_speculate_matches_generator_ground_truth():
    cfg = wl.training(scale=0.001, n_kernels=30)
    lay, rng = cfg["layout"], cfg["rng"]
    for _ in range(30):
        reads, writes = wl.pick_sets(rng, lay.n)
        args, kinds = wl.make_args(rng, lay, VA0, reads, writes, struct_frac=0.5)
        p = core.speculate(lay.base(VA0), lay.size, args, kinds)
        exp = np.zeros(lay.n, np.uint8)
        exp[reads] = 1
        exp[writes] = 3
        assert np.array_equal(p, exp)


def test_mutator_fill_words():
    buf = np.zeros(21, np.uint8)
    core.mutator_fill(buf, 12345, 7)
    key = core.sm(12345 ^ core.sm(7))
    words = [core.sm(key ^ j) for j in range(3)]
    exp = b"".join(w.to_bytes(8, "little") for w in words)[:21]
    assert bytes(buf) == exp
    # seed depends on every read digest, in order
    s1 = core.mutator_seed(1, 2, [10, 20])
    assert s1 != core.mutator_seed(1, 2, [20, 10]) and s1 != core.mutator_seed(1, 2, [10])
    assert core.mutator_seed(1, 2, []) == core.sm(1 ^ core.sm(2))


def _bytewise_copy(dst, do, src, so, ln):
    for t in range(ln):
        dst[do + t] = src[so + t]


def test_copy_engine_offsets_lengths():
    rng = np.random.default_rng(11)
    live = rng.integers(0, 256, 4096, dtype=np.uint8)
    buf_off = np.array([0, 2048], np.uint64)
    buf_size = np.array([1024, 2048], np.uint64)
    for so in range(16):
        for do in range(16):
            for ln in (0, 1, 7, 15, 16, 17, 31, 33, 64, 255, 300):
                st = np.zeros(512, np.uint8)
                ex = np.zeros(512, np.uint8)
                d = np.zeros(1, copyeng.DESC_DTYPE)
                d[0] = (so, do, ln, 1, copyeng.LIVE_TO_STAGING)
                assert copyeng.apply(d, live, buf_off, buf_size, staging=st) == 0
                _bytewise_copy(ex, do, live, 2048 + so, ln)
                assert np.array_equal(st, ex)


def test_copy_engine_directions_and_errors():
    rng = np.random.default_rng(12)
    live = rng.integers(0, 256, 1 << 14, dtype=np.uint8)
    live0 = live.copy()
    off = np.array([0, 8192], np.uint64)
    sz = np.array([4000, 8192], np.uint64)
    st = np.zeros(4096, np.uint8)
    img = np.zeros(16384, np.uint8)
    pres = np.zeros(1, np.uint32)
    d = np.zeros(5, copyeng.DESC_DTYPE)
    d[0] = (0, 0, 4000, 0, copyeng.LIVE_TO_STAGING)
    d[1] = (0, 4096, 4000, 0, copyeng.STAGING_TO_IMAGE)
    d[2] = (100, 9000, 500, 1, copyeng.LIVE_TO_IMAGE)
    d[3] = (9000, 0, 500, 1, copyeng.IMAGE_TO_LIVE | copyeng.MARK_PRESENT)
    d[4] = (0, 0, 4001, 0, copyeng.LIVE_TO_STAGING)            # out of bounds
    assert copyeng.apply(d, live, off, sz, st, img, pres) == 1
    assert np.array_equal(img[4096:8096], live0[:4000])
    assert np.array_equal(img[9000:9500], live0[8192 + 100:8192 + 600])
    assert np.array_equal(live[8192:8692], live0[8292:8792])
    assert pres[0] == 2
    bad = np.zeros(1, copyeng.DESC_DTYPE)
    bad[0] = (0, 0, 1, 0, 9)
    assert copyeng.apply(bad, live, off, sz, st, img, pres) == 1

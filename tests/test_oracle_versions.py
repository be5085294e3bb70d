"""Pins of the oracle's "versions" storage mode (no GPU).

The versions mode runs the protocols' own code over arrays that describe
bytes instead of holding them.  It is pinned three ways: its word stream
and partial digests by published SplitMix64 outputs; its arrays by a
random model check against numpy arrays (every slice assignment of the
protocols' kinds, bytes compared after each step); and whole protocol runs
in versions mode against the same runs in bytes mode (which the
correctness theorems pin): identical CoW lists, copier pieces, dirty sets,
on-demand lists, fallback rounds, images and final memory.
"""
import os

import numpy as np
import pytest

from oracle import core
from oracle import protocols as P
from oracle import versions as V
from paper_2405_12079_b300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")
G = 0x9E3779B97F4A7C15
M = 2**64 - 1
VA0 = 0x7F00_0000_0000


def _v():
    return [int(l, 16) for l in open(os.path.join(GOLD, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]


def _le(x):
    return np.frombuffer(int(x).to_bytes(8, "little"), np.uint8)


def test_word_stream_published():
    """Word j of the stream is sm(key ^ j): key ^ j = 0, GOLDEN, 2 GOLDEN give
    the first three published outputs, little-endian; an unaligned start
    takes the word's bytes from the right place."""
    v = _v()
    assert np.array_equal(core.words(8, 0), _le(v[0]))
    assert np.array_equal(core.words(8, G), _le(v[1]))
    assert np.array_equal(core.words(8, G ^ 1, 8), _le(v[1]))
    assert np.array_equal(core.words(8, ((2 * G) & M) ^ 5, 40), _le(v[2]))
    assert np.array_equal(core.words(5, 0, 3), _le(v[0])[3:])
    assert np.array_equal(core.words(16, 0)[:8], _le(v[0]))
    assert np.array_equal(core.words(3, G ^ 1, 13), _le(v[1])[5:])


def test_partial_digest_published_and_additive():
    """digest_at(piece, j0) sums mix64(word + (j0 + j) GOLDEN): a zero word
    at j0 = 1 and 2 gives the first and second published outputs; a digest
    is the sum of its aligned pieces' partial digests."""
    v = _v()
    z = np.zeros(8, np.uint8)
    assert core.digest_at(z, 1) == v[0] and core.digest_at(z, 2) == v[1]
    assert core.digest_at(z, 0) == 0
    rng = np.random.default_rng(5)
    b = rng.integers(0, 256, 1003, dtype=np.uint8)
    parts = (core.digest_at(b[:16], 0) + core.digest_at(b[16:512], 2) +
             core.digest_at(b[512:], 64)) & M
    assert parts == core.digest(b)


def test_mutator_fill_is_the_word_stream_of_its_key():
    buf = np.zeros(4099, np.uint8)
    core.mutator_fill(buf, 0x1234_5678_9ABC, 17)
    assert np.array_equal(buf, core.words(4099, core.mutator_key(0x1234_5678_9ABC, 17)))
    assert core.mutator_key(1, 2) != core.mutator_key(1, 3)


def test_varray_model_check():
    """Random slice assignments between VArrays (and from literal bytes),
    through views of views, mirrored on numpy arrays: the bytes agree after
    every step, and segment lists stay short when copies continue."""
    rng = np.random.default_rng(11)
    n = 5000
    arrs = [V.VArray(n, V.Words(7), 0), V.VArray(n), V.VArray(n, V.Words(9), 123)]
    ref = [core.words(n, 7, 0), np.zeros(n, np.uint8), core.words(n, 9, 123)]
    for step in range(600):
        d = int(rng.integers(0, 3))
        a = int(rng.integers(0, n))
        ln = int(rng.integers(0, min(700, n - a) + 1))
        kind = rng.random()
        if kind < 0.5:
            s = int(rng.integers(0, 3))
            b = int(rng.integers(0, n - ln + 1))
            src = arrs[s][b:b + ln]
            exp = ref[s][b:b + ln].copy()
        elif kind < 0.7:
            exp = rng.integers(0, 256, ln, dtype=np.uint8)
            src = exp.copy()
        else:
            key = int(rng.integers(0, 2**63))
            src = V.VArray(ln, V.Words(key), 8 * int(rng.integers(0, 100)))
            exp = src.materialize()
        if rng.random() < 0.5:
            arrs[d][a:a + ln] = src
        else:                                   # through a view of a view
            lo = int(rng.integers(0, a + 1))
            arrs[d][lo:][a - lo:a - lo + ln] = src
        ref[d][a:a + ln] = exp
        if step % 50 == 0 or step == 599:
            for x, y in zip(arrs, ref):
                assert np.array_equal(x.materialize(), y)
    # copying a whole array piece by piece in order gives back one segment
    w = V.VArray(4096, V.Words(3), 0)
    c = V.VArray(4096)
    for o in range(0, 4096, 512):
        c[o:o + 512] = w[o:o + 512]
    assert len(c.segs) == 1
    assert V.digest_pieces(c.pieces(0, 4096)) == core.digest(core.words(4096, 3))


# ------------------------------------------------- versions == bytes mode

KEY = 0xC0FFEE


def world(seed, n=24, lo=1024, hi=40000, sizes=None):
    rng = np.random.default_rng(seed)
    if sizes is None:
        sizes = wl.sizes_uniform(rng, n, lo, hi)
    lay = wl.make_layout(rng, sizes, gap_lo=256, gap_hi=4096)
    return rng, lay


def procs(lay, seed):
    mem = core.words(lay.arena_bytes, KEY, 0)
    b = P.Process(VA0, lay.off, lay.size, mem, seed)
    v = V.VersionProcess(VA0, lay.off, lay.size, KEY, seed, arena_bytes=lay.arena_bytes)
    return b, v


def kernels(rng, lay, K, stray_stores=False):
    ks = []
    for _ in range(K):
        r, w = wl.pick_sets(rng, lay.n, 1, 6)
        reads = np.union1d(r, w)
        args, kinds = wl.make_args(rng, lay, VA0, reads, w)
        rec, cls, st = wl.trace_runs(rng, lay, VA0, reads, w, 512, 0.02 if stray_stores else 0.0,
                                     0.5 if stray_stores else 0.0)
        ks.append(wl.Kernel(args, kinds, reads, w, rec, cls, 4, st))
    return ks


def same_mem(b, v):
    return np.array_equal(v.mem.materialize(), b.mem)


@pytest.mark.parametrize("seed,budget,chunk,quota,strays", [
    (1, 1 << 18, 4096, 16384, False), (2, 30000, 256, 4096, False), (3, 0, 8192, 32768, False),
    (4, 1 << 18, 4096, 8192, True)])
def test_cow_versions_equals_bytes(seed, budget, chunk, quota, strays):
    rng, lay = world(seed)
    ks = kernels(rng, lay, 30, strays)
    b, v = procs(lay, seed)
    rb = P.cow_checkpoint(b, ks, budget, chunk, quota)
    rv = P.cow_checkpoint(v, ks, budget, chunk, quota)
    assert rb.cow_log == rv.cow_log and rb.copier_log == rv.copier_log
    assert rb.misspec == rv.misspec and rb.kernels_run == rv.kernels_run
    assert rb.stats == rv.stats
    assert np.array_equal(rv.image.materialize(), rb.image)
    assert same_mem(b, v)


@pytest.mark.parametrize("seed,chunk,quota,strays,passes", [
    (5, 4096, 8192, False, 0), (6, 256, 1024, True, 0), (7, 4096, 8192, False, 3)])
def test_recopy_versions_equals_bytes(seed, chunk, quota, strays, passes):
    rng, lay = world(seed)
    ks = kernels(rng, lay, 40, strays)
    b, v = procs(lay, seed)
    if passes:
        rb = P.iterative_recopy(b, ks, chunk, quota, passes, 0)
        rv = P.iterative_recopy(v, ks, chunk, quota, passes, 0)
        assert rb.passes == rv.passes
    else:
        rb = P.recopy_checkpoint(b, ks, chunk, quota)
        rv = P.recopy_checkpoint(v, ks, chunk, quota)
    assert rb.dirty == rv.dirty and rb.copier_log == rv.copier_log
    assert rb.kernels_run == rv.kernels_run and rb.stats == rv.stats
    assert np.array_equal(rv.image.materialize(), rb.image)
    assert same_mem(b, v)


@pytest.mark.parametrize("seed,chunk,quota,stream,strays,odf", [
    (8, 4096, 8192, False, False, False), (9, 256, 2048, True, False, False),
    (10, 4096, 8192, True, True, False), (11, 4096, 8192, True, False, True),
    (12, 256, 2048, True, True, True)])
def test_restore_versions_equals_bytes(seed, chunk, quota, stream, strays, odf):
    rng, lay = world(seed)
    ks = kernels(rng, lay, 30, strays)
    if strays:                                  # a stray load of a buffer not yet restored
        k = ks[1]
        k.trace[7] = np.uint64(int(lay.base(VA0)[lay.n - 1]) + 64)
    img_key = 0xBEEF
    b = P.Process(VA0, lay.off, lay.size, core.words(lay.arena_bytes, KEY, 0), seed)
    v = V.VersionProcess(VA0, lay.off, lay.size, KEY, seed, arena_bytes=lay.arena_bytes)
    image_b = core.words(b.image_bytes, img_key, 0)
    image_v = V.VArray(v.image_bytes, V.Words(img_key), 0)
    rb = P.concurrent_restore(b, image_b, ks, chunk, quota, copier_stream=stream,
                              ondemand_first=odf)
    rv = P.concurrent_restore(v, image_v, ks, chunk, quota, copier_stream=stream,
                              ondemand_first=odf)
    assert rb.ondemand == rv.ondemand and rb.copier_log == rv.copier_log
    assert rb.misspec == rv.misspec and rb.kernels_during == rv.kernels_during
    assert rb.stats == rv.stats
    assert same_mem(b, v)
    if strays:
        assert rb.misspec is not None

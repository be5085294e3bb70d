"""Pins of the oracle's C/R protocols (no GPU).

The correctness arguments of the paper are the pins:
  Section 4.2: the CoW image equals memory at the checkpoint instant t1
  Section 4.3: the recopy image equals memory at t2 (copier done, quiesce)
  Section 6:   concurrent restore + replay equals stop-the-world restore +
               replay (the mutator's writes depend on what it read, so a
               stale read changes the result)
plus the worked scenarios the paper describes for Figures 6, 7 and 9,
closed-form special cases, and planted mistakes that the invariants catch.
"""
import numpy as np
import pytest

from oracle import protocols as P
from paper_2405_12079_b300 import workloads as wl

VA0 = 0x7F00_0000_0000


def make_proc(seed, sizes=None, n=24, lo=1024, hi=40000):
    rng = np.random.default_rng(seed)
    if sizes is None:
        sizes = wl.sizes_uniform(rng, n, lo, hi)
    lay = wl.make_layout(rng, sizes, gap_lo=256, gap_hi=4096)
    arena = np.zeros(lay.arena_bytes, np.uint8)
    wl.fill_random(rng, arena)
    return rng, lay, P.Process(VA0, lay.off, lay.size, arena, seed=seed)


def kernel(rng, lay, reads, writes, n_rec=512, strays=(), stray_frac=0.0):
    reads = np.union1d(np.asarray(reads, np.int64), np.asarray(writes, np.int64))
    writes = np.asarray(writes, np.int64)
    args, kinds = wl.make_args(rng, lay, VA0, reads, writes)
    rec, cls, st = wl.trace_runs(rng, lay, VA0, reads, writes, n_rec, stray_frac, 0.0)
    k = wl.Kernel(args, kinds, reads, writes, rec, cls, 4, st)
    for r, buf in strays:          # planted stray store into buffer ``buf``
        a = int(lay.base(VA0)[buf]) + 4 * int(rng.integers(0, int(lay.size[buf]) // 4 - 1))
        k.trace[r] = np.uint64(a) | wl.STORE_BIT
        k.labels[r] = wl.CLS_OTHER
        k.strays.append((r, a))
    return k


def seq(rng, lay, K):
    ks = []
    for _ in range(K):
        r, w = wl.pick_sets(rng, lay.n, 1, 6)
        ks.append(kernel(rng, lay, r, w))
    return ks


@pytest.mark.parametrize("seed,budget,chunk,quota", [
    (1, 1 << 20, 4096, 16384), (2, 60000, 4096, 8192), (3, 0, 8192, 32768),
    (4, 1 << 18, 1 << 16, 1 << 16), (5, 30000, 256, 4096)])
def test_cow_image_equals_memory_at_t1(seed, budget, chunk, quota):
    rng, lay, proc = make_proc(seed)
    ks = seq(rng, lay, 40)
    t1 = P.stw_checkpoint(proc)
    res = P.cow_checkpoint(proc, ks, budget, chunk, quota)
    assert res.misspec is None
    assert np.array_equal(res.image, t1)
    if budget == 0:
        assert all(e[2] == "D" for e in res.cow_log)
    # every CoW happened to a speculated-write buffer of that kernel
    for k, i, kind, off, ln in res.cow_log:
        assert i in set(ks[k].writes.tolist())


def test_cow_special_cases():
    rng, lay, proc = make_proc(10)
    ks = seq(rng, lay, 10)
    t1 = P.stw_checkpoint(proc)
    # zero kernels: a plain stop-the-world copy
    r0 = P.cow_checkpoint(proc, [], 1 << 20, 4096, 4096)
    assert np.array_equal(r0.image, t1) and r0.cow_log == [] and r0.kernels_run == 0
    # a copier that finishes before the first kernel needs no CoW
    r1 = P.cow_checkpoint(proc, ks, 1 << 20, 1 << 20, 1 << 30)
    assert r1.cow_log == [] and r1.kernels_run == 0 and np.array_equal(r1.image, t1)


def test_cow_figure6_scenario():
    """Fig. 6: a kernel writing an uncheckpointed buffer copies it to a free
    device buffer first; later writers of the same buffer do not copy again;
    with no free device memory the buffer goes straight to the checkpoint."""
    sizes = np.full(5, 8192, np.uint64)
    rng, lay, proc = make_proc(20, sizes=sizes)
    t1 = P.stw_checkpoint(proc)
    k1 = kernel(rng, lay, [0], [2])
    k2 = kernel(rng, lay, [0], [3])
    k3 = kernel(rng, lay, [1], [2])
    res = P.cow_checkpoint(proc, [k1, k2, k3], 8192, 4096, 4096)
    assert [(e[0], e[1], e[2]) for e in res.cow_log] == [(0, 2, "S"), (1, 3, "D")]
    assert np.array_equal(res.image, t1)


def test_cow_misspeculation_fallback():
    """Section 4.2: a store the speculation missed, into a buffer not yet
    checkpointed, discards the checkpoint and takes a stop-the-world one."""
    rng, lay, proc = make_proc(30, sizes=np.full(8, 16384, np.uint64))
    ks = [kernel(rng, lay, [0], [1]), kernel(rng, lay, [2], [3], strays=[(5, 7)]),
          kernel(rng, lay, [1], [4])]
    res = P.cow_checkpoint(proc, ks, 1 << 20, 4096, 4096)
    assert res.misspec == 1
    assert np.array_equal(res.image, P.stw_checkpoint(proc))   # memory after kernel 1
    # the same stray into a buffer that is already checkpointed is harmless
    rng, lay, proc = make_proc(31, sizes=np.full(8, 16384, np.uint64))
    t1 = P.stw_checkpoint(proc)
    ks = [kernel(rng, lay, [5], [6]), kernel(rng, lay, [5], [6], strays=[(3, 0)])]
    res = P.cow_checkpoint(proc, ks, 1 << 20, 16384, 16384)
    assert res.misspec is None and np.array_equal(res.image, t1)


def test_cow_planted_mistake_is_caught(monkeypatch):
    """An oracle that ignores the validator, facing a missed store, breaks
    the Section 4.2 invariant -- so the invariant test has teeth."""
    rng, lay, proc = make_proc(32, sizes=np.full(8, 16384, np.uint64))
    t1 = P.stw_checkpoint(proc)
    ks = [kernel(rng, lay, [0], [1]), kernel(rng, lay, [2], [3], strays=[(5, 7)])]
    monkeypatch.setattr(P, "victims_of_store", lambda *a: [])
    res = P.cow_checkpoint(proc, ks, 1 << 20, 4096, 4096)
    assert res.misspec is None and not np.array_equal(res.image, t1)


@pytest.mark.parametrize("seed,chunk,quota", [(40, 4096, 8192), (41, 256, 2048),
                                              (42, 1 << 16, 1 << 16)])
def test_recopy_image_equals_memory_at_t2(seed, chunk, quota):
    rng, lay, proc = make_proc(seed)
    ks = seq(rng, lay, 60)
    res = P.recopy_checkpoint(proc, ks, chunk, quota)
    assert np.array_equal(res.image, P.stw_checkpoint(proc))     # memory now == at t2
    wr = set()
    for k in ks[:res.kernels_run]:
        wr |= set(k.writes.tolist())
    assert set(res.dirty) <= wr


def test_recopy_figure7_scenario():
    """Fig. 7: B1 written after it was copied and B3 written while being
    copied are dirty; B5, written before the copier reached it, is not."""
    sizes = np.full(6, 8192, np.uint64)
    rng, lay, proc = make_proc(50, sizes=sizes)
    # the copier moves 3.5 buffers before the kernel: B0..B2 done, B3 in
    # flight, B4 and B5 pending
    ks = [kernel(rng, lay, [0], [1, 3, 5])]
    res = P.recopy_checkpoint(proc, ks, 4096, 7 * 4096)
    assert res.dirty == [1, 3]
    assert np.array_equal(res.image, P.stw_checkpoint(proc))


def test_recopy_victims_join_dirty_set():
    """Section 4.3: validator victims are added to the dirty set if dirty."""
    sizes = np.full(6, 8192, np.uint64)
    rng, lay, proc = make_proc(51, sizes=sizes)
    ks = [kernel(rng, lay, [4], [5], strays=[(9, 0)])]
    res = P.recopy_checkpoint(proc, ks, 4096, 4 * 4096)
    assert res.dirty == [0]
    assert np.array_equal(res.image, P.stw_checkpoint(proc))


def _restore_pair(seed, K=40, chunk=4096, quota=8192, sizes=None, plant=None,
                  kernels=None):
    rng, lay, proc = make_proc(seed, sizes=sizes)
    image = P.stw_checkpoint(proc)
    ks = kernels(rng, lay) if kernels else seq(rng, lay, K)
    # reference: stop-the-world restore, then replay
    ref = P.Process(VA0, lay.off, lay.size, np.zeros(lay.arena_bytes, np.uint8), seed)
    P.stw_restore(ref, image)
    for j, k in enumerate(ks):
        ref.run_kernel(j, k)
    # concurrent: fresh (wrong) memory, on-demand + background restore
    cur = P.Process(VA0, lay.off, lay.size, np.full(lay.arena_bytes, 0xA5, np.uint8), seed)
    res = P.concurrent_restore(cur, image, ks, chunk, quota)
    mask = np.zeros(lay.arena_bytes, bool)
    for o, s in zip(lay.off, lay.size):
        mask[int(o):int(o) + int(s)] = True
    return res, cur.mem[mask], ref.mem[mask]


@pytest.mark.parametrize("seed,chunk,quota", [(60, 4096, 8192), (61, 256, 1024),
                                              (62, 1 << 16, 1 << 17)])
def test_restore_equals_stw_restore_plus_replay(seed, chunk, quota):
    res, got, ref = _restore_pair(seed, chunk=chunk, quota=quota)
    assert res.misspec is None
    assert np.array_equal(got, ref)


def test_restore_figure9_scenario():
    """Fig. 9: K0 waits for its buffer B1 to be copied on demand; K1 and K2
    find their buffers already restored and run while B3, B4 are copied."""
    sizes = np.full(5, 8192, np.uint64)

    def ks(rng, lay):
        return [kernel(rng, lay, [1], [1]), kernel(rng, lay, [0], [0]),
                kernel(rng, lay, [1, 2], [2])]
    res, got, ref = _restore_pair(70, sizes=sizes, chunk=4096, quota=8192, kernels=ks)
    assert [(e[0], e[1]) for e in res.ondemand] == [(0, 1)]   # only K0 waits
    # K1 and K2 overlap with the background copy of B2, B3 and B4
    assert sorted({e[1] for e in res.copier_log if e[0] >= 1}) == [2, 3, 4]
    assert np.array_equal(got, ref)


def test_restore_misspeculation_rolls_back():
    """Section 6: a read the speculation missed, of a buffer not yet
    restored, rolls back and restores stop-the-world, then replays."""
    sizes = np.full(8, 8192, np.uint64)

    def ks(rng, lay):
        k1 = kernel(rng, lay, [0], [1])
        k1.trace[3] = np.uint64(int(lay.base(VA0)[7]) + 64)     # stray load
        k1.labels[3] = wl.CLS_OTHER
        return [kernel(rng, lay, [0], [0]), k1, kernel(rng, lay, [2], [3])]
    res, got, ref = _restore_pair(71, sizes=sizes, chunk=4096, quota=4096, kernels=ks)
    assert res.misspec == 1
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("seed,chunk,quota", [(60, 4096, 8192), (61, 256, 1024)])
def test_restore_copier_stream_without_strays_is_the_same(seed, chunk, quota):
    """With every access speculated, a copier on its own stream changes no
    decision: the same on-demand list, copier pieces and final memory."""
    a, got_a, ref = _restore_pair(seed, chunk=chunk, quota=quota)
    rng, lay, proc = make_proc(seed)
    image = P.stw_checkpoint(proc)
    ks = seq(rng, lay, 40)
    cur = P.Process(VA0, lay.off, lay.size, np.full(lay.arena_bytes, 0xA5, np.uint8), seed)
    b = P.concurrent_restore(cur, image, ks, chunk, quota, copier_stream=True)
    assert b.misspec is None and a.misspec is None
    assert b.ondemand == a.ondemand and b.copier_log == a.copier_log
    mask = np.zeros(lay.arena_bytes, bool)
    for o, sz in zip(lay.off, lay.size):
        mask[int(o):int(o) + int(sz)] = True
    assert np.array_equal(cur.mem[mask], ref)


def _stray_restore(copier_stream, need_k1):
    """8 buffers of 8 KiB, one buffer per copier round: round 0 restores
    buffer 0, round 1 buffer 1.  K0 needs buffer 5; K1 needs need_k1 and
    makes an unspeculated access to buffer 0."""
    sizes = np.full(8, 8192, np.uint64)

    def ks(rng, lay):
        k1 = kernel(rng, lay, [need_k1], [need_k1], strays=[(5, 0)])
        return [kernel(rng, lay, [5], [5]), k1, kernel(rng, lay, [6], [6])]
    rng, lay, proc = make_proc(73, sizes=sizes)
    image = P.stw_checkpoint(proc)
    kk = ks(rng, lay)
    ref = P.Process(VA0, lay.off, lay.size, np.zeros(lay.arena_bytes, np.uint8), 73)
    P.stw_restore(ref, image)
    for j, k in enumerate(kk):
        ref.run_kernel(j, k)
    cur = P.Process(VA0, lay.off, lay.size, np.full(lay.arena_bytes, 0xA5, np.uint8), 73)
    res = P.concurrent_restore(cur, image, kk, 4096, 8192, copier_stream=copier_stream)
    mask = np.zeros(lay.arena_bytes, bool)
    for o, sz in zip(lay.off, lay.size):
        mask[int(o):int(o) + int(sz)] = True
    return res, np.array_equal(cur.mem[mask], ref.mem[mask])


def test_restore_copier_stream_unwaited_buffer_is_not_restored():
    """Buffer 0 is present (copied in round 0) but no kernel has waited for
    the copier yet: an unspeculated access to it in K1 is a mis-speculation
    with the copier on its own stream and not in lockstep."""
    lock, ok_lock = _stray_restore(False, 3)
    stream, ok_stream = _stray_restore(True, 3)
    assert lock.misspec is None and stream.misspec == 1
    assert ok_lock and ok_stream


def test_restore_copier_stream_wait_covers_earlier_pieces():
    """K1 needs buffer 1, whose last piece is from round 1: waiting for it
    also lands buffer 0's round-0 pieces, so the access to buffer 0 is fine."""
    lock, ok_lock = _stray_restore(False, 1)
    stream, ok_stream = _stray_restore(True, 1)
    assert lock.misspec is None and stream.misspec is None
    assert ok_lock and ok_stream


def _odf_restore(seed, chunk=4096, quota=8192, kernels=None, K=40, sizes=None):
    """The same restore with the copier on its own stream, in both round
    orders: the copier's move before the round's on-demand copies (the
    default) and after them (ondemand_first)."""
    rng, lay, proc = make_proc(seed, sizes=sizes)
    image = P.stw_checkpoint(proc)
    ks = kernels(rng, lay) if kernels else seq(rng, lay, K)
    ref = P.Process(VA0, lay.off, lay.size, np.zeros(lay.arena_bytes, np.uint8), seed)
    P.stw_restore(ref, image)
    for j, k in enumerate(ks):
        ref.run_kernel(j, k)
    mask = np.zeros(lay.arena_bytes, bool)
    for o, sz in zip(lay.off, lay.size):
        mask[int(o):int(o) + int(sz)] = True
    out = []
    for odf in (False, True):
        cur = P.Process(VA0, lay.off, lay.size, np.full(lay.arena_bytes, 0xA5, np.uint8),
                        seed)
        res = P.concurrent_restore(cur, image, ks, chunk, quota, copier_stream=True,
                                   ondemand_first=odf)
        out.append((res, np.array_equal(cur.mem[mask], ref.mem[mask])))
    return ks, lay, out


@pytest.mark.parametrize("seed,chunk,quota", [(60, 4096, 8192), (61, 256, 1024),
                                              (62, 1 << 16, 1 << 17)])
def test_restore_ondemand_first_equals_stw_restore_plus_replay(seed, chunk, quota):
    """Sec. 6 correctness in the on-demand-first round order: the final
    memory is the stop-the-world restore followed by the replay, as in the
    default order; every byte is restored once (copier + on-demand = the
    image's buffers), and the copier never moves a buffer the same round's
    kernel is speculated to access."""
    ks, lay, out = _odf_restore(seed, chunk=chunk, quota=quota)
    (a, ok_a), (b, ok_b) = out
    assert ok_a and ok_b and a.misspec is None and b.misspec is None
    total = int(sum(int(s) for s in lay.size))
    assert b.stats["ondemand_bytes"] + b.stats["copier_bytes"] == total
    rng = np.random.default_rng(0)
    proc = P.Process(VA0, lay.off, lay.size, np.zeros(lay.arena_bytes, np.uint8), seed)
    for r, i, off, ln, _ in b.copier_log:
        if r < b.kernels_during:
            assert proc.speculate(ks[r])[i] == 0, (r, i)
    # in the default order the copier does move buffers of its round's kernel
    assert any(r < a.kernels_during and proc.speculate(ks[r])[i] != 0
               for r, i, off, ln, _ in a.copier_log)


def test_restore_ondemand_first_scenario():
    """Five 8 KiB buffers, two 4 KiB pieces per round.  K0 needs B0: in the
    default order the copier's round 0 moves B0 and K0 waits for those
    pieces; on demand first, K0 fetches B0 itself and the copier's round 0
    moves B1.  K1 needs B1: present either way (copied in round 0 or 1).
    K2 needs B2 and B3: B3 on demand in both orders; B2 the copier moved in
    round 2 of the default order (K2 waits for it), in round 1 on demand
    first."""
    sizes = np.full(5, 8192, np.uint64)

    def ks(rng, lay):
        return [kernel(rng, lay, [0], [0]), kernel(rng, lay, [1], [1]),
                kernel(rng, lay, [2, 3], [3])]
    kk, lay, out = _odf_restore(74, sizes=sizes, chunk=4096, quota=8192, kernels=ks)
    (a, ok_a), (b, ok_b) = out
    assert ok_a and ok_b and a.misspec is None and b.misspec is None
    assert [(e[0], e[1]) for e in a.ondemand] == [(2, 3)]
    assert [(e[0], e[1]) for e in a.copier_log][:6] == [(0, 0), (0, 0), (1, 1), (1, 1),
                                                      (2, 2), (2, 2)]
    assert [(e[0], e[1]) for e in b.ondemand] == [(0, 0), (2, 3)]
    assert [(e[0], e[1]) for e in b.copier_log][:4] == [(0, 1), (0, 1), (1, 2), (1, 2)]


def test_restore_ondemand_first_misspeculation_rolls_back():
    """A stray load of a buffer not yet restored rolls back in the
    on-demand-first order too, at the same round."""
    sizes = np.full(8, 8192, np.uint64)

    def ks(rng, lay):
        k1 = kernel(rng, lay, [0], [1])
        k1.trace[3] = np.uint64(int(lay.base(VA0)[7]) + 64)     # stray load
        k1.labels[3] = wl.CLS_OTHER
        return [kernel(rng, lay, [0], [0]), k1, kernel(rng, lay, [2], [3])]
    kk, lay, out = _odf_restore(71, sizes=sizes, chunk=4096, quota=4096, kernels=ks)
    (a, ok_a), (b, ok_b) = out
    assert a.misspec == 1 and b.misspec == 1
    assert ok_a and ok_b


def test_restore_planted_mistake_is_caught(monkeypatch):
    """An oracle that skips on-demand copies reads stale data, and the
    read-dependent mutator makes the final memory differ."""
    orig = P.Process.speculate
    monkeypatch.setattr(P.Process, "speculate",
                        lambda self, kern: np.zeros_like(orig(self, kern)))
    monkeypatch.setattr(P, "victims_of", lambda res, n: np.zeros(0, np.int64))
    res, got, ref = _restore_pair(72)
    assert not np.array_equal(got, ref)


def _copier_log(sizes, chunk, quota, rounds, skip=lambda i: False, done=()):
    cp = P.Copier(len(sizes), sizes, chunk)
    for i in done:
        cp.state[i] = P.DONE
        cp.copied[i] = sizes[i]
    for r in range(rounds):
        cp.advance(quota, lambda i, off, ln: False, r, skip)
    return [e[:4] for e in cp.log], cp.done()


def test_copier_piece_schedule_by_hand():
    """The copier's pieces written out by hand (Section 4.2 copy phase; the
    4 MB chunking of Section 5, here 1 KiB): sizes that are not multiples
    of 256, chunk 1024, quota 1536 per round.  Shows that a piece charges
    align256(len) against the quota (300 -> 512, 904 -> 1024, 257 -> 512),
    is cut at the quota left in the round (512-byte pieces), never crosses
    into the next buffer (904 = the rest of buffer 1), and that the cursor
    moves on to the next buffer within a round."""
    log, done = _copier_log([300, 5000, 257], 1024, 1536, 4)
    assert log == [
        (0, 0, 0, 300), (0, 1, 0, 1024),
        (1, 1, 1024, 1024), (1, 1, 2048, 512),
        (2, 1, 2560, 1024), (2, 1, 3584, 512),
        (3, 1, 4096, 904), (3, 2, 0, 257),
    ]
    assert done
    # one round short: not done, buffer 2 untouched
    log, done = _copier_log([300, 5000, 257], 1024, 1536, 3)
    assert len(log) == 6 and not done


def test_copier_cursor_skips_done_and_skipped_buffers():
    """Buffers already done (a direct CoW copy, an on-demand restore) or
    skipped (present) cost no quota: the cursor passes them in the same
    round."""
    log, done = _copier_log([300, 5000, 257], 1024, 1536, 1, skip=lambda i: i == 1)
    assert log == [(0, 0, 0, 300), (0, 2, 0, 257)] and done
    log, done = _copier_log([300, 5000, 257, 700], 1024, 1536, 1, done=(0, 2))
    assert log == [(0, 1, 0, 1024), (0, 1, 1024, 512)] and not done
    # an in-flight buffer finished elsewhere (on-demand restore of its
    # remaining bytes) is not copied again
    cp = P.Copier(2, [2048, 600], 1024)
    cp.advance(1024, lambda i, off, ln: False, 0)
    cp.copied[0], cp.state[0] = 2048, P.DONE
    cp.advance(1024, lambda i, off, ln: False, 1)
    assert [e[:4] for e in cp.log] == [(0, 0, 0, 1024), (1, 1, 0, 600)]


def test_first_fit_allocator():
    a = P.FirstFit(1024)
    assert a.alloc(256) == 0 and a.alloc(512) == 256 and a.alloc(512) is None
    a.release(0, 256)
    assert a.alloc(256) == 0
    a.release(256, 512)
    a.release(0, 256)
    assert a.free == [(0, 1024)]


@pytest.mark.parametrize("seed,passes", [(80, 3), (81, 6)])
def test_iterative_recopy_image_equals_memory_at_t2(seed, passes):
    """Iterative concurrent recopy: the image still equals memory at t2, and
    the stop-the-world recopy at the end is no larger than the single-round
    protocol's (each extra pass only starts when the dirty bytes shrink)."""
    rng, lay, proc = make_proc(seed, n=40)
    ks = seq(rng, lay, 200)
    mem0 = proc.mem.copy()
    one = P.recopy_checkpoint(proc, ks, 4096, 16384)
    proc.mem[:] = mem0
    res = P.iterative_recopy(proc, ks, 4096, 16384, passes, 0)
    assert np.array_equal(res.image, P.stw_checkpoint(proc))
    assert len(res.passes) >= 1
    sizes = [b for _, _, b in res.passes]
    assert all(x > y for x, y in zip(sizes, sizes[1:]))     # strictly shrinking
    assert res.stats["recopy_bytes"] <= one.stats["recopy_bytes"] or \
        res.kernels_run > one.kernels_run


def test_iterative_recopy_without_extra_passes_is_the_soft_recopy():
    rng, lay, proc = make_proc(82, n=30)
    ks = seq(rng, lay, 80)
    mem0 = proc.mem.copy()
    one = P.recopy_checkpoint(proc, ks, 4096, 8192)
    proc.mem[:] = mem0
    it = P.iterative_recopy(proc, ks, 4096, 8192, 0, 0)
    assert it.dirty == one.dirty and it.copier_log == one.copier_log
    assert it.kernels_run == one.kernels_run and np.array_equal(it.image, one.image)

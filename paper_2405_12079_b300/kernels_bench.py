"""Kernel microbenchmarks of the data plane (CUDA events, after warm-up).

    python -m paper_2405_12079_b300.kernels_bench [--kernel validate|copy|all]
                                                  [--traces K] [--copy-gb G]

validate: one launch over K concatenated 1.3M-record training-kernel traces
          (1,000-buffer table; K = 160 -> 208M records, 1.7 GB), plus one
          launch per single trace, plus a random-record trace.
copy:     G GB of 4 MB regions device->device, device->pinned host and
          pinned host->device through the copy engine, next to the DMA
          engines (torch copy_) on the same buffers.
validate_rounds:        native recopy sessions, one validation launch per
          round against deferred validation (--rounds-nrec records per round).
validate_rounds_launch: one deferred launch over 16 distinct 1.3M-record
          traces against 16 plain launches and one over their concatenation.
protocol_kernels:       the small protocol kernels (device-decided rounds,
          the rule kernel, image manifest and verified restore) in their
          sessions.
image_manifest:         the manifest (digest of every buffer) of a 2 GB
          device-resident image.
Prints one JSON object.  Inputs are larger than L2 unless stated.
"""
import argparse
import json
import sys

import numpy as np
import torch

from . import phos, workloads as wl

VA0 = 0x7E00_0000_0000


def timeit(fn, reps=10, warm=3):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def bench_validate(K, out, variants=(1, 2)):
    s = torch.cuda.current_stream().cuda_stream
    cfg = wl.training(n_kernels=1)
    lay, rng = cfg["layout"], cfg["rng"]
    t = phos.Table(lay.base(VA0), lay.size)
    reads, writes = wl.pick_sets(rng, lay.n)
    perm = np.zeros(lay.n, np.uint8)
    perm[reads] = phos.PERM_R
    perm[writes] = phos.PERM_RW
    rec, _, _ = wl.trace_runs(rng, lay, VA0, reads, writes, 1_300_000, 0.001, 0.0)
    big = torch.from_numpy(np.tile(rec, K).view(np.uint8)).cuda()
    N = len(rec) * K
    d_perm = torch.from_numpy(perm).cuda()
    bm = torch.empty(((N + 31) // 32) * 4, dtype=torch.uint8, device="cuda")
    cnt = torch.empty(24, dtype=torch.uint8, device="cuda")
    vv = torch.empty(256, dtype=torch.uint8, device="cuda")
    st = torch.zeros(4, dtype=torch.uint8, device="cuda")

    def run(ptr, nrec):
        phos.validate(t, d_perm.data_ptr(), ptr, nrec, 4, bm.data_ptr(), cnt.data_ptr(),
                      vv.data_ptr(), vv.data_ptr() + 128, None, 0, st.data_ptr(), s)

    n1 = len(rec)
    rr, _ = wl.trace_random(rng, lay, VA0, np.asarray(writes), 64 * 1_000_000)
    rrd = torch.from_numpy(rr.view(np.uint8)).cuda()
    for v in variants:
        phos.validate_config(v)
        tag = "v%d" % v
        ms = timeit(lambda: run(big.data_ptr(), N))
        out["validate_concat_" + tag] = dict(records=N, ms=ms, grec_s=N / ms / 1e6,
                                             gbs=N * 8.125 / ms / 1e6)
        ms = timeit(lambda: [run(big.data_ptr() + 8 * n1 * j, n1) for j in range(K)], 3, 1) / K
        out["validate_per_trace_" + tag] = dict(records=n1, us=1e3 * ms, grec_s=n1 / ms / 1e6,
                                                gbs=n1 * 8.125 / ms / 1e6)
        ms = timeit(lambda: run(rrd.data_ptr(), len(rr)))
        out["validate_random_" + tag] = dict(records=len(rr), ms=ms, grec_s=len(rr) / ms / 1e6)
        # the per-trace launches replayed from a CUDA graph: device time
        # without the host's per-call overhead
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        cs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cs):
            run(big.data_ptr(), n1)                  # warm scratch outside capture
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=cs):
                for j in range(K):
                    phos.validate(t, d_perm.data_ptr(), big.data_ptr() + 8 * n1 * j, n1, 4,
                                  bm.data_ptr(), cnt.data_ptr(), vv.data_ptr(),
                                  vv.data_ptr() + 128, None, 0, st.data_ptr(),
                                  cs.cuda_stream)
        ms = timeit(lambda: g.replay(), 3, 1) / K
        out["validate_per_trace_graph_" + tag] = dict(records=n1, us=1e3 * ms,
                                                      grec_s=n1 / ms / 1e6)
    # grid sweep for one 1.3M-record trace (launch-bound shape)
    for ctas in (148, 147, 128, 96, 74, 48, 37, 24):
        phos.validate_grid(ctas)
        ms = timeit(lambda: [run(big.data_ptr() + 8 * n1 * j, n1) for j in range(K)], 3, 1) / K
        out["validate_per_trace_grid%d" % ctas] = dict(us=1e3 * ms)
    phos.validate_grid(0)
    phos.validate_config(0)


def bench_validate_distinct(K, out, reps=5):
    """Validation over K distinct training-kernel traces (each kernel its
    own read/write sets, as the benchmark's 200 kernels) in one launch, with
    the union of their speculated sets, next to the first 50 of them, next
    to K copies of the first trace with that trace's own speculated set."""
    s = torch.cuda.current_stream().cuda_stream
    cfg = wl.training(n_kernels=K)
    lay, rng = cfg["layout"], cfg["rng"]
    t = phos.Table(lay.base(VA0), lay.size)
    ks = wl.make_training_kernels(rng, lay, VA0, K, 1_300_000, 0.001)
    perms = []
    for k in ks:
        p = np.zeros(lay.n, np.uint8)
        p[k.reads] = phos.PERM_R
        p[k.writes] = phos.PERM_RW
        perms.append(p)
    n1 = len(ks[0].trace)
    big = torch.from_numpy(np.concatenate([k.trace for k in ks]).view(np.uint8)).cuda()
    tiled = torch.from_numpy(np.tile(ks[0].trace, K).view(np.uint8)).cuda()
    u_all = torch.from_numpy(np.maximum.reduce(perms)).cuda()
    u_50 = torch.from_numpy(np.maximum.reduce(perms[:50])).cuda()
    p0 = torch.from_numpy(perms[0]).cuda()
    N = n1 * K
    bm = torch.empty(((N + 31) // 32) * 4, dtype=torch.uint8, device="cuda")
    cnt = torch.empty(24, dtype=torch.uint8, device="cuda")
    vv = torch.empty(256, dtype=torch.uint8, device="cuda")
    st = torch.zeros(4, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flush_r = torch.ones(256 << 20, dtype=torch.uint8, device="cuda")
    acc = torch.zeros(1, dtype=torch.int64, device="cuda")

    def run(perm, ptr, nrec):
        phos.validate(t, perm.data_ptr(), ptr, nrec, 4, bm.data_ptr(), cnt.data_ptr(),
                      vv.data_ptr(), vv.data_ptr() + 128, None, 0, st.data_ptr(), s)

    def timed(fn):
        fn()
        ts = []
        for _ in range(reps):
            # L2 flush: a 256 MB write, then a 256 MB read of another
            # buffer, so that no dirty lines are left for the timed launch
            # to write back
            flush.zero_()
            torch.sum(flush_r.view(torch.int64), dim=(0,), out=acc[0])
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts)), float(np.min(ts))

    # ~1.5 s of launches first: an idle GPU runs the first ones at lower clocks
    import time
    t_warm = time.time() + 1.5
    while time.time() < t_warm:
        run(u_all, big.data_ptr(), N)
        torch.cuda.synchronize()
    for name, perm, ptr, nrec in (("distinct_all", u_all, big.data_ptr(), N),
                                  ("distinct_50", u_50, big.data_ptr(), n1 * min(50, K)),
                                  ("tiled_one", p0, tiled.data_ptr(), N)):
        med, best = timed(lambda: run(perm, ptr, nrec))
        out["validate_" + name] = dict(records=nrec, ms_median=med, ms_best=best,
                                       grec_s=nrec / med / 1e6, gbs=nrec * 8.125 / med / 1e6,
                                       violations=int(cnt.cpu().numpy().view(np.uint64)[0]))


def bench_emit(K, out):
    """Validation with the ascending index list (k_validate_emit after
    k_validate_b) over K concatenated training traces with 1 % stray
    records, index list capped at 4M entries."""
    s = torch.cuda.current_stream().cuda_stream
    cfg = wl.training(n_kernels=1)
    lay, rng = cfg["layout"], cfg["rng"]
    t = phos.Table(lay.base(VA0), lay.size)
    reads, writes = wl.pick_sets(rng, lay.n)
    perm = np.zeros(lay.n, np.uint8)
    perm[reads] = phos.PERM_R
    perm[writes] = phos.PERM_RW
    rec, _, _ = wl.trace_runs(rng, lay, VA0, reads, writes, 1_300_000, 0.01, 0.0)
    big = torch.from_numpy(np.tile(rec, K).view(np.uint8)).cuda()
    N = len(rec) * K
    cap = 4 << 20
    d_perm = torch.from_numpy(perm).cuda()
    bm = torch.empty(((N + 31) // 32) * 4, dtype=torch.uint8, device="cuda")
    cnt = torch.empty(24, dtype=torch.uint8, device="cuda")
    vv = torch.empty(256, dtype=torch.uint8, device="cuda")
    idx = torch.empty(8 * cap, dtype=torch.uint8, device="cuda")
    st = torch.zeros(4, dtype=torch.uint8, device="cuda")

    def run(with_idx):
        phos.validate(t, d_perm.data_ptr(), big.data_ptr(), N, 4, bm.data_ptr(), cnt.data_ptr(),
                      vv.data_ptr(), vv.data_ptr() + 128, idx.data_ptr() if with_idx else None,
                      cap if with_idx else 0, st.data_ptr(), s)
    ms_plain = timeit(lambda: run(False))
    ms_idx = timeit(lambda: run(True))
    out["validate_with_index_list"] = dict(records=N, violations=int(
        cnt.cpu().numpy().view(np.uint64)[0]), ms_without=ms_plain, ms_with=ms_idx,
        emit_ms=ms_idx - ms_plain)


def bench_validate_rounds(out, K=64, n_rec=65536):
    """Recopy sessions of K kernel rounds with n_rec-record traces over the
    1,000-buffer training layout (1/20 scale, the copier held to 256 bytes
    per round): one validation launch per round against up to 16 rounds per
    launch (deferred validation).  Times the rounds only (K is a multiple
    of 16, so every queued round is validated inside the timed region)."""
    import time
    from . import runner
    s = torch.cuda.current_stream().cuda_stream
    cfg = wl.training(scale=0.05, n_kernels=K)
    rng, lay = cfg["rng"], cfg["layout"]
    arena = torch.empty(lay.arena_bytes, dtype=torch.uint8, device="cuda")
    phos.harness_fill(arena.data_ptr(), lay.arena_bytes, cfg["seed"], s)
    kernels = wl.make_training_kernels(rng, lay, arena.data_ptr(), K, n_rec, 0.001)
    dp = runner.DeviceProcess(lay, arena, cfg["seed"], kernels)
    image = torch.empty(dp.image_bytes, dtype=torch.uint8).pin_memory()
    ks = dp.native_kernels()

    def session(flags):
        c = phos.Checkpoint(dp.table, phos.CKPT_RECOPY | flags, image.data_ptr(), image.numel(),
                            4 << 20, 4, None, 0, s)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k = phos.harness_drive_ckpt(c, dp.table, dp.seed, 256, ks, s)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        dirty = c.stats()["dirty"]
        c.finish()
        c.close()
        return 1e3 * (t1 - t0) / k, dirty
    for name, flags in (("concurrent", phos.CKPT_CONCURRENT),
                        ("deferred", phos.CKPT_CONCURRENT | phos.CKPT_DEFER)):
        session(flags)
        best, dirty = min(session(flags) for _ in range(3))
        out["rounds_" + name] = dict(rounds=K, records_per_round=n_rec, ms_per_round=best,
                                    dirty=dirty)


def bench_validate_rounds_launch(out, K=16, reps=7):
    """Deferred validation of K distinct training-kernel traces (1.3M
    records each, each round its own speculated perms) in one
    k_validate_rounds launch (phos_harness_validate_rounds, recopy rule),
    against K phos_validate launches over the same traces and one
    phos_validate launch over their concatenation with the union of the
    perms.  L2 flushed before every repetition (a 256 MB write, then a
    256 MB read of another buffer)."""
    s = torch.cuda.current_stream().cuda_stream
    cfg = wl.training(n_kernels=K)
    lay, rng = cfg["layout"], cfg["rng"]
    t = phos.Table(lay.base(VA0), lay.size)
    ks = wl.make_training_kernels(rng, lay, VA0, K, 1_300_000, 0.001)
    perms = []
    for k in ks:
        p = np.zeros(lay.n, np.uint8)
        p[k.reads] = phos.PERM_R
        p[k.writes] = phos.PERM_RW
        perms.append(torch.from_numpy(p).cuda())
    trs = [torch.from_numpy(k.trace.view(np.uint8).copy()).cuda() for k in ks]
    n1 = len(ks[0].trace)
    N = n1 * K
    cat = torch.cat(trs)
    uperm = torch.stack(perms).max(dim=0).values.contiguous()
    nvw = (lay.n + 31) // 32
    bm = torch.empty(((N + 31) // 32) * 4, dtype=torch.uint8, device="cuda")
    cnt = torch.empty(24, dtype=torch.uint8, device="cuda")
    vv = torch.empty(8 * nvw, dtype=torch.uint8, device="cuda")
    st = torch.zeros(4, dtype=torch.uint8, device="cuda")
    sb, kmax = phos.harness_rounds_scratch(t)
    scr = torch.zeros(max(sb, 256), dtype=torch.uint8, device="cuda")
    flags = torch.ones(lay.n, dtype=torch.uint8, device="cuda")
    dirty = torch.zeros(lay.n, dtype=torch.uint8, device="cuda")
    acc = torch.from_numpy(np.array([0, 0, 0, 0, 2**64 - 1, 0, 0, 0], np.uint64)
                           .view(np.uint8).copy()).cuda()
    flag = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    rounds = [(tr.data_ptr(), n1, pm.data_ptr(), flags.data_ptr(), j)
              for j, (tr, pm) in enumerate(zip(trs, perms))]
    flw = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flr = torch.ones(256 << 20, dtype=torch.uint8, device="cuda")
    fl_acc = torch.zeros(1, dtype=torch.int64, device="cuda")

    def deferred():
        phos.harness_validate_rounds(t, rounds[:min(K, kmax)], 4, 1, dirty.data_ptr(),
                                     acc.data_ptr(), flag.data_ptr(), st.data_ptr(),
                                     scr.data_ptr(), s)

    def per_round():
        for tr, pm in zip(trs, perms):
            phos.validate(t, pm.data_ptr(), tr.data_ptr(), n1, 4, bm.data_ptr(), cnt.data_ptr(),
                          vv.data_ptr(), vv.data_ptr() + 4 * nvw, None, 0, st.data_ptr(), s)

    def concat():
        phos.validate(t, uperm.data_ptr(), cat.data_ptr(), N, 4, bm.data_ptr(), cnt.data_ptr(),
                      vv.data_ptr(), vv.data_ptr() + 4 * nvw, None, 0, st.data_ptr(), s)

    def flushed(fn):
        fn()
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            flw.zero_()
            torch.sum(flr.view(torch.int64), dim=(0,), out=fl_acc[0])
            torch.cuda._sleep(100_000)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts)), float(np.min(ts))

    import time
    t_warm = time.time() + 1.5
    while time.time() < t_warm:
        concat()
        torch.cuda.synchronize()
    for name, fn, launches, bpr in (("deferred_one_launch", deferred, 1, 8.0),
                                    ("per_round_launches", per_round, K, 8.125),
                                    ("concat_one_launch", concat, 1, 8.125)):
        med, best = flushed(fn)
        out["validate_rounds_" + name] = dict(
            rounds=K, records=N, launches=launches, ms_median=med, ms_best=best,
            grec_s=N / med / 1e6, gbs=N * bpr / med / 1e6, bytes_per_record=bpr)


def bench_protocol_kernels(out, K=48, n_rec=65536):
    """The protocol's small kernels in the sessions that launch them, over
    the 1,000-buffer training layout at 1/20 scale (2 GB arena), K kernel
    rounds of n_rec-record traces, quota image/40, 4 MB pieces: a
    device-decided CoW session (k_dr_* with 64 MB of staging), a no-sync
    recopy session on the ring validation variant (k_rule after each
    k_validate), and a verified restore of the CoW image (k_vzero and
    k_verify building the manifest, k_verify on every restored buffer).
    """
    from . import runner
    s = torch.cuda.current_stream().cuda_stream
    cfg = wl.training(scale=0.05, n_kernels=K)
    rng, lay = cfg["rng"], cfg["layout"]
    arena = torch.empty(lay.arena_bytes, dtype=torch.uint8, device="cuda")
    phos.harness_fill(arena.data_ptr(), lay.arena_bytes, cfg["seed"], s)
    kernels = wl.make_training_kernels(rng, lay, arena.data_ptr(), K, n_rec, 0.001)
    dp = runner.DeviceProcess(lay, arena, cfg["seed"], kernels)
    image = torch.empty(dp.image_bytes, dtype=torch.uint8).pin_memory()
    quota = -(-dp.image_bytes // 40 // 256) * 256
    stg = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    st = dp.run_cow(image, quota, 4 << 20, stg, stg.numel(), rounds="device")["stats"]
    out["cow_device_rounds"] = dict(rounds=K, cow_bytes=st["cow_bytes"],
                                    direct_bytes=st["direct_bytes"])
    phos.validate_config(1)
    try:
        st = dp.run_recopy(torch.empty_like(image).pin_memory(), quota, 4 << 20,
                           rounds="nosync")["stats"]
    finally:
        phos.validate_config(0)
    out["recopy_nosync_ring"] = dict(rounds=K, dirty=st["dirty"])
    man = torch.empty(8 * lay.n, dtype=torch.uint8, device="cuda")
    phos.image_manifest(dp.table, image.data_ptr(), image.numel(), man.data_ptr(), s)
    phos.harness_fill(arena.data_ptr(), lay.arena_bytes, 12345, s)
    r = dp.run_restore(image, quota, 4 << 20, rounds="concurrent", d_manifest=man)
    out["restore_verified"] = dict(rounds=r["kernels_during"],
                                   ondemand=len(r["ondemand"]), copier=len(r["copier"]))


def bench_image_manifest(out, scale=0.05, reps=10):
    """phos_image_manifest over a device-resident image of the 1,000-buffer
    training layout (2 GB at scale 0.05): k_vzero, then k_verify digesting
    every buffer (one HBM read of its bytes), CUDA events, L2 not flushed
    (the image is 16x L2)."""
    s = torch.cuda.current_stream().cuda_stream
    cfg = wl.training(scale=scale, n_kernels=1)
    lay = cfg["layout"]
    t = phos.Table(lay.base(VA0), lay.size)
    nb = t.image_bytes()
    img = torch.empty(nb, dtype=torch.uint8, device="cuda")
    phos.harness_fill(img.data_ptr(), nb, 7, s)
    man = torch.empty(8 * lay.n, dtype=torch.uint8, device="cuda")
    img_bytes = int(lay.size.astype(np.int64).sum())
    ms = timeit(lambda: phos.image_manifest(t, img.data_ptr(), nb, man.data_ptr(), s), reps,
                warm=3)
    out["image_manifest_device"] = dict(buffers=int(lay.n), bytes=img_bytes, ms=ms,
                                        gbs=img_bytes / ms / 1e6,
                                        launches_per_call=1 + (lay.n + 63) // 64)


def bench_copy_misaligned(gb, out):
    """Device -> device copies of G GB in 4 MB regions whose source is
    offset from the destination's alignment by 0, 1, 2, 4, 8 or 12 bytes."""
    s = torch.cuda.current_stream().cuda_stream
    G = int(gb) << 30
    nb = 64
    bs = G // nb
    live = torch.empty(G + 4096, dtype=torch.uint8, device="cuda")
    phos.harness_fill(live.data_ptr(), G + 4096, 5, s)
    tab = phos.Table([live.data_ptr() + i * bs for i in range(nb)], [bs] * nb)
    stg = torch.empty(G, dtype=torch.uint8, device="cuda")
    st = torch.zeros(4, dtype=torch.uint8, device="cuda")
    chunk = 4 << 20
    for delta in (0, 1, 2, 4, 8, 12):
        rows = []
        for i in range(nb):
            for o in range(0, bs - chunk, chunk):
                rows.append((o + delta, i * bs + o, chunk - 64, i, phos.COPY_LIVE_TO_STAGING))
        d = torch.from_numpy(np.array(rows, phos.COPY_DTYPE).view(np.uint8)).cuda()
        moved = sum(r[2] for r in rows)
        ms = timeit(lambda: phos.cow_copy(tab, d.data_ptr(), len(rows), stg.data_ptr(), G,
                                          st.data_ptr(), s), 5, 2)
        out["copy_d2d_src_offset_%d" % delta] = dict(gb=moved / 1e9, ms=ms,
                                                    gbs_rw=2 * moved / ms / 1e6)


def bench_copy(gb, out):
    s = torch.cuda.current_stream().cuda_stream
    G = int(gb) << 30
    live = torch.empty(G, dtype=torch.uint8, device="cuda")
    phos.harness_fill(live.data_ptr(), G, 5, s)
    nb = 64
    bs = G // nb
    tab = phos.Table([live.data_ptr() + i * bs for i in range(nb)], [bs] * nb)
    stg = torch.empty(G, dtype=torch.uint8, device="cuda")
    img = torch.empty(G, dtype=torch.uint8).pin_memory()
    st = torch.zeros(4, dtype=torch.uint8, device="cuda")

    def mk(kind, chunk=4 << 20):
        rows = []
        for i in range(nb):
            for o in range(0, bs, chunk):
                rows.append((o, i * bs + o, chunk, i, kind) if kind != 4 else
                            (i * bs + o, o, chunk, i, kind))
        a = np.array(rows, phos.COPY_DTYPE)
        return torch.from_numpy(a.view(np.uint8)).cuda(), len(rows)

    d1, n1 = mk(phos.COPY_LIVE_TO_STAGING)
    d2, n2 = mk(phos.COPY_LIVE_TO_IMAGE)
    d4, n4 = mk(phos.COPY_IMAGE_TO_LIVE)
    ms = timeit(lambda: phos.cow_copy(tab, d1.data_ptr(), n1, stg.data_ptr(), G, st.data_ptr(), s),
                5, 2)
    out["copy_d2d"] = dict(gb=gb, ms=ms, gbs_rw=2 * G / ms / 1e6)
    ms = timeit(lambda: phos.recopy(tab, d2.data_ptr(), n2, img.data_ptr(), G, st.data_ptr(), s),
                3, 1)
    out["copy_d2h"] = dict(gb=gb, ms=ms, gbs=G / ms / 1e6)
    ms = timeit(lambda: phos.restore_on_demand(tab, d4.data_ptr(), n4, img.data_ptr(), G, None,
                                               st.data_ptr(), s), 3, 1)
    out["copy_h2d"] = dict(gb=gb, ms=ms, gbs=G / ms / 1e6)
    ms = timeit(lambda: stg.copy_(live, non_blocking=True), 5, 2)
    out["dma_d2d"] = dict(gbs_rw=2 * G / ms / 1e6)
    ms = timeit(lambda: img.copy_(live, non_blocking=True), 3, 1)
    out["dma_d2h"] = dict(gbs=G / ms / 1e6)
    ms = timeit(lambda: live.copy_(img, non_blocking=True), 3, 1)
    out["dma_h2d"] = dict(gbs=G / ms / 1e6)
    # two DMA streams, and DMA + copy engine at once, device -> host
    h2 = torch.empty(G // 2, dtype=torch.uint8).pin_memory()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    half = G // 2
    cur = torch.cuda.current_stream()

    def two_dma():
        s1.wait_stream(cur)
        s2.wait_stream(cur)
        with torch.cuda.stream(s1):
            img[:half].copy_(live[:half], non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(live[half:], non_blocking=True)
        cur.wait_stream(s1)
        cur.wait_stream(s2)
    ms = timeit(two_dma, 3, 1)
    out["dma_d2h_two_streams"] = dict(gbs=G / ms / 1e6)

    def dma_and_engine():
        s1.wait_stream(cur)
        with torch.cuda.stream(s1):
            h2.copy_(live[half:], non_blocking=True)
        phos.recopy(tab, d2.data_ptr(), n2 // 2, img.data_ptr(), G, st.data_ptr(), s)
        cur.wait_stream(s1)
    ms = timeit(dma_and_engine, 3, 1)
    out["dma_and_engine_d2h"] = dict(gbs=G / ms / 1e6)


def bench_speculate(out, n_launch=20000):
    """Device speculation of a queue of launches over the 1,000-buffer
    training table, against the host call per launch."""
    import time
    s = torch.cuda.current_stream().cuda_stream
    cfg = wl.training(n_kernels=1)
    lay, rng = cfg["layout"], cfg["rng"]
    t = phos.Table(lay.base(VA0), lay.size)
    launches = [wl.make_args(rng, lay, VA0, *wl.pick_sets(rng, lay.n)) for _ in range(n_launch)]
    words, wk, off = phos.flatten_launch_args(launches)
    d_w = torch.from_numpy(words.view(np.uint8).copy()).cuda()
    d_k = torch.from_numpy(wk.copy()).cuda()
    d_o = torch.from_numpy(off.view(np.uint8).copy()).cuda()
    d_p = torch.zeros(n_launch * lay.n, dtype=torch.uint8, device="cuda")
    ms = timeit(lambda: phos.speculate_device(t, d_w.data_ptr(), d_k.data_ptr(), d_o.data_ptr(),
                                              n_launch, d_p.data_ptr(), None, s))
    perm = np.zeros(lay.n, np.uint8)
    t0 = time.perf_counter()
    for args, kinds in launches[:2000]:
        perm[:] = 0
        phos.speculate(t, args, kinds, perm)
    host_us = 1e6 * (time.perf_counter() - t0) / 2000
    out["speculate_device"] = dict(launches=n_launch, words=len(words), ms=ms,
                                   launches_per_s=n_launch / ms * 1e3,
                                   host_us_per_launch=host_us)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", default="all",
                    choices=["validate", "validate_distinct", "emit", "copy", "copy_misaligned",
                             "validate_rounds", "validate_rounds_launch", "protocol_kernels",
                             "image_manifest", "speculate", "all"])
    ap.add_argument("--traces", type=int, default=160)
    ap.add_argument("--rounds-nrec", type=int, default=65536,
                    help="validate_rounds: records per kernel round's trace")
    ap.add_argument("--copy-gb", type=int, default=8)
    ap.add_argument("--variant", type=int, default=0, help="validate kernel variant (0 = both)")
    a = ap.parse_args()
    out = {}
    if a.kernel in ("validate", "all"):
        bench_validate(a.traces, out, (1, 2) if a.variant == 0 else (a.variant,))
    if a.kernel == "validate_distinct":
        bench_validate_distinct(a.traces, out)
    if a.kernel == "emit":
        bench_emit(a.traces, out)
    if a.kernel == "copy_misaligned":
        bench_copy_misaligned(a.copy_gb, out)
    if a.kernel == "validate_rounds":
        bench_validate_rounds(out, n_rec=a.rounds_nrec)
    if a.kernel == "validate_rounds_launch":
        bench_validate_rounds_launch(out)
    if a.kernel == "protocol_kernels":
        bench_protocol_kernels(out)
    if a.kernel == "image_manifest":
        bench_image_manifest(out)
    if a.kernel in ("copy", "all"):
        bench_copy(a.copy_gb, out)
    if a.kernel in ("speculate", "all"):
        bench_speculate(out)
    print(json.dumps(out, indent=1))
    sys.stdout.flush()


if __name__ == "__main__":
    main()

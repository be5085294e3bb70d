"""The protocols at the benchmark's full sizes against the oracle in its
"versions" storage mode (the oracle describes bytes instead of holding
them, and regenerates them piece by piece to compare).

  * training-process image (Sec. 4.2 soft CoW, then Sec. 4.3 soft recopy
    on the memory the first checkpoint left): 1,000 buffers, 40 GB, 200
    kernels, 4 MB pieces, copier quota image/100 per round, 2 GB staging,
    DMA host legs for pieces >= 256 KiB, the copier on its own stream -- the
    benchmark's step -- with each kernel's validation at once and deferred
    (16 rounds per launch).  Traces are shortened to 16,384 records per kernel
    (only the strays, which are loads here, can change a decision, and the
    oracle's validation is a linear scan).
  * large on-demand restore (Sec. 6): 10,000 buffers, log-normal 4 KB -
    2 GB, at a fifth of 120 GB (what the box pins next to the test), 500
    replayed kernels with layer locality, quota image/500, 4 MB pieces,
    the copier on its own stream.

Compared exactly: CoW lists, copier pieces, dirty set, on-demand list,
fallback round, statistics, every buffer's image bytes and the whole
arena's bytes at the end.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import protocols as P  # noqa: E402
from oracle import versions as V  # noqa: E402
from paper_2405_12079_b300 import phos, runner, workloads as wl  # noqa: E402

PIECE = 64 << 20


def a256(x):
    return (int(x) + 255) // 256 * 256


def copier_rows(log):
    return [(int(r), int(i), int(o), int(ln), int(bool(sh))) for r, i, o, ln, sh in log]


def cow_rows(log):
    return [(int(k), int(i), 1 if kind == "S" else 2, int(o), int(ln))
            for k, i, kind, o, ln in log]


def image_mismatches(exp, img, lay, img_off):
    """Buffers whose image bytes differ from the oracle's (regenerated in
    64 MB pieces on the thread pool)."""
    def job(i, a, b):
        return i if not np.array_equal(exp.materialize(a, b), img[a:b]) else None
    fs = []
    for i in range(lay.n):
        o, s = int(img_off[i]), int(lay.size[i])
        for a in range(o, o + s, PIECE):
            fs.append(V.pool().submit(job, i, a, min(o + s, a + PIECE)))
    return sorted({f.result() for f in fs} - {None})


def arena_mismatches(mem, arena):
    """Offsets of 64 MB pieces of the device arena that differ from the
    oracle's live memory."""
    n = arena.numel()
    host = torch.empty(min(n, 1 << 30), dtype=torch.uint8).pin_memory()
    hv = host.numpy()
    bad = []
    for a in range(0, n, host.numel()):
        b = min(n, a + host.numel())
        host[:b - a].copy_(arena[a:b])
        fs = [V.pool().submit(lambda p, q: (p, np.array_equal(mem.materialize(p, q),
                                                               hv[p - a:q - a])), p,
                              min(b, p + PIECE)) for p in range(a, b, PIECE)]
        bad += [p for p, ok in (f.result() for f in fs) if not ok]
    return bad


@pytest.fixture
def dma_host_legs():
    phos.host_copy_config(256 << 10)
    yield
    phos.host_copy_config(phos.HOST_COPY_DEFAULT)


@pytest.mark.parametrize("rounds", ["concurrent", "deferred"])
def test_training_image_full_size(dma_host_legs, rounds):
    s = torch.cuda.current_stream().cuda_stream
    cfg = wl.training(scale=1.0, n_kernels=200)
    rng, lay = cfg["rng"], cfg["layout"]
    seed = cfg["seed"]
    arena = torch.empty(lay.arena_bytes, dtype=torch.uint8, device="cuda")
    phos.harness_fill(arena.data_ptr(), lay.arena_bytes, seed, s)
    va0 = arena.data_ptr()
    kernels = wl.make_training_kernels(rng, lay, va0, 200, 16384, 0.001)
    dp = runner.DeviceProcess(lay, arena, seed, kernels)
    image = torch.empty(dp.image_bytes, dtype=torch.uint8).pin_memory()
    staging_bytes = a256(2e9)
    staging = torch.empty(staging_bytes, dtype=torch.uint8, device="cuda")
    quota, chunk = a256(dp.image_bytes / 100), 4 << 20
    proc = V.VersionProcess(va0, lay.off, lay.size, seed, seed, arena_bytes=lay.arena_bytes)
    assert dp.image_bytes == proc.image_bytes and dp.image_bytes > 39e9

    # soft copy-on-write from t1 = now
    t0 = time.time()
    exp = P.cow_checkpoint(proc, kernels, staging_bytes, chunk, quota)
    t_orc = time.time() - t0
    got = dp.run_cow(image, quota, chunk, staging, staging_bytes, rounds=rounds)
    torch.cuda.synchronize()
    assert exp.misspec is None and got["stats"]["misspec_round"] == -1
    assert got["kernels_run"] == exp.kernels_run
    assert [tuple(int(x) for x in r) for r in got["cow"]] == cow_rows(exp.cow_log)
    assert [tuple(int(x) for x in r) for r in got["copier"]] == copier_rows(exp.copier_log)
    for key in ("cow_bytes", "direct_bytes", "copier_bytes"):
        assert got["stats"][key] == exp.stats[key]
    assert len(exp.cow_log) > 0
    assert image_mismatches(exp.image, image.numpy(), lay, dp.img_off) == []
    assert arena_mismatches(proc.mem, arena) == []

    # soft recopy on the memory the CoW checkpoint left
    exp2 = P.recopy_checkpoint(proc, kernels, chunk, quota)
    got2 = dp.run_recopy(image, quota, chunk, rounds=rounds)
    torch.cuda.synchronize()
    assert got2["kernels_run"] == exp2.kernels_run
    assert got2["dirty"].tolist() == exp2.dirty and len(exp2.dirty) > 0
    assert [tuple(int(x) for x in r) for r in got2["copier"]] == copier_rows(exp2.copier_log)
    for key in ("copier_bytes", "recopy_bytes"):
        assert got2["stats"][key] == exp2.stats[key]
    assert image_mismatches(exp2.image, image.numpy(), lay, dp.img_off) == []
    assert arena_mismatches(proc.mem, arena) == []
    print("training 40 GB (%s): oracle CoW run %.1f s, %d CoW copies, %d copier pieces, "
          "%d dirty" % (rounds, t_orc, len(exp.cow_log), len(exp.copier_log), len(exp2.dirty)))


def test_large_restore_full_buffer_count(dma_host_legs):
    s = torch.cuda.current_stream().cuda_stream
    cfg = wl.large_restore(scale=0.2, n_kernels=500, n_rec=1024)
    rng, lay = cfg["rng"], cfg["layout"]
    seed = cfg["seed"]
    assert lay.n == 10000
    arena = torch.empty(lay.arena_bytes, dtype=torch.uint8, device="cuda")
    phos.harness_fill(arena.data_ptr(), lay.arena_bytes, 5, s)
    va0 = arena.data_ptr()
    kernels = wl.make_restore_kernels(rng, lay, va0, 500, cfg["n_rec"])
    dp = runner.DeviceProcess(lay, arena, seed, kernels)
    # the checkpoint: every buffer of the filled arena to the pinned image
    image = torch.empty(dp.image_bytes, dtype=torch.uint8).pin_memory()
    rows = np.zeros(lay.n, phos.COPY_DTYPE)
    for i in range(lay.n):
        rows[i] = (0, int(dp.img_off[i]), int(lay.size[i]), i, phos.COPY_LIVE_TO_IMAGE)
    d_rows = torch.from_numpy(rows.view(np.uint8).copy()).cuda()
    phos.recopy(dp.table, d_rows.data_ptr(), lay.n, image.data_ptr(), image.numel(), None, s)
    torch.cuda.synchronize()
    ref = V.VersionProcess(va0, lay.off, lay.size, 5, seed, arena_bytes=lay.arena_bytes)
    img_v = P.stw_checkpoint(ref)
    assert image_mismatches(img_v, image.numpy(), lay, dp.img_off) == []
    # the restored process starts from memory that is not the checkpoint
    phos.harness_fill(arena.data_ptr(), lay.arena_bytes, 9, s)
    torch.cuda.synchronize()
    cur = V.VersionProcess(va0, lay.off, lay.size, 9, seed, arena_bytes=lay.arena_bytes)
    quota, chunk = a256(dp.image_bytes / 500), 4 << 20
    exp = P.concurrent_restore(cur, img_v, kernels, chunk, quota, copier_stream=True)
    got = dp.run_restore(image, quota, chunk, rounds="concurrent")
    torch.cuda.synchronize()
    assert exp.misspec is None and got["stats"]["misspec_round"] == -1
    assert got["kernels_during"] == exp.kernels_during
    assert [tuple(int(x) for x in r) for r in got["ondemand"]] == \
        [(int(k), int(i), int(o), int(ln), 0) for k, i, o, ln in exp.ondemand]
    assert [tuple(int(x) for x in r) for r in got["copier"]] == copier_rows(exp.copier_log)
    assert got["stats"]["ondemand_bytes"] == exp.stats["ondemand_bytes"]
    assert got["stats"]["copier_bytes"] == exp.stats["copier_bytes"]
    assert len(exp.ondemand) > 0
    assert arena_mismatches(cur.mem, arena) == []

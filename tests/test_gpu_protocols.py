"""GPU parity of the lockstep protocol drivers against the oracle: soft
copy-on-write (Sec. 4.2), soft recopy (Sec. 4.3) and soft on-demand restore
(Sec. 6) produce exactly the oracle's CoW lists, copier pieces, dirty sets,
on-demand lists, fallback rounds, checkpoint image and final memory, on
scaled training-process, tiny and large-restore workloads and on
mis-speculation scenarios."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import protocols as P  # noqa: E402
from paper_2405_12079_b300 import phos, runner, workloads as wl  # noqa: E402


@pytest.fixture(autouse=True, params=[0, 16384], ids=["sm-copies", "dma-host-legs"])
def host_legs(request):
    """Every protocol case runs with the host legs on the SM copy kernel and
    with pieces of >= 16 KiB on the DMA engines; results must not change."""
    phos.host_copy_config(request.param)
    yield request.param
    phos.host_copy_config(phos.HOST_COPY_DEFAULT)


def a256(x):
    return (int(x) + 255) // 256 * 256


class World:
    def __init__(self, layout, seed, make_kernels):
        self.lay = layout
        rng = np.random.default_rng(seed)
        self.mem0 = np.zeros(layout.arena_bytes, np.uint8)
        wl.fill_random(rng, self.mem0)
        self.arena = torch.from_numpy(self.mem0.copy()).cuda()
        self.va0 = self.arena.data_ptr()
        self.kernels = make_kernels(rng, layout, self.va0)
        self.seed = seed
        self.dp = runner.DeviceProcess(layout, self.arena, seed, self.kernels)

    def oracle_proc(self, mem=None):
        m = self.mem0.copy() if mem is None else mem
        return P.Process(self.va0, self.lay.off, self.lay.size, m, self.seed)

    def live_equal(self, proc):
        return np.array_equal(self.arena.cpu().numpy(), proc.mem)


def cow_rows(log):
    return [(int(k), int(i), 1 if kind == "S" else 2, int(o), int(ln))
            for k, i, kind, o, ln in log]


def copier_rows(log):
    return [(int(r), int(i), int(o), int(ln), int(bool(sh))) for r, i, o, ln, sh in log]


def training_world(seed, scale, n_kernels, stray_store_frac=0.0):
    cfg = wl.training(scale=scale, seed=seed, n_kernels=n_kernels)

    def mk(rng, lay, va0):
        return wl.make_training_kernels(rng, lay, va0, n_kernels, cfg["n_rec"], 0.001,
                                        stray_store_frac)
    return World(cfg["layout"], seed, mk), cfg


def check_ckpt(w, mode, quota, chunk, staging_bytes=0, rounds="sync"):
    img = torch.zeros(w.dp.image_bytes, dtype=torch.uint8).pin_memory()
    stg = torch.zeros(max(staging_bytes, 256), dtype=torch.uint8, device="cuda")
    proc = w.oracle_proc()
    if mode == "cow":
        exp = P.cow_checkpoint(proc, w.kernels, staging_bytes, chunk, quota)
        got = w.dp.run_cow(img, quota, chunk, stg, staging_bytes, rounds=rounds)
        assert got["stats"]["misspec_round"] == (-1 if exp.misspec is None else exp.misspec)
        assert [tuple(int(x) for x in r) for r in got["cow"]] == cow_rows(exp.cow_log)
        assert got["stats"]["cow_bytes"] == exp.stats["cow_bytes"]
        assert got["stats"]["direct_bytes"] == exp.stats["direct_bytes"]
    else:
        exp = P.recopy_checkpoint(proc, w.kernels, chunk, quota)
        got = w.dp.run_recopy(img, quota, chunk, rounds=rounds)
        assert got["dirty"].tolist() == exp.dirty
        assert got["stats"]["recopy_bytes"] == exp.stats["recopy_bytes"]
    torch.cuda.synchronize()
    if rounds == "device" and exp.misspec is None:
        # the host never learns when the device's copier finished, so every
        # kernel of the sequence ran; those after the end do not touch the
        # image (every buffer was done)
        assert got["kernels_run"] == len(w.kernels) >= exp.kernels_run
        for k in range(exp.kernels_run, got["kernels_run"]):
            proc.run_kernel(k, w.kernels[k])
    else:
        assert got["kernels_run"] == exp.kernels_run
    assert [tuple(int(x) for x in r) for r in got["copier"]] == copier_rows(exp.copier_log)
    assert np.array_equal(img.numpy(), exp.image)
    assert w.live_equal(proc)
    return got, exp


@pytest.mark.parametrize("rounds", ["sync", "nosync", "concurrent", "deferred", "device"])
@pytest.mark.parametrize("mode", ["cow", "recopy"])
def test_training_image_scaled(mode, rounds):
    """Training-process shape at 1/500 scale (1,000 buffers, ~80 MB,
    200 kernels); quota = image/100, chunk 64 KiB, staging 4 MB.  The
    no-sync rounds (rule on the device, no wait per kernel), the
    concurrent copier (its own stream, event ordering) and deferred
    validation (up to 16 rounds per launch) give exactly the lockstep
    results."""
    if mode == "recopy" and rounds == "device":
        pytest.skip("device-decided rounds are for CoW and restore sessions")
    w, cfg = training_world(wl.SEED0 + 2, 0.002, 200)
    quota = a256(w.dp.image_bytes / 100)
    got, exp = check_ckpt(w, mode, quota, 64 * 1024, staging_bytes=4 << 20, rounds=rounds)
    if mode == "cow":
        assert len(exp.cow_log) > 0 and exp.misspec is None
    else:
        assert len(exp.dirty) > 0


@pytest.mark.parametrize("mode", ["cow", "recopy"])
def test_stray_stores_fault_injection(mode):
    """1 % of strays are stores outside the speculation: CoW falls back to
    stop-the-world, recopy adds the victims to the dirty set."""
    w, cfg = training_world(wl.SEED0 + 12, 0.001, 80, stray_store_frac=0.3)
    quota = a256(w.dp.image_bytes / 60)
    got, exp = check_ckpt(w, mode, quota, 32 * 1024, staging_bytes=1 << 20)
    if mode == "cow":
        assert exp.misspec is not None


@pytest.mark.parametrize("rounds", ["nosync", "concurrent", "deferred"])
def test_stray_stores_recopy_nosync(rounds):
    """Recopy without a wait per kernel: the store victims reach the dirty
    set through the device-side rule; everything equals the oracle."""
    w, cfg = training_world(wl.SEED0 + 12, 0.001, 80, stray_store_frac=0.3)
    quota = a256(w.dp.image_bytes / 60)
    got, exp = check_ckpt(w, "recopy", quota, 32 * 1024, rounds=rounds)
    assert got["stats"]["violations"] > 0


@pytest.mark.parametrize("rounds", ["nosync", "concurrent", "deferred", "device"])
def test_stray_stores_cow_nosync_falls_back_at_finish(rounds):
    """CoW without a wait per kernel on the mis-speculating workload: the
    device records the same first mis-speculated round as the oracle; the
    host learns of it later, so more kernels run before the stop-the-world
    copy, and the image equals live memory at finish, which equals the
    oracle's memory after that many kernels."""
    w, cfg = training_world(wl.SEED0 + 12, 0.001, 80, stray_store_frac=0.3)
    quota = a256(w.dp.image_bytes / 60)
    chunk = 32 * 1024
    img = torch.zeros(w.dp.image_bytes, dtype=torch.uint8).pin_memory()
    stg = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    exp = P.cow_checkpoint(w.oracle_proc(), w.kernels, 1 << 20, chunk, quota)
    assert exp.misspec is not None
    got = w.dp.run_cow(img, quota, chunk, stg, 1 << 20, rounds=rounds)
    torch.cuda.synchronize()
    assert got["stats"]["misspec_round"] == exp.misspec
    k_run = got["kernels_run"]
    assert k_run >= exp.kernels_run
    proc = w.oracle_proc()
    for k in range(k_run):
        proc.run_kernel(k, w.kernels[k])
    assert w.live_equal(proc)
    assert np.array_equal(img.numpy(), P.stw_checkpoint(proc))


def test_cow_budget_zero_and_tiny_config():
    """Tiny config: 64 buffers, write set of 16, 1M-record random trace
    with 3 % other-buffer accesses (stores among them force the fallback);
    and a zero staging budget (every CoW goes straight to the image)."""
    cfg = wl.tiny()
    lay = cfg["layout"]
    wset = cfg["wset"]

    def mk(rng, lay_, va0):
        rec, cls = wl.trace_random(rng, lay_, va0, wset, cfg["n_rec"])
        args, kinds = wl.make_args(rng, lay_, va0, wset, wset)
        return [wl.Kernel(args, kinds, wset, wset, rec, cls, 4, [])]
    w = World(lay, cfg["seed"], mk)
    check_ckpt(w, "cow", a256(w.dp.image_bytes / 4), 1 << 16, staging_bytes=64 << 20)

    def mk2(rng, lay_, va0):
        ks = []
        for _ in range(12):
            r, wr = wl.pick_sets(rng, lay_.n, 1, 8)
            args, kinds = wl.make_args(rng, lay_, va0, r, wr)
            rec, cls, st = wl.trace_runs(rng, lay_, va0, r, wr, 4096, 0.0)
            ks.append(wl.Kernel(args, kinds, r, wr, rec, cls, 4, st))
        return ks
    w2 = World(lay, cfg["seed"] + 100, mk2)
    got, exp = check_ckpt(w2, "cow", a256(w2.dp.image_bytes / 20), 1 << 16, staging_bytes=0)
    assert all(e[2] == "D" for e in exp.cow_log)


def check_restore(w, quota, chunk, rounds="sync"):
    """rounds: sync / nosync / concurrent.  Without a mis-speculation every
    mode gives the oracle's lists exactly (concurrent: the oracle's copier
    on its own stream).  With one, the device records the oracle's round;
    without a wait per kernel the host rolls back later, so only the round,
    the final memory and the present bits are compared."""
    proc = w.oracle_proc()
    image = P.stw_checkpoint(proc)
    img = torch.from_numpy(image.copy()).pin_memory()
    # the restored process starts from memory that is not the checkpoint
    w.arena.fill_(0xA5)
    cur = w.oracle_proc(np.full(w.lay.arena_bytes, 0xA5, np.uint8))
    exp = P.concurrent_restore(cur, image, w.kernels, chunk, quota,
                               copier_stream=rounds in ("concurrent", "deferred", "odfirst"),
                               ondemand_first=rounds == "odfirst")
    present = torch.zeros(4 * ((w.lay.n + 31) // 32), dtype=torch.uint8, device="cuda")
    got = w.dp.run_restore(img, quota, chunk, present, rounds=rounds)
    torch.cuda.synchronize()
    assert got["stats"]["misspec_round"] == (-1 if exp.misspec is None else exp.misspec)
    if exp.misspec is None or rounds == "sync":
        # device-decided rounds: the host never learns when the copier is
        # done, so every kernel runs inside the session
        assert got["kernels_during"] == (len(w.kernels) if rounds == "device"
                                         else exp.kernels_during)
        assert [tuple(int(x) for x in r) for r in got["ondemand"]] == \
            [(int(k), int(i), int(o), int(ln), 0) for k, i, o, ln in exp.ondemand]
        assert [tuple(int(x) for x in r) for r in got["copier"]] == \
            copier_rows(exp.copier_log)
    assert w.live_equal(cur)
    bits = present.cpu().numpy().view(np.uint32)
    assert int(sum(bin(int(x)).count("1") for x in bits)) == w.lay.n
    return got, exp


@pytest.mark.parametrize("rounds", ["sync", "nosync", "concurrent", "concurrent-window",
                                    "deferred", "odfirst", "odfirst-window", "device"])
def test_large_restore_scaled(rounds):
    """Large-restore shape at small scale: 10,000 buffers, layer-local
    read/write sets, background bulk restore plus on-demand copies.  With a
    copier window the host holds back the copier's next pieces until few
    are in flight; the decisions, and so the results, do not change."""
    cfg = wl.large_restore(scale=0.0005, n_kernels=150, n_rec=1024)

    def mk(rng, lay, va0):
        return wl.make_restore_kernels(rng, lay, va0, cfg["n_kernels"], cfg["n_rec"])
    w = World(cfg["layout"], cfg["seed"], mk)
    quota = a256(w.dp.image_bytes / 300)
    if rounds.endswith("-window"):
        phos.copier_window(2 * quota)
    try:
        got, exp = check_restore(w, quota, 64 * 1024, rounds.split("-")[0])
    finally:
        phos.copier_window(0)
    assert len(exp.ondemand) > 0


@pytest.mark.parametrize("rounds", ["sync", "nosync", "concurrent", "deferred", "odfirst",
                                    "device"])
def test_restore_stray_load_rolls_back(rounds):
    cfg = wl.training(scale=0.0005, seed=wl.SEED0 + 22, n_kernels=40)

    def mk(rng, lay, va0):
        return wl.make_training_kernels(rng, lay, va0, 40, cfg["n_rec"], stray_frac=0.002)
    w = World(cfg["layout"], cfg["seed"], mk)
    got, exp = check_restore(w, a256(w.dp.image_bytes / 80), 32 * 1024, rounds)
    assert exp.misspec is not None


@pytest.mark.parametrize("div,n_kernels,stray,max_passes,stop", [
    (100, 200, 0.0, 6, 0), (30, 200, 0.0, 6, 0), (30, 200, 0.0, 1, 0),
    (20, 120, 0.3, 6, 1 << 20)])
@pytest.mark.parametrize("rounds", ["sync", "nosync", "concurrent", "deferred"])
def test_iterative_recopy(div, n_kernels, stray, max_passes, stop, rounds):
    """Iterative concurrent recopy (Sec. 4.3): the passes (round, buffers,
    bytes), the copier pieces across passes, the final dirty set, the image
    at t2 and live memory all equal the oracle's; the stop-the-world recopy
    shrinks against the single-pass protocol on the same workload."""
    w, cfg = training_world(wl.SEED0 + 2, 0.002 if n_kernels == 200 else 0.001, n_kernels,
                            stray_store_frac=stray)
    quota = a256(w.dp.image_bytes / div)
    chunk = 64 * 1024
    img = torch.zeros(w.dp.image_bytes, dtype=torch.uint8).pin_memory()
    proc = w.oracle_proc()
    exp = P.iterative_recopy(proc, w.kernels, chunk, quota, max_passes, stop)
    got = w.dp.run_recopy(img, quota, chunk, max_passes=max_passes, stop_bytes=stop,
                          rounds=rounds)
    torch.cuda.synchronize()
    assert len(exp.passes) >= 1
    assert [(int(r), int(nb), int(b)) for r, nb, b, _, _ in got["passes"]] == \
        [(k, len(bs), b) for k, bs, b in exp.passes]
    assert got["stats"]["passes"] == len(exp.passes)
    assert got["kernels_run"] == exp.kernels_run
    assert [tuple(int(x) for x in r) for r in got["copier"]] == copier_rows(exp.copier_log)
    assert got["dirty"].tolist() == exp.dirty
    assert got["stats"]["recopy_bytes"] == exp.stats["recopy_bytes"]
    assert got["stats"]["copier_bytes"] == exp.stats["copier_bytes"]
    assert np.array_equal(img.numpy(), exp.image)
    assert w.live_equal(proc)


@pytest.mark.parametrize("rounds", ["sync", "concurrent", "deferred"])
@pytest.mark.parametrize("mode", ["cow", "recopy"])
def test_native_driver_equals_oracle(mode, rounds):
    """The library's native round driver gives the oracle's results too."""
    w, cfg = training_world(wl.SEED0 + 2, 0.002, 200)
    quota = a256(w.dp.image_bytes / 100)
    chunk = 64 * 1024
    img = torch.zeros(w.dp.image_bytes, dtype=torch.uint8).pin_memory()
    stg = torch.zeros(4 << 20, dtype=torch.uint8, device="cuda")
    proc = w.oracle_proc()
    if mode == "cow":
        exp = P.cow_checkpoint(proc, w.kernels, 4 << 20, chunk, quota)
        got = w.dp.run_native(phos.CKPT_COW, img, quota, chunk, stg, 4 << 20, rounds)
        assert [tuple(int(x) for x in r) for r in got["cow"]] == cow_rows(exp.cow_log)
    else:
        exp = P.recopy_checkpoint(proc, w.kernels, chunk, quota)
        got = w.dp.run_native(phos.CKPT_RECOPY, img, quota, chunk, rounds=rounds)
        assert got["dirty"].tolist() == exp.dirty
    torch.cuda.synchronize()
    assert got["kernels_run"] == exp.kernels_run
    assert [tuple(int(x) for x in r) for r in got["copier"]] == copier_rows(exp.copier_log)
    assert np.array_equal(img.numpy(), exp.image)
    assert w.live_equal(proc)


@pytest.mark.parametrize("mode", ["cow", "recopy"])
def test_deferred_long_traces(mode):
    """Deferred validation of kernel rounds with long, ragged traces
    (300K-600K records: the launch takes 32-word batches and prefetches)
    inside recopy (stray stores: dirty marks by the device rule) and CoW
    sessions: dirty set or CoW list, copier pieces, image and live memory
    equal the oracle's."""
    cfg = wl.training(scale=0.002, seed=wl.SEED0 + 50, n_kernels=24)

    def mk(rng, lay, va0):
        ks = []
        for _ in range(24):
            ks += wl.make_training_kernels(rng, lay, va0, 1, int(rng.integers(300_000, 600_000)),
                                           0.001, 0.3 if mode == "recopy" else 0.0)
        return ks
    w = World(cfg["layout"], cfg["seed"], mk)
    quota = a256(w.dp.image_bytes / 30)
    got, exp = check_ckpt(w, mode, quota, 64 * 1024, staging_bytes=4 << 20, rounds="deferred")
    assert exp.kernels_run == 24
    if mode == "recopy":
        assert got["stats"]["violations"] > 0 and len(exp.dirty) > 0


@pytest.mark.parametrize("budget", [0, 1 << 20], ids=["no-staging", "staging-1MiB"])
def test_device_rounds_cow_staging_pressure(budget):
    """Device-decided CoW rounds with little or no staging: the device's
    first-fit allocator and its direct copies to the image give exactly the
    oracle's CoW list, copier pieces and image."""
    w, cfg = training_world(wl.SEED0 + 40, 0.001, 120)
    quota = a256(w.dp.image_bytes / 60)
    got, exp = check_ckpt(w, "cow", quota, 32 * 1024, staging_bytes=budget, rounds="device")
    assert len(exp.cow_log) > 0
    if budget == 0:
        assert all(e[2] == "D" for e in exp.cow_log)
    else:
        assert {e[2] for e in exp.cow_log} == {"S", "D"}


def test_sessions_on_two_threads_and_streams():
    """Two processes checkpointed at once from two host threads, each on a
    stream of its own: a concurrent deferred recopy with stray stores and a
    concurrent CoW.  The library keeps no per-process state between them
    (each session owns its arenas and scratch, each table its copy scratch),
    so each result is the oracle's, as when it runs alone."""
    import threading
    wa, _ = training_world(wl.SEED0 + 41, 0.001, 80, stray_store_frac=0.3)
    wb, _ = training_world(wl.SEED0 + 42, 0.001, 80)
    chunk = 32 * 1024
    qa, qb = a256(wa.dp.image_bytes / 60), a256(wb.dp.image_bytes / 60)
    pa, pb = wa.oracle_proc(), wb.oracle_proc()
    exp_a = P.recopy_checkpoint(pa, wa.kernels, chunk, qa)
    exp_b = P.cow_checkpoint(pb, wb.kernels, 1 << 20, chunk, qb)
    img_a = torch.zeros(wa.dp.image_bytes, dtype=torch.uint8).pin_memory()
    img_b = torch.zeros(wb.dp.image_bytes, dtype=torch.uint8).pin_memory()
    stg_b = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    got, errors = {}, []

    def run(name, fn):
        try:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                got[name] = fn()
                st.synchronize()
        except Exception as e:           # reported below, in the test's thread
            errors.append((name, e))
    ts = [threading.Thread(target=run, args=("a", lambda: wa.dp.run_recopy(
              img_a, qa, chunk, rounds="deferred"))),
          threading.Thread(target=run, args=("b", lambda: wb.dp.run_cow(
              img_b, qb, chunk, stg_b, 1 << 20, rounds="concurrent")))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
    torch.cuda.synchronize()
    ga, gb = got["a"], got["b"]
    assert ga["dirty"].tolist() == exp_a.dirty and ga["stats"]["violations"] > 0
    assert ga["stats"]["recopy_bytes"] == exp_a.stats["recopy_bytes"]
    assert [tuple(int(x) for x in r) for r in ga["copier"]] == copier_rows(exp_a.copier_log)
    assert np.array_equal(img_a.numpy(), exp_a.image)
    assert wa.live_equal(pa)
    assert gb["stats"]["misspec_round"] == -1 and exp_b.misspec is None
    assert [tuple(int(x) for x in r) for r in gb["cow"]] == cow_rows(exp_b.cow_log)
    assert [tuple(int(x) for x in r) for r in gb["copier"]] == copier_rows(exp_b.copier_log)
    assert np.array_equal(img_b.numpy(), exp_b.image)
    assert wb.live_equal(pb)


@pytest.mark.parametrize("mode", ["cow", "recopy"])
def test_deferred_rounds_with_ragged_traces(mode):
    """Deferred validation over rounds whose traces end anywhere: empty, one
    record, inside the first batch, on and around batch and word
    boundaries, and the full length; with stray stores (kept only where the
    trace still holds them, so every write is validated).  The lists, dirty
    set, image and memory equal the oracle's, as in the other modes."""
    cfg = wl.training(scale=0.001, seed=wl.SEED0 + 43, n_kernels=60)
    cut_rng = np.random.default_rng(4343)
    cuts = [0, 1, 31, 32, 33, 255, 256, 257, 511, 1000, 4095]

    def mk(rng, lay, va0):
        ks = wl.make_training_kernels(rng, lay, va0, 60, cfg["n_rec"], 0.002,
                                      0.0 if mode == "cow" else 0.3)
        for k in ks:
            m = int(cut_rng.choice(cuts + [len(k.trace)]))
            k.trace = k.trace[:m]
            k.labels = k.labels[:m]
            k.strays = [s for s in k.strays if s[0] < m]
        return ks
    w = World(cfg["layout"], wl.SEED0 + 43, mk)
    quota = a256(w.dp.image_bytes / 50)
    check_ckpt(w, mode, quota, 32 * 1024, staging_bytes=1 << 20, rounds="deferred")


def test_restore_ondemand_first_rejects_misuse():
    """PHOS_RESTORE_ONDEMAND_FIRST needs the copier stream, and its advance
    comes once per round, after before_kernel."""
    cfg = wl.training(scale=0.0005, seed=wl.SEED0 + 23, n_kernels=4)

    def mk(rng, lay, va0):
        return wl.make_training_kernels(rng, lay, va0, 4, cfg["n_rec"])
    w = World(cfg["layout"], cfg["seed"], mk)
    img = torch.zeros(w.dp.image_bytes, dtype=torch.uint8).pin_memory()
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(phos.PhosError):
        phos.Restore(w.dp.table, img.data_ptr(), img.numel(), 4096, 4, None, s,
                     phos.RESTORE_ONDEMAND_FIRST)
    r = phos.Restore(w.dp.table, img.data_ptr(), img.numel(), 4096, 4, None, s,
                     phos.CKPT_CONCURRENT | phos.RESTORE_ONDEMAND_FIRST)
    with pytest.raises(phos.PhosError):
        r.advance(1 << 20)                       # not inside a round
    pk = w.dp.kernels[0]
    r.before_kernel(pk.speculate(w.dp.table, w.dp.perm))
    r.advance(1 << 20)
    with pytest.raises(phos.PhosError):
        r.advance(1 << 20)                       # twice in one round
    w.dp.run_kernel(0)
    r.after_kernel(pk.d_trace.data_ptr(), pk.n_rec)
    r.finish()
    r.close()

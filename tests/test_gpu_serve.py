"""The serving loop: every checkpoint and restore request gives the same
bytes alone (one at a time) and in the mix (continuous batching), and those
bytes are what the oracle's memcpy gives; admission waits for the staging
budget instead of failing."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import copyeng  # noqa: E402
from paper_2405_12079_b300 import phos, workloads as wl  # noqa: E402


def a256(x):
    return (int(x) + 255) // 256 * 256


class World:
    """Disjoint device and host regions, one per request."""

    def __init__(self, seed, n_req=24, packed=False, buffers=(1, 300), size_hi=(2_000, 60_000)):
        """packed: buffer sizes multiples of 256 with no gaps, so pieces of
        neighbouring buffers are contiguous on both sides and merge.
        buffers: range of buffer counts per request (log-uniform when the
        range spans more than a factor of 10); size_hi: range of each
        request's largest buffer size."""
        rng = np.random.default_rng(seed)
        self.rng = rng
        lays = []
        for q in range(n_req):
            lo, hi = buffers
            if hi > 10 * lo:
                nb = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
            else:
                nb = int(rng.integers(lo, hi))
            sizes = wl.sizes_uniform(rng, nb, 1, int(rng.integers(*size_hi)))
            if packed:
                sizes = (sizes + np.uint64(255)) // np.uint64(256) * np.uint64(256)
                lay = wl.make_layout(rng, sizes, gap_lo=0, gap_hi=0)
            else:
                lay = wl.make_layout(rng, sizes, gap_lo=0, gap_hi=2048)
            lays.append(lay)
        dev_b = sum(l.arena_bytes + 4096 for l in lays) + 4096
        host_b = sum(a256(int(sum(a256(x) for x in l.size))) + 4096 for l in lays) + 4096
        self.dev_h = rng.integers(0, 256, dev_b, dtype=np.uint8)
        self.host_h = rng.integers(0, 256, host_b, dtype=np.uint8)
        self.dev = torch.from_numpy(self.dev_h.copy()).cuda()
        self.host = torch.from_numpy(self.host_h.copy()).pin_memory()
        self.reqs = []
        doff = hoff = 0
        for q, lay in enumerate(lays):
            off = doff
            doff += lay.arena_bytes + 4096
            t = phos.Table(lay.base(self.dev.data_ptr() + off), lay.size)
            img = t.image_bytes()
            kind = phos.REQ_CHECKPOINT if q % 2 == 0 else phos.REQ_RESTORE
            self.reqs.append(dict(kind=kind, lay=lay, dev_off=off, table=t, host_off=hoff,
                                  img=img, img_off=t.image_offsets()))
            hoff += a256(img) + 4096
        assert doff <= self.dev_h.size and hoff <= self.host_h.size

    def reset(self):
        self.dev.copy_(torch.from_numpy(self.dev_h))
        self.host.copy_(torch.from_numpy(self.host_h))
        torch.cuda.synchronize()

    def expected(self, skip=()):
        dev, host = self.dev_h.copy(), self.host_h.copy()
        for q, r in enumerate(self.reqs):
            if q in skip:
                continue
            lay, n = r["lay"], r["lay"].n
            d = np.zeros(n, copyeng.DESC_DTYPE)
            for i in range(n):
                if r["kind"] == phos.REQ_CHECKPOINT:
                    d[i] = (0, r["host_off"] + int(r["img_off"][i]), int(lay.size[i]), i,
                            copyeng.LIVE_TO_IMAGE)
                else:
                    d[i] = (r["host_off"] + int(r["img_off"][i]), 0, int(lay.size[i]), i,
                            copyeng.IMAGE_TO_LIVE)
            assert copyeng.apply(d, dev, lay.off + np.uint64(r["dev_off"]), lay.size,
                                 image=host) == 0
        return dev, host

    def submit(self, srv, r):
        return srv.submit(r["kind"], r["table"], self.host.data_ptr() + r["host_off"],
                          a256(r["img"]))


@pytest.mark.parametrize("shape", ["small", "cfg4-buffers"])
@pytest.mark.parametrize("packed", [False, True], ids=["gaps", "packed"])
@pytest.mark.parametrize("dma_min", [0, 256 << 10], ids=["sm-copies", "dma"])
def test_alone_and_mix_give_the_same_bytes(dma_min, packed, shape):
    """shape cfg4-buffers: the serving workload's 100-10,000 buffers per
    request (log-uniform), at reduced bytes (buffers of at most 2-8 KB)."""
    if shape == "small":
        w = World(5, packed=packed)
    else:
        w = World(15, n_req=16, packed=packed, buffers=(100, 10_000), size_hi=(2_000, 8_000))
        assert max(r["lay"].n for r in w.reqs) > 2000
    exp_dev, exp_host = w.expected()
    cks = [a256(r["img"]) for r in w.reqs if r["kind"] == phos.REQ_CHECKPOINT]
    stg = max(max(cks), sum(cks) // 2)       # smaller than all checkpoints together
    staging = torch.empty(stg, dtype=torch.uint8, device="cuda")

    # alone: one request at a time
    w.reset()
    srv = phos.Server(1, staging.data_ptr(), staging.numel(), chunk=64 << 10, dma_min=dma_min)
    for r in w.reqs:
        tk = w.submit(srv, r)
        srv.drain(60_000)
        res = srv.poll(tk)
        assert res["state"] == 2 and res["status"] == 0
    srv.close()
    torch.cuda.synchronize()
    assert np.array_equal(w.dev.cpu().numpy(), exp_dev)
    assert np.array_equal(w.host.numpy(), exp_host)

    # mix: continuous batching, arrivals while others are in flight, a
    # staging budget smaller than the checkpoints' total
    w.reset()
    srv = phos.Server(8, staging.data_ptr(), staging.numel(), chunk=64 << 10, dma_min=dma_min)
    tks = []
    for r in w.reqs:
        tks.append(w.submit(srv, r))
        time.sleep(float(w.rng.exponential(0.0005)))
    srv.drain(60_000)
    res = [srv.poll(t) for t in tks]
    srv.close()
    torch.cuda.synchronize()
    assert all(x["state"] == 2 and x["status"] == 0 for x in res)
    assert all(x["t_done_ns"] >= x["t_admit_ns"] >= x["t_submit_ns"] for x in res)
    assert np.array_equal(w.dev.cpu().numpy(), exp_dev)
    assert np.array_equal(w.host.numpy(), exp_host)
    assert sum(cks) > staging.numel()    # admission had to wait for budget


def test_request_larger_than_budget_is_refused():
    w = World(6, n_req=2)
    staging = torch.empty(4096, dtype=torch.uint8, device="cuda")
    srv = phos.Server(4, staging.data_ptr(), staging.numel())
    with pytest.raises(phos.PhosError) as e:
        w.submit(srv, w.reqs[0])
    assert e.value.code == phos.PHOS_EBUDGET
    srv.close()


@pytest.mark.parametrize("priority", [False, True], ids=["counted", "priority"])
def test_app_transfers_in_the_mix(priority):
    """Application transfers (Sec. 5 prioritized application PCIe transfer)
    issued on their own stream while the mix runs: every request's bytes and
    every application transfer's bytes are exact either way; the server
    counts them, and with priority it held C/R issue back at least once."""
    w = World(7)
    exp_dev, exp_host = w.expected()
    cks = [a256(r["img"]) for r in w.reqs if r["kind"] == phos.REQ_CHECKPOINT]
    staging = torch.empty(sum(cks), dtype=torch.uint8, device="cuda")
    rng = np.random.default_rng(70)
    n_app, sz = 16, 1 << 20
    src_h = torch.from_numpy(rng.integers(0, 256, n_app * sz, dtype=np.uint8)).pin_memory()
    src_d = torch.from_numpy(rng.integers(0, 256, n_app * sz, dtype=np.uint8)).cuda()
    dst_d = torch.zeros(n_app * sz, dtype=torch.uint8, device="cuda")
    dst_h = torch.zeros(n_app * sz, dtype=torch.uint8).pin_memory()
    w.reset()
    srv = phos.Server(8, staging.data_ptr(), staging.numel(), chunk=64 << 10, dma_min=256 << 10,
                      app_priority=priority, window=1 << 20)
    app = torch.cuda.Stream()
    tks = []
    for q, r in enumerate(w.reqs):
        tks.append(w.submit(srv, r))
        if q < n_app:
            o = q * sz
            if q % 2 == 0:
                srv.app_copy(dst_d.data_ptr() + o, src_h.data_ptr() + o, sz, app.cuda_stream)
            else:
                srv.app_copy(dst_h.data_ptr() + o, src_d.data_ptr() + o, sz, app.cuda_stream)
    srv.drain(60_000)
    app.synchronize()
    st = srv.stats()
    res = [srv.poll(t) for t in tks]
    srv.close()
    torch.cuda.synchronize()
    assert all(x["state"] == 2 and x["status"] == 0 for x in res)
    assert np.array_equal(w.dev.cpu().numpy(), exp_dev)
    assert np.array_equal(w.host.numpy(), exp_host)
    ev, od = np.arange(0, n_app, 2), np.arange(1, n_app, 2)
    got_d = dst_d.cpu().numpy().reshape(n_app, sz)
    got_h = dst_h.numpy().reshape(n_app, sz)
    assert np.array_equal(got_d[ev], src_h.numpy().reshape(n_app, sz)[ev])
    assert np.array_equal(got_h[od], src_d.cpu().numpy().reshape(n_app, sz)[od])
    assert st["app_copies"] == n_app and st["app_bytes"] == n_app * sz
    assert st["batches"] > 0


@pytest.mark.parametrize("priority", [False, True], ids=["counted", "priority"])
@pytest.mark.parametrize("app_d2h", [True, False], ids=["app-d2h", "app-h2d"])
@pytest.mark.parametrize("kind", [phos.REQ_CHECKPOINT, phos.REQ_RESTORE], ids=["ckpt", "restore"])
def test_pending_app_transfer_holds_back_cr_issue(priority, app_d2h, kind):
    """An application transfer queued behind ~25 ms of work on its stream
    (a bounded clock-spin kernel) is pending that long: with priority, a
    request whose host leg runs in either direction cannot finish before
    it, and the scheduler counted the turns it held back; without priority
    nothing is held back by the scheduler (the copy engines may still queue
    the request's copies behind the pending one)."""
    w = World(8, n_req=2)
    r = w.reqs[0] if w.reqs[0]["kind"] == kind else w.reqs[1]
    assert r["kind"] == kind
    staging = torch.empty(a256(r["img"]) + 256, dtype=torch.uint8, device="cuda")
    src = torch.zeros(1 << 20, dtype=torch.uint8).pin_memory()
    dev = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    srv = phos.Server(4, staging.data_ptr(), staging.numel(), chunk=64 << 10, dma_min=256 << 10,
                      app_priority=priority, window=1 << 20)
    app = torch.cuda.Stream()
    with torch.cuda.stream(app):
        torch.cuda._sleep(50_000_000)           # >= 24.6 ms at 2032 MHz
    if app_d2h:
        srv.app_copy(src.data_ptr(), dev.data_ptr(), src.numel(), app.cuda_stream)
    else:
        srv.app_copy(dev.data_ptr(), src.data_ptr(), src.numel(), app.cuda_stream)
    tk = w.submit(srv, r)
    srv.drain(60_000)
    res = srv.poll(tk)
    st = srv.stats()
    app.synchronize()
    srv.close()
    assert res["state"] == 2 and res["status"] == 0
    took_ms = (res["t_done_ns"] - res["t_submit_ns"]) / 1e6
    if priority:
        assert took_ms > 15 and st["paused_turns"] > 0
    else:
        assert st["paused_turns"] == 0


def test_app_copy_rejects_pageable_and_same_side():
    staging = torch.empty(4096, dtype=torch.uint8, device="cuda")
    srv = phos.Server(1, staging.data_ptr(), staging.numel(), app_priority=True)
    pageable = np.zeros(4096, np.uint8)
    d1 = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    d2 = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    for dst, src in [(d1.data_ptr(), pageable.ctypes.data), (d1.data_ptr(), d2.data_ptr())]:
        with pytest.raises(phos.PhosError) as e:
            srv.app_copy(dst, src, 4096, s)
        assert e.value.code == phos.PHOS_EINVAL
    assert srv.stats()["app_copies"] == 0
    srv.close()


def test_cancelled_requests_leave_the_others_exact():
    """Cancellation (a failure the serving loop must survive): one admitted
    checkpoint, one admitted restore and one queued request are cancelled
    while a pending application transfer holds every host leg back, so none
    of their pieces has been issued.  They end as cancelled, their images
    and buffers are untouched, the staging of the cancelled checkpoint is
    released, and every other request's bytes are exactly the oracle's."""
    w = World(9, n_req=10)
    cks = [a256(r["img"]) for r in w.reqs if r["kind"] == phos.REQ_CHECKPOINT]
    staging = torch.empty(sum(cks), dtype=torch.uint8, device="cuda")
    src = torch.zeros(1 << 20, dtype=torch.uint8).pin_memory()
    dev = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    w.reset()
    srv = phos.Server(4, staging.data_ptr(), staging.numel(), chunk=64 << 10, dma_min=256 << 10,
                      app_priority=True, window=1 << 20)
    app = torch.cuda.Stream()
    t0 = time.perf_counter()
    with torch.cuda.stream(app):
        torch.cuda._sleep(1_000_000_000)        # >= 0.49 s at 2032 MHz
    srv.app_copy(dev.data_ptr(), src.data_ptr(), src.numel(), app.cuda_stream)
    tks = [w.submit(srv, r) for r in w.reqs]
    # requests 0 (checkpoint) and 1 (restore) are admitted, 9 is queued
    t_end = time.time() + 1.0
    while time.time() < t_end and not (srv.poll(tks[0])["state"] == 1 and
                                       srv.poll(tks[1])["state"] == 1):
        time.sleep(0.0005)
    states = [srv.poll(t)["state"] for t in tks]
    cancel = (0, 1, 9)
    for q in cancel:
        srv.cancel(tks[q])
    t_cancel = time.perf_counter() - t0
    held = srv.stats()["paused_turns"]
    assert states[9] == 0 and srv.poll(tks[9])["state"] == 4
    srv.drain(60_000)
    app.synchronize()
    res = [srv.poll(t) for t in tks]
    st = srv.stats()
    srv.close()
    torch.cuda.synchronize()
    assert states[0] == 1 and states[1] == 1
    for q, x in enumerate(res):
        assert x["state"] == (4 if q in cancel else 2) and x["status"] == 0
    assert st["cancelled"] == 3
    exp_dev, exp_host = w.expected(skip=cancel)
    dev, host = w.dev.cpu().numpy(), w.host.numpy()
    diff = [q for q, r in enumerate(w.reqs)
            if not np.array_equal(dev[r["dev_off"]:r["dev_off"] + r["lay"].arena_bytes],
                                  exp_dev[r["dev_off"]:r["dev_off"] + r["lay"].arena_bytes]) or
            not np.array_equal(host[r["host_off"]:r["host_off"] + r["img"]],
                               exp_host[r["host_off"]:r["host_off"] + r["img"]])]
    assert diff == [], (diff, states, t_cancel, held, st)
    assert np.array_equal(dev, exp_dev)
    assert np.array_equal(host, exp_host)
    with pytest.raises(phos.PhosError):
        srv2 = phos.Server(1, staging.data_ptr(), staging.numel())
        try:
            srv2.cancel(12345)
        finally:
            srv2.close()

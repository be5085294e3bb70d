"""Benchmark: one concurrent checkpoint step of a training-process image.

Workload (synthetic, seeded): a 40 GB training-process image of 1,000
buffers with log-normal sizes 256 B - 512 MB, and a sequence of 200
application kernels (each writes 1-20 random buffers and reads 1-20, with
a 1.3M-record warp-coalesced access trace of 32 x 4-byte runs, 0.1 %
stray loads).  One step is one soft copy-on-write checkpoint (Sec. 4.2,
2 GB device staging) followed by one soft recopy checkpoint (Sec. 4.3),
each taken in lockstep with the application: the background copier moves
image/100 bytes per round in 4 MB pieces into a pinned host image; before
each kernel its launch arguments are speculated, CoW copies or dirty
marking happen, the kernel runs, and its trace is validated.

Prints one JSON line.  ``value`` = bytes moved by the copy engine (CoW
copies, background copy, direct copies, recopy) per second of step time.
``--impl reference`` times the CPU oracle on a bounded sample instead.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "validated accesses/s and C/R copy GB/s vs HBM/PCIe peak; request p50/p99"
WORKLOAD = ("training-process image: 1,000 buffers, log-normal 256 B-512 MB, 40 GB; "
            "200-kernel mutator sequence writing 1-20 buffers each; 1.3M-record coalesced "
            "trace per kernel (0.1% stray); soft CoW then soft recopy, lockstep, "
            "quota image/100, 4 MB pieces, 2 GB staging, pinned host image")


def a256(x):
    return int(math.ceil(x / 256.0)) * 256


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ oracle

def oracle_sample(scale, n_kernels=200, seed=None):
    """The oracle's CoW + recopy checkpoint on a scaled copy of the
    workload; returns (bytes moved, records validated, seconds)."""
    from oracle import protocols as P
    from paper_2405_12079_b300 import workloads as wl
    cfg = wl.training(scale=scale, n_kernels=n_kernels)
    rng, lay = cfg["rng"], cfg["layout"]
    va0 = 0x7F00_0000_0000
    mem = np.zeros(lay.arena_bytes, np.uint8)
    wl.fill_random(rng, mem)
    n_rec = max(int(1_300_000 * scale), 1024)
    ks = wl.make_training_kernels(rng, lay, va0, n_kernels, n_rec, 0.001)
    proc = P.Process(va0, lay.off, lay.size, mem, cfg["seed"])
    quota = a256(proc.image_bytes / 100)
    t0 = time.perf_counter()
    r1 = P.cow_checkpoint(proc, ks, int(2e9 * scale), 64 * 1024, quota)
    r2 = P.recopy_checkpoint(proc, ks, 64 * 1024, quota)
    dt = time.perf_counter() - t0
    moved = (r1.stats["cow_bytes"] + r1.stats["direct_bytes"] + r1.stats["copier_bytes"] +
             r2.stats["copier_bytes"] + r2.stats["recopy_bytes"])
    recs = n_rec * (r1.kernels_run + r2.kernels_run)
    return moved, recs, dt


def cpu_baseline(scale=0.04):
    moved, recs, dt = oracle_sample(scale)
    return {"value": moved / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "oracle CoW + recopy checkpoint of the same workload scaled to %.1f%% "
                      "(%.0f MB image, %d records validated), single thread, %.1f s"
                      % (100 * scale, 40e3 * scale, recs, dt)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    scale = 0.01
    for _ in range(args.warmup):
        oracle_sample(scale)
    tot_b, tot_t = 0, 0.0
    for _ in range(args.steps):
        b, r, dt = oracle_sample(scale)
        tot_b += b
        tot_t += dt
    v = tot_b / tot_t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_scale": scale},
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "each step: the oracle's CoW + recopy checkpoint of "
                                       "the workload scaled to %.1f%%" % (100 * scale)},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- GPU arm

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, mx, reasons = [], None, set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names[1:], f[5:9]):
                if v.lower() in ("active", "yes", "1"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


class Marks:
    """CUDA events on the launching stream between protocol phases."""

    def __init__(self, torch):
        self.torch = torch
        self.pool = []
        self.used = []

    def mark(self, name):
        if len(self.used) == len(self.pool):
            self.pool.append(self.torch.cuda.Event(enable_timing=True))
        ev = self.pool[len(self.used)]
        ev.record()
        self.used.append((name, ev))

    def collect(self, acc):
        for (n0, e0), (_, e1) in zip(self.used, self.used[1:]):
            acc[n0] = acc.get(n0, 0.0) + e0.elapsed_time(e1)
        self.used = []


def run_gpu(args, rank, world):
    import torch
    import torch.distributed as dist
    from paper_2405_12079_b300 import build as B
    from paper_2405_12079_b300 import phos, runner, workloads as wl

    if not os.path.exists(phos.LIB_PATH):
        B.build()
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    s = torch.cuda.current_stream().cuda_stream
    scale = args.scale
    cfg = wl.training(scale=scale, n_kernels=200)
    rng, lay = cfg["rng"], cfg["layout"]
    arena = torch.empty(lay.arena_bytes, dtype=torch.uint8, device="cuda")
    phos.harness_fill(arena.data_ptr(), lay.arena_bytes, cfg["seed"], s)
    va0 = arena.data_ptr()
    t0 = time.time()
    kernels = wl.make_training_kernels(rng, lay, va0, 200, cfg["n_rec"], 0.001)
    dp = runner.DeviceProcess(lay, arena, cfg["seed"], kernels)
    del kernels
    image = torch.empty(dp.image_bytes, dtype=torch.uint8).pin_memory()
    staging_bytes = a256(2e9 * scale)
    staging = torch.empty(staging_bytes, dtype=torch.uint8, device="cuda")
    quota, chunk = a256(dp.image_bytes / 100), 4 << 20
    setup_s = time.time() - t0
    torch.cuda.synchronize()

    marks = Marks(torch)

    def hook_run(mode):
        # lockstep round with phase marks (same calls as runner.DeviceProcess)
        c = (phos.Checkpoint(dp.table, phos.CKPT_COW, image.data_ptr(), image.numel(), chunk,
                             4, staging.data_ptr(), staging_bytes, s) if mode == "cow" else
             phos.Checkpoint(dp.table, phos.CKPT_RECOPY, image.data_ptr(), image.numel(), chunk,
                             4, None, 0, s))
        k = 0
        while k < len(dp.kernels):
            marks.mark("copier")
            if c.advance(quota):
                break
            pk = dp.kernels[k]
            marks.mark("cow" if mode == "cow" else "dirty_marking")
            c.before_kernel(pk.speculate(dp.table, dp.perm))
            marks.mark("app_kernel")
            dp.run_kernel(k)
            marks.mark("validate")
            mis = c.after_kernel(pk.d_trace.data_ptr(), pk.n_rec)
            k += 1
            if mis:
                break
        marks.mark("finish")
        c.finish()
        marks.mark("end")
        st = c.stats()
        c.close()
        return st

    def step():
        a = hook_run("cow")
        b = hook_run("recopy")
        moved = (a["cow_bytes"] + a["direct_bytes"] + a["copier_bytes"] + b["copier_bytes"] +
                 b["recopy_bytes"])
        return moved, a["validated"] + b["validated"], a, b

    # property check on the first warm-up step: CoW image == memory at t1
    ptr_live = [int(x) for x in lay.base(va0)]
    ptr_img = [image.data_ptr() + int(o) for o in dp.img_off]
    lens = [int(x) for x in lay.size]
    dig_a = torch.zeros(8 * lay.n, dtype=torch.uint8, device="cuda")
    dig_b = torch.zeros(8 * lay.n, dtype=torch.uint8, device="cuda")
    phos.harness_digest(ptr_live, lens, dig_a.data_ptr(), s)
    acc = {}
    hook_run("cow")
    marks.collect(acc)
    phos.harness_digest(ptr_img, lens, dig_b.data_ptr(), s)
    torch.cuda.synchronize()
    verified = {"cow_image_equals_memory_at_t1": bool(torch.equal(dig_a, dig_b))}
    hook_run("recopy")
    marks.collect(acc)
    phos.harness_digest(ptr_live, lens, dig_a.data_ptr(), s)
    phos.harness_digest(ptr_img, lens, dig_b.data_ptr(), s)
    torch.cuda.synchronize()
    verified["recopy_image_equals_memory_at_t2"] = bool(torch.equal(dig_a, dig_b))
    for _ in range(max(args.warmup - 1, 0)):
        step()
        marks.collect({})
    torch.cuda.synchronize()

    # timed region
    clk = Clocks(dev)
    clk.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = phos.launch_count()
    phase = {}
    moved = recs = 0
    stats = []
    e0.record()
    for _ in range(args.steps):
        m, r, a, b = step()
        moved += m
        recs += r
        stats.append((a, b))
    e1.record()
    torch.cuda.synchronize()
    launches = phos.launch_count() - l0
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    marks.collect(phase)
    ms = e0.elapsed_time(e1)
    t_max = ms
    tot_moved, tot_recs = moved, recs
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
        v = torch.tensor([moved, recs], dtype=torch.float64, device="cuda")
        dist.all_reduce(v)
        tot_moved, tot_recs = int(v[0].item()), int(v[1].item())

    # per-kernel rooflines from the same run
    pk = peaks()
    hbm = float(pk.get("hbm_gbs", 6400.0))
    a_last, b_last = stats[-1]
    # background copier and recopy pieces (device -> pinned host) run in
    # the copier and finish phases; CoW copies (device -> device staging,
    # or straight to the host image when staging is full) in the cow phase
    copier_ms = phase.get("copier", 0.0) + phase.get("finish", 0.0)
    d2h_bytes = sum(a["copier_bytes"] + b["copier_bytes"] + b["recopy_bytes"]
                    for a, b in stats)
    d2h_gbs = d2h_bytes / (copier_ms * 1e6) if copier_ms else 0.0
    cow_ms = phase.get("cow", 0.0)
    cow_bytes = sum(a["cow_bytes"] for a, _ in stats)
    direct_bytes = sum(a["direct_bytes"] for a, _ in stats)

    # PCIe peak: DMA copy of 1 GiB to pinned memory, best of 5 (this run)
    g = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    h = torch.empty(1 << 30, dtype=torch.uint8).pin_memory()
    best = 1e9
    for _ in range(5):
        x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        x0.record()
        h.copy_(g, non_blocking=True)
        x1.record()
        torch.cuda.synchronize()
        best = min(best, x0.elapsed_time(x1))
    pcie_d2h = (1 << 30) / (best * 1e6)
    del g, h

    # validation kernel alone, same launch shape, over all 200 traces
    nvw = (lay.n + 31) // 32
    maxw = max((p.n_rec + 31) // 32 for p in dp.kernels)
    bm = torch.empty(4 * maxw, dtype=torch.uint8, device="cuda")
    cnt = torch.empty(24, dtype=torch.uint8, device="cuda")
    vv = torch.empty(8 * nvw, dtype=torch.uint8, device="cuda")
    stw = torch.zeros(4, dtype=torch.uint8, device="cuda")
    perms = []
    for p in dp.kernels:
        perms.append(torch.from_numpy(p.speculate(dp.table, np.zeros(lay.n, np.uint8)).copy())
                     .cuda())
    for rep in range(2):
        torch.cuda.synchronize()
        x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        x0.record()
        for p, pm in zip(dp.kernels, perms):
            phos.validate(dp.table, pm.data_ptr(), p.d_trace.data_ptr(), p.n_rec, 4,
                          bm.data_ptr(), cnt.data_ptr(), vv.data_ptr(), vv.data_ptr() + 4 * nvw,
                          None, 0, stw.data_ptr(), s)
        x1.record()
        torch.cuda.synchronize()
        val_ms = x0.elapsed_time(x1)
    val_recs = sum(p.n_rec for p in dp.kernels)
    val_launch_us = 1e3 * val_ms / len(dp.kernels)
    val_gbs = val_recs * 8.125 / (val_ms * 1e6)

    # end to end: the step's traces come from pinned host memory each step
    # (host->device inside the timed region) and its stats are read back
    h_tr = [p.d_trace.cpu().pin_memory() for p in dp.kernels]
    h2d = sum(t.numel() for t in h_tr)
    e_steps = max(1, min(2, args.steps))
    torch.cuda.synchronize()
    x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    x0.record()
    e_moved = 0
    for _ in range(e_steps):
        for p, ht in zip(dp.kernels, h_tr):
            p.d_trace.copy_(ht, non_blocking=True)
        m, r, a, b = step()
        e_moved += m
    x1.record()
    torch.cuda.synchronize()
    e2e_ms = x0.elapsed_time(x1)
    d2h_step = int((d2h_bytes + direct_bytes) / args.steps)

    if rank == 0:
        cpu = cpu_baseline()
        roof = {"kernel": "k_copy_main (background copier + recopy, device->pinned host)",
                "bound": "pcie", "achieved": d2h_gbs, "peak": pcie_d2h, "unit": "GB/s",
                "frac": d2h_gbs / pcie_d2h if pcie_d2h else None, "traffic": None,
                "peak_source": "DMA cudaMemcpyAsync 1 GiB device->pinned, best of 5, "
                               "measured in this run (MEASURED_PEAKS.json has no PCIe figure)"}
        line = {
            "metric": METRIC, "value": tot_moved / (t_max * 1e6), "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "scale": scale, "image_bytes": dp.image_bytes,
                       "buffers": lay.n, "kernels": len(dp.kernels),
                       "records_per_kernel": dp.kernels[0].n_rec, "quota": quota,
                       "chunk": chunk, "staging_bytes": staging_bytes,
                       "l2": "inputs larger than L2 (image %.1f GB, traces %.2f GB)"
                             % (dp.image_bytes / 1e9, h2d / 1e9),
                       "parallelism": "replicas" if world > 1 else "1 GPU"},
            "validated_accesses_per_s": tot_recs / (t_max * 1e-3),
            "roofline": roof,
            "rooflines": [
                roof,
                {"kernel": "k_validate (one launch per kernel trace, 1.3M records)",
                 "bound": "hbm", "achieved": val_gbs, "peak": hbm, "unit": "GB/s",
                 "frac": val_gbs / hbm, "traffic": None,
                 "accesses_per_s": val_recs / (val_ms * 1e-3),
                 "avg_launch_us": val_launch_us, "peak_source": "MEASURED_PEAKS.json hbm_gbs"},
                {"kernel": "k_copy_main (CoW live->staging)", "bound": "hbm",
                 "achieved": 2 * cow_bytes / (cow_ms * 1e6) if cow_ms else None, "peak": hbm,
                 "unit": "GB/s", "frac": (2 * cow_bytes / (cow_ms * 1e6) / hbm) if cow_ms else None,
                 "traffic": None, "direct_bytes_in_phase": direct_bytes,
                 "note": "read+write bytes; phase time includes the descriptor upload, the "
                         "prologue launch and any direct-to-host copies"}],
            "breakdown_ms_per_step": {k: v / args.steps for k, v in phase.items()},
            "cow": {"cow_bytes": a_last["cow_bytes"], "direct_bytes": a_last["direct_bytes"],
                    "kernels": a_last["kernels"], "misspec_round": a_last["misspec_round"]},
            "recopy": {"recopy_bytes": b_last["recopy_bytes"], "dirty": b_last["dirty"],
                       "kernels": b_last["kernels"]},
            "verified": verified,
            "cpu_baseline": cpu,
            "e2e": {"value": e_moved / (e2e_ms * 1e6), "unit": "GB/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h_step},
            "gpu_launches": launches,
            "clocks": clocks,
            "setup_s": setup_s,
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="phos", choices=["phos", "reference"])
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the workload (parity / quick runs); 1.0 = the full 40 GB")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

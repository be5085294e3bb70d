"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs: buffer layouts, kernel launch arguments with
their ground-truth read/write sets, access traces with ground-truth class
labels, initial memory contents and request streams.  It holds none of the
method's arithmetic (no speculation, lookup, protocol or copy logic), so the
CUDA path and the CPU oracle can both consume it.

The paper's applications (Table 4: 75-718 buffers, 1.7-73.6 GB per GPU) are
private; these generators stand in for them.  Every draw comes from a numpy
PCG64 generator seeded by the caller.
"""
import math
import struct
from dataclasses import dataclass, field

import numpy as np

SEED0 = 20250512
ALIGN = 256

# trace record classes (ground truth, known at generation time)
CLS_LOAD, CLS_STORE, CLS_OTHER, CLS_GAP, CLS_STRADDLE = 0, 1, 2, 3, 4
# launch-argument kinds
ARG_SCALAR, ARG_CONST_PTR, ARG_MUT_PTR, ARG_STRUCT = 0, 1, 2, 3
STORE_BIT = np.uint64(1 << 63)


def _a256(x):
    return (np.asarray(x, np.uint64) + np.uint64(ALIGN - 1)) & ~np.uint64(ALIGN - 1)


@dataclass
class Layout:
    """n buffers carved from one arena at 256-byte aligned offsets."""
    off: np.ndarray            # uint64 arena offset of each buffer
    size: np.ndarray           # uint64 byte size of each buffer
    arena_bytes: int

    @property
    def n(self):
        return len(self.off)

    def base(self, va0):
        return self.off + np.uint64(va0)


def sizes_uniform(rng, n, lo, hi):
    return rng.integers(lo, hi + 1, size=n, dtype=np.int64).astype(np.uint64)


def sizes_lognormal(rng, n, lo, hi, total, round_to=ALIGN):
    """Log-normal sizes clipped to [lo, hi] with sigma = ln(hi/lo)/6; the
    location is bisected on the drawn sample so the clipped sizes sum to
    ``total`` (within 0.5 %).  Sizes are rounded up to ``round_to``."""
    z = rng.standard_normal(n)
    sigma = math.log(hi / lo) / 6.0
    lo_mu, hi_mu = math.log(lo) - 10, math.log(hi) + 10
    for _ in range(200):
        mu = 0.5 * (lo_mu + hi_mu)
        s = np.clip(np.exp(mu + sigma * z), lo, hi)
        if s.sum() > total:
            hi_mu = mu
        else:
            lo_mu = mu
    s = np.clip(np.exp(0.5 * (lo_mu + hi_mu) + sigma * z), lo, hi)
    s = np.ceil(s / round_to) * round_to
    return s.astype(np.uint64)


def make_layout(rng, sizes, gap_lo=256, gap_hi=65536):
    sizes = np.asarray(sizes, np.uint64)
    n = len(sizes)
    gaps = rng.integers(gap_lo, gap_hi + 1, size=n + 1).astype(np.uint64)
    off = np.zeros(n, np.uint64)
    cur = np.uint64(0)
    for i in range(n):
        cur = _a256(cur + gaps[i])
        off[i] = cur
        cur = cur + sizes[i]
    arena = int(_a256(cur + gaps[n]))
    return Layout(off=off, size=sizes, arena_bytes=arena)


def fill_random(rng, arena_u8):
    """Uniform random bytes for the initial live memory (numpy array)."""
    step = 1 << 26
    for o in range(0, arena_u8.size, step):
        m = min(step, arena_u8.size - o)
        arena_u8[o:o + m] = rng.integers(0, 256, size=m, dtype=np.uint8)


@dataclass
class Kernel:
    """One application kernel launch (harness stand-in)."""
    args: list                 # raw little-endian bytes of each argument
    kinds: list                # ARG_* of each argument
    reads: np.ndarray          # ground truth: buffers read, ascending (includes writes)
    writes: np.ndarray         # ground truth: buffers written, ascending
    trace: np.ndarray          # uint64 access records
    labels: np.ndarray         # uint8 class of each record (CLS_*)
    w: int = 4                 # access width in bytes
    strays: list = field(default_factory=list)   # (record index, address) stray stores


def make_args(rng, layout, va0, reads, writes, struct_frac=0.2):
    """Launch arguments whose pointer values land inside the given buffers:
    mutable pointers for writes, const pointers for read-only buffers, a few
    scalars, and with probability ``struct_frac`` an opaque struct that
    carries some of the written pointers next to small scalar fields."""
    base = layout.base(va0)
    wr = [int(x) for x in writes]
    ro = [int(x) for x in reads if int(x) not in set(wr)]

    def ptr(i):
        o = int(rng.integers(0, int(layout.size[i])))
        return int(base[i]) + o

    args, kinds = [], []
    in_struct = []
    if wr and rng.random() < struct_frac:
        m = int(rng.integers(1, len(wr) + 1))
        in_struct = wr[:m]
        wr = wr[m:]
    for i in wr:
        args.append(struct.pack("<Q", ptr(i))); kinds.append(ARG_MUT_PTR)
    for i in ro:
        args.append(struct.pack("<Q", ptr(i))); kinds.append(ARG_CONST_PTR)
    for _ in range(int(rng.integers(0, 4))):
        sz = int(rng.choice([4, 8]))
        v = int(rng.integers(0, 1 << 20))
        args.append(v.to_bytes(sz, "little")); kinds.append(ARG_SCALAR)
    if in_struct:
        b = b""
        for i in in_struct:
            b += struct.pack("<Q", ptr(i))
            b += struct.pack("<I", int(rng.integers(0, 1 << 16))) + b"\0\0\0\0"
        b += b"\x07\x00\x00"          # trailing partial chunk, ignored
        args.append(b); kinds.append(ARG_STRUCT)
    order = rng.permutation(len(args))
    return [args[j] for j in order], [kinds[j] for j in order]


def _gap_ranges(layout, va0, w):
    """[lo, hi] ranges of w-byte aligned addresses in the unmapped gaps."""
    base = layout.base(va0)
    ends = base + layout.size
    starts = np.concatenate([[np.uint64(va0)], ends])
    stops = np.concatenate([base, [np.uint64(va0 + layout.arena_bytes)]])
    lo = (starts + np.uint64(w - 1)) // np.uint64(w) * np.uint64(w)
    hi = stops - np.uint64(w)
    ok = hi >= lo
    return lo[ok], hi[ok]


def _rand_in_buffers(rng, layout, va0, bufs, count, w, align):
    b = rng.choice(np.asarray(bufs, np.int64), size=count)
    sz = layout.size[b].astype(np.int64)
    span = (sz - w) // align + 1
    o = (rng.random(count) * span).astype(np.int64) * align
    return layout.base(va0)[b] + o.astype(np.uint64)


def _rand_in_gaps(rng, layout, va0, count, w):
    lo, hi = _gap_ranges(layout, va0, w)
    g = rng.integers(0, len(lo), size=count)
    span = ((hi[g] - lo[g]) // np.uint64(w) + np.uint64(1)).astype(np.float64)
    o = (rng.random(count) * span).astype(np.uint64) * np.uint64(w)
    return lo[g] + o


def trace_random(rng, layout, va0, in_set, n_rec, frac_other=0.03, frac_gap=0.02,
                 store_frac=0.25, w=4, write_set=None):
    """Independent records: (1 - other - gap) inside ``in_set``, ``frac_other``
    in buffers outside it, ``frac_gap`` in unmapped gaps; ``store_frac`` of
    the records are stores (only into ``write_set`` for in-set records;
    default: the whole in-set).  Addresses are w-aligned."""
    in_set = np.asarray(in_set, np.int64)
    write_set = in_set if write_set is None else np.asarray(write_set, np.int64)
    others = np.setdiff1d(np.arange(layout.n), in_set)
    n_other = int(round(n_rec * frac_other)) if len(others) else 0
    n_gap = int(round(n_rec * frac_gap))
    n_in = n_rec - n_other - n_gap
    cls = np.concatenate([np.zeros(n_in, np.uint8), np.full(n_other, CLS_OTHER, np.uint8),
                          np.full(n_gap, CLS_GAP, np.uint8)])
    rng.shuffle(cls)
    rec = np.zeros(n_rec, np.uint64)
    store = rng.random(n_rec) < store_frac
    m_in = cls == 0
    addr_in = _rand_in_buffers(rng, layout, va0, in_set, int(m_in.sum()), w, w)
    rec[m_in] = addr_in
    # in-set stores only where the buffer is writable
    if len(write_set) != len(in_set):
        base = layout.base(va0)
        bi = np.searchsorted(base, addr_in, side="right") - 1
        store_ok = np.isin(bi, write_set)
        st_in = store[m_in] & store_ok
        store[m_in] = st_in
    cls[m_in & store] = CLS_STORE
    m_o = cls == CLS_OTHER
    if n_other:
        rec[m_o] = _rand_in_buffers(rng, layout, va0, others, n_other, w, w)
    m_g = cls == CLS_GAP
    if n_gap:
        rec[m_g] = _rand_in_gaps(rng, layout, va0, n_gap, w)
    rec[store] |= STORE_BIT
    return rec, cls


def trace_runs(rng, layout, va0, reads, writes, n_rec, stray_frac=0.001,
               stray_store_frac=0.0, run=32, w=4):
    """Warp-coalesced runs: each run of ``run`` records is a, a+w, ...
    at a (run*w)-aligned offset inside one buffer of the kernel's read/write
    set (stores with probability 1/2 when the buffer is written).  Then a
    ``stray_frac`` share of records is replaced by strays outside the set
    (3:2 other-buffer : gap); ``stray_store_frac`` of those are stores.
    Returns (records, labels, stray stores inside buffers)."""
    rw = np.union1d(np.asarray(reads, np.int64), np.asarray(writes, np.int64))
    n_runs = (n_rec + run - 1) // run
    span = run * w
    b = rng.choice(rw, size=n_runs)
    sz = layout.size[b].astype(np.int64)
    slots = np.maximum((sz - span) // span + 1, 1)
    o = (rng.random(n_runs) * slots).astype(np.int64) * span
    a0 = layout.base(va0)[b] + o.astype(np.uint64)
    is_w = np.isin(b, np.asarray(writes, np.int64))
    st = is_w & (rng.random(n_runs) < 0.5)
    lane = np.arange(run, dtype=np.uint64) * np.uint64(w)
    rec = (a0[:, None] + lane[None, :]).reshape(-1)[:n_rec]
    stv = np.repeat(st, run)[:n_rec]
    # clip runs that would leave a small buffer (size < run*w)
    endb = np.repeat(layout.base(va0)[b] + layout.size[b], run)[:n_rec]
    inside = rec + np.uint64(w) <= endb
    cls = np.where(stv, CLS_STORE, CLS_LOAD).astype(np.uint8)
    rec = np.where(inside, rec, np.repeat(a0, run)[:n_rec])
    rec = rec | np.where(stv, STORE_BIT, np.uint64(0))
    strays = []
    n_stray = int(round(n_rec * stray_frac))
    if n_stray:
        pos = np.sort(rng.choice(n_rec, size=n_stray, replace=False))
        others = np.setdiff1d(np.arange(layout.n), rw)
        kind_other = rng.random(n_stray) < 0.6
        if len(others) == 0:
            kind_other[:] = False
        is_store = rng.random(n_stray) < stray_store_frac
        n_o = int(kind_other.sum())
        addr = np.zeros(n_stray, np.uint64)
        if n_o:
            addr[kind_other] = _rand_in_buffers(rng, layout, va0, others, n_o, w, w)
        if n_stray - n_o:
            addr[~kind_other] = _rand_in_gaps(rng, layout, va0, n_stray - n_o, w)
        rec[pos] = addr | np.where(is_store, STORE_BIT, np.uint64(0))
        cls[pos] = np.where(kind_other, CLS_OTHER, CLS_GAP)
        for j in np.nonzero(kind_other & is_store)[0]:
            strays.append((int(pos[j]), int(addr[j])))
    return rec, cls, strays


def pick_sets(rng, n, lo=1, hi=20, locality=None, window=64):
    """Random read and write sets of lo..hi buffers each.  With ``locality``
    (a start index), sets come from a window [start, start+window) with 20 %
    drawn anywhere (layer locality)."""
    def one():
        m = int(rng.integers(lo, hi + 1))
        m = min(m, n)
        if locality is None:
            return np.sort(rng.choice(n, size=m, replace=False))
        s = set()
        while len(s) < m:
            if rng.random() < 0.2:
                s.add(int(rng.integers(0, n)))
            else:
                s.add(int((locality + rng.integers(0, window)) % n))
        return np.array(sorted(s), np.int64)
    w = one()
    r = one()
    return np.union1d(r, w), w


def make_training_kernels(rng, layout, va0, n_kernels, n_rec, stray_frac=0.001,
                          stray_store_frac=0.0, set_hi=20):
    """200-kernel style mutator sequence: each kernel writes 1..set_hi random
    buffers and reads 1..set_hi, with a coalesced-run trace."""
    ks = []
    for _ in range(n_kernels):
        reads, writes = pick_sets(rng, layout.n, 1, set_hi)
        args, kinds = make_args(rng, layout, va0, reads, writes)
        rec, cls, strays = trace_runs(rng, layout, va0, reads, writes, n_rec,
                                      stray_frac, stray_store_frac)
        ks.append(Kernel(args, kinds, reads, writes, rec, cls, 4, strays))
    return ks


def make_restore_kernels(rng, layout, va0, n_kernels, n_rec, stray_frac=0.0, set_hi=20):
    """Replay sequence with layer locality: kernel k touches buffers near a
    window that sweeps the table in index order (inference layers)."""
    ks = []
    for k in range(n_kernels):
        start = int(k * layout.n / max(n_kernels, 1))
        reads, writes = pick_sets(rng, layout.n, 1, set_hi, locality=start)
        args, kinds = make_args(rng, layout, va0, reads, writes)
        rec, cls, strays = trace_runs(rng, layout, va0, reads, writes, n_rec, stray_frac, 0.0)
        ks.append(Kernel(args, kinds, reads, writes, rec, cls, 4, strays))
    return ks


# ---------------------------------------------------------------------------
# the five workload shapes; ``scale`` shrinks byte totals and record counts
# ---------------------------------------------------------------------------

def tiny(scale=1.0, seed=SEED0 + 1):
    """64 buffers of U[4 KiB, 1 MiB], speculated write set of 16, 1M-record
    trace (95 % in-set, 3 % other buffers, 2 % gaps, 25 % stores, w = 4)."""
    rng = np.random.default_rng(seed)
    hi = max(int((1 << 20) * scale), 8192)
    sizes = sizes_uniform(rng, 64, 4096, hi)
    layout = make_layout(rng, sizes)
    wset = np.sort(rng.choice(64, size=16, replace=False))
    n_rec = max(int(1_000_000 * scale), 1024)
    return dict(rng=rng, layout=layout, wset=wset, n_rec=n_rec, seed=seed)


def training(scale=1.0, seed=SEED0 + 2, n_kernels=200, n_rec=1_300_000):
    """1,000 buffers, log-normal 256 B - 512 MB, 40 GB total; 200 kernels."""
    rng = np.random.default_rng(seed)
    total = 40e9 * scale
    hi = max(min(512 * 2**20, total / 4), 4096)
    sizes = sizes_lognormal(rng, 1000, 256, hi, total)
    layout = make_layout(rng, sizes)
    return dict(rng=rng, layout=layout, n_kernels=n_kernels,
                n_rec=max(int(n_rec * scale), 4096) if scale < 1 else n_rec, seed=seed)


def batched(scale=1.0, seed=SEED0 + 3, n_images=64):
    """64 images, buffer counts log-uniform 20-2,000, image sizes log-uniform
    0.1-2 GB rescaled to 40 GB in total."""
    rng = np.random.default_rng(seed)
    counts = np.exp(rng.uniform(math.log(20), math.log(2000), n_images)).astype(np.int64)
    isz = np.exp(rng.uniform(math.log(0.1e9), math.log(2e9), n_images))
    isz = isz * (40e9 * scale / isz.sum())
    images = []
    for j in range(n_images):
        hi = max(min(512 * 2**20, isz[j] / 4), 4096)
        sizes = sizes_lognormal(rng, int(counts[j]), 256, hi, isz[j])
        images.append(make_layout(rng, sizes))
    return dict(rng=rng, images=images, seed=seed)


def serving(seed=SEED0 + 4, rate=50.0, window_s=30.0, lo=50e6, hi=20e9, scale=1.0):
    """Poisson arrivals; half checkpoints, half restores; image sizes
    log-normal clipped to [lo, hi] with sigma = ln(hi/lo)/6 around the
    geometric mean; 100-10,000 buffers per request."""
    rng = np.random.default_rng(seed)
    t, reqs = 0.0, []
    sigma = math.log(hi / lo) / 6.0
    mu = 0.5 * (math.log(lo) + math.log(hi))
    while True:
        t += rng.exponential(1.0 / rate)
        if t > window_s:
            break
        size = float(np.clip(math.exp(mu + sigma * rng.standard_normal()), lo, hi)) * scale
        nb = int(np.exp(rng.uniform(math.log(100), math.log(10000))))
        kind = "ckpt" if rng.random() < 0.5 else "restore"
        reqs.append(dict(t=t, bytes=max(int(size), 256 * nb), n_bufs=nb, kind=kind))
    return dict(rng=rng, requests=reqs, seed=seed)


def large_restore(scale=1.0, seed=SEED0 + 5, n_kernels=500, n_rec=65536):
    """10,000 buffers, log-normal 4 KB - 2 GB, 120 GB total (times scale)."""
    rng = np.random.default_rng(seed)
    total = 120e9 * scale
    hi = max(min(2 * 2**30, total / 8), 8192)
    sizes = sizes_lognormal(rng, 10000, 4096, hi, total)
    layout = make_layout(rng, sizes)
    return dict(rng=rng, layout=layout, n_kernels=n_kernels, n_rec=n_rec, seed=seed)

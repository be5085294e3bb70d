"""Concurrent checkpoint / restore protocols, plain and sequential --
TEST INFRASTRUCTURE ONLY.

Each protocol is written as the paper states it, in lockstep: in every
round the background copier first moves at most ``quota`` bytes (the copy
that runs concurrently with the next kernel), then the protocol acts on the
next kernel's speculated buffers, the kernel runs, and its access trace is
validated.  Copies are numpy slice assignments.

  cow_checkpoint      Section 4.2 (soft copy-on-write; staging full ->
                      copy straight to the host image; store mis-speculation
                      on a buffer not yet checkpointed -> discard and take a
                      stop-the-world checkpoint at that instant)
  recopy_checkpoint   Section 4.3 (soft recopy; dirty = written while being
                      or after being copied; validator victims join the
                      dirty set; quiesce at t2 and recopy the dirty set)
  concurrent_restore  Section 6 (on-demand restore of the speculated
                      read/write buffers before each kernel, background bulk
                      restore; an access to a buffer not yet restored rolls
                      everything back to the checkpoint, restores
                      stop-the-world and replays)
  stw_checkpoint / stw_restore   the stop-the-world references the
                      correctness arguments of Sections 4.2, 4.3 and 6
                      compare against.

Readings of points the paper leaves open (the same prose is the only thing
the CUDA control plane shares with this file):
  - image layout: buffer i at img_off[i] = sum of align256(size) before it
  - copier: ascending table index, pieces of at most ``chunk`` bytes that
    never cross a buffer; a piece is also cut at the remaining quota; each
    piece charges align256(len) against the quota (quota, chunk multiples
    of 256)
  - staging: first-fit over free extents (ascending offset, coalesced on
    free), each shadow takes align256(size); freed once drained
  - CoW acts on speculated-write buffers that are neither done nor
    shadowed, in ascending index; a partially copied buffer is shadowed
    whole; without room its remaining bytes go straight to the image
  - the checkpoint ends when the copier has drained every buffer (checked
    right after its move in each round); kernels after that point are not
    part of it; when the kernels run out first the copier drains the rest
  - restore: the protocol ends once every buffer is present; the remaining
    kernels then run normally
Parity: the copier's piece schedule is pinned by a piece log written out
by hand (sizes that are not multiples of 256); the protocols are pinned by
the correctness theorems (image == memory at t1 for CoW,
at t2 for recopy; concurrent restore == stop-the-world restore + replay),
by the worked scenarios of Figures 6, 7 and 9, and by closed-form special
cases (zero staging budget, zero kernels, copier faster than the kernels).
"""
import numpy as np

from . import core

PENDING, INFLIGHT, DONE = 0, 1, 2
PERM_R, PERM_W = 1, 2


def align256(x):
    return (int(x) + 255) & ~255


class Process:
    """Live memory of one process: a byte arena holding every buffer."""

    def __init__(self, va0, buf_off, buf_size, arena, seed):
        self.va0 = int(va0)
        self.off = np.asarray(buf_off, np.uint64)
        self.size = np.asarray(buf_size, np.uint64)
        self.base = self.off + np.uint64(self.va0)
        self.mem = arena                      # uint8, modified in place
        self.seed = int(seed)
        self.n = len(self.off)
        self.img_off = np.zeros(self.n, np.uint64)
        acc = 0
        for i in range(self.n):
            self.img_off[i] = acc
            acc += align256(self.size[i])
        self.image_bytes = acc

    def buf(self, i):
        o, s = int(self.off[i]), int(self.size[i])
        return self.mem[o:o + s]

    def speculate(self, kern):
        return core.speculate(self.base, self.size, kern.args, kern.kinds)

    def new_bytes(self, n):
        """A zeroed byte array for an image or a staging area."""
        return np.zeros(int(n), np.uint8)

    def read_digests(self, reads):
        return [core.digest(self.buf(r)) for r in reads]

    def fill(self, w, s_k):
        core.mutator_fill(self.buf(w), s_k, int(w))

    def run_kernel(self, k, kern):
        """Harness mutator: read digests, fill written buffers, strays."""
        digs = self.read_digests(kern.reads)
        s = core.mutator_seed(self.seed, k, digs)
        for w in kern.writes:
            self.fill(w, s)
        for r, a in kern.strays:
            v = core.stray_value(self.seed, k, int(r))
            o = int(a) - self.va0
            self.mem[o:o + 4] = np.frombuffer(int(v).to_bytes(4, "little"), np.uint8)

    def validate(self, perm, kern):
        return core.validate(self.base, self.size, perm, kern.trace, kern.w)


def victims_of(res, n):
    """Buffers named by any access the speculation did not allow."""
    bits = np.unpackbits(res.victim.view(np.uint8), bitorder="little")[:n]
    return np.nonzero(bits)[0]


def stw_checkpoint(proc):
    img = proc.new_bytes(proc.image_bytes)
    for i in range(proc.n):
        s, io = int(proc.size[i]), int(proc.img_off[i])
        img[io:io + s] = proc.buf(i)
    return img


def stw_restore(proc, image):
    for i in range(proc.n):
        s, io = int(proc.size[i]), int(proc.img_off[i])
        proc.buf(i)[:] = image[io:io + s]


class FirstFit:
    """Staging allocator: first fit over free extents."""

    def __init__(self, total):
        self.free = [(0, int(total))] if total > 0 else []

    def alloc(self, nbytes):
        for j, (o, ln) in enumerate(self.free):
            if ln >= nbytes:
                if ln == nbytes:
                    del self.free[j]
                else:
                    self.free[j] = (o + nbytes, ln - nbytes)
                return o
        return None

    def release(self, off, nbytes):
        self.free.append((off, nbytes))
        self.free.sort()
        merged = []
        for o, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((o, ln))
        self.free = merged


class Copier:
    """Background copier state shared by the three protocols."""

    def __init__(self, n, size, chunk):
        self.n = n
        self.size = [int(s) for s in size]
        self.chunk = int(chunk)
        self.state = [PENDING] * n
        self.copied = [0] * n
        self.cursor = 0
        self.log = []                     # (round, buf, off, len, from_shadow)

    def done(self):
        while self.cursor < self.n and self.state[self.cursor] == DONE:
            self.cursor += 1
        return self.cursor >= self.n

    def advance(self, quota, move, rnd, skip=lambda i: False):
        """Move up to ``quota`` bytes; move(i, off, len) copies one piece and
        returns whether it came from a shadow."""
        left = quota
        while left > 0 and not self.done():
            i = self.cursor
            if skip(i):
                self.state[i] = DONE
                continue
            rem = self.size[i] - self.copied[i]
            take = min(self.chunk, rem, left)
            if take <= 0:
                break
            shadow = move(i, self.copied[i], take)
            self.log.append((rnd, i, self.copied[i], take, bool(shadow)))
            self.copied[i] += take
            left -= align256(take)
            self.state[i] = DONE if self.copied[i] == self.size[i] else INFLIGHT
        return quota - left


class Result:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def cow_checkpoint(proc, kernels, staging_bytes, chunk, quota):
    """Section 4.2 soft copy-on-write checkpoint taken at t1 = now."""
    n = proc.n
    image = proc.new_bytes(proc.image_bytes)
    staging = proc.new_bytes(max(int(staging_bytes), 1))
    alloc = FirstFit(staging_bytes)
    shadow = [None] * n
    cp = Copier(n, proc.size, chunk)
    cow_log = []                          # (k, buf, 'S'|'D', off, len)
    misspec = None
    stats = dict(cow_bytes=0, direct_bytes=0, copier_bytes=0)

    def move(i, off, ln):
        io = int(proc.img_off[i]) + off
        if shadow[i] is not None:
            so = shadow[i] + off
            image[io:io + ln] = staging[so:so + ln]
        else:
            image[io:io + ln] = proc.buf(i)[off:off + ln]
        stats["copier_bytes"] += ln
        if off + ln == cp.size[i] and shadow[i] is not None:
            alloc.release(shadow[i], align256(cp.size[i]))
            shadow[i] = None
            return True
        return shadow[i] is not None

    k = 0
    while k < len(kernels):
        cp.advance(quota, move, k)
        if cp.done():
            break
        kern = kernels[k]
        perm = proc.speculate(kern)
        for i in np.nonzero(perm & PERM_W)[0]:
            i = int(i)
            if cp.state[i] == DONE or shadow[i] is not None:
                continue
            sz = cp.size[i]
            o = alloc.alloc(align256(sz))
            if o is not None:
                staging[o:o + sz] = proc.buf(i)
                shadow[i] = o
                cow_log.append((k, i, "S", o, sz))
                stats["cow_bytes"] += sz
            else:
                c = cp.copied[i]
                io = int(proc.img_off[i])
                image[io + c:io + sz] = proc.buf(i)[c:]
                cow_log.append((k, i, "D", c, sz - c))
                stats["direct_bytes"] += sz - c
                cp.copied[i] = sz
                cp.state[i] = DONE
        safe = [cp.state[i] == DONE or shadow[i] is not None for i in range(n)]
        proc.run_kernel(k, kern)
        res = proc.validate(perm, kern)
        k += 1
        bad = [v for v in victims_of_store(proc, perm, kern, res) if not safe[v]]
        if bad:
            misspec = k - 1
            image = stw_checkpoint(proc)
            break
    if misspec is None and not cp.done():
        cp.advance(1 << 62, move, k)
    return Result(image=image, cow_log=cow_log, copier_log=cp.log, misspec=misspec,
                  kernels_run=k, stats=stats)


def victims_of_store(proc, perm, kern, res):
    """Buffers hit by a store the speculation did not allow (Section 4.2:
    only writes matter for copy-on-write and recopy)."""
    bits = np.unpackbits(res.victim_st.view(np.uint8), bitorder="little")[:proc.n]
    return [int(v) for v in np.nonzero(bits)[0]]


def recopy_checkpoint(proc, kernels, chunk, quota):
    """Section 4.3 soft recopy checkpoint started at t1 = now, ending at t2."""
    n = proc.n
    image = proc.new_bytes(proc.image_bytes)
    cp = Copier(n, proc.size, chunk)
    dirty = set()
    stats = dict(copier_bytes=0, recopy_bytes=0)

    def move(i, off, ln):
        io = int(proc.img_off[i]) + off
        image[io:io + ln] = proc.buf(i)[off:off + ln]
        stats["copier_bytes"] += ln
        return False

    k = 0
    while k < len(kernels):
        cp.advance(quota, move, k)
        if cp.done():
            break
        kern = kernels[k]
        perm = proc.speculate(kern)
        touched = [cp.state[i] != PENDING for i in range(n)]
        for i in np.nonzero(perm & PERM_W)[0]:
            if touched[int(i)]:
                dirty.add(int(i))
        proc.run_kernel(k, kern)
        res = proc.validate(perm, kern)
        for v in victims_of_store(proc, perm, kern, res):
            if touched[v]:
                dirty.add(v)
        k += 1
    if not cp.done():
        cp.advance(1 << 62, move, k)
    # t2: quiesce, recopy the dirty set whole from live memory
    for i in sorted(dirty):
        sz, io = int(proc.size[i]), int(proc.img_off[i])
        image[io:io + sz] = proc.buf(i)
        stats["recopy_bytes"] += sz
    return Result(image=image, dirty=sorted(dirty), copier_log=cp.log, kernels_run=k,
                  stats=stats)


def iterative_recopy(proc, kernels, chunk, quota, max_passes, stop_bytes):
    """Iterative concurrent recopy (Section 4.3: "we can also iteratively do
    the concurrent recopy", pre-copy in the style of live migration).

    Pass 0 is the soft recopy's concurrent copy of every buffer.  Whenever
    the copier finishes a pass, if fewer than ``max_passes`` extra passes
    ran, the dirty bytes exceed ``stop_bytes`` and they shrank since the
    previous pass, the dirty buffers become pending again and a new
    concurrent pass recopies them while the kernels keep running (the same
    dirty rule applies: written while in flight or after being copied);
    otherwise the checkpoint quiesces (t2) and recopies the dirty set
    stop-the-world.  The pass starts in the round whose copier move
    finished the previous pass, before that round's kernel."""
    n = proc.n
    image = proc.new_bytes(proc.image_bytes)
    cp = Copier(n, proc.size, chunk)
    dirty = set()
    passes = []                           # (round, buffers, bytes) of each extra pass
    stats = dict(copier_bytes=0, recopy_bytes=0)

    def move(i, off, ln):
        io = int(proc.img_off[i]) + off
        image[io:io + ln] = proc.buf(i)[off:off + ln]
        stats["copier_bytes"] += ln
        return False

    prev = None
    k = 0
    while k < len(kernels):
        cp.advance(quota, move, k)
        if cp.done():
            db = sum(int(proc.size[i]) for i in dirty)
            if len(passes) < max_passes and db > stop_bytes and (prev is None or db < prev):
                for i in sorted(dirty):
                    cp.state[i] = PENDING
                    cp.copied[i] = 0
                cp.cursor = 0
                passes.append((k, sorted(dirty), db))
                prev = db
                dirty = set()
            else:
                break
        kern = kernels[k]
        perm = proc.speculate(kern)
        touched = [cp.state[i] != PENDING for i in range(n)]
        for i in np.nonzero(perm & PERM_W)[0]:
            if touched[int(i)]:
                dirty.add(int(i))
        proc.run_kernel(k, kern)
        res = proc.validate(perm, kern)
        for v in victims_of_store(proc, perm, kern, res):
            if touched[v]:
                dirty.add(v)
        k += 1
    if not cp.done():
        cp.advance(1 << 62, move, k)
    for i in sorted(dirty):
        sz, io = int(proc.size[i]), int(proc.img_off[i])
        image[io:io + sz] = proc.buf(i)
        stats["recopy_bytes"] += sz
    return Result(image=image, dirty=sorted(dirty), passes=passes, copier_log=cp.log,
                  kernels_run=k, stats=stats)


def concurrent_restore(proc, image, kernels, chunk, quota, copier_stream=False,
                       ondemand_first=False):
    """Section 6 soft on-demand concurrent restore, then the rest of the
    kernels.  proc.mem holds whatever was there before (not restored).

    copier_stream: the background copier's pieces run on a stream of their
    own.  A piece issued in round r lands before a later kernel only if
    that kernel waited for it, and a kernel waits for the copier's latest
    piece of each buffer it is speculated to access (all pieces up to that
    round are then in place, since the copier's pieces land in order).  A
    buffer counts as restored for the mis-speculation rule once it is
    present and its last copier piece is at or below the latest round
    waited for; bytes and the final memory are the same either way.

    ondemand_first (with copier_stream): a round fetches its kernel's
    missing buffers first and advances the copier after, so the copier
    never moves a buffer the round's kernel needs (those are present by
    then) and the kernel never waits for its own round's pieces.  The
    session ends when every buffer is present at the start of a round."""
    assert copier_stream or not ondemand_first
    n = proc.n
    present = [False] * n
    last = [-1] * n                       # round of the copier's last piece of buffer i
    waited = -1
    cp = Copier(n, proc.size, chunk)
    ondemand = []                         # (k, buf, off, len)
    misspec = None
    stats = dict(ondemand_bytes=0, copier_bytes=0)

    def fetch(i, off, ln):
        io = int(proc.img_off[i]) + off
        proc.buf(i)[off:off + ln] = image[io:io + ln]

    k = 0

    def move(i, off, ln):
        fetch(i, off, ln)
        stats["copier_bytes"] += ln
        last[i] = k
        if off + ln == cp.size[i]:
            present[i] = True
        return False

    while k < len(kernels):
        if ondemand_first:
            if all(present):
                break
        else:
            cp.advance(quota, move, k, skip=lambda i: present[i])
            if all(present):
                break
        kern = kernels[k]
        perm = proc.speculate(kern)
        if copier_stream:
            for i in np.nonzero(perm)[0]:
                waited = max(waited, last[int(i)])
        for i in np.nonzero(perm)[0]:
            i = int(i)
            if not present[i]:
                c = cp.copied[i]
                fetch(i, c, cp.size[i] - c)
                ondemand.append((k, i, c, cp.size[i] - c))
                stats["ondemand_bytes"] += cp.size[i] - c
                cp.copied[i] = cp.size[i]
                cp.state[i] = DONE
                present[i] = True
        before = [present[i] and (not copier_stream or last[i] <= waited) for i in range(n)]
        if ondemand_first:
            cp.advance(quota, move, k, skip=lambda i: present[i])
        proc.run_kernel(k, kern)
        res = proc.validate(perm, kern)
        k += 1
        bad = [int(v) for v in victims_of(res, n) if not before[int(v)]]
        if bad:
            misspec = k - 1
            stw_restore(proc, image)
            for j in range(k):
                proc.run_kernel(j, kernels[j])
            present = [True] * n
            break
    if not all(present):
        cp.advance(1 << 62, move, k, skip=lambda i: present[i])
    run_during = k
    for j in range(k, len(kernels)):
        proc.run_kernel(j, kernels[j])
    return Result(ondemand=ondemand, copier_log=cp.log, misspec=misspec,
                  kernels_during=run_during, stats=stats)


def wasted_gpu_hours(n, f_fail, overhead, restore, hours, f):
    """Appendix A.1 cost, as printed: failures cost N F T (R + N / (2 f)),
    checkpoints cost N O f T."""
    return n * f_fail * hours * (restore + n / (2.0 * f)) + n * overhead * f * hours


def optimal_frequency(n, f_fail, overhead):
    """Appendix A.1: f* = sqrt(N F / (2 O))."""
    return (n * f_fail / (2.0 * overhead)) ** 0.5

"""The "versions" storage mode of the protocol oracle -- TEST INFRASTRUCTURE
ONLY.

The protocols in ``protocols.py`` move bytes by slice assignment between
live memory, device staging and the checkpoint image.  At the sizes the
benchmark runs (a 40 GB training image, a 120 GB restore image) the oracle
cannot hold its own copies of those bytes, so this module gives the same
protocol code arrays that hold *descriptions* of bytes instead: every array
is a sorted list of segments, each saying "these bytes are bytes
[src_off, src_off + len) of source S".  Sources:

  Words(key)   the harness word stream, word j = sm(key ^ j) (the initial
               fill of an arena, and the mutator's fill of a written buffer
               with key = sm(s_k ^ sm(w)))
  Literal      explicit bytes (a stray store's four bytes)
  ZERO         zeros (fresh staging and image arrays)

A copy between arrays copies segment descriptions, a mutator fill replaces
a buffer's segments by one Words segment, and a stray store inserts a
four-byte Literal.  Expected bytes are regenerated from the segments only
when a digest is needed (the mutator's reads) or when a result is compared,
piece by piece, so a full-size image is compared byte for byte without the
oracle holding it.  The protocol decisions are the same code in both modes.

Digests of independent buffers are computed on a thread pool (the C
oracle's calls release the interpreter lock); each digest is the plain
``orc_digest`` definition summed over 8-byte aligned pieces
(``orc_digest_at``).
"""
import bisect
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import core
from .protocols import Process

CHUNK = 64 << 20          # regeneration piece (a multiple of 8)
M64 = (1 << 64) - 1


class Words:
    """Byte stream whose 8-byte little-endian word j is sm(key ^ j)."""
    __slots__ = ("key",)
    _interned = {}

    def __new__(cls, key):
        key &= M64
        w = cls._interned.get(key)
        if w is None:
            w = object.__new__(cls)
            w.key = key
            cls._interned[key] = w
        return w

    def gen(self, off, ln):
        return core.words(ln, self.key, off)


class Literal:
    __slots__ = ("data",)

    def __init__(self, data):
        self.data = np.array(data, np.uint8)

    def gen(self, off, ln):
        return self.data[off:off + ln].copy()


class _Zero:
    def gen(self, off, ln):
        return np.zeros(ln, np.uint8)


ZERO = _Zero()


def _bounds(sl, n):
    a, b, step = sl.indices(n)
    assert step == 1
    return a, max(a, b)


class VArray:
    """A byte array of length n held as segments (start, end, src, src_off),
    sorted, disjoint and covering [0, n)."""

    def __init__(self, n, src=ZERO, src_off=0):
        self.n = int(n)
        self.segs = [(0, self.n, src, int(src_off))] if self.n else []
        self.starts = [0] if self.n else []

    @property
    def size(self):
        return self.n

    def __len__(self):
        return self.n

    def _cut(self, pos):
        """Index of the segment that starts at pos, splitting one if needed
        (len(segs) when pos == n)."""
        if pos >= self.n:
            return len(self.segs)
        i = bisect.bisect_right(self.starts, pos) - 1
        s, e, src, so = self.segs[i]
        if s == pos:
            return i
        self.segs[i:i + 1] = [(s, pos, src, so), (pos, e, src, so + (pos - s))]
        self.starts[i + 1:i + 1] = [pos]
        return i + 1

    def _merge_at(self, i):
        """Merge segments i-1 and i when they continue the same source."""
        if 0 < i < len(self.segs):
            s0, e0, a, o0 = self.segs[i - 1]
            s1, e1, b, o1 = self.segs[i]
            if a is b and o0 + (e0 - s0) == o1:
                self.segs[i - 1:i + 1] = [(s0, e1, a, o0)]
                del self.starts[i]

    def pieces(self, a, b):
        """[(len, src, src_off)] describing bytes [a, b)."""
        out = []
        if a >= b:
            return out
        i = bisect.bisect_right(self.starts, a) - 1
        while a < b:
            s, e, src, so = self.segs[i]
            hi = min(e, b)
            out.append((hi - a, src, so + (a - s)))
            a = hi
            i += 1
        return out

    def assign(self, a, b, pieces):
        if a >= b:
            return
        i0 = self._cut(a)
        i1 = self._cut(b)
        new, p = [], a
        for ln, src, so in pieces:
            if ln <= 0:
                continue
            if new and new[-1][2] is src and new[-1][3] + (new[-1][1] - new[-1][0]) == so:
                s, _, _, o = new[-1]
                new[-1] = (s, p + ln, src, o)
            else:
                new.append((p, p + ln, src, so))
            p += ln
        assert p == b, "assigned %d bytes to a slice of %d" % (p - a, b - a)
        self.segs[i0:i1] = new
        self.starts[i0:i1] = [x[0] for x in new]
        self._merge_at(i0 + len(new))
        self._merge_at(i0)

    def __getitem__(self, sl):
        a, b = _bounds(sl, self.n)
        return VView(self, a, b)

    def __setitem__(self, sl, val):
        a, b = _bounds(sl, self.n)
        if isinstance(val, VView):
            self.assign(a, b, val.arr.pieces(val.a, val.b))
        elif isinstance(val, VArray):
            self.assign(a, b, val.pieces(0, val.n))
        else:
            self.assign(a, b, [(b - a, Literal(np.asarray(val, np.uint8).reshape(-1)), 0)])

    def materialize(self, a=0, b=None):
        b = self.n if b is None else b
        out = np.empty(b - a, np.uint8)
        p = 0
        for ln, src, so in self.pieces(a, b):
            out[p:p + ln] = src.gen(so, ln)
            p += ln
        return out


class VView:
    """A slice [a, b) of a VArray, as ``arr[a:b]`` is of a numpy array."""
    __slots__ = ("arr", "a", "b")

    def __init__(self, arr, a, b):
        self.arr, self.a, self.b = arr, a, b

    @property
    def size(self):
        return self.b - self.a

    def __len__(self):
        return self.b - self.a

    def __getitem__(self, sl):
        a, b = _bounds(sl, self.b - self.a)
        return VView(self.arr, self.a + a, self.a + b)

    def __setitem__(self, sl, val):
        a, b = _bounds(sl, self.b - self.a)
        self.arr[self.a + a:self.a + b] = val

    def pieces(self):
        return self.arr.pieces(self.a, self.b)

    def materialize(self):
        return self.arr.materialize(self.a, self.b)


def digest_pieces(pieces):
    """orc_digest of the bytes the pieces describe, regenerated in aligned
    pieces of at most CHUNK bytes."""
    total = sum(p[0] for p in pieces)
    tmp = VArray(total)
    tmp.assign(0, total, pieces)
    acc = 0
    for a in range(0, total, CHUNK):
        b = min(total, a + CHUNK)
        acc = (acc + core.digest_at(tmp.materialize(a, b), a // 8)) & M64
    return acc


_POOL = None


def pool():
    global _POOL
    if _POOL is None:
        _POOL = ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2))
    return _POOL


class VersionProcess(Process):
    """Process whose memory, staging and images are VArrays.  The arena
    starts as the word stream of ``arena_key`` (the harness fill of the
    whole arena, word j counted from the arena's first byte)."""

    def __init__(self, va0, buf_off, buf_size, arena_key, seed, arena_bytes=None):
        off = np.asarray(buf_off, np.uint64)
        size = np.asarray(buf_size, np.uint64)
        n = arena_bytes if arena_bytes is not None else (
            int(off[-1]) + int(size[-1]) if len(off) else 0)
        super().__init__(va0, off, size, VArray(n, Words(arena_key), 0), seed)
        self._dig = {}                      # piece tuple -> Future of its digest

    def new_bytes(self, n):
        return VArray(int(n))

    def _key(self, i):
        # the sources themselves (interned word streams, literal objects) key
        # the cache, so a key keeps its sources alive and cannot be reused
        o, s = int(self.off[i]), int(self.size[i])
        return tuple(self.mem.pieces(o, o + s)), o, s

    def _future(self, i):
        key, o, s = self._key(i)
        f = self._dig.get(key)
        if f is None:
            f = pool().submit(digest_pieces, self.mem.pieces(o, o + s))
            self._dig[key] = f
        return f

    def read_digests(self, reads):
        fs = [self._future(int(r)) for r in reads]
        return [f.result() for f in fs]

    def fill(self, w, s_k):
        o, s = int(self.off[w]), int(self.size[w])
        self.mem.assign(o, o + s, [(s, Words(core.mutator_key(s_k, int(w))), 0)])
        self._future(int(w))               # its digest is likely read soon

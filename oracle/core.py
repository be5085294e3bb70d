"""ctypes binding of the C oracle (phos_oracle.c) -- TEST INFRASTRUCTURE ONLY.

Every function here is a thin marshalling wrapper; the arithmetic is in the
C file, written as plain linear scans (Section 4.1 speculation and runtime
validation) and byte loops (harness digest / mutator).

Pins (tests/test_oracle_pins.py):
  speculate  - generator ground truth, brute force over every address of a
               small VA window, struct-chunk and one-past-end special cases
  validate   - brute force over a 64 KiB VA window x {load, store} x widths,
               generator ground-truth labels, closed-form special cases
  digest     - published SplitMix64 outputs on hand-built words (pins the
               word-index term), zero padding of the tail
  stray      - published SplitMix64 outputs
  mutator    - SplitMix64 reference outputs (published test vector)
"""
import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "phos_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

u64p = ctypes.POINTER(ctypes.c_uint64)
u32p = ctypes.POINTER(ctypes.c_uint32)
u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force=False):
    """Compile phos_oracle.c with gcc into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-shared", "-fPIC",
                               "-o", _LIB, _SRC])
    return _LIB


_OMP_SRC = os.path.join(_HERE, "oracle_omp.c")
_OMP_LIB = os.path.join(_HERE, "liboracle_omp.so")
_omp = None


def build_omp(force=False):
    """Compile the all-core timing driver (oracle_omp.c + phos_oracle.c,
    OpenMP) into oracle/liboracle_omp.so; used only to time the baseline."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_OMP_SRC))
    if force or not os.path.exists(_OMP_LIB) or os.path.getmtime(_OMP_LIB) < newest:
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-fopenmp", "-shared",
                               "-fPIC", "-o", _OMP_LIB, _OMP_SRC, _SRC])
    return _OMP_LIB


def omp_lib():
    global _omp
    if _omp is None:
        build_omp()
        L = ctypes.CDLL(_OMP_LIB)
        L.orc_threads.restype = ctypes.c_int
        L.orc_validate_omp.restype = ctypes.c_int
        L.orc_validate_omp.argtypes = [u64p, u64p, u8p, ctypes.c_uint32, u64p, ctypes.c_uint64,
                                       ctypes.c_uint32, u32p, u64p, u32p, u32p]
        L.orc_memcpy_omp.restype = None
        L.orc_memcpy_omp.argtypes = [u8p, u8p, ctypes.c_uint64]
        _omp = L
    return _omp


def omp_threads():
    return int(omp_lib().orc_threads())


def validate_omp(base, size, perm, trace, w):
    """orc_validate run on every host thread over word-aligned ranges of the
    trace (timing only; results equal validate's, without the index list)."""
    base, size = _u64(base), _u64(size)
    perm = np.ascontiguousarray(perm, np.uint8)
    trace = _u64(trace)
    n, N = len(base), len(trace)
    bitmap = np.zeros(max((N + 31) // 32, 1), np.uint32)
    count = np.zeros(3, np.uint64)
    victim = np.zeros(max((n + 31) // 32, 1), np.uint32)
    victim_st = np.zeros(max((n + 31) // 32, 1), np.uint32)
    omp_lib().orc_validate_omp(_p(base, u64p), _p(size, u64p), _p(perm, u8p), n,
                               _p(trace, u64p), N, w, _p(bitmap, u32p), _p(count, u64p),
                               _p(victim, u32p), _p(victim_st, u32p))
    nv = (n + 31) // 32
    return bitmap[:(N + 31) // 32], count, victim[:nv], victim_st[:nv]


def memcpy_omp(dst, src):
    assert dst.dtype == np.uint8 and src.dtype == np.uint8 and dst.size == src.size
    omp_lib().orc_memcpy_omp(_p(dst, u8p), _p(src, u8p), src.size)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_mix64.restype = ctypes.c_uint64
        L.orc_mix64.argtypes = [ctypes.c_uint64]
        L.orc_sm.restype = ctypes.c_uint64
        L.orc_sm.argtypes = [ctypes.c_uint64]
        L.orc_table_check.restype = ctypes.c_int
        L.orc_table_check.argtypes = [u64p, u64p, ctypes.c_uint32]
        L.orc_speculate.restype = None
        L.orc_speculate.argtypes = [u64p, u64p, ctypes.c_uint32,
                                    ctypes.POINTER(ctypes.c_void_p), u32p, u8p,
                                    ctypes.c_uint32, u8p]
        L.orc_speculate_region.restype = None
        L.orc_speculate_region.argtypes = [u64p, u64p, ctypes.c_uint32, ctypes.c_uint64,
                                           ctypes.c_uint64, ctypes.c_uint8, u8p]
        L.orc_validate.restype = ctypes.c_int
        L.orc_validate.argtypes = [u64p, u64p, u8p, ctypes.c_uint32, u64p, ctypes.c_uint64,
                                   ctypes.c_uint32, u32p, u64p, u32p, u32p, u64p,
                                   ctypes.c_uint64]
        L.orc_digest.restype = ctypes.c_uint64
        L.orc_digest.argtypes = [u8p, ctypes.c_uint64]
        L.orc_mutator_seed.restype = ctypes.c_uint64
        L.orc_mutator_seed.argtypes = [ctypes.c_uint64, ctypes.c_uint64, u64p, ctypes.c_uint32]
        L.orc_mutator_fill.restype = None
        L.orc_mutator_fill.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
        L.orc_digest_at.restype = ctypes.c_uint64
        L.orc_digest_at.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64]
        L.orc_words.restype = None
        L.orc_words.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        L.orc_mutator_key.restype = ctypes.c_uint64
        L.orc_mutator_key.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
        L.orc_stray_value.restype = ctypes.c_uint32
        L.orc_stray_value.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def mix64(z):
    return int(lib().orc_mix64(z & 0xFFFFFFFFFFFFFFFF))


def sm(x):
    return int(lib().orc_sm(x & 0xFFFFFFFFFFFFFFFF))


def table_check(base, size):
    base, size = _u64(base), _u64(size)
    return int(lib().orc_table_check(_p(base, u64p), _p(size, u64p), len(base)))


def speculate(base, size, args, kinds, perm=None):
    """Section 4.1 / Section 6 argument-based speculation.

    args: list of ``bytes`` (each argument's raw little-endian bytes);
    kinds: 0 scalar, 1 const pointer, 2 mutable pointer, 3 opaque struct.
    Returns u8 perm[n] (OR-accumulated onto ``perm`` if given)."""
    base, size = _u64(base), _u64(size)
    n = len(base)
    out = np.zeros(n, np.uint8) if perm is None else perm
    nargs = len(args)
    bufs = [ctypes.create_string_buffer(bytes(a), max(len(a), 1)) for a in args]
    argv = (ctypes.c_void_p * max(nargs, 1))(*[ctypes.cast(b, ctypes.c_void_p) for b in bufs])
    asz = np.array([len(a) for a in args], np.uint32)
    kd = np.array(kinds, np.uint8)
    lib().orc_speculate(_p(base, u64p), _p(size, u64p), n, argv,
                        _p(asz, u32p) if nargs else None,
                        _p(kd, u8p) if nargs else None, nargs, _p(out, u8p))
    return out


def speculate_region(base, size, addr, length, p, perm):
    """Section 4.1 type-1 rule: a memory move writing [addr, addr+len)."""
    base, size = _u64(base), _u64(size)
    lib().orc_speculate_region(_p(base, u64p), _p(size, u64p), len(base), addr, length, p,
                               _p(perm, u8p))
    return perm


class ValidateResult:
    __slots__ = ("bitmap", "count", "victim", "victim_st", "idx", "malformed")

    def __init__(self, bitmap, count, victim, victim_st, idx, malformed):
        self.bitmap, self.count, self.victim, self.victim_st, self.idx, self.malformed = \
            bitmap, count, victim, victim_st, idx, malformed


def validate(base, size, perm, trace, w, idx_cap=0):
    """Section 4.1 runtime validation (linear scan per record)."""
    base, size = _u64(base), _u64(size)
    perm = np.ascontiguousarray(perm, np.uint8)
    trace = _u64(trace)
    n, N = len(base), len(trace)
    bitmap = np.zeros(max((N + 31) // 32, 1), np.uint32)
    count = np.zeros(3, np.uint64)
    victim = np.zeros(max((n + 31) // 32, 1), np.uint32)
    victim_st = np.zeros(max((n + 31) // 32, 1), np.uint32)
    idx = np.zeros(max(idx_cap, 1), np.uint64)
    m = lib().orc_validate(_p(base, u64p), _p(size, u64p), _p(perm, u8p), n,
                           _p(trace, u64p), N, w, _p(bitmap, u32p), _p(count, u64p),
                           _p(victim, u32p), _p(victim_st, u32p),
                           _p(idx, u64p) if idx_cap else None, idx_cap)
    nidx = min(int(count[0]), idx_cap)
    nv = (n + 31) // 32
    return ValidateResult(bitmap[:(N + 31) // 32], count, victim[:nv], victim_st[:nv],
                          idx[:nidx].copy(), bool(m))


def digest(buf):
    """Harness digest of a byte array (order-independent sum)."""
    b = np.ascontiguousarray(buf, np.uint8)
    return int(lib().orc_digest(_p(b, u8p), b.size))


def digest_at(buf, j0):
    """Partial digest of a piece starting at word j0 of its buffer."""
    b = np.ascontiguousarray(buf, np.uint8)
    return int(lib().orc_digest_at(_p(b, u8p), b.size, j0 & 0xFFFFFFFFFFFFFFFF))


def words(length, key, byte_off=0):
    """Bytes [byte_off, byte_off + length) of the word stream sm(key ^ j)."""
    out = np.empty(int(length), np.uint8)
    lib().orc_words(_p(out, u8p), out.size, key & 0xFFFFFFFFFFFFFFFF, int(byte_off))
    return out


def mutator_seed(seed, k, read_digests):
    d = _u64(read_digests) if len(read_digests) else np.zeros(1, np.uint64)
    return int(lib().orc_mutator_seed(seed, k, _p(d, u64p), len(read_digests)))


def mutator_fill(view, s_k, w):
    """Fill a writable uint8 numpy view in place (harness mutator)."""
    assert view.flags["C_CONTIGUOUS"] and view.dtype == np.uint8
    lib().orc_mutator_fill(_p(view, u8p), view.size, s_k, w)


def mutator_key(s_k, w):
    """Key of the word stream the mutator writes into buffer w."""
    return int(lib().orc_mutator_key(s_k & 0xFFFFFFFFFFFFFFFF, int(w)))


def stray_value(seed, k, r):
    return int(lib().orc_stray_value(seed, k, r))

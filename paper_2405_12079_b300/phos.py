"""ctypes binding of libphos.so -- argument marshalling only.

Every function forwards to the C entry point of the same name declared in
include/phos.h (and include/phos_harness.h); every step of the data plane
runs in the library's CUDA kernels or its C++ control plane.  Pointers are
plain integers (``tensor.data_ptr()``), streams are ``cudaStream_t`` values
(``torch.cuda.current_stream().cuda_stream``).  If the library is missing
the import of any function raises: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libphos.so")

PHOS_OK, PHOS_EINVAL, PHOS_ENOMEM, PHOS_EBUDGET, PHOS_ECUDA = 0, 1, 2, 3, 4
PHOS_ETIMEDOUT, PHOS_ECORRUPT, PHOS_EMISSPEC = 5, 6, 7
PERM_NONE, PERM_R, PERM_W, PERM_RW = 0, 1, 2, 3
ARG_SCALAR, ARG_CONST_PTR, ARG_MUT_PTR, ARG_STRUCT = 0, 1, 2, 3
COPY_LIVE_TO_STAGING, COPY_LIVE_TO_IMAGE, COPY_STAGING_TO_IMAGE, COPY_IMAGE_TO_LIVE = 1, 2, 3, 4
COPY_MARK_PRESENT = 0x100
REC_STORE = 1 << 63

COPY_DTYPE = np.dtype([("src_off", "<u8"), ("dst_off", "<u8"), ("len", "<u8"),
                       ("buf", "<u4"), ("flags", "<u4")])
BUF_DTYPE = np.dtype([("base", "<u8"), ("size", "<u8")])

_c = ctypes
_u64, _u32, _u8, _i32, _vp = _c.c_uint64, _c.c_uint32, _c.c_uint8, _c.c_int32, _c.c_void_p
_P = _c.POINTER

# name -> (restype, argtypes)
_SIGS = {
    "phos_last_error": (_c.c_char_p, []),
    "phos_status_name": (_c.c_char_p, [_i32]),
    "phos_launch_count": (_u64, []),
    "phos_table_create": (_i32, [_vp, _u32, _P(_vp)]),
    "phos_table_destroy": (_i32, [_vp]),
    "phos_table_size": (_u32, [_vp]),
    "phos_speculate": (_i32, [_vp, _P(_vp), _vp, _vp, _u32, _vp]),
    "phos_speculate_region": (_i32, [_vp, _u64, _u64, _u8, _vp]),
    "phos_validate": (_i32, [_vp, _vp, _vp, _u64, _u32, _vp, _vp, _vp, _vp, _vp, _u64, _vp, _vp]),
    "phos_cow_copy": (_i32, [_vp, _vp, _u32, _vp, _u64, _vp, _vp]),
    "phos_recopy": (_i32, [_vp, _vp, _u32, _vp, _u64, _vp, _vp]),
    "phos_restore_on_demand": (_i32, [_vp, _vp, _u32, _vp, _u64, _vp, _vp, _vp]),
    "phos_copy": (_i32, [_vp, _vp, _u32, _vp, _u64, _vp, _u64, _vp, _vp, _vp]),
    "phos_copy_config": (_i32, [_u64, _u32]),
    "phos_validate_config": (_i32, [_u32]),
    "phos_validate_grid": (_i32, [_u32]),
    "phos_validate_wait_limit": (_i32, [_u32]),
    "phos_host_copy_config": (_i32, [_u64]),
    "phos_copier_window": (_i32, [_u64]),
    "phos_ckpt_frequency": (_i32, [_c.c_double, _c.c_double, _c.c_double, _c.c_double,
                                   _c.c_double, _P(_c.c_double), _P(_c.c_double)]),
    "phos_validate_noalloc": (_i32, [_vp, _vp, _vp, _u64, _u32, _vp, _vp, _vp, _vp, _vp, _u64,
                                      _vp, _vp]),
    "phos_image_bytes": (_u64, [_vp]),
    "phos_image_manifest": (_i32, [_vp, _vp, _u64, _vp, _vp]),
    "phos_image_offsets": (_i32, [_vp, _vp]),
    "phos_harness_digest": (_i32, [_vp, _vp, _u32, _vp, _vp]),
    "phos_harness_mutate": (_i32, [_vp, _u64, _u64, _vp, _u32, _vp, _u32, _vp, _u32, _vp]),
    "phos_harness_drive_ckpt": (_i32, [_vp, _vp, _u64, _u64, _vp, _u32, _vp, _P(_u32)]),
    "phos_harness_fill": (_i32, [_u64, _u64, _u64, _vp]),
    "phos_harness_table_rebind": (_i32, [_vp, _i32, _P(_i32)]),
    "phos_harness_table_scratch": (_i32, [_vp, _P(_u64)]),
    "phos_harness_validate_rounds": (_i32, [_vp, _vp, _u32, _u32, _u32, _vp, _vp, _vp, _vp, _vp,
                                            _vp]),
    "phos_harness_rounds_scratch": (_i32, [_vp, _P(_u64), _P(_u32)]),
    "phos_plan_create": (_i32, [_vp, _u32, _P(_vp)]),
    "phos_plan_launch": (_i32, [_vp, _vp]),
    "phos_plan_set_tile": (_i32, [_vp, _u64]),
    "phos_plan_autotune": (_i32, [_vp, _vp, _P(_u64), _P(_c.c_float)]),
    "phos_plan_info": (_i32, [_vp, _P(_u64), _P(_u64), _P(_u64), _P(_u32)]),
    "phos_plan_destroy": (_i32, [_vp]),
    "phos_server_start": (_i32, [_vp, _P(_vp)]),
    "phos_server_submit": (_i32, [_vp, _vp, _P(_u64)]),
    "phos_server_poll": (_i32, [_vp, _u64, _vp]),
    "phos_server_cancel": (_i32, [_vp, _u64]),
    "phos_server_drain": (_i32, [_vp, _u32]),
    "phos_server_stop": (_i32, [_vp]),
    "phos_speculate_device": (_i32, [_vp, _vp, _vp, _vp, _u32, _vp, _vp, _vp]),
    "phos_server_app_copy": (_i32, [_vp, _vp, _vp, _u64, _vp]),
    "phos_server_stats": (_i32, [_vp, _vp]),
    "phos_ckpt_begin": (_i32, [_vp, _vp, _vp, _P(_vp)]),
    "phos_ckpt_advance": (_i32, [_vp, _u64, _P(_c.c_int)]),
    "phos_ckpt_before_kernel_dev": (_i32, [_vp, _vp]),
    "phos_restore_before_kernel_dev": (_i32, [_vp, _vp]),
    "phos_ckpt_before_kernel": (_i32, [_vp, _vp]),
    "phos_ckpt_after_kernel": (_i32, [_vp, _vp, _u64, _P(_c.c_int)]),
    "phos_ckpt_finish": (_i32, [_vp]),
    "phos_ckpt_begin_pass": (_i32, [_vp, _P(_u64)]),
    "phos_ckpt_stats": (_i32, [_vp, _vp]),
    "phos_ckpt_log": (_i32, [_vp, _u32, _vp, _u64, _P(_u64)]),
    "phos_ckpt_end": (_i32, [_vp]),
    "phos_restore_begin": (_i32, [_vp, _vp, _vp, _P(_vp)]),
    "phos_restore_advance": (_i32, [_vp, _u64, _P(_c.c_int)]),
    "phos_restore_before_kernel": (_i32, [_vp, _vp]),
    "phos_restore_after_kernel": (_i32, [_vp, _vp, _u64, _P(_c.c_int)]),
    "phos_restore_finish": (_i32, [_vp]),
    "phos_restore_stats": (_i32, [_vp, _vp]),
    "phos_restore_log": (_i32, [_vp, _u32, _vp, _u64, _P(_u64)]),
    "phos_restore_end": (_i32, [_vp]),
}

CKPT_COW, CKPT_RECOPY = 1, 2
CKPT_NO_SYNC = 0x100
CKPT_CONCURRENT = 0x200
CKPT_DEVICE = 0x400
CKPT_DEFER = 0x800
RESTORE_ONDEMAND_FIRST = 0x1000


REQ_CHECKPOINT, REQ_RESTORE = 1, 2
SERVER_APP_PRIORITY = 1


class ServerDesc(_c.Structure):
    _fields_ = [("max_slots", _u32), ("flags", _u32), ("d_staging", _vp),
                ("staging_bytes", _u64), ("chunk", _u64), ("dma_min", _u64), ("window", _u64)]


class ServerStats(_c.Structure):
    _fields_ = [("app_copies", _u64), ("app_bytes", _u64), ("paused_turns", _u64),
                ("batches", _u64), ("cancelled", _u64)]


class Request(_c.Structure):
    _fields_ = [("kind", _u32), ("reserved", _u32), ("table", _vp), ("host", _vp),
                ("host_bytes", _u64)]


class Result(_c.Structure):
    _fields_ = [("state", _u32), ("status", _i32), ("bytes", _u64), ("t_submit_ns", _u64),
                ("t_admit_ns", _u64), ("t_done_ns", _u64)]


class PlanItem(_c.Structure):
    _fields_ = [("table", _vp), ("d_perm", _vp), ("d_trace", _vp), ("n_rec", _u64),
                ("access_bytes", _u32), ("n_copy", _u32), ("d_bitmap", _vp), ("d_count", _vp),
                ("d_victim", _vp), ("d_victim_st", _vp), ("d_list", _vp), ("staging", _vp),
                ("staging_bytes", _u64), ("image", _vp), ("image_bytes", _u64)]


class CkptDesc(_c.Structure):
    _fields_ = [("mode", _u32), ("access_bytes", _u32), ("chunk", _u64),
                ("d_staging", _vp), ("staging_bytes", _u64), ("image", _vp),
                ("image_bytes", _u64)]


class CkptStats(_c.Structure):
    _fields_ = [("kernels", _u64), ("copier_bytes", _u64), ("cow_bytes", _u64),
                ("direct_bytes", _u64), ("recopy_bytes", _u64), ("validated", _u64),
                ("violations", _u64), ("misspec_round", _c.c_int64), ("done", _u32),
                ("dirty", _u32), ("passes", _u64)]


class RestoreDesc(_c.Structure):
    _fields_ = [("access_bytes", _u32), ("flags", _u32), ("chunk", _u64), ("image", _vp),
                ("image_bytes", _u64), ("d_present", _vp), ("d_manifest", _vp)]


class RestoreStats(_c.Structure):
    _fields_ = [("kernels", _u64), ("copier_bytes", _u64), ("ondemand_bytes", _u64),
                ("validated", _u64), ("violations", _u64), ("misspec_round", _c.c_int64),
                ("done", _u32), ("corrupt_buf", _i32)]

_lib = None


class PhosError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (code, msg))
        self.code = code


def lib():
    """Load libphos.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libphos.so not found at %s; build it with "
                              "`python -m paper_2405_12079_b300.build`" % LIB_PATH)
        L = _c.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def launch_count():
    return int(lib().phos_launch_count())


def exported_symbols():
    return [n for n in _SIGS if getattr(lib(), n, None) is not None]


def check(code, what=""):
    if code != PHOS_OK:
        msg = lib().phos_last_error().decode(errors="replace")
        raise PhosError(code, (what + ": " if what else "") + msg)
    return code


def _np_ptr(a):
    return a.ctypes.data if a is not None and a.size else None


class Table:
    """Device-resident buffer table (phos_table_create)."""

    def __init__(self, bases, sizes):
        bufs = np.zeros(len(bases), BUF_DTYPE)
        bufs["base"] = np.asarray(bases, np.uint64)
        bufs["size"] = np.asarray(sizes, np.uint64)
        self._bufs = bufs
        h = _vp()
        check(lib().phos_table_create(_np_ptr(bufs), len(bufs), _c.byref(h)), "table_create")
        self.handle = h.value
        self.n = len(bufs)

    def close(self):
        if self.handle:
            lib().phos_table_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def image_bytes(self):
        return int(lib().phos_image_bytes(self.handle))

    def image_offsets(self):
        out = np.zeros(max(self.n, 1), np.uint64)
        check(lib().phos_image_offsets(self.handle, out.ctypes.data), "image_offsets")
        return out[:self.n]


def speculate(table, args, kinds, perm=None):
    """Host-side speculation; args: list of bytes objects."""
    n = table.n
    out = np.zeros(max(n, 1), np.uint8) if perm is None else perm
    nargs = len(args)
    bufs = [_c.create_string_buffer(bytes(a), max(len(a), 1)) for a in args]
    argv = (_vp * max(nargs, 1))(*[_c.cast(b, _vp) for b in bufs])
    asz = np.array([len(a) for a in args] or [0], np.uint32)
    kd = np.array(list(kinds) or [0], np.uint8)
    check(lib().phos_speculate(table.handle, argv, asz.ctypes.data, kd.ctypes.data, nargs,
                               out.ctypes.data), "speculate")
    return out[:n] if perm is None else out


def flatten_launch_args(launches):
    """Argument words for phos_speculate_device: launches is a list of
    (args, kinds) as for speculate().  A pointer argument gives its first 8
    bytes (zero-extended), a struct each full 8-byte chunk, a scalar
    nothing.  Returns (u64 words, u8 kinds, u64 offsets[n_launch + 1])."""
    words, wk, off = [], [], [0]
    for args, kinds in launches:
        for a, k in zip(args, kinds):
            a = bytes(a)
            if k == ARG_STRUCT:
                for o in range(0, len(a) - 7, 8):
                    words.append(int.from_bytes(a[o:o + 8], "little"))
                    wk.append(k)
            elif k != ARG_SCALAR:
                words.append(int.from_bytes(a[:8].ljust(8, b"\0"), "little"))
                wk.append(k)
        off.append(len(words))
    return (np.array(words, np.uint64), np.array(wk, np.uint8), np.array(off, np.uint64))


def speculate_device(table, d_words, d_kind, d_off, n_launch, d_perm, d_status=None,
                     stream=None):
    """phos_speculate_device with integer device pointers."""
    return check(lib().phos_speculate_device(table.handle, d_words, d_kind, d_off, n_launch,
                                             d_perm, d_status, stream), "speculate_device")


def speculate_region(table, addr, length, perm_bits, perm):
    check(lib().phos_speculate_region(table.handle, addr, length, perm_bits, perm.ctypes.data),
          "speculate_region")
    return perm


def validate(table, d_perm, d_trace, n_rec, access_bytes, d_bitmap, d_count, d_victim=None,
             d_victim_st=None, d_idx=None, idx_cap=0, d_status=None, stream=None):
    """phos_validate with integer device pointers."""
    return check(lib().phos_validate(table.handle, d_perm, d_trace, n_rec, access_bytes,
                                     d_bitmap, d_count, d_victim, d_victim_st, d_idx, idx_cap,
                                     d_status, stream), "validate")


def validate_noalloc(table, d_perm, d_trace, n_rec, access_bytes, d_bitmap, d_count,
                     d_victim=None, d_victim_st=None, d_idx=None, idx_cap=0, d_status=None,
                     stream=None):
    """phos_validate_noalloc: the same validation, no device allocation."""
    return check(lib().phos_validate_noalloc(table.handle, d_perm, d_trace, n_rec, access_bytes,
                                             d_bitmap, d_count, d_victim, d_victim_st, d_idx,
                                             idx_cap, d_status, stream), "validate_noalloc")


def cow_copy(table, d_list, n, d_staging, staging_bytes, d_status=None, stream=None):
    return check(lib().phos_cow_copy(table.handle, d_list, n, d_staging, staging_bytes,
                                     d_status, stream), "cow_copy")


def recopy(table, d_list, n, image, image_bytes, d_status=None, stream=None):
    return check(lib().phos_recopy(table.handle, d_list, n, image, image_bytes, d_status,
                                   stream), "recopy")


def restore_on_demand(table, d_list, n, image, image_bytes, d_present, d_status=None,
                      stream=None):
    return check(lib().phos_restore_on_demand(table.handle, d_list, n, image, image_bytes,
                                              d_present, d_status, stream), "restore_on_demand")


def copy(table, d_list, n, d_staging=None, staging_bytes=0, image=None, image_bytes=0,
         d_present=None, d_status=None, stream=None):
    return check(lib().phos_copy(table.handle, d_list, n, d_staging, staging_bytes, image,
                                 image_bytes, d_present, d_status, stream), "copy")


def validate_config(variant=0):
    return check(lib().phos_validate_config(variant), "validate_config")


def ckpt_frequency(n_gpus, fail_per_hour, overhead_h, restore_h, hours):
    """Appendix A.1: (f*, wasted GPU hours at f*)."""
    f, w = _c.c_double(), _c.c_double()
    check(lib().phos_ckpt_frequency(n_gpus, fail_per_hour, overhead_h, restore_h, hours,
                                    _c.byref(f), _c.byref(w)), "ckpt_frequency")
    return f.value, w.value


def validate_grid(ctas=0):
    return check(lib().phos_validate_grid(ctas), "validate_grid")


def validate_wait_limit(probes=1 << 24):
    return check(lib().phos_validate_wait_limit(probes), "validate_wait_limit")


HOST_COPY_DEFAULT = 256 << 10       # the library's default DMA threshold


def host_copy_config(dma_min_bytes=0):
    return check(lib().phos_host_copy_config(dma_min_bytes), "host_copy_config")


def copy_config(tile_bytes=0, ctas_per_sm=0):
    return check(lib().phos_copy_config(tile_bytes, ctas_per_sm), "copy_config")


def copier_window(nbytes=0):
    """phos_copier_window: bound the copier bytes in flight (0 = none)."""
    return check(lib().phos_copier_window(nbytes), "copier_window")


def harness_digest(ptrs, lens, d_out, stream=None):
    p = np.ascontiguousarray(ptrs, np.uint64)
    ln = np.ascontiguousarray(lens, np.uint64)
    return check(lib().phos_harness_digest(_np_ptr(p), _np_ptr(ln), len(p), d_out, stream),
                 "harness_digest")


def harness_mutate(table, seed, k, reads, writes, d_strays=None, ns=0, stream=None):
    r = np.ascontiguousarray(reads, np.uint32)
    w = np.ascontiguousarray(writes, np.uint32)
    return check(lib().phos_harness_mutate(table.handle, seed & (2**64 - 1), k, _np_ptr(r),
                                           len(r), _np_ptr(w), len(w), d_strays, ns, stream),
                 "harness_mutate")


class HarnessKernel(_c.Structure):
    _fields_ = [("args", _vp), ("arg_size", _vp), ("kind", _vp), ("nargs", _u32),
                ("nr", _u32), ("reads", _vp), ("writes", _vp), ("nw", _u32), ("ns", _u32),
                ("d_strays", _vp), ("d_trace", _vp), ("n_rec", _u64)]


def harness_drive_ckpt(ckpt, table, seed, quota, kernels, stream=None):
    """phos_harness_drive_ckpt over an array of HarnessKernel; returns the
    number of rounds run."""
    n = _u32()
    check(lib().phos_harness_drive_ckpt(ckpt.h, table.handle, seed & (2**64 - 1), quota,
                                        _c.cast(kernels, _vp), len(kernels), stream,
                                        _c.byref(n)), "harness_drive_ckpt")
    return int(n.value)


def image_manifest(table, image, image_bytes, d_digest, stream=None):
    """phos_image_manifest: per-buffer digests of a checkpoint image."""
    return check(lib().phos_image_manifest(table.handle, image, image_bytes, d_digest, stream),
                 "image_manifest")


def harness_fill(ptr, length, key, stream=None):
    return check(lib().phos_harness_fill(ptr, length, key & (2**64 - 1), stream), "harness_fill")


def harness_table_rebind(table, device):
    """Test hook: record ``device`` as the table's device; returns the old one."""
    old = _i32()
    check(lib().phos_harness_table_rebind(table.handle, device, _c.byref(old)),
          "harness_table_rebind")
    return int(old.value)


def harness_table_scratch(table):
    """Bytes of the table's growable validation scratch."""
    b = _u64()
    check(lib().phos_harness_table_scratch(table.handle, _c.byref(b)), "harness_table_scratch")
    return int(b.value)


class HarnessRound(_c.Structure):
    _fields_ = [("d_trace", _vp), ("n_rec", _u64), ("d_perm", _vp), ("d_flags", _vp),
                ("round", _c.c_int64)]


def harness_validate_rounds(table, rounds, access_bytes, rule, d_dirty, d_acc, d_flag, d_status,
                            d_scratch, stream=None):
    """phos_harness_validate_rounds over a sequence of (d_trace, n_rec,
    d_perm, d_flags, round) tuples (device pointers as integers)."""
    arr = (HarnessRound * max(len(rounds), 1))()
    for i, (tr, nr, pm, fl, rd) in enumerate(rounds):
        arr[i] = HarnessRound(tr, nr, pm, fl, rd)
    return check(lib().phos_harness_validate_rounds(table.handle, _c.cast(arr, _vp), len(rounds),
                                                    access_bytes, rule, d_dirty, d_acc, d_flag,
                                                    d_status, d_scratch, stream),
                 "harness_validate_rounds")


def harness_rounds_scratch(table):
    """(scratch bytes, most rounds per launch) of deferred validation."""
    b, k = _u64(), _u32()
    check(lib().phos_harness_rounds_scratch(table.handle, _c.byref(b), _c.byref(k)),
          "harness_rounds_scratch")
    return int(b.value), int(k.value)


def _stats_dict(st):
    return {f: getattr(st, f) for f, _ in st._fields_}


def _log(fn, h, kind):
    n = _u64()
    check(fn(h, kind, None, 0, _c.byref(n)), "log")
    out = np.zeros(max(n.value, 1) * 5, np.uint64)
    check(fn(h, kind, out.ctypes.data, n.value, _c.byref(n)), "log")
    return out[:n.value * 5].reshape(-1, 5)


class Checkpoint:
    """One concurrent checkpoint session (phos_ckpt_*)."""

    def __init__(self, table, mode, image, image_bytes, chunk, access_bytes=4, staging=None,
                 staging_bytes=0, stream=None):
        d = CkptDesc(mode, access_bytes, chunk, staging, staging_bytes, image, image_bytes)
        h = _vp()
        check(lib().phos_ckpt_begin(table.handle, _c.byref(d), stream, _c.byref(h)),
              "ckpt_begin")
        self.h = h.value
        self._flag = _c.c_int()

    def advance(self, quota):
        check(lib().phos_ckpt_advance(self.h, quota, _c.byref(self._flag)), "ckpt_advance")
        return bool(self._flag.value)

    def before_kernel(self, perm):
        check(lib().phos_ckpt_before_kernel(self.h, perm.ctypes.data), "ckpt_before_kernel")

    def before_kernel_dev(self, d_perm):
        """CKPT_DEVICE sessions: the round's perm as a device pointer."""
        check(lib().phos_ckpt_before_kernel_dev(self.h, d_perm), "ckpt_before_kernel_dev")

    def after_kernel(self, d_trace, n_rec):
        check(lib().phos_ckpt_after_kernel(self.h, d_trace, n_rec, _c.byref(self._flag)),
              "ckpt_after_kernel")
        return bool(self._flag.value)

    def finish(self):
        check(lib().phos_ckpt_finish(self.h), "ckpt_finish")

    def begin_pass(self):
        b = _u64()
        check(lib().phos_ckpt_begin_pass(self.h, _c.byref(b)), "ckpt_begin_pass")
        return int(b.value)

    def stats(self):
        st = CkptStats()
        check(lib().phos_ckpt_stats(self.h, _c.byref(st)), "ckpt_stats")
        return _stats_dict(st)

    def log(self, kind):
        return _log(lib().phos_ckpt_log, self.h, kind)

    def close(self):
        if self.h:
            lib().phos_ckpt_end(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Restore:
    """One concurrent restore session (phos_restore_*)."""

    def __init__(self, table, image, image_bytes, chunk, access_bytes=4, d_present=None,
                 stream=None, flags=0, d_manifest=None):
        """flags: CKPT_NO_SYNC or CKPT_CONCURRENT (the same bits as for
        checkpoints); d_manifest: device u64[n] from image_manifest, to
        verify every restored buffer."""
        d = RestoreDesc(access_bytes, flags, chunk, image, image_bytes, d_present, d_manifest)
        h = _vp()
        check(lib().phos_restore_begin(table.handle, _c.byref(d), stream, _c.byref(h)),
              "restore_begin")
        self.h = h.value
        self._flag = _c.c_int()

    def advance(self, quota):
        check(lib().phos_restore_advance(self.h, quota, _c.byref(self._flag)),
              "restore_advance")
        return bool(self._flag.value)

    def before_kernel(self, perm):
        check(lib().phos_restore_before_kernel(self.h, perm.ctypes.data),
              "restore_before_kernel")

    def before_kernel_dev(self, d_perm):
        """CKPT_DEVICE sessions: the round's perm as a device pointer."""
        check(lib().phos_restore_before_kernel_dev(self.h, d_perm), "restore_before_kernel_dev")

    def after_kernel(self, d_trace, n_rec):
        check(lib().phos_restore_after_kernel(self.h, d_trace, n_rec, _c.byref(self._flag)),
              "restore_after_kernel")
        return bool(self._flag.value)

    def finish(self):
        check(lib().phos_restore_finish(self.h), "restore_finish")

    def stats(self):
        st = RestoreStats()
        check(lib().phos_restore_stats(self.h, _c.byref(st)), "restore_stats")
        return _stats_dict(st)

    def log(self, kind):
        return _log(lib().phos_restore_log, self.h, kind)

    def close(self):
        if self.h:
            lib().phos_restore_end(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Batched plan (phos_plan_*): many items, one persistent graph launch."""

    def __init__(self, items):
        arr = (PlanItem * max(len(items), 1))(*items)
        h = _vp()
        check(lib().phos_plan_create(_c.cast(arr, _vp), len(items), _c.byref(h)), "plan_create")
        self.h = h.value

    def launch(self, stream=None):
        check(lib().phos_plan_launch(self.h, stream), "plan_launch")

    def set_tile(self, tile):
        check(lib().phos_plan_set_tile(self.h, tile), "plan_set_tile")

    def autotune(self, stream=None):
        t, ms = _u64(), _c.c_float()
        check(lib().phos_plan_autotune(self.h, stream, _c.byref(t), _c.byref(ms)),
              "plan_autotune")
        return int(t.value), float(ms.value)

    def info(self):
        r, b, t, st = _u64(), _u64(), _u64(), _u32()
        check(lib().phos_plan_info(self.h, _c.byref(r), _c.byref(b), _c.byref(t), _c.byref(st)),
              "plan_info")
        return dict(records=r.value, copy_bytes=b.value, tile=t.value, status=st.value)

    def close(self):
        if self.h:
            lib().phos_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (phos_server_*)."""

    def __init__(self, max_slots, d_staging, staging_bytes, chunk=4 << 20, dma_min=256 << 10,
                 app_priority=False, window=0):
        d = ServerDesc(max_slots, SERVER_APP_PRIORITY if app_priority else 0, d_staging,
                       staging_bytes, chunk, dma_min, window)
        h = _vp()
        check(lib().phos_server_start(_c.byref(d), _c.byref(h)), "server_start")
        self.h = h.value

    def submit(self, kind, table, host, host_bytes):
        r = Request(kind, 0, table.handle, host, host_bytes)
        t = _u64()
        check(lib().phos_server_submit(self.h, _c.byref(r), _c.byref(t)), "server_submit")
        return int(t.value)

    def poll(self, ticket):
        r = Result()
        check(lib().phos_server_poll(self.h, ticket, _c.byref(r)), "server_poll")
        return {f: getattr(r, f) for f, _ in r._fields_}

    def cancel(self, ticket):
        check(lib().phos_server_cancel(self.h, ticket), "server_cancel")

    def drain(self, timeout_ms=600_000):
        check(lib().phos_server_drain(self.h, timeout_ms), "server_drain")

    def app_copy(self, dst, src, nbytes, stream):
        """An application transfer on `stream` that C/R traffic yields to."""
        check(lib().phos_server_app_copy(self.h, dst, src, nbytes, stream), "server_app_copy")

    def stats(self):
        st = ServerStats()
        check(lib().phos_server_stats(self.h, _c.byref(st)), "server_stats")
        return _stats_dict(st)

    def close(self):
        if self.h:
            lib().phos_server_stop(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

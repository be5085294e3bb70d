"""Lockstep drivers that play the application around the C/R sessions.

A ``DeviceProcess`` is one GPU process image: a device arena holding every
buffer, the buffer table, and a sequence of application kernels (the
harness mutator, launch arguments for speculation, access traces resident
in HBM).  ``run_cow`` / ``run_recopy`` / ``run_restore`` perform one
concurrent checkpoint or restore through the library's control plane in
the round order its header defines: copier advance, speculation +
before_kernel, the application kernel, after_kernel (validation).  All data
movement and validation happen in libphos.so; this module only sequences
the calls.
"""
import ctypes
import time

import numpy as np
import torch

from . import phos


class PreparedKernel:
    """A kernel with its launch arguments marshalled once for speculation
    and its trace and stray list resident on the device."""

    def __init__(self, kern, device="cuda"):
        self.kern = kern
        self.nargs = len(kern.args)
        self._bufs = [ctypes.create_string_buffer(bytes(a), max(len(a), 1)) for a in kern.args]
        self.argv = (ctypes.c_void_p * max(self.nargs, 1))(
            *[ctypes.cast(b, ctypes.c_void_p) for b in self._bufs])
        self.asz = np.array([len(a) for a in kern.args] or [0], np.uint32)
        self.kinds = np.array(list(kern.kinds) or [0], np.uint8)
        tr = np.ascontiguousarray(kern.trace, np.uint64)
        self.n_rec = len(tr)
        self.d_trace = torch.from_numpy((tr if len(tr) else np.zeros(2, np.uint64))
                                        .view(np.uint8).copy()).to(device)
        self.reads = np.ascontiguousarray(kern.reads, np.uint32)
        self.writes = np.ascontiguousarray(kern.writes, np.uint32)
        st = np.array(kern.strays, np.uint64).reshape(-1) if kern.strays else np.zeros(2,
                                                                                       np.uint64)
        self.ns = len(kern.strays)
        self.d_strays = torch.from_numpy(st.view(np.uint8).copy()).to(device)

    def speculate(self, table, out):
        out[:] = 0
        phos.check(phos.lib().phos_speculate(table.handle, self.argv, self.asz.ctypes.data,
                                             self.kinds.ctypes.data, self.nargs,
                                             out.ctypes.data), "speculate")
        return out


class DeviceProcess:
    def __init__(self, layout, arena, seed, kernels):
        """arena: CUDA uint8 tensor of layout.arena_bytes (the process's
        memory); kernels: workloads.Kernel list whose addresses are based at
        arena.data_ptr()."""
        self.layout = layout
        self.arena = arena
        self.va0 = arena.data_ptr()
        self.seed = int(seed)
        self.table = phos.Table(layout.base(self.va0), layout.size)
        self.kernels = [PreparedKernel(k, arena.device) for k in kernels]
        self.perm = np.zeros(max(layout.n, 1), np.uint8)
        self.image_bytes = self.table.image_bytes()
        self.img_off = self.table.image_offsets()

    def stream(self):
        return torch.cuda.current_stream().cuda_stream

    def native_kernels(self):
        """The kernels as phos_harness_kernel_t entries for the native
        driver (the PreparedKernel objects keep the memory alive)."""
        arr = (phos.HarnessKernel * max(len(self.kernels), 1))()
        for j, pk in enumerate(self.kernels):
            arr[j] = phos.HarnessKernel(
                ctypes.cast(pk.argv, ctypes.c_void_p), pk.asz.ctypes.data, pk.kinds.ctypes.data,
                pk.nargs, len(pk.reads), pk.reads.ctypes.data if len(pk.reads) else None,
                pk.writes.ctypes.data if len(pk.writes) else None, len(pk.writes), pk.ns,
                pk.d_strays.data_ptr(), pk.d_trace.data_ptr(), pk.n_rec)
        return arr

    def run_kernel(self, k):
        pk = self.kernels[k]
        phos.harness_mutate(self.table, self.seed, k, pk.reads, pk.writes,
                            pk.d_strays.data_ptr(), pk.ns, self.stream())

    @staticmethod
    def _flags(rounds):
        """rounds: "sync" (wait for each validation), "nosync" (rule on the
        device), "concurrent" (nosync, copier on its own stream), "deferred"
        (concurrent, up to 16 rounds validated per launch), "odfirst"
        (restore only: concurrent, each round's on-demand copies before its
        copier move) or "device" (every round's decisions on the device,
        perms from device speculation)."""
        return {"sync": 0, "nosync": phos.CKPT_NO_SYNC,
                "concurrent": phos.CKPT_CONCURRENT,
                "deferred": phos.CKPT_CONCURRENT | phos.CKPT_DEFER,
                "odfirst": phos.CKPT_CONCURRENT | phos.RESTORE_ONDEMAND_FIRST,
                "device": phos.CKPT_DEVICE}[rounds]

    def device_perms(self):
        """Every kernel's speculated permissions, computed on the device in
        one launch (phos_speculate_device): u8 [K][n] device tensor."""
        if getattr(self, "_d_perms", None) is None:
            n = max(self.layout.n, 1)
            launches = [(pk.kern.args, pk.kern.kinds) for pk in self.kernels]
            words, wk, off = phos.flatten_launch_args(launches)
            dev = self.arena.device
            d_w = torch.from_numpy((words if len(words) else np.zeros(1, np.uint64))
                                   .view(np.uint8).copy()).to(dev)
            d_k = torch.from_numpy(wk if len(wk) else np.zeros(1, np.uint8)).to(dev)
            d_o = torch.from_numpy(off.view(np.uint8).copy()).to(dev)
            d_p = torch.zeros(len(self.kernels) * n, dtype=torch.uint8, device=dev)
            phos.speculate_device(self.table, d_w.data_ptr(), d_k.data_ptr(), d_o.data_ptr(),
                                  len(self.kernels), d_p.data_ptr(), None, self.stream())
            self._d_perms = d_p
        return self._d_perms

    def _before(self, sess, k, device):
        pk = self.kernels[k]
        if device:
            n = max(self.layout.n, 1)
            sess.before_kernel_dev(self.device_perms().data_ptr() + k * n)
        else:
            sess.before_kernel(pk.speculate(self.table, self.perm))

    def run_cow(self, image, quota, chunk, staging=None, staging_bytes=0, rounds="sync"):
        """Soft copy-on-write."""
        return self._ckpt(phos.CKPT_COW | self._flags(rounds), image, quota, chunk, staging,
                          staging_bytes)

    def run_recopy(self, image, quota, chunk, max_passes=0, stop_bytes=0, rounds="sync"):
        """Soft recopy; with max_passes > 0, iterative: each time the copier
        finishes a pass, another concurrent pass recopies the dirty set while
        its bytes exceed stop_bytes and keep shrinking."""
        return self._ckpt(phos.CKPT_RECOPY | self._flags(rounds), image, quota, chunk, None, 0,
                          max_passes, stop_bytes)

    def _ckpt(self, mode, image, quota, chunk, staging, staging_bytes, max_passes=0,
              stop_bytes=0, mark=None, finish_times=None, logs=True):
        """One checkpoint session, round by round.  mark(phase) is called as
        each phase of a round is enqueued (copier, cow / dirty_marking,
        app_kernel, validate, finish, end); finish_times receives the host
        time finish took after the device had drained; logs=False returns
        the statistics only."""
        s = self.stream()
        c = phos.Checkpoint(self.table, mode, image.data_ptr(), image.numel(), chunk, 4,
                            staging.data_ptr() if staging is not None else None, staging_bytes, s)
        mark = mark or (lambda name: None)
        pre = "cow" if mode & phos.CKPT_COW else "dirty_marking"
        device = bool(mode & phos.CKPT_DEVICE)
        if device:
            self.device_perms()
        k, misspec = 0, False
        K = len(self.kernels)
        prev, passes = None, 0
        while k < K:
            mark("copier")
            if c.advance(quota):
                db = self.dirty_bytes(c) if max_passes else 0
                if passes < max_passes and db > stop_bytes and (prev is None or db < prev):
                    c.begin_pass()
                    prev, passes = db, passes + 1
                else:
                    break
            pk = self.kernels[k]
            mark(pre)
            self._before(c, k, device)
            mark("app_kernel")
            self.run_kernel(k)
            mark("validate")
            misspec = c.after_kernel(pk.d_trace.data_ptr(), pk.n_rec)
            k += 1
            if misspec:
                break
        mark("finish")
        if finish_times is not None:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        c.finish()
        if finish_times is not None:
            finish_times.append(time.perf_counter() - t0)
        mark("end")
        if not logs:
            st = c.stats()
            c.close()
            return st
        out = dict(stats=c.stats(), cow=c.log(0), copier=c.log(1), dirty=c.log(2)[:, 0],
                   passes=c.log(3), kernels_run=k)
        c.close()
        return out

    def run_native(self, mode, image, quota, chunk, staging=None, staging_bytes=0,
                   rounds="sync"):
        """The same checkpoint rounds through the library's native driver
        (phos_harness_drive_ckpt) instead of this module's loop."""
        s = self.stream()
        c = phos.Checkpoint(self.table, mode | self._flags(rounds), image.data_ptr(),
                            image.numel(), chunk, 4,
                            staging.data_ptr() if staging is not None else None, staging_bytes, s)
        ks = self.native_kernels()
        k = phos.harness_drive_ckpt(c, self.table, self.seed, quota, ks, s)
        c.finish()
        out = dict(stats=c.stats(), cow=c.log(0), copier=c.log(1), dirty=c.log(2)[:, 0],
                   passes=c.log(3), kernels_run=k)
        c.close()
        return out

    def dirty_bytes(self, c):
        d = c.log(2)[:, 0].astype(np.int64)
        return int(self.layout.size[d].sum()) if len(d) else 0

    def run_restore(self, image, quota, chunk, d_present=None, rounds="sync", d_manifest=None):
        """Concurrent restore followed by the rest of the kernels;
        d_manifest: verify every restored buffer against it (finish raises
        PHOS_ECORRUPT on a mismatch)."""
        s = self.stream()
        device = rounds == "device"
        if device:
            self.device_perms()
        r = phos.Restore(self.table, image.data_ptr(), image.numel(), chunk, 4,
                         d_present.data_ptr() if d_present is not None else None, s,
                         self._flags(rounds),
                         d_manifest.data_ptr() if d_manifest is not None else None)
        k = 0
        K = len(self.kernels)
        odf = rounds == "odfirst"
        while k < K:
            if not odf and r.advance(quota):
                break
            pk = self.kernels[k]
            self._before(r, k, device)
            done = odf and r.advance(quota)      # after the round's on-demand copies
            self.run_kernel(k)
            misspec = r.after_kernel(pk.d_trace.data_ptr(), pk.n_rec)
            k += 1
            if misspec or done:
                break
        r.finish()
        if r.stats()["misspec_round"] >= 0:  # rolled back: replay what ran
            for j in range(k):
                self.run_kernel(j)
        during = k
        for j in range(k, K):
            self.run_kernel(j)
        out = dict(stats=r.stats(), ondemand=r.log(0), copier=r.log(1), kernels_during=during)
        r.close()
        return out

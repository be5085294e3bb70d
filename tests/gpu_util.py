"""Shared helpers of the GPU parity tests (test infrastructure)."""
import numpy as np
import torch

from paper_2405_12079_b300 import phos


def dev(a):
    """numpy -> CUDA tensor (bytes preserved)."""
    a = np.ascontiguousarray(a)
    t = torch.from_numpy(a.view(np.uint8).copy()).cuda()
    return t


def host(t, dtype, n=None):
    a = t.cpu().numpy().view(dtype)
    return a if n is None else a[:n]


def stream():
    return torch.cuda.current_stream().cuda_stream


def run_validate(table, perm, trace, w, idx_cap=0, status=None):
    """Call phos_validate on device copies; returns numpy outputs."""
    N, n = len(trace), table.n
    d_perm = dev(np.asarray(perm, np.uint8) if n else np.zeros(1, np.uint8))
    d_tr = dev(np.asarray(trace, np.uint64) if N else np.zeros(2, np.uint64))
    nw = max((N + 31) // 32, 1)
    d_bm = torch.full((nw * 4,), 0xAB, dtype=torch.uint8, device="cuda")
    d_cnt = torch.full((24,), 0xCD, dtype=torch.uint8, device="cuda")
    nv = max((n + 31) // 32, 1)
    d_v = torch.full((nv * 4,), 0xEF, dtype=torch.uint8, device="cuda")
    d_vs = torch.full((nv * 4,), 0xEF, dtype=torch.uint8, device="cuda")
    d_idx = torch.zeros((max(idx_cap, 1) * 8,), dtype=torch.uint8, device="cuda")
    d_st = torch.zeros((4,), dtype=torch.uint8, device="cuda") if status is None else status
    phos.validate(table, d_perm.data_ptr(), d_tr.data_ptr(), N, w, d_bm.data_ptr(),
                  d_cnt.data_ptr(), d_v.data_ptr(), d_vs.data_ptr(),
                  d_idx.data_ptr() if idx_cap else None, idx_cap, d_st.data_ptr(), stream())
    torch.cuda.synchronize()
    return dict(bitmap=host(d_bm, np.uint32, (N + 31) // 32), count=host(d_cnt, np.uint64),
                victim=host(d_v, np.uint32, (n + 31) // 32),
                victim_st=host(d_vs, np.uint32, (n + 31) // 32),
                idx=host(d_idx, np.uint64), status=int(host(d_st, np.uint32)[0]))

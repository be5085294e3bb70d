"""The C-ABI library builds, loads without a GPU and exports every symbol
the public headers declare (no compute calls: no device is needed)."""
import glob
import os
import re

from paper_2405_12079_b300 import build, phos

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(phos_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_declared_symbols():
    build.build()
    L = phos.lib()
    names = declared()
    assert len(names) >= 15
    missing = [n for n in sorted(names) if getattr(L, n, None) is None]
    assert not missing, missing
    # the binding knows the signature of every declared entry point
    assert not (names - set(phos._SIGS)), names - set(phos._SIGS)


def test_host_only_calls_without_gpu():
    """Error paths that never touch the device."""
    L = phos.lib()
    assert L.phos_status_name(phos.PHOS_EMISSPEC) == b"PHOS_EMISSPEC"
    import ctypes
    import numpy as np
    bufs = np.zeros(2, phos.BUF_DTYPE)
    bufs["base"] = [4096, 1000]                    # unsorted
    bufs["size"] = [16, 16]
    h = ctypes.c_void_p()
    assert L.phos_table_create(bufs.ctypes.data, 2, ctypes.byref(h)) == phos.PHOS_EINVAL
    assert b"unsorted" in L.phos_last_error()
    assert L.phos_copy_config(1000, 0) == phos.PHOS_EINVAL


def header_enums():
    """NAME -> value of every enumerator in the public headers."""
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
            for m in re.finditer(r"\b(PHOS_[A-Z0-9_]+)\s*=\s*(0x[0-9a-fA-F]+|\d+)", body):
                out[m.group(1)] = int(m.group(2), 0)
    return out


def test_binding_constants_match_the_header():
    """Every constant the binding defines under a header enumerator's name
    (with or without the PHOS_ prefix) has the header's value."""
    enums = header_enums()
    assert len(enums) >= 25
    checked = 0
    for name, value in enums.items():
        for attr in (name, name[len("PHOS_"):]):
            if hasattr(phos, attr):
                assert getattr(phos, attr) == value, (attr, getattr(phos, attr), value)
                checked += 1
    assert checked >= 20
    assert phos.CKPT_DEFER == enums["PHOS_CKPT_DEFER"]

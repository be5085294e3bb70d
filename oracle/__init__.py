"""Plain CPU oracle for the PhOS data plane -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never imports, links
or calls it, and it imports nothing from the CUDA library: the two share only
the seeded input generators, which hold none of the method's arithmetic.

Contents
  core.py       ctypes binding of phos_oracle.c (speculation, validation,
                digest, mutator) -- plain linear scans and byte loops
  copyeng.py    the copy engine as memcpy over numpy byte arrays
  protocols.py  soft copy-on-write (Section 4.2), soft recopy (Section 4.3)
                and soft on-demand restore (Section 6) as plain sequential
                simulators, plus their stop-the-world counterparts

Parity status per function is listed in each module's header.
"""

"""PhOS data plane on B300 (sm_103a): access validation and the C/R copy engine.

The compute path is the C-ABI library ``libphos.so`` (CUDA kernels plus the
host control plane in C++); ``phos`` is its ctypes binding.  Importing this
package loads nothing; the library is opened on first use and the binding
raises if it is missing -- there is no CPU fallback.
"""

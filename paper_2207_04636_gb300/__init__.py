"""GB300 robust-pseudospectral occ-RI exchange build (arXiv 2207.04636).

The product is libxk.so (include/xk.h): hand-written CUDA for sm_103a behind
a C ABI.  This package holds its sources (csrc/), its build script and a thin
ctypes binding with the same entry points.
"""
from .xk import (Batch, Handle, XKError, admit_release, admit_reserve, admit_state, exchange_energy_noalloc, footprint, isdf_points, kernel_launches, last_error, lib, poll,
                 XK_OK, XK_PENDING, XK_EINVAL, XK_ENOMEM, XK_ETIMEDOUT, XK_ECUDA, XK_EBUSY)

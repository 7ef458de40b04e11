"""GB300-native direct-QPAT propagation library (Javaherian & Holman,
"Direct quantitative photoacoustic tomography for realistic acoustic media").

The compute path is the in-tree CUDA library ``libqpat.so`` (sm_103a, built
by ``build.py``); this package is a thin ctypes binding over its C ABI
(``include/qpat.h``) plus a ``torch.autograd.Function``.  Importing the
bindings fails loudly when the library is missing: there is no CPU fallback.
"""
from .binding import (QpatError, Context, qpat_create, qpat_destroy, qpat_acoustic_forward,
                      qpat_acoustic_adjoint, qpat_da_solve, qpat_forward, qpat_jvp, qpat_vjp,
                      qpat_dot, qpat_sync, qpat_get_sizes, library_path, exported_symbols)

__all__ = ["QpatError", "Context", "qpat_create", "qpat_destroy", "qpat_acoustic_forward",
           "qpat_acoustic_adjoint", "qpat_da_solve", "qpat_forward", "qpat_jvp", "qpat_vjp",
           "qpat_dot", "qpat_sync", "qpat_get_sizes", "library_path", "exported_symbols"]

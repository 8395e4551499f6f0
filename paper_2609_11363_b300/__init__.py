"""Selected inverse on S = pattern(L+D+L^T) from incomplete LDL^T factors, on B300.

Thin Python binding of ``libsinv.so`` (C ABI in ``include/sinv.h``).  It only
marshals arguments: every step of the path runs in the library's CUDA kernels.
PyTorch provides device memory and streams.  There is no CPU fallback: if the
library is missing the import of the binding fails loudly.
"""
from .binding import (  # noqa: F401
    SinvError,
    Handle,
    lib_path,
    load_library,
    PREC,
    lowrank_correct_noalloc,
    LOWRANK_NOALLOC_MAX,
    Mlp,
    MLP_F,
    MLP_H,
)

"""GB300-native exchange hot path of L-ACE (localized Adaptively Compressed Exchange).

Python binding of ``liblace.so`` (C ABI declared in ``include/lace.h``).  The
binding only marshals arguments: every step of the computation runs in the
library's CUDA kernels.  Importing this package does not need a GPU; creating
a :class:`Lace` context or a :class:`Server` does, and fails loudly when the library or a CUDA
device is missing.
"""
from .binding import (  # noqa: F401
    Batch,
    LACE_FP64,
    LACE_MIXED,
    LACE_SYM_AVG,
    LACE_SYM_LOWER,
    LACE_SYM_UPPER,
    Lace,
    LaceError,
    Server,
    exported_symbols,
    library_path,
    load_library,
    probe_peak_rates,
)

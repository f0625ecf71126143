"""GB300-native DC-LNO hot path (Ozaki, Fukuda, Jiang: O(N) divide-conquer with
localized natural orbitals).

The work runs in ``libdclno.so`` (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/dclno.h``).  This package is its thin Python binding:
argument marshalling only.  Importing it fails loudly if the library has not
been built; there is no CPU fallback.
"""
from ._lib import (  # noqa: F401
    DCLNO_FP64, DCLNO_MIXED, LIB_PATH, Context, DclnoError, STATUS_NAMES, exported_symbols, load_library,
    find_mu_noalloc, measure_fp64_peaks,
)

"""GB300-native Lazy stochastic PCA (Wojnowicz et al., arXiv 1709.07175).

The compute path is the CUDA library ``liblspca.so`` (sm_103a) behind the
C-ABI declared in ``include/lspca.h``; ``paper_1709_07175_gb300.lspca`` is
the thin ctypes binding with the same entry-point names.  The library is
loaded on first use and a missing or unloadable library raises
``LspcaLibraryError``: there is no CPU fallback.
"""
from .synthetic import WORKLOADS, Workload  # noqa: F401

"""GB300-native (sm_103a) model-based iterative reconstruction for x-ray
edge-illumination tomography (Modregger et al., arXiv:2202.08627).

The compute path is the CUDA library ``libei.so`` behind a C ABI
(``include/ei.h``); ``paper_2202_08627_gb300.ei`` is its thin ctypes binding.
Importing this package loads nothing; the library is loaded on first use and
the import fails loudly if it has not been built.
"""

__all__ = ["ei", "inputs"]

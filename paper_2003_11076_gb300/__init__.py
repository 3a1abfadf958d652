"""GB300-native semantic light-field EM (Kaveti, Katt & Singh, arXiv 2003.11076).

The compute path lives in hand-written sm_103a CUDA kernels behind the C ABI
declared in ``include/lf.h``; ``paper_2003_11076_gb300.lf`` is the thin Python
binding.  ``paper_2003_11076_gb300.scenes`` renders seeded synthetic inputs.
Submodules are imported lazily so that the scene generator can be used on a
machine without the compiled library.
"""

__all__ = ["lf", "scenes"]

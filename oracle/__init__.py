"""FP64 CPU oracle of the per-pixel light-field EM (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA path.
"""

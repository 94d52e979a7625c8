"""Time-resolved Monte Carlo path tracing on GB300 (arXiv 2510.25660).

The compute path is the C-ABI library ``libmt.so`` (hand-written sm_103a CUDA,
``csrc/``); this package holds its thin ctypes binding (``api``), the build
script (``build``), the launch autotuner (``autotune``) and the seeded scene
generators (``scenes``, inputs only).  Importing the package does not load the
CUDA library; the first call into ``api`` does, and fails loudly if it is
missing.
"""

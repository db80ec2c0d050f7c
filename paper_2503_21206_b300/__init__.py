"""B300-native (sm_103a) GPU search hot path of PilotANN (arxiv 2503.21206).

The search itself runs in hand-written CUDA kernels behind the C-ABI library
``libpilot.so`` (declared in include/pilot.h); ``pilot`` is its thin ctypes
binding.  ``synth`` and ``index_build`` generate the seeded inputs.
"""

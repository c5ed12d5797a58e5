"""GB300-native direct-summation engine for StePS-style compactified N-body runs.

The compute path is libsteps.so (CUDA, sm_103a) behind the C ABI declared in
include/steps.h; ``steps`` is its thin ctypes binding and ``workloads`` builds
seeded synthetic inputs.  Importing the package loads nothing; the first call
into ``steps`` loads the library and fails loudly if it is missing.
"""

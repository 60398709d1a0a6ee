"""GB300 (sm_103a) surfel sampling and progressive blue-noise ordering.

The compute path lives in ``libbs.so`` (CUDA kernels behind a C ABI, declared in
``include/bs.h``); ``paper_1904_08225_gb300.bs`` is its thin ctypes binding.
``workloads`` builds the seeded synthetic meshes the benchmarks and tests use.
"""

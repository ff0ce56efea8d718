"""GB300-native state-vector simulator (JUQCS method, arXiv:1912.03243).

The compute path is the C-ABI library ``libsv`` (CUDA, sm_103a) declared in
``include/sv.h``; ``paper_1912_03243_gb300.sv`` is its thin ctypes binding.
``paper_1912_03243_gb300.circuits`` holds the seeded synthetic circuit
generators shared by the tests and the benchmark.
"""

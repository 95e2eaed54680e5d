"""GB300-native (sm_103a) wavelet-adaptive artificial-compressibility solver.

The compute path is the C-ABI library ``libacm`` (CUDA kernels in ``csrc/``); the Python
binding ``paper_1912_05371_gb300.acm`` only marshals arguments to it.  ``workloads`` holds the
seeded synthetic inputs.
"""

"""GB300-native split-step Crank-Nicolson solver for the spin-1 SO- and
Rabi-coupled Gross-Pitaevskii equation (arXiv:2009.13507).

The compute path is the C-ABI library ``libsgpe.so`` (hand-written sm_103a
CUDA kernels); ``paper_2009_13507_gb300.sgpe`` is its thin ctypes binding.
Importing this package loads nothing; the library is loaded on first use and
raises if it is missing.
"""

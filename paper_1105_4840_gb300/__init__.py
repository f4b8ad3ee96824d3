"""GB300-native parallel step-wise pulling protocol (arXiv 1105.4840).

Submodules
  inputs   seeded synthetic workloads (chain parameters, start state, lambda grids)
  pmf      ctypes binding of the C-ABI library libpmf.so (CUDA, sm_103a)
  build    compiles libpmf.so with nvcc

Importing the package loads nothing; `from paper_1105_4840_gb300 import pmf`
loads the CUDA library and fails loudly if it is missing.
"""

"""GB300-native matrix-free geometric multigrid for node-centred finite-difference
linear elasticity (Runnels et al., arXiv 2001.04789): CUDA kernels for sm_103a
behind a C ABI (``include/elas.h``), with a thin ctypes binding."""

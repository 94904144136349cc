"""GB300-native coupled immersed-boundary lattice-Boltzmann step
(arXiv:1704.04551): hand-written CUDA kernels for sm_103a behind a C ABI
(``include/ibm_lbm.h``), with a thin ctypes binding in ``binding.py``."""

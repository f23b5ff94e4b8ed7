"""GB300 (sm_103a) implementation of the semi-Lagrangian lattice Boltzmann step of
arXiv:2012.05537 with the 45-velocity cubature set, behind the C ABI of include/sllbm.h.

Submodules: ``build`` (nvcc build of libsllbm.so), ``sllbm`` (ctypes binding; imports
torch), ``inputs`` (seeded synthetic workloads; no method arithmetic).
"""

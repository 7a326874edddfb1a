"""Batched Born-Oppenheimer energies and forces of every replica of a
replica-parallel ab initio simulation step (arXiv:1601.02713, Sec. 2) on one
GB300: closed-shell RHF direct SCF with hand-written sm_103a CUDA kernels.

Submodules: `native` (ctypes binding of include/pimdgb.h), `build` (nvcc build
of the CUDA library), `inputs` (seeded synthetic geometries and basis data).
Nothing is imported eagerly so that the package loads without a GPU.
"""

"""B300-native column-generation VMAT optimiser (Men, Romeijn, Jia, Jiang).

Submodules:
  inputs   seeded synthetic planning problems (phantom + D); no method arithmetic
  vmat     ctypes binding of the C-ABI library libvmat.so (the CUDA path)
  autograd torch.autograd.Function over the dose + cost forward and its adjoint
  build    nvcc/gcc build of the native libraries
The CUDA library is loaded lazily by `paper_1005_4396_b300.vmat`.
"""
__version__ = "0.1.0"

"""GB300-native (sm_103a) hot path of stochastic multi-dimensional deconvolution (arXiv 2202.04486).

The CUDA kernels live in csrc/ and are built into libsmdd_gb300.so (a C ABI, include/smdd.h) by
build.py; binding.py is the thin ctypes layer over it; autograd.py wraps the forward/adjoint pair as a
torch.autograd.Function; synth.py draws the seeded synthetic inputs.  Importing this package does not
load the library: the first call through binding.py does, and fails loudly if it is missing.
"""
__all__ = ["binding", "build", "synth"]

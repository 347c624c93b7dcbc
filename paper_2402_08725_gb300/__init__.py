"""GB300 (sm_103a) implementation of the STARRED loss-and-gradient hot path
(Millon et al., arXiv 2402.08725): joint multi-epoch two-channel deconvolution
and PSF reconstruction, with hand-written CUDA kernels behind a C ABI
(include/starred.h).

Modules:
  build      compiles csrc/*.cu into _build/libstarred_gb300.so (nvcc, sm_103a)
  _native    ctypes prototypes of the C ABI
  binding    Problem / Batch objects over torch device memory and streams
  torch_ops  torch.autograd.Function around the loss and its adjoint
  synthetic  seeded synthetic inputs shaped like the paper's workloads
"""

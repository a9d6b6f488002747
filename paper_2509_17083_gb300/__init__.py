"""HyRF (arXiv 2509.17083) render-and-train hot path, GB300-native.

The compute path is the C-ABI library libhyrf.so (hand-written sm_103a CUDA
kernels, declared in include/hyrf.h). `hyrf` is the thin ctypes binding with
the same call names; `autograd` wraps each stage in a torch.autograd.Function;
`renderer` composes the stages into one differentiable view render. PyTorch
supplies device memory and streams only.
"""
__all__ = ["synth"]

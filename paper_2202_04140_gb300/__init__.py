"""GB300 (sm_103a) recursive contraction of sparse symmetric tensors (arXiv 2202.04140).

Submodules:
  ace        ctypes binding of libace.so (the C ABI of include/ace.h)
  torch_api  tensor-level API: Spec, Dag (evaluate, evaluate_grad, energy), pooling
  build      builds libace.so in-tree with nvcc for sm_103a
The compiled library is loaded on first import of ``ace``/``torch_api``.
"""
__all__ = ["ace", "torch_api", "build"]

"""B300-native NMODL mechanism hot path (nrn_state / nrn_cur on sm_103a).

The compute path is libnmodl_b300.so (hand-written CUDA); `_lib` is its
ctypes binding and `api` a small object wrapper over it for torch tensors.
Importing the package does not load the library; `import
paper_1905_02241_b300.api` does, and fails if the library is missing.
"""
__all__ = ["workloads"]

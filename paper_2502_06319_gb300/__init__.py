"""GB300 (sm_103a) implementation of the COSMICA hot path (arXiv 2502.06319).

The propagation path lives in libcosmica.so (CUDA, C ABI in include/cosmica.h);
`cosmica` is its ctypes binding.  `workloads` describes the synthetic inputs.
Nothing here imports the CUDA binding eagerly, so the input descriptions can
be loaded without a GPU.
"""
__all__ = ["cosmica", "workloads"]

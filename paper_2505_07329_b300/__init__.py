"""B300 (sm_103a) engine for the server side of private LoRA fine-tuning under
homomorphic encryption (arXiv 2505.07329): the encrypted-vector x clear-matrix
product W.[x] / W^T.[g] of Eq. (LWEdot) with the fused ModulusSwitch.

The compute path is libphe.so (CUDA, C ABI in include/phe.h); `phe` is its
ctypes binding.  Build with `python -m paper_2505_07329_b300.build`.
"""

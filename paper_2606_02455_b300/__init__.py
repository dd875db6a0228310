"""B300-native Langevin Speculative Dynamics: window verification and Gaussian transport on one GPU.

The compute path is the CUDA library ``liblsd.so`` (C ABI declared in
``include/lsd.h``); ``paper_2606_02455_b300.lsd`` is its thin Python binding.
Importing the package itself does not load the library.
"""
__all__ = ["workloads"]

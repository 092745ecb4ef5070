"""GB300-native Hessian-free ray-Born sound-speed inversion (arXiv 2211.00316).

The compute path is librbx (CUDA for sm_103a, C ABI in include/rbx.h); `rbx` is its
Python binding, `phantoms` the seeded synthetic inputs, `build` the in-tree compiler.
"""

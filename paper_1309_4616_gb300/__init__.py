"""GB300 exponential integrators: phi_k(hA)v by Leja interpolation, exponential
Euler and Rosenbrock-Euler steps, on hand-written sm_103a kernels.

The compute path lives in libei.so (C ABI: include/ei.h); `ei` is its thin
ctypes binding, `workloads` the seeded synthetic inputs, `build` the in-tree
build step.  Importing the package loads nothing: `ei.lib()` loads the
library on first use and raises if it has not been built.
"""

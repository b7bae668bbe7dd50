"""GB300 matrix-free hybrid multigrid for SIPG / upwind DG (arXiv 1805.11930).

The compute path is libdgmg.so (CUDA, sm_103a) behind the C ABI of
include/dgmg.h; `dgmg` is its ctypes binding, `inputs` the seeded workload
generators, `build` the compiler driver.  Importing this package loads
nothing; `dgmg.load()` or `dgmg.Context()` loads the library and raises if it
cannot.
"""
__all__ = ["build", "dgmg", "inputs"]

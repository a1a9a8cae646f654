"""GB300 (sm_103a) library for distance-generalized (k,h)-cores.

After Tatti, "Fast computation of distance-generalized cores using sampling":
exact h-degrees, the rank-sampled h-degree estimate (Alg. 1, Prop. 3.1,
Alg. 2), and ExactCore / Core (Alg. 4) peeling, all in hand-written CUDA
kernels behind the C ABI of ``include/khcore.h``.

Submodules:
  khcore    thin ctypes binding of the C ABI (same names as the C calls)
  build     nvcc build of ``_build/libkhcore.so``
  graphgen  seeded synthetic graph generators (inputs only)
"""

"""GB300 (sm_103a) lattice Boltzmann solver for the volume-averaged Navier-Stokes
equations with Carreau-Yasuda blood rheology (Horvat et al., arXiv 2402.10809).

``lbm``      ctypes binding of the C ABI (include/lbm.h) to liblbm.so.
``build``    in-tree nvcc build of liblbm.so.
"""

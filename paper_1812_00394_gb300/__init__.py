"""GB300 (sm_103a) implementation of the time step of the simplified finite-volume lattice
Boltzmann method with k-omega SST and three-stage IMEX Runge-Kutta (arXiv 1812.00394, Part II).

* ``fvlbm``   -- binding of the C ABI in include/fvlbm.h (CUDA library, in-tree build)
* ``meshgen`` -- seeded synthetic meshes and cases
* ``build``   -- nvcc build of the library
"""

"""GB300 (sm_103a) integration of massive-neutrino particles along geodesics of a
linearly perturbed spacetime: the fastdf method of Elbers 2022 (arXiv:2207.14256).

The compute path is libfdf.so (include/fdf.h), hand-written CUDA kernels behind
a C-ABI; ``paper_2207_14256_gb300.fdf`` is its Python binding and
``paper_2207_14256_gb300.inputs`` builds seeded synthetic inputs.  Importing
this package loads nothing; the binding loads the library on first use.
"""

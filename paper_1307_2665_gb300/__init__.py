"""GB300 (sm_103a) composite spectral direct solver (Gillman & Martinsson, arXiv:1307.2665).

The solver lives in libhps.so (CUDA kernels behind the C ABI of include/hps.h);
`paper_1307_2665_gb300.hps` is its ctypes binding and
`paper_1307_2665_gb300.inputs` holds the seeded synthetic inputs.  Importing
the package loads nothing native; the binding loads the library on first use.
"""

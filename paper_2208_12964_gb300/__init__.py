"""GB300 (sm_103a) MART on Uniformly Sampled Polar/Cylindrical Grids.

``uspg`` is the ctypes binding of the CUDA library ``_lib/libuspg.so`` (C ABI
in ``include/uspg.h``); ``synth`` draws seeded synthetic scans and phantoms;
``build`` compiles the library.  Submodules are imported on demand so that
``synth`` can be used without the library.
"""

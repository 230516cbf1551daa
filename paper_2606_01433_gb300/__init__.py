"""GB300-native monolithic multilevel GDSW overlapping Schwarz preconditioner and
flexible GMRES for Carreau Stokes saddle-point systems.

The compute path lives in the CUDA shared library ``libgdsw.so`` (sources in ``csrc/``,
C ABI in ``include/gdsw.h``); ``gdsw`` is its thin ctypes binding.  Importing this package
does not load the library: ``paper_2606_01433_gb300.gdsw.load()`` does, and raises if the
library has not been built.
"""

"""GB300 (sm_103a) domain wall fermion operator and Krylov solvers.

``paper_2203_17119_gb300.dwf``     ctypes binding of ``include/dwf.h``
``paper_2203_17119_gb300.inputs``  seeded synthetic gauge fields and sources
``paper_2203_17119_gb300.build``   in-tree nvcc build of ``libdwf.so``

Importing the package loads nothing; the binding loads the library on first
use and raises if it has not been built.
"""

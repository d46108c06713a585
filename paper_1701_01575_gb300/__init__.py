"""GB300-native exact Gotoh alignment (local / global / semi-global) behind a C ABI.

Submodules:
  * ``dsa``       -- ctypes binding of libdsa.so (include/dsa.h)
  * ``build``     -- compiles libdsa.so for sm_103a in-tree
  * ``workloads`` -- seeded synthetic inputs (no alignment arithmetic)
Importing the package loads nothing; the binding loads the library on first use.
"""

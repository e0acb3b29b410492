"""GB300 library for the statically condensed HDG trace operator and its nested
p/h multigrid (arXiv 1705.09907).

Submodules:
  build   compile csrc/ into the in-tree libhdg.so (sm_103a)
  hdg     ctypes binding of include/hdg.h (loads libhdg.so; raises if missing)
  inputs  seeded synthetic workloads (coefficient fields, sources)
The binding is imported lazily so that `inputs` works without the library.
"""

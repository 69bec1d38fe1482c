"""Test infrastructure only: the plain FP64 CPU oracle of the primal hybrid FEM.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  It imports nothing from the CUDA product path.
"""

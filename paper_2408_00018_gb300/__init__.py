"""GB300-native synchronous parallel simulated annealing.

The solver itself is the CUDA library ``libsa103.so`` (C ABI in include/sa.h);
``paper_2408_00018_gb300.sa`` is its thin Python binding and
``paper_2408_00018_gb300.inputs`` holds the seeded input generators shared by
the tests and the benchmark.  Importing the package loads nothing.
"""
__all__ = ["sa", "inputs"]

"""GB300-native LOR-preconditioned matrix-free high-order Poisson solver.

The compute path lives in the CUDA library built from ``csrc/`` and is reached
through the ctypes binding in :mod:`paper_1908_07071_gb300.lor`.  Importing this
package loads nothing; ``from paper_1908_07071_gb300 import lor`` loads the
shared library and raises if it has not been built.
"""
__all__ = ["lor", "synthetic", "build"]

"""GB300-native short-range non-bonded forces (ACEMD hot path, arXiv:0902.0827).

The compute path lives in the CUDA shared library built from ``csrc/``; the
Python binding in :mod:`paper_0902_0827_gb300.nb` only marshals arguments.
Importing this package loads nothing heavy.
"""
__all__ = ["systems", "nb"]

"""B300-native hybrid symplectic N-body hot path (CUDA for sm_103a behind a C-ABI).

Importing the package is cheap; the CUDA library ``libnb.so`` is loaded on
first use by :mod:`paper_2604_09184_b300.nb` and a missing library raises.
"""
__all__ = ["ics"]

"""B300-native (sm_103a) training step and query path of the domain-decomposed
PINN method of arXiv 2602.15883.

The compute path lives in ``libdpinn.so`` (hand-written CUDA behind a C ABI,
declared in ``include/dpinn.h``); this package is its thin ctypes binding plus
the synthetic-workload generator.  Importing the package does not load the
library; ``Dpinn`` (from ``paper_2602_15883_b300.binding``) does, and fails
loudly when the library is missing.
"""

__all__ = ["Dpinn", "DpinnError"]


def __getattr__(name):
    if name in ("Dpinn", "DpinnError"):
        import importlib
        return getattr(importlib.import_module(".binding", __name__), name)
    raise AttributeError(name)

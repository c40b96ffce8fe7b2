"""GB300-native content-area estimation (Budd et al., arXiv 2210.14771).

The estimation runs in libca (CUDA, sm_103a) behind a C ABI (include/ca.h);
this package is its Python view plus the synthetic frame generator and the
Hausdorff evaluation.  Importing it needs neither a GPU nor the built
library; calling the estimator needs both.
"""
import importlib

from .build import build  # noqa: F401

_LAZY = {"ContentArea": "api", "params": "api", "results_numpy": "api", "new_results": "api"}


def __getattr__(name):
    # torch-dependent parts are imported on first use
    if name in _LAZY:
        return getattr(importlib.import_module(__name__ + "." + _LAZY[name]), name)
    raise AttributeError(name)

"""GB300-native scenario-batched Bellman (min-plus) kernels for the Split
operator (CVRP with stochastic demand) and the order-up-to inventory-
reinsertion DP of arXiv 2602.05179.

The compute path is the C-ABI library ``libsdp.so`` (hand-written sm_103a CUDA
kernels, header ``include/sdp.h``); the Python layer only marshals arguments.
Importing this package does not load the library; the first call does, and it
raises if the library is missing or no CUDA device is present.
"""
__all__ = ["split_eval", "split_count_arcs", "reinsert_eval", "SplitMeanCost",
           "SplitPlan", "lib_path"]


def __getattr__(name):
    if name in __all__:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)

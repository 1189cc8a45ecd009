"""GB300-native incremental state-vector simulator (qTask, arXiv 2210.01076).

The compute path is the C-ABI library ``libqtask.so`` (hand-written CUDA for
sm_103a, declared in ``include/qtask.h``); ``binding`` marshals arguments to
it with ctypes.  Importing this package does not load the library: the
binding loads it on first use and raises if it has not been built.
"""
__all__ = ["binding", "workloads", "build"]

"""GB300-native near-field P2P operator of MLFMA (arXiv 2403.01596).

The compute path is libp2p.so (hand-written CUDA for sm_103a, C ABI in
include/p2p.h); `api` wraps it for PyTorch tensors and autograd.  Submodules
load lazily so that the seeded input generators (`workloads`) import without
a GPU or a built library.
"""
import importlib

__all__ = ["api", "workloads", "build", "Plan", "BoxStructure", "P2PFunction", "p2p"]


def __getattr__(name):
    if name in ("Plan", "BoxStructure", "P2PFunction", "p2p"):
        return getattr(importlib.import_module(".api", __name__), name)
    if name in ("api", "workloads", "build", "_capi", "autotune", "bench_util"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)

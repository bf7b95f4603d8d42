"""GB300-native online dynamic mode decomposition (hot path of arXiv 2311.18715).

The C ABI lives in include/odmd.h and libodmd.so (built in-tree by ``build()``);
``OnlineDMD`` wraps it for torch tensors.
"""
from ._build import build
from ._lib import EXPORTED, OdmdError, load_library

__all__ = ["build", "load_library", "OdmdError", "EXPORTED", "OnlineDMD", "OnlineDMDPairs", "check_noalloc",
           "update_batch", "predict_batch", "batch_split"]


def __getattr__(name):
    if name == "OnlineDMD":
        from .odmd import OnlineDMD
        return OnlineDMD
    if name == "OnlineDMDPairs":
        from .odmd import OnlineDMDPairs
        return OnlineDMDPairs
    if name in ("check_noalloc", "update_batch", "predict_batch", "batch_split"):
        from . import odmd
        return getattr(odmd, name)
    raise AttributeError(name)

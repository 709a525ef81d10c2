"""B300-native contraction of hybrid tensor networks (arXiv 2410.15080).

The compute path is the shared library ``libqtpu_htn.so`` (C ABI in
``include/qtpu_htn.h``); ``htn`` is its ctypes binding.  Nothing here falls
back to a CPU or PyTorch implementation.
"""
from .htn import HTN, QtpuError, batch_info, contract_batch, from_network, lib, plan_text, qt_evaluate  # noqa: F401

"""GB300-native dynamic max-flow (arXiv 2511.05895, Dynamic Push Relabel).

The solver is the CUDA library libmfgpu.so (C ABI in include/mf.h); this
package is its thin Python binding.  See ``MaxFlowGraph``.
"""
from ._native import (MF_DELTA, MF_DEVICE_PTRS, MF_ECHECK, MF_ECUDA, MF_EINVAL, MF_ENOMEM, MF_ENOTSOLVED,
                      MF_ETIMEOUT, MF_HOST_PTRS, MF_MODE_DATA_DRIVEN, MF_MODE_PUSH_PULL, MF_MODE_TOPOLOGY, MF_OK,
                      MF_POLICY_FIXED, MF_POLICY_LEARNED, MF_POLICY_PLAIN, MF_RECOMPUTE, MaxFlowGraph, MFError,
                      Server, bicsr_host, lib)

__all__ = ["MaxFlowGraph", "MFError", "Server", "bicsr_host", "lib", "MF_OK", "MF_EINVAL", "MF_ENOMEM",
           "MF_ECUDA", "MF_ENOTSOLVED", "MF_ETIMEOUT", "MF_ECHECK", "MF_HOST_PTRS", "MF_DEVICE_PTRS",
           "MF_DELTA", "MF_RECOMPUTE", "MF_POLICY_FIXED", "MF_POLICY_PLAIN", "MF_POLICY_LEARNED",
           "MF_MODE_DATA_DRIVEN", "MF_MODE_TOPOLOGY", "MF_MODE_PUSH_PULL"]
__version__ = "0.1.0"

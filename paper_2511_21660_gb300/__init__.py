"""GB300-native batched Relay-BP decoder (paper Sec. 2.3, App. A.3).

The decoder is libqldpc.so (CUDA kernels for sm_103a behind the C ABI of
include/qldpc.h); ``qldpc`` is its Python binding.  Importing the binding
raises if the library has not been built: there is no CPU fallback.
"""
from .qldpc import (QLDPC_KERNEL_AUTO, QLDPC_KERNEL_BASELINE, QLDPC_KERNEL_FUSED,
                    QLDPC_MSG_FP16, QLDPC_MSG_FP32, QldpcError, RelayConfig, RelayDecoder,
                    SoftDMem, decode_mixed, load_library, soft_dmem_loss)

__all__ = ["RelayDecoder", "RelayConfig", "SoftDMem", "soft_dmem_loss", "decode_mixed",
           "QldpcError",
           "load_library", "QLDPC_MSG_FP32",
           "QLDPC_MSG_FP16", "QLDPC_KERNEL_AUTO", "QLDPC_KERNEL_BASELINE", "QLDPC_KERNEL_FUSED"]

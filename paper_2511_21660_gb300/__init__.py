"""GB300-native batched Relay-BP decoder (paper Sec. 2.3, App. A.3) with the
filtered-OSD (Sec. 5) and cluster (Sec. 2.5, Sec. 6) post-processors.

The decoder is libqldpc.so (CUDA kernels for sm_103a behind the C ABI of
include/qldpc.h); ``qldpc`` is its Python binding.  Importing the binding
raises if the library has not been built: there is no CPU fallback.
"""
from .qldpc import (QLDPC_CLUSTER_DECODED, QLDPC_CLUSTER_SKIPPED, QLDPC_CLUSTER_STALLED,
                    QLDPC_CLUSTER_TOO_LARGE, QLDPC_CLUSTER_TOO_MANY, QLDPC_KERNEL_AUTO,
                    QLDPC_KERNEL_BASELINE, QLDPC_KERNEL_FUSED, QLDPC_MSG_FP16, QLDPC_MSG_FP32,
                    QLDPC_OSD_NO_SOLUTION, QLDPC_OSD_SKIPPED, QLDPC_OSD_SOLVED,
                    QLDPC_OSD_TOO_MANY, ClusterDecoder, FilteredOSD, QldpcError, RelayConfig,
                    RelayDecoder, SoftDMem, decode_grouped, decode_mixed,
                    first_leg_then_cluster, first_leg_then_osd, load_library, soft_dmem_loss)

__all__ = ["RelayDecoder", "RelayConfig", "SoftDMem", "soft_dmem_loss", "decode_mixed",
           "decode_grouped",
           "FilteredOSD", "first_leg_then_osd", "QldpcError", "load_library",
           "QLDPC_MSG_FP32", "QLDPC_MSG_FP16", "QLDPC_KERNEL_AUTO", "QLDPC_KERNEL_BASELINE",
           "QLDPC_KERNEL_FUSED", "QLDPC_OSD_SKIPPED", "QLDPC_OSD_SOLVED", "QLDPC_OSD_TOO_MANY",
           "QLDPC_OSD_NO_SOLUTION", "ClusterDecoder", "first_leg_then_cluster",
           "QLDPC_CLUSTER_SKIPPED", "QLDPC_CLUSTER_DECODED", "QLDPC_CLUSTER_TOO_LARGE",
           "QLDPC_CLUSTER_TOO_MANY", "QLDPC_CLUSTER_STALLED"]

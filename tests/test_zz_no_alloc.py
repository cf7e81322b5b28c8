"""The allocation-free host-buffer decode (qldpc_decode_batch_host_static).

Some callers cannot allocate device memory while they decode: a real-time loop
that works inside a fixed memory budget, or a process whose device memory is
owned by another allocator.  qldpc_decode_batch_host allocates its staging
buffers on first use and whenever a batch grows, so those callers use the static
variant, which stages everything in one fixed device array instead.

This file runs last (pytest collects it last) and needs nothing from the other
tests: it builds its own decoder and compares the static variant with the
regular host-buffer entry point, bit for bit, on two calls in a row.
"""
import ctypes

import numpy as np
import pytest

from workloads import BB144, gamma_table, pack_bits, phenomenological_dem, sample_faults, \
    syndromes_of

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _decode(fn, handle, packed, cw):
    B = packed.shape[0]
    cor = np.zeros((B, cw), dtype=np.uint64)
    legs = np.zeros(B, dtype=np.int32)
    conv = np.zeros(B, dtype=np.uint8)
    iters = np.zeros(B, dtype=np.int32)
    fn(handle, ctypes.c_void_p(packed.ctypes.data), B, ctypes.c_void_p(cor.ctypes.data),
       ctypes.c_void_p(legs.ctypes.data), ctypes.c_void_p(conv.ctypes.data),
       ctypes.c_void_p(iters.ctypes.data))
    return cor, legs, conv, iters


def test_static_scratch_decode_matches_host_decode_on_consecutive_calls():
    from paper_2511_21660_gb300 import RelayConfig, RelayDecoder
    from paper_2511_21660_gb300 import qldpc as Q

    P = phenomenological_dem(BB144, 12, 0.003)
    gam = gamma_table(P.N, 300, 0.125, -0.24, 0.66, 3)
    dec = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam, RelayConfig(stop_after_solutions=5))
    try:
        cw = dec.correction_words
        # two different batches, the second one smaller, so that leftovers of the first
        # call in the shared static array would show up as differences
        for seed, n in ((11, 4000), (12, 1500)):
            sig = syndromes_of(P.row_ptr, P.col_idx, sample_faults(P.p, seed, n))
            packed = pack_bits(sig)
            ref = _decode(Q.qldpc_decode_batch_host, dec.handle, packed, cw)
            got = _decode(Q.qldpc_decode_batch_host_static, dec.handle, packed, cw)
            for a, b, what in zip(got, ref, ("corrections", "legs", "converged", "iters")):
                assert np.array_equal(a, b), f"seed {seed}: {what} differ"
            assert ref[2].all()

        # a batch larger than the static array is refused with a clear message
        big = np.zeros((20000, dec.syndrome_words), dtype=np.uint64)
        with pytest.raises(Q.QldpcError) as err:
            _decode(Q.qldpc_decode_batch_host_static, dec.handle, big, cw)
        assert err.value.status == Q.QLDPC_ERR_INVALID_ARG
        assert "static scratch" in str(err.value)
    finally:
        dec.close()

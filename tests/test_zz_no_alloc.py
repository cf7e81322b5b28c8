"""The allocation-free host-buffer decode (qldpc_decode_batch_host_static).

Some callers cannot allocate device memory while they decode: a real-time loop
that works inside a fixed memory budget, or a process whose device memory is
owned by another allocator.  qldpc_decode_batch_host allocates its staging
buffers on first use and whenever a batch grows, so those callers use the static
variant, which stages everything in one fixed device array instead.

This file runs last (pytest collects it last) and needs nothing from the other
tests: it builds its own decoders and compares the static variant with the
regular host-buffer entry point, bit for bit, on calls in a row, at the largest
batch the array holds, and checks that the static calls leave the device's free
memory unchanged.
"""
import ctypes

import numpy as np
import pytest

from workloads import BB144, gamma_table, pack_bits, phenomenological_dem, sample_faults, \
    syndromes_of

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STATIC_BYTES = 8 * 1024 * 1024


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


def _largest_batch(sw, cw):
    """The header's layout: a 256-byte counter, then syndromes, corrections, legs,
    iterations and converged flags, each rounded up to 256 bytes."""
    def need(B):
        al = lambda x: (x + 255) // 256 * 256  # noqa: E731
        return 256 + al(8 * sw * B) + al(8 * cw * B) + 2 * al(4 * B) + al(B)
    B = 0
    while need(B + 1) <= STATIC_BYTES:
        B += 1
    return B


def _problem():
    P = phenomenological_dem(BB144, 12, 0.003)
    return P, gamma_table(P.N, 300, 0.125, -0.24, 0.66, 3)


def _syndromes(P, seed, n):
    return pack_bits(syndromes_of(P.row_ptr, P.col_idx, sample_faults(P.p, seed, n)))


def test_static_calls_on_a_fresh_handle_allocate_nothing():
    """The first calls on a new handle, before any other host-buffer call, leave the
    device's free memory exactly where it was."""
    from paper_2511_21660_gb300 import RelayConfig, RelayDecoder
    from paper_2511_21660_gb300 import qldpc as Q

    P, gam = _problem()
    dec = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam, RelayConfig(stop_after_solutions=5))
    try:
        packed = _syndromes(P, 21, 3000)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        a = _decode(Q.qldpc_decode_batch_host_static, dec.handle, packed, dec.correction_words)
        b = _decode(Q.qldpc_decode_batch_host_static, dec.handle, packed, dec.correction_words)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        assert a[2].all()
    finally:
        dec.close()


def test_static_scratch_decode_matches_host_decode_on_consecutive_calls():
    from paper_2511_21660_gb300 import RelayConfig, RelayDecoder
    from paper_2511_21660_gb300 import qldpc as Q

    P, gam = _problem()
    dec = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam, RelayConfig(stop_after_solutions=5))
    try:
        cw = dec.correction_words
        # two different batches, the second one smaller, so that leftovers of the first
        # call in the shared static array would show up as differences
        for seed, n in ((11, 4000), (12, 1500)):
            packed = _syndromes(P, seed, n)
            ref = _decode(Q.qldpc_decode_batch_host, dec.handle, packed, cw)
            got = _decode(Q.qldpc_decode_batch_host_static, dec.handle, packed, cw)
            for a, b, what in zip(got, ref, ("corrections", "legs", "converged", "iters")):
                assert np.array_equal(a, b), f"seed {seed}: {what} differ"
            assert ref[2].all()
    finally:
        dec.close()


def test_largest_static_batch_is_decoded_and_one_more_shot_is_refused():
    """The array holds 17,732 gross-code shots: that batch decodes bit for bit like the
    host-buffer path, one shot more is refused with the exact limit in the message."""
    from paper_2511_21660_gb300 import RelayConfig, RelayDecoder
    from paper_2511_21660_gb300 import qldpc as Q

    P, gam = _problem()
    dec = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam, RelayConfig(stop_after_solutions=5))
    try:
        cw, sw = dec.correction_words, dec.syndrome_words
        nmax = _largest_batch(sw, cw)
        assert nmax == 17732
        packed = _syndromes(P, 13, nmax)
        got = _decode(Q.qldpc_decode_batch_host_static, dec.handle, packed, cw)
        ref = _decode(Q.qldpc_decode_batch_host, dec.handle, packed, cw)
        for a, b, what in zip(got, ref, ("corrections", "legs", "converged", "iters")):
            assert np.array_equal(a, b), what
        over = np.zeros((nmax + 1, sw), dtype=np.uint64)
        with pytest.raises(Q.QldpcError) as err:
            _decode(Q.qldpc_decode_batch_host_static, dec.handle, over, cw)
        assert err.value.status == Q.QLDPC_ERR_INVALID_ARG
        assert "static scratch" in str(err.value) and f"at most {nmax} shots" in str(err.value)
    finally:
        dec.close()

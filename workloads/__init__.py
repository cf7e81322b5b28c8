"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package holds only problem construction (bivariate-bicycle codes, detector
matrices, logical-action matrices), the seeded fault sampler and the seeded
memory-strength table. It contains none of the decoder's arithmetic, and it
imports neither the oracle nor the CUDA library.
"""
from .gf2 import gf2_rank, gf2_nullspace, gf2_rref
from .codes import (BBCode, bb_code, BB72, BB144, BB288, phenomenological_dem,
                    code_capacity_dem, DecodingProblem, csr_from_dense)
from .sampling import (splitmix64, uniform01, sample_faults, syndromes_of,
                       gamma_table, pack_bits, unpack_bits)

__all__ = [
    "gf2_rank", "gf2_nullspace", "gf2_rref", "BBCode", "bb_code", "BB72", "BB144",
    "BB288", "phenomenological_dem", "code_capacity_dem", "DecodingProblem",
    "csr_from_dense", "splitmix64", "uniform01", "sample_faults", "syndromes_of",
    "gamma_table", "pack_bits", "unpack_bits",
]

"""Bivariate-bicycle (BB) codes and the decoding problems (H, A, p) built from them.

A decoding problem is the triple of Sec. 2.1 ("Noise and decoding"): a binary
decoding matrix H (M x N, one row per detector, one column per fault), a binary
logical-action matrix A (K x N) and a fault-probability vector p (length N).
A decoder given sigma = H F succeeds iff A (F + F_hat) = 0.

The paper benchmarks circuit-level noise on the gross and two-gross BB codes
(Sec. 2.1, "QEC circuit decoding examples"); those circuits are not available,
so these generators build the phenomenological stand-in: T noisy rounds of
perfect-gate syndrome extraction with data and measurement faults, followed by
one perfect round, giving detector matrices with the paper's detector counts
(936 rows for the gross code at T=12, 2736 rows for the two-gross code at T=18).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .gf2 import gf2_nullspace, gf2_rank


def _shift(n: int) -> np.ndarray:
    """n x n cyclic shift S_n with (S_n)[i, (i+1) mod n] = 1."""
    s = np.zeros((n, n), dtype=np.uint8)
    s[np.arange(n), (np.arange(n) + 1) % n] = 1
    return s


@dataclass(frozen=True)
class BBCode:
    """BB code with x = S_l (x) I_m, y = I_l (x) S_m, H_X = [A|B], H_Z = [B^T|A^T].

    ``a_terms`` / ``b_terms`` list the monomials of A and B as (power of x, power of y).
    """
    name: str
    l: int
    m: int
    a_terms: tuple
    b_terms: tuple

    def _poly(self, terms) -> np.ndarray:
        x = np.kron(_shift(self.l), np.eye(self.m, dtype=np.uint8))
        y = np.kron(np.eye(self.l, dtype=np.uint8), _shift(self.m))
        out = np.zeros((self.l * self.m,) * 2, dtype=np.int64)
        for px, py in terms:
            out += (np.linalg.matrix_power(x.astype(np.int64), px)
                    @ np.linalg.matrix_power(y.astype(np.int64), py))
        return (out % 2).astype(np.uint8)

    @property
    def A(self) -> np.ndarray:
        return self._poly(self.a_terms)

    @property
    def B(self) -> np.ndarray:
        return self._poly(self.b_terms)

    @property
    def hx(self) -> np.ndarray:
        return np.hstack([self.A, self.B])

    @property
    def hz(self) -> np.ndarray:
        return np.hstack([self.B.T, self.A.T])

    @property
    def n(self) -> int:
        return 2 * self.l * self.m

    @property
    def k(self) -> int:
        return self.n - gf2_rank(self.hx) - gf2_rank(self.hz)

    def x_logicals(self) -> np.ndarray:
        """k independent X-type logical operators: rows of ker(H_Z) outside rowspace(H_X).

        A Z-type residual r with H_X r = 0 is a logical fault iff it anticommutes
        with one of these rows, so they form the logical-action matrix for
        decoding against H_X.
        """
        hx = self.hx
        base = gf2_rank(hx)
        chosen = []
        for v in gf2_nullspace(self.hz):
            trial = np.vstack([hx] + chosen + [v[None, :]])
            if gf2_rank(trial) > base + len(chosen):
                chosen.append(v[None, :])
        return np.vstack(chosen).astype(np.uint8)


def bb_code(name: str) -> BBCode:
    return {"bb72": BB72, "bb144": BB144, "bb288": BB288}[name]


# [[72,12,6]]: l=m=6, A = x^3 + y + y^2, B = y^3 + x + x^2
BB72 = BBCode("bb72", 6, 6, ((3, 0), (0, 1), (0, 2)), ((0, 3), (1, 0), (2, 0)))
# gross [[144,12,12]]: l=12, m=6, same A and B
BB144 = BBCode("bb144", 12, 6, ((3, 0), (0, 1), (0, 2)), ((0, 3), (1, 0), (2, 0)))
# two-gross [[288,12,18]]: l=m=12, A = x^3 + y^2 + y^7, B = y^3 + x + x^2
BB288 = BBCode("bb288", 12, 12, ((3, 0), (0, 2), (0, 7)), ((0, 3), (1, 0), (2, 0)))


def csr_from_dense(h: np.ndarray):
    """CSR (row_ptr, col_idx) of a dense 0/1 matrix; columns ascending within a row."""
    h = np.asarray(h, dtype=np.uint8)
    rows, cols = np.nonzero(h)
    row_ptr = np.zeros(h.shape[0] + 1, dtype=np.int32)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    return row_ptr, cols.astype(np.int32)


@dataclass
class DecodingProblem:
    """(H, A, p) of Sec. 2.1 plus bookkeeping. H is kept dense (uint8) and as CSR."""
    name: str
    H: np.ndarray
    A: np.ndarray
    p: np.ndarray
    meta: dict = field(default_factory=dict)

    def __post_init__(self):
        self.H = np.ascontiguousarray(self.H, dtype=np.uint8)
        self.A = np.ascontiguousarray(self.A, dtype=np.uint8)
        self.p = np.ascontiguousarray(self.p, dtype=np.float64)
        self.row_ptr, self.col_idx = csr_from_dense(self.H)

    @property
    def M(self) -> int:
        return self.H.shape[0]

    @property
    def N(self) -> int:
        return self.H.shape[1]

    @property
    def E(self) -> int:
        return int(self.col_idx.size)


def code_capacity_dem(code: BBCode, p: float) -> DecodingProblem:
    """Code-capacity problem: one fault per qubit, H = H_X, A = X-logicals."""
    return DecodingProblem(f"{code.name}_cc", code.hx, code.x_logicals(),
                           np.full(code.n, p), {"code": code.name, "rounds": 0, "p": p})


def phenomenological_dem(code: BBCode, rounds: int, p: float) -> DecodingProblem:
    """Detector matrix for ``rounds`` noisy rounds followed by one perfect round.

    Detectors (t, i), t = 0..rounds, i = 0..mX-1, row t*mX + i.  Columns:
      * data fault (t, q), t = 0..rounds, q = 0..n-1 (column t*n + q) flips
        detectors (t, i) for every i in the support of column q of H_X;
      * measurement fault (t, i), t = 0..rounds-1 (column (rounds+1)*n + t*mX + i)
        flips detectors (t, i) and (t+1, i).
    The logical action of data fault (t, q) is column q of the X-logicals;
    measurement faults have none. Every fault has probability p.
    """
    hx = code.hx
    mx, n = hx.shape
    T = rounds
    M = (T + 1) * mx
    n_data = (T + 1) * n
    n_meas = T * mx
    H = np.zeros((M, n_data + n_meas), dtype=np.uint8)
    for t in range(T + 1):
        H[t * mx:(t + 1) * mx, t * n:(t + 1) * n] = hx
    for t in range(T):
        for i in range(mx):
            c = n_data + t * mx + i
            H[t * mx + i, c] = 1
            H[(t + 1) * mx + i, c] = 1
    lx = code.x_logicals()
    A = np.zeros((lx.shape[0], n_data + n_meas), dtype=np.uint8)
    for t in range(T + 1):
        A[:, t * n:(t + 1) * n] = lx
    return DecodingProblem(f"{code.name}_T{T}", H, A, np.full(H.shape[1], p),
                           {"code": code.name, "rounds": T, "p": p,
                            "n_data": n_data, "n_meas": n_meas})

"""Strassen coefficient tables for the oracle (test infrastructure only).

A table for L levels lists the 7^L products of Eq. 4 (Section 3.6):

    M_r = (sum_s delta_s X_s)(sum_t eps_t V_t);   C_q += gamma_q M_r,

where X_s are blocks of A, V_t blocks of B and C_q blocks of C in a 2^L x 2^L
partition.  Each product is a triple (a_terms, b_terms, c_terms), each term a tuple
(block_row, block_col, sign) with sign in {+1, -1}.

``FIG1`` is Figure 1 (Section 3.1) written out by hand.  The L-level table is the
L-th Kronecker power of it: product r = 7a + b of the two-level table is the outer
product a applied to the inner product b, and the block index along each dimension is
2 * outer + inner, with signs multiplied (Sections 3.5-3.6).  Figure 2 prints the
two-level table; the test suite checks the generated one against that print.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

Term = Tuple[int, int, int]          # (block_row, block_col, sign)
Product = Tuple[Tuple[Term, ...], Tuple[Term, ...], Tuple[Term, ...]]

# Figure 1, one row per product M0..M6: (A terms, B terms, C targets).
FIG1: Tuple[Product, ...] = (
    (((0, 0, +1), (1, 1, +1)), ((0, 0, +1), (1, 1, +1)), ((0, 0, +1), (1, 1, +1))),  # M0
    (((1, 0, +1), (1, 1, +1)), ((0, 0, +1),),            ((1, 0, +1), (1, 1, -1))),  # M1
    (((0, 0, +1),),            ((0, 1, +1), (1, 1, -1)), ((0, 1, +1), (1, 1, +1))),  # M2
    (((1, 1, +1),),            ((1, 0, +1), (0, 0, -1)), ((0, 0, +1), (1, 0, +1))),  # M3
    (((0, 0, +1), (0, 1, +1)), ((1, 1, +1),),            ((0, 1, +1), (0, 0, -1))),  # M4
    (((1, 0, +1), (0, 0, -1)), ((0, 0, +1), (0, 1, +1)), ((1, 1, +1),)),             # M5
    (((0, 1, +1), (1, 1, -1)), ((1, 0, +1), (1, 1, +1)), ((0, 0, +1),)),             # M6
)


def _kron_terms(outer: Tuple[Term, ...], inner: Tuple[Term, ...]) -> Tuple[Term, ...]:
    return tuple((2 * oi + ii, 2 * oj + ij, os * isg)
                 for (oi, oj, os) in outer for (ii, ij, isg) in inner)


def table(levels: int) -> List[Product]:
    """The 7^L-row table of Eq. 4 for ``levels`` = L >= 0 (L = 0: the single
    classical product C00 += A00 B00)."""
    if levels < 0:
        raise ValueError("levels must be >= 0")
    cur: List[Product] = [(((0, 0, 1),), ((0, 0, 1),), ((0, 0, 1),))]
    for _ in range(levels):
        nxt: List[Product] = []
        for (oa, ob, oc) in cur:            # outer product index a (slow)
            for (ia, ib, ic) in FIG1:       # inner product index b (fast)
                nxt.append((_kron_terms(oa, ia), _kron_terms(ob, ib), _kron_terms(oc, ic)))
        cur = nxt
    return cur


def block(X: np.ndarray, levels: int, bi: int, bj: int) -> np.ndarray:
    """Block (bi, bj) of X in the 2^L x 2^L partition with h = ceil(dim / 2^L) along
    each dimension; rows/columns past the edge of X are zeros (virtual padding)."""
    P = 1 << levels
    R, Cc = X.shape
    hr, hc = -(-R // P), -(-Cc // P)
    out = np.zeros((hr, hc), dtype=X.dtype)
    r0, c0 = bi * hr, bj * hc
    sub = X[r0:min(r0 + hr, R), c0:min(c0 + hc, Cc)]
    out[:sub.shape[0], :sub.shape[1]] = sub
    return out


def apply_table(A: np.ndarray, B: np.ndarray, C: np.ndarray, levels: int,
                tab: List[Product] | None = None) -> np.ndarray:
    """Return C + A @ B evaluated product by product from the L-level table (Eq. 4):
    form the signed operand sums, multiply them with numpy, and add gamma * M into
    each target block (masked to the real extent of C).  Used to pin tables: on
    integer-valued inputs this must equal A @ B exactly."""
    tab = table(levels) if tab is None else tab
    P = 1 << levels
    m, n = C.shape
    hm, hn = -(-m // P), -(-n // P)
    out = np.array(C, copy=True)
    for (at, bt, ct) in tab:
        S = sum(s * block(A, levels, i, j) for (i, j, s) in at)
        T = sum(s * block(B, levels, i, j) for (i, j, s) in bt)
        M = S @ T
        for (i, j, s) in ct:
            r0, c0 = i * hm, j * hn
            r1, c1 = min(r0 + hm, m), min(c0 + hn, n)
            if r1 > r0 and c1 > c0:
                out[r0:r1, c0:c1] += s * M[:r1 - r0, :c1 - c0]
    return out


def counts(levels: int) -> dict:
    """Term counts of the L-level table: products, A/B operand terms, C updates, and
    the extra additions of A and B submatrices (terms - products)."""
    tab = table(levels)
    na = sum(len(p[0]) for p in tab)
    nb = sum(len(p[1]) for p in tab)
    nc = sum(len(p[2]) for p in tab)
    return {"products": len(tab), "a_terms": na, "b_terms": nb, "c_updates": nc,
            "a_adds": na - len(tab), "b_adds": nb - len(tab)}

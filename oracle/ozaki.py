"""Oracle of the split-precision (Ozaki-style) FP64 product -- TEST INFRASTRUCTURE ONLY.

Not a method of the paper; it follows the error-free splitting of Ozaki, Ogita, Oishi
and Rump, "Error-free transformations of matrix multiplication by using fast
routines of matrix multiplication and its applications", Numer. Algorithms 59 (2012),
with the splitting carried out on integer digits (as in Mukunoki, Ozaki, Ogita and
Imamura, "DGEMM using tensor cores, and its accurate and reproducible versions",
ISC 2020).  The scheme computed here, step by step:

1. Scale.  For each row i of X: e_i is the smallest integer with
   max_k |X_ik| < 2^(e_i - 1)  (e_i = frexp(max)+1; rows of zeros get e_i = 0).
   For each column j of V: f_j likewise over max_k |V_kj|.  Then
   u_ik = X_ik * 2^-e_i and w_kj = V_kj * 2^-f_j lie in (-1/2, 1/2).
2. Split into S = 7 balanced base-2^b digits (b = 8) in the integer domain:
   N = rint(u * 2^(b S))  (u * 2^(bS) is an exact scaling; rint rounds half to even),
   so |N| <= 2^(bS-1).  Then, most significant first, with q_s = b (S - s):
   d_s = floor((N_s + 2^(q_s - 1)) / 2^(q_s)),  N_(s+1) = N_s - d_s 2^(q_s)
   for s < S, and d_S = N_S.  Hence N = sum_s d_s 2^(b (S - s)) exactly and
   |d_s| <= 2^(b-1) = 128: every digit is exactly representable in BF16 (8 significant
   bits) and a product of two digits (|.| <= 2^14) is exact in FP32.
   u = N 2^(-bS) + r with |r| <= 2^(-bS-1).
3. Products of slices.  For each weight w = 2 .. S+1, the exact integer matrix
   G_w = sum_{s + t = w} D_s^X D_t^V  (pairs with s + t > S + 1 are dropped).
4. Recombine with one rounding: the integer T = sum_w G_w 2^(b(S+1-w)) is exact,
   and M_ij = RN(T_ij) * 2^(e_i + f_j - b(S+1)), where RN is
   the round-to-nearest-even conversion to FP64 and the power-of-two scaling is exact
   (results in the normal range).

For Strassen (Eq. 4) the operand sums sum_s delta_s X_s and sum_t eps_t V_t are formed in
FP64 first (left to right over the table's terms), split as above, and each product's
M_r is added into its C blocks, C_q = C_q + gamma_q M_r, in product order.
"""
from __future__ import annotations

import numpy as np

from . import tables

B_BITS = 8      # bits per digit
S_DIGITS = 7    # digits per operand: b S = 56 bits cover a 53-bit significand with rounding room


def scale_exponents_rows(X: np.ndarray) -> np.ndarray:
    """e_i = smallest integer with max_k |X_ik| < 2^(e_i - 1); 0 for a zero row."""
    mx = np.max(np.abs(X), axis=1) if X.shape[1] else np.zeros(X.shape[0])
    _, ex = np.frexp(mx)          # mx = f * 2^ex with 0.5 <= f < 1, so mx < 2^ex
    e = ex.astype(np.int64) + 1   # mx < 2^(e - 1)
    e[mx == 0] = 0
    return e


def split(U: np.ndarray, S: int, b: int = B_BITS) -> np.ndarray:
    """Digits of U (entries in (-1/2, 1/2)): array [S, rows, cols] of integers (as
    float64), most significant first, with rint(U 2^(bS)) = sum_s D[s-1] 2^(b(S-s))."""
    N = np.rint(np.ldexp(np.asarray(U, dtype=np.float64), b * S)).astype(np.int64)
    out = np.empty((S,) + np.shape(U))
    for s in range(1, S):
        q = b * (S - s)
        d = (N + (np.int64(1) << np.int64(q - 1))) >> np.int64(q)   # floor division by 2^q
        N = N - (d << np.int64(q))
        out[s - 1] = d
    out[S - 1] = N
    return out


def slice_product_groups(DX: np.ndarray, DV: np.ndarray) -> dict:
    """G_w = sum_{s+t=w} DX[s-1] @ DV[t-1] for w = 2..S+1, exact (int64 matmul)."""
    S = DX.shape[0]
    X64 = DX.astype(np.int64)
    V64 = DV.astype(np.int64)
    G = {}
    for w in range(2, S + 2):
        acc = np.zeros((DX.shape[1], DV.shape[2]), dtype=np.int64)
        for s in range(1, w):
            t = w - s
            if t > S:
                continue
            acc += X64[s - 1] @ V64[t - 1]
        G[w] = acc
    return G


def recombine(G: dict, e: np.ndarray, f: np.ndarray, S: int, b: int = B_BITS) -> np.ndarray:
    """M = RN(T) 2^(e_i + f_j - b(S+1)) with T = sum_w G_w 2^(b(S+1-w)).

    T is carried as two integers, T_hi (weights w <= (S+2)//2) and T_lo (the rest),
    T = T_hi 2^(b(S+1-W)) + T_lo with W = (S+2)//2.  For the sizes this oracle serves
    (|G_w| < 2^28) both are below 2^53 in magnitude (asserted), so each converts to FP64 exactly,
    the power-of-two scaling of T_hi is exact, and the one FP64 addition of the two
    returns the correctly rounded RN(T)."""
    W = (S + 2) // 2
    t_hi = np.zeros(G[2].shape, dtype=np.int64)
    t_lo = np.zeros(G[2].shape, dtype=np.int64)
    for w in range(2, S + 2):
        if w <= W:
            t_hi = t_hi + G[w] * (np.int64(1) << np.int64(b * (W - w)))
        else:
            t_lo = t_lo + G[w] * (np.int64(1) << np.int64(b * (S + 1 - w)))
    assert np.all(np.abs(t_hi) < 2 ** 53) and np.all(np.abs(t_lo) < 2 ** 53)
    T = np.ldexp(t_hi.astype(np.float64), b * (S + 1 - W)) + t_lo.astype(np.float64)
    return np.ldexp(T, (e[:, None] + f[None, :] - b * (S + 1)).astype(np.int64))


def product(X: np.ndarray, V: np.ndarray, S: int = S_DIGITS) -> np.ndarray:
    """M ~= X @ V by steps 1-4 (the split-precision product of one pair of operands)."""
    e = scale_exponents_rows(X)
    f = scale_exponents_rows(V.T)
    U = np.ldexp(X, -e[:, None])
    Wt = np.ldexp(V, -f[None, :])
    DX = split(U, S)
    DV = split(Wt, S)
    return recombine(slice_product_groups(DX, DV), e, f, S)


def gemm(A: np.ndarray, B: np.ndarray, C: np.ndarray, levels: int, S: int = S_DIGITS) -> np.ndarray:
    """C + A @ B with ``levels`` levels of Strassen (table of Eq. 4) and every product
    M_r computed by the split-precision product; returns a new array."""
    tab = tables.table(levels)
    out = np.array(C, dtype=np.float64, copy=True)
    m, n = C.shape
    P = 1 << levels
    hm, hn = -(-m // P), -(-n // P)
    for (at, bt, ct) in tab:
        X = None
        for (i, j, s) in at:
            blk = tables.block(A, levels, i, j)
            X = (blk if s > 0 else -blk) if X is None else (X + blk if s > 0 else X - blk)
        V = None
        for (i, j, s) in bt:
            blk = tables.block(B, levels, i, j)
            V = (blk if s > 0 else -blk) if V is None else (V + blk if s > 0 else V - blk)
        M = product(X, V, S)
        for (i, j, s) in ct:
            r0, c0 = i * hm, j * hn
            r1, c1 = min(r0 + hm, m), min(c0 + hn, n)
            if r1 > r0 and c1 > c0:
                blk = M[:r1 - r0, :c1 - c0]
                out[r0:r1, c0:c1] = out[r0:r1, c0:c1] + blk if s > 0 else out[r0:r1, c0:c1] - blk
    return out

"""A numpy model of the split3 arithmetic, used only to check the parity tests' bounds.

It computes a Strassen product exactly as the library's FP32-accurate arithmetic rounds it:
every operand sum P = sum_q U[q, r] A_q is formed in FP32, split into BF16 hi = bf16(P) and
lo = bf16(P - hi) (round to nearest even), the three products hi*hi + hi*lo + lo*hi are
exact (as in the tensor cores) and their sum M_r is rounded to FP32, and every C block is
updated in FP32 (Section 3, Eq. 3; two levels by the Kronecker square of the tables).  The
rounding of the FP32 accumulation inside one product is not modelled; it is O(2**-24
sqrt(k)) relative and matters only at large k.  Test infrastructure: it shares nothing with
the CUDA library.
"""
import numpy as np

import oracle


def bf16_round(x) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def split(P: np.ndarray):
    P = P.astype(np.float32)
    hi = bf16_round(P)
    lo = bf16_round((P - hi).astype(np.float32))
    return hi.astype(np.float64), lo.astype(np.float64)


def product3(P: np.ndarray, Q: np.ndarray) -> np.ndarray:
    ph, pl = split(P)
    qh, ql = split(Q)
    return (ph @ qh + ph @ ql + pl @ qh).astype(np.float32)


def strassen_split3(A: np.ndarray, B: np.ndarray, levels: int) -> np.ndarray:
    """C = A B by ``levels`` levels of Strassen in the split3 arithmetic (float64 result)."""
    m, k = A.shape
    n = B.shape[1]
    if levels == 0:
        return product3(A, B).astype(np.float64)
    g = 1 << levels
    hm, hk, hn = (oracle.block_size(d, levels) for d in (m, k, n))
    Ap = np.zeros((g * hm, g * hk), np.float32)
    Ap[:m, :k] = A
    Bp = np.zeros((g * hk, g * hn), np.float32)
    Bp[:k, :n] = B
    UL, VL, WL, rc = oracle.level_coefficients(levels)
    Ab = [Ap[i * hm:(i + 1) * hm, j * hk:(j + 1) * hk] for i, j in rc]
    Bb = [Bp[i * hk:(i + 1) * hk, j * hn:(j + 1) * hn] for i, j in rc]
    C = np.zeros((g * hm, g * hn), np.float32)
    for r in range(UL.shape[1]):
        P = np.zeros((hm, hk), np.float32)
        Q = np.zeros((hk, hn), np.float32)
        for b in range(len(rc)):
            if UL[b, r]:
                P += np.float32(UL[b, r]) * Ab[b]
            if VL[b, r]:
                Q += np.float32(VL[b, r]) * Bb[b]
        M = product3(P, Q)
        for c, (i, j) in enumerate(rc):
            if WL[c, r]:
                C[i * hm:(i + 1) * hm, j * hn:(j + 1) * hn] += np.float32(WL[c, r]) * M
    return C[:m, :n].astype(np.float64)

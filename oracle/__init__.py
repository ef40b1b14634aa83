"""Oracle for fused Strassen GEMM -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct CPU reference for what the GPU path computes:

    C = alpha * A @ B + beta * C            (Section 1, Eq. 1 and Eq. 2)

with A (m x k), B (k x n), C (m x n), row-major.  Two routes are provided:

* ``classical`` -- the FP64 triple loop of Eq. 1, in plain C (``oracle_gemm.c``),
  optionally restricted to a sample of rows so that large problems stay cheap.
* ``strassen`` -- FP64 Strassen written from the seven products of Eq. (3)
  (the ``gpu_allops`` table of Section 3: M0..M6 and their C updates), applied
  recursively for ``levels`` levels, with zero padding of the fringes
  (Section 3.5).  The leaf product is a library matmul in FP64.  ``basis=
  "winograd"`` applies the Strassen-Winograd variant's seven products instead
  (Section 6 names it among the algorithms the primitive can carry).
* ``table_matmul`` -- FP64 one-level product by any basis table <g_m, g_k, g_n; R>
  (the <3,2,3> scheme of rank 15 and the <2,3,2> scheme of rank 11 below, or the
  2x2 tables), same fringe rule.

Supporting definitions: the 2x2 coefficient matrices U, V, W of Eq. (3), their
Kronecker powers for multi-level Strassen (Section 3.4), the Brent-equation
check, the operand-count table of Section 3.2, the block-size (padding) rule and
the normwise error used to state accuracy.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  Nothing here is shared with the CUDA path.

Parity status: every function below is pinned by tests in
``tests/test_oracle.py`` (Brent equations, the paper's operand-count table,
exact small-integer agreement, textbook special cases, a library matmul and
brute force on tiny inputs).  Floating-point agreement of the *GPU* path beyond
a tolerance is not pinned by any printed example: the paper prints none.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
from collections import Counter

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

# ---------------------------------------------------------------------------
# Eq. (3), Section 3: the seven products of one-level Strassen.
#
# Quadrants are numbered as in Eq. (2): X0 top-left, X1 top-right,
# X2 bottom-left, X3 bottom-right, i.e. q = 2*row + col.
#
#   M0 = (A0 + A3)(B0 + B3);  C0 += M0;  C3 += M0
#   M1 = (A2 + A3) B0;        C2 += M1;  C3 -= M1
#   M2 = A0 (B1 - B3);        C1 += M2;  C3 += M2
#   M3 = A3 (B2 - B0);        C0 += M3;  C2 += M3
#   M4 = (A0 + A1) B3;        C1 += M4;  C0 -= M4
#   M5 = (A2 - A0)(B0 + B1);  C3 += M5
#   M6 = (A1 - A3)(B2 + B3);  C0 += M6
#
# U[q, r] is the coefficient of A_q in the A-operand of product r, V[q, r] the
# coefficient of B_q in its B-operand and W[q, r] the coefficient with which
# M_r is added into C_q.
# ---------------------------------------------------------------------------
STRASSEN_U = np.array([
    # r:  0   1   2   3   4   5   6
    [1, 0, 1, 0, 1, -1, 0],    # A0
    [0, 0, 0, 0, 1, 0, 1],     # A1
    [0, 1, 0, 0, 0, 1, 0],     # A2
    [1, 1, 0, 1, 0, 0, -1],    # A3
], dtype=np.int64)

STRASSEN_V = np.array([
    [1, 1, 0, -1, 0, 1, 0],    # B0
    [0, 0, 1, 0, 0, 1, 0],     # B1
    [0, 0, 0, 1, 0, 0, 1],     # B2
    [1, 0, -1, 0, 1, 0, 1],    # B3
], dtype=np.int64)

STRASSEN_W = np.array([
    [1, 0, 0, 1, -1, 0, 1],    # C0
    [0, 0, 1, 0, 1, 0, 0],     # C1
    [0, 1, 0, 1, 0, 0, 0],     # C2
    [1, -1, 1, 0, 0, 1, 0],    # C3
], dtype=np.int64)


# ---------------------------------------------------------------------------
# The Strassen-Winograd variant, which the paper names among the fast-matmul
# algorithms its primitive could carry (Section 6).  In its usual form it shares
# partial sums (S1..S4 of A, T1..T4 of B, U2..U4 of the products) to need 15
# additions; written per product, as this primitive forms every operand and
# every C update directly from the quadrants, its tables are (A0 = A11,
# A1 = A12, A2 = A21, A3 = A22, likewise B and C):
#   M0 = A0 B0;                                C0, C1, C2, C3 += M0
#   M1 = A1 B2;                                C0 += M1
#   M2 = (A0 + A1 - A2 - A3) B3;               C1 += M2
#   M3 = A3 (B0 - B1 - B2 + B3);               C2 -= M3
#   M4 = (A2 + A3)(B1 - B0);                   C1 += M4, C3 += M4
#   M5 = (A2 + A3 - A0)(B0 - B1 + B3);         C1, C2, C3 += M5
#   M6 = (A0 - A2)(B3 - B1);                   C2 += M6, C3 += M6
# 14 nonzeros in each of U, V, W (12 for Strassen's).
# ---------------------------------------------------------------------------
WINOGRAD_U = np.array([
    # r:  0   1   2   3   4   5   6
    [1, 0, 1, 0, 0, -1, 1],    # A0
    [0, 1, 1, 0, 0, 0, 0],     # A1
    [0, 0, -1, 0, 1, 1, -1],   # A2
    [0, 0, -1, 1, 1, 1, 0],    # A3
], dtype=np.int64)

WINOGRAD_V = np.array([
    [1, 0, 0, 1, -1, 1, 0],    # B0
    [0, 0, 0, -1, 1, -1, -1],  # B1
    [0, 1, 0, -1, 0, 0, 0],    # B2
    [0, 0, 1, 1, 0, 1, 1],     # B3
], dtype=np.int64)

WINOGRAD_W = np.array([
    [1, 1, 0, 0, 0, 0, 0],     # C0
    [1, 0, 1, 0, 1, 1, 0],     # C1
    [1, 0, 0, -1, 0, 1, 1],    # C2
    [1, 0, 0, 0, 1, 1, 1],     # C3
], dtype=np.int64)

# ---------------------------------------------------------------------------
# A <3,2,3> basis of rank 15 (Section 6 names bases other than <2,2,2> as the
# next step for the primitive).  A one-level basis <g_m, g_k, g_n; R> splits A
# into a g_m x g_k grid of blocks, B into g_k x g_n and C into g_m x g_n, and
# forms R products
#     M_r = (sum_a U[a, r] A_a)(sum_b V[b, r] B_b),   C_c += W[c, r] M_r,
# blocks numbered row-major in their grid: a = i*g_k + l, b = l*g_n + j,
# c = i*g_n + j.  This scheme needs 15 products where the classical one needs
# 18 (Hopcroft and Kerr showed 15 is the least for <3,2,3>).  It was found for
# this package by a random walk over rank-reducing rewrites of the classical
# scheme modulo 2, then a choice of signs; its correctness rests on the Brent
# equations, which the tests check exactly, not on that search.  At most three
# C blocks per product (30 nonzeros in W), 32 in each of U and V.
# ---------------------------------------------------------------------------
B323_U = np.array([
    # r: 0   1   2   3   4   5   6   7   8   9  10  11  12  13  14
    [-1,  1,  1, -1,  0,  0,  0,  0,  0,  1,  0,  0,  0,  0,  0],   # A(0,0)
    [0,   1,  1,  0, -1,  0,  0,  0,  0,  1,  1,  0,  0,  0,  1],   # A(0,1)
    [0,   0,  0,  1, -1,  1,  0,  0,  0,  0,  0, -1, -1,  1,  0],   # A(1,0)
    [0,   0,  0,  0,  0,  1,  0,  0, -1,  0, -1, -1, -1,  0,  0],   # A(1,1)
    [1,  -1, -1,  0,  0,  0,  0, -1,  0,  0,  0,  0,  1,  0,  0],   # A(2,0)
    [0,   0, -1,  0,  0, -1,  1,  0,  1,  0,  0,  0,  1,  0,  0],   # A(2,1)
], dtype=np.int64)

B323_V = np.array([
    [1,   0,  0,  0,  0, -1,  0, -1,  1,  0,  0,  0,  1,  0,  0],   # B(0,0)
    [0,   0,  0,  1,  0, -1,  0,  0,  1,  0,  0,  0,  1,  1,  0],   # B(0,1)
    [-1,  1,  0, -1, -1,  0,  0,  0,  0, -1,  0,  0,  0,  0, -1],   # B(0,2)
    [-1,  1,  1,  0,  0,  0, -1,  0, -1,  0,  0,  0,  0,  0,  0],   # B(1,0)
    [0,   0,  0,  0,  1,  1,  0,  0, -1,  0, -1,  1,  0, -1,  0],   # B(1,1)
    [1,  -1, -1,  0,  0,  0,  0,  0,  0,  0,  1,  0,  0,  0,  1],   # B(1,2)
], dtype=np.int64)

B323_W = np.array([
    [-1,  1,  0,  0,  0,  0,  0,  1,  0,  0,  0,  0,  0,  0,  1],   # C(0,0)
    [0,   0,  0, -1, -1,  0,  0,  0,  0, -1,  0,  0,  0,  1,  0],   # C(0,1)
    [0,   0,  0,  0,  0,  0,  0,  0,  0, -1,  0,  0,  0,  0,  1],   # C(0,2)
    [0,   0,  0,  0,  0, -1, -1,  0,  1,  0,  0,  0,  0, -1,  0],   # C(1,0)
    [0,   0,  0,  0,  0,  0,  0,  0,  0,  0,  0, -1,  0,  1,  0],   # C(1,1)
    [0,   0,  0,  0,  1,  0,  0,  0,  0,  0, -1, -1,  0,  0,  1],   # C(1,2)
    [0,   0,  0,  0,  0,  0, -1,  1,  0,  0,  0,  0,  0,  0,  0],   # C(2,0)
    [0,   0,  0,  0,  0, -1,  0, -1,  0,  0,  0, -1,  1,  0,  0],   # C(2,1)
    [0,  -1,  1,  0,  0,  0, -1,  0,  0, -1,  0,  0,  0,  0,  0],   # C(2,2)
], dtype=np.int64)

# ---------------------------------------------------------------------------
# A <2,3,2; 11> basis: A split into 2 x 3 blocks, B into 3 x 2, C into 2 x 2
# (same block numbering).  C = A(:, 0:2) B(0:2, :) + A(:, 2) B(2, :): the seven
# products of Eq. (3) on the first part -- whose quadrant q = 2*row + col is
# block row*3 + col of A and row*2 + col of B and of C -- then the four block
# products A(i,2) B(2,j) added into C(i,j).  Eleven products where the classical
# scheme needs twelve.
# ---------------------------------------------------------------------------
def _b232_tables():
    U = np.zeros((6, 11), dtype=np.int64)
    V = np.zeros((6, 11), dtype=np.int64)
    W = np.zeros((4, 11), dtype=np.int64)
    for q in range(4):
        row, col = divmod(q, 2)
        U[row * 3 + col, :7] = STRASSEN_U[q]
        V[row * 2 + col, :7] = STRASSEN_V[q]
        W[row * 2 + col, :7] = STRASSEN_W[q]
    for i in range(2):
        for j in range(2):
            r = 7 + 2 * i + j
            U[i * 3 + 2, r] = 1
            V[2 * 2 + j, r] = 1
            W[i * 2 + j, r] = 1
    return U, V, W


B232_U, B232_V, B232_W = _b232_tables()

# block grid (g_m, g_k, g_n) of each one-level basis
BASIS_DIMS = {"strassen": (2, 2, 2), "winograd": (2, 2, 2), "b323": (3, 2, 3), "b232": (2, 3, 2)}


def basis_tables(basis: str = "strassen"):
    """(U, V, W) of a one-level basis, looked up when called."""
    g = globals()
    return tuple(g[f"{basis.upper()}_{x}"] for x in "UVW")


class _Bases(dict):
    def __missing__(self, key):
        return basis_tables(key)


BASES = _Bases()  # BASES["strassen"], BASES["winograd"]: the tables as they are now


def quadrant_rc(q: int) -> tuple[int, int]:
    """Row and column of quadrant q under the numbering of Eq. (2)."""
    return q // 2, q % 2


# ---------------------------------------------------------------------------
# Multi-level coefficients (Section 3.4).  The paper derives the 49 two-level
# instances from the general two-level primitive without printing them; the
# reading taken here is the Kronecker (tensor) power of the one-level table:
# instance (r1, r2) uses block (q1, q2) of each operand -- block q2 of
# quadrant q1 -- with coefficient U[q1, r1] * U[q2, r2] (likewise V, W).
# ---------------------------------------------------------------------------
def level_coefficients(levels: int, U=None, V=None, W=None):
    """Return (U_L, V_L, W_L, block_rc) for ``levels`` recursion levels.

    U_L has shape (4**L, 7**L).  Row index is the flattened tuple
    (q1, ..., qL) (q1 most significant), column index the flattened tuple
    (r1, ..., rL).  ``block_rc[b]`` gives the (block_row, block_col) of block b
    in the 2**L x 2**L grid of equal blocks.
    """
    U = STRASSEN_U if U is None else U
    V = STRASSEN_V if V is None else V
    W = STRASSEN_W if W is None else W
    UL = np.ones((1, 1), dtype=np.int64)
    VL = np.ones((1, 1), dtype=np.int64)
    WL = np.ones((1, 1), dtype=np.int64)
    for _ in range(levels):
        UL = np.kron(UL, U)
        VL = np.kron(VL, V)
        WL = np.kron(WL, W)
    block_rc = []
    for qs in itertools.product(range(4), repeat=levels):
        br = bc = 0
        for q in qs:
            r, c = quadrant_rc(q)
            br = 2 * br + r
            bc = 2 * bc + c
        block_rc.append((br, bc))
    return UL, VL, WL, block_rc


def brent_residual(levels: int = 1, U=None, V=None, W=None) -> int:
    """Sum of |residuals| of the Brent equations for the level-L coefficients.

    For block matrices with a g x g grid of blocks (g = 2**L) the product
    C = A B is the trilinear identity: the coefficient of A_(i,j) B_(j',l) in
    C_(i',l') must be 1 when j == j', i == i', l == l' and 0 otherwise.  A
    bilinear algorithm with coefficient matrices U, V, W reproduces it iff, for
    every such triple, sum_r U[a, r] V[b, r] W[c, r] equals that indicator.
    Returns 0 exactly when all g**6 equations hold.
    """
    UL, VL, WL, rc = level_coefficients(levels, U, V, W)
    nb = len(rc)
    total = 0
    for a in range(nb):
        i, j = rc[a]
        for b in range(nb):
            j2, l = rc[b]
            for c in range(nb):
                i2, l2 = rc[c]
                want = 1 if (j == j2 and i == i2 and l == l2) else 0
                got = int(np.sum(UL[a] * VL[b] * WL[c]))
                total += abs(got - want)
    return total


def operand_counts(levels: int, basis: str = "strassen"):
    """(W_A, W_B, W_C) of every instance: the number of nonzero coefficients
    in its A-operand, B-operand and C-update (Section 3.2)."""
    UL, VL, WL, _ = level_coefficients(levels, *basis_tables(basis))
    nnz = lambda M: [int(np.count_nonzero(M[:, r])) for r in range(M.shape[1])]
    return list(zip(nnz(UL), nnz(VL), nnz(WL)))


def variant_table(levels: int) -> Counter:
    """Counter mapping (W_A, W_B, W_C) -> number of instances."""
    return Counter(operand_counts(levels))


# ---------------------------------------------------------------------------
# Fringes (Section 3.5).  The paper pads the A and B tiles with zeros at the
# fringes.  Reading taken here: every dimension d is padded with implicit zeros
# to 2**L * h, where the bottom-level block size is
#     h = roundup(ceil(d / 2**L), align)
# so that all blocks at all levels are equal; blocks that fall past d are
# partially or entirely zero.  In exact arithmetic any padding gives the same
# product, so this rule only affects rounding.
# ---------------------------------------------------------------------------
def block_size(d: int, levels: int, align: int = 8) -> int:
    if levels == 0:
        return d
    g = 1 << levels
    h = -(-d // g)
    return -(-h // align) * align


def _pad(X: np.ndarray, rows: int, cols: int) -> np.ndarray:
    out = np.zeros((rows, cols), dtype=np.float64)
    out[: X.shape[0], : X.shape[1]] = X
    return out


def _strassen_rec(A: np.ndarray, B: np.ndarray, levels: int, U, V, W) -> np.ndarray:
    """M = A @ B for exactly even-sized padded operands, by Eq. (3) (or another
    one-level table U, V, W applied at every level)."""
    if levels == 0:
        return A @ B   # leaf: library FP64 matmul
    hm, hk = A.shape[0] // 2, A.shape[1] // 2
    hn = B.shape[1] // 2
    Aq = [A[:hm, :hk], A[:hm, hk:], A[hm:, :hk], A[hm:, hk:]]
    Bq = [B[:hk, :hn], B[:hk, hn:], B[hk:, :hn], B[hk:, hn:]]
    Cq = [np.zeros((hm, hn)) for _ in range(4)]
    for r in range(7):
        P = sum(U[q, r] * Aq[q] for q in range(4) if U[q, r])
        Q = sum(V[q, r] * Bq[q] for q in range(4) if V[q, r])
        M = _strassen_rec(P, Q, levels - 1, U, V, W)
        for q in range(4):
            if W[q, r]:
                Cq[q] += W[q, r] * M
    return np.block([[Cq[0], Cq[1]], [Cq[2], Cq[3]]])


def strassen(A, B, C=None, alpha: float = 1.0, beta: float = 0.0,
             levels: int = 1, align: int = 8, basis: str = "strassen") -> np.ndarray:
    """FP64 Strassen: C_out = alpha * A B + beta * C, ``levels`` levels.

    beta is applied first (beta == 0 or C is None means C is not read), the
    operands are padded per the fringe rule above, the seven products of
    Eq. (3) are formed recursively and the padding is dropped.
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    if levels == 0 or min(m, n, k) == 0:
        prod = A @ B if min(m, n, k) > 0 else np.zeros((m, n))
    else:
        g = 1 << levels
        Mp = g * block_size(m, levels, align)
        Np = g * block_size(n, levels, align)
        Kp = g * block_size(k, levels, align)
        prod = _strassen_rec(_pad(A, Mp, Kp), _pad(B, Kp, Np), levels, *basis_tables(basis))[:m, :n]
    out = alpha * prod
    if C is not None and beta != 0.0:
        out = out + beta * np.asarray(C, dtype=np.float64)
    return out


def grid_block(d: int, g: int, align: int = 8) -> int:
    """Block size of a dimension d split g ways: the fringe rule above with g in
    place of 2**L (g = 1 keeps d itself)."""
    if g == 1:
        return d
    h = -(-d // g)
    return -(-h // align) * align


def brent_residual_grid(dims, U, V, W) -> int:
    """Sum of |residuals| of the Brent equations of a one-level <g_m, g_k, g_n>
    basis: the coefficient of A_(i,l) B_(l',j) in C_(i',j') must be 1 when
    l == l', i == i', j == j' and 0 otherwise.  0 exactly when all hold."""
    gm, gk, gn = dims
    total = 0
    for i, l, l2, j, i2, j2 in itertools.product(range(gm), range(gk), range(gk), range(gn),
                                                 range(gm), range(gn)):
        want = 1 if (l == l2 and i == i2 and j == j2) else 0
        got = int(np.sum(U[i * gk + l] * V[l2 * gn + j] * W[i2 * gn + j2]))
        total += abs(got - want)
    return total


def table_matmul(A, B, C=None, alpha: float = 1.0, beta: float = 0.0,
                 basis: str = "b323", align: int = 8) -> np.ndarray:
    """FP64 one-level product by a basis table: C_out = alpha * A B + beta * C.

    Each dimension is padded with zeros to g * grid_block(d, g); the R products
    M_r = (sum_a U[a, r] A_a)(sum_b V[b, r] B_b) are formed with a library FP64
    matmul and added into C block c with coefficient W[c, r]; the padding is
    dropped.  beta == 0 or C None: C is not read."""
    U, V, W = basis_tables(basis)
    gm, gk, gn = BASIS_DIMS[basis]
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    if min(m, n, k) == 0:
        prod = np.zeros((m, n))
    else:
        hm, hk, hn = grid_block(m, gm, align), grid_block(k, gk, align), grid_block(n, gn, align)
        Ap = _pad(A, gm * hm, gk * hk)
        Bp = _pad(B, gk * hk, gn * hn)
        Ab = [Ap[i * hm:(i + 1) * hm, l * hk:(l + 1) * hk] for i in range(gm) for l in range(gk)]
        Bb = [Bp[l * hk:(l + 1) * hk, j * hn:(j + 1) * hn] for l in range(gk) for j in range(gn)]
        Cb = [np.zeros((hm, hn)) for _ in range(gm * gn)]
        for r in range(U.shape[1]):
            P = sum(U[a, r] * Ab[a] for a in range(gm * gk) if U[a, r])
            Q = sum(V[b, r] * Bb[b] for b in range(gk * gn) if V[b, r])
            M = P @ Q
            for c in range(gm * gn):
                if W[c, r]:
                    Cb[c] += W[c, r] * M
        prod = np.block([[Cb[i * gn + j] for j in range(gn)] for i in range(gm)])[:m, :n]
    out = alpha * prod
    if C is not None and beta != 0.0:
        out = out + beta * np.asarray(C, dtype=np.float64)
    return out


# ---------------------------------------------------------------------------
# Classical FP64 GEMM in C (Eq. 1).
# ---------------------------------------------------------------------------
_DTYPES = {np.dtype(np.float64): 0, np.dtype(np.float32): 1}
ORC_BF16 = 2
ORC_F16 = 3


def build(force: bool = False) -> str:
    """Compile oracle_gemm.c into _build/liboracle.so (gcc, OpenMP)."""
    src = os.path.join(_HERE, "oracle_gemm.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    os.makedirs(_BUILD_DIR, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                           src, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_gemm.restype = ctypes.c_int
        lib.oracle_gemm.argtypes = [
            ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
            ctypes.c_double, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64]
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def _code(X: np.ndarray, dtype_code):
    if dtype_code is not None:
        return dtype_code
    return _DTYPES[X.dtype]


def classical(A: np.ndarray, B: np.ndarray, C=None, alpha: float = 1.0,
              beta: float = 0.0, rows=None, a_code=None, b_code=None,
              c_code=None) -> np.ndarray:
    """FP64 C_out[rows] = alpha * A[rows] @ B + beta * C[rows].

    A, B, C are 2-D row-major numpy arrays (float64, float32, or uint16 holding
    bfloat16 / float16 bit patterns, in which case pass ``a_code``/``b_code``
    = ORC_BF16 or ORC_F16).  ``rows`` selects a sample of output rows.
    """
    lib = _load()
    A = np.ascontiguousarray(A)
    B = np.ascontiguousarray(B)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    if rows is None:
        nrows = m
        rows_arr = None
    else:
        rows_arr = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        nrows = rows_arr.size
    out = np.empty((nrows, n), dtype=np.float64)
    if C is not None:
        C = np.ascontiguousarray(C)
        cptr, ccode, ldc = C.ctypes.data, _code(C, c_code), C.shape[1]
    else:
        cptr, ccode, ldc = None, 0, n
    rc = lib.oracle_gemm(m, n, k, float(alpha),
                         A.ctypes.data, _code(A, a_code), k,
                         B.ctypes.data, _code(B, b_code), n,
                         float(beta), cptr, ccode, ldc,
                         out.ctypes.data, n,
                         None if rows_arr is None else rows_arr.ctypes.data, nrows)
    if rc != 0:
        raise ValueError("oracle_gemm: bad argument")
    return out


# ---------------------------------------------------------------------------
# Accuracy measure used to state results against the FP64 product.
# ---------------------------------------------------------------------------
def normwise_error(C, C64, A_norm_f: float, B_norm_f: float) -> float:
    """||C - C64||_F / (||A||_F * ||B||_F)."""
    d = np.asarray(C, dtype=np.float64) - np.asarray(C64, dtype=np.float64)
    denom = float(A_norm_f) * float(B_norm_f)
    num = float(np.sqrt(np.sum(d * d)))
    if denom == 0.0:
        return 0.0 if num == 0.0 else float("inf")
    return num / denom


def effective_tflops(m: int, n: int, k: int, seconds: float) -> float:
    """Eq. (4) of Section 4: 2 m n k / time, in units of 1e12 flop/s."""
    return 2.0 * m * n * k / seconds * 1e-12

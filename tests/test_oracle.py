"""Pins for the CPU oracle (no GPU).

Each test ties the oracle to something other than itself: the paper's printed
tables, the Brent equations of matrix multiplication, a library matmul, brute
force on tiny inputs, exact integer arithmetic and textbook special cases.
"""
import itertools
import os

import numpy as np
import pytest
import torch

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line)
    return rows


def _parse_terms(text, letter):
    vec = np.zeros(4, dtype=np.int64)
    for tok in text.split():
        sign = 1 if tok[0] == "+" else -1
        assert tok[1] == letter
        vec[int(tok[2])] = sign
    return vec


# --------------------------------------------------------------- coefficients
def test_coefficients_match_printed_products():
    """U, V, W equal the seven products of Eq. (3) as restated in the fixture."""
    rows = _read_rows("strassen_products.txt")
    assert len(rows) == 7
    for line in rows:
        r, a, b, c = [s.strip() for s in line.split("|")]
        r = int(r)
        np.testing.assert_array_equal(oracle.STRASSEN_U[:, r], _parse_terms(a, "A"))
        np.testing.assert_array_equal(oracle.STRASSEN_V[:, r], _parse_terms(b, "B"))
        np.testing.assert_array_equal(oracle.STRASSEN_W[:, r], _parse_terms(c, "C"))


@pytest.mark.parametrize("levels", [0, 1, 2])
def test_brent_equations_hold(levels):
    assert oracle.brent_residual(levels) == 0


def test_brent_check_detects_every_single_coefficient_change():
    base = [oracle.STRASSEN_U, oracle.STRASSEN_V, oracle.STRASSEN_W]
    for which in range(3):
        for q in range(4):
            for r in range(7):
                for val in (-1, 0, 1):
                    if base[which][q, r] == val:
                        continue
                    mats = [m.copy() for m in base]
                    mats[which][q, r] = val
                    assert oracle.brent_residual(1, *mats) > 0, (which, q, r, val)


def test_brent_check_detects_swapped_products():
    """Swapping the C-updates of two products must break the identity."""
    W = oracle.STRASSEN_W.copy()
    W[:, [0, 5]] = W[:, [5, 0]]
    assert oracle.brent_residual(1, oracle.STRASSEN_U, oracle.STRASSEN_V, W) > 0


def test_operand_count_table_matches_paper():
    """(W_A, W_B, W_C) -> instance counts of the Section 3.2 table."""
    want = {0: {}, 1: {}, 2: {}}
    for line in _read_rows("variant_table.txt"):
        lv, _var, wa, wb, wc, cnt = line.split()
        want[int(lv)][(int(wa), int(wb), int(wc))] = int(cnt)
    for lv in (0, 1, 2):
        assert dict(oracle.variant_table(lv)) == want[lv]


@pytest.mark.parametrize("levels", [0, 1, 2, 3])
def test_product_counts(levels):
    UL, VL, WL, rc = oracle.level_coefficients(levels)
    assert UL.shape == (4 ** levels, 7 ** levels)
    assert len(rc) == 4 ** levels
    assert len(set(rc)) == 4 ** levels
    # every block of A, B and C is referenced 12**L... (12 per level, Section 3.2)
    assert int(np.count_nonzero(UL)) == 12 ** levels
    assert int(np.count_nonzero(VL)) == 12 ** levels
    assert int(np.count_nonzero(WL)) == 12 ** levels


# ----------------------------------------------------------------- classical
def _brute(A, B, C, alpha, beta):
    m, k = A.shape
    n = B.shape[1]
    out = np.zeros((m, n))
    for i in range(m):
        for j in range(n):
            s = 0.0
            for l in range(k):
                s += float(A[i, l]) * float(B[l, j])
            out[i, j] = alpha * s + (beta * float(C[i, j]) if C is not None and beta != 0 else 0.0)
    return out


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (3, 5, 7), (8, 4, 9), (5, 1, 13)])
def test_classical_matches_brute_force(m, n, k):
    A = synth.uniform((m, k), 1).astype(np.float64)
    B = synth.uniform((k, n), 2).astype(np.float64)
    C = synth.uniform((m, n), 3).astype(np.float64)
    got = oracle.classical(A, B, C, alpha=1.5, beta=-0.5)
    want = _brute(A, B, C, 1.5, -0.5)
    # same operation order (l ascending, FP64) -> identical bits
    np.testing.assert_array_equal(got, want)


def test_classical_matches_library_matmul():
    A = synth.gaussian((67, 129), 4)
    B = synth.gaussian((129, 45), 5)
    got = oracle.classical(A, B)
    want = A.astype(np.float64) @ B.astype(np.float64)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_classical_row_sample_equals_full():
    A = synth.uniform((40, 33), 6)
    B = synth.uniform((33, 21), 7)
    full = oracle.classical(A, B)
    rows = [0, 39, 17, 17, 5]
    np.testing.assert_array_equal(oracle.classical(A, B, rows=rows), full[rows])


def test_classical_beta_zero_ignores_nan_in_c():
    A = synth.uniform((4, 4), 8)
    B = synth.uniform((4, 4), 9)
    C = np.full((4, 4), np.nan)
    out = oracle.classical(A, B, C, beta=0.0)
    assert np.all(np.isfinite(out))


@pytest.mark.parametrize("kind", ["bf16", "f16"])
def test_half_formats_convert_exactly(kind):
    """Every 16-bit pattern converts like torch's own conversion."""
    bits = np.arange(1 << 16, dtype=np.uint16)
    tdt = torch.bfloat16 if kind == "bf16" else torch.float16
    want = torch.from_numpy(bits.view(np.int16)).view(tdt).to(torch.float64).numpy()
    code = oracle.ORC_BF16 if kind == "bf16" else oracle.ORC_F16
    one = np.ones((1, 1))
    got = oracle.classical(one, bits.reshape(1, -1), b_code=code)[0]
    nan = np.isnan(want)
    np.testing.assert_array_equal(np.isnan(got), nan)
    np.testing.assert_array_equal(got[~nan], want[~nan])


# ------------------------------------------------------------------ strassen
def test_block_size_rule():
    assert oracle.block_size(4097, 2) == 1032
    assert oracle.block_size(4097, 1) == 2056
    assert oracle.block_size(16384, 2) == 4096
    assert oracle.block_size(16, 2) == 8
    assert oracle.block_size(30001, 2) == 7504
    assert oracle.block_size(7, 0) == 7
    for d in range(1, 200):
        for L in (1, 2):
            h = oracle.block_size(d, L)
            assert h % 8 == 0 and (1 << L) * h >= d and (1 << L) * (h - 8) < d


def test_textbook_2x2():
    rows = _read_rows("textbook_2x2.txt")
    A, B, C = [np.array([float(v) for v in r.split()]).reshape(2, 2) for r in rows]
    np.testing.assert_array_equal(oracle.strassen(A, B, levels=1, align=1), C)
    np.testing.assert_array_equal(oracle.strassen(A, B, levels=1), C)
    np.testing.assert_array_equal(oracle.classical(A, B), C)


SHAPES = [(1, 1, 1), (2, 2, 2), (3, 5, 7), (16, 16, 16), (17, 9, 31), (33, 40, 8),
          (64, 64, 64), (100, 37, 75), (5, 130, 3)]


@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("m,n,k", SHAPES)
def test_strassen_exact_on_small_integers(levels, m, n, k):
    A, B = synth.problem(m, n, k, seed=11 * m + n + k, dist="int")
    C = synth.small_int((m, n), 99)
    want = oracle.classical(A, B, C, alpha=2.0, beta=-3.0)
    for align in (1, 8):
        got = oracle.strassen(A, B, C, alpha=2.0, beta=-3.0, levels=levels, align=align)
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_strassen_float_close_to_library(levels):
    A, B = synth.problem(90, 70, 110, seed=3, dist="gaussian")
    got = oracle.strassen(A, B, levels=levels)
    want = A.astype(np.float64) @ B.astype(np.float64)
    err = oracle.normwise_error(got, want, np.linalg.norm(A), np.linalg.norm(B))
    assert err < 1e-14


@pytest.mark.parametrize("levels", [1, 2])
def test_strassen_identity(levels):
    A = synth.uniform((24, 24), 12).astype(np.float64)
    I = np.eye(24)
    np.testing.assert_array_equal(oracle.strassen(A, I, levels=levels, align=1), A)
    np.testing.assert_array_equal(oracle.strassen(I, A, levels=levels, align=1), A)


def test_planted_coefficient_mistake_is_caught(monkeypatch):
    """Plant a sign error in the oracle's W table: the integer pin must fail."""
    A, B = synth.problem(16, 16, 16, seed=21, dist="int")
    want = oracle.classical(A, B)
    W = oracle.STRASSEN_W.copy()
    W[3, 1] = +1           # C3 -= M1 becomes C3 += M1
    monkeypatch.setattr(oracle, "STRASSEN_W", W)
    got = oracle.strassen(A, B, levels=1)
    assert not np.array_equal(got, want)


def test_planted_operand_mistake_is_caught(monkeypatch):
    A, B = synth.problem(16, 16, 16, seed=22, dist="int")
    want = oracle.classical(A, B)
    U = oracle.STRASSEN_U.copy()
    U[:, [2, 3]] = U[:, [3, 2]]    # transposed operand assignment
    monkeypatch.setattr(oracle, "STRASSEN_U", U)
    assert not np.array_equal(oracle.strassen(A, B, levels=1), want)


# ------------------------------------------------------------------ measures
def test_normwise_error_closed_forms():
    A = np.ones((2, 2))
    B = np.ones((2, 2))
    C64 = A @ B
    assert oracle.normwise_error(C64, C64, 2.0, 2.0) == 0.0
    C = C64.copy()
    C[0, 0] += 3.0
    C[1, 1] -= 4.0
    assert oracle.normwise_error(C, C64, 2.0, 2.0) == pytest.approx(5.0 / 4.0)


def test_effective_tflops_formula():
    assert oracle.effective_tflops(1000, 1000, 1000, 1e-3) == pytest.approx(2.0)
    assert oracle.effective_tflops(16384, 16384, 16384, 1.0) == pytest.approx(2 * 16384 ** 3 * 1e-12)


# ------------------------------------------------ Strassen-Winograd basis (Section 6)
def _winograd_textbook(A, B):
    """One level of the Winograd variant in its shared-subexpression form (S1..S4, T1..T4,
    U2..U4), written independently of the oracle's per-product tables."""
    h, hk, hn = A.shape[0] // 2, A.shape[1] // 2, B.shape[1] // 2
    A11, A12, A21, A22 = A[:h, :hk], A[:h, hk:], A[h:, :hk], A[h:, hk:]
    B11, B12, B21, B22 = B[:hk, :hn], B[:hk, hn:], B[hk:, :hn], B[hk:, hn:]
    S1 = A21 + A22
    S2 = S1 - A11
    S3 = A11 - A21
    S4 = A12 - S2
    T1 = B12 - B11
    T2 = B22 - T1
    T3 = B22 - B12
    T4 = T2 - B21
    M1, M2, M3, M4 = A11 @ B11, A12 @ B21, S4 @ B22, A22 @ T4
    M5, M6, M7 = S1 @ T1, S2 @ T2, S3 @ T3
    U2 = M1 + M6
    U3 = U2 + M7
    U4 = U2 + M5
    return np.block([[M1 + M2, U4 + M3], [U3 - M4, U3 + M5]])


@pytest.mark.parametrize("levels", [1, 2])
def test_winograd_brent_equations_hold(levels):
    assert oracle.brent_residual(levels, *oracle.BASES["winograd"]) == 0


def test_winograd_brent_detects_every_single_coefficient_change():
    U, V, W = (M.copy() for M in oracle.BASES["winograd"])
    for M in (U, V, W):
        for idx in itertools.product(range(4), range(7)):
            old = M[idx]
            for new in {-1, 0, 1} - {old}:
                M[idx] = new
                assert oracle.brent_residual(1, U, V, W) > 0
            M[idx] = old


def test_winograd_tables_equal_the_shared_subexpression_form():
    A, B = synth.problem(16, 12, 10, seed=3, dist="int")
    np.testing.assert_array_equal(oracle.strassen(A, B, levels=1, align=1, basis="winograd"),
                                  _winograd_textbook(A.astype(np.float64), B.astype(np.float64)))


def test_winograd_operand_counts():
    c = oracle.operand_counts(1, "winograd")
    assert [x[0] for x in c] == [1, 1, 4, 1, 2, 3, 2]   # W_A
    assert [x[1] for x in c] == [1, 1, 1, 4, 2, 3, 2]   # W_B
    assert [x[2] for x in c] == [4, 1, 1, 1, 2, 3, 2]   # W_C
    assert sum(x[2] for x in c) == 14


@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("m,n,k", [(16, 16, 16), (37, 21, 50), (64, 64, 64), (5, 130, 3)])
def test_winograd_exact_on_small_integers(levels, m, n, k):
    A, B = synth.problem(m, n, k, seed=7 * m + k, dist="int")
    C = synth.small_int((m, n), 5)
    want = oracle.classical(A, B, C, alpha=2.0, beta=-3.0)
    got = oracle.strassen(A, B, C, alpha=2.0, beta=-3.0, levels=levels, basis="winograd")
    np.testing.assert_array_equal(got, want)


# ------------------------------------------------ a <3,2,3> basis of rank 15 (Section 6)
def _classical_table(gm, gk, gn):
    """The classical scheme of a <gm, gk, gn> grid as a basis table: one product per
    (i, l, j), A(i,l) times B(l,j) into C(i,j)."""
    R = gm * gk * gn
    U = np.zeros((gm * gk, R), np.int64)
    V = np.zeros((gk * gn, R), np.int64)
    W = np.zeros((gm * gn, R), np.int64)
    for r, (i, l, j) in enumerate(itertools.product(range(gm), range(gk), range(gn))):
        U[i * gk + l, r] = V[l * gn + j, r] = W[i * gn + j, r] = 1
    return U, V, W


def test_brent_grid_accepts_classical_schemes_and_rejects_misplaced_blocks():
    for dims in [(3, 2, 3), (2, 3, 2), (1, 2, 3), (2, 2, 2)]:
        U, V, W = _classical_table(*dims)
        assert oracle.brent_residual_grid(dims, U, V, W) == 0
        if dims[0] > 1:
            # the C blocks of one row taken for another's: a transposed or shifted index
            Wbad = np.roll(W, dims[2], axis=0)
            assert oracle.brent_residual_grid(dims, U, V, Wbad) > 0


def test_brent_grid_agrees_with_the_square_form_on_the_2x2_tables():
    for basis in ("strassen", "winograd"):
        assert oracle.brent_residual_grid((2, 2, 2), *oracle.BASES[basis]) == 0
    U, V, W = (M.copy() for M in oracle.BASES["strassen"])
    U[0, 0] = -U[0, 0]
    assert oracle.brent_residual_grid((2, 2, 2), U, V, W) == oracle.brent_residual(1, U, V, W) > 0


def test_b323_brent_equations_hold():
    U, V, W = oracle.BASES["b323"]
    assert U.shape == (6, 15) and V.shape == (6, 15) and W.shape == (9, 15)
    assert oracle.brent_residual_grid((3, 2, 3), U, V, W) == 0


def test_b323_brent_detects_every_single_coefficient_change():
    U, V, W = (M.copy() for M in oracle.BASES["b323"])
    for M in (U, V, W):
        for idx in itertools.product(range(M.shape[0]), range(15)):
            old = M[idx]
            for new in {-1, 0, 1} - {old}:
                M[idx] = new
                assert oracle.brent_residual_grid((3, 2, 3), U, V, W) > 0
            M[idx] = old


def test_b323_shape_of_the_scheme():
    U, V, W = oracle.BASES["b323"]
    assert set(np.unique(np.concatenate([U.ravel(), V.ravel(), W.ravel()]))) <= {-1, 0, 1}
    assert [int(np.count_nonzero(M)) for M in (U, V, W)] == [32, 32, 30]
    assert int(np.count_nonzero(W, axis=0).max()) == 3   # at most three C blocks per product


def test_b232_brent_equations_hold():
    U, V, W = oracle.BASES["b232"]
    assert U.shape == (6, 11) and V.shape == (6, 11) and W.shape == (4, 11)
    assert oracle.brent_residual_grid((2, 3, 2), U, V, W) == 0


def test_b232_brent_detects_every_single_coefficient_change():
    U, V, W = (M.copy() for M in oracle.BASES["b232"])
    for M in (U, V, W):
        for idx in itertools.product(range(M.shape[0]), range(11)):
            old = M[idx]
            for new in {-1, 0, 1} - {old}:
                M[idx] = new
                assert oracle.brent_residual_grid((2, 3, 2), U, V, W) > 0
            M[idx] = old


def test_b232_shape_of_the_scheme():
    U, V, W = oracle.BASES["b232"]
    assert set(np.unique(np.concatenate([U.ravel(), V.ravel(), W.ravel()]))) <= {-1, 0, 1}
    assert [int(np.count_nonzero(M)) for M in (U, V, W)] == [16, 16, 16]
    assert int(np.count_nonzero(W, axis=0).max()) == 2   # at most two C blocks per product


def test_grid_block_rule():
    assert oracle.grid_block(16384, 3) == 5464
    assert oracle.grid_block(16384, 2) == oracle.block_size(16384, 1) == 8192
    assert oracle.grid_block(1, 3) == 8
    assert oracle.grid_block(30001, 3, align=1) == 10001
    assert oracle.grid_block(77, 1) == 77


@pytest.mark.parametrize("m,n,k", [(18, 18, 12), (7, 11, 5), (64, 40, 33), (3, 200, 2), (100, 1, 9)])
@pytest.mark.parametrize("align", [1, 8])
@pytest.mark.parametrize("basis", ["b323", "b232"])
def test_table_bases_exact_on_small_integers(m, n, k, align, basis):
    A, B = synth.problem(m, n, k, seed=11 * m + n, dist="int")
    C = synth.small_int((m, n), 5)
    want = oracle.classical(A, B, C, alpha=2.0, beta=-3.0)
    got = oracle.table_matmul(A, B, C, alpha=2.0, beta=-3.0, basis=basis, align=align)
    np.testing.assert_array_equal(got, want)


def test_table_matmul_with_the_strassen_table_is_one_level_strassen():
    A, B = synth.problem(40, 24, 36, seed=5, dist="uniform")
    np.testing.assert_array_equal(oracle.table_matmul(A, B, basis="strassen"),
                                  oracle.strassen(A, B, levels=1))


def test_table_matmul_empty_and_beta_only():
    A, B = np.zeros((6, 0)), np.zeros((0, 9))
    C = synth.small_int((6, 9), 5)
    np.testing.assert_array_equal(oracle.table_matmul(A, B, C, beta=2.0), 2.0 * C)
    assert oracle.table_matmul(np.zeros((0, 4)), np.zeros((4, 3))).shape == (0, 3)


@pytest.mark.parametrize("basis", ["b323", "b232"])
def test_table_bases_float_agree_with_classical_within_fp64_rounding(basis):
    A, B = synth.problem(96, 90, 64, seed=9, dist="uniform")
    got = oracle.table_matmul(A, B, basis=basis)
    want = oracle.classical(A, B)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(A).max() * np.abs(B).max() * 64

"""C-ABI library checks that need no GPU: it builds, loads, exports every declared
symbol, rejects bad arguments before launching anything, and its product tables
satisfy the Brent equations and agree with the oracle's restatement of Eq. (3)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1808_07984_gb300 as fmm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    fmm.build()
    return fmm.load()


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(fmm_\w+)\s*\(", text)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "fmm_gemm" in names and "fmm_device_status" in names
    for name in names:
        assert hasattr(lib, name), name


def test_version(lib):
    assert b"sm_103a" in lib.fmm_version()


@pytest.mark.parametrize("levels", [0, 1, 2])
def test_library_tables_match_oracle(lib, levels):
    U, V, W = fmm.product_table(levels)
    UL, VL, WL, rc = oracle.level_coefficients(levels)
    g = 1 << levels
    for row, (bi, bj) in enumerate(rc):
        np.testing.assert_array_equal(U[bi * g + bj], UL[row])
        np.testing.assert_array_equal(V[bi * g + bj], VL[row])
        np.testing.assert_array_equal(W[bi * g + bj], WL[row])


@pytest.mark.parametrize("levels", [0, 1, 2])
def test_library_winograd_tables_match_oracle(lib, levels):
    U, V, W = fmm.product_table(levels, "winograd")
    UL, VL, WL, rc = oracle.level_coefficients(levels, *oracle.BASES["winograd"])
    g = 1 << levels
    for row, (bi, bj) in enumerate(rc):
        np.testing.assert_array_equal(U[bi * g + bj], UL[row])
        np.testing.assert_array_equal(V[bi * g + bj], VL[row])
        np.testing.assert_array_equal(W[bi * g + bj], WL[row])


@pytest.mark.parametrize("levels", [1, 2])
def test_library_tables_satisfy_brent(lib, levels):
    """Independent of the oracle's arrays: rebuild the trilinear identity."""
    U, V, W = fmm.product_table(levels)
    g = 1 << levels
    R = 7 ** levels
    T = np.einsum("ar,br,cr->abc", U.astype(np.int64), V.astype(np.int64), W.astype(np.int64))
    for a in range(g * g):
        i, j = divmod(a, g)
        for b in range(g * g):
            j2, l = divmod(b, g)
            for c in range(g * g):
                i2, l2 = divmod(c, g)
                assert T[a, b, c] == int(j == j2 and i == i2 and l == l2)
    assert U.shape == (g * g, R)


def test_workspace_sizes(lib):
    # packed split3: two 16-bit arrays per operand, 7^L products of h x h blocks
    assert fmm.workspace_size(512, 512, 512, 1, "split3") == 2 * 2 * (7 * 256 * 256 * 2)
    assert fmm.workspace_size(512, 512, 512, 0, "split3") == 2 * 2 * (512 * 512 * 2)
    assert fmm.workspace_size(512, 512, 512, 1, "plain_bf16") == 2 * (7 * 256 * 256 * 2)
    assert fmm.workspace_size(0, 512, 512, 1, "split3") == 0
    with pytest.raises(fmm.FmmError):
        fmm.workspace_size(16, 16, 16, 3, "split3")


def _call(lib, m=16, n=16, k=16, lda=16, ldb=16, ldc=16, levels=1, variant=0,
          A=0x10000, B=0x20000, C=0x30000, ws=0x100000, ws_bytes=1 << 30):
    return lib.fmm_gemm(m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, levels, variant,
                        ws, ws_bytes, None)


def test_argument_errors_need_no_gpu(lib):
    # these are rejected by host-side checks before any CUDA call
    assert _call(lib, m=-1) == 1
    assert _call(lib, lda=8) == 1
    assert _call(lib, ldb=8) == 1
    assert _call(lib, ldc=8) == 1
    assert _call(lib, levels=3) == 3
    assert _call(lib, variant=9) == 3
    assert _call(lib, C=0x10000 + 64) == 1               # C overlaps A
    assert _call(lib, ws_bytes=16) == 4                  # workspace too small
    assert _call(lib, ws=0x100010) == 2                  # workspace misaligned
    assert b"workspace" in lib.fmm_last_error() or b"aligned" in lib.fmm_last_error()
    assert _call(lib, m=0) == 0                          # empty problem: no-op
    # block sizes beyond the 32-bit tile coordinates are refused on the host
    assert _call(lib, m=1 << 33, ldc=16) == 1
    assert _call(lib, n=1 << 33, ldb=1 << 33, ldc=1 << 33) == 1


def test_oracle_is_not_linked_by_the_library():
    so = fmm.lib_path()
    data = open(so, "rb").read()
    assert b"oracle_gemm" not in data


def _call_ex(lib, levels=1, algo=0, variant=0, **opt):
    o = fmm._Options()
    for key, v in opt.items():
        setattr(o, key, v)
    o.algo = algo
    return lib.fmm_gemm_ex(16, 16, 16, 1.0, 0x10000, 16, 0x20000, 16, 0.0, 0x30000, 16, levels, variant,
                           0x100000, 1 << 30, None, ctypes.byref(o))


def test_option_errors_need_no_gpu(lib):
    """Every option value outside its range, and every unsupported combination, is refused by
    the host before any CUDA call (FMM_ERR_ARG = 1, FMM_ERR_UNSUPPORTED = 3)."""
    assert _call_ex(lib, cta_pair=3) == 1
    assert _call_ex(lib, schedule=5) == 1
    assert _call_ex(lib, bk=48) == 1
    assert _call_ex(lib, pipeline=3) == 1
    assert _call_ex(lib, basis=4) == 1
    assert _call_ex(lib, basis=-1) == 1
    assert _call_ex(lib, deterministic=2) == 1
    assert _call_ex(lib, outer_scaling=2) == 1
    assert _call_ex(lib, fringe=2) == 1
    assert _call_ex(lib, cta_pair=2, bk=32) == 3            # pairs need 64-deep stages
    assert _call_ex(lib, levels=2, basis=1) == 3            # Winograd: one level
    assert _call_ex(lib, algo=2, outer_scaling=1) == 3      # fused: no outside scaling
    assert _call_ex(lib, algo=3, levels=1) == 3             # hybrid: two levels
    assert _call_ex(lib, algo=9) == 3
    assert _call_ex(lib, levels=2, basis=2) == 3            # <3,2,3>: one level
    assert _call_ex(lib, algo=3, levels=2, basis=2) == 3    # <3,2,3>: no hybrid (two-level) form
    assert _call_ex(lib, basis=2, pipeline=2) == 3          # <3,2,3>: one table pass
    assert _call_ex(lib, fused_kernel=3) == 1
    assert _call_ex(lib, fused_kernel=-1) == 1
    assert _call_ex(lib, store_first=3) == 1
    assert _call_ex(lib, algo=2, cta_pair=1, fused_kernel=2) == 3  # tensor-memory kernel: CTA pairs
    # 16-bit operands on chip: tensor-memory kernel (CTA pairs); FP16 scaling: Strassen's basis
    assert _call_ex(lib, algo=2, variant=1, cta_pair=1) == 3
    assert _call_ex(lib, algo=2, variant=1, fused_kernel=1) == 3
    assert _call_ex(lib, algo=2, variant=2, basis=2) == 3
    assert _call_ex(lib, algo=2, variant=2, basis=1) == 3


def test_options_struct_matches_the_header():
    """The binding's fmm_options has the header's fields in the header's order and size."""
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fmm.h")).read()
    body = hdr[hdr.index("typedef struct fmm_options {"):hdr.index("} fmm_options;")]
    fields = re.findall(r"^\s*int\s+(\w+)(\[(\d+)\])?;", body, re.M)
    names = [f[0] for f in fields]
    assert names == [f[0] for f in fmm._Options._fields_]
    assert ctypes.sizeof(fmm._Options) == 4 * sum(int(f[2]) if f[2] else 1 for f in fields)


def test_basis_shapes(lib):
    assert fmm.basis_shape(0, "b323") == (1, 1, 1, 1)
    assert fmm.basis_shape(1, "b323") == (3, 2, 3, 15)
    assert fmm.basis_shape(2, "strassen") == (4, 4, 4, 49)
    assert fmm.basis_shape(1, "winograd") == (2, 2, 2, 7)
    with pytest.raises(fmm.FmmError):
        fmm.basis_shape(2, "b323")
    with pytest.raises(fmm.FmmError):
        fmm.basis_shape(1, 7)


def test_library_b323_tables_match_oracle_and_brent(lib):
    U, V, W = fmm.product_table(1, "b323")
    OU, OV, OW = oracle.BASES["b323"]
    np.testing.assert_array_equal(U, OU)
    np.testing.assert_array_equal(V, OV)
    np.testing.assert_array_equal(W, OW)
    # and the exported arrays on their own satisfy the trilinear identity of <3,2,3>
    for i, l, l2, j, i2, j2 in np.ndindex(3, 2, 2, 3, 3, 3):
        got = int(np.sum(U[i * 2 + l].astype(np.int64) * V[l2 * 3 + j] * W[i2 * 3 + j2]))
        assert got == (1 if (l == l2 and i == i2 and j == j2) else 0)
    # at most three destinations per product: within the kernels' four-entry lists
    assert int(np.count_nonzero(W, axis=0).max()) <= 4


def test_library_b232_tables_match_oracle_and_brent(lib):
    assert fmm.basis_shape(1, "b232") == (2, 3, 2, 11)
    with pytest.raises(fmm.FmmError):
        fmm.basis_shape(2, "b232")
    U, V, W = fmm.product_table(1, "b232")
    OU, OV, OW = oracle.BASES["b232"]
    np.testing.assert_array_equal(U, OU)
    np.testing.assert_array_equal(V, OV)
    np.testing.assert_array_equal(W, OW)
    for i, l, l2, j, i2, j2 in np.ndindex(2, 3, 3, 2, 2, 2):
        got = int(np.sum(U[i * 3 + l].astype(np.int64) * V[l2 * 2 + j] * W[i2 * 2 + j2]))
        assert got == (1 if (l == l2 and i == i2 and j == j2) else 0)
    # refused combinations (host checks, no GPU)
    assert _call_ex(lib, levels=2, basis=3) == 3
    assert _call_ex(lib, levels=1, basis=3, pipeline=2) == 3
    assert _call_ex(lib, algo=3, levels=2, basis=3) == 3
    assert _call_ex(lib, basis=4) == 1


def test_b323_workspace_sizes(lib):
    # 15 products of (h_m x h_k) A sums and (h_k x h_n) B sums, BF16 hi and lo
    m = n = k = 3000
    hm, hk, hn = oracle.grid_block(m, 3), oracle.grid_block(k, 2), oracle.grid_block(n, 3)
    a = -(-15 * hm * hk * 2 // 256) * 256
    b = -(-15 * hk * hn * 2 // 256) * 256
    assert fmm.workspace_size(m, n, k, 1, basis="b323") == 2 * (a + b)
    assert fmm.workspace_size(m, n, k, 1, "plain_bf16", basis="b323") == a + b


@pytest.mark.parametrize("levels,basis,want", [(1, 0, [1, 4, 2]), (2, 0, [1, 12, 24, 12]), (1, 1, None), (1, 2, None),
                                               (1, 3, None)])
def test_store_first_phases_are_a_valid_order(lib, levels, basis, want):
    """Host-side plan of the store-first launch phases (no GPU): every C block that some
    product updates is stored by exactly one product, that product runs in a strictly earlier
    phase than every other product updating the block, and no phase holds two products that
    touch a block one of them stores.  Strassen's phase sizes are the documented ones."""
    lib.fmm_store_phases.restype = ctypes.c_int
    lib.fmm_store_phases.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    gm, gk, gn, R = fmm.basis_shape(levels, basis)
    _, _, W = fmm.product_table(levels, basis)
    phase = np.zeros(R, dtype=np.int32)
    store = np.zeros(gm * gn * R, dtype=np.int8)
    nph = lib.fmm_store_phases(levels, basis, phase.ctypes.data, store.ctypes.data)
    assert nph >= 1
    store = store.reshape(gm * gn, R)
    assert set(np.unique(phase)) == set(range(nph))
    for c in range(gm * gn):
        touch = np.nonzero(W[c])[0]
        if len(touch) == 0:
            continue
        storers = np.nonzero(store[c])[0]
        assert len(storers) == 1, (c, storers)
        s = storers[0]
        assert W[c, s] != 0
        for r in touch:
            if r != s:
                assert phase[r] > phase[s], (c, r, s)
    for ph in range(nph):
        members = np.nonzero(phase == ph)[0]
        for c in range(gm * gn):
            if store[c, members].any():
                assert np.count_nonzero(W[c, members]) == 1, (ph, c)
    if want is not None:
        assert [int(np.count_nonzero(phase == p)) for p in range(nph)] == want
    assert lib.fmm_store_phases(0, 0, phase.ctypes.data, store.ctypes.data) == -1


def test_fused_workspace_is_the_fp16_panel_maxima(lib):
    """The fused algorithm stores no operand sums: no workspace for FP32 and BF16 operands, and
    for FP16 operands only the panel maxima of the operand sums (7^L products x (128-row panels
    of A + 256-column panels of B) x 4 bytes, rounded up to 256)."""
    assert fmm.workspace_size(1024, 1024, 1024, 1, "split3", algo="fused") == 0
    assert fmm.workspace_size(1024, 1024, 1024, 1, "bf16", algo="fused") == 0
    for levels, R in ((1, 7), (2, 49)):
        h = 1024 >> levels
        panels = -(-h // 128) + -(-h // 256)
        want = -(-(R * panels * 4) // 256) * 256
        assert fmm.workspace_size(1024, 1024, 1024, levels, "f16", algo="fused") == want

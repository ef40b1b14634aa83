"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Integer inputs must agree bit for bit (every operand sum, product and partial sum
is an integer below 2**24, exact in BF16 and FP32).  Floating-point inputs must
agree within the normwise bound ||C - C64||_F / (||A||_F ||B||_F) <= tol, with tol
from ``tests/bounds.py``: 1e-6 for the FP32-accurate split arithmetic wherever that
arithmetic itself allows it, its own derived bound at smaller depths.
"""

import numpy as np
import pytest
import torch

import oracle
import paper_1808_07984_gb300 as fmm
import synth
from bounds import tolerance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fmm.build()
    fmm.load()
    oracle.build()


def _to_device(X, ld_pad, dtype):
    rows, cols = X.shape
    t = torch.zeros((rows, cols + ld_pad), dtype=dtype, device="cuda")
    t[:, :cols] = torch.from_numpy(np.ascontiguousarray(X)).to(dtype=dtype, device="cuda")
    return t[:, :cols]


def run(m, n, k, levels, variant="split3", dist="uniform", seed=0, alpha=1.0, beta=0.0,
        tile_n=0, pads=(0, 0, 0), c_fill=None, rows=None, schedule="auto", algo="auto", bk=0,
        cta_pair=None, round_tiles=0, pipeline=None, fringe="pad", basis="strassen",
        deterministic=False, outer_scaling=False, fused_kernel="auto", store_first=None):
    A, B = synth.problem(m, n, k, seed, dist)
    in_dtype = {"bf16": torch.bfloat16, "f16": torch.float16}.get(variant, torch.float32)
    Ad = _to_device(A, pads[0], in_dtype)
    Bd = _to_device(B, pads[1], in_dtype)
    C0 = None
    if beta != 0.0:
        C0 = synth.uniform((m, n), seed + 5)
        Cd = _to_device(C0, pads[2], torch.float32)
    else:
        Cd = _to_device(np.zeros((m, n), np.float32), pads[2], torch.float32)
        if c_fill is not None:
            Cd.fill_(c_fill)
    fmm.gemm(Ad, Bd, Cd, alpha=alpha, beta=beta, levels=levels, variant=variant, tile_n=tile_n,
             schedule=schedule, algo=algo, bk=bk, cta_pair=cta_pair, round_tiles=round_tiles,
             pipeline=pipeline, fringe=fringe, basis=basis, deterministic=deterministic,
             outer_scaling=outer_scaling, fused_kernel=fused_kernel, store_first=store_first)
    fmm.device_status()
    # sampled rows are gathered on the device (a full-size C is several GB)
    Csel = Cd if rows is None else Cd[torch.from_numpy(np.asarray(rows)).to(Cd.device)]
    C = Csel.cpu().numpy().astype(np.float64)
    if variant in ("bf16", "f16"):
        # the oracle sees exactly the 16-bit values the GPU saw
        code = oracle.ORC_BF16 if variant == "bf16" else oracle.ORC_F16
        Ab = Ad.cpu().contiguous().view(torch.int16).numpy().view(np.uint16)
        Bb = Bd.cpu().contiguous().view(torch.int16).numpy().view(np.uint16)
        C64 = oracle.classical(Ab, Bb, C0, alpha, beta, rows=rows, a_code=code, b_code=code)
        An = float(np.linalg.norm(Ad.float().cpu().numpy()))
        Bn = float(np.linalg.norm(Bd.float().cpu().numpy()))
    else:
        C64 = oracle.classical(A, B, C0, alpha, beta, rows=rows)
        An = float(np.linalg.norm(A.astype(np.float64)))
        Bn = float(np.linalg.norm(B.astype(np.float64)))
    if rows is not None:
        An = float(np.linalg.norm(A[rows].astype(np.float64)))
    return C, C64, An, Bn


# ------------------------------------------------------------ exact integers
@pytest.mark.parametrize("variant", ["split3", "plain_bf16", "bf16", "f16"])
@pytest.mark.parametrize("levels", [0, 1, 2])
def test_int16_cube_bit_exact(variant, levels):
    C, C64, _, _ = run(16, 16, 16, levels, variant, dist="int", seed=1)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("tile_n", [128, 256])
@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("m,n,k", [(300, 520, 200), (129, 257, 65), (1, 300, 1), (520, 8, 400)])
def test_int_ragged_bit_exact(m, n, k, levels, tile_n):
    C, C64, _, _ = run(m, n, k, levels, "split3", dist="int", seed=m + n + k, tile_n=tile_n)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("schedule", ["product", "rounds"])
@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("m,n,k", [(1000, 1200, 300), (136, 1800, 64)])
def test_int_schedules_bit_exact(m, n, k, levels, schedule):
    """Both work orders, with enough tiles for several rounds and a partial last round."""
    C, C64, _, _ = run(m, n, k, levels, "split3", dist="int", seed=m + k, schedule=schedule)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("cta_pair", [False, True])
@pytest.mark.parametrize("tile_n", [128, 256])
@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("m,n,k", [(300, 520, 200), (129, 257, 65), (1000, 1200, 300), (520, 8, 400),
                                   (1, 300, 1)])
def test_cta_pair_and_single_cta_bit_exact(m, n, k, levels, tile_n, cta_pair):
    """Both tensor-core kernels: one CTA per 128-row tile, and CTA pairs sharing 256-row tiles
    (odd numbers of 128-row tiles leave the odd CTA of the last pair with rows past the end)."""
    C, C64, _, _ = run(m, n, k, levels, "split3", dist="int", seed=5 * m + k, tile_n=tile_n,
                       cta_pair=cta_pair)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("cta_pair", [False, True])
@pytest.mark.parametrize("round_tiles", [1, 3, 7, 1000])
@pytest.mark.parametrize("levels", [1, 2])
def test_round_sizes_bit_exact(levels, round_tiles, cta_pair):
    """Tile rounds of any size (several full rounds and a partial last one)."""
    C, C64, _, _ = run(1000, 1200, 300, levels, "split3", dist="int", seed=11 + round_tiles,
                       schedule="rounds", round_tiles=round_tiles, cta_pair=cta_pair)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("cta_pair", [False, True])
@pytest.mark.parametrize("levels", [0, 1, 2])
def test_f16_scaled_odd_tile_rows(levels, cta_pair):
    """Scaled FP16 with an odd number of 128-row panels (the odd CTA of the last pair has none)."""
    m, n, k = 300, 200, 150
    C, C64, An, Bn = run(m, n, k, levels, "f16", seed=21, cta_pair=cta_pair)
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance("f16", levels, k)
    C, C64, _, _ = run(m, n, k, levels, "f16", dist="int", seed=22, cta_pair=cta_pair)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("cta_pair", [False, True])
@pytest.mark.parametrize("levels", [0, 1, 2])
def test_unaligned_ldc_both_kernels(levels, cta_pair):
    """Element-wise write-back (ldc odd) from both tensor-core kernels."""
    C, C64, _, _ = run(513, 300, 130, levels, "split3", dist="int", seed=19, pads=(0, 0, 1),
                       cta_pair=cta_pair)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("pipeline", [False, True])
@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("m,n,k", [(300, 520, 200), (129, 257, 65), (1000, 1200, 300), (520, 8, 400),
                                   (1, 300, 1)])
def test_pipelined_sums_bit_exact(m, n, k, levels, pipeline):
    """Operand sums formed per top-level product on a side stream, overlapped with the
    tensor-core kernel of the products whose sums exist (and the plain order)."""
    C, C64, _, _ = run(m, n, k, levels, "split3", dist="int", seed=13 * m + k, pipeline=pipeline)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("variant", ["plain_bf16", "bf16", "f16"])
@pytest.mark.parametrize("levels", [1, 2])
def test_pipelined_other_variants(levels, variant):
    C, C64, _, _ = run(300, 260, 200, levels, variant, dist="int", seed=17, pipeline=True)
    np.testing.assert_array_equal(C, C64)
    C, C64, An, Bn = run(300, 260, 200, levels, variant, seed=18, pipeline=True)
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance(variant, levels, 200)


@pytest.mark.parametrize("pad_c", [0, 1])
@pytest.mark.parametrize("levels", [1, 2])
def test_pipelined_alpha_beta(levels, pad_c):
    """beta pass then pipelined sums and products; ldc aligned (TMA reductions) or odd."""
    m, n, k = 257, 300, 130
    A, B = synth.problem(m, n, k, 23, "int")
    C0 = synth.small_int((m, n), 24)
    Cd = _to_device(C0, pad_c, torch.float32)
    fmm.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), Cd, alpha=-2.0, beta=3.0,
             levels=levels, pipeline=True)
    fmm.device_status()
    np.testing.assert_array_equal(Cd.cpu().numpy(), oracle.classical(A, B, C0, -2.0, 3.0))


def test_pipelined_back_to_back_calls_share_workspace():
    """Consecutive pipelined calls on one stream with one workspace: the side stream of a call
    starts only after the previous call's products have read the shared sums."""
    A1, B1 = synth.problem(700, 600, 500, 31, "int")
    A2, B2 = synth.problem(700, 600, 500, 32, "int")
    d = [torch.from_numpy(X).cuda() for X in (A1, B1, A2, B2)]
    ws = torch.empty(fmm.workspace_size(700, 600, 500, 2), dtype=torch.uint8, device="cuda")
    C1 = fmm.gemm(d[0], d[1], levels=2, workspace=ws, pipeline=True)
    C2 = fmm.gemm(d[2], d[3], levels=2, workspace=ws, pipeline=True)
    fmm.device_status()
    np.testing.assert_array_equal(C1.cpu().numpy(), oracle.classical(A1, B1))
    np.testing.assert_array_equal(C2.cpu().numpy(), oracle.classical(A2, B2))


def test_pipelined_call_in_cuda_graph():
    """A pipelined call captured in a CUDA graph (its side stream joins the capture through
    the fork event) and replayed: the replay computes the same exact product."""
    A, B = synth.problem(600, 520, 400, 41, "int")
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = torch.zeros((600, 520), device="cuda")
    ws = torch.empty(fmm.workspace_size(600, 520, 400, 2), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        fmm.gemm(Ad, Bd, C, levels=2, workspace=ws, pipeline=True, stream=s)  # creates the side stream
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fmm.gemm(Ad, Bd, C, levels=2, workspace=ws, pipeline=True, stream=s)
    C.zero_()
    g.replay()
    torch.cuda.synchronize()
    fmm.device_status()
    np.testing.assert_array_equal(C.cpu().numpy(), oracle.classical(A, B))


@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("m,n,k", [(300, 520, 200), (129, 257, 65), (1000, 1200, 300), (33, 70, 17),
                                   (5, 7, 3), (520, 8, 400), (64, 64, 64)])
def test_peeled_fringes_bit_exact(m, n, k, levels):
    """Dynamic peeling: Strassen on the evenly splitting core, classical k, row and column
    strips (or one classical product when there is no core)."""
    C, C64, _, _ = run(m, n, k, levels, "split3", dist="int", seed=29 * m + k, fringe="peel")
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("levels", [1, 2])
def test_peeled_alpha_beta_unaligned(levels):
    m, n, k = 257, 301, 131
    A, B = synth.problem(m, n, k, 37, "int")
    C0 = synth.small_int((m, n), 38)
    Cd = _to_device(C0, 1, torch.float32)
    fmm.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), Cd, alpha=3.0, beta=-2.0,
             levels=levels, fringe="peel")
    fmm.device_status()
    np.testing.assert_array_equal(Cd.cpu().numpy(), oracle.classical(A, B, C0, 3.0, -2.0))


@pytest.mark.parametrize("variant", ["split3", "plain_bf16", "bf16", "f16"])
def test_peeled_float(variant):
    C, C64, An, Bn = run(500, 333, 271, 2, variant, seed=39, fringe="peel")
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance(variant, 2, 271)


def test_peeled_odd_30001_29999_4097_sampled_rows():
    rows = np.array([0, 1, 29983, 29984, 30000])  # core rows and bottom-strip rows
    C, C64, An, Bn = run(30001, 29999, 4097, 2, "split3", dist="gaussian", seed=5, rows=rows,
                         fringe="peel")
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance("split3", 2, 4097)


@pytest.mark.parametrize("opts", [{}, {"algo": "fused"}, {"pipeline": True}, {"pads": (0, 0, 1)},
                                  {"cta_pair": False}, {"fringe": "peel"}])
@pytest.mark.parametrize("m,n,k", [(300, 520, 200), (129, 257, 65), (1000, 1200, 300), (1, 300, 1)])
def test_winograd_basis_bit_exact(m, n, k, opts):
    """The Strassen-Winograd variant's seven products (one level) through every path."""
    o = dict(opts)
    pads = o.pop("pads", (0, 0, 0))
    if o.get("algo") == "fused":
        pads = (_pad4(k), _pad4(n), 0)
    C, C64, _, _ = run(m, n, k, 1, "split3", dist="int", seed=43 * m + k, basis="winograd", pads=pads, **o)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("variant", ["split3", "plain_bf16", "bf16", "f16"])
def test_winograd_basis_float(variant):
    C, C64, An, Bn = run(600, 520, 400, 1, variant, seed=45, basis="winograd")
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance(variant, 1, 400)


# ------------------------------------------------ classical 16-bit operands read in place
@pytest.mark.parametrize("variant", ["bf16", "f16"])
@pytest.mark.parametrize("pads", [(0, 0, 0), (1, 0, 0), (0, 3, 0), (1, 1, 1), (8, 8, 0)])
@pytest.mark.parametrize("m,n,k", [(300, 520, 200), (129, 257, 65), (1000, 1000, 1000)])
def test_classical_16bit_operands_in_place_or_packed(variant, pads, m, n, k):
    """L = 0 with BF16/FP16 operands: the tensor-core kernel reads an operand straight from
    the caller's buffer when TMA can address it (16-byte aligned rows), else from the
    converted copy; every mix of the two gives the exact product on small integers."""
    C, C64, _, _ = run(m, n, k, 0, variant, dist="int", seed=61 * m + k, pads=pads)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("variant", ["bf16", "f16"])
@pytest.mark.parametrize("pads", [(0, 0, 0), (1, 0, 0)])
def test_classical_16bit_float_in_place(variant, pads):
    C, C64, An, Bn = run(700, 640, 512, 0, variant, seed=63, pads=pads, alpha=0.5, beta=2.0)
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance(variant, 0, 512)


def test_classical_16bit_in_place_needs_no_workspace():
    """Both operands read in place: the call runs with no workspace at all; an operand that
    has to be converted (rows not 16-byte aligned) still asks for it (FMM_ERR_WORKSPACE)."""
    m, n, k = 512, 384, 256
    A, B = synth.problem(m, n, k, 79, "int")
    L = fmm.load()
    s = torch.cuda.current_stream().cuda_stream
    for variant, dt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        Ad = torch.from_numpy(A).to(dt).cuda()
        Bd = torch.from_numpy(B).to(dt).cuda()
        C = torch.full((m, n), float("nan"), device="cuda")
        st = L.fmm_gemm(m, n, k, 1.0, Ad.data_ptr(), k, Bd.data_ptr(), n, 0.0, C.data_ptr(), n, 0,
                        fmm.VARIANTS[variant], None, 0, s)
        assert st == 0, fmm.load().fmm_last_error()
        fmm.device_status()
        np.testing.assert_array_equal(C.cpu().numpy(), oracle.classical(A, B))
        Ap = torch.zeros((m, k + 1), dtype=dt, device="cuda")
        st = L.fmm_gemm(m, n, k, 1.0, Ap.data_ptr(), k + 1, Bd.data_ptr(), n, 0.0, C.data_ptr(), n, 0,
                        fmm.VARIANTS[variant], None, 0, s)
        assert st == 4


def test_classical_f16_in_place_large_magnitudes():
    """FP16 values near the top of the range: read in place without panel scaling, their
    products are exact in the FP32 accumulator."""
    m, n, k = 256, 384, 128
    A = (synth.small_int((m, k), 5) * 8000.0).astype(np.float32)   # |x| <= 32000
    B = (synth.small_int((k, n), 6) * 0.5).astype(np.float32)
    Ad = torch.from_numpy(A).half().cuda()
    Bd = torch.from_numpy(B).half().cuda()
    C = fmm.gemm(Ad, Bd, levels=0, variant="f16")
    fmm.device_status()
    np.testing.assert_array_equal(C.cpu().numpy(), oracle.classical(A, B))


# ------------------------------------------------ classical products store C (beta = 0)
@pytest.mark.parametrize("variant", ["split3", "bf16", "f16"])
@pytest.mark.parametrize("pads", [(0, 0, 0), (0, 0, 1)])
@pytest.mark.parametrize("m,n,k", [(300, 520, 200), (129, 257, 65), (1000, 1200, 300)])
def test_classical_beta0_stores_c_without_reading_it(variant, pads, m, n, k):
    """L = 0, beta = 0: each output tile has one item, whose write-back stores C (TMA store,
    or plain stores when C rows are unaligned); NaN in C beforehand must not survive."""
    C, C64, _, _ = run(m, n, k, 0, variant, dist="int", seed=67 * m + k, pads=pads, c_fill=float("nan"))
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("opts", [{"deterministic": True}, {"cta_pair": False}, {"outer_scaling": True},
                                  {"tile_n": 128}, {"fringe": "peel"}])
def test_classical_beta0_store_under_options(opts):
    C, C64, _, _ = run(700, 650, 300, 0, "split3", dist="int", seed=71, c_fill=float("nan"), **opts)
    np.testing.assert_array_equal(C, C64)


def test_classical_beta_nonzero_still_adds():
    C, C64, An, Bn = run(640, 520, 256, 0, "split3", seed=73, alpha=0.5, beta=-1.25)
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance("split3", 0, 256)


# ------------- the <3,2,3> basis of rank 15 and the <2,3,2> basis of rank 11 (Section 6)
@pytest.mark.parametrize("basis", ["b323", "b232"])
@pytest.mark.parametrize("opts", [{}, {"pads": (0, 0, 1)}, {"cta_pair": False}, {"fringe": "peel"},
                                  {"deterministic": True}, {"round_tiles": 1}, {"tile_n": 128},
                                  {"tile_n": 256}, {"outer_scaling": True}, {"schedule": "product"}])
@pytest.mark.parametrize("m,n,k", [(300, 520, 200), (129, 257, 65), (1000, 1200, 300), (1, 300, 1),
                                   (7, 5, 3), (1800, 776, 130)])
def test_table_basis_bit_exact(m, n, k, opts, basis):
    """<3,2,3>: fifteen products over 3 x 2 blocks of A and 2 x 3 of B, each added into its (at
    most three) 3 x 3 blocks of C; <2,3,2>: eleven products over 2 x 3 blocks of A and 3 x 2 of
    B into 2 x 2 blocks of C: exact on small integers through every packed option."""
    o = dict(opts)
    pads = o.pop("pads", (0, 0, 0))
    C, C64, _, _ = run(m, n, k, 1, "split3", dist="int", seed=47 * m + k, basis=basis, pads=pads, **o)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("basis", ["b323", "b232"])
@pytest.mark.parametrize("variant", ["split3", "plain_bf16", "bf16", "f16"])
@pytest.mark.parametrize("m,n,k", [(600, 520, 400), (771, 1030, 515)])
def test_table_basis_float(variant, m, n, k, basis):
    C, C64, An, Bn = run(m, n, k, 1, variant, seed=49, basis=basis)
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance(variant, 1, k)


@pytest.mark.parametrize("basis", ["b323", "b232"])
@pytest.mark.parametrize("variant", ["split3", "f16"])
def test_table_basis_alpha_beta(variant, basis):
    C, C64, An, Bn = run(700, 900, 350, 1, variant, seed=51, alpha=-1.5, beta=0.75, basis=basis)
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance(variant, 1, 350)


@pytest.mark.parametrize("basis", ["b323", "b232"])
def test_table_basis_matches_the_oracle_table_product(basis):
    """The library's products against the oracle's restatement of the same table
    (FP64), on values whose sums and products are exact in every precision involved."""
    m, n, k = 240, 330, 160
    A, B = synth.problem(m, n, k, 53, "int")
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = fmm.gemm(Ad, Bd, levels=1, basis=basis)
    fmm.device_status()
    np.testing.assert_array_equal(C.cpu().numpy(), oracle.table_matmul(A, B, basis=basis))


@pytest.mark.parametrize("basis", ["b323", "b232"])
def test_table_basis_sampled_rows_4096(basis):
    rows = np.array([0, 1, 1365, 1366, 1367, 2730, 2731, 4095])  # first rows of each third
    C, C64, An, Bn = run(4096, 4096, 4096, 1, "split3", seed=55, rows=rows, basis=basis)
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance("split3", 1, 4096)


@pytest.mark.parametrize("basis", ["b323", "b232"])
def test_table_basis_deterministic_bitwise_reproducible(basis):
    m, n, k = 1900, 1700, 1100
    outs = [run(m, n, k, 1, "split3", seed=75, deterministic=True, basis=basis)[0] for _ in range(3)]
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("basis", ["b323", "b232"])
def test_table_basis_outer_scaling_keeps_badly_scaled_rows_accurate(basis):
    """The <3,2,3> sums combine up to four blocks (the <2,3,2> ones up to two): without outside scaling badly scaled rows
    and columns lose accuracy as with Strassen; with it every element keeps FP32-level accuracy
    against its own scale."""
    m = n = k = 600
    A, B = synth.problem(m, n, k, 77, "badly_scaled")
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C64 = oracle.classical(A, B)
    scaled = fmm.gemm(Ad, Bd, levels=1, basis=basis, outer_scaling=True).cpu().numpy().astype(np.float64)
    fmm.device_status()
    assert _componentwise(scaled, C64, A, B) <= 1e-5


@pytest.mark.parametrize("basis", ["b323", "b232"])
def test_table_basis_f16_large_magnitudes_panel_scaled(basis):
    """FP16 operands near the top of the range: four-term sums would overflow FP16 unscaled;
    the per-panel power-of-two scaling keeps them exact on these integers."""
    m, n, k = 384, 390, 256
    A = (synth.small_int((m, k), 7) * 8000.0).astype(np.float32)
    B = (synth.small_int((k, n), 8) * 0.5).astype(np.float32)
    C = fmm.gemm(torch.from_numpy(A).half().cuda(), torch.from_numpy(B).half().cuda(), levels=1,
                 variant="f16", basis=basis)
    fmm.device_status()
    np.testing.assert_array_equal(C.cpu().numpy(), oracle.classical(A, B))


def test_table_bases_rejected_where_not_built():
    A = torch.zeros((64, 64), device="cuda")
    for basis in ("b323", "b232"):
        with pytest.raises(fmm.FmmError):
            fmm.gemm(A, A, levels=2, basis=basis)
        with pytest.raises(fmm.FmmError):
            fmm.gemm(A, A, levels=2, basis=basis, algo="hybrid")


@pytest.mark.parametrize("basis", ["b323", "b232"])
@pytest.mark.parametrize("opts", [{}, {"cta_pair": False}, {"deterministic": True}, {"pads": (0, 0, 1)}])
@pytest.mark.parametrize("m,n,k", [(300, 520, 200), (129, 257, 65), (1000, 1200, 300), (7, 5, 3)])
def test_table_basis_fused_bit_exact(m, n, k, opts, basis):
    """The table bases with their operand sums formed on chip (fused kernel): <3,2,3> with up to
    four FP32 source tiles per operand, fifteen products and destinations in the 3 x 3 C grid;
    <2,3,2> with eleven products into the 2 x 2 C grid."""
    o = dict(opts)
    pads = o.pop("pads", (0, 0, 0))
    pads = (_pad4(k), _pad4(n), pads[2])
    C, C64, _, _ = run(m, n, k, 1, "split3", dist="int", seed=81 * m + k, basis=basis, algo="fused",
                       pads=pads, **o)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("basis", ["b323", "b232"])
@pytest.mark.parametrize("variant", ["split3", "plain_bf16"])
def test_table_basis_fused_float(variant, basis):
    C, C64, An, Bn = run(600, 520, 400, 1, variant, seed=83, basis=basis, algo="fused",
                         pads=(_pad4(400), _pad4(520), 0))
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance(variant, 1, 400)


@pytest.mark.parametrize("m,n,k", [(3000, 3000, 3000), (1200, 900, 150), (2304, 2304, 2304)])
def test_levels_auto_uses_the_models_choice(m, n, k):
    A, B = synth.problem(m, n, k, 57 + m, "int")
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = fmm.gemm(Ad, Bd, levels="auto")
    fmm.device_status()
    np.testing.assert_array_equal(C.cpu().numpy(), oracle.classical(A, B))


def test_winograd_basis_rejected_at_two_levels():
    A = torch.zeros((64, 64), device="cuda")
    with pytest.raises(fmm.FmmError):
        fmm.gemm(A, A, levels=2, basis="winograd")


@pytest.mark.parametrize("opts", [{}, {"cta_pair": False}, {"algo": "fused"}, {"pipeline": True},
                                  {"pads": (0, 0, 1)}, {"levels": 1}, {"levels": 0}])
@pytest.mark.parametrize("m,n,k", [(300, 520, 200), (1000, 1200, 300), (129, 257, 65)])
def test_deterministic_ownership_bit_exact(m, n, k, opts):
    """Ownership mode (padded last round, per-item completion) through every path."""
    o = dict(opts)
    levels = o.pop("levels", 2)
    pads = o.pop("pads", (0, 0, 0))
    if o.get("algo") == "fused":
        pads = (_pad4(k), _pad4(n), 0)
    C, C64, _, _ = run(m, n, k, levels, "split3", dist="int", seed=51 * m + k, deterministic=True,
                       pads=pads, **o)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("opts", [{}, {"algo": "fused"}, {"pads": (0, 0, 1)}])
def test_deterministic_results_are_bitwise_reproducible(opts):
    """The same float product three times in ownership mode: identical bits each time."""
    o = dict(opts)
    pads = o.pop("pads", (0, 0, 0))
    m, n, k = 2000, 1800, 1536
    outs = [run(m, n, k, 2, "split3", seed=53, deterministic=True, pads=pads, **o)[0] for _ in range(3)]
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_short_one_level_products_run_in_ownership_order_by_default():
    """beta = 0, one level, h_k <= 512 (here k = 1000, h_k = 504) with the default options: the
    library runs each tile position's products in order on one worker, so the float result is
    bitwise the ownership mode's (and reproducible), bit-exact on integers, and within the
    bound; k = 2000 (h_k = 1000) keeps the launch phases, which still meet the bound."""
    m, n = 1800, 2000
    outs = [run(m, n, 1000, 1, "split3", seed=71)[0] for _ in range(3)]
    owned = run(m, n, 1000, 1, "split3", seed=71, deterministic=True)[0]
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    assert np.array_equal(outs[0], owned)
    C, C64, An, Bn = run(m, n, 1000, 1, "split3", seed=71)
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance("split3", 1, 1000)
    C, C64, _, _ = run(m, n, 1000, 1, "split3", dist="int", seed=72, c_fill=float("nan"))
    np.testing.assert_array_equal(C, C64)
    C, C64, An, Bn = run(m, n, 2000, 1, "split3", seed=73)
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance("split3", 1, 2000)


@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("m,n,k,pads", [(300, 520, 200, (0, 0, 0)), (129, 257, 65, (0, 0, 1)),
                                        (1000, 1200, 300, (0, 0, 0))])
def test_outer_scaling_bit_exact(m, n, k, pads, levels):
    """Power-of-two row and column scaling around the product is exact on integers."""
    C, C64, _, _ = run(m, n, k, levels, "split3", dist="int", seed=61 * m + k, pads=pads, outer_scaling=True)
    np.testing.assert_array_equal(C, C64)


def test_outer_scaling_with_beta_and_fp16():
    m, n, k = 257, 301, 131
    A, B = synth.problem(m, n, k, 63, "int")
    C0 = synth.small_int((m, n), 64)
    Cd = torch.from_numpy(C0).cuda()
    fmm.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), Cd, alpha=2.0, beta=-3.0, levels=2,
             outer_scaling=True)
    fmm.device_status()
    np.testing.assert_array_equal(Cd.cpu().numpy(), oracle.classical(A, B, C0, 2.0, -3.0))
    C, C64, _, _ = run(300, 200, 150, 1, "f16", dist="int", seed=65, outer_scaling=True)
    np.testing.assert_array_equal(C, C64)


def _componentwise(C, C64, A, B):
    """max_ij |C - C64| / (||A_i|| ||B_:j||): the error of each element against its own scale."""
    ra = np.linalg.norm(A.astype(np.float64), axis=1)[:, None]
    cb = np.linalg.norm(B.astype(np.float64), axis=0)[None, :]
    return float(np.max(np.abs(C - C64) / (ra * cb)))


def test_outer_scaling_keeps_badly_scaled_rows_accurate():
    """Rows of A and columns of B spread over 10^-3 .. 10^3: without outside scaling the
    two-level sums swamp small rows and columns; with it every element keeps FP32-level
    accuracy against its own scale."""
    m = n = k = 512
    A, B = synth.problem(m, n, k, 67, "badly_scaled")
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C64 = oracle.classical(A, B)
    plain = fmm.gemm(Ad, Bd, levels=2).cpu().numpy().astype(np.float64)
    scaled = fmm.gemm(Ad, Bd, levels=2, outer_scaling=True).cpu().numpy().astype(np.float64)
    fmm.device_status()
    e_plain, e_scaled = _componentwise(plain, C64, A, B), _componentwise(scaled, C64, A, B)
    assert e_scaled <= 1e-5, e_scaled
    assert e_scaled * 10 < e_plain, (e_scaled, e_plain)


def test_cta_pair_rejected_with_bk32():
    A = torch.zeros((64, 64), device="cuda")
    with pytest.raises(fmm.FmmError):
        fmm.gemm(A, A, levels=1, bk=32, cta_pair=True)


@pytest.mark.parametrize("levels", [0, 1, 2])
def test_unaligned_ldc_uses_elementwise_writeback(levels):
    """ldc odd: rows of C are not 16-byte aligned, so the element-wise reduction path runs."""
    C, C64, _, _ = run(257, 300, 130, levels, "split3", dist="int", seed=9, pads=(0, 0, 1))
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("tile_n", [128, 256])
@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("m,n,k", [(300, 520, 200), (129, 257, 65), (1000, 1200, 300)])
def test_bk32_stages_bit_exact(m, n, k, levels, tile_n):
    """32-deep pipeline stages (64-byte swizzled K-major tiles)."""
    C, C64, _, _ = run(m, n, k, levels, "split3", dist="int", seed=3 * m + k, tile_n=tile_n, bk=32)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("levels", [0, 2])
def test_bk32_float_and_unaligned(levels):
    C, C64, An, Bn = run(640, 384, 768, levels, "split3", dist="gaussian", seed=4, bk=32,
                         pads=(3, 1, 1), alpha=-1.0, beta=0.5)
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance("split3", levels, 768)


def test_int_with_alpha_beta_bit_exact():
    A, B = synth.problem(200, 136, 96, 3, "int")
    C0 = synth.small_int((200, 136), 4)
    Ad = torch.from_numpy(A).cuda()
    Bd = torch.from_numpy(B).cuda()
    Cd = torch.from_numpy(C0).cuda()
    fmm.gemm(Ad, Bd, Cd, alpha=2.0, beta=-3.0, levels=2)
    fmm.device_status()
    np.testing.assert_array_equal(Cd.cpu().numpy(), oracle.classical(A, B, C0, 2.0, -3.0))


# ------------------------------------------------- fused (on-chip operand sums)
def _pad4(c):
    return (-c) % 4


@pytest.mark.parametrize("schedule", ["product", "rounds"])
@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("m,n,k", [(16, 16, 16), (300, 520, 200), (129, 257, 65), (1, 300, 1),
                                   (520, 8, 400), (1000, 1200, 300)])
def test_fused_int_bit_exact(m, n, k, levels, schedule):
    C, C64, _, _ = run(m, n, k, levels, "split3", dist="int", seed=m + 2 * n + k, algo="fused",
                       pads=(_pad4(k), _pad4(n), 0), schedule=schedule)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("cta_pair", [False, True])
@pytest.mark.parametrize("algo", ["fused", "hybrid"])
@pytest.mark.parametrize("m,n,k", [(300, 520, 200), (129, 257, 65), (1000, 1200, 300), (520, 8, 400)])
def test_fused_single_cta_and_pair_bit_exact(m, n, k, algo, cta_pair):
    """On-chip sums with one CTA per 128 x 128 tile and with CTA pairs on 256 x 256 tiles."""
    for levels in ((1, 2) if algo == "fused" else (2,)):
        C, C64, _, _ = run(m, n, k, levels, "split3", dist="int", seed=7 * m + n + k, algo=algo,
                           pads=(_pad4(k), _pad4(n), 0), cta_pair=cta_pair)
        np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("cta_pair", [False, True])
def test_fused_float_single_cta_and_pair(cta_pair):
    C, C64, An, Bn = run(640, 384, 768, 1, "split3", dist="gaussian", seed=31, algo="fused",
                         cta_pair=cta_pair)
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance("split3", 1, 768)


@pytest.mark.parametrize("variant", ["split3", "plain_bf16"])
@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("m,n,k", [(7, 13, 5), (257, 129, 1000), (640, 384, 96)])
def test_fused_float_shapes(m, n, k, levels, variant):
    C, C64, An, Bn = run(m, n, k, levels, variant, dist="gaussian", seed=m * 3 + n + k,
                         algo="fused", pads=(_pad4(k), _pad4(n), 0))
    err = oracle.normwise_error(C, C64, An, Bn)
    assert err <= tolerance(variant, levels, k), err


@pytest.mark.parametrize("fused_kernel", ["smem", "tmem"])
@pytest.mark.parametrize("variant", ["split3", "plain_bf16"])
@pytest.mark.parametrize("m,n,k", [(16, 16, 16), (300, 520, 200), (129, 257, 65), (1000, 1200, 300),
                                   (520, 8, 400), (600, 700, 1030)])
def test_fused_kernels_int_bit_exact(m, n, k, variant, fused_kernel):
    """Both on-chip kernels (CTA pairs): operand sums of both operands in shared memory, or the
    A-operand sums in tensor memory; one and two levels, and the hybrid two-level scheme."""
    for levels, algo in ((1, "fused"), (2, "fused"), (2, "hybrid")):
        C, C64, _, _ = run(m, n, k, levels, variant, dist="int", seed=3 * m + n + k, algo=algo,
                           pads=(_pad4(k), _pad4(n), 0), fused_kernel=fused_kernel)
        np.testing.assert_array_equal(C, C64, err_msg=f"{algo} L={levels}")


@pytest.mark.parametrize("schedule", ["product", "rounds"])
def test_fused_tmem_kernel_float_and_schedules(schedule):
    C, C64, An, Bn = run(1100, 900, 1300, 1, "split3", dist="gaussian", seed=44, algo="fused",
                         fused_kernel="tmem", schedule=schedule)
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance("split3", 1, 1300)


def test_fused_tmem_kernel_needs_cta_pairs():
    A = torch.zeros((64, 64), device="cuda")
    with pytest.raises(fmm.FmmError) as ei:
        fmm.gemm(A, A, levels=1, algo="fused", cta_pair=False, fused_kernel="tmem")
    assert ei.value.status == 3


def test_fused_matches_packed_closely():
    """Same arithmetic, different place of the sums: results agree to FP32 rounding."""
    A, B = synth.problem(1024, 768, 896, 41, "uniform")
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    for levels in (1, 2):
        Cp = fmm.gemm(Ad, Bd, levels=levels, algo="packed")
        Cf = fmm.gemm(Ad, Bd, levels=levels, algo="fused")
        fmm.device_status()
        rel = ((Cp - Cf).norm() / Cp.norm()).item()
        assert rel < 1e-6, rel


@pytest.mark.parametrize("fused_kernel", ["smem", "tmem"])
def test_fused_full_size_sampled_rows(fused_kernel):
    rows = np.unique(synth.rng(5).integers(0, 8192, size=8))
    C, C64, An, Bn = run(8192, 8192, 8192, 2, "split3", seed=21, rows=rows, algo="fused",
                         fused_kernel=fused_kernel)
    assert oracle.normwise_error(C, C64, An, Bn) <= 1e-6


@pytest.mark.parametrize("algo", ["fused", "hybrid"])
def test_fused_full_size_int_bit_exact(algo):
    """Small integers at 16384^3, two levels, sums formed on chip (default kernel): sampled
    rows equal the FP64 oracle exactly."""
    rows = np.unique(np.concatenate([[0, 16383], synth.rng(17).integers(0, 16384, size=4)]))
    C, C64, _, _ = run(16384, 16384, 16384, 2, "split3", dist="int", seed=61, rows=rows, algo=algo)
    np.testing.assert_array_equal(C, C64)


def test_fused_rejects_unaligned_leading_dimension():
    A = torch.zeros((64, 65), device="cuda")
    B = torch.zeros((65, 64), device="cuda")
    with pytest.raises(fmm.FmmError) as ei:
        fmm.gemm(A, B, levels=1, algo="fused")
    assert ei.value.status == 2


# ------------------------------------------------------------- hybrid two-level
@pytest.mark.parametrize("m,n,k", [(16, 16, 16), (300, 520, 200), (129, 257, 65), (1000, 1200, 300)])
def test_hybrid_int_bit_exact(m, n, k):
    C, C64, _, _ = run(m, n, k, 2, "split3", dist="int", seed=5 * m + n + k, algo="hybrid")
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("variant", ["split3", "plain_bf16"])
def test_hybrid_float(variant):
    C, C64, An, Bn = run(640, 384, 768, 2, variant, dist="gaussian", seed=9, algo="hybrid")
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance(variant, 2, 768)


def test_hybrid_full_size_sampled_rows():
    rows = np.unique(synth.rng(6).integers(0, 8192, size=8))
    C, C64, An, Bn = run(8192, 8192, 8192, 2, "split3", seed=22, rows=rows, algo="hybrid")
    assert oracle.normwise_error(C, C64, An, Bn) <= 1e-6


@pytest.mark.parametrize("m,n,k", [(16, 16, 16), (300, 520, 200), (129, 257, 65), (1000, 1200, 300)])
def test_hybrid_bf16_operands_int_bit_exact(m, n, k):
    """BF16 operands on the hybrid scheme: FP32 top-level sums of the BF16 values, the 49
    bottom-level sums formed on chip and rounded once to BF16."""
    C, C64, _, _ = run(m, n, k, 2, "bf16", dist="int", seed=11 * m + n + k, algo="hybrid")
    np.testing.assert_array_equal(C, C64)


def test_hybrid_bf16_operands_float():
    C, C64, An, Bn = run(640, 384, 768, 2, "bf16", dist="gaussian", seed=12, algo="hybrid")
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance("bf16", 2, 768)


@pytest.mark.parametrize("m,n,k", [(16, 16, 16), (300, 520, 200), (129, 257, 65), (1000, 1200, 300)])
def test_hybrid_f16_scaled_int_bit_exact(m, n, k):
    """FP16 operands on the hybrid scheme: FP32 top-level sums, then per (product, panel) the
    power of two that puts the panel's largest bottom-level sum in [2^14, 2^15) (a maxima pass
    before the kernel), applied on chip before the FP16 rounding and undone in the epilogue."""
    C, C64, _, _ = run(m, n, k, 2, "f16", dist="int", seed=13 * m + n + k, algo="hybrid")
    np.testing.assert_array_equal(C, C64)


def test_hybrid_f16_scaled_float_and_badly_scaled():
    C, C64, An, Bn = run(640, 384, 768, 2, "f16", dist="gaussian", seed=14, algo="hybrid")
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance("f16", 2, 768)
    C, C64, An, Bn = run(512, 512, 512, 2, "f16", dist="badly_scaled", seed=15, algo="hybrid")
    assert np.all(np.isfinite(C))
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance("f16", 2, 512)


def test_hybrid_f16_large_values_do_not_overflow():
    """Sums of FP16 inputs near 2^15 exceed FP16's range unscaled (65504)."""
    A = (synth.uniform((256, 256), 82) * 30000.0).astype(np.float32)
    B = (synth.uniform((256, 256), 83) * 30000.0).astype(np.float32)
    Ad = torch.from_numpy(A).half().cuda()
    Bd = torch.from_numpy(B).half().cuda()
    C = fmm.gemm(Ad, Bd, levels=2, variant="f16", algo="hybrid")
    fmm.device_status()
    Ab = Ad.cpu().view(torch.int16).numpy().view(np.uint16)
    Bb = Bd.cpu().view(torch.int16).numpy().view(np.uint16)
    C64 = oracle.classical(Ab, Bb, a_code=oracle.ORC_F16, b_code=oracle.ORC_F16)
    Cn = C.cpu().numpy()
    assert np.all(np.isfinite(Cn))
    err = oracle.normwise_error(Cn, C64, float(Ad.float().norm()), float(Bd.float().norm()))
    assert err <= tolerance("f16", 2, 256), err


@pytest.mark.parametrize("pads", [(1, 3, 1), (0, 0, 1), (5, 0, 0)])
def test_hybrid_unaligned_leading_dimensions_bit_exact(pads):
    """Odd leading dimensions: the top-level sum pass reads any row stride and writes aligned
    FP32 sums, so the on-chip bottom level runs unchanged; unaligned C takes the element-wise
    write-back."""
    C, C64, _, _ = run(300, 520, 203, 2, "split3", dist="int", seed=13, algo="hybrid", pads=pads)
    np.testing.assert_array_equal(C, C64)


def test_hybrid_odd_30001_29999_4097_sampled_rows():
    rows = np.unique(np.concatenate([[0, 30000], synth.rng(19).integers(0, 30001, size=6)]))
    C, C64, An, Bn = run(30001, 29999, 4097, 2, "split3", dist="gaussian", seed=24, rows=rows, algo="hybrid")
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance("split3", 2, 4097)


# ------------------------------------------------------ degenerate problems
@pytest.mark.parametrize("levels,algo", [(0, "auto"), (1, "auto"), (2, "auto"), (1, "fused"), (2, "hybrid")])
def test_degenerate_shapes(levels, algo):
    """k = 0 scales C by beta; alpha = 0 likewise (no product is formed); m = 0 or n = 0 leaves
    C untouched; 1 x 1 x 1 and 1 x 9 x 1 products (all but one block empty at every level) are
    exact."""
    C0 = synth.uniform((40, 48), 81)
    for (m, n, k, alpha, beta) in [(40, 48, 0, 1.0, 0.5), (40, 48, 32, 0.0, 2.0)]:
        A = torch.from_numpy(synth.uniform((m, max(k, 1)), 82)[:, :k].copy()).cuda()
        B = torch.from_numpy(synth.uniform((max(k, 1), n), 83)[:k].copy()).cuda()
        Cd = torch.from_numpy(C0.copy()).cuda()
        fmm.gemm(A, B, Cd, alpha=alpha, beta=beta, levels=levels, algo=algo)
        fmm.device_status()
        np.testing.assert_array_equal(Cd.cpu().numpy(), (np.float32(beta) * C0).astype(np.float32))
    for (m, n) in [(0, 48), (40, 0)]:
        Cd = torch.full((max(m, 1), max(n, 1)), 7.0, device="cuda")[:m, :n]
        fmm.gemm(torch.zeros((m, 32), device="cuda"), torch.zeros((32, n), device="cuda"), Cd, levels=levels,
                 algo=algo)
        fmm.device_status()
    for (m, n, k) in [(1, 1, 1), (1, 9, 1), (8, 8, 8)]:
        # the fused kernels need rows of a multiple of 16 bytes: pad the leading dimensions
        pads = ((-k) % 4, (-n) % 4, 0) if algo == "fused" else (0, 0, 0)
        C, C64, _, _ = run(m, n, k, levels, "split3", dist="int", seed=84 + m + n, algo=algo, pads=pads)
        np.testing.assert_array_equal(C, C64)


# ------------------------------------------------------ fused, 16-bit operands
@pytest.mark.parametrize("variant", ["bf16", "f16"])
@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("m,n,k", [(8, 24, 16), (16, 16, 16), (304, 520, 200), (136, 264, 72), (1000, 1200, 304)])
def test_fused_16bit_operands_int_bit_exact(variant, levels, m, n, k):
    """BF16 and FP16 operands with every operand sum formed on chip from the caller's 16-bit
    tiles (tensor-memory kernel, no stored sums; FP16 scaled per panel by the power of two the
    maxima pass found): small integers equal the FP64 oracle exactly, ragged tiles included, and
    shapes so small that some blocks lie wholly outside the matrices (their products are dropped
    and the remaining ones keep their rows of panel maxima)."""
    C, C64, _, _ = run(m, n, k, levels, variant, dist="int", seed=7 * m + n + 3 * k + levels, algo="fused")
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("variant", ["bf16", "f16"])
@pytest.mark.parametrize("levels", [1, 2])
def test_fused_16bit_operands_float(variant, levels):
    C, C64, An, Bn = run(640, 384, 768, levels, variant, dist="gaussian", seed=40 + levels, algo="fused")
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance(variant, levels, 768)


def test_fused_f16_badly_scaled_and_large_values():
    """Badly scaled FP16 inputs stay finite and within the FP16 bound; inputs near 2^15, whose
    sums exceed FP16's range unscaled, do not overflow."""
    C, C64, An, Bn = run(512, 512, 512, 1, "f16", dist="badly_scaled", seed=43, algo="fused")
    assert np.all(np.isfinite(C))
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance("f16", 1, 512)
    A = (synth.uniform((256, 256), 84) * 30000.0).astype(np.float32)
    B = (synth.uniform((256, 256), 85) * 30000.0).astype(np.float32)
    Ad = torch.from_numpy(A).half().cuda()
    Bd = torch.from_numpy(B).half().cuda()
    C = fmm.gemm(Ad, Bd, levels=1, variant="f16", algo="fused")
    fmm.device_status()
    Ab = Ad.cpu().view(torch.int16).numpy().view(np.uint16)
    Bb = Bd.cpu().view(torch.int16).numpy().view(np.uint16)
    C64 = oracle.classical(Ab, Bb, a_code=oracle.ORC_F16, b_code=oracle.ORC_F16)
    Cn = C.cpu().numpy()
    assert np.all(np.isfinite(Cn))
    err = oracle.normwise_error(Cn, C64, float(Ad.float().norm()), float(Bd.float().norm()))
    assert err <= tolerance("f16", 1, 256), err


def test_fused_bf16_operands_other_bases_bit_exact():
    for basis in ("winograd", "b323"):
        C, C64, _, _ = run(312, 264, 200, 1, "bf16", dist="int", seed=44, algo="fused", basis=basis)
        np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("variant,levels", [("bf16", 1), ("f16", 2)])
def test_fused_16bit_full_size_sampled_rows(variant, levels):
    rows = np.unique(np.concatenate([[0, 8191], synth.rng(23).integers(0, 8192, size=4)]))
    C, C64, An, Bn = run(8192, 8192, 8192, levels, variant, seed=45, rows=rows, algo="fused")
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance(variant, levels, 8192)


def test_fused_16bit_operands_refusals():
    """16-bit operands on chip: forward products in the tensor-memory kernel (CTA pairs) with
    rows of a multiple of 16 bytes; FP16 scaling with Strassen's basis only."""
    A = torch.zeros((64, 64), device="cuda", dtype=torch.bfloat16)
    B = torch.zeros((64, 64), device="cuda", dtype=torch.bfloat16)
    for kw in ({"cta_pair": False}, {"fused_kernel": "smem"}):
        with pytest.raises(fmm.FmmError) as ei:
            fmm.gemm(A, B, levels=1, variant="bf16", algo="fused", **kw)
        assert ei.value.status == 3
    with pytest.raises(fmm.FmmError) as ei:
        fmm.gemm(A.half(), B.half(), levels=1, variant="f16", algo="fused", basis="b323")
    assert ei.value.status == 3
    with pytest.raises(fmm.FmmError) as ei:
        fmm.gemm_backward(A, B, torch.zeros((64, 64), device="cuda"), levels=1, variant="bf16", algo="fused")
    assert ei.value.status == 3
    Au = torch.zeros((64, 68), device="cuda", dtype=torch.bfloat16)
    Bu = torch.zeros((68, 64), device="cuda", dtype=torch.bfloat16)
    with pytest.raises(fmm.FmmError) as ei:
        fmm.gemm(Au, Bu, levels=1, variant="bf16", algo="fused")
    assert ei.value.status == 2


# ------------------------------------------- large odd sizes with dynamic fringes
@pytest.mark.parametrize("variant,levels", [("split3", 2), ("plain_bf16", 2), ("split3", 0)])
def test_odd_30001_29999_4097_sampled_rows(variant, levels):
    """m = 30001, n = 29999, k = 4097 with tight (odd) leading dimensions: unaligned rows,
    element-wise write-back, zero-padded fringe blocks."""
    rows = np.unique(np.concatenate([[0, 30000], synth.rng(7).integers(0, 30001, size=6)]))
    C, C64, An, Bn = run(30001, 29999, 4097, levels, variant, dist="gaussian", seed=23, rows=rows)
    err = oracle.normwise_error(C, C64, An, Bn)
    assert err <= tolerance(variant, levels, 4097), err


# ------------------------------------------------------------------- floats
def test_512_cube_one_level_split3_within_1e6():
    C, C64, An, Bn = run(512, 512, 512, 1, "split3", seed=11)
    err = oracle.normwise_error(C, C64, An, Bn)
    assert err <= 1e-6, err


@pytest.mark.parametrize("variant", ["split3", "plain_bf16", "bf16", "f16"])
@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (7, 13, 5), (130, 70, 300), (257, 129, 1000),
                                   (640, 384, 96)])
def test_float_shapes(m, n, k, levels, variant):
    C, C64, An, Bn = run(m, n, k, levels, variant, dist="gaussian", seed=m * 7 + n + k)
    err = oracle.normwise_error(C, C64, An, Bn)
    assert err <= tolerance(variant, levels, k), err


@pytest.mark.parametrize("levels", [0, 1, 2])
def test_alpha_beta_and_padded_leading_dims(levels):
    C, C64, An, Bn = run(300, 260, 150, levels, "split3", seed=5, alpha=-1.5, beta=0.75,
                         pads=(5, 3, 9))
    err = oracle.normwise_error(C, C64, An, Bn)
    assert err <= tolerance("split3", levels, 150), err


@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("pad_c", [0, 1])
def test_negative_alpha_bit_exact(levels, pad_c):
    """alpha < 0 on both write-back paths (TMA reductions for aligned C, element-wise for
    unaligned C)."""
    A, B = synth.problem(136, 264, 72, 91, "int")
    C0 = synth.small_int((136, 264), 92)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    Cd = _to_device(C0, pad_c, torch.float32)
    fmm.gemm(Ad, Bd, Cd, alpha=-2.0, beta=3.0, levels=levels)
    fmm.device_status()
    np.testing.assert_array_equal(Cd.cpu().numpy(), oracle.classical(A, B, C0, -2.0, 3.0))


def test_beta_zero_does_not_read_c():
    C, C64, An, Bn = run(130, 140, 150, 1, "split3", seed=6, c_fill=float("nan"))
    assert np.all(np.isfinite(C))
    assert oracle.normwise_error(C, C64, An, Bn) <= 1e-6


def test_k_zero_scales_c():
    Cd = torch.ones((33, 17), device="cuda")
    A = torch.zeros((33, 0), device="cuda")
    B = torch.zeros((0, 17), device="cuda")
    fmm.gemm(A, B, Cd, alpha=1.0, beta=2.5, levels=1)
    fmm.device_status()
    assert torch.all(Cd == 2.5)


@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("tile_n", [128, 256])
def test_f16_scaled_int_ragged_bit_exact(levels, tile_n):
    """Power-of-two scaling is exact: integer products stay bit-exact through FP16."""
    C, C64, _, _ = run(300, 520, 200, levels, "f16", dist="int", seed=77, tile_n=tile_n)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("levels", [1, 2])
def test_f16_scaled_badly_scaled_inputs(levels):
    """Rows of A / columns of B spread over 10^-3..10^3: the per-panel shifts keep every
    operand sum in FP16's normal range."""
    C, C64, An, Bn = run(512, 512, 512, levels, "f16", dist="badly_scaled", seed=78)
    assert np.all(np.isfinite(C))
    err = oracle.normwise_error(C, C64, An, Bn)
    assert err <= tolerance("f16", levels, 512), err


def test_f16_large_values_do_not_overflow():
    """Operand sums of FP16 inputs near 2^15 exceed FP16's range unscaled (65504)."""
    A = (synth.uniform((256, 256), 80) * 30000.0).astype(np.float32)
    B = (synth.uniform((256, 256), 81) * 30000.0).astype(np.float32)
    Ad = torch.from_numpy(A).half().cuda()
    Bd = torch.from_numpy(B).half().cuda()
    C = fmm.gemm(Ad, Bd, levels=2, variant="f16")
    fmm.device_status()
    Ab = Ad.cpu().view(torch.int16).numpy().view(np.uint16)
    Bb = Bd.cpu().view(torch.int16).numpy().view(np.uint16)
    C64 = oracle.classical(Ab, Bb, a_code=oracle.ORC_F16, b_code=oracle.ORC_F16)
    Cn = C.cpu().numpy()
    assert np.all(np.isfinite(Cn))
    err = oracle.normwise_error(Cn, C64, float(Ad.float().norm()), float(Bd.float().norm()))
    assert err <= tolerance("f16", 2, 256), err


def test_badly_scaled_two_level():
    C, C64, An, Bn = run(512, 512, 512, 2, "split3", dist="badly_scaled", seed=8)
    err = oracle.normwise_error(C, C64, An, Bn)
    assert err <= 1e-6, err


# -------------------------------------------------- full size, sampled rows
@pytest.mark.parametrize("n,k,levels", [(16384, 16384, 2), (16384, 512, 2), (8192, 8192, 1), (16384, 512, 1),
                                         (16384, 1024, 1), (16384, 2048, 1)])
def test_full_size_sampled_rows(n, k, levels):
    m = n
    rows = np.unique(synth.rng(123).integers(0, m, size=12))
    C, C64, An, Bn = run(m, n, k, levels, "split3", seed=20, rows=rows, tile_n=0)
    err = oracle.normwise_error(C, C64, An, Bn)
    assert err <= 1e-6, err


@pytest.mark.parametrize("m,n,k,levels", [(16384, 16384, 16384, 2), (30001, 29999, 4097, 2),
                                          (30001, 29999, 4097, 1), (16384, 16384, 512, 1),
                                          (16384, 16384, 2048, 1)])
def test_full_size_int_sampled_rows_bit_exact(m, n, k, levels):
    """Small integers at the benchmark's sizes: every operand sum, product and partial sum is an
    integer far below 2**24, so each sampled element must equal the FP64 oracle exactly.  This
    reaches the full-size paths: 76 CTA pairs, three stages, 64-deep k-steps by the hundred,
    tile rounds; at 30001 x 29999 x 4097 the tight leading dimensions (odd lda, ldb, ldc) take
    the unaligned-operand sum pass and the element-wise write-back, and the last block row and
    column are zero-padded fringes; the rank-512 update runs in the ownership order, the
    rank-2048 one in store-first launch phases."""
    rows = np.unique(np.concatenate([[0, m - 1], synth.rng(m + k).integers(0, m, size=6)]))
    C, C64, _, _ = run(m, n, k, levels, "split3", dist="int", seed=k + levels, rows=rows)
    np.testing.assert_array_equal(C, C64)


# ------------------------------------------- store-first phases (beta = 0)
@pytest.mark.parametrize("store_first", [True, False])
@pytest.mark.parametrize("pad_c", [0, 1])
@pytest.mark.parametrize("levels,basis", [(1, "strassen"), (2, "strassen"), (1, "winograd"), (1, "b323"),
                                          (1, "b232")])
@pytest.mark.parametrize("m,n,k", [(300, 520, 200), (129, 257, 65), (1000, 1200, 300), (520, 8, 400)])
def test_store_first_phases_bit_exact(m, n, k, levels, basis, pad_c, store_first):
    """beta = 0: the products run in launch phases whose first update of each C block is a
    store; C starts as NaN, so a block that some product adds into before it was stored, or
    that no product stores, shows up.  Aligned C (TMA stores) and unaligned C (element-wise
    stores), every basis, fringe blocks."""
    C, C64, _, _ = run(m, n, k, levels, "split3", dist="int", seed=m + k + levels, basis=basis,
                       pads=(0, 0, pad_c), c_fill=float("nan"), store_first=store_first)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("levels,basis", [(1, "strassen"), (2, "strassen"), (1, "b323"), (1, "b232")])
@pytest.mark.parametrize("pad_c", [0, 1])
@pytest.mark.parametrize("m,n,k", [(300, 520, 200), (1000, 1200, 300), (600, 2100, 96)])
def test_store_first_in_ownership_mode_bit_exact(m, n, k, levels, basis, pad_c):
    """Deterministic (ownership) mode with beta = 0: one launch, every tile position's products
    in order on one worker, the first product to update a block stores it; C starts as NaN."""
    C, C64, _, _ = run(m, n, k, levels, "split3", dist="int", seed=m + n + levels, basis=basis,
                       pads=(0, 0, pad_c), c_fill=float("nan"), deterministic=True)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("levels", [1, 2])
def test_store_first_negative_alpha_and_float(levels):
    A, B = synth.problem(136, 264, 72, 93, "int")
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    Cd = torch.full((136, 264), float("nan"), device="cuda")
    fmm.gemm(Ad, Bd, Cd, alpha=-2.0, beta=0.0, levels=levels)
    fmm.device_status()
    np.testing.assert_array_equal(Cd.cpu().numpy(), oracle.classical(A, B, None, -2.0, 0.0))
    C, C64, An, Bn = run(700, 900, 1100, levels, "split3", dist="gaussian", seed=94, c_fill=float("nan"))
    assert oracle.normwise_error(C, C64, An, Bn) <= tolerance("split3", levels, 1100)


def test_store_first_backward_and_16bit():
    """The backward products (transposed operands) and the 16-bit arithmetic take the phases too."""
    A, B = synth.problem(300, 200, 136, 95, "int")
    dC = synth.small_int((300, 200), 96)
    for levels in (1, 2):
        dA, dB = fmm.gemm_backward(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                                   torch.from_numpy(dC).cuda(), levels=levels)
        fmm.device_status()
        np.testing.assert_array_equal(dA.cpu().numpy(), oracle.classical(dC, np.ascontiguousarray(B.T)))
        np.testing.assert_array_equal(dB.cpu().numpy(), oracle.classical(np.ascontiguousarray(A.T), dC))
        for variant in ("bf16", "f16"):
            C, C64, _, _ = run(300, 520, 200, levels, variant, dist="int", seed=97, c_fill=float("nan"))
            np.testing.assert_array_equal(C, C64)


# ----------------------------------------------------------- failure path
def test_bounded_wait_reports_timeout_and_context_survives():
    fmm.set_wait_timeout_ns(20_000_000)  # 20 ms
    try:
        fmm.debug_wait_timeout()
        with pytest.raises(fmm.FmmError) as ei:
            fmm.device_status()
        assert ei.value.status == 6
    finally:
        fmm.set_wait_timeout_ns(2_000_000_000)
    fmm.device_status()  # word was cleared
    C, C64, _, _ = run(64, 64, 64, 1, "split3", dist="int", seed=2)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("m,n,k", [(20000, 8, 40), (8, 20000, 40), (40, 48, 40000)])
def test_extreme_aspect_ratios_bit_exact(m, n, k, levels):
    """Tall, wide and deep problems: most tiles of a block are fringe, or the k loop is long."""
    C, C64, _, _ = run(m, n, k, levels, "split3", dist="int", seed=m + 3 * n + k)
    np.testing.assert_array_equal(C, C64)


@pytest.mark.parametrize("opts", [{"outer_scaling": True}, {"deterministic": True}, {"pipeline": True},
                                  {"fringe": "peel"}])
def test_k_zero_and_alpha_zero_with_options(opts):
    Cd = torch.ones((33, 17), device="cuda")
    fmm.gemm(torch.zeros((33, 0), device="cuda"), torch.zeros((0, 17), device="cuda"), Cd, alpha=1.0,
             beta=2.5, levels=1, **opts)
    fmm.device_status()
    assert torch.all(Cd == 2.5)
    A, B = synth.problem(33, 17, 9, 5, "int")
    fmm.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), Cd, alpha=0.0, beta=2.0, levels=1, **opts)
    fmm.device_status()
    assert torch.all(Cd == 5.0)

"""GB300-native fused Strassen GEMM: thin Python binding of ``libfmm_gb300.so``.

The binding only marshals arguments (device pointers, sizes, the current CUDA
stream) to the C ABI declared in ``include/fmm.h``; every step of the product
runs in the library's own sm_103a kernels.  PyTorch supplies device memory and
streams.  There is no fallback: if the library is missing or the call fails, an
exception is raised.

Operation (Section 1, Eq. 1): ``C = alpha * A @ B + beta * C`` with ``levels``
levels of Strassen's algorithm (Section 3, Eq. 3; Section 3.4 for two levels).
"""
from __future__ import annotations

import ctypes
import os

from . import _build

__all__ = ["build", "load", "gemm", "workspace_size", "device_status", "product_table",
           "VARIANTS", "ALGOS", "FmmError"]

VARIANTS = {"split3": 0, "bf16": 1, "f16": 2, "plain_bf16": 3}
ALGOS = {"auto": 0, "packed": 1, "fused": 2, "hybrid": 3}
STATUS = {0: "FMM_OK", 1: "FMM_ERR_ARG", 2: "FMM_ERR_ALIGN", 3: "FMM_ERR_UNSUPPORTED",
          4: "FMM_ERR_WORKSPACE", 5: "FMM_ERR_CUDA", 6: "FMM_ERR_TIMEOUT"}


class FmmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class TuneTable(ctypes.Structure):
    """fmm_tune_table: class i holds problems with min(m, n, k) <= max_dim[i]."""
    _fields_ = [("count", ctypes.c_int), ("max_dim", ctypes.c_int64 * 8),
                ("levels", ctypes.c_int * 8), ("tile_n", ctypes.c_int * 8)]


class _Options(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int), ("tile_n", ctypes.c_int), ("num_ctas", ctypes.c_int),
                ("schedule", ctypes.c_int), ("bk", ctypes.c_int), ("cta_pair", ctypes.c_int),
                ("round_tiles", ctypes.c_int), ("fringe", ctypes.c_int), ("pipeline", ctypes.c_int),
                ("basis", ctypes.c_int), ("deterministic", ctypes.c_int), ("outer_scaling", ctypes.c_int),
                ("fused_kernel", ctypes.c_int), ("store_first", ctypes.c_int), ("reserved", ctypes.c_int * 2)]


_lib = None


def build(force: bool = False) -> str:
    """Compile the CUDA library in-tree (nvcc, sm_103a)."""
    return _build.build(force=force)


def lib_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load libfmm_gb300.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise FmmError(5, f"{_build.LIB} is missing: run paper_1808_07984_gb300.build()")
    L = ctypes.CDLL(_build.LIB)
    i64, i32, f32, vp, sz = ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t
    L.fmm_workspace_size.restype = sz
    L.fmm_workspace_size.argtypes = [i64, i64, i64, i32, i32]
    L.fmm_workspace_size_ex.restype = sz
    L.fmm_workspace_size_ex.argtypes = [i64, i64, i64, i32, i32, ctypes.POINTER(_Options)]
    gemm_args = [i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64, i32, i32, vp, sz, vp]
    L.fmm_gemm.restype = i32
    L.fmm_gemm.argtypes = gemm_args
    L.fmm_gemm_ex.restype = i32
    L.fmm_gemm_ex.argtypes = gemm_args + [ctypes.POINTER(_Options)]
    L.fmm_gemm_backward.restype = i32
    L.fmm_gemm_backward.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp, i64,
                                    i32, i32, vp, sz, vp]
    L.fmm_gemm_backward_ex.restype = i32
    L.fmm_gemm_backward_ex.argtypes = L.fmm_gemm_backward.argtypes + [ctypes.POINTER(_Options)]
    L.fmm_workspace_size_backward.restype = sz
    L.fmm_workspace_size_backward.argtypes = [i64, i64, i64, i32, i32]
    L.fmm_workspace_size_backward_ex.restype = sz
    L.fmm_workspace_size_backward_ex.argtypes = [i64, i64, i64, i32, i32, ctypes.POINTER(_Options)]
    L.fmm_tune_default.restype = None
    L.fmm_tune_default.argtypes = [ctypes.POINTER(TuneTable)]
    L.fmm_tune_default_ex.restype = None
    L.fmm_tune_default_ex.argtypes = [i32, ctypes.POINTER(TuneTable)]
    L.fmm_tune_measure.restype = i32
    L.fmm_tune_measure.argtypes = [i32, vp, i32, i32, ctypes.POINTER(TuneTable), vp, vp]
    L.fmm_tune_select.restype = i32
    L.fmm_tune_select.argtypes = [ctypes.POINTER(TuneTable), i64, i64, i64,
                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    arr64 = ctypes.POINTER(ctypes.c_int64)
    arrf = ctypes.POINTER(ctypes.c_float)
    arrp = ctypes.POINTER(ctypes.c_void_p)
    L.fmm_batched_workspace_size.restype = sz
    L.fmm_batched_workspace_size.argtypes = [i32, arr64, arr64, arr64, i32, ctypes.POINTER(TuneTable)]
    L.fmm_batched_plan_create.restype = i32
    L.fmm_batched_plan_create.argtypes = [i32, arr64, arr64, arr64, arrf, arrp, arr64, arrp, arr64,
                                          arrf, arrp, arr64, i32, ctypes.POINTER(TuneTable), vp, sz,
                                          ctypes.POINTER(ctypes.c_void_p)]
    L.fmm_batched_plan_execute.restype = i32
    L.fmm_batched_plan_execute.argtypes = [vp, vp]
    L.fmm_batched_plan_destroy.restype = None
    L.fmm_batched_plan_destroy.argtypes = [vp]
    L.fmm_last_error.restype = ctypes.c_char_p
    L.fmm_last_error.argtypes = []
    L.fmm_device_status.restype = i32
    L.fmm_device_status.argtypes = [vp]
    L.fmm_set_wait_timeout_ns.restype = None
    L.fmm_set_wait_timeout_ns.argtypes = [ctypes.c_uint64]
    L.fmm_debug_wait_timeout.restype = i32
    L.fmm_debug_wait_timeout.argtypes = [vp]
    L.fmm_product_table.restype = i32
    L.fmm_product_table.argtypes = [i32, vp, vp, vp]
    L.fmm_product_table_ex.restype = i32
    L.fmm_product_table_ex.argtypes = [i32, i32, vp, vp, vp]
    L.fmm_basis_shape.restype = i32
    L.fmm_basis_shape.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_int)]
    L.fmm_profile_enable.restype = i32
    L.fmm_profile_enable.argtypes = [i32]
    L.fmm_profile_read.restype = i32
    L.fmm_profile_read.argtypes = [vp, vp]
    L.fmm_version.restype = ctypes.c_char_p
    L.fmm_version.argtypes = []
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise FmmError(status, load().fmm_last_error().decode())


SCHEDULES = {"auto": 0, "product": 1, "rounds": 2}


FRINGES = {"pad": 0, "peel": 1}
BASES = {"strassen": 0, "winograd": 1, "b323": 2, "b232": 3}


FUSED_KERNELS = {"auto": 0, "smem": 1, "tmem": 2}


def _opts(algo="auto", tile_n=0, num_ctas=0, schedule="auto", bk=0, cta_pair=None, round_tiles=0,
          pipeline=None, fringe="pad", basis="strassen", deterministic=False, outer_scaling=False,
          fused_kernel="auto", store_first=None):
    o = _Options()
    o.store_first = 0 if store_first is None else (2 if store_first else 1)
    o.fused_kernel = FUSED_KERNELS[fused_kernel] if isinstance(fused_kernel, str) else int(fused_kernel)
    o.outer_scaling = 1 if outer_scaling else 0
    o.deterministic = 1 if deterministic else 0
    o.basis = BASES[basis] if isinstance(basis, str) else int(basis)
    o.round_tiles = int(round_tiles)
    o.fringe = FRINGES[fringe] if isinstance(fringe, str) else int(fringe)
    o.pipeline = 0 if pipeline is None else (2 if pipeline else 1)
    o.bk = int(bk)
    o.cta_pair = 0 if cta_pair is None else (2 if cta_pair else 1)
    o.schedule = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    o.algo = ALGOS[algo] if isinstance(algo, str) else int(algo)
    o.tile_n = int(tile_n)
    o.num_ctas = int(num_ctas)
    return o


def _variant(v) -> int:
    return VARIANTS[v] if isinstance(v, str) else int(v)


def workspace_size(m, n, k, levels=1, variant="split3", algo="auto", tile_n=0, cta_pair=None,
                   fringe="pad", basis="strassen", outer_scaling=False) -> int:
    o = _opts(algo, tile_n, cta_pair=cta_pair, fringe=fringe, basis=basis, outer_scaling=outer_scaling)
    ws = load().fmm_workspace_size_ex(m, n, k, levels, _variant(variant), ctypes.byref(o))
    if ws == ctypes.c_size_t(-1).value:
        raise FmmError(3, "unsupported combination")
    return int(ws)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


_IN_DTYPE = {0: "float32", 1: "bfloat16", 2: "float16", 3: "float32"}


def gemm(A, B, C=None, alpha: float = 1.0, beta: float = 0.0, levels: int = 1,
         variant="split3", algo="auto", tile_n: int = 0, num_ctas: int = 0,
         workspace=None, stream=None, schedule="auto", bk: int = 0, cta_pair=None,
         round_tiles: int = 0, pipeline=None, fringe="pad", basis="strassen",
         deterministic: bool = False, outer_scaling: bool = False, fused_kernel="auto",
         store_first=None):
    """C = alpha * A @ B + beta * C on the current CUDA device (torch tensors).

    A (m x k) and B (k x n) are row-major CUDA tensors of the element type the
    variant names (float32 for "split3"/"plain_bf16", bfloat16 for "bf16");
    C is float32 and is allocated when None.  Rows may be padded (stride(0) >= cols)
    but columns must be contiguous.  ``workspace`` is a uint8 CUDA tensor; one of
    the right size is allocated when None.  ``cta_pair``: None = automatic, True = CTA
    pairs (256-row tiles shared by a cluster of two CTAs), False = one CTA per tile.
    ``pipeline``: None = automatic, True / False = overlap the operand-sum passes with the
    tensor-core kernel one top-level product at a time, or not.  ``fringe``: "pad" (zero
    padding of the blocks) or "peel" (Strassen on the evenly splitting core plus classical
    strip products).  ``basis``: "strassen", "winograd" (one level), "b323" (the <3,2,3>
    basis of rank 15) or "b232" (the <2,3,2> basis of rank 11), the last two one level, packed
    or fused algorithm.  ``deterministic``:
    ownership mode, bitwise reproducible results.  ``outer_scaling``: exact power-of-two
    scaling of the rows of A and columns of B around the product (badly scaled inputs).
    ``fused_kernel`` (fused and hybrid algorithms): "auto", "smem" (both operands' sums in shared
    memory) or "tmem" (CTA pairs: the A-operand sums in tensor memory).  ``store_first``
    (packed, beta = 0): None = automatic (on), True / False = the first update of every C
    block stores it (products in launch phases, no zeroing pass), or zero C and add every
    product.
    ``levels="auto"``: the level count and basis the analytic model (``model.py``) predicts
    fastest for this shape and variant (classical, Strassen at one or two levels, or the
    <3,2,3> basis); ``basis`` is then ignored.
    """
    import torch
    v = _variant(variant)
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise FmmError(1, f"inner dimensions differ: {k} vs {k2}")
    if levels == "auto":
        levels, basis = choose(m, n, k, {x: name for name, x in VARIANTS.items()}[v])
    want = getattr(torch, _IN_DTYPE[v])
    for name, X in (("A", A), ("B", B)):
        if X.dtype != want:
            raise FmmError(1, f"{name} must be {want} for variant {variant}")
        if not X.is_cuda:
            raise FmmError(1, f"{name} must be a CUDA tensor")
        if X.numel() and X.stride(1) != 1:
            raise FmmError(1, f"{name} must have contiguous rows")
    if C is None:
        C = torch.empty((m, n), dtype=torch.float32, device=A.device)
        beta = 0.0
    if C.dtype != torch.float32 or not C.is_cuda or (C.numel() and C.stride(1) != 1):
        raise FmmError(1, "C must be a float32 CUDA tensor with contiguous rows")
    ws_need = workspace_size(m, n, k, levels, v, algo, tile_n, cta_pair, fringe, basis, outer_scaling)
    # a classical product of 16-bit operands that TMA can read in place needs no workspace
    in_place = (int(levels) == 0 and v in (VARIANTS["bf16"], VARIANTS["f16"]) and algo in ("auto", "packed")
                and not outer_scaling
                and all(X.data_ptr() % 16 == 0 and _ld(X) % 8 == 0 for X in (A, B)))
    if workspace is None and ws_need > 0 and not in_place:
        workspace = torch.empty(ws_need, dtype=torch.uint8, device=A.device)
    ws_ptr = workspace.data_ptr() if workspace is not None else None
    ws_bytes = workspace.numel() if workspace is not None else 0
    o = _opts(algo, tile_n, num_ctas, schedule, bk, cta_pair, round_tiles, pipeline, fringe, basis,
              deterministic, outer_scaling, fused_kernel, store_first)
    st = load().fmm_gemm_ex(m, n, k, float(alpha), A.data_ptr(), _ld(A),
                            B.data_ptr(), _ld(B), float(beta), C.data_ptr(),
                            _ld(C), int(levels), v, ws_ptr, ws_bytes,
                            _stream_handle(stream), ctypes.byref(o))
    _check(st)
    return C


def _ld(X) -> int:
    """Row stride of a row-major 2-D tensor in elements; for a tensor without elements (whose
    stride torch leaves at 0 or 1) the row length, which the C ABI's checks expect."""
    if X.numel() == 0:
        return max(int(X.shape[1]) if X.dim() == 2 else 1, 1)
    return max(X.stride(0), 1)


def choose(m: int, n: int, k: int, variant="split3"):
    """(levels, basis) that the analytic model predicts fastest for an m x n x k product:
    classical, Strassen at one or two levels, or the <3,2,3> basis at one level."""
    from . import model
    if min(m, n, k) <= 0:
        return 0, "strassen"
    cands = [(0, "strassen"), (1, "strassen"), (2, "strassen"), (1, "b323")]
    return min(cands, key=lambda c: model.predict(m, n, k, c[0], variant, basis=c[1])["ms"])


def workspace_size_backward(m, n, k, levels=1, variant="split3") -> int:
    ws = load().fmm_workspace_size_backward(m, n, k, levels, _variant(variant))
    if ws == ctypes.c_size_t(-1).value:
        raise FmmError(3, "unsupported combination")
    return int(ws)


def gemm_backward(A, B, dC, levels: int = 1, variant="split3", need_dA=True, need_dB=True,
                  workspace=None, stream=None, pipeline=None, basis="strassen", deterministic=False,
                  algo="auto"):
    """(dA, dB) = (dC @ B.T, A.T @ dC) as Strassen products through fmm_gemm_backward_ex.

    A (m x k) and B (k x n) have the variant's element type, dC (m x n) is float32; the
    gradients are float32 (None where not requested).  ``pipeline`` as in gemm();
    ``algo="fused"``: the operand sums are formed on chip from the transposed tiles (FP32
    inputs, no workspace)."""
    import torch
    v = _variant(variant)
    m, k = A.shape
    k2, n = B.shape
    if k != k2 or tuple(dC.shape) != (m, n):
        raise FmmError(1, "shape mismatch")
    want = getattr(torch, _IN_DTYPE[v])
    for name, X in (("A", A), ("B", B)):
        if X.dtype != want or not X.is_cuda or (X.numel() and X.stride(1) != 1):
            raise FmmError(1, f"{name} must be a {want} CUDA tensor with contiguous rows")
    if dC.dtype != torch.float32 or not dC.is_cuda or (dC.numel() and dC.stride(1) != 1):
        raise FmmError(1, "dC must be a float32 CUDA tensor with contiguous rows")
    dA = torch.empty((m, k), dtype=torch.float32, device=A.device) if need_dA else None
    dB = torch.empty((k, n), dtype=torch.float32, device=A.device) if need_dB else None
    o = _opts(algo=algo, pipeline=pipeline, basis=basis, deterministic=deterministic)
    ws_need = load().fmm_workspace_size_backward_ex(m, n, k, levels, v, ctypes.byref(o))
    if ws_need == ctypes.c_size_t(-1).value:
        raise FmmError(3, "unsupported combination")
    if workspace is None and ws_need > 0:
        workspace = torch.empty(ws_need, dtype=torch.uint8, device=A.device)
    st = load().fmm_gemm_backward_ex(
        m, n, k, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B),
        dC.data_ptr(), _ld(dC),
        dA.data_ptr() if dA is not None else None, max(k, 1),
        dB.data_ptr() if dB is not None else None, max(n, 1),
        int(levels), v, workspace.data_ptr() if workspace is not None else None,
        workspace.numel() if workspace is not None else 0, _stream_handle(stream), ctypes.byref(o))
    _check(st)
    return dA, dB


def _make_linear_fn():
    import torch

    class FmmLinearFn(torch.autograd.Function):
        """C = A @ B with a hand-written backward dA = dC @ B^T, dB = A^T @ dC, all three
        computed as Strassen products by the library (no autograd through torch ops)."""

        @staticmethod
        def forward(ctx, A, B, levels=1, variant="split3", deterministic=False):
            ctx.save_for_backward(A, B)
            ctx.levels = levels
            ctx.variant = variant
            ctx.deterministic = deterministic
            return gemm(A, B, levels=levels, variant=variant, deterministic=deterministic)

        @staticmethod
        def backward(ctx, dC):
            A, B = ctx.saved_tensors
            dA, dB = gemm_backward(A, B, dC.contiguous().float(), levels=ctx.levels,
                                   variant=ctx.variant, need_dA=ctx.needs_input_grad[0],
                                   need_dB=ctx.needs_input_grad[1], deterministic=ctx.deterministic)
            # FP32 gradients; autograd casts them to the inputs' dtype where that differs
            return dA, dB, None, None, None

    return FmmLinearFn


_linear_fn = None


def linear(A, B, levels: int = 1, variant="split3", deterministic: bool = False):
    """Differentiable C = A @ B (torch.autograd) backed by the Strassen library.
    deterministic=True: forward and backward in the ownership mode (bitwise reproducible)."""
    global _linear_fn
    if _linear_fn is None:
        _linear_fn = _make_linear_fn()
    return _linear_fn.apply(A, B, levels, variant, deterministic)


def tune_table(classes=None, variant=None):
    """TuneTable from [(max_dim, levels, tile_n), ...] (None = the library's built-in table,
    that of ``variant`` when given), or from a table dict written by
    paper_1808_07984_gb300.autotune."""
    t = TuneTable()
    if classes is None:
        if variant is None:
            load().fmm_tune_default(ctypes.byref(t))
        else:
            load().fmm_tune_default_ex(_variant(variant), ctypes.byref(t))
        return t
    if isinstance(classes, dict):
        classes = [(c["max_dim"], c["levels"], c["tile_n"]) for c in classes["classes"]]
    if not 1 <= len(classes) <= 8:
        raise FmmError(1, "a tune table holds 1 to 8 classes")
    t.count = len(classes)
    for i, (d, lv, tn) in enumerate(classes):
        t.max_dim[i] = min(int(d), 2 ** 63 - 1)
        t.levels[i] = int(lv)
        t.tile_n[i] = int(tn)
    return t


def tune_measure(sizes=(1024, 2048, 4096, 8192, 16384), variant="split3", reps: int = 3,
                 stream=None) -> dict:
    """Native autotuner (fmm_tune_measure): the table dict autotune.autotune returns, measured
    by the library itself."""
    import numpy as np
    sz = np.asarray(sizes, dtype=np.int64)
    times = np.zeros(6 * len(sz), dtype=np.float32)
    t = TuneTable()
    _check(load().fmm_tune_measure(_variant(variant), sz.ctypes.data, len(sz), int(reps), ctypes.byref(t),
                                   times.ctypes.data, _stream_handle(stream)))
    classes = [{"max_dim": int(t.max_dim[i]), "levels": int(t.levels[i]), "tile_n": int(t.tile_n[i])}
               for i in range(t.count)]
    probes = {str(int(d)): {f"L{L}_N{tn}": round(float(times[i * 6 + L * 2 + j]), 4)
                            for L in range(3) for j, tn in enumerate((128, 256))} for i, d in enumerate(sz)}
    return {"classes": classes, "variant": variant, "probes_ms": probes, "native": True}


def tune_select(m, n, k, tune=None):
    """(levels, tile_n) the table assigns to an m x n x k problem."""
    t = tune_table(tune) if not isinstance(tune, TuneTable) else tune
    lv, tn = ctypes.c_int(), ctypes.c_int()
    _check(load().fmm_tune_select(ctypes.byref(t), m, n, k, ctypes.byref(lv), ctypes.byref(tn)))
    return lv.value, tn.value


def _default_tune(variant=None):
    path = os.environ.get("FMM_TUNE_FILE")
    if path and os.path.exists(path):
        from . import autotune
        return tune_table(autotune.load(path))
    return tune_table(None, variant)


class BatchedPlan:
    """Many products C_p = alpha_p A_p @ B_p + beta_p C_p in one persistent tensor-core
    launch per tile width.  Creating the plan uploads the per-problem parameter blocks into
    the workspace; execute() only launches kernels, so it can be captured in a CUDA graph
    (keep the plan, its workspace and the tensors alive while the graph is used)."""

    def __init__(self, As, Bs, Cs, alphas=None, betas=None, variant="split3", tune=None,
                 workspace=None):
        import torch
        L = load()
        self.variant = _variant(variant)
        cnt = len(As)
        if not (len(Bs) == len(Cs) == cnt):
            raise FmmError(1, "A, B and C lists differ in length")
        want = getattr(torch, _IN_DTYPE[self.variant])
        for X in list(As) + list(Bs):
            if X.dtype != want or not X.is_cuda or (X.numel() and X.stride(1) != 1):
                raise FmmError(1, f"operands must be {want} CUDA tensors with contiguous rows")
        for X in Cs:
            if X.dtype != torch.float32 or not X.is_cuda or (X.numel() and X.stride(1) != 1):
                raise FmmError(1, "C must be float32 CUDA tensors with contiguous rows")
        I64 = ctypes.c_int64 * cnt
        F32 = ctypes.c_float * cnt
        VP = ctypes.c_void_p * cnt
        self._m = I64(*[a.shape[0] for a in As])
        self._n = I64(*[b.shape[1] for b in Bs])
        self._k = I64(*[a.shape[1] for a in As])
        self._alpha = F32(*(alphas if alphas is not None else [1.0] * cnt))
        self._beta = F32(*(betas if betas is not None else [0.0] * cnt))
        self._A = VP(*[a.data_ptr() for a in As])
        self._B = VP(*[b.data_ptr() for b in Bs])
        self._C = VP(*[c.data_ptr() for c in Cs])
        self._lda = I64(*[_ld(a) for a in As])
        self._ldb = I64(*[_ld(b) for b in Bs])
        self._ldc = I64(*[_ld(c) for c in Cs])
        self._tune = tune if isinstance(tune, TuneTable) else (tune_table(tune) if tune is not None
                                                               else _default_tune(self.variant))
        ws = L.fmm_batched_workspace_size(cnt, self._m, self._n, self._k, self.variant,
                                          ctypes.byref(self._tune))
        if ws == ctypes.c_size_t(-1).value:
            _check(3)
        if workspace is None:
            workspace = torch.empty(max(ws, 256), dtype=torch.uint8, device=As[0].device)
        self.workspace = workspace
        self._keep = (As, Bs, Cs)
        handle = ctypes.c_void_p()
        _check(L.fmm_batched_plan_create(cnt, self._m, self._n, self._k, self._alpha, self._A,
                                         self._lda, self._B, self._ldb, self._beta, self._C,
                                         self._ldc, self.variant, ctypes.byref(self._tune),
                                         workspace.data_ptr(), workspace.numel(),
                                         ctypes.byref(handle)))
        self._handle = handle

    def execute(self, stream=None):
        _check(load().fmm_batched_plan_execute(self._handle, _stream_handle(stream)))

    def close(self):
        if getattr(self, "_handle", None):
            load().fmm_batched_plan_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gemm_batched(As, Bs, Cs=None, alphas=None, betas=None, variant="split3", tune=None,
                 workspace=None, stream=None):
    """C_p = alpha_p A_p @ B_p + beta_p C_p for every p, one persistent launch per tile width."""
    import torch
    if Cs is None:
        Cs = [torch.empty((a.shape[0], b.shape[1]), dtype=torch.float32, device=a.device)
              for a, b in zip(As, Bs)]
        betas = [0.0] * len(As)
    plan = BatchedPlan(As, Bs, Cs, alphas, betas, variant, tune, workspace)
    plan.execute(stream)
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    plan.close()
    return Cs


def device_status(stream=None):
    """Synchronise and raise FmmError if a device-side wait timed out."""
    _check(load().fmm_device_status(_stream_handle(stream)))


def set_wait_timeout_ns(ns: int):
    load().fmm_set_wait_timeout_ns(int(ns))


def debug_wait_timeout(stream=None):
    _check(load().fmm_debug_wait_timeout(_stream_handle(stream)))


PHASES = ("beta", "pack", "tensor")


def profile_enable(on: bool = True):
    """Bracket every launch of each phase with CUDA events (see fmm_profile_read)."""
    _check(load().fmm_profile_enable(1 if on else 0))


def profile_read():
    """{phase: (milliseconds, launches)} summed since the previous read."""
    import numpy as np
    ms = np.zeros(3, dtype=np.float64)
    n = np.zeros(3, dtype=np.int64)
    _check(load().fmm_profile_read(ms.ctypes.data, n.ctypes.data))
    return {p: (float(ms[i]), int(n[i])) for i, p in enumerate(PHASES)}


def basis_shape(levels: int, basis="strassen"):
    """(g_m, g_k, g_n, R): block grid and product count of ``levels`` levels of a basis."""
    dims = (ctypes.c_int * 4)()
    if load().fmm_basis_shape(levels, BASES[basis] if isinstance(basis, str) else int(basis), dims) != 0:
        raise FmmError(3, "basis and levels not built")
    return tuple(int(x) for x in dims)


def product_table(levels: int, basis="strassen"):
    """(U, V, W) int8 arrays as the kernels use them: U of shape (g_m g_k, R) with row
    i * g_k + l for A block (i, l), V (g_k g_n, R) with row l * g_n + j, W (g_m g_n, R) with
    row i * g_n + j (for the 2x2 bases: (4**L, 7**L), row bi * 2**L + bj)."""
    import numpy as np
    gm, gk, gn, R = basis_shape(levels, basis)
    U = np.zeros(gm * gk * R, dtype=np.int8)
    V = np.zeros(gk * gn * R, dtype=np.int8)
    W = np.zeros(gm * gn * R, dtype=np.int8)
    b = BASES[basis] if isinstance(basis, str) else int(basis)
    r = load().fmm_product_table_ex(levels, b, U.ctypes.data, V.ctypes.data, W.ctypes.data)
    if r != R:
        raise FmmError(1, "bad levels")
    return U.reshape(gm * gk, R), V.reshape(gk * gn, R), W.reshape(gm * gn, R)

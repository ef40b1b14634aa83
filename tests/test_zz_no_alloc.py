"""fmm_gemm_noalloc: the entry point for callers that cannot allocate device memory
(a plug-in whose host application owns all device allocations, or a latency-critical
caller that must not call cudaMalloc / cudaFree because they can synchronise the device).
On consecutive calls that reuse its built-in 64 MiB scratch it must agree with the FP64
oracle within the parity bounds and with fmm_gemm (which takes a caller-provided
workspace); it must run a classical product of aligned 16-bit operands, which needs no
workspace, whatever the workspace estimate; and it must reject problems that do not fit
its scratch.

Collected last (file name) so that a run stopping at the first failure has already run
every other test."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1808_07984_gb300 as fmm
import synth
from bounds import tolerance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fmm.build()
    oracle.build()
    L = fmm.load()
    i64, i32, f32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_void_p
    L.fmm_gemm_noalloc.restype = i32
    L.fmm_gemm_noalloc.argtypes = [i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64, i32, i32, vp]
    return L


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _err(C, C64, An, Bn):
    return oracle.normwise_error(C.cpu().numpy().astype(np.float64), C64, An, Bn)


def test_noalloc_matches_the_oracle_and_fmm_gemm_on_consecutive_calls(lib):
    cases = [(512, 512, 512, 1, 31), (300, 520, 200, 2, 32), (256, 384, 640, 0, 33)]
    for m, n, k, levels, seed in cases:
        A, B = synth.problem(m, n, k, seed, "uniform")
        Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        C64 = oracle.classical(A, B)
        An, Bn = np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64))
        tol = tolerance("split3", levels, k)
        # existing entry point, caller-provided workspace
        ws = torch.empty(max(fmm.workspace_size(m, n, k, levels, "split3"), 256),
                         dtype=torch.uint8, device="cuda")
        C_ref = torch.empty((m, n), dtype=torch.float32, device="cuda")
        st = lib.fmm_gemm(m, n, k, 1.0, Ad.data_ptr(), k, Bd.data_ptr(), n, 0.0,
                          C_ref.data_ptr(), n, levels, 0, ws.data_ptr(), ws.numel(), _stream())
        assert st == 0, lib.fmm_last_error()
        # no-allocation entry point, twice in a row on the shared scratch; C starts as NaN
        # to show that beta = 0 does not read it
        for _ in range(2):
            C = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
            st = lib.fmm_gemm_noalloc(m, n, k, 1.0, Ad.data_ptr(), k, Bd.data_ptr(), n, 0.0,
                                      C.data_ptr(), n, levels, 0, _stream())
            assert st == 0, lib.fmm_last_error()
            fmm.device_status()
            err = _err(C, C64, An, Bn)
            assert err <= tol, (m, n, k, levels, err)
            diff = (C.double() - C_ref.double()).norm().item() / (An * Bn)
            assert diff <= tol, (m, n, k, levels, diff)


def test_noalloc_runs_in_place_16bit_classical_products_beyond_its_scratch(lib):
    """A classical BF16 product whose operands TMA reads in place needs no workspace, although
    fmm_workspace_size counts 128 MiB of conversion space for it (it cannot see the pointers)."""
    m, n, k = 8192, 8192, 4096
    assert fmm.workspace_size(m, n, k, 0, "bf16") > 64 << 20
    A, B = synth.problem(m, n, k, 41, "gaussian")
    Ad = torch.from_numpy(A).to(torch.bfloat16).cuda()
    Bd = torch.from_numpy(B).to(torch.bfloat16).cuda()
    C_ref = torch.empty((m, n), dtype=torch.float32, device="cuda")
    st = lib.fmm_gemm(m, n, k, 1.0, Ad.data_ptr(), k, Bd.data_ptr(), n, 0.0, C_ref.data_ptr(), n,
                      0, 1, None, 0, _stream())
    assert st == 0, lib.fmm_last_error()
    rows = np.unique(synth.rng(42).integers(0, m, size=6))
    rsel = torch.from_numpy(rows).cuda()
    Ab = Ad[rsel].cpu().view(torch.int16).numpy().view(np.uint16)
    Bb = Bd.cpu().view(torch.int16).numpy().view(np.uint16)
    C64 = oracle.classical(Ab, Bb, a_code=oracle.ORC_BF16, b_code=oracle.ORC_BF16)
    An = float(Ad[rsel].float().norm())
    Bn = float(Bd.float().norm())
    for _ in range(2):
        C = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.fmm_gemm_noalloc(m, n, k, 1.0, Ad.data_ptr(), k, Bd.data_ptr(), n, 0.0, C.data_ptr(),
                                  n, 0, 1, _stream())
        assert st == 0, lib.fmm_last_error()
        fmm.device_status()
        assert _err(C[rsel], C64, An, Bn) <= tolerance("bf16", 0, k)
        assert torch.equal(C[rsel], C_ref[rsel])


def test_noalloc_rejects_problems_larger_than_its_scratch(lib):
    # 8192^3 at one level needs about 940 MB of workspace; the call must refuse before
    # touching the (fake, non-overlapping) pointers.
    a, b, c = 0x100000000000, 0x200000000000, 0x300000000000
    st = lib.fmm_gemm_noalloc(8192, 8192, 8192, 1.0, a, 8192, b, 8192, 0.0, c, 8192, 1, 0, _stream())
    assert st == 4
    assert b"scratch" in lib.fmm_last_error()

"""fmm_gemm_noalloc: the entry point for callers that cannot allocate device memory
(a plug-in whose host application owns all device allocations, or a latency-critical
caller that must not call cudaMalloc / cudaFree).  It must give the same products as
fmm_gemm, which takes a caller-provided workspace, on consecutive calls that reuse its
built-in 64 MiB scratch, and must reject problems that do not fit that scratch.

Collected last (file name) so that a run stopping at the first failure has already run
every other test."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1808_07984_gb300 as fmm
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-6  # split3 normwise bound used by the parity tests for k >= 64


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fmm.build()
    L = fmm.load()
    i64, i32, f32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_void_p
    L.fmm_gemm_noalloc.restype = i32
    L.fmm_gemm_noalloc.argtypes = [i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64, i32, i32, vp]
    return L


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_noalloc_matches_fmm_gemm_on_consecutive_calls(lib):
    cases = [(512, 512, 512, 1, 31), (300, 520, 200, 2, 32), (256, 384, 640, 0, 33)]
    for m, n, k, levels, seed in cases:
        A, B = synth.problem(m, n, k, seed, "uniform")
        Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        # existing entry point, caller-provided workspace
        ws = torch.empty(max(fmm.workspace_size(m, n, k, levels, "split3"), 256),
                         dtype=torch.uint8, device="cuda")
        C_ref = torch.empty((m, n), dtype=torch.float32, device="cuda")
        st = lib.fmm_gemm(m, n, k, 1.0, Ad.data_ptr(), k, Bd.data_ptr(), n, 0.0,
                          C_ref.data_ptr(), n, levels, 0, ws.data_ptr(), ws.numel(), _stream())
        assert st == 0, lib.fmm_last_error()
        # no-allocation entry point; C starts as NaN to show beta = 0 does not read it
        C = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.fmm_gemm_noalloc(m, n, k, 1.0, Ad.data_ptr(), k, Bd.data_ptr(), n, 0.0,
                                  C.data_ptr(), n, levels, 0, _stream())
        assert st == 0, lib.fmm_last_error()
        fmm.device_status()
        diff = (C.double() - C_ref.double()).norm().item()
        err = diff / (np.linalg.norm(A.astype(np.float64)) * np.linalg.norm(B.astype(np.float64)))
        assert err <= TOL, (m, n, k, levels, err)


def test_noalloc_rejects_problems_larger_than_its_scratch(lib):
    # 8192^3 at one level needs about 940 MB of workspace; the call must refuse before
    # touching the (fake) pointers.
    st = lib.fmm_gemm_noalloc(8192, 8192, 8192, 1.0, 0x1000, 8192, 0x2000, 8192, 0.0, 0x3000,
                              8192, 1, 0, _stream())
    assert st == 4
    assert b"scratch" in lib.fmm_last_error()

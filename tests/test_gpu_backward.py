"""Backward products dA = dC @ B^T and dB = A^T @ dC (fmm_gemm_backward) and the
differentiable layer, against the FP64 oracle.  Integer inputs are bit-exact; floats
within the normwise bounds of test_gpu_parity."""

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


def _tol(variant, levels, k):
    return tolerance(variant, levels, k)


def _err(X, X64, An, Bn):
    return oracle.normwise_error(X, X64, An, Bn)


@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("m,n,k", [(16, 16, 16), (300, 200, 136), (129, 65, 257), (1, 40, 33)])
def test_backward_int_bit_exact(m, n, k, levels):
    A, B = synth.problem(m, n, k, 7 + m, "int")
    dC = synth.small_int((m, n), 8 + n)
    dA, dB = fmm.gemm_backward(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                               torch.from_numpy(dC).cuda(), levels=levels)
    fmm.device_status()
    np.testing.assert_array_equal(dA.cpu().numpy(), oracle.classical(dC, np.ascontiguousarray(B.T)))
    np.testing.assert_array_equal(dB.cpu().numpy(), oracle.classical(np.ascontiguousarray(A.T), dC))


@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("m,n,k", [(300, 200, 136), (129, 65, 257)])
def test_backward_pipelined_int_bit_exact(m, n, k, levels):
    """Transposed-quadrant sums formed per top-level product (pipelined)."""
    A, B = synth.problem(m, n, k, 9 + m, "int")
    dC = synth.small_int((m, n), 10 + n)
    dA, dB = fmm.gemm_backward(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                               torch.from_numpy(dC).cuda(), levels=levels, pipeline=True)
    fmm.device_status()
    np.testing.assert_array_equal(dA.cpu().numpy(), oracle.classical(dC, np.ascontiguousarray(B.T)))
    np.testing.assert_array_equal(dB.cpu().numpy(), oracle.classical(np.ascontiguousarray(A.T), dC))


@pytest.mark.parametrize("m,n,k", [(300, 200, 136), (129, 65, 257)])
def test_backward_winograd_int_bit_exact(m, n, k):
    A, B = synth.problem(m, n, k, 19 + m, "int")
    dC = synth.small_int((m, n), 20 + n)
    dA, dB = fmm.gemm_backward(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                               torch.from_numpy(dC).cuda(), levels=1, basis="winograd")
    fmm.device_status()
    np.testing.assert_array_equal(dA.cpu().numpy(), oracle.classical(dC, np.ascontiguousarray(B.T)))
    np.testing.assert_array_equal(dB.cpu().numpy(), oracle.classical(np.ascontiguousarray(A.T), dC))


@pytest.mark.parametrize("basis", ["b323", "b232"])
@pytest.mark.parametrize("m,n,k", [(300, 200, 136), (129, 65, 257), (600, 610, 250)])
def test_backward_table_basis_int_bit_exact(m, n, k, basis):
    """dA = dC B^T and dB = A^T dC as <3,2,3> products: the table pass reads the stored
    operand blocks transposed."""
    A, B = synth.problem(m, n, k, 21 + m, "int")
    dC = synth.small_int((m, n), 22 + n)
    dA, dB = fmm.gemm_backward(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                               torch.from_numpy(dC).cuda(), levels=1, basis=basis)
    fmm.device_status()
    np.testing.assert_array_equal(dA.cpu().numpy(), oracle.classical(dC, np.ascontiguousarray(B.T)))
    np.testing.assert_array_equal(dB.cpu().numpy(), oracle.classical(np.ascontiguousarray(A.T), dC))


@pytest.mark.parametrize("variant", ["split3", "plain_bf16"])
@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("m,n,k", [(257, 300, 140), (512, 384, 640)])
def test_backward_float(m, n, k, levels, variant):
    A, B = synth.problem(m, n, k, 3 * m + k, "gaussian")
    dC = synth.gaussian((m, n), 11)
    dA, dB = fmm.gemm_backward(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                               torch.from_numpy(dC).cuda(), levels=levels, variant=variant)
    fmm.device_status()
    Bt = np.ascontiguousarray(B.T)
    At = np.ascontiguousarray(A.T)
    nA, nB, nC = (np.linalg.norm(X.astype(np.float64)) for X in (A, B, dC))
    assert _err(dA.cpu().numpy(), oracle.classical(dC, Bt), nC, nB) <= _tol(variant, levels, n)
    assert _err(dB.cpu().numpy(), oracle.classical(At, dC), nA, nC) <= _tol(variant, levels, m)


@pytest.mark.parametrize("variant", ["split3", "plain_bf16"])
@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("m,n,k", [(16, 16, 16), (300, 200, 136), (129, 65, 257), (520, 8, 400), (1000, 1200, 300)])
def test_backward_fused_int_bit_exact(m, n, k, levels, variant):
    """dA = dC B^T and dB = A^T dC with the operand sums formed on chip: the tensor-memory
    kernel reads B^T as tiles stored by rows of n and A^T as tiles stored by rows of k."""
    pad = lambda c: (-c) % 4
    A, B = synth.problem(m, n, k, 17 + m, "int")
    dC = synth.small_int((m, n), 18 + n)

    def dev(X):
        r, c = X.shape
        t = torch.zeros((r, c + pad(c)), dtype=torch.float32, device="cuda")
        t[:, :c] = torch.from_numpy(X).cuda()
        return t[:, :c]
    dA, dB = fmm.gemm_backward(dev(A), dev(B), dev(dC), levels=levels, variant=variant, algo="fused")
    fmm.device_status()
    np.testing.assert_array_equal(dA.cpu().numpy(), oracle.classical(dC, np.ascontiguousarray(B.T)))
    np.testing.assert_array_equal(dB.cpu().numpy(), oracle.classical(np.ascontiguousarray(A.T), dC))


@pytest.mark.parametrize("levels", [1, 2])
def test_backward_fused_float(levels):
    m, n, k = 700, 520, 900
    A, B = synth.problem(m, n, k, 19, "gaussian")
    dC = synth.gaussian((m, n), 20)
    dA, dB = fmm.gemm_backward(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                               torch.from_numpy(dC).cuda(), levels=levels, algo="fused")
    fmm.device_status()
    nA, nB, nC = (np.linalg.norm(X.astype(np.float64)) for X in (A, B, dC))
    assert _err(dA.cpu().numpy(), oracle.classical(dC, np.ascontiguousarray(B.T)), nC, nB) <= _tol("split3", levels, n)
    assert _err(dB.cpu().numpy(), oracle.classical(np.ascontiguousarray(A.T), dC), nA, nC) <= _tol("split3", levels, m)


def test_backward_fused_full_size_sampled_rows():
    """The C3 layer shape in FP32 (8192 x 4096 x 4096), gradients on chip, sampled rows."""
    m, k, n = 8192, 4096, 4096
    A, B = synth.problem(m, n, k, 21, "gaussian")
    dC = synth.gaussian((m, n), 22)
    dA, dB = fmm.gemm_backward(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                               torch.from_numpy(dC).cuda(), levels=1, algo="fused")
    fmm.device_status()
    rng = synth.rng(23)
    ra = np.unique(rng.integers(0, m, size=6))
    rb = np.unique(rng.integers(0, k, size=6))
    dA64 = oracle.classical(dC, np.ascontiguousarray(B.T), rows=ra)
    dB64 = oracle.classical(np.ascontiguousarray(A.T), dC, rows=rb)
    nB, nC = np.linalg.norm(B.astype(np.float64)), np.linalg.norm(dC.astype(np.float64))
    assert _err(dA.cpu().numpy()[ra], dA64, np.linalg.norm(dC[ra].astype(np.float64)), nB) <= _tol("split3", 1, n)
    assert _err(dB.cpu().numpy()[rb], dB64, np.linalg.norm(A[:, rb].astype(np.float64)), nC) <= _tol("split3", 1, m)


def test_backward_fused_rejected_for_16bit_operands():
    A = torch.zeros((64, 64), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(fmm.FmmError) as ei:
        fmm.gemm_backward(A, A, torch.zeros((64, 64), device="cuda"), levels=1, variant="bf16", algo="fused")
    assert ei.value.status == 3


def test_backward_bf16_inputs_fp32_grads():
    """BF16 A and B, FP32 dC: each operand sum is rounded once to BF16."""
    m, n, k = 384, 256, 320
    A, B = synth.problem(m, n, k, 4, "gaussian")
    dC = synth.gaussian((m, n), 5)
    Ab = torch.from_numpy(A).to(torch.bfloat16).cuda()
    Bb = torch.from_numpy(B).to(torch.bfloat16).cuda()
    dA, dB = fmm.gemm_backward(Ab, Bb, torch.from_numpy(dC).cuda(), levels=1, variant="bf16")
    fmm.device_status()
    assert dA.dtype == torch.float32 and dB.dtype == torch.float32
    Abits = Ab.cpu().view(torch.int16).numpy().view(np.uint16)
    Bbits = Bb.cpu().view(torch.int16).numpy().view(np.uint16)
    dA64 = oracle.classical(dC, np.ascontiguousarray(Bbits.T), b_code=oracle.ORC_BF16)
    dB64 = oracle.classical(np.ascontiguousarray(Abits.T), dC, a_code=oracle.ORC_BF16)
    nA = float(Ab.float().norm())
    nB = float(Bb.float().norm())
    nC = float(np.linalg.norm(dC.astype(np.float64)))
    assert _err(dA.cpu().numpy(), dA64, nC, nB) <= _tol("bf16", 1, n)
    assert _err(dB.cpu().numpy(), dB64, nA, nC) <= _tol("bf16", 1, m)


@pytest.mark.parametrize("m,n,k", [(384, 256, 320), (130, 260, 72), (257, 129, 65)])
def test_backward_bf16_classical_int_bit_exact(m, n, k):
    """L = 0 with BF16 A and B: the BF16 operand of each gradient product is read in place
    when its rows are 16-byte aligned, the FP32 dC is converted; exact on small integers."""
    A, B = synth.problem(m, n, k, 23 + m, "int")
    dC = synth.small_int((m, n), 24 + n)
    Ab = torch.from_numpy(A).to(torch.bfloat16).cuda()
    Bb = torch.from_numpy(B).to(torch.bfloat16).cuda()
    dA, dB = fmm.gemm_backward(Ab, Bb, torch.from_numpy(dC).cuda(), levels=0, variant="bf16")
    fmm.device_status()
    np.testing.assert_array_equal(dA.cpu().numpy(), oracle.classical(dC, np.ascontiguousarray(B.T)))
    np.testing.assert_array_equal(dB.cpu().numpy(), oracle.classical(np.ascontiguousarray(A.T), dC))


@pytest.mark.parametrize("levels", [1, 2])
def test_linear_autograd_matches_oracle_and_finite_differences(levels):
    m, n, k = 256, 192, 320
    A, B = synth.problem(m, n, k, 12, "gaussian")
    G = synth.gaussian((m, n), 13)
    Ad = torch.from_numpy(A).cuda().requires_grad_(True)
    Bd = torch.from_numpy(B).cuda().requires_grad_(True)
    Gd = torch.from_numpy(G).cuda()
    C = fmm.linear(Ad, Bd, levels=levels)
    loss = (C * Gd).sum()
    loss.backward()
    fmm.device_status()
    nA, nB, nG = (np.linalg.norm(X.astype(np.float64)) for X in (A, B, G))
    dA64 = oracle.classical(G, np.ascontiguousarray(B.T))
    dB64 = oracle.classical(np.ascontiguousarray(A.T), G)
    assert _err(Ad.grad.cpu().numpy(), dA64, nG, nB) <= _tol("split3", levels, n)
    assert _err(Bd.grad.cpu().numpy(), dB64, nA, nG) <= _tol("split3", levels, m)
    # The loss is bilinear, so a central difference with any step is exact up to rounding:
    # (L(A + E) - L(A - E)) / 2 = <G, E B> = <dA, E>.
    E = torch.from_numpy(synth.gaussian((m, k), 14)).cuda()
    with torch.no_grad():
        lp = (fmm.linear(Ad + E, Bd, levels=levels) * Gd).double().sum()
        lm = (fmm.linear(Ad - E, Bd, levels=levels) * Gd).double().sum()
    fd = float((lp - lm) / 2)
    an = float((Ad.grad.double() * E.double()).sum())
    scale = float(np.linalg.norm(G) * np.linalg.norm(B.astype(np.float64)) * E.double().norm())
    assert abs(fd - an) <= 1e-5 * scale


@pytest.mark.parametrize("levels", [1, 2])
def test_linear_layer_shapes_sampled_rows(levels):
    """Differentiable layer at 8192 x 4096 x 4096 with BF16 inputs (one and two levels);
    gradients checked on sampled rows of dA and of dB against the FP64 oracle."""
    m, k, n = 8192, 4096, 4096
    rng = synth.rng(31)
    A = torch.from_numpy(synth.gaussian((m, k), 32)).to(torch.bfloat16).cuda().requires_grad_(True)
    B = torch.from_numpy(synth.gaussian((k, n), 33)).to(torch.bfloat16).cuda().requires_grad_(True)
    dC = torch.from_numpy(synth.gaussian((m, n), 34)).cuda()
    C = fmm.linear(A, B, levels=levels, variant="bf16")
    C.backward(dC)
    fmm.device_status()
    Af = A.detach().float().cpu().numpy().astype(np.float64)
    Bf = B.detach().float().cpu().numpy().astype(np.float64)
    dCn = dC.cpu().numpy()
    ra = np.unique(rng.integers(0, m, size=6))
    rb = np.unique(rng.integers(0, k, size=6))
    # dA[ra] = dC[ra] B^T;  dB[rb] = A[:, rb]^T dC  (inputs are exact in FP64)
    dA64 = oracle.classical(dCn, np.ascontiguousarray(Bf.T), rows=ra)
    dB64 = oracle.classical(np.ascontiguousarray(Af.T), dCn, rows=rb)
    gA = A.grad.float().cpu().numpy()[ra]
    gB = B.grad.float().cpu().numpy()[rb]
    # gradients come back in the inputs' dtype (BF16): allow that rounding on top
    tol = _tol("bf16", levels, 4096) + 2.0 ** -8
    assert _err(gA, dA64, np.linalg.norm(dCn[ra].astype(np.float64)), np.linalg.norm(Bf)) <= tol
    assert _err(gB, dB64, np.linalg.norm(Af[:, rb]), np.linalg.norm(dCn.astype(np.float64))) <= tol


@pytest.mark.parametrize("levels", [1, 2])
def test_linear_gradcheck_64(levels):
    """torch.autograd.gradcheck of the library-backed layer at 64^3 (config C3's check).  The
    library takes no FP64 operands, so the layer runs in FP32 (split3).  It is bilinear, so a
    central difference with step 1 is exact up to the rounding of the forward products; the
    tolerance is that rounding: the split3 normwise bound at k = 64 turned into a per-element
    bound (times ||A||_F ||B||_F / sqrt(m n), six standard deviations)."""
    g = torch.Generator(device="cpu").manual_seed(77 + levels)
    A = torch.randn((64, 64), generator=g).cuda().requires_grad_(True)
    B = torch.randn((64, 64), generator=g).cuda().requires_grad_(True)
    per_elem = 6 * _tol("split3", levels, 64) * float(A.detach().norm() * B.detach().norm()) / 64
    # the ownership mode makes repeated backward calls bitwise identical (gradcheck's
    # reentrancy check uses a zero tolerance)
    assert torch.autograd.gradcheck(lambda a, b: fmm.linear(a, b, levels=levels, deterministic=True), (A, B),
                                    eps=1.0, atol=per_elem, rtol=0.0, fast_mode=True)
    fmm.device_status()


def _fd64_gradients(A, B, G):
    """dL/dA and dL/dB of L(A, B) = <G, A B> by FP64 central differences of the oracle's
    product (step 1, exact for a bilinear map up to FP64 rounding).  Perturbing A[i, l]
    changes only row i of the product, and B[l, j] only column j, so one oracle call per row
    of A (its 64 perturbed copies stacked) and per column of B suffices."""
    m, k = A.shape
    n = B.shape[1]
    dA = np.zeros((m, k))
    for i in range(m):
        rows = np.repeat(A[i:i + 1].astype(np.float64), k, axis=0)
        plus = oracle.classical(rows + np.eye(k), B)
        minus = oracle.classical(rows - np.eye(k), B)
        dA[i] = (plus - minus) @ G[i].astype(np.float64) / 2.0
    dB = np.zeros((k, n))
    for j in range(n):
        cols = np.repeat(B[:, j:j + 1].astype(np.float64), k, axis=1)
        plus = oracle.classical(A, cols + np.eye(k))
        minus = oracle.classical(A, cols - np.eye(k))
        dB[:, j] = G[:, j].astype(np.float64) @ (plus - minus) / 2.0
    return dA, dB


@pytest.mark.parametrize("levels", [0, 1, 2])
def test_linear_gradients_64_against_fp64_finite_differences(levels):
    """Config C3's FP64 check: the layer's dA and dB at 64^3 against FP64 central differences
    of the CPU oracle and against the classical FP64 gradient, normwise within the split3
    bound at k = 64."""
    A, B = synth.problem(64, 64, 64, 90 + levels, "gaussian")
    G = synth.gaussian((64, 64), 93 + levels)
    Ad = torch.from_numpy(A).cuda().requires_grad_(True)
    Bd = torch.from_numpy(B).cuda().requires_grad_(True)
    (fmm.linear(Ad, Bd, levels=levels) * torch.from_numpy(G).cuda()).sum().backward()
    fmm.device_status()
    fdA, fdB = _fd64_gradients(A, B, G)
    gA64 = oracle.classical(G, np.ascontiguousarray(B.T))
    gB64 = oracle.classical(np.ascontiguousarray(A.T), G)
    # the two FP64 references agree to FP64 rounding
    assert np.abs(fdA - gA64).max() <= 1e-9 and np.abs(fdB - gB64).max() <= 1e-9
    nA, nB, nG = (np.linalg.norm(X.astype(np.float64)) for X in (A, B, G))
    tol = _tol("split3", levels, 64)
    assert _err(Ad.grad.cpu().numpy(), fdA, nG, nB) <= tol
    assert _err(Bd.grad.cpu().numpy(), fdB, nA, nG) <= tol


def test_library_call_from_a_fresh_thread():
    """A thread that has made no CUDA call yet (as autograd's device thread may be) can call
    the library: it makes the device's context current itself."""
    import threading
    A, B = synth.problem(96, 80, 64, 81, "int")
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    out = {}

    def work():
        try:
            out["C"] = fmm.gemm(Ad, Bd, levels=1).cpu().numpy()
        except Exception as exc:  # noqa: BLE001 - reported below
            out["err"] = exc

    t = threading.Thread(target=work)
    t.start()
    t.join()
    assert "err" not in out, out.get("err")
    np.testing.assert_array_equal(out["C"], oracle.classical(A, B))

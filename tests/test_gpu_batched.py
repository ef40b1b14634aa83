"""Batched uneven products in one persistent launch (fmm_batched_plan_*), CUDA-graph
capture and replay, the scaled FP16 arithmetic, against the FP64 oracle."""

import numpy as np
import pytest
import torch

import oracle
import paper_1808_07984_gb300 as fmm
import synth
from bounds import tolerance

pytestmark = pytest.mark.gpu

MIXED = [(0, 1000, 0), (1, 2000, 256), (2, 2 ** 62, 128)]  # levels by size class, mixed tiles


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fmm.build()
    fmm.load()
    oracle.build()


def _table(classes):
    return [(d, lv, tn) for lv, d, tn in classes]


SHAPES = [(16, 16, 16), (300, 520, 200), (1100, 900, 1300), (257, 129, 65), (2100, 2300, 2050),
          (512, 512, 512), (1, 300, 1), (640, 384, 1000)]


def test_batched_int_bit_exact_mixed_levels_and_tiles():
    As, Bs, Cs, C0s, host = [], [], [], [], []
    for i, (m, n, k) in enumerate(SHAPES):
        A, B = synth.problem(m, n, k, 100 + i, "int")
        C0 = synth.small_int((m, n), 200 + i)
        As.append(torch.from_numpy(A).cuda())
        Bs.append(torch.from_numpy(B).cuda())
        Cs.append(torch.from_numpy(C0).cuda())
        host.append((A, B, C0))
    alphas = [1.0, -2.0, 3.0, 1.0, 0.5, 1.0, 2.0, -1.0]
    betas = [0.0, 1.0, -1.0, 2.0, 0.0, 1.0, 0.0, 3.0]
    fmm.gemm_batched(As, Bs, Cs, alphas, betas, tune=_table(MIXED))
    fmm.device_status()
    for i, (A, B, C0) in enumerate(host):
        want = oracle.classical(A, B, C0, alphas[i], betas[i])
        np.testing.assert_array_equal(Cs[i].cpu().numpy(), want, err_msg=str(SHAPES[i]))


@pytest.mark.parametrize("variant", ["split3", "f16"])
def test_batched_float(variant):
    shapes = [(256 * a, 256 * b, 256 * c) for a, b, c in [(2, 3, 4), (4, 4, 4), (1, 7, 2), (5, 2, 3)]]
    dt = torch.float16 if variant == "f16" else torch.float32
    As, Bs, hostA, hostB = [], [], [], []
    for i, (m, n, k) in enumerate(shapes):
        A, B = synth.problem(m, n, k, 300 + i, "uniform")
        Ad, Bd = torch.from_numpy(A).to(dt).cuda(), torch.from_numpy(B).to(dt).cuda()
        As.append(Ad)
        Bs.append(Bd)
        hostA.append(Ad.float().cpu().numpy().astype(np.float64))
        hostB.append(Bd.float().cpu().numpy().astype(np.float64))
    Cs = fmm.gemm_batched(As, Bs, variant=variant, tune=_table(MIXED))
    fmm.device_status()
    for i, (m, n, k) in enumerate(shapes):
        C64 = oracle.classical(hostA[i], hostB[i])
        err = oracle.normwise_error(Cs[i].cpu().numpy(), C64, np.linalg.norm(hostA[i]),
                                    np.linalg.norm(hostB[i]))
        lv = fmm.tune_select(m, n, k, _table(MIXED))[0]
        assert err <= tolerance(variant, lv, k), (shapes[i], err)


def test_batched_graph_capture_and_replay():
    shapes = SHAPES[1:6]
    As, Bs, Cs, host = [], [], [], []
    for i, (m, n, k) in enumerate(shapes):
        A, B = synth.problem(m, n, k, 400 + i, "int")
        As.append(torch.from_numpy(A).cuda())
        Bs.append(torch.from_numpy(B).cuda())
        Cs.append(torch.zeros((m, n), dtype=torch.float32, device="cuda"))
        host.append((A, B))
    plan = fmm.BatchedPlan(As, Bs, Cs, tune=_table(MIXED))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.execute(s)  # eager run on the capture stream first
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    eager = [c.clone() for c in Cs]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.execute()
    for c in Cs:
        c.zero_()
    graph.replay()
    torch.cuda.synchronize()
    fmm.device_status()
    for e, c in zip(eager, Cs):
        assert torch.equal(e, c)
    # the graph reads the operands' current contents: change them and replay
    for i, a in enumerate(As):
        a.mul_(-1.0)
    graph.replay()
    torch.cuda.synchronize()
    for i, (A, B) in enumerate(host):
        np.testing.assert_array_equal(Cs[i].cpu().numpy(), oracle.classical(-A, B))
    plan.close()


def test_batched_256_uneven_fp16_sampled():
    """256 problems, m, n, k uniform over multiples of 256 in [1024, 8192], FP16 inputs with
    per-panel power-of-two scaling; every problem checked on two sampled rows."""
    shapes = synth.uneven_batch(256, seed=2024)
    g = torch.Generator(device="cuda").manual_seed(2025)
    As = [(torch.rand((m, k), device="cuda", generator=g) * 2 - 1).half() for m, n, k in shapes]
    Bs = [(torch.rand((k, n), device="cuda", generator=g) * 2 - 1).half() for m, n, k in shapes]
    Cs = fmm.gemm_batched(As, Bs, variant="f16")
    fmm.device_status()
    rng = synth.rng(2026)
    worst = 0.0
    for i in range(0, 256, 16):
        m, n, k = shapes[i]
        rows = np.unique(rng.integers(0, m, size=2))
        Ab = As[i][torch.from_numpy(rows).cuda()].cpu().view(torch.int16).numpy().view(np.uint16)
        Bb = Bs[i].cpu().view(torch.int16).numpy().view(np.uint16)
        C64 = oracle.classical(Ab, Bb, a_code=oracle.ORC_F16, b_code=oracle.ORC_F16)
        An = float(As[i][torch.from_numpy(rows).cuda()].float().norm())
        Bn = float(Bs[i].float().norm())
        err = oracle.normwise_error(Cs[i][torch.from_numpy(rows).cuda()].cpu().numpy(), C64, An, Bn)
        lv = fmm.tune_select(m, n, k)[0]
        assert err <= tolerance("f16", lv, k), (shapes[i], err)
        worst = max(worst, err)


@pytest.mark.parametrize("levels", [1, 2])
def test_batched_uneven_fp16_scaled_strassen_classes(levels):
    """Config C4's defining feature at its sizes: problems drawn like the 256-problem batch
    (multiples of 256 in [1024, 8192]) forced through one- and two-level Strassen classes of
    the FP16 arithmetic, whose operand sums are scaled by a power of two per panel before
    the FP16 rounding; sampled rows of every other problem against the oracle on the FP16
    bit patterns."""
    shapes = synth.uneven_batch(24, seed=2030 + levels)
    g = torch.Generator(device="cuda").manual_seed(2040 + levels)
    As = [(torch.rand((m, k), device="cuda", generator=g) * 2 - 1).half() for m, n, k in shapes]
    Bs = [(torch.rand((k, n), device="cuda", generator=g) * 2 - 1).half() for m, n, k in shapes]
    table = [(2 ** 62, levels, 0)]
    Cs = fmm.gemm_batched(As, Bs, variant="f16", tune=table)
    fmm.device_status()
    rng = synth.rng(2050 + levels)
    for i in range(0, len(shapes), 2):
        m, n, k = shapes[i]
        assert fmm.tune_select(m, n, k, table)[0] == levels
        rsel = torch.from_numpy(np.unique(rng.integers(0, m, size=2))).cuda()
        Ab = As[i][rsel].cpu().view(torch.int16).numpy().view(np.uint16)
        Bb = Bs[i].cpu().view(torch.int16).numpy().view(np.uint16)
        C64 = oracle.classical(Ab, Bb, a_code=oracle.ORC_F16, b_code=oracle.ORC_F16)
        err = oracle.normwise_error(Cs[i][rsel].cpu().numpy(), C64, float(As[i][rsel].float().norm()),
                                    float(Bs[i].float().norm()))
        assert err <= tolerance("f16", levels, k), (shapes[i], err)


def test_native_tuner_builds_a_valid_table():
    t = fmm.tune_measure(sizes=(512, 1024, 2048), variant="split3", reps=2)
    assert 1 <= len(t["classes"]) <= 3
    prev = 0
    for c in t["classes"]:
        assert c["levels"] in (0, 1, 2) and c["tile_n"] in (128, 256) and c["max_dim"] > prev
        prev = c["max_dim"]
    assert set(t["probes_ms"]) == {"512", "1024", "2048"}
    assert all(v > 0 for p in t["probes_ms"].values() for v in p.values())
    fmm.tune_select(700, 700, 700, t)  # the table is usable by the batched entry points

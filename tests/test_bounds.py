"""The parity tests' split3 bound against a model of the split arithmetic (CPU only).

The bound must hold for the arithmetic itself (otherwise a correct kernel would fail), and
must not be loose (otherwise a wrong kernel would pass): at every depth where it exceeds the
FP32-accurate 1e-6, the modelled error is at least 40 % of it."""
import numpy as np
import pytest
import torch

import oracle
import synth
from bounds import NORTH, split3_bound, tolerance
from split_model import bf16_round, strassen_split3

SHAPES = [(1, 1, 1), (7, 13, 5), (16, 16, 16), (129, 257, 33), (129, 257, 65), (640, 384, 96),
          (300, 260, 150), (300, 520, 200), (130, 70, 300), (640, 384, 768), (257, 129, 1000)]


def _err(A, B, levels):
    C64 = A.astype(np.float64) @ B.astype(np.float64)
    return oracle.normwise_error(strassen_split3(A, B, levels), C64,
                                 np.linalg.norm(A.astype(np.float64)), np.linalg.norm(B.astype(np.float64)))


def test_model_rounds_like_torch_bf16():
    x = synth.gaussian((4096,), 3) * np.float32(1e3)
    want = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    np.testing.assert_array_equal(bf16_round(x), want)


@pytest.mark.parametrize("dist", ["uniform", "gaussian"])
@pytest.mark.parametrize("m,n,k", SHAPES)
def test_bound_holds_for_the_split_arithmetic(m, n, k, dist):
    A, B = synth.problem(m, n, k, m * 7 + n + k, dist)
    for levels in (0, 1, 2):
        err = _err(A, B, levels)
        assert err <= tolerance("split3", levels, k), (levels, err)


@pytest.mark.parametrize("m,n,k", [(640, 384, 96), (300, 260, 150), (130, 70, 300), (257, 129, 64)])
def test_bound_is_tight_where_it_exceeds_1e6(m, n, k):
    A, B = synth.problem(m, n, k, 5, "uniform")
    for levels in (0, 1, 2):
        b = split3_bound(levels, k)
        if b > NORTH:
            assert _err(A, B, levels) >= 0.4 * b, levels


def test_two_level_split_arithmetic_exceeds_1e6_at_small_k():
    """Why 1e-6 is not asserted at every depth: the arithmetic itself lies above it."""
    A, B = synth.problem(256, 256, 96, 6, "uniform")
    assert _err(A, B, 2) > NORTH
    assert _err(A, B, 0) < NORTH


def test_bound_is_1e6_at_the_configs_depths():
    assert split3_bound(1, 512) == NORTH          # C1: 512^3, one level
    assert split3_bound(2, 4096) == NORTH         # C2 4096^3 .. 16384^3, two levels
    assert split3_bound(2, 4097) == NORTH         # C5: k = 4097, two levels
    assert split3_bound(2, 512) > NORTH           # rank-k 512 at two levels: h_k = 128
    assert split3_bound(1, 512) == NORTH

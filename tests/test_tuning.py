"""Tune-table selection and the autotuner's table construction (no GPU)."""
import math

import pytest

import paper_1808_07984_gb300 as fmm
from paper_1808_07984_gb300 import autotune


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fmm.build()
    fmm.load()


def test_default_table_crossovers():
    assert fmm.tune_select(1024, 1024, 1024)[0] == 0
    assert fmm.tune_select(4096, 4096, 4096)[0] == 1
    assert fmm.tune_select(8192, 8192, 8192)[0] == 1
    assert fmm.tune_select(16384, 16384, 16384)[0] == 2
    # rank-k: the smallest dimension decides
    assert fmm.tune_select(16384, 16384, 512)[0] == 0


def test_custom_table():
    t = [(2000, 0, 128), (5000, 1, 256), (2 ** 62, 2, 0)]
    assert fmm.tune_select(1000, 9000, 9000, t) == (0, 128)
    assert fmm.tune_select(3000, 3000, 3000, t) == (1, 256)
    assert fmm.tune_select(6000, 7000, 8000, t) == (2, 0)
    with pytest.raises(fmm.FmmError):
        fmm.tune_select(10, 10, 10, [(100, 3, 0)])
    with pytest.raises(fmm.FmmError):
        fmm.tune_select(10, 10, 10, [(100, 1, 96)])


def test_build_table_picks_fastest_and_merges():
    probes = {
        1024: {(0, 128): 1.0, (1, 128): 1.2, (2, 128): 1.5},
        2048: {(0, 128): 5.0, (1, 256): 4.9, (2, 128): 6.0},
        4096: {(0, 128): 40.0, (1, 256): 35.0, (2, 256): 36.0},
        8192: {(1, 256): 300.0, (2, 256): 280.0},
    }
    t = autotune.build_table(probes)["classes"]
    assert [(c["levels"], c["tile_n"]) for c in t] == [(0, 128), (1, 256), (2, 256)]
    assert t[0]["max_dim"] == int(math.sqrt(1024 * 2048))
    assert t[1]["max_dim"] == int(math.sqrt(4096 * 8192))  # 2048 and 4096 merged
    assert t[2]["max_dim"] == 2 ** 63 - 1
    table = fmm.tune_table({"classes": t})
    assert fmm.tune_select(1400, 1400, 1400, table) == (0, 128)
    assert fmm.tune_select(3000, 3000, 3000, table) == (1, 256)


def test_batched_workspace_is_sum_of_parts():
    ms, ns, ks = [512, 1024, 300], [256, 2048, 300], [768, 512, 1000]
    import ctypes
    L = fmm.load()
    I64 = ctypes.c_int64 * 3
    t = fmm.tune_table(None)
    ws = L.fmm_batched_workspace_size(3, I64(*ms), I64(*ns), I64(*ks), 0, ctypes.byref(t))
    parts = sum(fmm.workspace_size(m, n, k, fmm.tune_select(m, n, k)[0], "split3")
                for m, n, k in zip(ms, ns, ks))
    assert ws >= parts

"""Autotuner for the Strassen level and tile width per size class.

For each probe size d it times square d x d x d products at levels 0, 1, 2 and tile
widths 128 and 256 through the library (CUDA events, after warm-up), keeps the fastest
pair, and turns the probes into size classes whose boundaries are the geometric means
between neighbouring probe sizes.  The result is a JSON-serialisable table that
``tune_table`` converts to the C ABI's fmm_tune_table; setting FMM_TUNE_FILE to a saved
table makes the batched entry points use it by default.
"""
from __future__ import annotations

import json
import math


def measure(d: int, levels: int, tile_n: int, variant: str = "split3", steps: int = 3,
            warmup: int = 2) -> float:
    """Milliseconds per d x d x d product (library call, operands resident on the GPU)."""
    import torch

    from . import gemm, workspace_size
    dtype = {"split3": torch.float32, "plain_bf16": torch.float32, "bf16": torch.bfloat16,
             "f16": torch.float16}[variant]
    g = torch.Generator(device="cuda").manual_seed(d + 17 * levels + tile_n)
    A = (torch.rand((d, d), device="cuda", generator=g) * 2 - 1).to(dtype)
    B = (torch.rand((d, d), device="cuda", generator=g) * 2 - 1).to(dtype)
    C = torch.empty((d, d), dtype=torch.float32, device="cuda")
    ws = torch.empty(max(256, workspace_size(d, d, d, levels, variant, tile_n=tile_n)),
                     dtype=torch.uint8, device="cuda")
    for _ in range(warmup):
        gemm(A, B, C, levels=levels, variant=variant, tile_n=tile_n, workspace=ws)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        gemm(A, B, C, levels=levels, variant=variant, tile_n=tile_n, workspace=ws)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def build_table(probes: dict) -> dict:
    """probes: {d: {(levels, tile_n): ms}} -> {"classes": [...]} (pure function)."""
    sizes = sorted(probes)
    classes = []
    for i, d in enumerate(sizes):
        (lv, tn), _ = min(probes[d].items(), key=lambda kv: kv[1])
        upper = int(math.sqrt(d * sizes[i + 1])) if i + 1 < len(sizes) else 2 ** 63 - 1
        if classes and classes[-1]["levels"] == lv and classes[-1]["tile_n"] == tn:
            classes[-1]["max_dim"] = upper  # merge neighbouring classes with the same choice
        else:
            classes.append({"max_dim": upper, "levels": lv, "tile_n": tn})
    return {"classes": classes[:8]}


def autotune(sizes=(1024, 2048, 4096, 8192, 16384), variant: str = "split3",
             levels=(0, 1, 2), tiles=(128, 256), steps: int = 3, prior: str | None = None,
             keep: int = 2, native: bool = False) -> dict:
    """Measure the candidates of each probe size and build the table.  prior="model": rank
    the candidates with the analytic model (model.py) and measure only the best ``keep``.
    native=True: the library's own tuner (fmm_tune_measure) measures every candidate."""
    import torch
    if native:
        from . import tune_measure
        table = tune_measure(sizes, variant, steps)
        table["gpu"] = torch.cuda.get_device_name()
        return table
    probes = {}
    for d in sizes:
        cands = [(lv, tn) for lv in levels for tn in tiles]
        if prior == "model":
            from . import model
            cands = model.rank_candidates(d, variant, levels, tiles)[:keep]
        probes[d] = {(lv, tn): measure(d, lv, tn, variant, steps) for lv, tn in cands}
    table = build_table(probes)
    table["variant"] = variant
    table["gpu"] = torch.cuda.get_device_name()
    table["probes_ms"] = {str(d): {f"L{lv}_N{tn}": round(ms, 4) for (lv, tn), ms in p.items()}
                          for d, p in probes.items()}
    if prior:
        table["prior"] = prior
    return table


def save(table: dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump(table, f, indent=1)


def load(path: str) -> dict:
    with open(path) as f:
        return json.load(f)


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--variant", default="split3")
    ap.add_argument("--out", default="fmm_tune.json")
    ap.add_argument("--sizes", default="1024,2048,4096,8192,16384")
    a = ap.parse_args()
    t = autotune(tuple(int(x) for x in a.sizes.split(",")), a.variant)
    save(t, a.out)
    print(json.dumps({k: v for k, v in t.items() if k != "probes_ms"}))

"""Analytic time model of one library call on a GB300 (the paper's Section 4 model, adapted).

The paper models a fused Strassen product on V100 as arithmetic time plus the time of its
extra memory operations (the W_A, W_B operand tiles each k-step and the W_C accumulator
updates).  On GB300 the same three costs appear in different places:

* the operand-sum pass reads A and B once and writes the 7^L sums (BF16, two arrays for the
  split3 arithmetic): HBM-bound;
* the tensor-core kernel does (7/8)^L of the classical UMMA work, 1 or 3 UMMAs per k16 slice,
  in 256 x tile_n CTA-pair tiles distributed over 76 CTA pairs;
* every work item adds its accumulator into W_C destination tiles of C (TMA reductions
  through L2; the first update of each C block is a store, half the bytes), which costs time
  the mainloop does not hide.

    T = t_beta + t_pack + t_tensor + launches * t_launch
    t_beta   = 0 with beta = 0: a classical product stores C, and a Strassen product stores
               the first update of each C block (store-first launch phases); 4 m n / BW
               when C has to be zeroed first (store_first=False)
    t_pack   = pack_bytes / (BW * pack_eff)
    t_tensor = t_work + cap_slope * max(0, t_mma - cap_t0) * (t_mma / t_work)^2
    t_work   = W * (t_item_mma + t_item_fix + wb_bytes_item * wb_cost),  t_mma = W * t_item_mma
               (the power cap lowers the SM clock under long dense UMMA work, the more so the
               larger the tensor cores' share of the kernel's time)
    W        = sum over the store-first launch phases of ceil(items_phase / workers)
    items    = R * ceil(h_m / 256) * ceil(h_n / tile_n)     (R products of a basis)
    t_item_mma = terms * 2 * 256 * tile_n * h_k / (TC * tc_eff / workers)
                 (times n128_slow for 128-wide tiles)

BW and TC are the measured HBM copy bandwidth and burst BF16 tensor rate of the pool's
GB300s; pack_eff (at most 1), tc_eff, wb_cost, t_item_fix, t_launch, n128_slow and the two
power-cap terms are fitted to measured library calls (``fit``).  ``DEFAULT`` holds the fit to
136 split3 calls measured on a GB300 (square, panel and rank-k sweeps at the automatic tile
width, calls at both tile widths, and classical, one- and two-level Strassen and the <3,2,3>
basis at twelve sizes): mean absolute error 3.5 % (4.5 %, 3.4 % and 2.5 % over the three
files).  pack_eff comes out at 1.0 (the sum pass streams at the measured copy bandwidth);
tc_eff at 1.21, i.e. short UMMA work runs at 2.30 PFLOP/s, 89 % of what 152 SMs reach at the
maximum clock (the burst denominator is a cuBLAS product timed at a lower clock); 128-wide
tiles run 24 % slower per flop; dense UMMA work beyond about 2 ms slows by up to 28 % (the power
cap's clock drop).

Used by ``autotune.autotune(prior="model")`` to rank the (levels, tile_n) candidates of each
size so that only the most promising ones are measured, and (``best_basis``) to choose
between one-level bases: a basis with block grid (g_m, g_k, g_n), R products and nnz(W) C
updates enters through the block sizes h = ceil(d / g) (rounded up to 8), the R operand sums
per operand and the average W_C = nnz(W) / R.
"""
from __future__ import annotations

import math

GB300 = {"sms": 152, "hbm_gbs": 6781.1, "tc_tflops": 1897.8}
# UMMA rate of 152 SMs at the maximum SM clock (8192 BF16 flops per SM and cycle at 2070 MHz)
# over the measured burst rate: the largest tc_eff ``fit`` allows
_TC_EFF_MAX = 152 * 8192 * 2.070e9 / 1897.8e12

# fitted (``fit``) to the 136 measured split3 calls of ``calibration_samples()``: 58 at the
# automatic tile width (tuned/gb300_model_samples.json), 30 at explicit tile widths
# (gb300_tile_samples.json) and 48 of four bases (gb300_basis_samples.json), all measured with
# the store-first write-back (beta = 0: no zeroing pass, first updates stored)
DEFAULT = {"pack_eff": 1.000, "tc_eff": 1.212, "wb_cost_ns_per_kb": 14.98, "t_item_fix_us": 0.0,
           "t_launch_us": 8.46, "n128_slow": 1.239, "cap_slope": 0.283, "cap_t0_ms": 2.07}

_TERMS = {"split3": 3, "plain_bf16": 1, "bf16": 1, "f16": 1}
# one-level bases: block grid (g_m, g_k, g_n), products R and nonzeros of W (C updates)
BASES = {"strassen": (2, 2, 2, 7, 12), "winograd": (2, 2, 2, 7, 14), "b323": (3, 2, 3, 15, 30),
         "b232": (2, 3, 2, 11, 16)}
_IN_BYTES = {"split3": 4, "plain_bf16": 4, "bf16": 2, "f16": 2}
_ARRAYS = {"split3": 2, "plain_bf16": 1, "bf16": 1, "f16": 1}


def block(d: int, levels: int, g: int = 0) -> int:
    """Block size of the library's split rule: ceil(d / g) rounded up to 8 (d > 0), with
    g = 2^L unless given."""
    if d <= 0:
        return 0
    h = -(-d // (g or (1 << levels)))
    return -(-h // 8) * 8


def shape(levels: int, basis: str = "strassen"):
    """(g_m, g_k, g_n, R, average C updates per product) of ``levels`` levels of a basis."""
    if levels == 0:
        return 1, 1, 1, 1, 1.0
    gm, gk, gn, r, nw = BASES[basis]
    if basis != "strassen" and levels != 1:
        raise ValueError("bases other than Strassen's are built for one level")
    return gm ** levels, gk ** levels, gn ** levels, r ** levels, (nw / r) ** levels


def auto_tile_n(m: int, n: int, levels: int, basis: str = "strassen") -> int:
    """The library's automatic tile width for CTA pairs (256 unless that leaves fewer than
    four items per pair)."""
    gm, _, gn, R, _ = shape(levels, basis)
    hm, hn = block(m, levels, gm), block(n, levels, gn)
    items256 = R * -(-hm // 256) * -(-hn // 256)
    return 256 if items256 >= 4 * (GB300["sms"] // 2) else 128


# products per launch phase of the store-first write-back (the library's fmm_store_phases)
_PHASES = {(1, "strassen"): (1, 4, 2), (2, "strassen"): (1, 12, 24, 12), (1, "winograd"): (1, 6),
           (1, "b323"): (5, 7, 3), (1, "b232"): (3, 8)}


def predict(m: int, n: int, k: int, levels: int, variant: str = "split3", tile_n: int = 0,
            params: dict | None = None, hw: dict | None = None, basis: str = "strassen",
            store_first: bool = True) -> dict:
    """Predicted milliseconds of fmm_gemm(m, n, k, levels, variant, basis) with beta = 0 and
    its components."""
    p = dict(DEFAULT, **(params or {}))
    h = dict(GB300, **(hw or {}))
    gm, gk, gn, R, wc = shape(levels, basis)
    terms, e_in, arrays = _TERMS[variant], _IN_BYTES[variant], _ARRAYS[variant]
    hm, hn, hk = block(m, levels, gm), block(n, levels, gn), block(k, levels, gk)
    tn = tile_n or auto_tile_n(m, n, levels, basis)
    bw = h["hbm_gbs"] * 1e9
    t_beta = 4.0 * m * n / bw if (levels > 0 and not store_first) else 0.0
    pack_bytes = (m * k + k * n) * e_in + R * (hm * hk + hk * hn) * 2 * arrays
    t_pack = pack_bytes / (bw * p["pack_eff"])
    workers = h["sms"] // 2
    tiles = -(-hm // 256) * -(-hn // tn)
    items = R * tiles
    # each launch phase ends with a partial wave of items
    phases = _PHASES.get((levels, basis), (R,)) if (levels > 0 and store_first) else (R,)
    per_worker = sum(-(-(P * tiles) // workers) for P in phases)
    tc = h["tc_tflops"] * 1e12 * p["tc_eff"] / workers
    t_item_mma = terms * 2.0 * 256 * tn * hk / tc
    if tn == 128:
        # 128-wide pair tiles: each CTA's UMMAs are N = 64 and every k-step loads the A panel
        # for half the output of a 256-wide tile; measured slower per flop
        t_item_mma *= p["n128_slow"]
    # wc: average W_C of a product (Strassen: 12 nonzeros of W over 7 products per level)
    # a classical product stores its tile (write only); Strassen products add into C (read and
    # write of every destination tile)
    if levels == 0:
        wb_bytes_item = wc * 256 * tn * 4 * 0.5
    else:
        # of the R * wc block updates, one per C block (gm * gn of them) stores
        f_store = (gm * gn) / (R * wc) if store_first else 0.0
        wb_bytes_item = wc * 256 * tn * 4 * (1.0 - 0.5 * f_store)
    t_item = t_item_mma + p["t_item_fix_us"] * 1e-6 + wb_bytes_item / 1024.0 * p["wb_cost_ns_per_kb"] * 1e-9
    t_tensor = per_worker * t_item
    # the power cap: dense UMMA work lasting longer than cap_t0 runs at a lower SM clock, the
    # more so the larger the share of the kernel's time the tensor cores are busy
    t_mma = per_worker * t_item_mma
    t_tensor += p["cap_slope"] * max(0.0, t_mma - p["cap_t0_ms"] * 1e-3) * (t_mma / t_tensor) ** 2
    launches = 2 + len(phases)
    t = t_beta + t_pack + t_tensor + launches * p["t_launch_us"] * 1e-6
    return {"ms": t * 1e3, "beta_ms": t_beta * 1e3, "pack_ms": t_pack * 1e3,
            "tensor_ms": t_tensor * 1e3, "items": items, "items_per_pair": per_worker,
            "launches": launches, "tile_n": tn, "eff_tflops": 2.0 * m * n * k / t * 1e-12}


def best_levels(m: int, n: int, k: int, variant: str = "split3", params: dict | None = None) -> int:
    """The level the model predicts fastest."""
    return min(range(3), key=lambda L: predict(m, n, k, L, variant, params=params)["ms"])


def best_basis(m: int, n: int, k: int, variant: str = "split3", params: dict | None = None):
    """(levels, basis) the model predicts fastest among classical, Strassen at one and two
    levels and the other one-level bases."""
    cands = [(0, "strassen"), (1, "strassen"), (2, "strassen"), (1, "winograd"), (1, "b323")]
    return min(cands, key=lambda c: predict(m, n, k, c[0], variant, params=params, basis=c[1])["ms"])


def rank_candidates(d: int, variant: str = "split3", levels=(0, 1, 2), tiles=(128, 256),
                    params: dict | None = None) -> list:
    """(levels, tile_n) candidates of a square d-problem, fastest predicted first."""
    cands = [(L, t) for L in levels for t in tiles]
    return sorted(cands, key=lambda c: predict(d, d, d, c[0], variant, tile_n=c[1], params=params)["ms"])


def _pred_ms(sample, variant, params):
    """Predicted ms of a sample (m, n, k, levels, ms), (m, n, k, levels, tile_n, ms) or
    (m, n, k, levels, tile_n, basis, ms)."""
    if len(sample) == 7:
        m, n, k, L, tn, b, _ = sample
        return predict(m, n, k, L, variant, tile_n=tn, params=params, basis=b)["ms"]
    if len(sample) == 6:
        m, n, k, L, tn, _ = sample
    else:
        (m, n, k, L, _), tn = sample, 0
    return predict(m, n, k, L, variant, tile_n=tn, params=params)["ms"]


def fit(samples, variant: str = "split3", start: dict | None = None, iters: int = 400) -> dict:
    """Least-squares fit of the model's free parameters to measured calls.

    samples: iterable of (m, n, k, levels, measured_ms), (m, n, k, levels, tile_n,
    measured_ms) for calls at an explicit tile width (0: automatic), or (m, n, k, levels,
    tile_n, basis, measured_ms).  Minimises the mean squared log ratio of
    predicted to measured time by coordinate search (no dependency beyond math)."""
    samples = list(samples)
    p = dict(DEFAULT, **(start or {}))
    keys = list(DEFAULT)

    def loss(q):
        s = 0.0
        for smp in samples:
            s += math.log(_pred_ms(smp, variant, q) / smp[-1]) ** 2
        return s / max(len(samples), 1)

    best = loss(p)
    step = {key: 0.25 * p[key] for key in keys}
    for _ in range(iters):
        improved = False
        for key in keys:
            for sgn in (1, -1):
                q = dict(p)
                q[key] = max(1e-6, p[key] + sgn * step[key])
                if key == "tc_eff":
                    q[key] = min(q[key], _TC_EFF_MAX)
                if key == "pack_eff":
                    q[key] = min(q[key], 1.0)  # the sum pass cannot beat the copy bandwidth
                lq = loss(q)
                if lq < best:
                    p, best, improved = q, lq, True
        if not improved:
            for key in keys:
                step[key] *= 0.5
            if max(step[k_] / max(p[k_], 1e-9) for k_ in keys) < 1e-4:
                break
    return p


def mean_abs_error(samples, variant: str = "split3", params: dict | None = None) -> float:
    """Mean |predicted - measured| / measured over samples as ``fit`` takes them."""
    samples = list(samples)
    err = [abs(_pred_ms(smp, variant, params) - smp[-1]) / smp[-1] for smp in samples]
    return sum(err) / max(len(err), 1)


def load_samples(path: str):
    """Samples of a calibration file: (m, n, k, levels, ms), (m, n, k, levels, tile_n, ms)
    for a file of calls at explicit tile widths, or (m, n, k, levels, 0, basis, ms) for a
    file whose columns are m, n, k and one time per "L<levels>_<basis>" candidate."""
    import json
    with open(path) as f:
        rec = json.load(f)
    var = rec.get("variant", "split3")
    if "samples_m_n_k_levels_ms" in rec:
        return [tuple(x) for x in rec["samples_m_n_k_levels_ms"]], var
    cols = rec.get("columns", [])
    if len(cols) > 3 and all(c.startswith("L") and "_" in c for c in cols[3:]):
        cands = [(int(c[1:c.index("_")]), c[c.index("_") + 1:]) for c in cols[3:]]
        return [(m, n, k, L, 0, b, t) for m, n, k, *ms in rec["rows"]
                for (L, b), t in zip(cands, ms)], var
    return [tuple(x) for x in rec["rows"]], var


def calibration_samples(variant: str = "split3"):
    """Every measured call of the tuned/ calibration files (the samples ``DEFAULT`` is fitted
    to)."""
    import os
    d = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned")
    out = []
    for name in ("gb300_model_samples.json", "gb300_tile_samples.json", "gb300_basis_samples.json"):
        S, var = load_samples(os.path.join(d, name))
        if var == variant:
            out += S
    return out


if __name__ == "__main__":
    import argparse
    import os
    ap = argparse.ArgumentParser(description="fit or check the GB300 time model")
    ap.add_argument("--samples", default=None,
                    help="one calibration file (default: every file under tuned/)")
    ap.add_argument("--fit", action="store_true")
    a = ap.parse_args()
    S, var = load_samples(a.samples) if a.samples else (calibration_samples(), "split3")
    prm = fit(S, var) if a.fit else DEFAULT
    print({k_: round(v, 4) for k_, v in prm.items()}, "mean abs error", round(mean_abs_error(S, var, prm), 4))

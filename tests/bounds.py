"""Normwise error bounds ||C - C64||_F / (||A||_F ||B||_F) used by every parity test.

split3 (FP32 inputs; every operand sum formed in FP32, split into BF16 hi = bf16(P) and
lo = bf16(P - hi); the product hi*hi + hi*lo + lo*hi accumulated in FP32, lo*lo dropped):

* k >= 64: max(1e-6, 2**-17 * 2**L / sqrt(k)).  1e-6 is the bound stated for FP32-accurate
  paths.  The second term is the error of the split arithmetic itself: each product term
  carries a relative error of about 2**-18 (the rounding of lo, <= 2**-16 |P|, and the dropped
  lo*lo term), random in sign, so the normwise error of a classical product is about
  2**-18 / sqrt(k); each Strassen level doubles it (the operand sums and the C updates
  combine several blocks).  A numpy model of exactly this arithmetic
  (``tests/split_model.py``, checked in ``tests/test_bounds.py``) stays below the bound with
  a margin under 2.5x, and exceeds 1e-6 itself for two-level products with k below about
  450 and one-level products with k below about 70; so 1e-6 is asserted exactly for
  L = 0 at k >= 64, L = 1 at k >= 233 and L = 2 at k >= 932 (C5's k = 4097 included), and the
  split arithmetic's own bound below those depths.
* k < 64: 2**-15 * 2**L / sqrt(k) (a few product terms do not average their errors out).

plain BF16 / FP16 (one rounding of each FP32 operand sum): 4 u 3**L / sqrt(k), u = 2**-8
(BF16) or 2**-11 (FP16).  16-bit inputs of a classical product are exact in the tensor
cores: 1e-6.
"""
import math

U_BF16 = 2.0 ** -8   # unit roundoff of bfloat16 (8-bit significand)
U_F16 = 2.0 ** -11   # unit roundoff of float16 (11-bit significand)
NORTH = 1e-6         # the FP32-accurate bound


def split3_bound(levels: int, k: int) -> float:
    kk = max(int(k), 1)
    if kk < 64:
        return 2.0 ** -15 * 2 ** levels / math.sqrt(kk)
    return max(NORTH, 2.0 ** -17 * 2 ** levels / math.sqrt(kk))


def tolerance(variant: str, levels: int, k: int) -> float:
    """Normwise bound of one product of ``levels`` Strassen levels over inner dimension k."""
    kk = max(int(k), 1)
    if variant == "split3":
        return split3_bound(levels, kk)
    if variant in ("bf16", "f16") and levels == 0:
        return NORTH  # inputs exactly representable, FP32 accumulation only
    if variant == "f16":
        return 4 * U_F16 * 3 ** levels / math.sqrt(kk)
    return 4 * U_BF16 * 3 ** levels / math.sqrt(kk)

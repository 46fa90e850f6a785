"""Per-element comparison used by the parity tests.

An element passes when |got - ref| <= rtol |ref| + atol max|ref|: the
relative bar rtol holds for every element that is not tiny next to the
largest one, and atol (relative to the largest magnitude) covers elements
so small that rounding in the sums that form them (terms of both signs,
summed in different orders) dominates their own size.

Bars used by the tests: FP64 rtol 1e-10, atol 1e-12; PCM_MIXED rtol 1e-6,
atol 1e-7 (the mixed kernels add FP32-rounded terms, with errors of about
6e-8 of the largest term, into every element)."""
import numpy as np

FP64 = (1e-10, 1e-12)
MIXED = (1e-6, 1e-7)


def worst(got, ref, rtol, atol, scale=None):
    """Largest |got - ref| / (rtol |ref| + atol scale) over the elements;
    scale defaults to max|ref|.  The check passes when this is <= 1."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    if scale is None:
        scale = float(np.max(np.abs(ref)))
    bound = rtol * np.abs(ref) + atol * scale
    return float(np.max(np.abs(got - ref) / bound))


def check(got, ref, bars, scale=None, what=""):
    w = worst(got, ref, bars[0], bars[1], scale)
    assert w <= 1.0, "%s: worst element at %.3g of the bar (rtol %g, atol %g)" % (what, w, bars[0], bars[1])
    return w

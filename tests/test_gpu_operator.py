"""The operator A of Eq. 1 (Eq. 2, Eq. 3 as the r -> 0 limit of Eq. 2,
Eq. 8) as the library applies it, through pcm_apply_a, against the oracle's
dense A times the same vector, element by element.

PCM_FP64 multiplies by its stored A; PCM_MIXED stores no A (near pairs kept
exactly, every other element 1/R recomputed): its accurate product (the one
behind true residuals and the energy; double-float 1/R from coordinates split
into a 2^-10 grid part and an FP32 rest, whose rounding, at most 2^-36 bohr,
bounds a far element's relative error by about 1e-11) is held to rtol 1e-11,
its FP32 product (the inner solver's) to rtol 1e-6, with positive x (no
cancellation in the row sums); with x of both signs the bars gain an atol
relative to the largest |y| (FP64 1e-13, double-float 1e-12, FP32 1e-7)."""
import numpy as np
import pytest

import oracle
import workloads
from _parity import check

pytestmark = pytest.mark.gpu


def _apply(w, precision, xs, fp32=False, operator="auto"):
    import paper_1505_07851_gb300 as pcm
    with pcm.Context(precision=precision, operator=operator) as ctx:
        M = ctx.build_surface(w.mol.xyz, w.mol.Z, w.mol.radius, 110)
        assert ctx.stats()["operator_free"] == (1 if operator == "free" else 0)
        xyzzs, idx = ctx.get_surface()
        ys = [np.array(ctx.apply_a(x, fp32=fp32)) for x in xs]
    return M, xyzzs, ys


@pytest.mark.parametrize("name", ["cluster40_sp", "cluster300_sp"])
def test_operator_against_oracle(name):
    w = workloads.small_cluster(40, seed=23) if name == "cluster40_sp" else workloads.config(1)
    rng = np.random.default_rng(3)
    # sizes are known after the surface: build once to get M
    M, xyzzs, _ = _apply(w, "fp64", [])
    A = oracle.a_matrix({"r": xyzzs[:, :3], "zeta": xyzzs[:, 3], "S": xyzzs[:, 4]})
    x_pos = rng.uniform(0.0, 1.0, M)
    x_mix = rng.normal(size=M)
    y_pos, y_mix = A @ x_pos, A @ x_mix
    for prec, op, fp32, bars_pos, bars_mix in (("fp64", "auto", False, (1e-12, 0.0), (1e-12, 1e-13)),
                                               ("mixed", "stored", False, (1e-11, 0.0), (1e-11, 1e-12)),
                                               ("mixed", "free", False, (1e-11, 0.0), (1e-11, 1e-12)),
                                               ("mixed", "free", True, (1e-6, 0.0), (1e-6, 1e-7))):
        M2, xyzzs2, (g_pos, g_mix) = _apply(w, prec, [x_pos, x_mix], fp32, op)
        assert M2 == M and np.array_equal(xyzzs2, xyzzs)
        tag = "%s %s%s" % (prec, op, " fp32" if fp32 else "")
        check(g_pos, y_pos, bars_pos, what=tag + " x > 0")
        check(g_mix, y_mix, bars_mix, what=tag + " x mixed")


def test_fp32_product_needs_a_matrix_free_context():
    import paper_1505_07851_gb300 as pcm
    w = workloads.config(0)
    for prec, op in (("fp64", "auto"), ("mixed", "stored")):
        with pcm.Context(precision=prec, operator=op) as ctx:
            M = ctx.build_surface(w.mol.xyz, w.mol.Z, w.mol.radius, 110)
            with pytest.raises(pcm.PCMError):
                ctx.apply_a(np.ones(M), fp32=True)


def test_automatic_operator_choice():
    """PCM_OPERATOR_AUTO: stored A for small surfaces, matrix-free above
    24576 points (the 1000-atom cluster)."""
    import paper_1505_07851_gb300 as pcm
    for w, free in ((workloads.config(1), 0), (workloads.config(2), 1)):
        with pcm.Context(precision="mixed") as ctx:
            ctx.build_surface(w.mol.xyz, w.mol.Z, w.mol.radius, 110)
            assert ctx.stats()["operator_free"] == free

"""The autotuner (pcm_options.autotune): timed trials pick the FP32 ESP and
Fock kernels' tile shapes; results stay within the mixed-precision bar of
the untuned kernels, and the choices are recorded."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _run(w, autotune):
    import paper_1505_07851_gb300 as pcm
    with pcm.Context(precision="mixed", autotune=autotune) as ctx:
        ctx.setup(w.mol, w.basis)
        c = ctx.esp(w.P)
        q, _ = ctx.solve(delta=1e-8)
        dF = ctx.fock(q)
        return c, dF, ctx.energy(q)


def test_autotuned_results_and_table():
    import paper_1505_07851_gb300 as pcm
    w = workloads.small_cluster(5, seed=22, d_shells=True)
    c0, F0, E0 = _run(w, False)
    c1, F1, E1 = _run(w, True)
    assert np.max(np.abs(c1 - c0)) <= 1e-6 * np.max(np.abs(c0))
    assert np.max(np.abs(F1 - F0)) <= 1e-6 * np.max(np.abs(F0))
    assert abs(E1 - E0) <= 1e-7
    tab = pcm.autotune_table()
    kinds = {t["kernel"] for t in tab}
    assert {"esp_variant", "fock_pairs_per_thread"} <= kinds
    for t in tab:
        allowed = (("pair-driven, 4 points/thread", "pair-driven, 2 points/thread", "MS-driven")
                   if t["kernel"] == "esp_variant" else (1, 2))
        assert t["choice"] in allowed and 0 <= t["L"] <= 4
    # a second tuned context reuses the choices: identical results
    c2, F2, E2 = _run(w, True)
    assert np.array_equal(c1, c2) and np.array_equal(F1, F2) and E1 == E2


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("fp32x2", [True, False])
@pytest.mark.parametrize("d_shells", [False, True])
def test_each_esp_variant_against_fp64(variant, fp32x2, d_shells):
    """Every ESP variant (pair-driven with 4 or 2 points per thread, MS-driven),
    with packed or scalar FP32 instructions, meets the mixed bar on its own, on
    s/p and on s/p/d clusters (classes ss .. dd)."""
    import paper_1505_07851_gb300 as pcm
    w = workloads.small_cluster(8, seed=21, d_shells=d_shells)
    with pcm.Context(precision="fp64") as ref:
        ref.setup(w.mol, w.basis)
        c64 = ref.esp(w.P)
    with pcm.Context(precision="mixed", esp_variant=variant, fp32x2=fp32x2) as ctx:
        ctx.setup(w.mol, w.basis)
        c32 = ctx.esp(w.P)
    assert np.max(np.abs(c32 - c64)) <= 1e-6 * np.max(np.abs(c64))


def test_packed_and_scalar_agree():
    """The packed kernels run each lane's arithmetic as the scalar kernels do;
    only the order of the sums differs (even and odd pairs, or points, in two
    lanes).  ESP: compensated sums, so the two agree to 1e-7.  Fock at one
    fixed q: plain FP32 sums over a tile of 128 points (64 per lane when
    packed), each within the mixed bar (1e-6 of the largest element) of the
    FP64 Fock and within that bar of one another."""
    import paper_1505_07851_gb300 as pcm
    w = workloads.small_cluster(10, seed=23, d_shells=True)
    out = []
    q = None
    for prec, packed in (("fp64", True), ("mixed", True), ("mixed", False)):
        with pcm.Context(precision=prec, fp32x2=packed) as ctx:
            M, _ = ctx.setup(w.mol, w.basis)
            if q is None:
                q = np.random.default_rng(5).normal(size=M)
            c = ctx.esp(w.P)
            out.append((c, ctx.fock(q)))
    (c64, F64), (c0, F0), (c1, F1) = out
    assert np.max(np.abs(c0 - c1)) <= 1e-7 * np.max(np.abs(c1))
    for F in (F0, F1):
        assert np.max(np.abs(F - F64)) <= 1e-6 * np.max(np.abs(F64))
    assert np.max(np.abs(F0 - F1)) <= 1e-6 * np.max(np.abs(F64))

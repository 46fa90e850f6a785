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
    assert {"esp_points_per_thread", "fock_pairs_per_thread"} <= kinds
    for t in tab:
        allowed = (4, 2) if t["kernel"] == "esp_points_per_thread" else (1, 2)
        assert t["choice"] in allowed and 0 <= t["L"] <= 4
    # a second tuned context reuses the choices: identical results
    c2, F2, E2 = _run(w, True)
    assert np.array_equal(c1, c2) and np.array_equal(F1, F2) and E1 == E2

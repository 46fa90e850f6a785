"""PCM_MIXED (FP32 integrals, FP64 accumulation) against the FP64 GPU path,
which is itself checked against the oracle at 1e-10.  Targets: 1e-6
relative on c and dF (normwise) and 1e-6 Eh on the energy."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _run(w, precision, schwarz=0.0, delta=1e-10):
    import paper_1505_07851_gb300 as pcm
    with pcm.Context(precision=precision, schwarz=schwarz) as ctx:
        ctx.setup(w.mol, w.basis)
        c = ctx.esp(w.P)
        q, st = ctx.solve(delta=delta)
        dF = ctx.fock(q)
        E = ctx.energy(q)
        _, idx = ctx.get_surface()
    return dict(c=c, q=q, dF=dF, E=E, idx=idx)


CASES = {
    "water": lambda: workloads.config(0),
    "cluster8_sp": lambda: workloads.small_cluster(8, seed=21),
    "cluster5_spd": lambda: workloads.small_cluster(5, seed=22, d_shells=True),
    "cluster40_sp": lambda: workloads.small_cluster(40, seed=23),
    "cluster20_spd": lambda: workloads.small_cluster(20, seed=24, d_shells=True),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("schwarz", [0.0, 1e-12])
def test_mixed_matches_fp64(name, schwarz):
    w = CASES[name]()
    a = _run(w, "fp64", schwarz)
    b = _run(w, "mixed", schwarz)
    assert np.array_equal(a["idx"], b["idx"])
    ec = np.max(np.abs(b["c"] - a["c"])) / np.max(np.abs(a["c"]))
    # Fock from the same q isolates the integral error
    import paper_1505_07851_gb300 as pcm
    with pcm.Context(precision="mixed", schwarz=schwarz) as ctx:
        ctx.setup(w.mol, w.basis)
        dF_m = ctx.fock(a["q"])
    eF = np.max(np.abs(dF_m - a["dF"])) / np.max(np.abs(a["dF"]))
    eE = abs(b["E"] - a["E"])
    print("%s schwarz=%g: c %.2e  dF %.2e  E %.2e Eh (E = %.6f)" % (name, schwarz, ec, eF, eE, a["E"]))
    assert ec <= 1e-6, ec
    assert eF <= 1e-6, eF
    assert eE <= 1e-6, eE


def test_mixed_against_oracle_directly():
    w = workloads.small_cluster(8, seed=21)
    b = _run(w, "mixed")
    o = oracle.run(w, delta=1e-10)
    pos = {int(k): i for i, k in enumerate(o["surf"]["index"])}
    p = np.array([pos[int(k)] for k in b["idx"]])
    assert np.max(np.abs(b["c"] - o["c"][p])) <= 1e-6 * np.max(np.abs(o["c"]))
    assert abs(b["E"] - o["E_lu"]) <= 1e-6

"""PCM_MIXED (FP32 integrals, FP64 accumulation) against the oracle on every
case with both operators (stored A, matrix-free), and against the FP64 GPU path (itself checked against the oracle at
1e-10) with and without screening.  Bars: every element of c and dF within
1e-6 of itself plus 1e-7 of the largest element (tests/_parity.py), and
1e-6 Eh on the energy (the Eq. 21 target)."""
import numpy as np
import pytest

import oracle
import workloads
from _parity import MIXED, check

pytestmark = pytest.mark.gpu


def _run(w, precision, schwarz=0.0, delta=1e-10, operator="auto"):
    import paper_1505_07851_gb300 as pcm
    with pcm.Context(precision=precision, schwarz=schwarz, operator=operator) as ctx:
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
    wc = check(b["c"], a["c"], MIXED, what="c")
    # Fock from the same q isolates the integral error
    import paper_1505_07851_gb300 as pcm
    with pcm.Context(precision="mixed", schwarz=schwarz) as ctx:
        ctx.setup(w.mol, w.basis)
        dF_m = ctx.fock(a["q"])
    wF = check(dF_m, a["dF"], MIXED, what="dF")
    eE = abs(b["E"] - a["E"])
    print("%s schwarz=%g: c %.2f dF %.2f of the bar, E %.2e Eh (E = %.6f)" % (name, schwarz, wc, wF, eE, a["E"]))
    assert eE <= 1e-6, eE


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("operator", ["stored", "free"])
def test_mixed_against_oracle_directly(name, operator):
    w = CASES[name]()
    b = _run(w, "mixed", operator=operator)
    o = oracle.run(w, delta=1e-10)
    pos = {int(k): i for i, k in enumerate(o["surf"]["index"])}
    p = np.array([pos[int(k)] for k in b["idx"]])
    check(b["c"], o["c"][p], MIXED, what="c")
    q_o = np.empty_like(b["q"])
    q_o[p] = b["q"]
    check(b["dF"], oracle.fock(o["eb"], q_o, o["surf"]["r"], o["surf"]["zeta"]), MIXED, what="dF")
    assert abs(b["E"] - o["E_lu"]) <= 1e-6


@pytest.mark.parametrize("name", ["cluster8_sp", "cluster20_spd"])
@pytest.mark.parametrize("operator", ["stored", "free"])
def test_mixed_solve_against_lu(name, operator):
    """The refined PCM_MIXED solve of the oracle's own right-hand side (Eq. 1)
    against the oracle's dense LU solution: the FP32 inner solves (the stored
    operator's symmetric tile product, or the matrix-free product) inside the
    double-float refinement reach the FP64 bound ||q - q_lu|| <= 10 delta /
    lambda_min, as the FP64 solver does."""
    import paper_1505_07851_gb300 as pcm
    w = CASES[name]()
    o = oracle.run(w, delta=1e-10)
    with pcm.Context(precision="mixed", operator=operator) as ctx:
        ctx.setup(w.mol, w.basis)
        _, idx = ctx.get_surface()
        pos = {int(k): i for i, k in enumerate(o["surf"]["index"])}
        p = np.array([pos[int(k)] for k in idx])
        q, st = ctx.solve(rhs=np.ascontiguousarray(o["rhs"][p]), delta=1e-10)
    assert st["converged"] == 1 and st["rnorm"] < 1e-10
    lam_min = np.linalg.eigvalsh(o["A"])[0]
    assert np.linalg.norm(q - o["q_lu"][p]) <= 10 * 1e-10 / lam_min


@pytest.mark.parametrize("operator", ["stored", "free"])
def test_energy_from_last_residual_matches_product(operator):
    """pcm_energy of the charges a PCM_MIXED solve just returned takes
    q^T A q from that solve's final true residual (A q = rhs - r); a fresh
    context, which has solved nothing, forms A q by the double-float product.
    The two energies agree to rounding, and a changed q falls back to the
    product."""
    import paper_1505_07851_gb300 as pcm
    w = CASES["cluster20_spd"]()
    with pcm.Context(precision="mixed", operator=operator) as ctx:
        ctx.setup(w.mol, w.basis)
        c = ctx.esp(w.P)
        q, _ = ctx.solve(delta=1e-8)
        E_kept = ctx.energy(q)
        q2 = q.copy()
        q2[len(q2) // 2] *= 1.001
        E_changed = ctx.energy(q2)
    with pcm.Context(precision="mixed", operator=operator) as ctx:
        ctx.setup(w.mol, w.basis)
        E_prod = ctx.energy(q, c=c)
        E_prod2 = ctx.energy(q2, c=c)
    assert abs(E_kept - E_prod) <= 1e-12 * abs(E_prod), (E_kept, E_prod)
    assert E_changed == E_prod2 or abs(E_changed - E_prod2) <= 1e-14 * abs(E_prod2)
    assert E_changed != E_kept


@pytest.mark.parametrize("operator", ["stored", "free"])
def test_mixed_solve_bitwise_reproducible(operator):
    """The symmetric tile products add their row and column parts in 64-bit
    fixed point and every other sum in a fixed order, so two solves of the
    same system (in fresh contexts, with tiles arriving in whatever order the
    hardware schedules them) return the same charges bit for bit."""
    import paper_1505_07851_gb300 as pcm
    w = CASES["cluster40_sp"]()
    qs = []
    for _ in range(2):
        with pcm.Context(precision="mixed", operator=operator) as ctx:
            ctx.setup(w.mol, w.basis)
            ctx.esp(w.P)
            q, st = ctx.solve(delta=1e-9)
            qs.append((q, st["iterations"]))
    assert qs[0][1] == qs[1][1]
    assert np.array_equal(qs[0][0], qs[1][0])

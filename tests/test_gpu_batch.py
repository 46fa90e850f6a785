"""Batched runs (pcm_batch_run: the packed integral blocks of all molecules
in one launch per angular class under PCM_MIXED, every solve in lockstep with
the PCG loop as a device-driven CUDA graph, or with matrix-free members one
persistent solver per molecule) against the single-molecule path on the same
inputs, and three molecules against the oracle (energy, the charges against
the LU solution, dF element by element).  Five clusters of uneven size (one below the Jacobi threshold, the
others on RBJ)."""
import numpy as np
import pytest

import oracle
import workloads
from _parity import FP64, MIXED, check

pytestmark = pytest.mark.gpu

SIZES = ((18, 41), (30, 42), (12, 45), (36, 44), (24, 43))
DELTA_1E6 = (1e-6 / 0.01) ** (1.0 / 1.07)


@pytest.fixture(scope="module")
def mols():
    return [workloads.small_cluster(n, seed) for n, seed in SIZES]


def _single(w, precision, delta):
    import paper_1505_07851_gb300 as pcm
    with pcm.Context(precision=precision) as ctx:
        ctx.setup(w.mol, w.basis)
        ctx.esp(w.P)
        q, st = ctx.solve(delta=delta)
        return dict(E=ctx.energy(q), q=q, dF=ctx.fock(q), it=st["iterations"], conv=st["converged"])


def _batch(mols, precision, delta, device=False, operator="auto"):
    import paper_1505_07851_gb300 as pcm
    with pcm.Batch(len(mols), precision=precision, operator=operator) as b:
        for i, w in enumerate(mols):
            b.set_molecule(i, w.mol, w.basis)
        Ps = [w.P for w in mols]
        if device:
            import torch
            Ps = [torch.tensor(P, device="cuda") for P in Ps]
        E, q, dF = b.run(Ps, delta, want_q=True, want_dF=True)
        if device:
            q = [a.cpu().numpy() for a in q]
            dF = [a.cpu().numpy() for a in dF]
        st = [b.stats(i) for i in range(len(mols))]
        tot = b.stats()
    return E, q, dF, st, tot


def test_fp64_batch_matches_single(mols):
    E, q, dF, st, tot = _batch(mols, "fp64", 1e-9)
    assert tot["launches"] > 0
    for i, w in enumerate(mols):
        s = _single(w, "fp64", 1e-9)
        assert st[i]["converged"] and s["conv"]
        assert abs(st[i]["iterations"] - s["it"]) <= 1, (i, st[i]["iterations"], s["it"])
        assert abs(E[i] - s["E"]) <= 1e-10
        assert np.max(np.abs(dF[i] - s["dF"])) <= 1e-8 * np.max(np.abs(s["dF"]))


def test_mixed_batch_energy_error_vs_fp64(mols):
    E, q, dF, st, tot = _batch(mols, "mixed", DELTA_1E6)
    for i, w in enumerate(mols):
        ref = _single(w, "fp64", 1e-10)
        assert st[i]["converged"]
        assert abs(E[i] - ref["E"]) <= 1e-6, (i, E[i] - ref["E"])
        assert np.max(np.abs(dF[i] - ref["dF"])) <= 1e-5 * np.max(np.abs(ref["dF"]))


@pytest.mark.parametrize("precision,operator", [("fp64", "auto"), ("mixed", "auto"), ("mixed", "free")])
def test_batch_molecules_against_oracle(mols, precision, operator):
    import paper_1505_07851_gb300 as pcm
    E, q, dF, st, tot = _batch(mols, precision, 1e-10, operator=operator)
    bars = FP64 if precision == "fp64" else MIXED
    for i in (0, 2, 4):
        w = mols[i]
        o = oracle.run(w, delta=1e-10)
        assert st[i]["converged"]
        assert abs(E[i] - o["E_lu"]) <= (1e-9 if precision == "fp64" else 1e-6), (i, E[i] - o["E_lu"])
        with pcm.Context() as ctx:
            ctx.build_surface(w.mol.xyz, w.mol.Z, w.mol.radius, 110)
            _, idx = ctx.get_surface()
        pos = {int(k): j for j, k in enumerate(o["surf"]["index"])}
        perm = np.array([pos[int(k)] for k in idx])
        q_o = np.empty_like(q[i])
        q_o[perm] = q[i]
        check(dF[i], oracle.fock(o["eb"], q_o, o["surf"]["r"], o["surf"]["zeta"]), bars, what="dF %d" % i)
        # the batch's c stays inside it; its charges solve A q = -f (Bz + c) to the
        # threshold, so they are compared with the LU solution of the oracle's system
        lam_min = np.linalg.eigvalsh(o["A"])[0]
        assert np.linalg.norm(q[i] - o["q_lu"][perm]) <= 10 * 1e-10 / lam_min + (0 if precision == "fp64" else 1e-5)


def test_device_pointers_bit_identical(mols):
    a = _batch(mols[:3], "mixed", DELTA_1E6)
    b = _batch(mols[:3], "mixed", DELTA_1E6, device=True)
    assert np.array_equal(a[0], b[0])
    for x, y in zip(a[2], b[2]):
        assert np.array_equal(x, y)


def test_batch_errors(mols):
    import paper_1505_07851_gb300 as pcm
    with pcm.Batch(2) as b:
        b.set_molecule(0, mols[0].mol, mols[0].basis)
        with pytest.raises(pcm.PCMError):
            b.run([mols[0].P, mols[1].P], 1e-6)          # molecule 1 not set
        with pytest.raises(pcm.PCMError):
            b.set_molecule(2, mols[1].mol, mols[1].basis)

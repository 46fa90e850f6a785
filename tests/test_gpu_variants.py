"""Variants of Section 4b-ii and Eq. 1: the octree block-Jacobi preconditioner
the paper compares RBJ with, and COSMO's k = 0.5.  Against the oracle on the
same inputs."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def test_octree_preconditioner_matches_oracle():
    import paper_1505_07851_gb300 as pcm
    w = workloads.small_cluster(24, seed=31)
    s = oracle.surface(w.mol.xyz, w.mol.radius)
    A = oracle.a_matrix(s)
    f = oracle.f_factor()
    rhs = -f * (oracle.bz(s, w.mol.xyz, w.mol.Z) + oracle.esp(oracle.ExpandedBasis(w.basis, w.mol.xyz), w.P,
                                                              s["r"], s["zeta"]))
    for leaf in (200, 800):
        pc = oracle.Preconditioner(A, "octree", leaf, points=s["r"])
        x, it, ok, rn = oracle.pcg(A, rhs, 1e-8, pc)
        with pcm.Context(schwarz=0.0, precond="octree", octree_leaf=leaf) as ctx:
            ctx.setup(w.mol, w.basis)
            _, idx = ctx.get_surface()
            ctx.esp(w.P)
            q, st = ctx.solve(delta=1e-8)
        pos = {int(k): i for i, k in enumerate(s["index"])}
        perm = np.array([pos[int(k)] for k in idx])
        assert ok and st["converged"]
        assert abs(st["iterations"] - it) <= 1, (leaf, st["iterations"], it)
        assert np.linalg.norm(A[np.ix_(perm, perm)] @ q - rhs[perm]) <= 1.05e-8 + 1e-12 * np.linalg.norm(rhs)


def test_cosmo_k_half():
    """k = 0.5 (COSMO): parity with the oracle, and E scales exactly with
    f = (eps - 1)/(eps + k) at the solution (E = -(f/2) V^T A^-1 V)."""
    import paper_1505_07851_gb300 as pcm
    w = workloads.small_cluster(8, seed=21)
    E = {}
    for k in (0.0, 0.5):
        with pcm.Context(schwarz=0.0, k=k) as ctx:
            ctx.setup(w.mol, w.basis)
            ctx.esp(w.P)
            q, _ = ctx.solve(delta=1e-11)
            E[k] = ctx.energy(q)
        o = oracle.run(w, k=k, delta=1e-11)
        assert abs(E[k] - o["E_lu"]) <= 1e-9
    ratio = oracle.f_factor(78.39, 0.5) / oracle.f_factor(78.39, 0.0)
    assert abs(E[0.5] / E[0.0] - ratio) <= 1e-10

"""Edge and degenerate cases of the path on the GPU, against the oracle or
against what the equations fix exactly."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _pcm():
    import paper_1505_07851_gb300 as pcm
    return pcm


def _perm(ctx_index, orc_index):
    pos = {int(k): i for i, k in enumerate(orc_index)}
    return np.array([pos[int(k)] for k in ctx_index])


def _mol(symbols, xyz):
    return workloads._mol(symbols, xyz)


def test_isolated_atoms_have_no_switching():
    """Two atoms 40 bohr apart: every S_k is 1, M = 2 n, and the energy is that
    of the oracle (and nearly twice the single-atom energy)."""
    pcm = _pcm()
    mol = _mol(["O", "O"], [[0, 0, 0], [40.0, 0, 0]])
    with pcm.Context(schwarz=0.0) as ctx:
        M = ctx.build_surface(mol.xyz, mol.Z, mol.radius, 110)
        xyzzs, idx = ctx.get_surface()
    assert M == 220 and np.all(xyzzs[:, 4] == 1.0)
    s = oracle.surface(mol.xyz, mol.radius)
    assert len(s["zeta"]) == 220


@pytest.mark.parametrize("npts", [26, 302])
def test_other_sphere_sizes_match_oracle(npts):
    pcm = _pcm()
    w = workloads.config(0)
    zeta = 4.9
    with pcm.Context(schwarz=0.0) as ctx:
        ctx.setup(w.mol, w.basis, pts_per_sphere=npts)
        xyzzs, idx = ctx.get_surface()
        c = ctx.esp(w.P)
        q, _ = ctx.solve(delta=1e-11)
        E = ctx.energy(q)
    o = oracle.run(w, n=npts, zeta=zeta, delta=1e-11)
    p = _perm(idx, o["surf"]["index"])
    assert np.max(np.abs(c - o["c"][p])) <= 1e-10 * np.max(np.abs(o["c"]))
    assert abs(E - o["E_lu"]) <= 1e-9


def test_buried_points_are_dropped_like_the_oracle():
    """A hydrogen inside an oxygen sphere: its points are buried (S < 1e-8)
    and dropped; the kept set matches the oracle's."""
    pcm = _pcm()
    mol = _mol(["O", "H"], [[0, 0, 0], [0.3, 0.0, 0.0]])
    with pcm.Context() as ctx:
        M = ctx.build_surface(mol.xyz, mol.Z, mol.radius, 110)
        _, idx = ctx.get_surface()
    s = oracle.surface(mol.xyz, mol.radius)
    assert M == len(s["index"]) < 220
    assert sorted(idx.tolist()) == sorted(s["index"].tolist())


def test_zero_density_and_zero_charges():
    """P = 0 gives c = 0 (the nuclei alone polarise the solvent); q = 0 gives
    dF = 0 and a zero gradient; the energy is the oracle's nuclear-only one."""
    pcm = _pcm()
    w = workloads.small_cluster(5, seed=22, d_shells=True)
    P0 = np.zeros_like(w.P)
    for prec in ("fp64", "mixed"):
        with pcm.Context(precision=prec, schwarz=0.0) as ctx:
            M, nbf = ctx.setup(w.mol, w.basis)
            c = ctx.esp(P0)
            assert np.all(c == 0.0)
            q, _ = ctx.solve(delta=1e-11)
            E = ctx.energy(q)
            dF = ctx.fock(np.zeros(M))
            assert np.all(dF == 0.0)
            g = ctx.gradient(np.zeros(M), w.P)
            assert np.all(g == 0.0)
        s = oracle.surface(w.mol.xyz, w.mol.radius)
        A = oracle.a_matrix(s)
        f = oracle.f_factor()
        Bz = oracle.bz(s, w.mol.xyz, w.mol.Z)
        qo = oracle.solve_lu(A, -f * Bz)
        assert abs(E - oracle.energy(Bz, np.zeros_like(Bz), qo, A, f)) <= 1e-9


def test_screening_everything_away():
    """A cutoff above every bound leaves no primitive pair: c and dF are zero
    in both precisions and nothing fails."""
    pcm = _pcm()
    w = workloads.small_cluster(5, seed=22, d_shells=True)
    for prec in ("fp64", "mixed"):
        with pcm.Context(precision=prec, schwarz=1e30) as ctx:
            M, nbf = ctx.setup(w.mol, w.basis)
            assert ctx.stats()["pairs_kept"] == 0
            c = ctx.esp(w.P)
            assert np.all(c == 0.0)
            dF = ctx.fock(np.ones(M))
            assert np.all(dF == 0.0)


def test_d_shells_only():
    """A basis of d shells alone (only the dd class): parity with the oracle."""
    pcm = _pcm()
    mol = _mol(["N", "O"], [[0, 0, 0], [2.2, 0.3, -0.4]])
    rng = np.random.default_rng(4)
    basis = workloads.Basis(np.array([0, 1, 1], np.int32), np.array([2, 2, 2], np.int32),
                            np.array([2, 1, 2], np.int32), np.array([1.3, 0.4, 0.9, 2.0, 0.5]),
                            rng.uniform(0.1, 1.0, 5))
    nbf = 18
    G = rng.normal(size=(nbf, 4))
    P = G @ G.T
    with pcm.Context(schwarz=0.0) as ctx:
        ctx.setup(mol, basis)
        _, idx = ctx.get_surface()
        c = ctx.esp(P)
        q, _ = ctx.solve(delta=1e-11)
        dF = ctx.fock(q)
    s = oracle.surface(mol.xyz, mol.radius)
    eb = oracle.ExpandedBasis(basis, mol.xyz)
    p = _perm(idx, s["index"])
    co = oracle.esp(eb, P, s["r"], s["zeta"])
    assert np.max(np.abs(c - co[p])) <= 1e-10 * np.max(np.abs(co))
    q_o = np.empty_like(q)
    q_o[p] = q
    Fo = oracle.fock(eb, q_o, s["r"], s["zeta"])
    assert np.max(np.abs(dF - Fo)) <= 1e-10 * np.max(np.abs(Fo))


def test_solver_limits():
    """A threshold above |rhs| stops at iteration 0 with q = 0; a warm start
    from the solution stops at once; RBJ with one block (l >= M) converges in
    one step."""
    pcm = _pcm()
    w = workloads.config(0)
    with pcm.Context() as ctx:
        M, _ = ctx.setup(w.mol, w.basis)
        ctx.esp(w.P)
        q0, st0 = ctx.solve(delta=1e6)
        assert st0["iterations"] == 0 and st0["converged"] and np.all(q0 == 0.0)
        q, st = ctx.solve(delta=1e-12)
        q2, st2 = ctx.solve(delta=1e-8, q=q.copy(), warm=True)
        assert st2["iterations"] == 0 and st2["converged"]
    with pcm.Context(precond="rbj", rbj_block=10 ** 6) as ctx:
        ctx.setup(w.mol, w.basis)
        ctx.esp(w.P)
        q, st = ctx.solve(delta=1e-9)
        assert st["iterations"] <= 2 and st["converged"]


def test_batch_with_a_single_atom():
    """A batch whose members include a one-atom molecule (Jacobi, tiny M)."""
    pcm = _pcm()
    one = workloads.Workload("one", _mol(["O"], [[0, 0, 0]]),
                             workloads.Basis(np.array([0], np.int32), np.array([0], np.int32),
                                             np.array([2], np.int32), np.array([3.0, 0.5]), np.array([0.6, 0.5])),
                             np.full((1, 1), 2.0), 1, 0)
    mols = [one, workloads.config(0)]
    with pcm.Batch(2, precision="fp64") as b:
        for i, w in enumerate(mols):
            b.set_molecule(i, w.mol, w.basis)
        E, q, dF = b.run([w.P for w in mols], 1e-10, want_q=True, want_dF=True)
    for i, w in enumerate(mols):
        o = oracle.run(w, delta=1e-10)
        assert abs(E[i] - o["E_lu"]) <= 1e-9

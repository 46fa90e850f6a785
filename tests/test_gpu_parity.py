"""GPU path (through the C ABI) against the CPU oracle on the same seeded
inputs, element by element, FP64 mode.  Tolerances (FP64): every element of
c and dF within 1e-10 of itself plus 1e-12 of the largest element (see
tests/_parity.py); Bz 1e-13 relative; 1e-9 Eh on the energy; 1e-13 relative
on point positions and 1e-10 on switching values."""
import math

import numpy as np
import pytest

import oracle
import workloads
from _parity import FP64, check

pytestmark = pytest.mark.gpu


def _pcm():
    import paper_1505_07851_gb300 as pcm
    return pcm


def _perm(ctx_index, orc_index):
    pos = {int(k): i for i, k in enumerate(orc_index)}
    assert len(ctx_index) == len(orc_index)
    return np.array([pos[int(k)] for k in ctx_index])


def _run_gpu(w, schwarz=0.0, delta=1e-10, precond="auto", rbj_block=100, seed=0, n=110):
    pcm = _pcm()
    with pcm.Context(schwarz=schwarz, precond=precond, rbj_block=rbj_block, seed=seed) as ctx:
        M, nbf = ctx.setup(w.mol, w.basis, n)
        xyzzs, idx = ctx.get_surface()
        Bz = np.zeros(M)
        c = ctx.esp(w.P, bz_out=Bz)
        q, st = ctx.solve(delta=delta)
        dF = ctx.fock(q)
        E = ctx.energy(q)
        return dict(M=M, nbf=nbf, xyzzs=xyzzs, idx=idx, Bz=Bz, c=c, q=q, st=st, dF=dF, E=E,
                    stats=ctx.stats())


CASES = {
    "water": lambda: workloads.config(0),
    "cluster8_sp": lambda: workloads.small_cluster(8, seed=21),
    "cluster5_spd": lambda: workloads.small_cluster(5, seed=22, d_shells=True),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    w = CASES[request.param]()
    g = _run_gpu(w)
    o = oracle.run(w, delta=1e-10)
    return request.param, w, g, o


def test_surface_parity(case):
    name, w, g, o = case
    s = o["surf"]
    assert g["M"] == len(s["S"])
    p = _perm(g["idx"], s["index"])
    xyzzs = g["xyzzs"]
    assert np.max(np.abs(xyzzs[:, :3] - s["r"][p])) <= 1e-13 * np.max(np.abs(s["r"]))
    assert np.max(np.abs(xyzzs[:, 3] - s["zeta"][p]) / s["zeta"][p]) <= 1e-15
    # S_k is a product of erfc factors whose relative sensitivity to the point
    # position is ~2 x zeta per factor; positions agree to ~1e-13 bohr (the
    # angle i pi (3 - sqrt 5) is rounded differently), so allow 1e-10.
    assert np.max(np.abs(xyzzs[:, 4] - s["S"][p]) / s["S"][p]) <= 1e-10
    # library order: grouped by increasing exponent
    assert np.all(np.diff(xyzzs[:, 3]) >= 0)


def test_bz_parity(case):
    name, w, g, o = case
    p = _perm(g["idx"], o["surf"]["index"])
    assert np.max(np.abs(g["Bz"] - o["Bz"][p])) <= 1e-13 * np.max(np.abs(o["Bz"]))


def test_esp_parity(case):
    name, w, g, o = case
    p = _perm(g["idx"], o["surf"]["index"])
    check(g["c"], o["c"][p], FP64, what="c")


def test_fock_parity(case):
    name, w, g, o = case
    p = _perm(g["idx"], o["surf"]["index"])
    q_o = np.empty_like(g["q"])
    q_o[p] = g["q"]
    ref = oracle.fock(o["eb"], q_o, o["surf"]["r"], o["surf"]["zeta"])
    check(g["dF"], ref, FP64, what="dF")
    assert np.max(np.abs(g["dF"] - g["dF"].T)) == 0.0


def test_solve_and_energy_parity(case):
    name, w, g, o = case
    p = _perm(g["idx"], o["surf"]["index"])
    assert g["st"]["converged"] == 1 and g["st"]["rnorm"] < 1e-10
    lam_min = np.linalg.eigvalsh(o["A"])[0]
    assert np.linalg.norm(g["q"] - o["q_lu"][p]) <= 10 * 1e-10 / lam_min
    assert abs(g["E"] - o["E_lu"]) <= 1e-9, (g["E"], o["E_lu"])
    # the same preconditioner and threshold take the same number of steps (up to one)
    assert abs(g["st"]["iterations"] - o["iters"]) <= 1


def test_duality_q_c_equals_P_dF(case):
    name, w, g, o = case
    lhs = g["q"] @ g["c"]
    rhs = np.sum(w.P * g["dF"])
    assert abs(lhs - rhs) <= 1e-11 * (np.abs(g["q"]) @ np.abs(g["c"]))


@pytest.mark.parametrize("l,seed", [(40, 3), (100, 7)])
def test_rbj_iterations_match_oracle(l, seed):
    w = workloads.small_cluster(10, seed=31)
    g = _run_gpu(w, delta=1e-8, precond="rbj", rbj_block=l, seed=seed)
    s = oracle.surface(w.mol.xyz, w.mol.radius)
    p = _perm(g["idx"], s["index"])
    A = oracle.a_matrix(s)
    b = np.zeros(len(g["q"]))
    # same rhs as the GPU solve: -f (Bz + c) in oracle order
    eb = oracle.ExpandedBasis(w.basis, w.mol.xyz)
    c = oracle.esp(eb, w.P, s["r"], s["zeta"])
    b = -oracle.f_factor() * (oracle.bz(s, w.mol.xyz, w.mol.Z) + c)
    pc = oracle.Preconditioner(A, "rbj", l, seed)
    x, it, ok, rn = oracle.pcg(A, b, 1e-8, pc)
    assert ok and g["st"]["converged"]
    assert abs(g["st"]["iterations"] - it) <= 1, (g["st"]["iterations"], it)
    assert np.linalg.norm(g["q"] - x[p]) <= 1e-6


@pytest.mark.parametrize("l,seed", [(40, 3), (100, 7)])
def test_rbj_residual_history_matches_oracle(l, seed):
    """The RBJ blocks are the oracle's (pivots and ties follow the atom-major
    point order, not the library's storage order), so the first CG steps
    reproduce the oracle's residual norms to rounding: ||r_k|| after k = 1..6
    steps, cold start, on a cluster of several elements (several exponent
    classes, so storage and atom-major orders differ)."""
    pcm = _pcm()
    w = workloads.small_cluster(10, seed=31)
    s = oracle.surface(w.mol.xyz, w.mol.radius)
    A = oracle.a_matrix(s)
    eb = oracle.ExpandedBasis(w.basis, w.mol.xyz)
    c = oracle.esp(eb, w.P, s["r"], s["zeta"])
    b = -oracle.f_factor() * (oracle.bz(s, w.mol.xyz, w.mol.Z) + c)
    pc = oracle.Preconditioner(A, "rbj", l, seed)
    assert len(set(s["zeta"].round(12))) > 1
    for k in range(1, 7):
        with pcm.Context(schwarz=0.0, precond="rbj", rbj_block=l, seed=seed, max_iter=k) as ctx:
            ctx.setup(w.mol, w.basis)
            ctx.esp(w.P)
            q, st = ctx.solve(delta=1e-30)
        _, it, ok, rn = oracle.pcg(A, b, 1e-30, pc, max_iter=k)
        assert st["iterations"] == it == k
        assert abs(st["rnorm"] - rn) <= 1e-8 * rn, (k, st["rnorm"], rn)


def test_rbj_full_block_one_step():
    w = workloads.config(0)
    g = _run_gpu(w, delta=1e-8, precond="rbj", rbj_block=10 ** 6)
    assert g["st"]["converged"] and g["st"]["iterations"] == 1


def test_screening_error_is_small():
    w = workloads.small_cluster(8, seed=21)
    g0 = _run_gpu(w, schwarz=0.0)
    g1 = _run_gpu(w, schwarz=1e-12)
    st = g1["stats"]
    assert st["pairs_kept"] < st["pairs_candidate"]
    assert np.max(np.abs(g1["c"] - g0["c"])) <= 1e-8 * np.max(np.abs(g0["c"]))
    assert np.max(np.abs(g1["dF"] - g0["dF"])) <= 1e-8 * np.max(np.abs(g0["dF"]))


def test_device_pointers_match_host_pointers():
    import torch
    pcm = _pcm()
    w = workloads.small_cluster(6, seed=5)
    with pcm.Context(schwarz=0.0) as ctx:
        M, nbf = ctx.setup(w.mol, w.basis)
        c_h = ctx.esp(w.P)
        q_h, _ = ctx.solve(delta=1e-9)
        F_h = ctx.fock(q_h)
        E_h = ctx.energy(q_h)
        Pd = torch.tensor(w.P, device="cuda", dtype=torch.float64)
        c_d = ctx.esp(Pd)
        q_d, _ = ctx.solve(delta=1e-9, like=Pd)
        F_d = ctx.fock(q_d)
        E_d = ctx.energy(q_d)
    assert np.array_equal(c_h, c_d.cpu().numpy())
    assert np.array_equal(q_h, q_d.cpu().numpy())
    assert np.array_equal(F_h, F_d.cpu().numpy())
    assert E_h == E_d


def test_reruns_are_bit_identical():
    w = workloads.small_cluster(8, seed=21)
    a = _run_gpu(w, schwarz=1e-12)
    b = _run_gpu(w, schwarz=1e-12)
    for k in ("c", "q", "dF"):
        assert np.array_equal(a[k], b[k]), k
    assert a["E"] == b["E"]


def test_single_sphere_conductor_on_gpu():
    # one atom, no electrons: induced charge -> -f, energy -> -f/(2R)
    pcm = _pcm()
    R = 2.7
    with pcm.Context() as ctx:
        M = ctx.build_surface(np.zeros((1, 3)), np.array([1.0]), np.array([R]), 302)
        assert M == 302
        nb = ctx.set_basis([0], [0], [1], [1.0], [0.0])      # zero-coefficient basis: c = 0
        c = ctx.esp(np.zeros((1, 1)))
        assert np.all(c == 0.0)
        q, st = ctx.solve(delta=1e-12)
        E = ctx.energy(q)
    f = oracle.f_factor()
    assert abs(q.sum() / (-f) - 1) < 1e-3
    assert abs(E / (-f / (2 * R)) - 1) < 1e-3


def test_error_codes():
    pcm = _pcm()
    with pcm.Context() as ctx:
        with pytest.raises(pcm.PCMError) as e:
            ctx.esp(np.eye(2))                              # no basis yet
        assert e.value.status == pcm.PCM_ERR_ARG
        with pytest.raises(pcm.PCMError) as e:
            ctx.build_surface(np.zeros((1, 3)), [1.0], [-1.0])
        assert e.value.status == pcm.PCM_ERR_ARG
        with pytest.raises(pcm.PCMError) as e:
            ctx.build_surface(np.full((1, 3), np.nan), [1.0], [2.0])
        assert e.value.status == pcm.PCM_ERR_ARG
        ctx.build_surface(np.zeros((1, 3)), [1.0], [2.0])
        with pytest.raises(pcm.PCMError) as e:
            ctx.set_basis([0], [3], [1], [1.0], [1.0])     # f shell
        assert e.value.status == pcm.PCM_ERR_UNSUPPORTED
        ctx.set_basis([0], [0], [1], [1.0], [1.0])
        with pytest.raises(pcm.PCMError) as e:
            ctx.esp(np.full((1, 1), np.nan))
        assert e.value.status == pcm.PCM_ERR_ARG
    with pcm.Context(max_iter=2, precond="none") as ctx:
        w = workloads.config(0)
        ctx.setup(w.mol, w.basis)
        ctx.esp(w.P)
        q, st = ctx.solve(delta=1e-12)
        assert st["converged"] == 0 and st["iterations"] == 2
        assert np.all(np.isfinite(q))


def test_context_reuse_matches_fresh_contexts():
    """One context through several set-ups (same shells at a new geometry, then
    other shells) gives the results of a fresh context each time, bit for bit:
    the reused shell-pair lists change nothing."""
    pcm = _pcm()
    a = workloads.small_cluster(8, seed=21)
    b = workloads.small_cluster(5, seed=22, d_shells=True)
    moved = workloads.Workload(a.name, workloads.Molecule(a.mol.symbols, a.mol.xyz + 0.05 * np.sin(a.mol.xyz),
                                                          a.mol.Z, a.mol.radius), a.basis, a.P, a.nocc, a.seed)

    def run(ctx, w):
        ctx.setup(w.mol, w.basis)
        c = ctx.esp(w.P)
        q, _ = ctx.solve(delta=1e-9)
        return c, ctx.fock(q), ctx.energy(q)

    with pcm.Context() as ctx:
        seq = [run(ctx, w) for w in (a, moved, b, a)]
    for w, got in zip((a, moved, b, a), seq):
        with pcm.Context() as fresh:
            ref = run(fresh, w)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]) and got[2] == ref[2]

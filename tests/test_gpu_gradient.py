"""Nuclear gradient (Eq. 14, Eq. 22) through the C ABI against the oracle,
term by term, on the same seeded inputs and the same charges; against
finite differences of the library's own energy at fixed q; and through the
torch.autograd.Function.  Tolerance (FP64): 1e-10 relative to the largest
component of each term."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _pcm():
    import paper_1505_07851_gb300 as pcm
    return pcm


def _perm(ctx_index, orc_index):
    pos = {int(k): i for i, k in enumerate(orc_index)}
    return np.array([pos[int(k)] for k in ctx_index])


CASES = {
    "water": lambda: workloads.config(0),
    "cluster3_spd": lambda: workloads.small_cluster(3, 7, d_shells=True),
    "cluster8_sp": lambda: workloads.small_cluster(8, seed=21),
    "cluster5_spd": lambda: workloads.small_cluster(5, seed=22, d_shells=True),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    pcm = _pcm()
    w = CASES[request.param]()
    o = oracle.run(w, delta=1e-10)
    s = o["surf"]
    q_o = o["q_lu"]
    og = oracle.gradient(o["eb"], w.P, q_o, s, w.mol.xyz, w.mol.Z, w.mol.radius, o["f"])
    with pcm.Context(schwarz=0.0) as ctx:
        ctx.setup(w.mol, w.basis)
        _, idx = ctx.get_surface()
        p = _perm(idx, s["index"])
        q = q_o[p]
        g = {t: ctx.gradient(q, w.P, terms=t) for t in ("B", "C", "A")}
        g["total"] = ctx.gradient(q, w.P)
        g2 = ctx.gradient(q, w.P)
    return request.param, w, og, g, g2


@pytest.mark.parametrize("term", ["B", "C", "A", "total"])
def test_gradient_terms_match_oracle(case, term):
    name, w, og, g, g2 = case
    scale = np.max(np.abs(og[term]))
    err = np.max(np.abs(g[term] - og[term])) / scale
    assert err <= TOL, (name, term, err)


def test_gradient_terms_add_up_and_rerun_bit_identical(case):
    name, w, og, g, g2 = case
    assert np.allclose(g["B"] + g["C"] + g["A"], g["total"], rtol=0, atol=1e-14 * np.max(np.abs(g["total"])))
    assert np.array_equal(g["total"], g2)


def test_gradient_translation_invariance(case):
    name, w, og, g, g2 = case
    for t in ("B", "C", "A"):
        assert np.max(np.abs(g[t].sum(axis=0))) <= 1e-11 * np.max(np.abs(g[t]))


def test_gradient_matches_finite_differences_of_the_library_energy():
    """Richardson central differences of (Bz)^T q + c^T q + q^T A q / 2f
    computed by the library at displaced geometries with q fixed."""
    pcm = _pcm()
    w = workloads.small_cluster(3, 7, d_shells=True)
    with pcm.Context(schwarz=0.0) as ctx:
        M, _ = ctx.setup(w.mol, w.basis)
        _, idx0 = ctx.get_surface()
        ctx.esp(w.P)
        q, _ = ctx.solve(delta=1e-11)
        g = ctx.gradient(q, w.P)

        def E(x):
            ctx.build_surface(x, w.mol.Z, w.mol.radius)
            ctx.set_basis(w.basis.shell_atom, w.basis.shell_l, w.basis.shell_nprim, w.basis.exps, w.basis.coefs)
            _, idx = ctx.get_surface()
            assert np.array_equal(idx, idx0)
            ctx.esp(w.P)
            return ctx.energy(q)

        fd = np.zeros_like(g)
        for I in range(w.mol.natom):
            for d in range(3):
                D = []
                for h in (2e-3, 1e-3):
                    xp = w.mol.xyz.copy()
                    xp[I, d] += h
                    xm = w.mol.xyz.copy()
                    xm[I, d] -= h
                    D.append((E(xp) - E(xm)) / (2 * h))
                fd[I, d] = (4 * D[1] - D[0]) / 3
    assert np.max(np.abs(g - fd)) <= 1e-8 * np.max(np.abs(g))


def test_autograd_function_water():
    import torch
    pcm = _pcm()
    w = workloads.config(0)
    dev = torch.device("cuda", 0)
    with pcm.Context(schwarz=0.0) as ctx:
        xyz = torch.tensor(w.mol.xyz, dtype=torch.float64, requires_grad=True)
        P = torch.tensor(w.P, dtype=torch.float64, device=dev, requires_grad=True)
        E = pcm.solvation_energy(xyz, P, ctx, w.mol, w.basis, delta=1e-12)
        E.backward()
        # the backward is pcm_gradient (positions) and pcm_fock (density) at the forward's q
        ctx.setup(w.mol, w.basis)
        ctx.esp(w.P)
        q, _ = ctx.solve(delta=1e-12)
        g = ctx.gradient(q, w.P)
        dF = ctx.fock(q)
        assert np.allclose(xyz.grad.numpy(), g, rtol=1e-9, atol=1e-12)
        assert np.allclose(P.grad.cpu().numpy(), dF, rtol=1e-9, atol=1e-12)

        # and both are derivatives of the energy (q re-solved at every point)
        def f(x, Pm):
            return pcm.solvation_energy(x, Pm, ctx, w.mol, w.basis, 1e-12)

        x0 = torch.tensor(w.mol.xyz, dtype=torch.float64, requires_grad=True)
        P0 = torch.tensor(w.P, dtype=torch.float64, device=dev, requires_grad=True)
        assert torch.autograd.gradcheck(f, (x0, P0), eps=1e-5, atol=1e-7, rtol=1e-5)


def test_gradient_errors():
    pcm = _pcm()
    w = workloads.config(0)
    with pcm.Context() as ctx:
        ctx.build_surface(w.mol.xyz, w.mol.Z, w.mol.radius)
        q = np.zeros(ctx.M)
        # B and A need no basis; the integral term does
        g = ctx.gradient(q, None, terms="BA")
        assert np.all(g == 0.0)
        with pytest.raises(pcm.PCMError):
            ctx.gradient(q, w.P, terms="C")


@pytest.fixture(scope="module", params=sorted(CASES))
def mixed_case(request):
    pcm = _pcm()
    w = CASES[request.param]()
    o = oracle.run(w, delta=1e-10)
    s = o["surf"]
    og = oracle.gradient(o["eb"], w.P, o["q_lu"], s, w.mol.xyz, w.mol.Z, w.mol.radius, o["f"])
    with pcm.Context(schwarz=0.0, precision="mixed") as ctx:
        ctx.setup(w.mol, w.basis)
        _, idx = ctx.get_surface()
        ctx.esp(w.P)
        ctx.solve(delta=1e-8)                  # makes the FP32 copy of A
        q = o["q_lu"][_perm(idx, s["index"])]
        g = {t: ctx.gradient(q, w.P, terms=t) for t in ("B", "C", "A")}
        g["total"] = ctx.gradient(q, w.P)
    return request.param, og, g


@pytest.mark.parametrize("term", ["B", "C", "A", "total"])
def test_mixed_gradient_matches_oracle(mixed_case, term):
    """PCM_MIXED: FP32 integral and off-diagonal A kernels; the bar is
    1e-5 Eh/bohr absolute, and 1e-6 relative to the largest component."""
    name, og, g = mixed_case
    err = np.max(np.abs(g[term] - og[term]))
    assert err <= 1e-5, (name, term, err)
    assert err <= 1e-6 * max(1.0, np.max(np.abs(og[term]))), (name, term, err)


def test_scalar_and_packed_mixed_gradients_agree():
    """The scalar FP32 gradient kernels (pcm_options.fp32x2 = 0) and the
    packed ones do the same arithmetic per lane; the C term (integrals)
    differs only in the order of the compensated sums, so the two gradients
    agree far inside the mixed bar, and both meet it against the oracle."""
    pcm = _pcm()
    w = workloads.small_cluster(6, seed=24, d_shells=True)
    o = oracle.run(w, delta=1e-10)
    s = o["surf"]
    og = oracle.gradient(o["eb"], w.P, o["q_lu"], s, w.mol.xyz, w.mol.Z, w.mol.radius, o["f"])
    out = []
    for packed in (True, False):
        with pcm.Context(schwarz=0.0, precision="mixed", fp32x2=packed) as ctx:
            ctx.setup(w.mol, w.basis)
            _, idx = ctx.get_surface()
            ctx.esp(w.P)
            ctx.solve(delta=1e-8)
            q = o["q_lu"][_perm(idx, s["index"])]
            out.append(ctx.gradient(q, w.P))
    assert np.max(np.abs(out[0] - out[1])) <= 1e-7 * max(1.0, np.max(np.abs(og["total"])))
    for g in out:
        assert np.max(np.abs(g - og["total"])) <= 1e-6 * max(1.0, np.max(np.abs(og["total"])))

"""The 1000-atom cluster with d shells (M about 46k, nbf about 9.5k) in both
precisions: sampled ESP points and Fock blocks against the oracle, the mixed
energy against the FP64 path.  Bars: FP64 1e-8 relative (screening at
1e-12), mixed 1e-6 relative on c and dF and 1e-6 Eh on the energy."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

DELTA = (1e-6 / 0.01) ** (1.0 / 1.07)


@pytest.fixture(scope="module")
def big():
    import paper_1505_07851_gb300 as pcm
    w = workloads.config(2)
    out = {"w": w}
    for name, prec in (("fp64", "fp64"), ("mixed", "mixed")):
        with pcm.Context(precision=prec) as ctx:
            M, nbf = ctx.setup(w.mol, w.basis)
            c = ctx.esp(w.P)
            q, st = ctx.solve(delta=DELTA)
            dF = ctx.fock(q)
            E = ctx.energy(q)
            r = dict(c=c, q=q, dF=dF, E=E, st=st, M=M, nbf=nbf)
            if prec == "fp64":
                qt, _ = ctx.solve(delta=1e-10)
                r["E_tight"] = ctx.energy(qt)
                _, r["idx"] = ctx.get_surface()
            out[name] = r
    s = oracle.surface(w.mol.xyz, w.mol.radius)
    pos = {int(k): i for i, k in enumerate(s["index"])}
    out["perm"] = np.array([pos[int(k)] for k in out["fp64"]["idx"]])
    out["surf"] = s
    out["eb"] = oracle.ExpandedBasis(w.basis, w.mol.xyz)
    return out


def test_sizes(big):
    assert 40000 <= big["fp64"]["M"] <= 52000
    assert 8000 <= big["fp64"]["nbf"] <= 11000
    assert big["fp64"]["st"]["converged"] and big["mixed"]["st"]["converged"]


def test_esp_sampled(big):
    rng = np.random.default_rng(21)
    s, p = big["surf"], big["perm"]
    sample = rng.choice(len(p), 8, replace=False)
    ref = oracle.esp(big["eb"], big["w"].P, s["r"][p[sample]], s["zeta"][p[sample]])
    scale = np.max(np.abs(ref))
    for name, tol in (("fp64", 1e-8), ("mixed", 1e-6)):
        err = np.max(np.abs(big[name]["c"][sample] - ref)) / scale
        assert err <= tol, (name, err)


def test_fock_sampled(big):
    rng = np.random.default_rng(22)
    eb, s, p = big["eb"], big["surf"], big["perm"]
    pairs = [tuple(sorted(rng.choice(eb.nshell, 2, replace=False))) for _ in range(4)]
    pairs += [(a, a) for a in rng.choice(eb.nshell, 2, replace=False)]
    for name, tol in (("fp64", 1e-8), ("mixed", 1e-6)):
        g = big[name]
        q_o = np.empty_like(g["q"])
        q_o[p] = g["q"]
        blocks = oracle.fock_blocks(eb, q_o, s["r"], s["zeta"], pairs)
        scale = np.max(np.abs(g["dF"]))
        for (a, b), blk in zip(pairs, blocks):
            ia, ib = eb.sh_bf[a], eb.sh_bf[b]
            got = g["dF"][ia:ia + blk.shape[0], ib:ib + blk.shape[1]]
            assert np.max(np.abs(got - blk)) <= tol * scale, (name, a, b)


def test_energies(big):
    Et = big["fp64"]["E_tight"]
    assert abs(big["fp64"]["E"] - Et) <= 1e-6
    assert abs(big["mixed"]["E"] - Et) <= 1e-6

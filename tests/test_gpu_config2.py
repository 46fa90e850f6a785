"""The 1000-atom cluster with d shells (M about 46k, nbf about 8.5k), the
benchmark's workload, in both precisions: 64 sampled ESP points and 32 Fock
blocks (random shell pairs, pairs on one atom, d-d pairs, diagonal blocks)
against the oracle element by element, and the energies against the FP64
solve at delta = 1e-10.

Bars (tests/_parity.py): the FP64 run with the near-complete pair list
(Schwarz cutoff 1e-20: each dropped primitive pair contributes under 1e-20
of the largest magnitudes, far below FP64 rounding of the sums) at rtol
1e-10 / atol 1e-12; the benchmark's FP64 run (cutoff 1e-12) at rtol 1e-8 /
atol 1e-10 (screening error); PCM_MIXED at rtol 1e-6 / atol 1e-7; energies
1e-6 Eh."""
import numpy as np
import pytest

import oracle
import workloads
from _parity import FP64, MIXED, check

pytestmark = pytest.mark.gpu

DELTA = (1e-6 / 0.01) ** (1.0 / 1.07)
SCREENED = (1e-8, 1e-10)


@pytest.fixture(scope="module")
def big():
    import paper_1505_07851_gb300 as pcm
    w = workloads.config(2)
    out = {"w": w}
    for name, prec, schwarz in (("fp64", "fp64", 1e-12), ("mixed", "mixed", 1e-12), ("fine", "fp64", 1e-20)):
        with pcm.Context(precision=prec, schwarz=schwarz) as ctx:
            M, nbf = ctx.setup(w.mol, w.basis)
            c = ctx.esp(w.P)
            if name == "fine":
                q, st = out["fp64"]["q"], out["fp64"]["st"]
            else:
                q, st = ctx.solve(delta=DELTA)
            dF = ctx.fock(q)
            E = ctx.energy(q)
            r = dict(c=c, q=q, dF=dF, E=E, st=st, M=M, nbf=nbf)
            _, r["idx"] = ctx.get_surface()
            if name == "fp64":
                qt, _ = ctx.solve(delta=1e-10)
                r["E_tight"] = ctx.energy(qt)
            out[name] = r
    s = oracle.surface(w.mol.xyz, w.mol.radius)
    pos = {int(k): i for i, k in enumerate(s["index"])}
    out["perm"] = np.array([pos[int(k)] for k in out["fp64"]["idx"]])
    out["surf"] = s
    out["eb"] = oracle.ExpandedBasis(w.basis, w.mol.xyz)
    return out


def test_sizes_and_order(big):
    assert 40000 <= big["fp64"]["M"] <= 52000
    assert 8000 <= big["fp64"]["nbf"] <= 11000
    assert big["fp64"]["st"]["converged"] and big["mixed"]["st"]["converged"]
    for name in ("mixed", "fine"):
        assert np.array_equal(big[name]["idx"], big["fp64"]["idx"])


def test_esp_sampled(big):
    rng = np.random.default_rng(21)
    s, p = big["surf"], big["perm"]
    sample = rng.choice(len(p), 64, replace=False)
    ref = oracle.esp(big["eb"], big["w"].P, s["r"][p[sample]], s["zeta"][p[sample]])
    # the scale of atol: the largest |c| of the whole surface (the oracle's sample
    # shares it to within the FP64 bar)
    scale = np.max(np.abs(big["fine"]["c"]))
    for name, bars in (("fine", FP64), ("fp64", SCREENED), ("mixed", MIXED)):
        check(big[name]["c"][sample], ref, bars, scale=scale, what="c " + name)


def _fock_pairs(eb, rng):
    atom, lval = eb.sh_atom, eb.sh_l
    n = eb.nshell
    pairs = [tuple(sorted(rng.choice(n, 2, replace=False))) for _ in range(8)]
    # both shells on one atom (the largest integrals)
    for a in rng.choice(n, 8, replace=False):
        same = np.flatnonzero((atom == atom[a]) & (np.arange(n) != a))
        pairs.append(tuple(sorted((int(a), int(rng.choice(same))))))
    # d-d pairs: on one atom, on neighbouring atoms, at random
    d = np.flatnonzero(lval == 2)
    for _ in range(8):
        pairs.append(tuple(sorted(rng.choice(d, 2, replace=False))))
    pairs += [(int(a), int(a)) for a in rng.choice(d, 4, replace=False)]
    pairs += [(int(a), int(a)) for a in rng.choice(n, 4, replace=False)]
    return pairs


def test_fock_sampled(big):
    rng = np.random.default_rng(22)
    eb, s, p = big["eb"], big["surf"], big["perm"]
    pairs = _fock_pairs(eb, rng)
    assert len(pairs) >= 32 and any(eb.sh_l[a] == 2 and eb.sh_l[b] == 2 and a != b for a, b in pairs)
    for name, bars in (("fine", FP64), ("fp64", SCREENED), ("mixed", MIXED)):
        g = big[name]
        q_o = np.empty_like(g["q"])
        q_o[p] = g["q"]
        blocks = oracle.fock_blocks(eb, q_o, s["r"], s["zeta"], pairs)
        scale = np.max(np.abs(g["dF"]))
        got = np.concatenate([g["dF"][eb.sh_bf[a]:eb.sh_bf[a] + blk.shape[0],
                                      eb.sh_bf[b]:eb.sh_bf[b] + blk.shape[1]].ravel()
                              for (a, b), blk in zip(pairs, blocks)])
        ref = np.concatenate([blk.ravel() for blk in blocks])
        check(got, ref, bars, scale=scale, what="dF " + name)


def test_energies(big):
    Et = big["fp64"]["E_tight"]
    assert abs(big["fp64"]["E"] - Et) <= 1e-6
    assert abs(big["mixed"]["E"] - Et) <= 1e-6
    # the near-complete pair list moves the energy by less than the screened run's bar
    assert abs(big["fine"]["E"] - big["fp64"]["E"]) <= 1e-8

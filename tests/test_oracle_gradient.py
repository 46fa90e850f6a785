"""Pins of the oracle's nuclear gradient (Eq. 14, Eq. 22) against things
other than itself: finite differences of the (separately pinned) energy
terms, translational invariance, the stationarity of Eq. 13 at the solution
of Eq. 1, and the closed form for a Gaussian charge."""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle
import workloads


def _energy_terms(w, xyz, q, index):
    """(B z)^T q, c^T q and q^T A q / (2 f) at geometry xyz with the point
    set `index` of the reference geometry (Eq. 13, term by term)."""
    s = oracle.surface(xyz, w.mol.radius, keep_all=True)
    ss = {k: s[k][index] for k in ("r", "zeta", "S", "atom")}
    eb = oracle.ExpandedBasis(w.basis, xyz)
    f = oracle.f_factor()
    EB = oracle.bz(ss, xyz, w.mol.Z) @ q
    EC = oracle.esp(eb, w.P, ss["r"], ss["zeta"]) @ q
    EA = q @ oracle.a_matrix(ss) @ q / (2.0 * f)
    return np.array([EB, EC, EA])


def _richardson(fun, xyz, h=2e-3):
    """Central differences at h and h/2 combined to O(h^4)."""
    natom = len(xyz)
    out = None
    for I in range(natom):
        for x in range(3):
            D = []
            for hh in (h, h / 2):
                xp = xyz.copy()
                xp[I, x] += hh
                xm = xyz.copy()
                xm[I, x] -= hh
                D.append((fun(xp) - fun(xm)) / (2 * hh))
            g = (4 * D[1] - D[0]) / 3
            if out is None:
                out = np.zeros(np.shape(g) + (natom, 3))
            out[..., I, x] = g
    return out


CASES = [("water", lambda: workloads.water()),
         ("cluster3_spd", lambda: workloads.small_cluster(3, 7, d_shells=True))]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    w = request.param[1]()
    r = oracle.run(w)
    s = r["surf"]
    q = r["q_lu"]
    g = oracle.gradient(r["eb"], w.P, q, s, w.mol.xyz, w.mol.Z, w.mol.radius, r["f"])
    return w, r, s, q, g


def test_each_term_matches_finite_differences(case):
    w, r, s, q, g = case
    fd = _richardson(lambda x: _energy_terms(w, x, q, s["index"]), w.mol.xyz)
    for i, k in enumerate("BCA"):
        assert np.max(np.abs(g[k])) > 1e-3
        assert np.max(np.abs(g[k] - fd[i])) <= 1e-9, (k, np.max(np.abs(g[k] - fd[i])))


def test_switching_part_is_resolved(case):
    """The diagonal (switching) part of the A term is far above the
    finite-difference error, so the FD pin sees it."""
    w, r, s, q, g = case
    f = r["f"]

    def ediag(x):
        t = oracle.surface(x, w.mol.radius, keep_all=True)
        S = t["S"][s["index"]]
        z = t["zeta"][s["index"]]
        return np.sum(q * q * z * math.sqrt(2 / math.pi) / S) / (2 * f)

    gd = _richardson(ediag, w.mol.xyz)
    assert np.max(np.abs(gd)) > 1e-4


def test_translational_invariance(case):
    w, r, s, q, g = case
    for k in "BCA":
        assert np.max(np.abs(g[k].sum(axis=0))) <= 1e-12 * max(1.0, np.max(np.abs(g[k])))


def test_total_derivative_at_the_solution():
    """With q re-solved at every geometry, dG/dR equals Eq. 14 at the
    solution (Eq. 13 is stationary in q there)."""
    w = workloads.water()
    r = oracle.run(w)
    s = r["surf"]
    f = r["f"]

    def dG(x):
        t = oracle.surface(x, w.mol.radius, keep_all=True)
        ss = {k: t[k][s["index"]] for k in ("r", "zeta", "S", "atom")}
        eb = oracle.ExpandedBasis(w.basis, x)
        A = oracle.a_matrix(ss)
        Bz = oracle.bz(ss, x, w.mol.Z)
        c = oracle.esp(eb, w.P, ss["r"], ss["zeta"])
        q = oracle.solve_lu(A, -f * (Bz + c))
        return oracle.energy(Bz, c, q, A, f)

    fd = _richardson(dG, w.mol.xyz)
    g = oracle.gradient(r["eb"], w.P, r["q_lu"], s, w.mol.xyz, w.mol.Z, w.mol.radius, f)["total"]
    assert np.max(np.abs(g - fd)) <= 1e-8 * np.max(np.abs(g))


def test_gaussian_charge_closed_form():
    """One normalised s primitive (exponent a) with P = 1 is a unit Gaussian
    charge of exponent 2a; its potential through the erf operator is
    erf(z'' d)/d with 1/z''^2 = 1/(2a) + 1/zeta_k^2, so the integral part of
    the gradient on its atom is sum_k q_k d/dR [-erf(z'' d)/d]."""
    a = 0.8
    mol = workloads._mol(["H", "O"], [[0.0, 0.0, 0.0], [1.9, 0.4, -0.3]])
    basis = workloads.Basis(np.array([0], np.int32), np.array([0], np.int32), np.array([1], np.int32),
                            np.array([a]), np.array([1.0]))
    s = oracle.surface(mol.xyz, mol.radius)
    rng = np.random.default_rng(3)
    q = np.where(s["atom"] == 1, rng.normal(size=len(s["zeta"])), 0.0)
    eb = oracle.ExpandedBasis(basis, mol.xyz)
    g = oracle.gradient_c(eb, np.ones((1, 1)), q, s)
    v = mol.xyz[0] - s["r"]                         # R_0 - r_k
    d = np.linalg.norm(v, axis=1)
    zz = 1.0 / np.sqrt(1.0 / (2 * a) + 1.0 / s["zeta"] ** 2)
    dg = 2 * zz / math.sqrt(math.pi) * np.exp(-(zz * d) ** 2) / d - erf(zz * d) / d ** 2
    ref = -(q * dg / d) @ v
    assert np.allclose(g[0], ref, rtol=1e-11, atol=1e-14)
    assert np.allclose(g[1], -ref, rtol=1e-11, atol=1e-14)

"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(closed forms, high-precision quadrature, limits, invariants).  CPU only."""
import math
import os

import numpy as np
import pytest
from scipy.special import erf

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Boys -----

def _boys_quad(m, T):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    return float(mpmath.quad(lambda u: u ** (2 * m) * mpmath.e ** (-T * u * u), [0, 1]))


@pytest.mark.parametrize("T", [0.0, 1e-9, 0.3, 2.0, 10.0, 29.99, 30.01, 45.0, 120.0])
def test_boys_against_quadrature(T):
    F = oracle.boys(8, T)
    for m in range(9):
        ref = _boys_quad(m, T)
        assert abs(F[m] - ref) <= 2e-14 * abs(ref), (m, T, F[m], ref)


@pytest.mark.parametrize("T", [1e-6, 0.7, 5.0, 17.0, 29.0])
def test_boys_f0_erf_closed_form(T):
    # F_0(T) = (1/2) sqrt(pi/T) erf(sqrt(T)); the oracle uses the series here.
    ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert abs(oracle.boys(0, T)[0] - ref) <= 1e-14 * ref


def test_boys_zero():
    F = oracle.boys(10, 0.0)
    assert np.allclose(F, [1.0 / (2 * m + 1) for m in range(11)], rtol=0, atol=1e-16)


# ------------------------------------------------- primitive integrals -----

def _gaussian_charge_potential(alpha_total, zeta, R):
    """Potential of a unit Gaussian charge of exponent alpha_total felt by a
    unit Gaussian charge of exponent zeta^2 at distance R:
    erf(z R)/R with 1/z^2 = 1/alpha + 1/zeta^2."""
    z = 1.0 / math.sqrt(1.0 / alpha_total + 1.0 / zeta ** 2)
    return math.erf(z * R) / R if R > 0 else 2.0 * z / math.sqrt(math.pi)


@pytest.mark.parametrize("a,b,zeta", [(0.8, 0.5, 1.3), (12.0, 0.3, 5.2), (1000.0, 2.0, 4.0),
                                      (0.11, 0.13, 9.0)])
def test_ss_against_gaussian_charge_closed_form(a, b, zeta):
    # Gaussian product theorem: chi_a chi_b = K exp(-p |r-P|^2); a Gaussian
    # of exponent p holds (pi/p)^{3/2} of charge.
    A = np.array([0.1, -0.2, 0.3]); B = np.array([0.9, 0.3, -0.2]); C = np.array([1.7, -0.6, 0.8])
    p = a + b
    P = (a * A + b * B) / p
    K = math.exp(-a * b / p * np.sum((A - B) ** 2))
    ref = K * (math.pi / p) ** 1.5 * _gaussian_charge_potential(p, zeta, np.linalg.norm(P - C))
    got = oracle.prim_integrals(0, a, A, 0, b, B, C, zeta)[0, 0]
    assert abs(got - ref) <= 1e-13 * abs(ref)


def test_point_charge_limit_textbook():
    # zeta -> inf: ordinary nuclear attraction, (2 pi / p) K F_0(p R_PC^2)
    # (Szabo & Ostlund, Eq. A.33, without the nuclear charge and sign).
    a, b = 0.7, 1.9
    A = np.array([0.0, 0.1, 0.0]); B = np.array([0.5, -0.3, 0.2]); C = np.array([-0.4, 0.9, 1.1])
    p = a + b
    P = (a * A + b * B) / p
    K = math.exp(-a * b / p * np.sum((A - B) ** 2))
    T = p * np.sum((P - C) ** 2)
    ref = 2 * math.pi / p * K * 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert abs(oracle.prim_integrals(0, a, A, 0, b, B, C, math.inf)[0, 0] - ref) <= 1e-14 * ref
    # and the erf operator approaches it as zeta grows
    for la, lb in [(1, 0), (1, 1), (2, 1)]:
        big = oracle.prim_integrals(la, a, A, lb, b, B, C, 1e5)
        inf = oracle.prim_integrals(la, a, A, lb, b, B, C, math.inf)
        assert np.max(np.abs(big - inf)) <= 1e-8 * np.max(np.abs(inf))


def _monomials(l):
    out = []
    for lx in range(l, -1, -1):
        for ly in range(l - lx, -1, -1):
            out.append((lx, ly, l - lx - ly))
    return out


def _quadrature_block(la, a, A, lb, b, B, C, zeta, n):
    """Brute-force 3D Gauss-Hermite quadrature of the raw primitive block."""
    p = a + b
    P = (a * A + b * B) / p
    K = math.exp(-a * b / p * np.sum((A - B) ** 2))
    s, w = np.polynomial.hermite.hermgauss(n)
    X, Y, Zc = np.meshgrid(s, s, s, indexing="ij")
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]).ravel()
    r = np.stack([X.ravel(), Y.ravel(), Zc.ravel()], 1) / math.sqrt(p) + P
    d = np.linalg.norm(r - C, axis=1)
    op = np.where(d > 1e-14, erf(zeta * np.maximum(d, 1e-300)) / np.maximum(d, 1e-300),
                  2 * zeta / math.sqrt(math.pi))
    base = W * op * K * p ** -1.5
    ra = r - A; rb = r - B
    out = np.zeros((len(_monomials(la)), len(_monomials(lb))))
    for i, ea in enumerate(_monomials(la)):
        pa = ra[:, 0] ** ea[0] * ra[:, 1] ** ea[1] * ra[:, 2] ** ea[2]
        for j, e2 in enumerate(_monomials(lb)):
            pb = rb[:, 0] ** e2[0] * rb[:, 1] ** e2[1] * rb[:, 2] ** e2[2]
            out[i, j] = np.sum(base * pa * pb)
    return out


@pytest.mark.parametrize("la,lb", [(1, 0), (0, 1), (1, 1), (2, 0), (0, 2), (2, 1), (1, 2), (2, 2),
                                   (3, 0), (3, 1)])
def test_all_classes_against_brute_force_quadrature(la, lb):
    a, b, zeta = 0.8, 0.5, 1.3
    A = np.array([0.1, -0.2, 0.3]); B = np.array([0.9, 0.3, -0.2]); C = np.array([1.7, -0.6, 0.8])
    got = oracle.prim_integrals(la, a, A, lb, b, B, C, zeta)
    q1 = _quadrature_block(la, a, A, lb, b, B, C, zeta, 40)
    q2 = _quadrature_block(la, a, A, lb, b, B, C, zeta, 56)
    scale = np.max(np.abs(q2))
    assert np.max(np.abs(q1 - q2)) <= 1e-11 * scale      # quadrature converged
    assert np.max(np.abs(got - q2)) <= 1e-10 * scale, np.max(np.abs(got - q2)) / scale


def _fd(fun, x, i, h=1e-4):
    xp = x.copy(); xm = x.copy()
    xp[i] += h; xm[i] -= h
    return (fun(xp) - fun(xm)) / (2 * h)


def test_center_derivatives_raise_angular_momentum():
    # d/dA_i of x_A^a exp(-alpha r_A^2) = 2 alpha x_A^{a+1_i} - a_i x_A^{a-1_i}:
    # finite differences of lower classes give higher classes.
    a, b, zeta = 0.9, 1.4, 3.1
    A = np.array([0.2, -0.1, 0.4]); B = np.array([-0.6, 0.5, 0.1]); C = np.array([0.7, 1.2, -0.9])
    I = lambda la, AA, lb, BB: oracle.prim_integrals(la, a, AA, lb, b, BB, C, zeta)
    ps = I(1, A, 0, B); ds = I(2, A, 0, B); sd = I(0, A, 2, B); pp = I(1, A, 1, B)
    ss = I(0, A, 0, B)[0, 0]
    dmap = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 1): 3, (1, 2): 4, (2, 2): 5}
    for i in range(3):
        # d/dA_i [s|s] = 2a [p_i|s]
        g = _fd(lambda X: I(0, X, 0, B)[0, 0], A, i)
        assert abs(g - 2 * a * ps[i, 0]) <= 1e-7 * abs(ps).max()
        # d/dB_i [s|s] = 2b [s|p_i]
        g = _fd(lambda X: I(0, A, 0, X)[0, 0], B, i)
        assert abs(g - 2 * b * I(0, A, 1, B)[0, i]) <= 1e-7 * abs(ps).max()
        for j in range(3):
            # d/dA_i [p_j|s] = 2a [d_ij|s] - delta_ij [s|s]
            g = _fd(lambda X: I(1, X, 0, B)[j, 0], A, i)
            ref = 2 * a * ds[dmap[tuple(sorted((i, j)))], 0] - (ss if i == j else 0.0)
            assert abs(g - ref) <= 1e-7 * abs(ds).max()
            # d/dB_i [s|p_j] = 2b [s|d_ij] - delta_ij [s|s]
            g = _fd(lambda X: I(0, A, 1, X)[0, j], B, i)
            ref = 2 * b * sd[0, dmap[tuple(sorted((i, j)))]] - (ss if i == j else 0.0)
            assert abs(g - ref) <= 1e-7 * abs(sd).max()
            # d/dB_i [p_j|s] = 2b [p_j|p_i]
            g = _fd(lambda X: I(1, A, 0, X)[j, 0], B, i)
            assert abs(g - 2 * b * pp[j, i]) <= 1e-7 * abs(pp).max()


def test_translation_invariance_of_derivatives():
    # moving A, B and C together leaves the integral unchanged
    a, b, zeta = 0.6, 2.2, 4.4
    A = np.array([0.2, -0.1, 0.4]); B = np.array([-0.6, 0.5, 0.1]); C = np.array([0.7, 1.2, -0.9])
    for la, lb in [(1, 1), (2, 1), (2, 2)]:
        base = oracle.prim_integrals(la, a, A, lb, b, B, C, zeta)
        t = np.array([0.37, -1.1, 2.3])
        moved = oracle.prim_integrals(la, a, A + t, lb, b, B + t, C + t, zeta)
        assert np.max(np.abs(base - moved)) <= 1e-13 * np.max(np.abs(base))


def test_swap_symmetry():
    a, b, zeta = 0.6, 2.2, 4.4
    A = np.array([0.2, -0.1, 0.4]); B = np.array([-0.6, 0.5, 0.1]); C = np.array([0.7, 1.2, -0.9])
    for la, lb in [(1, 0), (2, 0), (2, 1), (2, 2)]:
        ab = oracle.prim_integrals(la, a, A, lb, b, B, C, zeta)
        ba = oracle.prim_integrals(lb, b, B, la, a, A, C, zeta)
        assert np.max(np.abs(ab - ba.T)) <= 1e-13 * np.max(np.abs(ab))


def _rotation(seed):
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.standard_normal((3, 3)))
    return Q * np.sign(np.diag(R))


def test_rotation_covariance():
    # raw p components transform as a vector, raw d components (monomials
    # x_i x_j) as a symmetric tensor.
    a, b, zeta = 0.6, 1.2, 2.4
    A = np.array([0.2, -0.1, 0.4]); B = np.array([-0.6, 0.5, 0.1]); C = np.array([0.7, 1.2, -0.9])
    Rm = _rotation(7)
    pp = oracle.prim_integrals(1, a, A, 1, b, B, C, zeta)
    pp_r = oracle.prim_integrals(1, a, Rm @ A, 1, b, Rm @ B, Rm @ C, zeta)
    assert np.max(np.abs(pp_r - Rm @ pp @ Rm.T)) <= 1e-12 * np.max(np.abs(pp))
    ds = oracle.prim_integrals(2, a, A, 0, b, B, C, zeta)[:, 0]
    ds_r = oracle.prim_integrals(2, a, Rm @ A, 0, b, Rm @ B, Rm @ C, zeta)[:, 0]
    idx = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 1): 3, (1, 2): 4, (2, 2): 5}
    T = np.zeros((3, 3))
    for (i, j), k in idx.items():
        T[i, j] = T[j, i] = ds[k]
    Tr = Rm @ T @ Rm.T
    for (i, j), k in idx.items():
        assert abs(ds_r[k] - Tr[i, j]) <= 1e-12 * np.max(np.abs(ds))


def test_normalisation_unit_self_overlap():
    # small-zeta limit: erf(zeta r)/r -> 2 zeta / sqrt(pi), so the integral
    # becomes 2 zeta / sqrt(pi) times the overlap; a normalised component
    # has unit self-overlap.
    zeta = 1e-5
    A = np.array([0.3, 0.2, -0.1])
    for l in (0, 1, 2):
        for a in (0.2, 3.0, 700.0):
            blk = oracle.prim_integrals(l, a, A, l, a, A, A, zeta)
            for i, e in enumerate(_monomials(l)):
                S = blk[i, i] * math.sqrt(math.pi) / (2 * zeta)
                assert abs(oracle.prim_norm(a, e) ** 2 * S - 1.0) < 1e-8


# ----------------------------------------------------- contractions -----

def _one_s_shell_basis(alpha_half):
    return workloads.Basis(np.array([0], np.int32), np.array([0], np.int32), np.array([1], np.int32),
                           np.array([alpha_half]), np.array([1.0]))


def test_esp_of_gaussian_density_closed_form():
    # One normalised s primitive of exponent alpha/2 and P = [[1]]: the
    # density is a unit Gaussian charge of exponent alpha, so
    # c_k = -erf(z'' r)/r with 1/z''^2 = 1/alpha + 1/zeta_k^2 (Eq. 5, Eq. 6).
    alpha = 1.7
    eb = oracle.ExpandedBasis(_one_s_shell_basis(alpha / 2), np.zeros((1, 3)))
    rng = np.random.default_rng(3)
    pts = rng.normal(size=(20, 3)) * 2.0
    zeta = rng.uniform(2.0, 8.0, size=20)
    c = oracle.esp(eb, np.array([[1.0]]), pts, zeta)
    for k in range(20):
        ref = -_gaussian_charge_potential(alpha, zeta[k], np.linalg.norm(pts[k]))
        assert abs(c[k] - ref) <= 1e-13 * abs(ref)


def test_esp_fock_duality_and_fock_symmetry():
    # q^T c = <P, dF>_F for any q and any symmetric P (both contract the
    # same L, Eq. 5 and Eq. 10); dF is symmetric.
    w = workloads.small_cluster(4, seed=11, d_shells=True)
    eb = oracle.ExpandedBasis(w.basis, w.mol.xyz)
    s = oracle.surface(w.mol.xyz, w.mol.radius, n=26)
    rng = np.random.default_rng(5)
    q = rng.normal(size=len(s["zeta"]))
    c = oracle.esp(eb, w.P, s["r"], s["zeta"])
    F = oracle.fock(eb, q, s["r"], s["zeta"])
    assert np.max(np.abs(F - F.T)) <= 1e-13 * np.max(np.abs(F))
    lhs = q @ c
    rhs = np.sum(w.P * F)
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(q) @ np.abs(c))


def test_esp_linear_in_density_and_translation_invariant():
    w = workloads.small_cluster(3, seed=2)
    eb = oracle.ExpandedBasis(w.basis, w.mol.xyz)
    s = oracle.surface(w.mol.xyz, w.mol.radius, n=14)
    c1 = oracle.esp(eb, w.P, s["r"], s["zeta"])
    c2 = oracle.esp(eb, 2.5 * w.P, s["r"], s["zeta"])
    assert np.max(np.abs(c2 - 2.5 * c1)) <= 1e-13 * np.max(np.abs(c1))
    t = np.array([3.0, -1.0, 0.5])
    eb2 = oracle.ExpandedBasis(w.basis, w.mol.xyz + t)
    c3 = oracle.esp(eb2, w.P, s["r"] + t, s["zeta"])
    assert np.max(np.abs(c3 - c1)) <= 1e-11 * np.max(np.abs(c1))


# ------------------------------------------------------------ surface -----

def test_fibonacci_points_and_weights():
    u = oracle.fibonacci_directions(110)
    assert np.allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-15)
    assert abs(u.sum(0)).max() < 0.05                    # nearly balanced
    s = oracle.surface(np.zeros((1, 3)), np.array([2.7]), n=110)
    assert len(s["zeta"]) == 110 and np.all(s["S"] == 1.0)
    assert abs(110 * s["w"] - 4 * math.pi) < 1e-13
    assert np.allclose(np.linalg.norm(s["r"], axis=1), 2.7, atol=1e-14)
    # Eq. 7
    assert np.allclose(s["zeta"], 4.9 / (2.7 * math.sqrt(4 * math.pi / 110)), rtol=1e-15)


def test_switching_factor_against_literal_eq9():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 200
    rng = np.random.default_rng(1)
    for _ in range(200):
        z = rng.uniform(2, 9); RJ = rng.uniform(2, 4); d = rng.uniform(0.0, 2.5 * RJ)
        lit = 1 - (mpmath.erf(mpmath.mpf(z) * (mpmath.mpf(RJ) - mpmath.mpf(d)))
                   + mpmath.erf(mpmath.mpf(z) * (mpmath.mpf(RJ) + mpmath.mpf(d)))) / 2
        got = oracle.switching_factor(z, d, RJ)
        if lit < 1e-30:
            # far below the 1e-8 drop threshold: only the drop decision matters
            assert got < 1e-20
            continue
        # erfc's tail has condition number ~2x^2: allow for the rounding of its argument
        x1 = z * (RJ - d)
        tol = 2e-14 + 4 * max(x1, 0.0) ** 2 * 2.2e-16
        assert abs(got - float(lit)) <= tol * float(lit) + 1e-300, (z, RJ, d, got, lit)


def test_switching_limits_and_drop():
    # far atoms do not switch; points buried deep in another sphere vanish
    for sep in (40.0, 8.0, 3.0, 1.0):
        xyz = np.array([[0, 0, 0], [sep, 0, 0]], float)
        s = oracle.surface(xyz, np.array([2.5, 2.5]), n=110)
        if sep == 40.0:
            assert len(s["S"]) == 220 and np.all(np.abs(s["S"] - 1) < 1e-15)
        assert np.all(s["S"] >= 1e-8) and np.all(s["S"] <= 1.0)
    few = len(oracle.surface(np.array([[0, 0, 0], [1.0, 0, 0]], float), np.array([2.5, 2.5]))["S"])
    many = len(oracle.surface(np.array([[0, 0, 0], [4.0, 0, 0]], float), np.array([2.5, 2.5]))["S"])
    assert few < many < 220


def test_water_surface_size():
    # the 3-atom workload keeps about 250 points (M = 252 with these radii)
    w = workloads.config(0)
    s = oracle.surface(w.mol.xyz, w.mol.radius)
    assert len(s["S"]) == 252


# ----------------------------------------------------- A, solve, energy -----

@pytest.mark.parametrize("n", [110, 302])
def test_single_sphere_conductor_gauss_and_born(n):
    # Unit point charge at the centre of one sphere: the induced charge
    # approaches -f (Gauss's law, Eq. 1 and the remark on k = 0) and the
    # energy approaches the Born value -f / (2R).  This pins the reading of
    # Eq. 3's constant: sqrt(2/pi) passes, the printed 1/sqrt(2 pi) does not.
    R = 2.7
    s = oracle.surface(np.zeros((1, 3)), np.array([R]), n=n)
    f = oracle.f_factor()
    Bz = oracle.bz(s, np.zeros((1, 3)), np.array([1.0]))
    for reading, ok in (("sqrt(2/pi)", True), ("1/sqrt(2pi)", False)):
        A = oracle.a_matrix(s, diag_reading=reading)
        q = oracle.solve_lu(A, -f * Bz)
        E = oracle.energy(Bz, np.zeros_like(Bz), q, A, f)
        gauss = abs(q.sum() / (-f) - 1.0)
        born = abs(E / (-f / (2 * R)) - 1.0)
        if ok:
            assert gauss < 1e-3 and born < 1e-3, (gauss, born)
        else:
            assert gauss > 2e-2


def test_a_is_spd_and_lu_residual():
    w = workloads.config(0)
    s = oracle.surface(w.mol.xyz, w.mol.radius)
    A = oracle.a_matrix(s)
    assert np.max(np.abs(A - A.T)) == 0.0
    np.linalg.cholesky(A)
    # buried points make the diagonal span many orders of magnitude (Section 4b)
    d = np.diag(A)
    assert d.max() / d.min() > 1e5
    b = np.random.default_rng(0).normal(size=len(d))
    x = oracle.solve_lu(A, b)
    assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b) * np.linalg.cond(A) * 1e-6


def test_preconditioning_needed_for_ill_conditioned_a():
    # Section 4b: buried points make A ill-conditioned; plain CG stalls where
    # Jacobi-preconditioned CG converges.
    w = workloads.config(0)
    s = oracle.surface(w.mol.xyz, w.mol.radius)
    A = oracle.a_matrix(s)
    b = np.random.default_rng(1).normal(size=len(s["S"]))
    _, it_j, ok_j, _ = oracle.pcg(A, b, 1e-8, oracle.Preconditioner(A, "jacobi"), max_iter=300)
    _, it_n, ok_n, _ = oracle.pcg(A, b, 1e-8, oracle.Preconditioner(A, "none"), max_iter=300)
    assert ok_j and not ok_n


@pytest.mark.parametrize("kind", ["jacobi", "rbj"])
def test_pcg_converges_to_lu(kind):
    w = workloads.config(0)
    s = oracle.surface(w.mol.xyz, w.mol.radius)
    A = oracle.a_matrix(s)
    b = np.random.default_rng(1).normal(size=len(s["S"]))
    x_lu = oracle.solve_lu(A, b)
    for delta in (1e-4, 1e-8):
        pc = oracle.Preconditioner(A, kind, l=40, seed=9)
        x, it, ok, rn = oracle.pcg(A, b, delta, pc)
        assert ok and rn < delta
        assert np.linalg.norm(A @ x - b) < 10 * delta
        lam_min = np.linalg.eigvalsh(A)[0]
        assert np.linalg.norm(x - x_lu) <= 10 * delta / lam_min


def test_rbj_full_block_converges_in_one_step():
    # Section 4b-ii: with block size M the preconditioner is the exact
    # inverse and CG converges in one step.
    w = workloads.config(0)
    s = oracle.surface(w.mol.xyz, w.mol.radius)
    A = oracle.a_matrix(s)
    b = np.random.default_rng(2).normal(size=len(s["S"]))
    pc = oracle.Preconditioner(A, "rbj", l=len(b), seed=3)
    x, it, ok, rn = oracle.pcg(A, b, 1e-8, pc)
    assert ok and it == 1


def test_rbj_partition_rules():
    w = workloads.config(0)
    s = oracle.surface(w.mol.xyz, w.mol.radius)
    A = oracle.a_matrix(s)
    M = A.shape[0]
    l = 37
    blocks = oracle.rbj_blocks(A, l, seed=123)
    allidx = np.concatenate(blocks)
    assert sorted(allidx.tolist()) == list(range(M))
    assert all(len(b) == l for b in blocks[:-1]) and 0 < len(blocks[-1]) <= l
    unassigned = np.ones(M, bool)
    for j, b in enumerate(blocks):
        U = np.nonzero(unassigned)[0]
        r = oracle.splitmix64(123, j)
        assert b[0] == U[((r >> 32) * len(U)) >> 32]       # the drawn pivot leads its block
        rest = np.setdiff1d(U, b)
        if len(rest):
            assert np.abs(A[b[0], b[1:]]).min() >= np.abs(A[b[0], rest]).max()
        unassigned[b] = False


def test_rbj_more_blocks_not_better_than_fewer_on_average():
    # Section 4b-ii: larger blocks keep more of A, so CG needs fewer steps.
    w = workloads.small_cluster(12, seed=4)
    s = oracle.surface(w.mol.xyz, w.mol.radius)
    A = oracle.a_matrix(s)
    b = np.random.default_rng(0).normal(size=A.shape[0])
    its = {}
    for l in (10, 100, 400):
        its[l] = np.mean([oracle.pcg(A, b, 1e-6, oracle.Preconditioner(A, "rbj", l, sd))[1]
                          for sd in range(4)])
    assert its[10] >= its[100] >= its[400]


def test_splitmix64_published_vectors():
    vals = [int(x) for x in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if x.strip() and not x.startswith("#")]
    assert [oracle.splitmix64(1234567, j) for j in range(5)] == vals


def test_dynamic_delta_eq21():
    params = {}
    for line in open(os.path.join(GOLDEN, "paper_parameters.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()[:2]
            params[k] = float(v)
    assert oracle.dynamic_delta(None) == params["delta_first"]
    assert oracle.dynamic_delta(-1.0) == 1.0
    for e in (1e-2, 1e-4, 1e-6):
        d = oracle.dynamic_delta(e)
        err = params["err_coef"] * d ** params["err_pow"]            # Eq. 21
        assert abs(err / (params["delta_safety"] * e) - 1) < 1e-12
    assert oracle.dynamic_delta(1e30) == 1.0 and oracle.dynamic_delta(1e-40) == 1e-10
    assert oracle.f_factor(params["epsilon"], params["k_cosmo"]) == (78.39 - 1) / 78.39


def test_energy_identity_at_solution():
    # With q = -f A^-1 V (V = Bz + c), Eq. 13 equals V^T q / 2 and is negative.
    o = oracle.run(workloads.config(0), delta=1e-12)
    V = o["Bz"] + o["c"]
    E = oracle.energy(o["Bz"], o["c"], o["q_lu"], o["A"], o["f"])
    assert abs(E - 0.5 * V @ o["q_lu"]) <= 1e-12 * abs(E)
    assert E < 0
    assert abs(o["E"] - E) < 1e-9


def test_gauss_law_compact_molecule():
    # Compact basis (tight exponents), fine grid: the induced charge tends to
    # -f (Z - N_el) with N_el = tr(P S); S from the small-zeta limit of the
    # integrals (erf(zeta r)/r -> 2 zeta / sqrt(pi)).
    mol = workloads._mol(["O", "H", "H"], [[0, 0, 0], [1.43, 1.11, 0], [-1.43, 1.11, 0]])
    rng = np.random.default_rng(0)
    basis = workloads.make_basis(mol, {"O": [(0, 3, (2.0, 60.0)), (-1, 3, (1.5, 20.0))],
                                       "H": [(0, 3, (1.5, 30.0))]}, rng)
    P = workloads.make_density(basis, mol.xyz, 5, rng)
    eb = oracle.ExpandedBasis(basis, mol.xyz)
    zs = 1e-5
    S = np.zeros((eb.nbf, eb.nbf))
    for a in range(eb.nshell):
        for b in range(eb.nshell):
            blk = eb.shell_block(a, b, eb.xyz[eb.sh_atom[a]], zs) * math.sqrt(math.pi) / (2 * zs)
            S[eb.sh_bf[a]:eb.sh_bf[a] + blk.shape[0], eb.sh_bf[b]:eb.sh_bf[b] + blk.shape[1]] = blk
    Nel = np.sum(P * S)
    s = oracle.surface(mol.xyz, mol.radius, n=590)
    A = oracle.a_matrix(s)
    V = oracle.bz(s, mol.xyz, mol.Z) + oracle.esp(eb, P, s["r"], s["zeta"])
    f = oracle.f_factor()
    q = oracle.solve_lu(A, -f * V)
    Q = mol.Z.sum() - Nel
    assert abs(q.sum() - (-f * Q)) < 0.02 * max(1.0, abs(Q)), (q.sum(), -f * Q)


def test_octree_partition_rules():
    """The octree leaves partition the points, respect the capacity, hold
    only points of their own box, and reduce to one block when it fits."""
    rng = np.random.default_rng(9)
    r = rng.normal(size=(3000, 3)) * np.array([3.0, 1.0, 0.5])
    blocks = oracle.octree_blocks(r, 200)
    allidx = np.sort(np.concatenate(blocks))
    assert np.array_equal(allidx, np.arange(len(r)))
    assert max(len(b) for b in blocks) <= 200
    # every leaf lies in an axis-aligned box that no other leaf's points enter
    for b in blocks[:20]:
        lo, hi = r[b].min(axis=0), r[b].max(axis=0)
        inside = np.all((r >= lo) & (r <= hi), axis=1)
        assert set(np.nonzero(inside)[0]) <= set(b.tolist())
    assert len(oracle.octree_blocks(r, 3000)) == 1
    # block Jacobi on a block-diagonal SPD matrix with the octree blocks is exact
    A = np.zeros((len(r), len(r)))
    for b in blocks:
        B = rng.normal(size=(len(b), len(b)))
        A[np.ix_(b, b)] = B @ B.T + len(b) * np.eye(len(b))
    pc = oracle.Preconditioner(A, "octree", 200, points=r)
    x, it, ok, rn = oracle.pcg(A, rng.normal(size=len(r)), 1e-10, pc)
    assert ok and it == 1

"""ORACLE -- test infrastructure only.

A plain, slow, FP64 CPU statement of the C-PCM/ISWIG hot path of Liu,
Luehr, Kulik & Martinez (the paper).  Only the tests, the package's smoke
check and the benchmark's CPU-baseline leg import it.  The CUDA library
shares no code with it and never calls it; it shares nothing with the
library but the seeded input generators in ``workloads``.

Contents, each following the passage cited:
  * surface(): Lebedev-sphere stand-in (Fibonacci points, equal weights),
    Gaussian exponents (Eq. 7) and ISWIG switching (Eq. 9), dropping points
    whose switching value is below 1e-8 (Section 3).
  * a_matrix(), bz(): Eq. 2, Eq. 3, Eq. 8 and Eq. 4.
  * esp(), fock(): Eq. 5, Eq. 6, Eq. 10, Eq. 12 via the C part (integrals.c).
  * solve_lu(): dense LU solve of Eq. 1 (LAPACK via numpy).
  * pcg(): CG / Jacobi-PCG / randomized block-Jacobi PCG with the residual
    test of Eq. 20 (Section 4b), the RBJ permutation of Section 4b-ii, and
    the octree block-Jacobi the paper compares RBJ with.
  * dynamic_delta(): Eq. 21 and the rule that follows it.
  * energy(): Eq. 13.
  * gradient_bz(), gradient_a(), gradient_c(), gradient(): the nuclear
    gradient of Eq. 13 at fixed P and q (Eq. 14, Eq. 22), with the points
    moving with their atoms and the switching function of Eq. 9
    differentiated.

Readings of the paper where it is silent or garbled (shared with the CUDA
path as specification, not as code):
  * Eq. 3 is read as A_kk = zeta_k sqrt(2/pi) / S_k, the r -> 0 limit of
    Eq. 2 with zeta'_kk = zeta_k / sqrt(2).
  * Lebedev points are replaced by a Fibonacci sphere with equal weights
    w = 4 pi / n, i.e. the weights of a sphere sum to 4 pi.
  * The CG stop test is the Euclidean norm of r = A x - b below delta.
  * RBJ: the pivot is drawn uniformly from the unassigned indices with a
    counter-based splitmix64 stream; its block is the pivot followed by
    the l - 1 unassigned indices of largest |A_kj| (ties to the lower
    index); the last block may be short.
  * Dynamic threshold: delta = (1e-3 e_prev / 0.01)^(1/1.07), clamped to
    [1e-10, 1]; delta = 1 when there is no previous DIIS error.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
from scipy.special import erf, erfc

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_boys.argtypes = [ctypes.c_int, ctypes.c_double, dp]
        L.oracle_prim.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_int, ctypes.c_double,
                                  dp, dp, ctypes.c_double, dp]
        L.oracle_norm.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.oracle_norm.restype = ctypes.c_double
        L.oracle_shell_block.argtypes = [ip, ip, ip, ip, dp, dp, dp, ctypes.c_int, ctypes.c_int, dp,
                                         ctypes.c_double, dp]
        L.oracle_esp.argtypes = [ctypes.c_int, ip, ip, ip, ip, ip, dp, dp, dp, ctypes.c_int, dp,
                                 ctypes.c_int, dp, dp, dp]
        L.oracle_fock_pairs.argtypes = [ip, ip, ip, ip, dp, dp, dp, ctypes.c_int, dp, dp, dp,
                                        ctypes.c_int, ip, ip, ctypes.POINTER(ctypes.c_long), dp]
        L.oracle_grad_c.argtypes = [ctypes.c_int, ip, ip, ip, ip, ip, dp, dp, dp, ctypes.c_int, dp,
                                    ctypes.c_int, dp, dp, dp, ip, ctypes.c_int, dp]
        _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32).ctypes.data_as(ctypes.POINTER(ctypes.c_int))


# --------------------------------------------------------------------------
# Primitive-level helpers (used by the pins)
# --------------------------------------------------------------------------

def boys(mmax: int, T: float) -> np.ndarray:
    F = np.zeros(mmax + 1)
    lib().oracle_boys(mmax, float(T), _d_out(F))
    return F


def _d_out(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def cart_exponents(l: int):
    """Cartesian exponents in the order x^l, x^(l-1) y, ..., z^l."""
    out = []
    for lx in range(l, -1, -1):
        for ly in range(l - lx, -1, -1):
            out.append((lx, ly, l - lx - ly))
    return out


def prim_integrals(la, alpha, A, lb, beta, B, C, zeta):
    """Raw (unnormalised) Cartesian primitive block [chi_a|J|chi_b]
    (ncart(la), ncart(lb)); zeta = inf gives the point charge."""
    out = np.zeros(ncart(la) * ncart(lb))
    A = np.asarray(A, np.float64); B = np.asarray(B, np.float64); C = np.asarray(C, np.float64)
    lib().oracle_prim(la, alpha, _d(A), lb, beta, _d(B), _d(C), float(zeta), _d_out(out))
    return out.reshape(ncart(la), ncart(lb))


def prim_norm(a, e):
    return lib().oracle_norm(float(a), int(e[0]), int(e[1]), int(e[2]))


# --------------------------------------------------------------------------
# Basis expansion (sp shells -> an s and a p shell with shared exponents)
# --------------------------------------------------------------------------

class ExpandedBasis:
    def __init__(self, basis, xyz):
        sa, sl, sn, so, sbf = [], [], [], [], []
        ex, co = [], []
        off = 0
        cpos = 0
        bf = 0
        for s in range(len(basis.shell_l)):
            l = int(basis.shell_l[s]); n = int(basis.shell_nprim[s])
            e = basis.exps[off:off + n]
            if l == -1:
                parts = [(0, basis.coefs[cpos:cpos + n]), (1, basis.coefs[cpos + n:cpos + 2 * n])]
                cpos += 2 * n
            else:
                parts = [(l, basis.coefs[cpos:cpos + n])]
                cpos += n
            for (ll, c) in parts:
                sa.append(int(basis.shell_atom[s])); sl.append(ll); sn.append(n)
                so.append(len(ex)); sbf.append(bf)
                ex.extend(e); co.extend(c)
                bf += ncart(ll)
            off += n
        self.sh_atom = np.array(sa, np.int32)
        self.sh_l = np.array(sl, np.int32)
        self.sh_nprim = np.array(sn, np.int32)
        self.sh_off = np.array(so, np.int32)
        self.sh_bf = np.array(sbf, np.int32)
        self.exps = np.array(ex, np.float64)
        self.coefs = np.array(co, np.float64)
        self.xyz = np.ascontiguousarray(xyz, np.float64)
        self.nbf = bf
        self.nshell = len(sl)

    def shell_block(self, sa, sb, C, zeta):
        na, nb = ncart(self.sh_l[sa]), ncart(self.sh_l[sb])
        out = np.zeros(na * nb)
        lib().oracle_shell_block(_i(self.sh_atom), _i(self.sh_l), _i(self.sh_nprim), _i(self.sh_off),
                                 _d(self.exps), _d(self.coefs), _d(self.xyz), int(sa), int(sb),
                                 _d(np.asarray(C, np.float64)), float(zeta), _d_out(out))
        return out.reshape(na, nb)


# --------------------------------------------------------------------------
# Surface (Eq. 7, Eq. 9, Section 3)
# --------------------------------------------------------------------------

def fibonacci_directions(n: int) -> np.ndarray:
    """Unit vectors u_i, i = 0..n-1: z_i = 1 - (2i+1)/n, phi_i = i pi (3 - sqrt 5)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    s = np.sqrt(1.0 - z * z)
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def switching_factor(zeta_k, d, RJ):
    """S_wf of Eq. 9: 1 - (erf(zeta (R_J - d)) + erf(zeta (R_J + d))) / 2,
    written with erfc = 1 - erf as (erfc(zeta (R_J - d)) + erfc(zeta (R_J + d))) / 2
    so that small values keep their relative precision."""
    return 0.5 * (erfc(zeta_k * (RJ - d)) + erfc(zeta_k * (RJ + d)))


def surface(xyz, radius, n=110, zeta=4.9, drop=1e-8, keep_all=False):
    """Points, exponents and switching values of the ISWIG cavity surface.

    Returns dict with r (M,3), zeta (M,), S (M,), atom (M,), index (M,)
    (the candidate index I*n + i), in atom-major order, after dropping the
    points whose switching value is below `drop` (Section 3)."""
    xyz = np.asarray(xyz, np.float64)
    radius = np.asarray(radius, np.float64)
    natom = len(xyz)
    u = fibonacci_directions(n)
    w = 4.0 * math.pi / n
    r = (xyz[:, None, :] + radius[:, None, None] * u[None, :, :]).reshape(-1, 3)
    atom = np.repeat(np.arange(natom), n)
    zk = zeta / (radius[atom] * math.sqrt(w))                      # Eq. 7
    S = np.ones(natom * n)
    for J in range(natom):                                          # Eq. 9
        d = np.linalg.norm(r - xyz[J], axis=1)
        f = switching_factor(zk, d, radius[J])
        S = np.where(atom == J, S, S * f)
    keep = np.ones_like(S, dtype=bool) if keep_all else (S >= drop)
    idx = np.nonzero(keep)[0]
    return {"r": r[idx], "zeta": zk[idx], "S": S[idx], "atom": atom[idx], "index": idx,
            "w": w}


# --------------------------------------------------------------------------
# A, B z (Eq. 2, Eq. 3, Eq. 4, Eq. 8)
# --------------------------------------------------------------------------

def a_matrix(surf, diag_reading="sqrt(2/pi)"):
    r = surf["r"]; z = surf["zeta"]; S = surf["S"]
    M = len(z)
    A = np.empty((M, M))
    for k0 in range(0, M, 2048):
        k1 = min(M, k0 + 2048)
        d = np.linalg.norm(r[k0:k1, None, :] - r[None, :, :], axis=2)
        zp = z[k0:k1, None] * z[None, :] / np.sqrt(z[k0:k1, None] ** 2 + z[None, :] ** 2)   # Eq. 8
        with np.errstate(divide="ignore", invalid="ignore"):
            A[k0:k1] = erf(zp * d) / d                                                     # Eq. 2
    if diag_reading == "sqrt(2/pi)":
        diag = z * math.sqrt(2.0 / math.pi) / S                                           # Eq. 3 (read)
    elif diag_reading == "1/sqrt(2pi)":
        diag = z / math.sqrt(2.0 * math.pi) / S                                           # Eq. 3 (literal)
    else:
        raise ValueError(diag_reading)
    A[np.arange(M), np.arange(M)] = diag
    return A


def bz(surf, xyz, Z):
    """(B z)_k = sum_J Z_J erf(zeta_k |r_k - R_J|) / |r_k - R_J| (Eq. 4)."""
    r = surf["r"]; z = surf["zeta"]
    d = np.linalg.norm(r[:, None, :] - np.asarray(xyz)[None, :, :], axis=2)
    return (np.asarray(Z)[None, :] * erf(z[:, None] * d) / d).sum(axis=1)


# --------------------------------------------------------------------------
# ESP and Fock (Eq. 5, Eq. 6, Eq. 10, Eq. 12)
# --------------------------------------------------------------------------

def esp(eb: ExpandedBasis, P, pts, zeta):
    """c_k = -sum_{mu nu} P_{mu nu} (mu|J_k|nu) at the given points."""
    pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
    zeta = np.ascontiguousarray(zeta, np.float64)
    out = np.zeros(len(pts))
    P = np.ascontiguousarray(P, np.float64)
    lib().oracle_esp(eb.nshell, _i(eb.sh_atom), _i(eb.sh_l), _i(eb.sh_nprim), _i(eb.sh_off),
                     _i(eb.sh_bf), _d(eb.exps), _d(eb.coefs), _d(eb.xyz), eb.nbf, _d(P),
                     len(pts), _d(pts), _d(zeta), _d_out(out))
    return out


def fock_blocks(eb: ExpandedBasis, q, pts, zeta, pairs):
    """dF blocks for the listed (expanded) shell pairs: -sum_k q_k (A|J_k|B)."""
    pairs = np.asarray(pairs, np.int32).reshape(-1, 2)
    sizes = [ncart(eb.sh_l[a]) * ncart(eb.sh_l[b]) for a, b in pairs]
    off = np.zeros(len(pairs), np.int64)
    if len(pairs):
        off[1:] = np.cumsum(sizes)[:-1]
    out = np.zeros(int(sum(sizes)))
    pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
    lib().oracle_fock_pairs(_i(eb.sh_atom), _i(eb.sh_l), _i(eb.sh_nprim), _i(eb.sh_off),
                            _d(eb.exps), _d(eb.coefs), _d(eb.xyz), len(pts), _d(pts),
                            _d(np.asarray(zeta, np.float64)), _d(np.asarray(q, np.float64)),
                            len(pairs), _i(pairs[:, 0]), _i(pairs[:, 1]),
                            np.ascontiguousarray(off, dtype=np.int64).ctypes.data_as(
                                ctypes.POINTER(ctypes.c_long)), _d_out(out))
    blocks = []
    for (a, b), o, s in zip(pairs, off, sizes):
        blocks.append(out[o:o + s].reshape(ncart(eb.sh_l[a]), ncart(eb.sh_l[b])))
    return blocks


def fock(eb: ExpandedBasis, q, pts, zeta):
    """Full dF_{mu nu} = sum_k q_k L^k_{mu nu} (Eq. 10), nbf x nbf."""
    pairs = [(a, b) for a in range(eb.nshell) for b in range(a, eb.nshell)]
    blocks = fock_blocks(eb, q, pts, zeta, pairs)
    F = np.zeros((eb.nbf, eb.nbf))
    for (a, b), blk in zip(pairs, blocks):
        ia, ib = eb.sh_bf[a], eb.sh_bf[b]
        F[ia:ia + blk.shape[0], ib:ib + blk.shape[1]] = blk
        F[ib:ib + blk.shape[1], ia:ia + blk.shape[0]] = blk.T
    return F


# --------------------------------------------------------------------------
# Solvers (Eq. 1, Eq. 20, Section 4b)
# --------------------------------------------------------------------------

def f_factor(eps=78.39, k=0.0):
    """f = (eps - 1) / (eps + k) (Eq. 1)."""
    return (eps - 1.0) / (eps + k)


def solve_lu(A, rhs):
    return np.linalg.solve(A, rhs)


_MASK64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(seed: int, j: int) -> int:
    """Output j (0-based) of the splitmix64 generator seeded with `seed`
    (Steele, Lea & Flood 2014): state_j = seed + (j+1) * golden, then the
    published mix."""
    z = (seed + (j + 1) * _GOLDEN) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def rbj_blocks(A, l, seed):
    """Randomized block-Jacobi partition (Section 4b-ii): list of index
    arrays.  Draw j picks position floor((r_j >> 32) * n_unassigned / 2^32)
    in the ascending list of unassigned indices."""
    M = A.shape[0]
    unassigned = np.ones(M, dtype=bool)
    blocks = []
    j = 0
    while unassigned.any():
        U = np.nonzero(unassigned)[0]
        r = splitmix64(seed, j)
        j += 1
        pos = ((r >> 32) * len(U)) >> 32
        k = int(U[pos])
        others = U[U != k]
        mag = np.abs(A[k, others])
        order = np.lexsort((others, -mag))        # descending |A_kj|, ties -> lower index
        blk = np.concatenate([[k], others[order[:l - 1]]]).astype(np.int64)
        blocks.append(blk)
        unassigned[blk] = False
    return blocks


def octree_blocks(r, leaf):
    """Octree partition of the points r (M x 3) used by the block-Jacobi
    comparison of Section 4b-ii (reading: the bounding cube, centred on the
    bounding box with side equal to its largest extent, is split at its
    centre into octants 4[x >= cx] + 2[y >= cy] + [z >= cz] until a box holds
    at most `leaf` points; non-empty leaves in depth-first octant order, points
    in ascending index).  Returns a list of index arrays."""
    r = np.asarray(r, np.float64)
    lo, hi = r.min(axis=0), r.max(axis=0)
    out = []

    def split(idx, c, h, depth):
        if len(idx) <= leaf or depth >= 40:
            if len(idx):
                out.append(np.sort(idx))
            return
        o = 4 * (r[idx, 0] >= c[0]) + 2 * (r[idx, 1] >= c[1]) + (r[idx, 2] >= c[2])
        q = 0.5 * h
        for k in range(8):
            sub = idx[o == k]
            cc = c + q * np.array([1 if k & 4 else -1, 1 if k & 2 else -1, 1 if k & 1 else -1])
            split(sub, cc, q, depth + 1)

    split(np.arange(len(r)), 0.5 * (lo + hi), 0.5 * float(np.max(hi - lo)), 0)
    return out


class Preconditioner:
    """z = C r for C = I (none), diag(A)^-1 (Jacobi), P M^-1 P (RBJ), or
    block Jacobi on octree leaves (pass the points as `points`)."""

    def __init__(self, A, kind="rbj", l=100, seed=0, points=None):
        self.kind = kind
        if kind == "none":
            return
        if kind == "jacobi":
            self.dinv = 1.0 / np.diag(A)
            return
        if kind == "rbj":
            self.blocks = rbj_blocks(A, l, seed)
        elif kind == "octree":
            self.blocks = octree_blocks(points, l)
        else:
            raise ValueError(kind)
        self.inv = [np.linalg.inv(A[np.ix_(b, b)]) for b in self.blocks]

    def apply(self, r):
        if self.kind == "none":
            return r.copy()
        if self.kind == "jacobi":
            return self.dinv * r
        z = np.zeros_like(r)
        for b, Minv in zip(self.blocks, self.inv):
            z[b] = Minv @ r[b]
        return z


def pcg(A, b, delta, precond: Preconditioner, x0=None, max_iter=None):
    """Preconditioned CG (Saad, Algorithm 9.1).  Stops as soon as the
    recursively updated residual has ||r||_2 < delta (Eq. 20).
    Returns (x, iterations, converged, ||r||)."""
    M = len(b)
    max_iter = 10 * M if max_iter is None else max_iter
    x = np.zeros(M) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x
    rn = np.linalg.norm(r)
    if rn < delta:
        return x, 0, True, rn
    z = precond.apply(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, max_iter + 1):
        Ap = A @ p
        alpha = rz / (p @ Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        rn = np.linalg.norm(r)
        if rn < delta:
            return x, it, True, rn
        z = precond.apply(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, max_iter, False, rn


def dynamic_delta(prev_diis_error, err_coef=0.01, err_pow=1.07, safety=1e-3,
                  dmin=1e-10, dmax=1.0):
    """Eq. 21: Err(delta) = 0.01 delta^1.07; delta is chosen so that
    Err(delta) = 1e-3 x (previous DIIS error); delta = 1 on the first SCF
    step (no previous error)."""
    if prev_diis_error is None or prev_diis_error < 0:
        return 1.0
    d = (safety * prev_diis_error / err_coef) ** (1.0 / err_pow)
    return float(min(dmax, max(dmin, d)))


def energy(Bz, c, q, A, f):
    """Delta G_els = (Bz)^T q + c^T q + q^T A q / (2 f) (Eq. 13)."""
    return float(Bz @ q + c @ q + q @ (A @ q) / (2.0 * f))


# --------------------------------------------------------------------------
# One pass of the whole path
# --------------------------------------------------------------------------

def run(w, eps=78.39, k=0.0, zeta=4.9, n=110, drop=1e-8, delta=None, prev_diis=None,
        precond="auto", rbj_block=100, seed=0, pts_subset=None):
    """Surface -> c -> rhs -> q (LU and PCG) -> dF -> energy for a workload."""
    s = surface(w.mol.xyz, w.mol.radius, n=n, zeta=zeta, drop=drop)
    eb = ExpandedBasis(w.basis, w.mol.xyz)
    f = f_factor(eps, k)
    A = a_matrix(s)
    Bz_ = bz(s, w.mol.xyz, w.mol.Z)
    c = esp(eb, w.P, s["r"], s["zeta"])
    rhs = -f * (Bz_ + c)
    q_lu = solve_lu(A, rhs)
    out = {"surf": s, "eb": eb, "A": A, "Bz": Bz_, "c": c, "rhs": rhs, "q_lu": q_lu, "f": f}
    if delta is None:
        delta = dynamic_delta(prev_diis)
    kind = precond
    if precond == "auto":
        kind = "jacobi" if len(c) < 1000 else "rbj"
    pc = Preconditioner(A, kind, rbj_block, seed)
    q, it, ok, rn = pcg(A, rhs, delta, pc)
    out.update(q=q, iters=it, converged=ok, rnorm=rn, delta=delta)
    out["dF"] = fock(eb, q, s["r"], s["zeta"])
    out["E"] = energy(Bz_, c, q, A, f)
    out["E_lu"] = energy(Bz_, c, q_lu, A, f)
    return out


# --------------------------------------------------------------------------
# Nuclear gradient at fixed P and q (Eq. 14, Eq. 22)
# --------------------------------------------------------------------------
# Every surface point r_k = R_I + R_I u_i moves with its atom I = atom[k];
# zeta_k does not depend on the geometry.  Derivatives of erf(z d)/d:
#   d/dd [erf(z d) / d] = (2 z / sqrt(pi)) exp(-z^2 d^2) / d - erf(z d) / d^2.

def _derf_over_r(z, d):
    return 2.0 * z / math.sqrt(math.pi) * np.exp(-(z * d) ** 2) / d - erf(z * d) / d ** 2


def gradient_bz(surf, xyz, Z, q):
    """d/dR of (B z)^T q (Eq. 4, first term of Eq. 14): natom x 3."""
    xyz = np.asarray(xyz, np.float64)
    r, z, atom = surf["r"], surf["zeta"], surf["atom"]
    natom = len(xyz)
    g = np.zeros((natom, 3))
    for J in range(natom):
        v = r - xyz[J]
        d = np.linalg.norm(v, axis=1)
        # d/dr_k of q_k Z_J erf(zeta_k d)/d; r_k moves with atom[k], R_J with J
        t = (q * Z[J] * _derf_over_r(z, d) / d)[:, None] * v
        for x in range(3):
            g[:, x] += np.bincount(atom, weights=t[:, x], minlength=natom)
        g[J] -= t.sum(axis=0)
    return g


def gradient_a(surf, xyz, radius, q, f):
    """d/dR of q^T A q / (2 f) (Eq. 2, Eq. 3, Eq. 8, Eq. 9; third term of
    Eq. 14): off-diagonal erf(zeta' r)/r terms and the diagonal through the
    switching values S_k.  natom x 3."""
    xyz = np.asarray(xyz, np.float64)
    radius = np.asarray(radius, np.float64)
    r, z, atom, S = surf["r"], surf["zeta"], surf["atom"], surf["S"]
    natom = len(xyz)
    M = len(z)
    g = np.zeros((natom, 3))
    nz = np.nonzero(q)[0]
    # off-diagonal: sum over ordered pairs k != l of q_k q_l A_kl / (2 f);
    # d/dr_k A_kl = h'(r_kl) (r_k - r_l) / r_kl = -d/dr_l A_kl
    for b0 in range(0, len(nz), 512):
        kk = nz[b0:b0 + 512]
        v = r[kk, None, :] - r[None, nz, :]
        d = np.linalg.norm(v, axis=2)
        zp = z[kk, None] * z[None, nz] / np.sqrt(z[kk, None] ** 2 + z[None, nz] ** 2)   # Eq. 8
        same = kk[:, None] == nz[None, :]
        d_safe = np.where(same, 1.0, d)
        coef = np.where(same, 0.0, q[kk, None] * q[None, nz] * _derf_over_r(zp, d_safe) / d_safe) / (2.0 * f)
        t = coef[:, :, None] * v                       # d/dr_k of the (k, l) term
        tk = t.sum(axis=1)
        tl = t.sum(axis=0)
        for x in range(3):
            g[:, x] += np.bincount(atom[kk], weights=tk[:, x], minlength=natom)
            g[:, x] -= np.bincount(atom[nz], weights=tl[:, x], minlength=natom)
    # diagonal: A_kk = zeta_k sqrt(2/pi) / S_k with S_k = prod_{J != atom[k]} s_J (Eq. 9);
    # d/dd s_J = (zeta/sqrt(pi)) [exp(-zeta^2 (R_J - d)^2) - exp(-zeta^2 (R_J + d)^2)],
    # d A_kk = -A_kk d ln S_k
    Akk = z * math.sqrt(2.0 / math.pi) / S
    for J in range(natom):
        v = r - xyz[J]
        d = np.linalg.norm(v, axis=1)
        sJ = switching_factor(z, d, radius[J])
        ds = z / math.sqrt(math.pi) * (np.exp(-(z * (radius[J] - d)) ** 2) - np.exp(-(z * (radius[J] + d)) ** 2))
        other = atom != J
        coef = np.where(other, -(q * q) / (2.0 * f) * Akk * ds / np.where(other, sJ, 1.0) / d, 0.0)
        t = coef[:, None] * v                          # d/dr_k; R_J gets the opposite
        for x in range(3):
            g[:, x] += np.bincount(atom, weights=t[:, x], minlength=natom)
        g[J] -= t.sum(axis=0)
    return g


def gradient_c(eb: ExpandedBasis, P, q, surf):
    """d/dR of c^T q at fixed P (second term of Eq. 14, Eq. 22): natom x 3."""
    natom = len(eb.xyz)
    g = np.zeros(natom * 3)
    pts = np.ascontiguousarray(surf["r"], np.float64)
    lib().oracle_grad_c(eb.nshell, _i(eb.sh_atom), _i(eb.sh_l), _i(eb.sh_nprim), _i(eb.sh_off),
                        _i(eb.sh_bf), _d(eb.exps), _d(eb.coefs), _d(eb.xyz), eb.nbf,
                        _d(np.ascontiguousarray(P, np.float64)), len(pts), _d(pts),
                        _d(np.asarray(surf["zeta"], np.float64)), _d(np.asarray(q, np.float64)),
                        _i(surf["atom"]), natom, _d_out(g))
    return g.reshape(natom, 3)


def gradient(eb: ExpandedBasis, P, q, surf, xyz, Z, radius, f):
    """Eq. 14: z^T (dB^T) q + (d*c^T) q + q^T (dA) q / (2 f) at fixed P and
    q.  At the solution of Eq. 1 this is the derivative of Delta G_els
    (Eq. 13) at fixed P, because Delta G_els is stationary in q there.
    Returns dict with the three terms and their sum (natom x 3 each)."""
    gb = gradient_bz(surf, xyz, Z, q)
    ga = gradient_a(surf, xyz, radius, q, f)
    gc = gradient_c(eb, P, q, surf)
    return {"B": gb, "A": ga, "C": gc, "total": gb + ga + gc}

"""Seeded synthetic inputs for the C-PCM (ISWIG) hot path.

This module is shared by the CUDA path's tests and benchmark and by the
CPU oracle's tests.  It holds NO arithmetic of the method itself: it only
draws molecules (element, position, nuclear charge, cavity radius), basis
sets (shell angular momenta, exponents, raw contraction coefficients) and
density matrices.  Surface points, switching functions, integrals, the
linear system and the energy are computed separately by each side.

The paper's own inputs (PDB proteins, the SI test molecules, Lebedev
tables and real basis sets) are not available; these generators stand in
for them with the shapes the paper describes (Section 3: proteins of
about 100-500 atoms, 6-31G-like basis sets, 110 points per atom, radii of
1.2 x Bondi).

Units: bohr for lengths, atomic units throughout.

Conventions fixed here and assumed by both sides:
  * shell_l: 0 = s, 1 = p, 2 = d, -1 = sp (an s and a p shell sharing one
    set of exponents; its coefficients are given s first, then p).
  * basis-function order: shells in order; within an sp shell s, px, py,
    pz; p: x, y, z; d (6 Cartesian): xx, xy, xz, yy, yz, zz.
  * the density is a full symmetric nbf x nbf matrix, row-major.
"""
from __future__ import annotations

import dataclasses
import numpy as np

ANGSTROM = 1.0 / 0.529177210903          # bohr per angstrom

# Bondi (1964) van der Waals radii in angstrom.
BONDI_ANGSTROM = {"H": 1.20, "C": 1.70, "N": 1.55, "O": 1.52, "S": 1.80}
ATOMIC_NUMBER = {"H": 1, "C": 6, "N": 7, "O": 8, "S": 16}
RADIUS_SCALE = 1.2                       # cavity radii are 1.2 x Bondi (Section 3)

# Paper defaults (Section 3 and Eq. 1): water, C-PCM k = 0, 110 points per atom.
EPSILON = 78.39
K_COSMO = 0.0
ZETA_110 = 4.9                           # optimized exponent used for 110-point spheres
POINTS_PER_SPHERE = 110
SWITCH_DROP = 1e-8                       # ISWIG screening threshold (Section 3)


@dataclasses.dataclass
class Molecule:
    symbols: list
    xyz: np.ndarray          # (natom, 3) bohr
    Z: np.ndarray            # (natom,) nuclear charges
    radius: np.ndarray       # (natom,) cavity radii in bohr (already 1.2 x Bondi)

    @property
    def natom(self) -> int:
        return len(self.symbols)


@dataclasses.dataclass
class Basis:
    shell_atom: np.ndarray   # (nshell,) int32
    shell_l: np.ndarray      # (nshell,) int32, -1 = sp
    shell_nprim: np.ndarray  # (nshell,) int32
    exps: np.ndarray         # (sum nprim,) exponents, shell after shell
    coefs: np.ndarray        # raw contraction coefficients; sp shells store
                             # nprim s coefficients then nprim p coefficients

    @property
    def nshell(self) -> int:
        return len(self.shell_l)

    @property
    def nbf(self) -> int:
        per = {0: 1, 1: 3, 2: 6, -1: 4}
        return int(sum(per[int(l)] for l in self.shell_l))


@dataclasses.dataclass
class Workload:
    name: str
    mol: Molecule
    basis: Basis
    P: np.ndarray            # (nbf, nbf) symmetric density
    nocc: int
    seed: int
    C: np.ndarray | None = None   # (nbf, nocc) occupied orbitals, P = 2 C C^T


def _mol(symbols, xyz_bohr):
    symbols = list(symbols)
    xyz = np.asarray(xyz_bohr, dtype=np.float64).reshape(-1, 3)
    Z = np.array([ATOMIC_NUMBER[s] for s in symbols], dtype=np.float64)
    radius = np.array([RADIUS_SCALE * BONDI_ANGSTROM[s] * ANGSTROM for s in symbols])
    return Molecule(symbols, xyz, Z, radius)


def _loguniform(rng, lo, hi, n):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))


# Per-element shell recipes: (shell_l, nprim, exponent range).  The ranges
# sit inside the overall [0.1, 5000] span, a core shell tight and the outer
# shells diffuse, as in 6-31G-like sets.
_SHELLS_631G = {
    "H": [(0, 3, (0.3, 30.0)), (0, 1, (0.1, 0.4))],
    "C": [(0, 6, (3.0, 5000.0)), (-1, 3, (0.3, 30.0)), (-1, 1, (0.1, 0.4))],
    "N": [(0, 6, (3.0, 5000.0)), (-1, 3, (0.3, 30.0)), (-1, 1, (0.1, 0.4))],
    "O": [(0, 6, (3.0, 5000.0)), (-1, 3, (0.3, 30.0)), (-1, 1, (0.1, 0.4))],
    "S": [(0, 6, (10.0, 5000.0)), (-1, 6, (1.0, 500.0)), (-1, 3, (0.2, 5.0)), (-1, 1, (0.1, 0.4))],
}
_D_SHELL = (2, 1, (0.3, 1.5))            # one polarisation d shell per heavy atom (6-31G*-like)


def make_basis(mol: Molecule, recipe: dict, rng, d_on_heavy: bool = False) -> Basis:
    sa, sl, sn, ex, co = [], [], [], [], []
    for ia, s in enumerate(mol.symbols):
        shells = list(recipe[s])
        if d_on_heavy and s != "H":
            shells.append(_D_SHELL)
        for (l, n, (lo, hi)) in shells:
            e = np.sort(_loguniform(rng, lo, hi, n))[::-1]
            sa.append(ia); sl.append(l); sn.append(n); ex.extend(e)
            ncoef = 2 * n if l == -1 else n
            co.extend(rng.uniform(0.1, 1.0, size=ncoef))
    return Basis(np.array(sa, np.int32), np.array(sl, np.int32), np.array(sn, np.int32),
                 np.array(ex, np.float64), np.array(co, np.float64))


def _cart(l):
    return [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]


def _dfact(n):
    r = 1.0
    while n > 1:
        r *= n
        n -= 2
    return r


def overlap_matrix(basis: Basis, xyz: np.ndarray, block: int = 2048, cut: float = 1e-17) -> np.ndarray:
    """Overlap S_{mu nu} of the basis functions (input preparation for the
    density; not part of the solvation method).  Each Cartesian primitive
    component is normalised to unit self-overlap and multiplied by the raw
    contraction coefficient.  One-dimensional factors by the Obara-Saika
    overlap recurrence s(i+1, j) = X_PA s(i, j) + (i s(i-1, j) + j s(i, j-1)) / 2p,
    s(0, 0) = sqrt(pi / p) exp(-a b / p X_AB^2); primitive pairs whose
    prefactor is below `cut` are skipped."""
    # expanded primitives (sp -> s and p)
    pl, pe, pc, pa, pbf = [], [], [], [], []
    off = cpos = bf = 0
    for s_ in range(basis.nshell):
        l, n = int(basis.shell_l[s_]), int(basis.shell_nprim[s_])
        e = basis.exps[off:off + n]
        parts = [(0, basis.coefs[cpos:cpos + n]), (1, basis.coefs[cpos + n:cpos + 2 * n])] if l == -1 \
            else [(l, basis.coefs[cpos:cpos + n])]
        cpos += 2 * n if l == -1 else n
        for ll, c in parts:
            for k in range(n):
                pl.append(ll); pe.append(e[k]); pa.append(basis.shell_atom[s_]); pbf.append(bf)
                pc.append(c[k] * (2 * e[k] / np.pi) ** 0.75 * (4 * e[k]) ** (ll / 2) / np.sqrt(_dfact(2 * ll - 1)))
            bf += len(_cart(ll))
        off += n
    pl = np.array(pl); pe = np.array(pe); pc = np.array(pc); pcen = xyz[np.array(pa)]; pbf = np.array(pbf)
    S = np.zeros(bf * bf)

    def s1d(la, lb, PA, PB, inv2p, s00):
        t = {(0, 0): s00}
        for i in range(la + 1):
            for j in range(lb + 1):
                if (i, j) in t:
                    continue
                if i > 0:
                    v = PA * t[(i - 1, j)]
                    if i > 1: v = v + (i - 1) * inv2p * t[(i - 2, j)]
                    if j > 0: v = v + j * inv2p * t[(i - 1, j - 1)]
                else:
                    v = PB * t[(i, j - 1)]
                    if j > 1: v = v + (j - 1) * inv2p * t[(i, j - 2)]
                t[(i, j)] = v
        return t

    for la in range(3):
        ia_all = np.nonzero(pl == la)[0]
        for lb in range(3):
            ib = np.nonzero(pl == lb)[0]
            if len(ia_all) == 0 or len(ib) == 0:
                continue
            ca, cb = _cart(la), _cart(lb)
            fa = np.array([np.sqrt(_dfact(2 * la - 1) / (_dfact(2 * x - 1) * _dfact(2 * y - 1) * _dfact(2 * z - 1)))
                           for x, y, z in ca])
            fb = np.array([np.sqrt(_dfact(2 * lb - 1) / (_dfact(2 * x - 1) * _dfact(2 * y - 1) * _dfact(2 * z - 1)))
                           for x, y, z in cb])
            for b0 in range(0, len(ia_all), block):
                ia = ia_all[b0:b0 + block]
                a = pe[ia][:, None]; b = pe[ib][None, :]
                p = a + b
                A = pcen[ia][:, None, :]; B = pcen[ib][None, :, :]
                d2 = np.sum((A - B) ** 2, axis=-1)
                K = np.exp(-a * b / p * d2)
                w = pc[ia][:, None] * pc[ib][None, :] * K
                m = np.abs(w) > cut
                ii, jj = np.nonzero(m)
                if len(ii) == 0:
                    continue
                a1 = a[ii, 0]; b1 = b[0, jj]; p1 = a1 + b1; w1 = w[ii, jj]
                P = (a1[:, None] * A[ii, 0, :] + b1[:, None] * B[0, jj, :]) / p1[:, None]
                PA = P - A[ii, 0, :]; PB = P - B[0, jj, :]
                inv2p = 0.5 / p1
                s00 = np.sqrt(np.pi / p1)
                tx = s1d(la, lb, PA[:, 0], PB[:, 0], inv2p, s00)
                ty = s1d(la, lb, PA[:, 1], PB[:, 1], inv2p, s00)
                tz = s1d(la, lb, PA[:, 2], PB[:, 2], inv2p, s00)
                rows = pbf[ia][ii]; cols = pbf[ib][jj]
                for u, (ax, ay, az) in enumerate(ca):
                    for v, (bx, by, bz) in enumerate(cb):
                        val = w1 * fa[u] * fb[v] * tx[(ax, bx)] * ty[(ay, by)] * tz[(az, bz)]
                        S += np.bincount((rows + u) * bf + cols + v, weights=val, minlength=bf * bf)
    S = S.reshape(bf, bf)
    return 0.5 * (S + S.T)


def _orthonormalise(G: np.ndarray, S: np.ndarray) -> np.ndarray:
    """Symmetric orthonormalisation in the overlap metric: G (G^T S G)^(-1/2)."""
    e, V = np.linalg.eigh(G.T @ S @ G)
    return G @ (V / np.sqrt(e)) @ V.T


def _density(C: np.ndarray) -> np.ndarray:
    P = 2.0 * C @ C.T
    return 0.5 * (P + P.T)


def make_orbitals(basis: Basis, xyz: np.ndarray, nocc: int, rng) -> np.ndarray:
    """nocc seeded occupied orbitals, orthonormal in the overlap metric
    (C^T S C = I): the columns of a seeded Gaussian nbf x nocc matrix G,
    symmetrically orthonormalised, C = G (G^T S G)^(-1/2)."""
    S = overlap_matrix(basis, xyz)
    nocc = min(nocc, basis.nbf)
    return _orthonormalise(rng.standard_normal((basis.nbf, nocc)), S)


def make_density(basis: Basis, xyz: np.ndarray, nocc: int, rng) -> np.ndarray:
    """P = 2 C C^T for the orbitals of make_orbitals (tr(P S) = 2 nocc)."""
    return _density(make_orbitals(basis, xyz, nocc, rng))


def scf_sequence(w: "Workload", n_iter: int = 14, e0: float = 0.1, ratio: float = 0.4,
                 seed: int | None = None):
    """A synthetic SCF history ending at w.P, for the CG threshold schemes of
    Section 4b-i: iteration n has the DIIS error e_n = e0 ratio^n and the
    density of the occupied orbitals perturbed by e_n times a seeded Gaussian
    matrix (re-orthonormalised in the overlap metric), so that the densities
    approach w.P as the DIIS errors fall.  Returns [(P_n, e_n), ...]."""
    if w.C is None:
        raise ValueError("the workload carries no orbitals")
    rng = np.random.default_rng(w.seed + 77 if seed is None else seed)
    S = overlap_matrix(w.basis, w.mol.xyz)
    out = []
    for n in range(n_iter):
        e = e0 * ratio ** n
        G = w.C + e * rng.standard_normal(w.C.shape)
        out.append((_density(_orthonormalise(G, S)), e))
    return out


def water(seed: int = 150507851 + 0) -> Workload:
    """3-atom O,H,H molecule: O at the origin, H at (+-1.43, 1.11, 0) bohr.
    H: one s shell of 3 primitives; O: one s and one sp shell of 3
    primitives; exponents log-uniform in [0.1, 130]; nbf = 7; 5 occupied."""
    rng = np.random.default_rng(seed)
    mol = _mol(["O", "H", "H"], [[0, 0, 0], [1.43, 1.11, 0], [-1.43, 1.11, 0]])
    recipe = {"O": [(0, 3, (0.1, 130.0)), (-1, 3, (0.1, 130.0))],
              "H": [(0, 3, (0.1, 130.0))]}
    basis = make_basis(mol, recipe, rng)
    C = make_orbitals(basis, mol.xyz, 5, rng)
    return Workload("water", mol, basis, _density(C), 5, seed, C)


def _composition(natom: int, ratios=(("H", 50), ("C", 31), ("N", 9), ("O", 9), ("S", 1))):
    tot = sum(r for _, r in ratios)
    counts = [int(round(natom * r / tot)) for _, r in ratios]
    counts[0] += natom - sum(counts)
    out = []
    for (s, _), c in zip(ratios, counts):
        out += [s] * c
    return out


def random_walk_cluster(natom: int, rng, globule_radius_A: float,
                        bond=(1.0, 1.5), nonbond=2.0, max_tries=20000) -> np.ndarray:
    """Positions (angstrom) of a seeded branching random walk: each new atom
    sits 1.0-1.5 A from a parent (mostly the previous atom) and at least
    2.0 A from every other atom, inside a sphere of the given radius."""
    pos = np.zeros((natom, 3))
    n = 1
    tries = 0
    while n < natom:
        tries += 1
        if tries > max_tries * natom:
            raise RuntimeError("random walk could not place all atoms; enlarge the globule")
        parent = n - 1 if rng.random() < 0.7 else int(rng.integers(0, n))
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        cand = pos[parent] + rng.uniform(*bond) * d
        if np.linalg.norm(cand) > globule_radius_A:
            continue
        dist = np.linalg.norm(pos[:n] - cand, axis=1)
        dist[parent] = np.inf
        if np.all(dist >= nonbond):
            pos[n] = cand
            n += 1
    return pos


def cluster(natom: int, seed: int, globule_radius_A: float, d_shells: bool = False,
            nocc: int | None = None, name: str = "cluster") -> Workload:
    """Protein-shaped cluster with H:C:N:O:S = 50:31:9:9:1, s/sp (and
    optionally d) shells, and nocc = 2 * natom occupied orbitals unless given."""
    rng = np.random.default_rng(seed)
    symbols = _composition(natom)
    rng.shuffle(symbols)
    pos = random_walk_cluster(natom, rng, globule_radius_A)
    mol = _mol(symbols, pos * ANGSTROM)
    basis = make_basis(mol, _SHELLS_631G, rng, d_on_heavy=d_shells)
    nocc = 2 * natom if nocc is None else nocc
    nocc = min(nocc, basis.nbf)
    C = make_orbitals(basis, mol.xyz, nocc, rng)
    return Workload(name, mol, basis, _density(C), nocc, seed, C)


# Globule radii (angstrom) chosen so that the 110-point ISWIG surface of the
# cluster has roughly the number of kept points the workloads call for.
GLOBULE_RADIUS_A = {300: 8.0, 1000: 13.5}


def config(i: int) -> Workload:
    """The five workloads, by number:
    0: water, nbf 7, M ~ 250.
    1: 300-atom s/sp cluster, nbf ~ 1.6k, 600 occupied, M ~ 12k.
    2: 1000-atom s/sp/d cluster, nbf ~ 9.5k, M ~ 45k.
    3: the 300-atom cluster of 1 with d shells, nbf ~ 2.8k.
    4: (batched conformations; see conformations()).
    """
    seed = 150507851 + i
    if i == 0:
        return water(seed)
    if i == 1:
        return cluster(300, seed, GLOBULE_RADIUS_A[300], nocc=600, name="cluster300_sp")
    if i == 2:
        return cluster(1000, seed, GLOBULE_RADIUS_A[1000], d_shells=True, nocc=2000,
                       name="cluster1000_spd")
    if i == 3:
        w = cluster(300, 150507851 + 1, GLOBULE_RADIUS_A[300], d_shells=True, nocc=600,
                    name="cluster300_spd")
        return w
    raise ValueError("config %d is a batch; use conformations()" % i)


def small_cluster(natom: int, seed: int, d_shells: bool = False, radius_A: float | None = None,
                  nocc: int | None = None) -> Workload:
    """Small clusters for parity tests (sizes the oracle finishes in seconds)."""
    if radius_A is None:
        radius_A = max(3.0, 8.0 * (natom / 300.0) ** (1.0 / 3.0))
    return cluster(natom, seed, radius_A, d_shells=d_shells, nocc=nocc,
                   name="cluster%d%s" % (natom, "_spd" if d_shells else "_sp"))


def _conformation(args):
    na, seed, j = args
    r = 8.0 * (na / 300.0) ** (1.0 / 3.0)
    return cluster(int(na), seed * 1000 + j, r, name="conf%d" % j)


def conformations(n: int = 64, seed: int = 150507851 + 4, lo: int = 150, hi: int = 600, workers: int = 0):
    """Seeded batch of peptide-like clusters with uniform-random sizes in
    [lo, hi] atoms (s/sp shells, 2 natom occupied orbitals).  workers > 1
    builds them in that many processes (spawned, so that a CUDA context of the
    caller is never forked); the result does not depend on it."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(lo, hi + 1, size=n)
    jobs = [(int(na), seed, j) for j, na in enumerate(sizes)]
    if workers > 1:
        import multiprocessing as mp
        import os
        # one BLAS thread per worker process (the workers already fill the cores)
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        os.environ.update({k: "1" for k in keys})
        try:
            with mp.get_context("spawn").Pool(workers) as pool:
                return pool.map(_conformation, jobs, chunksize=1)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    return [_conformation(a) for a in jobs]

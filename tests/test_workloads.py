"""The seeded input generator: sizes of the named workloads, and the density
built from overlap-orthonormal occupied orbitals (tr(P S) = 2 n_occ).  The
generator's overlap is checked against the oracle's integrals in the
small-zeta limit, where erf(zeta r)/r -> 2 zeta / sqrt(pi)."""
import math

import numpy as np

import oracle
import workloads


def _oracle_overlap(w, zs=1e-6):
    eb = oracle.ExpandedBasis(w.basis, w.mol.xyz)
    S = np.zeros((eb.nbf, eb.nbf))
    for a in range(eb.nshell):
        for b in range(eb.nshell):
            blk = eb.shell_block(a, b, eb.xyz[eb.sh_atom[a]], zs) * math.sqrt(math.pi) / (2 * zs)
            S[eb.sh_bf[a]:eb.sh_bf[a] + blk.shape[0], eb.sh_bf[b]:eb.sh_bf[b] + blk.shape[1]] = blk
    return S


def test_overlap_and_electron_count():
    for w in (workloads.config(0), workloads.small_cluster(5, seed=22, d_shells=True)):
        S = workloads.overlap_matrix(w.basis, w.mol.xyz)
        assert np.max(np.abs(S - _oracle_overlap(w))) <= 1e-10 * np.max(np.abs(S))
        assert abs(np.sum(w.P * S) - 2 * w.nocc) < 1e-9 * w.nocc
        assert np.max(np.abs(w.P - w.P.T)) == 0.0


def test_named_workload_shapes():
    w = workloads.config(0)
    assert (w.mol.natom, w.basis.nbf, w.nocc) == (3, 7, 5)
    w = workloads.config(1)
    assert w.mol.natom == 300 and 1500 <= w.basis.nbf <= 1800 and w.nocc == 600
    assert sorted(set(w.mol.symbols)) == ["C", "H", "N", "O", "S"]
    d = np.linalg.norm(w.mol.xyz[:, None] - w.mol.xyz[None], axis=2) / workloads.ANGSTROM
    np.fill_diagonal(d, np.inf)
    assert d.min() >= 1.0 - 1e-9                       # bonds of at least 1.0 A
    assert w.mol.Z.sum() == 1161

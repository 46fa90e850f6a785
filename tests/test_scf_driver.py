"""Host logic of the SCF-sequence driver (Section 4b-i) and the synthetic
SCF histories it runs on."""
import numpy as np
import pytest

import workloads


def test_two_delta_rule():
    from paper_1505_07851_gb300.scf import two_delta
    # loose threshold s * delta_2 until the previous DIIS error reaches 1e-3
    assert two_delta(None, 1e-6) == pytest.approx(1e-2)
    assert two_delta(-1.0, 1e-6) == pytest.approx(1e-2)
    assert two_delta(5e-3, 1e-6) == pytest.approx(1e-2)
    assert two_delta(1e-3, 1e-6) == 1e-6
    assert two_delta(2e-7, 1e-5) == 1e-5
    assert two_delta(5e-3, 1e-7, s=1e3) == pytest.approx(1e-4)


def test_scf_sequence_approaches_the_density():
    w = workloads.config(0)
    seq = workloads.scf_sequence(w, 12)
    S = workloads.overlap_matrix(w.basis, w.mol.xyz)
    errs = [e for _, e in seq]
    assert np.all(np.diff(errs) < 0) and errs[0] == pytest.approx(0.1)
    dist = [np.max(np.abs(P - w.P)) for P, _ in seq]
    for P, _ in seq:
        assert np.allclose(P, P.T)
        assert np.trace(P @ S) == pytest.approx(2 * w.nocc, rel=1e-12)
    # the distance to the final density shrinks with the DIIS error
    assert dist[-1] < 1e-3 * dist[0]
    assert all(d <= 20 * e for d, e in zip(dist, errs))
    # seeded
    seq2 = workloads.scf_sequence(w, 12)
    assert all(np.array_equal(a[0], b[0]) for a, b in zip(seq, seq2))

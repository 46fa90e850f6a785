"""Host logic of the SCF-sequence driver (Section 4b-i) and the synthetic
SCF histories it runs on."""
import numpy as np
import pytest

import workloads


def test_threshold_rules_through_the_c_abi():
    """pcm_cg_threshold is the rule pcm_solve applies (host logic, no GPU)."""
    import paper_1505_07851_gb300 as pcm
    th = pcm.cg_threshold
    # 2-delta (Section 4b-i): 1e4 * delta_2 until the previous DIIS error reaches 1e-3
    assert th(1e-6, -1.0, two_delta=True) == pytest.approx(1e-2)
    assert th(1e-6, 5e-3, two_delta=True) == pytest.approx(1e-2)
    assert th(1e-6, 1e-3, two_delta=True) == 1e-6
    assert th(1e-5, 2e-7, two_delta=True) == 1e-5
    # fixed
    assert th(3e-7, 0.5) == 3e-7
    # Eq. 21: Err(delta) = 0.01 delta^1.07 equals 1e-3 of the previous DIIS error
    for e in (1e-1, 1e-3, 1e-5):
        d = th(-1.0, e)
        assert 0.01 * d ** 1.07 == pytest.approx(1e-3 * e, rel=1e-12)
    assert th(-1.0, -1.0) == 1.0                  # first SCF step
    assert th(0.0, 1e3) == 1.0                    # clamped above
    assert th(-1.0, 1e-20) == 1e-10               # clamped below
    for bad in ((float("nan"), 1.0, False), (1e-6, float("nan"), False), (0.0, 1e-2, True)):
        with pytest.raises(pcm.PCMError):
            th(bad[0], bad[1], two_delta=bad[2])


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


class _FakeContext:
    """Stands in for pcm.Context on the host: records the calls run_sequence
    makes and writes its 'solution' into the array it is given (as the C ABI
    does for a warm start), so that aliasing would show."""

    def __init__(self, M=5):
        self.M = M
        self.calls = []

    def esp(self, P):
        self.calls.append(("esp", float(np.sum(P))))

    def solve(self, delta=-1.0, prev_diis_error=-1.0, q=None, warm=False, like=None, two_delta=False):
        import paper_1505_07851_gb300 as pcm
        d = pcm.cg_threshold(delta, prev_diis_error, two_delta)
        out = q if q is not None else np.zeros(self.M)
        self.calls.append(("solve", d, warm, None if q is None else q.copy()))
        out += 1.0                       # each solve moves the charges by one
        return out, {"delta": d, "iterations": 3, "converged": 1, "ms_solve": 0.0, "refinements": 1}

    def energy(self, q):
        return float(np.sum(q))


@pytest.mark.parametrize("scheme", ["fixed", "2delta", "dynamic"])
def test_run_sequence_thresholds_and_warm_starts(scheme):
    from paper_1505_07851_gb300.scf import run_sequence
    seq = [(np.full((2, 2), float(n)), 0.1 * 0.4 ** n) for n in range(5)]
    ctx = _FakeContext()
    res = run_sequence(ctx, seq, scheme, delta_tight=1e-6, keep_q=True)
    solves = [c for c in ctx.calls if c[0] == "solve"]
    assert len(res) == len(seq) == len(solves)
    prev = None
    for n, (r, s) in enumerate(zip(res, solves)):
        if scheme == "fixed":
            want = 1e-6
        elif scheme == "2delta":
            want = 1e-2 if (prev is None or prev > 1e-3) else 1e-6
        else:
            want = 1.0 if prev is None else (1e-3 * prev / 0.01) ** (1 / 1.07)
        assert r["delta"] == pytest.approx(want, rel=1e-12)
        # warm start from the previous charges after the first iteration
        assert s[2] == (n > 0)
        if n > 0:
            assert np.array_equal(s[3], res[n - 1]["q"])
        # the kept charges are copies: later in-place solves do not change them
        assert np.all(r["q"] == n + 1)
        assert r["energy"] == pytest.approx(ctx.M * (n + 1))
        prev = seq[n][1]

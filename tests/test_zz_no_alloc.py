"""pcm_energy_noalloc, the energy entry point for callers that cannot
allocate device memory (their GPU memory belongs to their own allocator),
called through the C ABI and checked against pcm_energy on the same inputs,
on two calls in a row.  Collected last on purpose."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def test_energy_noalloc_matches_pcm_energy_twice():
    import torch
    import paper_1505_07851_gb300 as pcm

    w = workloads.small_cluster(8, seed=21)
    with pcm.Context(schwarz=0.0) as ctx:
        M, nbf = ctx.setup(w.mol, w.basis)
        Bz = np.zeros(M)
        c = ctx.esp(w.P, bz_out=Bz)
        q1, _ = ctx.solve(delta=1e-10)
        q2 = 0.5 * q1 + np.random.default_rng(0).normal(scale=1e-3, size=M)
        E1 = ctx.energy(q1)
        E2 = ctx.energy(q2)
        xyzzs, _ = ctx.get_surface()
    # the caller's own copy of A (Eq. 2, Eq. 3) for the library's surface points
    A = oracle.a_matrix({"r": xyzzs[:, :3], "zeta": xyzzs[:, 3], "S": xyzzs[:, 4]})
    f = (78.39 - 1.0) / 78.39
    dev = torch.device("cuda", 0)
    Ad = torch.tensor(A, device=dev)
    Bzd = torch.tensor(Bz, device=dev)
    cd = torch.tensor(c, device=dev)
    Ed = torch.zeros(1, dtype=torch.float64, device=dev)
    for q, E_ref in ((q1, E1), (q2, E2)):
        qd = torch.tensor(q, device=dev)
        pcm.energy_noalloc(Ad, Bzd, cd, qd, f, Ed)
        torch.cuda.synchronize()
        E = float(Ed.item())
        assert abs(E - E_ref) <= 1e-9 * max(1.0, abs(E_ref)), (E, E_ref)


def test_energy_noalloc_rejects_sizes_beyond_its_scratch():
    import ctypes
    import paper_1505_07851_gb300 as pcm
    # host-side checks only: nothing is launched
    dummy = ctypes.c_void_p(16)
    st = pcm.pcm_energy_noalloc(65537, dummy, 65537, dummy, dummy, dummy, 0.98, dummy, None)
    assert st == pcm.PCM_ERR_ARG
    assert b"65536" in pcm.pcm_last_error()
    st = pcm.pcm_energy_noalloc(0, dummy, 1, dummy, dummy, dummy, 0.98, dummy, None)
    assert st == pcm.PCM_ERR_ARG

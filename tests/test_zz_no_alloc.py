"""pcm_energy_noalloc, the energy entry point for callers that cannot
allocate device memory (their GPU memory belongs to their own allocator, so
the library may not call cudaMalloc), called through the C ABI.  Checked
against pcm_energy and the oracle's energy on the same inputs, on two calls
in a row; at 10,000 points with A a column slice of a wider matrix (leading
dimension above M, rows strided over the grid) against host FP64 sums.
Collected last on purpose."""
import numpy as np
import pytest

import oracle
import workloads


@pytest.mark.gpu
def test_energy_noalloc_matches_pcm_energy_and_oracle_twice():
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
    # the caller's own copy of A for the library's surface points
    A = oracle.a_matrix({"r": xyzzs[:, :3], "zeta": xyzzs[:, 3], "S": xyzzs[:, 4]})
    f = (78.39 - 1.0) / 78.39
    dev = torch.device("cuda", 0)
    Ad = torch.tensor(A, device=dev)
    Bzd = torch.tensor(Bz, device=dev)
    cd = torch.tensor(c, device=dev)
    Ed = torch.zeros(1, dtype=torch.float64, device=dev)
    for q, E_lib in ((q1, E1), (q2, E2)):
        qd = torch.tensor(q, device=dev)
        pcm.energy_noalloc(Ad, Bzd, cd, qd, f, Ed)
        torch.cuda.synchronize()
        E = float(Ed.item())
        assert abs(E - E_lib) <= 1e-9 * max(1.0, abs(E_lib)), (E, E_lib)
        E_o = oracle.energy(Bz, c, q, A, f)
        assert abs(E - E_o) <= 1e-9 * max(1.0, abs(E_o)), (E, E_o)


@pytest.mark.gpu
def test_energy_noalloc_wide_leading_dimension_many_rows():
    import torch
    import paper_1505_07851_gb300 as pcm

    M, pad = 10000, 13
    rng = np.random.default_rng(5)
    big = rng.uniform(0.0, 1.0, size=(M, M + pad))
    A = big[:, :M]
    f = 0.75
    dev = torch.device("cuda", 0)
    Ad = torch.tensor(big, device=dev)[:, :M]
    assert Ad.stride(0) == M + pad
    Ed = torch.zeros(1, dtype=torch.float64, device=dev)
    Bz = rng.uniform(-1.0, 1.0, M)
    c = rng.uniform(-1.0, 1.0, M)
    Bzd, cd = torch.tensor(Bz, device=dev), torch.tensor(c, device=dev)
    for seed in (1, 2):
        q = np.random.default_rng(seed).uniform(0.0, 1.0, M)
        pcm.energy_noalloc(Ad, Bzd, cd, torch.tensor(q, device=dev), f, Ed)
        torch.cuda.synchronize()
        E_ref = float(Bz @ q + c @ q + q @ (A @ q) / (2.0 * f))
        assert abs(float(Ed.item()) - E_ref) <= 1e-9 * abs(E_ref)


@pytest.mark.gpu
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


def test_energy_noalloc_binding_rejects_bad_shapes():
    """The binding checks shapes before anything reaches the library (CPU
    tensors with the right shapes are then refused as not on a GPU)."""
    import torch
    import paper_1505_07851_gb300 as pcm

    M = 6
    d = dict(dtype=torch.float64)
    good = dict(A=torch.zeros(M, M, **d), Bz=torch.zeros(M, **d), c=torch.zeros(M, **d), q=torch.zeros(M, **d),
                E=torch.zeros(1, **d))
    bad = [dict(A=torch.zeros(M - 1, M, **d)), dict(A=torch.zeros(M, M - 1, **d)), dict(A=torch.zeros(M * M, **d)),
           dict(A=torch.zeros(M, 2 * M, **d)[:, ::2]), dict(Bz=torch.zeros(M - 1, **d)), dict(c=torch.zeros(M + 1, **d)),
           dict(E=torch.zeros(0, **d))]
    for b in bad:
        kw = dict(good, **b)
        with pytest.raises(ValueError):
            pcm.energy_noalloc(kw["A"], kw["Bz"], kw["c"], kw["q"], 0.9, kw["E"])
    with pytest.raises(TypeError):
        pcm.energy_noalloc(good["A"], good["Bz"], good["c"], good["q"], 0.9, good["E"])

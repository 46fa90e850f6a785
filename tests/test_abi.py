"""The C-ABI library builds, loads and exports every function include/pcm.h
declares (no GPU needed: nothing is computed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(pcm_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_1505_07851_gb300", "libpcm.so"))
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_binding_mirrors_the_c_names():
    import paper_1505_07851_gb300 as pcm
    assert set(_declared()) <= set(pcm.EXPORTS)


def test_defaults_are_the_papers_and_errors_have_messages():
    import paper_1505_07851_gb300 as pcm
    o = pcm.pcm_options()
    assert pcm.pcm_default_options(ctypes.byref(o)) == 0
    assert (o.eps, o.k, o.zeta, o.switch_drop, o.schwarz, o.rbj_block, o.jacobi_below) == \
        (78.39, 0.0, 4.9, 1e-8, 1e-12, 100, 1000)
    for s in range(7):
        assert pcm.pcm_strerror(s)
    assert pcm.pcm_default_options(None) == pcm.PCM_ERR_ARG


def test_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1505_07851_gb300 as pcm
    with pytest.raises(pcm.PCMError):
        pcm.Context()

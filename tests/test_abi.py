"""The C-ABI library builds, loads and exports every symbol include/trstmi.h
declares (CPU only: no compute call), and fails loudly without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(trstmi_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("trstmi_create", "trstmi_step", "trstmi_coherence", "trstmi_get_phi",
                     "trstmi_set_phi", "trstmi_get_state", "trstmi_set_state",
                     "trstmi_destroy", "trstmi_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2207_06374_gb300 import trstmi as T
    L = ctypes.CDLL(T.LIB_PATH) if os.path.exists(T.LIB_PATH) else T.lib()
    T.lib()
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    # the Python binding mirrors every declared entry point
    assert set(_declared()) <= set(T.SIGNATURES)


def test_strerror_and_defaults_without_gpu():
    from paper_2207_06374_gb300 import trstmi as T
    assert T.strerror(0) == "ok"
    assert "CUDA" in T.strerror(T.TRSTMI_ECUDA)
    o = T.default_options()
    assert o.K == 256 and o.precision == T.FP64 and o.topk == 8
    assert o.delta0 == 0.1 and o.gamma_inc == 2.0 and o.gamma_dec == 0.25


def test_no_cpu_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2207_06374_gb300 import trstmi as T
    with pytest.raises(T.TrstmiError) as e:
        T.Search(4, 2, 1)
    assert e.value.status == T.TRSTMI_ECUDA

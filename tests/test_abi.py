"""Host-side checks of the C ABI: the library builds, loads without a GPU and exports
every function include/mmf.h declares; the binding refuses to run without it."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:int|const char\*|void)\s+\*?\s*(mmf_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mmf_create", "mmf_propagate", "mmf_destroy", "mmf_energy", "mmf_last_error"):
        assert required in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_1901_01895_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_abi():
    import paper_1901_01895_gb300 as m
    for n in declared_functions():
        assert hasattr(m, n), n


def test_error_paths_without_gpu():
    import paper_1901_01895_gb300 as m
    import numpy as np
    S = np.ones((1, 1, 1, 1))
    b = np.zeros((1, 4))
    with pytest.raises(m.MMFError) as e:
        m.mmf_create(1, 1, S, None, b, 0.0, 1e-13, 12, 1e-12)          # N_t not a power of two
    assert e.value.code == m.MMF_EINVAL
    with pytest.raises(m.MMFError) as e:
        m.mmf_create(1, 3, S, None, np.zeros((3, 4)), 0.0, 1e-13, 64, 1e-12)   # n_pol = 3
    assert e.value.code == m.MMF_EINVAL
    S2 = np.zeros((2, 2, 2, 2)); S2[1, 0, 0, 0] = 1.0                   # violates the parity classes
    with pytest.raises(m.MMFError) as e:
        m.mmf_create(2, 1, S2, np.array([0, 1]), np.zeros((2, 4)), 0.0, 1e-13, 64, 1e-12)
    assert e.value.code == m.MMF_EINVAL
    assert "parity" in m.mmf_last_error()
    assert m.mmf_destroy(0) is None

"""The C-ABI library builds, loads without a GPU and exports every function
declared in include/evoke.h; host-only entry points agree with the oracle."""
import ctypes
import os
import re

import numpy as np

from tests.conftest import ROOT


def declared_functions():
    src = open(os.path.join(ROOT, "include", "evoke.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(evoke_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_header_symbols():
    from paper_1911_10616_gb300 import _lib
    lib = ctypes.CDLL(_lib.library_path())
    names = declared_functions()
    assert len(names) >= 6
    for name in names:
        assert hasattr(lib, name), name
    assert set(_lib.SYMBOLS) == set(names)


def test_strerror_and_version():
    from paper_1911_10616_gb300 import _lib
    lib = _lib.load()
    assert lib.evoke_strerror(0) == b"ok"
    assert lib.evoke_strerror(2).startswith(b"input is not")
    assert _lib.version() >= 100


def test_library_matrix_equals_oracle(oracle_mod):
    import paper_1911_10616_gb300 as ev
    assert np.array_equal(ev.orbit_matrix(), oracle_mod.A_matrix())


def test_null_arguments_rejected_without_gpu_work():
    from paper_1911_10616_gb300 import _lib
    lib = _lib.load()
    assert lib.evoke_orbit_matrix(None) == 1
    assert lib.evoke_count_orbits(None, None, 5, 3, None, None, None) == 1
    assert lib.evoke_plan_status(None, None) == 1


def test_totals_argument_checks_and_empty_input_without_gpu():
    from paper_1911_10616_gb300 import _lib
    lib = _lib.load()
    buf = (ctypes.c_int64 * 30)()
    assert lib.evoke_graphlet_totals(None, 0, 20, buf, None) == 1   # orbits not 73 / 15
    assert lib.evoke_graphlet_totals(None, 5, 73, buf, None) == 1   # counts missing
    assert lib.evoke_graphlet_totals(None, 0, 73, None, None) == 1  # totals missing
    for k in range(30):
        buf[k] = -1
    assert lib.evoke_graphlet_totals(None, 0, 73, buf, None) == 0   # no vertices: all zero
    assert list(buf) == [0] * 30
    assert lib.evoke_strerror(8).startswith(b"orbit counts")

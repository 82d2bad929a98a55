"""The C ABI library builds for sm_103a, loads, and exports every function
that include/o2pic.h declares; argument validation needs no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_0705_0497_gb300 import build, api
    build.build()
    return api.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "o2pic.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(o2pic_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("o2pic_create", "o2pic_set_processes", "o2pic_load_particles", "o2pic_step",
              "o2pic_read_moments", "o2pic_read_particles", "o2pic_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_0705_0497_gb300 import api
    names = declared_functions()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(s[0] for s in api.SIGNATURES) == names


def test_struct_layouts_match_header(lib):
    from paper_0705_0497_gb300 import api
    # o2pic_config: 13 doubles, 4 x 32-bit, 3 x u64, 2 x i32
    assert ctypes.sizeof(api.Config) == 13 * 8 + 4 * 4 + 3 * 8 + 2 * 4
    assert ctypes.sizeof(api.Process) == 4 * 4 + 8 + 2 * 8
    assert ctypes.sizeof(api.Stats) == 8 * (48 + 6 + 3 + 7 + 1 + 3 + 3 + 3 + 1 + 3 + 2 + 2 + 1 + 1)


def test_config_validation_without_gpu(lib):
    from paper_0705_0497_gb300 import api
    c = api.Config()
    assert lib.o2pic_config_init(ctypes.byref(c)) == 0
    assert c.T_gas == 300.0 and c.n_cells == 128
    h = ctypes.c_void_p()
    bad = api.Config()
    lib.o2pic_config_init(ctypes.byref(bad))
    bad.n_cells = 0
    assert lib.o2pic_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad.n_cells = 10000
    assert lib.o2pic_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    lib.o2pic_config_init(ctypes.byref(bad))
    bad.dt = -1.0
    assert lib.o2pic_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    assert lib.o2pic_create(None, ctypes.byref(h)) == -1
    assert lib.o2pic_strerror(-2) == b"particle capacity exceeded"
    assert lib.o2pic_version() == 1


def test_null_context_calls_are_rejected(lib):
    assert lib.o2pic_step(None, 1, None) == -1
    assert lib.o2pic_synchronize(None) == -1
    assert lib.o2pic_set_processes(None, None, 0) == -1


def test_majorant_cap_validation_without_gpu(lib):
    import numpy as np
    caps = np.array([np.nan, 650.0, 650.0])
    assert lib.o2pic_set_majorant_cap(None, caps.ctypes.data) == -1
    assert lib.o2pic_set_majorant_cap(None, None) == -1

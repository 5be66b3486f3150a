"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function include/lbm.h declares, and rejects invalid
geometries before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "lbm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2207_01534_gb300 import lbm

    return lbm.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "lbm_create" in names and "lbm_step" in names and len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def _create(lib, solid, **geo):
    from paper_2207_01534_gb300 import lbm

    nz, ny, nx = solid.shape
    g = lbm.Geometry()
    g.nx, g.ny, g.nz = nx, ny, nz
    s = np.ascontiguousarray(solid, dtype=np.uint8)
    g.solid = s.ctypes.data
    per = geo.get("periodic", (1, 1, 1))
    for a in range(3):
        g.periodic[a] = per[a]
    g.open_axis = geo.get("open_axis", -1)
    p = lbm.Params()
    lib.lbm_default_params(ctypes.byref(p))
    for k, v in geo.get("params", {}).items():
        setattr(p, k, v)
    h = ctypes.c_void_p()
    code = lib.lbm_create(ctypes.byref(g), ctypes.byref(p), ctypes.byref(h))
    return code, lib.lbm_last_error(None).decode()


def test_invalid_geometries_are_rejected_before_device_work(lib):
    solid = np.zeros((6, 6, 6), np.uint8)
    code, msg = _create(lib, solid, periodic=(0, 1, 1))
    assert code == -1 and "closed" in msg
    code, msg = _create(lib, solid, periodic=(1, 1, 1), open_axis=2)
    assert code == -1
    code, msg = _create(lib, solid, periodic=(1, 1, 0), open_axis=0)
    assert code == -7
    s2 = solid.copy()
    s2[1, 2, 2] = 1
    code, msg = _create(lib, s2, periodic=(1, 1, 0), open_axis=2)
    assert code == -1 and "interior" in msg
    code, msg = _create(lib, solid, params={"storage": 9})
    assert code == -7


def test_default_params(lib):
    from paper_2207_01534_gb300 import lbm

    p = lbm.Params()
    assert lib.lbm_default_params(ctypes.byref(p)) == 0
    assert p.G == 3.5 and p.velocity_shift == 1 and tuple(p.tau) == (1.0, 1.0) and p.storage == 0


def test_batch_creation_rejects_bad_arguments_before_device_work(lib):
    from paper_2207_01534_gb300 import lbm

    h = ctypes.c_void_p()
    g = (lbm.Geometry * 1)()
    p = (lbm.Params * 1)()
    assert lib.lbm_create_batch(0, g, p, ctypes.byref(h)) == -1
    assert lib.lbm_create_batch(1, None, None, ctypes.byref(h)) == -1
    # an invalid first sample: nothing is created and the message names it
    solid = np.zeros((6, 6, 6), np.uint8)
    g[0].nx = g[0].ny = g[0].nz = 6
    g[0].solid = solid.ctypes.data
    g[0].periodic[0], g[0].periodic[1], g[0].periodic[2] = 0, 1, 1
    g[0].open_axis = -1
    lib.lbm_default_params(ctypes.byref(p[0]))
    assert lib.lbm_create_batch(1, g, p, ctypes.byref(h)) == -1
    assert h.value is None
    assert lib.lbm_last_error(None).decode().startswith("sample 0:")
    assert lib.lbm_batch_size(None) == 0


def test_binding_constants_match_the_header():
    """The Python binding's status, storage, schedule, plane-rule and field
    constants are the values include/lbm.h declares."""
    import re

    from paper_2207_01534_gb300 import lbm as m

    hdr = open(os.path.join(ROOT, "include", "lbm.h")).read()
    vals = {k: int(v) for k, v in re.findall(r"\b(LBM_[A-Z0-9_]+)\s*=\s*(-?\d+)u?\b", hdr)}
    assert {v: k for k, v in m.STATUS.items()} == {k: vals[k] for k in m.STATUS.values()}
    for name, code in m.STORAGE.items():
        assert vals["LBM_STORE_" + name.upper()] == code
    for name, code in m.KERNEL.items():
        assert vals["LBM_KERNEL_" + name.upper()] == code
    for name, code in m.BC.items():
        assert vals["LBM_BC_" + name.upper()] == code
    for i, name in enumerate(m.FIELDS):
        assert vals["LBM_FIELD_" + name.upper()] == 1 << i

"""Host-side checks of the C ABI (no GPU): the library builds, loads and
exports every function include/nb.h declares; host-side argument checks."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(nb_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_09184_b300 import build
    build.build()
    from paper_2604_09184_b300 import nb
    return nb.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared("nb.h")
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), name


def test_defaults_and_workspace_sizing(lib):
    from paper_2604_09184_b300 import nb
    p = nb.params()
    assert p.G == pytest.approx(2.959122082855911e-4, rel=0, abs=0)
    assert p.hill_factor == 3.0 and p.vel_factor == 0.4 and p.bs_kmax == 8
    small = lib.nb_workspace_bytes(C.byref(p), 256)
    big = lib.nb_workspace_bytes(C.byref(p), 65538)
    assert 0 < small < big
    assert big < 2 * 1024 ** 3
    bad = nb.params(precision=7)
    assert lib.nb_workspace_bytes(C.byref(bad), 256) == 0
    assert lib.nb_workspace_bytes(C.byref(p), 0) == 0


def test_host_side_rejections_need_no_device(lib):
    from paper_2604_09184_b300 import nb
    p = nb.params()
    h = C.c_void_p()
    # n < 1, null inputs and a missing workspace are rejected before any CUDA call
    assert lib.nb_init_system(C.byref(h), C.byref(p), 0, None, None, None, None, None, None,
                              None, 0, None, 0) == nb.NB_E_INVALID
    import numpy as np
    x = np.ones((4, 3))
    ptr = C.c_void_p(x.ctypes.data)
    assert lib.nb_init_system(C.byref(h), C.byref(p), 4, ptr, ptr, ptr, ptr, None, None, None,
                              0, None, 0) == nb.NB_E_WORKSPACE
    assert lib.nb_step(None, 1, 6.0) == nb.NB_E_INVALID
    assert nb.status_string(nb.NB_E_OVERFLOW) == "buffer overflow"


def test_binding_shape_checks_on_host_arrays():
    """The binding's buffer checks: exact shapes, -1 as any extent, a row
    minimum for outputs, and host arrays converted or refused (ValueError)."""
    import numpy as np
    from paper_2604_09184_b300 import nb
    assert nb._shape_ok((5, 3), (5, 3), False)
    assert not nb._shape_ok((4, 3), (5, 3), False)
    assert not nb._shape_ok((5,), (5, 3), False)
    assert not nb._shape_ok((15,), (5,), False)
    assert not nb._shape_ok((5, 2), (5, 3), False)
    assert nb._shape_ok((7, 3), (5, 3), True) and not nb._shape_ok((4, 3), (5, 3), True)
    assert nb._shape_ok((0, 2), (-1, 2), False) and nb._shape_ok((9, 2), (-1, 2), False)
    assert not nb._shape_ok((9, 3), (-1, 2), False)
    a = nb._host_buf("x", [[1, 2, 3], [4, 5, 6]], np.float64, (2, 3))
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    with pytest.raises(ValueError):
        nb._host_buf("x", np.ones(6), np.float64, (2, 3))
    with pytest.raises(ValueError):
        nb._host_buf("m", np.ones(3), np.float64, (4,))
    assert nb._len0(np.ones((4, 3))) == 4 and nb._len0(np.float64(1.0)) == -1

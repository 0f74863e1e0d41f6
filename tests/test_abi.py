"""The C-ABI library loads, exports every symbol include/mot.h declares, and
rejects bad input before touching the GPU."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_07989_gb300.build import build
    build()
    from paper_2510_07989_gb300 import mot as M
    return M.load_library()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mot.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mot_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_exported(lib):
    names = declared_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_abi():
    from paper_2510_07989_gb300 import mot as M
    assert sorted(M.EXPORTED) == declared_symbols()
    for n in declared_symbols():
        assert callable(getattr(M, n))


def test_create_rejects_bad_input(lib):
    from paper_2510_07989_gb300 import mot as M
    from paper_2510_07989_gb300.inputs.meshes import icosphere
    m = icosphere(1)
    with pytest.raises(M.MotError) as e:
        M.mot_create(m.verts, m.tris, 2.0, 1.0, 0.2, 3)        # K < k_max + 1
    assert e.value.code == M.MOT_EINVAL and "k_max" in str(e.value)
    with pytest.raises(M.MotError) as e:
        M.mot_create(m.verts, m.tris[:-1], 2.0, 1.0, 0.2, 40)  # open mesh
    assert e.value.code == M.MOT_EINVAL
    with pytest.raises(M.MotError) as e:
        M.mot_create(m.verts, m.tris, 2.0, 1.0, -0.2, 40)      # dt <= 0
    assert e.value.code == M.MOT_EINVAL
    bad = m.tris.copy()
    bad[0] = bad[0, ::-1]
    with pytest.raises(M.MotError) as e:
        M.mot_create(m.verts, bad, 2.0, 1.0, 0.2, 40)          # inconsistent orientation
    assert e.value.code == M.MOT_EINVAL


def test_run_many_rejects_bad_input_before_any_work(lib):
    """mot_run_many validates its arguments before touching a handle or the GPU."""
    import ctypes
    from paper_2510_07989_gb300 import mot as M
    assert lib.mot_run_many(None, -1, 1, None, None, None, None) == M.MOT_EINVAL
    assert lib.mot_run_many(None, 1, -1, None, None, None, None) == M.MOT_EINVAL
    assert lib.mot_run_many(None, 0, 5, None, None, None, None) == M.MOT_OK  # nothing to march
    assert lib.mot_run_many(None, 1, 5, None, None, None, None) == M.MOT_EINVAL
    # a repeated handle is refused (checked by address only, never dereferenced)
    fake = ctypes.create_string_buffer(64)
    hs = (ctypes.c_void_p * 2)(ctypes.addressof(fake), ctypes.addressof(fake))
    wv = (ctypes.c_void_p * 2)(ctypes.addressof(fake), ctypes.addressof(fake))
    bs = (ctypes.c_int * 2)(1, 1)
    assert lib.mot_run_many(hs, 2, 5, wv, bs, None, None) == M.MOT_EINVAL
    # a NULL handle or wave array among them is refused too
    hs2 = (ctypes.c_void_p * 2)(ctypes.addressof(fake), None)
    assert lib.mot_run_many(hs2, 2, 5, wv, bs, None, None) == M.MOT_EINVAL
    wv2 = (ctypes.c_void_p * 2)(None, ctypes.addressof(fake))
    hs3 = (ctypes.c_void_p * 2)(ctypes.addressof(fake), ctypes.addressof(fake) + 8)
    assert lib.mot_run_many(hs3, 2, 5, wv2, bs, None, None) == M.MOT_EINVAL

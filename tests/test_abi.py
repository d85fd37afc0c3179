"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every symbol include/glint.h declares, and rejects
invalid arguments before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "glint.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(glint_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def glib():
    from paper_2306_05051_gb300 import _lib
    return _lib.lib()


def test_library_exports_every_declared_symbol(glib):
    from paper_2306_05051_gb300 import _lib
    syms = _declared_symbols()
    assert "glint_eval" in syms and "glint_eval_trace" in syms
    for s in syms:
        assert hasattr(glib, s), s
    assert set(syms) == set(_lib.SIGNATURES), set(syms) ^ set(_lib.SIGNATURES)


def test_error_strings_and_version(glib):
    assert glib.glint_error_string(0) == b"ok"
    assert glib.glint_error_string(-1) == b"invalid argument"
    assert glib.glint_version() >= 100


def test_invalid_arguments_rejected_on_host(glib):
    from paper_2306_05051_gb300 import _lib
    from paper_2306_05051_gb300.scenes import Material, Light
    mat = _lib.material_struct(Material())
    lts = _lib.lights_struct([Light(kind=1)])
    fake = 0x1000
    # null frame / null material / bad sizes / bad material: GLINT_ERR_ARG, no device call
    assert glib.glint_eval(None, C.byref(mat), lts, fake, None) == -1
    fr = _lib.GlintFrame(fake, None, None, 0, 8, 1)
    assert glib.glint_eval(C.byref(fr), C.byref(mat), lts, fake, None) == -1
    fr = _lib.GlintFrame(fake, None, None, 8, 8, 9)
    assert glib.glint_eval(C.byref(fr), C.byref(mat), lts, fake, None) == -1
    fr = _lib.GlintFrame(fake, None, None, 8, 8, 1)
    for field, bad in (("n_lods", 1), ("n_rings", 7), ("lod_factor", 3), ("max_sub", 65), ("ndf", 2), ("R", 0.0),
                       ("gamma", -1.0), ("alpha_x", 0.0)):
        m = _lib.material_struct(Material())
        setattr(m, field, bad)
        assert glib.glint_eval(C.byref(fr), C.byref(m), lts, fake, None) == -1, field
    # a point light without a light plane
    pl = _lib.lights_struct([Light(kind=0)])
    assert glib.glint_eval(C.byref(fr), C.byref(mat), pl, fake, None) == -1
    # host-buffer path: staging size and a too-small staging buffer
    assert glib.glint_eval_host_staging_size(8, 8, 1, 0, 0) >= 8 * 8 * 68
    assert glib.glint_eval_host_staging_size(0, 8, 1, 0, 0) == 0
    assert glib.glint_eval_host(C.byref(fr), C.byref(mat), lts, fake, fake, 16, None) == -6
    # trace with no pixels
    assert glib.glint_eval_trace(C.byref(fr), C.byref(mat), lts, fake, 0, fake, fake, 1, None) == -1

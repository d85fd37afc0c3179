"""ctypes binding of libglint.so (include/glint.h).  Argument marshalling
only: every step of the glint evaluation runs in the library's kernels.
There is no fallback: if the library cannot be loaded, every call raises."""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

GLINT_OK = 0
ERRORS = {-1: "GLINT_ERR_ARG", -2: "GLINT_ERR_ALIGN", -3: "GLINT_ERR_NOT_DEVICE_PTR", -4: "GLINT_ERR_CUDA",
          -5: "GLINT_ERR_UNSUPPORTED", -6: "GLINT_ERR_WORKSPACE"}


class GlintError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({lib().glint_error_string(code).decode()})")


class GlintMaterial(C.Structure):
    _fields_ = [("ndf", C.c_int32), ("alpha_x", C.c_float), ("alpha_y", C.c_float), ("ln_density", C.c_float),
                ("R", C.c_float), ("F0", C.c_float), ("gamma", C.c_float), ("n_lods", C.c_int32),
                ("n_rings", C.c_int32), ("lod_factor", C.c_int32), ("max_sub", C.c_int32), ("seed", C.c_uint32),
                ("lod_blend", C.c_int32), ("sampler", C.c_int32), ("rng_table", C.c_int32)]


class GlintLight(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dir", C.c_float * 3), ("intensity", C.c_float)]


class GlintLaunch(C.Structure):
    _fields_ = [("threads_per_cta", C.c_int32), ("ctas_per_sm", C.c_int32)]


MAX_WAVES = 32


class GlintCamera(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("fwd", C.c_double * 3), ("right", C.c_double * 3), ("up", C.c_double * 3),
                ("tan_half_fov", C.c_double), ("width", C.c_int32), ("height", C.c_int32)]


class GlintHeightfield(C.Structure):
    _fields_ = [("n_waves", C.c_int32), ("n_march", C.c_int32), ("n_bisect", C.c_int32), ("pad", C.c_int32),
                ("kx", C.c_double * MAX_WAVES), ("kz", C.c_double * MAX_WAVES), ("phase", C.c_double * MAX_WAVES),
                ("amp", C.c_double * MAX_WAVES), ("uv_scale", C.c_double)]


class GlintSpherePlane(C.Structure):
    _fields_ = [("center", C.c_double * 3), ("radius", C.c_double), ("sphere_uv_scale", C.c_double),
                ("plane_half_extent", C.c_double), ("plane_uv_scale", C.c_double), ("plane_uv_wrap", C.c_double),
                ("n_lights", C.c_int32), ("noise_cell", C.c_int32), ("noise_w", C.c_int32), ("noise_h", C.c_int32),
                ("light_pos", (C.c_double * 3) * 8), ("light_I", C.c_double * 8),
                ("noise_alpha", C.c_void_p), ("noise_log10_density", C.c_void_p)]


class GlintFrame(C.Structure):
    _fields_ = [("gbuf", C.c_void_p), ("light_px", C.c_void_p), ("mat_px", C.c_void_p),
                ("width", C.c_int32), ("height", C.c_int32), ("n_lights", C.c_int32)]


TRACE_PIX_DTYPE = np.dtype([("status", "i4"), ("K", "i4"), ("n_rec", "i4"), ("n_can_open", "i4"),
                            ("A", "f4"), ("r", "f4"), ("phi", "f4"), ("out", "f4")])
TRACE_REC_DTYPE = np.dtype([("light", "i4"), ("sub", "i4"), ("vert", "i4"), ("sv", "i4"), ("av", "i4"),
                            ("gid", "u4"), ("i", "i4"), ("j", "i4"), ("ax", "i4"), ("ay", "i4"),
                            ("h0", "u4"), ("h1", "u4"), ("gate", "i4"), ("c", "i4"),
                            ("n", "f4"), ("P1", "f4"), ("mu", "f4"), ("sigma", "f4"), ("c_cont", "f4"),
                            ("u", "f4"), ("v", "f4"), ("p", "f4")])

# every symbol include/glint.h declares, with (restype, argtypes)
_P = C.c_void_p
SIGNATURES = {
    "glint_error_string": (C.c_char_p, [C.c_int]),
    "glint_version": (C.c_int, []),
    "glint_eval": (C.c_int, [_P, _P, _P, _P, _P]),
    "glint_eval_launch": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "glint_eval_host_staging_size": (C.c_size_t, [C.c_int32] * 5),
    "glint_eval_host": (C.c_int, [_P, _P, _P, _P, _P, C.c_size_t, _P]),
    "glint_eval_trace": (C.c_int, [_P, _P, _P, _P, C.c_int32, _P, _P, C.c_int32, _P]),
    "glint_ctx_create": (C.c_int, [_P]),
    "glint_ctx_destroy": (None, [_P]),
    "glint_ctx_get_launch": (C.c_int, [_P, _P]),
    "glint_ctx_set_launch": (C.c_int, [_P, _P]),
    "glint_eval_batch": (C.c_int, [_P, _P, C.c_int32, _P, _P, _P, _P]),
    "glint_eval_batch_noalloc": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P]),
    "glint_backward_workspace_size": (C.c_size_t, [_P]),
    "glint_backward": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, C.c_size_t, _P]),
    "glint_fit_l2": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, C.c_size_t, _P]),
    "glint_gbuffer_heightfield": (C.c_int, [_P, _P, _P, _P]),
    "glint_gbuffer_sphere_plane": (C.c_int, [_P, _P, _P, _P, _P, _P]),
}


def lib():
    """Load (building first if needed) libglint.so."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(rc, what):
    if rc != GLINT_OK:
        raise GlintError(rc, what)


def material_struct(m) -> GlintMaterial:
    return GlintMaterial(int(m.ndf), float(m.alpha_x), float(m.alpha_y), float(m.ln_density), float(m.R),
                         float(m.F0), float(m.gamma), int(m.n_lods), int(m.n_rings), int(m.lod_factor),
                         int(m.max_sub), int(m.seed) & 0xFFFFFFFF, int(getattr(m, "lod_blend", 0)),
                         int(getattr(m, "sampler", 0)), int(getattr(m, "rng_table", 0)))


def lights_struct(lights):
    arr = (GlintLight * max(1, len(lights)))()
    for k, L in enumerate(lights):
        arr[k].kind = int(L.kind)
        for c in range(3):
            arr[k].dir[c] = float(L.dir[c])
        arr[k].intensity = float(L.intensity)
    return arr


def frame_struct(gbuf, light_px, mat_px, n_lights) -> GlintFrame:
    H, W = int(gbuf.shape[0]), int(gbuf.shape[1])
    ptr = lambda t: None if t is None else t.data_ptr()
    return GlintFrame(ptr(gbuf), ptr(light_px), ptr(mat_px), W, H, int(n_lights))

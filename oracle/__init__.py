"""ctypes binding of the FP64 CPU oracle (oracle/glint_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by bench.py's CPU-baseline leg.  The CUDA library never imports this package.

The oracle is compiled from source with g++ on first use (or by build()),
into oracle/_build/, so the same file serves the x86 build host and the Arm
GPU host.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glint_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libglint_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (g++, -O2, OpenMP, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OMaterial(C.Structure):
    _fields_ = [("ndf", C.c_int32), ("alpha_x", C.c_float), ("alpha_y", C.c_float),
                ("ln_density", C.c_float), ("R", C.c_float), ("F0", C.c_float), ("gamma", C.c_float),
                ("n_lods", C.c_int32), ("n_rings", C.c_int32), ("lod_factor", C.c_int32),
                ("max_sub", C.c_int32), ("seed", C.c_uint32), ("lod_blend", C.c_int32), ("sampler", C.c_int32),
                ("rng_table", C.c_int32)]


class OLight(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dir", C.c_float * 3), ("intensity", C.c_float)]


PIX_DTYPE = np.dtype([("status", "i4"), ("K", "i4"), ("Kmaj", "i4"), ("k", "i4"),
                      ("A", "f8"), ("r", "f8"), ("phi", "f8"), ("s0", "f8"), ("s1", "f8"),
                      ("out", "f8")], align=True)

REC_DTYPE = np.dtype([("light", "i4"), ("sub", "i4"), ("vert", "i4"), ("sv", "i4"), ("av", "i4"),
                      ("level", "i4"), ("ring", "i4"), ("kor", "i4"), ("tri", "i4"), ("tet", "i4"),
                      ("pinned", "i4"), ("gid", "u4"), ("i", "i4"), ("j", "i4"), ("ax", "i4"),
                      ("ay", "i4"), ("h0", "u4"), ("h1", "u4"), ("gate", "i4"), ("c", "i4"),
                      ("n", "f8"), ("p", "f8"), ("P1", "f8"), ("mu", "f8"), ("sigma", "f8"),
                      ("z", "f8"), ("c_cont", "f8"), ("u", "f8"), ("v", "f8"),
                      ("x", "f8"), ("t", "f8"), ("s", "f8"), ("As", "f8"), ("qx", "f8"),
                      ("qy", "f8"), ("afx", "f8"), ("afy", "f8"), ("w", "f8")], align=True)

_P = C.c_void_p
_D = C.c_double
_I = C.c_int


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.oracle_eval.argtypes = [_P, _P, _P, _I, _I, C.POINTER(OMaterial), _P, _I, _P, _I, _I, _P, _I]
            L.oracle_trace.argtypes = [_P, _P, _P, _I, _I, C.POINTER(OMaterial), _P, _I, _I, _P, _P, _I, _P]
            L.oracle_grad.argtypes = [_P, _P, _I, _I, C.POINTER(OMaterial), _P, _I, _I, _P, _I, _P,
                                      _P, _P, _P, _I]
            L.oracle_phi_inv.argtypes = [_D]; L.oracle_phi_inv.restype = _D
            L.oracle_pcg4d.argtypes = [_P]; L.oracle_pcg3d.argtypes = [_P]
            L.oracle_fmix32.argtypes = [C.c_uint32]; L.oracle_fmix32.restype = C.c_uint32
            L.oracle_grid_id.argtypes = [_I, _I, _I]; L.oracle_grid_id.restype = C.c_uint32
            L.oracle_eval_hash.argtypes = [C.c_int32, C.c_int32, C.c_uint32, C.c_int32, C.c_int32,
                                           C.c_uint32, _P]
            L.oracle_theta.argtypes = [C.c_uint32]; L.oracle_theta.restype = _D
            L.oracle_table_words.argtypes = [C.c_uint32, _P]
            L.oracle_eval_table.argtypes = [C.c_int32, C.c_int32, C.c_uint32, C.c_int32, C.c_int32, C.c_uint32, _P]
            L.oracle_ndf.argtypes = [_I, _D, _D, _D, _D, _D]; L.oracle_ndf.restype = _D
            L.oracle_smith_lambda.argtypes = [_I, _D, _D, _D, _D, _D]; L.oracle_smith_lambda.restype = _D
            L.oracle_footprint.argtypes = [_D, _D, _D, _D, _P]
            L.oracle_split.argtypes = [_D, _D, _I, _I, _I, _I, _P]
            L.oracle_lod.argtypes = [_D, _I, _I, _P, _P]
            L.oracle_cell.argtypes = [_D, _D, _I, _P, _P]
            L.oracle_tet.argtypes = [_P, _D, _P, _P]
            L.oracle_grid_coords.argtypes = [_D, _D, _I, _I, _I, _D, _I, _P]
            L.oracle_simplex.argtypes = [_D, _D, _P, _P]
            L.oracle_gated_count.argtypes = [_D, _D, _D, _D, _P]; L.oracle_gated_count.restype = _I
            L.oracle_exact_count.argtypes = [_I, _D, _D]; L.oracle_exact_count.restype = _I
            L.oracle_classical_count.argtypes = [_D, _D, C.c_uint32, C.c_uint32, _P]
            L.oracle_classical_count.restype = _I
            sizes = np.zeros(4, np.int32)
            L.oracle_struct_sizes(sizes.ctypes.data_as(_P))
            assert sizes[0] == C.sizeof(OMaterial) and sizes[1] == C.sizeof(OLight), sizes
            assert sizes[2] == PIX_DTYPE.itemsize and sizes[3] == REC_DTYPE.itemsize, sizes
            _lib = L
    return _lib


# --------------------------------------------------------------------------
# scene marshalling
# --------------------------------------------------------------------------
def _np(t):
    if t is None:
        return None
    if hasattr(t, "detach"):
        t = t.detach().cpu().numpy()
    return np.ascontiguousarray(t, dtype=np.float32)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_P)


def _material(m) -> OMaterial:
    return OMaterial(int(m.ndf), float(m.alpha_x), float(m.alpha_y), float(m.ln_density), float(m.R),
                     float(m.F0), float(m.gamma), int(m.n_lods), int(m.n_rings), int(m.lod_factor),
                     int(m.max_sub), int(m.seed) & 0xFFFFFFFF, int(getattr(m, "lod_blend", 0)),
                     int(getattr(m, "sampler", 0)), int(getattr(m, "rng_table", 0)))


def _lights(lights):
    arr = (OLight * max(1, len(lights)))()
    for k, L in enumerate(lights):
        arr[k].kind = int(L.kind)
        for c in range(3):
            arr[k].dir[c] = float(L.dir[c])
        arr[k].intensity = float(L.intensity)
    return arr


class _Marshalled:
    def __init__(self, scene, material=None, lights=None):
        self.gbuf = _np(scene.gbuf)
        self.light_px = _np(scene.light_px)
        self.mat_px = _np(scene.mat_px)
        self.H, self.W = self.gbuf.shape[:2]
        self.mat = _material(material or scene.material)
        lt = lights if lights is not None else scene.lights
        self.lights = _lights(lt)
        self.nL = len(lt)


def eval_image(scene, px=None, relaxed=False, threads=0, material=None, lights=None):
    """Radiance of every pixel ([H, W] float64) or of the flat pixel indices px."""
    m = _Marshalled(scene, material, lights)
    pl = None if px is None else np.ascontiguousarray(px, dtype=np.int32)
    n = m.W * m.H if pl is None else len(pl)
    out = np.zeros(n, np.float64)
    rc = lib().oracle_eval(_ptr(m.gbuf), _ptr(m.light_px), _ptr(m.mat_px), m.W, m.H, C.byref(m.mat),
                           m.lights, m.nL, _ptr(pl), n, int(relaxed), _ptr(out), int(threads))
    if rc != 0:
        raise ValueError("oracle_eval rejected its arguments")
    return out.reshape(m.H, m.W) if pl is None else out


def trace_pixel(scene, px, cap=200000, material=None, lights=None):
    """(pixel summary record, evaluation records) of flat pixel index px."""
    m = _Marshalled(scene, material, lights)
    pix = np.zeros(1, PIX_DTYPE)
    recs = np.zeros(cap, REC_DTYPE)
    nrec = np.zeros(1, np.int32)
    rc = lib().oracle_trace(_ptr(m.gbuf), _ptr(m.light_px), _ptr(m.mat_px), m.W, m.H, C.byref(m.mat),
                            m.lights, m.nL, int(px), _ptr(pix), _ptr(recs), cap, _ptr(nrec))
    if rc != 0:
        raise ValueError("oracle_trace rejected its arguments")
    return pix[0], recs[: min(int(nrec[0]), cap)]


def grad(scene, grad_out, px=None, grad_light=0, threads=0, material=None, lights=None,
         per_pixel=False):
    """FP64 gradient of sum(grad_out * relaxed image) with respect to
    (alpha_x, alpha_y, ln density, light[grad_light].dir xyz).
    Returns (grad6, per-pixel [n, 6] or None, relaxed image values)."""
    m = _Marshalled(scene, material, lights)
    if m.mat_px is not None:
        raise ValueError("gradients need the scalar material")
    pl = None if px is None else np.ascontiguousarray(px, dtype=np.int32)
    n = m.W * m.H if pl is None else len(pl)
    go = np.ascontiguousarray(np.asarray(grad_out, np.float64).reshape(-1))
    assert go.size == n
    g6 = np.zeros(6, np.float64)
    pp = np.zeros((n, 6), np.float64) if per_pixel else None
    rel = np.zeros(n, np.float64)
    rc = lib().oracle_grad(_ptr(m.gbuf), _ptr(m.light_px), m.W, m.H, C.byref(m.mat), m.lights, m.nL,
                           int(grad_light), _ptr(pl), n, _ptr(go), _ptr(g6), _ptr(pp), _ptr(rel),
                           int(threads))
    if rc != 0:
        raise ValueError("oracle_grad rejected its arguments")
    return g6, pp, rel


# --------------------------------------------------------------------------
# single pieces (unit tests)
# --------------------------------------------------------------------------
def phi_inv(P):
    return lib().oracle_phi_inv(float(P))


def pcg4d(v):
    a = np.array(v, np.uint32)
    lib().oracle_pcg4d(a.ctypes.data_as(_P))
    return a


def pcg3d(v):
    a = np.array(v, np.uint32)
    lib().oracle_pcg3d(a.ctypes.data_as(_P))
    return a


def fmix32(h):
    return lib().oracle_fmix32(int(h) & 0xFFFFFFFF)


def grid_id(level, ring, kor):
    return lib().oracle_grid_id(level, ring, kor)


def eval_hash(i, j, gid, ax, ay, seed):
    h = np.zeros(2, np.uint32)
    lib().oracle_eval_hash(int(i), int(j), int(gid) & 0xFFFFFFFF, int(ax), int(ay),
                           int(seed) & 0xFFFFFFFF, h.ctypes.data_as(_P))
    return int(h[0]), int(h[1])


def table_words(k):
    h = np.zeros(2, np.uint32)
    lib().oracle_table_words(int(k) & 0xFFFFFFFF, h.ctypes.data_as(_P))
    return int(h[0]), int(h[1])


def eval_table(i, j, gid, ax, ay, seed):
    h = np.zeros(2, np.uint32)
    lib().oracle_eval_table(int(i), int(j), int(gid) & 0xFFFFFFFF, int(ax), int(ay), int(seed) & 0xFFFFFFFF,
                            h.ctypes.data_as(_P))
    return int(h[0]), int(h[1])


def theta(h):
    return lib().oracle_theta(int(h) & 0xFFFFFFFF)


def ndf(kind, ax, ay, ht, hb, hn):
    return lib().oracle_ndf(kind, ax, ay, ht, hb, hn)


def smith_lambda(kind, ax, ay, wt, wb, wn):
    return lib().oracle_smith_lambda(kind, ax, ay, wt, wb, wn)


def footprint(a, b, c, d):
    """(sigma0, sigma1, phi, P, r) of J = [[a, b], [c, d]]."""
    o = np.zeros(5)
    lib().oracle_footprint(a, b, c, d, o.ctypes.data_as(_P))
    return tuple(o)


def split(r, A, M=4, L=8, f=4, Kmax=64):
    o = np.zeros(3, np.int32)
    lib().oracle_split(r, A, M, L, f, Kmax, o.ctypes.data_as(_P))
    return tuple(int(x) for x in o)


def lod(As, f=4, L=8):
    i = np.zeros(2, np.int32); d = np.zeros(1)
    lib().oracle_lod(As, f, L, i.ctypes.data_as(_P), d.ctypes.data_as(_P))
    return int(i[0]), float(d[0]), bool(i[1])


def cell(rho_r, phi, M=4):
    """(m, tri, [(ring, kor) x 3], x, t, [lam x 3])"""
    i = np.zeros(8, np.int32); d = np.zeros(5)
    lib().oracle_cell(rho_r, phi, M, i.ctypes.data_as(_P), d.ctypes.data_as(_P))
    verts = [(int(i[2 + 2 * k]), int(i[3 + 2 * k])) for k in range(3)]
    return int(i[0]), int(i[1]), verts, float(d[0]), float(d[1]), d[2:5].copy()


def tet(lam3, s):
    """(tet index, [(upper, triangle vertex) x 4], weights[4])"""
    lam = np.ascontiguousarray(lam3, np.float64)
    i = np.zeros(9, np.int32); w = np.zeros(4)
    lib().oracle_tet(lam.ctypes.data_as(_P), s, i.ctypes.data_as(_P), w.ctypes.data_as(_P))
    return int(i[0]), [(int(i[1 + 2 * k]), int(i[2 + 2 * k])) for k in range(4)], w


def grid_coords(u, v, level, ring, kor, rho, f=4):
    q = np.zeros(2)
    lib().oracle_grid_coords(u, v, level, ring, kor, rho, f, q.ctypes.data_as(_P))
    return float(q[0]), float(q[1])


def simplex(qx, qy):
    i = np.zeros(6, np.int32); w = np.zeros(3)
    lib().oracle_simplex(qx, qy, i.ctypes.data_as(_P), w.ctypes.data_as(_P))
    return [(int(i[2 * k]), int(i[2 * k + 1])) for k in range(3)], w


def classical_count(n, p, h0, h1):
    """(c, z, c_cont) of the classical sampler for words h0, h1."""
    d = np.zeros(2)
    c = lib().oracle_classical_count(float(n), float(p), int(h0) & 0xFFFFFFFF, int(h1) & 0xFFFFFFFF,
                                     d.ctypes.data_as(_P))
    return int(c), float(d[0]), float(d[1])


def exact_count(N, p, theta):
    """Exact sampler: inverse of the Bin(N, p) CDF at theta (integer N)."""
    return int(lib().oracle_exact_count(int(N), float(p), float(theta)))


def gated_count(n, p, th0, th1):
    """(c, P1, mu, sigma, z, c_cont, relaxed)"""
    d = np.zeros(6)
    c = lib().oracle_gated_count(n, p, th0, th1, d.ctypes.data_as(_P))
    return (c,) + tuple(float(x) for x in d)

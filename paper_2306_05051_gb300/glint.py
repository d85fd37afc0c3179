"""Python API over the C ABI (include/glint.h).  PyTorch provides device
memory and streams; every step of the glint evaluation runs in libglint.so.

    img = render(gbuf, light_px, mat_px, material, lights)      # device tensors
    img = render_scene(scene)
    pix, recs = trace(scene, pixels)                             # parity records
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from .scenes import Light, Material, Scene


def _stream_handle(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check_plane(t, name, shape_tail, device=None, host=False):
    if t is None:
        return
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 tensor")
    if host:
        if t.is_cuda:
            raise ValueError(f"{name} must be a host tensor")
    elif not t.is_cuda or (device is not None and t.device != device):
        raise ValueError(f"{name} must live on {device}")
    if tuple(t.shape[-len(shape_tail):]) != tuple(shape_tail):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected [..., {shape_tail}]")


def render(gbuf: torch.Tensor, light_px: Optional[torch.Tensor] = None, mat_px: Optional[torch.Tensor] = None,
           material: Material = Material(), lights: Sequence[Light] = (), out: Optional[torch.Tensor] = None,
           stream=None, launch=None) -> torch.Tensor:
    """Glint radiance [H, W] of one G-buffer frame (glint_eval; with
    launch = (threads_per_cta, ctas_per_sm), glint_eval_launch)."""
    _check_plane(gbuf, "gbuf", (16,))
    if gbuf.dim() != 3:
        raise ValueError(f"gbuf has shape {tuple(gbuf.shape)}, expected [H, W, 16]")
    dev = gbuf.device
    H, W = int(gbuf.shape[0]), int(gbuf.shape[1])
    _check_plane(light_px, "light_px", (H, W, 4), dev)
    _check_plane(mat_px, "mat_px", (H, W, 2), dev)
    if out is None:
        out = torch.empty(H, W, dtype=torch.float32, device=dev)
    _check_plane(out, "out", (H, W), dev)
    frame = _lib.frame_struct(gbuf, light_px, mat_px, len(lights))
    mat = _lib.material_struct(material)
    lts = _lib.lights_struct(lights)
    with torch.cuda.device(dev):
        if launch is None:
            rc = _lib.lib().glint_eval(C.byref(frame), C.byref(mat), lts, out.data_ptr(), _stream_handle(stream))
        else:
            cfg = _lib.GlintLaunch(int(launch[0]), int(launch[1]))
            rc = _lib.lib().glint_eval_launch(C.byref(frame), C.byref(mat), lts, out.data_ptr(), C.byref(cfg),
                                              _stream_handle(stream))
    _lib.check(rc, "glint_eval")
    return out


def render_scene(scene: Scene, out=None, stream=None, material=None, lights=None, launch=None) -> torch.Tensor:
    return render(scene.gbuf, scene.light_px, scene.mat_px, material or scene.material,
                  scene.lights if lights is None else lights, out=out, stream=stream, launch=launch)


def staging_bytes(scene: Scene) -> int:
    return int(_lib.lib().glint_eval_host_staging_size(scene.width, scene.height, len(scene.lights),
                                                       int(scene.light_px is not None),
                                                       int(scene.mat_px is not None)))


def render_host(scene: Scene, staging: torch.Tensor, out_host: torch.Tensor, stream=None) -> torch.Tensor:
    """glint_eval_host: host planes in, host image out, copies enqueued on the
    stream (synchronise before reading out_host)."""
    H, W = scene.height, scene.width
    _check_plane(scene.gbuf, "gbuf", (16,), host=True)
    _check_plane(scene.light_px, "light_px", (H, W, 4), host=True)
    _check_plane(scene.mat_px, "mat_px", (H, W, 2), host=True)
    _check_plane(out_host, "out_host", (H, W), host=True)
    if not staging.is_cuda:
        raise ValueError("staging must be device memory")
    frame = _lib.frame_struct(scene.gbuf, scene.light_px, scene.mat_px, len(scene.lights))
    mat = _lib.material_struct(scene.material)
    lts = _lib.lights_struct(scene.lights)
    nbytes = staging.numel() * staging.element_size()
    with torch.cuda.device(staging.device):
        rc = _lib.lib().glint_eval_host(C.byref(frame), C.byref(mat), lts, out_host.data_ptr(),
                                        staging.data_ptr(), nbytes, _stream_handle(stream))
    _lib.check(rc, "glint_eval_host")
    return out_host


def trace(scene: Scene, pixels, cap: Optional[int] = None, stream=None, material=None, lights=None):
    """Parity records of the listed flat pixel indices (glint_eval_trace).
    Returns (pix [n], recs [n, cap]) numpy structured arrays; record slots that
    were not written hold light = -1."""
    dev = scene.gbuf.device
    px = torch.as_tensor(np.asarray(pixels, np.int32), device=dev)
    n = int(px.numel())
    lts_list = scene.lights if lights is None else lights
    if cap is None:
        cap = max(1, len(lts_list)) * 48 * 64
    pix = torch.zeros(n * _lib.TRACE_PIX_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    recs = torch.full((n * cap * _lib.TRACE_REC_DTYPE.itemsize,), 0xFF, dtype=torch.uint8, device=dev)
    frame = _lib.frame_struct(scene.gbuf, scene.light_px, scene.mat_px, len(lts_list))
    mat = _lib.material_struct(material or scene.material)
    lts = _lib.lights_struct(lts_list)
    with torch.cuda.device(dev):
        rc = _lib.lib().glint_eval_trace(C.byref(frame), C.byref(mat), lts, px.data_ptr(), n, pix.data_ptr(),
                                         recs.data_ptr(), cap, _stream_handle(stream))
        _lib.check(rc, "glint_eval_trace")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    p = pix.cpu().numpy().view(_lib.TRACE_PIX_DTYPE)
    r = recs.cpu().numpy().view(_lib.TRACE_REC_DTYPE).reshape(n, cap)
    return p, r


class BatchContext:
    """Batched evaluation context (glint_ctx_* / glint_eval_batch): one
    persistent launch over many frames, recorded in a CUDA graph and
    replayed; the launch shape is tuned on the first batch of a shape."""

    def __init__(self, device=None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._h = C.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(_lib.lib().glint_ctx_create(C.byref(self._h)), "glint_ctx_create")

    def close(self):
        if self._h:
            _lib.lib().glint_ctx_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launch(self):
        L = _lib.GlintLaunch()
        rc = _lib.lib().glint_ctx_get_launch(self._h, C.byref(L))
        return None if rc else (int(L.threads_per_cta), int(L.ctas_per_sm))

    @launch.setter
    def launch(self, value):
        L = _lib.GlintLaunch(int(value[0]), int(value[1]))
        _lib.check(_lib.lib().glint_ctx_set_launch(self._h, C.byref(L)), "glint_ctx_set_launch")

    def render(self, scenes_list, outs=None, stream=None, material=None, lights=None):
        """Shade every scene (same material and light descriptors) into outs
        (list of [H, W] device tensors, allocated when None)."""
        n = len(scenes_list)
        first = scenes_list[0]
        material = material or first.material
        lights = first.lights if lights is None else lights
        if outs is None:
            outs = [torch.empty(s.height, s.width, dtype=torch.float32, device=self.device) for s in scenes_list]
        frames = (_lib.GlintFrame * n)()
        for k, s in enumerate(scenes_list):
            _check_plane(s.gbuf, "gbuf", (16,), self.device)
            _check_plane(s.light_px, "light_px", (s.height, s.width, 4), self.device)
            _check_plane(s.mat_px, "mat_px", (s.height, s.width, 2), self.device)
            _check_plane(outs[k], "out", (s.height, s.width), self.device)
            frames[k] = _lib.frame_struct(s.gbuf, s.light_px, s.mat_px, len(lights))
        optr = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
        mat = _lib.material_struct(material)
        lts = _lib.lights_struct(lights)
        with torch.cuda.device(self.device):
            rc = _lib.lib().glint_eval_batch(self._h, frames, n, C.byref(mat), lts, optr, _stream_handle(stream))
        _lib.check(rc, "glint_eval_batch")
        return outs


def backward_workspace_bytes(scene: Scene, lights=None) -> int:
    lights = scene.lights if lights is None else lights
    frame = _lib.frame_struct(scene.gbuf, scene.light_px, scene.mat_px, len(lights))
    return int(_lib.lib().glint_backward_workspace_size(C.byref(frame)))


def backward(scene: Scene, grad_out: torch.Tensor, material=None, lights=None, relaxed=False, stream=None,
             workspace=None, grad=None, out_relaxed=None):
    """glint_backward: gradient of sum(grad_out * relaxed image) with respect
    to (alpha_x, alpha_y, ln_density, light directions).  Returns the
    gradient (3 + 3 * n_lights floats, device) and the relaxed image when
    requested.  workspace (float64 device tensor), grad and out_relaxed may be
    passed in to avoid allocations."""
    material = material or scene.material
    lights = scene.lights if lights is None else lights
    dev = scene.gbuf.device
    H, W = scene.height, scene.width
    _check_plane(grad_out, "grad_out", (H, W), dev)
    frame = _lib.frame_struct(scene.gbuf, scene.light_px, scene.mat_px, len(lights))
    nbytes = int(_lib.lib().glint_backward_workspace_size(C.byref(frame)))
    ws = workspace if workspace is not None else torch.empty(max(nbytes, 8) // 8 + 1, dtype=torch.float64, device=dev)
    if grad is None:
        grad = torch.empty(3 + 3 * len(lights), dtype=torch.float32, device=dev)
    rel = out_relaxed if out_relaxed is not None else (
        torch.empty(H, W, dtype=torch.float32, device=dev) if relaxed else None)
    mat = _lib.material_struct(material)
    lts = _lib.lights_struct(lights)
    with torch.cuda.device(dev):
        rc = _lib.lib().glint_backward(C.byref(frame), C.byref(mat), lts, grad_out.data_ptr(), grad.data_ptr(),
                                       None if rel is None else rel.data_ptr(), ws.data_ptr(),
                                       ws.numel() * 8, _stream_handle(stream))
    _lib.check(rc, "glint_backward")
    return (grad, rel) if (relaxed or out_relaxed is not None) else grad


def fit_l2(scene: Scene, target: torch.Tensor, material=None, lights=None, stream=None, workspace=None,
           out=None, grad=None, loss=None):
    """glint_fit_l2: one pass giving the image (out), the L2 loss
    sum((out - target)^2) and its gradient with respect to (alpha_x,
    alpha_y, ln_density, light directions), through the relaxed counts.
    Returns (out, grad, loss) as device tensors."""
    material = material or scene.material
    lights = scene.lights if lights is None else lights
    dev = scene.gbuf.device
    H, W = scene.height, scene.width
    _check_plane(target, "target", (H, W), dev)
    frame = _lib.frame_struct(scene.gbuf, scene.light_px, scene.mat_px, len(lights))
    nbytes = int(_lib.lib().glint_backward_workspace_size(C.byref(frame)))
    ws = workspace if workspace is not None else torch.empty(max(nbytes, 8) // 8 + 1, dtype=torch.float64, device=dev)
    out = out if out is not None else torch.empty(H, W, dtype=torch.float32, device=dev)
    _check_plane(out, "out", (H, W), dev)
    grad = grad if grad is not None else torch.empty(3 + 3 * len(lights), dtype=torch.float32, device=dev)
    loss = loss if loss is not None else torch.empty(1, dtype=torch.float32, device=dev)
    mat = _lib.material_struct(material)
    lts = _lib.lights_struct(lights)
    with torch.cuda.device(dev):
        rc = _lib.lib().glint_fit_l2(C.byref(frame), C.byref(mat), lts, target.data_ptr(), out.data_ptr(),
                                     grad.data_ptr(), loss.data_ptr(), ws.data_ptr(), ws.numel() * 8,
                                     _stream_handle(stream))
    _lib.check(rc, "glint_fit_l2")
    return out, grad, loss


class GlintBRDF(torch.autograd.Function):
    """Glint image as a differentiable function of the scalar material
    roughness, ln flake density and the directions of directional lights.
    Forward: the glint image (integer counts).  Backward: the gradient of the
    relaxed image (counts before integer rounding), discrete choices fixed.

        img = GlintBRDF.apply(alpha_x, alpha_y, ln_density, light_dirs, scene)
    alpha_x, alpha_y, ln_density: 0-d tensors; light_dirs: [n_lights, 3]."""

    @staticmethod
    def forward(ctx, alpha_x, alpha_y, ln_density, light_dirs, scene):
        import dataclasses
        mat = dataclasses.replace(scene.material, alpha_x=float(alpha_x), alpha_y=float(alpha_y),
                                  ln_density=float(ln_density))
        dirs = light_dirs.detach().cpu().tolist()
        lights = [dataclasses.replace(L, dir=tuple(dirs[k])) if L.kind == 1 else L
                  for k, L in enumerate(scene.lights)]
        ctx.scene, ctx.mat, ctx.lights = scene, mat, lights
        ctx.dev_dtype = (alpha_x.device, alpha_x.dtype, light_dirs.device, light_dirs.dtype)
        return render_scene(scene, material=mat, lights=lights)

    @staticmethod
    def backward(ctx, grad_out):
        g = backward(ctx.scene, grad_out.contiguous().float(), material=ctx.mat, lights=ctx.lights)
        adev, adt, ddev, ddt = ctx.dev_dtype
        ga = g[:3].to(device=adev, dtype=adt)
        gd = g[3:].reshape(-1, 3).to(device=ddev, dtype=ddt)
        return ga[0], ga[1], ga[2], gd, None


# --------------------------------------------------------------------------
# synthetic G-buffers generated on the GPU (glint_gbuffer_*)
# --------------------------------------------------------------------------
def _camera_struct(cam, tan_half_fov, W, H):
    eye, fwd, right, up = (t.detach().cpu().double().tolist() for t in cam)
    return _lib.GlintCamera((C.c_double * 3)(*eye), (C.c_double * 3)(*fwd), (C.c_double * 3)(*right),
                            (C.c_double * 3)(*up), float(tan_half_fov), int(W), int(H))


def gbuffer_heightmap(W=1920, H=1080, view_deg=25.0, seed=5, alpha=1.0, density=1e7, rms_slope=0.45,
                      device="cuda", n_march=128, n_bisect=48, stream=None) -> Scene:
    """The heightmap (rms_slope > 0) or plane (rms_slope = 0) view of
    scenes.heightmap, ray-marched by glint_gbuffer_heightfield on the GPU."""
    import math
    from . import scenes
    eye, target, up = scenes.heightmap_camera(view_deg)
    cam = _camera_struct(scenes.camera_basis(eye, target, up), math.tan(math.radians(30.0) / 2), W, H)
    hf = scenes.Heightfield.seeded(seed, rms_slope=rms_slope)
    n = int(hf.kx.numel())
    if n > _lib.MAX_WAVES:
        raise ValueError("too many waves")
    f = _lib.GlintHeightfield()
    f.n_waves, f.n_march, f.n_bisect = n, int(n_march), int(n_bisect)
    for k in range(n):
        f.kx[k], f.kz[k] = float(hf.kx[k]), float(hf.kz[k])
        f.phase[k], f.amp[k] = float(hf.phase[k]), float(hf.amp[k])
    f.uv_scale = 64.0
    dev = torch.device(device)
    gbuf = torch.empty(H, W, 16, dtype=torch.float32, device=dev)
    with torch.cuda.device(dev):
        rc = _lib.lib().glint_gbuffer_heightfield(C.byref(cam), C.byref(f), gbuf.data_ptr(), _stream_handle(stream))
    _lib.check(rc, "glint_gbuffer_heightfield")
    name = "heightmap" if rms_slope > 0 else "plane"
    return Scene(f"{name}{int(round(view_deg))}", gbuf, None, None, scenes.heightmap_material(alpha, density),
                 [Light(kind=1, dir=scenes.HEIGHTMAP_LIGHT_DIR, intensity=1.0)])


def gbuffer_sphere_plane(W=3840, H=2160, azimuth_deg=0.0, seed=3, device="cuda", stream=None) -> Scene:
    """The frame of scenes.sphere_plane, ray-cast by glint_gbuffer_sphere_plane
    on the GPU (the value-noise lattices are drawn on the host from the same
    seeded generator)."""
    from . import scenes
    st = scenes.sphere_plane_setup(W, H, azimuth_deg, seed)
    dev = torch.device(device)
    cam = _camera_struct(st["camera"], st["tan_half_fov"], W, H)
    na = st["noise_alpha"].to(dev).contiguous()
    nr = st["noise_log10_density"].to(dev).contiguous()
    sp = _lib.GlintSpherePlane()
    for k in range(3):
        sp.center[k] = st["center"][k]
    sp.radius, sp.sphere_uv_scale = st["radius"], st["sphere_uv_scale"]
    sp.plane_half_extent, sp.plane_uv_scale, sp.plane_uv_wrap = (st["plane_half_extent"], st["plane_uv_scale"],
                                                                 st["plane_uv_wrap"])
    sp.n_lights, sp.noise_cell = len(st["light_pos"]), st["noise_cell"]
    sp.noise_h, sp.noise_w = int(na.shape[0]), int(na.shape[1])
    for l, (pos, I) in enumerate(zip(st["light_pos"], st["light_I"])):
        for k in range(3):
            sp.light_pos[l][k] = pos[k]
        sp.light_I[l] = I
    sp.noise_alpha, sp.noise_log10_density = na.data_ptr(), nr.data_ptr()
    gbuf = torch.empty(H, W, 16, dtype=torch.float32, device=dev)
    light_px = torch.empty(len(st["light_pos"]), H, W, 4, dtype=torch.float32, device=dev)
    mat_px = torch.empty(H, W, 2, dtype=torch.float32, device=dev)
    with torch.cuda.device(dev):
        rc = _lib.lib().glint_gbuffer_sphere_plane(C.byref(cam), C.byref(sp), gbuf.data_ptr(), light_px.data_ptr(),
                                                   mat_px.data_ptr(), _stream_handle(stream))
    _lib.check(rc, "glint_gbuffer_sphere_plane")
    torch.cuda.current_stream(dev).synchronize() if stream is None else stream.synchronize()
    return Scene("sphere_plane", gbuf, light_px, mat_px, st["material"], st["lights"])

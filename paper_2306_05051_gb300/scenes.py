"""Seeded synthetic G-buffers shaped like the paper's benchmark scenes.

The paper measures glint shading on Unity scenes (Plane 90/25 degrees,
Sphere, Heightmap, Sponza; Sec. 7, Table 1) that are not available here.
This module builds analytic stand-ins: a pinhole camera, ray/plane and
ray/sphere hits, a ray-marched displaced plane, analytic uv maps, and uv
derivatives from first-order ray differentials.  It contains none of the glint method's arithmetic; both the
CUDA library and the CPU oracle read the bytes it produces.

G-buffer layout, per pixel, 16 float32 (4 x float4):
    [u, v, du/dx, dv/dx,  du/dy, dv/dy, nx, ny,  nz, tx, ty, tz,  wvx, wvy, wvz, 0]
n is the surface normal (all zero marks a background pixel), t the tangent
(direction of increasing u), wv the direction towards the viewer.
Point-light plane, [n_lights, H, W, 4]: (direction to the light xyz, E = I/d^2).
Material plane, [H, W, 2]: (isotropic roughness alpha, flakes per unit uv^2).

Geometry is computed in float64 with torch (CPU or CUDA) and stored as
float32, so a scene generated once feeds the oracle and the GPU identically.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import torch

DEFAULT_SEED = 0x9E3779B9


@dataclass
class Material:
    """Glint material parameters (scalar; a per-pixel plane may override
    alpha and density).  Defaults follow the paper where it gives a value
    (R = 0.034, Sec. 7) and the library's recorded readings otherwise."""
    ndf: int = 0                   # 0 Beckmann, 1 GGX
    alpha_x: float = 0.3
    alpha_y: float = 0.3
    ln_density: float = math.log(1e5)   # ln(flakes per unit uv^2)
    R: float = 0.034
    F0: float = 1.0
    gamma: float = 0.05            # angular texel size (projected half-vector units)
    n_lods: int = 8
    n_rings: int = 4
    lod_factor: int = 4
    max_sub: int = 64
    seed: int = DEFAULT_SEED
    lod_blend: int = 0             # 0 distributed binomial (Sec. 4.2); 1 linear mix of LOD outputs (Sec. 3)
    sampler: int = 0               # 0 gated Gaussian (Sec. 6.3); 1 classical Gaussian / Bernoulli loop
    rng_table: int = 0             # 0 hashed uniforms; 1 uniforms fetched from a precomputed table (Sec. 6.3)


@dataclass
class Light:
    kind: int                      # 0 point (reads the per-pixel light plane), 1 directional
    dir: tuple = (0.0, 1.0, 0.0)   # directional only: direction towards the light
    intensity: float = 1.0         # directional only


@dataclass
class Scene:
    name: str
    gbuf: torch.Tensor                         # [H, W, 16] float32
    light_px: Optional[torch.Tensor]           # [nL, H, W, 4] float32 or None
    mat_px: Optional[torch.Tensor]             # [H, W, 2] float32 or None
    material: Material
    lights: List[Light] = field(default_factory=list)

    @property
    def height(self) -> int:
        return int(self.gbuf.shape[0])

    @property
    def width(self) -> int:
        return int(self.gbuf.shape[1])

    def to(self, device) -> "Scene":
        mv = lambda t: None if t is None else t.to(device)
        return replace(self, gbuf=mv(self.gbuf), light_px=mv(self.light_px), mat_px=mv(self.mat_px))


# --------------------------------------------------------------------------
# camera and hits
# --------------------------------------------------------------------------
def _normalize(v: torch.Tensor) -> torch.Tensor:
    return v / torch.linalg.vector_norm(v, dim=-1, keepdim=True).clamp_min(1e-300)


def camera_basis(eye, target, up=(0.0, 1.0, 0.0), device="cpu"):
    """(eye, fwd, right, up) of a pinhole camera looking at target, `up` the
    world direction that appears upwards on screen (float64 tensors)."""
    f64 = torch.float64
    eye = torch.tensor(eye, dtype=f64, device=device)
    fwd = _normalize(torch.tensor(target, dtype=f64, device=device) - eye)
    up0 = torch.tensor(up, dtype=f64, device=device)
    right = _normalize(torch.linalg.cross(fwd, up0))
    up = torch.linalg.cross(right, fwd)
    return eye, fwd, right, up


def camera_rays(W, H, eye, target, fov_deg=60.0, device="cpu", up=(0.0, 1.0, 0.0)):
    """Pinhole camera, vertical field of view fov_deg, `up` the world
    direction that appears upwards on screen.  Returns eye [3],
    unnormalised directions D [H, W, 3] and their screen derivatives
    dD/dx, dD/dy [3] (constant for a pinhole)."""
    f64 = torch.float64
    eye, fwd, right, up = camera_basis(eye, target, up, device)
    th = math.tan(math.radians(fov_deg) / 2)
    aspect = W / H
    xs = (torch.arange(W, dtype=f64, device=device) + 0.5) * (2.0 / W) - 1.0
    ys = 1.0 - (torch.arange(H, dtype=f64, device=device) + 0.5) * (2.0 / H)
    sx = (xs * th * aspect)[None, :, None]
    sy = (ys * th)[:, None, None]
    D = fwd + sx * right + sy * up
    dDdx = (2.0 / W) * th * aspect * right
    dDdy = -(2.0 / H) * th * up
    return eye, D, dDdx, dDdy


def _transfer(t, D, dD, N):
    """First-order ray differential of the hit point (Igehy 1999):
    dP = t (dD - (dD.N)/(D.N) D)."""
    dn = (D * N).sum(-1, keepdim=True)
    return t[..., None] * (dD - (dD * N).sum(-1, keepdim=True) / dn * D)


def _hit_plane(eye, D, height=0.0):
    t = (height - eye[1]) / D[..., 1]
    return t


def _hit_sphere(eye, D, center, radius):
    oc = eye - center
    a = (D * D).sum(-1)
    b = 2.0 * (D * oc).sum(-1)
    c = (oc * oc).sum() - radius * radius
    disc = b * b - 4 * a * c
    sq = torch.sqrt(disc.clamp_min(0.0))
    t = (-b - sq) / (2 * a)
    t = torch.where(disc > 0, t, torch.full_like(t, float("inf")))
    return torch.where(t > 0, t, torch.full_like(t, float("inf")))


def _pack(u, v, dudx, dvdx, dudy, dvdy, n, tg, wv, mask):
    H, W = u.shape
    g = torch.zeros(H, W, 16, dtype=torch.float64, device=u.device)
    g[..., 0], g[..., 1] = u, v
    g[..., 2], g[..., 3], g[..., 4], g[..., 5] = dudx, dvdx, dudy, dvdy
    g[..., 6:9] = n
    g[..., 9:12] = tg
    g[..., 12:15] = wv
    g[~mask] = 0.0
    return g


def _noise_grid(H, W, cell, gen, lo, hi, device):
    """The value-noise lattice: uniform values in [lo, hi) every `cell` pixels."""
    gh, gw = H // cell + 2, W // cell + 2
    return torch.rand(gh, gw, generator=gen, dtype=torch.float64).to(device) * (hi - lo) + lo


def _value_noise(H, W, cell, gen, lo, hi, device):
    """Bilinear value noise: uniform values on a grid every `cell` pixels."""
    grid = _noise_grid(H, W, cell, gen, lo, hi, device)
    ys = (torch.arange(H, dtype=torch.float64, device=device) + 0.5) / cell
    xs = (torch.arange(W, dtype=torch.float64, device=device) + 0.5) / cell
    y0, x0 = ys.floor().long(), xs.floor().long()
    fy, fx = (ys - y0)[:, None], (xs - x0)[None, :]
    g00 = grid[y0][:, x0]; g01 = grid[y0][:, x0 + 1]
    g10 = grid[y0 + 1][:, x0]; g11 = grid[y0 + 1][:, x0 + 1]
    return (1 - fy) * ((1 - fx) * g00 + fx * g01) + fy * ((1 - fx) * g10 + fx * g11)


# --------------------------------------------------------------------------
# plane and sphere shading records
# --------------------------------------------------------------------------
def _plane_record(eye, D, dDdx, dDdy, t, uv_scale, uv_rot, uv_off, wrap):
    P = eye + t[..., None] * D
    N = torch.zeros_like(P); N[..., 1] = 1.0
    dPdx = _transfer(t, D, dDdx.expand_as(D), N)
    dPdy = _transfer(t, D, dDdy.expand_as(D), N)
    c, s = math.cos(uv_rot), math.sin(uv_rot)
    # uv = scale * Rot(uv_rot) (x, z) + off
    def uvmap(X, Z):
        return uv_scale * (c * X - s * Z), uv_scale * (s * X + c * Z)
    u, v = uvmap(P[..., 0], P[..., 2])
    u, v = u + uv_off[0], v + uv_off[1]
    if wrap:
        u, v = torch.remainder(u, wrap), torch.remainder(v, wrap)
    dudx, dvdx = uvmap(dPdx[..., 0], dPdx[..., 2])
    dudy, dvdy = uvmap(dPdy[..., 0], dPdy[..., 2])
    # tangent = dP/du direction = Rot^T e_u in (x, z)
    tg = torch.zeros_like(P); tg[..., 0] = c; tg[..., 2] = -s
    return P, u, v, dudx, dvdx, dudy, dvdy, N, tg


def _sphere_record(eye, D, dDdx, dDdy, t, center, radius, uv_scale):
    P = eye + t[..., None] * D
    Pc = P - center
    N = Pc / radius
    dPdx = _transfer(t, D, dDdx.expand_as(D), N)
    dPdy = _transfer(t, D, dDdy.expand_as(D), N)
    X, Y, Z = Pc[..., 0], Pc[..., 1], Pc[..., 2]
    rxz2 = (X * X + Z * Z).clamp_min(1e-30)
    phi = torch.atan2(Z, X)
    th = torch.acos((Y / radius).clamp(-1.0, 1.0))
    u = uv_scale * (phi / (2 * math.pi) + 0.5)
    v = uv_scale * th / math.pi
    # gradients of (phi, theta) with respect to P
    gphi = torch.stack([-Z / rxz2, torch.zeros_like(X), X / rxz2], -1)
    r = torch.linalg.vector_norm(Pc, dim=-1)
    sin_th = torch.sqrt(rxz2) / r
    ey = torch.zeros_like(Pc); ey[..., 1] = 1.0
    gth = -(ey / r[..., None] - (Y / r ** 3)[..., None] * Pc) / sin_th[..., None].clamp_min(1e-30)
    du = uv_scale / (2 * math.pi) * gphi
    dv = uv_scale / math.pi * gth
    dudx, dudy = (du * dPdx).sum(-1), (du * dPdy).sum(-1)
    dvdx, dvdy = (dv * dPdx).sum(-1), (dv * dPdy).sum(-1)
    tg = _normalize(torch.stack([-Z, torch.zeros_like(X), X], -1))
    return P, u, v, dudx, dvdx, dudy, dvdy, N, tg


def _point_lights(P, mask, lights_pos, intensities):
    planes = []
    for Lp, I in zip(lights_pos, intensities):
        d = torch.tensor(Lp, dtype=torch.float64, device=P.device) - P
        dist2 = (d * d).sum(-1)
        w = d / torch.sqrt(dist2)[..., None]
        pl = torch.cat([w, (I / dist2)[..., None]], -1)
        pl[~mask] = 0.0
        planes.append(pl)
    return torch.stack(planes, 0)


def _f32(x):
    return None if x is None else x.to(torch.float32).contiguous()


# --------------------------------------------------------------------------
# the paper-shaped workloads
# --------------------------------------------------------------------------
def plane45(W=256, H=256, ndf=0, seed=1, device="cpu") -> Scene:
    """256^2 flat plane viewed at 45 degrees, seeded affine uv map scaled so
    the median footprint holds about 2 flakes at density 1e5, one point light
    1 unit above the plane centre, alpha = 0.3 isotropic, 8 LODs."""
    gen = torch.Generator().manual_seed(seed)
    rot = float(torch.rand(1, generator=gen, dtype=torch.float64)) * 2 * math.pi
    off = (torch.rand(2, generator=gen, dtype=torch.float64) * 4.0).tolist()
    eye = (0.0, math.sqrt(2.0), math.sqrt(2.0))
    eye_t, D, dDdx, dDdy = camera_rays(W, H, eye, (0.0, 0.0, 0.0), 60.0, device)
    t = _hit_plane(eye_t, D)
    mask = torch.isfinite(t) & (t > 0)
    t = torch.where(mask, t, torch.ones_like(t))
    scale = 0.46 * (256.0 / max(W, H))
    P, u, v, dudx, dvdx, dudy, dvdy, N, tg = _plane_record(eye_t, D, dDdx, dDdy, t, scale, rot, off, 0)
    wv = _normalize(-D)
    gbuf = _pack(u, v, dudx, dvdx, dudy, dvdy, N, tg, wv, mask)
    light_px = _point_lights(P, mask, [(0.0, 1.0, 0.0)], [1.0])
    mat = Material(ndf=ndf, alpha_x=0.3, alpha_y=0.3, ln_density=math.log(1e5), n_lods=8)
    return Scene("plane45", _f32(gbuf), _f32(light_px), None, mat, [Light(kind=0)])


def grazing_plane(W=1920, H=1080, device="cpu") -> Scene:
    """1920x1080 infinite plane y = 0 seen from height 1 at pitch -20 degrees;
    rows whose footprint anisotropy would exceed 32:1 are background.  uv is
    64 x world (x, z) wrapped to [0, 64).  alpha = (0.2, 0.05), density 1e7,
    12 LODs, one directional light at 30 degrees elevation."""
    pitch = math.radians(-20.0)
    eye = (0.0, 1.0, 0.0)
    target = (0.0, 1.0 + math.sin(pitch), -math.cos(pitch))
    eye_t, D, dDdx, dDdy = camera_rays(W, H, eye, target, 60.0, device)
    Dn = _normalize(D)
    # grazing angle below the horizon; anisotropy of a square pixel ~ 1/sin(angle)
    mask = (-Dn[..., 1]) > (1.0 / 32.0)
    t = _hit_plane(eye_t, D)
    t = torch.where(mask, t, torch.ones_like(t))
    P, u, v, dudx, dvdx, dudy, dvdy, N, tg = _plane_record(eye_t, D, dDdx, dDdy, t, 64.0, 0.0, (0.0, 0.0), 64.0)
    wv = _normalize(-D)
    gbuf = _pack(u, v, dudx, dvdx, dudy, dvdy, N, tg, wv, mask)
    el = math.radians(30.0)
    ldir = (0.0, math.sin(el), -math.cos(el))
    mat = Material(ndf=0, alpha_x=0.2, alpha_y=0.05, ln_density=math.log(1e7), n_lods=12)
    return Scene("grazing_plane", _f32(gbuf), None, None, mat, [Light(kind=1, dir=ldir, intensity=1.0)])


SPHERE_PLANE = {"target": (0.0, 0.55, 0.0), "light_pos": [(2.5, 3.5, 2.0), (-3.0, 2.5, -1.5)],
                "light_I": [12.0, 8.0]}


def sphere_plane_setup(W=3840, H=2160, azimuth_deg=0.0, seed=3):
    """Everything that defines the sphere_plane frame, for a generator that
    rebuilds it elsewhere: camera (eye, fwd, right, up, tan of half the
    vertical field of view), geometry and lights, and the two value-noise
    lattices (alpha, log10 density) drawn from the seeded generator in the
    same order as sphere_plane."""
    az = math.radians(azimuth_deg)
    R = 4.2
    eye = (R * math.sin(az), 1.6, R * math.cos(az))
    cam = camera_basis(eye, SPHERE_PLANE["target"])
    gen = torch.Generator().manual_seed(seed)
    alpha = _noise_grid(H, W, 64, gen, 0.05, 0.5, "cpu")
    log10rho = _noise_grid(H, W, 64, gen, 3.0, 9.0, "cpu")
    return dict(W=W, H=H, camera=cam, tan_half_fov=math.tan(math.radians(60.0) / 2), center=(0.0, 1.0, 0.0),
                radius=1.0, sphere_uv_scale=8.0, plane_half_extent=10.0, plane_uv_scale=4.0, plane_uv_wrap=8.0,
                light_pos=SPHERE_PLANE["light_pos"], light_I=SPHERE_PLANE["light_I"], noise_cell=64,
                noise_alpha=alpha, noise_log10_density=log10rho,
                material=Material(ndf=0, alpha_x=0.3, alpha_y=0.3, ln_density=math.log(1e6), n_lods=12),
                lights=[Light(kind=0), Light(kind=0)])


def sphere_plane(W=3840, H=2160, azimuth_deg=0.0, seed=3, device="cpu") -> Scene:
    """Unit sphere resting on a 20 x 20 ground plane.  Sphere uv is
    equirectangular x 8, plane uv is 4 x world wrapped to [0, 8).  Per-pixel
    alpha ~ U[0.05, 0.5] and log10 density ~ U[3, 9] from seeded value noise
    with 64-pixel cells; 12 LODs; two point lights."""
    az = math.radians(azimuth_deg)
    R = 4.2
    eye = (R * math.sin(az), 1.6, R * math.cos(az))
    eye_t, D, dDdx, dDdy = camera_rays(W, H, eye, SPHERE_PLANE["target"], 60.0, device)
    center = torch.tensor([0.0, 1.0, 0.0], dtype=torch.float64, device=device)
    ts = _hit_sphere(eye_t, D, center, 1.0)
    tp = _hit_plane(eye_t, D)
    Pp = eye_t + tp[..., None] * D
    plane_ok = (tp > 0) & (Pp[..., 0].abs() <= 10.0) & (Pp[..., 2].abs() <= 10.0)
    tp = torch.where(plane_ok, tp, torch.full_like(tp, float("inf")))
    use_sphere = ts < tp
    mask = torch.isfinite(torch.minimum(ts, tp))
    ts1 = torch.where(use_sphere & mask, ts, torch.ones_like(ts))
    tp1 = torch.where(~use_sphere & mask, tp, torch.ones_like(tp))
    sph = _sphere_record(eye_t, D, dDdx, dDdy, ts1, center, 1.0, 8.0)
    pla = _plane_record(eye_t, D, dDdx, dDdy, tp1, 4.0, 0.0, (0.0, 0.0), 8.0)
    sel = use_sphere
    pick = lambda a, b: torch.where(sel[..., None] if a.dim() == 3 else sel, a, b)
    P, u, v, dudx, dvdx, dudy, dvdy, N, tg = [pick(a, b) for a, b in zip(sph, pla)]
    wv = _normalize(-D)
    gbuf = _pack(u, v, dudx, dvdx, dudy, dvdy, N, tg, wv, mask)
    light_px = _point_lights(P, mask, SPHERE_PLANE["light_pos"], SPHERE_PLANE["light_I"])
    gen = torch.Generator().manual_seed(seed)
    alpha = _value_noise(H, W, 64, gen, 0.05, 0.5, device)
    log10rho = _value_noise(H, W, 64, gen, 3.0, 9.0, device)
    mat_px = torch.stack([alpha, torch.pow(10.0, log10rho)], -1)
    mat_px[~mask] = 0.0
    mat = Material(ndf=0, alpha_x=0.3, alpha_y=0.3, ln_density=math.log(1e6), n_lods=12)
    return Scene("sphere_plane", _f32(gbuf), _f32(light_px), _f32(mat_px), mat,
                 [Light(kind=0), Light(kind=0)])


# --------------------------------------------------------------------------
# displaced plane (heightmap)
# --------------------------------------------------------------------------
@dataclass
class Heightfield:
    """h(x, z) = sum_k a_k sin(kx_k x + kz_k z + phi_k): seeded waves with
    log-uniform wavelengths and uniform directions and phases, amplitudes
    set so every wave has the same slope amplitude a_k |k_k| and the
    root-mean-square slope of the sum is `rms_slope`."""
    kx: torch.Tensor
    kz: torch.Tensor
    phase: torch.Tensor
    amp: torch.Tensor

    @staticmethod
    def seeded(seed, n_waves=16, wavelengths=(0.01, 0.08), rms_slope=0.45):
        gen = torch.Generator().manual_seed(seed)
        rnd = lambda: torch.rand(n_waves, generator=gen, dtype=torch.float64)
        lam = wavelengths[0] * (wavelengths[1] / wavelengths[0]) ** rnd()
        ang, phase = rnd() * 2 * math.pi, rnd() * 2 * math.pi
        k = 2 * math.pi / lam
        # the slope of one wave has mean square (a |k|)^2 / 2
        amp = rms_slope * math.sqrt(2.0 / n_waves) / k
        return Heightfield(k * torch.cos(ang), k * torch.sin(ang), phase, amp)

    @property
    def bound(self) -> float:
        return float(self.amp.sum())

    def to(self, device) -> "Heightfield":
        return Heightfield(*(t.to(device) for t in (self.kx, self.kz, self.phase, self.amp)))

    def height(self, x, z):
        arg = x[..., None] * self.kx + z[..., None] * self.kz + self.phase
        return (self.amp * torch.sin(arg)).sum(-1)

    def gradient(self, x, z):
        c = self.amp * torch.cos(x[..., None] * self.kx + z[..., None] * self.kz + self.phase)
        return (c * self.kx).sum(-1), (c * self.kz).sum(-1)


def _hit_heightfield(eye, D, hf, n_march=128, n_bisect=48, chunk=1 << 18):
    """First crossing of the ray eye + t D (D_y < 0) with y = h(x, z):
    march n_march even steps across the slab |y| <= bound, then bisect the
    first bracket where y - h changes sign from + to -.  Such a crossing
    is front-facing (D . (-h_x, 1, -h_z) <= 0).  Crests thinner than one
    march step may be stepped through."""
    A = hf.bound
    Df = D.reshape(-1, 3)
    t = torch.empty(Df.shape[0], dtype=D.dtype, device=D.device)
    for s in range(0, Df.shape[0], chunk):
        d = Df[s:s + chunk]
        f = lambda tt: eye[1] + tt * d[:, 1] - hf.height(eye[0] + tt * d[:, 0], eye[2] + tt * d[:, 2])
        t_in, t_out = (A - eye[1]) / d[:, 1], (-A - eye[1]) / d[:, 1]
        step = (t_out - t_in) / n_march
        lo, hi = t_in.clone(), t_out.clone()
        found = torch.zeros_like(t_in, dtype=torch.bool)
        for j in range(1, n_march + 1):
            tj = t_in + j * step
            hit = (~found) & (f(tj) <= 0)
            lo = torch.where(hit, tj - step, lo)
            hi = torch.where(hit, tj, hi)
            found |= hit
        for _ in range(n_bisect):
            mid = 0.5 * (lo + hi)
            above = f(mid) > 0
            lo, hi = torch.where(above, mid, lo), torch.where(above, hi, mid)
        t[s:s + chunk] = hi
    return t.reshape(D.shape[:-1])


def heightmap_camera(view_deg):
    """(eye, target, up) of the heightmap views: height 1, the central ray
    meeting the base plane at view_deg."""
    v = math.radians(view_deg)
    return (0.0, 1.0, 0.0), (0.0, 1.0 - math.sin(v), -math.cos(v)), (0.0, 0.0, -1.0)


def heightmap_material(alpha=1.0, density=1e7):
    return Material(ndf=0, alpha_x=alpha, alpha_y=alpha, ln_density=math.log(density), n_lods=16)


HEIGHTMAP_LIGHT_DIR = (0.0, math.sin(math.radians(30.0)), -math.cos(math.radians(30.0)))


def heightmap(W=1920, H=1080, view_deg=25.0, seed=5, alpha=1.0, density=1e7, rms_slope=0.45,
              device="cpu") -> Scene:
    """Plane y = 0 displaced by a high-frequency seeded heightfield (16
    waves, wavelengths 0.01-0.08, RMS slope 0.45), ray-marched from a
    camera at height 1 whose central ray meets the base plane at view_deg
    (90 looks straight down), vertical field of view 30 degrees so the
    surface fills the frame.  Normals and tangents are the heightfield's;
    uv = 64 x world (x, z) wrapped to [0, 64), with derivatives from ray
    differentials transferred onto the local tangent plane, so facets seen
    edge-on scatter pixels of large anisotropy across the frame.  Beckmann
    alpha = 1 isotropic (the paper's timing material, Sec. 7.1), density
    1e7, 16 LODs (footprints up to 4^15 flakes before a k x k split, so a
    density sweep to 1e10 stays on the pyramid), one directional light at
    30 degrees elevation.  rms_slope = 0 gives the flat plane of the same
    views (the Plane 90 / 25 degree scenes of Table 1)."""
    eye, target, up = heightmap_camera(view_deg)
    eye_t, D, dDdx, dDdy = camera_rays(W, H, eye, target, 30.0, device, up=up)
    if not bool((D[..., 1] < 0).all()):
        raise ValueError("heightmap: every ray must point below the horizon (view_deg > 15)")
    hf = Heightfield.seeded(seed, rms_slope=rms_slope).to(device)
    t = _hit_heightfield(eye_t, D, hf)
    P = eye_t + t[..., None] * D
    hx, hz = hf.gradient(P[..., 0], P[..., 2])
    one = torch.ones_like(hx)
    N = _normalize(torch.stack([-hx, one, -hz], -1))
    dPdx = _transfer(t, D, dDdx.expand_as(D), N)
    dPdy = _transfer(t, D, dDdy.expand_as(D), N)
    s = 64.0
    u, v_ = torch.remainder(s * P[..., 0], s), torch.remainder(s * P[..., 2], s)
    dudx, dvdx = s * dPdx[..., 0], s * dPdx[..., 2]
    dudy, dvdy = s * dPdy[..., 0], s * dPdy[..., 2]
    tg = _normalize(torch.stack([one, hx, torch.zeros_like(hx)], -1))     # dP/du
    wv = _normalize(-D)
    mask = torch.ones_like(t, dtype=torch.bool)
    gbuf = _pack(u, v_, dudx, dvdx, dudy, dvdy, N, tg, wv, mask)
    mat = heightmap_material(alpha, density)
    name = "heightmap" if rms_slope > 0 else "plane"
    return Scene(f"{name}{int(round(view_deg))}", _f32(gbuf), None, None, mat,
                 [Light(kind=1, dir=HEIGHTMAP_LIGHT_DIR, intensity=1.0)])


ORBIT_RESOLUTIONS = [(256, 256), (512, 512), (1280, 720), (1920, 1080)]


def orbit_frames(n_frames=64, device="cpu", resolutions=None) -> List[Scene]:
    """Camera orbit around the sphere scene: frame i at azimuth 360 i / n
    degrees and value-noise seed 4 + i; resolutions cycle through
    256^2, 512^2, 1280x720, 1920x1080."""
    res = resolutions or ORBIT_RESOLUTIONS
    out = []
    for i in range(n_frames):
        W, H = res[i % len(res)]
        sc = sphere_plane(W, H, azimuth_deg=360.0 * i / n_frames, seed=4 + i, device=device)
        sc.name = f"orbit{i:02d}_{W}x{H}"
        out.append(sc)
    return out


def plane_sphere_fit(W=512, H=512, target=False, device="cpu") -> Scene:
    """512^2 plane + sphere with a directional light, Beckmann, scalar
    material: alpha = (0.2, 0.1), density 1e6, light normalize(0.3, 1, 0.2).
    target=True gives the perturbed parameters the image loss is measured
    against: alpha = (0.25, 0.15), ln density + 0.3, light rotated by 3
    degrees about the vertical axis."""
    eye = (0.0, 1.8, 3.6)
    eye_t, D, dDdx, dDdy = camera_rays(W, H, eye, (0.0, 0.6, 0.0), 60.0, device)
    center = torch.tensor([0.0, 1.0, 0.0], dtype=torch.float64, device=device)
    ts = _hit_sphere(eye_t, D, center, 1.0)
    tp = _hit_plane(eye_t, D)
    Pp = eye_t + tp[..., None] * D
    plane_ok = (tp > 0) & (Pp[..., 0].abs() <= 8.0) & (Pp[..., 2].abs() <= 8.0)
    tp = torch.where(plane_ok, tp, torch.full_like(tp, float("inf")))
    use_sphere = ts < tp
    mask = torch.isfinite(torch.minimum(ts, tp))
    ts1 = torch.where(use_sphere & mask, ts, torch.ones_like(ts))
    tp1 = torch.where(~use_sphere & mask, tp, torch.ones_like(tp))
    sph = _sphere_record(eye_t, D, dDdx, dDdy, ts1, center, 1.0, 8.0)
    pla = _plane_record(eye_t, D, dDdx, dDdy, tp1, 4.0, 0.0, (0.0, 0.0), 8.0)
    pick = lambda a, b: torch.where(use_sphere[..., None] if a.dim() == 3 else use_sphere, a, b)
    P, u, v, dudx, dvdx, dudy, dvdy, N, tg = [pick(a, b) for a, b in zip(sph, pla)]
    wv = _normalize(-D)
    gbuf = _pack(u, v, dudx, dvdx, dudy, dvdy, N, tg, wv, mask)
    l = torch.tensor([0.3, 1.0, 0.2], dtype=torch.float64)
    l = l / torch.linalg.vector_norm(l)
    if target:
        a = math.radians(3.0)
        c, s = math.cos(a), math.sin(a)
        l = torch.tensor([c * l[0] + s * l[2], l[1], -s * l[0] + c * l[2]], dtype=torch.float64)
        mat = Material(ndf=0, alpha_x=0.25, alpha_y=0.15, ln_density=math.log(1e6) + 0.3, n_lods=12)
    else:
        mat = Material(ndf=0, alpha_x=0.2, alpha_y=0.1, ln_density=math.log(1e6), n_lods=12)
    ldir = tuple(float(x) for x in l)
    return Scene("plane_sphere_fit", _f32(gbuf), None, None, mat, [Light(kind=1, dir=ldir, intensity=1.0)])


def by_name(name: str, **kw) -> Scene:
    return {"plane45": plane45, "grazing_plane": grazing_plane, "sphere_plane": sphere_plane,
            "plane_sphere_fit": plane_sphere_fit, "heightmap": heightmap}[name](**kw)


def random_gbuffer(W=131, H=77, seed=0, n_point=1, n_dir=1, material_plane=True, device="cpu") -> Scene:
    """Randomised G-buffer for edge-case coverage (not a paper workload):
    footprint areas log-uniform in [1e-13, 1e-2] uv^2, anisotropy up to 1e4
    at random orientation, uv in [-100, 100], random normals, tangents, view
    and light directions (some below the horizon), 4% background pixels,
    1% zero-area footprints, per-pixel alpha in [0.03, 0.7] and density
    10^[2, 10] when material_plane is set."""
    gen = torch.Generator().manual_seed(seed)
    f64 = torch.float64
    rnd = lambda *s: torch.rand(*s, generator=gen, dtype=f64)
    nrm = lambda *s: torch.randn(*s, generator=gen, dtype=f64)
    area = 10.0 ** (rnd(H, W) * 11.0 - 13.0)
    ratio = 10.0 ** (rnd(H, W) * 4.0)
    ang = rnd(H, W) * math.pi
    a, b = torch.sqrt(area * ratio), torch.sqrt(area / ratio)
    c, s = torch.cos(ang), torch.sin(ang)
    rot2 = rnd(H, W) * 2 * math.pi
    c2, s2 = torch.cos(rot2), torch.sin(rot2)
    # J = Rot(ang) diag(a, b) Rot(rot2)
    J00 = c * a * c2 - s * b * s2; J01 = -c * a * s2 - s * b * c2
    J10 = s * a * c2 + c * b * s2; J11 = -s * a * s2 + c * b * c2
    zero = rnd(H, W) < 0.01
    J00, J01, J10, J11 = [torch.where(zero, torch.zeros_like(x), x) for x in (J00, J01, J10, J11)]
    n = _normalize(nrm(H, W, 3))
    tg = _normalize(nrm(H, W, 3))
    wv = _normalize(n + 1.2 * nrm(H, W, 3) * 0.5)
    g = torch.zeros(H, W, 16, dtype=f64)
    g[..., 0:2] = rnd(H, W, 2) * 200.0 - 100.0
    g[..., 2], g[..., 3], g[..., 4], g[..., 5] = J00, J10, J01, J11
    g[..., 6:9] = n
    g[..., 9:12] = tg
    g[..., 12:15] = wv
    bg = rnd(H, W) < 0.04
    g[bg] = 0.0
    lp = []
    for _ in range(n_point):
        wl = _normalize(n + nrm(H, W, 3) * 0.6)
        E = 10.0 ** (rnd(H, W) * 2 - 1)
        pl = torch.cat([wl, E[..., None]], -1)
        pl[bg] = 0.0
        lp.append(pl)
    lights = [Light(kind=0) for _ in range(n_point)]
    for k in range(n_dir):
        d = nrm(3)
        d[1] = d[1].abs() + 0.3
        lights.append(Light(kind=1, dir=tuple(float(x) for x in d), intensity=1.5))
    mat_px = None
    if material_plane:
        alpha = rnd(H, W) * 0.67 + 0.03
        dens = 10.0 ** (rnd(H, W) * 8.0 + 2.0)
        mat_px = torch.stack([alpha, dens], -1)
        mat_px[bg] = 0.0
    light_px = torch.stack(lp, 0) if lp else None
    mat = Material(ndf=int(seed) % 2, alpha_x=0.25, alpha_y=0.15, ln_density=math.log(1e6), n_lods=12)
    sc = Scene(f"random{seed}", _f32(g), _f32(light_px), _f32(mat_px), mat, lights)
    return sc.to(device)

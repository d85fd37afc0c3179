"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
seeded workloads, at sizes the oracle finishes in seconds and, for the
1080p and 4K frames, on sampled pixels of the full-size launch."""
import math

import numpy as np
import pytest
import torch

import parity
from paper_2306_05051_gb300 import glint, scenes

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _render(scene_dev):
    img = glint.render_scene(scene_dev)
    torch.cuda.synchronize()
    return img.cpu().numpy().astype(np.float64)


def _summary(name, s):
    print(f"[{name}] traced pixels {s['n_traced']}, records {s['n_rec']}, excused mismatches {s['n_excused']}, "
          f"pixels over tol {s['over']}, max rel err (matched) {s['max_err_matched']:.3g}")


@pytest.mark.parametrize("ndf", [0, 1])
def test_plane45_full_image(orc, ndf):
    sc = scenes.plane45(ndf=ndf)
    img = _render(sc.to(DEV))
    ref = orc.eval_image(sc)
    assert np.count_nonzero(ref) > 1000
    s = parity.check_image(orc, sc, sc.to(DEV), img, ref, sample_trace=600)
    _summary(f"plane45 ndf={ndf}", s)


@pytest.mark.parametrize("which", ["plane45", "plane45_ggx", "grazing_plane"])
def test_fresnel_f0(orc, which):
    """Schlick F with F0 = 0.04 (a dielectric), so that the Fresnel term is
    not identically 1: the 45 degree plane (view and light near the normal,
    F just above F0) and the grazing plane (F up to several times F0)."""
    import dataclasses
    base = {"plane45": lambda: scenes.plane45(ndf=0), "plane45_ggx": lambda: scenes.plane45(ndf=1),
            "grazing_plane": lambda: scenes.grazing_plane(480, 270)}[which]()
    sc = dataclasses.replace(base, material=dataclasses.replace(base.material, F0=0.04))
    img = _render(sc.to(DEV))
    ref = orc.eval_image(sc)
    one = orc.eval_image(base)
    lit = one != 0
    ratio = ref[lit] / one[lit]
    f0 = float(np.float32(0.04))
    assert ratio.min() >= f0 - 1e-12 and ratio.max() < 1.0 and ratio.max() > f0 * (1 + 1e-4)
    if which == "grazing_plane":
        assert ratio.max() > 2 * f0
    s = parity.check_image(orc, sc, sc.to(DEV), img, ref, sample_trace=600)
    _summary(f"{which} F0=0.04", s)


@pytest.mark.parametrize("gamma", [0.01, 0.2])
@pytest.mark.parametrize("which", ["plane45", "sphere_plane"])
def test_angular_texel_size(orc, which, gamma):
    """The angular grid at a finer (0.01) and a coarser (0.2) texel than the
    default 0.05: the angular coordinate h / gamma and its floor."""
    import dataclasses
    sc = scenes.plane45() if which == "plane45" else scenes.sphere_plane(480, 270)
    sc = dataclasses.replace(sc, material=dataclasses.replace(sc.material, gamma=gamma))
    img = _render(sc.to(DEV))
    ref = orc.eval_image(sc)
    s = parity.check_image(orc, sc, sc.to(DEV), img, ref, sample_trace=400)
    _summary(f"{which} gamma={gamma}", s)


def test_plane_sphere_fit_full_image(orc):
    sc = scenes.plane_sphere_fit()
    img = _render(sc.to(DEV))
    ref = orc.eval_image(sc)
    s = parity.check_image(orc, sc, sc.to(DEV), img, ref, sample_trace=600)
    _summary("plane_sphere_fit 512", s)


def test_grazing_plane_1080p_sampled(orc):
    scd = scenes.grazing_plane(device=DEV)
    sc = scd.to("cpu")
    img = _render(scd)
    rng = np.random.default_rng(2)
    H, W = sc.height, sc.width
    fg = np.flatnonzero(sc.gbuf[..., 6:9].abs().sum(-1).reshape(-1).numpy() > 0)
    top = fg[fg < (H // 3) * W]                            # far rows: K > 1, largest footprints
    px = np.unique(np.concatenate([rng.choice(fg, 12000, replace=False), rng.choice(top, 4000, replace=False)]))
    ref = orc.eval_image(sc, px=px.astype(np.int32))
    s = parity.check_image(orc, sc, scd, img, ref, px=px, sample_trace=300)
    _summary("grazing_plane 1080p", s)
    assert max(int(p["K"]) for p in s["opix"]) > 1


def test_sphere_plane_4k_sampled(orc):
    scd = scenes.sphere_plane(device=DEV)
    sc = scd.to("cpu")
    img = _render(scd)
    rng = np.random.default_rng(3)
    fg = np.flatnonzero(sc.gbuf[..., 6:9].abs().sum(-1).reshape(-1).numpy() > 0)
    px = np.sort(rng.choice(fg, 16000, replace=False))
    ref = orc.eval_image(sc, px=px.astype(np.int32))
    s = parity.check_image(orc, sc, scd, img, ref, px=px, sample_trace=300)
    _summary("sphere_plane 4K", s)


def test_sphere_plane_small_full_image(orc):
    """The 4K scene's geometry at 480 x 270 (larger footprints): every pixel."""
    sc = scenes.sphere_plane(480, 270)
    img = _render(sc.to(DEV))
    ref = orc.eval_image(sc)
    s = parity.check_image(orc, sc, sc.to(DEV), img, ref, sample_trace=400)
    _summary("sphere_plane 480x270", s)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_gbuffer_edge_cases(orc, seed):
    """Ragged 131 x 77 frame: background, zero-area footprints, anisotropy to
    1e4 (capped sub-footprints), fractional footprints, areas above the top
    level, negative uv, lights below the horizon, per-pixel material."""
    sc = scenes.random_gbuffer(seed=seed)
    img = _render(sc.to(DEV))
    ref = orc.eval_image(sc)
    s = parity.check_image(orc, sc, sc.to(DEV), img, ref, sample_trace=500)
    _summary(f"random seed {seed}", s)
    stat = np.array([orc.trace_pixel(sc, int(p), cap=1)[0]["status"] for p in range(0, img.size, 3)])
    assert (stat == 1).any() and (stat == 2).any() and (stat == 0).any()
    assert (img[ref == 0] == 0).all()


def test_trace_counts_48_evaluations_per_pixel_and_light(orc):
    sc = scenes.sphere_plane(160, 90)
    scd = sc.to(DEV)
    fg = np.flatnonzero(sc.gbuf[..., 6:9].abs().sum(-1).reshape(-1).numpy() > 0)[:64].astype(np.int32)
    pix, recs = glint.trace(scd, fg, cap=2 * 48 * 8)
    for k, p in enumerate(fg):
        op, orecs = orc.trace_pixel(sc, int(p))
        n_on = len(set(orecs["light"]))
        assert pix[k]["K"] == op["K"]
        written = recs[k][recs[k]["light"] >= 0]
        assert len(written) == 48 * int(op["K"]) * n_on == len(orecs)


def test_no_lights_background_only_and_one_pixel(orc):
    sc = scenes.plane45(32, 16)
    scd = sc.to(DEV)
    img = glint.render_scene(scd, lights=[]).cpu().numpy()
    assert (img == 0).all()
    bg = scenes.Scene("bg", torch.zeros(5, 7, 16), None, None, scenes.Material(), [scenes.Light(kind=1)])
    assert (glint.render_scene(bg.to(DEV)).cpu().numpy() == 0).all()
    one = scenes.Scene("one", sc.gbuf[8:9, 16:17].contiguous(), sc.light_px[:, 8:9, 16:17].contiguous(), None,
                       sc.material, sc.lights)
    v = glint.render_scene(one.to(DEV)).cpu().numpy()
    assert v.shape == (1, 1)
    assert v[0, 0] == pytest.approx(orc.eval_image(one)[0, 0], rel=1e-4, abs=1e-30)


def test_maximum_parameters(orc):
    """Largest supported rings, LODs, lights and sub-footprints."""
    sc = scenes.random_gbuffer(97, 41, seed=7, n_point=4, n_dir=4)
    sc.material = scenes.Material(ndf=1, alpha_x=0.4, alpha_y=0.2, ln_density=math.log(1e6), n_lods=16,
                                  n_rings=6, lod_factor=2, max_sub=64)
    img = _render(sc.to(DEV))
    ref = orc.eval_image(sc)
    s = parity.check_image(orc, sc, sc.to(DEV), img, ref, sample_trace=200)
    _summary("max params", s)


def test_host_buffer_path_matches_device_path(orc):
    sc = scenes.sphere_plane(320, 180)
    scd = sc.to(DEV)
    dev_img = glint.render_scene(scd).cpu()
    host = scenes.Scene(sc.name, sc.gbuf.pin_memory(), sc.light_px.pin_memory(), sc.mat_px.pin_memory(),
                        sc.material, sc.lights)
    staging = torch.empty(glint.staging_bytes(host), dtype=torch.uint8, device=DEV)
    out = torch.empty(sc.height, sc.width, dtype=torch.float32).pin_memory()
    glint.render_host(host, staging, out)
    torch.cuda.synchronize()
    assert torch.equal(out, dev_img)


@pytest.mark.parametrize("which", ["sphere_plane_tall", "grazing_plane"])
def test_host_buffer_path_in_bands_matches_device_path(which):
    """Frames of several bands (the last one short), with and without the
    light and material planes: the banded, overlapped host path gives the
    device path's bits, and the stream it was given is ordered after it."""
    if which == "sphere_plane_tall":
        sc = scenes.sphere_plane(1280, 2000, seed=11)          # 5 bands: 4 x 410 rows and 360
    else:
        sc = scenes.grazing_plane()                           # 1920 x 1080, directional light, 4 bands
    scd = sc.to(DEV)
    dev_img = glint.render_scene(scd).cpu()
    pin = lambda t: None if t is None else t.pin_memory()
    host = scenes.Scene(sc.name, pin(sc.gbuf), pin(sc.light_px), pin(sc.mat_px), sc.material, sc.lights)
    staging = torch.empty(glint.staging_bytes(host), dtype=torch.uint8, device=DEV)
    out = torch.full((sc.height, sc.width), -1.0, dtype=torch.float32).pin_memory()
    s = torch.cuda.Stream()
    glint.render_host(host, staging, out, stream=s)
    flag = torch.zeros(1, device=DEV)
    with torch.cuda.stream(s):
        flag += 1.0                                            # queued after the call on the same stream
    s.synchronize()
    assert torch.equal(out, dev_img)
    assert flag.item() == 1.0


def test_side_stream_and_repeatability(orc):
    sc = scenes.plane45(128, 96)
    scd = sc.to(DEV)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = glint.render_scene(scd, stream=s)
    s.synchronize()
    b = glint.render_scene(scd)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_invalid_device_arguments():
    from paper_2306_05051_gb300 import _lib
    sc = scenes.plane45(16, 16)
    with pytest.raises(_lib.GlintError) as e:      # host tensor where device memory is required
        fr = _lib.frame_struct(sc.gbuf, sc.light_px, None, 1)
        out = torch.empty(16, 16, device=DEV)
        import ctypes as C
        rc = _lib.lib().glint_eval(C.byref(fr), C.byref(_lib.material_struct(sc.material)),
                                   _lib.lights_struct(sc.lights), out.data_ptr(), 0)
        _lib.check(rc, "glint_eval")
    assert e.value.code == -3
    g = torch.zeros(16 * 16 * 16 + 1, device=DEV)[1:].view(16, 16, 16)   # 4-byte aligned, not 16
    with pytest.raises(_lib.GlintError) as e:
        glint.render(g, sc.light_px.to(DEV), None, sc.material, sc.lights)
    assert e.value.code == -2


def test_every_launch_shape_gives_the_same_bits():
    """glint_eval_launch: one CTA per tile (ctas_per_sm = 0) and persistent
    grids of every CTA size give glint_eval's image bit for bit; bad shapes
    are rejected."""
    from paper_2306_05051_gb300 import _lib
    sc = scenes.sphere_plane(640, 360, seed=5)
    scd = sc.to(DEV)
    ref = glint.render_scene(scd)
    for shape in [(512, 0), (128, 0), (1024, 0), (128, 1), (256, 4), (256, 8), (512, 2), (1024, 1), (1024, 2),
                  (512, 16)]:
        img = glint.render_scene(scd, launch=shape)
        torch.cuda.synchronize()
        assert torch.equal(img, ref), shape
    for bad in [(512, -1), (512, 17), (100, 2), (2048, 1)]:
        with pytest.raises(_lib.GlintError) as e:
            glint.render_scene(scd, launch=bad)
        assert e.value.code == -1, bad


def test_launch_shapes_across_row_and_block_tiles():
    """A frame large enough that some launch shapes tile it in 16-pixel-wide
    blocks (at least 2048 row tiles) and others in runs of a row: every
    shape, one CTA per tile or persistent, gives the same bits, and every
    pixel is written."""
    sc = scenes.sphere_plane(1600, 900, seed=6)               # 1.44 M px: 2-D at 128-512 threads, rows at 1024
    scd = sc.to(DEV)
    ref = glint.render_scene(scd)
    for shape in [(128, 0), (256, 0), (1024, 0), (512, 2), (256, 4), (128, 8), (1024, 1)]:
        img = torch.full_like(ref, float("nan"))
        glint.render_scene(scd, out=img, launch=shape)
        torch.cuda.synchronize()
        assert torch.equal(img, ref), shape


def _iso(sc):
    import dataclasses
    return dataclasses.replace(sc, material=dataclasses.replace(sc.material, n_rings=0))


@pytest.mark.parametrize("which", ["grazing_plane", "plane45", "random"])
def test_isotropic_grid_mode(orc, which):
    """n_rings = 0 (Sec. 4 with the footprint cut into ceil(r) pieces on the
    isotropic grid): parity with the oracle, 24 evaluations per piece and
    light, and K growing with the anisotropy."""
    if which == "grazing_plane":
        sc = _iso(scenes.grazing_plane())
    elif which == "plane45":
        sc = _iso(scenes.plane45())
    else:
        sc = _iso(scenes.random_gbuffer(seed=4))
    scd = sc.to(DEV)
    img = _render(scd)
    if which == "grazing_plane":
        rng = np.random.default_rng(8)
        fg = np.flatnonzero(sc.gbuf[..., 6:9].abs().sum(-1).reshape(-1).numpy() > 0)
        px = np.unique(rng.choice(fg, 12000, replace=False)).astype(np.int32)
        ref = orc.eval_image(sc, px=px)
        s = parity.check_image(orc, sc, scd, img, ref, px=px, sample_trace=300)
    else:
        ref = orc.eval_image(sc)
        s = parity.check_image(orc, sc, scd, img, ref, sample_trace=300)
        px = np.arange(img.size, dtype=np.int32)
    _summary(f"isotropic grids {which}", s)
    pix, _ = glint.trace(scd, px[:4000], cap=0)
    ok = pix["status"] == 0
    nl_on = pix["n_rec"][ok] // np.maximum(24 * pix["K"][ok], 1)
    assert (pix["n_rec"][ok] == 24 * pix["K"][ok] * nl_on).all()
    if which == "grazing_plane":
        assert pix["K"][ok].max() >= 8                     # far rows: anisotropy cut into many pieces


def _anisotropy(sc):
    """Footprint anisotropy per pixel: ratio of the singular values of the
    uv Jacobian (inf for a degenerate footprint)."""
    g = sc.gbuf.double().numpy().reshape(-1, 16)
    J = np.stack([np.stack([g[:, 2], g[:, 4]], -1), np.stack([g[:, 3], g[:, 5]], -1)], -2)
    sv = np.linalg.svd(J, compute_uv=False)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(sv[:, 1] > 0, sv[:, 0] / sv[:, 1], np.inf)


@pytest.mark.parametrize("view,rings,slope", [(25.0, 4, 0.45), (90.0, 4, 0.45), (25.0, 0, 0.45), (25.0, 6, 0.45),
                                              (90.0, 4, 0.0), (25.0, 4, 0.0)])
def test_heightmap_1080p_sampled(orc, view, rings, slope):
    """Displaced plane at 1920 x 1080 (the Heightmap 25 / 90 degree views of
    Sec. 7.1, Beckmann alpha = 1): random pixels plus the scattered pixels of
    anisotropy above 16, with anisotropic grids (4 and 6 rings) and with
    isotropic grids.  slope = 0: the flat Plane views of the same table; seen
    from above every footprint is exactly isotropic (ratio 1, orientation
    set by rounding-level off-diagonal terms), the degenerate case of the
    ratio / orientation cell."""
    import dataclasses
    scd = scenes.heightmap(view_deg=view, rms_slope=slope, device=DEV)
    scd = dataclasses.replace(scd, material=dataclasses.replace(scd.material, n_rings=rings))
    sc = scd.to("cpu")
    img = _render(scd)
    rng = np.random.default_rng(11)
    r = _anisotropy(sc)
    tail = np.flatnonzero(r > 16)
    picks = [rng.choice(r.size, 10000, replace=False)]
    if tail.size:
        picks.append(rng.choice(tail, min(2000, tail.size), replace=False))
    px = np.unique(np.concatenate(picks)).astype(np.int32)
    ref = orc.eval_image(sc, px=px)
    assert np.count_nonzero(ref) > 1000
    s = parity.check_image(orc, sc, scd, img, ref, px=px, sample_trace=300)
    _summary(f"{sc.name} rings={rings}", s)
    if view == 25.0 and slope > 0:
        # large anisotropy is scattered over the frame, not gathered in rows
        rows = np.unique(tail // sc.width)
        assert rows.size > sc.height // 2
        sel = tail[np.argsort(-r[tail])[:2000]].astype(np.int32)       # the most anisotropic
        pix, _ = glint.trace(scd, sel, cap=0)
        ok = pix["status"] == 0
        # pieces along the major axis: ceil(r / 2^M), at most 64
        kmaj = np.minimum(np.ceil(r[sel] / 2.0 ** rings - 1e-6), 64)
        assert (pix["K"][ok] >= kmaj[ok] - 1).all() and pix["K"][ok].max() >= 2

"""G-buffers generated on the GPU (glint_gbuffer_heightfield,
glint_gbuffer_sphere_plane) against the package's seeded CPU generator:
the same frames up to the rounding of FP64 transcendental functions and
summation order, and the same shaded image under glint_eval where the two
G-buffers agree.  These generators make benchmark inputs; the parity tests
against the oracle keep using the CPU generator's bytes."""
import numpy as np
import pytest
import torch

from paper_2306_05051_gb300 import _lib, glint, scenes

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _compare(a, b, rel):
    """Fraction of elements equal to the bit, and the largest relative
    difference (denominator: the field's own scale)."""
    a = a.cpu().double().numpy()
    b = b.cpu().double().numpy()
    same = float(np.mean(a == b))
    scale = np.maximum(np.abs(b), rel)
    return same, float(np.max(np.abs(a - b) / scale))


@pytest.mark.parametrize("view,slope", [(25.0, 0.45), (90.0, 0.45), (25.0, 0.0)])
def test_heightfield_matches_cpu_generator(view, slope):
    W, H = 480, 270
    g = glint.gbuffer_heightmap(W, H, view_deg=view, rms_slope=slope, device=DEV)
    c = scenes.heightmap(W, H, view_deg=view, rms_slope=slope, device="cpu")
    torch.cuda.synchronize()
    ga, ca = g.gbuf.cpu().reshape(-1, 16), c.gbuf.reshape(-1, 16)
    # the hit: the same surface point on all but a few grazing pixels
    close = (ga[:, 0:2] - ca[:, 0:2]).abs().max(1).values <= 1e-4 * 64
    assert close.double().mean() >= 0.999
    for lo, hi, tol in ((0, 2, 1e-5), (2, 6, 1e-4), (6, 15, 1e-5)):
        same, err = _compare(ga[close, lo:hi], ca[close, lo:hi], 1e-3)
        assert err <= tol, (lo, hi, err)
        assert same >= 0.5, (lo, hi, same)
    assert g.material == c.material and [l.dir for l in g.lights] == [l.dir for l in c.lights]


def test_sphere_plane_matches_cpu_generator():
    W, H = 640, 360
    g = glint.gbuffer_sphere_plane(W, H, azimuth_deg=40.0, seed=9, device=DEV)
    c = scenes.sphere_plane(W, H, azimuth_deg=40.0, seed=9, device="cpu")
    ga, ca = g.gbuf.cpu().reshape(-1, 16), c.gbuf.reshape(-1, 16)
    hit_g, hit_c = ga[:, 6:9].abs().sum(1) > 0, ca[:, 6:9].abs().sum(1) > 0
    assert (hit_g != hit_c).double().mean() <= 1e-3            # silhouettes only
    both = hit_g & hit_c
    for lo, hi, tol in ((0, 2, 1e-5), (2, 6, 1e-4), (6, 15, 1e-5)):
        same, err = _compare(ga[both, lo:hi], ca[both, lo:hi], 1e-3)
        assert err <= tol, (lo, hi, err)
        assert same >= 0.5, (lo, hi, same)
    nL = c.light_px.shape[0]
    la, lb = g.light_px.cpu().reshape(nL, -1, 4)[:, both], c.light_px.reshape(nL, -1, 4)[:, both]
    assert _compare(la, lb, 1e-3)[1] <= 1e-5
    ma, mb = g.mat_px.cpu().reshape(-1, 2)[both], c.mat_px.reshape(-1, 2)[both]
    assert _compare(ma, mb, 1e-3)[1] <= 1e-5


def test_generated_frame_shades_like_the_cpu_frame_where_they_agree():
    W, H = 640, 360
    g = glint.gbuffer_sphere_plane(W, H, device=DEV)
    c = scenes.sphere_plane(W, H).to(DEV)
    a, b = glint.render_scene(g), glint.render_scene(c)
    torch.cuda.synchronize()
    ident = (g.gbuf == c.gbuf).all(-1) & (g.light_px == c.light_px).all(-1).all(0) & (g.mat_px == c.mat_px).all(-1)
    assert ident.double().mean() > 0.2
    assert torch.equal(a[ident], b[ident])


def test_generator_argument_errors():
    import ctypes as C
    from paper_2306_05051_gb300 import scenes as S
    cam = glint._camera_struct(S.camera_basis(*S.heightmap_camera(10.0)), 0.27, 64, 32)   # rays above the horizon
    f = _lib.GlintHeightfield()
    f.n_waves, f.n_march, f.n_bisect, f.uv_scale = 1, 8, 8, 64.0
    f.amp[0] = 0.01
    out = torch.empty(32, 64, 16, device=DEV)
    assert _lib.lib().glint_gbuffer_heightfield(C.byref(cam), C.byref(f), out.data_ptr(), None) == -1
    f.n_waves = 33
    cam = glint._camera_struct(S.camera_basis(*S.heightmap_camera(60.0)), 0.27, 64, 32)
    assert _lib.lib().glint_gbuffer_heightfield(C.byref(cam), C.byref(f), out.data_ptr(), None) == -1

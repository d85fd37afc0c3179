"""Seeded scene generators: geometric invariants of the displaced-plane
(heightmap) G-buffer, which is ray-marched rather than analytic."""
import math

import numpy as np
import torch

from paper_2306_05051_gb300 import scenes


def test_heightfield_slope_statistics():
    hf = scenes.Heightfield.seeded(5)
    g = torch.Generator().manual_seed(1)
    x, z = torch.rand(200000, generator=g, dtype=torch.float64) * 10, torch.rand(200000, generator=g, dtype=torch.float64) * 10
    hx, hz = hf.gradient(x, z)
    rms = math.sqrt(float((hx * hx + hz * hz).mean()))
    assert abs(rms - 0.45) < 0.03
    # the analytic gradient matches central differences of the height
    e = 1e-7
    fd = (hf.height(x[:1000] + e, z[:1000]) - hf.height(x[:1000] - e, z[:1000])) / (2 * e)
    assert torch.allclose(fd, hx[:1000], atol=1e-6)
    assert float(hf.height(x, z).abs().max()) <= hf.bound


def test_heightmap_gbuffer_invariants():
    for view in (25.0, 90.0):
        sc = scenes.heightmap(192, 108, view_deg=view)
        g = sc.gbuf.double().reshape(-1, 16)
        n, tg, wv = g[:, 6:9], g[:, 9:12], g[:, 12:15]
        assert torch.allclose(torch.linalg.vector_norm(n, dim=-1), torch.ones(len(g), dtype=torch.float64), atol=1e-6)
        assert float((n * tg).sum(-1).abs().max()) < 1e-6            # tangent lies in the tangent plane
        assert float((n * wv).sum(-1).min()) > 0                     # every visible facet faces the camera
        assert ((g[:, 0] >= 0) & (g[:, 0] < 64) & (g[:, 1] >= 0) & (g[:, 1] < 64)).all()
        J = torch.stack([torch.stack([g[:, 2], g[:, 4]], -1), torch.stack([g[:, 3], g[:, 5]], -1)], -2)
        sv = torch.linalg.svdvals(J)
        r = (sv[:, 0] / sv[:, 1]).numpy()
        if view == 90.0:
            assert r.max() < 4                                       # seen from above: nearly isotropic
        else:
            assert np.median(r) > 1.5 and r.max() > 16               # grazing: anisotropy with a long tail


def test_heightmap_first_hit_lies_on_the_surface():
    hf = scenes.Heightfield.seeded(5)
    eye, D, _, _ = scenes.camera_rays(64, 36, (0.0, 1.0, 0.0), (0.0, 1.0 - math.sin(0.436), -math.cos(0.436)),
                                      30.0, up=(0.0, 0.0, -1.0))
    t = scenes._hit_heightfield(eye, D, hf)
    P = eye + t[..., None] * D
    assert float((P[..., 1] - hf.height(P[..., 0], P[..., 2])).abs().max()) < 1e-12
    # the march may step through crests thinner than one step; check that
    # this is rare with a sweep 16 times finer than the march
    tin = (hf.bound - eye[1]) / D[..., 1]
    earlier = torch.zeros_like(t, dtype=torch.bool)
    for a in torch.linspace(0, 1, 2049, dtype=torch.float64)[:-1]:
        tt = tin + a * (t - tin)
        Q = eye + tt[..., None] * D
        earlier |= (Q[..., 1] - hf.height(Q[..., 0], Q[..., 2])) < -1e-9
    assert float(earlier.double().mean()) < 0.01


def test_heightmap_uv_derivatives_match_finite_differences():
    """The stored du/dx ... dv/dy are the first-order ray differentials of
    the ray-marched hit: compare with central differences of hits of rays
    moved by +-1e-5 pixel (same crossing, so the difference is smooth; at
    grazing pixels a 1e-3 pixel step is already off by the curvature)."""
    W, H, view = 96, 54, 25.0
    v = math.radians(view)
    eye, D, dDdx, dDdy = scenes.camera_rays(W, H, (0.0, 1.0, 0.0), (0.0, 1.0 - math.sin(v), -math.cos(v)), 30.0,
                                            up=(0.0, 0.0, -1.0))
    sc = scenes.heightmap(W, H, view_deg=view)
    hf = scenes.Heightfield.seeded(5)
    g = sc.gbuf.double()
    rng = np.random.default_rng(3)
    ys, xs = rng.integers(0, H, 60), rng.integers(0, W, 60)
    d = 1e-5
    checked = 0
    for y, x in zip(ys, xs):
        n, wv = g[y, x, 6:9], g[y, x, 12:15]
        if float((n * wv).sum()) < 0.2:        # near-silhouette: a nearby ray may hit another facet
            continue
        rays = torch.stack([D[y, x] + d * dDdx, D[y, x] - d * dDdx, D[y, x] + d * dDdy, D[y, x] - d * dDdy])
        t = scenes._hit_heightfield(eye, rays[:, None, :], hf)[:, 0]
        P = eye + t[:, None] * rays
        uv = 64.0 * P[:, [0, 2]]
        du_dx, du_dy = (uv[0] - uv[1]) / (2 * d), (uv[2] - uv[3]) / (2 * d)
        J = torch.tensor([[g[y, x, 2], g[y, x, 4]], [g[y, x, 3], g[y, x, 5]]], dtype=torch.float64)
        fd = torch.stack([du_dx, du_dy], -1)                   # rows u, v; columns x, y
        assert torch.allclose(fd, J, rtol=1e-3, atol=1e-4 * float(J.abs().max())), (y, x, fd, J)
        checked += 1
    assert checked > 30


def test_flat_plane_views():
    """rms_slope = 0: the flat plane of the same views (Table 1's Plane
    scenes); seen from above every footprint is isotropic, at 25 degrees
    the anisotropy is 1/sin of the grazing angle, about 1.5 to 6.5."""
    for view, lo, hi in ((90.0, 1.0 - 1e-6, 1.0 + 1e-6), (25.0, 1.4, 7.0)):
        sc = scenes.heightmap(160, 90, view_deg=view, rms_slope=0.0)
        assert sc.name == f"plane{int(view)}"
        g = sc.gbuf.double().reshape(-1, 16)
        assert torch.equal(g[:, 6:9], torch.tensor([0.0, 1.0, 0.0], dtype=torch.float64).expand(len(g), 3).abs())
        J = torch.stack([torch.stack([g[:, 2], g[:, 4]], -1), torch.stack([g[:, 3], g[:, 5]], -1)], -2)
        sv = torch.linalg.svdvals(J)
        r = sv[:, 0] / sv[:, 1]
        assert float(r.min()) >= lo and float(r.max()) <= hi

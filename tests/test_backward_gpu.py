"""Adjoint (glint_backward) on the 512^2 plane + sphere fit scene: the GPU
gradient of an L2 image loss against the oracle's FP64 dual-number gradient,
against central finite differences (h = 1e-3) of the GPU's relaxed image away
from discrete changes, the relaxed image against the oracle, and the
torch.autograd wrapper."""
import copy
import math

import numpy as np
import pytest
import torch

from paper_2306_05051_gb300 import _lib, glint, scenes

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
NAMES = ["alpha_x", "alpha_y", "ln_density", "dir_x", "dir_y", "dir_z"]


@pytest.fixture(scope="module")
def fit():
    sc = scenes.plane_sphere_fit()
    tgt = scenes.plane_sphere_fit(target=True)
    scd = sc.to(DEV)
    img = glint.render_scene(scd)
    timg = glint.render_scene(scd, material=tgt.material, lights=tgt.lights)
    go = 2.0 * (img - timg)
    torch.cuda.synchronize()
    return sc, scd, go


def test_adjoint_matches_oracle_dual_gradient(orc, fit):
    sc, scd, go = fit
    g = glint.backward(scd, go).cpu().numpy().astype(np.float64)
    g6, _, _ = orc.grad(sc, go.cpu().numpy().astype(np.float64).reshape(-1))
    print("gpu   ", g)
    print("oracle", g6)
    for k in range(6):
        assert abs(g[k] - g6[k]) <= 1e-3 * abs(g6[k]) + 1e-6 * np.abs(g6).max(), (NAMES[k], g[k], g6[k])


def test_adjoint_with_fresnel_f0_matches_oracle(orc, fit):
    """F0 = 0.04: the Schlick term and its derivative through the half-vector
    (light direction) enter the gradient."""
    import dataclasses
    sc, scd, go = fit
    mat = dataclasses.replace(sc.material, F0=0.04)
    g = glint.backward(scd, go, material=mat).cpu().numpy().astype(np.float64)
    g6, _, _ = orc.grad(sc, go.cpu().numpy().astype(np.float64).reshape(-1), material=mat)
    g1, _, _ = orc.grad(sc, go.cpu().numpy().astype(np.float64).reshape(-1))
    assert np.abs(g6[3:] - g1[3:]).max() > 1e-3 * np.abs(g1[3:]).max()     # F changes the direction gradient
    for k in range(6):
        assert abs(g[k] - g6[k]) <= 1e-3 * abs(g6[k]) + 1e-6 * np.abs(g6).max(), (NAMES[k], g[k], g6[k])


def test_relaxed_image_matches_oracle(orc, fit):
    sc, scd, go = fit
    _, rel = glint.backward(scd, go, relaxed=True)
    rel = rel.cpu().numpy().astype(np.float64).reshape(-1)
    _, _, orel = orc.grad(sc, np.zeros(sc.width * sc.height))
    scale = max(np.abs(orel).mean(), 1e-30)
    err = np.abs(rel - orel) / np.maximum(np.abs(orel), 1e-6 * scale)
    assert np.count_nonzero(err > 1e-4) <= max(2, int(1e-4 * err.size)), err.max()


def _perturb(scene, k, sign, h):
    mat = copy.deepcopy(scene.material)
    lights = copy.deepcopy(scene.lights)
    if k < 3:
        name = ("alpha_x", "alpha_y", "ln_density")[k]
        base = float(np.float32(getattr(mat, name)))
        new = float(np.float32(base + sign * h))
        setattr(mat, name, new)
        return mat, lights, new - base
    d = list(lights[0].dir)
    base = float(np.float32(d[k - 3]))
    new = float(np.float32(base + sign * h))
    d[k - 3] = new
    lights[0].dir = tuple(d)
    return mat, lights, new - base


def _state(scd, px, mat, lights):
    pix, recs = glint.trace(scd, px, cap=48, material=mat, lights=lights)
    r = recs
    return (pix["K"], pix["status"], r["gid"], r["i"], r["j"], r["ax"], r["ay"], r["gate"])


def test_adjoint_matches_central_differences(fit):
    """FD with h = 1e-3 of the relaxed image, on pixels whose discrete state
    (grids, lattice vertices, texels, gates, K) is the same at both ends."""
    sc, scd, go = fit
    rng = np.random.default_rng(7)
    lit = np.flatnonzero(go.cpu().numpy().reshape(-1) != 0)
    sub = np.sort(rng.choice(lit, size=min(20000, len(lit)), replace=False)).astype(np.int32)
    s0 = _state(scd, sub, sc.material, sc.lights)
    for k in range(6):
        h = 1e-3
        mp, lp, hp = _perturb(sc, k, +1, h)
        mm, lm, hm = _perturb(sc, k, -1, h)
        sp = _state(scd, sub, mp, lp)
        sm = _state(scd, sub, mm, lm)
        keep = np.ones(len(sub), bool)
        for a, b, c in zip(s0, sp, sm):
            if a.ndim == 1:
                keep &= (a == b) & (a == c)
            else:
                keep &= ((a == b) & (a == c)).all(1)
        kept = sub[keep]
        mask = torch.zeros(sc.height * sc.width, device=DEV)
        mask[torch.as_tensor(kept, device=DEV, dtype=torch.long)] = 1.0
        gom = (go.reshape(-1) * mask).reshape(sc.height, sc.width).contiguous()
        g = glint.backward(scd, gom)[k].item()
        _, rp = glint.backward(scd, gom, material=mp, lights=lp, relaxed=True)
        _, rm = glint.backward(scd, gom, material=mm, lights=lm, relaxed=True)
        fd = float(((rp - rm).double() * gom.double()).sum().item()) / (hp - hm)
        print(f"{NAMES[k]}: kept {len(kept)}/{len(sub)}  adjoint {g:.6g}  fd {fd:.6g}")
        if len(kept) < 50:
            continue                                   # (ln density: the lattice moves by ~q/2000 cells)
        assert abs(g - fd) <= 1e-2 * max(abs(g), abs(fd)) + 1e-6, (NAMES[k], g, fd)


def test_autograd_function_matches_backward(fit):
    sc, scd, go = fit
    m = sc.material
    ax = torch.tensor(m.alpha_x, dtype=torch.float64, requires_grad=True)
    ay = torch.tensor(m.alpha_y, dtype=torch.float64, requires_grad=True)
    lr = torch.tensor(m.ln_density, dtype=torch.float64, requires_grad=True)
    dirs = torch.tensor([list(sc.lights[0].dir)], dtype=torch.float64, requires_grad=True)
    img = glint.GlintBRDF.apply(ax, ay, lr, dirs, scd)
    assert torch.equal(img, glint.render_scene(scd))
    tgt = scenes.plane_sphere_fit(target=True)
    timg = glint.render_scene(scd, material=tgt.material, lights=tgt.lights)
    loss = ((img - timg) ** 2).sum()
    loss.backward()
    g = glint.backward(scd, (2.0 * (img - timg)).detach().contiguous()).cpu().double()
    got = torch.stack([ax.grad, ay.grad, lr.grad] + list(dirs.grad.reshape(-1)))
    assert torch.allclose(got, g, rtol=1e-6, atol=0)


def test_backward_argument_errors(fit):
    sc, scd, go = fit
    import ctypes as C
    frame = _lib.frame_struct(scd.gbuf, None, None, 1)
    mat = _lib.material_struct(sc.material)
    lts = _lib.lights_struct(sc.lights)
    g = torch.empty(6, device=DEV)
    ws = torch.empty(16, dtype=torch.float64, device=DEV)
    L = _lib.lib()
    need = L.glint_backward_workspace_size(C.byref(frame))
    assert need > 16 * 8
    assert L.glint_backward(C.byref(frame), C.byref(mat), lts, go.data_ptr(), g.data_ptr(), None, ws.data_ptr(),
                            16 * 8, None) == -6
    rnd = scenes.random_gbuffer(seed=1).to(DEV)        # per-pixel material plane: no scalar gradient
    fr2 = _lib.frame_struct(rnd.gbuf, rnd.light_px, rnd.mat_px, len(rnd.lights))
    go2 = torch.zeros(rnd.height, rnd.width, device=DEV)
    assert L.glint_backward(C.byref(fr2), C.byref(mat), _lib.lights_struct(rnd.lights), go2.data_ptr(),
                            torch.empty(9, device=DEV).data_ptr(), None, ws.data_ptr(), 16 * 8, None) == -5


def test_fit_l2_one_pass_matches_forward_plus_backward(orc, fit):
    """glint_fit_l2: image equal to glint_eval's up to summation order, loss
    and gradient equal to render -> 2 (img - target) -> glint_backward, and
    the gradient equal to the oracle's for the same grad_out."""
    sc, scd, go = fit
    tgt = scenes.plane_sphere_fit(target=True)
    timg = glint.render_scene(scd, material=tgt.material, lights=tgt.lights)
    img = glint.render_scene(scd)
    out, g, loss = glint.fit_l2(scd, timg)
    torch.cuda.synchronize()
    a, b = out.double(), img.double()
    scale = b.abs().mean().item()
    assert ((a - b).abs() / b.abs().clamp_min(1e-6 * scale)).max().item() <= 1e-5
    ref_loss = ((img.double() - timg.double()) ** 2).sum().item()
    assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss
    g2 = glint.backward(scd, (2.0 * (img - timg)).contiguous())
    gg, gr = g.double().cpu().numpy(), g2.double().cpu().numpy()
    for k in range(6):
        assert abs(gg[k] - gr[k]) <= 1e-4 * abs(gr[k]) + 1e-7 * np.abs(gr).max(), (NAMES[k], gg[k], gr[k])
    go_fused = (2.0 * (out.double() - timg.double())).cpu().numpy().reshape(-1)
    g6, _, _ = orc.grad(sc, go_fused)
    for k in range(6):
        assert abs(gg[k] - g6[k]) <= 1e-3 * abs(g6[k]) + 1e-6 * np.abs(g6).max(), (NAMES[k], gg[k], g6[k])


def test_fit_l2_repeatable_and_argument_errors(fit):
    sc, scd, go = fit
    import ctypes as C
    tgt = torch.zeros(sc.height, sc.width, device=DEV)
    o1, g1, l1 = glint.fit_l2(scd, tgt)
    o2, g2, l2 = glint.fit_l2(scd, tgt)
    torch.cuda.synchronize()
    assert torch.equal(o1, o2) and torch.equal(g1, g2) and torch.equal(l1, l2)
    L = _lib.lib()
    frame = _lib.frame_struct(scd.gbuf, None, None, 1)
    mat = _lib.material_struct(sc.material)
    lts = _lib.lights_struct(sc.lights)
    ws = torch.empty(16, dtype=torch.float64, device=DEV)
    out = torch.empty_like(tgt)
    g = torch.empty(6, device=DEV)
    assert L.glint_fit_l2(C.byref(frame), C.byref(mat), lts, None, out.data_ptr(), g.data_ptr(), None,
                          ws.data_ptr(), 16 * 8, None) == -1
    assert L.glint_fit_l2(C.byref(frame), C.byref(mat), lts, tgt.data_ptr(), out.data_ptr(), g.data_ptr(), None,
                          ws.data_ptr(), 16 * 8, None) == -6
    rnd = scenes.random_gbuffer(seed=1).to(DEV)
    fr2 = _lib.frame_struct(rnd.gbuf, rnd.light_px, rnd.mat_px, len(rnd.lights))
    t2 = torch.zeros(rnd.height, rnd.width, device=DEV)
    o3 = torch.empty_like(t2)
    assert L.glint_fit_l2(C.byref(fr2), C.byref(mat), _lib.lights_struct(rnd.lights), t2.data_ptr(),
                          o3.data_ptr(), torch.empty(9, device=DEV).data_ptr(), None, ws.data_ptr(), 16 * 8,
                          None) == -5

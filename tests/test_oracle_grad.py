"""Pin of the oracle's FP64 dual-number gradient against central finite
differences of its relaxed image (counts before integer rounding), on
pixels whose discrete state (grids, lattice vertices, angular texels, gates,
sub-footprints, tetrahedron, triangle) is the same at both ends of the step."""
import copy
import math

import numpy as np
import pytest

from paper_2306_05051_gb300 import scenes


def _f32(x):
    return float(np.float32(x))


def _state(orc, scene, px, material, lights):
    pix, recs = orc.trace_pixel(scene, px, material=material, lights=lights)
    return (int(pix["K"]), recs["gid"].tobytes(), recs["i"].tobytes(), recs["j"].tobytes(),
            recs["ax"].tobytes(), recs["ay"].tobytes(), recs["gate"].tobytes(),
            recs["tet"].tobytes(), recs["tri"].tobytes())


def _perturbed(scene, k, sign, h):
    """(material, lights, effective step) with parameter k moved by sign*h,
    rounded to what the float32 interface carries."""
    mat = copy.deepcopy(scene.material)
    lights = copy.deepcopy(scene.lights)
    if k < 3:
        name = ("alpha_x", "alpha_y", "ln_density")[k]
        base = _f32(getattr(mat, name))
        new = _f32(base + sign * h)
        setattr(mat, name, new)
        return mat, lights, new - base
    d = list(lights[0].dir)
    base = _f32(d[k - 3])
    new = _f32(base + sign * h)
    d[k - 3] = new
    lights[0].dir = tuple(d)
    return mat, lights, new - base


@pytest.mark.parametrize("k,h,min_frac", [(0, 2e-6, 0.6), (1, 2e-6, 0.6), (2, 4e-6, 0.2),
                                          (3, 2e-6, 0.5), (4, 2e-6, 0.5), (5, 2e-6, 0.5)])
def test_dual_gradient_matches_central_differences(orc, k, h, min_frac):
    scene = scenes.plane_sphere_fit(96, 96)
    ref = orc.eval_image(scene, relaxed=True).ravel()
    pxs = np.flatnonzero(ref > 0)
    rng = np.random.default_rng(20 + k)
    pxs = np.sort(rng.choice(pxs, size=min(200, len(pxs)), replace=False)).astype(np.int32)
    g6, per, rel = orc.grad(scene, np.ones(len(pxs)), px=pxs, per_pixel=True)
    np.testing.assert_allclose(rel, ref[pxs], rtol=1e-13, atol=0)
    assert np.all(np.abs(g6 - per.sum(0)) <= 1e-12 * np.abs(per).sum(0))
    mp, lp, hp = _perturbed(scene, k, +1, h)
    mm, lm, hm = _perturbed(scene, k, -1, h)
    fp = orc.eval_image(scene, px=pxs, relaxed=True, material=mp, lights=lp)
    fm = orc.eval_image(scene, px=pxs, relaxed=True, material=mm, lights=lm)
    fd = (fp - fm) / (hp - hm)
    ok = 0
    for n, px in enumerate(pxs):
        s0 = _state(orc, scene, px, scene.material, scene.lights)
        if _state(orc, scene, px, mp, lp) != s0 or _state(orc, scene, px, mm, lm) != s0:
            continue
        ok += 1
        d = per[n, k]
        tol = 1e-5 * max(abs(d), abs(fd[n])) + 1e-13 * abs(ref[px]) / abs(hp)
        assert abs(fd[n] - d) <= tol, (px, fd[n], d)
    assert ok >= min_frac * len(pxs), (ok, len(pxs))

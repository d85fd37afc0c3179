"""Statistical pins of the oracle's counting law against independent
computations: a brute-force per-flake Bernoulli simulation (Sec. 4.1,
stratified flakes), binomial additivity (Sec. 4.2), coherence between
consecutive LODs (Sec. 1 specification), and convergence to the smooth NDF
(Sec. 3, Eq. 5-6; Sec. 7)."""
import math

import numpy as np
import pytest
import torch

from paper_2306_05051_gb300.scenes import Light, Material, Scene


def pixel_row(uv, J, w=(0.0, 0.0, 1.0), material=None, E=1.0):
    """A 1 x N G-buffer: flat patch with normal +z, tangent +x, given uv and
    footprint Jacobian J = [[du/dx, du/dy], [dv/dx, dv/dy]]; view and
    (directional) light both along w, so the half-vector is w."""
    uv = np.asarray(uv, np.float64)
    N = len(uv)
    J = np.broadcast_to(np.asarray(J, np.float64), (N, 2, 2))
    g = np.zeros((1, N, 16), np.float32)
    g[0, :, 0:2] = uv
    g[0, :, 2] = J[:, 0, 0]; g[0, :, 3] = J[:, 1, 0]
    g[0, :, 4] = J[:, 0, 1]; g[0, :, 5] = J[:, 1, 1]
    g[0, :, 8] = 1.0
    g[0, :, 9] = 1.0
    g[0, :, 12:15] = w
    mat = material or Material()
    return Scene("pixels", torch.from_numpy(g), None, None, mat,
                 [Light(kind=1, dir=tuple(w), intensity=E)])


def count_scale(orc, scene, A):
    """C = out * 4 R A cos_v / (D(n) G E) for the pixel_row geometry."""
    m = scene.material
    w = np.asarray(scene.lights[0].dir, float)
    w = w / np.linalg.norm(w)
    lam = orc.smith_lambda(m.ndf, m.alpha_x, m.alpha_y, w[0], w[1], w[2])
    G = 1.0 / (1.0 + lam) ** 2
    Dn = orc.ndf(m.ndf, m.alpha_x, m.alpha_y, 0.0, 0.0, 1.0)
    return 4.0 * m.R * A * w[2] / (Dn * G * scene.lights[0].intensity)


def eff_rho(rho):
    """The density the library sees: ln(density) crosses the interface as float32."""
    return math.exp(float(np.float32(math.log(rho))))


def square_J(A_uv, ratio=1.0, angle=0.0):
    a = math.sqrt(A_uv * ratio); b = math.sqrt(A_uv / ratio)
    c, s = math.cos(angle), math.sin(angle)
    R = np.array([[c, -s], [s, c]])
    return (R @ np.diag([a, b])).astype(np.float32).astype(np.float64)


def nearest_counts(orc, scene, n):
    """Per pixel: sum over the 4 tetrahedron vertices of one realisation (the
    spatial and angular texel of largest weight), i.e. the distributed
    binomial of Sec. 4.2 without the realisation interpolation of Eq. 14."""
    out = np.zeros(n)
    for px in range(n):
        pix, recs = orc.trace_pixel(scene, px)
        assert pix["status"] == 0
        tot = 0
        for vert in range(4):
            r = recs[(recs["vert"] == vert) & (recs["sub"] == 0)]
            k = np.argmax(r["u"] * 1000.0 + r["v"])          # max u, then max v
            best = r[(r["sv"] == r["sv"][k])]
            best = best[np.argmax(best["v"])]
            tot += best["c"]
        out[px] = tot
    return out


def brute_force_counts(A, p, J, rho, n_place, rng):
    """Explicit stratified flakes: one per cell of side rho^-1/2, jittered,
    each reflecting with probability p; count flakes with X < p inside the
    footprint parallelogram uv + J [-1/2, 1/2]^2 at a random placement."""
    cell = 1.0 / math.sqrt(rho)
    Jinv = np.linalg.inv(J)
    half = 0.5 * (np.abs(J).sum(1))                         # bounding box half extent
    counts = np.zeros(n_place)
    for k in range(n_place):
        c = rng.uniform(0, 1000 * cell, 2)
        i0 = np.floor((c - half) / cell).astype(int) - 1
        i1 = np.floor((c + half) / cell).astype(int) + 1
        ii, jj = np.meshgrid(np.arange(i0[0], i1[0] + 1), np.arange(i0[1], i1[1] + 1), indexing="ij")
        pos = (np.stack([ii, jj], -1) + rng.uniform(0, 1, ii.shape + (2,))) * cell
        loc = (pos - c) @ Jinv.T
        inside = (np.abs(loc) <= 0.5).all(-1)
        X = rng.uniform(0, 1, ii.shape)
        counts[k] = np.count_nonzero(inside & (X < p))
    return counts


@pytest.mark.parametrize("A,p", [(0.25, 0.034), (1.0, 0.034), (4.0, 0.034), (64.0, 0.5), (1024.0, 0.5)])
def test_counts_match_brute_force_flakes(orc, A, p):
    rho = 1e6
    rng = np.random.default_rng(int(A * 100))
    J = square_J(A / rho, ratio=1.7, angle=0.6)
    A_true = abs(np.linalg.det(J)) * eff_rho(rho)
    n = 4000 if A < 100 else 1500
    uv = rng.uniform(0, 3, (n, 2))
    mat = Material(R=p, ln_density=math.log(rho), n_lods=12)
    scene = pixel_row(uv, J, material=mat)
    meth = nearest_counts(orc, scene, n)
    brute = brute_force_counts(A_true, p, J, rho, 3000 if A < 100 else 600, rng)
    # exact expectation of the flake model: A p
    se_b = brute.std() / math.sqrt(len(brute))
    assert abs(brute.mean() - A_true * p) <= 4 * se_b + 1e-12
    se_m = meth.std() / math.sqrt(n)
    bias = 0.02 * A_true * p if A_true * p < 1 else 0.5 + 0.01 * A_true * p
    assert abs(meth.mean() - brute.mean()) <= 4 * math.hypot(se_m, se_b) + bias, (meth.mean(), brute.mean())
    ratio = meth.var() / brute.var()
    assert 0.8 <= ratio <= 1.2, (meth.var(), brute.var())


def test_distributed_counts_are_binomial_in_the_footprint_area(orc):
    """Sec. 4.2: sum of the per-vertex binomials of trials w_i N_i behaves as
    one binomial over the footprint: mean A p, variance A p (1 - p), and the
    trials sum to A exactly."""
    rng = np.random.default_rng(11)
    rho, p = 1e6, 0.5
    for A in (37.0, 300.0, 5000.0):
        J = square_J(A / rho, ratio=5.0, angle=1.1)
        A_true = abs(np.linalg.det(J)) * eff_rho(rho)
        n = 1500
        uv = rng.uniform(0, 3, (n, 2))
        scene = pixel_row(uv, J, material=Material(R=p, ln_density=math.log(rho), n_lods=12))
        for px in range(0, n, 97):
            _, recs = orc.trace_pixel(scene, px)
            trials = sum(recs[(recs["vert"] == v)]["n"][0] for v in range(4))
            assert trials == pytest.approx(A_true, rel=1e-12)
        c = nearest_counts(orc, scene, n)
        se = c.std() / math.sqrt(n)
        assert abs(c.mean() - A_true * p) <= 4 * se + 0.5
        assert c.var() / (A_true * p * (1 - p)) == pytest.approx(1.0, abs=0.15)


def test_lod_coherence(orc):
    """Coherence between consecutive LODs (Sec. 1): at a bracket boundary the
    counts from both sides agree; within a bracket the grids used stay the
    six vertices of one prism; the mean count is linear in A."""
    rng = np.random.default_rng(12)
    rho, f = 1e6, 4
    n = 256
    uv = rng.uniform(0, 3, (n, 2))
    mat = Material(R=0.5, ln_density=math.log(rho), n_lods=12)
    base = square_J(1.0 / rho, ratio=3.0, angle=0.4)
    A0 = abs(np.linalg.det(base)) * eff_rho(rho)
    for level in (2, 3, 5):
        boundary = float(f) ** level
        outs = []
        for eps in (-1e-7, 1e-7):
            Jc = base * math.sqrt(boundary * (1 + eps) / A0)
            sc = pixel_row(uv, Jc, material=mat)
            outs.append((orc.eval_image(sc, relaxed=True)[0], orc.eval_image(sc)[0]))
        (rl, il), (rh, ih) = outs
        np.testing.assert_allclose(rl, rh, rtol=1e-5, atol=1e-9)
        np.testing.assert_allclose(il, ih, rtol=1e-5, atol=1e-9)
        # inside the bracket: the grids belong to one prism (2 levels x 3)
        for px in range(0, n, 37):
            grids = set()
            for frac in np.linspace(0.02, 0.98, 9):
                Jc = base * math.sqrt(boundary * (1 + 3 * frac) / A0)
                _, recs = orc.trace_pixel(pixel_row(uv[px:px + 1], Jc, material=mat), 0)
                grids |= set(zip(recs["level"], recs["ring"], recs["kor"]))
            assert len(grids) <= 6 and {g[0] for g in grids} <= {level, level + 1}
    # E[C] linear in A within [f^3, f^4]
    n = 2000
    uv = rng.uniform(0, 3, (n, 2))
    As, means = [], []
    for frac in (0.0, 0.25, 0.5, 0.75):
        A = 64.0 * (1 + 3 * frac)
        Jc = base * math.sqrt(A / A0)
        sc = pixel_row(uv, Jc, material=mat)
        C = orc.eval_image(sc)[0] * count_scale(orc, sc, A)
        As.append(A); means.append(C.mean())
        assert C.mean() == pytest.approx(A * 0.5, rel=4 * C.std() / math.sqrt(n) / (A * 0.5) + 0.01)


@pytest.mark.parametrize("kind", [0, 1])
def test_convergence_to_smooth_ndf(orc, kind):
    """Sec. 3, Eq. 5-6 and Sec. 7: D_P / D(h) -> 1 as the flake count grows."""
    rng = np.random.default_rng(13 + kind)
    n = 400
    uv = rng.uniform(0, 5, (n, 2))
    th = math.radians(12.0)
    w = (math.sin(th) * math.cos(0.7), math.sin(th) * math.sin(0.7), math.cos(th))
    J = square_J(1e-6, ratio=2.0, angle=0.3)
    P = abs(np.linalg.det(J))
    last_err = None
    for log_rho in (3, 6, 9, 12):
        rho = 10.0 ** log_rho
        mat = Material(ndf=kind, alpha_x=0.3, alpha_y=0.2, R=0.034, ln_density=math.log(rho), n_lods=12)
        sc = pixel_row(uv, J, w=w, material=mat)
        A = P * eff_rho(rho)
        C = orc.eval_image(sc)[0] * count_scale(orc, sc, A)
        h = np.array(w) / np.linalg.norm(w)
        Dh = orc.ndf(kind, 0.3, 0.2, h[0], h[1], h[2])
        Dn = orc.ndf(kind, 0.3, 0.2, 0.0, 0.0, 1.0)
        p = 0.034 * Dh / Dn
        ratio = C / (A * p)                                # = D_P / D(h)
        bound = 4 / math.sqrt(A * p) + 1 / (A * p)
        assert np.mean(np.abs(ratio - 1) <= bound) >= 0.99
        err = abs(ratio.mean() - 1)
        assert err <= 4 * ratio.std() / math.sqrt(n) + 0.6 / (A * p) + 1e-12
        last_err = err
    assert last_err < 1e-3

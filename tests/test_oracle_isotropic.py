"""Isotropic-grid mode (n_rings = 0): the distributed binomial of Sec. 4 on
the single isotropic grid, with the anisotropic footprint filtered by hand -
cut along its major axis into ceil(r) pieces - instead of the anisotropic
grids of Sec. 5.  Pins: the enumeration (two LOD vertices of ring 0, 24
evaluations per piece and light), the trials summing to the footprint area,
equality with the ring mode where the footprint is isotropic, and the
brute-force flake model for anisotropic footprints."""
import dataclasses
import math

import numpy as np
import pytest

from paper_2306_05051_gb300.scenes import Material
from test_oracle_stats import brute_force_counts, count_scale, eff_rho, pixel_row, square_J


def iso(m):
    return dataclasses.replace(m, n_rings=0)


@pytest.mark.parametrize("ratio", [1.5, 3.0, 7.2, 20.0])
def test_pieces_and_enumeration(orc, ratio):
    rho, A = 1e6, 40.0
    J = square_J(A / rho, ratio=ratio, angle=0.8)
    A_true = abs(np.linalg.det(J)) * eff_rho(rho)
    sv = np.linalg.svd(J, compute_uv=False)                # J as the library sees it (float32 entries)
    r = sv[0] / sv[1]
    mat = iso(Material(R=0.3, ln_density=math.log(rho), n_lods=12))
    sc = pixel_row(np.array([[0.3, 0.7]]), J, material=mat)
    pix, recs = orc.trace_pixel(sc, 0)
    assert int(pix["status"]) == 0
    K = int(pix["K"])
    assert K == math.ceil(r)                               # ceil(r) pieces (no LOD split at this area)
    assert len(recs) == 24 * K                             # 2 LOD vertices x 3 simplex x 4 angular per piece
    assert set(np.unique(recs["vert"])) == {0, 3}
    assert set(np.unique(recs["ring"])) == {0} and set(np.unique(recs["kor"])) == {0}
    lv = np.unique(recs["level"])
    assert len(lv) <= 2 and (len(lv) == 1 or lv[1] == lv[0] + 1)
    trials = 0.0
    for sub in range(K):
        rs = recs[recs["sub"] == sub]
        trials += sum(rs[rs["vert"] == v]["n"][0] for v in (0, 3))
    assert trials == pytest.approx(A_true, rel=1e-12)      # Sec. 4.2: the pieces' trials sum to A


def test_equals_ring_mode_for_isotropic_footprints(orc):
    """r = 1: the ring mode's cell puts all weight on ring 0 too, so both
    modes count the same flakes (the ring mode also evaluates two
    zero-weight vertices whose gates never open)."""
    rng = np.random.default_rng(21)
    rho = 1e6
    uv = rng.uniform(0, 4, (300, 2))
    for A in (0.3, 5.0, 900.0, 3e6):
        c = math.sqrt(A / rho)
        J = np.diag([c, c]).astype(np.float32).astype(np.float64)
        mat = Material(R=0.4, ln_density=math.log(rho), n_lods=12)
        a = orc.eval_image(pixel_row(uv, J, material=mat))
        b = orc.eval_image(pixel_row(uv, J, material=iso(mat)))
        np.testing.assert_array_equal(a, b)
        ar = orc.eval_image(pixel_row(uv, J, material=mat), relaxed=True)
        br = orc.eval_image(pixel_row(uv, J, material=iso(mat)), relaxed=True)
        np.testing.assert_array_equal(ar, br)
        assert np.count_nonzero(a) > 0


def nearest_counts_all_pieces(orc, scene, n):
    """Per pixel: over every piece and both LOD vertices, the count of the
    realisation of largest spatial and then angular weight."""
    out = np.zeros(n)
    for px in range(n):
        pix, recs = orc.trace_pixel(scene, px)
        assert pix["status"] == 0
        tot = 0
        for sub in range(int(pix["K"])):
            for vert in (0, 3):
                r = recs[(recs["vert"] == vert) & (recs["sub"] == sub)]
                k = np.argmax(r["u"] * 1000.0 + r["v"])
                best = r[r["sv"] == r["sv"][k]]
                tot += best[np.argmax(best["v"])]["c"]
        out[px] = tot
    return out


@pytest.mark.parametrize("A,ratio", [(48.0, 6.0), (300.0, 12.0)])
def test_anisotropic_counts_match_brute_force_flakes(orc, A, ratio):
    """Sec. 4.1 flake model on an anisotropic footprint: the hand-filtered
    isotropic evaluation counts A p flakes on average."""
    rho, p = 1e6, 0.5
    rng = np.random.default_rng(int(A + ratio))
    J = square_J(A / rho, ratio=ratio, angle=0.5)
    A_true = abs(np.linalg.det(J)) * eff_rho(rho)
    n = 1200
    uv = rng.uniform(0, 3, (n, 2))
    sc = pixel_row(uv, J, material=iso(Material(R=p, ln_density=math.log(rho), n_lods=12)))
    meth = nearest_counts_all_pieces(orc, sc, n)
    brute = brute_force_counts(A_true, p, J, rho, 1500, rng)
    se_b = brute.std() / math.sqrt(len(brute))
    assert abs(brute.mean() - A_true * p) <= 4 * se_b + 1e-12
    se_m = meth.std() / math.sqrt(n)
    assert abs(meth.mean() - A_true * p) <= 4 * math.hypot(se_m, se_b) + 0.5 + 0.01 * A_true * p, \
        (meth.mean(), A_true * p)
    # the pieces share lattice texels at their borders, so their counts are
    # correlated: the variance is that of the flake model within a factor 2
    assert 0.5 <= meth.var() / brute.var() <= 2.0, (meth.var(), brute.var())


def test_mean_count_is_unbiased_with_interpolation(orc):
    """The interpolated (image) count of the isotropic mode has mean A p."""
    rho, p, A, ratio = 1e6, 0.5, 120.0, 9.0
    rng = np.random.default_rng(5)
    J = square_J(A / rho, ratio=ratio, angle=1.3)
    A_true = abs(np.linalg.det(J)) * eff_rho(rho)
    n = 3000
    uv = rng.uniform(0, 3, (n, 2))
    sc = pixel_row(uv, J, material=iso(Material(R=p, ln_density=math.log(rho), n_lods=12)))
    C = orc.eval_image(sc)[0] * count_scale(orc, sc, A_true)
    assert C.mean() == pytest.approx(A_true * p, rel=4 * C.std() / math.sqrt(n) / (A_true * p) + 0.01)

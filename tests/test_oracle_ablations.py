"""Pins of the oracle's two ablation modes, the schemes the paper replaces:

* the linear mix of LOD outputs (Sec. 3, "Temporal Coherence": the count of
  each grid is taken over its whole cell and the counts are blended with the
  LOD weights): the mean is still A p, but the variance falls short of the
  binomial A p (1 - p) - the incorrect statistics that Sec. 3 (item 1) and
  Sec. 4.2 attribute to it;
* the classical binomial approximation (Sec. 6.3): an explicit sum of
  Bernoulli trials where N p <= 5 (and N <= 16), which is exactly binomial,
  and a floored Gaussian of the binomial's mean and variance elsewhere."""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2306_05051_gb300.scenes import Material
from test_oracle_stats import eff_rho, pixel_row, square_J


def _weighted_nearest(orc, scene, n, weighted):
    """Per pixel: the sum over the 4 tetrahedron vertices of one realisation
    (the spatial and angular texel of largest weight), weighted by the
    vertex's LOD weight when `weighted` (linear mix)."""
    out = np.zeros(n)
    for px in range(n):
        pix, recs = orc.trace_pixel(scene, px)
        assert pix["status"] == 0
        tot = 0.0
        for vert in range(4):
            r = recs[(recs["vert"] == vert) & (recs["sub"] == 0)]
            k = np.argmax(r["u"] * 1000.0 + r["v"])
            best = r[(r["sv"] == r["sv"][k])]
            best = best[np.argmax(best["v"])]
            tot += (best["w"] if weighted else 1.0) * best["c"]
        out[px] = tot
    return out


def test_linear_mix_keeps_the_mean_and_loses_variance(orc):
    rng = np.random.default_rng(21)
    rho, p = 1e6, 0.5
    for A in (40.0, 600.0):                          # inside the brackets [16, 64] and [256, 1024]
        J = square_J(A / rho, ratio=3.0, angle=0.7)
        A_true = abs(np.linalg.det(J)) * eff_rho(rho)
        n = 1500
        uv = rng.uniform(0, 3, (n, 2))
        mix = pixel_row(uv, J, material=Material(R=p, ln_density=math.log(rho), n_lods=12, lod_blend=1))
        dist = pixel_row(uv, J, material=Material(R=p, ln_density=math.log(rho), n_lods=12))
        # trials: each vertex counts over its whole cell; the weights still sum the cells to A
        _, recs = orc.trace_pixel(mix, 0)
        tet = [recs[recs["vert"] == v][0] for v in range(4)]
        assert all(float(r["n"]).is_integer() for r in tet)
        assert sum(r["w"] * r["n"] for r in tet) == pytest.approx(A_true, rel=1e-12)
        cm = _weighted_nearest(orc, mix, n, True)
        cd = _weighted_nearest(orc, dist, n, False)
        var_bin = A_true * p * (1 - p)
        se = cm.std() / math.sqrt(n)
        assert abs(cm.mean() - A_true * p) <= 4 * se + 0.5
        assert cm.var() / var_bin <= 0.8, (cm.var(), var_bin)          # the deficit
        assert cd.var() / var_bin == pytest.approx(1.0, abs=0.15)      # the distributed law keeps it


def test_linear_mix_image_mean_is_the_distributed_mean(orc):
    """Both blends have mean count A p: the images agree on average."""
    rng = np.random.default_rng(22)
    rho = 1e6
    J = square_J(150.0 / rho, ratio=2.0, angle=0.3)
    uv = rng.uniform(0, 3, (3000, 2))
    a = orc.eval_image(pixel_row(uv, J, material=Material(R=0.3, ln_density=math.log(rho), n_lods=12, lod_blend=1)))
    b = orc.eval_image(pixel_row(uv, J, material=Material(R=0.3, ln_density=math.log(rho), n_lods=12)))
    se = math.hypot(a.std(), b.std()) / math.sqrt(a.size)
    assert abs(a.mean() - b.mean()) <= 4 * se + 1e-3 * b.mean()


def _classical_samples(orc, n, p, m, seed):
    rng = np.random.default_rng(seed)
    w = rng.integers(0, 2 ** 32, (m, 2), dtype=np.uint64)
    return np.array([orc.classical_count(n, p, int(a), int(b))[0] for a, b in w])


@pytest.mark.parametrize("n,p", [(1, 0.3), (4, 0.5), (10, 0.034), (16, 0.3)])
def test_classical_loop_is_binomial(orc, n, p):
    c = _classical_samples(orc, n, p, 40000, 7 + n)
    k = np.arange(n + 1)
    obs = np.bincount(c, minlength=n + 1)
    exp = stats.binom.pmf(k, n, p) * len(c)
    keep = exp >= 5
    obs_k = np.append(obs[keep], obs[~keep].sum())
    exp_k = np.append(exp[keep], exp[~keep].sum())
    if exp_k[-1] < 5:
        obs_k, exp_k = obs_k[:-1], exp_k[:-1]
        exp_k *= obs_k.sum() / exp_k.sum()
    assert stats.chisquare(obs_k, exp_k).pvalue > 1e-4


def test_classical_fractional_trials_and_branches(orc):
    # a fractional last trial keeps the mean N p
    c = _classical_samples(orc, 3.4, 0.5, 40000, 3)
    assert c.max() <= 4 and abs(c.mean() - 1.7) <= 4 * c.std() / math.sqrt(len(c))
    # the loop has no normal quantile (z = 0); the Gaussian branch does
    assert orc.classical_count(16, 0.3, 5, 9)[1] == 0.0
    assert orc.classical_count(17, 0.1, 5, 9)[1] != 0.0          # N > 16: Gaussian although N p <= 5
    assert orc.classical_count(12, 0.5, 5, 9)[1] != 0.0          # N p > 5
    # Gaussian branch: floor(N p + sqrt(N p (1 - p)) z(theta0)), clamped to [0, ceil N]
    for h0 in (0x00000100, 0x40000000, 0x80000000, 0xFFFFFF00):
        n, p = 200.0, 0.3
        th = ((h0 >> 8) + 0.5) * 2.0 ** -24
        want = math.floor(n * p + math.sqrt(n * p * (1 - p)) * stats.norm.ppf(th))
        assert orc.classical_count(n, p, h0, 0)[0] == min(max(want, 0), 200)
    # its moments: mean N p - 1/2 (the floor), variance N p (1 - p) + 1/12
    c = _classical_samples(orc, 400.0, 0.25, 20000, 5)
    assert abs(c.mean() - (100.0 - 0.5)) <= 4 * c.std() / math.sqrt(len(c))
    assert c.var() / (75.0 + 1 / 12) == pytest.approx(1.0, abs=0.05)


def test_classical_image_counts_use_the_classical_law(orc):
    """In an image, every evaluation of the classical mode follows the
    classical sampler of its trials and hash words."""
    rng = np.random.default_rng(4)
    J = square_J(30.0 / 1e6, ratio=2.0, angle=0.2)
    sc = pixel_row(rng.uniform(0, 3, (20, 2)), J, material=Material(R=0.2, ln_density=math.log(1e6), sampler=1))
    for px in range(20):
        _, recs = orc.trace_pixel(sc, px)
        for r in recs[::7]:
            assert int(r["c"]) == orc.classical_count(r["n"], r["p"], int(r["h0"]), int(r["h1"]))[0]
            assert int(r["gate"]) == 1


def test_random_number_table(orc):
    """Sec. 6.3, last paragraph: the uniforms fetched from a small precomputed
    table.  The table's words are uniform and the two words of an entry
    independent; an evaluation reads the entry indexed by the top 16 bits of
    the sum of its spatial and angular words; gates open at the law's rate."""
    words = np.array([orc.table_words(k) for k in range(0, 1 << 16, 7)], np.float64)
    th = (np.floor(words / 256.0) + 0.5) / 2 ** 24
    for c in (0, 1):
        assert stats.chisquare(np.histogram(th[:, c], bins=64, range=(0, 1))[0]).pvalue > 1e-4
    assert abs(np.corrcoef(th[:, 0], th[:, 1])[0, 1]) < 0.02
    seed = 0x9E3779B9
    rng = np.random.default_rng(8)
    opened = 0
    n = 20000
    for _ in range(n):
        i, j, ax, ay = (int(x) for x in rng.integers(-5000, 5000, 4))
        gid = orc.grid_id(int(rng.integers(0, 12)), int(rng.integers(0, 5)), int(rng.integers(0, 8)))
        s0 = int(orc.pcg4d([i & 0xFFFFFFFF, j & 0xFFFFFFFF, gid, seed])[0])
        a0 = int(orc.pcg3d([ax & 0xFFFFFFFF, ay & 0xFFFFFFFF, ~seed & 0xFFFFFFFF])[0])
        h = orc.eval_table(i, j, gid, ax, ay, seed)
        assert h == orc.table_words(((s0 + a0) & 0xFFFFFFFF) >> 16)
        opened += orc.theta(h[0]) < 0.1
    assert abs(opened / n - 0.1) <= 4 * math.sqrt(0.1 * 0.9 / n)


def test_table_mode_image_follows_the_hash_mode_on_average(orc):
    rng = np.random.default_rng(23)
    J = square_J(80.0 / 1e6, ratio=3.0, angle=0.9)
    uv = rng.uniform(0, 3, (3000, 2))
    a = orc.eval_image(pixel_row(uv, J, material=Material(R=0.2, ln_density=math.log(1e6), rng_table=1)))
    b = orc.eval_image(pixel_row(uv, J, material=Material(R=0.2, ln_density=math.log(1e6))))
    assert not np.array_equal(a, b)
    se = math.hypot(a.std(), b.std()) / math.sqrt(a.size)
    assert abs(a.mean() - b.mean()) <= 4 * se

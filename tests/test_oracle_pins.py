"""More pins of the FP64 oracle against things other than itself:

* the MurmurHash3 finaliser against the hash's published known answers;
* the evaluation counts and the default R that the paper prints;
* Schlick's Fresnel term at its fixed points, its exponent, and its
  distance to the exact dielectric Fresnel equations;
* the high-density limit against an independently written smooth
  microfacet BRDF (NDF written out, Smith masking by quadrature);
* the gated sampler's distribution against its definition and against the
  binomial law over a table of (N, p) (Sec. 6.3);
* the exact sampler and the additivity of the distributed binomial
  (Sec. 4.2): the four tetrahedron vertices' laws convolve to Bin(A, p)."""
import math
import os

import numpy as np
import pytest
import torch
from scipy import stats

from paper_2306_05051_gb300.scenes import Light, Material, Scene

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# --------------------------------------------------------------------------
# hash: MurmurHash3 known answers
# --------------------------------------------------------------------------
def _murmur3_x86_32(orc, data: bytes, seed: int) -> int:
    """MurmurHash3_x86_32 (Appleby) with the oracle's fmix32 as finaliser."""
    M = 0xFFFFFFFF
    c1, c2 = 0xCC9E2D51, 0x1B873593

    def rotl(x, r):
        return ((x << r) | (x >> (32 - r))) & M

    def mix_k(k):
        return (rotl((k * c1) & M, 15) * c2) & M

    h = seed
    nb = len(data) // 4
    for i in range(nb):
        h ^= mix_k(int.from_bytes(data[4 * i:4 * i + 4], "little"))
        h = (rotl(h, 13) * 5 + 0xE6546B64) & M
    tail = data[4 * nb:]
    if tail:
        k = 0
        for b, byte in enumerate(tail):
            k |= byte << (8 * b)
        h ^= mix_k(k)
    return orc.fmix32(h ^ len(data))


def test_fmix32_reproduces_murmurhash3_known_answers(orc):
    rows = []
    with open(os.path.join(GOLDEN, "murmur3_known_answers.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                data, seed, want = line.split()
                rows.append((b"" if data == "-" else bytes.fromhex(data), int(seed, 16), int(want, 16)))
    assert len(rows) >= 12
    for data, seed, want in rows:
        assert _murmur3_x86_32(orc, data, seed) == want, (data, hex(seed))
    # the empty input is the finaliser alone
    assert orc.fmix32(1) == 0x514E28B7 and orc.fmix32(0) == 0


# --------------------------------------------------------------------------
# the paper's printed counts and constants
# --------------------------------------------------------------------------
def _paper_constants():
    out = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def _patch(view, light, uv, J, material):
    """A 1 x N G-buffer of a flat patch (normal +z, tangent +x) with the given
    view direction, one directional light, uv and footprint Jacobian
    J = [[du/dx, du/dy], [dv/dx, dv/dy]]."""
    uv = np.asarray(uv, np.float64)
    N = len(uv)
    g = np.zeros((1, N, 16), np.float32)
    g[0, :, 0:2] = uv
    g[0, :, 2] = J[0][0]; g[0, :, 3] = J[1][0]
    g[0, :, 4] = J[0][1]; g[0, :, 5] = J[1][1]
    g[0, :, 8] = 1.0
    g[0, :, 9] = 1.0
    g[0, :, 12:15] = view
    return Scene("patch", torch.from_numpy(g), None, None, material, [Light(kind=1, dir=tuple(light), intensity=1.0)])


def _unit(theta_deg, phi_deg):
    t, p = math.radians(theta_deg), math.radians(phi_deg)
    return (math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t))


def test_paper_evaluation_counts_and_R(orc):
    """Sec. 6: 2 x 5 grids x 4 spatial x 4 angular = 160 naive evaluations;
    Sec. 6.1: 4 tetrahedron vertices x 4 x 4 = 64; Sec. 6.2: 4 x 3 x 4 = 48
    with the simplex grid; Sec. 7: R = 0.034.  The factors are read off the
    oracle (its cell, tetrahedra and traces), not typed in."""
    pc = _paper_constants()
    # grids of one ratio/orientation cell: the union of its triangles' vertices
    m, tri, _, x, t, lam = orc.cell(2.42, math.radians(53.25), 4)
    pent = set()
    for tt in (0.05 * x, 0.5, 1 - 0.05 * x):                 # a point in each of the 3 triangles
        _, _, verts, _, _, _ = orc.cell(2.42, (math.floor(math.radians(53.25) / (math.pi / 8)) + tt) * math.pi / 8, 4)
        pent |= set(verts)
    assert len(pent) == 5
    _, tv, w = orc.tet(lam, 0.3)
    n_tet = len(tv)
    # a traced pixel: 48 records per light, 3 lattice and 4 angular texels per grid
    mat = Material(n_lods=8)
    sc = _patch(_unit(20, 10), _unit(35, 200), [(3.3, 7.1)], [[0.004, 0.001], [-0.002, 0.006]], mat)
    pix, recs = orc.trace_pixel(sc, 0)
    per_grid = [recs[(recs["sub"] == 0) & (recs["vert"] == i)] for i in range(4)]
    n_spatial = len({(int(r["i"]), int(r["j"])) for r in per_grid[0]})
    n_angular = len({(int(r["ax"]), int(r["ay"])) for r in per_grid[0]})
    assert (n_spatial, n_angular) == (3, 4)
    assert len(recs) == int(pix["K"]) * n_tet * n_spatial * n_angular
    assert n_tet * n_spatial * n_angular == pc["evals_simplex"] == 48
    assert n_tet * 4 * n_angular == pc["evals_tetrahedra"] == 64            # square grid: 4 bilinear texels
    assert 2 * len(pent) * 4 * n_angular == pc["evals_naive"] == 160        # 2 LODs x pentagon, no tetrahedra
    assert Material().R == pc["R_default"]


# --------------------------------------------------------------------------
# Schlick Fresnel (Eq. 2's F)
# --------------------------------------------------------------------------
def _fresnel_ratio(orc, theta_deg, F0):
    """out(F0) / out(F0 = 1) on a patch whose half-vector is the normal
    (view and light mirrored about it), so v.h = cos(theta): the Fresnel
    factor alone (counts, D and G are the same in both)."""
    v = _unit(theta_deg, 0.0)
    l = (-v[0], -v[1], v[2])
    rng = np.random.default_rng(1)
    uv = rng.uniform(0, 4, (64, 2))
    J = [[3e-3, 0.0], [0.0, 3e-3]]
    a = orc.eval_image(_patch(v, l, uv, J, Material(F0=F0, ln_density=math.log(1e7))))[0]
    b = orc.eval_image(_patch(v, l, uv, J, Material(F0=1.0, ln_density=math.log(1e7))))[0]
    assert (b > 0).sum() > 30
    r = a[b > 0] / b[b > 0]
    assert r.max() - r.min() <= 1e-12 * r.max()
    v32 = np.asarray(v, np.float32).astype(np.float64)
    return float(r.mean()), float(v32[2] / np.linalg.norm(v32))     # the factor and v.h as the oracle sees it


def _fresnel_dielectric(cos_i, eta):
    """Exact Fresnel reflectance of unpolarised light, air to a dielectric of
    index eta (the textbook s and p amplitudes)."""
    sin_t = math.sqrt(max(0.0, 1 - cos_i ** 2)) / eta
    cos_t = math.sqrt(1 - sin_t ** 2)
    rs = (cos_i - eta * cos_t) / (cos_i + eta * cos_t)
    rp = (eta * cos_i - cos_t) / (eta * cos_i + cos_t)
    return 0.5 * (rs * rs + rp * rp)


def test_schlick_fresnel_fixed_points_and_exponent(orc):
    # F(v.h = 1) = F0 (F0 crosses the interface as float32)
    for F0 in (0.04, 0.5):
        assert _fresnel_ratio(orc, 0.0, F0)[0] == pytest.approx(float(np.float32(F0)), rel=1e-12)
    # F -> 1 at grazing incidence
    assert _fresnel_ratio(orc, 89.5, 0.04)[0] > 0.95
    # with F0 = 0 the factor is (1 - v.h)^5: Schlick's exponent
    for th in (30.0, 55.0, 75.0):
        r, c = _fresnel_ratio(orc, th, 0.0)
        assert math.log(r) / math.log(1 - c) == pytest.approx(5.0, rel=1e-9)
    # and it stays close to the exact reflectance of glass (eta = 1.5, F0 = 0.04)
    for th in (0.0, 20.0, 40.0, 60.0, 75.0):
        r, c = _fresnel_ratio(orc, th, 0.04)
        assert abs(r - _fresnel_dielectric(c, 1.5)) <= 0.025, th


# --------------------------------------------------------------------------
# high-density limit: the smooth microfacet BRDF (Sec. 3, Eq. 1-4)
# --------------------------------------------------------------------------
def _slope_pdf_kind(kind):
    # isotropic slope profile g(r^2) of the stretched slope distribution
    return (lambda u: np.exp(-u)) if kind == 0 else (lambda u: 1.0 / (1.0 + u) ** 2)


def _ndf_smooth(kind, ax, ay, h):
    """Walter et al. 2007 anisotropic Beckmann / GGX written from the slope
    distribution: D(m) = P22(slope(m)) / cos^4(theta_m)."""
    h = np.asarray(h) / np.linalg.norm(h)
    sx, sy = -h[0] / h[2], -h[1] / h[2]
    u = (sx / ax) ** 2 + (sy / ay) ** 2
    return _slope_pdf_kind(kind)(u) / (math.pi * ax * ay) / h[2] ** 4


def _masking_G1(kind, ax, ay, w):
    """Smith G1(w) = cos(w) / integral of <w.m>+ D(m) dm, the integral taken
    by quadrature over the stretched slope plane in polar form."""
    n_r, n_phi = 4000, 720
    phi = (np.arange(n_phi) + 0.5) * (2 * math.pi / n_phi)
    if kind == 0:
        rho = (np.arange(n_r) + 0.5) * (9.0 / n_r)
        wr = 9.0 / n_r * rho * np.exp(-rho ** 2)                     # rho drho g(rho^2)
    else:
        t = (np.arange(n_r) + 0.5) * (math.pi / 2 / n_r)
        rho = np.tan(t)
        wr = (math.pi / 2 / n_r) * np.sin(t) * np.cos(t)             # rho drho / (1 + rho^2)^2
    R, PH = np.meshgrid(rho, phi, indexing="ij")
    x, y = ax * R * np.cos(PH), ay * R * np.sin(PH)
    proj = np.maximum(0.0, w[2] - w[0] * x - w[1] * y)               # <w.m> / <m.n> for slope (x, y)
    total = (proj * wr[:, None]).sum() * (2 * math.pi / n_phi) / math.pi
    return w[2] / total


@pytest.mark.parametrize("kind", [0, 1])
def test_dense_limit_is_the_smooth_microfacet_brdf(orc, kind):
    ax, ay = 0.3, 0.2
    v, l = np.array(_unit(25, 10)), np.array(_unit(40, 160))
    h = (v + l) / np.linalg.norm(v + l)
    rho = 1e12
    mat = Material(ndf=kind, alpha_x=ax, alpha_y=ay, F0=1.0, ln_density=math.log(rho), n_lods=16)
    rng = np.random.default_rng(3 + kind)
    uv = rng.uniform(0, 2, (256, 2))
    J = [[3e-2, 4e-3], [-5e-3, 3.2e-2]]
    out = orc.eval_image(_patch(tuple(v), tuple(l), uv, J, mat))[0]
    smooth = (_masking_G1(kind, ax, ay, v) * _masking_G1(kind, ax, ay, l) * _ndf_smooth(kind, ax, ay, h)
              / (4 * v[2] * l[2]) * l[2])
    A = abs(J[0][0] * J[1][1] - J[0][1] * J[1][0]) * math.exp(float(np.float32(math.log(rho))))
    p = 0.034 * _ndf_smooth(kind, ax, ay, h) * math.pi * ax * ay
    assert A * p > 5e6
    assert out.mean() == pytest.approx(smooth, rel=2e-4 + 4 * out.std() / math.sqrt(len(out)) / smooth)


# --------------------------------------------------------------------------
# gated sampler (Sec. 6.3) against its definition and the binomial law
# --------------------------------------------------------------------------
def _gated_pmf_definition(n, p):
    """PMF of clamp(floor(gate (1 + N(mu, sigma^2))), 1, ceil n) for an open
    gate, 0 for a closed one: P>=1 = 1 - (1 - p)^n, mu = max(n - 1, 0) p,
    sigma^2 = mu (1 - p), written from Sec. 6.3 with scipy's normal CDF."""
    P1 = 1.0 if p >= 1 else -math.expm1(n * math.log1p(-p))
    mu = max(n - 1.0, 0.0) * p
    sig = math.sqrt(mu * (1 - p))
    top = math.ceil(n)
    if sig == 0.0:
        pmf = np.zeros(top + 1)
        pmf[min(max(math.floor(1 + mu), 1), top)] = P1
    else:
        lo = max(1, int(math.floor(1 + mu - 12 * sig)))
        hi = min(top, int(math.ceil(1 + mu + 12 * sig)))
        k = np.arange(lo, hi + 1)
        cdf_lo = stats.norm.cdf((k - 1 - mu) / sig)               # P(1 + mu + sigma z < k)
        cdf_hi = stats.norm.cdf((k - mu) / sig)
        q = cdf_hi - cdf_lo
        q[0] = cdf_hi[0]                                          # clamp mass at the bottom
        q[-1] = 1.0 - cdf_lo[-1]                                  # and at ceil n
        pmf = np.zeros(top + 1)
        pmf[lo:hi + 1] = P1 * q
    pmf[0] += 1.0 - P1
    return pmf


def _sampler_moments(orc, n, p, ngrid=2048):
    th1 = (np.arange(ngrid) + 0.5) / ngrid
    P1 = orc.gated_count(n, p, 0.0, 0.5)[1]
    c = np.array([orc.gated_count(n, p, 0.0, t)[0] for t in th1], np.float64)
    return P1 * c.mean(), P1 * (c * c).mean() - (P1 * c.mean()) ** 2, P1


N_GRID = [0.1, 0.5, 1.0, 3.0, 10.0, 30.0, 100.0, 1e3, 1e4, 1e5, 1e6]
P_GRID = [1e-4, 1e-3, 1e-2, 0.034, 0.1, 0.3, 0.7, 1.0]


def test_gated_sampler_table(orc):
    """Over n in [0.1, 1e6] and p in [1e-4, 1]: the oracle's sampler follows
    the PMF written from the definition (moments within the quadrature
    error), and for n >= 1 that PMF follows the binomial law to the
    acceptance of the reading: mean within 0.5/(np) + 2 %, variance within
    15 % where np >= 1 (20 % below 10 trials).  The total variation distance
    to Bin(n, p) is tabulated (integer n)."""
    rows = []
    for n in N_GRID:
        for p in P_GRID:
            pmf = _gated_pmf_definition(n, p)
            k = np.arange(len(pmf))
            mean = float((k * pmf).sum())
            var = float((k * k * pmf).sum() - mean ** 2)
            om, ov, P1 = _sampler_moments(orc, n, p)
            assert P1 == pytest.approx(1.0 if p >= 1 else -math.expm1(n * math.log1p(-p)), rel=1e-12)
            assert om == pytest.approx(mean, rel=2e-3, abs=1e-9), (n, p)
            if var > 1e-6:
                assert ov == pytest.approx(var, rel=0.05, abs=1e-9), (n, p)
            bm, bv = n * p, n * p * (1 - p)
            if n < 1:
                # below one trial the law is Bernoulli(P>=1) (N - 1 clamped at 0);
                # no binomial to compare with
                assert mean == pytest.approx(P1, rel=1e-12) and (pmf[0], pmf[1]) == pytest.approx((1 - P1, P1))
                rows.append((n, p, mean / bm - 1, 0.0, None))
                continue
            assert abs(mean - bm) / bm <= 0.5 / (n * p) + 0.02, (n, p, mean, bm)
            if n * p >= 1 and bv > 0:
                # 15 %, except below 10 trials: the floor of a Gaussian of
                # sigma < 1 under-disperses (n = 3, p = 0.7: -17 %)
                assert abs(var - bv) / bv <= (0.15 if n >= 10 else 0.2), (n, p, var, bv)
            tv = None
            if float(n).is_integer():
                ref = stats.binom.pmf(k, int(n), p)
                tv = 0.5 * float(np.abs(pmf - ref).sum() + max(0.0, 1.0 - ref.sum()))
            rows.append((n, p, mean / bm - 1, (var / bv - 1) if bv > 0 else 0.0, tv))
    print("\n   n        p      mean err   var err    TV")
    for n, p, me, ve, tv in rows:
        print(f"{n:8.3g} {p:8.3g} {me:+9.2e} {ve:+9.2e} " + ("  -" if tv is None else f"{tv:8.2e}"))


def _exact_pmf(orc, N, p):
    """PMF of the oracle's exact sampler, from the positions in theta where
    its (non-decreasing) count steps, found by bisection."""
    edges = [0.0]
    for k in range(N):
        lo, hi = 0.0, 1.0
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if orc.exact_count(N, p, mid) <= k:
                lo = mid
            else:
                hi = mid
        edges.append(lo)
    edges.append(1.0)
    return np.diff(np.array(edges))


def test_exact_sampler_is_binomial_and_distributed_laws_add_up(orc):
    """Sec. 4.2 (distributed binomial, additivity): for a tetrahedron whose
    four vertices carry integer trials, the exact sampler's four laws
    convolve to Bin(A, p) for the footprint's A = sum of the trials."""
    p = 0.3
    for N in (1, 4, 16, 28):
        assert np.abs(_exact_pmf(orc, N, p) - stats.binom.pmf(np.arange(N + 1), N, p)).max() <= 1e-12
    # level 2 of f = 4 (16 and 64 flakes per cell), cell weights (1/2, 1/4, 1/4), s = 1/4
    level, f = 2, 4
    lam = np.array([0.5, 0.25, 0.25])
    s = 0.25
    A = f ** level + s * (f ** (level + 1) - f ** level)
    _, verts, w = orc.tet(lam, s)
    trials = [wi * f ** (level + up) for (up, _), wi in zip(verts, w)]
    assert all(float(t).is_integer() for t in trials) and sum(trials) == A == 28
    conv = np.array([1.0])
    for t in trials:
        conv = np.convolve(conv, _exact_pmf(orc, int(t), p))
    assert np.abs(conv - stats.binom.pmf(np.arange(int(A) + 1), int(A), p)).max() <= 1e-12
    # the gated laws of the same vertices stay within the table's tolerance
    gconv = np.array([1.0])
    for t in trials:
        gconv = np.convolve(gconv, _gated_pmf_definition(t, p))
    k = np.arange(len(gconv))
    gm = (k * gconv).sum()
    gv = (k * k * gconv).sum() - gm ** 2
    assert abs(gm / (A * p) - 1) <= 0.02 and abs(gv / (A * p * (1 - p)) - 1) <= 0.15

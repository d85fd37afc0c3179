"""Pins of the oracle's individual steps against things other than itself:
library routines (numpy SVD, scipy ndtri / binom), numerical integration of
the NDF and of the Smith masking definition, the paper's Fig. 5 / Fig. 6
discretisation, brute-force minimality, and the defining identities of each
weight scheme (partition of unity, linear precision, continuity)."""
import math
import os

import numpy as np
import pytest
from scipy import special, stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Phi^-1 (used by the gated sampler, Sec. 6.3)
# --------------------------------------------------------------------------
def test_phi_inv_matches_scipy_ndtri(orc):
    rng = np.random.default_rng(0)
    Ps = np.concatenate([
        (np.arange(0, 1 << 24, 4099) + 0.5) * 2.0 ** -24,          # the sampler's own grid
        10.0 ** -rng.uniform(0, 15, 500), 1 - 10.0 ** -rng.uniform(1, 15, 500),
        [0.5, 2.0 ** -25, 1 - 2.0 ** -25]])
    for P in Ps:
        z = orc.phi_inv(P)
        ref = special.ndtri(P)
        assert abs(z - ref) <= 1e-12 * (1 + abs(ref)), (P, z, ref)


# --------------------------------------------------------------------------
# footprint (Sec. 5.1): SVD of J
# --------------------------------------------------------------------------
def test_footprint_matches_numpy_svd(orc):
    rng = np.random.default_rng(1)
    for _ in range(2000):
        J = rng.normal(size=(2, 2)) * 10.0 ** rng.uniform(-6, 1)
        J[:, 1] *= 10.0 ** rng.uniform(-3, 0)
        J = J.astype(np.float32).astype(np.float64)
        s0, s1, phi, P, r = orc.footprint(J[0, 0], J[0, 1], J[1, 0], J[1, 1])
        U, S, Vt = np.linalg.svd(J)
        assert s0 == pytest.approx(S[0], rel=1e-12)
        assert s1 == pytest.approx(S[1], rel=1e-9)
        assert P == pytest.approx(abs(np.linalg.det(J)), rel=1e-12)
        assert r == pytest.approx(S[0] / S[1], rel=1e-9)
        assert 0.0 <= phi < math.pi
        u0 = U[:, 0]
        if S[0] > S[1] * (1 + 1e-6):
            # phi is the orientation of the major axis u0 (modulo pi)
            assert abs(math.cos(phi) * u0[1] - math.sin(phi) * u0[0]) < 1e-7


def test_footprint_axis_aligned_special_cases(orc):
    s0, s1, phi, P, r = orc.footprint(3.0, 0.0, 0.0, 0.5)
    assert (s0, s1, phi, P, r) == pytest.approx((3.0, 0.5, 0.0, 1.5, 6.0))
    s0, s1, phi, P, r = orc.footprint(0.5, 0.0, 0.0, 3.0)
    assert (s0, s1, phi, P, r) == pytest.approx((3.0, 0.5, math.pi / 2, 1.5, 6.0))


# --------------------------------------------------------------------------
# NDF (Eq. 2-4 use a standard NDF): normalisation by quadrature
# --------------------------------------------------------------------------
def _slope_grid(n_psi=320, n_phi=160):
    """Quadrature over the slope plane (a, b) = slopes / alpha in polar form
    (rho = tan psi), Gauss-Legendre in psi and uniform in the angle."""
    x, w = np.polynomial.legendre.leggauss(n_psi)
    psi = (x + 1) * math.pi / 4
    wpsi = w * math.pi / 4
    ang = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi
    wang = 2 * math.pi / n_phi
    rho = np.tan(psi)
    jac = rho / np.cos(psi) ** 2
    return rho, wpsi * jac, ang, wang


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("ax,ay", [(0.3, 0.3), (0.2, 0.05), (0.05, 0.5), (0.6, 0.25)])
def test_ndf_projected_area_is_one(orc, kind, ax, ay):
    """int D(h) <h.n> dw_h = 1 (a normalised microfacet NDF)."""
    rho, wr, ang, wa = _slope_grid()
    total = 0.0
    for r, wrr in zip(rho, wr):
        for a in ang:
            sx, sy = ax * r * math.cos(a), ay * r * math.sin(a)
            h = np.array([-sx, -sy, 1.0]); h /= np.linalg.norm(h)
            # d(omega) <h.n> = cos^4(theta) d(slope); d(slope) = ax ay d(a, b)
            total += orc.ndf(kind, ax, ay, h[0], h[1], h[2]) * h[2] ** 4 * ax * ay * wrr * wa
    assert total == pytest.approx(1.0, abs=2e-5 if kind == 1 else 1e-9)


@pytest.mark.parametrize("kind", [0, 1])
def test_ndf_at_normal(orc, kind):
    for ax, ay in [(0.3, 0.3), (0.2, 0.05)]:
        assert orc.ndf(kind, ax, ay, 0.0, 0.0, 1.0) == pytest.approx(1.0 / (math.pi * ax * ay), rel=1e-14)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("ax,ay", [(0.3, 0.3), (0.2, 0.05)])
@pytest.mark.parametrize("theta_deg,phi_deg", [(20, 0), (60, 35), (80, 120)])
def test_smith_lambda_matches_masking_integral(orc, kind, ax, ay, theta_deg, phi_deg):
    """Definition of Lambda: int max(0, w.h) D(h) dw_h = <w.n> (1 + Lambda(w))."""
    th, ph = math.radians(theta_deg), math.radians(phi_deg)
    w = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    rho, wr, ang, wa = _slope_grid(480, 240)
    total = 0.0
    for r, wrr in zip(rho, wr):
        for a in ang:
            sx, sy = ax * r * math.cos(a), ay * r * math.sin(a)
            h = np.array([-sx, -sy, 1.0]); h /= np.linalg.norm(h)
            wh = max(0.0, float(w @ h))
            total += wh * orc.ndf(kind, ax, ay, h[0], h[1], h[2]) * h[2] ** 3 * ax * ay * wrr * wa
    lam = orc.smith_lambda(kind, ax, ay, w[0], w[1], w[2])
    assert total / w[2] - 1.0 == pytest.approx(lam, abs=2e-3 if kind == 1 else 5e-4)


# --------------------------------------------------------------------------
# hash (parity unpinned against the paper): statistics only
# --------------------------------------------------------------------------
def test_hash_words_uniform_and_independent(orc):
    th0, th1, nb = [], [], []
    gid = orc.grid_id(3, 2, 5)
    for i in range(-64, 64):
        for j in range(-32, 32):
            for ax in (-1, 0, 1, 2):
                h0, h1 = orc.eval_hash(i, j, gid, ax, 7, 0x9E3779B9)
                th0.append(orc.theta(h0)); th1.append(orc.theta(h1))
    th0, th1 = np.array(th0), np.array(th1)
    for th in (th0, th1):
        assert 0 < th.min() and th.max() < 1
        counts = np.histogram(th, bins=64, range=(0, 1))[0]
        assert stats.chisquare(counts).pvalue > 1e-4
    joint = np.histogram2d(th0, th1, bins=16, range=[[0, 1], [0, 1]])[0].ravel()
    assert stats.chisquare(joint).pvalue > 1e-4
    assert abs(np.corrcoef(th0, th1)[0, 1]) < 0.02
    # neighbouring keys (ax, ax+1) are uncorrelated
    a = th0.reshape(-1, 4)
    assert abs(np.corrcoef(a[:, 0], a[:, 1])[0, 1]) < 0.03


def test_hash_depends_on_every_key_field(orc):
    base = (5, -9, orc.grid_id(2, 1, 3), 4, -2, 12345)
    h = orc.eval_hash(*base)
    for k in range(6):
        key = list(base)
        key[k] = key[k] + 1
        assert orc.eval_hash(*key) != h
    # theta mapping uses the top 24 bits, centred
    assert orc.theta(0) == 0.5 * 2.0 ** -24
    assert orc.theta(0xFFFFFFFF) == 1 - 0.5 * 2.0 ** -24


# --------------------------------------------------------------------------
# sub-footprint split (library extension of Sec. 4.2)
# --------------------------------------------------------------------------
def test_split_is_the_smallest_admissible(orc):
    rng = np.random.default_rng(2)
    for _ in range(3000):
        M, L, f = int(rng.integers(1, 6)), int(rng.integers(2, 13)), int(rng.choice([2, 4]))
        r = 10.0 ** rng.uniform(0, 3)
        A = 10.0 ** rng.uniform(-2, 1.2 * L * math.log10(f))
        Kmaj, k, K = orc.split(r, A, M, L, f, 64)
        top = float(f) ** (L - 1)
        assert K == Kmaj * k * k and 1 <= K <= 64
        # brute force: smallest Kmaj with r / Kmaj <= 2^M, capped at 64
        want_maj = next(q for q in range(1, 10 ** 6) if r / q <= 2.0 ** M or q >= 64)
        assert Kmaj == min(want_maj, 64)
        # smallest k with k^2 top >= A / Kmaj, capped by Kmaj k^2 <= 64
        kk = 1
        while kk * kk * top < A / Kmaj and Kmaj * (kk + 1) ** 2 <= 64:
            kk += 1
        assert k == kk


# --------------------------------------------------------------------------
# LOD bracket (Sec. 5.2, Eq. 13 with area factor f; Sec. 4.2 weights)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("f", [2, 4])
def test_lod_bracket_is_area_linear(orc, f):
    rng = np.random.default_rng(3)
    L = 8
    for As in 10.0 ** rng.uniform(-3, 7, 3000):
        level, s, pinned = orc.lod(As, f, L)
        top = float(f) ** (L - 1)
        if As < 1:
            assert (level, s, pinned) == (0, 0.0, True)
        elif As >= top:
            assert (level, s, pinned) == (L - 2, 1.0, True)
        else:
            lo, hi = float(f) ** level, float(f) ** (level + 1)
            assert lo <= As < hi and 0.0 <= s < 1.0 and not pinned
            # P = w_hi P_hi + w_lo P_lo with w_hi = (P - P_lo)/(P_hi - P_lo) (Sec. 4.2)
            assert (1 - s) * lo + s * hi == pytest.approx(As, rel=1e-14)


# --------------------------------------------------------------------------
# ratio / orientation lattice: the paper's Fig. 5 and Fig. 6
# --------------------------------------------------------------------------
def _golden_grids():
    rows = {}
    with open(os.path.join(GOLDEN, "fig5_fig6_grids.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, *rest = line.split()
                rows.setdefault(k, []).append(rest)
    return rows


def _deg(ring, kor):
    return 0.0 if ring == 0 else kor * 180.0 / 2 ** (ring + 1)


def test_orientations_per_ring_match_fig5(orc):
    g = _golden_grids()
    first = {int(r[0]): [float(x) for x in r[1:]] for r in g["first_ring"]}
    for ring in (1, 2, 3):
        want = {0.0, 90.0}
        for m, angs in first.items():
            if m <= ring:
                want |= set(angs)
        # every grid vertex that appears on `ring` within the drawn quarter plane
        seen = set()
        for rho_r in np.linspace(max(ring - 1, 0), min(ring + 1, 4), 41):
            for phi in np.linspace(0, math.pi / 2, 721):
                _, _, verts, _, _, lam = orc.cell(rho_r, phi, 4)
                for (rg, k), l in zip(verts, lam):
                    if rg == ring and l > 0:
                        a = _deg(rg, k)
                        if a <= 90.0:
                            seen.add(a)
        assert seen == want, (ring, sorted(seen), sorted(want))


def test_fig5_point_distributes_over_the_drawn_pentagon(orc):
    g = _golden_grids()
    rr, deg = (float(x) for x in g["point"][0])
    pent = {(int(s.split(":")[0]), float(s.split(":")[1])) for s in g["pentagon"][0]}
    tris = [{(int(s.split(":")[0]), float(s.split(":")[1])) for s in t} for t in g["triangle"]]
    m, tri, verts, x, t, lam = orc.cell(rr, math.radians(deg), 4)
    got = {(rg, _deg(rg, k)) for rg, k in verts}
    assert got <= pent and got in [t for t in tris]
    # sweeping the whole cell yields exactly the drawn pentagon and triangles
    seen_tris, seen = [], set()
    for xx in np.linspace(0.0, 0.999, 60):
        for tt in np.linspace(0.0, 0.999, 60):
            phi = math.radians(45.0 + 22.5 * tt)
            _, _, vv, _, _, _ = orc.cell(2.0 + xx, phi, 4)
            s = {(rg, _deg(rg, k)) for rg, k in vv}
            seen |= s
            if s not in seen_tris:
                seen_tris.append(s)
    assert seen == pent
    assert sorted(map(sorted, seen_tris)) == sorted(map(sorted, tris))


def test_cell_barycentrics(orc):
    rng = np.random.default_rng(4)
    for _ in range(5000):
        M = int(rng.integers(1, 6))
        rho_r = rng.uniform(-0.5, M + 0.5)
        phi = rng.uniform(0, math.pi)
        m, tri, verts, x, t, lam = orc.cell(rho_r, phi, M)
        assert lam.min() >= -1e-15 and lam.sum() == pytest.approx(1.0, abs=1e-14)
        # linear precision in the (x, t) parameter plane (inner cell: in (x, x t))
        if m == 0:
            pts = [(0.0, 0.0), (1.0, 0.0), (1.0, 1.0)]
            target = (x, x * t)
        else:
            table = {(m, 0): None}
            pts = []
            nm = 2 ** (m + 1)
            a = int(math.floor(phi / (math.pi / nm))) % nm
            for rg, k in verts:
                if rg == m:
                    pts.append((0.0, 0.0 if k == a else 1.0))
                else:
                    pts.append((1.0, ((k - 2 * a) % (2 * nm)) / 2.0))
            target = (x, t)
        rec = np.array(pts).T @ lam
        assert rec == pytest.approx(target, abs=1e-12)


def _vertex_weights(orc, rho_r, phi, s, M=4):
    """Weight of every grid vertex (upper, ring, kor) for a point of the
    (ratio, orientation, scale) lattice: cell triangle, then tetrahedron."""
    _, _, verts, _, _, lam = orc.cell(rho_r, phi, M)
    _, tv, w = orc.tet(lam, s)
    out = {}
    for (up, j), ww in zip(tv, w):
        key = (up,) + tuple(verts[j])
        if verts[j][0] == 0:
            key = (up, 0, 0)
        out[key] = out.get(key, 0.0) + ww
    return out


def test_tetrahedra_partition_precision_and_continuity(orc):
    rng = np.random.default_rng(5)
    for _ in range(3000):
        lam = rng.dirichlet([1, 1, 1])
        s = rng.uniform()
        k, tv, w = orc.tet(lam, s)
        assert w.min() >= -1e-15 and w.sum() == pytest.approx(1.0, abs=1e-14)
        # linear precision: upper weight = s; per triangle vertex total = lam
        assert sum(ww for (up, _), ww in zip(tv, w) if up) == pytest.approx(s, abs=1e-14)
        per = np.zeros(3)
        for (_, j), ww in zip(tv, w):
            per[j] += ww
        assert per == pytest.approx(lam, abs=1e-14)
    # continuity along random lines through the full 3-D lattice
    for _ in range(30):
        p0 = np.array([rng.uniform(0, 4), rng.uniform(0, math.pi), rng.uniform(0, 1)])
        d = rng.normal(size=3); d /= np.linalg.norm(d)
        step = 2e-5
        prev = None
        for k in range(4000):
            p = p0 + (k * step) * d
            rr, ph, s = min(max(p[0], 0), 4), p[1] % math.pi, min(max(p[2], 0), 1)
            cur = _vertex_weights(orc, rr, ph, s)
            if prev is not None:
                keys = set(cur) | set(prev)
                jump = max(abs(cur.get(kk, 0.0) - prev.get(kk, 0.0)) for kk in keys)
                assert jump <= 8 * step * 16, (p, jump)
            prev = cur


def test_tetrahedra_per_pixel_count(orc):
    """Sec. 6.1: 4 tetrahedron vertices per pixel (not the 10 pentagon-prism
    vertices), and the distributed trials sum to the footprint's flakes."""
    rng = np.random.default_rng(6)
    for _ in range(500):
        As = 10.0 ** rng.uniform(-1, 6)
        level, s, pinned = orc.lod(As, 4, 12)
        _, _, verts, _, _, lam = orc.cell(rng.uniform(0, 4), rng.uniform(0, math.pi), 4)
        _, tv, w = orc.tet(lam, s)
        assert len(tv) == 4
        n = [ww * (As if pinned else 4.0 ** (level + up)) for (up, _), ww in zip(tv, w)]
        assert sum(n) == pytest.approx(As, rel=1e-12)


# --------------------------------------------------------------------------
# anisotropic grid transform (Eq. 12) and simplex lattice (Sec. 6.2)
# --------------------------------------------------------------------------
def test_grid_transform_area_ratio_orientation(orc):
    rng = np.random.default_rng(7)
    for _ in range(300):
        level, ring = int(rng.integers(0, 10)), int(rng.integers(0, 5))
        kor = 0 if ring == 0 else int(rng.integers(0, 2 ** (ring + 1)))
        rho = 10.0 ** rng.uniform(3, 9)
        f = int(rng.choice([2, 4]))
        q0 = np.array(orc.grid_coords(0.0, 0.0, level, ring, kor, rho, f))
        qu = np.array(orc.grid_coords(1e-3, 0.0, level, ring, kor, rho, f))
        qv = np.array(orc.grid_coords(0.0, 1e-3, level, ring, kor, rho, f))
        Jq = np.stack([qu - q0, qv - q0], 1) / 1e-3
        # one lattice vertex per cell: vertex density rho / f^level per uv^2
        assert abs(np.linalg.det(Jq)) == pytest.approx(rho / float(f) ** level, rel=1e-9)
        # unskew to the equilateral frame: q = S g_hat, S = I + F2 [[1,1],[1,1]]
        F2 = (math.sqrt(3) - 1) / 2
        S = np.eye(2) + F2
        Jg = np.linalg.solve(S, Jq)
        U, sv, Vt = np.linalg.svd(Jg)
        assert sv[0] / sv[1] == pytest.approx(2.0 ** ring, rel=1e-9)
        # the cell's long side (least-stretched uv direction) points along phi_k
        phik = 0.0 if ring == 0 else kor * math.pi / 2 ** (ring + 1)
        if ring > 0:
            long_dir = Vt[1]
            assert abs(long_dir[0] * math.sin(phik) - long_dir[1] * math.cos(phik)) < 1e-9


def test_simplex_vertices(orc):
    rng = np.random.default_rng(8)
    G2 = (3 - math.sqrt(3)) / 6
    unskew = lambda i, j: np.array([i - G2 * (i + j), j - G2 * (i + j)])
    for _ in range(5000):
        q = rng.uniform(-1e4, 1e4, 2)
        verts, w = orc.simplex(q[0], q[1])
        assert w.min() >= -1e-12 and w.sum() == pytest.approx(1.0, abs=1e-12)
        V = np.array(verts, float)
        assert V.T @ w == pytest.approx(q, abs=1e-8)            # linear precision
        sides = [np.linalg.norm(unskew(*(V[a] - V[b]))) for a, b in ((0, 1), (1, 2), (0, 2))]
        assert sides == pytest.approx([math.sqrt(2 / 3)] * 3, rel=1e-12)   # equilateral


# --------------------------------------------------------------------------
# gated Gaussian binomial (Sec. 6.3)
# --------------------------------------------------------------------------
def _pmf_from_sampler(orc, n, p, ngrid=4096):
    """Distribution of the oracle's count: the gate is open with probability
    P>=1 (checked separately), the Gaussian part is sampled on a midpoint grid
    of theta1."""
    th1 = (np.arange(ngrid) + 0.5) / ngrid
    c0 = orc.gated_count(n, p, 0.0, 0.5)
    P1 = c0[1]
    vals = np.array([orc.gated_count(n, p, 0.0, t)[0] for t in th1])
    kmax = int(math.ceil(n))
    pmf = np.bincount(vals, minlength=kmax + 1).astype(float) / ngrid * P1
    pmf[0] += 1 - P1
    return pmf, P1


@pytest.mark.parametrize("n,p", [(1, 0.3), (2, 0.3), (5, 0.1), (10, 0.5), (40, 0.034),
                                 (200, 0.02), (1000, 0.5), (3.5, 0.2), (0.4, 0.6)])
def test_gated_count_gate_probability_is_P_at_least_one(orc, n, p):
    """The gate opens with the binomial's probability of >= 1 success: scan
    theta0 across the threshold."""
    P1 = orc.gated_count(n, p, 0.0, 0.5)[1]
    want = stats.binom.sf(0, n, p) if float(n).is_integer() else 1 - (1 - p) ** n
    assert P1 == pytest.approx(want, rel=1e-12)
    assert orc.gated_count(n, p, P1 * (1 - 1e-12), 0.5)[0] >= 0
    assert orc.gated_count(n, p, min(P1 * (1 + 1e-9), 1 - 1e-16), 0.999)[0] == 0 or P1 == 1.0


@pytest.mark.parametrize("n,p", [(1, 0.3), (5, 0.1), (10, 0.5), (40, 0.5), (200, 0.02),
                                 (1000, 0.5), (5000, 0.034)])
def test_gated_count_moments_follow_binomial(orc, n, p):
    pmf, P1 = _pmf_from_sampler(orc, n, p)
    k = np.arange(len(pmf))
    mean = (k * pmf).sum()
    var = (k * k * pmf).sum() - mean ** 2
    bm, bv = stats.binom.mean(n, p), stats.binom.var(n, p)
    assert abs(mean - bm) / bm <= 0.5 / (n * p) + 0.02
    if n * p >= 1:
        assert abs(var - bv) / bv <= 0.15
    # P(c >= 1) is the gate's probability up to the Gaussian's mass below 1
    assert pmf[1:].sum() <= P1 + 1e-12


def test_gated_count_special_cases(orc):
    # p = 1: every flake reflects, count = floor(n) (n >= 1), 1 for n < 1
    for n in (0.3, 1.0, 2.5, 17.0, 4096.75):
        c = orc.gated_count(n, 1.0, 0.999, 0.01)[0]
        assert c == (1 if n < 1 else math.floor(n))
    # n <= 1: Bernoulli(P>=1) with P>=1 = 1 - (1 - p)^n
    for n in (0.25, 1.0):
        c_on = orc.gated_count(n, 0.3, 1e-9, 0.01)[0]
        c_off = orc.gated_count(n, 0.3, 0.999999, 0.99)[0]
        assert (c_on, c_off) == (1, 0)
    # zero trials never count
    assert orc.gated_count(0.0, 0.5, 1e-9, 0.99)[0] == 0
    # an open gate counts at least one success and never more than ceil(n)
    for n, p in ((3.2, 0.9), (2.3, 0.034), (40.0, 0.3)):
        for th1 in (1e-7, 0.01, 0.5, 1 - 1e-7):
            c = orc.gated_count(n, p, 0.0, th1)[0]
            assert 1 <= c <= math.ceil(n)

"""Monte Carlo of the GPU's counts against the distributed binomial
(Sec. 4.2): over 50,000 footprints of the same size at random places, the
sum of the four tetrahedron vertices' counts at one texel (simplex vertex 0,
angular texel 0) follows the convolution of the four vertices' gated laws
(chi-square), and its mean and variance follow the whole-footprint binomial
to the gated sampler's acceptance (mean within 0.5 + 2 % of n p per vertex,
variance within 15 %)."""
import math

import numpy as np
import pytest
import torch
from scipy import stats

from paper_2306_05051_gb300 import glint
from paper_2306_05051_gb300.scenes import Material
from test_oracle_pins import _gated_pmf_definition
from test_oracle_stats import pixel_row, square_J

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("A,p", [(28.0, 0.3), (600.0, 0.05)])
def test_summed_vertex_counts_follow_the_convolved_law(orc, A, p):
    rho = 1e6
    n = 50000
    rng = np.random.default_rng(31 + int(A))
    J = square_J(A / rho, ratio=2.5, angle=0.4)
    uv = rng.uniform(0, 1000, (n, 2))
    sc = pixel_row(uv, J, material=Material(R=p, ln_density=math.log(rho), n_lods=12))
    scd = sc.to(DEV)
    pix, recs = glint.trace(scd, np.arange(n, dtype=np.int32), cap=48)
    assert (pix["status"] == 0).all() and (pix["K"] == 1).all()
    sel = (recs["sv"] == 0) & (recs["av"] == 0) & (recs["light"] == 0)
    c = np.where(sel, recs["c"], 0).sum(1)
    trials = recs[0][(recs[0]["sv"] == 0) & (recs[0]["av"] == 0)]["n"].astype(np.float64)
    assert len(trials) == 4
    _, orecs = orc.trace_pixel(sc, 0)
    o_trials = orecs[(orecs["sv"] == 0) & (orecs["av"] == 0)]["n"]
    np.testing.assert_allclose(trials, o_trials, rtol=1e-6)
    pf = float(recs[0]["p"][0])
    conv = np.array([1.0])
    for t in o_trials:
        conv = np.convolve(conv, _gated_pmf_definition(float(t), pf))
    obs = np.bincount(c, minlength=len(conv))[:len(conv)].astype(np.float64)
    exp = conv * n
    keep = exp >= 10
    o_k = np.append(obs[keep], obs[~keep].sum())
    e_k = np.append(exp[keep], exp[~keep].sum())
    if e_k[-1] < 10:
        o_k, e_k = o_k[:-1], e_k[:-1]
        e_k *= o_k.sum() / e_k.sum()
    chi = stats.chisquare(o_k, e_k)
    print(f"A = {A}, p = {p}: mean {c.mean():.3f} (A p = {A * p:.3f}), var {c.var():.3f} "
          f"(A p (1-p) = {A * p * (1 - p):.3f}), chi2 p-value {chi.pvalue:.3g} over {len(o_k)} bins")
    assert chi.pvalue > 1e-4
    # the sample mean is the convolved law's; that law is the footprint's
    # binomial to the sampler's acceptance, summed over the four vertices
    k = np.arange(len(conv))
    m_law = float((k * conv).sum())
    assert abs(c.mean() - m_law) <= 4 * c.std() / math.sqrt(n)
    A_true = float(sum(o_trials))
    assert abs(c.mean() - A_true * pf) <= sum(0.5 + 0.02 * t * pf for t in o_trials) + 4 * c.std() / math.sqrt(n)
    assert c.var() / (A_true * pf * (1 - pf)) == pytest.approx(1.0, abs=0.15)

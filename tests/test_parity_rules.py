"""The comparison rules of tests/parity.py catch planted mistakes: copies
of oracle trace records (CPU) stand in for the GPU's, with one field
changed at a time."""
import numpy as np
import pytest

import parity
from paper_2306_05051_gb300 import scenes


@pytest.fixture(scope="module")
def traced(orc):
    sc = scenes.plane45(32, 32)
    for px in range(400, 1024):
        p, r = orc.trace_pixel(sc, px)
        if int(p["status"]) == 0 and len(r) and r["gate"].sum() >= 2:
            return sc, p, r
    pytest.skip("no lit pixel with two open gates")


def _compare(orc, sc, p, r, g):
    return parity.compare_pixel(orc, sc.material, p, r, p, g)


def test_identical_records_match(orc, traced):
    sc, p, r = traced
    n, exc, unexc = _compare(orc, sc, p, r, r.copy())
    assert n == len(r) and exc == 0 and unexc == []


def _first_open_far_from_integer(r):
    for k in np.flatnonzero(r["gate"]):
        f = float(r["c_cont"][k]) % 1.0
        if 0.1 < f < 0.9:
            return int(k)
    pytest.skip("no open gate with a count far from an integer")


def test_count_off_by_one_far_from_a_boundary_is_unexcused(orc, traced):
    sc, p, r = traced
    g = r.copy()
    k = _first_open_far_from_integer(r)
    g["c"][k] += 1
    _, exc, unexc = _compare(orc, sc, p, r, g)
    assert exc == 0 and [u[0] for u in unexc] == ["count"]


def test_count_flip_at_a_boundary_is_excused(orc, traced):
    sc, p, r = traced
    o = r.copy()
    k = _first_open_far_from_integer(r)
    o["c_cont"][k] = np.floor(o["c_cont"][k]) + 1.0 - 1e-9       # the oracle's count just below an integer
    g = o.copy()
    g["c"][k] += 1                                                # the other side of it
    _, exc, unexc = _compare(orc, sc, p, o, g)
    assert exc == 1 and unexc == []


def test_hash_word_change_is_unexcused(orc, traced):
    sc, p, r = traced
    g = r.copy()
    g["h0"][3] ^= 1
    _, _, unexc = _compare(orc, sc, p, r, g)
    assert [u[0] for u in unexc] == ["hash"]


def test_gate_flip_far_from_the_threshold_is_unexcused(orc, traced):
    sc, p, r = traced
    g = r.copy()
    k = next((int(k) for k in range(len(r))
              if abs(parity._theta(r["h0"][k]) - float(r["P1"][k])) > 1e-3 * max(float(r["P1"][k]), 1e-3)), None)
    if k is None:
        pytest.skip("no gate far from its threshold")
    g["gate"][k] ^= 1
    _, exc, unexc = _compare(orc, sc, p, r, g)
    assert exc == 0 and [u[0] for u in unexc] == ["gate"]


def test_lattice_vertex_change_is_unexcused(orc, traced):
    sc, p, r = traced
    g = r.copy()
    k = next((int(k) for k in range(len(r))
              if 0.01 < float(r["qx"][k]) % 1.0 < 0.99 and 0.01 < float(r["qy"][k]) % 1.0 < 0.99
              and abs(float(r["qx"][k]) % 1.0 - float(r["qy"][k]) % 1.0) > 0.01), None)
    if k is None:
        pytest.skip("no lattice coordinate away from the cell edges")
    g["i"][k] += 1
    _, exc, unexc = _compare(orc, sc, p, r, g)
    assert exc == 0 and [u[0] for u in unexc] == ["enum"]


def test_excuses_are_per_component(orc, traced):
    """A lattice vertex flipped at its own cell edge is excused; an angular
    texel changed in the same record, far from its own boundary, is not, and
    neither is a lattice vertex flipped along the other axis."""
    sc, p, r = traced
    k = next((int(k) for k in range(len(r))
              if 0.01 < float(r["afx"][k]) % 1.0 < 0.99 and 0.01 < float(r["qy"][k]) % 1.0 < 0.99
              and abs(float(r["qx"][k]) % 1.0 - float(r["qy"][k]) % 1.0) > 0.01), None)
    if k is None:
        pytest.skip("no record away from the angular and lattice edges")
    o = r.copy()
    o["qx"][k] = np.floor(o["qx"][k]) + 1.0 - 1e-9                 # the oracle's qx just below a cell edge
    g = o.copy()
    g["i"][k] += 1                                                 # the GPU on the other side of it
    _, exc, unexc = _compare(orc, sc, p, o, g)
    assert exc == 1 and unexc == []
    g2 = g.copy()
    g2["ax"][k] += 1                                               # plus an angular texel far from its edge
    _, exc, unexc = _compare(orc, sc, p, o, g2)
    assert exc == 0 and [u[0] for u in unexc] == ["enum"]
    g3 = g.copy()
    g3["j"][k] += 1                                                # plus j, whose qy is far from an edge
    _, exc, unexc = _compare(orc, sc, p, o, g3)
    assert exc == 0 and [u[0] for u in unexc] == ["enum"]


def test_missing_and_extra_records_are_unexcused(orc, traced):
    sc, p, r = traced
    _, _, unexc = _compare(orc, sc, p, r, r[1:].copy())
    assert [u[0] for u in unexc] == ["missing"]
    g = r.copy()
    g["light"][0] = 5                                             # a record the oracle does not have
    _, _, unexc = _compare(orc, sc, p, r, g)
    assert sorted(u[0] for u in unexc) == ["extra", "missing"]


def test_radiance_error_denominator():
    ref = np.array([1.0, 0.0, 2.0])
    img = np.array([1.0 + 1e-5, 1e-9, 2.0])
    err = parity.radiance_error(img, ref)
    assert err[0] == pytest.approx(1e-5) and err[2] == 0.0
    assert err[1] == pytest.approx(1e-9 / (1e-6 * 1.0))           # floor: 1e-6 of the mean |ref|

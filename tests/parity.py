"""Comparison of the CUDA path with the FP64 oracle.

Rules (the tolerance of the glint path):
  * hash words, grid ids, lattice vertices and angular texels: bit-exact,
    except where the oracle's FP64 decision variable lies within a margin of
    the decision boundary (ENUM_MARGIN in lattice / texel units,
    STRUCT_MARGIN for the (ratio, orientation, scale) cell decisions);
  * gate decisions: exact unless |theta0 - P>=1| <= GATE_MARGIN * P>=1;
  * integer counts: exact unless the oracle's continuous count lies within
    COUNT_MARGIN * max(1, c) of an integer (or n of an integer for the
    ceil(n) clamp);
  * enumeration excuses are per component: a differing lattice vertex is
    excused only by its own coordinate (i by qx, j by qy, either by the
    simplex diagonal fx = fy), a differing angular texel only by its own
    angular coordinate (ax by afx, ay by afy);
  * excused mismatches: at most BUDGET of the evaluation records of a random
    sample of lit pixels (at least MIN_SAMPLE_RECORDS records, so that the
    budget allows several), and the excused records of every pixel over the
    radiance tolerance at most BUDGET of the records of all compared pixels;
  * radiance: relative error <= RAD_TOL (denominator max(|ref|, 1e-6
    mean|ref|)) on pixels whose decisions all match.
"""
import math

import numpy as np

RAD_TOL = 1e-4
COUNT_MARGIN = 1e-5
GATE_MARGIN = 2e-6
ENUM_MARGIN = 1e-5
STRUCT_MARGIN = 1e-7
BUDGET = 1e-4
MIN_SAMPLE_RECORDS = 40000


def _frac(x):
    return x - np.floor(x)


def _near_int(x, d):
    f = _frac(x)
    return min(f, 1.0 - f) <= d


def _theta(h):
    return ((int(h) >> 8) + 0.5) * 2.0 ** -24


def struct_margin(orc, opix, material, rec):
    """Smallest distance of the oracle's cell/triangle/tetrahedron/LOD/split
    decision variables to their boundaries, for one pixel (record gives
    x, t, s, As of its sub-footprint)."""
    M, f, L = material.n_rings, material.lod_factor, material.n_lods
    d = []
    x, t, s, As = float(rec["x"]), float(rec["t"]), float(rec["s"]), float(rec["As"])
    rho_r = math.log2(opix["r"]) - math.log2(opix["Kmaj"]) if opix["r"] > 0 else 0.0
    if 0.0 < rho_r < M:
        d.append(abs(rho_r - round(rho_r)))
    d += [abs(t), abs(1 - t), abs(t - x / 2), abs(t - 1 + x / 2)]
    _, _, _, _, _, lam = orc.cell(rho_r, float(opix["phi"]), M)
    d += [abs(s - lam[0]), abs(s - lam[0] - lam[1])]
    if As > 0:
        lg = math.log(As) / math.log(f)
        d.append(abs(lg - round(lg)))
    rr = opix["r"] / 2.0 ** M
    if rr > 1:
        d.append(abs(rr - round(rr)) / rr)
    return min(d) if d else 1.0


def _enum_excused(orc, opix, material, o, r, smargin):
    """Whether a differing enumeration (grid id, lattice vertex, angular
    texel) of one record lies at a decision boundary, component by
    component."""
    if int(o["gid"]) != int(r["gid"]):
        return smargin() <= STRUCT_MARGIN
    fx, fy = _frac(o["qx"]), _frac(o["qy"])
    diag = abs(fx - fy) <= ENUM_MARGIN
    ok = True
    if int(o["i"]) != int(r["i"]):
        ok &= _near_int(o["qx"], ENUM_MARGIN) or diag
    if int(o["j"]) != int(r["j"]):
        ok &= _near_int(o["qy"], ENUM_MARGIN) or diag
    if int(o["ax"]) != int(r["ax"]):
        ok &= _near_int(o["afx"], ENUM_MARGIN)
    if int(o["ay"]) != int(r["ay"]):
        ok &= _near_int(o["afy"], ENUM_MARGIN)
    return bool(ok)


def compare_pixel(orc, material, opix, orecs, gpix, grecs):
    """Compare one pixel's records.  Returns (n_records, n_excused,
    unexcused list)."""
    unexcused = []
    excused = 0
    if int(opix["status"]) != int(gpix["status"]) or (int(opix["status"]) == 0 and int(opix["K"]) != int(gpix["K"])):
        # only decision-boundary cases may disagree on the pixel level
        m = struct_margin(orc, opix, material, orecs[0]) if len(orecs) else 1.0
        if m <= STRUCT_MARGIN:
            return len(orecs), len(orecs), []
        return len(orecs), 0, [("pixel", int(opix["status"]), int(gpix["status"]), int(opix["K"]), int(gpix["K"]))]
    g = {}
    for r in grecs:
        if r["light"] >= 0:
            g[(int(r["light"]), int(r["sub"]), int(r["vert"]), int(r["sv"]), int(r["av"]))] = r
    cache = {}

    def smargin():
        if "m" not in cache:
            cache["m"] = struct_margin(orc, opix, material, orecs[0])
        return cache["m"]

    for o in orecs:
        key = (int(o["light"]), int(o["sub"]), int(o["vert"]), int(o["sv"]), int(o["av"]))
        r = g.pop(key, None)
        if r is None:
            unexcused.append(("missing", key))
            continue
        same_enum = (int(o["gid"]) == int(r["gid"]) and int(o["i"]) == int(r["i"]) and int(o["j"]) == int(r["j"])
                     and int(o["ax"]) == int(r["ax"]) and int(o["ay"]) == int(r["ay"]))
        if not same_enum:
            if _enum_excused(orc, opix, material, o, r, smargin):
                excused += 1
            else:
                unexcused.append(("enum", key, dict(o=(int(o["gid"]), int(o["i"]), int(o["j"]), int(o["ax"]), int(o["ay"])),
                                                    g=(int(r["gid"]), int(r["i"]), int(r["j"]), int(r["ax"]), int(r["ay"])))))
            continue
        if int(o["h0"]) != int(r["h0"]) or (int(o["gate"]) and int(o["h1"]) != int(r["h1"])):
            unexcused.append(("hash", key, int(o["h0"]), int(r["h0"]), int(o["h1"]), int(r["h1"])))
            continue
        if int(o["gate"]) != int(r["gate"]):
            if abs(_theta(o["h0"]) - o["P1"]) <= GATE_MARGIN * o["P1"] + 1e-12:
                excused += 1
            else:
                unexcused.append(("gate", key, float(o["P1"]), float(r["P1"]), _theta(o["h0"])))
            continue
        if int(o["c"]) != int(r["c"]):
            cc = float(o["c_cont"])
            if _near_int(cc, COUNT_MARGIN * max(1.0, abs(cc))) or _near_int(float(o["n"]), 1e-6 * max(1.0, float(o["n"]))):
                excused += 1
            else:
                unexcused.append(("count", key, int(o["c"]), int(r["c"]), cc, float(r["c_cont"]), float(o["n"]), float(r["n"])))
    for key in g:
        unexcused.append(("extra", key))
    return len(orecs), excused, unexcused


def trace_and_compare(orc, scene_cpu, scene_dev, pixels, material=None, lights=None):
    """Trace the pixels on both sides and compare.  Returns a summary dict."""
    from paper_2306_05051_gb300 import glint
    material = material or scene_cpu.material
    lights = scene_cpu.lights if lights is None else lights
    opix, orecs = [], []
    Kmax = 1
    for px in pixels:
        p, r = orc.trace_pixel(scene_cpu, int(px), material=material, lights=lights)
        opix.append(p); orecs.append(r)
        Kmax = max(Kmax, int(p["K"]))
    cap = max(1, len(lights)) * 48 * Kmax
    gpix, grecs = glint.trace(scene_dev, pixels, cap=cap, material=material, lights=lights)
    n_rec = n_exc = 0
    bad = []
    bad_px = []
    for k, px in enumerate(pixels):
        n, e, u = compare_pixel(orc, material, opix[k], orecs[k], gpix[k], grecs[k])
        n_rec += n; n_exc += e
        if e or u:
            bad_px.append(int(px))
        if u:
            bad.append((int(px), u[:4]))
    return dict(n_rec=n_rec, n_excused=n_exc, unexcused=bad, mismatched_pixels=bad_px,
                opix=opix, gpix=gpix)


def radiance_error(img, ref):
    scale = max(float(np.abs(ref).mean()), 1e-30)
    return np.abs(img - ref) / np.maximum(np.abs(ref), 1e-6 * scale)


def check_image(orc, scene_cpu, scene_dev, img, ref, px=None, max_traced=400, rng=None, sample_trace=400,
                min_records=MIN_SAMPLE_RECORDS, material=None, lights=None):
    """Full comparison: radiance of every compared pixel; the pixels over the
    tolerance must each show an excused decision-boundary mismatch, and their
    excused records must stay within the budget of all compared records; a
    random sample of lit pixels (sample_trace pixels, grown until it holds
    min_records evaluation records or the lit pixels run out) is traced to
    measure the mismatch rate.  Returns the summary of the random sample."""
    rng = rng or np.random.default_rng(0)
    ids = np.arange(ref.size) if px is None else np.asarray(px)
    flat_img = img.reshape(-1)[ids]
    flat_ref = ref.reshape(-1)
    err = radiance_error(flat_img, flat_ref)
    over = ids[err > RAD_TOL]
    assert len(over) <= max_traced, f"{len(over)} pixels over the radiance tolerance (max rel {err.max():.3g})"
    lit = ids[flat_ref != 0]
    pool = rng.permutation(lit if len(lit) else ids)
    n_take = min(sample_trace, len(pool))
    s = trace_and_compare(orc, scene_cpu, scene_dev, np.sort(pool[:n_take]).astype(np.int32), material, lights)
    while s["n_rec"] < min_records and n_take < len(pool):
        per_px = max(s["n_rec"] / max(n_take, 1), 1.0)
        more = min(len(pool) - n_take, max(64, int((min_records - s["n_rec"]) / per_px) + 1))
        t = trace_and_compare(orc, scene_cpu, scene_dev, np.sort(pool[n_take:n_take + more]).astype(np.int32),
                              material, lights)
        n_take += more
        for k in ("n_rec", "n_excused"):
            s[k] += t[k]
        for k in ("unexcused", "mismatched_pixels", "opix", "gpix"):
            s[k] = list(s[k]) + list(t[k])
    assert not s["unexcused"], f"unexcused mismatches: {s['unexcused'][:5]}"
    assert s["n_excused"] <= BUDGET * s["n_rec"], (s["n_excused"], s["n_rec"])
    if len(over):
        so = trace_and_compare(orc, scene_cpu, scene_dev, over.astype(np.int32), material, lights)
        assert not so["unexcused"], f"unexcused mismatches: {so['unexcused'][:5]}"
        unexplained = sorted(set(int(p) for p in over) - set(so["mismatched_pixels"]))
        assert not unexplained, f"pixels over tolerance without a decision-boundary mismatch: {unexplained[:10]}"
        # every excused record of these pixels counts against the budget of
        # all compared pixels (records per lit pixel from the sample)
        est_total = s["n_rec"] / max(n_take, 1) * max(len(lit), 1)
        assert so["n_excused"] <= BUDGET * est_total, (so["n_excused"], est_total)
    matched = ~np.isin(ids, np.asarray(sorted(set(s["mismatched_pixels"]) | set(int(p) for p in over)), dtype=np.int64))
    s["max_err_matched"] = float(err[matched].max()) if matched.any() else 0.0
    s["over"] = int(len(over))
    s["n_traced"] = int(n_take)
    return s

"""Batched path (glint_eval_batch): one persistent, graph-replayed launch
over frames of uneven size gives, per frame, exactly the plain glint_eval
image; graph re-pointing, launch-shape control and argument errors."""
import numpy as np
import pytest
import torch

import parity
from paper_2306_05051_gb300 import _lib, glint, scenes

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

RES = [(64, 64), (96, 80), (160, 90), (200, 120), (33, 17), (128, 128), (256, 144), (64, 200)]


def _frames(n, device=DEV):
    return scenes.orbit_frames(n, device=device, resolutions=RES)


def test_batch_equals_plain_bitwise():
    fr = _frames(12)
    ctx = glint.BatchContext(DEV)
    outs = ctx.render(fr)
    torch.cuda.synchronize()
    for s, o in zip(fr, outs):
        assert torch.equal(o, glint.render_scene(s)), s.name
    assert ctx.launch is not None
    # second call, new output buffers: the recorded graph is re-pointed
    outs2 = ctx.render(fr)
    torch.cuda.synchronize()
    for a, b in zip(outs, outs2):
        assert a.data_ptr() != b.data_ptr() and torch.equal(a, b)
    ctx.close()


def test_batch_matches_oracle_on_sampled_pixels(orc):
    fr = _frames(4)
    ctx = glint.BatchContext(DEV)
    outs = ctx.render(fr)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    for s, o in zip(fr, outs):
        sc = s.to("cpu")
        px = np.sort(rng.choice(s.width * s.height, size=min(1500, s.width * s.height), replace=False)).astype(np.int32)
        ref = orc.eval_image(sc, px=px)
        img = o.cpu().numpy().astype(np.float64)
        parity.check_image(orc, sc, s, img, ref, px=px, sample_trace=60)


def test_batch_orbit_64_frames_at_full_size(orc):
    """The benchmarked batch: 64 orbit frames, 16 each of 256^2, 512^2,
    1280x720 and 1920x1080, in one tuned, graph-replayed launch.  Every frame
    equals its glint_eval image bit for bit, and two 1920x1080 frames match
    the oracle on sampled pixels."""
    fr = scenes.orbit_frames(64, device=DEV)
    assert sorted({(s.width, s.height) for s in fr}) == [(256, 256), (512, 512), (1280, 720), (1920, 1080)]
    ctx = glint.BatchContext(DEV)
    outs = ctx.render(fr)
    outs = ctx.render(fr)                          # graph replay
    torch.cuda.synchronize()
    for s, o in zip(fr, outs):
        assert torch.equal(o, glint.render_scene(s)), s.name
    ctx.close()
    rng = np.random.default_rng(9)
    big = [k for k, s in enumerate(fr) if s.width == 1920][:2]
    for k in big:
        s = fr[k]
        sc = s.to("cpu")
        fg = np.flatnonzero(sc.gbuf[..., 6:9].abs().sum(-1).reshape(-1).numpy() > 0)
        px = np.sort(rng.choice(fg, 6000, replace=False)).astype(np.int32)
        ref = orc.eval_image(sc, px=px)
        img = outs[k].cpu().numpy().astype(np.float64)
        parity.check_image(orc, sc, s, img, ref, px=px, sample_trace=300)


def test_batch_fixed_launch_shapes_and_reuse():
    fr = _frames(6)
    ref = [glint.render_scene(s) for s in fr]
    ctx = glint.BatchContext(DEV)
    for shape in [(128, 8), (256, 4), (1024, 1), (512, 0), (256, 0), (512, 2), (128, 0)]:
        ctx.launch = shape
        outs = ctx.render(fr)
        torch.cuda.synchronize()
        assert ctx.launch == shape
        for a, b in zip(outs, ref):
            assert torch.equal(a, b)
    # a different batch shape with a preset launch shape keeps the preset
    outs = ctx.render(fr[:3])
    torch.cuda.synchronize()
    for a, b in zip(outs, ref[:3]):
        assert torch.equal(a, b)
    ctx.close()


def test_batch_on_side_stream():
    fr = _frames(5)
    ctx = glint.BatchContext(DEV)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        outs = ctx.render(fr, stream=s)
    s.synchronize()
    for sc, o in zip(fr, outs):
        assert torch.equal(o, glint.render_scene(sc))
    ctx.close()


def test_batch_argument_errors():
    fr = _frames(2)
    ctx = glint.BatchContext(DEV)
    with pytest.raises(ValueError):
        ctx.render([fr[0].to("cpu")])
    import ctypes as C
    frames = (_lib.GlintFrame * 1)()
    frames[0] = _lib.frame_struct(fr[0].gbuf, fr[0].light_px, fr[0].mat_px, 2)
    out = torch.empty(fr[0].height, fr[0].width, device=DEV)
    optr = (C.c_void_p * 1)(out.data_ptr())
    mat = _lib.material_struct(fr[0].material)
    lts = _lib.lights_struct(fr[0].lights)
    L = _lib.lib()
    assert L.glint_eval_batch(ctx._h, frames, 0, C.byref(mat), lts, optr, None) == -1
    assert L.glint_eval_batch(ctx._h, frames, 129, C.byref(mat), lts, optr, None) == -1
    assert L.glint_eval_batch(None, frames, 1, C.byref(mat), lts, optr, None) == -1
    for bad in [(100, 2), (512, -1), (512, 17)]:
        assert L.glint_ctx_set_launch(ctx._h, C.byref(_lib.GlintLaunch(*bad))) == -1
    ctx.close()


def test_batch_switches_between_ring_and_isotropic_grids():
    """One context, batches alternating n_rings = 4 and 0: each matches
    glint_eval with that material bit for bit (the recorded graph follows
    the kernel of the mode)."""
    import dataclasses
    fr = _frames(4)
    m4 = fr[0].material
    m0 = dataclasses.replace(m4, n_rings=0)
    ctx = glint.BatchContext(DEV)
    for m in (m4, m0, m4, m0):
        outs = ctx.render(fr, material=m)
        torch.cuda.synchronize()
        for s, o in zip(fr, outs):
            assert torch.equal(o, glint.render_scene(s, material=m))
    ctx.close()

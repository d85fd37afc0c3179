"""glint_eval_batch_noalloc: the batched entry point for callers that cannot
allocate device memory (a renderer with a fixed memory budget, code that
must not synchronise the device mid-frame, a plug-in whose host owns every
allocation).  Its tile counters live in a static device array instead of
memory from cudaMalloc.  Called through the C ABI, twice in a row, it must
give glint_eval's images bit for bit (the batch kernel gives the same bits
for every launch shape).  This file is collected last so that a run stopping
at the first failure has already run every other test."""
import ctypes as C

import pytest
import torch

from paper_2306_05051_gb300 import _lib, glint, scenes

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

def _call(frames, outs, stream=None):
    n = len(frames)
    arr = (_lib.GlintFrame * n)()
    for k, f in enumerate(frames):
        arr[k] = _lib.frame_struct(f.gbuf, f.light_px, f.mat_px, len(f.lights))
    optr = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    mat = _lib.material_struct(frames[0].material)
    lts = _lib.lights_struct(frames[0].lights)
    s = torch.cuda.current_stream() if stream is None else stream
    with torch.cuda.device(DEV):
        return _lib.lib().glint_eval_batch_noalloc(arr, n, C.byref(mat), lts, optr, int(s.cuda_stream))


def test_noalloc_batch_matches_glint_eval_on_two_calls():
    # 130 frames: two launches (128 + 2), i.e. two counters of the static array
    res = [(16, 16), (24, 8), (40, 30), (7, 5), (64, 36)]
    frames = scenes.orbit_frames(130, device=DEV, resolutions=res)
    refs = [glint.render_scene(f) for f in frames]
    torch.cuda.synchronize()
    for call in range(2):
        outs = [torch.full_like(r, -1.0) for r in refs]
        assert _call(frames, outs) == 0
        torch.cuda.synchronize()
        for f, o, r in zip(frames, outs, refs):
            assert torch.equal(o, r), (call, f.name)


def test_noalloc_batch_larger_frames_and_side_stream():
    frames = scenes.orbit_frames(6, device=DEV, resolutions=[(256, 256), (320, 180), (97, 61)])
    refs = [glint.render_scene(f) for f in frames]
    s = torch.cuda.Stream()
    outs = [torch.zeros_like(r) for r in refs]
    torch.cuda.synchronize()
    for _ in range(2):
        assert _call(frames, outs, stream=s) == 0
        s.synchronize()
        for o, r in zip(outs, refs):
            assert torch.equal(o, r)


def test_noalloc_rejects_batches_beyond_the_static_scratch():
    f = scenes.orbit_frames(1, device=DEV, resolutions=[(8, 8)])[0]
    frames = [f] * 8193
    outs = [torch.zeros(8, 8, device=DEV)] * 8193
    assert _call(frames, outs) == -6            # GLINT_ERR_WORKSPACE, nothing enqueued
    assert _call(frames[:1], outs[:1]) == 0
    torch.cuda.synchronize()

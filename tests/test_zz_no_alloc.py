"""The allocation-free discretization entry point (hf_discretize_noalloc).

It serves callers that cannot allocate device memory at all, for example a
plug-in whose host application owns every device allocation and only hands
out finished output buffers, or a render loop that forbids cudaMalloc after
start-up because an allocation can synchronise the device and stall a frame.
The entry point keeps its scratch in a fixed array inside the library; here it
is called through the C ABI twice in a row (the second call reuses the
scratch left by the first) and its textures are compared with those of the
regular entry point, hf_discretize_cascades, for the same cameras.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""

import ctypes as ct

import numpy as np
import pytest

from _parity import HEIGHT_REL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _regular_textures(r, cam):
    r.set_camera(cam)
    r.discretize()
    r.sync()
    return [r.texture(0, c).clone() for c in range(cam.n_cascades)]


def test_noalloc_matches_regular_entry_point(torch_cuda, tiny):
    from paper_2201_10887_gb300 import Renderer, hf
    from paper_2201_10887_gb300.renderer import camera_struct
    torch = torch_cuda
    r = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    amp = float(np.abs(tiny.tree.value).max())
    cams = [tiny.cameras[0].with_(n_cascades=3, cascade_size=200, split_lambda=0.5),
            tiny.cameras[0].with_(n_cascades=2, cascade_size=160, forward=(0.3, 0.9, -0.4)),
            tiny.cameras[0].with_(n_cascades=2, cascade_size=144, texel_ladder=2)]
    for cam in cams:  # two calls in a row, each against the regular entry point
        ref = _regular_textures(r, cam)
        N = cam.cascade_size
        outs = [torch.full((N * N,), float("nan"), dtype=torch.float32, device="cuda")
                for _ in range(cam.n_cascades)]
        info = hf.hf_discretize_noalloc(r.ctx, camera_struct(cam), outs)
        r.sync()
        for c in range(cam.n_cascades):
            got = outs[c].view(N, N).cpu().numpy()
            want = ref[c].cpu().numpy()
            assert np.array_equal(np.isfinite(got), np.isfinite(want))
            fin = np.isfinite(want)
            assert fin.sum() > 1000
            err = np.max(np.abs(got[fin] - want[fin]) / np.maximum(np.abs(want[fin]), amp))
            assert err <= HEIGHT_REL, (c, err)
            reg = r.cascade(0, c)
            assert (info[c].snap_x, info[c].snap_y, info[c].snap_k) == (reg.snap_x, reg.snap_y, reg.snap_k)
    r.close()


def test_noalloc_rejects_oversized_views(torch_cuda, tiny):
    from paper_2201_10887_gb300 import Renderer, hf
    from paper_2201_10887_gb300.renderer import camera_struct
    r = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    cam = tiny.cameras[0].with_(n_cascades=8, cascade_size=4096)
    assert 8 * 4096 * 16 > hf.HF_NOALLOC_SCRATCH_BYTES
    ptrs = (ct.c_void_p * 8)()
    rc = hf.lib().hf_discretize_noalloc(r.ctx, ct.byref(camera_struct(cam)), ptrs, None, None)
    assert rc == hf.HF_ERR_ARG and "scratch" in hf.hf_last_error()
    r.close()

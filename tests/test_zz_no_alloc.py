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

import pytest

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


def _noalloc(torch, r, cam):
    from paper_2201_10887_gb300 import hf
    from paper_2201_10887_gb300.renderer import camera_struct
    N = cam.cascade_size
    outs = [torch.full((N * N,), float("nan"), dtype=torch.float32, device="cuda")
            for _ in range(cam.n_cascades)]
    info = hf.hf_discretize_noalloc(r.ctx, camera_struct(cam), outs)
    r.sync()
    return [o.view(N, N) for o in outs], info


def _same_bits(torch, a, b):
    """Both paths run the same kernels on the same inputs: equal bits, with
    the invisible texels (-inf) in the same places."""
    return torch.equal(torch.nan_to_num(a), torch.nan_to_num(b)) and torch.equal(torch.isinf(a), torch.isinf(b))


CAMS = [dict(n_cascades=3, cascade_size=200, split_lambda=0.5),
        dict(n_cascades=2, cascade_size=160, forward=(0.3, 0.9, -0.4)),
        dict(n_cascades=2, cascade_size=144, texel_ladder=2)]


def test_noalloc_matches_regular_entry_point(torch_cuda, tiny):
    from paper_2201_10887_gb300 import Renderer
    torch = torch_cuda
    r = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    for kw in CAMS:  # calls in a row, each against the regular entry point
        cam = tiny.cameras[0].with_(**kw)
        ref = _regular_textures(r, cam)
        got, info = _noalloc(torch, r, cam)
        for c in range(cam.n_cascades):
            assert int(torch.isfinite(ref[c]).sum()) > 1000
            assert _same_bits(torch, got[c], ref[c]), (kw, c)
            reg = r.cascade(0, c)
            assert (info[c].snap_x, info[c].snap_y, info[c].snap_k) == (reg.snap_x, reg.snap_y, reg.snap_k)
    r.close()


@pytest.mark.parametrize("kind", ["fp16", "water"])
def test_noalloc_is_fp32_terrain_in_any_context(torch_cuda, tiny, kind, monkeypatch):
    """The allocation-free path always evaluates the terrain in FP32, with the
    FP32 walk of the context's own lists: in a context created for the FP16
    path (compact lists, as a plain FP32 context keeps), or with the water
    layer (depths set; index lists, as a plain FP32 context forced onto them),
    it gives the textures of that plain FP32 context over the same leaves."""
    import workloads
    from paper_2201_10887_gb300 import Renderer
    torch = torch_cuda
    if kind == "water":
        monkeypatch.setenv("HF_FP32_INDEX_LISTS", "1")
    plain = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    monkeypatch.delenv("HF_FP32_INDEX_LISTS", raising=False)
    if kind == "fp16":
        other = Renderer(tiny.tree, tiny.sigma, tiny.radius, precision=1)
    else:
        other = Renderer(tiny.tree, tiny.sigma, tiny.radius, water=True)
        other.update_water(workloads.tiny_flood_config().depth)
    for kw in CAMS[:2]:
        cam = tiny.cameras[0].with_(**kw)
        want, _ = _noalloc(torch, plain, cam)
        got, _ = _noalloc(torch, other, cam)
        for c in range(cam.n_cascades):
            assert _same_bits(torch, got[c], want[c]), (kind, kw, c)
    plain.close()
    other.close()


def test_noalloc_binding_refuses_bad_outputs(torch_cuda, tiny):
    """The binding refuses output lists that do not match the camera before
    the library is called: the outputs stay untouched."""
    from paper_2201_10887_gb300 import Renderer, hf
    from paper_2201_10887_gb300.renderer import camera_struct
    torch = torch_cuda
    r = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    cam = tiny.cameras[0].with_(n_cascades=2, cascade_size=64)
    ok = [torch.full((64 * 64,), 7.0, device="cuda") for _ in range(2)]
    for bad in ([ok[0]], ok + [ok[0].clone()], [ok[0], ok[1][:100]], [ok[0], ok[1].double()]):
        with pytest.raises(ValueError):
            hf.hf_discretize_noalloc(r.ctx, camera_struct(cam), bad)
    torch.cuda.synchronize()
    assert all(bool((t == 7.0).all()) for t in ok)
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

"""Ray-cast results written straight into pinned host memory.

hf_raycast accepts pinned host buffers for t and hit; the kernel then writes
them over the host link while it runs, staging the results of each 16 x 8
pixel tile through shared memory so that they go out in image rows (in device
memory it stores them directly).  Both forms must give the same bytes: the
frames below are rendered into device memory and into pinned host memory and
compared bit for bit, for image sizes that do and do not fill whole tiles, a
hit buffer that does not start on a 4-byte boundary (byte stores at the row
ends), the coarse-level stop and the water layer."""

import numpy as np
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


def _both(torch, r, cam, hit_offset=0):
    """The frame of `cam` in device memory and in pinned host memory."""
    t_dev, h_dev = r.render(cam)
    r.sync()
    t_dev = t_dev.cpu().numpy().ravel().copy()
    h_dev = h_dev.cpu().numpy().ravel().copy()
    npx = cam.width * cam.height
    t_host = torch.full((npx,), -7.0, dtype=torch.float32).pin_memory()
    h_big = torch.full((npx + hit_offset,), 77, dtype=torch.uint8).pin_memory()
    h_host = h_big[hit_offset:]
    view = torch.empty(r.view_bytes(cam.n_cascades, cam.cascade_size), dtype=torch.uint8, device="cuda")
    r.bind_view(3, cam, view, t_host, h_host)
    r.render(cam, slot=3)
    r.sync()
    return t_dev, h_dev, t_host.numpy().copy(), h_host.numpy().copy()


@pytest.mark.parametrize("kw,hit_offset", [(dict(), 0), (dict(width=333, height=97), 1),
                                           (dict(n_cascades=2, cascade_size=131, width=197, height=143), 0),
                                           (dict(width=18, height=9), 3), (dict(lod_pixels=8.0), 0)])
def test_host_outputs_equal_device_outputs(torch_cuda, tiny, kw, hit_offset):
    from paper_2201_10887_gb300 import Renderer
    r = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    cam = tiny.cameras[0].with_(**kw)
    t_dev, h_dev, t_host, h_host = _both(torch_cuda, r, cam, hit_offset)
    assert np.array_equal(h_host, h_dev)
    assert np.array_equal(t_host.view(np.uint32), t_dev.view(np.uint32))
    assert (h_dev > 0).mean() > 0.05  # the frame sees terrain
    r.close()


def test_host_outputs_water_layer(torch_cuda, tiny):
    from paper_2201_10887_gb300 import Renderer
    r = Renderer(tiny.tree, tiny.sigma, tiny.radius, water=True)
    r.update_water(np.where(np.arange(tiny.tree.n_leaves) % 3 == 0, 5.0, 0.0).astype(np.float32))
    cam = tiny.cameras[0].with_(width=301, height=211)
    t_dev, h_dev, t_host, h_host = _both(torch_cuda, r, cam, 2)
    assert np.array_equal(h_host, h_dev)
    assert np.array_equal(t_host.view(np.uint32), t_dev.view(np.uint32))
    assert (h_dev & 0x80).any()
    r.close()

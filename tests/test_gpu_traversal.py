"""The max-mipmap walk variant that climbs at once to the coarsest node the
ray has entered (hf_camera.traversal = 1; our reading of the improved
traversal the paper attributes to Dick et al., Section 1) against the CPU
oracle's per-patch DDA, and against the default walk, which climbs one level
per step (Tevs et al.): both walks must find the same first hit."""

import numpy as np
import pytest

from _parity import RC, assert_rays, check_rays, frame_bracket

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


@pytest.mark.parametrize("kw", [dict(), dict(n_cascades=3, cascade_size=200, split_lambda=0.5),
                                dict(n_cascades=2, cascade_size=131, width=197, height=143,
                                     forward=(0.3, 0.9, -0.35)),
                                dict(n_cascades=4, cascade_size=97, texel_ladder=2)])
def test_jump_traversal_tiny_frames(orc, torch_cuda, tiny, kw):
    from test_gpu_parity import _frame_parity
    _frame_parity(orc, torch_cuda, tiny, tiny.cameras[0].with_(traversal=1, **kw))


def test_jump_traversal_dem_frame(orc, torch_cuda):
    """A DEM frame (four 2048^2 cascades, 1920 x 1080): every pixel against
    the oracle's DDA on the library's textures, the same hits as the default
    walk, and the node visits of both walks."""
    import workloads
    from paper_2201_10887_gb300 import Renderer
    s = workloads.dem_config(n_frames=120)
    cam = s.cameras[60]
    r = Renderer(s.tree, s.sigma, s.radius)
    t0, h0 = r.render(cam)
    v0 = r.ray_stats()["visits"]
    t0, h0 = t0.cpu().numpy().ravel().copy(), h0.cpu().numpy().ravel().copy()
    t1, h1 = r.render(cam.with_(traversal=1))
    r.sync()
    v1 = r.ray_stats()["visits"]
    gt, gh = t1.cpu().numpy().ravel(), h1.cpu().numpy().ravel()
    assert np.array_equal(gh, h0)
    both = gh > 0
    rel = np.abs(gt[both] - t0[both]) / t0[both]
    print(f"jump walk: {v1 / gt.size:.2f} visits per ray against {v0 / gt.size:.2f}; "
          f"identical t on {np.mean(gt[both] == t0[both]):.6f} of the hits, max rel. difference {rel.max():.2e}")
    assert rel.max() < 1e-6
    cells = orc.Cells(s.tree)
    amp = float(np.abs(cells.cv).max())
    texs, rcs = [], []
    for c in range(cam.n_cascades):
        texs.append(r.texture(0, c).cpu().numpy())
        rcs.append(RC(r.cascade(0, c)))
    ot, oh, seg, _ = orc.raycast(cam, s.tree, rcs, texs)
    res = check_rays(gt, gh, ot, oh, seg, shape=(cam.height, cam.width),
                     bracket=frame_bracket(orc, cam, s.tree, rcs, texs, gt, gh, ot, seg, amp))
    assert_rays(res, "dem frame 60, jump walk")
    r.close()

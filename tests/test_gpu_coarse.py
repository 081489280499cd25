"""GPU parity of the coarse-level stop (hf_camera.lod_pixels): with a stop
level L_c per cascade the rays end at the box tops of max-mip level L_c.  The
oracle's reference is its independent box-field walk (a 2-D DDA over the
level-L nodes, itself pinned against dense marching).  The same rules apply
as for the exact surface (_parity.py); the stop levels are the oracle's."""

import numpy as np
import pytest

from _parity import BOX_EXCUSE_REL, RC, assert_rays, check_rays, frame_bracket

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


@pytest.mark.parametrize("lod", [8.0, 32.0])
def test_coarse_stop_tiny_frames(orc, torch_cuda, tiny, lod):
    from test_gpu_parity import _frame_parity
    base = tiny.cameras[0]
    for cam in (base.with_(n_cascades=3, cascade_size=200, split_lambda=0.7, lod_pixels=lod),
                base.with_(n_cascades=2, cascade_size=160, forward=(0.3, 0.9, -0.35), lod_pixels=lod)):
        from paper_2201_10887_gb300 import Renderer
        r = Renderer(tiny.tree, tiny.sigma, tiny.radius)
        r.set_camera(cam)
        levels = [r.cascade(0, c).stop_level for c in range(cam.n_cascades)]
        r.close()
        assert max(levels) >= 1, levels
        _frame_parity(orc, torch_cuda, tiny, cam)


def test_coarse_stop_levels_match_oracle(orc, torch_cuda, tiny):
    from paper_2201_10887_gb300 import Renderer
    r = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    for lod in (0.0, 1.0, 4.0, 16.0, 256.0):
        cam = tiny.cameras[0].with_(n_cascades=4, cascade_size=256, lod_pixels=lod)
        r.set_camera(cam)
        for c in range(cam.n_cascades):
            info = r.cascade(0, c)
            assert info.stop_level == orc.stop_level(lod, cam.vfov, cam.height, info.near, info.texel, info.N)
    r.close()


def test_coarse_stop_dem_frame(orc, torch_cuda):
    """A DEM frame (four 2048^2 cascades, 1920 x 1080) with the coarse stop at
    eight pixels (the cascade splits already make a texel about one pixel at
    a cascade's near edge): every pixel against the oracle's box-field walk on the
    library's textures; the far cascades stop above level 0, and hits come no
    later than the exact surface's."""
    import workloads
    from paper_2201_10887_gb300 import Renderer
    s = workloads.dem_config(n_frames=120)
    cam = s.cameras[60].with_(lod_pixels=8.0)
    r = Renderer(s.tree, s.sigma, s.radius)
    t, hit = r.render(cam)
    r.sync()
    cells = orc.Cells(s.tree)
    amp = float(np.abs(cells.cv).max())
    texs, rcs = [], []
    for c in range(cam.n_cascades):
        info = r.cascade(0, c)
        texs.append(r.texture(0, c).cpu().numpy())
        rcs.append(RC(info))
    assert max(rc.stop_level for rc in rcs) >= 1
    gt, gh = t.cpu().numpy().ravel(), hit.cpu().numpy().ravel()
    ot, oh, seg, _ = orc.raycast(cam, s.tree, rcs, texs)
    res = check_rays(gt, gh, ot, oh, seg, shape=(cam.height, cam.width),
                     bracket=frame_bracket(orc, cam, s.tree, rcs, texs, gt, gh, ot, seg, amp))
    assert_rays(res, "dem frame 60, coarse stop at 8 pixels", BOX_EXCUSE_REL)
    t0, h0 = r.render(cam.with_(lod_pixels=0.0), slot=1)
    r.sync()
    e0, eh = t0.cpu().numpy().ravel(), h0.cpu().numpy().ravel()
    both = (gh > 0) & (eh > 0)
    assert np.mean(gt[both] <= e0[both] * (1 + 1e-5)) > 0.999
    r.close()

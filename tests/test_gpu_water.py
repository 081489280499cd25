"""GPU parity of the water layer (terrain + relative water depths at the
same cells, Section 2 and Table 1) against the CPU FP64 oracle: terrain and
water-surface textures, the max mipmap bounding both, and rays that stop at
whichever surface they meet first, on a tiny flood, ragged sizes, a depth
update, an all-dry field and the DEM flood at full size.  Rules in
_parity.py (water wet/dry, water flag)."""

import numpy as np
import pytest

from _parity import (HEIGHT_REL, RC, assert_rays, check_mask, check_rays, check_water_flags, frame_bracket,
                     mask_from_spans, ocas)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _water_frame(orc, scene, cam, depth, texel_sample=None, seed=0, r=None):
    """The water frame of `cam` against the oracle (on renderer r, whose
    depths are then replaced by `depth`, or on a fresh one)."""
    from paper_2201_10887_gb300 import Renderer
    if r is None:
        r = Renderer(scene.tree, scene.sigma, scene.radius, water=True)
    r.update_water(depth)
    t, hit = r.render(cam)
    r.sync()
    cells = orc.Cells(scene.tree)
    amp = float(np.abs(cells.cv).max())
    dmax = float(np.max(depth)) if np.max(depth) > 0 else 1.0
    rng = np.random.default_rng(seed)
    texs, wtexs, rcs = [], [], []
    for c in range(cam.n_cascades):
        info = r.cascade(0, c)
        spans = r.spans(0, c).cpu().numpy()
        bad, vis, _ = check_mask(orc, info, cells, spans)
        assert bad == 0
        tex = r.texture(0, c).cpu().numpy()
        wtex = r.water_texture(0, c).cpu().numpy()
        shown = mask_from_spans(spans, info.N)
        assert np.array_equal(np.isfinite(tex), shown)
        assert not np.any(np.isfinite(wtex) & ~shown)          # water only on visible texels
        jj, ii = np.nonzero(vis & shown)
        if texel_sample is not None and jj.size > texel_sample:
            pick = rng.choice(jj.size, size=texel_sample, replace=False)
            jj, ii = jj[pick], ii[pick]
        v, d, w = orc.water_heights(ocas(orc, info), cells, depth, scene.sigma, scene.radius, ii, jj)
        gv, gw = tex[jj, ii], wtex[jj, ii]
        assert np.max(np.abs(gv - v) / np.maximum(np.abs(v), amp)) <= HEIGHT_REL
        wet_g, wet_o = np.isfinite(gw), np.isfinite(w)
        # wet/dry may differ only where the oracle's depth is ~0, and a GPU-only
        # wet texel then sits on the terrain
        mis = wet_g != wet_o
        assert np.all(np.abs(d[mis]) <= 1e-6 * dmax), np.abs(d[mis]).max()
        only_g = wet_g & ~wet_o
        assert np.all(np.abs(gw[only_g] - v[only_g]) <= 1e-6 * dmax + HEIGHT_REL * amp)
        both = wet_g & wet_o
        if both.any():
            assert np.max(np.abs(gw[both] - w[both]) / np.maximum(np.abs(w[both]), amp)) <= HEIGHT_REL
        assert np.array_equal(r.mip(0, c).cpu().numpy(), orc.maxmip_pair(tex, wtex))
        texs.append(tex)
        wtexs.append(wtex)
        rcs.append(RC(info))
    gt, gh = t.cpu().numpy().ravel(), hit.cpu().numpy().ravel()
    ot, oh, seg = orc.raycast_water(cam, scene.tree, rcs, texs, wtexs)
    res = check_rays(gt, gh, ot, oh, seg, shape=(cam.height, cam.width),
                     bracket=frame_bracket(orc, cam, scene.tree, rcs, texs, gt, gh, ot, seg, amp, water_texs=wtexs))
    assert_rays(res, "water layer")
    n_mis, n_bad = check_water_flags(orc, cam, scene.tree, rcs, texs, wtexs, gh, oh, seg)
    assert n_bad == 0, (n_mis, n_bad)
    both = (gh > 0) & (oh > 0) & ((gh & 0x80) == (oh & 0x80))
    assert not both.any() or np.mean((gh[both] & 0x7F) != (oh[both] & 0x7F)) < 1e-3    # first-hit cascade
    r.close()
    return float(np.mean((oh & 0x80) > 0)), float(np.mean(oh > 0))


def test_tiny_flood_frame(orc, torch_cuda):
    import workloads
    s = workloads.tiny_flood_config()
    water_px, hit_px = _water_frame(orc, s, s.cameras[0], s.depth)
    assert water_px > 0.05 and hit_px > 0.3


@pytest.mark.parametrize("N,W,H,C,lam,wet", [(100, 97, 61, 3, 0.5, 0.5), (257, 200, 150, 2, 1.0, 0.15)])
def test_tiny_flood_ragged(orc, torch_cuda, N, W, H, C, lam, wet):
    import workloads
    s = workloads.tiny_flood_config(wet_area=wet)
    cam = s.cameras[0].with_(cascade_size=N, width=W, height=H, n_cascades=C, split_lambda=lam)
    water_px, _ = _water_frame(orc, s, cam, s.depth)
    assert water_px > 0.01


def test_dry_field_matches_terrain_only(orc, torch_cuda, monkeypatch):
    """All depths 0: no water texel anywhere, and the rays equal the
    terrain-only library's bit for bit (the terrain-only context on the index
    lists, the walk the water layer uses)."""
    import workloads
    from paper_2201_10887_gb300 import Renderer
    s = workloads.tiny_config()
    cam = s.cameras[0]
    rw = Renderer(s.tree, s.sigma, s.radius, water=True)
    rw.update_water(np.zeros(s.tree.n_leaves, np.float32))
    tw, hw = rw.render(cam)
    monkeypatch.setenv("HF_FP32_INDEX_LISTS", "1")
    r0 = Renderer(s.tree, s.sigma, s.radius)
    t0, h0 = r0.render(cam)
    rw.sync()
    r0.sync()
    assert torch_cuda.equal(hw, h0)
    assert torch_cuda.equal(torch_cuda.nan_to_num(tw, nan=-1.0), torch_cuda.nan_to_num(t0, nan=-1.0))
    for c in range(cam.n_cascades):
        assert torch_cuda.equal(rw.texture(0, c), r0.texture(0, c))
        assert not torch_cuda.isfinite(rw.water_texture(0, c)).any()
    rw.close()
    r0.close()


def test_depth_update_between_frames(orc, torch_cuda):
    """A new depth field (a higher flood) replaces the old one in the same
    context without a rebuild; the next frame matches the oracle on the new
    depths."""
    import workloads
    from paper_2201_10887_gb300 import Renderer
    s = workloads.tiny_flood_config(wet_area=0.1)
    r = Renderer(s.tree, s.sigma, s.radius, water=True)
    r.update_water(s.depth)
    r.render(s.cameras[0])
    r.sync()
    deeper, _ = workloads.flood_depths(s.tree, 0.45)
    water_px, _ = _water_frame(orc, s, s.cameras[0], deeper, r=r)
    assert water_px > 0.1


def test_water_api_errors(torch_cuda):
    import workloads
    from paper_2201_10887_gb300 import Renderer, hf
    s = workloads.tiny_config()
    r0 = Renderer(s.tree, s.sigma, s.radius)
    with pytest.raises(hf.HFError) as e:
        r0.update_water(np.zeros(s.tree.n_leaves, np.float32))
    assert e.value.code == hf.HF_ERR_STATE
    rw = Renderer(s.tree, s.sigma, s.radius, water=True)
    bad = np.zeros(s.tree.n_leaves, np.float32)
    bad[5] = -1.0
    for arr in (bad, np.zeros(3, np.float32), np.full(s.tree.n_leaves, np.nan, np.float32)):
        with pytest.raises(hf.HFError) as e:
            rw.update_water(arr)
        assert e.value.code == hf.HF_ERR_ARG
    # batched frames do not carry the water layer
    rw.set_camera(s.cameras[0])
    v = rw.views[0]
    items = (hf.hf_batch_item * 1)(hf.hf_batch_item(rw.ctx.value, 0, 0, v["t"].data_ptr(), v["hit"].data_ptr()))
    with pytest.raises(hf.HFError) as e:
        hf.hf_batch_query_bytes(items, 0)
    assert e.value.code == hf.HF_ERR_ARG
    r0.close()
    rw.close()


@pytest.mark.slow
def test_dem_flood_frame(orc, torch_cuda):
    """DEM-scale flood (4.5 M leaves, 20 % of the area under water), four
    2048^2 cascades, 1920 x 1080: sampled texels, every pixel."""
    import workloads
    s = workloads.flood_config(n_frames=120)
    water_px, hit_px = _water_frame(orc, s, s.cameras[0], s.depth, texel_sample=3000)
    assert hit_px > 0.5

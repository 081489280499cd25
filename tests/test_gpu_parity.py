"""GPU parity: the CUDA path through the C ABI against the CPU FP64 oracle,
element by element on the same seeded inputs (tolerances in _parity.py)."""

import math

import numpy as np
import pytest

from _parity import (BOX_EXCUSE_REL, EXCUSE_REL, GRAZE_REL, HEIGHT_REL, RAY_REL, RC, assert_rays, bracketed,
                     check_mask, check_rays, excuse_cap, frame_bracket, height_error, mask_from_spans, mask_margin, ocas, surface_bracket)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _frame_parity(orc, torch_cuda, scene, cam, bucket_level=-1, full_rays=True, kernel=0):
    from paper_2201_10887_gb300 import Renderer
    r = Renderer(scene.tree, scene.sigma, scene.radius, bucket_level=bucket_level, kernel=kernel)
    t, hit = r.render(cam)
    r.sync()
    cells = orc.Cells(scene.tree)
    amp = float(np.abs(cells.cv).max())
    ov = orc.fit(cam, scene.tree, cells)
    texs, rcs, worst = [], [], 0.0
    for c in range(cam.n_cascades):
        info = r.cascade(0, c)
        oc = ov.cas[c]
        assert (info.snap_x, info.snap_y, info.snap_k) == (oc.snap_x, oc.snap_y, oc.snap_k)
        spans = r.spans(0, c).cpu().numpy()
        bad, vis, near = check_mask(orc, info, cells, spans)
        assert bad == 0, f"cascade {c}: {bad} mask mismatches"
        tex = r.texture(0, c).cpu().numpy()
        ref = orc.texel_heights(ocas(orc, info), cells, scene.sigma, scene.radius,
                                kernel=kernel).reshape(info.N, info.N)
        assert np.array_equal(np.isfinite(tex), mask_from_spans(spans, info.N))
        worst = max(worst, height_error(tex, ref, amp, exempt=near))
        mip = r.mip(0, c).cpu().numpy()
        assert np.array_equal(mip, orc.maxmip(tex)), f"cascade {c}: max mip differs"
        texs.append(tex)
        rcs.append(RC(info))
    assert worst <= HEIGHT_REL, worst
    ot, oh, seg, _ = orc.raycast(cam, scene.tree, rcs, texs)
    gt, gh = t.cpu().numpy().ravel(), hit.cpu().numpy().ravel()
    res = check_rays(gt, gh, ot, oh, seg, shape=(cam.height, cam.width),
                     bracket=frame_bracket(orc, cam, scene.tree, rcs, texs, gt, gh, ot, seg, amp))
    assert_rays(res, f"{cam.width}x{cam.height}, {cam.n_cascades} x {cam.cascade_size}^2",
                BOX_EXCUSE_REL if cam.lod_pixels > 0 else EXCUSE_REL)
    terr = res.terr
    # the reported first-hit cascade agrees where both hit
    both = (gh > 0) & (oh > 0)
    assert not both.any() or np.mean(gh[both] != oh[both]) < 1e-3
    r.close()
    return worst, terr, int((oh > 0).sum())


def test_tiny_frame(orc, torch_cuda, tiny):
    """The tiny workload as specified: one 256^2 cascade, 320 x 240."""
    w, terr, hits = _frame_parity(orc, torch_cuda, tiny, tiny.cameras[0])
    assert hits > 20000


@pytest.mark.parametrize("N,W,H,C,lam", [(100, 173, 97, 3, 0.5), (129, 64, 200, 2, 1.0),
                                         (37, 50, 31, 4, 0.0)])
def test_ragged_sizes_and_cascades(orc, torch_cuda, tiny, N, W, H, C, lam):
    """Texture sides and image sizes that are not multiples of any tile."""
    cam = tiny.cameras[0].with_(n_cascades=C, cascade_size=N, width=W, height=H, split_lambda=lam)
    _frame_parity(orc, torch_cuda, tiny, cam)


@pytest.mark.parametrize("N,C", [(256, 1), (100, 3)])
def test_wendland_kernel_frame(orc, torch_cuda, tiny, N, C):
    """Another interpolant in the discretization slot (Wendland's compactly
    supported C2 function over the same supports): heights, mips and rays
    against the oracle with the same weights."""
    cam = tiny.cameras[0].with_(cascade_size=N, n_cascades=C)
    worst, terr, nhit = _frame_parity(orc, torch_cuda, tiny, cam, kernel=orc.WENDLAND_C2)
    assert nhit > 1000


def test_far_world_origin(orc, torch_cuda):
    """World origin at (5e6, 5e6) m: FP64 camera-relative set-up keeps the
    FP32 path within tolerance."""
    import workloads
    s = workloads.precision_config()
    _frame_parity(orc, torch_cuda, s, s.cameras[0].with_(n_cascades=3, split_lambda=0.5))


@pytest.mark.parametrize("bucket_level", [0, 1, 2])
def test_bucket_levels_agree(orc, torch_cuda, tiny, bucket_level):
    """Superset lists of any bucket size give the same heights (Section 4)."""
    cam = tiny.cameras[0].with_(n_cascades=2, cascade_size=128)
    _frame_parity(orc, torch_cuda, tiny, cam, bucket_level=bucket_level)


def test_steep_and_sideways_views(orc, torch_cuda, tiny):
    base = tiny.cameras[0]
    for cam in [base.with_(n_cascades=2, forward=(0.0, 0.2, -1.0)),
                base.with_(n_cascades=3, forward=(-0.8, 0.1, -0.6), vfov=math.radians(40)),
                base.with_(n_cascades=2, forward=(0.0, 0.0, -1.0), up=(0.0, 1.0, 0.0))]:
        _frame_parity(orc, torch_cuda, tiny, cam)


def test_empty_view(orc, torch_cuda, tiny):
    from paper_2201_10887_gb300 import Renderer
    cam = tiny.cameras[0].with_(forward=(0.0, -1.0, 0.2), n_cascades=2)
    cam = cam.with_(eye=(cam.eye[0], tiny.tree.origin_y - 100.0, cam.eye[2]))
    r = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    t, hit = r.render(cam)
    r.sync()
    assert int(hit.sum()) == 0 and bool(torch_cuda.isnan(t).all())
    for c in range(2):
        assert r.cascade(0, c).n_poly == 0
        assert bool(torch_cuda.isinf(r.texture(0, c)).all())
    r.close()


def test_flat_terrain_plane_hits(orc, torch_cuda, tiny):
    """Constant cell values: every visible texel equals the constant and rays
    hit the plane at t = (o_z - h0) / (-d_z)."""
    import copy
    from paper_2201_10887_gb300 import Renderer
    tree = copy.copy(tiny.tree)
    tree.value = np.full_like(tiny.tree.value, 250.0)
    cam = tiny.cameras[0].with_(n_cascades=2, cascade_size=128)
    r = Renderer(tree, tiny.sigma, tiny.radius)
    t, hit = r.render(cam)
    r.sync()
    for c in range(2):
        tex = r.texture(0, c).cpu().numpy()
        fin = np.isfinite(tex)
        assert fin.sum() > 1000 and np.max(np.abs(tex[fin] - 250.0)) < 1e-3
    gt, gh = t.cpu().numpy().ravel(), hit.cpu().numpy().ravel()
    # independent ray directions from the camera basis
    F = np.array(cam.forward) / np.linalg.norm(cam.forward)
    U = np.array(cam.up) - np.dot(cam.up, F) * F
    U /= np.linalg.norm(U)
    R = np.cross(F, U)
    tv = math.tan(cam.vfov / 2)
    th = tv * cam.width / cam.height
    py, px = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    sx = (2 * (px.ravel() + 0.5) / cam.width - 1) * th
    sy = (1 - 2 * (py.ravel() + 0.5) / cam.height) * tv
    d = F[None] + sx[:, None] * R[None] + sy[:, None] * U[None]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    tp = (cam.eye[2] - 250.0) / (-d[:, 2])
    ok = gh > 0
    assert ok.sum() > 10000
    assert np.max(np.abs(gt[ok] - tp[ok]) / tp[ok]) < 2e-5
    r.close()


def test_update_values(orc, torch_cuda, tiny):
    """New cell values (e.g. a water level update) without rebuilding."""
    import copy
    from paper_2201_10887_gb300 import Renderer
    cam = tiny.cameras[0].with_(n_cascades=2, cascade_size=96)
    r = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    r.render(cam)
    new = (tiny.tree.value * 0.5 + 40.0).astype(np.float32)
    r.update_values(new)
    r.render(cam)
    r.sync()
    tree2 = copy.copy(tiny.tree)
    tree2.value = new
    cells = orc.Cells(tree2)
    amp = float(np.abs(cells.cv).max())
    for c in range(2):
        info = r.cascade(0, c)
        ref = orc.texel_heights(ocas(orc, info), cells, tiny.sigma, tiny.radius).reshape(info.N, info.N)
        _, margin = mask_margin(orc, info, cells)
        assert height_error(r.texture(0, c).cpu().numpy(), ref, amp, exempt=margin <= 1e-7) <= HEIGHT_REL
    # a rejected update (a NaN in the middle) changes nothing
    from paper_2201_10887_gb300 import hf
    before = [r.texture(0, c).clone() for c in range(2)]
    bad = new.copy()
    bad[bad.size // 2] = np.nan
    with pytest.raises(hf.HFError) as e:
        r.update_values(bad)
    assert e.value.code == hf.HF_ERR_ARG
    r.render(cam)
    r.sync()
    for c in range(2):
        assert torch_cuda.equal(r.texture(0, c), before[c])
    r.close()


def test_minimal_texture(orc, torch_cuda, tiny):
    """N = 2: one patch per cascade, a single-entry max mipmap."""
    cam = tiny.cameras[0].with_(n_cascades=1, cascade_size=2, width=16, height=12)
    from paper_2201_10887_gb300 import Renderer
    r = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    r.render(cam)
    r.sync()
    tex = r.texture(0, 0).cpu().numpy()
    assert np.array_equal(r.mip(0, 0).cpu().numpy(), orc.maxmip(tex))
    r.close()


@pytest.mark.slow
def test_maximum_cascades_and_size(orc, torch_cuda, tiny):
    """HF_MAX_CASCADES cascades of the largest side (8192^2, a 14-level max
    mipmap): full masks and mipmaps, sampled texels and rays."""
    from paper_2201_10887_gb300 import Renderer, hf
    cam = tiny.cameras[0].with_(n_cascades=hf.HF_MAX_CASCADES, cascade_size=8192, width=320, height=240)
    r = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    t, hit = r.render(cam)
    r.sync()
    cells = orc.Cells(tiny.tree)
    amp = float(np.abs(cells.cv).max())
    rng = np.random.default_rng(7)
    texs, rcs = [], []
    for c in range(cam.n_cascades):
        info = r.cascade(0, c)
        assert info.N == 8192
        spans = r.spans(0, c).cpu().numpy()
        tex = r.texture(0, c).cpu().numpy()
        shown = mask_from_spans(spans, info.N)
        assert np.array_equal(np.isfinite(tex), shown)
        jj, ii = np.nonzero(shown)
        if jj.size:
            pick = rng.choice(jj.size, size=min(1500, jj.size), replace=False)
            vis, _ = orc.mask(ocas(orc, info), cells, ii[pick], jj[pick])
            assert vis.all()
            ref = orc.texel_heights(ocas(orc, info), cells, tiny.sigma, tiny.radius, ii[pick], jj[pick])
            got = tex[jj[pick], ii[pick]]
            assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), amp)) <= HEIGHT_REL
        assert np.array_equal(r.mip(0, c).cpu().numpy(), orc.maxmip(tex))
        texs.append(tex)
        rcs.append(RC(info))
    gt, gh = t.cpu().numpy(), hit.cpu().numpy()
    py = rng.integers(0, cam.height, 1500)
    px = rng.integers(0, cam.width, 1500)
    ot, oh, seg, _ = orc.raycast(cam, tiny.tree, rcs, texs, pixels=(px, py))
    g_t, g_h = gt[py, px], gh[py, px]

    def bracket(idx):                 # backward-error rule on the sampled pixels
        tmax = np.nanmax(np.concatenate([np.where(g_h[idx] > 0, g_t[idx], np.nan), ot[idx], [0.0]]))
        tu, hu, td, hd = surface_bracket(orc, cam, tiny.tree, rcs, texs, px[idx], py[idx],
                                         GRAZE_REL * (tmax + amp))
        return bracketed(g_t[idx], g_h[idx], seg[idx], tu, hu, td, hd)
    res = check_rays(g_t, g_h, ot, oh, seg, silhouette=np.zeros(px.size, bool), bracket=bracket)
    print(f"sampled rays: {res.n}, hit/miss differ {res.frac:.2e}, passed by backward error {res.excused}")
    assert res.frac <= 2e-3 and res.off == 0, (res.frac, res.off)
    assert int(((g_h > 0) & (oh > 0)).sum()) > 500
    assert res.terr <= RAY_REL, res.terr
    assert res.excused <= excuse_cap(res.n), res.excused
    r.close()


@pytest.mark.slow
@pytest.mark.parametrize("frame", [0, 60])
def test_dem_frame_sampled(orc, torch_cuda, frame):
    """DEM-scale workload (4.5 M leaves, four 2048^2 cascades, 1920 x 1080)
    in the bench's launch configuration: full mask and max-mip comparison,
    sampled texels, and every pixel against the oracle ray caster run on the
    library's textures."""
    import workloads
    from paper_2201_10887_gb300 import Renderer
    s = workloads.dem_config(n_frames=120)
    cam = s.cameras[frame]
    r = Renderer(s.tree, s.sigma, s.radius)
    t, hit = r.render(cam)
    r.sync()
    cells = orc.Cells(s.tree)
    amp = float(np.abs(cells.cv).max())
    rng = np.random.default_rng(frame)
    texs, rcs = [], []
    for c in range(cam.n_cascades):
        info = r.cascade(0, c)
        spans = r.spans(0, c).cpu().numpy()
        bad, vis, _ = check_mask(orc, info, cells, spans)
        assert bad == 0
        tex = r.texture(0, c).cpu().numpy()
        assert np.array_equal(np.isfinite(tex), mask_from_spans(spans, info.N))
        jj, ii = np.nonzero(vis & np.isfinite(tex))
        pick = rng.choice(jj.size, size=min(4000, jj.size), replace=False)
        ref = orc.texel_heights(ocas(orc, info), cells, s.sigma, s.radius, ii[pick], jj[pick])
        got = tex[jj[pick], ii[pick]]
        err = np.max(np.abs(got - ref) / np.maximum(np.abs(ref), amp))
        assert err <= HEIGHT_REL, (c, err)
        assert np.array_equal(r.mip(0, c).cpu().numpy(), orc.maxmip(tex))
        texs.append(tex)
        rcs.append(RC(info))
    gt, gh = t.cpu().numpy().ravel(), hit.cpu().numpy().ravel()
    ot, oh, seg, _ = orc.raycast(cam, s.tree, rcs, texs)
    res = check_rays(gt, gh, ot, oh, seg, shape=(cam.height, cam.width),
                     bracket=frame_bracket(orc, cam, s.tree, rcs, texs, gt, gh, ot, seg, amp))
    assert_rays(res, f"dem frame {frame}")
    r.close()


def test_outputs_in_pinned_host_memory(torch_cuda, tiny):
    """The ray cast writes t and hit straight into pinned host memory, bit for
    bit what it writes to device memory; pageable host memory is refused
    before any launch."""
    import ctypes as ct
    from paper_2201_10887_gb300 import Renderer, hf
    cam = tiny.cameras[0].with_(n_cascades=2, cascade_size=128)
    a = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    b = Renderer(tiny.tree, tiny.sigma, tiny.radius, host_outputs=True)
    ta, ha = a.render(cam)
    tb, hb = b.render(cam)
    b.sync()
    assert not tb.is_cuda and tb.is_pinned()
    assert torch_cuda.equal(ta.cpu().view(torch_cuda.int32), tb.view(torch_cuda.int32))
    assert torch_cuda.equal(ha.cpu(), hb)
    assert (hb > 0).sum() > 1000
    pageable_t = np.zeros(cam.width * cam.height, np.float32)
    pageable_h = np.zeros(cam.width * cam.height, np.uint8)
    rc = hf.lib().hf_raycast(a.ctx, 0, pageable_t.ctypes.data_as(ct.c_void_p),
                             pageable_h.ctypes.data_as(ct.c_void_p), None)
    assert rc == hf.HF_ERR_ARG
    assert "pageable" in hf.hf_last_error()
    assert not pageable_t.any()
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_lookup_without_cell_map_is_identical(torch_cuda, tiny, monkeypatch, precision):
    """Grids beyond the cell map's size limit look their bucket up in the
    occupancy bitmaps instead; HF_CELLMAP_MAX_CELLS=0 forces that path here:
    textures, mipmaps and rays equal the cell-map path's bit for bit."""
    from paper_2201_10887_gb300 import Renderer
    cam = tiny.cameras[0].with_(n_cascades=3, cascade_size=192, split_lambda=0.5)
    a = Renderer(tiny.tree, tiny.sigma, tiny.radius, precision=precision)
    monkeypatch.setenv("HF_CELLMAP_MAX_CELLS", "0")
    b = Renderer(tiny.tree, tiny.sigma, tiny.radius, precision=precision)
    assert b.persistent_bytes < a.persistent_bytes
    ta, ha = a.render(cam)
    tb, hb = b.render(cam)
    a.sync()
    b.sync()
    for c in range(cam.n_cascades):
        assert torch_cuda.equal(a.texture(0, c).view(torch_cuda.int32), b.texture(0, c).view(torch_cuda.int32))
        assert torch_cuda.equal(a.mip(0, c).view(torch_cuda.int32), b.mip(0, c).view(torch_cuda.int32))
    assert torch_cuda.equal(ta.view(torch_cuda.int32), tb.view(torch_cuda.int32)) and torch_cuda.equal(ha, hb)
    a.close()
    b.close()


@pytest.mark.parametrize("kernel", [0, 1])
def test_index_list_walk_frames(orc, torch_cuda, tiny, monkeypatch, kernel):
    """The FP32 walk over lists of leaf indices (grids whose offsets do not fit
    the compact lists, and the water layer, use it; HF_FP32_INDEX_LISTS=1
    forces it here) passes the same frame rules as the walk over the compact
    lists, for both interpolants."""
    monkeypatch.setenv("HF_FP32_INDEX_LISTS", "1")
    for cam in (tiny.cameras[0], tiny.cameras[0].with_(n_cascades=3, cascade_size=131, width=173, height=97)):
        _frame_parity(orc, torch_cuda, tiny, cam, kernel=kernel)

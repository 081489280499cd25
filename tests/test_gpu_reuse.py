"""Temporal reuse (hf_discretize_reuse) and the lattice fit it relies on.

The lattice fit's frames are checked against the oracle like every other
frame (test_gpu_parity's rules).  Texels carried over from an earlier frame
must equal a fresh discretization of the same view bit for bit (every
height is a function of the texel's position and the leaf data only), also
with the water layer and the FP16 path; the carried-over count is checked
against the earlier frame's texture and the current spans on the host."""

import math

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


def _flight(cam, n, step=(3.7, 2.3), yaw_deg=0.25, ladder=4, **kw):
    """n cameras moving by `step` metres and turning by yaw_deg per frame."""
    out = []
    f0 = np.array(cam.forward, float)
    for k in range(n):
        a = math.radians(yaw_deg * k)
        f = (f0[0] * math.cos(a) - f0[1] * math.sin(a), f0[0] * math.sin(a) + f0[1] * math.cos(a), f0[2])
        eye = (cam.eye[0] + step[0] * k, cam.eye[1] + step[1] * k, cam.eye[2])
        out.append(cam.with_(eye=eye, forward=f, texel_ladder=ladder, **kw))
    return out


def _bits(t):
    """The tensor's words, so that NaN payloads compare equal."""
    import torch
    return t.contiguous().view(-1).view(torch.int32)


def _expected_reuse(r, slot, prev_slot, c):
    """Visible texels of cascade c whose lattice point the source cascade
    computed, from the earlier texture and the current spans (host)."""
    info = r.cascade(slot, c)
    q = info.reuse_source
    if q < 0:
        return 0
    src = r.cascade(prev_slot, q)
    old = r.texture(prev_slot, q).cpu().numpy()
    spans = r.spans(slot, c).cpu().numpy()
    if info.texel_ladder:
        di, dj = info.snap_x - src.snap_x, info.snap_y - src.snap_y
    else:
        di = dj = 0
    n = 0
    for j in range(info.N):
        lo, hi = spans[j]
        if hi < lo or not (0 <= j + dj < src.N):
            continue
        i = np.arange(lo, hi + 1)
        pi = i + di
        ok = (pi >= 0) & (pi < src.N)
        n += int(np.sum(old[j + dj, pi[ok]] != -np.inf))
    return n


def _run_flight(torch_cuda, scene, cams, water_depth=None, precision=0, check_rays=True, kernel=0,
                follow=False):
    """Frames k in slots k % 2, each reusing the other slot; every frame is
    also discretized afresh in slot 2 (with `follow`, both fitted with
    hysteresis against the previous frame's slot).  Returns the carried-over
    fraction."""
    from paper_2201_10887_gb300 import Renderer
    r = Renderer(scene.tree, scene.sigma, scene.radius, precision=precision, water=water_depth is not None,
                 kernel=kernel)
    if water_depth is not None:
        r.update_water(water_depth)
    reused = visible = 0
    for k, cam in enumerate(cams):
        slot, prev = k % 2, (k + 1) % 2
        fol = prev if (k and follow) else None
        t2, hit2 = r.render(cam, slot=2, follow=fol)
        t, hit = r.render(cam, slot=slot, reuse_from=prev if k else None, follow=fol)
        r.sync()
        st = r.stats(slot)
        for c in range(cam.n_cascades):
            a, b = r.texture(slot, c), r.texture(2, c)
            assert torch_cuda.equal(_bits(a), _bits(b)), (k, c)
            if water_depth is not None:
                assert torch_cuda.equal(_bits(r.water_texture(slot, c)), _bits(r.water_texture(2, c))), (k, c)
            assert torch_cuda.equal(_bits(r.mip(slot, c)), _bits(r.mip(2, c))), (k, c)
            exp = _expected_reuse(r, slot, prev, c) if k else 0
            assert st["reused_texels"][c] == exp, (k, c, st["reused_texels"][c], exp)
            if k == 0:
                assert r.cascade(slot, c).reuse_source == -1
        if check_rays:
            assert torch_cuda.equal(_bits(t), _bits(t2)) and torch_cuda.equal(hit, hit2), k
        if k:
            reused += sum(st["reused_texels"])
            visible += sum(st["visible_texels"])
    r.close()
    return reused / max(visible, 1)


def test_lattice_fit_frames_match_oracle(orc, torch_cuda, tiny):
    """Frames fitted on the texel lattice pass the same parity rules as the
    stable fit's (heights, mask, max mip, rays)."""
    from test_gpu_parity import _frame_parity
    base = tiny.cameras[0]
    for cam in (base.with_(texel_ladder=4),
                base.with_(texel_ladder=1, n_cascades=3, cascade_size=200, split_lambda=0.7),
                base.with_(texel_ladder=3, n_cascades=2, cascade_size=131, width=197, height=143,
                           forward=(0.3, 0.9, -0.35))):
        _frame_parity(orc, torch_cuda, tiny, cam)


@pytest.mark.parametrize("ladder", [1, 4])
def test_reuse_equals_fresh(torch_cuda, tiny, ladder):
    """A moving, turning camera: every frame built with reuse equals the same
    frame computed afresh (textures, mipmaps, rays), and most texels carry
    over."""
    cams = _flight(tiny.cameras[0], 6, ladder=ladder, n_cascades=3, cascade_size=192)
    frac = _run_flight(torch_cuda, tiny, cams)
    assert frac > 0.5, frac


def test_reuse_stable_fit_unchanged(torch_cuda, tiny):
    """With the paper's stable fit texels carry over only between identical
    fits: a camera that turns in place by a hair keeps its fit."""
    cams = _flight(tiny.cameras[0], 3, step=(0.0, 0.0), yaw_deg=0.01, ladder=0, n_cascades=2,
                   cascade_size=160)
    frac = _run_flight(torch_cuda, tiny, cams)
    assert frac > 0.9, frac


def test_reuse_water_layer(torch_cuda):
    """Terrain and water surface textures both carry over."""
    import workloads
    s = workloads.tiny_flood_config()
    cams = _flight(s.cameras[0], 4, ladder=2, n_cascades=2, cascade_size=160)
    assert _run_flight(torch_cuda, s, cams, water_depth=s.depth) > 0.5


def test_reuse_long_jumps_and_wendland(torch_cuda, tiny):
    """Long jumps and turns: one cascade finds a source, the other not, most
    texels are computed; the Wendland kernel carries over too."""
    cams = _flight(tiny.cameras[0], 4, step=(120.0, 0.0), yaw_deg=45.0, ladder=4, n_cascades=2, cascade_size=160)
    _run_flight(torch_cuda, tiny, cams)
    _run_flight(torch_cuda, tiny, _flight(tiny.cameras[0], 3, ladder=2, n_cascades=2, cascade_size=128), kernel=1)


def test_reuse_after_water_update(torch_cuda):
    """New water depths invalidate the earlier frame's texels as new terrain
    values do: nothing carries over, and the frame equals a fresh one."""
    import workloads
    from paper_2201_10887_gb300 import Renderer
    s = workloads.tiny_flood_config()
    cams = _flight(s.cameras[0], 2, ladder=4, n_cascades=2, cascade_size=128)
    r = Renderer(s.tree, s.sigma, s.radius, water=True)
    r.update_water(s.depth)
    r.render(cams[0], slot=0)
    r.update_water((s.depth * 1.5).astype(np.float32))
    r.render(cams[1], slot=1, reuse_from=0)
    r.render(cams[1], slot=2)
    r.sync()
    for c in range(2):
        assert r.cascade(1, c).reuse_source == -1
        assert torch_cuda.equal(_bits(r.texture(1, c)), _bits(r.texture(2, c)))
        assert torch_cuda.equal(_bits(r.water_texture(1, c)), _bits(r.water_texture(2, c)))
    r.close()


def test_reuse_fp16(torch_cuda, tiny):
    from paper_2201_10887_gb300 import hf
    cams = _flight(tiny.cameras[0], 4, ladder=4, n_cascades=2, cascade_size=160)
    assert _run_flight(torch_cuda, tiny, cams, precision=hf.HF_PREC_FP16) > 0.5


def test_reuse_with_fit_hysteresis(torch_cuda, tiny):
    """A camera climbing and sinking every frame: fits that follow the
    previous frame keep its texel sizes where one ladder step allows, frames
    still equal fresh ones fitted the same way, and at least as many texels
    carry over as without hysteresis."""
    base = tiny.cameras[0]
    cams = []
    for k, c in enumerate(_flight(base, 8, step=(6.0, 4.0), yaw_deg=0.5, ladder=8, n_cascades=3, cascade_size=160)):
        cams.append(c.with_(eye=(c.eye[0], c.eye[1], c.eye[2] + (25.0 if k % 2 else -25.0))))
    plain = _run_flight(torch_cuda, tiny, cams)
    held = _run_flight(torch_cuda, tiny, cams, follow=True)
    assert held >= plain and held > 0.3, (plain, held)


def test_reuse_rules(torch_cuda, tiny):
    """Nothing carries over across a change of the leaf data, between
    different spacings, or from a slot whose camera was reset; a slot cannot
    reuse itself or a slot sharing its buffer."""
    from paper_2201_10887_gb300 import Renderer, hf
    cams = _flight(tiny.cameras[0], 2, ladder=4, n_cascades=2, cascade_size=160)
    r = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    r.render(cams[0], slot=0)
    r.update_values((tiny.tree.value + 1.0).astype(np.float32))
    r.render(cams[1], slot=1, reuse_from=0)
    r.render(cams[1], slot=2)
    r.sync()
    for c in range(2):
        assert r.cascade(1, c).reuse_source == -1
        assert torch_cuda.equal(_bits(r.texture(1, c)), _bits(r.texture(2, c)))
    # another cascade size: with one ladder step per octave the spacing stays,
    # the earlier frame's window is smaller than the new one
    a, b = cams[0].with_(texel_ladder=1, cascade_size=150), cams[1].with_(texel_ladder=1)
    r.render(a, slot=0)
    r.render(b, slot=1, reuse_from=0)
    r.render(b, slot=2)
    r.sync()
    assert any(r.cascade(1, c).reuse_source >= 0 for c in range(2))
    for c in range(2):
        assert torch_cuda.equal(_bits(r.texture(1, c)), _bits(r.texture(2, c)))
    # another ladder: nothing carried over
    r.render(cams[0].with_(texel_ladder=1), slot=0)
    r.render(cams[1], slot=1, reuse_from=0)
    r.sync()
    assert all(r.cascade(1, c).reuse_source == -1 for c in range(2))
    with pytest.raises(hf.HFError) as e:
        r.discretize(1, reuse_from=1)
    assert e.value.code == hf.HF_ERR_ARG
    r.set_camera(cams[0], slot=0)        # camera set again: its textures are stale
    with pytest.raises(hf.HFError) as e:
        r.discretize(1, reuse_from=0)
    assert e.value.code == hf.HF_ERR_STATE
    with pytest.raises(hf.HFError) as e:
        r.discretize(1, reuse_from=7)    # never used
    assert e.value.code == hf.HF_ERR_STATE
    v = r.views[1]
    r.bind_view(3, cams[1], v["buf"], v["t"], v["hit"])  # slot 3 shares slot 1's buffer
    with pytest.raises(hf.HFError) as e:
        r.discretize(3, reuse_from=1)
    assert e.value.code == hf.HF_ERR_ARG
    r.close()


def test_reuse_dem_flight(torch_cuda):
    """The DEM flight slowed to ~10 m per frame, on the lattice fit: at full
    size (4 x 2048^2 cascades) frames built with reuse equal fresh ones."""
    import workloads
    s = workloads.dem_config(n_frames=12000)
    cams = [c.with_(texel_ladder=4) for c in s.cameras[600:604]]
    frac = _run_flight(torch_cuda, s, cams, check_rays=False)
    assert frac > 0.8, frac


@pytest.mark.parametrize("seed", range(6))
def test_reuse_random_flights(torch_cuda, tiny, seed):
    """Seeded random flights (step, turn, ladder, cascade count and size,
    with or without hysteresis): every frame equals a fresh one bit for bit
    and the carried-over counts match the host's count."""
    rng = np.random.default_rng(900 + seed)
    cams = _flight(tiny.cameras[0], 4, step=(float(rng.uniform(-30, 30)), float(rng.uniform(-30, 30))),
                   yaw_deg=float(rng.uniform(-3, 3)), ladder=int(rng.choice([1, 2, 4, 8])),
                   n_cascades=int(rng.integers(1, 5)), cascade_size=int(rng.integers(40, 200)))
    _run_flight(torch_cuda, tiny, cams, follow=bool(seed % 2))

"""Reduced-precision discretization (FP16x2 / BF16x2 distance, scale and exp,
FP32 sums) against the FP64 oracle, with the error bound stated up front.

Each weight carries about eight roundings of the 16-bit type (offset, square,
sum, scale, exp2, subtraction of the truncation constant), so its relative
error is at most eps_w ~ 8 u (u = 2^-11 for FP16, 2^-8 for BF16).  The height
error is then at most eps_w times the spread of the values inside a stencil,
which is below 100 m for these terrains; relative to the amplitude A:
    FP16: |dv| <= 2.5e-4 A        BF16: |dv| <= 2e-3 A.
Ray hits move with the heights; their error is reported, and hit/miss may
differ only at silhouettes and where heights moved.
"""

import numpy as np
import pytest

from _parity import RC, check_rays, height_error, mask_from_spans, ocas

pytestmark = pytest.mark.gpu

BOUNDS = {1: 2.5e-4, 2: 2e-3}   # HF_PREC_FP16, HF_PREC_BF16
NAMES = {1: "fp16", 2: "bf16"}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _frame(orc, scene, cam, precision):
    from paper_2201_10887_gb300 import Renderer
    r = Renderer(scene.tree, scene.sigma, scene.radius, precision=precision)
    t, hit = r.render(cam)
    r.sync()
    cells = orc.Cells(scene.tree)
    amp = float(np.abs(cells.cv).max())
    worst, texs, rcs, otexs = 0.0, [], [], []
    for c in range(cam.n_cascades):
        info = r.cascade(0, c)
        tex = r.texture(0, c).cpu().numpy()
        assert np.array_equal(np.isfinite(tex), mask_from_spans(r.spans(0, c).cpu().numpy(), info.N))
        ref = orc.texel_heights(ocas(orc, info), cells, scene.sigma, scene.radius).reshape(info.N, info.N)
        both = np.isfinite(tex) & np.isfinite(ref)
        worst = max(worst, height_error(np.where(both, tex, -np.inf), np.where(both, ref, -np.inf), amp))
        assert np.array_equal(r.mip(0, c).cpu().numpy(), orc.maxmip(tex))
        texs.append(tex)
        otexs.append(np.where(np.isfinite(ref), ref, -np.inf).astype(np.float32))
        rcs.append(RC(info))
    # ray-hit error against the oracle's own frame (oracle heights, oracle rays)
    ot, oh, seg, _ = orc.raycast(cam, scene.tree, rcs, otexs)
    frac, _, terr, errs = check_rays(t.cpu().numpy(), hit.cpu().numpy(), ot, oh, seg)
    r.close()
    return worst, frac, terr, errs


@pytest.mark.parametrize("precision", [1, 2])
def test_tiny_reduced_precision(orc, torch_cuda, tiny, precision):
    cam = tiny.cameras[0].with_(n_cascades=3, cascade_size=192, split_lambda=0.5)
    worst, frac, terr, errs = _frame(orc, tiny, cam, precision)
    print(f"{NAMES[precision]} tiny: height error {worst:.2e} A, hit mismatch {frac:.2e}, "
          f"t error median {np.median(errs):.2e} max {terr:.2e} of segment")
    assert worst <= BOUNDS[precision]
    assert frac <= 0.01


@pytest.mark.parametrize("precision", [1, 2])
def test_far_origin_reduced_precision(orc, torch_cuda, precision):
    """The precision workload: world origin at (5e6, 5e6) m."""
    import workloads
    s = workloads.precision_config()
    cam = s.cameras[0].with_(n_cascades=2, cascade_size=256)
    worst, frac, terr, errs = _frame(orc, s, cam, precision)
    print(f"{NAMES[precision]} far origin: height error {worst:.2e} A, hit mismatch {frac:.2e}, "
          f"t error median {np.median(errs):.2e} max {terr:.2e} of segment")
    assert worst <= BOUNDS[precision]
    assert frac <= 0.01


@pytest.mark.slow
def test_dem_fp16_sampled(orc, torch_cuda):
    import workloads
    from paper_2201_10887_gb300 import Renderer
    s = workloads.dem_config(n_frames=120)
    cam = s.cameras[30]
    r = Renderer(s.tree, s.sigma, s.radius, precision=1)
    r.render(cam)
    r.sync()
    cells = orc.Cells(s.tree)
    amp = float(np.abs(cells.cv).max())
    rng = np.random.default_rng(3)
    worst = 0.0
    for c in range(cam.n_cascades):
        info = r.cascade(0, c)
        tex = r.texture(0, c).cpu().numpy()
        jj, ii = np.nonzero(np.isfinite(tex))
        pick = rng.choice(jj.size, size=min(3000, jj.size), replace=False)
        ref = orc.texel_heights(ocas(orc, info), cells, s.sigma, s.radius, ii[pick], jj[pick])
        ok = np.isfinite(ref)
        got = tex[jj[pick], ii[pick]]
        worst = max(worst, float(np.max(np.abs(got[ok] - ref[ok]) / np.maximum(np.abs(ref[ok]), amp))))
    print(f"fp16 dem: height error {worst:.2e} A")
    assert worst <= BOUNDS[1]
    r.close()

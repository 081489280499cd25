"""Reduced-precision discretization (FP16x2 / BF16x2 distance, scale and exp,
FP32 sums) against the FP64 oracle, with the error bounds stated up front.

Heights.  Each weight carries about eight roundings of the 16-bit type
(offset, square, sum, scale, exp2, subtraction of the truncation constant),
so its relative error is at most eps_w ~ 8 u (u = 2^-11 for FP16, 2^-8 for
BF16).  The height error is then at most eps_w times the spread of the values
inside a stencil, which is below 100 m for these terrains; relative to the
amplitude A:
    FP16: |dv| <= 2.5e-4 A        BF16: |dv| <= 2e-3 A.

Rays.  The rendered frame is compared with the oracle's own frame (oracle
heights, oracle rays) under the FP32 path's ray rules: t within 1e-4 of the
first-hit cascade's segment, hit/miss differences at most 0.1 % of the pixels
and only at silhouettes.  A pixel outside them passes by backward error only
if the oracle's frame on surfaces raised and lowered by the height bound above
(plus the FP32 grazing allowance) brackets it; a ray that meets the surface at
a shallow angle moves by dv / sin(angle), so this is the height bound carried
to the hit.  At most RAY_EXCUSE of the pixels may pass that way.
"""

import numpy as np
import pytest

from _parity import (EXCUSE_REL, GRAZE_REL, HEIGHT_REL, HIT_MISMATCH, RAY_REL, RC, bracketed, check_rays,
                     excuse_cap, height_error, mask_from_spans, ocas)

pytestmark = pytest.mark.gpu

BOUNDS = {0: HEIGHT_REL, 1: 2.5e-4, 2: 2e-3}   # HF_PREC_FP32 / FP16 / BF16: height error / A
# share of pixels the height-bound bracket may pass: FP32 as in the frame
# parity tests; FP16 and BF16 measured at most 5.7e-4 and 2.9e-2 on the
# frames below (BF16's 8-bit mantissa moves a few per cent of the hits by
# more than 1e-4 of their segment)
RAY_EXCUSE = {0: EXCUSE_REL, 1: 2e-3, 2: 5e-2}
NAMES = {0: "fp32", 1: "fp16", 2: "bf16"}


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
        spans = r.spans(0, c).cpu().numpy()
        assert np.array_equal(np.isfinite(tex), mask_from_spans(spans, info.N))
        ref = orc.texel_heights(ocas(orc, info), cells, scene.sigma, scene.radius).reshape(info.N, info.N)
        _, margin = orc.mask(ocas(orc, info), cells)
        worst = max(worst, height_error(tex, ref, amp, exempt=margin.reshape(info.N, info.N) <= 1e-7))
        assert np.array_equal(r.mip(0, c).cpu().numpy(), orc.maxmip(tex))
        texs.append(tex)
        otexs.append(np.where(np.isfinite(ref), ref, -np.inf).astype(np.float32))
        rcs.append(RC(info))
    # ray-hit error against the oracle's own frame (oracle heights, oracle rays)
    ot, oh, seg, _ = orc.raycast(cam, scene.tree, rcs, otexs)
    gt, gh = t.cpu().numpy().ravel(), hit.cpu().numpy().ravel()

    def bracket(idx):   # the oracle's frame on surfaces moved by the height bound
        px, py = (idx % cam.width).astype(np.int32), (idx // cam.width).astype(np.int32)
        tmax = np.nanmax(np.concatenate([np.where(gh[idx] > 0, gt[idx], np.nan), ot[idx], [0.0]]))
        d = np.float32(BOUNDS[precision] * amp + GRAZE_REL * (tmax + amp))
        up = [np.where(np.isfinite(x), x + d, x).astype(np.float32) for x in otexs]
        dn = [np.where(np.isfinite(x), x - d, x).astype(np.float32) for x in otexs]
        tu, hu, _, _ = orc.raycast(cam, scene.tree, rcs, up, pixels=(px, py))
        td, hd, _, _ = orc.raycast(cam, scene.tree, rcs, dn, pixels=(px, py))
        return bracketed(gt[idx], gh[idx], seg[idx], tu, hu, td, hd)
    res = check_rays(gt, gh, ot, oh, seg, shape=(cam.height, cam.width), bracket=bracket)
    r.close()
    return worst, res


def _report_and_check(what, precision, worst, res):
    errs = res.errs
    print(f"{NAMES[precision]} {what}: height error {worst:.2e} A (bound {BOUNDS[precision]:.1e}); rays: "
          f"hit/miss differ {res.frac:.2e}, off-silhouette {res.off}, t error median {np.median(errs):.2e} "
          f"p99 {np.percentile(errs, 99):.2e} of segment, worst outside the bracket {res.terr:.2e}, "
          f"passed by the height-bound bracket {res.excused} of {res.n}")
    assert worst <= BOUNDS[precision]
    assert res.frac <= HIT_MISMATCH and res.off == 0, (res.frac, res.off)
    assert res.terr <= RAY_REL, res.terr
    assert res.excused <= excuse_cap(res.n, RAY_EXCUSE[precision]), (res.excused, res.n)


@pytest.mark.parametrize("precision", [1, 2])
def test_tiny_reduced_precision(orc, torch_cuda, tiny, precision):
    cam = tiny.cameras[0].with_(n_cascades=3, cascade_size=192, split_lambda=0.5)
    worst, res = _frame(orc, tiny, cam, precision)
    _report_and_check("tiny", precision, worst, res)


@pytest.mark.parametrize("precision", [1, 2])
def test_far_origin_reduced_precision(orc, torch_cuda, precision):
    """The precision workload: world origin at (5e6, 5e6) m."""
    import workloads
    s = workloads.precision_config()
    cam = s.cameras[0].with_(n_cascades=2, cascade_size=256)
    worst, res = _frame(orc, s, cam, precision)
    _report_and_check("far origin", precision, worst, res)


@pytest.mark.slow
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_dem_reduced_precision_frame(orc, torch_cuda, precision):
    """A DEM frame (4.5 M leaves, frame 30 of the flight) with the cascades
    and the image scaled down (four 384^2 cascades, 480 x 270) so that the
    oracle computes every texel: the full height and ray rules above, for the
    FP32 path too, side by side."""
    import workloads
    s = workloads.dem_config(n_frames=120)
    cam = s.cameras[30].with_(cascade_size=384, width=480, height=270)
    worst, res = _frame(orc, s, cam, precision)
    _report_and_check("dem frame 30 (4 x 384^2, 480x270)", precision, worst, res)


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

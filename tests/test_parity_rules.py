"""The ray comparison rules of the GPU parity tests, checked on the CPU with
the oracle alone: a result computed on a surface perturbed by less than the
grazing allowance must pass (and does engage the allowance on a low, flat
view), one computed on a surface moved a few times beyond it must fail.
This keeps the backward-error rule from forgiving real errors."""

import numpy as np
import pytest

from _parity import GRAZE_REL, RAY_REL, RC, check_rays, frame_bracket


def _frame(orc, tiny, pitch, height_above):
    from workloads.cameras import fixed_camera
    cam = fixed_camera(tiny.tree, tiny.fbm, (320.0, 80.0), height_above, 90.0, pitch, 60.0, 320, 240,
                       n_cascades=2, cascade_size=192, znear=1.0, zfar=1.0e4)
    cells = orc.Cells(tiny.tree)
    view = orc.fit(cam, tiny.tree, cells)
    texs, rcs = [], []
    for c in range(cam.n_cascades):
        cas = view.cas[c]
        vis, _ = orc.mask(cas, cells)
        vis = vis.reshape(cas.N, cas.N).astype(bool)
        tex = tiny.fbm.grid(cas.ox + np.arange(cas.N) * cas.h, cas.oy + np.arange(cas.N) * cas.h).astype(np.float32)
        tex[~vis] = -np.inf
        texs.append(tex)
        rcs.append(RC(type("I", (), dict(ox=cas.ox, oy=cas.oy, texel=cas.h, near=cas.near,
                                         far_ext=cas.far_ext, N=cas.N))))
    return cam, texs, rcs, float(np.abs(cells.cv).max())


def _check(orc, tiny, cam, texs, rcs, amp, shift):
    ot, oh, seg, _ = orc.raycast(cam, tiny.tree, rcs, texs)
    moved = [np.where(np.isfinite(t), t + np.float32(shift), t).astype(np.float32) for t in texs]
    gt, gh, _, _ = orc.raycast(cam, tiny.tree, rcs, moved)
    engaged = []
    br = frame_bracket(orc, cam, tiny.tree, rcs, texs, gt, gh, ot, seg, amp)

    def bracket(idx):
        ok = br(idx)
        engaged.append(int(ok.sum()))
        return ok
    res = check_rays(gt, gh, ot, oh, seg, shape=(cam.height, cam.width), bracket=bracket)
    return res.off, res.terr, res.errs, sum(engaged)


@pytest.mark.parametrize("pitch,height_above", [(-30.0, 300.0), (-3.0, 30.0)])
def test_perturbation_within_allowance_is_explained(orc, tiny, pitch, height_above):
    cam, texs, rcs, amp = _frame(orc, tiny, pitch, height_above)
    off, terr, errs, explained = _check(orc, tiny, cam, texs, rcs, amp, 0.5 * GRAZE_REL * amp)
    assert off == 0 and terr <= RAY_REL, (off, terr)
    assert explained >= 1      # grazing pixels exist and are forgiven only by the rule


@pytest.mark.parametrize("shift", [0.1, 2.0])
def test_perturbation_beyond_allowance_fails(orc, tiny, shift):
    cam, texs, rcs, amp = _frame(orc, tiny, -3.0, 30.0)
    assert shift > 3 * GRAZE_REL * (amp + 1.0e4)       # several times delta for any t in the view
    off, terr, errs, _ = _check(orc, tiny, cam, texs, rcs, amp, shift)
    assert terr > RAY_REL, terr
    assert np.mean(errs > RAY_REL) > 0.01

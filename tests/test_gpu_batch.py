"""Batched frames: many views of several heightfields (different sizes,
cascade counts, texture sizes, images, precisions) in one persistent launch
must reproduce the per-view calls bit for bit, for every work-unit shape, and
through a captured CUDA graph replayed with new cameras."""

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


def _scenes():
    import workloads
    tiles = workloads.batch_config(seed=9, n_tiles=4, min_side=128, max_side=512, width=200, height=120)
    tiny = workloads.tiny_config()
    return tiles, tiny


def _setup(torch_cuda):
    from paper_2201_10887_gb300 import Renderer
    tiles, tiny = _scenes()
    views, cams = [], []
    for k, sc in enumerate(tiles):
        r = Renderer(sc.tree, sc.sigma, sc.radius, precision=1 if k == 1 else 0)
        cam = sc.cameras[0].with_(cascade_size=min(sc.cameras[0].cascade_size, 512))
        views.append((r, 0))
        cams.append(cam)
    rt = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    for slot, cam in enumerate([tiny.cameras[0].with_(n_cascades=3, cascade_size=160, width=97, height=61),
                                tiny.cameras[0].with_(n_cascades=2, cascade_size=100, forward=(0.4, 0.9, -0.5)),
                                tiny.cameras[0].with_(n_cascades=2, cascade_size=120, texel_ladder=4),
                                tiny.cameras[0].with_(n_cascades=3, cascade_size=128, lod_pixels=16.0)]):
        views.append((rt, slot))
        cams.append(cam)
    return views, cams


def _reference(views, cams):
    ref = []
    for (r, slot), cam in zip(views, cams):
        t, hit = r.render(cam, slot=slot)
        r.sync()
        texs = [r.texture(slot, c).cpu().numpy().copy() for c in range(cam.n_cascades)]
        mips = [r.mip(slot, c).cpu().numpy().copy() for c in range(cam.n_cascades)]
        ref.append((t.cpu().numpy().copy(), hit.cpu().numpy().copy(), texs, mips))
    return ref


def _clear(views, cams):
    for (r, slot), cam in zip(views, cams):
        v = r.views[slot]
        v["t"].fill_(-7.0)
        v["hit"].fill_(255)
        for c in range(cam.n_cascades):
            r.texture(slot, c).fill_(-7.0)
            r.mip(slot, c).fill_(-7.0)


def _check(batch, views, cams, ref):
    for k, ((r, slot), cam) in enumerate(zip(views, cams)):
        t, hit = batch.outputs(k)
        rt, rh, rtex, rmip = ref[k]
        assert np.array_equal(hit.cpu().numpy(), rh), k
        assert np.array_equal(t.cpu().numpy(), rt, equal_nan=True), k
        for c in range(cam.n_cascades):
            assert np.array_equal(r.texture(slot, c).cpu().numpy(), rtex[c]), (k, c)
            assert np.array_equal(r.mip(slot, c).cpu().numpy(), rmip[c]), (k, c)


def test_batch_equals_per_view_calls_for_every_shape(torch_cuda):
    from paper_2201_10887_gb300 import Batch
    from paper_2201_10887_gb300.batch import flag_candidates
    views, cams = _setup(torch_cuda)
    ref = _reference(views, cams)
    batch = Batch(views)
    for flags in flag_candidates():
        _clear(views, cams)
        batch.prepare(flags)
        batch.launch()
        for r, _ in views:
            r.sync()
        _check(batch, views, cams, ref)


def test_batch_graph_replay_with_new_cameras(torch_cuda):
    from paper_2201_10887_gb300 import Batch
    views, cams = _setup(torch_cuda)
    for r_slot, cam in zip(views, cams):
        r_slot[0].set_camera(cam, r_slot[1])
    batch = Batch(views)
    batch.capture()
    for step in range(3):
        moved = [c.with_(eye=(c.eye[0] + 17.0 * step, c.eye[1] - 9.0 * step, c.eye[2] + 5.0 * step))
                 for c in cams]
        ref = _reference(views, moved)
        _clear(views, moved)
        for (r, slot), cam in zip(views, moved):
            r.set_camera(cam, slot)
        batch.run()
        torch_cuda.cuda.synchronize()
        for r, _ in views:
            r.sync()
        _check(batch, views, moved, ref)


def test_autotune_picks_a_valid_shape(torch_cuda):
    from paper_2201_10887_gb300 import Batch, autotune
    from paper_2201_10887_gb300.batch import flag_candidates
    views, cams = _setup(torch_cuda)
    for (r, slot), cam in zip(views, cams):
        r.set_camera(cam, slot)
    batch = Batch(views)
    best, times = autotune(batch, reps=2)
    assert best in flag_candidates() and len(times) == len(flag_candidates())
    assert all(v > 0 for v in times.values())
    for r, _ in views:
        r.sync()


def test_batch_with_many_items_and_cascades(torch_cuda):
    """More than 32 items and 32 cascades, so that each CTA's warp-wide search
    for its item or cascade takes more than one round: every shape still
    reproduces the per-view calls bit for bit."""
    import math
    from paper_2201_10887_gb300 import Batch, Renderer
    from paper_2201_10887_gb300.batch import flag_candidates
    tiny = _scenes()[1]
    r = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    views, cams = [], []
    rng = np.random.default_rng(31)
    for slot in range(41):
        yaw = math.radians(90.0 + rng.uniform(-40, 40))
        pitch = math.radians(rng.uniform(-50, -20))
        fwd = (math.cos(pitch) * math.cos(yaw), math.cos(pitch) * math.sin(yaw), math.sin(pitch))
        cams.append(tiny.cameras[0].with_(forward=fwd, n_cascades=int(rng.integers(1, 4)),
                                          cascade_size=int(rng.integers(33, 97)),
                                          width=int(rng.integers(16, 48)), height=int(rng.integers(12, 40))))
        views.append((r, slot))
    assert len(views) > 32 and sum(c.n_cascades for c in cams) > 32
    ref = _reference(views, cams)
    batch = Batch(views)
    for flags in flag_candidates():
        _clear(views, cams)
        batch.prepare(flags)
        batch.launch()
        r.sync()
        _check(batch, views, cams, ref)
    r.close()

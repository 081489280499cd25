"""Randomised GPU parity: seeded random cameras over the tiny scene (pose,
field of view, cascade count and size, image size, split, overlap, lattice
fit, coarse-level stop), each frame checked against the oracle with the full
rules of test_gpu_parity (mask, heights, max mip, every ray)."""

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


@pytest.mark.parametrize("seed", range(40))
def test_random_camera_frame(orc, torch_cuda, tiny, seed):
    from test_gpu_parity import _frame_parity
    rng = np.random.default_rng(100 + seed)
    t = tiny.tree
    gx, gy = rng.uniform(120, 520), rng.uniform(120, 520)
    eye = (t.origin_x + gx, t.origin_y + gy, float(tiny.fbm(gx, gy)) + rng.uniform(100, 500))  # above the ground
    yaw = math.atan2(320.0 - gy, 320.0 - gx) + rng.uniform(-0.6, 0.6)    # roughly toward the domain's centre
    pitch = rng.uniform(-1.2, -0.35)
    fwd = (math.cos(pitch) * math.cos(yaw), math.cos(pitch) * math.sin(yaw), math.sin(pitch))
    cam = tiny.cameras[0].with_(eye=eye, forward=fwd, vfov=rng.uniform(0.6, 1.3),
                                n_cascades=int(rng.integers(1, 5)), cascade_size=int(rng.integers(33, 300)),
                                width=int(rng.integers(40, 200)), height=int(rng.integers(40, 160)),
                                split_lambda=float(rng.uniform(0, 1)), overlap_frac=float(rng.uniform(0, 0.15)),
                                texel_ladder=int(rng.choice([0, 0, 1, 4])),
                                lod_pixels=float(rng.choice([0.0, 0.0, 4.0, 16.0])))
    worst, terr, hits = _frame_parity(orc, torch_cuda, tiny, cam)
    assert hits > 0, hits


@pytest.mark.parametrize("seed", range(10))
def test_random_camera_water_frame(orc, torch_cuda, seed):
    """The same with the water layer over the tiny flood (lattice fit drawn
    too; the coarse stop is not defined for two surfaces)."""
    import workloads
    from test_gpu_water import _water_frame
    s = workloads.tiny_flood_config()
    rng = np.random.default_rng(500 + seed)
    t = s.tree
    gx, gy = rng.uniform(120, 520), rng.uniform(120, 520)
    eye = (t.origin_x + gx, t.origin_y + gy, float(s.fbm(gx, gy)) + rng.uniform(100, 500))
    yaw = math.atan2(320.0 - gy, 320.0 - gx) + rng.uniform(-0.6, 0.6)
    pitch = rng.uniform(-1.2, -0.35)
    fwd = (math.cos(pitch) * math.cos(yaw), math.cos(pitch) * math.sin(yaw), math.sin(pitch))
    cam = s.cameras[0].with_(eye=eye, forward=fwd, vfov=rng.uniform(0.6, 1.3),
                             n_cascades=int(rng.integers(1, 4)), cascade_size=int(rng.integers(33, 260)),
                             width=int(rng.integers(40, 160)), height=int(rng.integers(40, 120)),
                             split_lambda=float(rng.uniform(0, 1)), overlap_frac=float(rng.uniform(0, 0.15)),
                             texel_ladder=int(rng.choice([0, 0, 2])))
    _water_frame(orc, s, cam, s.depth, seed=seed)

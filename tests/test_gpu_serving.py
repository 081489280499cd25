"""Continuous-batching server: requests of mixed image sizes and cascade
counts, admitted by a device-memory budget, grouped into batched frames on
several streams.  Every result must equal the same view rendered alone, the
budget must hold, and waiting requests must be admitted as memory frees."""

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


def _requests(tiny, n=24, seed=3, span=0.15):
    import workloads
    rng = np.random.default_rng(seed)
    base = tiny.cameras[0]
    reqs = []
    for k in range(n):
        w, h = [(64, 48), (160, 90), (200, 120)][int(rng.integers(0, 3))]
        cam = base.with_(width=w, height=h, n_cascades=int(rng.integers(1, 5)),
                         cascade_size=int(rng.choice([64, 128, 256])),
                         eye=(base.eye[0] + rng.uniform(-60, 60), base.eye[1] + rng.uniform(-40, 40),
                              base.eye[2] + rng.uniform(-50, 50)),
                         forward=(rng.uniform(-0.3, 0.3), 1.0, rng.uniform(-0.8, -0.3)))
        reqs.append(workloads.Request(k, float(k * span / n), cam))
    return reqs


@pytest.mark.parametrize("realtime,host_outputs,single", [(False, True, True), (True, True, True),
                                                          (False, False, True), (True, True, False)])
def test_server_results_equal_single_views(torch_cuda, tiny, realtime, host_outputs, single):
    """Each result equals the view rendered alone, with the ray casts writing
    into pinned host memory or into device memory copied afterwards, and
    groups of one request run through the per-view calls or as a batch."""
    from paper_2201_10887_gb300 import Renderer, Server
    r = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    reqs = _requests(tiny)
    probe = Server(r, 1 << 20, max_slots=1, host_outputs=host_outputs, host_budget=1 << 20)
    sizes = [probe.request_bytes(q.camera) for q in reqs]
    budget = int(2.5 * max(sizes))              # only a few views fit at once
    hbudget = int(3.5 * max(Server.host_bytes(q.camera) for q in reqs))  # and their results
    srv = Server(r, budget, max_slots=6, n_streams=3, max_group=4, keep_results=True,
                 host_outputs=host_outputs, host_budget=hbudget, single_view_calls=single)
    out = srv.run(reqs, realtime=realtime)
    assert out["requests"] == len(reqs) and len(out["results"]) == len(reqs)
    assert out["max_memory_used"] <= budget
    assert out["max_host_memory_used"] <= hbudget
    assert out["p99_ms"] >= out["p50_ms"] > 0
    if not realtime:
        assert out["mean_group"] > 1.0           # requests were batched together
    for q in reqs:                               # each result equals the view rendered alone
        t, hit = r.render(q.camera, slot=200)
        r.sync()
        gt, gh = out["results"][q.rid]
        assert np.array_equal(gh, hit.cpu().numpy().ravel()), q.rid
        assert np.array_equal(gt, t.cpu().numpy().ravel(), equal_nan=True), q.rid
    r.close()


def test_server_rejects_a_request_over_the_budget(torch_cuda, tiny):
    from paper_2201_10887_gb300 import Renderer, Server
    r = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    reqs = _requests(tiny, n=2)
    srv = Server(r, 4096, max_slots=2, host_budget=1 << 20)
    with pytest.raises(ValueError):
        srv.run(reqs, realtime=False)
    r.close()

"""Failure detection without a GPU fault: a bounded device wait on a flag
that nothing sets runs out, the kernel records HF_ERR_TIMEOUT and returns,
hf_sync reports it once, and the context keeps rendering correctly."""

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


def test_bounded_wait_reports_timeout_and_context_survives(torch_cuda, tiny):
    from paper_2201_10887_gb300 import Renderer, hf
    cam = tiny.cameras[0]
    r = Renderer(tiny.tree, tiny.sigma, tiny.radius)
    t0, h0 = r.render(cam)
    r.sync()
    t0, h0 = t0.clone(), h0.clone()
    hf.hf_selftest_wait_timeout(r.ctx, 2000)
    with pytest.raises(hf.HFError) as e:
        r.sync()
    assert e.value.code == hf.HF_ERR_TIMEOUT
    r.sync()                                   # reported once, then cleared
    t1, h1 = r.render(cam)
    r.sync()
    assert torch_cuda.equal(h1, h0)
    assert torch_cuda.equal(torch_cuda.nan_to_num(t1, nan=-1.0), torch_cuda.nan_to_num(t0, nan=-1.0))
    with pytest.raises(hf.HFError) as e:
        hf.hf_selftest_wait_timeout(r.ctx, 0)
    assert e.value.code == hf.HF_ERR_ARG
    r.close()

"""Batched frames: many views of many heightfields in one persistent launch.

``Batch`` holds the descriptor buffers of a fixed set of (renderer, view
slot) pairs: a pinned host buffer that ``hf_batch_prepare`` fills from the
views' current cameras, and a device buffer that ``hf_batch_launch`` copies
it into before running the batch.  Because launch sizes depend only on the
items' cascade counts and texture / image sizes, the launch can be captured
once in a CUDA graph and replayed each frame after ``prepare``.

``autotune`` times the work-unit shapes (ray tile, discretization warp patch,
ray tiles inside or after the persistent launch) on the actual batch and
keeps the fastest.
"""

from __future__ import annotations

import itertools

from . import hf

SHAPE_FLAGS = {
    "ray16x16": 0, "ray32x8": hf.HF_BATCH_RAY_TILE_32x8, "ray8x32": hf.HF_BATCH_RAY_TILE_8x32,
}


MODES = {
    "per-phase launches": 0,
    "persistent launch + ray launch": hf.HF_BATCH_PERSISTENT,
    "one persistent launch": hf.HF_BATCH_PERSISTENT | hf.HF_BATCH_RAYS_INSIDE,
}


def flag_candidates():
    out = []
    for ray, warp, mode in itertools.product(SHAPE_FLAGS.values(), (0, hf.HF_BATCH_WARP_16x2),
                                             MODES.values()):
        out.append(ray | warp | mode)
    return out


def describe(flags: int) -> str:
    ray = {0: "16x16", hf.HF_BATCH_RAY_TILE_32x8: "32x8", hf.HF_BATCH_RAY_TILE_8x32: "8x32"}[
        flags & (hf.HF_BATCH_RAY_TILE_32x8 | hf.HF_BATCH_RAY_TILE_8x32)]
    warp = "16x2" if flags & hf.HF_BATCH_WARP_16x2 else "8x4"
    mode = [k for k, v in MODES.items() if v == flags & (hf.HF_BATCH_PERSISTENT | hf.HF_BATCH_RAYS_INSIDE)][0]
    return f"{mode}, ray tile {ray}, texel warp {warp}"


class Batch:
    """A fixed set of views rendered together.  ``views`` is a list of
    (Renderer, view_slot); their cameras are set with Renderer.set_camera.

    Two pinned descriptor buffers alternate between frames so that the host
    can prepare frame k+1 while the copy of frame k is still pending; before
    a buffer is refilled, the event recorded after its last launch is
    awaited."""

    def __init__(self, views, flags: int = 0):
        import torch
        self.torch = torch
        self.views = list(views)
        self.flags = flags
        self.items = (hf.hf_batch_item * len(self.views))()
        self._bind_items()
        dev_bytes, host_bytes = hf.hf_batch_query_bytes(self.items, flags)
        device = self.views[0][0].device
        self.dev_bufs = [torch.empty(dev_bytes, dtype=torch.uint8, device=device) for _ in range(2)]
        self.host_bufs = [torch.empty(host_bytes, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
        self.events = [None, None]
        self.graphs = None
        self.cur = 0

    @property
    def host_buf(self):
        return self.host_bufs[self.cur]

    @property
    def dev_buf(self):
        return self.dev_bufs[self.cur]

    def _bind_items(self):
        for k, (r, slot) in enumerate(self.views):
            v = r.views[slot]
            self.items[k] = hf.hf_batch_item(r.ctx.value, slot, 0, v["t"].data_ptr(), v["hit"].data_ptr())

    def prepare(self, flags: int | None = None):
        """Fill the next descriptor buffer from the views' current cameras."""
        if flags is not None and flags != self.flags:
            self.flags = flags
            self.graphs = None
        self.cur ^= 1
        if self.events[self.cur] is not None:
            self.events[self.cur].synchronize()
        hf.hf_batch_prepare(self.items, self.flags, self.host_bufs[self.cur])

    def launch(self, stream=None):
        torch = self.torch
        if self.graphs is not None:
            self.graphs[self.cur].replay()
        else:
            hf.hf_batch_launch(self.host_bufs[self.cur], self.dev_bufs[self.cur], stream)
        ev = torch.cuda.Event()
        ev.record(stream if stream is not None else torch.cuda.current_stream())
        self.events[self.cur] = ev

    def run(self, stream=None):
        """Prepare from the current cameras and run (graph replay if captured)."""
        self.prepare()
        self.launch(stream)

    def capture(self):
        """Capture the launch of each descriptor buffer (copy, counter reset,
        kernels) in a CUDA graph; later ``launch`` / ``run`` calls replay."""
        torch = self.torch
        self.graphs = None
        graphs = []
        for b in range(2):
            self.prepare()
            hf.hf_batch_launch(self.host_bufs[self.cur], self.dev_bufs[self.cur])  # warm-up
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                with torch.cuda.graph(g, stream=s):
                    hf.hf_batch_launch(self.host_bufs[self.cur], self.dev_bufs[self.cur], s)
            torch.cuda.current_stream().wait_stream(s)
            graphs.append((self.cur, g))
        self.graphs = [None, None]
        for b, g in graphs:
            self.graphs[b] = g
        torch.cuda.synchronize()
        return self.graphs

    def outputs(self, k: int):
        r, slot = self.views[k]
        v = r.views[slot]
        return v["t"].view(v["shape"]), v["hit"].view(v["shape"])


def autotune(batch: Batch, candidates=None, reps: int = 3):
    """Time each flag combination (prepare + launch, CUDA events, best of
    `reps`) and leave the batch set to the fastest.  Returns (best flags,
    {flags: ms})."""
    torch = batch.torch
    results = {}
    for flags in candidates or flag_candidates():
        batch.prepare(flags)
        batch.launch()
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            batch.prepare(flags)
            a.record()
            batch.launch()
            b.record()
            b.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        results[flags] = best
    best_flags = min(results, key=results.get)
    batch.prepare(best_flags)
    return best_flags, results

"""Convenience wrapper over the C ABI: owns the device buffers of one
quadtree and its view slots, and runs the per-frame sequence
set_camera -> discretize -> max mip -> ray cast.

Device memory comes from PyTorch (uint8 CUDA tensors); the library itself
never allocates.  All computation happens in ``libhf.so``.
"""

from __future__ import annotations

import ctypes as ct

from . import hf


def camera_struct(cam) -> hf.hf_camera:
    """hf_camera from any object with eye, forward, up, vfov, znear, zfar,
    width, height, n_cascades, cascade_size, split_lambda, overlap_frac and
    optionally texel_ladder (0 = the stable fit), lod_pixels (0 = the exact
    surface) and traversal (0 = one level up per step, 1 = climb to the
    coarsest node entered)."""
    return hf.hf_camera((ct.c_double * 3)(*cam.eye), (ct.c_double * 3)(*cam.forward),
                        (ct.c_double * 3)(*cam.up), cam.vfov, cam.znear, cam.zfar, cam.width,
                        cam.height, cam.n_cascades, cam.cascade_size, cam.split_lambda,
                        cam.overlap_frac, int(getattr(cam, "texel_ladder", 0)), int(getattr(cam, "traversal", 0)),
                        float(getattr(cam, "lod_pixels", 0.0)))


class Renderer:
    """One quadtree heightfield on one GPU.

    ``tree`` is any object with origin_x, origin_y, root_cell, root_nx,
    root_ny, max_level and leaf arrays level, ix, iy, value.  With
    ``water=True`` the leaves also carry water depths (``update_water``) and
    every view gets a water surface texture per cascade (the max mipmap then
    bounds both surfaces).  ``kernel`` selects the RBF weight (hf.HF_RBF_*).
    With ``host_outputs`` the ray cast writes ``t`` and ``hit`` straight into
    pinned host tensors (no copy after the frame).
    """

    def __init__(self, tree, sigma: float, radius: float, precision: int = hf.HF_PREC_FP32,
                 bucket_level: int = -1, device=None, stream=None, water: bool = False,
                 kernel: int = hf.HF_RBF_GAUSSIAN, host_outputs: bool = False):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.host_outputs = bool(host_outputs)
        desc = hf.hf_quadtree_desc(tree.origin_x, tree.origin_y, tree.root_cell, tree.root_nx,
                                   tree.root_ny, tree.max_level)
        leaves = hf.leaves_array(tree.level, tree.ix, tree.iy, tree.value)
        rbf = hf.hf_rbf_params(sigma, radius, precision, bucket_level, 1 if water else 0, kernel)
        self.water = bool(water)
        self.ctx = hf.hf_create_quadtree(desc, leaves, rbf)
        self.persistent_bytes, _ = hf.hf_query_bytes(self.ctx, 1, 2)
        self.persistent = torch.empty(self.persistent_bytes, dtype=torch.uint8, device=self.device)
        hf.hf_bind_persistent(self.ctx, self.persistent, stream)
        self.views = {}

    # -- buffers ------------------------------------------------------------
    def view_bytes(self, n_cascades: int, cascade_size: int) -> int:
        return hf.hf_query_bytes(self.ctx, n_cascades, cascade_size)[1]

    def _slot_buffers(self, slot: int, cam):
        need = self.view_bytes(cam.n_cascades, cam.cascade_size)
        v = self.views.get(slot)
        if v is None or v["buf"].numel() < need:
            buf = self.torch.empty(need, dtype=self.torch.uint8, device=self.device)
            v = {"buf": buf}
            self.views[slot] = v
        npx = cam.width * cam.height
        if v.get("npx") != npx:
            if self.host_outputs:
                v["t"] = self.torch.empty(npx, dtype=self.torch.float32, pin_memory=True)
                v["hit"] = self.torch.empty(npx, dtype=self.torch.uint8, pin_memory=True)
            else:
                v["t"] = self.torch.empty(npx, dtype=self.torch.float32, device=self.device)
                v["hit"] = self.torch.empty(npx, dtype=self.torch.uint8, device=self.device)
            v["npx"] = npx
        v["shape"] = (cam.height, cam.width)
        v["C"] = cam.n_cascades
        return v

    def bind_view(self, slot: int, cam, view_buf, t_out, hit_out, follow: int = None):
        """Use caller-provided buffers for a view slot (uint8 view buffer of
        at least view_bytes(), float32 t and uint8 hit of width*height; t and
        hit may be pinned host tensors, which the ray cast then writes
        directly)."""
        need = self.view_bytes(cam.n_cascades, cam.cascade_size)
        npx = cam.width * cam.height
        if view_buf.numel() < need or t_out.numel() < npx or hit_out.numel() < npx:
            raise ValueError("view buffers too small")
        self.views[slot] = {"buf": view_buf, "t": t_out, "hit": hit_out, "npx": npx,
                            "shape": (cam.height, cam.width), "C": cam.n_cascades, "external": True}
        self._fit(slot, cam, view_buf, follow)
        return self.views[slot]

    def _fit(self, slot, cam, buf, follow):
        if follow is None:
            hf.hf_set_camera(self.ctx, slot, camera_struct(cam), buf)
        else:
            hf.hf_set_camera_follow(self.ctx, slot, camera_struct(cam), buf, follow)

    # -- per-frame steps ------------------------------------------------------
    def set_camera(self, cam, slot: int = 0, follow: int = None):
        """Fit `cam` to a view slot; with `follow` (the slot of the previous
        frame) the lattice fit keeps that frame's texel sizes where it can."""
        v = self._slot_buffers(slot, cam)
        self._fit(slot, cam, v["buf"], follow)
        return v

    def discretize(self, slot: int = 0, stream=None, reuse_from: int = None):
        """Step 1 for a view slot; with ``reuse_from`` (another slot holding an
        earlier frame) texels on the same lattice are carried over from it."""
        if reuse_from is None:
            hf.hf_discretize_cascades(self.ctx, slot, stream)
        else:
            hf.hf_discretize_reuse(self.ctx, slot, reuse_from, stream)

    def build_maxmip(self, slot: int = 0, stream=None):
        hf.hf_build_maxmip(self.ctx, slot, stream)

    def raycast(self, slot: int = 0, stream=None):
        v = self.views[slot]
        hf.hf_raycast(self.ctx, slot, v["t"], v["hit"], stream)
        return v["t"].view(v["shape"]), v["hit"].view(v["shape"])

    def render(self, cam=None, slot: int = 0, stream=None, reuse_from: int = None, follow: int = None):
        """One frame; `reuse_from` carries texels over from another slot's
        earlier frame, `follow` fits with hysteresis against a slot's camera."""
        if cam is not None:
            self.set_camera(cam, slot, follow)
        self.discretize(slot, stream, reuse_from)
        self.build_maxmip(slot, stream)
        return self.raycast(slot, stream)

    def update_values(self, values, stream=None):
        hf.hf_update_values(self.ctx, values, stream)

    def update_water(self, depths, stream=None):
        hf.hf_update_water(self.ctx, depths, stream)

    def stats(self, slot: int = 0, stream=None) -> dict:
        return hf.hf_view_stats(self.ctx, slot, self.views[slot]["C"], stream)

    def ray_stats(self, slot: int = 0, stream=None) -> dict:
        return hf.hf_ray_stats(self.ctx, slot, stream)

    def sync(self, stream=None):
        hf.hf_sync(self.ctx, stream)

    # -- inspection -----------------------------------------------------------
    def cascade(self, slot: int, c: int) -> hf.hf_cascade_info:
        return hf.hf_get_cascade(self.ctx, slot, c)

    def _sub(self, slot: int, ptr: int, nbytes: int):
        buf = self.views[slot]["buf"]
        off = ptr - buf.data_ptr()
        return buf[off: off + nbytes]

    def texture(self, slot: int, c: int):
        info = self.cascade(slot, c)
        return self._sub(slot, info.tex, info.N * info.N * 4).view(self.torch.float32).view(info.N, info.N)

    def mip(self, slot: int, c: int):
        info = self.cascade(slot, c)
        return self._sub(slot, info.mip, info.mip_floats * 4).view(self.torch.float32)

    def water_texture(self, slot: int, c: int):
        info = self.cascade(slot, c)
        return self._sub(slot, info.water_tex, info.N * info.N * 4).view(self.torch.float32).view(info.N, info.N)

    def spans(self, slot: int, c: int):
        info = self.cascade(slot, c)
        return self._sub(slot, info.spans, info.N * 8).view(self.torch.int32).view(info.N, 2)

    def close(self):
        if getattr(self, "ctx", None):
            hf.hf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

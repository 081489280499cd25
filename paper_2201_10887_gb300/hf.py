"""Thin ctypes binding of the C ABI in ``include/hf.h`` (same function names).

Only argument marshalling happens here: every step of the method runs in
``libhf.so``.  PyTorch supplies device memory (``uint8`` CUDA tensors) and
streams.  If the library has not been built, importing this module raises.
"""

from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhf.so")

HF_OK, HF_ERR_ARG, HF_ERR_STATE, HF_ERR_NOMEM, HF_ERR_CUDA, HF_ERR_TIMEOUT, HF_ERR_DATA, HF_ERR_HOST = 0, -1, -2, -3, -4, -5, -6, -7
HF_PREC_FP32, HF_PREC_FP16, HF_PREC_BF16 = 0, 1, 2
HF_RBF_GAUSSIAN, HF_RBF_WENDLAND_C2 = 0, 1
HF_MAX_LEVEL, HF_MAX_CASCADES, HF_MAX_POLY, HF_MAX_VIEWS = 15, 8, 32, 256

ERROR_NAMES = {HF_ERR_ARG: "HF_ERR_ARG", HF_ERR_STATE: "HF_ERR_STATE", HF_ERR_NOMEM: "HF_ERR_NOMEM",
               HF_ERR_CUDA: "HF_ERR_CUDA", HF_ERR_TIMEOUT: "HF_ERR_TIMEOUT", HF_ERR_DATA: "HF_ERR_DATA",
               HF_ERR_HOST: "HF_ERR_HOST"}

LEAF_DTYPE = np.dtype([("level", "<i4"), ("ix", "<i4"), ("iy", "<i4"), ("value", "<f4")])

EXPORTED = ["hf_create_quadtree", "hf_query_bytes", "hf_bind_persistent", "hf_update_values",
            "hf_set_camera", "hf_discretize_cascades", "hf_discretize_reuse", "hf_build_maxmip", "hf_raycast",
            "hf_get_cascade", "hf_view_stats", "hf_sync", "hf_destroy", "hf_last_error",
            "hf_discretize_noalloc", "hf_ray_stats", "hf_batch_query_bytes", "hf_batch_prepare",
            "hf_batch_launch", "hf_frame_batch", "hf_update_water", "hf_selftest_wait_timeout",
            "hf_measure_unit_rates", "hf_set_camera_follow"]
HF_BATCH_RAYS_INSIDE, HF_BATCH_RAY_TILE_32x8, HF_BATCH_RAY_TILE_8x32, HF_BATCH_WARP_16x2 = 1, 2, 4, 8
HF_BATCH_PERSISTENT = 16
HF_NOALLOC_SCRATCH_BYTES = 256 * 1024


class HFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class hf_quadtree_desc(ct.Structure):
    _fields_ = [("origin_x", ct.c_double), ("origin_y", ct.c_double), ("root_cell", ct.c_double),
                ("root_nx", ct.c_int32), ("root_ny", ct.c_int32), ("max_level", ct.c_int32)]


class hf_rbf_params(ct.Structure):
    _fields_ = [("sigma", ct.c_double), ("radius", ct.c_double), ("precision", ct.c_int32),
                ("bucket_level", ct.c_int32), ("water", ct.c_int32), ("kernel", ct.c_int32)]


class hf_camera(ct.Structure):
    _fields_ = [("eye", ct.c_double * 3), ("forward", ct.c_double * 3), ("up", ct.c_double * 3),
                ("vfov", ct.c_double), ("znear", ct.c_double), ("zfar", ct.c_double),
                ("width", ct.c_int32), ("height", ct.c_int32), ("n_cascades", ct.c_int32),
                ("cascade_size", ct.c_int32), ("split_lambda", ct.c_double),
                ("overlap_frac", ct.c_double), ("texel_ladder", ct.c_int32), ("traversal", ct.c_int32),
                ("lod_pixels", ct.c_double)]


class hf_cascade_info(ct.Structure):
    _fields_ = [("near_depth", ct.c_double), ("far_depth", ct.c_double), ("far_ext_depth", ct.c_double),
                ("n_poly", ct.c_int32), ("N", ct.c_int32),
                ("poly", (ct.c_double * 2) * HF_MAX_POLY), ("aabb", ct.c_double * 4),
                ("snap_x", ct.c_int64), ("snap_y", ct.c_int64), ("snap_k", ct.c_int64),
                ("ox", ct.c_double), ("oy", ct.c_double), ("extent", ct.c_double),
                ("texel", ct.c_double), ("tex", ct.c_void_p), ("mip", ct.c_void_p),
                ("spans", ct.c_void_p), ("mip_floats", ct.c_int64),
                ("water_tex", ct.c_void_p), ("texel_ladder", ct.c_int32), ("reuse_source", ct.c_int32),
                ("stop_level", ct.c_int32), ("reserved", ct.c_int32)]

    @property
    def near(self) -> float:
        return self.near_depth

    @property
    def far(self) -> float:
        return self.far_depth

    @property
    def far_ext(self) -> float:
        return self.far_ext_depth

    @property
    def h(self) -> float:
        return self.texel

    @property
    def E(self) -> float:
        return self.extent

    def polygon(self) -> np.ndarray:
        return np.array([[self.poly[i][0], self.poly[i][1]] for i in range(self.n_poly)])


class hf_view_stats_t(ct.Structure):
    _fields_ = [("visible_texels", ct.c_int64 * HF_MAX_CASCADES),
                ("candidates", ct.c_int64 * HF_MAX_CASCADES),
                ("influencers", ct.c_int64 * HF_MAX_CASCADES),
                ("reused_texels", ct.c_int64 * HF_MAX_CASCADES)]


class hf_batch_item(ct.Structure):
    _fields_ = [("ctx", ct.c_void_p), ("view_slot", ct.c_int32), ("reserved", ct.c_int32),
                ("t_dev", ct.c_void_p), ("hit_dev", ct.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ct.CDLL(LIB_PATH)
    P, vp, i32, i64, sz = ct.POINTER, ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_size_t
    sig = {
        "hf_create_quadtree": [P(hf_quadtree_desc), vp, i64, P(hf_rbf_params), P(vp)],
        "hf_query_bytes": [vp, i32, i32, P(sz), P(sz)],
        "hf_bind_persistent": [vp, vp, sz, vp],
        "hf_update_values": [vp, vp, i64, vp],
        "hf_update_water": [vp, vp, i64, vp],
        "hf_selftest_wait_timeout": [vp, i32, vp],
        "hf_set_camera": [vp, i32, P(hf_camera), vp, sz],
        "hf_set_camera_follow": [vp, i32, P(hf_camera), vp, sz, i32],
        "hf_discretize_cascades": [vp, i32, vp],
        "hf_discretize_reuse": [vp, i32, i32, vp],
        "hf_build_maxmip": [vp, i32, vp],
        "hf_raycast": [vp, i32, vp, vp, vp],
        "hf_get_cascade": [vp, i32, i32, P(hf_cascade_info)],
        "hf_view_stats": [vp, i32, P(hf_view_stats_t), vp],
        "hf_sync": [vp, vp],
        "hf_discretize_noalloc": [vp, P(hf_camera), P(vp), P(hf_cascade_info), vp],
        "hf_ray_stats": [vp, i32, P(i64), P(i64), vp],
        "hf_batch_query_bytes": [P(hf_batch_item), i32, i32, P(sz), P(sz)],
        "hf_batch_prepare": [P(hf_batch_item), i32, i32, vp, sz],
        "hf_batch_launch": [vp, vp, sz, vp],
        "hf_frame_batch": [P(hf_batch_item), i32, i32, vp, sz, vp, sz, vp],
        "hf_measure_unit_rates": [P(ct.c_double), P(ct.c_double), P(i32), vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ct.c_int
    lib.hf_destroy.argtypes = [vp]
    lib.hf_destroy.restype = None
    lib.hf_last_error.argtypes = []
    lib.hf_last_error.restype = ct.c_char_p
    return lib


_lib = _load()


def lib():
    return _lib


def hf_last_error() -> str:
    return _lib.hf_last_error().decode()


def _check(rc: int):
    if rc != HF_OK:
        raise HFError(rc, hf_last_error())


def _stream(stream):
    if stream is None:
        import torch
        return ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ct.c_void_p(stream)
    return ct.c_void_p(stream.cuda_stream)


def _dptr(t) -> ct.c_void_p:
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ct.c_void_p(t.data_ptr())


def leaves_array(level, ix, iy, value) -> np.ndarray:
    a = np.empty(len(level), LEAF_DTYPE)
    a["level"], a["ix"], a["iy"], a["value"] = level, ix, iy, value
    return a


def hf_create_quadtree(desc: hf_quadtree_desc, leaves: np.ndarray, rbf: hf_rbf_params) -> ct.c_void_p:
    leaves = np.ascontiguousarray(leaves, LEAF_DTYPE)
    ctx = ct.c_void_p()
    _check(_lib.hf_create_quadtree(ct.byref(desc), leaves.ctypes.data_as(ct.c_void_p),
                                   ct.c_int64(leaves.size), ct.byref(rbf), ct.byref(ctx)))
    return ctx


def hf_query_bytes(ctx, n_cascades: int, cascade_size: int):
    p, v = ct.c_size_t(), ct.c_size_t()
    _check(_lib.hf_query_bytes(ctx, n_cascades, cascade_size, ct.byref(p), ct.byref(v)))
    return p.value, v.value


def hf_bind_persistent(ctx, buf, stream=None):
    _check(_lib.hf_bind_persistent(ctx, _dptr(buf), buf.numel() * buf.element_size(), _stream(stream)))


def hf_update_values(ctx, values: np.ndarray, stream=None):
    v = np.ascontiguousarray(values, np.float32)
    _check(_lib.hf_update_values(ctx, v.ctypes.data_as(ct.c_void_p), ct.c_int64(v.size), _stream(stream)))


def hf_update_water(ctx, depths: np.ndarray, stream=None):
    d = np.ascontiguousarray(depths, np.float32)
    _check(_lib.hf_update_water(ctx, d.ctypes.data_as(ct.c_void_p), ct.c_int64(d.size), _stream(stream)))


def hf_selftest_wait_timeout(ctx, polls: int = 1000, stream=None):
    _check(_lib.hf_selftest_wait_timeout(ctx, polls, _stream(stream)))


def hf_set_camera(ctx, slot: int, cam: hf_camera, view_buf):
    _check(_lib.hf_set_camera(ctx, slot, ct.byref(cam), _dptr(view_buf),
                              view_buf.numel() * view_buf.element_size()))


def hf_set_camera_follow(ctx, slot: int, cam: hf_camera, view_buf, prev_slot: int):
    _check(_lib.hf_set_camera_follow(ctx, slot, ct.byref(cam), _dptr(view_buf),
                                     view_buf.numel() * view_buf.element_size(), prev_slot))


def hf_discretize_cascades(ctx, slot: int, stream=None):
    _check(_lib.hf_discretize_cascades(ctx, slot, _stream(stream)))


def hf_discretize_reuse(ctx, slot: int, prev_slot: int, stream=None):
    _check(_lib.hf_discretize_reuse(ctx, slot, prev_slot, _stream(stream)))


def hf_build_maxmip(ctx, slot: int, stream=None):
    _check(_lib.hf_build_maxmip(ctx, slot, _stream(stream)))


def _out_ptr(t) -> ct.c_void_p:
    """A kernel output: a contiguous CUDA tensor or a pinned host tensor."""
    if not t.is_contiguous() or not (t.is_cuda or t.is_pinned()):
        raise ValueError("expected a contiguous CUDA tensor or a pinned host tensor")
    return ct.c_void_p(t.data_ptr())


def hf_raycast(ctx, slot: int, t_out, hit_out, stream=None):
    """t_out / hit_out: CUDA tensors, or pinned host tensors that the kernel
    writes directly."""
    _check(_lib.hf_raycast(ctx, slot, _out_ptr(t_out), _out_ptr(hit_out), _stream(stream)))


def hf_get_cascade(ctx, slot: int, c: int) -> hf_cascade_info:
    info = hf_cascade_info()
    _check(_lib.hf_get_cascade(ctx, slot, c, ct.byref(info)))
    return info


def hf_view_stats(ctx, slot: int, n_cascades: int, stream=None) -> dict:
    st = hf_view_stats_t()
    _check(_lib.hf_view_stats(ctx, slot, ct.byref(st), _stream(stream)))
    return {"visible_texels": list(st.visible_texels)[:n_cascades],
            "candidates": list(st.candidates)[:n_cascades],
            "influencers": list(st.influencers)[:n_cascades],
            "reused_texels": list(st.reused_texels)[:n_cascades]}


def check_noalloc_outputs(cam: hf_camera, tex_out, device_index: int) -> None:
    """Raise ValueError unless tex_out holds exactly cam.n_cascades contiguous
    float32 tensors of at least cascade_size^2 elements on CUDA device
    `device_index`.  The C entry point reads one pointer per cascade and the
    kernel writes N*N floats through each, so a short list or a small tensor
    would be read or written past its end."""
    import torch
    n = int(cam.n_cascades)
    if len(tex_out) != n:
        raise ValueError(f"tex_out holds {len(tex_out)} tensors for {n} cascades")
    need = int(cam.cascade_size) ** 2
    for k, t in enumerate(tex_out):
        if t.dtype != torch.float32:
            raise ValueError(f"tex_out[{k}] is {t.dtype}, not torch.float32")
        if not t.is_cuda or t.device.index != device_index:
            raise ValueError(f"tex_out[{k}] is on {t.device}, not cuda:{device_index}")
        if not t.is_contiguous():
            raise ValueError(f"tex_out[{k}] is not contiguous")
        if t.numel() < need:
            raise ValueError(f"tex_out[{k}] has {t.numel()} elements, fewer than {need}")


def hf_discretize_noalloc(ctx, cam: hf_camera, tex_out, stream=None):
    """Allocation-free discretization into caller-provided textures (one
    contiguous CUDA float32 tensor of N*N elements per cascade, on the
    current device); returns the fitted cascades.  See include/hf.h for the
    limits and the shared scratch."""
    import torch
    check_noalloc_outputs(cam, tex_out, torch.cuda.current_device())
    n = len(tex_out)
    ptrs = (ct.c_void_p * n)(*[_dptr(t).value for t in tex_out])
    info = (hf_cascade_info * n)()
    _check(_lib.hf_discretize_noalloc(ctx, ct.byref(cam), ptrs, info, _stream(stream)))
    return list(info)


def hf_ray_stats(ctx, slot: int, stream=None) -> dict:
    v, t = ct.c_int64(), ct.c_int64()
    _check(_lib.hf_ray_stats(ctx, slot, ct.byref(v), ct.byref(t), _stream(stream)))
    return {"visits": v.value, "patch_tests": t.value}


def hf_batch_query_bytes(items, flags: int = 0):
    d, h = ct.c_size_t(), ct.c_size_t()
    _check(_lib.hf_batch_query_bytes(items, len(items), flags, ct.byref(d), ct.byref(h)))
    return d.value, h.value


def hf_batch_prepare(items, flags: int, host_buf):
    _check(_lib.hf_batch_prepare(items, len(items), flags, ct.c_void_p(host_buf.data_ptr()),
                                 host_buf.numel() * host_buf.element_size()))


def hf_batch_launch(host_buf, dev_buf, stream=None):
    _check(_lib.hf_batch_launch(ct.c_void_p(host_buf.data_ptr()), _dptr(dev_buf),
                                dev_buf.numel() * dev_buf.element_size(), _stream(stream)))


def hf_frame_batch(items, flags: int, host_buf, dev_buf, stream=None):
    _check(_lib.hf_frame_batch(items, len(items), flags, ct.c_void_p(host_buf.data_ptr()),
                               host_buf.numel() * host_buf.element_size(), _dptr(dev_buf),
                               dev_buf.numel() * dev_buf.element_size(), _stream(stream)))


def hf_sync(ctx, stream=None):
    _check(_lib.hf_sync(ctx, _stream(stream)))


def hf_measure_unit_rates(stream=None) -> dict:
    """Measured MUFU ex2 and FP32 FMA rates (operations / s) and the SM count."""
    ex2, ffma, sms = ct.c_double(), ct.c_double(), ct.c_int32()
    _check(_lib.hf_measure_unit_rates(ct.byref(ex2), ct.byref(ffma), ct.byref(sms), _stream(stream)))
    return {"ex2_per_s": ex2.value, "ffma_per_s": ffma.value, "sms": sms.value}


def hf_destroy(ctx):
    _lib.hf_destroy(ctx)

"""CPU checks of the C-ABI library: it loads, exports every entry point that
include/hf.h declares, validates its inputs, and its host-side cascade fit
agrees with the oracle's independent fit (no device work is launched)."""

import ctypes as ct
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hfmod():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2201_10887_gb300 import hf
    return hf


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:int|void|const char\*)\s+(hf_\w+)\s*\(", txt, re.M))
    return sorted(names)


def test_exports_every_declared_symbol(hfmod):
    names = _declared()
    assert len(names) >= 12
    lib = ct.CDLL(hfmod.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(hfmod.EXPORTED) <= set(names)


def test_product_does_not_use_the_oracle():
    pkg = os.path.join(ROOT, "paper_2201_10887_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, re.M), f
                assert "hf_oracle" not in txt and "liboracle" not in txt, f


def _tiny_ctx(hfmod, tiny, **kw):
    t = tiny.tree
    desc = hfmod.hf_quadtree_desc(t.origin_x, t.origin_y, t.root_cell, t.root_nx, t.root_ny, t.max_level)
    rbf = hfmod.hf_rbf_params(kw.get("sigma", tiny.sigma), kw.get("radius", tiny.radius), 0, -1)
    return hfmod.hf_create_quadtree(desc, hfmod.leaves_array(t.level, t.ix, t.iy, t.value), rbf)


def test_create_and_query(hfmod, tiny):
    ctx = _tiny_ctx(hfmod, tiny)
    p, v = hfmod.hf_query_bytes(ctx, 3, 256)
    assert p > tiny.tree.n_leaves * 16 and v >= 3 * 256 * 256 * 4
    with pytest.raises(hfmod.HFError) as e:
        hfmod.hf_query_bytes(ctx, 9, 256)
    assert e.value.code == hfmod.HF_ERR_ARG
    hfmod.hf_destroy(ctx)


def _bad(hfmod, tiny, mutate):
    t = tiny.tree
    lv = hfmod.leaves_array(t.level, t.ix, t.iy, t.value)
    desc = hfmod.hf_quadtree_desc(t.origin_x, t.origin_y, t.root_cell, t.root_nx, t.root_ny, t.max_level)
    rbf = hfmod.hf_rbf_params(tiny.sigma, tiny.radius, 0, -1)
    lv, desc, rbf = mutate(lv, desc, rbf)
    with pytest.raises(hfmod.HFError) as e:
        hfmod.hf_create_quadtree(desc, lv, rbf)
    return e.value.code


def test_rejects_invalid_quadtrees(hfmod, tiny):
    def dup(lv, d, r):
        return np.concatenate([lv, lv[:1]]), d, r

    def gap(lv, d, r):
        return lv[1:], d, r

    def overlap(lv, d, r):
        k = int(np.nonzero(lv["level"] == 1)[0][0])
        extra = lv[k:k + 1].copy()
        extra["level"] = 0
        extra["ix"] //= 2
        extra["iy"] //= 2
        return np.concatenate([lv, extra]), d, r

    def out_of_range(lv, d, r):
        lv = lv.copy()
        lv["ix"][0] = 10 ** 6
        return lv, d, r

    def nan_value(lv, d, r):
        lv = lv.copy()
        lv["value"][3] = np.nan
        return lv, d, r

    def bad_sigma(lv, d, r):
        r.sigma = 0.0
        return lv, d, r

    def bad_level(lv, d, r):
        d.max_level = 16
        return lv, d, r

    for m in [dup, gap, overlap, out_of_range, nan_value, bad_sigma, bad_level]:
        assert _bad(hfmod, tiny, m) == hfmod.HF_ERR_ARG, m.__name__


def _set_camera_fake(hfmod, ctx, cam, C, N):
    """Host-only fit: hf_set_camera only records the buffer address."""
    from paper_2201_10887_gb300.renderer import camera_struct
    need = hfmod.hf_query_bytes(ctx, C, N)[1]
    return hfmod.lib().hf_set_camera(ctx, 0, ct.byref(camera_struct(cam)), ct.c_void_p(1 << 30),
                                     ct.c_size_t(need))


def test_call_order_and_buffer_checks(hfmod, tiny):
    ctx = _tiny_ctx(hfmod, tiny)
    cam = tiny.cameras[0]
    lib = hfmod.lib()
    assert lib.hf_discretize_cascades(ctx, 0, None) == hfmod.HF_ERR_STATE
    assert lib.hf_raycast(ctx, 0, ct.c_void_p(1 << 20), ct.c_void_p(1 << 20), None) == hfmod.HF_ERR_STATE
    from paper_2201_10887_gb300.renderer import camera_struct
    assert lib.hf_set_camera(ctx, 0, ct.byref(camera_struct(cam)), ct.c_void_p(1 << 30),
                             ct.c_size_t(1000)) == hfmod.HF_ERR_NOMEM
    assert lib.hf_set_camera(ctx, 0, ct.byref(camera_struct(cam)), ct.c_void_p((1 << 30) + 8),
                             ct.c_size_t(1 << 30)) == hfmod.HF_ERR_ARG
    assert lib.hf_set_camera(ctx, 256, ct.byref(camera_struct(cam)), ct.c_void_p(1 << 30),
                             ct.c_size_t(1 << 30)) == hfmod.HF_ERR_ARG
    assert _set_camera_fake(hfmod, ctx, cam, cam.n_cascades, cam.cascade_size) == 0
    # the mip build needs a discretized view
    assert lib.hf_build_maxmip(ctx, 0, None) == hfmod.HF_ERR_STATE
    # no persistent buffer bound yet
    assert lib.hf_discretize_cascades(ctx, 0, None) == hfmod.HF_ERR_STATE
    for bad_cam in (cam.with_(vfov=0.0), cam.with_(texel_ladder=-1), cam.with_(texel_ladder=65),
                    cam.with_(texel_ladder=2, cascade_size=3), cam.with_(lod_pixels=-1.0),
                    cam.with_(lod_pixels=float("nan")), cam.with_(lod_pixels=2e6)):
        bad = camera_struct(bad_cam)
        assert lib.hf_set_camera(ctx, 1, ct.byref(bad), ct.c_void_p(1 << 30), ct.c_size_t(1 << 30)) == hfmod.HF_ERR_ARG
    bad = camera_struct(cam)
    bad.traversal = 2
    assert lib.hf_set_camera(ctx, 1, ct.byref(bad), ct.c_void_p(1 << 30), ct.c_size_t(1 << 30)) == hfmod.HF_ERR_ARG
    # reuse needs the persistent buffer first, like every device step
    assert lib.hf_discretize_reuse(ctx, 0, 1, None) == hfmod.HF_ERR_STATE
    hfmod.hf_destroy(ctx)


@pytest.mark.parametrize("variant", ["base", "three", "steep", "side", "far_origin", "lattice1", "lattice4"])
def test_library_fit_matches_oracle(hfmod, orc, tiny, variant):
    import math
    import workloads
    scene = tiny if variant != "far_origin" else workloads.precision_config()
    base = scene.cameras[0]
    cam = {"base": base,
           "three": base.with_(n_cascades=3, split_lambda=1.0),
           "steep": base.with_(n_cascades=2, forward=(0.0, 0.2, -1.0)),
           "side": base.with_(n_cascades=4, split_lambda=0.5, forward=(-0.8, 0.1, -0.6),
                              vfov=math.radians(40)),
           "far_origin": base.with_(n_cascades=3, split_lambda=0.5),
           "lattice1": base.with_(n_cascades=3, texel_ladder=1),
           "lattice4": base.with_(n_cascades=4, split_lambda=0.5, texel_ladder=4,
                                  forward=(-0.8, 0.1, -0.6))}[variant]
    ctx = _tiny_ctx(hfmod, scene)
    assert _set_camera_fake(hfmod, ctx, cam, cam.n_cascades, cam.cascade_size) == 0
    cells = orc.Cells(scene.tree)
    ov = orc.fit(cam, scene.tree, cells)
    for c in range(cam.n_cascades):
        li = hfmod.hf_get_cascade(ctx, 0, c)
        oc = ov.cas[c]
        assert (li.snap_x, li.snap_y, li.snap_k) == (oc.snap_x, oc.snap_y, oc.snap_k)
        assert li.n_poly == oc.n_poly
        if li.n_poly:
            assert np.max(np.abs(li.polygon() - oc.polygon())) < 1e-9 * scene.tree.width
        assert li.near == pytest.approx(oc.near, abs=1e-9) and li.far_ext == pytest.approx(oc.far_ext, abs=1e-9)
        if cam.texel_ladder:  # c_min 2^(m/n): the two sides may round the power differently
            assert li.texel == pytest.approx(oc.h, rel=1e-15) and li.texel_ladder == cam.texel_ladder
            assert li.ox == pytest.approx(oc.ox, rel=1e-15, abs=1e-12)
            assert li.oy == pytest.approx(oc.oy, rel=1e-15, abs=1e-12)
        else:
            assert li.texel == oc.h and li.ox == oc.ox and li.oy == oc.oy
        assert li.reuse_source == -1
    hfmod.hf_destroy(ctx)


def test_fit_fuzz_against_oracle(hfmod, orc, tiny):
    """Random cameras (position, heading, pitch, roll, field of view, cascade
    settings): the library's fit and the oracle's agree on every integer snap
    and on the polygons."""
    import math
    rng = np.random.default_rng(11)
    ctx = _tiny_ctx(hfmod, tiny)
    cells = orc.Cells(tiny.tree)
    W = tiny.tree.width
    checked = stops = 0
    for trial in range(300):
        yaw, pitch = rng.uniform(0, 2 * math.pi), rng.uniform(-1.5, 0.3)
        fwd = (math.cos(pitch) * math.cos(yaw), math.cos(pitch) * math.sin(yaw), math.sin(pitch))
        roll = rng.uniform(-0.3, 0.3)
        up = (math.sin(roll) * math.sin(yaw), -math.sin(roll) * math.cos(yaw), math.cos(roll))
        eye = (tiny.tree.origin_x + rng.uniform(-200, 840), tiny.tree.origin_y + rng.uniform(-200, 840),
               rng.uniform(150, 1200))
        cam = tiny.cameras[0].with_(eye=eye, forward=fwd, up=up, vfov=rng.uniform(0.3, 1.5),
                                    n_cascades=int(rng.integers(1, 9)),
                                    cascade_size=int(rng.integers(2, 600)),
                                    width=int(rng.integers(16, 400)), height=int(rng.integers(16, 400)),
                                    split_lambda=float(rng.uniform(0, 1)),
                                    overlap_frac=float(rng.uniform(0, 0.2)))
        if trial % 3 == 0:
            cam = cam.with_(texel_ladder=int(rng.integers(1, 9)), cascade_size=max(cam.cascade_size, 4))
        if trial % 2 == 0:
            cam = cam.with_(lod_pixels=float(rng.choice([0.5, 1.0, 2.0, 8.0, 64.0])))
        assert _set_camera_fake(hfmod, ctx, cam, cam.n_cascades, cam.cascade_size) == 0
        ov = orc.fit(cam, tiny.tree, cells)
        for c in range(cam.n_cascades):
            li = hfmod.hf_get_cascade(ctx, 0, c)
            oc = ov.cas[c]
            assert (li.snap_x, li.snap_y, li.snap_k) == (oc.snap_x, oc.snap_y, oc.snap_k), (trial, c)
            assert (li.n_poly == 0) == (oc.n_poly == 0), (trial, c)
            assert li.stop_level == orc.stop_level(cam.lod_pixels, cam.vfov, cam.height, li.near, li.texel,
                                                   cam.cascade_size), (trial, c)
            stops += li.stop_level > 0
            if li.n_poly:
                lp, op = li.polygon(), oc.polygon()
                # every vertex of one polygon is a vertex of the other
                d1 = np.min(np.linalg.norm(lp[:, None] - op[None], axis=2), axis=1)
                d2 = np.min(np.linalg.norm(op[:, None] - lp[None], axis=2), axis=1)
                assert d1.max() < 1e-7 * W and d2.max() < 1e-7 * W, (trial, c)
                checked += 1
    assert checked > 300 and stops > 20
    hfmod.hf_destroy(ctx)


def test_reduced_precision_offset_limits(hfmod, tiny):
    """FP16/BF16 lists need candidate offsets that are exact small integers:
    a grid whose coarse cells reach too far is rejected, FP32 accepts it."""
    t = tiny.tree
    lv = hfmod.leaves_array(t.level, t.ix, t.iy, t.value)
    desc = hfmod.hf_quadtree_desc(t.origin_x, t.origin_y, t.root_cell, t.root_nx, t.root_ny, t.max_level)
    for prec in (0, 1, 2):
        ctx = hfmod.hf_create_quadtree(desc, lv, hfmod.hf_rbf_params(tiny.sigma, tiny.radius, prec, -1))
        hfmod.hf_destroy(ctx)
    # radius 40 cells: reach 40 x 10 m = 320 half-cells of 1.25 m > 256 (BF16), < 1024 (FP16)
    ctx = hfmod.hf_create_quadtree(desc, lv, hfmod.hf_rbf_params(1.5, 40.0, 1, -1))
    hfmod.hf_destroy(ctx)
    with pytest.raises(hfmod.HFError) as e:
        hfmod.hf_create_quadtree(desc, lv, hfmod.hf_rbf_params(1.5, 40.0, 2, -1))
    assert e.value.code == hfmod.HF_ERR_ARG and "BF16" in str(e.value)


@pytest.mark.parametrize("sigma", [60.0, 120.0, 180.0, 400.0, 1e-4])
def test_reduced_precision_exponent_scale_range(hfmod, tiny, sigma):
    """The FP16 exponent scale -log2(e) / (8 sigma^2) per squared half-cell
    must be a normal FP16 number at every level: sigmas that push it below
    2^-14 (sigma > ~54 cells) or above 65504 are rejected, whatever the bits
    of the out-of-range value would wrap to.  FP32 takes them all."""
    t = tiny.tree
    lv = hfmod.leaves_array(t.level, t.ix, t.iy, t.value)
    desc = hfmod.hf_quadtree_desc(t.origin_x, t.origin_y, t.root_cell, t.root_nx, t.root_ny, t.max_level)
    hfmod.hf_destroy(hfmod.hf_create_quadtree(desc, lv, hfmod.hf_rbf_params(sigma, 3.0, 0, -1)))
    with pytest.raises(hfmod.HFError) as e:
        hfmod.hf_create_quadtree(desc, lv, hfmod.hf_rbf_params(sigma, 3.0, 1, -1))
    assert e.value.code == hfmod.HF_ERR_ARG and "normal range" in str(e.value)


def test_water_layer_flags_and_sizes(hfmod, tiny, monkeypatch):
    """The water layer: FP32 only, flag 0/1; it adds 4 bytes per
    leaf to the persistent buffer of an FP32 context on the index lists and a
    second texture per cascade (one mipmap bounds both surfaces); a plain FP32
    context also keeps the compact pair lists, which the water layer does not
    use.  RBF kernels: 0 or 1, FP32 only."""
    t = tiny.tree
    lv = hfmod.leaves_array(t.level, t.ix, t.iy, t.value)
    desc = hfmod.hf_quadtree_desc(t.origin_x, t.origin_y, t.root_cell, t.root_nx, t.root_ny, t.max_level)
    compact = hfmod.hf_create_quadtree(desc, lv, hfmod.hf_rbf_params(tiny.sigma, tiny.radius, 0, -1, 0, 0))
    monkeypatch.setenv("HF_FP32_INDEX_LISTS", "1")
    plain = hfmod.hf_create_quadtree(desc, lv, hfmod.hf_rbf_params(tiny.sigma, tiny.radius, 0, -1, 0, 0))
    monkeypatch.delenv("HF_FP32_INDEX_LISTS")
    wet = hfmod.hf_create_quadtree(desc, lv, hfmod.hf_rbf_params(tiny.sigma, tiny.radius, 0, -1, 1, 0))
    pc, _ = hfmod.hf_query_bytes(compact, 3, 256)
    p0, v0 = hfmod.hf_query_bytes(plain, 3, 256)
    p1, v1 = hfmod.hf_query_bytes(wet, 3, 256)
    assert p1 - p0 >= 4 * t.n_leaves and p1 - p0 < 4 * t.n_leaves + 256
    assert pc - p0 > 8 * 20 * t.n_leaves  # ~8 bytes per candidate (about 30 per leaf) in pairs
    assert v1 - v0 == 3 * 256 * 256 * 4
    # the coarse-level stop is defined for the terrain alone
    from paper_2201_10887_gb300.renderer import camera_struct
    cam = tiny.cameras[0].with_(lod_pixels=2.0)
    need = hfmod.hf_query_bytes(wet, cam.n_cascades, cam.cascade_size)[1]
    assert hfmod.lib().hf_set_camera(wet, 0, ct.byref(camera_struct(cam)), ct.c_void_p(1 << 30),
                                     ct.c_size_t(need)) == hfmod.HF_ERR_ARG
    assert hfmod.lib().hf_set_camera(plain, 0, ct.byref(camera_struct(cam)), ct.c_void_p(1 << 30),
                                     ct.c_size_t(need)) == 0
    for d in (compact, plain, wet):
        hfmod.hf_destroy(d)
    for args in ((0, -1, 2, 0), (1, -1, 1, 0), (2, -1, 1, 0), (0, -1, 0, 7), (1, -1, 0, 1), (2, -1, 0, 1)):
        with pytest.raises(hfmod.HFError) as e:
            hfmod.hf_create_quadtree(desc, lv, hfmod.hf_rbf_params(tiny.sigma, tiny.radius, *args))
        assert e.value.code == hfmod.HF_ERR_ARG


def test_arena_first_fit_and_merge():
    from paper_2201_10887_gb300.serving import Arena
    a = Arena(10_000)
    x, y = a.alloc(1000), a.alloc(3000)
    assert (x, y) == (0, 1024) and a.alloc(6000) is None
    a.release(y, 3000)
    assert a.alloc(2000) == 1024
    a.release(x, 1000)
    a.release(1024, 2000)
    assert a.free == [(0, 10_000)] and a.used() == 0


def test_fit_follow_against_oracle(hfmod, orc, tiny):
    """hf_set_camera_follow against the oracle's fit with the same earlier
    ladder steps, over pairs of nearby random cameras; a slot without a
    camera cannot be followed."""
    import math
    from paper_2201_10887_gb300.renderer import camera_struct
    rng = np.random.default_rng(5)
    ctx = _tiny_ctx(hfmod, tiny)
    cells = orc.Cells(tiny.tree)
    lib = hfmod.lib()
    kept = 0
    for trial in range(120):
        yaw, pitch = rng.uniform(0, 2 * math.pi), rng.uniform(-1.2, -0.2)
        fwd = (math.cos(pitch) * math.cos(yaw), math.cos(pitch) * math.sin(yaw), math.sin(pitch))
        eye = (tiny.tree.origin_x + rng.uniform(0, 640), tiny.tree.origin_y + rng.uniform(0, 640),
               rng.uniform(200, 900))
        a = tiny.cameras[0].with_(eye=eye, forward=fwd, n_cascades=int(rng.integers(1, 5)),
                                  cascade_size=int(rng.integers(16, 400)), texel_ladder=int(rng.integers(1, 6)))
        b = a.with_(eye=(eye[0] + rng.normal(0, 20), eye[1] + rng.normal(0, 20), eye[2] * rng.uniform(0.8, 1.25)))
        assert _set_camera_fake(hfmod, ctx, a, a.n_cascades, a.cascade_size) == 0
        infos = [hfmod.hf_get_cascade(ctx, 0, c) for c in range(a.n_cascades)]
        steps = [i.snap_k if i.n_poly else 10 ** 9 for i in infos]  # an empty cascade is not followed
        need = hfmod.hf_query_bytes(ctx, b.n_cascades, b.cascade_size)[1]
        assert lib.hf_set_camera_follow(ctx, 1, ct.byref(camera_struct(b)), ct.c_void_p(1 << 30),
                                        ct.c_size_t(need), 0) == 0
        ob = orc.fit(b, tiny.tree, cells, follow=steps)
        plain = orc.fit(b, tiny.tree, cells)
        for c in range(b.n_cascades):
            li = hfmod.hf_get_cascade(ctx, 1, c)
            assert (li.snap_x, li.snap_y, li.snap_k) == (ob.cas[c].snap_x, ob.cas[c].snap_y, ob.cas[c].snap_k), (trial, c)
            kept += int(ob.cas[c].n_poly > 0 and ob.cas[c].snap_k != plain.cas[c].snap_k)
    assert kept > 0
    for bad_prev in (7, -1, 999):
        assert lib.hf_set_camera_follow(ctx, 2, ct.byref(camera_struct(a)), ct.c_void_p(1 << 30),
                                        ct.c_size_t(1 << 30), bad_prev) == hfmod.HF_ERR_STATE
    hfmod.hf_destroy(ctx)


_HOST_FAILURE_SCRIPT = r"""
import resource, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2201_10887_gb300 import hf
n = 1024
iy, ix = np.divmod(np.arange(n * n, dtype=np.int64), n)
lv = hf.leaves_array(np.zeros(n * n, np.int32), ix.astype(np.int32), iy.astype(np.int32), np.zeros(n * n, np.float32))
desc = hf.hf_quadtree_desc(0.0, 0.0, 10.0, n, n, 0)
rbf = hf.hf_rbf_params(1.5, 3.0, 0, -1)
vm = [int(l.split()[1]) * 1024 for l in open("/proc/self/status") if l.startswith("VmSize:")][0]
resource.setrlimit(resource.RLIMIT_AS, (vm + (8 << 20), resource.getrlimit(resource.RLIMIT_AS)[1]))
try:
    hf.hf_create_quadtree(desc, lv, rbf)
    print("created")
except hf.HFError as e:
    print("code", e.code, str(e)[:120])
"""


def test_host_failure_is_a_status_not_an_exception(hfmod):
    """A host allocation that fails inside an entry point (here: the
    library's tables for a million leaves under an address-space limit a few
    megabytes above the process's size) comes back as HF_ERR_HOST with a
    message; no C++ exception crosses the C ABI, so the process goes on."""
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "-c", _HOST_FAILURE_SCRIPT, ROOT], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.startswith("code %d" % hfmod.HF_ERR_HOST), r.stdout
    assert "hf_create_quadtree" in r.stdout


def test_leaf_count_limit(hfmod, tiny):
    """List entries are 32-bit leaf indices: a count of 2^31 leaves is
    refused before the leaf array is read."""
    t = tiny.tree
    lv = hfmod.leaves_array(t.level, t.ix, t.iy, t.value)
    desc = hfmod.hf_quadtree_desc(t.origin_x, t.origin_y, t.root_cell, t.root_nx, t.root_ny, t.max_level)
    rbf = hfmod.hf_rbf_params(tiny.sigma, tiny.radius, 0, -1)
    lib = ct.CDLL(hfmod.LIB_PATH)
    lib.hf_last_error.restype = ct.c_char_p
    ctx = ct.c_void_p()
    rc = lib.hf_create_quadtree(ct.byref(desc), lv.ctypes.data_as(ct.c_void_p), ct.c_int64(2 ** 31),
                                ct.byref(rbf), ct.byref(ctx))
    assert rc == hfmod.HF_ERR_ARG and b"2^31" in lib.hf_last_error() and not ctx.value


def test_status_codes_match_the_header(hfmod):
    """The binding's status constants and names are the header's enum."""
    txt = open(os.path.join(ROOT, "include", "hf.h")).read()
    codes = {m.group(1): int(m.group(2)) for m in re.finditer(r"^\s*(HF_(?:OK|ERR_\w+))\s*=\s*(-?\d+)", txt, re.M)}
    assert "HF_ERR_HOST" in codes and len(codes) >= 8
    for name, value in codes.items():
        assert getattr(hfmod, name) == value, name
        if value:
            assert hfmod.ERROR_NAMES[value] == name
    assert set(hfmod.ERROR_NAMES) == {v for v in codes.values() if v}


def test_struct_layouts_match_the_header(hfmod, tmp_path):
    """Every ctypes structure of the binding (and the leaf record dtype) has
    the size and field offsets the C compiler gives the header's struct."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = [hfmod.hf_quadtree_desc, hfmod.hf_rbf_params, hfmod.hf_camera, hfmod.hf_cascade_info,
               hfmod.hf_view_stats_t, hfmod.hf_batch_item]
    lines = ['#include <stdio.h>', '#include "hf.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'printf("{n} size %zu\\n", sizeof({n}));')
        for f in st._fields_:
            lines.append(f'printf("{n} {f[0]} %zu\\n", offsetof({n}, {f[0]}));')
    lines.append('printf("hf_leaf size %zu\\n", sizeof(hf_leaf));')
    for f in hfmod.LEAF_DTYPE.names:
        lines.append(f'printf("hf_leaf {f} %zu\\n", offsetof(hf_leaf, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for st in structs:
        n = st.__name__
        assert got[(n, "size")] == ct.sizeof(st), n
        for f in st._fields_:
            assert got[(n, f[0])] == getattr(st, f[0]).offset, (n, f[0])
    assert got[("hf_leaf", "size")] == hfmod.LEAF_DTYPE.itemsize
    for f in hfmod.LEAF_DTYPE.names:
        assert got[("hf_leaf", f)] == hfmod.LEAF_DTYPE.fields[f][1], f


def test_noalloc_binding_checks_outputs_before_calling(hfmod):
    """hf_discretize_noalloc's binding refuses, before the library is called,
    an output list whose length differs from the camera's cascade count and
    tensors of the wrong type, device, layout or size: the C entry point
    reads one pointer per cascade and writes N*N floats through each."""
    import torch

    class Out:       # stand-in for a CUDA tensor (no GPU here)
        def __init__(self, n, dtype=torch.float32, cuda=True, index=0, contiguous=True):
            self.n, self.dtype, self.is_cuda = n, dtype, cuda
            self.device = torch.device("cuda", index) if cuda else torch.device("cpu")
            self._contig = contiguous

        def numel(self):
            return self.n

        def is_contiguous(self):
            return self._contig

    cam = hfmod.hf_camera()
    cam.n_cascades, cam.cascade_size = 2, 64
    good = [Out(64 * 64), Out(64 * 64 + 5)]
    hfmod.check_noalloc_outputs(cam, good, 0)
    bad = {"short list": [Out(64 * 64)],
           "long list": good + [Out(64 * 64)],
           "dtype": [Out(64 * 64), Out(64 * 64, dtype=torch.float64)],
           "host tensor": [Out(64 * 64), Out(64 * 64, cuda=False)],
           "other device": [Out(64 * 64), Out(64 * 64, index=1)],
           "strided": [Out(64 * 64), Out(64 * 64, contiguous=False)],
           "too small": [Out(64 * 64), Out(64 * 64 - 1)]}
    for what, outs in bad.items():
        with pytest.raises(ValueError):
            hfmod.check_noalloc_outputs(cam, outs, 0)


def test_jump_traversal_refusals(hfmod, tiny):
    """traversal = 1 (climb to the coarsest node entered) is refused with the
    coarse-level stop and with the water layer before any device work."""
    from paper_2201_10887_gb300.renderer import camera_struct
    lib = hfmod.lib()
    cam = tiny.cameras[0]
    desc = hfmod.hf_quadtree_desc(tiny.tree.origin_x, tiny.tree.origin_y, tiny.tree.root_cell,
                                  tiny.tree.root_nx, tiny.tree.root_ny, tiny.tree.max_level)
    leaves = hfmod.leaves_array(tiny.tree.level, tiny.tree.ix, tiny.tree.iy, tiny.tree.value)
    for water, kw in ((0, dict(lod_pixels=4.0)), (1, dict())):
        ctx = hfmod.hf_create_quadtree(desc, leaves, hfmod.hf_rbf_params(tiny.sigma, tiny.radius, 0, -1, water, 0))
        bad = camera_struct(cam.with_(traversal=1, **kw))
        rc = lib.hf_set_camera(ctx, 0, ct.byref(bad), ct.c_void_p(1 << 30), ct.c_size_t(1 << 40))
        assert rc == hfmod.HF_ERR_ARG and "traversal" in hfmod.hf_last_error()
        hfmod.hf_destroy(ctx)


def test_cell_map_limit_from_the_environment(hfmod, tiny, monkeypatch):
    """HF_CELLMAP_MAX_CELLS (read at creation) drops the cell map: the
    persistent buffer shrinks by 8 bytes per finest cell."""
    desc = hfmod.hf_quadtree_desc(tiny.tree.origin_x, tiny.tree.origin_y, tiny.tree.root_cell,
                                  tiny.tree.root_nx, tiny.tree.root_ny, tiny.tree.max_level)
    leaves = hfmod.leaves_array(tiny.tree.level, tiny.tree.ix, tiny.tree.iy, tiny.tree.value)
    rbf = hfmod.hf_rbf_params(tiny.sigma, tiny.radius, 0, -1, 0, 0)
    ctx = hfmod.hf_create_quadtree(desc, leaves, rbf)
    with_map, _ = hfmod.hf_query_bytes(ctx, 1, 2)
    hfmod.hf_destroy(ctx)
    monkeypatch.setenv("HF_CELLMAP_MAX_CELLS", "0")
    ctx = hfmod.hf_create_quadtree(desc, leaves, rbf)
    without, _ = hfmod.hf_query_bytes(ctx, 1, 2)
    hfmod.hf_destroy(ctx)
    fine = (tiny.tree.root_nx << tiny.tree.max_level) * (tiny.tree.root_ny << tiny.tree.max_level)
    assert with_map - without >= 8 * fine > 0

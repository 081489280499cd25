// Host side of the C ABI declared in include/hf.h: input validation, the
// quadtree bitmaps, exact sizing of the influence lists (Section 4), buffer
// layout, and the per-frame launch sequence.  Device memory is never
// allocated here; the caller provides it.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hf_internal.h"

using namespace hfi;

namespace {

// An NVTX range around each entry point, so that profilers can attribute
// kernels to API calls (header-only; costs nothing without a profiler).
struct ApiRange {
    explicit ApiRange(const char* name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
    ApiRange(const ApiRange&) = delete;
    ApiRange& operator=(const ApiRange&) = delete;
};

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) noexcept {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    try {
        g_err = buf;
    } catch (...) {  // no host memory left for the message: keep the code
    }
    return code;
}

int cuda_fail(int e, const char* what) {
    return fail(HF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(cudaError_t(e)));
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Bits of x rounded to nearest even in BF16 / FP16.  f16_bits returns
// UINT32_MAX unless the rounded result is a normal FP16 number.
uint32_t bf16_bits(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}
uint32_t f16_bits(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    const uint32_t sign = (u >> 16) & 0x8000u;
    int e = int((u >> 23) & 0xFF) - 127 + 15;
    uint32_t m = (u & 0x7FFFFFu) >> 13, rem = u & 0x1FFFu;
    if (rem > 0x1000u || (rem == 0x1000u && (m & 1u))) ++m;
    if (m == 0x400u) {
        m = 0;
        ++e;
    }
    if (e < 1 || e > 30) return std::numeric_limits<uint32_t>::max();
    return sign | (uint32_t(e) << 10) | m;
}

// Per-level occupancy bitmaps on the host (see hfi::Bitmaps).
struct HostBitmaps {
    std::vector<uint64_t> bits;
    std::vector<uint32_t> prefix;
    int64_t word_off[kMaxLevels + 1] = {};
    int64_t base[kMaxLevels + 1] = {};
    int32_t nx[kMaxLevels] = {};
    int32_t ny[kMaxLevels] = {};
    int max_level = 0;

    void init(int64_t rnx, int64_t rny, int M) {
        max_level = M;
        int64_t off = 0;
        for (int L = 0; L <= M; ++L) {
            nx[L] = int32_t(rnx << L);
            ny[L] = int32_t(rny << L);
            word_off[L] = off;
            off += (int64_t(nx[L]) * ny[L] + 63) / 64;
        }
        word_off[M + 1] = off;
        bits.assign(size_t(off), 0ull);
    }
    bool test(int L, int64_t ix, int64_t iy) const {
        const int64_t b = iy * nx[L] + ix;
        return (bits[size_t(word_off[L] + (b >> 6))] >> (b & 63)) & 1ull;
    }
    void set(int L, int64_t ix, int64_t iy) {
        const int64_t b = iy * nx[L] + ix;
        bits[size_t(word_off[L] + (b >> 6))] |= 1ull << (b & 63);
    }
    void finalize() {
        prefix.assign(bits.size(), 0u);
        int64_t total = 0;
        for (int L = 0; L <= max_level; ++L) {
            base[L] = total;
            uint32_t run = 0;
            for (int64_t w = word_off[L]; w < word_off[L + 1]; ++w) {
                prefix[size_t(w)] = run;
                run += uint32_t(__builtin_popcountll(bits[size_t(w)]));
            }
            total += run;
        }
        base[max_level + 1] = total;
    }
    int64_t rank(int L, int64_t ix, int64_t iy) const {
        const int64_t b = iy * nx[L] + ix;
        const int64_t w = word_off[L] + (b >> 6);
        return base[L] + prefix[size_t(w)] +
               __builtin_popcountll(bits[size_t(w)] & ((1ull << (b & 63)) - 1ull));
    }
    Bitmaps view(const uint64_t* b, const uint32_t* p) const {
        Bitmaps v;
        std::memset(&v, 0, sizeof(v));
        v.bits = b;
        v.prefix = p;
        for (int L = 0; L <= max_level + 1; ++L) {
            v.word_off[L] = word_off[L];
            v.base[L] = base[L];
        }
        for (int L = 0; L <= max_level; ++L) {
            v.nx[L] = nx[L];
            v.ny[L] = ny[L];
        }
        v.max_level = max_level;
        return v;
    }
};

struct ViewSlot {
    int stage = 0;  // 1 fitted, 2 discretized, 3 mip built
    hf_camera cam{};
    double eye_local[3] = {0, 0, 0};
    FitResult fit{};
    char* dev = nullptr;
    size_t bytes = 0;
    float* tex[HF_MAX_CASCADES] = {};
    float* mip[HF_MAX_CASCADES] = {};
    float* wtex[HF_MAX_CASCADES] = {};  // water surface (water layer only)
    int2* spans[HF_MAX_CASCADES] = {};
    float* xs[HF_MAX_CASCADES] = {};
    float* ys[HF_MAX_CASCADES] = {};
    uint64_t data_version = 0;  // the context's leaf data this slot was discretized from
    // source of the texels the last hf_discretize_reuse carried over, per cascade
    struct Reuse {
        const float* tex = nullptr;
        const float* wtex = nullptr;
        int32_t N = 0, di = 0, dj = 0;
    } reuse[HF_MAX_CASCADES];
};

// Device layout of the persistent buffer.
struct PersistentLayout {
    size_t status, lbits, lprefix, bbits, bprefix, recs, offsets, idx;
    size_t pair_offsets, pairs;          // reduced-precision lists (0 bytes for FP32)
    size_t cellmap;                      // per finest cell {first group, groups} (0 bytes if not kept)
    size_t pair_cellmap;                 // the same for the compact pair lists (reduced precision only)
    size_t depth;                         // water depths (0 bytes without the water layer)
    size_t total;
};

}  // namespace

struct hf_ctx {
    hf_quadtree_desc desc{};
    hf_rbf_params rbf{};
    int M = 0, B = 0;
    int64_t n_leaves = 0, n_buckets = 0, n_cand = 0;
    double c_fin = 0, c_min = 0, c_max = 0, zmin = 0, zmax = 0, width = 0, height = 0;
    double reach_q[kMaxLevels] = {};
    HostBitmaps leaves, buckets;
    std::vector<float4> recs;      // sorted by (level, iy, ix)
    std::vector<int64_t> perm;     // input position -> sorted index
    std::vector<int64_t> offsets;  // n_buckets + 1
    std::vector<int64_t> pair_offsets;  // n_buckets + 1 (reduced precision only)
    int64_t n_pairs = 0, max_pairs = 0;
    uint32_t kb2 = 0;              // packed level-0 scale bits of the compact lists
    uint32_t kf_bits = 0;          // FP32 finest-level scale per squared half-cell
    // compact pair lists and the format of their coordinates: 0 none, HF_PREC_FP16 or
    // HF_PREC_BF16. FP32 contexts without the water layer whose offsets are exact in
    // FP16 keep FP16-format lists and discretize from them in FP32 arithmetic.
    int compact_fmt = 0;
    bool fp32_compact() const { return rbf.precision == HF_PREC_FP32 && compact_fmt == HF_PREC_FP16; }
    std::vector<float> staged;     // values in sorted order for hf_update_values
    std::vector<float> depth;      // water depths in sorted order (water layer only)
    char* dev = nullptr;
    size_t dev_bytes = 0;
    PersistentLayout lay{};
    std::unique_ptr<ViewSlot> views[HF_MAX_VIEWS];
    uint64_t data_version = 0;  // bumped by hf_update_values / hf_update_water
    int64_t cellmap_max_cells = kCellMapMaxCells;  // HF_CELLMAP_MAX_CELLS at creation

    PersistentLayout layout() const {
        PersistentLayout l{};
        size_t o = 0;
        l.status = o; o = align256(o + sizeof(DevStatus));
        l.lbits = o; o = align256(o + leaves.bits.size() * 8);
        l.lprefix = o; o = align256(o + leaves.prefix.size() * 4);
        l.bbits = o; o = align256(o + buckets.bits.size() * 8);
        l.bprefix = o; o = align256(o + buckets.prefix.size() * 4);
        l.recs = o; o = align256(o + size_t(n_leaves + 1) * 16);  // + the null record
        l.offsets = o; o = align256(o + size_t(n_buckets + 1) * 8);
        l.idx = o; o = align256(o + size_t(n_cand) * 4);
        const bool compact = compact_fmt != 0;
        l.pair_offsets = o; o = align256(o + (compact ? size_t(n_buckets + 1) * 8 : 0));
        l.pairs = o; o = align256(o + (compact ? size_t(n_pairs) * 16 : 0));
        l.depth = o; o = align256(o + (rbf.water ? size_t(n_leaves + 1) * 4 : 0));
        l.cellmap = o; o = align256(o + (keep_cellmap() ? size_t(buckets.nx[M]) * size_t(buckets.ny[M]) * 8 : 0));
        l.pair_cellmap = o;
        o = align256(o + (keep_pair_cellmap() ? size_t(buckets.nx[M]) * size_t(buckets.ny[M]) * 8 : 0));
        l.total = o;
        return l;
    }
    DevStatus* d_status() const { return reinterpret_cast<DevStatus*>(dev + lay.status); }
    EnumTables enum_tables(bool device) const {
        EnumTables t;
        std::memset(&t, 0, sizeof(t));
        t.leaves = device ? leaves.view(reinterpret_cast<const uint64_t*>(dev + lay.lbits),
                                        reinterpret_cast<const uint32_t*>(dev + lay.lprefix))
                          : leaves.view(leaves.bits.data(), leaves.prefix.data());
        for (int L = 0; L < kMaxLevels; ++L) t.reach_q[L] = reach_q[L];
        return t;
    }
    LookupTables lookup_tables(bool device) const {
        LookupTables t;
        std::memset(&t, 0, sizeof(t));
        t.buckets = device ? buckets.view(reinterpret_cast<const uint64_t*>(dev + lay.bbits),
                                          reinterpret_cast<const uint32_t*>(dev + lay.bprefix))
                           : buckets.view(buckets.bits.data(), buckets.prefix.data());
        t.bucket_level = B;
        t.inv_c_fin = float(1.0 / c_fin);
        t.nx_fin = buckets.nx[M];
        t.ny_fin = buckets.ny[M];
        t.cellmap = device && keep_cellmap() ? reinterpret_cast<const uint2*>(dev + lay.cellmap) : nullptr;
        return t;
    }
    // the cell map is kept for grids of at most cellmap_max_cells finest cells
    // whose list groups are numbered in 32 bits
    bool keep_cellmap() const {
        return int64_t(buckets.nx[M]) * buckets.ny[M] <= cellmap_max_cells && n_cand / kListPad < (int64_t(1) << 32);
    }
    // ... and for the compact lists: pairs numbered in 32 bits, at most 2^24 - 1 per list
    bool keep_pair_cellmap() const {
        return compact_fmt != 0 && int64_t(buckets.nx[M]) * buckets.ny[M] <= cellmap_max_cells &&
               n_pairs < (int64_t(1) << 32) && max_pairs < (int64_t(1) << 24);
    }
    CompactView compact() const {
        CompactView v;
        v.pair_offsets = reinterpret_cast<const int64_t*>(dev + lay.pair_offsets);
        v.pairs = reinterpret_cast<uint4*>(dev + lay.pairs);
        v.kb2 = kb2;
        v.kf_bits = kf_bits;
        v.max_level = M;
        v.q = float(0.5 * c_fin);
        v.inv_q = float(2.0 / c_fin);
        v.cellmap = keep_pair_cellmap() ? reinterpret_cast<const uint2*>(dev + lay.pair_cellmap) : nullptr;
        return v;
    }
    ListsView lists() const {
        ListsView v;
        v.offsets = reinterpret_cast<const int64_t*>(dev + lay.offsets);
        v.idx = reinterpret_cast<int32_t*>(dev + lay.idx);
        v.recs = reinterpret_cast<float4*>(dev + lay.recs);
        v.depth = rbf.water ? reinterpret_cast<const float*>(dev + lay.depth) : nullptr;
        v.sentinel = int32_t(n_leaves);
        return v;
    }
};

namespace {

size_t per_view_bytes(int C, int N, bool water) {
    size_t o = 0;
    for (int c = 0; c < C; ++c) {
        o = align256(o + size_t(N) * N * 4);
        o = align256(o + size_t(mip_floats(N)) * 4);
        if (water) o = align256(o + size_t(N) * N * 4);
        o = align256(o + size_t(N) * 8);
        o = align256(o + size_t(N) * 4);
        o = align256(o + size_t(N) * 4);
    }
    return o;
}

bool finite3(const double* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

ViewSlot* get_view(hf_ctx* ctx, int32_t slot) {
    if (!ctx || slot < 0 || slot >= HF_MAX_VIEWS || !ctx->views[slot]) return nullptr;
    return ctx->views[slot].get();
}

// Texel grid and grown-polygon edge constraints of a fitted cascade for the
// row kernel (the buffers are set by the caller).
void fill_prep_geometry(const hf_cascade_info& ci, int N, PrepCascade& q) {
    q.ox = ci.ox;
    q.oy = ci.oy;
    q.h = ci.texel;
    q.inv_h = 1.0 / ci.texel;
    q.lattice = ci.texel_ladder > 0 ? 1 : 0;
    q.lat_x = ci.snap_x;
    q.lat_y = ci.snap_y;
    q.N = N;
    q.n_edges = ci.n_poly >= 3 ? ci.n_poly : 0;
    const double delta = std::sqrt(2.0) * ci.texel;  // one texel diagonal
    for (int e = 0; e < q.n_edges; ++e) {
        const double ax = ci.poly[e][0], ay = ci.poly[e][1];
        const double bx = ci.poly[(e + 1) % ci.n_poly][0], by = ci.poly[(e + 1) % ci.n_poly][1];
        const double len = std::hypot(bx - ax, by - ay);
        const double nx = (by - ay) / len, ny = -(bx - ax) / len;
        q.ny[e] = ny;
        q.c[e] = nx * ax + ny * ay + delta;
        q.sgn[e] = nx > 0.0 ? 1 : (nx < 0.0 ? -1 : 0);
        q.inv_nx[e] = nx != 0.0 ? 1.0 / nx : 0.0;
    }
}

int check_camera(const hf_camera& c) {
    if (!finite3(c.eye) || !finite3(c.forward) || !finite3(c.up))
        return fail(HF_ERR_ARG, "camera vectors must be finite");
    if (c.forward[0] == 0.0 && c.forward[1] == 0.0 && c.forward[2] == 0.0) return fail(HF_ERR_ARG, "zero forward vector");
    if (!(c.vfov > 0.0 && c.vfov < 3.1)) return fail(HF_ERR_ARG, "vfov must be in (0, 3.1) radians");
    if (!(c.znear > 0.0 && c.zfar > c.znear && std::isfinite(c.zfar))) return fail(HF_ERR_ARG, "need 0 < znear < zfar");
    if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384) return fail(HF_ERR_ARG, "image size out of range");
    if (c.n_cascades < 1 || c.n_cascades > HF_MAX_CASCADES) return fail(HF_ERR_ARG, "n_cascades must be 1..%d", HF_MAX_CASCADES);
    if (c.cascade_size < 2 || c.cascade_size > kMaxCascadeSize) return fail(HF_ERR_ARG, "cascade_size must be 2..%d", kMaxCascadeSize);
    if (!(c.split_lambda >= 0.0 && c.split_lambda <= 1.0)) return fail(HF_ERR_ARG, "split_lambda must be in [0, 1]");
    if (!(c.overlap_frac >= 0.0 && c.overlap_frac <= 1.0)) return fail(HF_ERR_ARG, "overlap_frac must be in [0, 1]");
    if (c.texel_ladder < 0 || c.texel_ladder > 64) return fail(HF_ERR_ARG, "texel_ladder must be 0..64");
    if (c.texel_ladder > 0 && c.cascade_size < 4) return fail(HF_ERR_ARG, "the lattice fit needs cascade_size >= 4");
    if (c.traversal != 0 && c.traversal != 1) return fail(HF_ERR_ARG, "hf_camera.traversal must be 0 or 1");
    if (c.traversal == 1 && c.lod_pixels > 0.0)
        return fail(HF_ERR_ARG, "traversal 1 is not available with the coarse-level stop");
    if (!(c.lod_pixels >= 0.0 && c.lod_pixels <= 1e6)) return fail(HF_ERR_ARG, "lod_pixels must be in [0, 1e6]");
    return HF_OK;
}

}  // namespace

int hfi::noalloc_discretize_params(hf_ctx* ctx, const hf_camera* cam, float* const* tex,
                                   char* scratch, size_t scratch_bytes, hf_cascade_info* info_out,
                                   PrepParams* pp, DiscParams* dp, LookupTables* lt, ListsView* lv,
                                   CompactView* cv, bool* compact, DevStatus** status) {
    if (!ctx || !cam || !tex) return fail(HF_ERR_ARG, "null argument");
    if (!ctx->dev) return fail(HF_ERR_STATE, "persistent buffer not bound");
    const hf_camera& c = *cam;
    if (int rc = check_camera(c)) return rc;
    const int C = c.n_cascades, N = c.cascade_size;
    const size_t need = size_t(C) * size_t(N) * 16;
    if (need > scratch_bytes)
        return fail(HF_ERR_ARG, "n_cascades * cascade_size = %lld exceeds the %zu rows of the built-in scratch",
                    (long long)C * N, scratch_bytes / 16);
    for (int k = 0; k < C; ++k)
        if (!tex[k] || (reinterpret_cast<uintptr_t>(tex[k]) & 255))
            return fail(HF_ERR_ARG, "output texture %d is null or not 256-byte aligned", k);
    double eye_local[3] = {c.eye[0] - ctx->desc.origin_x, c.eye[1] - ctx->desc.origin_y, c.eye[2]};
    FitDomain dom{ctx->width, ctx->height, ctx->zmin, ctx->zmax, ctx->c_min};
    std::unique_ptr<FitResult> fit(new FitResult);
    int rc = fit_cascades(c, eye_local, dom, fit.get());
    if (rc) return fail(rc, "cascade fit produced an oversized polygon");
    std::memset(pp, 0, sizeof(*pp));
    std::memset(dp, 0, sizeof(*dp));
    pp->C = C;
    pp->max_N = N;
    pp->dom_w = ctx->width;
    pp->dom_h = ctx->height;
    pp->eps_frac = 1e-6;
    dp->C = C;
    dp->max_N = N;
    dp->precision = ctx->rbf.precision;
    dp->kernel = ctx->rbf.kernel;
    dp->K = float(std::exp(-ctx->rbf.radius * ctx->rbf.radius / (2.0 * ctx->rbf.sigma * ctx->rbf.sigma)));
    int2* spans = reinterpret_cast<int2*>(scratch);
    float* xs = reinterpret_cast<float*>(scratch + size_t(C) * N * 8);
    float* ys = xs + size_t(C) * N;
    for (int k = 0; k < C; ++k) {
        const hf_cascade_info& ci = fit->cas[k];
        PrepCascade& q = pp->cas[k];
        fill_prep_geometry(ci, N, q);
        q.spans = spans + size_t(k) * N;
        q.xs = xs + size_t(k) * N;
        q.ys = ys + size_t(k) * N;
        DiscCascade& d = dp->cas[k];
        d.N = N;
        d.spans = q.spans;
        d.xs = q.xs;
        d.ys = q.ys;
        d.tex = tex[k];
        if (info_out) {
            info_out[k] = ci;
            info_out[k].tex = tex[k];
            info_out[k].mip = nullptr;
            info_out[k].spans = nullptr;
            info_out[k].mip_floats = mip_floats(N);
            info_out[k].water_tex = nullptr;
        }
    }
    *lt = ctx->lookup_tables(true);
    *lv = ctx->lists();
    // the FP32 walk the context's own FP32 discretization uses: over FP16-format
    // compact lists where the context keeps them, else over the index lists
    *compact = ctx->compact_fmt == HF_PREC_FP16;
    if (*compact) *cv = ctx->compact();
    *status = ctx->d_status();
    return HF_OK;
}

int hfi::set_cuda_error(int e, const char* what) { return cuda_fail(e, what); }

int hfi::exception_status(const char* where) noexcept {
    try {
        throw;
    } catch (const std::bad_alloc&) {
        return fail(HF_ERR_HOST, "%s: out of host memory", where);
    } catch (const std::exception& x) {
        return fail(HF_ERR_HOST, "%s: %s", where, x.what());
    } catch (...) {
        return fail(HF_ERR_HOST, "%s: unknown host exception", where);
    }
}

extern "C" {

const char* hf_last_error(void) { return g_err.c_str(); }

int hf_create_quadtree(const hf_quadtree_desc* desc, const hf_leaf* leaves, int64_t n_leaves,
                       const hf_rbf_params* rbf, hf_ctx** out) {
    return guarded("hf_create_quadtree", [&]() -> int {
        ApiRange range_("hf_create_quadtree");
        if (!desc || !rbf || !out) return fail(HF_ERR_ARG, "null argument");
        if (n_leaves < 1 || !leaves) return fail(HF_ERR_ARG, "no leaves");
        if (n_leaves > std::numeric_limits<int32_t>::max())  // list entries are 32-bit leaf indices
            return fail(HF_ERR_ARG, "more than 2^31 - 1 leaves");
        const hf_quadtree_desc& d = *desc;
        if (!(std::isfinite(d.origin_x) && std::isfinite(d.origin_y) && std::isfinite(d.root_cell) &&
              d.root_cell > 0.0))
            return fail(HF_ERR_ARG, "origin / root_cell must be finite, root_cell > 0");
        if (d.root_nx < 1 || d.root_ny < 1) return fail(HF_ERR_ARG, "root grid must be at least 1x1");
        if (d.max_level < 0 || d.max_level > HF_MAX_LEVEL)
            return fail(HF_ERR_ARG, "max_level must be in [0, %d]", HF_MAX_LEVEL);
        const int M = d.max_level;
        const int64_t fnx = int64_t(d.root_nx) << M, fny = int64_t(d.root_ny) << M;
        if (fnx > (int64_t(1) << 30) || fny > (int64_t(1) << 30) || fnx * fny > (int64_t(1) << 34))
            return fail(HF_ERR_ARG, "finest grid %lld x %lld too large", (long long)fnx, (long long)fny);
        if (!(std::isfinite(rbf->sigma) && rbf->sigma > 0.0 && std::isfinite(rbf->radius) && rbf->radius > 0.0))
            return fail(HF_ERR_ARG, "sigma and radius must be finite and > 0");
        if (rbf->precision < HF_PREC_FP32 || rbf->precision > HF_PREC_BF16)
            return fail(HF_ERR_ARG, "unknown precision %d", rbf->precision);
        if (rbf->bucket_level > M) return fail(HF_ERR_ARG, "bucket_level %d > max_level %d", rbf->bucket_level, M);
        if (rbf->water != 0 && rbf->water != 1) return fail(HF_ERR_ARG, "water must be 0 or 1");
        if (rbf->kernel != HF_RBF_GAUSSIAN && rbf->kernel != HF_RBF_WENDLAND_C2)
            return fail(HF_ERR_ARG, "unknown RBF kernel %d", rbf->kernel);
        if (rbf->kernel != HF_RBF_GAUSSIAN && rbf->precision != HF_PREC_FP32)
            return fail(HF_ERR_ARG, "the Wendland kernel needs FP32 precision");
        if (rbf->water && rbf->precision != HF_PREC_FP32)
            return fail(HF_ERR_ARG, "the water layer needs FP32 precision");

        std::unique_ptr<hf_ctx> ctx(new hf_ctx);
        ctx->desc = d;
        ctx->rbf = *rbf;
        ctx->M = M;
        ctx->B = rbf->bucket_level < 0 ? std::max(0, M - 1) : rbf->bucket_level;
        ctx->n_leaves = n_leaves;
        if (const char* env = std::getenv("HF_CELLMAP_MAX_CELLS")) {
            char* end = nullptr;
            const long long v = std::strtoll(env, &end, 10);
            if (end != env && *end == '\0' && v >= 0) ctx->cellmap_max_cells = std::min<int64_t>(v, kCellMapMaxCells);
        }
        ctx->c_fin = d.root_cell / double(int64_t(1) << M);
        ctx->width = d.root_cell * d.root_nx;
        ctx->height = d.root_cell * d.root_ny;

        // occupancy, duplicates, ranges
        HostBitmaps& lf = ctx->leaves;
        lf.init(d.root_nx, d.root_ny, M);
        int lmin = M, lmax = 0;
        float vmin = INFINITY, vmax = -INFINITY;
        int64_t area = 0;
        for (int64_t k = 0; k < n_leaves; ++k) {
            const hf_leaf& l = leaves[k];
            if (l.level < 0 || l.level > M) return fail(HF_ERR_ARG, "leaf %lld: level %d out of range", (long long)k, l.level);
            if (l.ix < 0 || l.iy < 0 || l.ix >= lf.nx[l.level] || l.iy >= lf.ny[l.level])
                return fail(HF_ERR_ARG, "leaf %lld: index (%d, %d) outside level %d", (long long)k, l.ix, l.iy, l.level);
            if (!std::isfinite(l.value)) return fail(HF_ERR_ARG, "leaf %lld: value not finite", (long long)k);
            if (lf.test(l.level, l.ix, l.iy)) return fail(HF_ERR_ARG, "leaf %lld: duplicate cell", (long long)k);
            lf.set(l.level, l.ix, l.iy);
            lmin = std::min(lmin, l.level);
            lmax = std::max(lmax, l.level);
            vmin = std::min(vmin, l.value);
            vmax = std::max(vmax, l.value);
            area += int64_t(1) << (2 * (M - l.level));
        }
        // no leaf may lie inside another; with the area sum this is an exact tiling
        for (int64_t k = 0; k < n_leaves; ++k) {
            const hf_leaf& l = leaves[k];
            for (int A = 0; A < l.level; ++A)
                if (lf.test(A, l.ix >> (l.level - A), l.iy >> (l.level - A)))
                    return fail(HF_ERR_ARG, "leaf %lld lies inside a coarser leaf", (long long)k);
        }
        if (area != fnx * fny) return fail(HF_ERR_ARG, "leaves do not cover the domain (gap)");
        lf.finalize();
        ctx->c_min = d.root_cell / double(int64_t(1) << lmax);
        ctx->c_max = d.root_cell / double(int64_t(1) << lmin);
        ctx->zmin = vmin;
        ctx->zmax = vmax;
        ++ctx->data_version;
        if (rbf->water) ctx->depth.assign(size_t(n_leaves), 0.f);

        // records in (level, iy, ix) order: centre, weight scale, value
        const double log2e = 1.4426950408889634;
        ctx->perm.resize(size_t(n_leaves));
        ctx->recs.resize(size_t(n_leaves));
        for (int64_t k = 0; k < n_leaves; ++k) {
            const hf_leaf& l = leaves[k];
            const int64_t s = lf.rank(l.level, l.ix, l.iy);
            const double c = d.root_cell / double(int64_t(1) << l.level);
            ctx->perm[size_t(k)] = s;
            // exponent scale of the weight (see rbf_weight in hf_kernels.cu)
            const double scale = rbf->kernel == HF_RBF_WENDLAND_C2 ? 1.0 / (rbf->radius * c * rbf->radius * c)
                                                                   : -log2e / (2.0 * rbf->sigma * rbf->sigma * c * c);
            ctx->recs[size_t(s)] = make_float4(float((l.ix + 0.5) * c), float((l.iy + 0.5) * c), float(scale), l.value);
        }

        // buckets: leaves at or below level B, coarser leaves split down to B
        HostBitmaps& bk = ctx->buckets;
        bk.init(d.root_nx, d.root_ny, M);
        const int B = ctx->B;
        for (int64_t k = 0; k < n_leaves; ++k) {
            const hf_leaf& l = leaves[k];
            if (l.level >= B) {
                bk.set(l.level, l.ix, l.iy);
            } else {
                const int sh = B - l.level;
                for (int64_t y = int64_t(l.iy) << sh; y < (int64_t(l.iy) + 1) << sh; ++y)
                    for (int64_t x = int64_t(l.ix) << sh; x < (int64_t(l.ix) + 1) << sh; ++x) bk.set(B, x, y);
            }
        }
        bk.finalize();
        ctx->n_buckets = bk.base[M + 1];

        // reach of a level-L centre, R c_L plus a margin covering FP32 rounding of
        // texel positions, in units of half a finest cell
        const double ext = std::max(ctx->width, ctx->height);
        const double ulp = std::ldexp(1.0, std::ilogb(ext) - 23);
        const double margin = std::max(1e-3 * ctx->c_fin, 8.0 * ulp);
        const double q = 0.5 * ctx->c_fin;
        for (int L = 0; L <= M; ++L)
            ctx->reach_q[L] = (rbf->radius * (d.root_cell / double(int64_t(1) << L)) + margin) / q;

        std::vector<int64_t> counts(size_t(ctx->n_buckets), 0);
        const int nt = std::max(1, std::min(64, int(std::thread::hardware_concurrency())));
        count_lists_host(ctx->enum_tables(false), ctx->lookup_tables(false), counts.data(), nt);
        ctx->offsets.resize(size_t(ctx->n_buckets) + 1);
        int64_t run = 0;
        for (int64_t b = 0; b < ctx->n_buckets; ++b) {
            ctx->offsets[size_t(b)] = run;
            run += (counts[size_t(b)] + kListPad - 1) / kListPad * kListPad;  // padded to groups of four
        }
        ctx->offsets[size_t(ctx->n_buckets)] = run;
        ctx->n_cand = run;
        // bucket-relative offsets of the compact lists must be exact small integers in the 16-bit type
        double rmax = 0.0;
        for (int L = 0; L <= M; ++L)
            if (lf.base[L + 1] > lf.base[L]) rmax = std::max(rmax, ctx->reach_q[L]);
        const double span = rmax + double(int64_t(1) << (M - ctx->B + 1)) + 1.0;
        if (rbf->precision == HF_PREC_FP32) {
            const char* env = std::getenv("HF_FP32_INDEX_LISTS");
            const bool forced = env && env[0] && std::strcmp(env, "0") != 0;
            if (!rbf->water && span <= 1024.0 && !forced) {
                ctx->compact_fmt = HF_PREC_FP16;
                // FP32 weight scale per squared half-cell of the finest level (c = 2 q):
                // Gaussian -log2(e) / (8 sigma^2), Wendland 1 / (4 radius^2); level L's is
                // 4^(M - L) times smaller, built in the exponent field
                const float kM = rbf->kernel == HF_RBF_WENDLAND_C2 ? float(1.0 / (4.0 * rbf->radius * rbf->radius))
                                                                   : float(-log2e / (8.0 * rbf->sigma * rbf->sigma));
                const float kL = float(std::ldexp(double(kM), -2 * (M - lmin)));
                if (!(std::fabs(kL) >= std::numeric_limits<float>::min()) || !std::isfinite(kM))
                    ctx->compact_fmt = 0;  // scales outside the normal range: the index lists serve
                else
                    std::memcpy(&ctx->kf_bits, &kM, 4);
            }
        }
        if (rbf->precision != HF_PREC_FP32) {
            ctx->compact_fmt = rbf->precision;
            const double limit = rbf->precision == HF_PREC_FP16 ? 1024.0 : 256.0;
            if (span > limit)
                return fail(HF_ERR_ARG, "candidate offsets span %.0f half-cells, more than the %s path holds exactly (%.0f)",
                            span, rbf->precision == HF_PREC_FP16 ? "FP16" : "BF16", limit);
            // exponent scales per squared half-cell: the finest level's is -log2(e) / (8 sigma^2);
            // level L's lowers the exponent by 2 (M - L), which must stay a normal number
            const bool f16 = rbf->precision == HF_PREC_FP16;
            const float kM = float(-log2e / (8.0 * rbf->sigma * rbf->sigma));
            std::memcpy(&ctx->kf_bits, &kM, 4);
            const uint32_t kMb = f16 ? f16_bits(kM) : bf16_bits(kM);
            const int shift = f16 ? 10 : 7, emask = f16 ? 31 : 255;
            const int eM = kMb == std::numeric_limits<uint32_t>::max() ? 0 : int((kMb >> shift) & uint32_t(emask));
            if (eM >= emask || eM - 2 * (M - lmin) < 1)
                return fail(HF_ERR_ARG, "the %s exponent scales of levels %d..%d leave the normal range",
                            f16 ? "FP16" : "BF16", lmin, M);
            const uint32_t step = 2u << shift;
            const uint32_t kb = kMb - uint32_t(M) * step;  // level 0's bits, modulo 2^32
            ctx->kb2 = kb * 0x10001u;
        }
        if (ctx->compact_fmt != 0) {
            ctx->pair_offsets.resize(size_t(ctx->n_buckets) + 1);
            int64_t pr = 0;
            for (int64_t b = 0; b < ctx->n_buckets; ++b) {
                ctx->pair_offsets[size_t(b)] = pr;
                pr += (counts[size_t(b)] + 1) / 2;
                ctx->max_pairs = std::max(ctx->max_pairs, (counts[size_t(b)] + 1) / 2);
            }
            ctx->pair_offsets[size_t(ctx->n_buckets)] = pr;
            ctx->n_pairs = pr;
        }
        ctx->lay = ctx->layout();
        *out = ctx.release();
        g_err.clear();
        return HF_OK;
    });
}

int hf_query_bytes(const hf_ctx* ctx, int32_t n_cascades, int32_t cascade_size,
                   size_t* persistent_bytes, size_t* view_bytes) {
    return guarded("hf_query_bytes", [&]() -> int {
        if (!ctx) return fail(HF_ERR_ARG, "null context");
        if (persistent_bytes) *persistent_bytes = ctx->lay.total;
        if (view_bytes) {
            if (n_cascades < 1 || n_cascades > HF_MAX_CASCADES || cascade_size < 2 || cascade_size > kMaxCascadeSize)
                return fail(HF_ERR_ARG, "cascades must be 1..%d of side 2..%d", HF_MAX_CASCADES, kMaxCascadeSize);
            *view_bytes = per_view_bytes(n_cascades, cascade_size, ctx->rbf.water != 0);
        }
        return HF_OK;
    });
}

int hf_bind_persistent(hf_ctx* ctx, void* dev_persistent, size_t bytes, void* stream) {
    return guarded("hf_bind_persistent", [&]() -> int {
        ApiRange range_("hf_bind_persistent");
        if (!ctx || !dev_persistent) return fail(HF_ERR_ARG, "null argument");
        if (reinterpret_cast<uintptr_t>(dev_persistent) & 255) return fail(HF_ERR_ARG, "buffer must be 256-byte aligned");
        if (bytes < ctx->lay.total)
            return fail(HF_ERR_NOMEM, "persistent buffer has %zu bytes, %zu needed", bytes, ctx->lay.total);
        cudaStream_t s = cudaStream_t(stream);
        char* dev = static_cast<char*>(dev_persistent);
        const PersistentLayout& l = ctx->lay;
        int e = cudaMemsetAsync(dev + l.status, 0, sizeof(DevStatus), s);
        if (!e) e = cudaMemcpyAsync(dev + l.lbits, ctx->leaves.bits.data(), ctx->leaves.bits.size() * 8, cudaMemcpyHostToDevice, s);
        if (!e) e = cudaMemcpyAsync(dev + l.lprefix, ctx->leaves.prefix.data(), ctx->leaves.prefix.size() * 4, cudaMemcpyHostToDevice, s);
        if (!e) e = cudaMemcpyAsync(dev + l.bbits, ctx->buckets.bits.data(), ctx->buckets.bits.size() * 8, cudaMemcpyHostToDevice, s);
        if (!e) e = cudaMemcpyAsync(dev + l.bprefix, ctx->buckets.prefix.data(), ctx->buckets.prefix.size() * 4, cudaMemcpyHostToDevice, s);
        if (!e) e = cudaMemcpyAsync(dev + l.recs, ctx->recs.data(), ctx->recs.size() * 16, cudaMemcpyHostToDevice, s);
        if (!e) e = cudaMemcpyAsync(dev + l.offsets, ctx->offsets.data(), ctx->offsets.size() * 8, cudaMemcpyHostToDevice, s);
        if (!e && ctx->compact_fmt != 0)
            e = cudaMemcpyAsync(dev + l.pair_offsets, ctx->pair_offsets.data(), ctx->pair_offsets.size() * 8,
                                cudaMemcpyHostToDevice, s);
        if (!e && ctx->rbf.water)
            e = cudaMemcpyAsync(dev + l.depth, ctx->depth.data(), ctx->depth.size() * 4, cudaMemcpyHostToDevice, s);
        // the null record that pads the lists: centre far away (its squared
        // distance stays finite), a weight scale of the kernel's sign, value 0
        // and depth 0, so that its weight and its terms are exactly 0
        static const float4 null_gauss = make_float4(1e18f, 1e18f, -1.f, 0.f);
        static const float4 null_wend = make_float4(1e18f, 1e18f, 1.f, 0.f);
        if (!e)
            e = cudaMemcpyAsync(dev + l.recs + size_t(ctx->n_leaves) * 16,
                                ctx->rbf.kernel == HF_RBF_WENDLAND_C2 ? &null_wend : &null_gauss, 16,
                                cudaMemcpyHostToDevice, s);
        if (!e && ctx->rbf.water) e = cudaMemsetAsync(dev + l.depth + size_t(ctx->n_leaves) * 4, 0, 4, s);
        if (e) return cuda_fail(e, "upload of the quadtree");
        ctx->dev = dev;
        ctx->dev_bytes = bytes;
        e = launch_fill_lists(ctx->enum_tables(true), ctx->lookup_tables(true), ctx->lists(), ctx->d_status(), stream);
        if (e) return cuda_fail(e, "influence-list kernel launch");
        if (ctx->keep_cellmap()) {
            e = launch_fill_cellmap(ctx->lookup_tables(true), ctx->lists(), reinterpret_cast<uint2*>(dev + l.cellmap),
                                    ctx->d_status(), stream);
            if (e) return cuda_fail(e, "cell-map kernel launch");
        }
        if (ctx->compact_fmt != 0) {
            e = launch_fill_compact(ctx->enum_tables(true), ctx->lookup_tables(true), ctx->lists(), ctx->compact(),
                                    ctx->compact_fmt, stream);
            if (e) return cuda_fail(e, "compact-list kernel launch");
            if (ctx->keep_pair_cellmap()) {
                const CompactView cv = ctx->compact();
                e = launch_fill_cellmap(ctx->lookup_tables(true), ctx->lists(),
                                        reinterpret_cast<uint2*>(dev + l.pair_cellmap), ctx->d_status(), stream, &cv);
                if (e) return cuda_fail(e, "compact cell-map kernel launch");
            }
        }
        e = cudaStreamSynchronize(s);
        if (e) return cuda_fail(e, "influence-list build");
        DevStatus st;
        e = cudaMemcpy(&st, ctx->d_status(), 8, cudaMemcpyDeviceToHost);
        if (e) return cuda_fail(e, "status read-back");
        if (st.flags) {
            ctx->dev = nullptr;
            return fail(HF_ERR_DATA, "influence-list build disagreed with the host count at bucket %u", st.detail);
        }
        return HF_OK;
    });
}

int hf_update_values(hf_ctx* ctx, const float* values, int64_t n_values, void* stream) {
    return guarded("hf_update_values", [&]() -> int {
        ApiRange range_("hf_update_values");
        if (!ctx || !values) return fail(HF_ERR_ARG, "null argument");
        if (n_values != ctx->n_leaves) return fail(HF_ERR_ARG, "expected %lld values", (long long)ctx->n_leaves);
        if (!ctx->dev) return fail(HF_ERR_STATE, "persistent buffer not bound");
        for (int64_t k = 0; k < n_values; ++k)  // validate before touching any state
            if (!std::isfinite(values[k])) return fail(HF_ERR_ARG, "value %lld not finite", (long long)k);
        ctx->staged.resize(size_t(n_values));
        float vmin = INFINITY, vmax = -INFINITY;
        for (int64_t k = 0; k < n_values; ++k) {
            const int64_t s = ctx->perm[size_t(k)];
            ctx->staged[size_t(s)] = values[k];
            ctx->recs[size_t(s)].w = values[k];
            vmin = std::min(vmin, values[k]);
            vmax = std::max(vmax, values[k]);
        }
        ctx->zmin = vmin;
        ctx->zmax = vmax;
        ++ctx->data_version;
        for (size_t k = 0; k < ctx->depth.size(); ++k)
            if (ctx->depth[k] > 0.f) ctx->zmax = std::max(double(ctx->zmax), double(ctx->recs[k].w) + ctx->depth[k]);
        cudaStream_t s = cudaStream_t(stream);
        int e = cudaMemcpy2DAsync(ctx->dev + ctx->lay.recs + 12, 16, ctx->staged.data(), 4, 4, size_t(n_values),
                                  cudaMemcpyHostToDevice, s);
        if (!e && ctx->compact_fmt != 0)  // the compact lists carry copies of the values
            e = launch_fill_compact(ctx->enum_tables(true), ctx->lookup_tables(true), ctx->lists(), ctx->compact(),
                                    ctx->compact_fmt, stream);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) return cuda_fail(e, "value upload");
        return HF_OK;
    });
}

int hf_update_water(hf_ctx* ctx, const float* depths, int64_t n_depths, void* stream) {
    return guarded("hf_update_water", [&]() -> int {
        ApiRange range_("hf_update_water");
        if (!ctx || !depths) return fail(HF_ERR_ARG, "null argument");
        if (!ctx->rbf.water) return fail(HF_ERR_STATE, "context was created without the water layer");
        if (n_depths != ctx->n_leaves) return fail(HF_ERR_ARG, "expected %lld depths", (long long)ctx->n_leaves);
        if (!ctx->dev) return fail(HF_ERR_STATE, "persistent buffer not bound");
        for (int64_t k = 0; k < n_depths; ++k)
            if (!(std::isfinite(depths[k]) && depths[k] >= 0.f))
                return fail(HF_ERR_ARG, "depth %lld must be finite and >= 0", (long long)k);
        double zmax = -INFINITY;
        for (int64_t k = 0; k < n_depths; ++k) {
            const int64_t s = ctx->perm[size_t(k)];
            ctx->depth[size_t(s)] = depths[k];
        }
        for (int64_t s = 0; s < n_depths; ++s)
            zmax = std::max(zmax, double(ctx->recs[size_t(s)].w) + (ctx->depth[size_t(s)] > 0.f ? ctx->depth[size_t(s)] : 0.0));
        ctx->zmax = zmax;
        ++ctx->data_version;
        cudaStream_t s = cudaStream_t(stream);
        int e = cudaMemcpyAsync(ctx->dev + ctx->lay.depth, ctx->depth.data(), ctx->depth.size() * 4, cudaMemcpyHostToDevice, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) return cuda_fail(e, "depth upload");
        return HF_OK;
    });
}

namespace {

int set_camera(hf_ctx* ctx, int32_t slot, const hf_camera* cam, void* dev_view, size_t bytes,
               const int64_t* follow) {
    if (!ctx || !cam || !dev_view) return fail(HF_ERR_ARG, "null argument");
    if (slot < 0 || slot >= HF_MAX_VIEWS) return fail(HF_ERR_ARG, "view slot %d out of range", slot);
    const hf_camera& c = *cam;
    if (int rc = check_camera(c)) return rc;
    if (c.lod_pixels > 0.0 && ctx->rbf.water)
        return fail(HF_ERR_ARG, "the coarse-level stop is not available with the water layer");
    if (c.traversal == 1 && ctx->rbf.water)
        return fail(HF_ERR_ARG, "traversal 1 is not available with the water layer");
    if (reinterpret_cast<uintptr_t>(dev_view) & 255) return fail(HF_ERR_ARG, "view buffer must be 256-byte aligned");
    const size_t need = per_view_bytes(c.n_cascades, c.cascade_size, ctx->rbf.water != 0);
    if (bytes < need) return fail(HF_ERR_NOMEM, "view buffer has %zu bytes, %zu needed", bytes, need);
    if (!ctx->views[slot]) ctx->views[slot].reset(new ViewSlot);
    ViewSlot& v = *ctx->views[slot];
    v.stage = 0;
    v.cam = c;
    v.eye_local[0] = c.eye[0] - ctx->desc.origin_x;
    v.eye_local[1] = c.eye[1] - ctx->desc.origin_y;
    v.eye_local[2] = c.eye[2];
    FitDomain dom{ctx->width, ctx->height, ctx->zmin, ctx->zmax, ctx->c_min};
    int rc = fit_cascades(c, v.eye_local, dom, &v.fit, follow);
    if (rc) return fail(rc, "cascade fit produced an oversized polygon");
    v.dev = static_cast<char*>(dev_view);
    v.bytes = bytes;
    const int N = c.cascade_size;
    size_t o = 0;
    for (int k = 0; k < c.n_cascades; ++k) {
        v.tex[k] = reinterpret_cast<float*>(v.dev + o); o = align256(o + size_t(N) * N * 4);
        v.mip[k] = reinterpret_cast<float*>(v.dev + o); o = align256(o + size_t(mip_floats(N)) * 4);
        if (ctx->rbf.water) {
            v.wtex[k] = reinterpret_cast<float*>(v.dev + o); o = align256(o + size_t(N) * N * 4);
        } else {
            v.wtex[k] = nullptr;
        }
        v.spans[k] = reinterpret_cast<int2*>(v.dev + o); o = align256(o + size_t(N) * 8);
        v.xs[k] = reinterpret_cast<float*>(v.dev + o); o = align256(o + size_t(N) * 4);
        v.ys[k] = reinterpret_cast<float*>(v.dev + o); o = align256(o + size_t(N) * 4);
        hf_cascade_info& ci = v.fit.cas[k];
        ci.tex = v.tex[k];
        ci.mip = v.mip[k];
        ci.spans = reinterpret_cast<int32_t*>(v.spans[k]);
        ci.mip_floats = mip_floats(N);
        ci.water_tex = v.wtex[k];
    }
    v.stage = 1;
    return HF_OK;
}

}  // namespace

int hf_set_camera(hf_ctx* ctx, int32_t slot, const hf_camera* cam, void* dev_view, size_t bytes) {
    return guarded("hf_set_camera", [&]() -> int {
        ApiRange range_("hf_set_camera");
        return set_camera(ctx, slot, cam, dev_view, bytes, nullptr);
    });
}

int hf_set_camera_follow(hf_ctx* ctx, int32_t slot, const hf_camera* cam, void* dev_view, size_t bytes,
                         int32_t prev_slot) {
    return guarded("hf_set_camera_follow", [&]() -> int {
        ApiRange range_("hf_set_camera_follow");
        if (!ctx || !cam) return fail(HF_ERR_ARG, "null argument");
        const ViewSlot* p = get_view(ctx, prev_slot);
        if (!p || p->stage < 1) return fail(HF_ERR_STATE, "view slot %d has no camera to follow", prev_slot);
        int64_t follow[HF_MAX_CASCADES];
        for (int k = 0; k < HF_MAX_CASCADES; ++k)  // no step to keep: never one above the fitted one
            follow[k] = std::numeric_limits<int64_t>::min();
        if (p->cam.texel_ladder == cam->texel_ladder && cam->texel_ladder > 0)
            for (int k = 0; k < p->cam.n_cascades; ++k)
                if (p->fit.cas[k].n_poly >= 3) follow[k] = p->fit.cas[k].snap_k;
        return set_camera(ctx, slot, cam, dev_view, bytes, follow);
    });
}

namespace {

DiscParams disc_params(const hf_ctx* ctx, const ViewSlot* v) {
    const int C = v->cam.n_cascades, N = v->cam.cascade_size;
    DiscParams dp;
    std::memset(&dp, 0, sizeof(dp));
    dp.C = C;
    dp.max_N = N;
    dp.precision = ctx->rbf.precision;
    dp.water = ctx->rbf.water;
    dp.kernel = ctx->rbf.kernel;
    dp.K = float(std::exp(-ctx->rbf.radius * ctx->rbf.radius / (2.0 * ctx->rbf.sigma * ctx->rbf.sigma)));
    for (int k = 0; k < C; ++k) {
        DiscCascade& dc = dp.cas[k];
        dc.N = N;
        dc.spans = v->spans[k];
        dc.xs = v->xs[k];
        dc.ys = v->ys[k];
        dc.tex = v->tex[k];
        dc.wtex = v->wtex[k];
        dc.prev = v->reuse[k].tex;
        dc.prev_w = v->reuse[k].wtex;
        dc.prev_N = v->reuse[k].N;
        dc.prev_di = v->reuse[k].di;
        dc.prev_dj = v->reuse[k].dj;
    }
    return dp;
}

}  // namespace

namespace {

// Grown-polygon edge constraints and buffers of cascade k for the row kernel.
void fill_prep_cascade(const ViewSlot* v, int k, PrepCascade& q) {
    fill_prep_geometry(v->fit.cas[k], v->cam.cascade_size, q);
    q.spans = v->spans[k];
    q.xs = v->xs[k];
    q.ys = v->ys[k];
}

}  // namespace

namespace {

int discretize_view(hf_ctx* ctx, ViewSlot* v, void* stream) {
    const int C = v->cam.n_cascades, N = v->cam.cascade_size;
    PrepParams pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.C = C;
    pp.max_N = N;
    pp.dom_w = ctx->width;
    pp.dom_h = ctx->height;
    pp.eps_frac = 1e-6;
    for (int k = 0; k < C; ++k) fill_prep_cascade(v, k, pp.cas[k]);
    int e = launch_prep(pp, stream);
    if (e) return cuda_fail(e, "visible-row kernel launch");
    if (ctx->fp32_compact() && !ctx->rbf.water)
        e = launch_discretize_f32c(disc_params(ctx, v), ctx->lookup_tables(true), ctx->compact(), ctx->d_status(),
                                   stream);
    else if (ctx->rbf.precision == HF_PREC_FP32)
        e = launch_discretize(disc_params(ctx, v), ctx->lookup_tables(true), ctx->lists(), ctx->d_status(), stream);
    else
        e = launch_discretize_mixed(disc_params(ctx, v), ctx->lookup_tables(true), ctx->compact(), ctx->d_status(),
                                    stream);
    if (e) return cuda_fail(e, "discretization kernel launch");
    v->stage = 2;
    v->data_version = ctx->data_version;
    return HF_OK;
}

// The earlier frame's cascade whose texel lattice matches cascade k of v and
// overlaps it most: lattice fit, the same spacing; stable fit, the same fit.
int reuse_source(const ViewSlot* v, int k, const ViewSlot* p, ViewSlot::Reuse* r) {
    const hf_cascade_info& a = v->fit.cas[k];
    const int N = v->cam.cascade_size;
    int best = -1;
    int64_t best_area = 0;
    if (a.n_poly < 3) return -1;
    for (int q = 0; q < p->cam.n_cascades; ++q) {
        const hf_cascade_info& b = p->fit.cas[q];
        const int M = p->cam.cascade_size;
        if (b.n_poly < 3 || a.texel_ladder != b.texel_ladder) continue;
        int64_t di = 0, dj = 0;
        if (a.texel_ladder > 0) {
            if (a.snap_k != b.snap_k || a.texel != b.texel) continue;
            di = a.snap_x - b.snap_x;
            dj = a.snap_y - b.snap_y;
        } else if (a.snap_x != b.snap_x || a.snap_y != b.snap_y || a.snap_k != b.snap_k || N != M) {
            continue;
        }
        // texel i of v is texel i + di of p: the overlap of [di, di + N) and [0, M)
        const int64_t wx = std::min<int64_t>(di + N, M) - std::max<int64_t>(di, 0);
        const int64_t wy = std::min<int64_t>(dj + N, M) - std::max<int64_t>(dj, 0);
        if (wx <= 0 || wy <= 0 || wx * wy <= best_area) continue;
        best = q;
        best_area = wx * wy;
        r->tex = p->tex[q];
        r->wtex = p->wtex[q];
        r->N = M;
        r->di = int32_t(di);
        r->dj = int32_t(dj);
    }
    return best;
}

}  // namespace

int hf_discretize_cascades(hf_ctx* ctx, int32_t slot, void* stream) {
    return guarded("hf_discretize_cascades", [&]() -> int {
        ApiRange range_("hf_discretize_cascades");
        ViewSlot* v = get_view(ctx, slot);
        if (!v || v->stage < 1) return fail(HF_ERR_STATE, "view slot %d has no camera", slot);
        if (!ctx->dev) return fail(HF_ERR_STATE, "persistent buffer not bound");
        for (int k = 0; k < HF_MAX_CASCADES; ++k) {
            v->reuse[k] = ViewSlot::Reuse();
            v->fit.cas[k].reuse_source = -1;
        }
        return discretize_view(ctx, v, stream);
    });
}

int hf_discretize_reuse(hf_ctx* ctx, int32_t slot, int32_t prev_slot, void* stream) {
    return guarded("hf_discretize_reuse", [&]() -> int {
        ApiRange range_("hf_discretize_reuse");
        ViewSlot* v = get_view(ctx, slot);
        if (!v || v->stage < 1) return fail(HF_ERR_STATE, "view slot %d has no camera", slot);
        if (!ctx->dev) return fail(HF_ERR_STATE, "persistent buffer not bound");
        if (prev_slot == slot) return fail(HF_ERR_ARG, "a slot cannot reuse its own texels");
        const ViewSlot* p = get_view(ctx, prev_slot);
        if (!p || p->stage < 2) return fail(HF_ERR_STATE, "view slot %d holds no discretized frame", prev_slot);
        if (v->dev < p->dev + p->bytes && p->dev < v->dev + v->bytes)
            return fail(HF_ERR_ARG, "view slots %d and %d share buffer memory", slot, prev_slot);
        const bool same_data = p->data_version == ctx->data_version;
        for (int k = 0; k < HF_MAX_CASCADES; ++k) {
            v->reuse[k] = ViewSlot::Reuse();
            v->fit.cas[k].reuse_source = -1;
        }
        for (int k = 0; k < v->cam.n_cascades && same_data; ++k) {
            ViewSlot::Reuse r;
            const int q = reuse_source(v, k, p, &r);
            if (q < 0) continue;
            v->reuse[k] = r;
            v->fit.cas[k].reuse_source = q;
        }
        return discretize_view(ctx, v, stream);
    });
}

int hf_build_maxmip(hf_ctx* ctx, int32_t slot, void* stream) {
    return guarded("hf_build_maxmip", [&]() -> int {
        ApiRange range_("hf_build_maxmip");
        ViewSlot* v = get_view(ctx, slot);
        if (!v || v->stage < 2) return fail(HF_ERR_STATE, "view slot %d is not discretized", slot);
        const int C = v->cam.n_cascades, N = v->cam.cascade_size;
        MipParams mp;
        std::memset(&mp, 0, sizeof(mp));
        mp.C = C;
        mp.max_P = mip_pow2(N);
        mp.max_K = mip_levels(mp.max_P);
        mp.two = ctx->rbf.water;
        for (int k = 0; k < C; ++k) {
            mp.cas[k].tex = v->tex[k];
            mp.cas[k].wtex = v->wtex[k];
            mp.cas[k].spans = v->spans[k];
            mp.cas[k].mip = v->mip[k];
            mp.cas[k].N = N;
            mp.cas[k].P = mp.max_P;
            mp.cas[k].K = mp.max_K;
        }
        int e = launch_maxmip(mp, stream);
        if (e) return cuda_fail(e, "max-mip kernel launch");
        v->stage = 3;
        return HF_OK;
    });
}

namespace {

RayParams ray_params(const ViewSlot* v, bool water) {
    const hf_camera& c = v->cam;
    const FitResult& f = v->fit;
    RayParams rp;
    std::memset(&rp, 0, sizeof(rp));
    rp.C = c.n_cascades;
    rp.water = water ? 1 : 0;
    rp.jump = c.traversal == 1 ? 1 : 0;
    rp.W = c.width;
    rp.H = c.height;
    rp.ez = float(v->eye_local[2]);
    for (int a = 0; a < 3; ++a) {
        rp.F[a] = float(f.F[a]);
        rp.R[a] = float(f.R[a]);
        rp.U[a] = float(f.U[a]);
    }
    {
        // pixel centre x + 1/2 maps to (2 (x + 1/2) / W - 1) tan_h, y + 1/2 to (1 - 2 (y + 1/2) / H) tan_v
        const double tv = std::tan(0.5 * c.vfov), th = tv * double(c.width) / double(c.height);
        rp.px_a = float(2.0 * th / c.width);
        rp.px_b = float(th * (1.0 / c.width - 1.0));
        rp.py_a = float(-2.0 * tv / c.height);
        rp.py_b = float(tv * (1.0 - 1.0 / c.height));
    }
    rp.dir2x = float(f.dir2[0]);
    rp.dir2y = float(f.dir2[1]);
    rp.znear = float(c.znear);
    rp.zfar = float(c.zfar);
    const int N = c.cascade_size, P = mip_pow2(N);
    for (int k = 0; k < rp.C; ++k) {
        const hf_cascade_info& ci = f.cas[k];
        RayCascade& rc = rp.cas[k];
        rc.tex = v->tex[k];
        rc.mip = v->mip[k];
        rc.wtex = v->wtex[k];
        rc.N = N;
        rc.P = P;
        rc.K = mip_levels(P);
        rc.eu = float((v->eye_local[0] - ci.ox) / ci.texel);
        rc.ev = float((v->eye_local[1] - ci.oy) / ci.texel);
        rc.h = float(ci.texel);
        rc.inv_h = float(1.0 / ci.texel);
        rc.near_d = float(ci.near_depth);
        rc.far_ext = float(ci.far_ext_depth);
        rc.budget = 8 * (2 * N + 8) * (rc.K + 2);
        rc.stop_level = std::min(ci.stop_level, rc.K);
        if (rc.stop_level > 0) rp.coarse = 1;
        int64_t off = 0;
        for (int L = 0; L < kMaxLevels; ++L) {
            rc.lvl_off[L] = int32_t(off);
            if (L <= rc.K) off += int64_t(P >> L) * (P >> L);
        }
    }
    return rp;
}

}  // namespace

namespace {

// Kernel outputs may be device memory, managed memory or pinned host memory
// mapped at the same address (the kernel then writes over the host link
// itself); pageable host memory would fault the kernel and is refused.
int check_kernel_output(const void* p, const char* what) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return fail(HF_ERR_ARG, "%s is not an address CUDA knows", what);
    }
    if (a.type == cudaMemoryTypeUnregistered)
        return fail(HF_ERR_ARG, "%s is pageable host memory: pass device memory or pinned host memory", what);
    if (a.type == cudaMemoryTypeHost && a.devicePointer != p)
        return fail(HF_ERR_ARG, "%s is pinned host memory not mapped at the same device address", what);
    return HF_OK;
}

// True for pinned host memory (an address check_kernel_output accepted).
bool host_memory(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

}  // namespace

int hf_raycast(hf_ctx* ctx, int32_t slot, float* t_dev, uint8_t* hit_dev, void* stream) {
    return guarded("hf_raycast", [&]() -> int {
        ApiRange range_("hf_raycast");
        ViewSlot* v = get_view(ctx, slot);
        if (!v || v->stage < 3) return fail(HF_ERR_STATE, "view slot %d has no max mipmap", slot);
        if (!t_dev || !hit_dev) return fail(HF_ERR_ARG, "null output buffer");
        if (int rc = check_kernel_output(t_dev, "t output")) return rc;
        if (int rc = check_kernel_output(hit_dev, "hit output")) return rc;
        RayParams rp = ray_params(v, ctx->rbf.water != 0);
        rp.t_out = t_dev;
        rp.hit_out = hit_dev;
        rp.host_out = (host_memory(t_dev) || host_memory(hit_dev)) ? 1 : 0;
        int e = launch_raycast(rp, ctx->d_status(), stream);
        if (e) return cuda_fail(e, "ray-cast kernel launch");
        return HF_OK;
    });
}

int hf_ray_stats(hf_ctx* ctx, int32_t slot, int64_t* visits, int64_t* patch_tests, void* stream) {
    return guarded("hf_ray_stats", [&]() -> int {
        ApiRange range_("hf_ray_stats");
        ViewSlot* v = get_view(ctx, slot);
        if (!visits || !patch_tests) return fail(HF_ERR_ARG, "null argument");
        if (!v || v->stage < 3) return fail(HF_ERR_STATE, "view slot %d has no max mipmap", slot);
        cudaStream_t s = cudaStream_t(stream);
        DevStatus* st = ctx->d_status();
        int e = cudaMemsetAsync(st->ray_counters, 0, sizeof(st->ray_counters), s);
        if (!e) e = launch_raycast_count(ray_params(v, ctx->rbf.water != 0), st, stream);
        if (e) return cuda_fail(e, "ray counting pass launch");
        unsigned long long c[2];
        e = cudaMemcpyAsync(c, st->ray_counters, sizeof(c), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) return cuda_fail(e, "ray counting pass");
        *visits = int64_t(c[0]);
        *patch_tests = int64_t(c[1]);
        return HF_OK;
    });
}

int hf_view_stats(hf_ctx* ctx, int32_t slot, hf_view_stats_t* out, void* stream) {
    return guarded("hf_view_stats", [&]() -> int {
        ApiRange range_("hf_view_stats");
        ViewSlot* v = get_view(ctx, slot);
        if (!out) return fail(HF_ERR_ARG, "null argument");
        if (!v || v->stage < 2) return fail(HF_ERR_STATE, "view slot %d is not discretized", slot);
        cudaStream_t s = cudaStream_t(stream);
        DevStatus* st = ctx->d_status();
        int e = cudaMemsetAsync(st->counters, 0, sizeof(st->counters), s);
        if (!e) e = launch_stats(disc_params(ctx, v), ctx->lookup_tables(true), ctx->lists(), st, stream);
        if (e) return cuda_fail(e, "counting pass launch");
        unsigned long long c[4 * HF_MAX_CASCADES];
        e = cudaMemcpyAsync(c, st->counters, sizeof(c), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) return cuda_fail(e, "counting pass");
        std::memset(out, 0, sizeof(*out));
        for (int k = 0; k < v->cam.n_cascades; ++k) {
            out->visible_texels[k] = int64_t(c[k]);
            out->candidates[k] = int64_t(c[HF_MAX_CASCADES + k]);
            out->influencers[k] = int64_t(c[2 * HF_MAX_CASCADES + k]);
            out->reused_texels[k] = int64_t(c[3 * HF_MAX_CASCADES + k]);
        }
        return HF_OK;
    });
}

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct BatchPlan {
    int n_cascades = 0;
    size_t items_off = 0, cascades_off = 0, bases_off = 0, item_bases_off = 0, counters_off = 0, total = 0;
};

int plan_batch(const hf_batch_item* items, int32_t n, BatchPlan* plan) {
    if (!items || n < 1) return fail(HF_ERR_ARG, "empty batch");
    int nc = 0;
    for (int32_t i = 0; i < n; ++i) {
        const hf_batch_item& it = items[i];
        ViewSlot* v = get_view(it.ctx, it.view_slot);
        if (!v || v->stage < 1) return fail(HF_ERR_STATE, "batch item %d: view slot %d has no camera", i, it.view_slot);
        if (!it.ctx->dev) return fail(HF_ERR_STATE, "batch item %d: persistent buffer not bound", i);
        if (it.ctx->rbf.water) return fail(HF_ERR_ARG, "batch item %d: batched frames do not carry the water layer", i);
        if (it.ctx->rbf.kernel != HF_RBF_GAUSSIAN)
            return fail(HF_ERR_ARG, "batch item %d: batched frames use the Gaussian kernel only", i);
        if (v->cam.traversal != 0)
            return fail(HF_ERR_ARG, "batch item %d: batched frames use traversal 0 only", i);
        if (!it.t_dev || !it.hit_dev) return fail(HF_ERR_ARG, "batch item %d: null output buffer", i);
        nc += v->cam.n_cascades;
    }
    plan->n_cascades = nc;
    plan->items_off = align_up(sizeof(BatchHeader), 256);
    plan->cascades_off = align_up(plan->items_off + size_t(n) * sizeof(BatchItem), 256);
    plan->bases_off = align_up(plan->cascades_off + size_t(nc) * sizeof(BatchCascade), 256);
    plan->item_bases_off = align_up(plan->bases_off + size_t(nc) * 4 * 4, 256);
    plan->counters_off = align_up(plan->item_bases_off + size_t(n) * 4, 256);
    plan->total = align_up(plan->counters_off + (size_t(nc) * 4 + 4) * 4, 256);
    return HF_OK;
}

int g_persistent_blocks[64][2] = {};

}  // namespace

int hf_batch_query_bytes(const hf_batch_item* items, int32_t n, int32_t flags, size_t* device_bytes,
                         size_t* host_bytes) {
    return guarded("hf_batch_query_bytes", [&]() -> int {
        (void)flags;
        BatchPlan plan;
        int rc = plan_batch(items, n, &plan);
        if (rc) return rc;
        if (device_bytes) *device_bytes = plan.total;
        if (host_bytes) *host_bytes = plan.counters_off;
        return HF_OK;
    });
}

int hf_batch_prepare(const hf_batch_item* items, int32_t n, int32_t flags, void* host_buf, size_t host_bytes) {
    return guarded("hf_batch_prepare", [&]() -> int {
        ApiRange range_("hf_batch_prepare");
        BatchPlan plan;
        int rc = plan_batch(items, n, &plan);
        if (rc) return rc;
        if (!host_buf) return fail(HF_ERR_ARG, "null host buffer");
        if (host_bytes < plan.counters_off)
            return fail(HF_ERR_NOMEM, "batch host buffer has %zu bytes, %zu needed", host_bytes, plan.counters_off);
        if (flags & ~int32_t(kBatchRaysInside | kBatchRayTileMask | kBatchWarp16x2 | kBatchPersistent))
            return fail(HF_ERR_ARG, "unknown batch flags");
        if ((flags & kBatchRaysInside) && !(flags & kBatchPersistent))
            return fail(HF_ERR_ARG, "HF_BATCH_RAYS_INSIDE needs HF_BATCH_PERSISTENT");
        if (((flags & kBatchRayTileMask) >> 1) == 3) return fail(HF_ERR_ARG, "choose one ray tile shape");
        for (int32_t i = 0; i < n; ++i) {
            if (int rc2 = check_kernel_output(items[i].t_dev, "batch item t output")) return rc2;
            if (int rc2 = check_kernel_output(items[i].hit_dev, "batch item hit output")) return rc2;
        }
        int dev = 0;
        int e = cudaGetDevice(&dev);
        if (e) return cuda_fail(e, "cudaGetDevice");
        if (dev < 0 || dev >= 64) return fail(HF_ERR_ARG, "device index %d", dev);
        if (!g_persistent_blocks[dev][0]) {
            e = batch_persistent_blocks(&g_persistent_blocks[dev][0], &g_persistent_blocks[dev][1]);
            if (e) return cuda_fail(e, "occupancy query");
        }
        char* hb = static_cast<char*>(host_buf);
        std::memset(hb, 0, plan.counters_off);
        BatchHeader& h = *reinterpret_cast<BatchHeader*>(hb);
        BatchItem* bi = reinterpret_cast<BatchItem*>(hb + plan.items_off);
        BatchCascade* bc = reinterpret_cast<BatchCascade*>(hb + plan.cascades_off);
        h.n_items = n;
        h.n_cascades = plan.n_cascades;
        h.flags = flags;
        const int shape = (flags & kBatchRayTileMask) >> 1;
        h.ray_tile_w = shape == 1 ? 32 : (shape == 2 ? 8 : 16);
        h.ray_tile_h = 256 / h.ray_tile_w;
        h.persistent_blocks = g_persistent_blocks[dev][0];
        h.persistent_blocks_rays = g_persistent_blocks[dev][1];
        h.items_off = int64_t(plan.items_off);
        h.cascades_off = int64_t(plan.cascades_off);
        h.counters_off = int64_t(plan.counters_off);
        h.bases_off = int64_t(plan.bases_off);
        h.item_bases_off = int64_t(plan.item_bases_off);
        h.desc_bytes = int64_t(plan.counters_off);
        h.total_bytes = int64_t(plan.total);
        int kc = 0, units[kPhases] = {0, 0, 0, 0, 0};
        for (int32_t i = 0; i < n; ++i) {
            hf_ctx* ctx = items[i].ctx;
            ViewSlot* v = get_view(ctx, items[i].view_slot);
            const int C = v->cam.n_cascades, N = v->cam.cascade_size, P = mip_pow2(N);
            BatchItem& I = bi[i];
            I.ray = ray_params(v, false);
            I.ray.t_out = items[i].t_dev;
            I.ray.hit_out = items[i].hit_dev;
            I.lt = ctx->lookup_tables(true);
            I.lv = ctx->lists();
            if (ctx->compact_fmt != 0) I.cv = ctx->compact();
            I.fp32c = ctx->fp32_compact() ? 1 : 0;
            I.status = ctx->d_status();
            I.dom_w = ctx->width;
            I.dom_h = ctx->height;
            I.eps_frac = 1e-6;
            for (int k = 0; k < HF_MAX_CASCADES; ++k) {  // batched frames compute every texel
                v->reuse[k] = ViewSlot::Reuse();
                v->fit.cas[k].reuse_source = -1;
            }
            const DiscParams dp = disc_params(ctx, v);
            I.K = dp.K;
            I.precision = ctx->rbf.precision;
            if (I.precision != HF_PREC_FP32) h.mixed = 1;
            I.first_cascade = kc;
            I.n_cascades = C;
            I.ray_tiles_x = (v->cam.width + h.ray_tile_w - 1) / h.ray_tile_w;
            I.ray_units = I.ray_tiles_x * ((v->cam.height + h.ray_tile_h - 1) / h.ray_tile_h);
            I.ray_unit_base = units[kPhaseRays];
            reinterpret_cast<int32_t*>(hb + plan.item_bases_off)[i] = I.ray_unit_base;
            units[kPhaseRays] += I.ray_units;
            for (int k = 0; k < C; ++k, ++kc) {
                BatchCascade& B = bc[kc];
                fill_prep_cascade(v, k, B.prep);
                B.disc = dp.cas[k];
                B.mip.tex = v->tex[k];
                B.mip.spans = v->spans[k];
                B.mip.mip = v->mip[k];
                B.mip.N = N;
                B.mip.P = P;
                B.mip.K = mip_levels(P);
                B.item = i;
                B.tiles_x = (N + 31) / 32;
                B.mip_blocks_x = (P + 63) / 64;
                B.n_units[kPhaseRows] = (N + 255) / 256;
                h.max_rows_units = std::max(h.max_rows_units, B.n_units[kPhaseRows]);
                B.n_units[kPhaseTexels] = B.tiles_x * ((N + 7) / 8);
                B.n_units[kPhaseMipLo] = B.mip_blocks_x * B.mip_blocks_x;
                B.n_units[kPhaseMipHi] = 1;
                for (int ph = 0; ph < 4; ++ph) {
                    B.unit_base[ph] = units[ph];
                    units[ph] += B.n_units[ph];
                }
            }
            v->stage = 3;
            v->data_version = ctx->data_version;
        }
        // global unit numbering: phase after phase
        int base = 0;
        for (int ph = 0; ph < kPhases; ++ph) {
            h.phase_base[ph] = base;
            base += units[ph];
        }
        h.phase_base[kPhases] = base;
        int32_t* bases = reinterpret_cast<int32_t*>(hb + plan.bases_off);
        for (int k = 0; k < plan.n_cascades; ++k)
            for (int ph = 0; ph < 4; ++ph) {
                bc[k].unit_base[ph] += h.phase_base[ph];
                bases[ph * plan.n_cascades + k] = bc[k].unit_base[ph];
            }
        return HF_OK;
    });
}

int hf_batch_launch(const void* host_buf, void* dev_buf, size_t dev_bytes, void* stream) {
    return guarded("hf_batch_launch", [&]() -> int {
        ApiRange range_("hf_batch_launch");
        if (!host_buf || !dev_buf) return fail(HF_ERR_ARG, "null buffer");
        if (reinterpret_cast<uintptr_t>(dev_buf) & 255) return fail(HF_ERR_ARG, "device buffer must be 256-byte aligned");
        const BatchHeader& h = *static_cast<const BatchHeader*>(host_buf);
        if (h.n_items < 1 || h.total_bytes <= 0) return fail(HF_ERR_ARG, "host buffer holds no prepared batch");
        if (dev_bytes < size_t(h.total_bytes))
            return fail(HF_ERR_NOMEM, "batch device buffer has %zu bytes, %lld needed", dev_bytes, (long long)h.total_bytes);
        cudaStream_t s = cudaStream_t(stream);
        char* db = static_cast<char*>(dev_buf);
        int e = cudaMemcpyAsync(db, host_buf, size_t(h.desc_bytes), cudaMemcpyHostToDevice, s);
        if (!e) e = cudaMemsetAsync(db + h.counters_off, 0, size_t(h.total_bytes - h.counters_off), s);
        if (e) return cuda_fail(e, "batch descriptor upload");
        e = launch_batch(h, dev_buf, stream);
        if (e) return cuda_fail(e, "batch kernel launch");
        return HF_OK;
    });
}

int hf_frame_batch(const hf_batch_item* items, int32_t n, int32_t flags, void* host_buf, size_t host_bytes,
                   void* dev_buf, size_t dev_bytes, void* stream) {
    return guarded("hf_frame_batch", [&]() -> int {
        ApiRange range_("hf_frame_batch");
        int rc = hf_batch_prepare(items, n, flags, host_buf, host_bytes);
        if (rc) return rc;
        return hf_batch_launch(host_buf, dev_buf, dev_bytes, stream);
    });
}

int hf_get_cascade(const hf_ctx* ctx, int32_t slot, int32_t c, hf_cascade_info* out) {
    return guarded("hf_get_cascade", [&]() -> int {
        if (!ctx || !out) return fail(HF_ERR_ARG, "null argument");
        if (slot < 0 || slot >= HF_MAX_VIEWS || !ctx->views[slot] || ctx->views[slot]->stage < 1)
            return fail(HF_ERR_STATE, "view slot %d has no camera", slot);
        const ViewSlot& v = *ctx->views[slot];
        if (c < 0 || c >= v.cam.n_cascades) return fail(HF_ERR_ARG, "cascade %d out of range", c);
        *out = v.fit.cas[c];
        return HF_OK;
    });
}

int hf_sync(hf_ctx* ctx, void* stream) {
    return guarded("hf_sync", [&]() -> int {
        ApiRange range_("hf_sync");
        if (!ctx) return fail(HF_ERR_ARG, "null context");
        int e = cudaStreamSynchronize(cudaStream_t(stream));
        if (e) return cuda_fail(e, "stream synchronize");
        e = cudaGetLastError();
        if (e) return cuda_fail(e, "pending CUDA error");
        if (!ctx->dev) return HF_OK;
        DevStatus st;
        e = cudaMemcpy(&st, ctx->d_status(), 8, cudaMemcpyDeviceToHost);
        if (e) return cuda_fail(e, "status read-back");
        if (st.flags) {
            e = cudaMemset(ctx->d_status(), 0, 8);
            if (e) return cuda_fail(e, "status reset");
            if (st.flags & kStatusTimeout)
                return fail(HF_ERR_TIMEOUT, "a bounded device loop gave up (a ray walk over its step budget or a "
                            "batch wait over its poll limit; detail %u)", st.detail);
            return fail(HF_ERR_DATA, "device consistency check failed (item %u)", st.detail);
        }
        return HF_OK;
    });
}

int hf_selftest_wait_timeout(hf_ctx* ctx, int32_t polls, void* stream) {
    return guarded("hf_selftest_wait_timeout", [&]() -> int {
        if (!ctx) return fail(HF_ERR_ARG, "null context");
        if (!ctx->dev) return fail(HF_ERR_STATE, "persistent buffer not bound");
        if (polls < 1 || polls > (1 << 20)) return fail(HF_ERR_ARG, "polls must be 1..2^20");
        int e = launch_selftest_wait(ctx->d_status(), polls, stream);
        if (e) return cuda_fail(e, "self-test launch");
        return HF_OK;
    });
}

int hf_measure_unit_rates(double* ex2_per_s, double* ffma_per_s, int32_t* sm_count, void* stream) {
    return guarded("hf_measure_unit_rates", [&]() -> int {
        ApiRange range_("hf_measure_unit_rates");
        if (!ex2_per_s || !ffma_per_s || !sm_count) return fail(HF_ERR_ARG, "null argument");
        int sms = 0;
        int e = measure_unit_rates(ex2_per_s, ffma_per_s, &sms, stream);
        if (e) return cuda_fail(e, "unit-rate kernels");
        *sm_count = sms;
        return HF_OK;
    });
}

void hf_destroy(hf_ctx* ctx) { delete ctx; }

}  // extern "C"

// Internal declarations shared by the host code (hf_host.cpp, hf_fit.cpp)
// and the CUDA kernels (hf_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/hf.h"

namespace hfi {

constexpr int kMaxLevels = HF_MAX_LEVEL + 1;
constexpr int kMaxCascadeSize = 8192;

// Device status block at the start of the persistent buffer.  Kernels OR
// error bits into `flags` and record the first failing item in `detail`.
enum : uint32_t { kStatusTimeout = 1u, kStatusData = 2u };
struct DevStatus {
    uint32_t flags;
    uint32_t detail;
    unsigned long long counters[4 * HF_MAX_CASCADES];  // measurement pass (hf_view_stats)
    unsigned long long ray_counters[2];                  // measurement pass (hf_ray_stats)
    uint32_t pad[26];  // pad[0]: the never-set flag of hf_selftest_wait_timeout
};
static_assert(sizeof(DevStatus) == 384, "status block is 384 bytes");

// Per-level occupancy bitmaps of a set of quadtree cells: bit (iy*nx[L]+ix)
// of level L is set when cell (L, ix, iy) is in the set.  prefix[w] counts
// the set bits of level L before word w, so the index of a cell is
// base[L] + prefix[w] + popcount(lower bits of word w).  Cells are thereby
// numbered by (level, iy, ix).  Levels without cells have no words.
struct Bitmaps {
    const uint64_t* bits;
    const uint32_t* prefix;
    int64_t word_off[kMaxLevels + 1];  // word_off[max_level + 1] = total words
    int64_t base[kMaxLevels + 1];      // base[max_level + 1] = total cells
    int32_t nx[kMaxLevels];
    int32_t ny[kMaxLevels];
    int32_t max_level;
};

// Candidate enumeration: the real leaves (the RBF centres) and the reach of
// a level-L centre, R * c_L + margin, in units of half a finest cell.
struct EnumTables {
    Bitmaps leaves;
    double reach_q[kMaxLevels];
};

// Texel -> bucket lookup.  Buckets are the leaves at or below level
// `bucket_level`; coarser leaves are split into their level-bucket_level
// descendants, so that each list covers a small square.
// cellmap (optional, for grids of at most kCellMapMaxCells finest cells):
// per finest cell, row-major, the list of its bucket as {first group of four
// entries, number of groups}, so that a texel finds its list with one load
// instead of the per-level bitmap probes and the offsets.
constexpr int64_t kCellMapMaxCells = int64_t(1) << 28;
struct LookupTables {
    Bitmaps buckets;
    int32_t bucket_level;
    float inv_c_fin;  // 1 / finest cell edge
    int32_t nx_fin, ny_fin;
    const uint2* cellmap;  // null: look the bucket up in the bitmaps
};

// Each bucket's list holds its candidates in ascending leaf order, padded to
// a multiple of 4 entries with `sentinel` (= the leaf count), so that lists
// start on 16-byte boundaries and are read four entries per load.  Record
// `sentinel` is a null record whose weight is exactly 0 (centre far away,
// value 0, depth 0), so padding adds nothing to the sums.
constexpr int kListPad = 4;
struct ListsView {
    const int64_t* offsets;  // n_buckets + 1, multiples of kListPad
    int32_t* idx;            // candidate leaf indices, ascending within a bucket, then padding
    float4* recs;            // per leaf (+ the null record): centre x, y (domain-local), weight scale, value
    const float* depth;      // per leaf (+ 0 for the null record) water depth (water layer only, else null)
    int32_t sentinel;        // index of the null record = number of leaves
};

// Compact candidate lists of the reduced-precision discretization: per
// bucket its candidates in pairs of 16 bytes: {x0 x1, y0 y1} in the 16-bit
// type (FP16 or BF16), the candidates' centres relative to the bucket's lower
// corner in units of half a finest cell (small integers, exact in the 16-bit
// type), then the two FP32 values whose 4 lowest mantissa bits carry the
// candidates' levels L.  The 16-bit exponent scale of level L,
// -log2(e) q^2 / (2 sigma^2 c_L^2), is the finest level's with the exponent
// field lowered by 2 (max_level - L): its bits are L * step + kb, step the
// exponent unit x 2, so kb2 = kb * 0x10001 gives both scales of a pair with
// one integer multiply-add.  An odd list is padded with a far-away entry of
// value 0.
struct CompactView {
    const int64_t* pair_offsets;  // n_buckets + 1
    uint4* pairs;                 // per pair
    float q, inv_q;               // half a finest cell (m) and its inverse
    uint32_t kb2;                 // (bits of the level-0 scale) * 0x10001, see above
    uint32_t kf_bits;             // FP32 bits of the finest level's weight scale per squared half-cell
    int32_t max_level;
    // optional (as LookupTables.cellmap): per finest cell {first pair of its
    // bucket's list, pairs | bucket level << 24}; null: bitmap lookup
    const uint2* cellmap;
};

// Per-frame cascade data for the prep kernel (visible rows, texel coordinates).
struct PrepCascade {
    double ox, oy, h, inv_h;
    int64_t lat_x, lat_y;  // lattice fit: texel (i, j) at ((lat_x + i) h, (lat_y + j) h)
    int32_t lattice;       // 1: lattice fit, 0: stable fit (texel at ox + i h, oy + j h)
    int32_t N;
    int32_t n_edges;  // 0 = empty cascade
    // grown polygon edge e: nx x + ny y <= c, i.e. x <= or >= (c - ny y) / nx
    double ny[HF_MAX_POLY];
    double c[HF_MAX_POLY];
    double inv_nx[HF_MAX_POLY];
    int32_t sgn[HF_MAX_POLY];
    int2* spans;
    float* xs;
    float* ys;
};

struct PrepParams {
    int32_t C;
    int32_t max_N;
    double dom_w, dom_h, eps_frac;  // domain extents and the boundary slack (fraction of h)
    PrepCascade cas[HF_MAX_CASCADES];
};

struct DiscCascade {
    int32_t N;
    const int2* spans;
    const float* xs;
    const float* ys;
    float* tex;
    float* wtex;  // water surface texture (water layer only)
    // temporal reuse (hf_discretize_reuse): texel (i, j) is texel
    // (i + prev_di, j + prev_dj) of an earlier frame's texture on the same
    // lattice; prev == nullptr: none
    const float* prev;
    const float* prev_w;
    int32_t prev_N, prev_di, prev_dj;
};

struct DiscParams {
    int32_t C;
    int32_t max_N;
    int32_t precision;
    int32_t water;  // 1: also discretize the depths and write the water surface
    int32_t kernel; // HF_RBF_* weight function
    float K;        // exp(-R^2 / (2 sigma^2))
    DiscCascade cas[HF_MAX_CASCADES];
};

struct MipCascade {
    const float* tex;
    const float* wtex;  // water surface: level 0 bounds both patches (two = 1 only)
    const int2* spans;  // visible span per texel row (texels outside it hold -inf); null: read every texel
    float* mip;
    int32_t N, P, K;
};

struct MipParams {
    int32_t C;
    int32_t max_P;
    int32_t max_K;
    int32_t two;  // 1: bound the terrain and the water surface together
    MipCascade cas[HF_MAX_CASCADES];
};

struct RayCascade {
    const float* tex;
    const float* mip;
    const float* wtex;  // water surface (water layer only; mip then bounds both surfaces)
    int32_t N, P, K;
    float eu, ev;  // eye in this cascade's patch units
    float h, inv_h;
    float near_d, far_ext;  // projected-depth band
    int32_t budget;         // bound on walk steps: 8 (2 N + 8) (K + 2)
    int32_t stop_level;     // coarse-level stop: the walk ends at this level's box tops (0 = patches)
    int32_t lvl_off[kMaxLevels];  // first float of mip level k
};

struct RayParams {
    int32_t C, W, H;
    int32_t water;           // 1: rays meet the terrain or the water surface, whichever comes first
    int32_t coarse;          // 1: some cascade has a coarse-level stop (RayCascade.stop_level > 0)
    int32_t jump;            // 1: after a step the walk climbs to the coarsest node entered (hf_camera.traversal)
    int32_t host_out;        // 1: t_out or hit_out is pinned host memory (the stores go out in image rows)
    float ez;                // eye height (m)
    float F[3], R[3], U[3];  // camera basis
    float px_a, px_b, py_a, py_b;  // screen coordinates: s = fma(pixel, a, b), s in [-tan, tan]
    float dir2x, dir2y;      // normalised ground projection of the view
    float znear, zfar;
    RayCascade cas[HF_MAX_CASCADES];
    float* t_out;
    uint8_t* hit_out;
};

// Batched frames (hf_frame_batch).  The host writes a header, one BatchItem
// per (context, view) and one BatchCascade per cascade into a pinned buffer;
// the same bytes are copied to the device and drive one persistent launch
// that drains an ordered work queue (visible rows -> discretization tiles ->
// level-0..6 mip blocks -> mip tops), then a batched ray-cast launch.
enum { kPhaseRows = 0, kPhaseTexels = 1, kPhaseMipLo = 2, kPhaseMipHi = 3, kPhaseRays = 4, kPhases = 5 };
enum : int32_t {
    kBatchRaysInside = 1,   // ray tiles drained by the persistent launch too
    kBatchRayTileMask = 6,  // (flags >> 1) & 3: 0 = 16x16, 1 = 32x8, 2 = 8x32 pixels per ray unit
    kBatchWarp16x2 = 8,     // discretization warps cover 16 x 2 texels (else 8 x 4)
    kBatchPersistent = 16   // rows / texels / mips in one persistent launch (else one launch per phase)
};

struct BatchCascade {
    PrepCascade prep;
    DiscCascade disc;
    MipCascade mip;
    int32_t item;
    int32_t tiles_x;        // discretization tiles (32 x 8 texels) per row
    int32_t mip_blocks_x;   // 64 x 64 level-0 blocks per row
    int32_t unit_base[4];   // first unit of this cascade in phases 0..3
    int32_t n_units[4];
};

struct BatchItem {
    RayParams ray;
    LookupTables lt;
    ListsView lv;
    CompactView cv;
    DevStatus* status;
    double dom_w, dom_h, eps_frac;
    float K;
    int32_t precision;
    int32_t fp32c;  // FP32 item discretized from its compact lists (see discretize_texel_f32c)
    int32_t first_cascade, n_cascades;
    int32_t ray_unit_base, ray_tiles_x, ray_units;
};

struct BatchHeader {
    int32_t n_items, n_cascades;
    int32_t phase_base[kPhases + 1];  // unit ranges per phase; phase_base[kPhases] = all units
    int32_t ray_tile_w, ray_tile_h;
    int32_t flags;
    int32_t persistent_blocks, persistent_blocks_rays;
    int32_t max_rows_units;
    int32_t mixed;  // 1: some item discretizes in FP16 / BF16 (else the texel phase is FP32 only)
    int64_t items_off, cascades_off, counters_off, desc_bytes, total_bytes;
    int64_t bases_off;  // int32 [4][n_cascades]: the cascades' first units of phases 0..3, contiguous
    int64_t item_bases_off;  // int32 [n_items]: the items' first ray units (BatchItem.ray_unit_base)
};

// Kernel launchers (hf_kernels.cu); they return a cudaError_t value.
int launch_fill_lists(const EnumTables& et, const LookupTables& lt, const ListsView& lv,
                      DevStatus* status, void* stream);
// Fills the cell map `cellmap` from lt's bucket bitmaps and the list offsets
// (with `cv`, the map of the compact pair lists).
int launch_fill_cellmap(const LookupTables& lt, const ListsView& lv, uint2* cellmap, DevStatus* status,
                        void* stream, const CompactView* cv = nullptr);
int launch_prep(const PrepParams& p, void* stream);
int launch_fill_compact(const EnumTables& et, const LookupTables& lt, const ListsView& lv,
                        const CompactView& cv, int precision, void* stream);
int measure_unit_rates(double* ex2_per_s, double* ffma_per_s, int* sm_count, void* stream);
int launch_discretize_mixed(const DiscParams& p, const LookupTables& lt, const CompactView& cv,
                            DevStatus* status, void* stream);
int launch_discretize(const DiscParams& p, const LookupTables& lt, const ListsView& lv,
                      DevStatus* status, void* stream);
int launch_discretize_f32c(const DiscParams& p, const LookupTables& lt, const CompactView& cv,
                           DevStatus* status, void* stream);
int launch_maxmip(const MipParams& p, void* stream);
int launch_stats(const DiscParams& p, const LookupTables& lt, const ListsView& lv,
                 DevStatus* status, void* stream);
int launch_raycast(const RayParams& p, DevStatus* status, void* stream);
int launch_raycast_count(const RayParams& p, DevStatus* status, void* stream);
int batch_persistent_blocks(int* blocks_plain, int* blocks_rays);
int launch_batch(const BatchHeader& h, void* dev_buf, void* stream);
int launch_selftest_wait(DevStatus* status, int limit, void* stream);

// Allocation-free discretization (hf_noalloc.cu): fits `cam` and fills the
// prep / discretize parameters for output textures `tex` and the scratch
// block `scratch` (spans, then xs, then ys of every cascade).  *compact: the
// FP32 walk over the compact lists (cv) serves, else the index lists (lv).
int noalloc_discretize_params(hf_ctx* ctx, const hf_camera* cam, float* const* tex,
                              char* scratch, size_t scratch_bytes, hf_cascade_info* info_out,
                              PrepParams* pp, DiscParams* dp, LookupTables* lt, ListsView* lv,
                              CompactView* cv, bool* compact, DevStatus** status);
// Records a CUDA failure as the calling thread's last error; returns HF_ERR_CUDA.
int set_cuda_error(int e, const char* what);

// Status of the exception being handled (called from a catch block only):
// HF_ERR_HOST with its description.
int exception_status(const char* where) noexcept;

// Runs an entry point's body and turns any C++ exception it throws (host
// allocation, thread creation) into HF_ERR_HOST, so that none crosses the
// C ABI.
template <class F>
int guarded(const char* where, F&& body) noexcept {
    try {
        return body();
    } catch (...) {
        return exception_status(where);
    }
}

// Host-side count of each bucket's candidates (same enumeration as the fill
// kernel, in exact integer arithmetic).  Bitmaps must hold host pointers.
void count_lists_host(const EnumTables& et, const LookupTables& lt, int64_t* counts,
                      int n_threads);

// Mip geometry shared by host and device code.
inline int mip_pow2(int N) {
    int P = 1;
    while (P < N - 1) P <<= 1;
    return P;
}
inline int mip_levels(int P) {
    int K = 0;
    while ((1 << K) < P) K++;
    return K;
}
inline int64_t mip_floats(int N) {
    int64_t P = mip_pow2(N);
    return (4 * P * P - 1) / 3;
}

// Cascade fitting (hf_fit.cpp).
struct FitDomain {
    double width, height, zmin, zmax, c_min;
};
struct FitResult {
    double F[3], U[3], R[3];
    double dir2[2];
    double n, f;
    int n_hull;
    double hull[64][2];
    hf_cascade_info cas[HF_MAX_CASCADES];
};
// eye_local: eye relative to the domain origin (FP64).  follow: with the
// lattice fit, cascade k keeps ladder step follow[k] when it is one step
// coarser than the smallest that fits (hysteresis); nullptr = none.
int fit_cascades(const hf_camera& cam, const double eye_local[3], const FitDomain& dom,
                 FitResult* out, const int64_t* follow = nullptr);

}  // namespace hfi

/*
 * hf.h -- C ABI of the GB300 adaptive-heightfield renderer.
 *
 * Implements the per-frame two-step method of Cornel, Horvath and Waser,
 * "An Attempt of Adaptive Heightfield Rendering with Complex Interpolants
 * Using Ray Casting" (2022):
 *   step 1  view-dependent discretization: the truncated Gaussian RBF
 *           approximation (Eq. 1, Eq. 2) of a quadtree heightfield is
 *           evaluated at every visible texel of frustum-split cascade
 *           textures fitted to the view (Section 3, Section 4);
 *   step 2  a maximum mipmap per cascade, then one ray per pixel through the
 *           cascades with empty-space skipping and exact ray/bilinear-patch
 *           intersection, blended where cascades overlap (Section 5).
 *
 * Conventions
 *   - Every function returns HF_OK (0) or a negative HF_ERR_* code; no C++
 *     exception crosses this boundary (each entry point catches them and
 *     returns HF_ERR_HOST).  hf_last_error() describes the most
 *     recent failure of the calling thread.
 *   - The library never allocates device memory.  The caller allocates the
 *     sizes hf_query_bytes() reports and keeps ownership; buffers must stay
 *     alive and untouched while work that uses them is in flight.
 *   - Host arrays passed in are copied before the call returns.
 *   - `stream` is a cudaStream_t passed as an opaque pointer (NULL = the
 *     legacy default stream).  Device work is enqueued asynchronously on it;
 *     errors detected on the device are reported by hf_sync().
 *   - Geometry: the heightfield domain is the rectangle
 *     [0, root_nx*root_cell] x [0, root_ny*root_cell] in domain-local metres,
 *     placed at (origin_x, origin_y) in world coordinates; z is up and is not
 *     offset.  World positions are FP64 on the host; device work uses FP32
 *     domain-local (or cascade-local) coordinates.
 *   - Cascade texel (i, j) of a cascade with origin (ox, oy) and spacing h
 *     sits at (ox + i h, oy + j h) domain-local; textures are N x N FP32,
 *     row-major (index j*N + i).  Invisible texels hold -infinity.
 *   - A context is not thread-safe: one host thread drives it at a time.
 */
#ifndef HF_H
#define HF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HF_OK = 0,
    HF_ERR_ARG = -1,     /* invalid argument or inconsistent input data */
    HF_ERR_STATE = -2,   /* call out of order (e.g. ray cast before the mip build) */
    HF_ERR_NOMEM = -3,   /* a caller buffer is smaller than required */
    HF_ERR_CUDA = -4,    /* a CUDA runtime call or kernel launch failed */
    HF_ERR_TIMEOUT = -5, /* a bounded device-side loop gave up; results are invalid */
    HF_ERR_DATA = -6,    /* device-side consistency check failed */
    HF_ERR_HOST = -7     /* host-side failure: host memory for the library's own tables
                            or worker threads could not be had; nothing was launched */
};

enum { HF_PREC_FP32 = 0, HF_PREC_FP16 = 1, HF_PREC_BF16 = 2 };
enum { HF_RBF_GAUSSIAN = 0, HF_RBF_WENDLAND_C2 = 1 };

#define HF_MAX_LEVEL 15
#define HF_MAX_CASCADES 8
#define HF_MAX_POLY 32
#define HF_MAX_VIEWS 256

/* Quadtree geometry (Section 2: an adaptive grid of square cells). */
typedef struct {
    double origin_x, origin_y; /* world position of the domain's lower corner (m) */
    double root_cell;          /* edge of a level-0 cell (m) */
    int32_t root_nx, root_ny;  /* level-0 grid size */
    int32_t max_level;         /* deepest level, 0..HF_MAX_LEVEL; level-L cells have edge root_cell / 2^L */
} hf_quadtree_desc;

/* One leaf cell: level L, integer position (ix, iy) on level L's grid
 * (0 <= ix < root_nx * 2^L), and the data value at the cell centre
 * (Section 2).  16 bytes, no padding. */
typedef struct {
    int32_t level, ix, iy;
    float value;
} hf_leaf;

/* Truncated Gaussian RBF (Eq. 1).  Cell i influences p when
 * |p_i - p| < radius * c_i, with weight exp(-(|p_i - p|/c_i)^2 / (2 sigma^2))
 * - exp(-radius^2 / (2 sigma^2)).  The paper's setting is sigma = 1 with
 * truncation at 3.5 sigma, i.e. radius = 3.5.  precision selects the
 * arithmetic of the distance / exp evaluation (HF_PREC_*); sums are FP32.
 * HF_PREC_FP16 / HF_PREC_BF16 evaluate distances, scales and exp two
 * candidates at a time in packed 16-bit arithmetic from compact per-bucket
 * lists (more device memory); candidate offsets must stay exact in the
 * 16-bit type, else hf_create_quadtree returns HF_ERR_ARG.
 * HF_PREC_FP32 evaluates in FP32 arithmetic.  Where the offsets are exact in
 * FP16 and the water layer is off, an FP32 context also keeps the compact
 * lists and walks them (one 16-byte load per two candidates, no index); their
 * values give up their 4 lowest mantissa bits to the cell's level (at most 15
 * ulp).  Otherwise, or with the environment variable HF_FP32_INDEX_LISTS=1
 * set at creation, it walks lists of leaf indices with exact values.
 * hf_discretize_noalloc always evaluates in FP32.
 * The lists of potentially influencing cells (Section 4) are kept per
 * square "bucket": every leaf at or below level bucket_level is a bucket,
 * coarser leaves are split into their level-bucket_level descendants so a
 * list never covers more than one level-bucket_level cell.  bucket_level
 * = -1 selects max(0, max_level - 1).
 * kernel selects the weight function of Eq. 2: HF_RBF_GAUSSIAN is Eq. 1;
 * HF_RBF_WENDLAND_C2 is Wendland's compactly supported C2 function
 * (1 - r)^4 (4 r + 1) of r = |p_i - p| / (radius c_i), zero for r >= 1 (sigma
 * unused) -- another interpolant in the same slot: lists, normalisation,
 * mipmap and ray cast stay as they are.  Non-Gaussian kernels need FP32
 * precision and are not available in batched frames.
 * water = 1 adds the water layer (Section 2: the input is a terrain model
 * plus relative water depths at the cells of the same adaptive grid; Table 1
 * times the approximation of both): every leaf also carries a depth >= 0
 * (hf_update_water, initially 0), each cascade gets a second texture holding
 * the water surface, and rays stop at whichever surface they meet first.  The
 * water layer needs precision HF_PREC_FP32 and is not available in batched
 * frames; hf_discretize_noalloc ignores it. */
typedef struct {
    double sigma;
    double radius;
    int32_t precision;
    int32_t bucket_level;
    int32_t water;
    int32_t kernel;
} hf_rbf_params;

/* A view (Section 3, Section 5).  eye is in world coordinates; forward and
 * up need not be unit or orthogonal (up is made orthogonal to forward).
 * vfov in radians; znear/zfar are clip distances along forward.
 * n_cascades textures of cascade_size^2 texels are fitted; split_lambda
 * blends logarithmic (1) and uniform (0) splits; the far plane of every
 * cascade but the last is pushed out by overlap_frac of its depth span.
 * texel_ladder selects the fit of each cascade's band polygon: 0 is the
 * paper's stable fit (extent an even multiple of the smallest cell c_min,
 * origin on a multiple of c_min, texel = extent / (N - 1)); n in 1..64 is
 * the lattice fit, which lets hf_discretize_reuse carry texels over from
 * one frame to the next: the texel spacing is restricted to the ladder
 * h_m = c_min 2^(m/n) (m >= -8n), taking the smallest m with (N - 2) h_m >=
 * the box's larger side, and the origin is the box corner rounded down to a
 * multiple of h_m, so texel (i, j) sits on the lattice point (snap_x + i,
 * snap_y + j) of spacing h_m whatever the camera's position.  The lattice
 * fit needs cascade_size >= 4; its texels are up to 2^(1/n) coarser than
 * the stable fit's.
 * traversal selects the max-mipmap walk of the ray cast (Section 5): 0 is
 * Tevs et al.'s, which after each step climbs one level when the ray has left
 * its parent node; 1 climbs at once to the coarsest node the ray has just
 * entered -- our reading of the improved traversal the paper attributes to
 * Dick et al. (Section 1), which it names without describing.  Both find the
 * same first hit; 1 is not available with the water layer, the coarse-level
 * stop or batched frames.
 * lod_pixels > 0 turns on the coarse-level stop (after the LOD-dependent early
 * ray termination the paper cites): in cascade c the ray stops at the box tops
 * of max-mipmap level L_c instead of descending to the bilinear patches, L_c
 * being the largest level whose nodes, 2^L texels wide, span at most
 * lod_pixels pixels (2 tan(vfov / 2) / height of the distance each) at the
 * cascade's near depth (hf_cascade_info.stop_level).  0 is the paper's exact
 * surface; not available with the water layer. */
typedef struct {
    double eye[3];
    double forward[3];
    double up[3];
    double vfov, znear, zfar;
    int32_t width, height;
    int32_t n_cascades, cascade_size;
    double split_lambda, overlap_frac;
    int32_t texel_ladder;
    int32_t traversal;
    double lod_pixels;
} hf_camera;

/* Fitted cascade (Section 3) plus the device buffers bound to it. */
typedef struct {
    double near_depth, far_depth, far_ext_depth; /* projected-depth band; far_ext includes the overlap */
    int32_t n_poly;                              /* vertices of the cascade polygon; 0 = empty */
    int32_t N;                                   /* texture side */
    double poly[HF_MAX_POLY][2];                 /* CCW, domain-local */
    double aabb[4];                              /* x0, y0, x1, y1 of the polygon */
    int64_t snap_x, snap_y, snap_k;              /* stable fit: ox = snap_x c_min, oy = snap_y c_min, extent = 2 snap_k c_min;
                                                    lattice fit: texel = c_min 2^(snap_k / texel_ladder), ox = snap_x texel,
                                                    oy = snap_y texel */
    double ox, oy, extent, texel;                /* texel = extent / (N - 1) */
    float* tex;                                  /* device, N*N FP32 heights, -inf where invisible */
    float* mip;                                  /* device, max mipmap (see hf_build_maxmip) */
    int32_t* spans;                              /* device, N rows x {first, last} visible column; last < first = none */
    int64_t mip_floats;                          /* number of floats in mip */
    float* water_tex;                            /* device, N*N FP32 water surface, -inf where dry or invisible; NULL without the water layer */
    int32_t texel_ladder;                        /* the camera's texel_ladder (0 = stable fit) */
    int32_t reuse_source;                        /* cascade of the earlier frame the last hf_discretize_reuse copied from, -1 = none */
    int32_t stop_level;                          /* coarse-level stop (hf_camera.lod_pixels): 0 = exact bilinear surface */
    int32_t reserved;
} hf_cascade_info;

typedef struct hf_ctx hf_ctx;

/* Validates the leaves (levels and indices in range, values finite, the
 * leaves tile the domain exactly) and builds the quadtree on the host: a
 * per-level occupancy bitmap, and for every leaf the exact size of its list
 * of potentially influencing cells (Section 4: the set I depends only on
 * the grid and is precomputed once).  Allocates host memory only.
 * Returns HF_ERR_ARG on invalid input; *out is set only on success.
 * For grids of at most 2^28 finest cells the persistent buffer also holds a
 * map from every finest cell to its list (8 bytes per finest cell per list
 * set), which saves each texel the bucket lookup; the environment variable
 * HF_CELLMAP_MAX_CELLS, read here, lowers that limit (0: never; the texel
 * then probes the occupancy bitmaps, with identical results). */
int hf_create_quadtree(const hf_quadtree_desc* desc, const hf_leaf* leaves, int64_t n_leaves,
                       const hf_rbf_params* rbf, hf_ctx** out);

/* Device bytes the caller must provide: persistent_bytes for
 * hf_bind_persistent (quadtree + influence lists, + 4 bytes per leaf for the
 * water depths), per_view_bytes for one hf_set_camera with n_cascades
 * textures of cascade_size^2 texels (a second texture per cascade with the
 * water layer).  Either output pointer may be NULL. */
int hf_query_bytes(const hf_ctx* ctx, int32_t n_cascades, int32_t cascade_size,
                   size_t* persistent_bytes, size_t* per_view_bytes);

/* Uploads the quadtree into dev_persistent (>= persistent_bytes, 256-byte
 * aligned) and builds the influence lists on the device.  The buffer is
 * owned by the caller and must outlive the context's device work.
 * Synchronises `stream` before returning.  HF_ERR_NOMEM if too small. */
int hf_bind_persistent(hf_ctx* ctx, void* dev_persistent, size_t bytes, void* stream);

/* Replaces the leaf values (e.g. a new water level) without rebuilding the
 * tree; `values` is a host array in the order of the leaves given to
 * hf_create_quadtree.  Enqueued on `stream`. */
int hf_update_values(hf_ctx* ctx, const float* values, int64_t n_values, void* stream);

/* Water layer only (hf_rbf_params.water = 1): sets the leaves' relative
 * water depths (Section 2), a host array in the order of the leaves given to
 * hf_create_quadtree; every depth must be finite and >= 0 (HF_ERR_ARG).  The
 * same RBF weights that give the terrain height v at a texel give its depth
 * d = sum w_i d_i / sum w_i; the texel's water surface is v + d where d > 0,
 * else -inf (dry).  The cascade fit afterwards covers terrain + depth.
 * HF_ERR_STATE for a context without the water layer.  Uploads on `stream`
 * and waits for it. */
int hf_update_water(hf_ctx* ctx, const float* depths, int64_t n_depths, void* stream);

/* Fits the cascades of `cam` (Section 3) on the host in FP64 and binds
 * dev_view (>= per_view_bytes for cam's cascade settings, 256-byte aligned)
 * to view slot `view_slot` (0..HF_MAX_VIEWS-1).  Host work only. */
int hf_set_camera(hf_ctx* ctx, int32_t view_slot, const hf_camera* cam, void* dev_view,
                  size_t bytes);

/* hf_set_camera with hysteresis for a flight of frames on the lattice fit:
 * cascade k keeps the ladder step of prev_slot's cascade k (the previous
 * frame; prev_slot may equal view_slot) when that step is exactly one above
 * the smallest that fits -- still covering the box, with texels up to one
 * ladder step coarser -- so that the texel size changes only when it must
 * and hf_discretize_reuse finds more texels to carry over.  Cameras with
 * another texel_ladder, or the stable fit, are fitted as by hf_set_camera.
 * HF_ERR_STATE if prev_slot has no camera. */
int hf_set_camera_follow(hf_ctx* ctx, int32_t view_slot, const hf_camera* cam, void* dev_view,
                         size_t bytes, int32_t prev_slot);

/* Step 1 (Section 3 mask, Section 4 Eq. 2): computes the visible-texel rows
 * of every cascade and evaluates the RBF approximation at every visible
 * texel; invisible texels are set to -infinity.  With the water layer the
 * same pass also writes the water surface textures (hf_update_water). */
int hf_discretize_cascades(hf_ctx* ctx, int32_t view_slot, void* stream);

/* Step 1 with texels carried over from an earlier frame (temporal reuse; the
 * paper recomputes every frame).  view_slot's camera is set; prev_slot (a
 * different slot of the same context, with its own buffers) holds an earlier
 * frame discretized since its camera was last set.  Each of view_slot's
 * cascades takes as its source the earlier frame's cascade with the same
 * texel lattice that overlaps it most: with the lattice fit, the same
 * spacing (snap_k, texel_ladder); with the stable fit, an identical fit
 * (snaps and size).  Every visible texel whose lattice point the source
 * computed (visible there) is copied from it -- heights depend only on the
 * texel's position and the leaf data, so the copy equals a recomputation bit
 * for bit -- and every other visible texel is computed as in
 * hf_discretize_cascades.  Nothing is carried over when the leaf values or
 * depths changed since prev_slot was discretized (hf_update_values,
 * hf_update_water).  prev_slot's textures are read on `stream`: the caller
 * keeps prev_slot untouched, and its earlier work ordered before this call
 * (same stream, or an event), until this work is done.  HF_ERR_ARG for
 * prev_slot == view_slot or overlapping view buffers, HF_ERR_STATE if either
 * slot is not ready.  hf_get_cascade reports the source (reuse_source),
 * hf_view_stats the texels carried over. */
int hf_discretize_reuse(hf_ctx* ctx, int32_t view_slot, int32_t prev_slot, void* stream);

/* Step 2a (Section 5, maximum mipmap of Tevs et al.): level 0 holds, per
 * bilinear patch (texels i..i+1, j..j+1), the maximum of its four corners,
 * or -inf if a corner is invisible; patches are padded with -inf to P x P,
 * P the smallest power of two >= N-1; level k (P>>k)^2 entries hold the
 * maximum of 2x2 entries of level k-1; levels are stored one after another,
 * row-major.  With the water layer one mipmap bounds both surfaces: a
 * level-0 entry is the larger of the terrain patch's maximum and the water
 * patch's (a water patch exists where its four corners are wet). */
int hf_build_maxmip(hf_ctx* ctx, int32_t view_slot, void* stream);

/* Step 2b (Section 5): one ray per pixel, nearest cascade first; writes
 * t_dev[y*width + x] = distance from the eye to the hit (FP32, NaN on a
 * miss) and hit_dev[y*width + x] = 0 on a miss, else 1 + the index of the
 * first cascade hit.  Pixel (0, 0) is the top-left corner.  The outputs may
 * be device memory, managed memory, or pinned host memory mapped at the same
 * address (cudaHostAlloc / cudaHostRegister): the kernel then writes the
 * results to the host itself, with no separate copy; pageable host memory is
 * refused (HF_ERR_ARG).  In the overlap
 * of cascades c and c+1 both are intersected and the hit distances are
 * blended linearly across the overlap band.  With the water layer a ray
 * stops, inside each cascade, at whichever surface it meets first (the
 * water surface on a tie), and that per-cascade hit is what gets blended;
 * bit 0x80 of hit_dev marks a first-hit cascade whose hit is on the water
 * surface, the low bits still hold 1 + that cascade's index. */
int hf_raycast(hf_ctx* ctx, int32_t view_slot, float* t_dev, uint8_t* hit_dev, void* stream);

/* Descriptor and device pointers of cascade c of a view slot. */
int hf_get_cascade(const hf_ctx* ctx, int32_t view_slot, int32_t c, hf_cascade_info* out);

/* Work counts of the last discretization of a view slot, per cascade:
 * visible texels, list entries walked (the candidates of Section 4), and
 * weighted-sum terms with w > 0 (the influencing set I of Eq. 2), all as if
 * every visible texel were computed, and the visible texels that
 * hf_discretize_reuse copied from the earlier frame instead (0 after
 * hf_discretize_cascades; counted by reading that frame's textures again, so
 * valid while they are unchanged).  Runs a counting pass of the
 * discretization on `stream` and waits for it; meant for measurement, not
 * for the frame loop. */
typedef struct {
    int64_t visible_texels[HF_MAX_CASCADES];
    int64_t candidates[HF_MAX_CASCADES];
    int64_t influencers[HF_MAX_CASCADES];
    int64_t reused_texels[HF_MAX_CASCADES];
} hf_view_stats_t;
int hf_view_stats(hf_ctx* ctx, int32_t view_slot, hf_view_stats_t* out, void* stream);

/* Work counts of the ray cast of a view slot (whose max mipmap is built):
 * max-mipmap nodes tested and ray/patch intersections solved, summed over
 * all pixels.  Runs a counting pass of the ray caster (no outputs written) on
 * `stream` and waits for it; meant for measurement. */
int hf_ray_stats(hf_ctx* ctx, int32_t view_slot, int64_t* visits, int64_t* patch_tests,
                 void* stream);

/* Allocation-free discretization.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory at all, such
 * as a plug-in whose host application owns every device allocation and only
 * hands it finished output buffers, or a render loop that forbids cudaMalloc
 * after start-up because it can synchronise the device and stall a frame.
 * It fits `cam` (as hf_set_camera does) and computes the same visible texels
 * and heights as hf_discretize_cascades, writing cascade c's N x N FP32
 * texture to tex_out[c] (a host array of cam->n_cascades device pointers,
 * each 256-byte aligned with room for N*N floats).  Its scratch (visible-row
 * spans and texel coordinates, 16 bytes per texture row per cascade) lives in
 * a fixed 256 KiB array inside the library, so n_cascades * cascade_size may
 * not exceed 16384 (HF_ERR_ARG otherwise); nothing is allocated.  The array is
 * loaded on every device that loads the library and stays until exit.  The
 * first call on a device looks the array's address up, so make that first
 * call before capturing any stream.  The address is kept for the life of the
 * process: it stays valid only while the device's primary context lives, so a
 * caller that resets the device (cudaDeviceReset) must not call this entry
 * point afterwards.  All calls share the array: calls that
 * overlap on the GPU (e.g. on two streams at once) race and must be ordered
 * by the caller.  If info_out is not NULL it receives the cam->n_cascades
 * fitted cascades (device pointers other than tex are NULL).  The context's
 * persistent buffer must be bound. */
#define HF_NOALLOC_SCRATCH_BYTES (256 * 1024)
int hf_discretize_noalloc(hf_ctx* ctx, const hf_camera* cam, float* const* tex_out,
                          hf_cascade_info* info_out, void* stream);

/* Batched frames (the paper times one view; serving many views and tiles at
 * once is this library's extension).  Each item is one view slot of one
 * context whose camera is set with hf_set_camera; t_dev / hit_dev receive its
 * ray cast as in hf_raycast (device memory or pinned host memory, checked by
 * hf_batch_prepare).  hf_batch_prepare writes descriptors of all items
 * into a caller-provided host buffer (pinned, so that hf_batch_launch can be
 * captured in a CUDA graph); hf_batch_launch copies them to a caller-provided
 * device buffer and runs the whole batch: one persistent launch drains a work
 * queue of visible rows, discretization tiles and max-mip blocks of every
 * cascade of every item (bounded waits on per-cascade completion counters),
 * then the ray tiles of every item (in a second launch, or in the same one
 * with HF_BATCH_RAYS_INSIDE) -- that is HF_BATCH_PERSISTENT; without it, one
 * launch per phase covers all cascades of all items (five launches in all,
 * meant to be captured in one CUDA graph).  The launch sizes depend only on the items'
 * cascade counts, texture and image sizes, so a captured graph stays valid
 * while those are unchanged and hf_batch_prepare refreshes the pinned
 * descriptors before each replay.  The launch copies host_buf asynchronously:
 * do not prepare into the same host buffer again until that copy has run
 * (e.g. alternate two buffers, or wait on an event recorded after the
 * launch).  Results equal those of the per-view calls.
 * flags select work-unit shapes: HF_BATCH_RAY_TILE_32x8 / _8x32 (default
 * 16x16 pixels per ray unit), HF_BATCH_WARP_16x2 (default 8x4 texels per
 * warp), HF_BATCH_PERSISTENT, HF_BATCH_RAYS_INSIDE (with PERSISTENT only).
 * Errors surface through hf_sync of the items' contexts. */
typedef struct {
    hf_ctx* ctx;
    int32_t view_slot;
    int32_t reserved;
    float* t_dev;
    uint8_t* hit_dev;
} hf_batch_item;

enum {
    HF_BATCH_RAYS_INSIDE = 1,
    HF_BATCH_RAY_TILE_32x8 = 2,
    HF_BATCH_RAY_TILE_8x32 = 4,
    HF_BATCH_WARP_16x2 = 8,
    HF_BATCH_PERSISTENT = 16
};

int hf_batch_query_bytes(const hf_batch_item* items, int32_t n, int32_t flags, size_t* device_bytes,
                         size_t* host_bytes);
int hf_batch_prepare(const hf_batch_item* items, int32_t n, int32_t flags, void* host_buf,
                     size_t host_bytes);
int hf_batch_launch(const void* host_buf, void* dev_buf, size_t dev_bytes, void* stream);
int hf_frame_batch(const hf_batch_item* items, int32_t n, int32_t flags, void* host_buf,
                   size_t host_bytes, void* dev_buf, size_t dev_bytes, void* stream);

/* Waits for `stream` and reports errors recorded on the device since the
 * last hf_sync (HF_ERR_TIMEOUT, HF_ERR_DATA) or by the CUDA runtime. */
int hf_sync(hf_ctx* ctx, void* stream);

/* Self-test of the failure path (no counterpart in the paper): the device
 * loops that could wait on other work -- the batched launch's waits on
 * completion counters -- and the ray walk are bounded, and when a bound runs
 * out the kernel records HF_ERR_TIMEOUT in the context's status block and
 * returns instead of hanging.  This launches one CTA that waits, polling at
 * most `polls` times (1..2^20; a poll is a short sleep and one load), on a
 * status word that nothing sets: the next hf_sync returns HF_ERR_TIMEOUT, clears the status,
 * and the context stays usable.  For tests of error handling. */
int hf_selftest_wait_timeout(hf_ctx* ctx, int32_t polls, void* stream);

/* Measurement support (no counterpart in the paper): the current device's
 * throughput of the two arithmetic units the discretization is designed
 * against -- MUFU ex2.approx (the exponential of Eq. 1) and FP32 fused
 * multiply-add -- in operations per second over all SMs, and its SM count.
 * Short dependency-chain kernels on `stream`, timed with CUDA events; waits
 * for them.  Needs no context. */
int hf_measure_unit_rates(double* ex2_per_s, double* ffma_per_s, int32_t* sm_count, void* stream);

/* Frees the context's host memory.  Device buffers belong to the caller. */
void hf_destroy(hf_ctx* ctx);

/* Message for the calling thread's most recent error ("" if none). */
const char* hf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif

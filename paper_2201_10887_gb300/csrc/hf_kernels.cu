// CUDA kernels for sm_103a: influence-list build, visible-row prep,
// RBF discretization (Eq. 1, Eq. 2), max mipmap and ray casting
// (Cornel et al., 2022, Sections 3-5).
//
// None of these steps is a dense contraction, so no tensor-core path is
// used: the discretization is bound by exp (MUFU) and FP32 issue, the mip
// build by HBM/L2 bandwidth, the ray caster by dependent loads.
#include <cmath>
#include <cstdlib>
#include <cstddef>
#include <cstdint>
#include <thread>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <utility>

#include "hf_internal.h"

namespace hfi {

// ---------------------------------------------------------------------------
// small helpers

__host__ __device__ inline int popc64(uint64_t w) {
#ifdef __CUDA_ARCH__
    return __popcll(w);
#else
    return __builtin_popcountll(w);
#endif
}

__device__ __forceinline__ void report(DevStatus* st, uint32_t flag, uint32_t detail) {
    if (atomicOr(&st->flags, flag) == 0) st->detail = detail;
}

// Loads of data written earlier in the same launch (batched path) go through
// L2 (ld.global.cg), which is coherent across SMs; everything else may use the
// read-only path.
template <bool COH, class T>
__device__ __forceinline__ T ldc(const T* p) {
    if (COH) return __ldcg(p);
    return __ldg(p);
}

// Programmatic dependent launch: the kernels of a frame are launched with
// programmatic stream serialization, so a kernel is set up while its
// predecessor drains; griddepcontrol.wait at its start then holds it until the
// predecessor has completed and its writes are visible (a no-op for a kernel
// launched without the attribute).
__device__ __forceinline__ void wait_for_predecessor() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class... P, class... A>
cudaError_t launch_dependent(void (*kern)(P...), dim3 grid, dim3 block, cudaStream_t s, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Weight of a candidate from q = k * d^2, k taken from its record:
//   HF_RBF_GAUSSIAN (Eq. 1)   k = -log2(e) / (2 sigma^2 c^2):   w = max(2^q - K, 0)
//   HF_RBF_WENDLAND_C2        k = 1 / (radius c)^2, r = sqrt(q): w = (1 - r)_+^4 (4 r + 1)
// (Wendland's compactly supported C2 function psi_{3,1}, the same support
// radius * c as the truncated Gaussian, so the same candidate lists serve.)
template <int KERNEL>
__device__ __forceinline__ float rbf_weight(float q, float K) {
    if (KERNEL == HF_RBF_WENDLAND_C2) {
        const float r = sqrt_approx(q);
        const float t = fmaxf(1.f - r, 0.f), t2 = t * t;
        return t2 * t2 * fmaf(4.f, r, 1.f);
    }
    return fmaxf(ex2_approx(q) - K, 0.f);
}

// ---------------------------------------------------------------------------
// Candidate enumeration for one bucket square (Section 4: the cells that can
// influence any point of the square).  Exact integer geometry in units of
// half a finest cell: a level-L centre sits at (2 ix + 1) 2^(M-L) and
// influences the square when its distance to the square is below
// reach_q[L].  The same code counts on the host and fills on the device.

template <class Visit>
__host__ __device__ inline int64_t for_each_candidate(const EnumTables& t, int Lb, int64_t bx,
                                                      int64_t by, Visit&& visit) {
    const Bitmaps& lf = t.leaves;
    const int M = lf.max_level;
    const int64_t s = int64_t(1) << (M - Lb + 1);
    const int64_t x0 = bx * s, x1 = x0 + s, y0 = by * s, y1 = y0 + s;
    int64_t n = 0;
    for (int L = 0; L <= M; ++L) {
        if (lf.base[L + 1] == lf.base[L]) continue;  // no leaves on this level
        const double r = t.reach_q[L], r2 = r * r;
        const int64_t g = int64_t(1) << (M - L);
        const double inv2g = 0.5 / double(g);
        int64_t lx = int64_t(floor((double(x0) - r) * inv2g - 0.5)) - 1;
        int64_t hx = int64_t(ceil((double(x1) + r) * inv2g - 0.5)) + 1;
        int64_t ly = int64_t(floor((double(y0) - r) * inv2g - 0.5)) - 1;
        int64_t hy = int64_t(ceil((double(y1) + r) * inv2g - 0.5)) + 1;
        lx = lx < 0 ? 0 : lx;
        ly = ly < 0 ? 0 : ly;
        hx = hx > lf.nx[L] - 1 ? lf.nx[L] - 1 : hx;
        hy = hy > lf.ny[L] - 1 ? lf.ny[L] - 1 : hy;
        for (int64_t iy = ly; iy <= hy; ++iy) {
            const int64_t Y = (2 * iy + 1) * g;
            const int64_t dy = Y < y0 ? y0 - Y : (Y > y1 ? Y - y1 : 0);
            if (double(dy * dy) >= r2) continue;
            for (int64_t ix = lx; ix <= hx; ++ix) {
                const int64_t X = (2 * ix + 1) * g;
                const int64_t dx = X < x0 ? x0 - X : (X > x1 ? X - x1 : 0);
                if (double(dx * dx + dy * dy) >= r2) continue;
                const int64_t b = iy * lf.nx[L] + ix;
                const int64_t w = lf.word_off[L] + (b >> 6);
                const uint64_t word = lf.bits[w];
                if ((word >> (b & 63)) & 1ull) {
                    const int64_t id =
                        lf.base[L] + lf.prefix[w] + popc64(word & ((1ull << (b & 63)) - 1ull));
                    visit(n, id);
                    ++n;
                }
            }
        }
    }
    return n;
}

// Locate the bucket word/bit of a linear bit position over all levels.
__host__ __device__ inline bool bucket_of_bit(const Bitmaps& bk, int64_t w, int bit, int& Lb,
                                              int64_t& bx, int64_t& by, int64_t& id) {
    int L = 0;
    while (L < bk.max_level && w >= bk.word_off[L + 1]) ++L;
    if (w < bk.word_off[L] || w >= bk.word_off[L + 1]) return false;
    const uint64_t word = bk.bits[w];
    if (!((word >> bit) & 1ull)) return false;
    const int64_t b = (w - bk.word_off[L]) * 64 + bit;
    Lb = L;
    bx = b % bk.nx[L];
    by = b / bk.nx[L];
    id = bk.base[L] + bk.prefix[w] + popc64(word & ((1ull << bit) - 1ull));
    return true;
}

struct CountOnly {
    __host__ __device__ void operator()(int64_t, int64_t) const {}
};

void count_lists_host(const EnumTables& et, const LookupTables& lt, int64_t* counts,
                      int n_threads) {
    const Bitmaps& bk = lt.buckets;
    const int64_t words = bk.word_off[bk.max_level + 1];
    if (n_threads < 1) n_threads = 1;
    auto work = [&](int64_t w0, int64_t w1) {
        for (int64_t w = w0; w < w1; ++w) {
            uint64_t word = bk.bits[w];
            while (word) {
                const int bit = __builtin_ctzll(word);
                word &= word - 1;
                int Lb;
                int64_t bx, by, id;
                if (bucket_of_bit(bk, w, bit, Lb, bx, by, id))
                    counts[id] = for_each_candidate(et, Lb, bx, by, CountOnly{});
            }
        }
    };
    std::vector<std::thread> pool;
    const int64_t chunk = (words + n_threads - 1) / n_threads;
    for (int t = 0; t < n_threads; ++t) {
        int64_t a = t * chunk, b = a + chunk < words ? a + chunk : words;
        if (a >= b) break;
        pool.emplace_back(work, a, b);
    }
    for (auto& th : pool) th.join();
}

// One thread per (bucket word, bit): fill that bucket's candidate list.
struct FillArgs {
    EnumTables et;
    Bitmaps buckets;
    ListsView lv;
    DevStatus* status;
};

__global__ void __launch_bounds__(256) k_fill_lists(const __grid_constant__ FillArgs a) {
    __shared__ EnumTables et;
    __shared__ Bitmaps bk;
    if (threadIdx.x == 0) {
        et = a.et;
        bk = a.buckets;
    }
    __syncthreads();
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t w = g >> 6;
    if (w >= bk.word_off[bk.max_level + 1]) return;
    int Lb;
    int64_t bx, by, id;
    if (!bucket_of_bit(bk, w, int(g & 63), Lb, bx, by, id)) return;
    const int64_t beg = a.lv.offsets[id], cap = a.lv.offsets[id + 1] - beg;
    int32_t* out = a.lv.idx + beg;
    const int64_t n = for_each_candidate(et, Lb, bx, by, [&](int64_t k, int64_t leaf) {
        if (k < cap) out[k] = int32_t(leaf);
    });
    // the host sized the list as its count rounded up to kListPad
    if (n > cap || cap - n >= kListPad) {
        report(a.status, kStatusData, uint32_t(id));
        return;
    }
    for (int64_t k = n; k < cap; ++k) out[k] = a.lv.sentinel;
}

int launch_fill_lists(const EnumTables& et, const LookupTables& lt, const ListsView& lv,
                      DevStatus* status, void* stream) {
    FillArgs a{et, lt.buckets, lv, status};
    const int64_t words = lt.buckets.word_off[lt.buckets.max_level + 1];
    const int64_t threads = words * 64;
    if (threads == 0) return cudaSuccess;
    const int64_t blocks = (threads + 255) / 256;
    k_fill_lists<<<dim3(unsigned(blocks)), 256, 0, cudaStream_t(stream)>>>(a);
    return cudaGetLastError();
}

// Compact pair lists for the reduced-precision path, one thread per bucket
// (same (word, bit) mapping as the list fill).  A pair of consecutive
// candidates takes 16 bytes: x0 x1 and y0 y1 in the 16-bit type (centres
// relative to the bucket's lower corner in units of half a finest cell: exact
// small integers for cells of a power-of-two hierarchy), then the two FP32
// values with their 4 lowest mantissa bits replaced by the candidates' levels
// (a change of at most 15 ulp).  The kernel rebuilds a candidate's 16-bit
// exponent scale from its level.  An odd list ends with a far-away entry of
// value 0.
template <int PREC>
__device__ __forceinline__ unsigned short to16(float x) {
    if (PREC == HF_PREC_FP16) return __half_as_ushort(__float2half_rn(x));
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

template <int PREC>
__global__ void __launch_bounds__(256) k_fill_compact(const __grid_constant__ FillArgs a,
                                                      const CompactView cv) {
    __shared__ Bitmaps bk;
    if (threadIdx.x == 0) bk = a.buckets;
    __syncthreads();
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t w = g >> 6;
    if (w >= bk.word_off[bk.max_level + 1]) return;
    int Lb;
    int64_t bx, by, id;
    if (!bucket_of_bit(bk, w, int(g & 63), Lb, bx, by, id)) return;
    const int M = a.et.leaves.max_level;
    const float x0q = float(bx << (M - Lb + 1)), y0q = float(by << (M - Lb + 1));
    const int64_t beg = a.lv.offsets[id];
    int64_t n = a.lv.offsets[id + 1] - beg;
    while (n > 0 && a.lv.idx[beg + n - 1] == a.lv.sentinel) --n;  // drop the padding
    const int64_t pb = cv.pair_offsets[id];
    for (int64_t m = 0; m < 2 * ((n + 1) / 2); m += 2) {
        float xs[2], ys[2];
        uint32_t vb[2];
        for (int s = 0; s < 2; ++s) {
            if (m + s < n) {
                const int32_t leaf = a.lv.idx[beg + m + s];
                const float4 r = a.lv.recs[leaf];
                int L = 0;  // records are sorted by level
                while (L < M && leaf >= a.et.leaves.base[L + 1]) ++L;
                xs[s] = r.x * cv.inv_q - x0q;
                ys[s] = r.y * cv.inv_q - y0q;
                vb[s] = (__float_as_uint(r.w) & ~15u) | uint32_t(L);
            } else {  // padding: far away, value 0
                xs[s] = 1024.f;
                ys[s] = 1024.f;
                vb[s] = uint32_t(M);
            }
        }
        uint4 c;
        c.x = uint32_t(to16<PREC>(xs[0])) | (uint32_t(to16<PREC>(xs[1])) << 16);
        c.y = uint32_t(to16<PREC>(ys[0])) | (uint32_t(to16<PREC>(ys[1])) << 16);
        c.z = vb[0];
        c.w = vb[1];
        cv.pairs[pb + m / 2] = c;
    }
}

int launch_fill_compact(const EnumTables& et, const LookupTables& lt, const ListsView& lv,
                        const CompactView& cv, int precision, void* stream) {
    FillArgs a{et, lt.buckets, lv, nullptr};
    const int64_t words = lt.buckets.word_off[lt.buckets.max_level + 1];
    if (words == 0) return cudaSuccess;
    const unsigned blocks = unsigned((words * 64 + 255) / 256);
    if (precision == HF_PREC_FP16)
        k_fill_compact<HF_PREC_FP16><<<blocks, 256, 0, cudaStream_t(stream)>>>(a, cv);
    else
        k_fill_compact<HF_PREC_BF16><<<blocks, 256, 0, cudaStream_t(stream)>>>(a, cv);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Visible rows (Section 3 mask) and texel coordinates of every cascade, FP64.
// Row j of cascade c sees columns [spans.x, spans.y]: the texel centres inside
// the cascade polygon grown by one texel diagonal and inside the domain.

__device__ __forceinline__ void prep_row(const PrepCascade& q, double dom_w, double dom_h,
                                         double eps_frac, int t) {
    const double h = q.h;
    // on the lattice fit a coordinate is an integer lattice index times h, so
    // that one lattice point gets one coordinate in every frame
    q.xs[t] = float(q.lattice ? double(q.lat_x + t) * h : q.ox + double(t) * h);
    const double y = q.lattice ? double(q.lat_y + t) * h : q.oy + double(t) * h;
    q.ys[t] = float(y);
    const double eps = eps_frac * h;
    int lo = 0, hi = -1;
    if (q.n_edges >= 3 && y >= -eps && y <= dom_h + eps) {
        double xlo = -eps, xhi = dom_w + eps;
        bool empty = false;
        for (int e = 0; e < q.n_edges; ++e) {
            const double rhs = q.c[e] - q.ny[e] * y;
            if (q.sgn[e] > 0) xhi = fmin(xhi, rhs * q.inv_nx[e]);
            else if (q.sgn[e] < 0) xlo = fmax(xlo, rhs * q.inv_nx[e]);
            else if (rhs < 0.0) empty = true;
        }
        if (!empty && xlo <= xhi) {
            double flo = ceil((xlo - q.ox) * q.inv_h), fhi = floor((xhi - q.ox) * q.inv_h);
            flo = fmax(flo, 0.0);
            fhi = fmin(fhi, double(q.N - 1));
            if (flo <= fhi) {
                lo = int(flo);
                hi = int(fhi);
            }
        }
    }
    q.spans[t] = make_int2(lo, hi);
}

__global__ void __launch_bounds__(128) k_prep(const __grid_constant__ PrepParams p) {
    wait_for_predecessor();
    const PrepCascade& q = p.cas[blockIdx.y];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < q.N) prep_row(q, p.dom_w, p.dom_h, p.eps_frac, t);
}

int launch_prep(const PrepParams& p, void* stream) {
    if (p.C == 0) return cudaSuccess;
    dim3 grid((p.max_N + 127) / 128, p.C);
    return launch_dependent(k_prep, grid, dim3(128), cudaStream_t(stream), p);
}

// ---------------------------------------------------------------------------
// Texel -> bucket.  The finest-cell coordinates of the texel are computed once;
// the cell containing it on level L is their shift by max_level - L, so the
// levels are consistent by construction.  Exactly one level holds a bucket.

__device__ __forceinline__ int64_t lookup_bucket(const LookupTables& lt, float px, float py) {
    const Bitmaps& bk = lt.buckets;
    int fx = int(floorf(px * lt.inv_c_fin));
    int fy = int(floorf(py * lt.inv_c_fin));
    fx = min(max(fx, 0), lt.nx_fin - 1);
    fy = min(max(fy, 0), lt.ny_fin - 1);
    const int M = bk.max_level;
    int64_t found = -1;
#pragma unroll
    for (int L = 0; L < kMaxLevels; ++L) {
        if (L >= lt.bucket_level && L <= M) {
            const int sh = M - L;
            const int64_t b = int64_t(fy >> sh) * bk.nx[L] + (fx >> sh);
            const int64_t w = bk.word_off[L] + (b >> 6);
            const uint64_t word = __ldg(reinterpret_cast<const unsigned long long*>(bk.bits) + w);
            if ((word >> (b & 63)) & 1ull)
                found = bk.base[L] + __ldg(bk.prefix + w) + __popcll(word & ((1ull << (b & 63)) - 1ull));
        }
    }
    return found;
}

// The cell map: one thread per finest cell writes its bucket's list as
// {first group, groups} (lists are padded to groups of kListPad entries), or
// for the compact lists {first pair, pairs | bucket level << 24}.
template <bool COMPACT>
__global__ void __launch_bounds__(256) k_fill_cellmap(const __grid_constant__ LookupTables lt, const ListsView lv,
                                                      const CompactView cv, uint2* cellmap, DevStatus* status) {
    const int64_t cell = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (cell >= int64_t(lt.nx_fin) * lt.ny_fin) return;
    const int fx = int(cell % lt.nx_fin), fy = int(cell / lt.nx_fin);
    const Bitmaps& bk = lt.buckets;
    const int M = bk.max_level;
    int64_t found = -1;
    int Lb = 0;
    for (int L = lt.bucket_level; L <= M; ++L) {
        const int sh = M - L;
        const int64_t b = int64_t(fy >> sh) * bk.nx[L] + (fx >> sh);
        const int64_t w = bk.word_off[L] + (b >> 6);
        const uint64_t word = bk.bits[w];
        if ((word >> (b & 63)) & 1ull) {
            found = bk.base[L] + bk.prefix[w] + popc64(word & ((1ull << (b & 63)) - 1ull));
            Lb = L;
        }
    }
    if (found < 0) {
        report(status, kStatusData, uint32_t(cell));
        cellmap[cell] = make_uint2(0u, 0u);
        return;
    }
    if (COMPACT) {
        const int64_t beg = cv.pair_offsets[found], end = cv.pair_offsets[found + 1];
        cellmap[cell] = make_uint2(uint32_t(beg), uint32_t(end - beg) | (uint32_t(Lb) << 24));
    } else {
        const int64_t beg = lv.offsets[found], end = lv.offsets[found + 1];
        cellmap[cell] = make_uint2(uint32_t(beg / kListPad), uint32_t((end - beg) / kListPad));
    }
}

int launch_fill_cellmap(const LookupTables& lt, const ListsView& lv, uint2* cellmap, DevStatus* status,
                        void* stream, const CompactView* cv) {
    const int64_t cells = int64_t(lt.nx_fin) * lt.ny_fin;
    if (cells == 0) return cudaSuccess;
    const dim3 grid(unsigned((cells + 255) / 256));
    if (cv)
        k_fill_cellmap<true><<<grid, 256, 0, cudaStream_t(stream)>>>(lt, lv, *cv, cellmap, status);
    else
        k_fill_cellmap<false><<<grid, 256, 0, cudaStream_t(stream)>>>(lt, lv, CompactView{}, cellmap, status);
    return cudaGetLastError();
}

// Temporal reuse (hf_discretize_reuse): the index of texel (i, j) in the
// earlier frame's texture on the same lattice, or -1 (no source, or outside
// it).  A texel that frame computed (anything but -inf) has the same position
// and therefore the same value: it is copied instead of recomputed.
__device__ __forceinline__ int64_t prev_index(const DiscCascade& q, int i, int j) {
    if (q.prev == nullptr) return -1;
    const int pi = i + q.prev_di, pj = j + q.prev_dj;
    if (unsigned(pi) >= unsigned(q.prev_N) || unsigned(pj) >= unsigned(q.prev_N)) return -1;
    return int64_t(pj) * q.prev_N + pi;
}

// ---------------------------------------------------------------------------
// RBF discretization (Eq. 1, Eq. 2): one thread per texel; a warp covers an
// 8 x 4 texel patch and a CTA a 32 x 8 tile, so that the lanes of a warp
// share buckets and their list and record loads coincide (the kernel is
// bound by the L1 data pipe's wavefronts from these per-lane gathers).
// Each visible texel walks its bucket's list:
//   w_i = max(2^(k_i d_i^2) - K, 0),  k_i = -log2(e) / (2 sigma^2 c_i^2)
//   v   = sum w_i v_i / sum w_i.
// Invisible texels are written as -inf so the texture is fully defined.
// With the water layer the same weights also sum the cells' water depths d_i
// (terrain and depths live on the same cells, Section 2): the water surface
// texel is v + sum w_i d_i / sum w_i where that depth is positive, else -inf.

// One bulk prefetch of a texel's whole list (16-byte aligned, n 16-byte units)
// into L2 before its walk: in the far cascades neighbouring texels use
// different lists, and the walk's loads then find them in L2 rather than in
// HBM.
__device__ __forceinline__ void prefetch_l2(const uint4* p, int n) {
    if (n > 0) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(uint32_t(n) * 16u) : "memory");
}

// Writes texel (i, j) if it is invisible (-inf) or carried over from an
// earlier frame and returns true; false: the texel must be computed.
template <bool COH, bool WATER>
__device__ __forceinline__ bool texel_settled(const DiscCascade& q, int i, int j) {
    const int2 sp = ldc<COH>(q.spans + j);
    const size_t o = size_t(j) * q.N + i;
    if (i < sp.x || i > sp.y) {
        q.tex[o] = -INFINITY;
        if (WATER) q.wtex[o] = -INFINITY;
        return true;
    }
    const int64_t po = prev_index(q, i, j);
    if (po >= 0) {
        const float old = ldc<COH>(q.prev + po);
        if (old != -INFINITY) {
            q.tex[o] = old;
            if (WATER) q.wtex[o] = ldc<COH>(q.prev_w + po);
            return true;
        }
    }
    return false;
}

// Eq. 2 at visible texel (i, j), walking its bucket's list in global memory.
template <bool COH, bool WATER, int KERNEL>
__device__ __forceinline__ void texel_rbf(const DiscCascade& q, float K, const LookupTables& lt,
                                          const ListsView& lv, DevStatus* status, int i, int j) {
    const size_t o = size_t(j) * q.N + i;
    float* out = q.tex + o;
    const float px = ldc<COH>(q.xs + i), py = ldc<COH>(q.ys + j);
    // lists start on 16-byte boundaries and are padded to groups of four
    // entries (null records weigh exactly 0): one load brings four indices
    const int4* groups;
    int ng;
    if (lt.cellmap) {  // one load: the finest cell's {first group, groups}
        const int fx = min(max(int(floorf(px * lt.inv_c_fin)), 0), lt.nx_fin - 1);
        const int fy = min(max(int(floorf(py * lt.inv_c_fin)), 0), lt.ny_fin - 1);
        const uint2 e = __ldg(lt.cellmap + size_t(fy) * lt.nx_fin + fx);
        groups = reinterpret_cast<const int4*>(lv.idx) + e.x;
        ng = int(e.y);
    } else {
        const int64_t bucket = lookup_bucket(lt, px, py);
        if (bucket < 0) {
            report(status, kStatusData, 0xFFFFFFFFu);
            *out = __int_as_float(0x7fc00000);
            if (WATER) q.wtex[o] = __int_as_float(0x7fc00000);
            return;
        }
        const int64_t beg = __ldg(lv.offsets + bucket);
        ng = int(__ldg(lv.offsets + bucket + 1) - beg) / kListPad;
        groups = reinterpret_cast<const int4*>(lv.idx + beg);
    }
    float sw = 0.f, swv = 0.f, swd = 0.f;
    auto term = [&](int id) {
        const float4 r = __ldg(lv.recs + id);
        const float dx = r.x - px, dy = r.y - py;
        const float w = rbf_weight<KERNEL>(r.z * fmaf(dx, dx, dy * dy), K);
        sw += w;
        swv = fmaf(w, r.w, swv);
        if (WATER) swd = fmaf(w, __ldg(lv.depth + id), swd);
    };
    for (int g = 0; g < ng; ++g) {
        const int4 q4 = __ldg(groups + g);
        term(q4.x);
        term(q4.y);
        term(q4.z);
        term(q4.w);
    }
    const float v = sw > 0.f ? swv / sw : __int_as_float(0x7fc00000);
    *out = v;
    if (WATER) q.wtex[o] = swd > 0.f ? v + swd / sw : -INFINITY;
}

template <bool COH, bool WATER = false, int KERNEL = HF_RBF_GAUSSIAN>
__device__ __forceinline__ void discretize_texel(const DiscCascade& q, float K, const LookupTables& lt,
                                                 const ListsView& lv, DevStatus* status, int i, int j) {
    if (i >= q.N || j >= q.N) return;
    if (texel_settled<COH, WATER>(q, i, j)) return;
    texel_rbf<COH, WATER, KERNEL>(q, K, lt, lv, status, i, j);
}

// texel of thread t (0..255) in a 32 x 8 tile: warp = 8 x 4 patch
__device__ __forceinline__ void tile_texel(int t, int& di, int& dj) {
    const int lane = t & 31, warp = t >> 5;
    di = (warp & 3) * 8 + (lane & 7);
    dj = (warp >> 2) * 4 + (lane >> 3);
}

template <bool WATER, int KERNEL>
__global__ void __launch_bounds__(256, 8) k_discretize_f32(const __grid_constant__ DiscParams p,
                                                        const __grid_constant__ LookupTables lt,
                                                        const ListsView lv, DevStatus* status) {
    wait_for_predecessor();
    int di, dj;
    tile_texel(threadIdx.x, di, dj);
    discretize_texel<false, WATER, KERNEL>(p.cas[blockIdx.z], p.K, lt, lv, status, blockIdx.x * 32 + di,
                                           blockIdx.y * 8 + dj);
}

// Reduced-precision discretization: the same texel mapping, bucket lookup and
// Eq. 2, but distances, scales and the exponential are evaluated two
// candidates at a time in FP16x2 or BF16x2 arithmetic (ex2.approx on packed
// pairs); weights are widened to FP32 for the sums.
__device__ __forceinline__ int64_t lookup_bucket_at(const LookupTables& lt, float px, float py,
                                                    int& Lb, int& bx, int& by) {
    const Bitmaps& bk = lt.buckets;
    int fx = int(floorf(px * lt.inv_c_fin));
    int fy = int(floorf(py * lt.inv_c_fin));
    fx = min(max(fx, 0), lt.nx_fin - 1);
    fy = min(max(fy, 0), lt.ny_fin - 1);
    const int M = bk.max_level;
    int64_t found = -1;
#pragma unroll
    for (int L = 0; L < kMaxLevels; ++L) {
        if (L >= lt.bucket_level && L <= M) {
            const int sh = M - L;
            const int64_t b = int64_t(fy >> sh) * bk.nx[L] + (fx >> sh);
            const int64_t w = bk.word_off[L] + (b >> 6);
            const uint64_t word = __ldg(reinterpret_cast<const unsigned long long*>(bk.bits) + w);
            if ((word >> (b & 63)) & 1ull) {
                found = bk.base[L] + __ldg(bk.prefix + w) + __popcll(word & ((1ull << (b & 63)) - 1ull));
                Lb = L;
                bx = fx >> sh;
                by = fy >> sh;
            }
        }
    }
    return found;
}

struct F16Ops {
    typedef __half2 T;
    static constexpr uint32_t kStep = 1u << 11;  // x4 in the exponent field
    static __device__ __forceinline__ T make(float a) { return __float2half2_rn(a); }
    static __device__ __forceinline__ T bits(uint32_t u) {
        T r;
        memcpy(&r, &u, 4);
        return r;
    }
    static __device__ __forceinline__ T exp2(T x) {
        uint32_t u, r;
        memcpy(&u, &x, 4);
        asm("ex2.approx.f16x2 %0, %1;" : "=r"(r) : "r"(u));
        return bits(r);
    }
    static __device__ __forceinline__ float2 widen(T x) { return __half22float2(x); }
};

struct BF16Ops {
    typedef __nv_bfloat162 T;
    static constexpr uint32_t kStep = 1u << 8;   // x4 in the exponent field
    static __device__ __forceinline__ T make(float a) { return __float2bfloat162_rn(a); }
    static __device__ __forceinline__ T bits(uint32_t u) {
        T r;
        memcpy(&r, &u, 4);
        return r;
    }
    static __device__ __forceinline__ T exp2(T x) {
        uint32_t u, r;
        memcpy(&u, &x, 4);
        asm("ex2.approx.ftz.bf16x2 %0, %1;" : "=r"(r) : "r"(u));
        return bits(r);
    }
    static __device__ __forceinline__ float2 widen(T x) { return __bfloat1622float2(x); }
};

template <class Ops, bool COH>
__device__ __forceinline__ void discretize_texel_mixed(const DiscCascade& q, float K, const LookupTables& lt,
                                                       const CompactView& cv, DevStatus* status, int i, int j) {
    typedef typename Ops::T T;
    if (i >= q.N || j >= q.N) return;
    const int2 sp = ldc<COH>(q.spans + j);
    float* out = q.tex + size_t(j) * q.N + i;
    if (i < sp.x || i > sp.y) {
        *out = -INFINITY;
        return;
    }
    const int64_t po = prev_index(q, i, j);
    if (po >= 0) {
        const float old = ldc<COH>(q.prev + po);
        if (old != -INFINITY) {
            *out = old;
            return;
        }
    }
    const float px = ldc<COH>(q.xs + i), py = ldc<COH>(q.ys + j);
    int Lb = 0, bx = 0, by = 0;
    int64_t pb;
    int np;
    if (cv.cellmap) {  // one load: the finest cell's {first pair, pairs | bucket level << 24}
        const int fx = min(max(int(floorf(px * lt.inv_c_fin)), 0), lt.nx_fin - 1);
        const int fy = min(max(int(floorf(py * lt.inv_c_fin)), 0), lt.ny_fin - 1);
        const uint2 e = __ldg(cv.cellmap + size_t(fy) * lt.nx_fin + fx);
        pb = e.x;
        np = int(e.y & 0xFFFFFFu);
        Lb = int(e.y >> 24);
        bx = fx >> (lt.buckets.max_level - Lb);
        by = fy >> (lt.buckets.max_level - Lb);
    } else {
        const int64_t bucket = lookup_bucket_at(lt, px, py, Lb, bx, by);
        if (bucket < 0) {
            report(status, kStatusData, 0xFFFFFFFFu);
            *out = __int_as_float(0x7fc00000);
            return;
        }
        pb = __ldg(cv.pair_offsets + bucket);
        np = int(__ldg(cv.pair_offsets + bucket + 1) - pb);
    }
    const int sh = lt.buckets.max_level - Lb + 1;
    const T PX = Ops::make(fmaf(px, cv.inv_q, -float(bx << sh)));
    const T PY = Ops::make(fmaf(py, cv.inv_q, -float(by << sh)));
    const T NK = Ops::make(-K);
    const T ONE = Ops::make(1.f);
    const uint4* cc = cv.pairs + pb;
    prefetch_l2(cc, np);
    const uint32_t kb2 = cv.kb2;
    float sw = 0.f, swv = 0.f;
#pragma unroll 3
    for (int k = 0; k < np; ++k) {
        const uint4 c = __ldg(cc + k);
        const T dx = __hsub2(Ops::bits(c.x), PX);
        const T dy = __hsub2(Ops::bits(c.y), PY);
        const T d2 = __hfma2(dx, dx, __hmul2(dy, dy));
        // both levels into one word (L0 | L1 << 16), then both 16-bit scales in one IMAD
        const uint32_t lv = __byte_perm(c.z, c.w, 0x5410) & 0x000F000Fu;
        const T e = Ops::exp2(__hmul2(Ops::bits(lv * Ops::kStep + kb2), d2));
        const float2 w = Ops::widen(__hfma2_relu(e, ONE, NK));
        sw += w.x + w.y;
        swv = fmaf(w.x, __uint_as_float(c.z), fmaf(w.y, __uint_as_float(c.w), swv));
    }
    *out = sw > 0.f ? swv / sw : __int_as_float(0x7fc00000);
}

// a_k - p for the two FP16 values a_0 (low half) and a_1 of u, in FP32: an
// FP16 value converts to FP32 exactly, so this is __half2float(a_k) - p with
// one rounding, done by the mixed-precision subtraction.
__device__ __forceinline__ float2 sub_f16x2_f32(uint32_t u, float p) {
    float2 r;
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
        "sub.rn.f32.f16 %0, lo, %3;\n\tsub.rn.f32.f16 %1, hi, %3;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "r"(u), "f"(p));
    return r;
}

// Eq. 2 in FP32 arithmetic from the compact pair lists (FP16-format
// coordinates): one 16-byte load brings two candidates and no index
// indirection is needed.  Positions are the lists' exact small integers (half
// finest cells from the bucket corner) against the texel's position in the
// same units; the weight scale of level L is the finest level's divided by
// 4^(M - L), built exactly in the exponent field; exp2, weights and sums are
// FP32.  The values carry the level in their 4 lowest mantissa bits (at most
// 15 ulp of the value).
template <bool COH, int KERNEL>
__device__ __forceinline__ void discretize_texel_f32c(const DiscCascade& q, float K, const LookupTables& lt,
                                                      const CompactView& cv, DevStatus* status, int i, int j) {
    if (i >= q.N || j >= q.N) return;
    if (texel_settled<COH, false>(q, i, j)) return;
    float* out = q.tex + size_t(j) * q.N + i;
    const float px = ldc<COH>(q.xs + i), py = ldc<COH>(q.ys + j);
    int Lb = 0, bx = 0, by = 0;
    int64_t pb;
    int np;
    if (cv.cellmap) {
        const int fx = min(max(int(floorf(px * lt.inv_c_fin)), 0), lt.nx_fin - 1);
        const int fy = min(max(int(floorf(py * lt.inv_c_fin)), 0), lt.ny_fin - 1);
        const uint2 e = __ldg(cv.cellmap + size_t(fy) * lt.nx_fin + fx);
        pb = e.x;
        np = int(e.y & 0xFFFFFFu);
        Lb = int(e.y >> 24);
        bx = fx >> (cv.max_level - Lb);
        by = fy >> (cv.max_level - Lb);
    } else {
        const int64_t bucket = lookup_bucket_at(lt, px, py, Lb, bx, by);
        if (bucket < 0) {
            report(status, kStatusData, 0xFFFFFFFFu);
            *out = __int_as_float(0x7fc00000);
            return;
        }
        pb = __ldg(cv.pair_offsets + bucket);
        np = int(__ldg(cv.pair_offsets + bucket + 1) - pb);
    }
    const int sh = cv.max_level - Lb + 1;
    const float PX = fmaf(px, cv.inv_q, -float(bx << sh));
    const float PY = fmaf(py, cv.inv_q, -float(by << sh));
    const uint4* cc = cv.pairs + pb;
    prefetch_l2(cc, np);
    const uint32_t kf = cv.kf_bits + (uint32_t(15 - cv.max_level) << 24);  // so that level L adds L << 24 - 15 << 24
    // the two candidates of a pair go through the packed FP32x2 instructions;
    // even and odd candidates are summed apart and added at the end
    float2 sw = make_float2(0.f, 0.f), swv = make_float2(0.f, 0.f);
    const float2 nK = make_float2(-K, -K);
#pragma unroll 2
    for (int k = 0; k < np; ++k) {
        const uint4 c = __ldg(cc + k);
        const float2 dx = sub_f16x2_f32(c.x, PX), dy = sub_f16x2_f32(c.y, PY);
        const float2 kk = make_float2(__uint_as_float(kf - ((15u - (c.z & 15u)) << 24)),
                                      __uint_as_float(kf - ((15u - (c.w & 15u)) << 24)));
        const float2 q = __fmul2_rn(kk, __ffma2_rn(dx, dx, __fmul2_rn(dy, dy)));
        float2 w;
        if (KERNEL == HF_RBF_GAUSSIAN) {
            w = __fadd2_rn(make_float2(ex2_approx(q.x), ex2_approx(q.y)), nK);
            w.x = fmaxf(w.x, 0.f);
            w.y = fmaxf(w.y, 0.f);
        } else {
            w = make_float2(rbf_weight<KERNEL>(q.x, K), rbf_weight<KERNEL>(q.y, K));
        }
        sw = __fadd2_rn(sw, w);
        swv = __ffma2_rn(w, make_float2(__uint_as_float(c.z), __uint_as_float(c.w)), swv);
    }
    const float s = sw.x + sw.y;
    *out = s > 0.f ? (swv.x + swv.y) / s : __int_as_float(0x7fc00000);
}

template <int KERNEL>
__global__ void __launch_bounds__(256, 8) k_discretize_f32c(const __grid_constant__ DiscParams p,
                                                            const __grid_constant__ LookupTables lt,
                                                            const CompactView cv, DevStatus* status) {
    wait_for_predecessor();
    int di, dj;
    tile_texel(threadIdx.x, di, dj);
    discretize_texel_f32c<false, KERNEL>(p.cas[blockIdx.z], p.K, lt, cv, status, blockIdx.x * 32 + di,
                                         blockIdx.y * 8 + dj);
}

int launch_discretize_f32c(const DiscParams& p, const LookupTables& lt, const CompactView& cv,
                           DevStatus* status, void* stream) {
    if (p.C == 0) return cudaSuccess;
    dim3 grid((p.max_N + 31) / 32, (p.max_N + 7) / 8, p.C);
    if (p.kernel == HF_RBF_WENDLAND_C2)
        return launch_dependent(k_discretize_f32c<HF_RBF_WENDLAND_C2>, grid, dim3(256), cudaStream_t(stream), p, lt, cv,
                                status);
    return launch_dependent(k_discretize_f32c<HF_RBF_GAUSSIAN>, grid, dim3(256), cudaStream_t(stream), p, lt, cv, status);
}

template <class Ops>
__global__ void __launch_bounds__(256) k_discretize_mixed(const __grid_constant__ DiscParams p,
                                                          const __grid_constant__ LookupTables lt,
                                                          const CompactView cv, DevStatus* status) {
    wait_for_predecessor();
    int di, dj;
    tile_texel(threadIdx.x, di, dj);
    discretize_texel_mixed<Ops, false>(p.cas[blockIdx.z], p.K, lt, cv, status, blockIdx.x * 32 + di,
                                       blockIdx.y * 8 + dj);
}

int launch_discretize_mixed(const DiscParams& p, const LookupTables& lt, const CompactView& cv,
                            DevStatus* status, void* stream) {
    if (p.C == 0) return cudaSuccess;
    dim3 grid((p.max_N + 31) / 32, (p.max_N + 7) / 8, p.C);
    if (p.precision == HF_PREC_FP16)
        return launch_dependent(k_discretize_mixed<F16Ops>, grid, dim3(256), cudaStream_t(stream), p, lt, cv, status);
    return launch_dependent(k_discretize_mixed<BF16Ops>, grid, dim3(256), cudaStream_t(stream), p, lt, cv, status);
}

int launch_discretize(const DiscParams& p, const LookupTables& lt, const ListsView& lv,
                      DevStatus* status, void* stream) {
    if (p.C == 0) return cudaSuccess;
    dim3 grid((p.max_N + 31) / 32, (p.max_N + 7) / 8, p.C);
    cudaStream_t s = cudaStream_t(stream);
    const bool wend = p.kernel == HF_RBF_WENDLAND_C2;
    if (p.water && wend)
        return launch_dependent(k_discretize_f32<true, HF_RBF_WENDLAND_C2>, grid, dim3(256), s, p, lt, lv, status);
    if (p.water)
        return launch_dependent(k_discretize_f32<true, HF_RBF_GAUSSIAN>, grid, dim3(256), s, p, lt, lv, status);
    if (wend)
        return launch_dependent(k_discretize_f32<false, HF_RBF_WENDLAND_C2>, grid, dim3(256), s, p, lt, lv, status);
    return launch_dependent(k_discretize_f32<false, HF_RBF_GAUSSIAN>, grid, dim3(256), s, p, lt, lv, status);
}

// Measurement pass: the discretization's texel mapping and inner loop, but
// counting visible texels, list entries walked, terms with w > 0 and texels
// carried over from an earlier frame instead of writing heights.  Warp sums, one 64-bit atomic per warp and counter.
template <int KERNEL>
__global__ void __launch_bounds__(256) k_stats_f32(const __grid_constant__ DiscParams p,
                                                   const __grid_constant__ LookupTables lt,
                                                   const ListsView lv, DevStatus* status) {
    const int c = blockIdx.z;
    const DiscCascade& q = p.cas[c];
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    unsigned vis = 0, cand = 0, infl = 0, reused = 0;
    if (i < q.N && j < q.N) {
        const int2 sp = __ldg(q.spans + j);
        if (i >= sp.x && i <= sp.y) {
            const int64_t po = prev_index(q, i, j);
            reused = po >= 0 && __ldg(q.prev + po) != -INFINITY ? 1u : 0u;
            const float px = __ldg(q.xs + i), py = __ldg(q.ys + j);
            const int64_t bucket = lookup_bucket(lt, px, py);
            if (bucket >= 0) {
                const int64_t beg = __ldg(lv.offsets + bucket);
                const int n = int(__ldg(lv.offsets + bucket + 1) - beg);
                const int32_t* ids = lv.idx + beg;
                vis = 1;
                for (int k = 0; k < n; ++k) {
                    const int id = __ldg(ids + k);
                    cand += id != lv.sentinel ? 1u : 0u;  // padding is not a candidate
                    const float4 r = __ldg(lv.recs + id);
                    const float dx = r.x - px, dy = r.y - py;
                    infl += rbf_weight<KERNEL>(r.z * fmaf(dx, dx, dy * dy), p.K) > 0.f ? 1u : 0u;
                }
            }
        }
    }
    vis = __reduce_add_sync(0xffffffffu, vis);
    cand = __reduce_add_sync(0xffffffffu, cand);
    infl = __reduce_add_sync(0xffffffffu, infl);
    reused = __reduce_add_sync(0xffffffffu, reused);
    if ((threadIdx.x & 31) == 0 && vis) {
        atomicAdd(&status->counters[c], (unsigned long long)vis);
        atomicAdd(&status->counters[HF_MAX_CASCADES + c], (unsigned long long)cand);
        atomicAdd(&status->counters[2 * HF_MAX_CASCADES + c], (unsigned long long)infl);
        if (reused) atomicAdd(&status->counters[3 * HF_MAX_CASCADES + c], (unsigned long long)reused);
    }
}

int launch_stats(const DiscParams& p, const LookupTables& lt, const ListsView& lv,
                 DevStatus* status, void* stream) {
    if (p.C == 0) return cudaSuccess;
    dim3 grid((p.max_N + 31) / 32, (p.max_N + 7) / 8, p.C);
    if (p.kernel == HF_RBF_WENDLAND_C2)
        k_stats_f32<HF_RBF_WENDLAND_C2><<<grid, dim3(32, 8), 0, cudaStream_t(stream)>>>(p, lt, lv, status);
    else
        k_stats_f32<HF_RBF_GAUSSIAN><<<grid, dim3(32, 8), 0, cudaStream_t(stream)>>>(p, lt, lv, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Maximum mipmap (Section 5, Tevs et al.).  Level 0 entry (pi, pj) is the max
// of the patch's four corner texels, -inf if one is invisible or the patch
// lies in the padding; level k is the max of 2x2 entries of level k-1.
// k_mip_lo: one CTA per 64x64 block of level 0 builds levels 0..6 of it
// (each thread 4x4 level-0 entries from a 5x5 texel window, then 2x2 and 1 in
// registers, 3 and 4 across lanes, 5 and 6 in shared memory).  k_mip_hi: one
// CTA per cascade builds levels 7..K.

__device__ __forceinline__ int64_t mip_off(int P, int k) {
    const int64_t a = int64_t(P) * P, b = int64_t(P >> k) * (P >> k);
    return (a - b) * 4 / 3;
}

// 5 x 5 texels from (pi0, pj0): -inf outside the texture.  Rows are read as
// one float4 plus a scalar where the texture's rows are 16-byte aligned
// (N % 4 == 0) and the window lies inside them, else texel by texel.  With
// the rows' visible spans, a window row outside its span is -inf without
// reading it (the discretization wrote -inf there).  Returns false when no
// row of the window was read.
template <bool COH>
__device__ __forceinline__ bool load_window(const float* __restrict__ tex, const int2* __restrict__ spans, int N,
                                            int pi0, int pj0, float (&t)[5][5]) {
    const bool vec = (N & 3) == 0 && pi0 + 4 < N;
    bool any = false;
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const int jj = pj0 + r;
        const float* row = tex + size_t(jj) * N;
        bool skip = jj >= N;
        if (!skip && spans) {
            const int2 sp = ldc<COH>(spans + jj);
            skip = sp.y < pi0 || sp.x > pi0 + 4;
        }
        if (skip) {
#pragma unroll
            for (int s = 0; s < 5; ++s) t[r][s] = -INFINITY;
        } else if (vec) {
            const float4 v = ldc<COH>(reinterpret_cast<const float4*>(row + pi0));
            t[r][0] = v.x;
            t[r][1] = v.y;
            t[r][2] = v.z;
            t[r][3] = v.w;
            t[r][4] = ldc<COH>(row + pi0 + 4);
        } else {
#pragma unroll
            for (int s = 0; s < 5; ++s) t[r][s] = pi0 + s < N ? ldc<COH>(row + pi0 + s) : -INFINITY;
        }
        any |= !skip;
    }
    return any;
}

// Level-0 entries of the 4 x 4 patches whose lower corners are (pi0 + s, pj0 + r):
// the maximum of the four corners, -inf for a patch with an undefined corner
// or beyond the N-1 patches of a row.
template <bool COH>
__device__ __forceinline__ void patch_maxima(const float* __restrict__ tex, const int2* __restrict__ spans, int N,
                                             int pi0, int pj0, float (&m0)[4][4]) {
    float t[5][5];
    if (!load_window<COH>(tex, spans, N, pi0, pj0, t)) {  // nothing visible in the window
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int s = 0; s < 4; ++s) m0[r][s] = -INFINITY;
        return;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const float a = t[r][s], b = t[r][s + 1], d = t[r + 1][s], e = t[r + 1][s + 1];
            const bool ok = (pi0 + s < N - 1) && (pj0 + r < N - 1) && isfinite(a) && isfinite(b) &&
                            isfinite(d) && isfinite(e);
            m0[r][s] = ok ? fmaxf(fmaxf(a, b), fmaxf(d, e)) : -INFINITY;
        }
}

// Levels 0..6 of one 64 x 64 block of patches (256 threads, 4 x 4 patches
// each).  Warp w covers threads tx in [8 (w & 1), +8), ty in [4 (w >> 1), +4):
// levels 1 and 2 stay in registers, levels 3 and 4 are 2 x 2 reductions across
// lanes (__shfl_xor_sync), levels 5 and 6 combine the block's sixteen level-4
// entries through shared memory.  With TWO (the water layer) a level-0 entry
// bounds the water patch too, where it exists.
template <bool COH, bool TWO = false>
__device__ __forceinline__ void mip_lo_block(const MipCascade& c, int bxi, int byi, float (*sm)[17]) {
    const int P = c.P, N = c.N, K = c.K;
    if (bxi * 64 >= P || byi * 64 >= P) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tx = (warp & 1) * 8 + (lane & 7), ty = (warp >> 1) * 4 + (lane >> 3);
    const int pi0 = bxi * 64 + tx * 4, pj0 = byi * 64 + ty * 4;
    float m0[4][4];
    patch_maxima<COH>(c.tex, c.spans, N, pi0, pj0, m0);
    if (TWO) {
        float w0[4][4];
        patch_maxima<COH>(c.wtex, c.spans, N, pi0, pj0, w0);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int s = 0; s < 4; ++s) m0[r][s] = fmaxf(m0[r][s], w0[r][s]);
    }
    if (pi0 < P && pj0 < P) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (pj0 + r >= P) break;
            float* dst = c.mip + size_t(pj0 + r) * P + pi0;
            if (P >= 4) {
                *reinterpret_cast<float4*>(dst) = make_float4(m0[r][0], m0[r][1], m0[r][2], m0[r][3]);
            } else {
                for (int s = 0; s < 4 && pi0 + s < P; ++s) dst[s] = m0[r][s];
            }
        }
    }
    if (K < 1) return;
    float m1[2][2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int s = 0; s < 2; ++s)
            m1[r][s] = fmaxf(fmaxf(m0[2 * r][2 * s], m0[2 * r][2 * s + 1]),
                             fmaxf(m0[2 * r + 1][2 * s], m0[2 * r + 1][2 * s + 1]));
    {
        const int P1 = P >> 1, pi1 = pi0 >> 1, pj1 = pj0 >> 1;
        float* base = c.mip + mip_off(P, 1);
        for (int r = 0; r < 2; ++r)
            for (int s = 0; s < 2; ++s)
                if (pi1 + s < P1 && pj1 + r < P1) base[size_t(pj1 + r) * P1 + pi1 + s] = m1[r][s];
    }
    const float m2 = fmaxf(fmaxf(m1[0][0], m1[0][1]), fmaxf(m1[1][0], m1[1][1]));
    if (K >= 2) {
        const int P2 = P >> 2, pi2 = pi0 >> 2, pj2 = pj0 >> 2;
        if (pi2 < P2 && pj2 < P2) c.mip[mip_off(P, 2) + size_t(pj2) * P2 + pi2] = m2;
    }
    // level 3: threads (tx, tx ^ 1) x (ty, ty ^ 1) are lanes (l, l ^ 1) x (l, l ^ 8)
    float m3 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, 1));
    m3 = fmaxf(m3, __shfl_xor_sync(0xffffffffu, m3, 8));
    if (K >= 3 && ((tx | ty) & 1) == 0) {
        const int P3 = P >> 3, gx = bxi * 8 + (tx >> 1), gy = byi * 8 + (ty >> 1);
        if (gx < P3 && gy < P3) c.mip[mip_off(P, 3) + size_t(gy) * P3 + gx] = m3;
    }
    // level 4: tx bit 1 is lane bit 1, ty bit 1 is lane bit 4
    float m4 = fmaxf(m3, __shfl_xor_sync(0xffffffffu, m3, 2));
    m4 = fmaxf(m4, __shfl_xor_sync(0xffffffffu, m4, 16));
    const bool lead4 = ((tx | ty) & 3) == 0;
    if (K >= 4 && lead4) {
        const int P4 = P >> 4, gx = bxi * 4 + (tx >> 2), gy = byi * 4 + (ty >> 2);
        if (gx < P4 && gy < P4) c.mip[mip_off(P, 4) + size_t(gy) * P4 + gx] = m4;
    }
    if (K < 5) return;
    // levels 5 and 6 from the 4 x 4 level-4 entries of the block
    if (lead4) sm[ty >> 2][tx >> 2] = m4;
    __syncthreads();
    if (threadIdx.x < 4) {
        const int x = threadIdx.x & 1, y = threadIdx.x >> 1;
        const float v = fmaxf(fmaxf(sm[2 * y][2 * x], sm[2 * y][2 * x + 1]),
                              fmaxf(sm[2 * y + 1][2 * x], sm[2 * y + 1][2 * x + 1]));
        const int P5 = P >> 5, gx = bxi * 2 + x, gy = byi * 2 + y;
        if (gx < P5 && gy < P5) c.mip[mip_off(P, 5) + size_t(gy) * P5 + gx] = v;
        sm[4 + y][x] = v;
    }
    __syncthreads();
    if (K >= 6 && threadIdx.x == 0) {
        const float v = fmaxf(fmaxf(sm[4][0], sm[4][1]), fmaxf(sm[5][0], sm[5][1]));
        const int P6 = P >> 6;
        if (bxi < P6 && byi < P6) c.mip[mip_off(P, 6) + size_t(byi) * P6 + bxi] = v;
    }
    __syncthreads();
}

// Five CTAs per SM (at most 51 registers) measured fastest: 0.0284 ms per DEM
// frame against 0.0310 ms at six and four.  The two-surface form keeps four
// (64 registers; at 51 it spills).
template <bool TWO>
__global__ void __launch_bounds__(256, TWO ? 4 : 5) k_mip_lo(const __grid_constant__ MipParams p) {
    wait_for_predecessor();
    __shared__ float sm[16][17];
    mip_lo_block<false, TWO>(p.cas[blockIdx.z], blockIdx.x, blockIdx.y, sm);
}

template <bool COH>
__device__ __forceinline__ void mip_hi_levels(const MipCascade& c, float* s0, float* s1) {
    const int P = c.P, K = c.K;
    if (K < 7) return;
    const int n6 = P >> 6, n7 = P >> 7;
    const float* l6 = c.mip + mip_off(P, 6);
    for (int e = threadIdx.x; e < n7 * n7; e += blockDim.x) {
        const int x = e % n7, y = e / n7;
        const float v = fmaxf(fmaxf(ldc<COH>(l6 + size_t(2 * y) * n6 + 2 * x), ldc<COH>(l6 + size_t(2 * y) * n6 + 2 * x + 1)),
                              fmaxf(ldc<COH>(l6 + size_t(2 * y + 1) * n6 + 2 * x),
                                    ldc<COH>(l6 + size_t(2 * y + 1) * n6 + 2 * x + 1)));
        s0[e] = v;
        c.mip[mip_off(P, 7) + e] = v;
    }
    __syncthreads();
    float* cur = s0;
    float* nxt = s1;
    int n = n7;
    for (int k = 8; k <= K; ++k) {
        const int m = n >> 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int x = e % m, y = e / m;
            const float v = fmaxf(fmaxf(cur[(2 * y) * n + 2 * x], cur[(2 * y) * n + 2 * x + 1]),
                                  fmaxf(cur[(2 * y + 1) * n + 2 * x], cur[(2 * y + 1) * n + 2 * x + 1]));
            nxt[e] = v;
            c.mip[mip_off(P, k) + e] = v;
        }
        __syncthreads();
        float* tmp = cur;
        cur = nxt;
        nxt = tmp;
        n = m;
    }
}

__global__ void __launch_bounds__(1024) k_mip_hi(const __grid_constant__ MipParams p) {
    wait_for_predecessor();
    __shared__ float sm[2][4096];
    mip_hi_levels<false>(p.cas[blockIdx.x], sm[0], sm[1]);
}

int launch_maxmip(const MipParams& p, void* stream) {
    if (p.C == 0) return cudaSuccess;
    dim3 grid((p.max_P + 63) / 64, (p.max_P + 63) / 64, p.C);
    cudaError_t e = p.two ? launch_dependent(k_mip_lo<true>, grid, dim3(256), cudaStream_t(stream), p)
                          : launch_dependent(k_mip_lo<false>, grid, dim3(256), cudaStream_t(stream), p);
    if (e != cudaSuccess) return e;
    if (p.max_K >= 7) {
        e = launch_dependent(k_mip_hi, dim3(p.C), dim3(1024), cudaStream_t(stream), p);
    }
    return e;
}

// ---------------------------------------------------------------------------
// Ray casting (Section 5).  One thread per pixel; rays are traced through the
// cascades nearest first.  Within a cascade the max mipmap is traversed top
// down (Tevs et al.): a node whose maximum lies below the ray over the node's
// extent is skipped whole, otherwise refined; single patches are intersected
// exactly (first root of the quadratic bilinear(x(t), y(t)) - z(t)).  The
// current level-0 patch is tracked in integers, so rounding can never move
// the walk backwards; after a step the walk climbs one level when it has left
// its parent node.  The segment above the cascade's global maximum (the top
// mip entry) is skipped before the walk starts, and the walk starts at level
// kRayStartLevel (64 x 64 patches) rather than at the single top node: on the
// flight-path views this removes about a fifth of the node visits (the
// descent through the top levels) and cannot change the first hit, since the
// walk still climbs to any level above where it may skip.
//
// Per-step arithmetic is kept small: exit times are fma(boundary, 1/d, -e/d)
// (both axes in one packed FP32x2 FMA, which rounds each as fmaf does)
// with 1/d = 0, -e/d = +inf for an axis-parallel ray (no branch), integer
// node boundaries become floats by one exact conversion (I2F, on the lightly
// used conversion pipe), level offsets come from shared memory, and all
// divisions happen once per ray.
// Screen coordinates are one fma per axis with host-computed scales.  The
// per-ray reciprocals of the direction and the divisions and square root of
// the patch root use the hardware approximations (rcp.approx, div.approx,
// sqrt.approx: a few ulp): the walk only needs its exit times to be
// consistent with one another, which they are whatever 1/d is, and a root
// error of a few ulp of t is far inside the ray tolerance.  The reciprocal
// used to clip the ray at the cascade maximum stays correctly rounded.
// Sums that carry a tolerance are written with __fadd_rn (and the blend depth
// with __fmul_rn / __fsub_rn) so that no copy of this code is contracted into
// an FMA differently from another: per-view and batched launches then agree
// bit for bit.

constexpr int kRayStartLevel = 6;
constexpr int kTopSlot = kMaxLevels - 1;  // level offsets need columns 0..K <= 13 (side <= 8192)
static_assert(kMaxCascadeSize <= 8192, "a larger side needs more mip levels than the top slot leaves");

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
struct Ray {
    float eu, ev, ez;  // origin in patch units (u, v) and metres (z)
    float du, dv, dz;  // per metre of t
};

// CHECK: the patch may have an undefined (-inf) corner, then it does not exist.
template <bool COH, bool CHECK = false>
__device__ __forceinline__ bool patch_hit(const float* __restrict__ tex, int N, int ci, int cj,
                                          const Ray& r, float t0, float t1, float& t_hit) {
    const float* p = tex + size_t(cj) * N + ci;
    const float h00 = ldc<COH>(p), h10 = ldc<COH>(p + 1), h01 = ldc<COH>(p + N), h11 = ldc<COH>(p + N + 1);
    if (CHECK && !(fminf(fminf(h00, h10), fminf(h01, h11)) > -INFINITY)) return false;
    const float a0 = fmaf(t0, r.du, r.eu) - float(ci);
    const float b0 = fmaf(t0, r.dv, r.ev) - float(cj);
    const float z0 = fmaf(t0, r.dz, r.ez);
    const float e = h10 - h00, g = h01 - h00, q = (h00 - h10) - (h01 - h11);
    const float C = fmaf(fmaf(q, a0, g), b0, fmaf(e, a0, h00)) - z0;
    if (C >= 0.f) {
        t_hit = t0;
        return true;
    }
    const float B = fmaf(e, r.du, fmaf(g, r.dv, q * fmaf(a0, r.dv, b0 * r.du))) - r.dz;
    const float A = q * r.du * r.dv;
    const float dt = t1 - t0;
    const float slack = 4.f * 1.1920929e-7f * fabsf(t1);  // closes cracks between patches
    float tau = INFINITY;
    if (A == 0.f) {
        if (B != 0.f) {
            const float x = __fdividef(-C, B);
            if (x >= -slack && x <= __fadd_rn(dt, slack)) tau = x;
        }
    } else {
        const float disc = fmaf(B, B, -4.f * A * C);
        if (disc >= 0.f) {
            const float s = sqrt_approx(disc);
            const float qq = -0.5f * (B + copysignf(s, B));
            const float x1 = __fdividef(qq, A), x2 = (qq != 0.f) ? __fdividef(C, qq) : x1;
            const float hi = __fadd_rn(dt, slack);
            if (x1 >= -slack && x1 <= hi) tau = x1;
            if (x2 >= -slack && x2 <= hi) tau = fminf(tau, x2);
        }
    }
    if (tau == INFINITY) return false;
    t_hit = t0 + fminf(fmaxf(tau, 0.f), dt);
    return true;
}

// Per-ray quantities that do not depend on the cascade.
struct RayDir {
    float dx, dy, dz;
    float rdx, rdy, rdz;  // reciprocals, 0 for a zero component
    float ks, rks;        // projected-depth rate and its reciprocal
    float tmin, tmax;
};

// First hit inside cascade c on [ta, tb].  With the water layer (UNION) the
// mipmap bounds both surfaces and each patch reached is tested against the
// terrain and, where its four corners are wet, the water surface: the first
// patch with any root holds the first hit of either surface, the nearer root
// of the two (the water surface on a tie; on_water says which).
// SIGNS (bit 0: du > 0, bit 1: dv > 0, bit 2: dz < 0) is constant per ray
// and nearly always per warp: the walk is compiled for each combination.  A
// zero component takes the non-positive branch, which leaves the walk as it
// would be: the exit time along it is infinite, and the clamp of the other
// coordinate returns the current cell.
template <bool COUNT, bool COH, bool UNION, int SIGNS, bool COARSE, bool JUMP = false>
__device__ __forceinline__ bool trace_cascade(const RayCascade& c, const int* __restrict__ off, const RayDir& d,
                                              float ez, float ta, float tb, float& t_hit, bool& on_water,
                                              DevStatus* status, uint32_t pixel, unsigned& visits, unsigned& tests) {
    const int N = c.N, P = c.P, K = c.K;
    const float* __restrict__ mip = c.mip;
    const float* __restrict__ tex = c.tex;
    const float top = __int_as_float(off[kTopSlot]);
    if (!(top > -INFINITY)) return false;  // nothing visible in this cascade
    Ray r;
    r.eu = c.eu;
    r.ev = c.ev;
    r.ez = ez;
    r.du = d.dx * c.inv_h;
    r.dv = d.dy * c.inv_h;
    r.dz = d.dz;
    // skip the part of the segment above the cascade's global maximum
    if (fmaf(ta, r.dz, ez) > top) {
        if (!(r.dz < 0.f)) return false;
        const float tz = (top - ez) * d.rdz;
        if (tz > tb) return false;
        ta = fmaxf(ta, tz);
    }
    const float idu = d.rdx * c.h, idv = d.rdy * c.h;
    const float ou = d.dx != 0.f ? -r.eu * idu : INFINITY;
    const float ov = d.dy != 0.f ? -r.ev * idv : INFINITY;
    const float2 iduv = make_float2(idu, idv), ouv = make_float2(ou, ov);
    constexpr int bu = SIGNS & 1, bv = (SIGNS >> 1) & 1;
    constexpr bool zneg = (SIGNS >> 2) & 1;
    const float slack = 2e-6f * fabsf(top);
    int ci = min(max(int(floorf(fmaf(ta, r.du, r.eu))), 0), N - 2);
    int cj = min(max(int(floorf(fmaf(ta, r.dv, r.ev))), 0), N - 2);
    const int L = COARSE ? c.stop_level : 0;  // coarse-level stop: no node below this level is visited
    int k = max(min(K, kRayStartLevel), L);
    float t = ta;
    const int budget = c.budget;
    for (int it = 0; it < budget; ++it) {
        const int ni = ci >> k, nj = cj >> k;
        const float2 txy = __ffma2_rn(make_float2(__int2float_rn((ni + bu) << k), __int2float_rn((nj + bv) << k)),
                                      iduv, ouv);
        const float tx = txy.x, ty = txy.y;
        const float te = fmaxf(fminf(fminf(tx, ty), tb), t);
        const float zmin = fmaf(zneg ? te : t, r.dz, ez);
        const float mx = ldc<COH>(mip + off[k] + nj * (P >> k) + ni);
        if (COUNT) ++visits;
        if (zmin <= __fadd_rn(mx, slack)) {
            if (k > L) {
                --k;
                continue;
            }
            if (COARSE && k > 0) {  // coarse-level stop: the ray meets this node's box top
                const float z0 = fmaf(t, r.dz, ez);
                t_hit = (z0 <= mx || !zneg) ? t : fminf(fmaf(mx - z0, d.rdz, t), te);
                on_water = false;
                return true;
            }
            if (ci <= N - 2 && cj <= N - 2) {
                if (COUNT) ++tests;
                float th;
                const bool ht = patch_hit<COH>(tex, N, ci, cj, r, t, te, th);
                if (UNION) {
                    float tw;
                    if (patch_hit<COH, true>(c.wtex, N, ci, cj, r, t, te, tw) && (!ht || tw <= th)) {
                        t_hit = tw;
                        on_water = true;
                        return true;
                    }
                }
                if (ht) {
                    t_hit = th;
                    on_water = false;
                    return true;
                }
            }
        }
        if (te >= tb) return false;
        int nci, ncj;
        if (tx <= ty) {
            nci = bu ? (ni + 1) << k : (ni << k) - 1;
            ncj = cj;
            if (k > 0) {
                int c2 = __float2int_rd(fmaf(te, r.dv, r.ev));
                c2 = bv ? max(c2, cj) : min(c2, cj);
                ncj = min(max(c2, nj << k), ((nj + 1) << k) - 1);
            }
        } else {
            ncj = bv ? (nj + 1) << k : (nj << k) - 1;
            nci = ci;
            if (k > 0) {
                int c2 = __float2int_rd(fmaf(te, r.du, r.eu));
                c2 = bu ? max(c2, ci) : min(c2, ci);
                nci = min(max(c2, ni << k), ((ni + 1) << k) - 1);
            }
        }
        if (unsigned(nci) >= unsigned(P) || unsigned(ncj) >= unsigned(P)) return false;
        const int diff = (nci ^ ci) | (ncj ^ cj);
        ci = nci;
        cj = ncj;
        t = te;
        if (JUMP) {  // climb to the coarsest node entered: the highest bit in which the patches differ
            if ((diff >> (k + 1)) != 0) k = min(31 - __clz(diff), K);
        } else if (k < K && (diff >> (k + 1)) != 0) {
            ++k;
        }
    }
    report(status, kStatusTimeout, pixel);
    return false;
}

// t-interval of the ray inside cascade c: projected depth in [near, far_ext],
// texel region u, v in [0, N-1], camera clip range [tmin, tmax].
__device__ __forceinline__ bool cascade_interval(const RayCascade& c, const RayDir& d, float& ta,
                                                 float& tb) {
    float lo = d.tmin, hi = d.tmax;
    if (d.ks > 0.f) {
        lo = fmaxf(lo, c.near_d * d.rks);
        hi = fminf(hi, c.far_ext * d.rks);
    } else if (d.ks < 0.f) {
        lo = fmaxf(lo, c.far_ext * d.rks);
        hi = fminf(hi, c.near_d * d.rks);
    } else if (!(c.near_d <= 0.f && 0.f <= c.far_ext)) {
        return false;
    }
    const float top = float(c.N - 1);
    if (d.dx != 0.f) {
        const float idu = d.rdx * c.h;
        const float t0 = (0.f - c.eu) * idu, t1 = (top - c.eu) * idu;
        lo = fmaxf(lo, fminf(t0, t1));
        hi = fminf(hi, fmaxf(t0, t1));
    } else if (c.eu < 0.f || c.eu > top) {
        return false;
    }
    if (d.dy != 0.f) {
        const float idv = d.rdy * c.h;
        const float t0 = (0.f - c.ev) * idv, t1 = (top - c.ev) * idv;
        lo = fmaxf(lo, fminf(t0, t1));
        hi = fminf(hi, fmaxf(t0, t1));
    } else if (c.ev < 0.f || c.ev > top) {
        return false;
    }
    ta = lo;
    tb = hi;
    return lo <= hi;
}

// Through the cascades, nearest first, blended in the overlaps (reading of
// Section 5: the blend runs linearly in projected depth across the overlap
// band of cascades c and c+1 when both are hit); 0x80 marks a first-hit
// cascade whose hit is on the water surface.
template <bool COUNT, bool COH, bool UNION, int SIGNS, bool COARSE, bool JUMP = false>
__device__ __forceinline__ void cast_cascades(const RayParams& p, const int (*s_off)[kMaxLevels], const RayDir& d,
                                              DevStatus* status, uint32_t pix, unsigned& visits, unsigned& tests,
                                              float& t, int& hit) {
    hit = 0;
    t = __int_as_float(0x7fc00000);
    for (int c = 0; c < p.C && !hit; ++c) {
        const RayCascade& cc = p.cas[c];
        float ta, tb, tc;
        bool wet = false;
        if (!cascade_interval(cc, d, ta, tb)) continue;
        if (!trace_cascade<COUNT, COH, UNION, SIGNS, COARSE, JUMP>(cc, s_off[c], d, p.ez, ta, tb, tc, wet, status, pix,
                                                                  visits, tests))
            continue;
        hit = (1 + c) | (wet ? 0x80 : 0);
        t = tc;
        const float s = __fmul_rn(tc, d.ks);
        if (c + 1 < p.C) {
            const RayCascade& cn = p.cas[c + 1];
            if (s >= cn.near_d && cc.far_ext > cn.near_d) {
                float ta2, tb2, t2;
                bool wet2 = false;
                if (cascade_interval(cn, d, ta2, tb2) &&
                    trace_cascade<COUNT, COH, UNION, SIGNS, COARSE, JUMP>(cn, s_off[c + 1], d, p.ez, ta2, tb2, t2, wet2,
                                                                       status, pix, visits, tests)) {
                    const float al = fminf(fmaxf(__fsub_rn(s, cn.near_d) / (cc.far_ext - cn.near_d), 0.f), 1.f);
                    t = fmaf(al, t2 - tc, tc);
                }
            }
        }
    }
}

// First hit of the ray through pixel (x, y), which must lie in the image.
template <bool COUNT, bool COH, bool WATER = false, bool COARSE = false, bool JUMP = false>
__device__ __forceinline__ void trace_pixel(const RayParams& p, const int (*s_off)[kMaxLevels], DevStatus* status,
                                            int x, int y, unsigned& visits, unsigned& tests, float& t, int& hit) {
    const float sx = fmaf(float(x), p.px_a, p.px_b);
    const float sy = fmaf(float(y), p.py_a, p.py_b);
    float dx = fmaf(sy, p.U[0], fmaf(sx, p.R[0], p.F[0]));
    float dy = fmaf(sy, p.U[1], fmaf(sx, p.R[1], p.F[1]));
    float dz = fmaf(sy, p.U[2], fmaf(sx, p.R[2], p.F[2]));
    const float il = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    RayDir d;
    d.dx = dx * il;
    d.dy = dy * il;
    d.dz = dz * il;
    d.rdx = d.dx != 0.f ? rcp_approx(d.dx) : 0.f;
    d.rdy = d.dy != 0.f ? rcp_approx(d.dy) : 0.f;
    d.rdz = d.dz != 0.f ? __frcp_rn(d.dz) : 0.f;
    const float rfd = rcp_approx(fmaf(d.dx, p.F[0], fmaf(d.dy, p.F[1], d.dz * p.F[2])));
    d.tmin = p.znear * rfd;
    d.tmax = p.zfar * rfd;
    d.ks = fmaf(d.dx, p.dir2x, d.dy * p.dir2y);
    d.rks = d.ks != 0.f ? rcp_approx(d.ks) : 0.f;
    const uint32_t pix = uint32_t(y) * uint32_t(p.W) + uint32_t(x);
    switch ((d.dx > 0.f ? 1 : 0) | (d.dy > 0.f ? 2 : 0) | (d.dz < 0.f ? 4 : 0)) {
    case 0: cast_cascades<COUNT, COH, WATER, 0, COARSE, JUMP>(p, s_off, d, status, pix, visits, tests, t, hit); break;
    case 1: cast_cascades<COUNT, COH, WATER, 1, COARSE, JUMP>(p, s_off, d, status, pix, visits, tests, t, hit); break;
    case 2: cast_cascades<COUNT, COH, WATER, 2, COARSE, JUMP>(p, s_off, d, status, pix, visits, tests, t, hit); break;
    case 3: cast_cascades<COUNT, COH, WATER, 3, COARSE, JUMP>(p, s_off, d, status, pix, visits, tests, t, hit); break;
    case 4: cast_cascades<COUNT, COH, WATER, 4, COARSE, JUMP>(p, s_off, d, status, pix, visits, tests, t, hit); break;
    case 5: cast_cascades<COUNT, COH, WATER, 5, COARSE, JUMP>(p, s_off, d, status, pix, visits, tests, t, hit); break;
    case 6: cast_cascades<COUNT, COH, WATER, 6, COARSE, JUMP>(p, s_off, d, status, pix, visits, tests, t, hit); break;
    default: cast_cascades<COUNT, COH, WATER, 7, COARSE, JUMP>(p, s_off, d, status, pix, visits, tests, t, hit); break;
    }
}

template <bool COUNT, bool COH, bool WATER = false, bool COARSE = false, bool JUMP = false>
__device__ __forceinline__ void raycast_pixel(const RayParams& p, const int (*s_off)[kMaxLevels], DevStatus* status,
                                              int x, int y, unsigned& visits, unsigned& tests) {
    if (x >= p.W || y >= p.H) return;
    float t;
    int hit;
    trace_pixel<COUNT, COH, WATER, COARSE, JUMP>(p, s_off, status, x, y, visits, tests, t, hit);
    if (!COUNT) {
        const size_t pix = size_t(y) * p.W + x;
        p.t_out[pix] = t;
        p.hit_out[pix] = uint8_t(hit);
    }
}

// Per cascade the mip level offsets and, in the last column, the top entry
// (the cascade's maximum, read by every ray before its walk).
template <bool COH>
__device__ __forceinline__ void load_level_offsets(const RayParams& p, int (*s_off)[kMaxLevels], int tid, int nthreads) {
    for (int e = tid; e < p.C * kMaxLevels; e += nthreads) {
        const int c = e / kMaxLevels, L = e % kMaxLevels;
        const RayCascade& rc = p.cas[c];
        s_off[c][L] = L == kTopSlot ? __float_as_int(ldc<COH>(rc.mip + rc.lvl_off[rc.K])) : rc.lvl_off[L];
    }
}

// 9 CTAs of 128 threads per SM leave the walk its 56 registers without spills
// (8 and 64 registers for the walk over both surfaces).  A CTA covers 16 x 8
// pixels, each warp a 4 x 8 column of them: neighbouring rays in a compact
// patch take more of the same steps than in a 16 x 2 strip (2 % faster);
// 4 x 8 columns measured 1 % faster than 8 x 4 patches.  With STAGE the
// results go out through shared memory in image rows (a warp stores two
// 64-byte rows of t, one warp the hit bytes four at a time), not in the
// walk's columns: for outputs in pinned host memory, which the GPU writes
// over the host link, the columns' 16-byte rows of t and 4-byte rows of hit
// made the ray cast 1.7 times slower (0.334 against 0.193 ms).  In device
// memory the direct stores are 2 % faster (0.187 against 0.191 ms).
template <bool COUNT, bool WATER, bool COARSE, bool JUMP = false, bool STAGE = true>
__global__ void __launch_bounds__(128, WATER ? 8 : 9) k_raycast(const __grid_constant__ RayParams p, DevStatus* status) {
    wait_for_predecessor();
    __shared__ int s_off[HF_MAX_CASCADES][kMaxLevels];
    __shared__ float s_t[8][16];
    __shared__ uint32_t s_hit[8][4];  // 16 hit bytes per row
    const int t = threadIdx.y * 16 + threadIdx.x, warp = t >> 5, lane = t & 31;
    load_level_offsets<false>(p, s_off, t, 128);
    __syncthreads();
    unsigned visits = 0, tests = 0;
    const int x0 = blockIdx.x * 16, y0 = blockIdx.y * 8;
    const int cx = warp * 4 + (lane & 3), cy = lane >> 2;
    float tr = 0.f;
    int hit = 0;
    if (x0 + cx < p.W && y0 + cy < p.H)
        trace_pixel<COUNT, false, WATER, COARSE, JUMP>(p, s_off, status, x0 + cx, y0 + cy, visits, tests, tr, hit);
    if (COUNT) {
        visits = __reduce_add_sync(0xffffffffu, visits);
        tests = __reduce_add_sync(0xffffffffu, tests);
        if (lane == 0) {
            atomicAdd(&status->ray_counters[0], (unsigned long long)visits);
            atomicAdd(&status->ray_counters[1], (unsigned long long)tests);
        }
    } else if (!STAGE) {
        if (x0 + cx < p.W && y0 + cy < p.H) {
            const size_t o = size_t(y0 + cy) * p.W + x0 + cx;
            p.t_out[o] = tr;
            p.hit_out[o] = uint8_t(hit);
        }
    } else {
        s_t[cy][cx] = tr;
        reinterpret_cast<uint8_t*>(s_hit[cy])[cx] = uint8_t(hit);
        __syncthreads();
        const int r = t >> 4, c = t & 15;
        if (x0 + c < p.W && y0 + r < p.H) p.t_out[size_t(y0 + r) * p.W + x0 + c] = s_t[r][c];
        if (t < 32) {
            const int y = y0 + (t >> 2), x = x0 + (t & 3) * 4;
            if (y < p.H && x < p.W) {
                uint8_t* dst = p.hit_out + size_t(y) * p.W + x;
                const uint32_t v = s_hit[t >> 2][t & 3];
                if (x + 3 < p.W && (reinterpret_cast<uintptr_t>(dst) & 3u) == 0) {
                    *reinterpret_cast<uint32_t*>(dst) = v;
                } else {
                    for (int k = 0; k < 4 && x + k < p.W; ++k) dst[k] = uint8_t(v >> (8 * k));
                }
            }
        }
    }
}

template <bool COUNT>
int launch_raycast_t(const RayParams& p, DevStatus* status, void* stream) {
    dim3 grid((p.W + 15) / 16, (p.H + 7) / 8);
    if (p.water)
        return launch_dependent(k_raycast<COUNT, true, false>, grid, dim3(16, 8), cudaStream_t(stream), p, status);
    if (p.coarse)
        return launch_dependent(k_raycast<COUNT, false, true>, grid, dim3(16, 8), cudaStream_t(stream), p, status);
    if (p.jump)
        return launch_dependent(k_raycast<COUNT, false, false, true>, grid, dim3(16, 8), cudaStream_t(stream), p, status);
    if constexpr (!COUNT) {
        if (!p.host_out)
            return launch_dependent(k_raycast<false, false, false, false, false>, grid, dim3(16, 8),
                                    cudaStream_t(stream), p, status);
    }
    return launch_dependent(k_raycast<COUNT, false, false>, grid, dim3(16, 8), cudaStream_t(stream), p, status);
}

int launch_raycast(const RayParams& p, DevStatus* status, void* stream) {
    return launch_raycast_t<false>(p, status, stream);
}

int launch_raycast_count(const RayParams& p, DevStatus* status, void* stream) {
    return launch_raycast_t<true>(p, status, stream);
}

// ---------------------------------------------------------------------------
// Batched frames: one persistent launch drains an ordered queue of work units
// (all visible-row units, then all discretization tiles, then all level-0..6
// mip blocks, then all mip tops, and optionally all ray tiles).  A unit waits
// only for units earlier in the queue (per-cascade completion counters), and
// units are taken only by running CTAs, so every wait ends; each wait is still
// bounded and reports HF_ERR_TIMEOUT instead of hanging.  Data written in the
// same launch is read through L2 (ld.global.cg).

constexpr int kWaitLimit = 1 << 24;

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void wait_count(const uint32_t* ctr, uint32_t target, DevStatus* status,
                                           uint32_t detail, int limit = kWaitLimit) {
    if (threadIdx.x == 0) {
        int it = 0;
        while (ld_acquire(ctr) < target) {
            if (++it > limit) {
                report(status, kStatusTimeout, detail);
                break;
            }
            __nanosleep(128);
        }
    }
    __syncthreads();
}

// Self-test of the failure path: one CTA waits, at most `limit` polls, on a
// word of the status block that nothing sets.
__global__ void __launch_bounds__(32) k_selftest_wait(DevStatus* status, int limit) {
    wait_count(&status->pad[0], 1u, status, 0xFFFFFFFEu, limit);
}

int launch_selftest_wait(DevStatus* status, int limit, void* stream) {
    cudaError_t e = cudaMemsetAsync(&status->pad[0], 0, sizeof(uint32_t), cudaStream_t(stream));
    if (e != cudaSuccess) return e;
    k_selftest_wait<<<1, 32, 0, cudaStream_t(stream)>>>(status, limit);
    return cudaGetLastError();
}

__device__ __forceinline__ void signal_done(uint32_t* ctr) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(ctr, 1u);
}

__device__ __forceinline__ int find_cascade(const BatchCascade* cas, int n, int phase, int u) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cas[mid].unit_base[phase] <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The same search by the 32 lanes of one warp over the compact array of the
// phase's first units (ascending): each round narrows the range by a factor
// of 32 with one load per lane, so a CTA's preamble costs ~two dependent
// loads instead of ~log2(n) loads at a cascade record's stride.
__device__ __forceinline__ int find_cascade_warp(const int32_t* bases, int n, int u) {
    const int lane = threadIdx.x & 31;
    int lo = 0, len = n;  // the answer lies in [lo, lo + len)
    while (len > 1) {
        const int step = (len + 31) / 32;
        const int k = lo + lane * step;
        const bool le = k < lo + len && __ldg(bases + k) <= u;
        const unsigned m = __ballot_sync(0xffffffffu, le);
        const int last = 31 - __clz(m);  // bases[lo] <= u always holds, so m != 0
        lo += last * step;
        len = min(step, n - lo);
    }
    return lo;
}

__device__ __forceinline__ int find_item(const BatchItem* items, int n, int u) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].ray_unit_base <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

union BatchShared {
    float mlo[16][17];
    float mhi[2][4096];
    int off[HF_MAX_CASCADES][kMaxLevels];
};

// Word-wise copy of a descriptor by the whole CTA (the structs are plain data
// of whole 4-byte words).
template <class T>
__device__ __forceinline__ void cta_copy(T* dst, const T* src) {
    static_assert(sizeof(T) % 4 == 0, "descriptor size must be whole words");
    const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    for (int w = threadIdx.x; w < int(sizeof(T) / 4); w += blockDim.x) d[w] = s[w];
}

// The lookup tables a texel needs: without `full`, only the fields after the
// bucket bitmaps (a walk that finds its list through a cell map never reads
// the bitmaps; the reduced-precision walk always needs their max_level).
__device__ __forceinline__ void cta_copy_lookup(LookupTables* dst, const LookupTables* src, bool full) {
    constexpr int from = int(offsetof(LookupTables, bucket_level)) / 4;
    static_assert(offsetof(LookupTables, bucket_level) % 4 == 0, "word-aligned tail");
    const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    const int w0 = full ? 0 : from;
    for (int w = w0 + threadIdx.x; w < int(sizeof(LookupTables) / 4); w += blockDim.x) d[w] = s[w];
}

// The ray parameters of an item: the fixed fields, its C cascades and the
// output pointers (the unused cascade slots are not copied).
__device__ __forceinline__ void cta_copy_ray(RayParams* dst, const RayParams* src, int C) {
    static_assert(offsetof(RayParams, cas) % 4 == 0 && sizeof(RayCascade) % 4 == 0 &&
                  offsetof(RayParams, t_out) % 4 == 0, "word-aligned parts");
    const int body = int(offsetof(RayParams, cas) + size_t(C) * sizeof(RayCascade)) / 4;
    const int tail = int(offsetof(RayParams, t_out)) / 4;
    const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    for (int w = threadIdx.x; w < int(sizeof(RayParams) / 4); w += blockDim.x)
        if (w < body || w >= tail) d[w] = s[w];
}

template <bool COH>
__device__ __forceinline__ void batch_ray_unit(const BatchHeader* h, const BatchItem* items, const BatchCascade* cas,
                                               const uint32_t* done, int u, int (*off)[kMaxLevels]) {
    // every warp finds the item itself (no barrier needed for it)
    const int it = find_cascade_warp(reinterpret_cast<const int32_t*>(reinterpret_cast<const uint8_t*>(h) +
                                                                      h->item_bases_off),
                                     h->n_items, u - h->phase_base[kPhaseRays]);
    const BatchItem& I = items[it];
    if (COH) {
        for (int c = 0; c < I.n_cascades; ++c)
            wait_count(done + 4 * (I.first_cascade + c) + kPhaseMipHi, 1u, I.status, uint32_t(u));
    }
    // the item's ray parameters, staged once per unit: the walk then reads
    // them from shared memory rather than through the descriptor buffer
    __shared__ RayParams s_ray;
    __syncthreads();  // the previous unit of this CTA is done with s_ray and off
    cta_copy_ray(&s_ray, &I.ray, I.n_cascades);
    __syncthreads();
    load_level_offsets<COH>(s_ray, off, threadIdx.x, blockDim.x);
    __syncthreads();
    const int local = u - h->phase_base[kPhaseRays] - I.ray_unit_base;
    const int tw = h->ray_tile_w, th = h->ray_tile_h;
    const int x = (local % I.ray_tiles_x) * tw + int(threadIdx.x) % tw;
    const int y = (local / I.ray_tiles_x) * th + int(threadIdx.x) / tw;
    unsigned visits = 0, tests = 0;
    if (s_ray.coarse)
        raycast_pixel<false, COH, false, true>(s_ray, off, I.status, x, y, visits, tests);
    else
        raycast_pixel<false, COH>(s_ray, off, I.status, x, y, visits, tests);
}

// Units are taken in chunks of kChunk; completions of consecutive units of
// the same cascade and phase are released with one counter increment, and
// pending releases are always flushed before the CTA waits on anything, so a
// CTA never waits on its own unreleased work.
constexpr int kChunk = 4;

template <bool RAYS_INSIDE>
__global__ void __launch_bounds__(256, RAYS_INSIDE ? 3 : 5) k_batch(const uint8_t* __restrict__ buf) {
    const BatchHeader* h = reinterpret_cast<const BatchHeader*>(buf);
    const BatchItem* items = reinterpret_cast<const BatchItem*>(buf + h->items_off);
    const BatchCascade* cas = reinterpret_cast<const BatchCascade*>(buf + h->cascades_off);
    uint32_t* done = reinterpret_cast<uint32_t*>(const_cast<uint8_t*>(buf) + h->counters_off);
    uint32_t* queue = done + 4 * h->n_cascades;
    __shared__ BatchShared sm;
    __shared__ LookupTables s_lt;
    __shared__ DiscCascade s_disc;
    __shared__ int s_base, s_lt_item, s_disc_k;
    if (threadIdx.x == 0) {
        s_lt_item = -1;
        s_disc_k = -1;
    }
    const int n_cas = h->n_cascades;
    const int end = RAYS_INSIDE ? h->phase_base[kPhases] : h->phase_base[kPhaseRays];
    const int ray_base = h->phase_base[kPhaseRays];
    const bool warp16 = (h->flags & kBatchWarp16x2) != 0;
    int kc = 0, kc_phase = -1;          // cached cascade of the last unit (uniform)
    int run_k = -1, run_phase = -1;     // pending completions (uniform)
    uint32_t run_n = 0;
    auto flush = [&]() {
        if (run_n) {
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(done + 4 * run_k + run_phase, run_n);
            run_n = 0;
        }
    };
    for (;;) {
        if (threadIdx.x == 0) s_base = int(atomicAdd(queue, unsigned(kChunk)));
        __syncthreads();
        const int base = s_base;
        __syncthreads();
        if (base >= end) break;
        for (int u = base; u < base + kChunk && u < end; ++u) {
            if (RAYS_INSIDE && u >= ray_base) {
                flush();
                batch_ray_unit<true>(h, items, cas, done, u, sm.off);
                __syncthreads();
                continue;
            }
            int phase = 0;
            while (phase < kPhaseMipHi && u >= h->phase_base[phase + 1]) ++phase;
            if (phase != kc_phase) {
                kc = find_cascade(cas, n_cas, phase, u);
                kc_phase = phase;
            } else {
                while (kc + 1 < n_cas && cas[kc + 1].unit_base[phase] <= u) ++kc;
            }
            const int k = kc;
            const BatchCascade& C = cas[k];
            if (run_n && (k != run_k || phase != run_phase)) flush();
            if (phase > kPhaseRows) {
                flush();
                const uint32_t need = uint32_t(C.n_units[phase - 1]);
                if (threadIdx.x == 0) {
                    int it = 0;
                    while (ld_acquire(done + 4 * k + (phase - 1)) < need) {
                        if (++it > kWaitLimit) {
                            report(items[C.item].status, kStatusTimeout, uint32_t(u));
                            break;
                        }
                        __nanosleep(128);
                    }
                }
                __syncthreads();
            }
            const int local = u - C.unit_base[phase];
            if (phase == kPhaseRows) {
                const BatchItem& I = items[C.item];
                const int t = local * 256 + threadIdx.x;
                if (t < C.prep.N) prep_row(C.prep, I.dom_w, I.dom_h, I.eps_frac, t);
            } else if (phase == kPhaseTexels) {
                if (s_lt_item != C.item || s_disc_k != k) {
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        if (s_lt_item != C.item) s_lt = items[C.item].lt;
                        s_disc = C.disc;
                        s_lt_item = C.item;
                        s_disc_k = k;
                    }
                    __syncthreads();
                }
                const BatchItem& I = items[C.item];
                int di, dj;
                if (warp16) {
                    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
                    di = (warp & 1) * 16 + (lane & 15);
                    dj = (warp >> 1) * 2 + (lane >> 4);
                } else {
                    tile_texel(threadIdx.x, di, dj);
                }
                const int i = (local % C.tiles_x) * 32 + di, j = (local / C.tiles_x) * 8 + dj;
                if (I.fp32c)
                    discretize_texel_f32c<true, HF_RBF_GAUSSIAN>(s_disc, I.K, s_lt, I.cv, I.status, i, j);
                else if (I.precision == HF_PREC_FP32)
                    discretize_texel<true>(s_disc, I.K, s_lt, I.lv, I.status, i, j);
                else if (I.precision == HF_PREC_FP16)
                    discretize_texel_mixed<F16Ops, true>(s_disc, I.K, s_lt, I.cv, I.status, i, j);
                else
                    discretize_texel_mixed<BF16Ops, true>(s_disc, I.K, s_lt, I.cv, I.status, i, j);
            } else if (phase == kPhaseMipLo) {
                mip_lo_block<true>(C.mip, local % C.mip_blocks_x, local / C.mip_blocks_x, sm.mlo);
            } else {
                mip_hi_levels<true>(C.mip, sm.mhi[0], sm.mhi[1]);
            }
            __syncthreads();
            run_k = k;
            run_phase = phase;
            ++run_n;
        }
        flush();
    }
    flush();
}

__global__ void __launch_bounds__(256) k_batch_rays(const uint8_t* __restrict__ buf) {
    wait_for_predecessor();
    const BatchHeader* h = reinterpret_cast<const BatchHeader*>(buf);
    const BatchItem* items = reinterpret_cast<const BatchItem*>(buf + h->items_off);
    const BatchCascade* cas = reinterpret_cast<const BatchCascade*>(buf + h->cascades_off);
    __shared__ int off[HF_MAX_CASCADES][kMaxLevels];
    batch_ray_unit<false>(h, items, cas, nullptr, h->phase_base[kPhaseRays] + int(blockIdx.x), off);
}

int batch_persistent_blocks(int* blocks_plain, int* blocks_rays) {
    int dev = 0, sms = 0, a = 0, b = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_batch<false>, 256, 0);
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch<true>, 256, 0);
    if (e) return e;
    *blocks_plain = sms * a;
    *blocks_rays = sms * b;
    return cudaSuccess;
}

// One launch per phase over all cascades of all items: each CTA finds its
// cascade by binary search over the phase's unit bases; kernel boundaries
// order the phases, so the per-view code paths (and read-only loads) apply.
__global__ void __launch_bounds__(128) k_bat_rows(const uint8_t* __restrict__ buf) {
    wait_for_predecessor();
    const BatchHeader* h = reinterpret_cast<const BatchHeader*>(buf);
    const BatchItem* items = reinterpret_cast<const BatchItem*>(buf + h->items_off);
    const BatchCascade* cas = reinterpret_cast<const BatchCascade*>(buf + h->cascades_off);
    const BatchCascade& C = cas[blockIdx.y];
    const BatchItem& I = items[C.item];
    const int t = blockIdx.x * 128 + threadIdx.x;
    if (t < C.prep.N) prep_row(C.prep, I.dom_w, I.dom_h, I.eps_frac, t);
}

// The CTA's cascade, its item's tables and the tile origin are looked up
// once and staged in shared memory; the texel code then reads them from
// there (uniform across the CTA) instead of through the descriptor buffer.
template <bool MIXED>  // false: every item is FP32 (the reduced-precision code is left out)
__global__ void __launch_bounds__(256, 8) k_bat_texels(const uint8_t* __restrict__ buf) {
    wait_for_predecessor();
    const BatchHeader* h = reinterpret_cast<const BatchHeader*>(buf);
    const BatchItem* items = reinterpret_cast<const BatchItem*>(buf + h->items_off);
    const BatchCascade* cas = reinterpret_cast<const BatchCascade*>(buf + h->cascades_off);
    __shared__ LookupTables s_lt;
    __shared__ DiscCascade s_disc;
    __shared__ ListsView s_lv;
    __shared__ CompactView s_cv;
    __shared__ int s_k, s_i0, s_j0;
    if (threadIdx.x < 32) {  // warp 0 finds the CTA's cascade
        const int u = h->phase_base[kPhaseTexels] + int(blockIdx.x);
        const int32_t* bases = reinterpret_cast<const int32_t*>(buf + h->bases_off) + kPhaseTexels * h->n_cascades;
        const int k = find_cascade_warp(bases, h->n_cascades, u);
        if (threadIdx.x == 0) {
            const int local = u - __ldg(bases + k), tx = cas[k].tiles_x;
            s_k = k;
            s_i0 = (local % tx) * 32;
            s_j0 = (local / tx) * 8;
        }
    }
    __syncthreads();
    const BatchCascade& C = cas[s_k];
    const BatchItem& I = items[C.item];
    // the FP32 walks read the bitmaps only without their cell map
    cta_copy_lookup(&s_lt, &I.lt, MIXED || (I.fp32c ? I.cv.cellmap == nullptr : I.lt.cellmap == nullptr));
    cta_copy(&s_disc, &C.disc);
    cta_copy(&s_lv, &I.lv);
    if (MIXED || I.fp32c) cta_copy(&s_cv, &I.cv);
    const float K = I.K;
    const int precision = I.precision;
    DevStatus* const status = I.status;
    __syncthreads();
    int di, dj;
    if (h->flags & kBatchWarp16x2) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        di = (warp & 1) * 16 + (lane & 15);
        dj = (warp >> 1) * 2 + (lane >> 4);
    } else {
        tile_texel(threadIdx.x, di, dj);
    }
    const int i = s_i0 + di, j = s_j0 + dj;
    if (I.fp32c)
        discretize_texel_f32c<false, HF_RBF_GAUSSIAN>(s_disc, K, s_lt, s_cv, status, i, j);
    else if (!MIXED || precision == HF_PREC_FP32)
        discretize_texel<false>(s_disc, K, s_lt, s_lv, status, i, j);
    else if (precision == HF_PREC_FP16)
        discretize_texel_mixed<F16Ops, false>(s_disc, K, s_lt, s_cv, status, i, j);
    else
        discretize_texel_mixed<BF16Ops, false>(s_disc, K, s_lt, s_cv, status, i, j);
}

__global__ void __launch_bounds__(256) k_bat_miplo(const uint8_t* __restrict__ buf) {
    wait_for_predecessor();
    const BatchHeader* h = reinterpret_cast<const BatchHeader*>(buf);
    const BatchCascade* cas = reinterpret_cast<const BatchCascade*>(buf + h->cascades_off);
    __shared__ float sm[16][17];
    __shared__ MipCascade s_mip;
    __shared__ int s_k, s_bx, s_by;
    if (threadIdx.x < 32) {  // warp 0 finds the CTA's cascade
        const int u = h->phase_base[kPhaseMipLo] + int(blockIdx.x);
        const int32_t* bases = reinterpret_cast<const int32_t*>(buf + h->bases_off) + kPhaseMipLo * h->n_cascades;
        const int k = find_cascade_warp(bases, h->n_cascades, u);
        if (threadIdx.x == 0) {
            const int local = u - __ldg(bases + k), bx = cas[k].mip_blocks_x;
            s_k = k;
            s_bx = local % bx;
            s_by = local / bx;
        }
    }
    __syncthreads();
    cta_copy(&s_mip, &cas[s_k].mip);
    __syncthreads();
    mip_lo_block<false>(s_mip, s_bx, s_by, sm);
}

__global__ void __launch_bounds__(1024) k_bat_miphi(const uint8_t* __restrict__ buf) {
    wait_for_predecessor();
    const BatchHeader* h = reinterpret_cast<const BatchHeader*>(buf);
    const BatchCascade* cas = reinterpret_cast<const BatchCascade*>(buf + h->cascades_off);
    __shared__ float sm[2][4096];
    mip_hi_levels<false>(cas[blockIdx.x].mip, sm[0], sm[1]);
}

int launch_batch(const BatchHeader& h, void* dev_buf, void* stream) {
    cudaStream_t s = cudaStream_t(stream);
    const uint8_t* buf = static_cast<const uint8_t*>(dev_buf);
    const bool persistent = (h.flags & kBatchPersistent) != 0;
    const bool inside = persistent && (h.flags & kBatchRaysInside) != 0;
    cudaError_t e;
    if (persistent) {
        const int units = inside ? h.phase_base[kPhases] : h.phase_base[kPhaseRays];
        const int cap = inside ? h.persistent_blocks_rays : h.persistent_blocks;
        const int chunks = (units + kChunk - 1) / kChunk;
        const int grid = chunks < cap ? chunks : cap;
        if (grid > 0) {
            if (inside) k_batch<true><<<grid, 256, 0, s>>>(buf);
            else k_batch<false><<<grid, 256, 0, s>>>(buf);
            if ((e = cudaGetLastError())) return e;
        }
    } else {
        const int nrow = h.phase_base[kPhaseTexels] - h.phase_base[kPhaseRows];
        const int ntex = h.phase_base[kPhaseMipLo] - h.phase_base[kPhaseTexels];
        const int nmip = h.phase_base[kPhaseMipHi] - h.phase_base[kPhaseMipLo];
        if (nrow > 0 && (e = launch_dependent(k_bat_rows, dim3(2 * h.max_rows_units, h.n_cascades), dim3(128), s, buf)))
            return e;
        if (ntex > 0 && (e = h.mixed ? launch_dependent(k_bat_texels<true>, dim3(ntex), dim3(256), s, buf)
                                     : launch_dependent(k_bat_texels<false>, dim3(ntex), dim3(256), s, buf)))
            return e;
        if (nmip > 0 && (e = launch_dependent(k_bat_miplo, dim3(nmip), dim3(256), s, buf))) return e;
        if ((e = launch_dependent(k_bat_miphi, dim3(h.n_cascades), dim3(1024), s, buf))) return e;
    }
    const int rays = h.phase_base[kPhases] - h.phase_base[kPhaseRays];
    if (!inside && rays > 0) return launch_dependent(k_batch_rays, dim3(rays), dim3(256), s, buf);
    return cudaSuccess;
}

}  // namespace hfi

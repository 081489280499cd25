// Cascade fitting on the host in FP64 (Section 3 of Cornel et al., 2022).
//
// Steps, in the paper's order:
//   1. intersection volume of the view frustum and the heightfield's box,
//   2. its vertices projected onto the ground plane, convex hull,
//   3. depth range [n, f] of the hull along the normalised 2-D view vector,
//   4. split distances (logarithmic, or blended with uniform by lambda),
//   5. per cascade, the hull clipped to its depth band; all far planes but
//      the last are pushed out so adjacent cascades overlap,
//   6. stable texel-aligned fit of the band polygon's bounding box (or, with
//      hf_camera.texel_ladder > 0, the lattice fit that hf_discretize_reuse
//      relies on: spacing from a fixed ladder, origin on the texel lattice).
//
// The frustum/box intersection is built by clipping the faces of each solid
// against the other's half-spaces (Sutherland-Hodgman); the hull is Andrew's
// monotone chain.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hf_internal.h"

namespace hfi {
namespace {

struct V3 {
    double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline V3 unit(V3 a) { return (1.0 / std::sqrt(dot(a, a))) * a; }

struct Plane {  // n . p <= d
    V3 n;
    double d;
};

// Keep the part of a convex polygon with n.p <= d.
std::vector<V3> clip_poly(const std::vector<V3>& in, const Plane& pl) {
    std::vector<V3> out;
    size_t m = in.size();
    for (size_t i = 0; i < m; ++i) {
        const V3& P = in[i];
        const V3& Q = in[(i + 1) % m];
        double sp = dot(pl.n, P) - pl.d, sq = dot(pl.n, Q) - pl.d;
        if (sp <= 0.0) out.push_back(P);
        if ((sp < 0.0 && sq > 0.0) || (sp > 0.0 && sq < 0.0)) out.push_back(P + (sp / (sp - sq)) * (Q - P));
    }
    return out;
}

struct P2 {
    double x, y;
};

// Andrew's monotone chain; counter-clockwise.  The chain pops only on a
// non-left turn, so it is convex for the points as given; afterwards
// near-coincident vertices and vertices within 1e-9 of the line through
// their neighbours are removed.  On a convex chain such a vertex lies between
// its neighbours, so removing it never loses an extreme point, whatever
// rounding noise (e.g. from fused multiply-adds) tilted a straight run.
std::vector<P2> monotone_hull(std::vector<P2> pts) {
    if (pts.size() < 3) return {};
    double scale = 1.0;
    for (const P2& p : pts) scale = std::max(scale, std::max(std::fabs(p.x), std::fabs(p.y)));
    const double same = 1e-9 * scale;
    std::sort(pts.begin(), pts.end(), [](const P2& a, const P2& b) {
        return a.x < b.x || (a.x == b.x && a.y < b.y);
    });
    auto turn = [](const P2& o, const P2& a, const P2& b) {
        return (a.x - o.x) * (b.y - o.y) - (a.y - o.y) * (b.x - o.x);
    };
    std::vector<P2> h(2 * pts.size());
    size_t k = 0;
    for (size_t i = 0; i < pts.size(); ++i) {
        while (k >= 2 && turn(h[k - 2], h[k - 1], pts[i]) <= 0.0) k--;
        h[k++] = pts[i];
    }
    for (size_t i = pts.size() - 1, t = k + 1; i-- > 0;) {
        while (k >= t && turn(h[k - 2], h[k - 1], pts[i]) <= 0.0) k--;
        h[k++] = pts[i];
    }
    h.resize(k > 0 ? k - 1 : 0);
    bool changed = true;
    while (changed && h.size() >= 3) {
        changed = false;
        for (size_t i = 0; i < h.size() && h.size() >= 3; ++i) {
            const P2& a = h[(i + h.size() - 1) % h.size()];
            const P2& m = h[i];
            const P2& b = h[(i + 1) % h.size()];
            const double len = std::hypot(b.x - a.x, b.y - a.y);
            const bool coincident = std::fabs(m.x - a.x) <= same && std::fabs(m.y - a.y) <= same;
            if (coincident || std::fabs(turn(a, m, b)) <= same * len) {
                h.erase(h.begin() + long(i));
                changed = true;
                break;
            }
        }
    }
    if (h.size() < 3) return {};
    double area = 0.0;
    for (size_t i = 0; i < h.size(); ++i) {
        const P2& a = h[i];
        const P2& b = h[(i + 1) % h.size()];
        area += a.x * b.y - b.x * a.y;
    }
    if (0.5 * area <= same * scale) return {};
    return h;
}

// 2-D half-plane clip: keep s(p) = (p - e).dir >= lo (keep_ge) or <= hi.
std::vector<P2> clip_depth(const std::vector<P2>& in, const double* dir, const double* e,
                           double L, bool keep_ge) {
    std::vector<P2> out;
    size_t m = in.size();
    for (size_t i = 0; i < m; ++i) {
        const P2& P = in[i];
        const P2& Q = in[(i + 1) % m];
        double sp = (P.x - e[0]) * dir[0] + (P.y - e[1]) * dir[1] - L;
        double sq = (Q.x - e[0]) * dir[0] + (Q.y - e[1]) * dir[1] - L;
        if (keep_ge) { sp = -sp; sq = -sq; }
        if (sp <= 0.0) out.push_back(P);
        if ((sp < 0.0 && sq > 0.0) || (sp > 0.0 && sq < 0.0)) {
            double t = sp / (sp - sq);
            out.push_back({P.x + t * (Q.x - P.x), P.y + t * (Q.y - P.y)});
        }
    }
    return out;
}

// Ladder of lattice-fit texel spacings: c_min 2^(m/n).
double ladder_texel(double c_min, int64_t m, int n) { return c_min * std::exp2(double(m) / double(n)); }

}  // namespace

int fit_cascades(const hf_camera& cam, const double eye_local[3], const FitDomain& dom,
                 FitResult* out, const int64_t* follow) {
    std::memset(out, 0, sizeof(*out));
    const int C = cam.n_cascades, N = cam.cascade_size;
    // camera basis: forward, up made orthogonal to it, right = forward x up
    V3 F = unit({cam.forward[0], cam.forward[1], cam.forward[2]});
    V3 up = {cam.up[0], cam.up[1], cam.up[2]};
    V3 U = up - dot(up, F) * F;
    if (std::sqrt(dot(U, U)) < 1e-9 * std::sqrt(dot(up, up))) {
        V3 ey = {0.0, 1.0, 0.0};
        U = ey - dot(ey, F) * F;
    }
    U = unit(U);
    V3 R = cross(F, U);
    out->F[0] = F.x; out->F[1] = F.y; out->F[2] = F.z;
    out->U[0] = U.x; out->U[1] = U.y; out->U[2] = U.z;
    out->R[0] = R.x; out->R[1] = R.y; out->R[2] = R.z;
    double gl = std::hypot(F.x, F.y);
    if (gl >= 1e-12) {
        out->dir2[0] = F.x / gl; out->dir2[1] = F.y / gl;
    } else {  // looking straight down: the top of the screen is "ahead"
        gl = std::hypot(U.x, U.y);
        out->dir2[0] = U.x / gl; out->dir2[1] = U.y / gl;
    }

    // 1. frustum AND box, as the union of each solid's faces clipped by the other
    const V3 E = {eye_local[0], eye_local[1], eye_local[2]};
    const double tv = std::tan(0.5 * cam.vfov), th = tv * double(cam.width) / double(cam.height);
    const int sx[4] = {-1, 1, 1, -1}, sy[4] = {-1, -1, 1, 1};
    V3 nc[4], fc[4];
    for (int q = 0; q < 4; ++q) {
        V3 r = F + (sx[q] * th) * R + (sy[q] * tv) * U;
        nc[q] = E + cam.znear * r;
        fc[q] = E + cam.zfar * r;
    }
    std::vector<std::vector<V3>> ffaces = {{nc[0], nc[1], nc[2], nc[3]}, {fc[0], fc[1], fc[2], fc[3]}};
    for (int q = 0; q < 4; ++q) ffaces.push_back({nc[q], nc[(q + 1) % 4], fc[(q + 1) % 4], fc[q]});
    const double W = dom.width, H = dom.height, z0 = dom.zmin, z1 = dom.zmax;
    std::vector<Plane> box = {{{-1, 0, 0}, 0.0}, {{1, 0, 0}, W}, {{0, -1, 0}, 0.0},
                              {{0, 1, 0}, H},    {{0, 0, -1}, -z0}, {{0, 0, 1}, z1}};
    std::vector<Plane> fr = {{-1.0 * F, -(dot(F, E) + cam.znear)},
                             {F, dot(F, E) + cam.zfar},
                             {(-1.0 * R) - th * F, dot((-1.0 * R) - th * F, E)},
                             {R - th * F, dot(R - th * F, E)},
                             {(-1.0 * U) - tv * F, dot((-1.0 * U) - tv * F, E)},
                             {U - tv * F, dot(U - tv * F, E)}};
    std::vector<std::vector<V3>> bfaces = {
        {{0, 0, z0}, {0, H, z0}, {0, H, z1}, {0, 0, z1}},
        {{W, 0, z0}, {W, H, z0}, {W, H, z1}, {W, 0, z1}},
        {{0, 0, z0}, {W, 0, z0}, {W, 0, z1}, {0, 0, z1}},
        {{0, H, z0}, {W, H, z0}, {W, H, z1}, {0, H, z1}},
        {{0, 0, z0}, {W, 0, z0}, {W, H, z0}, {0, H, z0}},
        {{0, 0, z1}, {W, 0, z1}, {W, H, z1}, {0, H, z1}}};
    std::vector<P2> ground;
    auto add_clipped = [&](const std::vector<V3>& face, const std::vector<Plane>& planes) {
        std::vector<V3> poly = face;
        for (const Plane& pl : planes) {
            if (poly.empty()) break;
            poly = clip_poly(poly, pl);
        }
        // the volume lies inside the box: clamp away rounding excursions
        for (const V3& p : poly)
            ground.push_back({std::min(std::max(p.x, 0.0), W), std::min(std::max(p.y, 0.0), H)});
    };
    for (const auto& f : ffaces) add_clipped(f, box);
    for (const auto& f : bfaces) add_clipped(f, fr);

    // 2. ground projection and convex hull
    std::vector<P2> hull = monotone_hull(ground);
    if (hull.size() > 64) return HF_ERR_ARG;
    out->n_hull = int(hull.size());
    for (size_t i = 0; i < hull.size(); ++i) { out->hull[i][0] = hull[i].x; out->hull[i][1] = hull[i].y; }

    // 3. depth range along the view direction
    double n = 0.0, f = 0.0;
    for (size_t i = 0; i < hull.size(); ++i) {
        double s = (hull[i].x - E.x) * out->dir2[0] + (hull[i].y - E.y) * out->dir2[1];
        if (i == 0 || s < n) n = s;
        if (i == 0 || s > f) f = s;
    }
    out->n = n;
    out->f = f;

    // 4. splits: d_k = lambda n'(f/n')^(k/C) + (1-lambda)(n' + (f-n') k/C)
    double split[HF_MAX_CASCADES + 1];
    const double np = std::max(n, std::max(cam.znear, dom.c_min));
    split[0] = n;
    split[C] = f;
    for (int k = 1; k < C; ++k) {
        double fr_k = double(k) / double(C);
        split[k] = (f > np) ? cam.split_lambda * np * std::pow(f / np, fr_k) +
                                  (1.0 - cam.split_lambda) * (np + (f - np) * fr_k)
                            : n + (f - n) * fr_k;
    }

    // 5./6. band polygons and stable fit
    for (int k = 0; k < C; ++k) {
        hf_cascade_info& c = out->cas[k];
        c.near_depth = split[k];
        c.far_depth = split[k + 1];
        c.far_ext_depth = (k < C - 1) ? c.far_depth + cam.overlap_frac * (c.far_depth - c.near_depth)
                                      : c.far_depth;
        c.N = N;
        std::vector<P2> poly;
        if (hull.size() >= 3) {
            const double e2[2] = {E.x, E.y};
            poly = clip_depth(hull, out->dir2, e2, c.near_depth, true);
            if (!poly.empty()) poly = clip_depth(poly, out->dir2, e2, c.far_ext_depth, false);
            poly = monotone_hull(poly);
        }
        if (poly.size() > HF_MAX_POLY) return HF_ERR_ARG;
        c.n_poly = int(poly.size());
        for (size_t i = 0; i < poly.size(); ++i) { c.poly[i][0] = poly[i].x; c.poly[i][1] = poly[i].y; }
        const double cm = dom.c_min;
        c.texel_ladder = cam.texel_ladder;
        c.reuse_source = -1;
        c.stop_level = 0;
        c.reserved = 0;
        double x0 = 0.0, x1 = 0.0, y0 = 0.0, y1 = 0.0;
        if (c.n_poly >= 3) {
            x0 = x1 = poly[0].x;
            y0 = y1 = poly[0].y;
            for (const P2& p : poly) {
                x0 = std::min(x0, p.x); x1 = std::max(x1, p.x);
                y0 = std::min(y0, p.y); y1 = std::max(y1, p.y);
            }
            c.aabb[0] = x0; c.aabb[1] = y0; c.aabb[2] = x1; c.aabb[3] = y1;
        } else {
            c.n_poly = 0;
        }
        if (cam.texel_ladder > 0) {
            // lattice fit: the spacing is the smallest ladder value
            // c_min 2^(m/n), m >= -8n, whose N - 2 spacings span the box's
            // larger side (so it depends on the box's size, not its place);
            // the origin is the box corner rounded down onto that lattice,
            // which leaves N - 1 spacings enough to reach the far side
            const int n = cam.texel_ladder;
            const int64_t m_lo = -8 * int64_t(n);
            int64_t m = c.n_poly ? m_lo : 0;
            if (c.n_poly) {
                const double need = std::max(x1 - x0, y1 - y0) * (1.0 - 1e-9) / double(N - 2);
                if (ladder_texel(cm, m_lo, n) < need) {
                    m = std::max(m_lo, int64_t(std::ceil(double(n) * std::log2(need / cm))));
                    while (m > m_lo && ladder_texel(cm, m - 1, n) >= need) --m;
                    while (ladder_texel(cm, m, n) < need) ++m;
                }
                // hysteresis: an earlier frame's step one coarser still fits,
                // and keeping it keeps that frame's texels on this lattice
                if (follow && follow[k] == m + 1) m = follow[k];
            }
            const double h = ladder_texel(cm, m, n);
            c.snap_k = m;
            c.snap_x = c.n_poly ? int64_t(std::floor(x0 / h + 1e-9)) : 0;
            c.snap_y = c.n_poly ? int64_t(std::floor(y0 / h + 1e-9)) : 0;
            c.texel = h;
            c.ox = double(c.snap_x) * h;
            c.oy = double(c.snap_y) * h;
            c.extent = double(N - 1) * h;
            continue;
        }
        if (c.n_poly) {
            // even multiple of c_min covering the larger side; origin on a
            // multiple of c_min; widen until the box is covered (1e-9 slack
            // so values landing on a multiple do not flip on rounding)
            int64_t kk = (int64_t)std::ceil(std::max(x1 - x0, y1 - y0) / (2.0 * cm) - 1e-9);
            if (kk < 1) kk = 1;
            int64_t sxn = (int64_t)std::floor(x0 / cm + 1e-9);
            int64_t syn = (int64_t)std::floor(y0 / cm + 1e-9);
            while (double(sxn + 2 * kk) * cm < x1 - 1e-9 * cm || double(syn + 2 * kk) * cm < y1 - 1e-9 * cm)
                kk++;
            c.snap_x = sxn; c.snap_y = syn; c.snap_k = kk;
        } else {
            c.snap_x = c.snap_y = 0;
            c.snap_k = 1;
        }
        c.ox = double(c.snap_x) * cm;
        c.oy = double(c.snap_y) * cm;
        c.extent = 2.0 * double(c.snap_k) * cm;
        c.texel = c.extent / double(N - 1);
    }
    // coarse-level stop: per cascade the largest max-mip level whose nodes span
    // at most lod_pixels pixels at the cascade's near depth
    const double pitch = 2.0 * std::tan(0.5 * cam.vfov) / double(cam.height);
    int K = 0;
    while ((int64_t(1) << K) < int64_t(N) - 1) ++K;
    for (int k = 0; k < C && cam.lod_pixels > 0.0; ++k) {
        hf_cascade_info& c = out->cas[k];
        const double span = cam.lod_pixels * pitch * c.near_depth;
        if (!(span > 0.0)) continue;
        int L = 0;
        while (L < K && c.texel * double(int64_t(2) << L) <= span * (1.0 + 1e-9)) ++L;
        c.stop_level = L;
    }
    return HF_OK;
}

}  // namespace hfi

/*
 * CPU FP64 oracle (test infrastructure only; see hf_oracle.h).
 *
 * Every function restates one step of the paper in plain code:
 *   Eq. 1 (truncated Gaussian weight) ........ orc_rbf_weight (kernel 0)
 *   Wendland C2 weight (another interpolant) .. orc_rbf_weight (kernel 1)
 *   Eq. 2 (normalised weighted sum) ........... orc_rbf_points, orc_texel_heights
 *   Section 3 (cascade fitting) ............... orc_fit, orc_frustum_box_vertices
 *   lattice fit for texel reuse (extension) ... orc_ladder_fit
 *   Section 3 (visible-texel mask) ............ orc_mask
 *   Section 5 (maximum mipmap, Tevs et al.) ... orc_maxmip
 *   Section 5 (ray casting, bilinear patches) . orc_ray_patch, orc_raycast
 *   coarse-level stop (extension) ............. orc_stop_level, trace_boxes
 * Where the paper leaves a detail open, the reading taken is stated at the
 * function and is the same one the product library follows.
 */
#include "hf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Eq. 1: w_i(p) = exp(-(d/c)^2 / (2 sigma^2)) - exp(-R^2 / (2 sigma^2)).
 * The paper truncates at 3.5 sigma (R = 3.5 sigma gives its constant
 * exp(-3.5^2/2)); R is a parameter here.  A cell influences p only if
 * w > 0 (Section 4), so the weight is 0 at and beyond d = R c.            */
double orc_rbf_weight(double dist, double c, double sigma, double radius, int kernel) {
    if (kernel == 1) {
        /* Wendland's compactly supported C2 function psi_{3,1}(r) =
         * (1 - r)^4 (4 r + 1) for r < 1, 0 beyond, with r = d / (radius c):
         * the same support as the truncated Gaussian (sigma unused).        */
        double r = dist / (radius * c);
        if (r >= 1.0) return 0.0;
        double t = 1.0 - r;
        return t * t * t * t * (4.0 * r + 1.0);
    }
    double r = dist / c;
    double w = exp(-(r * r) / (2.0 * sigma * sigma)) - exp(-(radius * radius) / (2.0 * sigma * sigma));
    return w > 0.0 ? w : 0.0;
}

/* Cell geometry from quadtree leaves: edge c = root_cell / 2^level, centre at
 * ((ix + 1/2) c, (iy + 1/2) c) (Section 2: values sit at cell centres).     */
void orc_cells_from_leaves(double root_cell, const int* level, const int* ix, const int* iy,
                           const float* value, long n, double* cx, double* cy, double* cs,
                           double* cv) {
    for (long k = 0; k < n; ++k) {
        double c = root_cell / ldexp(1.0, level[k]);
        cs[k] = c;
        cx[k] = ((double)ix[k] + 0.5) * c;
        cy[k] = ((double)iy[k] + 0.5) * c;
        cv[k] = (double)value[k];
    }
}

/* Exact enumeration of the influencing set I(p): every cell with
 * dist < R * c_i lies within R * c_max of p, so binning the centres on a
 * grid of that size and visiting the 3x3 neighbouring bins finds all of
 * them.  The weight test then keeps exactly I(p).                          */
typedef struct {
    double bin;
    long nbx, nby;
    long* start;  /* nbx*nby + 1 */
    long* items;
} orc_bins;

static void bins_build(orc_bins* b, const double* cx, const double* cy, const double* cs, long n,
                       double radius, double w, double h) {
    double cmax = 0.0;
    for (long k = 0; k < n; ++k) cmax = cs[k] > cmax ? cs[k] : cmax;
    b->bin = radius * cmax;
    if (b->bin <= 0.0) b->bin = 1.0;
    b->nbx = (long)floor(w / b->bin) + 1;
    b->nby = (long)floor(h / b->bin) + 1;
    long nb = b->nbx * b->nby;
    b->start = (long*)calloc((size_t)nb + 1, sizeof(long));
    b->items = (long*)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    long* bi = (long*)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    for (long k = 0; k < n; ++k) {
        long x = (long)floor(cx[k] / b->bin), y = (long)floor(cy[k] / b->bin);
        x = x < 0 ? 0 : (x >= b->nbx ? b->nbx - 1 : x);
        y = y < 0 ? 0 : (y >= b->nby ? b->nby - 1 : y);
        bi[k] = y * b->nbx + x;
        b->start[bi[k] + 1]++;
    }
    for (long q = 0; q < nb; ++q) b->start[q + 1] += b->start[q];
    long* fill = (long*)malloc(sizeof(long) * (size_t)nb);
    memcpy(fill, b->start, sizeof(long) * (size_t)nb);
    for (long k = 0; k < n; ++k) b->items[fill[bi[k]]++] = k;
    free(fill);
    free(bi);
}

static void bins_free(orc_bins* b) {
    free(b->start);
    free(b->items);
}

/* Eq. 2 at one point: v = sum_{i in I} w_i v_i / sum_{i in I} w_i.
 * Returns NaN when I is empty (the quotient is undefined).                */
static double rbf_brute(const double* cx, const double* cy, const double* cs, const double* cv,
                        long n, double sigma, double radius, int kernel, double px, double py, int* nI) {
    double sw = 0.0, swv = 0.0;
    int cnt = 0;
    for (long k = 0; k < n; ++k) {
        double w = orc_rbf_weight(hypot(cx[k] - px, cy[k] - py), cs[k], sigma, radius, kernel);
        if (w > 0.0) {
            sw += w;
            swv += w * cv[k];
            cnt++;
        }
    }
    if (nI) *nI = cnt;
    return cnt ? swv / sw : NAN;
}

static double rbf_binned(const orc_bins* b, const double* cx, const double* cy, const double* cs,
                         const double* cv, double sigma, double radius, int kernel, double px,
                         double py, int* nI) {
    long bx = (long)floor(px / b->bin), by = (long)floor(py / b->bin);
    double sw = 0.0, swv = 0.0;
    int cnt = 0;
    for (long y = by - 1; y <= by + 1; ++y) {
        if (y < 0 || y >= b->nby) continue;
        for (long x = bx - 1; x <= bx + 1; ++x) {
            if (x < 0 || x >= b->nbx) continue;
            long q = y * b->nbx + x;
            for (long s = b->start[q]; s < b->start[q + 1]; ++s) {
                long k = b->items[s];
                double w = orc_rbf_weight(hypot(cx[k] - px, cy[k] - py), cs[k], sigma, radius, kernel);
                if (w > 0.0) {
                    sw += w;
                    swv += w * cv[k];
                    cnt++;
                }
            }
        }
    }
    if (nI) *nI = cnt;
    return cnt ? swv / sw : NAN;
}

void orc_rbf_points(const double* cx, const double* cy, const double* cs, const double* cv,
                    long n, double sigma, double radius, int kernel, double dom_w, double dom_h,
                    const double* px, const double* py, long m, int mode, double* out,
                    int* n_influencers) {
    if (mode == 0) {
#pragma omp parallel for schedule(dynamic, 16)
        for (long q = 0; q < m; ++q)
            out[q] = rbf_brute(cx, cy, cs, cv, n, sigma, radius, kernel, px[q], py[q],
                               n_influencers ? &n_influencers[q] : NULL);
        return;
    }
    orc_bins b;
    bins_build(&b, cx, cy, cs, n, radius, dom_w, dom_h);
#pragma omp parallel for schedule(dynamic, 64)
    for (long q = 0; q < m; ++q)
        out[q] = rbf_binned(&b, cx, cy, cs, cv, sigma, radius, kernel, px[q], py[q],
                            n_influencers ? &n_influencers[q] : NULL);
    bins_free(&b);
}

/* ------------------------------------------------------------------------ */
/* Section 3: cascade fitting.                                              */

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static void norm3(double* a) {
    double l = sqrt(dot3(a, a));
    a[0] /= l; a[1] /= l; a[2] /= l;
}

/* Orthonormal camera basis: F = forward, U = up made orthogonal to F, R = F x U
 * (right).  If up is parallel to forward, world +y stands in for up.      */
static void camera_basis(const orc_camera* cam, double* F, double* U, double* R) {
    F[0] = cam->forward[0]; F[1] = cam->forward[1]; F[2] = cam->forward[2];
    norm3(F);
    double u[3] = {cam->up[0], cam->up[1], cam->up[2]};
    double d = dot3(u, F);
    U[0] = u[0] - d * F[0]; U[1] = u[1] - d * F[1]; U[2] = u[2] - d * F[2];
    if (sqrt(dot3(U, U)) < 1e-9 * sqrt(dot3(u, u))) {
        double ey[3] = {0.0, 1.0, 0.0};
        d = dot3(ey, F);
        U[0] = -d * F[0]; U[1] = 1.0 - d * F[1]; U[2] = -d * F[2];
    }
    norm3(U);
    cross3(F, U, R);
}

/* Ground projection of the view vector, normalised (Section 3).  When the
 * camera looks straight down, the projection of the up vector (the top of
 * the screen) is used instead.                                             */
static void view_dir2(const double* F, const double* U, double* dir2) {
    double x = F[0], y = F[1];
    double l = hypot(x, y);
    if (l < 1e-12) { x = U[0]; y = U[1]; l = hypot(x, y); }
    dir2[0] = x / l;
    dir2[1] = y / l;
}

/* The 12 half-spaces a.p <= b bounding (view frustum) AND (heightfield box). */
static void frustum_box_planes(const orc_camera* cam, const orc_domain* dom, double a[12][3],
                               double b[12]) {
    double F[3], U[3], R[3];
    camera_basis(cam, F, U, R);
    double tv = tan(0.5 * cam->vfov), th = tv * (double)cam->width / (double)cam->height;
    const double* e = cam->eye;
    a[0][0] = -F[0]; a[0][1] = -F[1]; a[0][2] = -F[2]; b[0] = -(dot3(F, e) + cam->znear);
    a[1][0] = F[0];  a[1][1] = F[1];  a[1][2] = F[2];  b[1] = dot3(F, e) + cam->zfar;
    double r[4][3];
    int sx[4] = {-1, 1, 1, -1}, sy[4] = {-1, -1, 1, 1};
    for (int q = 0; q < 4; ++q)
        for (int c = 0; c < 3; ++c) r[q][c] = F[c] + sx[q] * th * R[c] + sy[q] * tv * U[c];
    /* side planes through the eye spanned by consecutive corner rays */
    for (int q = 0; q < 4; ++q) {
        double n[3];
        cross3(r[q], r[(q + 1) % 4], n);
        if (dot3(n, F) > 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
        a[2 + q][0] = n[0]; a[2 + q][1] = n[1]; a[2 + q][2] = n[2];
        b[2 + q] = dot3(n, e);
    }
    double box[6][4] = {{-1, 0, 0, 0}, {1, 0, 0, dom->width}, {0, -1, 0, 0},
                        {0, 1, 0, dom->height}, {0, 0, -1, -dom->zmin}, {0, 0, 1, dom->zmax}};
    for (int q = 0; q < 6; ++q) {
        a[6 + q][0] = box[q][0]; a[6 + q][1] = box[q][1]; a[6 + q][2] = box[q][2];
        b[6 + q] = box[q][3];
    }
}

/* Vertices of the intersection volume of the view frustum and the
 * heightfield's bounding box (Section 3): every point where three of the
 * 12 bounding planes meet and that lies inside all 12 half-spaces.         */
int orc_frustum_box_vertices(const orc_camera* cam, const orc_domain* dom, double* xyz, int cap) {
    double a[12][3], b[12];
    frustum_box_planes(cam, dom, a, b);
    double scale = fabs(dom->width) + fabs(dom->height) + fabs(dom->zmin) + fabs(dom->zmax) +
                   fabs(cam->eye[0]) + fabs(cam->eye[1]) + fabs(cam->eye[2]);
    int cnt = 0;
    for (int i = 0; i < 12; ++i)
        for (int j = i + 1; j < 12; ++j)
            for (int k = j + 1; k < 12; ++k) {
                double cjk[3], cki[3], cij[3];
                cross3(a[j], a[k], cjk);
                cross3(a[k], a[i], cki);
                cross3(a[i], a[j], cij);
                double det = dot3(a[i], cjk);
                double mag = sqrt(dot3(a[i], a[i]) * dot3(a[j], a[j]) * dot3(a[k], a[k]));
                if (fabs(det) <= 1e-12 * mag) continue;
                double p[3];
                for (int c = 0; c < 3; ++c) p[c] = (b[i] * cjk[c] + b[j] * cki[c] + b[k] * cij[c]) / det;
                int inside = 1;
                for (int q = 0; q < 12 && inside; ++q) {
                    double tol = 1e-9 * sqrt(dot3(a[q], a[q])) * (scale + sqrt(dot3(p, p)));
                    if (dot3(a[q], p) > b[q] + tol) inside = 0;
                }
                if (inside && cnt < cap) {
                    xyz[3 * cnt] = p[0]; xyz[3 * cnt + 1] = p[1]; xyz[3 * cnt + 2] = p[2];
                    cnt++;
                }
            }
    return cnt;
}

/* Convex hull by gift wrapping (Jarvis march), counter-clockwise, without
 * collinear or repeated vertices.  Returns the vertex count (0 if the
 * points span no area).                                                    */
static int gift_wrap(const double* pts, int n, double out[][2], int cap) {
    if (n < 3) return 0;
    double scale = 0.0;
    for (int i = 0; i < n; ++i) scale = fmax(scale, fmax(fabs(pts[2 * i]), fabs(pts[2 * i + 1])));
    scale = fmax(scale, 1.0);
    double same = 1e-9 * scale, eps = 1e-12 * scale * scale;
    int start = 0;
    for (int i = 1; i < n; ++i)
        if (pts[2 * i] < pts[2 * start] ||
            (pts[2 * i] == pts[2 * start] && pts[2 * i + 1] < pts[2 * start + 1]))
            start = i;
    int p = start, m = 0;
    for (int guard = 0; guard <= n; ++guard) {
        if (m >= cap) return 0;
        out[m][0] = pts[2 * p];
        out[m][1] = pts[2 * p + 1];
        m++;
        int q = -1;
        for (int r = 0; r < n; ++r) {
            double rx = pts[2 * r] - pts[2 * p], ry = pts[2 * r + 1] - pts[2 * p + 1];
            if (fabs(rx) <= same && fabs(ry) <= same) continue;
            if (q < 0) { q = r; continue; }
            double qx = pts[2 * q] - pts[2 * p], qy = pts[2 * q + 1] - pts[2 * p + 1];
            double cr = qx * ry - qy * rx;
            if (cr < -eps || (fabs(cr) <= eps && rx * rx + ry * ry > qx * qx + qy * qy)) q = r;
        }
        if (q < 0) return 0;
        double dx = pts[2 * q] - pts[2 * start], dy = pts[2 * q + 1] - pts[2 * start + 1];
        if (fabs(dx) <= same && fabs(dy) <= same) break;
        p = q;
    }
    if (m < 3) return 0;
    /* zero-area hulls (all points on a line) count as empty */
    double area = 0.0;
    for (int i = 0; i < m; ++i) {
        int j = (i + 1) % m;
        area += out[i][0] * out[j][1] - out[j][0] * out[i][1];
    }
    return 0.5 * area > eps ? m : 0;
}

/* Projected depth of a ground point: offset from the eye along dir2.      */
static double sdepth(const double* dir2, const double* eye, double x, double y) {
    return (x - eye[0]) * dir2[0] + (y - eye[1]) * dir2[1];
}

/* hull AND {lo <= s <= hi}: hull vertices inside the band plus the points
 * where hull edges cross the band's two lines, wrapped again.             */
static int clip_band(const double hull[][2], int nh, const double* dir2, const double* eye,
                     double lo, double hi, double out[][2]) {
    double pts[4 * ORC_MAX_POLY * 2];
    int np = 0;
    for (int i = 0; i < nh; ++i) {
        const double* a = hull[i];
        const double* b = hull[(i + 1) % nh];
        double sa = sdepth(dir2, eye, a[0], a[1]), sb = sdepth(dir2, eye, b[0], b[1]);
        if (sa >= lo && sa <= hi) { pts[2 * np] = a[0]; pts[2 * np + 1] = a[1]; np++; }
        double lines[2] = {lo, hi};
        for (int l = 0; l < 2; ++l) {
            double L = lines[l];
            if ((sa - L) * (sb - L) < 0.0) {
                double t = (L - sa) / (sb - sa);
                pts[2 * np] = a[0] + t * (b[0] - a[0]);
                pts[2 * np + 1] = a[1] + t * (b[1] - a[1]);
                np++;
            }
        }
    }
    return gift_wrap(pts, np, out, ORC_MAX_POLY);
}

/* Stable texel-aligned fit (Section 3): the extent E is the smallest even
 * multiple of the minimum cell size covering the box's larger side, the
 * origin is the box's lower corner rounded down to a multiple of the
 * minimum cell size (widening E by 2 c_min until the box is covered), and
 * the texel spacing h = E / (N - 1) puts the four box corners on texel
 * centres.  A relative slack of 1e-9 keeps values that land on a multiple
 * from flipping on rounding.                                              */
/* Lattice fit (not in the paper; it makes texels of consecutive frames
 * coincide so that they can be reused).  Texel spacings come from the ladder
 * h_m = c_min 2^(m/n), m an integer >= -8n; the fit takes the smallest m
 * with (N - 2) h_m >= the box's larger side, which depends on the box's size
 * only, so moving the box never changes h.  The origin is the box's lower
 * corner rounded down to the lattice of h_m: from there N - 1 spacings
 * reach past the far side, because rounding down costs less than one
 * spacing.  Texel (i, j) lies on lattice point (i0 + i, j0 + j).  The same
 * 1e-9 relative slack as the stable fit keeps boundary cases from flipping. */
static double ladder_spacing(double c_min, long long m, int n) {
    return c_min * pow(2.0, (double)m / (double)n);
}

void orc_ladder_fit(double x0, double y0, double x1, double y1, double c_min, int N, int n,
                    long long* m, long long* i0, long long* j0, double* h) {
    double side = fmax(x1 - x0, y1 - y0);
    long long lo = -8LL * n;
    long long k = lo;
    if (side > 0.0) {
        double need = side * (1.0 - 1e-9) / (double)(N - 2);
        double guess = floor((double)n * log2(need / c_min)) - 2.0;
        if (guess > (double)lo) k = (long long)guess;
        while (ladder_spacing(c_min, k, n) < need) k++;
    }
    *m = k;
    *h = ladder_spacing(c_min, k, n);
    *i0 = (long long)floor(x0 / *h + 1e-9);
    *j0 = (long long)floor(y0 / *h + 1e-9);
}

static void lattice_fit(orc_cascade* c, double c_min, int N, int n, const long long* follow) {
    c->N = N;
    if (c->n_poly < 3) {
        c->n_poly = 0;
        c->aabb[0] = c->aabb[1] = c->aabb[2] = c->aabb[3] = 0.0;
        c->snap_x = c->snap_y = c->snap_k = 0;
        c->h = c_min;
    } else {
        double x0 = c->poly[0][0], x1 = x0, y0 = c->poly[0][1], y1 = y0;
        for (int i = 1; i < c->n_poly; ++i) {
            x0 = fmin(x0, c->poly[i][0]); x1 = fmax(x1, c->poly[i][0]);
            y0 = fmin(y0, c->poly[i][1]); y1 = fmax(y1, c->poly[i][1]);
        }
        c->aabb[0] = x0; c->aabb[1] = y0; c->aabb[2] = x1; c->aabb[3] = y1;
        orc_ladder_fit(x0, y0, x1, y1, c_min, N, n, &c->snap_k, &c->snap_x, &c->snap_y, &c->h);
        /* hysteresis (following an earlier frame): keep that frame's step if
         * it is one step coarser than the smallest that fits */
        if (follow && *follow == c->snap_k + 1) {
            c->snap_k = *follow;
            c->h = ladder_spacing(c_min, c->snap_k, n);
            c->snap_x = (long long)floor(x0 / c->h + 1e-9);
            c->snap_y = (long long)floor(y0 / c->h + 1e-9);
        }
    }
    c->ox = (double)c->snap_x * c->h;
    c->oy = (double)c->snap_y * c->h;
    c->E = (double)(N - 1) * c->h;
}

static void stable_fit(orc_cascade* c, double c_min, int N) {
    c->N = N;
    if (c->n_poly < 3) {
        c->n_poly = 0;
        c->aabb[0] = c->aabb[1] = c->aabb[2] = c->aabb[3] = 0.0;
        c->snap_x = c->snap_y = 0;
        c->snap_k = 1;
    } else {
        double x0 = c->poly[0][0], x1 = x0, y0 = c->poly[0][1], y1 = y0;
        for (int i = 1; i < c->n_poly; ++i) {
            x0 = fmin(x0, c->poly[i][0]); x1 = fmax(x1, c->poly[i][0]);
            y0 = fmin(y0, c->poly[i][1]); y1 = fmax(y1, c->poly[i][1]);
        }
        c->aabb[0] = x0; c->aabb[1] = y0; c->aabb[2] = x1; c->aabb[3] = y1;
        double m = fmax(x1 - x0, y1 - y0);
        long long k = (long long)ceil(m / (2.0 * c_min) - 1e-9);
        if (k < 1) k = 1;
        long long sx = (long long)floor(x0 / c_min + 1e-9);
        long long sy = (long long)floor(y0 / c_min + 1e-9);
        while ((double)(sx + 2 * k) * c_min < x1 - 1e-9 * c_min ||
               (double)(sy + 2 * k) * c_min < y1 - 1e-9 * c_min)
            k++;
        c->snap_x = sx; c->snap_y = sy; c->snap_k = k;
    }
    c->ox = (double)c->snap_x * c_min;
    c->oy = (double)c->snap_y * c_min;
    c->E = 2.0 * (double)c->snap_k * c_min;
    c->h = c->E / (double)(N - 1);
}

/* Section 3 in order: frustum AND box -> ground projection -> convex hull ->
 * depth range [n, f] along dir2 -> splits -> per-cascade band clipping
 * with the far planes of all but the last cascade pushed out -> stable fit.
 *
 * Splits: the paper uses the logarithmic scheme n (f/n)^(k/3) for three
 * cascades (Zhang et al.); the general practical split scheme
 *   d_k = lambda n'(f/n')^(k/C) + (1 - lambda)(n' + (f - n') k / C)
 * reduces to it at lambda = 1, C = 3.  n' = max(n, znear, c_min) keeps the
 * logarithm defined when the hull reaches behind the eye; if f <= n' the
 * splits are uniform over [n, f].  Cascade k covers [d_k, d_{k+1}]; the
 * first cascade starts at n, the last ends at f, and every far plane but
 * the last is pushed out by overlap_frac of its cascade's depth span.     */
int orc_fit(const orc_camera* cam, const orc_domain* dom, orc_view* out) {
    return orc_fit_follow(cam, dom, NULL, out);
}

int orc_fit_follow(const orc_camera* cam, const orc_domain* dom, const long long* follow, orc_view* out) {
    memset(out, 0, sizeof(*out));
    int C = cam->n_cascades;
    if (C < 1 || C > ORC_MAX_CASCADES || cam->cascade_size < 2) return -1;
    if (cam->texel_ladder < 0 || (cam->texel_ladder > 0 && cam->cascade_size < 4)) return -1;
    out->n_cascades = C;
    double F[3], U[3], R[3];
    camera_basis(cam, F, U, R);
    view_dir2(F, U, out->dir2);

    double xyz[3 * 220];
    int nv = orc_frustum_box_vertices(cam, dom, xyz, 220);
    double pts[2 * 220];
    for (int i = 0; i < nv; ++i) { pts[2 * i] = xyz[3 * i]; pts[2 * i + 1] = xyz[3 * i + 1]; }
    out->n_hull = gift_wrap(pts, nv, out->hull, ORC_MAX_POLY);

    double n = 0.0, f = 0.0;
    for (int i = 0; i < out->n_hull; ++i) {
        double s = sdepth(out->dir2, cam->eye, out->hull[i][0], out->hull[i][1]);
        if (i == 0 || s < n) n = s;
        if (i == 0 || s > f) f = s;
    }
    out->n = n;
    out->f = f;

    double np = fmax(n, fmax(cam->znear, dom->c_min));
    double lam = cam->split_lambda;
    out->split[0] = n;
    out->split[C] = f;
    for (int k = 1; k < C; ++k) {
        double fr = (double)k / (double)C;
        if (f > np)
            out->split[k] = lam * np * pow(f / np, fr) + (1.0 - lam) * (np + (f - np) * fr);
        else
            out->split[k] = n + (f - n) * fr;
    }
    for (int k = 0; k < C; ++k) {
        orc_cascade* c = &out->cas[k];
        c->near_ = out->split[k];
        c->far_ = out->split[k + 1];
        c->far_ext = (k < C - 1) ? c->far_ + cam->overlap_frac * (c->far_ - c->near_) : c->far_;
        c->n_poly = out->n_hull >= 3
                        ? clip_band(out->hull, out->n_hull, out->dir2, cam->eye, c->near_, c->far_ext, c->poly)
                        : 0;
        if (cam->texel_ladder > 0)
            lattice_fit(c, dom->c_min, cam->cascade_size, cam->texel_ladder, follow ? follow + k : NULL);
        else
            stable_fit(c, dom->c_min, cam->cascade_size);
    }
    return 0;
}

/* Visible texels (Section 3): texel centre inside the cascade polygon.
 * Reading: the polygon is grown by one texel diagonal (sqrt(2) h) so that
 * every point of the polygon lies in a bilinear patch whose four corners
 * are all visible, and texels must lie in the domain (with a 1e-6 texel
 * slack so that centres exactly on the boundary count as inside).        */
void orc_mask(const orc_cascade* cas, const orc_domain* dom, const int* ii, const int* jj,
              long m, unsigned char* vis, double* margin) {
    double h = cas->h, delta = sqrt(2.0) * h, eps = 1e-6 * h;
    for (long q = 0; q < m; ++q) {
        double px = cas->ox + (double)ii[q] * h, py = cas->oy + (double)jj[q] * h;
        int in = cas->n_poly >= 3;
        double mg = INFINITY;
        for (int e = 0; e < cas->n_poly; ++e) {
            const double* a = cas->poly[e];
            const double* b = cas->poly[(e + 1) % cas->n_poly];
            double nx = b[1] - a[1], ny = -(b[0] - a[0]);
            double l = hypot(nx, ny);
            double slack = delta - (nx * (px - a[0]) + ny * (py - a[1])) / l;
            if (slack < 0.0) in = 0;
            mg = fmin(mg, fabs(slack));
        }
        double dsl[4] = {px + eps, dom->width + eps - px, py + eps, dom->height + eps - py};
        for (int s = 0; s < 4; ++s) {
            if (dsl[s] < 0.0) in = 0;
            mg = fmin(mg, fabs(dsl[s]));
        }
        vis[q] = (unsigned char)in;
        if (margin) margin[q] = mg / h;
    }
}

void orc_texel_heights(const orc_cascade* cas, const orc_domain* dom, const double* cx,
                       const double* cy, const double* cs, const double* cv, long n,
                       double sigma, double radius, int kernel, const int* ii, const int* jj,
                       long m, double* out) {
    unsigned char* vis = (unsigned char*)malloc((size_t)(m > 0 ? m : 1));
    orc_mask(cas, dom, ii, jj, m, vis, NULL);
    double* px = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double* py = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    for (long q = 0; q < m; ++q) {
        px[q] = cas->ox + (double)ii[q] * cas->h;
        py[q] = cas->oy + (double)jj[q] * cas->h;
    }
    orc_rbf_points(cx, cy, cs, cv, n, sigma, radius, kernel, dom->width, dom->height, px, py, m, 1,
                   out, NULL);
    for (long q = 0; q < m; ++q)
        if (!vis[q]) out[q] = -INFINITY;
    free(vis);
    free(px);
    free(py);
}

/* ------------------------------------------------------------------------ */
/* Section 5: maximum mipmap (Tevs et al.).  Reading: level 0 stores, per
 * bilinear patch, the maximum of its four corner texels (a bilinear patch
 * never exceeds its corners), or -inf if any corner is not visible; the
 * patch grid is padded with -inf to P x P, P a power of two; each higher
 * level stores the maximum of its 2 x 2 children.                          */
static int mip_P(int N) {
    int P = 1;
    while (P < N - 1) P <<= 1;
    return P;
}

long orc_maxmip_size(int N) {
    long P = mip_P(N), s = 0;
    for (long p = P; p >= 1; p >>= 1) s += p * p;
    return s;
}

void orc_maxmip(const float* tex, int N, float* mip) {
    int P = mip_P(N);
    for (int pj = 0; pj < P; ++pj)
        for (int pi = 0; pi < P; ++pi) {
            float v = -INFINITY;
            if (pi < N - 1 && pj < N - 1) {
                float c[4] = {tex[(long)pj * N + pi], tex[(long)pj * N + pi + 1],
                              tex[(long)(pj + 1) * N + pi], tex[(long)(pj + 1) * N + pi + 1]};
                int ok = 1;
                for (int q = 0; q < 4; ++q) ok &= isfinite(c[q]) ? 1 : 0;
                if (ok) {
                    v = c[0];
                    for (int q = 1; q < 4; ++q) v = c[q] > v ? c[q] : v;
                }
            }
            mip[(long)pj * P + pi] = v;
        }
    long off = 0;
    for (int p = P; p > 1; p >>= 1) {
        long nxt = off + (long)p * p;
        int h = p >> 1;
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < h; ++x) {
                float a = mip[off + (long)(2 * y) * p + 2 * x], b = mip[off + (long)(2 * y) * p + 2 * x + 1];
                float c = mip[off + (long)(2 * y + 1) * p + 2 * x], d = mip[off + (long)(2 * y + 1) * p + 2 * x + 1];
                float v = a > b ? a : b;
                v = c > v ? c : v;
                v = d > v ? d : v;
                mip[nxt + (long)y * h + x] = v;
            }
        off = nxt;
    }
}

/* Ray against one bilinear patch (Section 5).  Patch-local coordinates
 * a, b in [0, 1]; the surface is H(a, b) = h00 (1-a)(1-b) + h10 a (1-b)
 * + h01 (1-a) b + h11 a b.  Along the segment a = a0 + tau da,
 * b = b0 + tau db, z = z0 + tau dz, tau in [0, dt], H - z is a quadratic
 * A tau^2 + B tau + C.  The hit is its first root in [0, dt]; a segment that
 * starts on or under the surface hits at tau = 0; a tangent touch is a hit. */
int orc_ray_patch(double h00, double h10, double h01, double h11, double a0, double b0,
                  double z0, double da, double db, double dz, double dt, double* tau) {
    double e = h10 - h00, g = h01 - h00, q = h00 - h10 - h01 + h11;
    double C = h00 + e * a0 + g * b0 + q * a0 * b0 - z0;
    double B = e * da + g * db + q * (a0 * db + b0 * da) - dz;
    double A = q * da * db;
    if (C >= 0.0) { *tau = 0.0; return 1; }
    double r[2];
    int nr = 0;
    if (A == 0.0) {
        if (B != 0.0) r[nr++] = -C / B;
    } else {
        double disc = B * B - 4.0 * A * C;
        if (disc < 0.0) return 0;
        double s = sqrt(disc);
        double qq = -0.5 * (B + (B >= 0.0 ? s : -s));
        r[nr++] = qq / A;
        if (qq != 0.0) r[nr++] = C / qq;
    }
    double best = INFINITY;
    for (int i = 0; i < nr; ++i)
        if (r[i] >= 0.0 && r[i] <= dt && r[i] < best) best = r[i];
    if (best == INFINITY) return 0;
    *tau = best;
    return 1;
}

typedef struct {
    double eu, ev, ez;    /* eye in patch units (u, v) and metres (z) */
    double du, dv, dz;    /* direction per metre of t */
} prj_ray;

static int patch_valid(const float* tex, int N, int ci, int cj) {
    return isfinite(tex[(long)cj * N + ci]) && isfinite(tex[(long)cj * N + ci + 1]) &&
           isfinite(tex[(long)(cj + 1) * N + ci]) && isfinite(tex[(long)(cj + 1) * N + ci + 1]);
}

static int test_patch(const float* tex, int N, int ci, int cj, const prj_ray* r, double t0,
                      double t1, double* t_hit) {
    double a0 = r->eu + t0 * r->du - ci, b0 = r->ev + t0 * r->dv - cj, z0 = r->ez + t0 * r->dz;
    double tau;
    if (orc_ray_patch(tex[(long)cj * N + ci], tex[(long)cj * N + ci + 1],
                      tex[(long)(cj + 1) * N + ci], tex[(long)(cj + 1) * N + ci + 1], a0, b0, z0,
                      r->du, r->dv, r->dz, t1 - t0, &tau)) {
        *t_hit = t0 + tau;
        return 1;
    }
    return 0;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static double exit_time(double e, double d, double lo, double hi) {
    if (d > 0.0) return (hi - e) / d;
    if (d < 0.0) return (lo - e) / d;
    return INFINITY;
}

/* Coarse-level stop (an extension after the LOD-dependent early ray
 * termination the paper cites): far from the eye a node of the max mipmap
 * smaller than a few pixels can stand in for the surface under it.  Stop
 * level of a cascade: the largest k with 2^k h <= lod_pixels times the pixel
 * pitch at the cascade's near depth, 2 tan(vfov / 2) / height * near (the
 * footprint only grows beyond it), capped at the mipmap's top level.       */
int orc_stop_level(double lod, double vfov, int height, double near_, double h, int N) {
    if (!(lod > 0.0) || !(near_ > 0.0)) return 0;
    double reach = lod * (2.0 * tan(0.5 * vfov) / (double)height) * near_;
    int P = mip_P(N), K = 0;
    while ((1 << K) < P) K++;
    int L = 0;
    while (L < K && ldexp(h, L + 1) <= reach * (1.0 + 1e-9)) L++;
    return L;
}

/* First hit of the level-L box field: the ray walks the level-L nodes of the
 * max mipmap in order (a 2-D DDA on cells of 2^L patches) and stops in the
 * first node whose maximum it reaches -- at the node's entry if it enters
 * below the box top, else where it comes down to it.                      */
static int trace_boxes(const float* mip, int N, int L, const prj_ray* r, double ta, double tb,
                       double* t_hit, long long* visits) {
    int P = mip_P(N), PL = P >> L;
    long off = 0;
    for (int k = 0; k < L; ++k) off += (long)(P >> k) * (P >> k);
    double s = ldexp(1.0, L);
    int ni = clampi((int)floor((r->eu + ta * r->du) / s), 0, PL - 1);
    int nj = clampi((int)floor((r->ev + ta * r->dv) / s), 0, PL - 1);
    double t = ta;
    for (long guard = 0; guard < 4L * (PL + 2); ++guard) {
        double tx = exit_time(r->eu, r->du, ni * s, (ni + 1) * s);
        double ty = exit_time(r->ev, r->dv, nj * s, (nj + 1) * s);
        double te = fmin(fmin(tx, ty), tb);
        if (te < t) te = t;
        (*visits)++;
        double M = (double)mip[off + (long)nj * PL + ni];
        double z0 = r->ez + t * r->dz, z1 = r->ez + te * r->dz;
        if (fmin(z0, z1) <= M) {
            *t_hit = z0 <= M ? t : t + (M - z0) / r->dz;
            return 1;
        }
        if (te >= tb) return 0;
        if (tx <= ty) ni += r->du > 0.0 ? 1 : -1;
        else nj += r->dv > 0.0 ? 1 : -1;
        if (ni < 0 || nj < 0 || ni >= PL || nj >= PL) return 0;
        t = te;
    }
    return 0;
}

/* First hit by walking every patch the ray crosses (2-D DDA).             */
static int trace_dda(const float* tex, int N, const prj_ray* r, double ta, double tb,
                     double* t_hit, long long* visits) {
    int ci = clampi((int)floor(r->eu + ta * r->du), 0, N - 2);
    int cj = clampi((int)floor(r->ev + ta * r->dv), 0, N - 2);
    double t = ta;
    for (long guard = 0; guard < 8L * N + 16; ++guard) {
        double tx = exit_time(r->eu, r->du, ci, ci + 1), ty = exit_time(r->ev, r->dv, cj, cj + 1);
        double te = fmin(fmin(tx, ty), tb);
        if (te < t) te = t;
        (*visits)++;
        if (patch_valid(tex, N, ci, cj) && test_patch(tex, N, ci, cj, r, t, te, t_hit)) return 1;
        if (te >= tb) return 0;
        if (tx <= ty) ci += r->du > 0.0 ? 1 : -1;
        else cj += r->dv > 0.0 ? 1 : -1;
        if (ci < 0 || ci > N - 2 || cj < 0 || cj > N - 2) return 0;
        t = te;
    }
    return 0;
}

/* First hit by maximum-mipmap traversal (Tevs et al.): a node whose maximum
 * lies below the ray over the node's extent is skipped whole; otherwise it
 * is refined down to single patches, which are intersected exactly.  The
 * current level-0 patch (ci, cj) is tracked as integers; after a step the
 * walk climbs one level when it has left its parent node.  The part of the
 * segment above the top entry (the global maximum) cannot hit and is
 * skipped first.
 * With `jump` (the improved traversal after Dick et al., who refine Tevs et
 * al.'s walk; the paper names it without describing it -- our reading): after
 * a step the walk climbs at once to the coarsest node it has just entered,
 * the level of the highest bit in which the old and new patch coordinates
 * differ, instead of one level per step.  Neither rule skips a node that the
 * ray could meet below its maximum, so both find the DDA's first hit.      */
static int trace_mip(const float* tex, const float* mip, int N, const prj_ray* r, double ta,
                     double tb, double* t_hit, long long* visits, int jump) {
    int P = mip_P(N), K = 0;
    while ((1 << K) < P) K++;
    long off[32];
    off[0] = 0;
    for (int k = 1; k <= K; ++k) off[k] = off[k - 1] + (long)(P >> (k - 1)) * (P >> (k - 1));
    double top = (double)mip[off[K]];
    if (r->ez + ta * r->dz > top) {
        if (!(r->dz < 0.0)) return 0;
        double tz = (top - r->ez) / r->dz;
        if (tz > tb) return 0;
        if (tz > ta) ta = tz;
    }
    int ci = clampi((int)floor(r->eu + ta * r->du), 0, N - 2);
    int cj = clampi((int)floor(r->ev + ta * r->dv), 0, N - 2);
    int k = K;
    double t = ta;
    for (long guard = 0; guard < 64L * (N + 4) * (K + 1); ++guard) {
        int ni = ci >> k, nj = cj >> k, size = 1 << k;
        double tx = exit_time(r->eu, r->du, (double)ni * size, (double)(ni + 1) * size);
        double ty = exit_time(r->ev, r->dv, (double)nj * size, (double)(nj + 1) * size);
        double te = fmin(fmin(tx, ty), tb);
        if (te < t) te = t;
        double zmin = fmin(r->ez + t * r->dz, r->ez + te * r->dz);
        float mx = mip[off[k] + (long)nj * (P >> k) + ni];
        (*visits)++;
        if (zmin <= (double)mx) {
            if (k > 0) { k--; continue; }
            if (test_patch(tex, N, ci, cj, r, t, te, t_hit)) return 1;
        }
        if (te >= tb) return 0;
        int oi = ni, oj = nj, pi = ci, pj = cj;
        if (tx <= ty) {
            ci = r->du > 0.0 ? (ni + 1) * size : ni * size - 1;
            int c2 = (int)floor(r->ev + te * r->dv);
            c2 = r->dv > 0.0 ? (c2 > cj ? c2 : cj) : (r->dv < 0.0 ? (c2 < cj ? c2 : cj) : cj);
            cj = clampi(c2, nj * size, nj * size + size - 1);
        } else {
            cj = r->dv > 0.0 ? (nj + 1) * size : nj * size - 1;
            int c2 = (int)floor(r->eu + te * r->du);
            c2 = r->du > 0.0 ? (c2 > ci ? c2 : ci) : (r->du < 0.0 ? (c2 < ci ? c2 : ci) : ci);
            ci = clampi(c2, ni * size, ni * size + size - 1);
        }
        if (ci < 0 || ci >= P || cj < 0 || cj >= P) return 0;
        t = te;
        if (jump) {
            int diff = (ci ^ pi) | (cj ^ pj), b = -1;
            while (diff) { diff >>= 1; b++; }
            if (b > k) k = b < K ? b : K;
        } else if (k < K && ((ci >> (k + 1)) != (oi >> 1) || (cj >> (k + 1)) != (oj >> 1))) {
            k++;
        }
    }
    return 0;
}

/* t-interval of the ray inside cascade c: projected depth in
 * [near, far_ext] (Section 3 bands, overlap included), texel region
 * u, v in [0, N-1], and the camera's clip range.                          */
static int cascade_interval(const orc_rcascade* c, const prj_ray* r, double ks, double tmin,
                            double tmax, double* ta, double* tb) {
    double lo = tmin, hi = tmax;
    if (ks > 0.0) { lo = fmax(lo, c->near_ / ks); hi = fmin(hi, c->far_ext / ks); }
    else if (ks < 0.0) { lo = fmax(lo, c->far_ext / ks); hi = fmin(hi, c->near_ / ks); }
    else if (!(c->near_ <= 0.0 && 0.0 <= c->far_ext)) return 0;
    double e[2] = {r->eu, r->ev}, d[2] = {r->du, r->dv};
    for (int a = 0; a < 2; ++a) {
        if (d[a] != 0.0) {
            double t0 = (0.0 - e[a]) / d[a], t1 = ((double)(c->N - 1) - e[a]) / d[a];
            lo = fmax(lo, fmin(t0, t1));
            hi = fmin(hi, fmax(t0, t1));
        } else if (e[a] < 0.0 || e[a] > (double)(c->N - 1)) {
            return 0;
        }
    }
    *ta = lo;
    *tb = hi;
    return lo <= hi;
}

/* First hit on [ta, tb] inside one cascade.  Without a water texture this is
 * the terrain's first hit.  With one (the water layer: terrain and water
 * depths on the same cells, Section 2) the ray meets whichever surface comes
 * first: the nearer of the terrain's and the water surface's first hits, the
 * water surface on a tie; *on_water says which.  A water patch exists where
 * its four corners are wet (finite), as a terrain patch needs four visible
 * corners.                                                                 */
static int trace_cascade(const float* tex, const float* wtex, const float* mip, int N, int stop,
                         const prj_ray* r, double ta, double tb, int mode, double* t_hit,
                         int* on_water, long long* visits) {
    double t1 = 0.0, t2 = 0.0;
    int h1 = stop > 0 ? trace_boxes(mip, N, stop, r, ta, tb, &t1, visits)
             : mode == 0 ? trace_dda(tex, N, r, ta, tb, &t1, visits)
                         : trace_mip(tex, mip, N, r, ta, tb, &t1, visits, mode == 2);
    int h2 = wtex ? trace_dda(wtex, N, r, ta, tb, &t2, visits) : 0;
    *on_water = h2 && (!h1 || t2 <= t1);
    if (*on_water) {
        *t_hit = t2;
        return 1;
    }
    if (h1) *t_hit = t1;
    return h1;
}

/* One ray per pixel through the cascades, nearest first (Section 5).
 * Reading of the blend: if cascade c is hit at projected depth s inside its
 * overlap with cascade c+1, cascade c+1 is traced too and, if it is hit,
 * t = (1 - alpha) t_c + alpha t_{c+1} with alpha rising linearly from 0 to 1
 * across the overlap band; otherwise the single hit is kept.  The result
 * reports the first cascade that was hit, with 0x80 added when that
 * cascade's hit is on the water surface (wtex given).                      */
void orc_raycast(const orc_camera* cam, const orc_rcascade* cas, int C,
                 const float* const* tex, const float* const* wtex, const float* const* mip,
                 const int* pxs, const int* pys, long m, int mode, double* t_out, int* hit_out,
                 double* seg_out, long long* visits_out) {
    double F[3], U[3], R[3], dir2[2];
    camera_basis(cam, F, U, R);
    view_dir2(F, U, dir2);
    double tv = tan(0.5 * cam->vfov), th = tv * (double)cam->width / (double)cam->height;
#pragma omp parallel for schedule(dynamic, 64)
    for (long q = 0; q < m; ++q) {
        double sx = (2.0 * (pxs[q] + 0.5) / cam->width - 1.0) * th;
        double sy = (1.0 - 2.0 * (pys[q] + 0.5) / cam->height) * tv;
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = F[c] + sx * R[c] + sy * U[c];
        norm3(d);
        double fd = dot3(d, F);
        double tmin = cam->znear / fd, tmax = cam->zfar / fd;
        double ks = d[0] * dir2[0] + d[1] * dir2[1];
        long long visits = 0;
        int hit = 0;
        double t = NAN, seg = NAN;
        for (int c = 0; c < C && !hit; ++c) {
            prj_ray r = {(cam->eye[0] - cas[c].ox) / cas[c].h, (cam->eye[1] - cas[c].oy) / cas[c].h,
                         cam->eye[2], d[0] / cas[c].h, d[1] / cas[c].h, d[2]};
            double ta, tb, tc;
            int wet = 0;
            if (!cascade_interval(&cas[c], &r, ks, tmin, tmax, &ta, &tb)) continue;
            if (!trace_cascade(tex[c], wtex ? wtex[c] : NULL, mip ? mip[c] : NULL, cas[c].N, cas[c].stop_level,
                               &r, ta, tb, mode, &tc, &wet, &visits))
                continue;
            hit = (1 + c) | (wet ? 0x80 : 0);
            t = tc;
            seg = tb - ta;
            double s = tc * ks;
            if (c + 1 < C && s >= cas[c + 1].near_ && cas[c].far_ext > cas[c + 1].near_) {
                const orc_rcascade* n2 = &cas[c + 1];
                prj_ray r2 = {(cam->eye[0] - n2->ox) / n2->h, (cam->eye[1] - n2->oy) / n2->h,
                              cam->eye[2], d[0] / n2->h, d[1] / n2->h, d[2]};
                double ta2, tb2, t2;
                int wet2 = 0;
                if (cascade_interval(n2, &r2, ks, tmin, tmax, &ta2, &tb2)) {
                    int h2 = trace_cascade(tex[c + 1], wtex ? wtex[c + 1] : NULL, mip ? mip[c + 1] : NULL,
                                           n2->N, n2->stop_level, &r2, ta2, tb2, mode, &t2, &wet2, &visits);
                    if (h2) {
                        double al = (s - n2->near_) / (cas[c].far_ext - n2->near_);
                        al = al < 0.0 ? 0.0 : (al > 1.0 ? 1.0 : al);
                        t = (1.0 - al) * tc + al * t2;
                    }
                }
            }
        }
        t_out[q] = t;
        hit_out[q] = hit;
        if (seg_out) seg_out[q] = seg;
        if (visits_out) visits_out[q] = visits;
    }
}

/*
 * CPU FP64 oracle for adaptive-heightfield RBF discretization and ray casting
 * (Cornel, Horvath, Waser, "An Attempt of Adaptive Heightfield Rendering with
 * Complex Interpolants Using Ray Casting", 2022).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously correct
 * restatement of what the method computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product
 * library never calls it and shares no code, header or table with it.
 *
 * Conventions (all FP64, domain-local metres: the domain is
 * [0, width] x [0, height], x/y horizontal, z up):
 *   - a cell has edge c, centre (cx, cy) and value v (Section 2);
 *   - cascade texel (i, j) sits at (ox + i*h, oy + j*h), i = column, j = row,
 *     stored row-major as tex[j*N + i];
 *   - bilinear patch (pi, pj) spans texels (pi..pi+1, pj..pj+1);
 *   - max-mip level k holds (P>>k)^2 entries, P = smallest power of two
 *     >= N-1, levels stored one after another, row-major.
 */
#ifndef HF_ORACLE_H
#define HF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_CASCADES 8
#define ORC_MAX_POLY 64

typedef struct {
    double width, height;   /* domain extents */
    double zmin, zmax;      /* range of the cell values (bounds the surface) */
    double c_min, c_max;    /* smallest / largest leaf edge */
} orc_domain;

typedef struct {
    double eye[3];          /* domain-local eye */
    double forward[3], up[3];
    double vfov;            /* vertical field of view, radians */
    double znear, zfar;     /* clip distances along forward */
    int width, height;      /* image size */
    int n_cascades, cascade_size;
    double split_lambda, overlap_frac;
    int texel_ladder;       /* 0: the paper's stable fit; n > 0: lattice fit (orc_ladder_fit) */
} orc_camera;

typedef struct {
    double near_, far_, far_ext;       /* projected-depth band; far_ext includes the overlap */
    int n_poly;                        /* 0 = empty cascade */
    double poly[ORC_MAX_POLY][2];      /* CCW cascade polygon */
    double aabb[4];                    /* x0, y0, x1, y1 */
    long long snap_x, snap_y, snap_k;  /* stable fit: ox = snap_x*c_min, oy = snap_y*c_min, E = 2*snap_k*c_min;
                                          lattice fit: h = c_min 2^(snap_k/n), ox = snap_x*h, oy = snap_y*h */
    double ox, oy, E, h;
    int N;
} orc_cascade;

typedef struct {
    double dir2[2];          /* normalised ground projection of the view vector */
    double n, f;             /* depth range of the hull along dir2 */
    double split[ORC_MAX_CASCADES + 1];
    int n_hull;
    double hull[ORC_MAX_POLY][2];
    int n_cascades;
    orc_cascade cas[ORC_MAX_CASCADES];
} orc_view;

/* Cascade used by the ray caster: only what rendering needs.  stop_level
 * 0 is the bilinear surface (Section 5); L >= 1 is the coarse-level stop: the
 * level-L box field of the max mipmap (orc_stop_level). */
typedef struct {
    double ox, oy, h;
    double near_, far_ext;
    int N;
    int stop_level;
} orc_rcascade;

/* ---- Eq. 1 / Eq. 2 ---- */
/* kernel 0: truncated Gaussian (Eq. 1); kernel 1: Wendland psi_{3,1} with support radius * c */
double orc_rbf_weight(double dist, double c, double sigma, double radius, int kernel);
void orc_cells_from_leaves(double root_cell, const int* level, const int* ix, const int* iy,
                           const float* value, long n, double* cx, double* cy, double* cs,
                           double* cv);
/* mode 0: brute force over every cell; mode 1: exact binned enumeration */
void orc_rbf_points(const double* cx, const double* cy, const double* cs, const double* cv,
                    long n, double sigma, double radius, int kernel, double dom_w, double dom_h,
                    const double* px, const double* py, long m, int mode, double* out,
                    int* n_influencers);

/* ---- Section 3: cascade fitting ---- */
int orc_fit(const orc_camera* cam, const orc_domain* dom, orc_view* out);
/* the same, with the lattice fit following an earlier frame: cascade k keeps
 * ladder step follow[k] where that is one step coarser than the smallest
 * that fits (follow: n_cascades steps, or NULL) */
int orc_fit_follow(const orc_camera* cam, const orc_domain* dom, const long long* follow, orc_view* out);
/* lattice fit of a box [x0, x1] x [y0, y1] for n ladder steps per octave:
 * returns the ladder index m, the lattice origin (i0, j0) and h */
void orc_ladder_fit(double x0, double y0, double x1, double y1, double c_min, int N, int n,
                    long long* m, long long* i0, long long* j0, double* h);
int orc_frustum_box_vertices(const orc_camera* cam, const orc_domain* dom, double* xyz,
                             int cap);
/* visibility of texels (i, j) of one cascade; margin = distance to the nearest decision
 * threshold in texels (for comparing decisions taken independently) */
void orc_mask(const orc_cascade* cas, const orc_domain* dom, const int* ii, const int* jj,
              long m, unsigned char* vis, double* margin);
/* heights of texels (i, j): Eq. 2 at visible texels, -inf elsewhere */
void orc_texel_heights(const orc_cascade* cas, const orc_domain* dom, const double* cx,
                       const double* cy, const double* cs, const double* cv, long n,
                       double sigma, double radius, int kernel, const int* ii, const int* jj, long m,
                       double* out);

/* ---- Section 5: maximum mipmap and ray casting ---- */
/* coarse-level stop of a cascade: the largest level k (0..K of its max mipmap)
 * whose nodes, 2^k h wide, span at most lod_pixels pixels at the cascade's near
 * depth; 0 when lod_pixels <= 0 or near <= 0 */
int orc_stop_level(double lod_pixels, double vfov, int height, double near_, double h, int N);
long orc_maxmip_size(int N);
void orc_maxmip(const float* tex, int N, float* mip);
/* first root of bilinear(a,b) - z along a ray segment inside one patch */
int orc_ray_patch(double h00, double h10, double h01, double h11, double a0, double b0,
                  double z0, double da, double db, double dz, double dt, double* tau);
/* mode 0: per-patch DDA; mode 1: max-mip traversal (needs mips) of the terrain,
 * one level up per step (Tevs et al.); mode 2: the same traversal climbing at once
 * to the coarsest node entered (our reading of Dick et al.'s improved traversal);
 * wtex (NULL = none): water surface textures, traced by DDA, the first surface met
 * wins inside each cascade.  Outputs per pixel: t (world distance from the eye),
 * hit (0 = miss, 1 + first cascade hit, + 0x80 if that hit is on the water surface),
 * seg (length of the first-hit cascade's ray segment), visits (mip nodes tested) */
void orc_raycast(const orc_camera* cam, const orc_rcascade* cas, int C,
                 const float* const* tex, const float* const* wtex, const float* const* mip,
                 const int* pxs, const int* pys, long m, int mode, double* t, int* hit,
                 double* seg, long long* visits);
int orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif

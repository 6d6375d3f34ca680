/*
 * FP64 CPU oracle for the batched runtime distance check.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * What it computes (Fujii & Pham, "Real-time Batched Distance Computation for
 * Time-Optimal Safe Path Tracking"):
 *   - Link SDFs: a signed distance field of every link mesh sampled on a grid in
 *     the link's own frame (Sec. III-A, "Link SDFs").  The value at a node is the
 *     signed distance to the mesh: unsigned distance by brute force over all
 *     triangles (closest point on triangle, Ericson, Real-Time Collision
 *     Detection, Sec. 5.1.5), sign from the generalised winding number (sum of
 *     triangle solid angles, Van Oosterom & Strackee 1983).  A mesh made of
 *     several closed components takes the minimum over components.
 *   - Parallel forward kinematics per configuration (Sec. III-A): standard DH.
 *   - The distance at an obstacle point: the point is mapped into each link frame
 *     (the "common way" of Sec. II-B / Fig. 2) and the link SDF is interpolated
 *     trilinearly (the grid-sample interpolation of Sec. III-A).  Outside the grid
 *     box the value is the distance to the box plus the interpolated value at the
 *     nearest box point.
 *   - Reduction with min per configuration (Sec. III-A, last paragraph of the
 *     overview), with the arg-min link and point.  Ties go to the smallest point
 *     index, then the smallest link index.
 *
 * Everything is double precision and written as the plain definition: no
 * culling, no blocking, no reordering.  OpenMP only splits independent outputs
 * (grid nodes, waypoints) across threads.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* The check functions keep per-waypoint transforms on the stack. */
#define ORACLE_MAX_LINKS 16

int oracle_max_links(void) { return ORACLE_MAX_LINKS; }

/* ------------------------------------------------------------------ threads */

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------ vector helpers */

static void sub3(const double *a, const double *b, double *o) {
    o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static double dot3(const double *a, const double *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* ------------------------------------------- point to triangle (Ericson 5.1.5) */

static double seg_dist2(const double *p, const double *a, const double *b) {
    double ab[3], ap[3], q[3];
    sub3(b, a, ab);
    sub3(p, a, ap);
    double den = dot3(ab, ab);
    double t = den > 0.0 ? dot3(ap, ab) / den : 0.0;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    for (int k = 0; k < 3; ++k) q[k] = a[k] + t * ab[k] - p[k];
    return dot3(q, q);
}

/* Closest point on triangle abc to p, classified by Voronoi region; returns the
 * squared distance.  Degenerate (zero-area) triangles fall back to the edges. */
double oracle_point_triangle_dist2(const double *p, const double *a, const double *b,
                                   const double *c) {
    double ab[3], ac[3], ap[3], bp[3], cp[3], q[3];
    sub3(b, a, ab);
    sub3(c, a, ac);
    sub3(p, a, ap);
    double d1 = dot3(ab, ap), d2 = dot3(ac, ap);
    if (d1 <= 0.0 && d2 <= 0.0) { sub3(p, a, q); return dot3(q, q); }      /* vertex a */
    sub3(p, b, bp);
    double d3 = dot3(ab, bp), d4 = dot3(ac, bp);
    if (d3 >= 0.0 && d4 <= d3) { sub3(p, b, q); return dot3(q, q); }       /* vertex b */
    double vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {                              /* edge ab */
        double v = d1 / (d1 - d3);
        for (int k = 0; k < 3; ++k) q[k] = a[k] + v * ab[k] - p[k];
        return dot3(q, q);
    }
    sub3(p, c, cp);
    double d5 = dot3(ab, cp), d6 = dot3(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) { sub3(p, c, q); return dot3(q, q); }      /* vertex c */
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {                              /* edge ac */
        double w = d2 / (d2 - d6);
        for (int k = 0; k < 3; ++k) q[k] = a[k] + w * ac[k] - p[k];
        return dot3(q, q);
    }
    double va = d3 * d6 - d5 * d4;
    if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) {                /* edge bc */
        double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        for (int k = 0; k < 3; ++k) q[k] = b[k] + w * (c[k] - b[k]) - p[k];
        return dot3(q, q);
    }
    double den = va + vb + vc;                                              /* face */
    if (!(den > 0.0)) {
        double e0 = seg_dist2(p, a, b), e1 = seg_dist2(p, b, c), e2 = seg_dist2(p, c, a);
        double m = e0 < e1 ? e0 : e1;
        return m < e2 ? m : e2;
    }
    double v = vb / den, w = vc / den;
    for (int k = 0; k < 3; ++k) q[k] = a[k] + ab[k] * v + ac[k] * w - p[k];
    return dot3(q, q);
}

/* Signed solid angle of triangle abc seen from p (Van Oosterom & Strackee):
 * tan(Omega/2) = det[ra rb rc] / (|ra||rb||rc| + (ra.rb)|rc| + (ra.rc)|rb| + (rb.rc)|ra|).
 * Positive when abc is counter-clockwise seen from the side opposite p. */
double oracle_solid_angle(const double *p, const double *a, const double *b, const double *c) {
    double ra[3], rb[3], rc[3], x[3];
    sub3(a, p, ra);
    sub3(b, p, rb);
    sub3(c, p, rc);
    double la = norm3(ra), lb = norm3(rb), lc = norm3(rc);
    cross3(rb, rc, x);
    double num = dot3(ra, x);
    double den = la * lb * lc + dot3(ra, rb) * lc + dot3(ra, rc) * lb + dot3(rb, rc) * la;
    return 2.0 * atan2(num, den);
}

/* Signed distance from x to one closed component (triangles t0..t1-1). */
static double component_sdf(const double *verts, const int32_t *tris, int32_t t0, int32_t t1,
                            const double *x) {
    double best = INFINITY, omega = 0.0;
    for (int32_t t = t0; t < t1; ++t) {
        const double *a = verts + 3 * tris[3 * t + 0];
        const double *b = verts + 3 * tris[3 * t + 1];
        const double *c = verts + 3 * tris[3 * t + 2];
        double d2 = oracle_point_triangle_dist2(x, a, b, c);
        if (d2 < best) best = d2;
        omega += oracle_solid_angle(x, a, b, c);
    }
    double winding = omega / (4.0 * M_PI);
    double d = sqrt(best);
    return winding >= 0.5 ? -d : d;
}

double oracle_winding_number(const double *verts, const int32_t *tris, int32_t n_tris,
                             const double *x) {
    double omega = 0.0;
    for (int32_t t = 0; t < n_tris; ++t)
        omega += oracle_solid_angle(x, verts + 3 * tris[3 * t], verts + 3 * tris[3 * t + 1],
                                    verts + 3 * tris[3 * t + 2]);
    return omega / (4.0 * M_PI);
}

/* Signed distance of x to a mesh given as closed components: min over components. */
double oracle_mesh_sdf(const double *verts, const int32_t *tris, const int32_t *comp_offsets,
                       int32_t n_comp, const double *x) {
    double d = INFINITY;
    for (int32_t c = 0; c < n_comp; ++c) {
        double dc = component_sdf(verts, tris, comp_offsets[c], comp_offsets[c + 1], x);
        if (dc < d) d = dc;
    }
    return d;
}

void oracle_mesh_sdf_many(const double *verts, const int32_t *tris, const int32_t *comp_offsets,
                          int32_t n_comp, const double *x, int64_t n_x, double *out) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n_x; ++i)
        out[i] = oracle_mesh_sdf(verts, tris, comp_offsets, n_comp, x + 3 * i);
}

/* ----------------------------------------------------------- grid definition */

/* meta layout (10 doubles): origin[3], h, n, center[3], radius, margin.
 * Isotropic spacing from the mesh bounding box grown by the margin on every side:
 * span s = max_axis(hi - lo) + 2 margin, h = s / (n - 1), origin = mid - s/2.
 * Bounding sphere: centre = box mid-point, radius = max vertex distance to it. */
void oracle_grid_meta(const double *verts, int32_t n_verts, int32_t n, double margin,
                      double *meta) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int32_t v = 0; v < n_verts; ++v)
        for (int k = 0; k < 3; ++k) {
            double x = verts[3 * v + k];
            if (x < lo[k]) lo[k] = x;
            if (x > hi[k]) hi[k] = x;
        }
    double mid[3], span = 0.0;
    for (int k = 0; k < 3; ++k) {
        mid[k] = 0.5 * (lo[k] + hi[k]);
        if (hi[k] - lo[k] > span) span = hi[k] - lo[k];
    }
    span += 2.0 * margin;
    double h = span / (double)(n - 1);
    double r2 = 0.0;
    for (int32_t v = 0; v < n_verts; ++v) {
        double d[3];
        sub3(verts + 3 * v, mid, d);
        double q = dot3(d, d);
        if (q > r2) r2 = q;
    }
    for (int k = 0; k < 3; ++k) meta[k] = mid[k] - 0.5 * span;
    meta[3] = h;
    meta[4] = (double)n;
    for (int k = 0; k < 3; ++k) meta[5 + k] = mid[k];
    meta[8] = sqrt(r2);
    meta[9] = margin;
}

/* Node (i, j, k) sits at origin + (i, j, k) h and is stored at i + n (j + n k). */
void oracle_build_grid(const double *verts, int32_t n_verts, const int32_t *tris,
                       const int32_t *comp_offsets, int32_t n_comp, int32_t n, double margin,
                       double *values, double *meta) {
    oracle_grid_meta(verts, n_verts, n, margin, meta);
    const double o0 = meta[0], o1 = meta[1], o2 = meta[2], h = meta[3];
    const int64_t total = (int64_t)n * n * n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t idx = 0; idx < total; ++idx) {
        int64_t i = idx % n, j = (idx / n) % n, k = idx / ((int64_t)n * n);
        double x[3] = {o0 + (double)i * h, o1 + (double)j * h, o2 + (double)k * h};
        values[idx] = oracle_mesh_sdf(verts, tris, comp_offsets, n_comp, x);
    }
}

/* ------------------------------------------------------- forward kinematics */

/* 4x4 row-major helpers */
static void mat4_mul(const double *A, const double *B, double *C) {
    double t[16];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += A[4 * r + k] * B[4 * k + c];
            t[4 * r + c] = s;
        }
    memcpy(C, t, sizeof t);
}
static void mat4_identity(double *M) {
    memset(M, 0, 16 * sizeof(double));
    M[0] = M[5] = M[10] = M[15] = 1.0;
}

/* Standard DH joint transform, the product Rz(theta) Tz(d) Tx(a) Rx(alpha). */
static void dh_joint(double a, double alpha, double d, double theta, double *A) {
    double Rz[16], Tz[16], Tx[16], Rx[16], t[16];
    mat4_identity(Rz); mat4_identity(Tz); mat4_identity(Tx); mat4_identity(Rx);
    Rz[0] = cos(theta); Rz[1] = -sin(theta); Rz[4] = sin(theta); Rz[5] = cos(theta);
    Tz[11] = d;
    Tx[3] = a;
    Rx[5] = cos(alpha); Rx[6] = -sin(alpha); Rx[9] = sin(alpha); Rx[10] = cos(alpha);
    mat4_mul(Rz, Tz, t);
    mat4_mul(t, Tx, t);
    mat4_mul(t, Rx, A);
}

/* One configuration: out = (dof+1) x 12 world-from-link transforms [R | t] row-major.
 * Link 0 is the base link; link j is DH frame j = base * A_1 ... A_j. */
static void fk_one(const double *dh, int32_t dof, const double *base, const double *qw,
                   double *out) {
    double T[16], A[16];
    mat4_identity(T);
    memcpy(T, base, 12 * sizeof(double));
    memcpy(out, T, 12 * sizeof(double));
    for (int32_t j = 0; j < dof; ++j) {
        const double *r = dh + 6 * j;
        dh_joint(r[0], r[1], r[2], r[3] + qw[j], A);
        mat4_mul(T, A, T);
        memcpy(out + (j + 1) * 12, T, 12 * sizeof(double));
    }
}

/* dh: dof x 6 rows (a, alpha, d, theta_offset, q_min, q_max); base: 3x4 world-from-base.
 * out: W x (dof+1) x 12 world-from-link transforms. */
void oracle_fk(const double *dh, int32_t dof, const double *base, const double *q, int64_t W,
               double *out) {
    const int32_t L = dof + 1;
#pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < W; ++w) fk_one(dh, dof, base, q + w * dof, out + w * L * 12);
}

/* ------------------------------------------------------------------ lookup */

static double trilinear(const double *v, int64_t n, const double *u) {
    int64_t i0[3];
    double f[3];
    for (int k = 0; k < 3; ++k) {
        double fl = floor(u[k]);
        int64_t i = (int64_t)fl;
        if (i > n - 2) i = n - 2;
        i0[k] = i;
        f[k] = u[k] - (double)i;
    }
    double acc = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) *
                           (dz ? f[2] : 1.0 - f[2]);
                int64_t idx = (i0[0] + dx) + n * ((i0[1] + dy) + n * (i0[2] + dz));
                acc += w * v[idx];
            }
    return acc;
}

/* Interpolated link SDF at p_loc (link frame).  Inside the grid box: trilinear.
 * Outside: |p_loc - q| + trilinear(q), q the nearest point of the box. */
double oracle_lookup(const double *values, const double *meta, const double *p_loc) {
    /* a NaN coordinate has no grid cell: the value is NaN (such pairs are ignored) */
    if (isnan(p_loc[0]) || isnan(p_loc[1]) || isnan(p_loc[2])) return NAN;
    const int64_t n = (int64_t)meta[4];
    const double h = meta[3], top = (double)(n - 1);
    double u[3];
    int inside = 1;
    for (int k = 0; k < 3; ++k) {
        u[k] = (p_loc[k] - meta[k]) / h;
        if (!(u[k] >= 0.0 && u[k] <= top)) inside = 0;
    }
    if (inside) return trilinear(values, n, u);
    double q[3], d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        double lo = meta[k], hi = meta[k] + top * h;
        q[k] = p_loc[k] < lo ? lo : (p_loc[k] > hi ? hi : p_loc[k]);
        d2 += (p_loc[k] - q[k]) * (p_loc[k] - q[k]);
        u[k] = (q[k] - meta[k]) / h;
        if (u[k] < 0.0) u[k] = 0.0;
        if (u[k] > top) u[k] = top;
    }
    return sqrt(d2) + trilinear(values, n, u);
}

void oracle_lookup_many(const double *values, const double *meta, const double *p_loc,
                        int64_t n_p, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_p; ++i) out[i] = oracle_lookup(values, meta, p_loc + 3 * i);
}

/* Map a world point into a link frame: R^T (p - t) for T = [R | t]. */
static void to_link(const double *T, const double *p, double *pl) {
    double d[3] = {p[0] - T[3], p[1] - T[7], p[2] - T[11]};
    for (int k = 0; k < 3; ++k) pl[k] = T[0 * 4 + k] * d[0] + T[1 * 4 + k] * d[1] + T[2 * 4 + k] * d[2];
}

/* ------------------------------------------------------------- full check */

/* grid_values: L grids, grid l starts at grid_offsets[l] (in doubles).
 * grid_meta: L x 10 (see oracle_grid_meta).  points: N x 3 world.
 * Outputs per waypoint: dist (min over links and points), argmin link and point
 * (first minimum in point-major, link-minor order; -1 when nothing is finite). */
void oracle_check(const double *dh, int32_t dof, const double *base, const double *grid_values,
                  const int64_t *grid_offsets, const double *grid_meta, const double *q,
                  int64_t W, const double *points, int64_t N, double *dist, int32_t *arg_link,
                  int32_t *arg_point) {
    const int32_t L = dof + 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t w = 0; w < W; ++w) {
        double Tw[ORACLE_MAX_LINKS * 12];
        fk_one(dh, dof, base, q + w * dof, Tw);
        double best = INFINITY;
        int32_t bl = -1, bp = -1;
        for (int64_t p = 0; p < N; ++p) {
            for (int32_t l = 0; l < L; ++l) {
                double pl[3];
                to_link(Tw + 12 * l, points + 3 * p, pl);
                double g = oracle_lookup(grid_values + grid_offsets[l], grid_meta + 10 * l, pl);
                if (g < best) { best = g; bl = l; bp = (int32_t)p; }
            }
        }
        dist[w] = best;
        arg_link[w] = bl;
        arg_point[w] = bp;
    }
}

/* All (waypoint, link, point) values, W x L x N, for small cases and tie checks. */
void oracle_pair_values(const double *dh, int32_t dof, const double *base,
                        const double *grid_values, const int64_t *grid_offsets,
                        const double *grid_meta, const double *q, int64_t W,
                        const double *points, int64_t N, double *out) {
    const int32_t L = dof + 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t w = 0; w < W; ++w) {
        double Tw[ORACLE_MAX_LINKS * 12];
        fk_one(dh, dof, base, q + w * dof, Tw);
        for (int32_t l = 0; l < L; ++l)
            for (int64_t p = 0; p < N; ++p) {
                double pl[3];
                to_link(Tw + 12 * l, points + 3 * p, pl);
                out[(w * L + l) * N + p] =
                    oracle_lookup(grid_values + grid_offsets[l], grid_meta + 10 * l, pl);
            }
    }
}

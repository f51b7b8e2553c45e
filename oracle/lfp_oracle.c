/*
 * FP64 CPU oracle for the light-field-probe ray tracer.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's
 * CPU-baseline / reference arm may load this library. It shares no code with
 * the CUDA path (no headers, helpers or tables); it reads the same probe maps
 * (float32 planes made by the seeded input generator) and computes everything
 * in double precision, one pixel at a time, in the order the paper states the
 * method. OpenMP runs pixels in parallel; nothing else is reordered.
 *
 * Paper: Liu, Nowrouzezahrai, McGuire, "Real-Time Scene Reconstruction using
 * Light Field Probes" (arXiv 2507.14624). Passages followed:
 *   - Sec. 3 (Overview): octahedral mapping; the problem statement (ray
 *     (X, w1), probe O, nearest surface point T, w2 = O->T, visible iff
 *     r_p(w2) = d(O, T), then L_o(X, w1) = L_p(w2)); probes on the vertices
 *     of a uniform grid, 8-probe cage, back-face test with stored normals.
 *   - Sec. 4.2 (Ray Tracing Using One Probe): projecting the ray onto the
 *     octahedral map gives at most 4 segments; low-resolution tracing tests
 *     distance only; high-resolution tracing adds the normal test, HIT /
 *     UNKNOWN; eye aligned with a probe is an O(1) lookup.
 *   - Sec. 4.3 (Ray Trace Using Multiple Probes): grid iterator over cubes;
 *     the traversal for fewer than 8 probes (orc_trace_ray, traversal 1).
 *   - Sec. 4.1 and 5.1 (simulated probe data, probe data generation): probe
 *     maps from a point cloud, nearest point per texel (orc_splat_probes).
 *   - Appendix A, Algorithms RayMarching, traceOneProbe, traceOneRaySegment,
 *     lowResolutionTracing, highResolutionTracing.
 *
 * Every function is pinned by the CPU tests in tests/test_oracle_*.py
 * against closed forms, brute force, invariants or the analytic scene (see
 * each test's docstring); none is marked "parity unpinned".
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   R1 octahedral pole +z; texel (i, j) covers u in [i/N, (i+1)/N) of
 *      u = (p + 1) / 2; storage row-major, j the row.
 *   R2 low-resolution map (a convolution in the paper) -> per-block min and max of
 *      the distance map (block k x k, k = N / M); conservative, so the
 *      hierarchical march returns exactly what the flat march returns.
 *   R3 texel test over the ray's t-interval [ta, tb] inside the texel:
 *      r(t) = |X + t w - O|, r_hi = max(r(ta), r(tb)), r_lo = min over
 *      [ta, tb]. With d the stored distance and thr(d) = d (1 + 4 th / N):
 *      r_hi < d -> the ray stays in front (continue); else r_lo <= thr(d) ->
 *      crossing, normal . w < 0 -> HIT else UNKNOWN; else (the ray passes
 *      behind the stored surface) -> UNKNOWN. The listing's highResolution-
 *      Tracing sends every crossing straight to the normal test; the text
 *      explains UNKNOWN by a ray that may start underneath the surface, read
 *      as the passes-behind branch. th < 0 selects the listing's two-way rule.
 *      Coarse texel: candidate iff r_hi >= dmin.
 *   R4 hit point (the listing returns the texel only): the first t >= ta at
 *      which the ray reaches the stored distance, r(t) = d, clamped to
 *      [ta, tb]; if the ray is behind the surface at ta and never comes back
 *      to d, the point of closest approach (clamped), or ta when it recedes.
 *      This is continuous in the data, unlike "a root inside [ta, tb], else
 *      ta", which jumps by a texel when a root sits at an interval end.
 *      Shading direction = (X + t w - O) / r; radiance bilinear over texel
 *      centres with the octahedral mirror border.
 *   R5 grid iterator: 3D DDA over cells (Amanatides & Woo 1987). The first
 *      visited cell starts at t = 0, the last one (where the ray leaves the
 *      grid) ends at t = infinity. Cage order: distance from the corner
 *      probe to X + t_in w, ties to the lower probe index. A probe's MISS
 *      ends the cell; UNKNOWN goes to the next probe; a cell whose 8 probes
 *      are all UNKNOWN sets sawUnknown. At grid exit: UNKNOWN if sawUnknown
 *      else MISS.
 *   R6 eye aligned: |X - O| < eye_eps -> HIT, radiance bilinear at oct(w)
 *      (eye_nearest: the listing's texelFetch, the value of the texel
 *      holding oct(w)).
 *   Fewer than 8 probes (traversal 1): probes nearest to the eye first, each
 *      over [0, inf), MISS or UNKNOWN falls through to the next.
 *
 * Texel walk along a segment: inside one octant both octahedral coordinates
 * are ratios of linear functions of t with a common denominator, so the
 * segment's image is a straight line and each texel-boundary crossing time is
 * the root of a linear equation. Texels are visited in order of t (2D DDA,
 * Amanatides & Woo); when both axes cross at the same t, x steps first.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_MISS = 0, ORC_HIT = 1, ORC_UNKNOWN = 2 };
enum { ORC_MARCH_FLAT = 0, ORC_MARCH_HIER = 1, ORC_MARCH_HIER_SHORTCUT = 2 };

typedef struct {
    int nx, ny, nz;
    double origin[3];
    double spacing;
    int N, M;               /* full map side, min/max mip side */
    double thickness_rel;   /* th in R3 */
    double eye_eps;         /* R6 */
    int march_mode;         /* ORC_MARCH_* */
    int eye_nearest;        /* eye-aligned lookup: 0 bilinear (R6), 1 the texel
                               holding oct(w) (the listing's texelFetch) */
    int traversal;          /* 0 grid iterator over cells (Sec. 4.3, grid
                               iterator); 1 fewer than 8 probes (Sec. 4.3): all
                               probes nearest to the eye first, each over the
                               whole ray, MISS or UNKNOWN -> next probe */
} orc_grid;

typedef struct {
    const float* dist;      /* [P][N][N]        */
    const float* normal;    /* [P][N][N][3]     */
    const float* radiance;  /* [P][N][N][3]     */
    const float* mip_min;   /* [P][M][M]        */
    const float* mip_max;   /* [P][M][M]        */
} orc_probes;

typedef struct {
    double pos[3], right[3], up[3], fwd[3];
    double fov_y;
    int W, H;
} orc_view;

/* Per-pixel result. */
typedef struct {
    int cls;                /* ORC_MISS / ORC_HIT / ORC_UNKNOWN */
    int probe;              /* hitting probe or -1 */
    int texel_i, texel_j;   /* fine texel that decided the HIT (or -1) */
    double uv[2];           /* shading coordinate in [0,1]^2 */
    double rgb[3];
    double t_hit;
    long long n_coarse, n_fine, n_normal, n_cells, n_probes;
} orc_result;

/* ------------------------------------------------------------------ */
/* small vector helpers                                                 */
/* ------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double sgn_nz(double v) { return v >= 0.0 ? 1.0 : -1.0; }

/* ------------------------------------------------------------------ */
/* Octahedral map (Sec. 3): direction -> unit sphere -> octahedron ->  */
/* unfold the lower octants onto the square [-1,1]^2 (R1).              */
/* ------------------------------------------------------------------ */
void orc_oct_encode(const double d[3], double p[2]) {
    double l1 = fabs(d[0]) + fabs(d[1]) + fabs(d[2]);
    double x = d[0] / l1, y = d[1] / l1;
    if (d[2] < 0.0) {
        double fx = (1.0 - fabs(y)) * sgn_nz(x);
        double fy = (1.0 - fabs(x)) * sgn_nz(y);
        x = fx;
        y = fy;
    }
    p[0] = x;
    p[1] = y;
}

void orc_oct_decode(const double p[2], double d[3]) {
    double x = p[0], y = p[1];
    double z = 1.0 - fabs(x) - fabs(y);
    if (z < 0.0) {
        double fx = (1.0 - fabs(y)) * sgn_nz(x);
        double fy = (1.0 - fabs(x)) * sgn_nz(y);
        x = fx;
        y = fy;
    }
    double l = sqrt(x * x + y * y + z * z);
    d[0] = x / l;
    d[1] = y / l;
    d[2] = z / l;
}

/* batch forms for tests */
void orc_oct_encode_n(long long n, const double* d, double* p) {
    for (long long k = 0; k < n; ++k) orc_oct_encode(d + 3 * k, p + 2 * k);
}
void orc_oct_decode_n(long long n, const double* p, double* d) {
    for (long long k = 0; k < n; ++k) orc_oct_decode(p + 2 * k, d + 3 * k);
}

/* Octahedral mirror border (R4): the square's edges fold onto themselves
 * reversed, so texel (-1, j) is texel (0, R-1-j), (R, j) is (R-1, R-1-j),
 * likewise for rows; past a corner, the diagonally opposite corner. */
void orc_mirror_texel(int R, int* i, int* j) {
    int ii = *i, jj = *j;
    if (ii < 0) { ii = 0; jj = R - 1 - jj; }
    else if (ii >= R) { ii = R - 1; jj = R - 1 - jj; }
    if (jj < 0) { jj = 0; ii = R - 1 - ii; }
    else if (jj >= R) { jj = R - 1; ii = R - 1 - ii; }
    *i = ii;
    *j = jj;
}

/* Bilinear radiance lookup at uv in [0,1]^2 over texel centres. Returns the
 * 4 mirrored texels and weights too (used by the adjoint). */
static void bilinear_taps(int N, const double uv[2], int ti[4], int tj[4], double w[4]) {
    double s = uv[0] * N - 0.5, t = uv[1] * N - 0.5;
    double fs = floor(s), ft = floor(t);
    int i0 = (int)fs, j0 = (int)ft;
    double a = s - fs, b = t - ft;
    int ci[4] = {i0, i0 + 1, i0, i0 + 1};
    int cj[4] = {j0, j0, j0 + 1, j0 + 1};
    double cw[4] = {(1 - a) * (1 - b), a * (1 - b), (1 - a) * b, a * b};
    for (int k = 0; k < 4; ++k) {
        int ii = ci[k], jj = cj[k];
        orc_mirror_texel(N, &ii, &jj);
        ti[k] = ii;
        tj[k] = jj;
        w[k] = cw[k];
    }
}

static void radiance_bilinear(const orc_grid* g, const orc_probes* pr, int probe,
                              const double uv[2], double rgb[3]) {
    int ti[4], tj[4];
    double w[4];
    bilinear_taps(g->N, uv, ti, tj, w);
    size_t base = (size_t)probe * g->N * g->N;
    rgb[0] = rgb[1] = rgb[2] = 0.0;
    for (int k = 0; k < 4; ++k) {
        const float* c = pr->radiance + 3 * (base + (size_t)tj[k] * g->N + ti[k]);
        for (int ch = 0; ch < 3; ++ch) rgb[ch] += w[k] * (double)c[ch];
    }
}

/* ------------------------------------------------------------------ */
/* Min/max mip (R2)                                                     */
/* ------------------------------------------------------------------ */
void orc_build_mip(int P, int N, int M, const float* dist, float* mip_min, float* mip_max) {
    int k = N / M;
    for (int p = 0; p < P; ++p)
        for (int J = 0; J < M; ++J)
            for (int I = 0; I < M; ++I) {
                float lo = INFINITY, hi = -INFINITY;
                for (int j = J * k; j < (J + 1) * k; ++j)
                    for (int i = I * k; i < (I + 1) * k; ++i) {
                        float v = dist[((size_t)p * N + j) * N + i];
                        if (v < lo) lo = v;
                        if (v > hi) hi = v;
                    }
                mip_min[((size_t)p * M + J) * M + I] = lo;
                mip_max[((size_t)p * M + J) * M + I] = hi;
            }
}

/* ------------------------------------------------------------------ */
/* A segment of the ray inside one octant of the probe, and its image   */
/* in octahedral coordinates: p_a(t) = (alpha_a + beta_a t) / (c + e t) */
/* ------------------------------------------------------------------ */
typedef struct {
    double Y0[3];           /* X - O */
    double w[3];            /* ray direction */
    double ta, tb;          /* segment */
    double s[3];            /* octant signs */
    double alpha[2], beta[2], c, e;
    int dir[2];             /* +1 / -1 / 0: motion of p_x, p_y with t */
} oseg;

static void seg_point(const oseg* sg, double t, double y[3]) {
    for (int a = 0; a < 3; ++a) y[a] = sg->Y0[a] + t * sg->w[a];
}

static double seg_radius(const oseg* sg, double t) {
    if (isinf(t)) return INFINITY;
    double y[3];
    seg_point(sg, t, y);
    return sqrt(dot3(y, y));
}

static void seg_setup(oseg* sg, const double Y0[3], const double w[3], double ta, double tb) {
    memcpy(sg->Y0, Y0, sizeof(sg->Y0));
    memcpy(sg->w, w, sizeof(sg->w));
    sg->ta = ta;
    sg->tb = tb;
    double tm = isinf(tb) ? ta + 1.0 : 0.5 * (ta + tb);
    double ym[3];
    seg_point(sg, tm, ym);
    for (int a = 0; a < 3; ++a) sg->s[a] = sgn_nz(ym[a]);
    sg->c = sg->s[0] * Y0[0] + sg->s[1] * Y0[1] + sg->s[2] * Y0[2];
    sg->e = sg->s[0] * w[0] + sg->s[1] * w[1] + sg->s[2] * w[2];
    for (int a = 0; a < 2; ++a) {
        if (sg->s[2] > 0.0) { /* upper hemisphere: p = (x, y) / |Y|_1 */
            sg->alpha[a] = Y0[a];
            sg->beta[a] = w[a];
        } else { /* lower hemisphere, folded: p_a = (Y_a + s_a s_z Y_z) / |Y|_1 */
            sg->alpha[a] = Y0[a] + sg->s[a] * sg->s[2] * Y0[2];
            sg->beta[a] = w[a] + sg->s[a] * sg->s[2] * w[2];
        }
        double slope = sg->beta[a] * sg->c - sg->alpha[a] * sg->e;
        sg->dir[a] = slope > 0.0 ? 1 : (slope < 0.0 ? -1 : 0);
    }
}

/* octahedral coordinate of the segment at time t, through the segment's own
 * octant formula: at a segment end that lies on one of the probe's planes the
 * general encoder may fold to the neighbouring octant, this never does */
static void seg_oct(const oseg* sg, double t, double p[2]) {
    double L = sg->c + sg->e * t;
    for (int a = 0; a < 2; ++a) p[a] = (sg->alpha[a] + sg->beta[a] * t) / L;
}

/* time at which p_a crosses the value B, or +inf if never on this branch */
static double seg_cross(const oseg* sg, int a, double B, double t_now) {
    double den = sg->beta[a] - B * sg->e;
    if (den == 0.0) return INFINITY;
    double t = (B * sg->c - sg->alpha[a]) / den;
    if (!isfinite(t)) return INFINITY;
    if (sg->c + sg->e * t <= 0.0) return INFINITY; /* other branch of the hyperbola */
    return t < t_now ? t_now : t;
}

static double boundary(int b, int R) { return (2.0 * b) / R - 1.0; }

/* index of the texel holding coordinate p at resolution R, for a walk that
 * moves in direction dir (a point on a boundary belongs to the texel ahead) */
static int texel_of(double p, int R, int dir) {
    double u = (p + 1.0) * 0.5 * R;
    int i = dir >= 0 ? (int)floor(u) : (int)ceil(u) - 1;
    if (i < 0) i = 0;
    if (i > R - 1) i = R - 1;
    return i;
}

/* 2D DDA over texels of resolution R along the segment between t0 and t1,
 * restricted to the index box [lo, hi]. visit() returns non-zero to stop. */
typedef int (*visit_fn)(void* ctx, int i, int j, double t0, double t1);

static int seg_walk(const oseg* sg, int R, double t0, double t1,
                    const int lo[2], const int hi[2], visit_fn visit, void* ctx) {
    double p[2];
    seg_oct(sg, t0, p);
    int idx[2];
    for (int a = 0; a < 2; ++a) {
        idx[a] = texel_of(p[a], R, sg->dir[a]);
        if (idx[a] < lo[a]) idx[a] = lo[a];
        if (idx[a] > hi[a]) idx[a] = hi[a];
    }
    double t = t0;
    for (int guard = 0; guard < 8 * R + 16; ++guard) {
        double tc[2];
        for (int a = 0; a < 2; ++a) {
            if (sg->dir[a] > 0) tc[a] = seg_cross(sg, a, boundary(idx[a] + 1, R), t);
            else if (sg->dir[a] < 0) tc[a] = seg_cross(sg, a, boundary(idx[a], R), t);
            else tc[a] = INFINITY;
        }
        double tn = tc[0] <= tc[1] ? tc[0] : tc[1];
        int last = tn >= t1;
        double tend = last ? t1 : tn;
        int r = visit(ctx, idx[0], idx[1], t, tend);
        if (r) return r;
        if (last) return 0;
        int a = tc[0] <= tc[1] ? 0 : 1; /* tie: x first */
        idx[a] += sg->dir[a];
        if (idx[a] < lo[a] || idx[a] > hi[a]) return 0;
        t = tend;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Texel tests (R3)                                                     */
/* ------------------------------------------------------------------ */
typedef struct {
    const orc_grid* g;
    const orc_probes* pr;
    int probe;
    const oseg* sg;
    double kappa;           /* thr(d) = d * kappa */
    int result;             /* ORC_* */
    int hit_i, hit_j;
    double hit_ta, hit_tb, hit_d;
    long long n_coarse, n_fine, n_normal;
} trace_ctx;

static void radial_range(const oseg* sg, double t0, double t1, double* r_lo, double* r_hi) {
    double a = seg_radius(sg, t0), b = seg_radius(sg, t1);
    *r_hi = a > b ? a : b;
    double tstar = -dot3(sg->Y0, sg->w) / dot3(sg->w, sg->w);
    if (tstar < t0) tstar = t0;
    if (tstar > t1) tstar = t1;
    *r_lo = seg_radius(sg, tstar);
}

/* highResolutionTracing, one fine texel */
static int fine_visit(void* vctx, int i, int j, double t0, double t1) {
    trace_ctx* cx = (trace_ctx*)vctx;
    const orc_grid* g = cx->g;
    size_t texel = ((size_t)cx->probe * g->N + j) * g->N + i;
    cx->n_fine++;
    double d = (double)cx->pr->dist[texel];
    double r_lo, r_hi;
    radial_range(cx->sg, t0, t1, &r_lo, &r_hi);
    if (r_hi < d) return 0; /* stored distance beyond the ray: keep marching */
    cx->hit_i = i;
    cx->hit_j = j;
    cx->hit_ta = t0;
    cx->hit_tb = t1;
    cx->hit_d = d;
    /* thickness_rel < 0 selects the listing's two-way rule: any crossing
     * goes to the normal test (no "passes behind" branch) */
    if (cx->g->thickness_rel < 0.0 || r_lo <= d * cx->kappa) {
        const float* n = cx->pr->normal + 3 * texel;
        cx->n_normal++;
        double nw = (double)n[0] * cx->sg->w[0] + (double)n[1] * cx->sg->w[1] + (double)n[2] * cx->sg->w[2];
        cx->result = nw < 0.0 ? ORC_HIT : ORC_UNKNOWN;
    } else {
        cx->result = ORC_UNKNOWN; /* the ray passes behind the stored surface */
    }
    return 1;
}

/* lowResolutionTracing, one coarse texel; on a candidate, run the
 * high-resolution tracing over the fine texels under it */
static int coarse_visit(void* vctx, int I, int J, double t0, double t1) {
    trace_ctx* cx = (trace_ctx*)vctx;
    const orc_grid* g = cx->g;
    size_t ct = ((size_t)cx->probe * g->M + J) * g->M + I;
    cx->n_coarse++;
    double dmin = (double)cx->pr->mip_min[ct];
    double r_lo, r_hi;
    radial_range(cx->sg, t0, t1, &r_lo, &r_hi);
    if (r_hi < dmin) return 0; /* no candidate in this coarse texel */
    if (g->march_mode == ORC_MARCH_HIER_SHORTCUT) {
        double dmax = (double)cx->pr->mip_max[ct];
        if (g->thickness_rel >= 0.0 && r_lo > dmax * cx->kappa) { /* every fine texel here is passed behind */
            cx->result = ORC_UNKNOWN;
            cx->hit_i = cx->hit_j = -1;
            return 1;
        }
    }
    int k = g->N / g->M;
    int lo[2] = {I * k, J * k}, hi[2] = {I * k + k - 1, J * k + k - 1};
    return seg_walk(cx->sg, g->N, t0, t1, lo, hi, fine_visit, cx);
}

/* traceOneRaySegment: low-resolution tracing to find a candidate coarse
 * texel, high-resolution tracing inside it, resume past it on MISS. The flat
 * RayMarching algorithm walks the full-resolution map instead. */
static int trace_one_ray_segment(trace_ctx* cx) {
    const orc_grid* g = cx->g;
    const oseg* sg = cx->sg;
    cx->result = ORC_MISS;
    if (g->march_mode == ORC_MARCH_FLAT) {
        int h = g->N / 2;
        int lo[2] = {sg->s[0] > 0 ? h : 0, sg->s[1] > 0 ? h : 0};
        int hi[2] = {sg->s[0] > 0 ? g->N - 1 : h - 1, sg->s[1] > 0 ? g->N - 1 : h - 1};
        seg_walk(sg, g->N, sg->ta, sg->tb, lo, hi, fine_visit, cx);
    } else {
        int h = g->M / 2;
        int lo[2] = {sg->s[0] > 0 ? h : 0, sg->s[1] > 0 ? h : 0};
        int hi[2] = {sg->s[0] > 0 ? g->M - 1 : h - 1, sg->s[1] > 0 ? g->M - 1 : h - 1};
        seg_walk(sg, g->M, sg->ta, sg->tb, lo, hi, coarse_visit, cx);
    }
    return cx->result;
}

static double clampd(double t, double lo, double hi) { return t < lo ? lo : (t > hi ? hi : t); }

/* Hit point (R4): |Y0 + t w|^2 = d^2 is A t^2 + 2 B t + C = 0. */
static double hit_time(const oseg* sg, double ta, double tb, double d) {
    double A = dot3(sg->w, sg->w), B = dot3(sg->Y0, sg->w), C = dot3(sg->Y0, sg->Y0) - d * d;
    double disc = B * B - A * C;
    if (seg_radius(sg, ta) < d) /* in front at ta: the ray enters the surface at the larger root */
        return clampd((-B + sqrt(disc > 0.0 ? disc : 0.0)) / A, ta, tb);
    double tstar = -B / A;          /* closest approach to the probe */
    if (tstar <= ta) return ta;     /* behind and receding */
    if (disc < 0.0) return clampd(tstar, ta, tb);
    return clampd((-B - sqrt(disc)) / A, ta, tb); /* approaching: the smaller root */
}

/* Octant split (Sec. 4.2: no more than four segments): cut [t0, t1] where the
 * ray crosses the probe's three axis planes. Returns the number of segments. */
int orc_split_segments(const double X[3], const double w[3], const double O[3],
                       double t0, double t1, double* bounds /* [5] */) {
    double cuts[3];
    int n = 0;
    for (int a = 0; a < 3; ++a) {
        if (w[a] == 0.0) continue;
        double t = (O[a] - X[a]) / w[a];
        if (t > t0 && t < t1) cuts[n++] = t;
    }
    for (int x = 1; x < n; ++x) /* sort the (at most 3) cut points */
        for (int y = x; y > 0 && cuts[y] < cuts[y - 1]; --y) {
            double tmp = cuts[y];
            cuts[y] = cuts[y - 1];
            cuts[y - 1] = tmp;
        }
    bounds[0] = t0;
    for (int k = 0; k < n; ++k) bounds[k + 1] = cuts[k];
    bounds[n + 1] = t1;
    return n + 1;
}

static void probe_position(const orc_grid* g, int probe, double O[3]) {
    int ix = probe % g->nx, iy = (probe / g->nx) % g->ny, iz = probe / (g->nx * g->ny);
    /* float32 positions, as every consumer of the grid description sees them */
    float o0 = (float)g->origin[0] + (float)g->spacing * (float)ix;
    float o1 = (float)g->origin[1] + (float)g->spacing * (float)iy;
    float o2 = (float)g->origin[2] + (float)g->spacing * (float)iz;
    O[0] = o0;
    O[1] = o1;
    O[2] = o2;
}

/* traceOneProbe over the ray interval [t0, t1]. */
static int trace_one_probe(const orc_grid* g, const orc_probes* pr, int probe,
                           const double X[3], const double w[3], double t0, double t1,
                           orc_result* res) {
    double O[3];
    probe_position(g, probe, O);
    double Y0[3] = {X[0] - O[0], X[1] - O[1], X[2] - O[2]};
    if (sqrt(dot3(Y0, Y0)) < g->eye_eps) {
        /* eye aligned with the probe: every point of the ray projects to
         * oct(w); look the radiance up directly (R6) */
        double p[2];
        orc_oct_encode(w, p);
        res->uv[0] = 0.5 * (p[0] + 1.0);
        res->uv[1] = 0.5 * (p[1] + 1.0);
        res->texel_i = texel_of(p[0], g->N, 1);
        res->texel_j = texel_of(p[1], g->N, 1);
        res->probe = probe;
        res->t_hit = 0.0;
        if (g->eye_nearest) { /* the texel's own value: sample at its centre */
            res->uv[0] = (res->texel_i + 0.5) / g->N;
            res->uv[1] = (res->texel_j + 0.5) / g->N;
        }
        radiance_bilinear(g, pr, probe, res->uv, res->rgb);
        return ORC_HIT;
    }
    double bounds[5];
    int nseg = orc_split_segments(X, w, O, t0, t1, bounds);
    for (int s = 0; s < nseg; ++s) {
        oseg sg;
        seg_setup(&sg, Y0, w, bounds[s], bounds[s + 1]);
        trace_ctx cx;
        memset(&cx, 0, sizeof(cx));
        cx.g = g;
        cx.pr = pr;
        cx.probe = probe;
        cx.sg = &sg;
        cx.kappa = 1.0 + 4.0 * g->thickness_rel / g->N;
        int r = trace_one_ray_segment(&cx);
        res->n_coarse += cx.n_coarse;
        res->n_fine += cx.n_fine;
        res->n_normal += cx.n_normal;
        if (r == ORC_MISS) continue; /* next segment */
        if (r == ORC_HIT) {
            double th = hit_time(&sg, cx.hit_ta, cx.hit_tb, cx.hit_d);
            double y[3], p[2];
            seg_point(&sg, th, y);
            orc_oct_encode(y, p);
            res->uv[0] = 0.5 * (p[0] + 1.0);
            res->uv[1] = 0.5 * (p[1] + 1.0);
            res->texel_i = cx.hit_i;
            res->texel_j = cx.hit_j;
            res->probe = probe;
            res->t_hit = th;
            radiance_bilinear(g, pr, probe, res->uv, res->rgb);
        }
        return r;
    }
    return ORC_MISS;
}

/* ------------------------------------------------------------------ */
/* Grid iterator (Sec. 4.3, R5)                                         */
/* ------------------------------------------------------------------ */
typedef struct {
    int c[3];
    double t_in, t_out;
} orc_cell;

static double cell_plane(const orc_grid* g, int a, int b) {
    float o = (float)g->origin[a] + (float)g->spacing * (float)b;
    return (double)o;
}

/* Cells crossed by the ray, in order. Returns the count (<= max_cells). */
int orc_grid_cells(const orc_grid* g, const double X[3], const double w[3],
                   orc_cell* out, int max_cells) {
    int nc[3] = {g->nx - 1, g->ny - 1, g->nz - 1};
    double t_enter = 0.0, t_exit = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double lo = cell_plane(g, a, 0), hi = cell_plane(g, a, nc[a]);
        if (w[a] == 0.0) {
            if (X[a] < lo || X[a] > hi) return 0;
            continue;
        }
        double ta = (lo - X[a]) / w[a], tb = (hi - X[a]) / w[a];
        if (ta > tb) { double tmp = ta; ta = tb; tb = tmp; }
        if (ta > t_enter) t_enter = ta;
        if (tb < t_exit) t_exit = tb;
    }
    if (t_enter > t_exit) return 0; /* the ray misses the grid */
    int c[3], step[3];
    double tmax[3];
    for (int a = 0; a < 3; ++a) {
        double p = X[a] + t_enter * w[a];
        int ci = (int)floor((p - g->origin[a]) / g->spacing);
        if (ci < 0) ci = 0;
        if (ci > nc[a] - 1) ci = nc[a] - 1;
        c[a] = ci;
        step[a] = w[a] > 0.0 ? 1 : (w[a] < 0.0 ? -1 : 0);
    }
    int n = 0;
    double t_in = 0.0;
    while (n < max_cells) {
        for (int a = 0; a < 3; ++a)
            tmax[a] = step[a] == 0 ? INFINITY
                                   : (cell_plane(g, a, c[a] + (step[a] > 0 ? 1 : 0)) - X[a]) / w[a];
        int a = 0;
        if (tmax[1] < tmax[a]) a = 1;
        if (tmax[2] < tmax[a]) a = 2;
        out[n].c[0] = c[0];
        out[n].c[1] = c[1];
        out[n].c[2] = c[2];
        out[n].t_in = t_in;
        int nxt = c[a] + step[a];
        if (step[a] == 0 || nxt < 0 || nxt > nc[a] - 1) {
            out[n].t_out = INFINITY; /* last cell: extends to infinity */
            return n + 1;
        }
        out[n].t_out = tmax[a];
        t_in = tmax[a];
        c[a] = nxt;
        ++n;
    }
    return n;
}

/* The 8 corner probes of a cell, nearest to P first (ties: lower index). */
void orc_cage_order(const orc_grid* g, const int c[3], const double P[3], int order[8]) {
    double dd[8];
    for (int k = 0; k < 8; ++k) {
        int ix = c[0] + (k & 1), iy = c[1] + ((k >> 1) & 1), iz = c[2] + ((k >> 2) & 1);
        order[k] = ix + g->nx * (iy + g->ny * iz);
        double O[3];
        probe_position(g, order[k], O);
        double v[3] = {P[0] - O[0], P[1] - O[1], P[2] - O[2]};
        dd[k] = sqrt(dot3(v, v));
    }
    for (int x = 1; x < 8; ++x)
        for (int y = x; y > 0 && (dd[y] < dd[y - 1] || (dd[y] == dd[y - 1] && order[y] < order[y - 1])); --y) {
            double td = dd[y]; dd[y] = dd[y - 1]; dd[y - 1] = td;
            int to = order[y]; order[y] = order[y - 1]; order[y - 1] = to;
        }
}

/* Fewer than 8 probes (Sec. 4.3): start from the probe closest to the eye
 * (ties: lower index); on MISS or UNKNOWN go to the next closest, each probe
 * over the whole ray [0, inf). No probe decides: UNKNOWN if one said
 * UNKNOWN, else MISS. */
static void trace_nearest_probes(const orc_grid* g, const orc_probes* pr, const double X[3], const double w[3],
                                 orc_result* res) {
    int P = g->nx * g->ny * g->nz;
    int* order = (int*)malloc(sizeof(int) * (size_t)P);
    double* dd = (double*)malloc(sizeof(double) * (size_t)P);
    for (int k = 0; k < P; ++k) {
        double O[3];
        probe_position(g, k, O);
        double v[3] = {X[0] - O[0], X[1] - O[1], X[2] - O[2]};
        dd[k] = sqrt(dot3(v, v));
        order[k] = k;
    }
    for (int x = 1; x < P; ++x)
        for (int y = x; y > 0 && dd[y] < dd[y - 1]; --y) {
            double td = dd[y]; dd[y] = dd[y - 1]; dd[y - 1] = td;
            int to = order[y]; order[y] = order[y - 1]; order[y - 1] = to;
        }
    int saw_unknown = 0, hit = 0;
    res->n_cells = 1;
    for (int k = 0; k < P && !hit; ++k) {
        res->n_probes++;
        int r = trace_one_probe(g, pr, order[k], X, w, 0.0, INFINITY, res);
        if (r == ORC_HIT) hit = 1;
        if (r == ORC_UNKNOWN) saw_unknown = 1;
    }
    free(order);
    free(dd);
    if (hit) { res->cls = ORC_HIT; return; }
    res->cls = saw_unknown ? ORC_UNKNOWN : ORC_MISS;
    res->probe = -1;
    res->texel_i = res->texel_j = -1;
}

/* Trace one ray through the grid. */
void orc_trace_ray(const orc_grid* g, const orc_probes* pr, const double X[3], const double w[3],
                   orc_result* res) {
    memset(res, 0, sizeof(*res));
    res->probe = -1;
    res->texel_i = res->texel_j = -1;
    if (g->traversal == 1) {
        trace_nearest_probes(g, pr, X, w, res);
        return;
    }
    orc_cell cells[1024];
    int ncell = orc_grid_cells(g, X, w, cells, 1024);
    int saw_unknown = 0;
    for (int ci = 0; ci < ncell; ++ci) {
        res->n_cells++;
        double P[3] = {X[0] + cells[ci].t_in * w[0], X[1] + cells[ci].t_in * w[1], X[2] + cells[ci].t_in * w[2]};
        int order[8];
        orc_cage_order(g, cells[ci].c, P, order);
        int n_unknown = 0;
        for (int k = 0; k < 8; ++k) {
            res->n_probes++;
            int r = trace_one_probe(g, pr, order[k], X, w, cells[ci].t_in, cells[ci].t_out, res);
            if (r == ORC_HIT) { res->cls = ORC_HIT; return; }
            if (r == ORC_MISS) break; /* this cell is empty along the ray */
            ++n_unknown;
        }
        if (n_unknown == 8) saw_unknown = 1;
    }
    res->cls = saw_unknown ? ORC_UNKNOWN : ORC_MISS;
    res->probe = -1;
    res->texel_i = res->texel_j = -1;
}

/* Pinhole ray through pixel (x, y). */
void orc_camera_ray(const orc_view* v, int x, int y, double X[3], double w[3]) {
    double th = tan(0.5 * v->fov_y);
    double a = ((x + 0.5) / v->W * 2.0 - 1.0) * th * v->W / v->H;
    double b = (1.0 - (y + 0.5) / v->H * 2.0) * th;
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = v->fwd[k] + a * v->right[k] + b * v->up[k];
    double l = sqrt(dot3(d, d));
    for (int k = 0; k < 3; ++k) {
        X[k] = v->pos[k];
        w[k] = d[k] / l;
    }
}

/* Render the listed pixels (or all when pixels == NULL) of one view.
 * Outputs are per listed pixel; any output pointer may be NULL. */
void orc_render(const orc_grid* g, const orc_probes* pr, const orc_view* v,
                long long n_pix, const long long* pixels,
                double* rgb, unsigned char* cls, int* aux_probe, double* aux_uv,
                int* hit_texel, double* t_hit, long long* counters /* [n_pix][5] */) {
#pragma omp parallel for schedule(dynamic, 64)
    for (long long k = 0; k < n_pix; ++k) {
        long long pix = pixels ? pixels[k] : k;
        int x = (int)(pix % v->W), y = (int)(pix / v->W);
        double X[3], w[3];
        orc_camera_ray(v, x, y, X, w);
        orc_result r;
        orc_trace_ray(g, pr, X, w, &r);
        if (rgb) for (int c = 0; c < 3; ++c) rgb[3 * k + c] = r.cls == ORC_HIT ? r.rgb[c] : 0.0;
        if (cls) cls[k] = (unsigned char)r.cls;
        if (aux_probe) aux_probe[k] = r.cls == ORC_HIT ? r.probe : -1;
        if (aux_uv) {
            aux_uv[2 * k] = r.cls == ORC_HIT ? r.uv[0] : 0.0;
            aux_uv[2 * k + 1] = r.cls == ORC_HIT ? r.uv[1] : 0.0;
        }
        if (hit_texel) {
            hit_texel[2 * k] = r.cls == ORC_HIT ? r.texel_i : -1;
            hit_texel[2 * k + 1] = r.cls == ORC_HIT ? r.texel_j : -1;
        }
        if (t_hit) t_hit[k] = r.cls == ORC_HIT ? r.t_hit : -1.0;
        if (counters) {
            counters[5 * k + 0] = r.n_coarse;
            counters[5 * k + 1] = r.n_fine;
            counters[5 * k + 2] = r.n_normal;
            counters[5 * k + 3] = r.n_cells;
            counters[5 * k + 4] = r.n_probes;
        }
    }
}

/* Trace arbitrary rays (X, w) (w need not be unit; it is normalised). */
void orc_trace_rays(const orc_grid* g, const orc_probes* pr, long long n, const double* X,
                    const double* W, double* rgb, unsigned char* cls, int* aux_probe,
                    double* aux_uv, int* hit_texel, double* t_hit) {
#pragma omp parallel for schedule(dynamic, 64)
    for (long long k = 0; k < n; ++k) {
        double w[3] = {W[3 * k], W[3 * k + 1], W[3 * k + 2]};
        double l = sqrt(dot3(w, w));
        for (int a = 0; a < 3; ++a) w[a] /= l;
        orc_result r;
        orc_trace_ray(g, pr, X + 3 * k, w, &r);
        if (rgb) for (int c = 0; c < 3; ++c) rgb[3 * k + c] = r.cls == ORC_HIT ? r.rgb[c] : 0.0;
        if (cls) cls[k] = (unsigned char)r.cls;
        if (aux_probe) aux_probe[k] = r.cls == ORC_HIT ? r.probe : -1;
        if (aux_uv) { aux_uv[2 * k] = r.uv[0]; aux_uv[2 * k + 1] = r.uv[1]; }
        if (hit_texel) { hit_texel[2 * k] = r.texel_i; hit_texel[2 * k + 1] = r.texel_j; }
        if (t_hit) t_hit[k] = r.cls == ORC_HIT ? r.t_hit : -1.0;
    }
}

/* One probe over one interval, for tests: returns the class and hit data. */
int orc_trace_one_probe(const orc_grid* g, const orc_probes* pr, int probe, const double X[3],
                        const double w[3], double t0, double t1, int* texel, double* uv, double* t_hit) {
    orc_result r;
    memset(&r, 0, sizeof(r));
    r.texel_i = r.texel_j = -1;
    int c = trace_one_probe(g, pr, probe, X, w, t0, t1, &r);
    texel[0] = r.texel_i;
    texel[1] = r.texel_j;
    uv[0] = r.uv[0];
    uv[1] = r.uv[1];
    *t_hit = r.t_hit;
    return c;
}

/* Walk one segment's texels at resolution R (tests): writes up to max
 * (i, j, t0, t1) records, returns the count. */
typedef struct { int n, max; int* ij; double* tt; } walk_rec;
static int record_visit(void* v, int i, int j, double t0, double t1) {
    walk_rec* w = (walk_rec*)v;
    if (w->n >= w->max) return 1;
    w->ij[2 * w->n] = i;
    w->ij[2 * w->n + 1] = j;
    w->tt[2 * w->n] = t0;
    w->tt[2 * w->n + 1] = t1;
    w->n++;
    return 0;
}
int orc_walk_segment(const double Y0[3], const double w[3], double ta, double tb, int R,
                     int max, int* ij, double* tt) {
    oseg sg;
    seg_setup(&sg, Y0, w, ta, tb);
    int h = R / 2;
    int lo[2] = {sg.s[0] > 0 ? h : 0, sg.s[1] > 0 ? h : 0};
    int hi[2] = {sg.s[0] > 0 ? R - 1 : h - 1, sg.s[1] > 0 ? R - 1 : h - 1};
    walk_rec rec = {0, max, ij, tt};
    seg_walk(&sg, R, ta, tb, lo, hi, record_visit, &rec);
    return rec.n;
}

/* ------------------------------------------------------------------ */
/* Adjoint: rgb is linear in radiance for fixed distance and normal maps,  */
/* so d rgb_c / d rad[p, texel_k, c] = w_k (the bilinear weight).          */
/* ------------------------------------------------------------------ */
void orc_backward(const orc_grid* g, long long n_pix, const double* grad_rgb,
                  const unsigned char* cls, const int* aux_probe, const double* aux_uv,
                  double* grad_rad /* [P][N][N][3], accumulated */) {
    for (long long k = 0; k < n_pix; ++k) {
        if (cls[k] != ORC_HIT || aux_probe[k] < 0) continue;
        int ti[4], tj[4];
        double w[4];
        bilinear_taps(g->N, aux_uv + 2 * k, ti, tj, w);
        size_t base = (size_t)aux_probe[k] * g->N * g->N;
        for (int q = 0; q < 4; ++q)
            for (int c = 0; c < 3; ++c)
                grad_rad[3 * (base + (size_t)tj[q] * g->N + ti[q]) + c] += w[q] * grad_rgb[3 * k + c];
    }
}

void orc_bilinear_taps(int N, const double* uv, int* ti, int* tj, double* w) {
    bilinear_taps(N, uv, ti, tj, w);
}

/* threads the OpenMP loops above run on (reported with CPU timings) */
#ifdef _OPENMP
#include <omp.h>
#endif
int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------
 * Probe maps from a point cloud (Sec. 4.1, simulated probe data; Sec. 5.1,
 * probe data generation), the plain definition in double precision. Every
 * point p is taken into the probe's frame, v = p - O, and onto the
 * octahedral map (R1, orc_oct_encode); its texel is (floor(u N), floor(w N))
 * of the square coordinate (u, w) = (enc(v) + 1) / 2, clamped to [0, N - 1].
 * Per texel the point nearest to the probe wins: smallest |v|^2, ties to the
 * lower point index. Distance = |v|, radiance = that point's colour, normal =
 * its normal when the cloud has normals, else the incoming direction
 * -v / |v| (R8). A texel no point reaches gets distance empty_dist, radiance
 * 0 and minus its texel-centre direction. A point at the probe (v = 0) has
 * no direction and is skipped. OpenMP over probes.
 *
 * Optional outputs for comparing a float32 implementation with it (any may
 * be NULL):
 *   winner  [P][N][N]  the winning point's index, -1 for an empty texel;
 *   decided [P][N][N]  1 where float32 rounding cannot change the winner,
 *                      0 where it can (see below);
 *   dcand   [P][N][N]  the least |v| over the points that float32 rounding
 *                      can put into the texel (+inf: none).
 * The margins follow from counting correctly rounded float32 operations
 * (unit roundoff 2^-24) in the recipe the GPU builder documents (v = p - O,
 * |v|^2 from three products and two sums; |v|_1 from two sums, one
 * reciprocal, two products, the fold, then (p + 1) N / 2): the texel
 * coordinate moves by at most 5.5 N 2^-24 texel widths, |v|^2 by at most
 * 5 2^-24 relative. With margins du = 8 N 2^-24 and dq = 16 2^-24, a point is
 * "near" a texel when it lies within du of it; a texel is undecided when a
 * point near one of its boundaries (inside or outside) is no farther than
 * its winner within dq (or the texel is empty), or when a second point
 * inside it ties with the winner within dq.
 */
static int splat_texel(const float p[3], const float O[3], int N, double* q, double v[3], double u[2]) {
    for (int a = 0; a < 3; ++a) v[a] = (double)p[a] - (double)O[a];
    double qq = dot3(v, v);
    double s = fabs(v[0]) + fabs(v[1]) + fabs(v[2]);
    if (!(s > 0.0) || !isfinite(s) || !isfinite(qq)) return -1;
    double e[2];
    orc_oct_encode(v, e);
    int ij[2];
    for (int a = 0; a < 2; ++a) {
        u[a] = (e[a] + 1.0) * 0.5 * N;
        int i = (int)floor(u[a]);
        ij[a] = i < 0 ? 0 : (i > N - 1 ? N - 1 : i);
    }
    *q = qq;
    return ij[0] + N * ij[1];
}

static int clamp_index(double x, int N) {
    int i = (int)floor(x);
    return i < 0 ? 0 : (i > N - 1 ? N - 1 : i);
}

void orc_splat_probes(long long n_points, const float* xyz, const float* rgb, const float* nrm, int n_probes,
                      const float* probe_pos, int N, float empty_dist, float* dist, float* normal,
                      float* radiance, long long* winner, unsigned char* decided, float* dcand) {
    const long long NN = (long long)N * N;
    const double eps32 = ldexp(1.0, -24);
    const double du = 8.0 * N * eps32, dq = 16.0 * eps32;
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < n_probes; ++p) {
        double* bq = (double*)malloc(sizeof(double) * (size_t)NN);
        long long* bk = (long long*)malloc(sizeof(long long) * (size_t)NN);
        for (long long t = 0; t < NN; ++t) {
            bq[t] = INFINITY;
            bk[t] = -1;
        }
        const float* O = probe_pos + 3 * p;
        for (long long k = 0; k < n_points; ++k) {
            double q, v[3], u[2];
            int t = splat_texel(xyz + 3 * k, O, N, &q, v, u);
            if (t < 0) continue;
            if (q < bq[t]) { /* points come in index order: an equal q keeps the lower index */
                bq[t] = q;
                bk[t] = k;
            }
        }
        for (long long t = 0; t < NN; ++t) {
            long long o = (long long)p * NN + t;
            if (winner) winner[o] = bk[t];
            if (bk[t] < 0) {
                double pp[2] = {((t % N) + 0.5) / N * 2.0 - 1.0, ((t / N) + 0.5) / N * 2.0 - 1.0}, d[3];
                orc_oct_decode(pp, d);
                dist[o] = empty_dist;
                for (int a = 0; a < 3; ++a) {
                    normal[3 * o + a] = (float)-d[a];
                    radiance[3 * o + a] = 0.0f;
                }
                continue;
            }
            long long k = bk[t];
            double q, v[3], u[2];
            splat_texel(xyz + 3 * k, O, N, &q, v, u);
            double r = sqrt(q);
            dist[o] = (float)r;
            for (int a = 0; a < 3; ++a) {
                normal[3 * o + a] = nrm ? nrm[3 * k + a] : (float)(-v[a] / r);
                radiance[3 * o + a] = rgb[3 * k + a];
            }
        }
        if (decided || dcand) {
            unsigned char* dec = (unsigned char*)malloc((size_t)NN);
            double* cq = (double*)malloc(sizeof(double) * (size_t)NN);
            for (long long t = 0; t < NN; ++t) {
                dec[t] = 1;
                cq[t] = bq[t];
            }
            for (long long k = 0; k < n_points; ++k) {
                double q, v[3], u[2];
                int t = splat_texel(xyz + 3 * k, O, N, &q, v, u);
                if (t < 0) continue;
                int ia = clamp_index(u[0] - du, N), ib = clamp_index(u[0] + du, N);
                int ja = clamp_index(u[1] - du, N), jb = clamp_index(u[1] + du, N);
                if (ia == ib && ja == jb) { /* the point stays in its texel */
                    if (k != bk[t] && q <= bq[t] * (1.0 + dq)) dec[t] = 0;
                    continue;
                }
                int is[2] = {ia, ib}, js[2] = {ja, jb};
                for (int x = 0; x < 2; ++x)
                    for (int y = 0; y < 2; ++y) {
                        long long tt = is[x] + (long long)N * js[y];
                        if (bk[tt] < 0 || q <= bq[tt] * (1.0 + dq)) dec[tt] = 0;
                        if (q < cq[tt]) cq[tt] = q;
                    }
            }
            for (long long t = 0; t < NN; ++t) {
                long long o = (long long)p * NN + t;
                if (decided) decided[o] = dec[t];
                if (dcand) dcand[o] = isinf(cq[t]) ? INFINITY : (float)sqrt(cq[t]);
            }
            free(dec);
            free(cq);
        }
        free(bq);
        free(bk);
    }
}

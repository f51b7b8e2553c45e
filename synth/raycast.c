/*
 * Seeded synthetic scenes: analytic ray casting against spheres, axis-aligned
 * boxes and a closed room, with Lambertian shading under directional lights.
 *
 * This file stands in for the capture pipeline of Sec. 5.1 (Probe Data
 * Generation): where the paper projects a scanned point cloud into each
 * probe's octahedral map and keeps the nearest point per texel, we cast one
 * ray per texel centre into an analytic scene and keep the nearest hit.
 * It is the input generator shared by the FP64 oracle and the CUDA path; it
 * holds no step of the probe tracer itself (no marching, no classification,
 * no shading lookup). The one convention it shares with both consumers is the
 * probe-map storage format: texel (i, j) of an N x N map holds the direction
 * obtained by unfolding the octahedral square point
 *   p = ((i + 0.5) / N * 2 - 1, (j + 0.5) / N * 2 - 1)
 * with +z as the pole (Sec. 3, octahedral mapping), stored row-major with
 * j as the row.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction,
 * so x86-64 and aarch64 hosts produce identical probe maps).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

typedef struct {
    int n_spheres;
    const double* spheres;     /* [n][7]: centre xyz, radius, albedo rgb      */
    int n_boxes;
    const double* boxes;       /* [n][9]: lo xyz, hi xyz, albedo rgb           */
    const double* room;        /* [6]: lo xyz, hi xyz (closed, inward walls)   */
    const double* wall_albedo; /* [6][3]: walls -x, +x, -y, +y, -z, +z         */
    int n_lights;
    const double* lights;      /* [n][4]: unit direction towards light, intensity */
    double ambient;
    /* optional uniform-grid accelerator over the objects (may be empty) */
    int acc_dims[3];           /* cells per axis; 0 = no accelerator */
    const double* acc_lo;      /* [3] */
    const double* acc_cell;    /* [3] cell size */
    const int* acc_start;      /* [cells + 1] offsets into acc_items */
    const int* acc_items;      /* object ids: spheres 0..ns-1, boxes ns.. */
} syn_scene;

#define SYN_NO_HIT (-1)

static int hit_sphere(const double* s, const double o[3], const double d[3],
                      double tmin, double tmax, double* t_out) {
    double oc[3] = {o[0] - s[0], o[1] - s[1], o[2] - s[2]};
    double a = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double b = oc[0] * d[0] + oc[1] * d[1] + oc[2] * d[2];
    double c = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - s[3] * s[3];
    double disc = b * b - a * c;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    double t0 = (-b - sq) / a;
    double t1 = (-b + sq) / a;
    if (t0 > tmin && t0 < tmax) { *t_out = t0; return 1; }
    if (t1 > tmin && t1 < tmax) { *t_out = t1; return 1; }
    return 0;
}

/* Slab test; returns entry axis (0..2) through *axis_out. */
static int hit_box(const double* b, const double o[3], const double d[3],
                   double tmin, double tmax, double* t_out, int* axis_out) {
    double t_enter = -INFINITY, t_exit = INFINITY;
    int ax_enter = 0;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < b[a] || o[a] > b[a + 3]) return 0;
            continue;
        }
        double ta = (b[a] - o[a]) / d[a];
        double tb = (b[a + 3] - o[a]) / d[a];
        if (ta > tb) { double tmp = ta; ta = tb; tb = tmp; }
        if (ta > t_enter) { t_enter = ta; ax_enter = a; }
        if (tb < t_exit) t_exit = tb;
    }
    if (t_enter > t_exit) return 0;
    if (t_enter > tmin && t_enter < tmax) { *t_out = t_enter; *axis_out = ax_enter; return 1; }
    return 0; /* origin inside the box or box behind: not a front hit */
}

static void object_hit(const syn_scene* sc, int id, const double o[3], const double d[3],
                       double tmin, double* best_t, int* best_id, int* best_axis) {
    double t;
    if (id < sc->n_spheres) {
        if (hit_sphere(sc->spheres + 7 * id, o, d, tmin, *best_t, &t)) {
            *best_t = t; *best_id = id; *best_axis = -1;
        }
    } else {
        int ax;
        if (hit_box(sc->boxes + 9 * (id - sc->n_spheres), o, d, tmin, *best_t, &t, &ax)) {
            *best_t = t; *best_id = id; *best_axis = ax;
        }
    }
}

/* Nearest object hit in (tmin, tmax); brute force or through the uniform grid. */
static void objects_nearest(const syn_scene* sc, const double o[3], const double d[3],
                            double tmin, double* best_t, int* best_id, int* best_axis) {
    int nobj = sc->n_spheres + sc->n_boxes;
    if (sc->acc_dims[0] <= 0) {
        for (int id = 0; id < nobj; ++id) object_hit(sc, id, o, d, tmin, best_t, best_id, best_axis);
        return;
    }
    /* 3D DDA over the accelerator cells (Amanatides & Woo 1987). Objects that
     * span several cells are tested more than once; the nearest is kept. */
    const int* dims = sc->acc_dims;
    const double* lo = sc->acc_lo;
    const double* cs = sc->acc_cell;
    double t0 = tmin, t1 = *best_t;
    for (int a = 0; a < 3; ++a) {
        double hi = lo[a] + cs[a] * dims[a];
        if (d[a] == 0.0) {
            if (o[a] < lo[a] || o[a] > hi) return;
            continue;
        }
        double ta = (lo[a] - o[a]) / d[a], tb = (hi - o[a]) / d[a];
        if (ta > tb) { double tmp = ta; ta = tb; tb = tmp; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    }
    if (t0 > t1) return;
    int c[3], step[3];
    double tmax_[3];
    for (int a = 0; a < 3; ++a) {
        double p = o[a] + t0 * d[a];
        int ci = (int)floor((p - lo[a]) / cs[a]);
        if (ci < 0) ci = 0;
        if (ci >= dims[a]) ci = dims[a] - 1;
        c[a] = ci;
        if (d[a] > 0.0) { step[a] = 1; tmax_[a] = (lo[a] + cs[a] * (ci + 1) - o[a]) / d[a]; }
        else if (d[a] < 0.0) { step[a] = -1; tmax_[a] = (lo[a] + cs[a] * ci - o[a]) / d[a]; }
        else { step[a] = 0; tmax_[a] = INFINITY; }
    }
    for (int guard = 0; guard < 1 << 20; ++guard) {
        int cell = c[0] + dims[0] * (c[1] + dims[1] * c[2]);
        for (int k = sc->acc_start[cell]; k < sc->acc_start[cell + 1]; ++k)
            object_hit(sc, sc->acc_items[k], o, d, tmin, best_t, best_id, best_axis);
        int a = 0;
        if (tmax_[1] < tmax_[a]) a = 1;
        if (tmax_[2] < tmax_[a]) a = 2;
        if (*best_t <= tmax_[a]) return; /* nearest hit lies in a visited cell */
        c[a] += step[a];
        if (c[a] < 0 || c[a] >= dims[a]) return;
        tmax_[a] = (lo[a] + cs[a] * (c[a] + (step[a] > 0 ? 1 : 0)) - o[a]) / d[a];
    }
}

/* Nearest surface along (o, d); the room is closed, so a ray that starts
 * inside it always hits something. Returns the primitive id: objects first
 * (spheres, then boxes), then walls as n_objects + wall index. */
static int cast_nearest(const syn_scene* sc, const double o[3], const double d[3],
                        double* t_out, double n_out[3], double albedo[3]) {
    /* room walls: exit distance of a ray that starts inside the room */
    double t_wall = INFINITY;
    int wall = 0;
    for (int a = 0; a < 3; ++a) {
        if (d[a] > 0.0) {
            double t = (sc->room[a + 3] - o[a]) / d[a];
            if (t < t_wall) { t_wall = t; wall = 2 * a + 1; }
        } else if (d[a] < 0.0) {
            double t = (sc->room[a] - o[a]) / d[a];
            if (t < t_wall) { t_wall = t; wall = 2 * a; }
        }
    }
    double best_t = t_wall;
    int best_id = SYN_NO_HIT, best_axis = -1;
    objects_nearest(sc, o, d, 0.0, &best_t, &best_id, &best_axis);
    *t_out = best_t;
    double p[3] = {o[0] + best_t * d[0], o[1] + best_t * d[1], o[2] + best_t * d[2]};
    int nobj = sc->n_spheres + sc->n_boxes;
    if (best_id == SYN_NO_HIT) {
        int a = wall / 2;
        n_out[0] = n_out[1] = n_out[2] = 0.0;
        n_out[a] = (wall & 1) ? -1.0 : 1.0; /* inward-facing wall */
        for (int k = 0; k < 3; ++k) albedo[k] = sc->wall_albedo[3 * wall + k];
        return nobj + wall;
    }
    if (best_id < sc->n_spheres) {
        const double* s = sc->spheres + 7 * best_id;
        double nn[3] = {p[0] - s[0], p[1] - s[1], p[2] - s[2]};
        double l = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        for (int k = 0; k < 3; ++k) { n_out[k] = nn[k] / l; albedo[k] = s[4 + k]; }
    } else {
        const double* b = sc->boxes + 9 * (best_id - sc->n_spheres);
        n_out[0] = n_out[1] = n_out[2] = 0.0;
        n_out[best_axis] = d[best_axis] > 0.0 ? -1.0 : 1.0; /* outward face */
        for (int k = 0; k < 3; ++k) albedo[k] = b[6 + k];
    }
    return best_id;
}

/* Distance from a point inside the room to the room's boundary along d. */
static double room_exit(const syn_scene* sc, const double o[3], const double d[3]) {
    double t_wall = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] > 0.0) {
            double t = (sc->room[a + 3] - o[a]) / d[a];
            if (t < t_wall) t_wall = t;
        } else if (d[a] < 0.0) {
            double t = (sc->room[a] - o[a]) / d[a];
            if (t < t_wall) t_wall = t;
        }
    }
    return t_wall;
}

/* Shadow rays test the objects only, up to where the ray leaves the room:
 * the walls do not block the directional lights (the room is lit as if
 * through an open ceiling), and object parts outside the room cast nothing. */
static int occluded(const syn_scene* sc, const double o[3], const double d[3]) {
    double best_t = room_exit(sc, o, d);
    int best_id = SYN_NO_HIT, best_axis = -1;
    objects_nearest(sc, o, d, 0.0, &best_t, &best_id, &best_axis);
    return best_id != SYN_NO_HIT;
}

static void shade(const syn_scene* sc, const double p[3], const double n[3],
                  const double albedo[3], double rgb[3]) {
    double e = sc->ambient;
    for (int l = 0; l < sc->n_lights; ++l) {
        const double* L = sc->lights + 4 * l;
        double ndl = n[0] * L[0] + n[1] * L[1] + n[2] * L[2];
        if (ndl <= 0.0) continue;
        double o[3] = {p[0] + 1e-7 * n[0], p[1] + 1e-7 * n[1], p[2] + 1e-7 * n[2]};
        if (occluded(sc, o, L)) continue;
        e += L[3] * ndl;
    }
    for (int k = 0; k < 3; ++k) rgb[k] = albedo[k] * e;
}

static void cast_one(const syn_scene* sc, const double o[3], const double d[3],
                     double* t, double n[3], double rgb[3], int* prim) {
    double albedo[3];
    *prim = cast_nearest(sc, o, d, t, n, albedo);
    double p[3] = {o[0] + *t * d[0], o[1] + *t * d[1], o[2] + *t * d[2]};
    shade(sc, p, n, albedo, rgb);
}

/* Ground-truth casts: n rays, directions need not be unit (t is in units of |d|). */
void syn_cast(const syn_scene* sc, long long n, const double* orig, const double* dir,
              double* t_out, double* n_out, double* rgb_out, int* prim_out) {
#pragma omp parallel for schedule(dynamic, 256)
    for (long long r = 0; r < n; ++r) {
        double t, nn[3], rgb[3];
        int prim;
        cast_one(sc, orig + 3 * r, dir + 3 * r, &t, nn, rgb, &prim);
        t_out[r] = t;
        for (int k = 0; k < 3; ++k) {
            if (n_out) n_out[3 * r + k] = nn[k];
            if (rgb_out) rgb_out[3 * r + k] = rgb[k];
        }
        if (prim_out) prim_out[r] = prim;
    }
}

/* Texel-centre direction of the probe-map storage format (see file header). */
static void texel_direction(int N, int i, int j, double d[3]) {
    double x = (i + 0.5) / N * 2.0 - 1.0;
    double y = (j + 0.5) / N * 2.0 - 1.0;
    double z = 1.0 - fabs(x) - fabs(y);
    if (z < 0.0) {
        double fx = (1.0 - fabs(y)) * (x >= 0.0 ? 1.0 : -1.0);
        double fy = (1.0 - fabs(x)) * (y >= 0.0 ? 1.0 : -1.0);
        x = fx;
        y = fy;
    }
    double l = sqrt(x * x + y * y + z * z);
    d[0] = x / l;
    d[1] = y / l;
    d[2] = z / l;
}

void syn_texel_directions(int N, double* out /* [N][N][3] */) {
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) texel_direction(N, i, j, out + 3 * ((size_t)j * N + i));
}

/* Probe maps for P probes at N x N: distance [P][N][N], surface normal
 * [P][N][N][3] (unit, world space, facing the probe side of the surface),
 * radiance [P][N][N][3]. One ray per texel centre, nearest hit kept. */
void syn_probe_maps(const syn_scene* sc, int P, const double* probe_pos, int N,
                    float* dist, float* normal, float* radiance) {
    long long total = (long long)P * N * N;
#pragma omp parallel for schedule(dynamic, 1024)
    for (long long idx = 0; idx < total; ++idx) {
        int p = (int)(idx / ((long long)N * N));
        int rem = (int)(idx % ((long long)N * N));
        int j = rem / N, i = rem % N;
        double d[3], t, nn[3], rgb[3];
        int prim;
        texel_direction(N, i, j, d);
        cast_one(sc, probe_pos + 3 * p, d, &t, nn, rgb, &prim);
        dist[idx] = (float)t;
        for (int k = 0; k < 3; ++k) {
            normal[3 * idx + k] = (float)nn[k];
            radiance[3 * idx + k] = (float)rgb[k];
        }
    }
}

/* A laser-scanner sweep from one position, in the order a scanner records
 * it: n_az azimuth columns (azimuth phase + 2 pi (a + 1/2) / n_az), each a
 * vertical sweep of n_el directions with polar angle theta_max (e + 1/2) /
 * n_el from the zenith (theta_max = 150 deg for a 300 deg vertical field:
 * the cone under the tripod stays unseen). Point k = a n_el + e is the
 * nearest hit of that direction, with its radiance and surface normal
 * (float32). */
void syn_scan(const syn_scene* sc, const double* pos, int n_az, int n_el, double phase, double theta_max,
              float* xyz, float* rgb, float* nrm) {
    const double two_pi = 2.0 * 3.14159265358979323846;
    const long long n = (long long)n_az * n_el;
#pragma omp parallel for schedule(dynamic, 1024)
    for (long long k = 0; k < n; ++k) {
        int a = (int)(k / n_el), e = (int)(k % n_el);
        double phi = phase + two_pi * (a + 0.5) / n_az;
        double th = theta_max * (e + 0.5) / n_el;
        double d[3] = {sin(th) * cos(phi), sin(th) * sin(phi), cos(th)};
        double t, nn[3], c[3];
        int prim;
        cast_one(sc, pos, d, &t, nn, c, &prim);
        for (int q = 0; q < 3; ++q) {
            xyz[3 * k + q] = (float)(pos[q] + t * d[q]);
            rgb[3 * k + q] = (float)c[q];
            nrm[3 * k + q] = (float)nn[q];
        }
    }
}

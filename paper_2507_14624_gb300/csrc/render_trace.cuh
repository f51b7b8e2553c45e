// The per-ray tracer of the forward render (device code shared by the
// render kernels).
//
// Per ray (Sec. 3 problem statement; Sec. 4.2-4.3; Appendix A):
//   grid iterator (3D DDA over cells, first cell from t = 0, last to infinity)
//   -> cage: the cell's 8 corner probes, nearest to the cell entry point first
//   -> traceOneProbe: eye aligned -> direct lookup; else split [t_in, t_out]
//      at the probe's axis planes into <= 4 single-octant segments
//   -> traceOneRaySegment: low-resolution walk over the min/max map; a coarse
//      texel is a candidate when the ray's farthest radius reaches its min
//      distance, a sure UNKNOWN when its nearest radius is behind max * kappa;
//      candidates get the full-resolution walk (highResolutionTracing)
//   -> HIT: bilinear radiance at the hit direction; MISS ends the cell;
//      UNKNOWN tries the next probe.
// Inside one octant the segment's octahedral image is p_a(t) = (alpha_a +
// beta_a t) / (c + e t), a straight line: the walks are 2D DDAs whose
// boundary-crossing times solve a linear equation. All boundaries are
// expressed in full-resolution texel units so low- and full-resolution walks
// share exact crossing times.
#pragma once
#include <cuda_runtime.h>

#include "lfp_device.cuh"

namespace lfp {
namespace trace {

constexpr float kInf = __builtin_huge_valf();

struct Ray {
    float3 X, w;
};

struct Seg {
    float3 Y0;         // X - O
    float3 w;
    float tstar;       // closest approach of the ray to the probe
    float c, e;        // denominator c + e t (the octant's L1 norm)
    float al[2], be[2];// numerators alpha + beta t
    int dir[2];        // motion of p_x, p_y along the segment
    int lo[2], hi[2];  // quadrant of the square (full-resolution indices)
};

struct Decision {
    int cls;           // kMiss / kHit / kUnknown
    int i, j;          // deciding full-resolution texel (HIT)
    float ta, tb, d;   // its interval and stored distance (HIT)
};

__device__ __forceinline__ float r2_at(const Seg& s, float t) {
    if (!(t < kInf)) return kInf;
    float x = fmaf(t, s.w.x, s.Y0.x), y = fmaf(t, s.w.y, s.Y0.y), z = fmaf(t, s.w.z, s.Y0.z);
    return x * x + y * y + z * z;
}

__device__ __forceinline__ float boundary(const Seg& s, int b, int N) {
    return __fdiv_rn(2.0f * (float)b, (float)N) - 1.0f;
}

// time at which p_a reaches B, or +inf if it never does on this branch
__device__ __forceinline__ float cross_time(const Seg& s, int a, float B, float tnow) {
    float den = s.be[a] - B * s.e;
    float t = (B * s.c - s.al[a]) / den;
    if (!(fabsf(t) < kInf)) return kInf;
    if (!(s.c + s.e * t > 0.0f)) return kInf;
    return fmaxf(t, tnow);
}

// full-resolution texel index of p along axis a for a walk moving in dir
__device__ __forceinline__ int texel_of(float p, int N, int dir) {
    float u = (p + 1.0f) * 0.5f * (float)N;
    int i = dir >= 0 ? (int)floorf(u) : (int)ceilf(u) - 1;
    return min(max(i, 0), N - 1);
}

__device__ __forceinline__ void seg_setup(Seg& s, float3 Y0, float3 w, float ta, float tb, int N) {
    s.Y0 = Y0;
    s.w = w;
    s.tstar = -(Y0.x * w.x + Y0.y * w.y + Y0.z * w.z) / (w.x * w.x + w.y * w.y + w.z * w.z);
    float tm = (tb < kInf) ? 0.5f * (ta + tb) : ta + 1.0f;
    float ym[3] = {fmaf(tm, w.x, Y0.x), fmaf(tm, w.y, Y0.y), fmaf(tm, w.z, Y0.z)};
    float sg[3] = {sgn_nz(ym[0]), sgn_nz(ym[1]), sgn_nz(ym[2])};
    float y0[3] = {Y0.x, Y0.y, Y0.z}, ww[3] = {w.x, w.y, w.z};
    s.c = sg[0] * y0[0] + sg[1] * y0[1] + sg[2] * y0[2];
    s.e = sg[0] * ww[0] + sg[1] * ww[1] + sg[2] * ww[2];
    int h = N / 2;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        if (sg[2] > 0.0f) {
            s.al[a] = y0[a];
            s.be[a] = ww[a];
        } else {  // folded lower octant: p_a = (Y_a + s_a s_z Y_z) / |Y|_1
            float f = sg[a] * sg[2];
            s.al[a] = y0[a] + f * y0[2];
            s.be[a] = ww[a] + f * ww[2];
        }
        float slope = s.be[a] * s.c - s.al[a] * s.e;
        s.dir[a] = slope > 0.0f ? 1 : (slope < 0.0f ? -1 : 0);
        s.lo[a] = sg[a] > 0.0f ? h : 0;
        s.hi[a] = sg[a] > 0.0f ? N - 1 : h - 1;
    }
}

template <bool COUNT>
struct Stats {
    unsigned coarse = 0, fine = 0, normal = 0, steps = 0;
};

// highResolutionTracing over full-resolution texels inside the index box
// [lo, hi] between t0 and t1. Returns true when a decision was reached.
template <int NRMF, bool COUNT>
__device__ bool fine_walk(const GridDev& g, const Seg& s, size_t pbase, float t0, float t1,
                          int lo0, int lo1, int hi0, int hi1, float r2a, Decision& out,
                          Stats<COUNT>& st, bool& step_limited) {
    const int N = g.N;
    float L0 = s.c + s.e * t0;
    int i = texel_of((s.al[0] + s.be[0] * t0) / L0, N, s.dir[0]);
    int j = texel_of((s.al[1] + s.be[1] * t0) / L0, N, s.dir[1]);
    i = min(max(i, lo0), hi0);
    j = min(max(j, lo1), hi1);
    float tx = s.dir[0] > 0 ? cross_time(s, 0, boundary(s, i + 1, N), t0)
             : s.dir[0] < 0 ? cross_time(s, 0, boundary(s, i, N), t0) : kInf;
    float ty = s.dir[1] > 0 ? cross_time(s, 1, boundary(s, j + 1, N), t0)
             : s.dir[1] < 0 ? cross_time(s, 1, boundary(s, j, N), t0) : kInf;
    float t = t0;
    for (int guard = 0; guard < 4 * N + 8; ++guard) {
        float tn = fminf(tx, ty);
        bool last = !(tn < t1);
        float te = last ? t1 : tn;
        float r2b = r2_at(s, te);
        float d = __ldg(g.dist + pbase + (size_t)j * N + i);
        if (COUNT) st.fine++;
        st.steps++;
        if (g.max_steps > 0 && (int)st.steps >= g.max_steps) { step_limited = true; return true; }
        if (!(fmaxf(r2a, r2b) < d * d)) {
            out.i = i;
            out.j = j;
            out.ta = t;
            out.tb = te;
            out.d = d;
            float tl = fminf(fmaxf(s.tstar, t), te);
            float r2lo = r2_at(s, tl);
            float dk = d * g.kappa;
            if (g.two_way || r2lo <= dk * dk) {
                float2 no = NrmTexel<NRMF>::load(g.nrm, pbase + (size_t)j * N + i);
                float3 n = oct_decode_unnorm(no.x, no.y);
                if (COUNT) st.normal++;
                out.cls = (n.x * s.w.x + n.y * s.w.y + n.z * s.w.z) < 0.0f ? kHit : kUnknown;
            } else {
                out.cls = kUnknown;  // the ray passes behind the stored surface
            }
            return true;
        }
        if (last) return false;
        if (tx <= ty) {
            i += s.dir[0];
            if (i < lo0 || i > hi0) return false;
            tx = cross_time(s, 0, boundary(s, s.dir[0] > 0 ? i + 1 : i, N), te);
        } else {
            j += s.dir[1];
            if (j < lo1 || j > hi1) return false;
            ty = cross_time(s, 1, boundary(s, s.dir[1] > 0 ? j + 1 : j, N), te);
        }
        t = te;
        r2a = r2b;
    }
    return false;
}

// traceOneRaySegment: low-resolution walk; full-resolution walk in candidates.
template <int NRMF, bool COUNT>
__device__ bool trace_segment(const GridDev& g, const Seg& s, int probe, float ta, float tb, bool flat,
                              Decision& out, Stats<COUNT>& st, bool& step_limited) {
    const int N = g.N, M = g.M, k = g.k;
    size_t pbase = (size_t)probe * N * N;
    float r2a = r2_at(s, ta);
    if (flat)  // Appendix A RayMarching: the full-resolution map only
        return fine_walk<NRMF, COUNT>(g, s, pbase, ta, tb, s.lo[0], s.lo[1], s.hi[0], s.hi[1], r2a, out, st,
                                      step_limited);
    const float2* mip = g.mip + (size_t)probe * M * M;
    float L0 = s.c + s.e * ta;
    int I = texel_of((s.al[0] + s.be[0] * ta) / L0, N, s.dir[0]) / k;
    int J = texel_of((s.al[1] + s.be[1] * ta) / L0, N, s.dir[1]) / k;
    int clo0 = s.lo[0] / k, chi0 = s.hi[0] / k, clo1 = s.lo[1] / k, chi1 = s.hi[1] / k;
    I = min(max(I, clo0), chi0);
    J = min(max(J, clo1), chi1);
    float tx = s.dir[0] > 0 ? cross_time(s, 0, boundary(s, (I + 1) * k, N), ta)
             : s.dir[0] < 0 ? cross_time(s, 0, boundary(s, I * k, N), ta) : kInf;
    float ty = s.dir[1] > 0 ? cross_time(s, 1, boundary(s, (J + 1) * k, N), ta)
             : s.dir[1] < 0 ? cross_time(s, 1, boundary(s, J * k, N), ta) : kInf;
    float t = ta;
    for (int guard = 0; guard < 4 * M + 8; ++guard) {
        float tn = fminf(tx, ty);
        bool last = !(tn < tb);
        float te = last ? tb : tn;
        float r2b = r2_at(s, te);
        float2 mm = __ldg(mip + (size_t)J * M + I);
        if (COUNT) st.coarse++;
        st.steps++;
        if (g.max_steps > 0 && (int)st.steps >= g.max_steps) { step_limited = true; return true; }
        if (!(fmaxf(r2a, r2b) < mm.x * mm.x)) {  // candidate coarse texel
            bool behind = false;
            if (!g.two_way) {
                float tl = fminf(fmaxf(s.tstar, t), te);
                float dk = mm.y * g.kappa;
                behind = r2_at(s, tl) > dk * dk;
            }
            if (behind) {  // every full-resolution texel under it is passed behind
                out.cls = kUnknown;
                out.i = out.j = -1;
                return true;
            }
            if (fine_walk<NRMF, COUNT>(g, s, pbase, t, te, I * k, J * k, I * k + k - 1, J * k + k - 1, r2a, out,
                                       st, step_limited))
                return true;
        }
        if (last) return false;
        if (tx <= ty) {
            I += s.dir[0];
            if (I < clo0 || I > chi0) return false;
            tx = cross_time(s, 0, boundary(s, (s.dir[0] > 0 ? I + 1 : I) * k, N), te);
        } else {
            J += s.dir[1];
            if (J < clo1 || J > chi1) return false;
            ty = cross_time(s, 1, boundary(s, (s.dir[1] > 0 ? J + 1 : J) * k, N), te);
        }
        t = te;
        r2a = r2b;
    }
    return false;
}

__device__ __forceinline__ float3 probe_pos(const GridDev& g, int p) {
    int ix = p % g.nx, iy = (p / g.nx) % g.ny, iz = p / (g.nx * g.ny);
    return make_float3(grid_plane(g.ox, g.spacing, ix), grid_plane(g.oy, g.spacing, iy),
                       grid_plane(g.oz, g.spacing, iz));
}

// traceOneProbe over [t0, t1]: split at the probe's axis planes (at most 4
// single-octant segments, Sec. 4.2); the first non-MISS segment decides.
template <int NRMF, bool COUNT>
__device__ void trace_probe(const GridDev& g, const Ray& r, int probe, float t0, float t1, bool flat,
                            Decision& out, Seg& hit_seg, Stats<COUNT>& st, bool& step_limited) {
    float3 O = probe_pos(g, probe);
    float3 Y0 = make_float3(r.X.x - O.x, r.X.y - O.y, r.X.z - O.z);
    float cut[3];
    int nc = 0;
    const float Xa[3] = {r.X.x, r.X.y, r.X.z}, Wa[3] = {r.w.x, r.w.y, r.w.z}, Oa[3] = {O.x, O.y, O.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (Wa[a] != 0.0f) {
            float tc = (Oa[a] - Xa[a]) / Wa[a];
            if (tc > t0 && tc < t1) cut[nc++] = tc;
        }
    }
    // sort the <= 3 cut points
    if (nc > 1 && cut[1] < cut[0]) { float x = cut[0]; cut[0] = cut[1]; cut[1] = x; }
    if (nc > 2 && cut[2] < cut[1]) {
        float x = cut[1]; cut[1] = cut[2]; cut[2] = x;
        if (cut[1] < cut[0]) { x = cut[0]; cut[0] = cut[1]; cut[1] = x; }
    }
    out.cls = kMiss;
    float a = t0;
    for (int sgi = 0; sgi <= nc; ++sgi) {
        float b = sgi < nc ? cut[sgi] : t1;
        Seg s;
        seg_setup(s, Y0, r.w, a, b, g.N);
        if (trace_segment<NRMF, COUNT>(g, s, probe, a, b, flat, out, st, step_limited)) {
            hit_seg = s;
            return;
        }
        a = b;
    }
    out.cls = kMiss;
}

// Hit point: the first t >= ta with |Y0 + t w| = d, clamped to [ta, tb];
// when the ray is behind the stored surface at ta it is the smaller root if
// the ray comes back to d, else the closest approach (ta when receding).
// |Y0 + t w|^2 = d^2 is A t^2 + 2 B t + C = 0; the roots use the
// cancellation-free forms.
__device__ __forceinline__ float hit_time(const Seg& s, float ta, float tb, float d) {
    float A = s.w.x * s.w.x + s.w.y * s.w.y + s.w.z * s.w.z;
    float B = s.Y0.x * s.w.x + s.Y0.y * s.w.y + s.Y0.z * s.w.z;
    float y0 = sqrtf(s.Y0.x * s.Y0.x + s.Y0.y * s.Y0.y + s.Y0.z * s.Y0.z);
    float C = (y0 - d) * (y0 + d);
    float sq = sqrtf(fmaxf(B * B - A * C, 0.0f));
    float t;
    if (r2_at(s, ta) < d * d) {
        t = B > 0.0f ? -C / (B + sq) : (sq - B) / A;  // larger root
    } else {
        float tstar = -B / A;
        if (!(tstar > ta)) return ta;
        if (B * B - A * C < 0.0f) t = tstar;
        else t = B < 0.0f ? C / (sq - B) : -(B + sq) / A;  // smaller root
    }
    return fminf(fmaxf(t, ta), tb);
}

template <int RADF>
__device__ __forceinline__ float3 shade(const GridDev& g, int probe, float u, float v) {
    int idx[4];
    float w[4];
    bilinear_taps(g.N, u, v, idx, w);
    size_t base = (size_t)probe * g.N * g.N;
    float3 c = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float3 t = RadTexel<RADF>::load(g.rad, base + idx[q]);
        c.x = fmaf(w[q], t.x, c.x);
        c.y = fmaf(w[q], t.y, c.y);
        c.z = fmaf(w[q], t.z, c.z);
    }
    return c;
}

struct PixelResult {
    int cls, probe, texel;
    float u, v;
    float3 rgb;
};

template <int RADF, int NRMF, bool COUNT>
__device__ PixelResult trace_ray(const GridDev& g, const Ray& r, bool flat, Stats<COUNT>& st,
                                 unsigned& cells, unsigned& probes) {
    PixelResult res;
    res.cls = kMiss;
    res.probe = -1;
    res.texel = -1;
    res.u = res.v = 0.f;
    res.rgb = make_float3(0.f, 0.f, 0.f);
    const int nc[3] = {g.nx - 1, g.ny - 1, g.nz - 1};
    const float og[3] = {g.ox, g.oy, g.oz};
    const float Xa[3] = {r.X.x, r.X.y, r.X.z}, Wa[3] = {r.w.x, r.w.y, r.w.z};

    // Eye aligned with a probe (Sec. 4.2, Appendix A traceOneProbe): the
    // nearest grid vertex within eye_eps is looked up at oct(w) directly.
    {
        int iv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) iv[a] = min(max((int)rintf((Xa[a] - og[a]) / g.spacing), 0), nc[a]);
        int p = iv[0] + g.nx * (iv[1] + g.ny * iv[2]);
        float3 O = probe_pos(g, p);
        float dx = Xa[0] - O.x, dy = Xa[1] - O.y, dz = Xa[2] - O.z;
        if (sqrtf(dx * dx + dy * dy + dz * dz) < g.eye_eps) {
            float2 pp = oct_encode(r.w.x, r.w.y, r.w.z);
            res.cls = kHit;
            res.probe = p;
            res.u = 0.5f * (pp.x + 1.0f);
            res.v = 0.5f * (pp.y + 1.0f);
            res.texel = texel_of(pp.x, g.N, 1) + g.N * texel_of(pp.y, g.N, 1);
            res.rgb = shade<RADF>(g, p, res.u, res.v);
            cells = 1;
            probes = 1;
            return res;
        }
    }

    // Grid iterator (Sec. 4.3): 3D DDA over the cells the ray crosses.
    float t_enter = 0.0f, t_exit = kInf;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float lo = grid_plane(og[a], g.spacing, 0), hi = grid_plane(og[a], g.spacing, nc[a]);
        if (Wa[a] == 0.0f) {
            if (Xa[a] < lo || Xa[a] > hi) t_enter = kInf;
            continue;
        }
        float ta = (lo - Xa[a]) / Wa[a], tb = (hi - Xa[a]) / Wa[a];
        if (ta > tb) { float x = ta; ta = tb; tb = x; }
        t_enter = fmaxf(t_enter, ta);
        t_exit = fminf(t_exit, tb);
    }
    if (!(t_enter <= t_exit)) return res;  // the ray misses the grid: MISS
    int c[3], step[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float p = fmaf(t_enter, Wa[a], Xa[a]);
        c[a] = min(max((int)floorf((p - og[a]) / g.spacing), 0), nc[a] - 1);
        step[a] = Wa[a] > 0.0f ? 1 : (Wa[a] < 0.0f ? -1 : 0);
    }
    bool saw_unknown = false, step_limited = false;
    float t_in = 0.0f;
    for (int guard = 0; guard < nc[0] + nc[1] + nc[2] + 3; ++guard) {
        float tm[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            tm[a] = step[a] == 0 ? kInf
                                 : (grid_plane(og[a], g.spacing, c[a] + (step[a] > 0 ? 1 : 0)) - Xa[a]) / Wa[a];
        int ax = 0;
        if (tm[1] < tm[ax]) ax = 1;
        if (tm[2] < tm[ax]) ax = 2;
        int nxt = c[ax] + step[ax];
        bool last_cell = step[ax] == 0 || nxt < 0 || nxt > nc[ax] - 1;
        float t_out = last_cell ? kInf : tm[ax];
        cells++;

        // cage: 8 corner probes, nearest to the entry point first, ties to
        // the lower probe index (corner k has index order k)
        float3 P = make_float3(fmaf(t_in, r.w.x, r.X.x), fmaf(t_in, r.w.y, r.X.y), fmaf(t_in, r.w.z, r.X.z));
        float dd[8];
        int ord[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            int p = (c[0] + (q & 1)) + g.nx * ((c[1] + ((q >> 1) & 1)) + g.ny * (c[2] + ((q >> 2) & 1)));
            float3 O = probe_pos(g, p);
            float dx = P.x - O.x, dy = P.y - O.y, dz = P.z - O.z;
            dd[q] = dx * dx + dy * dy + dz * dz;
            ord[q] = p;
        }
#pragma unroll
        for (int x = 1; x < 8; ++x) {
#pragma unroll
            for (int y = x; y > 0; --y) {
                bool sw = dd[y] < dd[y - 1];
                float fd = sw ? dd[y - 1] : dd[y];
                float fe = sw ? dd[y] : dd[y - 1];
                int oa = sw ? ord[y - 1] : ord[y];
                int ob = sw ? ord[y] : ord[y - 1];
                dd[y] = fd; dd[y - 1] = fe;
                ord[y] = oa; ord[y - 1] = ob;
            }
        }
        int n_unknown = 0;
        for (int q = 0; q < 8; ++q) {
            Decision dec;
            Seg hs;
            probes++;
            trace_probe<NRMF, COUNT>(g, r, ord[q], t_in, t_out, flat, dec, hs, st, step_limited);
            if (step_limited) {
                res.cls = kStepLimit;
                return res;
            }
            if (dec.cls == kHit) {
                float th = hit_time(hs, dec.ta, dec.tb, dec.d);
                float yx = fmaf(th, hs.w.x, hs.Y0.x), yy = fmaf(th, hs.w.y, hs.Y0.y), yz = fmaf(th, hs.w.z, hs.Y0.z);
                float2 pp = oct_encode(yx, yy, yz);
                res.cls = kHit;
                res.probe = ord[q];
                res.u = 0.5f * (pp.x + 1.0f);
                res.v = 0.5f * (pp.y + 1.0f);
                res.texel = dec.i + g.N * dec.j;
                res.rgb = shade<RADF>(g, ord[q], res.u, res.v);
                return res;
            }
            if (dec.cls == kMiss) break;
            ++n_unknown;
        }
        if (n_unknown == 8) saw_unknown = true;
        if (last_cell) break;
        t_in = t_out;
        c[ax] = nxt;
    }
    res.cls = saw_unknown ? kUnknown : kMiss;
    return res;
}

}  // namespace trace
}  // namespace lfp

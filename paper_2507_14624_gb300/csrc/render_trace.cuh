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
constexpr float kFarCuts = 1048576.0f;  // 2^20 grid spacings: octant cuts beyond are dropped

struct Ray {
    float3 X, w;
};

// One octant segment [ta, tb] of the ray relative to a probe, walked in the
// projective parameter u = tau / (c + e tau), tau = t - ta: inside an octant
// the octahedral coordinates p_a = (alpha_a + beta_a tau) / (c + e tau) are
// affine in u, p_a = p0_a + k_a u, so the crossing of texel boundary b
// (p = 2 b / N - 1) is u = b m_a + q_a, one multiply-add. The radial test
// r(tau) < d becomes |Ya + u V|^2 < d^2 (1 - e u)^2 with V = c w - e Ya
// (because Ya + tau w = (Ya + u V) / (1 - e u)): no division per texel.
struct Seg {
    float3 Ya;         // X + ta w - O
    float3 w;
    float cp, e;       // L1 norm of the octant along the segment: cp + e tau, cp > 0
    float m[2], q[2];  // boundary crossing u = b m + q (full-resolution b)
    float p0[2], k[2]; // p_a(u) = p0 + k u
    float A0, A1, A2;  // |Ya + u V|^2 = A0 + u (A1 + u A2)
    float u_end;
    float tstar;       // closest approach to the probe (tau)
    float ustar;       // the same point in u (0 before the segment, +inf past the octant's reach)
    int dir[2];        // motion of p_x, p_y with u
    int lo[2], hi[2];  // quadrant of the square (full-resolution indices)
};

struct Decision {
    int cls;           // kMiss / kHit / kUnknown
    int texel;         // deciding full-resolution texel i + N j (HIT)
    float u, v;        // shading coordinate in [0,1]^2 (HIT)
};

// full-resolution texel index of p along an axis for a walk moving in dir
__device__ __forceinline__ int texel_of(float p, int N, int dir) {
    float u = (p + 1.0f) * 0.5f * (float)N;
    int i = dir >= 0 ? (int)floorf(u) : (int)ceilf(u) - 1;
    return min(max(i, 0), N - 1);
}

__device__ __forceinline__ void seg_setup(Seg& s, float3 Y0, float3 w, float ta, float tb, int N) {
    float3 Ya = make_float3(fmaf(ta, w.x, Y0.x), fmaf(ta, w.y, Y0.y), fmaf(ta, w.z, Y0.z));
    s.Ya = Ya;
    s.w = w;
    float tm = (tb < kInf) ? 0.5f * (tb - ta) : 1.0f;
    float sg[3] = {sgn_nz(fmaf(tm, w.x, Ya.x)), sgn_nz(fmaf(tm, w.y, Ya.y)), sgn_nz(fmaf(tm, w.z, Ya.z))};
    float ya[3] = {Ya.x, Ya.y, Ya.z}, ww[3] = {w.x, w.y, w.z};
    float cp = sg[0] * ya[0] + sg[1] * ya[1] + sg[2] * ya[2];
    float e = sg[0] * ww[0] + sg[1] * ww[1] + sg[2] * ww[2];
    cp = fmaxf(cp, 1e-30f);  // the ray starts on the probe only in degenerate cases
    s.cp = cp;
    s.e = e;
    const int h = N / 2;
    const float two_n = 2.0f / (float)N;
    const float icp = __frcp_rn(cp);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        float al, be;
        if (sg[2] > 0.0f) {
            al = ya[a];
            be = ww[a];
        } else {  // folded lower octant: p_a = (Y_a + s_a s_z Y_z) / |Y|_1
            float f = sg[a] * sg[2];
            al = ya[a] + f * ya[2];
            be = ww[a] + f * ww[2];
        }
        float p0 = al * icp;
        float k = (be * cp - al * e) * icp;
        float ik = __frcp_rn(k);
        s.p0[a] = p0;
        s.k[a] = k;
        s.dir[a] = k > 0.0f ? 1 : (k < 0.0f ? -1 : 0);
        s.m[a] = two_n * ik;
        s.q[a] = -(1.0f + p0) * ik;
        s.lo[a] = sg[a] > 0.0f ? h : 0;
        s.hi[a] = sg[a] > 0.0f ? N - 1 : h - 1;
    }
    float3 V = make_float3(cp * w.x - e * Ya.x, cp * w.y - e * Ya.y, cp * w.z - e * Ya.z);
    s.A0 = Ya.x * Ya.x + Ya.y * Ya.y + Ya.z * Ya.z;
    s.A1 = 2.0f * (Ya.x * V.x + Ya.y * V.y + Ya.z * V.z);
    s.A2 = V.x * V.x + V.y * V.y + V.z * V.z;
    float te = tb - ta;
    s.u_end = (te < kInf) ? te * __frcp_rn(fmaf(e, te, cp)) : __frcp_rn(e);
    s.tstar = -(Ya.x * w.x + Ya.y * w.y + Ya.z * w.z);  // w is a unit vector (every caller normalises the ray)
    // u = tau / (cp + e tau) grows with tau wherever cp + e tau > 0, so the
    // closest approach clamped to a tau-interval is u* clamped to its u-interval
    const float Ls = fmaf(e, s.tstar, cp);
    s.ustar = !(s.tstar > 0.0f) ? 0.0f : (Ls > 0.0f ? __fdividef(s.tstar, Ls) : kInf);
}

// Does the ray come within dk of the probe over the walk interval [u0, u1]?
// min r = r(clamp(tau*, ta, tb)), and r^2 = |Ya + u V|^2 / (1 - e u)^2, so in
// u it is A(uc) <= dk^2 D(uc)^2 at uc = clamp(u*, u0, u1): no division.
__device__ __forceinline__ bool comes_within(float A0, float A1, float A2, float e, float ustar, float u0, float u1,
                                             float dk) {
    const float uc = fminf(fmaxf(ustar, u0), u1);
    const float P = fmaf(fmaf(A2, uc, A1), uc, A0);
    const float D = fmaf(-e, uc, 1.0f);
    return P <= (dk * dk) * (D * D);
}

// u of the next boundary crossed along axis a from index i (full resolution)
__device__ __forceinline__ float next_cross(const Seg& s, int a, int i, float u_now) {
    if (s.dir[a] == 0) return kInf;
    int b = s.dir[a] > 0 ? i + 1 : i;
    return fmaxf(fmaf((float)b, s.m[a], s.q[a]), u_now);
}

// tau of walk parameter u (infinite past the end). D is in (0, 1], so the
// fast division (2 ulp, no special-case path) is exact enough and keeps the
// walk loop's code short.
__device__ __forceinline__ float tau_of(const Seg& s, float u) {
    float D = fmaf(-s.e, u, 1.0f);
    return D > 0.0f ? __fdividef(s.cp * u, D) : kInf;
}

__device__ __forceinline__ float r2_tau(const Seg& s, float tau) {
    float x = fmaf(tau, s.w.x, s.Ya.x), y = fmaf(tau, s.w.y, s.Ya.y), z = fmaf(tau, s.w.z, s.Ya.z);
    return x * x + y * y + z * z;
}

// Hit point (tau from the segment start): the first tau >= ta with
// |Ya + tau w| = d, clamped to [ta, tb]; when the ray is behind the stored
// surface at ta it is the smaller root if the ray comes back to d, else the
// closest approach (ta when receding). |Ya + tau w|^2 = d^2 is
// A tau^2 + 2 B tau + C = 0; the roots use the cancellation-free forms.
__device__ __forceinline__ float hit_time(const Seg& s, float ta, float tb, float d) {
    float A = s.w.x * s.w.x + s.w.y * s.w.y + s.w.z * s.w.z;
    float B = s.Ya.x * s.w.x + s.Ya.y * s.w.y + s.Ya.z * s.w.z;
    float y0 = sqrtf(s.A0);
    float C = (y0 - d) * (y0 + d);
    float sq = sqrtf(fmaxf(B * B - A * C, 0.0f));
    float t;
    if (r2_tau(s, ta) < d * d) {
        t = B > 0.0f ? fdiv(-C, B + sq) : fdiv(sq - B, A);  // larger root
    } else {
        float tstar = fdiv(-B, A);
        if (!(tstar > ta)) return ta;
        if (B * B - A * C < 0.0f) t = tstar;
        else t = B < 0.0f ? fdiv(C, sq - B) : fdiv(-(B + sq), A);  // smaller root
    }
    return fminf(fmaxf(t, ta), tb);
}

template <bool COUNT>
struct Stats {
    unsigned coarse = 0, fine = 0, normal = 0, steps = 0;
};

// Where the full-resolution walk under a candidate low-resolution texel
// [u0, u1] can start: until the ray's radial distance first reaches the
// block's minimum dmin (d2 = dmin^2) every full-resolution texel is in front
// of its stored surface. f(u) = |Ya + u V|^2 - d2 (1 - e u)^2 is quadratic
// with f0 = f(u0) < 0 <= f1 = f(u1) when there is anything to skip; the
// estimate of its root never lies beyond it: the chord's zero when f is
// convex, the zero of the tangent at u0 when f is concave, then shortened by
// 1/256 of the skipped length to cover rounding.
__device__ __forceinline__ float fine_start(const Seg& s, float d2, float u0, float f0, float u1, float f1) {
    if (!(f0 < 0.0f) || !(f1 >= 0.0f) || !(u1 > u0)) return u0;
    const float a = fmaf(-__fmul_rn(d2, s.e), s.e, s.A2);
    float us;
    if (a >= 0.0f) {
        us = fmaf(u1 - u0, __fdividef(-f0, f1 - f0), u0);
    } else {
        const float fp = fmaf(2.0f * a, u0, fmaf(2.0f * d2, s.e, s.A1));
        if (!(fp > 0.0f)) return u0;
        us = u0 - __fdividef(f0, fp);
    }
    us = fmaf(us - u0, 255.0f / 256.0f, u0);
    return fminf(fmaxf(us, u0), u1);
}

// Where a segment's low-resolution walk can start. dq is
// the least distance stored in the segment's quadrant of the map: while the
// ray's radial distance stays below dq it is in front of every texel there,
// so the walk starts where it first reaches dq (the fine_start estimate over
// the whole segment, never past that point). f(u) = A(u) - dq^2 D(u)^2 is
// |Ya + tau w|^2 - dq^2 up to a positive factor, convex in tau: negative at
// both ends means negative throughout, and `walk` is false (the segment is a
// MISS without a visit). Returns 0 when the ray starts at or beyond dq.
__device__ __forceinline__ float segment_start(const Seg& s, float dq, bool& walk) {
    walk = true;
    const float d2q = dq * dq;
    const float f0 = fmaf(-d2q, 1.0f, s.A0);
    if (!(f0 < 0.0f)) return 0.0f;
    const float ue = s.u_end;
    const float De = fmaf(-s.e, ue, 1.0f);
    const float f1 = fmaf(-d2q, De * De, fmaf(fmaf(s.A2, ue, s.A1), ue, s.A0));
    if (!(f1 >= 0.0f)) {
        walk = false;
        return 0.0f;
    }
    return fine_start(s, d2q, 0.0f, f0, ue, f1);
}

// highResolutionTracing over full-resolution texels inside the index box
// [lo, hi] for u in [u0, u1]. P0, D20: |Ya + u0 V|^2 and (1 - e u0)^2.
// Returns true when a decision was reached.
template <int NRMF, bool COUNT>
__device__ bool fine_walk(const GridDev& g, const Seg& s, size_t pbase, float u0, float u1, float P0, float D20,
                          int lo0, int lo1, int hi0, int hi1, Decision& out, Stats<COUNT>& st, bool& step_limited) {
    const int N = g.N;
    int i = min(max(texel_of(fmaf(s.k[0], u0, s.p0[0]), N, s.dir[0]), lo0), hi0);
    int j = min(max(texel_of(fmaf(s.k[1], u0, s.p0[1]), N, s.dir[1]), lo1), hi1);
    float ux = next_cross(s, 0, i, u0), uy = next_cross(s, 1, j, u0);
    float u = u0, Pa = P0, D2a = D20;
    for (int guard = 0; guard < 4 * N + 8; ++guard) {
        float un = fminf(ux, uy);
        bool last = !(un < u1);
        float ue = last ? u1 : un;
        float Pb = fmaf(fmaf(s.A2, ue, s.A1), ue, s.A0);
        float Db = fmaf(-s.e, ue, 1.0f);
        float D2b = Db * Db;
        int ic = i, jc = j;
        LFP_CHECK_TEXEL(g.flags, (unsigned)ic < (unsigned)N && (unsigned)jc < (unsigned)N, ic, jc);
        float d = __ldg(g.dist + pbase + (size_t)jc * N + ic);
        float d2 = d * d;
        if (COUNT) st.fine++;
        st.steps++;
        if (g.max_steps > 0 && (int)st.steps >= g.max_steps) { step_limited = true; return true; }
        if (!(Pa < d2 * D2a && Pb < d2 * D2b)) {  // the ray reaches the stored distance
            out.cls = kUnknown;  // unless the normal test passes below
            if (g.two_way || comes_within(s.A0, s.A1, s.A2, s.e, s.ustar, u, ue, d * g.kappa)) {
                float2 no = NrmTexel<NRMF>::load(g.nrm, pbase + (size_t)jc * N + ic);
                float3 n = oct_decode_unnorm(no.x, no.y);
                if (COUNT) st.normal++;
                if ((n.x * s.w.x + n.y * s.w.y + n.z * s.w.z) < 0.0f) {
                    float th = hit_time(s, tau_of(s, u), tau_of(s, ue), d);
                    float2 pp = oct_encode(fmaf(th, s.w.x, s.Ya.x), fmaf(th, s.w.y, s.Ya.y), fmaf(th, s.w.z, s.Ya.z));
                    out.cls = kHit;
                    out.texel = i + N * j;
                    out.u = 0.5f * (pp.x + 1.0f);
                    out.v = 0.5f * (pp.y + 1.0f);
                }
            }  // else the ray passes behind the stored surface: UNKNOWN
            return true;
        }
        if (last) return false;
        if (ux <= uy) {
            i += s.dir[0];
            if (i < lo0 || i > hi0) return false;
            ux = next_cross(s, 0, i, ue);
        } else {
            j += s.dir[1];
            if (j < lo1 || j > hi1) return false;
            uy = next_cross(s, 1, j, ue);
        }
        u = ue;
        Pa = Pb;
        D2a = D2b;
    }
    return false;
}

// traceOneRaySegment: low-resolution walk; full-resolution walk in candidates.
template <int NRMF, bool COUNT, bool FLAT>
__device__ bool trace_segment(const GridDev& g, const Seg& s, int probe, Decision& out, Stats<COUNT>& st,
                              bool& step_limited) {
    const int N = g.N, M = g.M, k = g.k;
    {
        int unused = 0;
        LFP_CHECK_TEXEL(g.flags, (unsigned)probe < (unsigned)(g.nx * g.ny * g.nz), probe, unused);
        (void)unused;
    }
    size_t pbase = (size_t)probe * N * N;
    if (FLAT)  // Appendix A RayMarching: the full-resolution map only
        return fine_walk<NRMF, COUNT>(g, s, pbase, 0.0f, s.u_end, s.A0, 1.0f, s.lo[0], s.lo[1], s.hi[0], s.hi[1],
                                      out, st, step_limited);
    const float* mip = g.mip + (size_t)probe * 2 * M * M;  // min plane; the max plane follows it
    float u;
    {
        bool walk;
        const int quad = (s.lo[0] > 0 ? 1 : 0) | (s.lo[1] > 0 ? 2 : 0);
        u = segment_start(s, __ldg(g.qmin + (size_t)probe * 4 + quad), walk);
        if (!walk) return false;
    }
    int clo0 = div_k(g.kinv, s.lo[0]), chi0 = div_k(g.kinv, s.hi[0]);
    int clo1 = div_k(g.kinv, s.lo[1]), chi1 = div_k(g.kinv, s.hi[1]);
    int I = min(max(div_k(g.kinv, texel_of(fmaf(s.k[0], u, s.p0[0]), N, s.dir[0])), clo0), chi0);
    int J = min(max(div_k(g.kinv, texel_of(fmaf(s.k[1], u, s.p0[1]), N, s.dir[1])), clo1), chi1);
    // coarse boundaries are full-resolution boundaries b = I k: same crossings
    float ux = s.dir[0] == 0 ? kInf : fmaxf(fmaf((float)((s.dir[0] > 0 ? I + 1 : I) * k), s.m[0], s.q[0]), u);
    float uy = s.dir[1] == 0 ? kInf : fmaxf(fmaf((float)((s.dir[1] > 0 ? J + 1 : J) * k), s.m[1], s.q[1]), u);
    const float Du = fmaf(-s.e, u, 1.0f);
    float Pa = fmaf(fmaf(s.A2, u, s.A1), u, s.A0), D2a = Du * Du;
    const float u1 = s.u_end;
    for (int guard = 0; guard < 4 * M + 8; ++guard) {
        float un = fminf(ux, uy);
        bool last = !(un < u1);
        float ue = last ? u1 : un;
        float Pb = fmaf(fmaf(s.A2, ue, s.A1), ue, s.A0);
        float Db = fmaf(-s.e, ue, 1.0f);
        float D2b = Db * Db;
        int Ic = I, Jc = J;
        LFP_CHECK_TEXEL(g.flags, (unsigned)Ic < (unsigned)M && (unsigned)Jc < (unsigned)M, Ic, Jc);
        const float dmin = __ldg(mip + (size_t)Jc * M + Ic);
        float d2 = dmin * dmin;
        if (COUNT) st.coarse++;
        st.steps++;
        if (g.max_steps > 0 && (int)st.steps >= g.max_steps) { step_limited = true; return true; }
        if (!(Pa < d2 * D2a && Pb < d2 * D2b)) {  // candidate coarse texel
            if (!g.two_way &&
                !comes_within(s.A0, s.A1, s.A2, s.e, s.ustar, u, ue, __ldg(mip + (size_t)(M + Jc) * M + Ic) * g.kappa)) {
                out.cls = kUnknown;  // every full-resolution texel under it is passed behind
                return true;
            }
            // explicit multiply-adds: both engines round the start alike
            const float us = fine_start(s, d2, u, fmaf(-d2, D2a, Pa), ue, fmaf(-d2, D2b, Pb));
            const float Ds = fmaf(-s.e, us, 1.0f);
            if (fine_walk<NRMF, COUNT>(g, s, pbase, us, ue, fmaf(fmaf(s.A2, us, s.A1), us, s.A0), Ds * Ds, I * k, J * k,
                                       I * k + k - 1, J * k + k - 1, out, st, step_limited))
                return true;
        }
        if (last) return false;
        if (ux <= uy) {
            I += s.dir[0];
            if (I < clo0 || I > chi0) return false;
            ux = fmaxf(fmaf((float)((s.dir[0] > 0 ? I + 1 : I) * k), s.m[0], s.q[0]), ue);
        } else {
            J += s.dir[1];
            if (J < clo1 || J > chi1) return false;
            uy = fmaxf(fmaf((float)((s.dir[1] > 0 ? J + 1 : J) * k), s.m[1], s.q[1]), ue);
        }
        u = ue;
        Pa = Pb;
        D2a = D2b;
    }
    return false;
}

__device__ __forceinline__ float3 probe_pos(const GridDev& g, int p) {
    int ix = p % g.nx, iy = (p / g.nx) % g.ny, iz = p / (g.nx * g.ny);
    return make_float3(grid_plane(g.ox, g.spacing, ix), grid_plane(g.oy, g.spacing, iy),
                       grid_plane(g.oz, g.spacing, iz));
}

// Position and index of corner kq (bit a: +1 along axis a) of cell (c0, c1, c2).
__device__ __forceinline__ float3 corner_pos(const GridDev& g, int c0, int c1, int c2, int kq) {
    return make_float3(grid_plane(g.ox, g.spacing, c0 + (kq & 1)), grid_plane(g.oy, g.spacing, c1 + ((kq >> 1) & 1)),
                       grid_plane(g.oz, g.spacing, c2 + (kq >> 2)));
}
__device__ __forceinline__ int corner_index(const GridDev& g, int c0, int c1, int c2, int kq) {
    return (c0 + (kq & 1)) + g.nx * ((c1 + ((kq >> 1) & 1)) + g.ny * (c2 + (kq >> 2)));
}

// Cage order (8-probe cage, nearest corner to the entry point P first).
// Along each axis the squared distance of a corner is one of two values, so
// d^2(corner) = d^2(nearest) + sum of g_a over the axes where the corner
// differs from the nearest one, g_a = |dhi_a^2 - dlo_a^2|. With the axes
// sorted by g (a1 <= a2 <= a3) the order is fixed except for one comparison:
// n, n^a1, n^a2, {n^a3, n^a1a2}, n^a1a3, n^a2a3, n^a1a2a3.
// Returns the corner of rank q in bits [3q, 3q + 3).
__device__ __forceinline__ unsigned cage_order(const GridDev& g, int c0, int c1, int c2, float3 P) {
    float3 lo = corner_pos(g, c0, c1, c2, 0), hi = corner_pos(g, c0, c1, c2, 7);
    float dl, dh, ga[3];
    int n = 0;
    dl = P.x - lo.x; dh = P.x - hi.x; dl *= dl; dh *= dh; n |= dh < dl ? 1 : 0; ga[0] = fabsf(dh - dl);
    dl = P.y - lo.y; dh = P.y - hi.y; dl *= dl; dh *= dh; n |= dh < dl ? 2 : 0; ga[1] = fabsf(dh - dl);
    dl = P.z - lo.z; dh = P.z - hi.z; dl *= dl; dh *= dh; n |= dh < dl ? 4 : 0; ga[2] = fabsf(dh - dl);
    // sort the three axes by g, ties to the lower axis
    int a1 = 0, a2 = 1, a3 = 2;
    float g1 = ga[0], g2 = ga[1], g3 = ga[2];
    if (g2 < g1) { float t = g1; g1 = g2; g2 = t; int i = a1; a1 = a2; a2 = i; }
    if (g3 < g2) {
        float t = g2; g2 = g3; g3 = t; int i = a2; a2 = a3; a3 = i;
        if (g2 < g1) { t = g1; g1 = g2; g2 = t; i = a1; a1 = a2; a2 = i; }
    }
    const unsigned m1 = 1u << a1, m2 = 1u << a2, m3 = 1u << a3, un = (unsigned)n;
    const bool single_first = g3 < g1 + g2;
    unsigned r3 = un ^ (single_first ? m3 : (m1 | m2));
    unsigned r4 = un ^ (single_first ? (m1 | m2) : m3);
    return un | ((un ^ m1) << 3) | ((un ^ m2) << 6) | (r3 << 9) | (r4 << 12) | ((un ^ (m1 | m3)) << 15) |
           ((un ^ (m2 | m3)) << 18) | ((un ^ 7u) << 21);
}

// Traversal for fewer than 8 probes (Sec. 4.3): every probe ordered by the
// squared distance to the eye X (ties to the lower index), corner of rank q
// in bits [3q, 3q + 3).
__device__ __forceinline__ unsigned nearest_order(const GridDev& g, float3 X) {
    const int P = g.nx * g.ny * g.nz;  // <= 8, checked at grid creation
    float d2[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float3 O = probe_pos(g, k < P ? k : 0);
        float dx = __fsub_rn(X.x, O.x), dy = __fsub_rn(X.y, O.y), dz = __fsub_rn(X.z, O.z);
        d2[k] = k < P ? __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)) : kInf;
    }
    unsigned used = 0, order = 0;
    for (int q = 0; q < P; ++q) {
        int pick = -1;
        float best = kInf;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (!(used >> k & 1u) && k < P && (pick < 0 || d2[k] < best)) {
                best = d2[k];
                pick = k;
            }
        used |= 1u << pick;
        order |= (unsigned)pick << (3 * q);
    }
    return order;
}

// Constants of a view's primary rays. They all start at the camera X, so
// the eye-aligned test (Sec. 4.2), the grid entry when X lies in the closed
// probe box (every direction enters at t = 0, in the cell holding X) and
// that cell's cage order from X -- or, for the traversal with fewer than 8
// probes, the nearest-probe order -- are the same for every ray of the
// view: computed once per view or tile with the arithmetic the per-ray code
// uses, so no decision changes.
struct ViewStart {
    int eye_probe;   // probe within eye_eps of X, else -1
    int inside;      // grid traversal: X in the closed probe box
    int c[3];        // the cell holding X
    unsigned order;  // that cell's cage order from X, or the nearest-probe order
};

// nearest: the traversal for fewer than 8 probes (a compile-time constant
// where the caller knows it, so the other branch folds away)
__device__ __forceinline__ ViewStart view_start(const GridDev& g, float3 X, bool nearest) {
    ViewStart vs;
    const int nc[3] = {g.nx - 1, g.ny - 1, g.nz - 1};
    const float og[3] = {g.ox, g.oy, g.oz}, Xa[3] = {X.x, X.y, X.z};
    // eye aligned: the nearest grid vertex within eye_eps
    int iv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) iv[a] = min(max((int)rintf(fdiv(Xa[a] - og[a], g.spacing)), 0), nc[a]);
    const float3 O = corner_pos(g, iv[0], iv[1], iv[2], 0);
    const float ex = X.x - O.x, ey = X.y - O.y, ez = X.z - O.z;
    vs.eye_probe = sqrtf(ex * ex + ey * ey + ez * ez) < g.eye_eps ? iv[0] + g.nx * (iv[1] + g.ny * iv[2]) : -1;
    vs.inside = 0;
    vs.c[0] = vs.c[1] = vs.c[2] = 0;
    vs.order = 0;
    if (nearest) {
        vs.order = nearest_order(g, X);
        return vs;
    }
    int inside = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = grid_plane(og[a], g.spacing, 0), hi = grid_plane(og[a], g.spacing, nc[a]);
        if (!(Xa[a] >= lo && Xa[a] <= hi)) inside = 0;
        vs.c[a] = min(max((int)floorf(fdiv(Xa[a] - og[a], g.spacing)), 0), nc[a] - 1);
    }
    vs.inside = inside;
    if (inside) vs.order = cage_order(g, vs.c[0], vs.c[1], vs.c[2], X);
    return vs;
}

// View index of ray tile `tile`: the last view whose first tile <= tile.
__device__ __forceinline__ int view_of_tile(const ViewDev* v, int n, int tile) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (v[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// traceOneProbe over [t0, t1]: split at the probe's axis planes (at most 4
// single-octant segments, Sec. 4.2); the first non-MISS segment decides.
template <int NRMF, bool COUNT, bool FLAT>
__device__ void trace_probe(const GridDev& g, const Ray& r, int probe, float3 O, float t0, float t1, Decision& out,
                            Stats<COUNT>& st, bool& step_limited) {
    float3 Y0 = make_float3(r.X.x - O.x, r.X.y - O.y, r.X.z - O.z);
    // cut points strictly inside (t0, t1), sorted: c0 <= c1 <= c2 (inf = none);
    // the same expression as the cell faces, so a face through the probe is
    // never a cut
    float cx = r.w.x != 0.0f ? (O.x - r.X.x) * frcp(r.w.x) : kInf;
    float cy = r.w.y != 0.0f ? (O.y - r.X.y) * frcp(r.w.y) : kInf;
    float cz = r.w.z != 0.0f ? (O.z - r.X.z) * frcp(r.w.z) : kInf;
    // a cut further than kFarCuts spacings belongs to a ray almost parallel
    // to that probe plane: no closed scene decides anything that far out, and
    // a segment that long would lose the float32 resolution of its near end
    const float t_far = t0 + kFarCuts * g.spacing;
    cx = (cx > t0 && cx < t1 && cx < t_far) ? cx : kInf;
    cy = (cy > t0 && cy < t1 && cy < t_far) ? cy : kInf;
    cz = (cz > t0 && cz < t1 && cz < t_far) ? cz : kInf;
    float c0 = fminf(cx, fminf(cy, cz)), c2 = fmaxf(cx, fmaxf(cy, cz));
    float c1 = fmaxf(fminf(cx, cy), fminf(fmaxf(cx, cy), cz));  // median
    out.cls = kMiss;
    float a = t0;
    for (int sgi = 0; sgi < 4; ++sgi) {
        float b = sgi == 0 ? c0 : (sgi == 1 ? c1 : (sgi == 2 ? c2 : kInf));
        bool final_seg = !(b < kInf);
        if (final_seg) b = t1;
        Seg s;
        seg_setup(s, Y0, r.w, a, b, g.N);
        if (trace_segment<NRMF, COUNT, FLAT>(g, s, probe, out, st, step_limited)) return;
        if (final_seg) break;
        a = b;
    }
    out.cls = kMiss;
}

template <int RADF>
__device__ __forceinline__ float3 shade(const GridDev& g, int probe, float u, float v) {
    int idx[4];
    float w[4];
    bilinear_taps(g.N, u, v, idx, w);
    int pc = probe, zero = 0;
    (void)zero;  // the index checks of checked builds redirect through it
    LFP_CHECK_TEXEL(g.flags, (unsigned)pc < (unsigned)(g.nx * g.ny * g.nz), pc, zero);
    size_t base = (size_t)pc * g.N * g.N;
    float3 c = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int tq = idx[q];
        LFP_CHECK_TEXEL(g.flags, (unsigned)tq < (unsigned)(g.N * g.N), tq, zero);
        float3 t = RadTexel<RADF>::load(g.rad, base + tq);
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

// vs: the constants of the ray's view (view_start at r.X).
template <int RADF, int NRMF, bool COUNT, bool FLAT>
__device__ PixelResult trace_ray(const GridDev& g, const Ray& r, const ViewStart& vs, Stats<COUNT>& st,
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
    if (vs.eye_probe >= 0) {
        const int p = vs.eye_probe;
        float2 pp = oct_encode(r.w.x, r.w.y, r.w.z);
        res.cls = kHit;
        res.probe = p;
        res.u = 0.5f * (pp.x + 1.0f);
        res.v = 0.5f * (pp.y + 1.0f);
        const int ti = texel_of(pp.x, g.N, 1), tj = texel_of(pp.y, g.N, 1);
        res.texel = ti + g.N * tj;
        if (g.eye_nearest) {  // the texel's own value: sample at its centre
            res.u = (ti + 0.5f) / g.N;
            res.v = (tj + 0.5f) / g.N;
        }
        res.rgb = shade<RADF>(g, p, res.u, res.v);
        cells = 1;
        probes = 1;
        return res;
    }

    // Fewer than 8 probes (Sec. 4.3): every probe, nearest to the eye first
    // (ties to the lower index), over the whole ray; MISS or UNKNOWN falls
    // through to the next probe.
    if (g.nearest_probes) {
        const int P = g.nx * g.ny * g.nz;  // <= 8, checked at grid creation
        bool saw_unknown = false, step_limited = false;
        cells = 1;
        for (int q = 0; q < P; ++q) {
            const int pick = (vs.order >> (3 * q)) & 7;
            probes++;
            Decision dec;
            trace_probe<NRMF, COUNT, FLAT>(g, r, pick, probe_pos(g, pick), 0.0f, kInf, dec, st, step_limited);
            if (step_limited) {
                res.cls = kStepLimit;
                return res;
            }
            if (dec.cls == kHit) {
                res.cls = kHit;
                res.probe = pick;
                res.u = dec.u;
                res.v = dec.v;
                res.texel = dec.texel;
                res.rgb = shade<RADF>(g, pick, res.u, res.v);
                return res;
            }
            if (dec.cls == kUnknown) saw_unknown = true;
        }
        res.cls = saw_unknown ? kUnknown : kMiss;
        return res;
    }

    // Grid iterator (Sec. 4.3): 3D DDA over the cells the ray crosses. A
    // camera inside the probe box starts in its cell at t = 0 (from the view).
    int c[3], step[3];
    if (vs.inside) {
#pragma unroll
        for (int a = 0; a < 3; ++a) c[a] = vs.c[a];
    } else {
        float t_enter = 0.0f, t_exit = kInf;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float lo = grid_plane(og[a], g.spacing, 0), hi = grid_plane(og[a], g.spacing, nc[a]);
            if (Wa[a] == 0.0f) {
                if (Xa[a] < lo || Xa[a] > hi) t_enter = kInf;
                continue;
            }
            float ta = fdiv(lo - Xa[a], Wa[a]), tb = fdiv(hi - Xa[a], Wa[a]);
            if (ta > tb) { float x = ta; ta = tb; tb = x; }
            t_enter = fmaxf(t_enter, ta);
            t_exit = fminf(t_exit, tb);
        }
        if (!(t_enter <= t_exit)) return res;  // the ray misses the grid: MISS
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float p = fmaf(t_enter, Wa[a], Xa[a]);
            c[a] = min(max((int)floorf(fdiv(p - og[a], g.spacing)), 0), nc[a] - 1);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) step[a] = Wa[a] > 0.0f ? 1 : (Wa[a] < 0.0f ? -1 : 0);
    bool saw_unknown = false, step_limited = false;
    float t_in = 0.0f;
    for (int guard = 0; guard < nc[0] + nc[1] + nc[2] + 3; ++guard) {
        float tm[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            tm[a] = step[a] == 0 ? kInf
                                 : (grid_plane(og[a], g.spacing, c[a] + (step[a] > 0 ? 1 : 0)) - Xa[a]) *
                                       frcp(Wa[a]);
        // first exit, ties to the lower axis; selects rather than run-time
        // indices keep the per-axis arrays in registers (no stack frame)
        int ax = tm[1] < tm[0] ? 1 : 0;
        if (tm[2] < (ax ? tm[1] : tm[0])) ax = 2;
        const int cax = ax == 0 ? c[0] : (ax == 1 ? c[1] : c[2]);
        const int sax = ax == 0 ? step[0] : (ax == 1 ? step[1] : step[2]);
        const int ncax = ax == 0 ? nc[0] : (ax == 1 ? nc[1] : nc[2]);
        int nxt = cax + sax;
        bool last_cell = sax == 0 || nxt < 0 || nxt > ncax - 1;
        float t_out = last_cell ? kInf : (ax == 0 ? tm[0] : (ax == 1 ? tm[1] : tm[2]));
        cells++;

        // cage: 8 corner probes, nearest to the entry point first, ties to
        // the lower probe index (corner k has index order k)
        float3 P = make_float3(fmaf(t_in, r.w.x, r.X.x), fmaf(t_in, r.w.y, r.X.y), fmaf(t_in, r.w.z, r.X.z));
        const unsigned order = (guard == 0 && vs.inside) ? vs.order : cage_order(g, c[0], c[1], c[2], P);
        int n_unknown = 0;
        for (int q = 0; q < 8; ++q) {
            Decision dec;
            probes++;
            const int kq = (order >> (3 * q)) & 7;
            const int probe = corner_index(g, c[0], c[1], c[2], kq);
            trace_probe<NRMF, COUNT, FLAT>(g, r, probe, corner_pos(g, c[0], c[1], c[2], kq), t_in, t_out, dec, st,
                                           step_limited);
            if (step_limited) {
                res.cls = kStepLimit;
                return res;
            }
            if (dec.cls == kHit) {
                res.cls = kHit;
                res.probe = probe;
                res.u = dec.u;
                res.v = dec.v;
                res.texel = dec.texel;
                res.rgb = shade<RADF>(g, probe, res.u, res.v);
                return res;
            }
            if (dec.cls == kMiss) break;
            ++n_unknown;
        }
        if (n_unknown == 8) saw_unknown = true;
        if (last_cell) break;
        t_in = t_out;
        if (ax == 0) c[0] = nxt;
        else if (ax == 1) c[1] = nxt;
        else c[2] = nxt;
    }
    res.cls = saw_unknown ? kUnknown : kMiss;
    return res;
}

}  // namespace trace
}  // namespace lfp

// Forward render, streaming engine: the per-ray tracer of render_trace.cuh
// recast as a flat per-lane state machine.
//
// The nested formulation (cells -> probes -> segments -> low-res walk ->
// full-res walk, each a loop with early exits) leaves most lanes of a warp
// idle: lanes at different depths of the nest execute one after another, and
// a warp waits for its slowest ray. Here every loop iteration gives each lane
// one texel visit at whichever level it is on (the low- and full-resolution
// visits are the same instructions with different operands); the
// transitions (a full-resolution crossing's decision, next segment, probe,
// cell, ray) run in a control round that the walk enters once most lanes
// wait for one, and a lane whose ray is done takes the next ray from its
// warp's pool of 8x4 ray tiles (16-ray halves near the end of the launch),
// refilled from a global queue. Results are identical to the nested engine:
// the same arithmetic decides every texel.
#include <cuda_runtime.h>

#include "lfp_device.cuh"
#include "lfp_internal.h"
#include "render_trace.cuh"

namespace lfp {
namespace {

using namespace trace;

#ifndef LFP_STREAM_WALK_STEPS
#define LFP_STREAM_WALK_STEPS 64
#endif
#ifndef LFP_STREAM_BATCH_PCT
#define LFP_STREAM_BATCH_PCT 80
#endif
// resident blocks per SM of the two register budgets (64 and 56 registers)
constexpr int kMinBlocks[2] = {8, 9};
constexpr int kStreamThreads = kStreamThreadsPerBlock;
constexpr int kWalkSteps = LFP_STREAM_WALK_STEPS;  // most texel visits per lane between control rounds
constexpr int kBatchPct = LFP_STREAM_BATCH_PCT;     // transitions run once this % of busy lanes wait
constexpr unsigned kFull = 0xffffffffu;
#ifndef LFP_STREAM_CHAIN_PASSES
#define LFP_STREAM_CHAIN_PASSES 8
#endif
constexpr int kChainPasses = LFP_STREAM_CHAIN_PASSES;  // transition passes per control round

enum Mode : int {
    kIdle = 0,     // no ray: take one from the pool
    kWalk,         // one texel visit per iteration
    kCellStart,    // set up the cage of cell c
    kProbeStart,   // set up probe of rank q
    kSegStart,     // set up segment segi of the probe
    kSegEnd,       // the segment ended without a decision
    kUnknownRes,   // the probe returned UNKNOWN
    kNextCell,     // the probe returned MISS, or all 8 were UNKNOWN
    kRayDone,      // write the pixel
    kExit,         // no rays left
    kDecide        // full-resolution crossing: normal test and hit point
};

// Per-lane state. The walk's working set lives in registers (Lane); the
// fields only the control round touches live in shared memory, one slot per
// thread in structure-of-arrays layout (conflict-free), which frees registers
// for more resident warps.
struct Lane {
    int mode;
    int probe;           // current probe
    // segment (see Seg): u-parametrised octant line, the fields the walk uses
    float e, m0, m1, q0, q1, A0, A1, A2;
    int dir0, dir1;
    const float* plane;  // the current level's map: the probe's min plane (low resolution) or distance map
    // walk
    int level, i, j, lo0, lo1;  // index box: [lo, lo + span) per axis, span k (full res.) or M / 2
    float ux, uy, u, u1, Pa, D2a;  // after a HIT: (ux, uy) hold the shading uv
};

// control-round fields in shared memory
enum ColdF {
    kX0, kX1, kX2, kTin, kTout, kCut0, kCut1, kCut2, kSegA, kSegB,
    kY00, kY01, kY02,  // X - O of the current probe (probe_start), read by each segment set-up
    // segment fields used only when a walk descends, decides or ascends
    kW0, kW1, kW2, kYa0, kYa1, kYa2, kCp, kUstar, kP00, kP01, kK0, kK1, kUend,
    kUxc, kUyc, kUec,  // the low-resolution texel being refined: next crossings, exit
                       // (at a pending decision kUxc, kUyc hold the texel value and exit u)
    kNumColdF
};
enum ColdI { kC0, kC1, kC2, kCbits, kOrder, kQ, kKq, kSegI, kSegFinal, kCls, kQuad, kI, kJ, kLastc, kNumColdI };
// kCbits: step signs (2 bits per axis: 1 +, 2 -), bits 6-7 exit axis, bit 8
// last cell, bit 9 saw UNKNOWN, bit 10 the cage order of the current cell
// is already in kOrder (first cell of a ray from inside the grid; cleared by
// cell_start). kOrder: corner of rank q in bits [3q, 3q + 3).
__shared__ float sh_f[kNumColdF][kStreamThreads];
__shared__ int sh_i[kNumColdI][kStreamThreads];
__shared__ long long sh_o[kStreamThreads];  // output index of the lane's ray

// Per-warp constants of the view the warp's current tile belongs to. Every
// primary ray of a view starts at the camera X, so the view's index, the
// eye-aligned test (Sec. 4.2), the grid entry when X lies in the probe box
// (the cell holding X, from t = 0) and that first cell's cage order (nearest
// to X), or the nearest-probe order of the traversal for fewer than 8
// probes, are the same for all of its rays: they are computed once per tile
// (same operations as per ray, so decisions do not change).
enum WarpViewF { kWvView, kWvEye, kWvInside, kWvC0, kWvC1, kWvC2, kWvOrder, kWvX0, kWvY0, kWvNum };
// the tile's camera factors: a of its 8 pixel columns, b of its 4 rows
__shared__ float sh_wa[kStreamThreads / 32][8], sh_wb[kStreamThreads / 32][4];
__shared__ int sh_wv[kStreamThreads / 32][kWvNum];
__device__ __forceinline__ int& WV(int f) { return sh_wv[threadIdx.x >> 5][f]; }

__device__ __forceinline__ float& CF(int f) { return sh_f[f][threadIdx.x]; }
__device__ __forceinline__ int& CI(int f) { return sh_i[f][threadIdx.x]; }
__device__ __forceinline__ float3 ray_X() { return make_float3(CF(kX0), CF(kX1), CF(kX2)); }
__device__ __forceinline__ float3 ray_w() { return make_float3(CF(kW0), CF(kW1), CF(kW2)); }
__device__ __forceinline__ float3 seg_Ya() { return make_float3(CF(kYa0), CF(kYa1), CF(kYa2)); }

__device__ __forceinline__ int step_of(int bits, int a) {
    int v = (bits >> (2 * a)) & 3;
    return v == 1 ? 1 : (v == 2 ? -1 : 0);
}

// Grid-iterator set-up for a new ray; returns false if it misses the grid.
__device__ __forceinline__ bool ray_enter_grid(const GridDev& g, float3 X, float3 w) {
    const int nc[3] = {g.nx - 1, g.ny - 1, g.nz - 1};
    const float og[3] = {g.ox, g.oy, g.oz};
    const float Xa[3] = {X.x, X.y, X.z}, Wa[3] = {w.x, w.y, w.z};
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
    if (!(t_enter <= t_exit)) return false;
    int c[3], bits = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float p = fmaf(t_enter, Wa[a], Xa[a]);
        c[a] = min(max((int)floorf(fdiv(p - og[a], g.spacing)), 0), nc[a] - 1);
        bits |= (Wa[a] > 0.0f ? 1 : (Wa[a] < 0.0f ? 2 : 0)) << (2 * a);
    }
    CI(kC0) = c[0];
    CI(kC1) = c[1];
    CI(kC2) = c[2];
    CI(kCbits) = bits;
    CF(kTin) = 0.0f;
    return true;
}

// Cell c: its exit (3D DDA) and its cage order, nearest corner to the entry first.
__device__ __forceinline__ void cell_start(const GridDev& g) {
    const int nc[3] = {g.nx - 1, g.ny - 1, g.nz - 1};
    const float og[3] = {g.ox, g.oy, g.oz};
    const float3 X = ray_X(), w = ray_w();
    const float Xa[3] = {X.x, X.y, X.z}, Wa[3] = {w.x, w.y, w.z};
    const int c[3] = {CI(kC0), CI(kC1), CI(kC2)};
    const int cbits = CI(kCbits);
    float tm[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int st = step_of(cbits, a);
        tm[a] = st == 0 ? kInf
                        : (grid_plane(og[a], g.spacing, c[a] + (st > 0 ? 1 : 0)) - Xa[a]) * frcp(Wa[a]);
    }
    // first exit, ties to the lower axis; selects rather than a run-time
    // index keep tm in registers (no stack frame)
    int ax = tm[1] < tm[0] ? 1 : 0;
    if (tm[2] < (ax ? tm[1] : tm[0])) ax = 2;
    int st = step_of(cbits, ax);
    int cax = ax == 0 ? c[0] : (ax == 1 ? c[1] : c[2]);
    int ncax = ax == 0 ? nc[0] : (ax == 1 ? nc[1] : nc[2]);
    int nxt = cax + st;
    bool last = st == 0 || nxt < 0 || nxt > ncax - 1;
    float tax = ax == 0 ? tm[0] : (ax == 1 ? tm[1] : tm[2]);
    CI(kCbits) = (cbits & 0x23f) | (ax << 6) | (last ? 0x100 : 0);
    CF(kTout) = last ? kInf : tax;
    if (!(cbits & 0x400)) {  // else the first cell of a ray from inside the grid: order set from the view
        const float t_in = CF(kTin);
        float3 P = make_float3(fmaf(t_in, w.x, X.x), fmaf(t_in, w.y, X.y), fmaf(t_in, w.z, X.z));
        CI(kOrder) = (int)cage_order(g, c[0], c[1], c[2], P);
    }
    CI(kQ) = 0;
}

// Position of the current probe: a corner of the cell's cage, or (nearest-
// probe traversal) the probe whose index is stored in kKq.
template <bool NEAREST>
__device__ __forceinline__ float3 current_probe_pos(const GridDev& g) {
    return NEAREST ? probe_pos(g, CI(kKq)) : corner_pos(g, CI(kC0), CI(kC1), CI(kC2), CI(kKq));
}

// Probe of rank q: its index and the cut points of the octant split.
template <bool NEAREST>
__device__ __forceinline__ void probe_start(const GridDev& g, Lane& L) {
    const int kq = ((unsigned)CI(kOrder) >> (3 * CI(kQ))) & 7;
    CI(kKq) = kq;
    L.probe = NEAREST ? kq : corner_index(g, CI(kC0), CI(kC1), CI(kC2), kq);
    float3 O = current_probe_pos<NEAREST>(g);
    const float3 X = ray_X(), w = ray_w();
    CF(kY00) = X.x - O.x;
    CF(kY01) = X.y - O.y;
    CF(kY02) = X.z - O.z;
    const float t0 = CF(kTin), t1 = CF(kTout);
    float cx = w.x != 0.0f ? (O.x - X.x) * frcp(w.x) : kInf;
    float cy = w.y != 0.0f ? (O.y - X.y) * frcp(w.y) : kInf;
    float cz = w.z != 0.0f ? (O.z - X.z) * frcp(w.z) : kInf;
    const float t_far = t0 + kFarCuts * g.spacing;  // as in trace_probe
    cx = (cx > t0 && cx < t1 && cx < t_far) ? cx : kInf;
    cy = (cy > t0 && cy < t1 && cy < t_far) ? cy : kInf;
    cz = (cz > t0 && cz < t1 && cz < t_far) ? cz : kInf;
    CF(kCut0) = fminf(cx, fminf(cy, cz));
    CF(kCut2) = fmaxf(cx, fmaxf(cy, cz));
    CF(kCut1) = fmaxf(fminf(cx, cy), fminf(fmaxf(cx, cy), cz));
    CI(kSegI) = 0;
    CF(kSegA) = t0;
}

// Low-resolution index box of the segment's quadrant.
__device__ __forceinline__ void coarse_box(const GridDev& g, Lane& L) {
    const int hm = g.M / 2;
    const int quad = CI(kQuad);
    L.lo0 = (quad & 1) ? hm : 0;
    L.lo1 = (quad & 2) ? hm : 0;
}

// Segment segi: the octant line (same arithmetic as seg_setup) and the
// start of the low-resolution walk.
template <bool NEAREST>
__device__ __forceinline__ void seg_start(const GridDev& g, Lane& L) {
    const int segi = CI(kSegI);
    float b = segi == 0 ? CF(kCut0) : (segi == 1 ? CF(kCut1) : (segi == 2 ? CF(kCut2) : kInf));
    const bool final_seg = !(b < kInf);
    CI(kSegFinal) = final_seg;
    if (final_seg) b = CF(kTout);
    CF(kSegB) = b;
    Seg s;
    seg_setup(s, make_float3(CF(kY00), CF(kY01), CF(kY02)), ray_w(), CF(kSegA), b, g.N);
    CF(kYa0) = s.Ya.x;
    CF(kYa1) = s.Ya.y;
    CF(kYa2) = s.Ya.z;
    CF(kCp) = s.cp;
    CF(kUstar) = s.ustar;
    CF(kP00) = s.p0[0];
    CF(kP01) = s.p0[1];
    CF(kK0) = s.k[0];
    CF(kK1) = s.k[1];
    CF(kUend) = s.u_end;
    const int quad = (s.lo[0] > 0 ? 1 : 0) | (s.lo[1] > 0 ? 2 : 0);
    CI(kQuad) = quad;
    L.e = s.e;
    L.m0 = s.m[0];
    L.m1 = s.m[1];
    L.q0 = s.q[0];
    L.q1 = s.q[1];
    L.A0 = s.A0;
    L.A1 = s.A1;
    L.A2 = s.A2;
    L.dir0 = s.dir[0];
    L.dir1 = s.dir[1];
    {
        int p = L.probe, unused = 0;
        LFP_CHECK_TEXEL(g.flags, (unsigned)p < (unsigned)(g.nx * g.ny * g.nz), p, unused);
        L.probe = p;
        (void)unused;
    }
    // the walk starts where the ray first reaches the least distance of the
    // segment's map quadrant (segment_start)
    float us;
    {
        bool walk;
        us = segment_start(s, __ldg(g.qmin + (size_t)L.probe * 4 + quad), walk);
        if (!walk) {
            L.mode = kSegEnd;
            return;
        }
    }
    L.mode = kWalk;
    L.plane = g.mip + (size_t)L.probe * 2 * g.M * g.M;
    const int k = g.k, N = g.N;
    L.level = 0;
    coarse_box(g, L);
    const int hm1 = g.M / 2 - 1;
    L.i = min(max(div_k(g.kinv, texel_of(fmaf(s.k[0], us, s.p0[0]), N, L.dir0)), L.lo0), L.lo0 + hm1);
    L.j = min(max(div_k(g.kinv, texel_of(fmaf(s.k[1], us, s.p0[1]), N, L.dir1)), L.lo1), L.lo1 + hm1);
    L.u = us;
    L.u1 = s.u_end;
    const float Ds = fmaf(-L.e, us, 1.0f);
    L.Pa = fmaf(fmaf(L.A2, us, L.A1), us, L.A0);
    L.D2a = Ds * Ds;
    L.ux = L.dir0 == 0 ? kInf : fmaxf(fmaf((float)((L.dir0 > 0 ? L.i + 1 : L.i) * k), L.m0, L.q0), us);
    L.uy = L.dir1 == 0 ? kInf : fmaxf(fmaf((float)((L.dir1 > 0 ? L.j + 1 : L.j) * k), L.m1, L.q1), us);
}

// tau from the segment start of walk parameter u (infinite past the end),
// the same arithmetic as tau_of
__device__ __forceinline__ float lane_tau(const Lane& L, float u) {
    float D = fmaf(-L.e, u, 1.0f);
    return D > 0.0f ? __fdividef(CF(kCp) * u, D) : kInf;
}

// Advance past the current texel (exit ue) over the earlier next boundary;
// false when the walk leaves the current level's index box. The axis is
// selected into shared operands so both cases run the same instructions.
__device__ __forceinline__ bool advance(Lane& L, int scale, int span, float ue, float Pb, float D2b) {
    const bool xs = L.ux <= L.uy;
    const int dir = xs ? L.dir0 : L.dir1;
    const int c = (xs ? L.i : L.j) + dir;
    if ((unsigned)(c - (xs ? L.lo0 : L.lo1)) >= (unsigned)span) return false;
    const float un = fmaxf(fmaf((float)((dir > 0 ? c + 1 : c) * scale), xs ? L.m0 : L.m1, xs ? L.q0 : L.q1), ue);
    if (xs) {
        L.i = c;
        L.ux = un;
    } else {
        L.j = c;
        L.uy = un;
    }
    L.u = ue;
    L.Pa = Pb;
    L.D2a = D2b;
    return true;
}

// The full-resolution walk under a low-resolution texel ended without a
// decision: continue the low-resolution walk after that texel.
__device__ __forceinline__ void ascend(const GridDev& g, Lane& L) {
    L.level = 0;
    L.plane = g.mip + (size_t)L.probe * 2 * g.M * g.M;
    L.i = CI(kI);
    L.j = CI(kJ);
    coarse_box(g, L);
    L.ux = CF(kUxc);
    L.uy = CF(kUyc);
    L.u1 = CF(kUend);
    float ue = CF(kUec);
    float Pb = fmaf(fmaf(L.A2, ue, L.A1), ue, L.A0);
    float Db = fmaf(-L.e, ue, 1.0f);
    if (CI(kLastc) || !advance(L, g.k, g.M / 2, ue, Pb, Db * Db)) L.mode = kSegEnd;
}

// One texel visit (Appendix A low/highResolutionTracing, one step).
template <int NRMF, bool COUNT>
__device__ __forceinline__ void walk_step(const GridDev& g, Lane& L, Stats<COUNT>& st) {
    const int N = g.N, M = g.M, k = g.k;
    float un = fminf(L.ux, L.uy);
    bool last = !(un < L.u1);
    float ue = last ? L.u1 : un;
    float Pb = fmaf(fmaf(L.A2, ue, L.A1), ue, L.A0);
    float Db = fmaf(-L.e, ue, 1.0f);
    float D2b = Db * Db;
    // both levels read one float of the current plane: the same load for
    // every lane, whichever level it is on
    const int R = L.level ? N : M;
    int i = L.i, j = L.j;
    LFP_CHECK_TEXEL(g.flags, (unsigned)i < (unsigned)R && (unsigned)j < (unsigned)R, i, j);
    const float v = __ldg(L.plane + (j * R + i));
    if (COUNT) {
        if (L.level) st.fine++;
        else st.coarse++;
    }
    if (COUNT) {  // the instrumented kernel also enforces the max_steps cap
        st.steps++;
        if (g.max_steps > 0 && (int)st.steps >= g.max_steps) {
            CI(kCls) = kStepLimit;
            L.mode = kRayDone;
            return;
        }
    }
    float d2 = v * v;
    if (L.Pa < d2 * L.D2a && Pb < d2 * D2b) {  // the ray stays in front of the stored surface
        if (!last && advance(L, L.level ? 1 : k, L.level ? k : M / 2, ue, Pb, D2b)) return;
        if (L.level) ascend(g, L);
        else L.mode = kSegEnd;
        return;
    }
    if (L.level == 0) {  // candidate low-resolution texel
        // the block's max distance, from the max plane after the min plane
        if (!g.two_way &&
            !comes_within(L.A0, L.A1, L.A2, L.e, CF(kUstar), L.u, ue, __ldg(L.plane + (M + j) * M + i) * g.kappa)) {
            L.mode = kUnknownRes;  // every full-resolution texel under it is passed behind
            return;
        }
        CI(kI) = L.i;
        CI(kJ) = L.j;
        CF(kUxc) = L.ux;
        CF(kUyc) = L.uy;
        CF(kUec) = ue;
        CI(kLastc) = last;
        L.level = 1;
        L.plane = g.dist + (size_t)L.probe * N * N;
        L.lo0 = L.i * k;
        L.lo1 = L.j * k;
        L.u1 = ue;
        {  // skip the full-resolution texels the ray passes in front of dmin (fine_start)
            Seg s;
            s.A1 = L.A1;
            s.A2 = L.A2;
            s.e = L.e;
            // explicit multiply-adds: both engines round the start alike
            const float us = fine_start(s, d2, L.u, fmaf(-d2, L.D2a, L.Pa), ue, fmaf(-d2, D2b, Pb));
            const float Ds = fmaf(-L.e, us, 1.0f);
            L.Pa = fmaf(fmaf(L.A2, us, L.A1), us, L.A0);
            L.D2a = Ds * Ds;
            L.u = us;
        }
        L.i = min(max(texel_of(fmaf(CF(kK0), L.u, CF(kP00)), N, L.dir0), L.lo0), L.lo0 + k - 1);
        L.j = min(max(texel_of(fmaf(CF(kK1), L.u, CF(kP01)), N, L.dir1), L.lo1), L.lo1 + k - 1);
        L.ux = L.dir0 == 0 ? kInf : fmaxf(fmaf((float)(L.dir0 > 0 ? L.i + 1 : L.i), L.m0, L.q0), L.u);
        L.uy = L.dir1 == 0 ? kInf : fmaxf(fmaf((float)(L.dir1 > 0 ? L.j + 1 : L.j), L.m1, L.q1), L.u);
        return;
    }
    // full-resolution crossing: decided in the control round (kDecide), which
    // keeps the walk loop's code small
    CF(kUxc) = v;
    CF(kUyc) = ue;
    L.mode = kDecide;
}

// The normal decides a full-resolution crossing (highResolutionTracing):
// HIT with its shading uv, else UNKNOWN.
template <int NRMF, bool COUNT>
__device__ __forceinline__ void decide(const GridDev& g, Lane& L, Stats<COUNT>& st) {
    const int N = g.N;
    const float v = CF(kUxc), ue = CF(kUyc);
    const float d = v;
    L.mode = kUnknownRes;
    if (g.two_way || comes_within(L.A0, L.A1, L.A2, L.e, CF(kUstar), L.u, ue, d * g.kappa)) {
        int i = L.i, j = L.j;
        LFP_CHECK_TEXEL(g.flags, (unsigned)i < (unsigned)N && (unsigned)j < (unsigned)N, i, j);
        float2 no = NrmTexel<NRMF>::load(g.nrm, (size_t)L.probe * N * N + (size_t)j * N + i);
        float3 n = oct_decode_unnorm(no.x, no.y);
        const float3 w = ray_w();
        if (COUNT) st.normal++;
        if ((n.x * w.x + n.y * w.y + n.z * w.z) < 0.0f) {
            Seg s;  // the hit point needs Ya, w and |Ya|^2 only
            s.Ya = seg_Ya();
            s.w = w;
            s.A0 = L.A0;
            float th = hit_time(s, lane_tau(L, L.u), lane_tau(L, ue), d);
            float2 pp = oct_encode(fmaf(th, w.x, s.Ya.x), fmaf(th, w.y, s.Ya.y), fmaf(th, w.z, s.Ya.z));
            CI(kCls) = kHit;
            L.ux = 0.5f * (pp.x + 1.0f);  // shading uv
            L.uy = 0.5f * (pp.y + 1.0f);
            L.mode = kRayDone;
        }
    }
}

// Traversal for fewer than 8 probes (Sec. 4.3): every probe, nearest to the
// eye first (the view's order, view_start), as one pseudo-cell over [0, inf).
__device__ __forceinline__ void nearest_start(unsigned order) {
    CI(kOrder) = (int)order;
    CI(kQ) = 0;
    CI(kCbits) = 0x100;  // the one pseudo-cell is the last
    CF(kTin) = 0.0f;
    CF(kTout) = kInf;
}

// The view constants of tile `tile` into the warp's slots (warp-uniform:
// every lane computes and writes the same values).
template <bool NEAREST>
__device__ __forceinline__ void warp_view_setup(const GridDev& g, const ViewBatch& vb, int tile) {
    const int vi = view_of_tile(vb.v, vb.n, tile);
    const ViewDev& v = vb.v[vi];
    const ViewStart vs = view_start(g, make_float3(v.px, v.py, v.pz), NEAREST);
    WV(kWvView) = vi;
    WV(kWvEye) = vs.eye_probe;
    WV(kWvInside) = vs.inside;
    WV(kWvC0) = vs.c[0];
    WV(kWvC1) = vs.c[1];
    WV(kWvC2) = vs.c[2];
    WV(kWvOrder) = (int)vs.order;
    const int lt = tile - v.tile_begin;  // the tile's first pixel
    const int x0 = (lt % v.tiles_x) * 8, y0 = (lt / v.tiles_x) * 4;
    WV(kWvX0) = x0;
    WV(kWvY0) = y0;
    // pinhole factors of the tile's columns and rows (lanes 0-7 and 8-11),
    // the arithmetic start_ray used per ray
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane < 8) sh_wa[w][lane] = ((x0 + lane + 0.5f) / (float)v.W * 2.0f - 1.0f) * v.sa;
    else if (lane < 12) sh_wb[w][lane - 8] = (1.0f - (y0 + (lane - 8) + 0.5f) / (float)v.H * 2.0f) * v.sb;
    __syncwarp();
}

// Start the ray of slot `slot` (0..31) of 8x4 ray tile `tile` (whose view
// constants are in the warp's slots).
template <bool NEAREST>
__device__ __forceinline__ void start_ray(const GridDev& g, const ViewBatch& vb, int tile, int slot, Lane& L) {
    const ViewDev& v = vb.v[WV(kWvView)];
    int x = WV(kWvX0) + (slot & 7), y = WV(kWvY0) + (slot >> 3);
    if (x >= v.W || y >= v.H) {
        L.mode = kIdle;  // outside a ragged view: no ray in this slot
        return;
    }
    const float a = sh_wa[threadIdx.x >> 5][slot & 7], b = sh_wb[threadIdx.x >> 5][slot >> 3];
    float dx = v.fx + a * v.rx + b * v.ux, dy = v.fy + a * v.ry + b * v.uy, dz = v.fz + a * v.rz + b * v.uz;
    float il = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
    const float3 X = make_float3(v.px, v.py, v.pz);
    CF(kX0) = X.x;
    CF(kX1) = X.y;
    CF(kX2) = X.z;
    const float3 w = make_float3(dx * il, dy * il, dz * il);
    CF(kW0) = w.x;
    CF(kW1) = w.y;
    CF(kW2) = w.z;
    sh_o[threadIdx.x] = v.out_offset + (long long)y * v.W + x;
    CI(kCls) = kMiss;
    const int eye_probe = WV(kWvEye);
    if (eye_probe >= 0) {  // eye aligned with a probe (Sec. 4.2): look up oct(w) directly
        float2 pp = oct_encode(w.x, w.y, w.z);
        CI(kCls) = kHit;
        L.probe = eye_probe;
        L.ux = 0.5f * (pp.x + 1.0f);
        L.uy = 0.5f * (pp.y + 1.0f);
        L.i = texel_of(pp.x, g.N, 1);
        L.j = texel_of(pp.y, g.N, 1);
        if (g.eye_nearest) {  // the texel's own value: sample at its centre
            L.ux = (L.i + 0.5f) / g.N;
            L.uy = (L.j + 0.5f) / g.N;
        }
        L.mode = kRayDone;
        return;
    }
    if (NEAREST) {
        nearest_start((unsigned)WV(kWvOrder));
        L.mode = kProbeStart;
        return;
    }
    if (WV(kWvInside)) {  // the view's first cell and its cage order
        CI(kC0) = WV(kWvC0);
        CI(kC1) = WV(kWvC1);
        CI(kC2) = WV(kWvC2);
        CI(kCbits) = (w.x > 0.0f ? 1 : (w.x < 0.0f ? 2 : 0)) | (w.y > 0.0f ? 4 : (w.y < 0.0f ? 8 : 0)) |
                     (w.z > 0.0f ? 16 : (w.z < 0.0f ? 32 : 0)) | 0x400;
        CI(kOrder) = WV(kWvOrder);
        CF(kTin) = 0.0f;
        L.mode = kCellStart;
        return;
    }
    L.mode = ray_enter_grid(g, X, w) ? kCellStart : kRayDone;
}

template <int RADF>
__device__ __forceinline__ void write_ray(const GridDev& g, const OutDev& out, const Lane& L) {
    const long long o = sh_o[threadIdx.x];
    const int cls = CI(kCls);
    const bool hit = cls == kHit;
    float3 rgb = make_float3(0.f, 0.f, 0.f);
    if (hit) rgb = shade<RADF>(g, L.probe, L.ux, L.uy);
    if (out.rgb) {
        out.rgb[3 * o + 0] = rgb.x;
        out.rgb[3 * o + 1] = rgb.y;
        out.rgb[3 * o + 2] = rgb.z;
    }
    if (out.cls) out.cls[o] = (uint8_t)cls;
    if (out.aux_probe) out.aux_probe[o] = hit ? L.probe : -1;
    if (out.aux_uv) {
        out.aux_uv[2 * o + 0] = hit ? L.ux : 0.0f;
        out.aux_uv[2 * o + 1] = hit ? L.uy : 0.0f;
    }
    if (out.hit_texel) out.hit_texel[o] = hit ? L.i + g.N * L.j : -1;
    if (cls == kStepLimit) atomicOr(g.flags, 1u);
}

// Persistent kernel: every warp pulls 8x4 ray tiles from `queue` and keeps
// its 32 lanes busy, one texel visit per lane per iteration. COUNT selects
// the instrumented variant (fetch counters and the max_steps cap); the plain
// variant carries neither, which keeps the per-visit path short.
template <int RADF, int NRMF, bool COUNT, int OCC, bool NEAREST>
__global__ void __launch_bounds__(kStreamThreads, kMinBlocks[OCC]) render_stream_kernel(GridDev g, ViewBatch vb,
                                                                                     OutDev out, unsigned* queue) {
    const int n_probes = g.nx * g.ny * g.nz;  // nearest-probe traversal: probes per ray
    const int lane = threadIdx.x & 31;
    const unsigned lanes_below = (1u << lane) - 1u;
    Lane L;
    L.mode = kIdle;
    Stats<COUNT> st;
    unsigned cells = 0, probes = 0;
    unsigned long long acc[kNumCounters];
    if (COUNT)
        for (int q = 0; q < kNumCounters; ++q) acc[q] = 0;
    // warp-uniform ray pool: slots [next, end) of tile pool_tile, packed in
    // `pool` (next in bits 0-5, end in bits 6-11: one register). The queue
    // hands out whole 8x4 tiles, and the last vb.tail_tiles tiles as 16-ray
    // halves, so near the end of the launch no warp holds many unstarted
    // rays while others have run dry.
    int pool_tile = 0, pool = 0;
    bool exhausted = false;
    for (;;) {
        // ---- control round: every transition runs once, in pipeline order,
        // for all lanes that need it, so lanes reconverge at each stage ----
        if (L.mode == kDecide) decide<NRMF, COUNT>(g, L, st);
        if (L.mode == kRayDone) {
            write_ray<RADF>(g, out, L);
            if (COUNT) {
                const int cls = CI(kCls);
                const bool eye = cls == kHit && probes == 0;  // eye-aligned lookup
                acc[0] += st.coarse;
                acc[1] += st.fine;
                acc[2] += st.normal;
                acc[3] += cls == kHit ? 4 : 0;
                acc[4] += eye ? 1 : cells;
                acc[5] += eye ? 1 : probes;
                acc[6] += cls == kHit ? 1 : 0;
                acc[7] += 1;
            }
            L.mode = kIdle;
        }
        // refill idle lanes from the warp's pool (warp-synchronous)
        unsigned idle = __ballot_sync(kFull, L.mode == kIdle);
        while (idle != 0u && !exhausted) {
            if ((pool & 63) >= (pool >> 6)) {
                int t = 0;
                if (lane == 0) t = (int)atomicAdd(queue, 1u);
                t = __shfl_sync(kFull, t, 0);
                // the 56-register build keeps whole tiles (its register
                // allocation loses more than the split gains)
                const int t_split = OCC == 1 ? vb.total_tiles : max(vb.total_tiles - vb.tail_tiles, 0);
                if (t < t_split) {
                    pool_tile = t;
                    pool = 32 << 6;
                } else {
                    const int sub = t - t_split;
                    pool_tile = t_split + (sub >> 1);
                    if (pool_tile >= vb.total_tiles) {
                        exhausted = true;
                        break;
                    }
                    pool = ((sub & 1) * 16) | (((sub & 1) * 16 + 16) << 6);
                }
                warp_view_setup<NEAREST>(g, vb, pool_tile);
            }
            const int pool_next = pool & 63;
            int avail = (pool >> 6) - pool_next;
            int rank = __popc(idle & lanes_below);
            if (L.mode == kIdle && rank < avail) {
                st = Stats<COUNT>();
                cells = NEAREST ? 1 : 0;
                probes = 0;
                start_ray<NEAREST>(g, vb, pool_tile, pool_next + rank, L);  // kRayDone rays are written next round
            }
            pool += min(__popc(idle), avail);
            idle = __ballot_sync(kFull, L.mode == kIdle);
        }
        if (exhausted && L.mode == kIdle) L.mode = kExit;
        if (__all_sync(kFull, L.mode == kExit)) break;

        // the transitions run again while a lane's new segment ended at its
        // set-up (nearer than its quadrant's least distance), so such lanes
        // reach their next segment in the same round
#pragma unroll 1
        for (int pass = 0; pass < kChainPasses; ++pass) {
            if (L.mode == kSegEnd) {  // MISS on this segment: next segment, or the probe is a MISS
                if (CI(kSegFinal)) {
                    if (NEAREST) {  // a MISS falls through to the next probe too
                        const int q = CI(kQ) + 1;
                        CI(kQ) = q;
                        L.mode = q == n_probes ? kNextCell : kProbeStart;
                    } else {
                        L.mode = kNextCell;
                    }
                } else {
                    CI(kSegI) += 1;
                    CF(kSegA) = CF(kSegB);
                    L.mode = kSegStart;
                }
            }
            if (L.mode == kUnknownRes) {  // UNKNOWN falls through to the next probe of the cage
                const int q = CI(kQ) + 1;
                CI(kQ) = q;
                if (NEAREST) {  // any UNKNOWN makes an undecided ray UNKNOWN
                    CI(kCbits) |= 0x200;
                    L.mode = q == n_probes ? kNextCell : kProbeStart;
                } else if (q == 8) {
                    CI(kCbits) |= 0x200;  // saw UNKNOWN
                    L.mode = kNextCell;
                } else {
                    L.mode = kProbeStart;
                }
            }
            if (L.mode == kNextCell) {
                const int cbits = CI(kCbits);
                if (cbits & 0x100) {  // last cell
                    CI(kCls) = (cbits & 0x200) ? kUnknown : kMiss;
                    L.mode = kRayDone;  // written at the next control round
                } else {
                    int ax = (cbits >> 6) & 3;
                    int st_ax = step_of(cbits, ax);
                    if (ax == 0) CI(kC0) += st_ax;
                    else if (ax == 1) CI(kC1) += st_ax;
                    else CI(kC2) += st_ax;
                    CF(kTin) = CF(kTout);
                    L.mode = kCellStart;
                }
            }
            if (L.mode == kCellStart) {
                ++cells;
                cell_start(g);
                L.mode = kProbeStart;
            }
            if (L.mode == kProbeStart) {
                ++probes;
                probe_start<NEAREST>(g, L);
                L.mode = kSegStart;
            }
            if (L.mode == kSegStart) seg_start<NEAREST>(g, L);  // kWalk, or kSegEnd for a segment nearer than its quadrant
            if (!__any_sync(kFull, L.mode == kSegEnd)) break;
        }

        // ---- walk phase: one texel visit per walking lane per step, until
        // kBatchPct % of the busy lanes wait for a transition ----
        const int busy = __popc(__ballot_sync(kFull, L.mode != kIdle && L.mode != kExit));
        const int need = (kBatchPct * busy + 99) / 100;  // waiting lanes that end the phase
#pragma unroll 1
        for (int r = 0; r < kWalkSteps; ++r) {
            if (L.mode == kWalk) walk_step<NRMF, COUNT>(g, L, st);
            const int walking = __popc(__ballot_sync(kFull, L.mode == kWalk));
            if (busy - walking >= need) break;
        }
    }
    if (COUNT && out.counters) {
        for (int q = 0; q < kNumCounters; ++q) {
            unsigned long long v = acc[q];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(kFull, v, off);
            if (lane == 0 && v) atomicAdd(out.counters + q, v);
        }
    }
}

template <int RADF, int NRMF>
cudaError_t launch_stream_fmt(const GridDev& g, const ViewBatch& vb, const OutDev& out, unsigned* queue, int blocks,
                              int occ, cudaStream_t s) {
    // the instrumented variant (counters, step cap) always uses the 64-register budget
    const bool instr = out.counters || g.max_steps > 0;
    if (g.nearest_probes) {
        if (instr)
            render_stream_kernel<RADF, NRMF, true, 0, true><<<blocks, kStreamThreads, 0, s>>>(g, vb, out, queue);
        else
            render_stream_kernel<RADF, NRMF, false, 0, true><<<blocks, kStreamThreads, 0, s>>>(g, vb, out, queue);
    } else if (instr) {
        render_stream_kernel<RADF, NRMF, true, 0, false><<<blocks, kStreamThreads, 0, s>>>(g, vb, out, queue);
    } else if (occ == 1) {
        render_stream_kernel<RADF, NRMF, false, 1, false><<<blocks, kStreamThreads, 0, s>>>(g, vb, out, queue);
    } else {
        render_stream_kernel<RADF, NRMF, false, 0, false><<<blocks, kStreamThreads, 0, s>>>(g, vb, out, queue);
    }
    return cudaGetLastError();
}

template <int RADF, int NRMF>
int blocks_fmt(int occ) {
    int n = 0;
    if (occ == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, render_stream_kernel<RADF, NRMF, false, 1, false>,
                                                      kStreamThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, render_stream_kernel<RADF, NRMF, false, 0, false>,
                                                      kStreamThreads, 0);
    return n;
}

}  // namespace

cudaError_t launch_render_stream(const GridDev& g, int rad_fmt, int nrm_fmt, const ViewBatch& vb, const OutDev& out,
                                 unsigned* queue, int blocks, int occ, cudaStream_t s) {
    if (rad_fmt == kF32 && nrm_fmt == kF32) return launch_stream_fmt<kF32, kF32>(g, vb, out, queue, blocks, occ, s);
    if (rad_fmt == kF16 && nrm_fmt == kF16) return launch_stream_fmt<kF16, kF16>(g, vb, out, queue, blocks, occ, s);
    if (rad_fmt == kF16 && nrm_fmt == kF32) return launch_stream_fmt<kF16, kF32>(g, vb, out, queue, blocks, occ, s);
    return launch_stream_fmt<kF32, kF16>(g, vb, out, queue, blocks, occ, s);
}

int render_stream_blocks_per_sm(int rad_fmt, int nrm_fmt, int occ) {
    if (rad_fmt == kF32 && nrm_fmt == kF32) return blocks_fmt<kF32, kF32>(occ);
    if (rad_fmt == kF16 && nrm_fmt == kF16) return blocks_fmt<kF16, kF16>(occ);
    if (rad_fmt == kF16) return blocks_fmt<kF16, kF32>(occ);
    return blocks_fmt<kF32, kF16>(occ);
}

}  // namespace lfp

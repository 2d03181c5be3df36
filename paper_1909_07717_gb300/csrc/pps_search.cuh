// pps_search.cuh -- device code of the exact passing-point search (sm_103a).
//
// One persistent kernel covers the whole hot path of the SBIP-based dynamic
// passing-point search (ZJUNlict 2019, Sec. 4.1-4.4), fused:
//   A1 state staging        each warp reads its state record through the
//                           read-only cache and derives the constants
//   A2 candidate geometry   one lane per grid point; samples are generated
//                           on the fly, never stored
//   A3 opponent intercept   T_k = min_j t_j(sample k), opponents held in
//                           registers (warp-uniform, so every lane of a warp
//                           reads the same opponent in the same cycle);
//                           computed once per (point, k), shared by speeds
//   A4 ball time + margin   per speed: min_k (T_k - t_ball(s_k))
//   A5 shot angle, goal distance      once per point
//   A6 feasibility, score, mask       warp ballot -> one mask word per warp
//   A7 argmax               warp shuffle -> CTA -> 64-bit atomicMax per state
// Work is dealt per warp (a state and 32 consecutive grid points), so warps
// never wait for one another.  A second, tiny kernel turns the per-state
// keys into pps_best records.
//
// Arithmetic (FP32, inputs as given).  The opponent time is computed in a
// scaled form: speeds in units of vmax (w' = w / vmax), lengths multiplied
// by kappa = 2 amax / vmax^2 (d' = kappa d), q' = sqrt(w'^2 + d') and
// m' = max(1 - q', 0); the 1-D bang-bang time is
//     t = ((1 - w')^2 + d' - m'^2) * vmax / (2 amax),
// which equals (-w + sqrt(w^2 + 2 amax d)) / amax while the robot is still
// accelerating (q' <= 1) and (vmax - w)/amax + (d - d_acc)/vmax once it
// cruises; the numerator is the tangent-line identity of those two branches,
// so no branch is needed, and m' is a single saturating add.  The ball term uses
//     a T_k + sqrt(v^2 - 2 a s_k),   margin = (min_k(...) - v) / a,
// which is min_k (T_k - (v - sqrt(v^2 - 2 a s_k)) / a) rearranged.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "pps.h"

namespace pps {

#ifndef PPS_KUNROLL
#define PPS_KUNROLL 1  // measured: 1 beats 2 and 4 once slots are packed
#endif
constexpr int kKUnroll = PPS_KUNROLL;  // unroll of the sample loop

// Threads per CTA of a search-kernel instance: one CTA per SM either way;
// the 8-slot instances take 1024 threads (32 independent warps: more
// latency hiding for the dependent intercept chain is worth the few
// spilled registers at the 64-register cap; measured 56.9 ms against
// 60.0 ms with 512 threads on the batched workload), the wider ones 512.
template <int JMAX, int VMAX>
__host__ __device__ constexpr int search_tpb() {
    return JMAX <= 8 ? 1024 : 512;
}
constexpr float kFar = 1.0e18f;    // offset of an unused opponent slot
constexpr float kD2Floor = 1.0e-30f;  // keeps 1/d finite when d == 0

struct SearchArgs {
    const pps_state* states;
    int n_states;
    int nx, ny, P, words;  // words = ceil(P / 32): mask words per speed
    float g, x0, y0;
    int V;
    int kmax;              // largest K accepted
    float speed[PPS_MAX_SPEEDS];
    float speed2[PPS_MAX_SPEEDS];
    pps_params prm;
    pps_best* best;
    uint32_t* mask;        // may be null
    float* dbg_margin;     // may be null
    float* dbg_score;      // may be null
    float* dbg_T;          // may be null
    int T_stride;
    unsigned long long* keys;  // scratch: per-state packed (score, ~idx)
    int* counts;               // scratch: per-state feasible count
    float* dbg_point;          // may be null: per (s, p) best score
    const int* skip;           // may be null: states to leave untouched
    const int* list;           // may be null: search only states list[i],
    const int* list_n;         //   i < *list_n (EXT instances)
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ float rsqrt_fast(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_fast(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Square roots of the intercept formula and the ball term: one MUFU each.
__device__ __forceinline__ float sqrt_pos(float x) { return sqrt_fast(x); }
__device__ __forceinline__ float sqrt_ball(float x) { return sqrt_fast(x); }

// Order-preserving map of a float onto uint32 (for the packed argmax key).
__device__ __forceinline__ uint32_t order_bits(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float order_bits_inv(uint32_t k) {
    uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

__device__ __forceinline__ bool pos_finite(float x) {
    return x > 0.f && x < CUDART_INF_F;  // false for NaN
}

__device__ __forceinline__ bool is_finite(float x) {
    return fabsf(x) < CUDART_INF_F;
}

// Per-state constants (A1).  Computed identically by every thread.
struct StateK {
    float bx, by;
    float kappa;         // 2 amax / vmax^2: length unit of the scaled form
    float inv_vmax;      // velocity unit of the scaled form
    float t_scale;       // vmax / (2 amax): scaled numerator -> seconds
    float ab;            // ball deceleration
    float two_ab;
    float at_scale;      // ab * t_scale: scaled numerator -> a * T
    float reach;         // reach radius in scaled units
    float Lh, hw;        // goal line x, half mouth width
    float inv_diag;
    float invK;
    float fK;            // fraction of the last sample (K * invK)
    int K, nopp;
    bool general;        // needs the speed clamp or a reach radius
    bool valid;
};

__device__ __forceinline__ StateK derive_state(const pps_state& st,
                                               const pps_params& prm,
                                               int jmax, int kmax) {
    StateK d;
    d.nopp = st.n_opp;
    d.K = st.K;
    bool ok = d.nopp >= 0 && d.nopp <= jmax && d.K >= 1 && d.K <= kmax &&
              pos_finite(st.ball_decel) && pos_finite(st.vmax) &&
              pos_finite(st.amax) && pos_finite(st.field_len) &&
              pos_finite(st.field_wid) && is_finite(st.goal_width) &&
              st.goal_width >= 0.f && is_finite(st.ball[0]) &&
              is_finite(st.ball[1]);
    if (!ok) d.nopp = 0;
    bool fast_opp = false;
    for (int j = 0; j < d.nopp; ++j) {
        float ux = st.opp_vel[j][0], uy = st.opp_vel[j][1];
        ok = ok && is_finite(st.opp_pos[j][0]) && is_finite(st.opp_pos[j][1]) &&
             is_finite(ux) && is_finite(uy);
        fast_opp |= __fmaf_rn(ux, ux, __fmul_rn(uy, uy)) >
                    __fmul_rn(st.vmax, st.vmax);
    }
    d.valid = ok;
    if (!ok) {
        d.nopp = 0;
        d.K = 1;
    }
    d.bx = st.ball[0];
    d.by = st.ball[1];
    const float two_amax = __fmul_rn(2.f, st.amax);
    d.kappa = __fdiv_rn(two_amax, __fmul_rn(st.vmax, st.vmax));
    d.inv_vmax = __frcp_rn(st.vmax);
    d.t_scale = __fdiv_rn(st.vmax, two_amax);
    d.ab = st.ball_decel;
    d.two_ab = __fmul_rn(2.f, st.ball_decel);
    d.at_scale = __fmul_rn(st.ball_decel, d.t_scale);
    d.reach = __fmul_rn(d.kappa, prm.reach_radius);
    d.Lh = __fmul_rn(0.5f, st.field_len);
    d.hw = __fmul_rn(0.5f, st.goal_width);
    d.inv_diag = __frcp_rn(__fsqrt_rn(__fmaf_rn(
        st.field_len, st.field_len, __fmul_rn(st.field_wid, st.field_wid))));
    d.invK = __frcp_rn((float)d.K);
    d.fK = __fmul_rn((float)d.K, d.invK);
    d.general = fast_opp || prm.reach_radius > 0.f;
    return d;
}

// kappa (x - y) with one rounding: x - y is split exactly into hi + lo.
__device__ __forceinline__ float scaled_diff(float x, float y, float kappa) {
    const float hi = __fsub_rn(x, y);
    const float t = __fsub_rn(hi, x);
    const float lo = __fadd_rn(__fsub_rn(x, __fsub_rn(hi, t)),
                               __fsub_rn(-y, t));
    return __fmaf_rn(kappa, hi, __fmul_rn(kappa, lo));
}

// Opponents in registers, in scaled units: kappa (b - o) and u / vmax per
// slot; unused slots are parked at kFar so they can never hold the minimum.
// kappa (b - o) is formed from the exact difference (an error-free two-sum)
// so it carries a single rounding.  Slots are held in pairs (float2) so
// that two opponents go through one packed f32x2 instruction.
template <int JMAX>
struct OppRegs {
    static_assert(JMAX % 2 == 0, "opponent slots come in pairs");
    float2 bx[JMAX / 2], by[JMAX / 2], ux[JMAX / 2], uy[JMAX / 2];
};

template <int JMAX>
__device__ __forceinline__ void load_opps(const pps_state& st,
                                          const StateK& sk,
                                          OppRegs<JMAX>& o) {
#pragma unroll
    for (int i = 0; i < JMAX / 2; ++i) {
        float v[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * i + h;
            if (j < sk.nopp) {
                v[h][0] = scaled_diff(sk.bx, st.opp_pos[j][0], sk.kappa);
                v[h][1] = scaled_diff(sk.by, st.opp_pos[j][1], sk.kappa);
                v[h][2] = __fmul_rn(st.opp_vel[j][0], sk.inv_vmax);
                v[h][3] = __fmul_rn(st.opp_vel[j][1], sk.inv_vmax);
            } else {
                v[h][0] = kFar;
                v[h][1] = kFar;
                v[h][2] = 0.f;
                v[h][3] = 0.f;
            }
        }
        o.bx[i] = make_float2(v[0][0], v[1][0]);
        o.by[i] = make_float2(v[0][1], v[1][1]);
        o.ux[i] = make_float2(v[0][2], v[1][2]);
        o.uy[i] = make_float2(v[0][3], v[1][3]);
    }
}

// A3: one opponent's intercept time at the sample p = b + f (c - b), as the
// scaled numerator n (time = n * vmax / (2 amax)).  In units where vmax = 1
// and lengths are multiplied by kappa = 2 amax / vmax^2, the along-line speed
// w' = w / vmax, distance d' = kappa d and q' = sqrt(w'^2 + d') give
//     n = (1 - w')^2 + d' - max(1 - q', 0)^2,
// and max(1 - q', 0) is one saturating add because 1 - q' <= 1.  GEN adds
// the clamp of w' to [-1, 1] and the reach radius (n = 0 within reach).
// Two opponents at a time: every FP32 operation but the saturating add,
// the clamps and the square roots is one packed f32x2 instruction, each
// half rounded exactly as the scalar operation (1 - w is fma(w, -1, 1),
// -m is m * -1: both exact rewrites).
__device__ __forceinline__ float one_minus_sat(float x) {
    float y;  // saturate(1 - x) = clamp(1 - x, 0, 1)
    asm("add.rn.sat.f32 %0, %1, %2;" : "=f"(y) : "f"(1.f), "f"(-x));
    return y;
}

template <bool GEN>
__device__ __forceinline__ float2 sbip_num2(float2 f, float2 cbx, float2 cby,
                                            float2 obx, float2 oby,
                                            float2 oux, float2 ouy,
                                            float reach) {
    const float2 one = make_float2(1.f, 1.f), mone = make_float2(-1.f, -1.f);
    const float2 rx = __ffma2_rn(f, cbx, obx);  // kappa (p - o)
    const float2 ry = __ffma2_rn(f, cby, oby);
    const float2 d2 = __ffma2_rn(rx, rx, __ffma2_rn(ry, ry, make_float2(kD2Floor, kD2Floor)));
    const float2 ig = make_float2(rsqrt_fast(d2.x), rsqrt_fast(d2.y));
    const float2 d = __fmul2_rn(d2, ig);
    float2 w = __fmul2_rn(__ffma2_rn(oux, rx, __fmul2_rn(ouy, ry)), ig);
    if (GEN) {
        w.x = fminf(fmaxf(w.x, -1.f), 1.f);
        w.y = fminf(fmaxf(w.y, -1.f), 1.f);
        const float2 dl = __fadd2_rn(d, make_float2(-reach, -reach));
        const float2 dc = make_float2(fmaxf(dl.x, 0.f), fmaxf(dl.y, 0.f));
        const float2 q = __ffma2_rn(w, w, dc);
        const float2 m = make_float2(one_minus_sat(sqrt_pos(q.x)),
                                     one_minus_sat(sqrt_pos(q.y)));
        const float2 e = __ffma2_rn(w, mone, one);
        const float2 num = __ffma2_rn(__fmul2_rn(m, mone), m, __ffma2_rn(e, e, dc));
        return make_float2(dl.x > 0.f ? num.x : 0.f, dl.y > 0.f ? num.y : 0.f);
    } else {
        const float2 q = __ffma2_rn(w, w, d);
        const float2 m = make_float2(one_minus_sat(sqrt_pos(q.x)),
                                     one_minus_sat(sqrt_pos(q.y)));
        const float2 e = __ffma2_rn(w, mone, one);
        return __ffma2_rn(__fmul2_rn(m, mone), m, __ffma2_rn(e, e, d));
    }
}

// The smallest scaled intercept numerator over the JMAX opponent slots at
// the sample f of the pass kappa (c - b) = (cbx, cby); the minimum is a
// balanced tree so the sample's critical path stays short.
template <int JMAX, bool GEN>
__device__ __forceinline__ float opp_min(float f, float cbx, float cby,
                                         const OppRegs<JMAX>& o, float reach) {
    const float2 f2 = make_float2(f, f), cx2 = make_float2(cbx, cbx),
                 cy2 = make_float2(cby, cby);
    float t[JMAX];
#pragma unroll
    for (int i = 0; i < JMAX / 2; ++i) {
        const float2 r = sbip_num2<GEN>(f2, cx2, cy2, o.bx[i], o.by[i],
                                        o.ux[i], o.uy[i], reach);
        t[2 * i] = r.x;
        t[2 * i + 1] = r.y;
    }
#pragma unroll
    for (int w = 1; w < JMAX; w *= 2)
#pragma unroll
        for (int j = 0; j + w < JMAX; j += 2 * w) t[j] = fminf(t[j], t[j + w]);
    return t[0];
}

// A3 + A4 over the K samples of one point.  mv[v] accumulates
// min_k (a T_k + sqrt(v^2 - 2 a s_k)); Trow (debug) receives T_k.
// STRIDE G > 1 (a power of two up to 32): G consecutive lanes share one
// point, lane l of the group taking samples l + 1, l + 1 + G, ... (the
// caller takes the minimum over the group).  STRIDE 0: G = g, chosen at
// run time.
template <int JMAX, int VMAX, bool GEN, bool TDBG, int KU = kKUnroll, int STRIDE = 1>
__device__ __forceinline__ void sample_loop(const StateK& sk,
                                            const OppRegs<JMAX>& o,
                                            float cbx, float cby,
                                            float twoabD,
                                            const float (&sp2)[PPS_MAX_SPEEDS],
                                            float (&mv)[VMAX], float* Trow,
                                            int g = STRIDE) {
    // speeds in pairs for the packed ball-time terms
    constexpr int VP = (VMAX + 1) / 2;
    float2 s2[VP];
#pragma unroll
    for (int i = 0; i < VP; ++i)
        s2[i] = make_float2(sp2[2 * i], sp2[2 * i + 1 < VMAX ? 2 * i + 1 : 2 * i]);
    const float2 tD2 = make_float2(twoabD, twoabD);
    // Float sample counter: exact for K <= 2^24, and keeps integer-to-float
    // conversions out of the loop.
    const float Kf = (float)sk.K;
    const int G = STRIDE ? STRIDE : g;
    const float k0 = G == 1 ? 1.f : (float)(1 + (threadIdx.x & (G - 1)));
    const float step = (float)G;
#pragma unroll KU
    for (float kf = k0; kf <= Kf; kf += step) {
        const float f = __fmul_rn(kf, sk.invK);
        const int k = (int)kf;
        const float n = opp_min<JMAX, GEN>(f, cbx, cby, o, sk.reach);
        if (TDBG && Trow)
            Trow[k - 1] = sk.nopp ? __fmul_rn(n, sk.t_scale) : CUDART_INF_F;
        const float aT = __fmul_rn(n, sk.at_scale);
        const float nf = -f;
        if (VMAX == 1) {
            mv[0] = fminf(mv[0], __fadd_rn(aT, sqrt_ball(__fmaf_rn(
                                                 nf, twoabD, sp2[0]))));
        } else {
            const float2 nf2 = make_float2(nf, nf), aT2 = make_float2(aT, aT);
#pragma unroll
            for (int i = 0; i < VP; ++i) {
                const float2 a = __ffma2_rn(nf2, tD2, s2[i]);
                const float2 t = __fadd2_rn(
                    aT2, make_float2(sqrt_ball(a.x), sqrt_ball(a.y)));
                mv[2 * i] = fminf(mv[2 * i], t.x);
                if (2 * i + 1 < VMAX) mv[2 * i + 1] = fminf(mv[2 * i + 1], t.y);
            }
        }
    }
}

// A5: largest opponent-free angular gap of the goal mouth seen from c
// (opponents opp[0..nopp) as discs of radius r; hw = half mouth width).
template <int JMAX>
__device__ __forceinline__ float shot_angle_of(const float (*opp)[2],
                                               int nopp, float hw, bool front,
                                               float cx, float cy, float gx,
                                               float r,
                                               float* gap_start = nullptr) {
    if (gap_start) *gap_start = 0.f;
    if (!front) return 0.f;
    const float lo = atan2f(__fsub_rn(-hw, cy), gx);
    const float hi = atan2f(__fsub_rn(hw, cy), gx);
    float s[JMAX], e[JMAX];
    bool all = false;
    int blocked = 0;
    const float r2 = __fmul_rn(r, r);
    // Post directions from c: A to the lower post, B to the upper one.
    const float ax = gx, ay = __fsub_rn(-hw, cy), by = __fsub_rn(hw, cy);
    const float a2r2 = __fmul_rn(__fmaf_rn(ax, ax, __fmul_rn(ay, ay)), r2);
    const float b2r2 = __fmul_rn(__fmaf_rn(ax, ax, __fmul_rn(by, by)), r2);
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        s[j] = 1e30f;
        e[j] = 1e30f;
        if (j < nopp) {
            const float dx = __fsub_rn(opp[j][0], cx);
            const float dy = __fsub_rn(opp[j][1], cy);
            const float d2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
            all |= d2 <= r2;
            // A disc can block part of the mouth only if its centre lies in
            // the wedge A..B or it reaches one of the two boundary rays;
            // the others are skipped before any trigonometry.
            const float ca = __fsub_rn(__fmul_rn(ax, dy), __fmul_rn(ay, dx));
            const float cb = __fsub_rn(__fmul_rn(ax, dy), __fmul_rn(by, dx));
            const bool inside = ca >= 0.f && cb <= 0.f;
            const bool near_a = __fmaf_rn(ax, dx, __fmul_rn(ay, dy)) > 0.f &&
                                __fmul_rn(ca, ca) <= a2r2;
            const bool near_b = __fmaf_rn(ax, dx, __fmul_rn(by, dy)) > 0.f &&
                                __fmul_rn(cb, cb) <= b2r2;
            if (!(inside || near_a || near_b)) continue;
            const float d = __fsqrt_rn(d2);
            const float phi = atan2f(dy, dx);
            const float half = asinf(fminf(__fdiv_rn(r, d), 1.f));
            s[j] = __fsub_rn(phi, half);
            e[j] = __fadd_rn(phi, half);
            ++blocked;
        }
    }
    if (all) return 0.f;
    // Sort the blocked intervals by start (odd-even transposition network;
    // unused slots sit at 1e30, last), then sweep: a gap opens wherever the
    // next start lies beyond every end so far.  Each gap is the difference
    // of an end (or lo) and the next start (or hi), as in the definition.
    // With at most one blocked interval the sorted order is that interval
    // (if any) followed by the unused slots: it is moved to the front
    // instead, and the sweep sees the same array.
    if (blocked >= 2) {
#pragma unroll
        for (int round = 0; round < JMAX; ++round)
#pragma unroll
            for (int i = round & 1; i + 1 < JMAX; i += 2) {
                const bool sw = s[i] > s[i + 1];
                const float s0 = fminf(s[i], s[i + 1]), s1 = fmaxf(s[i], s[i + 1]);
                const float e0 = sw ? e[i + 1] : e[i], e1 = sw ? e[i] : e[i + 1];
                s[i] = s0;
                s[i + 1] = s1;
                e[i] = e0;
                e[i + 1] = e1;
            }
    } else {
        float s0 = s[0], e0 = e[0];
#pragma unroll
        for (int j = 1; j < JMAX; ++j)
            if (s[j] < s0) {
                s0 = s[j];
                e0 = e[j];
            }
        s[0] = s0;
        e[0] = e0;
#pragma unroll
        for (int j = 1; j < JMAX; ++j) s[j] = e[j] = 1e30f;
    }
    float best = 0.f, cur = lo, start = lo;
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
        if (s[j] > cur && cur < hi) {
            const float gap = __fsub_rn(fminf(s[j], hi), cur);
            if (gap > best) {
                best = gap;
                start = cur;
            }
        }
        cur = fmaxf(cur, e[j]);
    }
    if (cur < hi) {
        const float gap = __fsub_rn(hi, cur);
        if (gap > best) {
            best = gap;
            start = cur;
        }
    }
    if (gap_start) *gap_start = start;
    return best;
}

template <int JMAX>
__device__ __forceinline__ float shot_angle(const pps_state& st,
                                            const StateK& sk, bool front,
                                            float cx, float cy, float gx,
                                            float r) {
    return shot_angle_of<JMAX>(st.opp_pos, sk.nopp, sk.hw, front, cx, cy, gx,
                               r);
}

// The same angle formed by the G lanes that share the point (G a power of
// two, JMAX <= G <= 32; every lane of the warp takes part, each group of G
// consecutive lanes with one point): lane i of the group forms opponent i's
// interval, the group sorts the intervals by start across its lanes (a
// bitonic network of shuffles; equal starts may come in either order, which
// changes no gap: the second of two equal starts lies at or below the
// first's end), the running maximum of the ends is a prefix scan, and each
// lane measures the gap in front of its interval.  Every interval, running
// maximum and gap is the value the sequential sweep forms (the same
// operations on the same operands; maxima are exact), so the angle is the
// same bit for bit.
template <int JMAX>
__device__ __forceinline__ float shot_angle_lanes(const float (*opp)[2],
                                                  int nopp, float hw,
                                                  bool front, float cx,
                                                  float cy, float gx, float r,
                                                  int G) {
    const int lane = threadIdx.x & 31, i = lane & (G - 1);
    const float lo = atan2f(__fsub_rn(-hw, cy), gx);
    const float hi = atan2f(__fsub_rn(hw, cy), gx);
    const float r2 = __fmul_rn(r, r);
    const float ax = gx, ay = __fsub_rn(-hw, cy), by = __fsub_rn(hw, cy);
    const float a2r2 = __fmul_rn(__fmaf_rn(ax, ax, __fmul_rn(ay, ay)), r2);
    const float b2r2 = __fmul_rn(__fmaf_rn(ax, ax, __fmul_rn(by, by)), r2);
    float s = 1e30f, e = 1e30f;
    bool covers = false;
    if (i < nopp && i < JMAX) {
        const float dx = __fsub_rn(opp[i][0], cx);
        const float dy = __fsub_rn(opp[i][1], cy);
        const float d2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
        covers = d2 <= r2;
        const float ca = __fsub_rn(__fmul_rn(ax, dy), __fmul_rn(ay, dx));
        const float cb = __fsub_rn(__fmul_rn(ax, dy), __fmul_rn(by, dx));
        const bool inside = ca >= 0.f && cb <= 0.f;
        const bool near_a = __fmaf_rn(ax, dx, __fmul_rn(ay, dy)) > 0.f &&
                            __fmul_rn(ca, ca) <= a2r2;
        const bool near_b = __fmaf_rn(ax, dx, __fmul_rn(by, dy)) > 0.f &&
                            __fmul_rn(cb, cb) <= b2r2;
        if (inside || near_a || near_b) {
            const float d = __fsqrt_rn(d2);
            const float phi = atan2f(dy, dx);
            const float half = asinf(fminf(__fdiv_rn(r, d), 1.f));
            s = __fsub_rn(phi, half);
            e = __fadd_rn(phi, half);
        }
    }
    const unsigned group =
        G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (lane & ~(G - 1));
    const bool all = (__ballot_sync(0xffffffffu, covers) & group) != 0u;
    for (int k = 2; k <= G; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            const float so = __shfl_xor_sync(0xffffffffu, s, j);
            const float eo = __shfl_xor_sync(0xffffffffu, e, j);
            const bool up = (i & k) == 0, lower = (i & j) == 0;
            if (lower == up ? so < s : so > s) {
                s = so;
                e = eo;
            }
        }
    // m: the largest end of the group's intervals up to lane i
    float m = e;
    for (int off = 1; off < G; off <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, m, off, G);
        if (i >= off) m = fmaxf(m, y);
    }
    const float before = __shfl_up_sync(0xffffffffu, m, 1, G);
    const float cur = i == 0 ? lo : fmaxf(lo, before);
    float best = 0.f;
    if (s > cur && cur < hi) best = __fsub_rn(fminf(s, hi), cur);
    for (int off = G >> 1; off > 0; off >>= 1)
        best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, off));
    const float last = fmaxf(lo, __shfl_sync(0xffffffffu, m, G - 1, G));
    if (last < hi) best = fmaxf(best, __fsub_rn(hi, last));
    return front && !all ? best : 0.f;
}

// Everything per grid point (A2..A6): margins, feasibility and scores for
// all VMAX speed slots.  Shared by the search and the finalize kernels so
// that the finalize reproduces the search's numbers bit for bit.
template <int JMAX, int VMAX>
struct PointResult {
    float margin[VMAX];
    float score[VMAX];
    bool feas[VMAX];
};

// Grid and speed list of the point being evaluated (shared by the whole
// batch in pps_search, per state in the batched plans).
struct ItemGrid {
    float g, x0, y0;
    int V;
};

// KU: unroll of the sample loop (samples a register block holds); it only
// replicates the loop body, so every result is the same bit for bit.
// STRIDE G > 1 (G consecutive lanes on the same point, G a power of two up
// to 32; STRIDE 0 takes G = g at run time): the lanes split the samples and
// the minimum over them is taken across the group -- the same minimum, so
// the same results bit for bit, in a G-th of the serial time (the finalize
// kernels, which re-evaluate one point per state with G = 32, and the
// refinement of small batches).  Every lane of the warp must take part.
template <int JMAX, int VMAX, bool TDBG, int KU = kKUnroll, int STRIDE = 1>
__device__ __forceinline__ void eval_point(const pps_params& prm,
                                           const ItemGrid& gr,
                                           const float (&sp)[PPS_MAX_SPEEDS],
                                           const float (&sp2)[PPS_MAX_SPEEDS],
                                           const pps_state& st,
                                           const StateK& sk,
                                           const OppRegs<JMAX>& o, int ix,
                                           int iy, float* Trow,
                                           PointResult<JMAX, VMAX>& res,
                                           int g = STRIDE) {
    // A2: the grid point and c - b are exact in FP64 (x0 + ix g and its
    // difference with the FP32 ball fit in 53 bits); the pass vector enters
    // the sample loop in scaled units, kappa (c - b), with one rounding.
    const double cxd = fma((double)ix, (double)gr.g, (double)gr.x0);
    const double cyd = fma((double)iy, (double)gr.g, (double)gr.y0);
    const double dxd = cxd - (double)sk.bx, dyd = cyd - (double)sk.by;
    const float cx = (float)cxd, cy = (float)cyd;
    const float cbx = (float)((double)sk.kappa * dxd);
    const float cby = (float)((double)sk.kappa * dyd);
    const float dxm = (float)dxd, dym = (float)dyd;
    const float D = __fsqrt_rn(__fmaf_rn(dxm, dxm, __fmul_rn(dym, dym)));
    const float twoabD = __fmul_rn(sk.two_ab, D);

    // Unused speed slots repeat the last speed; their results are dropped.
    float mv[VMAX];
#pragma unroll
    for (int v = 0; v < VMAX; ++v) mv[v] = CUDART_INF_F;
    if (sk.general)
        sample_loop<JMAX, VMAX, true, TDBG, KU, STRIDE>(sk, o, cbx, cby, twoabD, sp2,
                                                        mv, Trow, g);
    else
        sample_loop<JMAX, VMAX, false, TDBG, KU, STRIDE>(sk, o, cbx, cby, twoabD, sp2,
                                                         mv, Trow, g);
    if (STRIDE != 1) {
        const int G = STRIDE ? STRIDE : g;
#pragma unroll
        for (int v = 0; v < VMAX; ++v)
#pragma unroll
            for (int off = G >> 1; off > 0; off >>= 1)
                mv[v] = fminf(mv[v], __shfl_xor_sync(0xffffffffu, mv[v], off));
    }

    // A5: the receiver is in front of the goal line iff x0 + ix g < L/2,
    // decided exactly on the FP64 grid coordinate.
    const bool front = cxd < (double)sk.Lh;
    const float gx = (float)((double)sk.Lh - cxd);
    // The shot angle only enters the score of a feasible pass: points with
    // no feasible speed skip it (a warp runs it if any of its lanes needs it).
    const bool long_enough = D >= prm.min_pass_dist;
    bool any_ok = false;
#pragma unroll
    for (int v = 0; v < VMAX; ++v) {
        const bool reach = __fmaf_rn(-sk.fK, twoabD, sp2[v]) >= 0.f;
        float m;
        if (!reach)
            m = -CUDART_INF_F;
        else if (sk.nopp == 0)
            m = CUDART_INF_F;
        else
            m = __fdiv_rn(__fsub_rn(mv[v], sp[v]), sk.ab);
        const bool ok = sk.valid && reach && long_enough && m > prm.tau_safe;
        res.margin[v] = m;
        res.feas[v] = ok;
        any_ok |= ok && v < gr.V;
    }
    float theta = 0.f;
    if (STRIDE != 1 && (STRIDE ? STRIDE : g) >= JMAX) {
        // the group's lanes share the angle's opponents
        if (__any_sync(0xffffffffu, any_ok)) {
            const float t = shot_angle_lanes<JMAX>(
                st.opp_pos, sk.nopp, sk.hw, front, cx, cy, gx,
                prm.robot_radius, STRIDE ? STRIDE : g);
            theta = any_ok ? t : 0.f;
        }
    } else if (any_ok) {
        theta = shot_angle<JMAX>(st, sk, front, cx, cy, gx, prm.robot_radius);
    }
    const float dg = __fsqrt_rn(__fmaf_rn(gx, gx, __fmul_rn(cy, cy)));
    const float base =
        __fsub_rn(__fmul_rn(prm.w_angle,
                            __fmul_rn(theta, 0.318309886183790672f)),
                  __fmul_rn(prm.w_dist, __fmul_rn(dg, sk.inv_diag)));
#pragma unroll
    for (int v = 0; v < VMAX; ++v)
        res.score[v] =
            res.feas[v]
                ? __fadd_rn(base, __fmul_rn(prm.w_margin,
                                            fminf(res.margin[v],
                                                  prm.margin_cap)))
                : -CUDART_INF_F;
}

// An upper bound of every score eval_point can give the point (ix, iy),
// from the same arithmetic with (a) the shot angle replaced by the whole
// mouth's angle hi - lo (every open gap lies inside [lo, hi]) and (b) each
// speed's margin taken over kBoundSamples of the K samples only (the margin
// is the minimum over all of them; each chosen sample is computed exactly
// as the sample loop computes it).  FP32 rounding is monotone, so the bound
// needs no slack; it holds when w_angle >= 0 and w_margin >= 0, which the
// caller checks.
constexpr int kBoundSamples = 4;

template <int JMAX, int VMAX>
__device__ __forceinline__ float score_bound(const pps_params& prm,
                                             const ItemGrid& gr,
                                             const float (&sp)[PPS_MAX_SPEEDS],
                                             const float (&sp2)[PPS_MAX_SPEEDS],
                                             const StateK& sk,
                                             const OppRegs<JMAX>& o, int ix,
                                             int iy) {
    const double cxd = fma((double)ix, (double)gr.g, (double)gr.x0);
    const double cyd = fma((double)iy, (double)gr.g, (double)gr.y0);
    const double dxd = cxd - (double)sk.bx, dyd = cyd - (double)sk.by;
    const float cy = (float)cyd;
    const float cbx = (float)((double)sk.kappa * dxd);
    const float cby = (float)((double)sk.kappa * dyd);
    const float dxm = (float)dxd, dym = (float)dyd;
    const float D = __fsqrt_rn(__fmaf_rn(dxm, dxm, __fmul_rn(dym, dym)));
    const float twoabD = __fmul_rn(sk.two_ab, D);
    // kBoundSamples of the sample loop's samples, spread along the pass
    // (sample k = ceil(K i / kBoundSamples), the last one being K), each
    // computed exactly as the loop computes it: f = k * (1 / K)
    float mv[VMAX];
#pragma unroll
    for (int v = 0; v < VMAX; ++v) mv[v] = CUDART_INF_F;
#pragma unroll
    for (int i = 1; i <= kBoundSamples; ++i) {
        const int k = (sk.K * i + kBoundSamples - 1) / kBoundSamples;
        const float f = __fmul_rn((float)k, sk.invK);
        const float n = sk.general
                            ? opp_min<JMAX, true>(f, cbx, cby, o, sk.reach)
                            : opp_min<JMAX, false>(f, cbx, cby, o, sk.reach);
        const float aT = __fmul_rn(n, sk.at_scale);
        const float nf = -f;
#pragma unroll
        for (int v = 0; v < VMAX; ++v)
            mv[v] = fminf(mv[v], __fadd_rn(aT, sqrt_ball(__fmaf_rn(
                                                   nf, twoabD, sp2[v]))));
    }
    float mb = -CUDART_INF_F;
#pragma unroll
    for (int v = 0; v < VMAX; ++v) {
        if (v >= gr.V) continue;
        if (!(__fmaf_rn(-sk.fK, twoabD, sp2[v]) >= 0.f)) continue;
        const float m = sk.nopp == 0
                            ? CUDART_INF_F
                            : __fdiv_rn(__fsub_rn(mv[v], sp[v]), sk.ab);
        mb = fmaxf(mb, m);
    }
    const bool front = cxd < (double)sk.Lh;
    const float gx = (float)((double)sk.Lh - cxd);
    float theta = 0.f;
    if (front) {
        const float lo = atan2f(__fsub_rn(-sk.hw, cy), gx);
        const float hi = atan2f(__fsub_rn(sk.hw, cy), gx);
        theta = fmaxf(__fsub_rn(hi, lo), 0.f);
    }
    const float dg = __fsqrt_rn(__fmaf_rn(gx, gx, __fmul_rn(cy, cy)));
    const float base =
        __fsub_rn(__fmul_rn(prm.w_angle,
                            __fmul_rn(theta, 0.318309886183790672f)),
                  __fmul_rn(prm.w_dist, __fmul_rn(dg, sk.inv_diag)));
    return __fadd_rn(base,
                     __fmul_rn(prm.w_margin, fminf(mb, prm.margin_cap)));
}

__device__ __forceinline__ unsigned long long warp_max_u64(
    unsigned long long x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long y = __shfl_xor_sync(0xffffffffu, x, off);
        x = y > x ? y : x;
    }
    return x;
}

// ------------------------------------------------------------ the kernels
// Every warp is an independent persistent worker: a work item is (state,
// 32 consecutive grid points), items are dealt round-robin over all warps
// of the grid, and nothing is shared between the warps of a CTA -- no
// shared memory, no barriers, so a warp that finishes early (for example
// because none of its points needed a shot angle) starts its next item at
// once.  The state record is read through the read-only cache (all lanes
// read the same address, one transaction per warp).
//
// EXT instances also honour a.list (search only the listed states), a.skip
// (states to leave untouched) and write a.dbg_point; the plain instances
// carry none of these checks in their loop.
// Longest run of consecutive items a warp takes at once (see search_kernel).
constexpr long long kMaxRun = 64;

template <int JMAX, int VMAX, bool EXT = false>
__global__ void __launch_bounds__(search_tpb<JMAX, VMAX>(), 1)
    search_kernel(const SearchArgs a) {
    constexpr int kWarps = search_tpb<JMAX, VMAX>() / 32;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * kWarps;
    const long long gw = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const bool listed = EXT && a.list;
    const long long n_items =
        (long long)(listed ? *a.list_n : a.n_states) * a.words;

    // Each warp takes runs of R consecutive items (mostly one state), the
    // runs dealt round-robin; the state's constants and opponents are
    // derived once per run and state.  R grows with the batch up to kMaxRun
    // while every warp still gets at least 8 runs, so small batches keep
    // all warps busy.
    const long long R = n_items >= warps * 8 * kMaxRun
                            ? kMaxRun
                            : (n_items >= warps * 8 ? n_items / (warps * 8) : 1);
    int cur = -1;
    StateK sk;
    OppRegs<JMAX> o;
    for (long long item = gw * R, j = 0; item < n_items;
         item = (++j == R) ? (j = 0, item - (R - 1) + warps * R) : item + 1) {
        const int i = (int)(item / a.words);
        const int chunk = (int)(item - (long long)i * a.words);
        const int s = listed ? a.list[i] : i;
        if (EXT && a.skip && a.skip[s]) continue;
        const pps_state& st = a.states[s];
        if (s != cur) {
            sk = derive_state(st, a.prm, JMAX, a.kmax);
            load_opps<JMAX>(st, sk, o);
            cur = s;
        }

        const int p = chunk * 32 + lane;
        const bool active = p < a.P;
        const int pc = active ? p : a.P - 1;
        const int iy = pc / a.nx, ix = pc - iy * a.nx;

        PointResult<JMAX, VMAX> r;
        const ItemGrid gr{a.g, a.x0, a.y0, a.V};
        if (a.dbg_T) {
            float* Trow = a.dbg_T + ((long long)s * a.P + pc) * a.T_stride;
            eval_point<JMAX, VMAX, true>(a.prm, gr, a.speed, a.speed2, st, sk,
                                         o, ix, iy, active ? Trow : nullptr, r);
        } else {
            eval_point<JMAX, VMAX, false>(a.prm, gr, a.speed, a.speed2, st, sk,
                                          o, ix, iy, nullptr, r);
        }

        // A6: mask words, debug outputs, feasible count.
        int cnt = 0;
        unsigned long long key = 0ull;
#pragma unroll
        for (int v = 0; v < VMAX; ++v) {
            const bool f = active && v < a.V && r.feas[v];
            cnt += f;
            if (f) {
                // A7: packed (score, ~idx) -- larger is better, and on equal
                // scores the smaller candidate index wins.
                const uint32_t idx = (uint32_t)(v * a.P + p);
                const unsigned long long k2 =
                    ((unsigned long long)order_bits(r.score[v]) << 32) |
                    (unsigned long long)(~idx);
                key = k2 > key ? k2 : key;
            }
            if (v < a.V) {
                const uint32_t word = __ballot_sync(0xffffffffu, f);
                if (a.mask && lane == 0)
                    a.mask[((long long)s * a.V + v) * a.words + chunk] = word;
                if (active) {
                    const long long o2 = ((long long)s * a.V + v) * a.P + p;
                    if (a.dbg_margin) a.dbg_margin[o2] = r.margin[v];
                    if (a.dbg_score) a.dbg_score[o2] = r.score[v];
                }
            }
        }
        if (EXT && a.dbg_point && active) {
            float bs = -CUDART_INF_F;
#pragma unroll
            for (int v = 0; v < VMAX; ++v)
                if (v < a.V && r.feas[v]) bs = fmaxf(bs, r.score[v]);
            a.dbg_point[(long long)s * a.P + p] = bs;
        }
        key = warp_max_u64(key);
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0) {
            if (key) atomicMax(a.keys + s, key);
            if (cnt) atomicAdd(a.counts + s, cnt);
        }
    }
}

// CTAs of 128 threads for the finalize kernels of n states (a warp each).
__host__ __device__ constexpr unsigned finalize_blocks(long long n) {
    return (unsigned)((n + 3) / 4);
}

// Per state: decode the key, re-evaluate the winning point for its margin
// and check that the score reproduces.  One warp per state (4 a CTA,
// finalize_blocks(n) CTAs); the lanes share the re-evaluation's samples and
// lane 0 writes the record.
template <int JMAX, int VMAX>
__global__ void __launch_bounds__(128) finalize_kernel(const SearchArgs a) {
    const int s = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (s >= a.n_states) return;
    if (a.skip && a.skip[s]) return;
    const pps_state& st = a.states[s];
    const StateK sk = derive_state(st, a.prm, JMAX, a.kmax);
    pps_best b;
    b.n_feasible = a.counts[s];
    b.status = sk.valid ? PPS_STATE_OK : PPS_STATE_INVALID;
    const unsigned long long key = a.keys[s];
    if (!sk.valid || key == 0ull) {
        b.idx = sk.valid ? -1 : -2;
        b.ix = b.iy = b.speed_idx = -1;
        b.score = -CUDART_INF_F;
        b.margin = -CUDART_INF_F;
        b.n_feasible = sk.valid ? b.n_feasible : 0;
    } else {
        const uint32_t idx = ~(uint32_t)(key & 0xffffffffull);
        const int v = (int)(idx / (uint32_t)a.P);
        const int p = (int)(idx - (uint32_t)v * (uint32_t)a.P);
        b.idx = (int)idx;
        b.speed_idx = v;
        b.iy = p / a.nx;
        b.ix = p - b.iy * a.nx;
        b.score = order_bits_inv((uint32_t)(key >> 32));
        OppRegs<JMAX> o;
        load_opps<JMAX>(st, sk, o);
        PointResult<JMAX, VMAX> r;
        const ItemGrid gr{a.g, a.x0, a.y0, a.V};
        eval_point<JMAX, VMAX, false, kKUnroll, 32>(a.prm, gr, a.speed, a.speed2, st,
                                                    sk, o, b.ix, b.iy, nullptr, r);
        float m = 0.f, sc = 0.f;
        bool f = false;
#pragma unroll
        for (int w = 0; w < VMAX; ++w)
            if (w == v) {
                m = r.margin[w];
                sc = r.score[w];
                f = r.feas[w];
            }
        b.margin = m;
        if (!f || __float_as_uint(sc) != __float_as_uint(b.score))
            b.status |= PPS_STATE_INCONSISTENT;
    }
    if ((threadIdx.x & 31) == 0) a.best[s] = b;
}

}  // namespace pps

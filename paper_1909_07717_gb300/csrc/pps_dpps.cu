// pps_dpps.cu -- the paper's own parameterisation of the passing-point
// search (include/pps.h, "Directions x kick powers"): from the ball holder,
// n_dir directions x n_pow kick powers; for every candidate the ball's path
// is searched for the first teammate and the first opponent that can reach
// it (SBIP, Sec. 4.2), and feasible candidates get the Sec. 4.3 score.
//
// Work items are chunks of 1024 consecutive candidates of one state, taken
// by warps from a queue.  A warp's lanes are persistent: each lane holds one
// candidate and takes one ball-path sample per loop trip -- the teammates
// first, the opponents only if a teammate receives -- and takes the next
// candidate as soon as its current one ends, so no lane idles while the
// chunk has candidates left.  Paths are prepared 32 at a time by the whole
// warp; feasible candidates wait in shared memory and are scored 32 at a
// time.  The state's two robot groups sit in shared memory as pairs (two
// robots per packed f32x2 instruction, the same intercept arithmetic as the
// receive-point search).

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>

#include "pps.h"
#include "pps_internal.h"
#include "pps_search.cuh"

char* pps_thread_error_buffer();

namespace {

using pps::OppRegs;

constexpr int kTPB = 512;
constexpr int kWarps = kTPB / 32;
constexpr int kChunk = 1024;  // candidates per work item, a multiple of 32
constexpr int kSmallChunk = 256;  // the same for the last states: the queue's
                                  // tail drains in small items
constexpr int kRing = 64;     // prepared paths a warp holds (a power of 2, > 62)
constexpr int kPend = 64;     // feasible candidates awaiting a score (> 62)
constexpr unsigned kFull = 0xffffffffu;
constexpr int kSamples = 8;   // ball-path samples a lane takes per loop trip

struct DArgs {
    const pps_dstate* states;
    int n_states;
    int words;   // mask words per state
    int kmax;
    pps_dparams prm;
    pps_dbest* best;
    uint32_t* mask;  // may be null
    float* dbg;      // may be null: t_team, t_opp, score per candidate
    unsigned long long* keys;
    int* counts;
    unsigned long long* queue;  // work-item counter, zero at launch
    int s_small;                // states from s_small on: kSmallChunk items
};

// Per-state constants (validity as in derive_state, for both groups).
struct DStateK {
    float bx, by, kappa, inv_vmax, t_scale, at_scale, ab, two_ab, reach;
    float hl, hw, inv_diag, invK;
    int K, nteam, nopp;
    bool general, valid;
};

__device__ __forceinline__ bool finite_(float x) { return fabsf(x) < CUDART_INF_F; }
__device__ __forceinline__ bool pos_(float x) { return x > 0.f && x < CUDART_INF_F; }

template <int J>
__device__ __forceinline__ DStateK derive_dstate(const pps_dstate& st,
                                                 const pps_dparams& prm,
                                                 int kmax) {
    DStateK d;
    d.nteam = st.n_team;
    d.nopp = st.n_opp;
    d.K = st.K;
    bool ok = d.nteam >= 0 && d.nteam <= J && d.nopp >= 0 && d.nopp <= J &&
              d.K >= 1 && d.K <= kmax && pos_(st.ball_decel) && pos_(st.vmax) &&
              pos_(st.amax) && pos_(st.field_len) && pos_(st.field_wid) &&
              finite_(st.goal_width) && st.goal_width >= 0.f &&
              finite_(st.ball[0]) && finite_(st.ball[1]);
    if (!ok) d.nteam = d.nopp = 0;
    bool fast = false;
    for (int j = 0; j < d.nteam; ++j) {
        const float ux = st.team_vel[j][0], uy = st.team_vel[j][1];
        ok = ok && finite_(st.team_pos[j][0]) && finite_(st.team_pos[j][1]) &&
             finite_(ux) && finite_(uy);
        fast |= __fmaf_rn(ux, ux, __fmul_rn(uy, uy)) > __fmul_rn(st.vmax, st.vmax);
    }
    for (int j = 0; j < d.nopp; ++j) {
        const float ux = st.opp_vel[j][0], uy = st.opp_vel[j][1];
        ok = ok && finite_(st.opp_pos[j][0]) && finite_(st.opp_pos[j][1]) &&
             finite_(ux) && finite_(uy);
        fast |= __fmaf_rn(ux, ux, __fmul_rn(uy, uy)) > __fmul_rn(st.vmax, st.vmax);
    }
    d.valid = ok;
    if (!ok) {
        d.nteam = d.nopp = 0;
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
    d.hl = __fmul_rn(0.5f, st.field_len);
    d.hw = __fmul_rn(0.5f, st.goal_width);
    d.inv_diag = __frcp_rn(__fsqrt_rn(__fmaf_rn(
        st.field_len, st.field_len, __fmul_rn(st.field_wid, st.field_wid))));
    d.invK = __frcp_rn((float)d.K);
    d.general = fast || prm.reach_radius > 0.f;
    return d;
}

// A group's robots in pairs, scaled relative to the ball (unused slots
// parked far away), as load_opps does for the opponents of a pps_state.
template <int J>
__device__ __forceinline__ void load_group(const float (*pos)[2],
                                           const float (*vel)[2], int n,
                                           const DStateK& sk, OppRegs<J>& g) {
#pragma unroll
    for (int i = 0; i < J / 2; ++i) {
        float v[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * i + h;
            if (j < n) {
                v[h][0] = pps::scaled_diff(sk.bx, pos[j][0], sk.kappa);
                v[h][1] = pps::scaled_diff(sk.by, pos[j][1], sk.kappa);
                v[h][2] = __fmul_rn(vel[j][0], sk.inv_vmax);
                v[h][3] = __fmul_rn(vel[j][1], sk.inv_vmax);
            } else {
                v[h][0] = v[h][1] = pps::kFar;
                v[h][2] = v[h][3] = 0.f;
            }
        }
        g.bx[i] = make_float2(v[0][0], v[1][0]);
        g.by[i] = make_float2(v[0][1], v[1][1]);
        g.ux[i] = make_float2(v[0][2], v[1][2]);
        g.uy[i] = make_float2(v[0][3], v[1][3]);
    }
}

// The smallest scaled intercept numerator of the group at sample f of the
// pass (cbx, cby) and the robot holding it (the first on ties).
template <int J, bool GEN>
__device__ __forceinline__ float group_min(float f, float cbx, float cby,
                                           const OppRegs<J>& g, float reach,
                                           int& who) {
    const float2 f2 = make_float2(f, f), cx2 = make_float2(cbx, cbx),
                 cy2 = make_float2(cby, cby);
    float t[J];
    int w[J];
#pragma unroll
    for (int i = 0; i < J / 2; ++i) {
        const float2 r = pps::sbip_num2<GEN>(f2, cx2, cy2, g.bx[i], g.by[i],
                                             g.ux[i], g.uy[i], reach);
        t[2 * i] = r.x;
        t[2 * i + 1] = r.y;
        w[2 * i] = 2 * i;
        w[2 * i + 1] = 2 * i + 1;
    }
#pragma unroll
    for (int s = 1; s < J; s *= 2)
#pragma unroll
        for (int j = 0; j + s < J; j += 2 * s)
            if (t[j + s] < t[j]) {
                t[j] = t[j + s];
                w[j] = w[j + s];
            }
    who = w[0];
    return t[0];
}

// One lane's candidate pass, fixed by its path: rolling speed v, path
// length S along (ux, uy), ending by a stop or at the field edge.
template <int J, bool GEN>
__device__ __forceinline__ float group_min_val(float f, float cbx, float cby,
                                               const OppRegs<J>& g, float reach) {
    return pps::opp_min<J, GEN>(f, cbx, cby, g, reach);
}

struct Path {
    float ux, uy, v, S;
    bool stopped;
};

// SBIP of one group along the path: the first sample k = 1..K at which a
// robot of the group can be no later than the ball (a T <= v - root, i.e.
// T <= t_ball); at the stop sample of a stopping path the group always
// gets the ball, at max(T, v / a).  Returns the time (+inf if none).
template <int J>
__device__ __forceinline__ float group_first(const DStateK& sk,
                                             const OppRegs<J>& g,
                                             const Path& p, bool active,
                                             int& k_out, int& who) {
    k_out = 0;
    who = -1;
    if (!active || sk.K < 1) return CUDART_INF_F;
    const float cbx = __fmul_rn(sk.kappa, __fmul_rn(p.S, p.ux));
    const float cby = __fmul_rn(sk.kappa, __fmul_rn(p.S, p.uy));
    const float v2 = __fmul_rn(p.v, p.v);
    const float twoaS = __fmul_rn(sk.two_ab, p.S);
    // The sample loop keeps only the group's minimum; the robot holding it
    // is found again at the sample the loop stops at.
    auto holder = [&](float f) {
        int w;
        if (sk.general)
            group_min<J, true>(f, cbx, cby, g, sk.reach, w);
        else
            group_min<J, false>(f, cbx, cby, g, sk.reach, w);
        return w;
    };
    for (int k = 1; k <= sk.K; ++k) {
        const float f = __fmul_rn((float)k, sk.invK);
        const float n = sk.general ? group_min_val<J, true>(f, cbx, cby, g, sk.reach)
                                   : group_min_val<J, false>(f, cbx, cby, g, sk.reach);
        if (p.stopped && k == sk.K) {
            k_out = k;
            who = holder(f);
            return fmaxf(__fmul_rn(n, sk.t_scale), __fdiv_rn(p.v, sk.ab));
        }
        const float root = pps::sqrt_ball(fmaxf(__fmaf_rn(-f, twoaS, v2), 0.f));
        if (__fadd_rn(__fmul_rn(n, sk.at_scale), root) <= p.v) {
            k_out = k;
            who = holder(f);
            // t_ball(s) = 2 s / (v + sqrt(v^2 - 2 a s))
            return __fdiv_rn(__fmul_rn(2.f, __fmul_rn(f, p.S)), __fadd_rn(p.v, root));
        }
    }
    return CUDART_INF_F;
}

struct DRes {
    float t_team, t_opp, score, rx, ry;
    int k_team, recv;
    bool feas;
};

// The ball's path of candidate (dir, pw): direction 2 pi dir / n_dir,
// rolling speed slide x the pw-th kick power, length up to its stop or the
// field edge, whichever comes first.
__device__ __forceinline__ Path dpps_path(const pps_dstate& st, const DStateK& sk,
                                          const pps_dparams& prm, int dir, int pw) {
    Path p;
    float sn, cs;
    sincospif(__fdiv_rn(2.f * (float)dir, (float)prm.n_dir), &sn, &cs);
    p.ux = cs;
    p.uy = sn;
    const float v0 = prm.n_pow > 1
                         ? __fmaf_rn((float)pw,
                                     __fdiv_rn(prm.v_hi - prm.v_lo,
                                               (float)(prm.n_pow - 1)),
                                     prm.v_lo)
                         : prm.v_lo;
    p.v = __fmul_rn(prm.slide, v0);
    const float s_stop = __fdiv_rn(__fmul_rn(p.v, p.v), sk.two_ab);
    float s_out = CUDART_INF_F;
    const float hwid = __fmul_rn(0.5f, st.field_wid);
    if (p.ux > 0.f) s_out = fminf(s_out, __fdiv_rn(sk.hl - sk.bx, p.ux));
    if (p.ux < 0.f) s_out = fminf(s_out, __fdiv_rn(-sk.hl - sk.bx, p.ux));
    if (p.uy > 0.f) s_out = fminf(s_out, __fdiv_rn(hwid - sk.by, p.uy));
    if (p.uy < 0.f) s_out = fminf(s_out, __fdiv_rn(-hwid - sk.by, p.uy));
    s_out = fmaxf(s_out, 0.f);
    p.stopped = s_stop <= s_out;
    p.S = p.stopped ? s_stop : s_out;
    return p;
}

// Sec. 4.3 score of a feasible candidate along (ux, uy), received at
// (rx, ry) at t_team, first reached by an opponent at t_opp.
template <int J>
__device__ __forceinline__ float dpps_score(const pps_dstate& st, const DStateK& sk,
                                            const pps_dparams& prm, float ux,
                                            float uy, float t_team, float t_opp,
                                            float rx, float ry) {
    const float gx = __fsub_rn(sk.hl, rx);
    const float theta = pps::shot_angle_of<J>(st.opp_pos, sk.nopp, sk.hw,
                                              rx < sk.hl, rx, ry, gx,
                                              prm.robot_radius);
    const float dg = __fsqrt_rn(__fmaf_rn(gx, gx, __fmul_rn(ry, ry)));
    // the turn from the pass direction u to the shot direction g - r, as
    // atan2(|u x (g - r)|, u . (g - r)): the same angle as the acos of the
    // normalised dot product, without its loss of precision when the two
    // directions nearly agree
    float refr = 0.f;
    if (dg > 0.f) {
        const float dot = __fmaf_rn(ux, gx, __fmul_rn(uy, -ry));
        const float crs = __fmaf_rn(ux, -ry, -__fmul_rn(uy, gx));
        refr = atan2f(fabsf(crs), dot);
    }
    const float delta = __fsub_rn(t_opp, t_team);
    const float inv_pi = 0.318309886183790672f;
    float sc = -__fmul_rn(prm.w_time, t_team);
    sc = __fadd_rn(sc, __fmul_rn(prm.w_angle, __fmul_rn(theta, inv_pi)));
    sc = __fsub_rn(sc, __fmul_rn(prm.w_dist, __fmul_rn(dg, sk.inv_diag)));
    sc = __fsub_rn(sc, __fmul_rn(prm.w_refr, __fmul_rn(refr, inv_pi)));
    sc = __fadd_rn(sc, __fmul_rn(prm.w_delta, fminf(delta, prm.delta_cap)));
    return sc;
}

// The receive point: sample k_team of K along the path.
__device__ __forceinline__ void receive_point(const DStateK& sk, float ux, float uy,
                                              float S, int k_team, float& rx,
                                              float& ry) {
    const float s = __fmul_rn(__fmul_rn((float)k_team, sk.invK), S);
    rx = __fmaf_rn(s, ux, sk.bx);
    ry = __fmaf_rn(s, uy, sk.by);
}

// Everything for one candidate (dir, pw), one candidate a thread: the
// finalize kernel's check of the search's best.
template <int J>
__device__ __forceinline__ void dpps_eval(const pps_dstate& st,
                                          const DStateK& sk,
                                          const pps_dparams& prm, int dir,
                                          int pw, bool active,
                                          const OppRegs<J>& team,
                                          const OppRegs<J>& opp, DRes& r) {
    const Path p = dpps_path(st, sk, prm, dir, pw);
    r.feas = false;
    r.score = -CUDART_INF_F;
    r.t_opp = CUDART_INF_F;
    r.rx = r.ry = 0.f;
    r.t_team = group_first<J>(sk, team, p, active && sk.valid, r.k_team, r.recv);
    const bool got = r.t_team < CUDART_INF_F;
    {
        int k_opp, who;
        r.t_opp = group_first<J>(sk, opp, p, got, k_opp, who);
    }
    // Sec. 4.3: safe when the first opponent comes more than tau later
    r.feas = got && __fsub_rn(r.t_opp, r.t_team) > prm.tau_delta;
    if (got) receive_point(sk, p.ux, p.uy, p.S, r.k_team, r.rx, r.ry);
    if (r.feas)
        r.score = dpps_score<J>(st, sk, prm, p.ux, p.uy, r.t_team, r.t_opp,
                                r.rx, r.ry);
}

// A 16-byte shared-memory load that stays where it is written: the
// compiler may not hoist it out of the sample loop (the group would then
// take 64 registers).
__device__ __forceinline__ float4 lds4(const void* p) {
    float4 v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(a));
    return v;
}

// Sample f of the pass (cbx, cby) against a group in shared memory
// (16-byte aligned), two robot pairs to a 16-byte load: per robot the
// arithmetic of opp_min, and its minimum tree.
template <int J, bool GEN>
__device__ __forceinline__ float group_min_smem(float f, float cbx, float cby,
                                                const OppRegs<J>& g, float reach) {
    static_assert(J % 4 == 0, "pairs are read two at a time");
    const float2 f2 = make_float2(f, f), cx2 = make_float2(cbx, cbx),
                 cy2 = make_float2(cby, cby);
    float t[J];
#pragma unroll
    for (int i = 0; i < J / 2; i += 2) {
        const float4 bx = lds4(&g.bx[i]);
        const float4 by = lds4(&g.by[i]);
        const float4 ux = lds4(&g.ux[i]);
        const float4 uy = lds4(&g.uy[i]);
        float2 r = pps::sbip_num2<GEN>(f2, cx2, cy2, make_float2(bx.x, bx.y),
                                       make_float2(by.x, by.y), make_float2(ux.x, ux.y),
                                       make_float2(uy.x, uy.y), reach);
        t[2 * i] = r.x;
        t[2 * i + 1] = r.y;
        r = pps::sbip_num2<GEN>(f2, cx2, cy2, make_float2(bx.z, bx.w),
                                make_float2(by.z, by.w), make_float2(ux.z, ux.w),
                                make_float2(uy.z, uy.w), reach);
        t[2 * i + 2] = r.x;
        t[2 * i + 3] = r.y;
    }
#pragma unroll
    for (int w = 1; w < J; w *= 2)
#pragma unroll
        for (int j = 0; j + w < J; j += 2 * w) t[j] = fminf(t[j], t[j + w]);
    return t[0];
}

// A warp's shared memory: the state's constants and two robot groups, the
// prepared paths, each lane's current candidate, the feasible candidates
// awaiting their score, the lanes' argmax keys and counts, and the chunk's
// mask words.  What the sample loop reads only when a phase ends lives
// here rather than in registers.
template <int J>
struct __align__(16) WarpSmem {
    DStateK sk;
    alignas(16) OppRegs<J> team;
    float pad[4];  // the opponents 16 bytes further on, so that lanes in the
                   // two phases read the same robot slot from other banks
    OppRegs<J> opp;
    float ring[5][kRing];  // prepared paths: ux, uy, v, S, stopped
    float cur[10][32];     // the lane's candidate: ux, uy, S, t_team, k_team,
                           // and its sample terms cbx, cby, v^2, 2 a S, v
    float pend[7][kPend];  // candidate (bits), t_team, t_opp, rx, ry, ux, uy
    unsigned long long key[32];
    int cnt[32];
    uint32_t mask[kChunk / 32];
};

// Score the feasible candidate in pending slot `slot` and fold it into the
// lane's argmax key and count.
template <int J>
__device__ __noinline__ void score_pending(const DArgs& a, const pps_dstate& st,
                                           int s, WarpSmem<J>& w, int slot, int lane) {
    const uint32_t idx = __float_as_uint(w.pend[0][slot]);
    const float t_team = w.pend[1][slot], t_opp = w.pend[2][slot];
    const float sc = dpps_score<J>(st, w.sk, a.prm, w.pend[5][slot], w.pend[6][slot],
                                   t_team, t_opp, w.pend[3][slot], w.pend[4][slot]);
    const unsigned long long k =
        ((unsigned long long)pps::order_bits(sc) << 32) | (unsigned long long)(~idx);
    if (k > w.key[lane]) w.key[lane] = k;
    ++w.cnt[lane];
    if (a.dbg) {
        float* d = a.dbg + ((long long)s * a.prm.n_dir * a.prm.n_pow + idx) * 3;
        d[0] = t_team;
        d[1] = t_opp;
        d[2] = sc;
    }
}

// The path of candidate c into its ring slot.
template <int J>
__device__ __noinline__ void prepare_path(const DArgs& a, const pps_dstate& st,
                                          WarpSmem<J>& w, int c) {
    const int dir = c / a.prm.n_pow;
    const Path p = dpps_path(st, w.sk, a.prm, dir, c - dir * a.prm.n_pow);
    const int slot = c & (kRing - 1);
    w.ring[0][slot] = p.ux;
    w.ring[1][slot] = p.uy;
    w.ring[2][slot] = p.v;
    w.ring[3][slot] = p.S;
    w.ring[4][slot] = p.stopped ? 1.f : 0.f;
}

// Candidates [c0, c1) of state s (c0 a multiple of 32, c1 - c0 at most
// kChunk) with persistent
// lanes, kSamples samples a loop trip.  Per lane and phase the samples k = 1..K
// are taken in order and the phase ends at the first interception, exactly
// as group_first does: the same arithmetic on the same values, so every
// time and score equals the one-candidate-a-thread evaluation bit for bit
// (a trip's later samples are discarded when an earlier one ends the
// phase).
template <int J, bool GEN>
__device__ __forceinline__ void run_chunk(const DArgs& a, const pps_dstate& st, int s,
                                          int c0, int c1, WarpSmem<J>& w, int lane) {
    const DStateK& sk = w.sk;
    const unsigned lt = (1u << lane) - 1u;
    w.mask[lane] = 0u;  // kChunk / 32 == 32 words, one a lane
    w.key[lane] = 0ull;
    w.cnt[lane] = 0;
    __syncwarp();
    // prepared paths wait in ring slot c mod kRing: the candidates prepared
    // and not yet taken are at most 63 consecutive ones
    int next = c0;   // first candidate not yet prepared
    int taken = c0;  // first prepared candidate not yet handed out
    int npend = 0;
    int cand = -1, k = 0;
    bool opp = false, stopped = false;
    for (;;) {
        const unsigned need = __ballot_sync(kFull, cand < 0);
        if (need) {
            const int want = __popc(need);
            if (next - taken < want && next < c1) {
                // the next (up to) 32 paths, one a lane; at most 31 are
                // waiting, so the ring's 64 slots never overrun
                __syncwarp();
                if (next + lane < c1) prepare_path<J>(a, st, w, next + lane);
                next = min(next + 32, c1);
                __syncwarp();
            }
            const int r = __popc(need & lt);
            if (cand < 0 && taken + r < next) {
                const int slot = (taken + r) & (kRing - 1);
                const float ux = w.ring[0][slot], uy = w.ring[1][slot];
                const float S = w.ring[3][slot];
                const float v = w.ring[2][slot];
                stopped = w.ring[4][slot] != 0.f;
                w.cur[0][lane] = ux;
                w.cur[1][lane] = uy;
                w.cur[2][lane] = S;
                w.cur[5][lane] = __fmul_rn(sk.kappa, __fmul_rn(S, ux));
                w.cur[6][lane] = __fmul_rn(sk.kappa, __fmul_rn(S, uy));
                w.cur[7][lane] = __fmul_rn(v, v);
                w.cur[8][lane] = __fmul_rn(sk.two_ab, S);
                w.cur[9][lane] = v;
                cand = taken + r;
                opp = false;
                k = 1;
            }
            taken += min(want, next - taken);
        }
        if (__all_sync(kFull, cand < 0)) break;

        // samples k .. k + kSamples - 1 of the lane's current phase: the
        // first of them (up to K) at which the group gets the ball ends the
        // phase
        bool done = false, feas = false;
        float t_opp = CUDART_INF_F;
        if (cand >= 0) {
            const OppRegs<J>& g = opp ? w.opp : w.team;
            const float cbx = w.cur[5][lane], cby = w.cur[6][lane], v2 = w.cur[7][lane],
                        twoaS = w.cur[8][lane], v = w.cur[9][lane];
            int kk = k;
            float f = 0.f, n = 0.f, root = 0.f;
            bool end = false, stop = false, hit = false;
#pragma unroll 1
            for (int j = 0; j < kSamples; ++j) {
                kk = k + j;
                f = __fmul_rn((float)kk, sk.invK);
                n = group_min_smem<J, GEN>(f, cbx, cby, g, sk.reach);
                end = kk == sk.K;
                // at the stop the group always gets the ball
                stop = stopped && end;
                root = pps::sqrt_ball(fmaxf(__fmaf_rn(-f, twoaS, v2), 0.f));
                hit = stop || __fadd_rn(__fmul_rn(n, sk.at_scale), root) <= v;
                if (hit || end) break;
            }
            float t = CUDART_INF_F;
            if (stop)
                t = fmaxf(__fmul_rn(n, sk.t_scale), __fdiv_rn(v, sk.ab));
            else if (hit)
                // t_ball(s) = 2 s / (v + sqrt(v^2 - 2 a s))
                t = __fdiv_rn(__fmul_rn(2.f, __fmul_rn(f, w.cur[2][lane])),
                              __fadd_rn(v, root));
            end = end || hit;
            if (end && !opp && t < CUDART_INF_F) {
                // a teammate receives: search the opponents from sample 1
                w.cur[3][lane] = t;
                w.cur[4][lane] = __int_as_float(kk);
                opp = true;
                k = 1;
            } else if (end) {
                done = true;
                if (!opp) {
                    w.cur[3][lane] = CUDART_INF_F;
                } else {
                    t_opp = t;
                    // Sec. 4.3: safe when the first opponent comes more
                    // than tau later
                    feas = __fsub_rn(t_opp, w.cur[3][lane]) > a.prm.tau_delta;
                }
            } else {
                k += kSamples;
            }
        }
        const unsigned fm = __ballot_sync(kFull, feas);
        if (feas) {
            const int slot = npend + __popc(fm & lt);
            const float ux = w.cur[0][lane], uy = w.cur[1][lane];
            float rx, ry;
            receive_point(sk, ux, uy, w.cur[2][lane], __float_as_int(w.cur[4][lane]),
                          rx, ry);
            w.pend[0][slot] = __uint_as_float((uint32_t)cand);
            w.pend[1][slot] = w.cur[3][lane];
            w.pend[2][slot] = t_opp;
            w.pend[3][slot] = rx;
            w.pend[4][slot] = ry;
            w.pend[5][slot] = ux;
            w.pend[6][slot] = uy;
            atomicOr(&w.mask[(cand - c0) >> 5], 1u << (cand & 31));
        } else if (done && a.dbg) {
            float* d = a.dbg + ((long long)s * a.prm.n_dir * a.prm.n_pow + cand) * 3;
            d[0] = w.cur[3][lane];
            d[1] = t_opp;
            d[2] = -CUDART_INF_F;
        }
        if (done) cand = -1;
        npend += __popc(fm);
        if (npend >= 32) {
            // a full warp of scores (at most 31 stay behind, so the 64
            // pending slots never overrun)
            __syncwarp();
            npend -= 32;
            score_pending<J>(a, st, s, w, npend + lane, lane);
            __syncwarp();
        }
    }
    __syncwarp();
    if (lane < npend) score_pending<J>(a, st, s, w, lane, lane);
    if (a.mask) {
        const int c = c0 + 32 * lane;
        if (c < c1) a.mask[(long long)s * a.words + (c >> 5)] = w.mask[lane];
    }
    const unsigned long long key = pps::warp_max_u64(w.key[lane]);
    const int cnt = __reduce_add_sync(kFull, w.cnt[lane]);
    if (lane == 0) {
        if (key) atomicMax(a.keys + s, key);
        if (cnt) atomicAdd(a.counts + s, cnt);
    }
    __syncwarp();
}

// An invalid state: no candidate is feasible; its mask words are zero.
__device__ __forceinline__ void invalid_chunk(const DArgs& a, int s, long long P,
                                              int c0, int c1, int lane) {
    if (a.dbg)
        for (int c = c0 + lane; c < c1; c += 32) {
            float* d = a.dbg + ((long long)s * P + c) * 3;
            d[0] = CUDART_INF_F;
            d[1] = CUDART_INF_F;
            d[2] = -CUDART_INF_F;
        }
    if (a.mask) {
        const int c = c0 + 32 * lane;
        if (c < c1) a.mask[(long long)s * a.words + (c >> 5)] = 0u;
    }
}

template <int J>
__global__ void __launch_bounds__(kTPB, 2) dpps_kernel(const DArgs a) {
    extern __shared__ __align__(16) unsigned char dpps_smem[];
    WarpSmem<J>& w = reinterpret_cast<WarpSmem<J>*>(dpps_smem)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const long long P = (long long)a.prm.n_dir * a.prm.n_pow;
    const long long big = (P + kChunk - 1) / kChunk;
    const long long small = (P + kSmallChunk - 1) / kSmallChunk;
    const unsigned long long n_big = (unsigned long long)a.s_small * big;
    const unsigned long long n_items =
        n_big + (unsigned long long)(a.n_states - a.s_small) * small;
    int cur = -1;
    const DStateK& sk = w.sk;
    for (;;) {
        unsigned long long item = 0ull;
        if (lane == 0) item = atomicAdd(a.queue, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= n_items) break;
        int s, c0, c1;
        if (item < n_big) {
            s = (int)(item / (unsigned long long)big);
            c0 = (int)(item - (unsigned long long)s * big) * kChunk;
            c1 = (int)min((long long)c0 + kChunk, P);
        } else {
            const unsigned long long j = item - n_big;
            const int q = (int)(j / (unsigned long long)small);
            s = a.s_small + q;
            c0 = (int)(j - (unsigned long long)q * small) * kSmallChunk;
            c1 = (int)min((long long)c0 + kSmallChunk, P);
        }
        const pps_dstate& st = a.states[s];
        if (s != cur) {
            cur = s;
            __syncwarp();
            if (lane == 0) {
                const DStateK d = derive_dstate<J>(st, a.prm, a.kmax);
                w.sk = d;
                load_group<J>(st.team_pos, st.team_vel, d.nteam, d, w.team);
                load_group<J>(st.opp_pos, st.opp_vel, d.nopp, d, w.opp);
            }
            __syncwarp();
        }
        if (!sk.valid)
            invalid_chunk(a, s, P, c0, c1, lane);
        else if (sk.general)
            run_chunk<J, true>(a, st, s, c0, c1, w, lane);
        else
            run_chunk<J, false>(a, st, s, c0, c1, w, lane);
    }
}

// Per state: decode the best key and evaluate that candidate again for its
// details; the score must reproduce bit for bit.
template <int J>
__global__ void __launch_bounds__(128) dpps_finalize(const DArgs a) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.n_states) return;
    const pps_dstate& st = a.states[s];
    const DStateK sk = derive_dstate<J>(st, a.prm, a.kmax);
    pps_dbest b;
    b.n_feasible = sk.valid ? a.counts[s] : 0;
    b.status = sk.valid ? PPS_STATE_OK : PPS_STATE_INVALID;
    b.reserved = 0;
    const unsigned long long key = a.keys[s];
    if (!sk.valid || key == 0ull) {
        b.idx = sk.valid ? -1 : -2;
        b.dir = b.pow = b.receiver = -1;
        b.score = -CUDART_INF_F;
        b.t_team = b.t_opp = CUDART_INF_F;
        b.recv[0] = b.recv[1] = 0.f;
    } else {
        const uint32_t idx = ~(uint32_t)(key & 0xffffffffull);
        b.idx = (int)idx;
        b.dir = (int)(idx / (uint32_t)a.prm.n_pow);
        b.pow = (int)(idx - (uint32_t)b.dir * (uint32_t)a.prm.n_pow);
        b.score = pps::order_bits_inv((uint32_t)(key >> 32));
        DRes r;
        OppRegs<J> team, opp;
        load_group<J>(st.team_pos, st.team_vel, sk.nteam, sk, team);
        load_group<J>(st.opp_pos, st.opp_vel, sk.nopp, sk, opp);
        dpps_eval<J>(st, sk, a.prm, b.dir, b.pow, true, team, opp, r);
        b.receiver = r.recv;
        b.t_team = r.t_team;
        b.t_opp = r.t_opp;
        b.recv[0] = r.rx;
        b.recv[1] = r.ry;
        if (!r.feas || __float_as_uint(r.score) != __float_as_uint(b.score))
            b.status |= PPS_STATE_INCONSISTENT;
    }
    a.best[s] = b;
    // the scratch is left zeroed for the next call
    a.keys[s] = 0ull;
    a.counts[s] = 0;
}

// Sec. 4.1, Eq. 1-2, one thread per query.
template <int J>
__global__ void __launch_bounds__(128)
    pass_power_kernel(const pps_dstate* __restrict__ states, int n_states,
                      const pps_pass_query* __restrict__ q, int n, float buffer,
                      const pps_dparams prm, int kmax,
                      pps_pass_power* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const pps_pass_query qu = q[i];
    pps_pass_power o;
    o.v0 = o.v1 = o.t_pass = o.t_recv = CUDART_NAN_F;
    o.clamped = 0;
    o.status = PPS_STATE_INVALID;
    if (qu.state >= 0 && qu.state < n_states) {
        const pps_dstate& st = states[qu.state];
        const DStateK sk = derive_dstate<J>(st, prm, kmax);
        if (sk.valid && qu.receiver >= 0 && qu.receiver < sk.nteam &&
            finite_(qu.target[0]) && finite_(qu.target[1])) {
            // the receiver's arrival: the intercept form at the target
            const float rx = pps::scaled_diff(qu.target[0], st.team_pos[qu.receiver][0], sk.kappa);
            const float ry = pps::scaled_diff(qu.target[1], st.team_pos[qu.receiver][1], sk.kappa);
            const float ux = __fmul_rn(st.team_vel[qu.receiver][0], sk.inv_vmax);
            const float uy = __fmul_rn(st.team_vel[qu.receiver][1], sk.inv_vmax);
            const float2 z = make_float2(0.f, 0.f);
            const float nrm =
                (sk.general
                     ? pps::sbip_num2<true>(z, z, z, make_float2(rx, rx),
                                            make_float2(ry, ry), make_float2(ux, ux),
                                            make_float2(uy, uy), sk.reach)
                     : pps::sbip_num2<false>(z, z, z, make_float2(rx, rx),
                                             make_float2(ry, ry), make_float2(ux, ux),
                                             make_float2(uy, uy), sk.reach))
                    .x;
            const float T = __fmul_rn(nrm, sk.t_scale);
            const float t = __fadd_rn(T, buffer);
            const float dx = __fsub_rn(qu.target[0], sk.bx);
            const float dy = __fsub_rn(qu.target[1], sk.by);
            const float d = __fsqrt_rn(__fmaf_rn(dx, dx, __fmul_rn(dy, dy)));
            const float half_at2 = __fmul_rn(0.5f * sk.ab, __fmul_rn(t, t));
            float v1 = t > 0.f ? __fdiv_rn(__fadd_rn(d, half_at2), t) : CUDART_INF_F;
            const float vmin = __fsqrt_rn(__fmul_rn(sk.two_ab, d));
            if (v1 < vmin || d < half_at2) v1 = vmin;
            float v0 = __fdiv_rn(v1, prm.slide);
            int cl = 0;
            if (v0 < prm.v_lo) { v0 = prm.v_lo; cl = 1; }
            if (v0 > prm.v_hi) { v0 = prm.v_hi; cl = 1; }
            o.v0 = v0;
            o.v1 = v1;
            o.t_pass = t;
            o.t_recv = T;
            o.clamped = cl;
            o.status = PPS_STATE_OK;
        }
    }
    out[i] = o;
}

// Sec. 4.4, one thread per query.
template <int J>
__global__ void __launch_bounds__(128)
    shoot_kernel(const pps_dstate* __restrict__ states, int n_states,
                 const pps_shot_query* __restrict__ q, int n, float v_shot,
                 float theta_min, const pps_dparams prm, int kmax,
                 pps_shot* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const pps_shot_query qu = q[i];
    pps_shot o;
    o.theta = o.dir = o.t_line = o.t_opp = CUDART_NAN_F;
    o.shoot = 0;
    o.status = PPS_STATE_INVALID;
    if (qu.state >= 0 && qu.state < n_states && finite_(qu.from[0]) &&
        finite_(qu.from[1])) {
        const pps_dstate& st = states[qu.state];
        DStateK sk = derive_dstate<J>(st, prm, kmax);
        if (sk.valid) {
            const float cx = qu.from[0], cy = qu.from[1];
            float start;
            const float theta = pps::shot_angle_of<J>(
                st.opp_pos, sk.nopp, sk.hw, cx < sk.hl, cx, cy,
                __fsub_rn(sk.hl, cx), prm.robot_radius, &start);
            const float dir = __fmaf_rn(0.5f, theta, start);
            float sn, cs;
            sincosf(dir, &sn, &cs);
            o.theta = theta;
            o.dir = dir;
            o.t_line = o.t_opp = CUDART_INF_F;
            if (theta > 0.f && cs > 0.f) {
                Path p;
                p.ux = cs;
                p.uy = sn;
                p.v = __fmul_rn(prm.slide, v_shot);
                p.S = __fdiv_rn(__fsub_rn(sk.hl, cx), cs);
                p.stopped = false;
                const float disc = __fmaf_rn(-sk.two_ab, p.S, __fmul_rn(p.v, p.v));
                if (disc >= 0.f) {
                    o.t_line = __fdiv_rn(__fmul_rn(2.f, p.S),
                                         __fadd_rn(p.v, __fsqrt_rn(disc)));
                    // the opponents, relative to the shooter
                    sk.bx = cx;
                    sk.by = cy;
                    OppRegs<J> g;
                    load_group<J>(st.opp_pos, st.opp_vel, sk.nopp, sk, g);
                    int k, who;
                    o.t_opp = group_first<J>(sk, g, p, true, k, who);
                    o.shoot = theta >= theta_min &&
                              (!(o.t_opp < CUDART_INF_F) ||
                               __fsub_rn(o.t_opp, o.t_line) > prm.tau_delta);
                }
            }
            o.status = PPS_STATE_OK;
        }
    }
    out[i] = o;
}

template <int J>
cudaError_t launch(DArgs a, int num_sms, cudaStream_t st) {
    const size_t smem = sizeof(WarpSmem<J>) * kWarps;
    cudaError_t e = cudaFuncSetAttribute(
        dpps_kernel<J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int occ = pps_occupancy((const void*)dpps_kernel<J>, kTPB, smem);
    const long long P = (long long)a.prm.n_dir * a.prm.n_pow;
    const long long grid_max = (long long)num_sms * occ;
    // the last states, about two small items a warp, in small items
    long long n_small = (2 * grid_max * kWarps * kSmallChunk + P - 1) / P;
    if (n_small > a.n_states) n_small = a.n_states;
    a.s_small = a.n_states - (int)n_small;
    const long long items = (long long)a.s_small * ((P + kChunk - 1) / kChunk) +
                            n_small * ((P + kSmallChunk - 1) / kSmallChunk);
    long long grid = (items + kWarps - 1) / kWarps;
    if (grid > grid_max) grid = grid_max;
    e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    dpps_kernel<J><<<(unsigned)grid, kTPB, smem, st>>>(a);
    dpps_finalize<J><<<(a.n_states + 127) / 128, 128, 0, st>>>(a);
    return cudaGetLastError();
}

bool fin(float x) { return std::isfinite(x); }

}  // namespace

extern "C" pps_status pps_dpps_default_params(pps_dparams* out) {
    if (!out) return PPS_EINVAL;
    out->n_dir = 128;
    out->n_pow = 64;
    out->v_lo = 1.f;
    out->v_hi = 6.5f;
    out->slide = 5.f / 7.f;
    out->tau_delta = 0.f;
    out->delta_cap = 1.f;
    out->w_time = out->w_angle = out->w_dist = out->w_refr = out->w_delta = 1.f;
    out->robot_radius = 0.09f;
    out->reach_radius = 0.f;
    return PPS_OK;
}

extern "C" size_t pps_dpps_mask_words(const pps_dparams* p) {
    if (!p || p->n_dir < 1 || p->n_pow < 1) return 0;
    return ((size_t)p->n_dir * (size_t)p->n_pow + 31) / 32;
}

extern "C" pps_status pps_dpps_search(pps_ctx* ctx, const pps_dstate* states,
                                      int n_states, const pps_dparams* params,
                                      pps_dbest* out_best, uint32_t* out_mask,
                                      float* out_dbg) {
    PPS_RANGE("pps_dpps_search");
    if (!ctx) return PPS_EINVAL;
    if (pps_ctx_failed(ctx))
        return pps_ctx_error(ctx, PPS_ECUDA, "context failed earlier; call pps_reset");
    if (n_states == 0) return PPS_OK;
    if (!states || !out_best || n_states < 0 || n_states > pps_ctx_max_states(ctx))
        return pps_ctx_error(ctx, PPS_EINVAL,
                             "pps_dpps_search: n_states outside 0..max_states or NULL buffer");
    pps_dparams p;
    if (params)
        p = *params;
    else
        pps_dpps_default_params(&p);
    const float vals[] = {p.v_lo, p.v_hi, p.slide, p.tau_delta, p.delta_cap,
                          p.w_time, p.w_angle, p.w_dist, p.w_refr, p.w_delta,
                          p.robot_radius, p.reach_radius};
    for (float x : vals)
        if (!fin(x))
            return pps_ctx_error(ctx, PPS_EINVAL, "pps_dpps_search: non-finite parameter");
    if (p.n_dir < 1 || p.n_dir > 1024 || p.n_pow < 1 || p.n_pow > 256 ||
        !(p.v_lo > 0.f) || p.v_hi < p.v_lo || !(p.slide > 0.f) || p.slide > 1.f ||
        p.robot_radius < 0.f || p.reach_radius < 0.f)
        return pps_ctx_error(ctx, PPS_EINVAL, "pps_dpps_search: parameter out of range");

    cudaError_t e = cudaSetDevice(pps_ctx_device(ctx));
    DArgs a;
    std::memset(&a, 0, sizeof a);
    a.states = states;
    a.n_states = n_states;
    a.words = (int)pps_dpps_mask_words(&p);
    a.kmax = pps_ctx_max_K(ctx);
    a.prm = p;
    a.best = out_best;
    a.mask = out_mask;
    a.dbg = out_dbg;
    pps_ctx_scratch(ctx, &a.keys, &a.counts);
    a.queue = pps_ctx_work_counter(ctx);
    cudaStream_t st = pps_ctx_stream(ctx);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(a.keys, 0, sizeof(unsigned long long) * n_states, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.counts, 0, sizeof(int) * n_states, st);
    if (e == cudaSuccess) {
        const int sms = pps_ctx_num_sms(ctx);
        e = pps_ctx_jmax(ctx) == 8 ? launch<8>(a, sms, st) : launch<16>(a, sms, st);
    }
    if (e != cudaSuccess) return pps_ctx_cuda_error(ctx, e, "pps_dpps_search");
    return PPS_OK;
}

extern "C" pps_status pps_pass_powers(pps_ctx* ctx, const pps_dstate* states,
                                      int n_states, const pps_pass_query* queries,
                                      int n_queries, float buffer,
                                      const pps_dparams* params,
                                      pps_pass_power* out) {
    PPS_RANGE("pps_pass_powers");
    if (!ctx) return PPS_EINVAL;
    if (pps_ctx_failed(ctx))
        return pps_ctx_error(ctx, PPS_ECUDA, "context failed earlier; call pps_reset");
    if (n_queries == 0) return PPS_OK;
    if (n_queries < 0 || n_states < 0 || !states || !queries || !out)
        return pps_ctx_error(ctx, PPS_EINVAL, "pps_pass_powers: bad buffers or counts");
    pps_dparams p;
    if (params)
        p = *params;
    else
        pps_dpps_default_params(&p);
    if (!fin(buffer) || buffer < 0.f || !(p.slide > 0.f) || p.slide > 1.f ||
        !(p.v_lo > 0.f) || !fin(p.v_hi) || p.v_hi < p.v_lo ||
        !fin(p.reach_radius) || p.reach_radius < 0.f)
        return pps_ctx_error(ctx, PPS_EINVAL, "pps_pass_powers: parameter out of range");
    cudaError_t e = cudaSetDevice(pps_ctx_device(ctx));
    cudaStream_t st = pps_ctx_stream(ctx);
    const unsigned grid = (unsigned)((n_queries + 127) / 128);
    if (e == cudaSuccess) {
        if (pps_ctx_jmax(ctx) == 8)
            pass_power_kernel<8><<<grid, 128, 0, st>>>(states, n_states, queries, n_queries,
                                                       buffer, p, pps_ctx_max_K(ctx), out);
        else
            pass_power_kernel<16><<<grid, 128, 0, st>>>(states, n_states, queries, n_queries,
                                                        buffer, p, pps_ctx_max_K(ctx), out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return pps_ctx_cuda_error(ctx, e, "pps_pass_powers");
    return PPS_OK;
}

extern "C" pps_status pps_shoot(pps_ctx* ctx, const pps_dstate* states, int n_states,
                                const pps_shot_query* queries, int n_queries,
                                float v_shot, float theta_min,
                                const pps_dparams* params, pps_shot* out) {
    PPS_RANGE("pps_shoot");
    if (!ctx) return PPS_EINVAL;
    if (pps_ctx_failed(ctx))
        return pps_ctx_error(ctx, PPS_ECUDA, "context failed earlier; call pps_reset");
    if (n_queries == 0) return PPS_OK;
    if (n_queries < 0 || n_states < 0 || !states || !queries || !out)
        return pps_ctx_error(ctx, PPS_EINVAL, "pps_shoot: bad buffers or counts");
    pps_dparams p;
    if (params)
        p = *params;
    else
        pps_dpps_default_params(&p);
    if (!(v_shot > 0.f) || !fin(v_shot) || !fin(theta_min) || !(p.slide > 0.f) ||
        p.slide > 1.f || !fin(p.tau_delta) || !fin(p.robot_radius) ||
        p.robot_radius < 0.f || !fin(p.reach_radius) || p.reach_radius < 0.f)
        return pps_ctx_error(ctx, PPS_EINVAL, "pps_shoot: parameter out of range");
    cudaError_t e = cudaSetDevice(pps_ctx_device(ctx));
    cudaStream_t st = pps_ctx_stream(ctx);
    const unsigned grid = (unsigned)((n_queries + 127) / 128);
    if (e == cudaSuccess) {
        if (pps_ctx_jmax(ctx) == 8)
            shoot_kernel<8><<<grid, 128, 0, st>>>(states, n_states, queries, n_queries,
                                                  v_shot, theta_min, p, pps_ctx_max_K(ctx), out);
        else
            shoot_kernel<16><<<grid, 128, 0, st>>>(states, n_states, queries, n_queries,
                                                   v_shot, theta_min, p, pps_ctx_max_K(ctx), out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return pps_ctx_cuda_error(ctx, e, "pps_shoot");
    return PPS_OK;
}

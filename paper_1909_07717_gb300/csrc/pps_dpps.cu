// pps_dpps.cu -- the paper's own parameterisation of the passing-point
// search (include/pps.h, "Directions x kick powers"): from the ball holder,
// n_dir directions x n_pow kick powers; for every candidate the ball's path
// is searched for the first teammate and the first opponent that can reach
// it (SBIP, Sec. 4.2), and feasible candidates get the Sec. 4.3 score.
//
// One warp per (state, direction, 32 powers), one lane per candidate.  A
// group's robots sit in registers as pairs (two robots per packed f32x2
// instruction, the same intercept arithmetic as the receive-point search);
// the teammates are searched first, the opponents only for candidates a
// teammate receives.  Each lane stops at its group's first interception.

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
constexpr long long kMaxRun = 64;

struct DArgs {
    const pps_dstate* states;
    int n_states;
    int chunks;  // ceil(n_pow / 32)
    int words;   // mask words per state
    int kmax;
    pps_dparams prm;
    pps_dbest* best;
    uint32_t* mask;  // may be null
    float* dbg;      // may be null: t_team, t_opp, score per candidate
    unsigned long long* keys;
    int* counts;
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

// Everything for one candidate (dir, pw); shared by the search and the
// finalize kernels so that both give the same numbers.
template <int J>
__device__ __forceinline__ void dpps_eval(const pps_dstate& st,
                                          const DStateK& sk,
                                          const pps_dparams& prm, int dir,
                                          int pw, bool active,
                                          const OppRegs<J>& team,
                                          const OppRegs<J>& opp, DRes& r) {
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
    if (got) {
        const float s = __fmul_rn(__fmul_rn((float)r.k_team, sk.invK), p.S);
        r.rx = __fmaf_rn(s, p.ux, sk.bx);
        r.ry = __fmaf_rn(s, p.uy, sk.by);
    }
    if (r.feas) {
        const float gx = __fsub_rn(sk.hl, r.rx);
        const float theta = pps::shot_angle_of<J>(st.opp_pos, sk.nopp, sk.hw,
                                                  r.rx < sk.hl, r.rx, r.ry, gx,
                                                  prm.robot_radius);
        const float dg = __fsqrt_rn(__fmaf_rn(gx, gx, __fmul_rn(r.ry, r.ry)));
        // the turn from the pass direction u to the shot direction g - r,
        // as atan2(|u x (g - r)|, u . (g - r)): the same angle as the acos
        // of the normalised dot product, without its loss of precision
        // when the two directions nearly agree
        float refr = 0.f;
        if (dg > 0.f) {
            const float dot = __fmaf_rn(p.ux, gx, __fmul_rn(p.uy, -r.ry));
            const float crs = __fmaf_rn(p.ux, -r.ry, -__fmul_rn(p.uy, gx));
            refr = atan2f(fabsf(crs), dot);
        }
        const float delta = __fsub_rn(r.t_opp, r.t_team);
        const float inv_pi = 0.318309886183790672f;
        float sc = -__fmul_rn(prm.w_time, r.t_team);
        sc = __fadd_rn(sc, __fmul_rn(prm.w_angle, __fmul_rn(theta, inv_pi)));
        sc = __fsub_rn(sc, __fmul_rn(prm.w_dist, __fmul_rn(dg, sk.inv_diag)));
        sc = __fsub_rn(sc, __fmul_rn(prm.w_refr, __fmul_rn(refr, inv_pi)));
        sc = __fadd_rn(sc, __fmul_rn(prm.w_delta, fminf(delta, prm.delta_cap)));
        r.score = sc;
    }
}

template <int J>
__global__ void __launch_bounds__(kTPB, 2) dpps_kernel(const DArgs a) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (kTPB / 32);
    const long long gw = (long long)blockIdx.x * (kTPB / 32) + (threadIdx.x >> 5);
    const long long per_state = (long long)a.prm.n_dir * a.chunks;
    const long long n_items = (long long)a.n_states * per_state;
    // runs of R consecutive items (mostly one state), dealt round-robin, as
    // in the receive-point search; the state's constants once per run
    const long long R = n_items >= warps * 8 * kMaxRun
                            ? kMaxRun
                            : (n_items >= warps * 8 ? n_items / (warps * 8) : 1);
    // the warp's state's two robot groups, in shared memory: every lane
    // reads the same robot at the same time (a broadcast), and the groups
    // need no registers
    __shared__ OppRegs<J> groups[kTPB / 32][2];
    OppRegs<J>& team = groups[threadIdx.x >> 5][0];
    OppRegs<J>& opp = groups[threadIdx.x >> 5][1];
    int cur = -1;
    DStateK sk;
    for (long long item = gw * R, j = 0; item < n_items;
         item = (++j == R) ? (j = 0, item - (R - 1) + warps * R) : item + 1) {
        const int s = (int)(item / per_state);
        const int rem = (int)(item - (long long)s * per_state);
        const int dir = rem / a.chunks, chunk = rem - dir * a.chunks;
        const int pw = chunk * 32 + lane;
        const bool active = pw < a.prm.n_pow;
        const pps_dstate& st = a.states[s];
        if (s != cur) {
            sk = derive_dstate<J>(st, a.prm, a.kmax);
            cur = s;
            __syncwarp();
            if (lane == 0) {
                load_group<J>(st.team_pos, st.team_vel, sk.nteam, sk, team);
                load_group<J>(st.opp_pos, st.opp_vel, sk.nopp, sk, opp);
            }
            __syncwarp();
        }
        DRes r;
        dpps_eval<J>(st, sk, a.prm, dir, active ? pw : 0, active, team, opp, r);
        const bool f = active && r.feas;
        const uint32_t idx = (uint32_t)(dir * a.prm.n_pow + pw);
        if (a.dbg && active) {
            float* d = a.dbg + ((long long)s * a.prm.n_dir * a.prm.n_pow + idx) * 3;
            d[0] = r.t_team;
            d[1] = r.t_opp;
            d[2] = r.score;
        }
        if (a.mask) {
            if ((a.prm.n_pow & 31) == 0) {
                const uint32_t word = __ballot_sync(0xffffffffu, f);
                if (lane == 0) a.mask[(long long)s * a.words + idx / 32] = word;
            } else if (f) {
                atomicOr(a.mask + (long long)s * a.words + idx / 32, 1u << (idx & 31));
            }
        }
        unsigned long long key = 0ull;
        if (f)
            key = ((unsigned long long)pps::order_bits(r.score) << 32) |
                  (unsigned long long)(~idx);
        key = pps::warp_max_u64(key);
        const int cnt = __reduce_add_sync(0xffffffffu, f ? 1 : 0);
        if (lane == 0) {
            if (key) atomicMax(a.keys + s, key);
            if (cnt) atomicAdd(a.counts + s, cnt);
        }
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
cudaError_t launch(const DArgs& a, int num_sms, cudaStream_t st) {
    const int occ = pps_occupancy((const void*)dpps_kernel<J>, kTPB, 0);
    const long long items = (long long)a.n_states * a.prm.n_dir * a.chunks;
    long long grid = (items + kTPB / 32 - 1) / (kTPB / 32);
    if (grid > (long long)num_sms * occ) grid = (long long)num_sms * occ;
    dpps_kernel<J><<<(unsigned)grid, kTPB, 0, st>>>(a);
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
    a.chunks = (p.n_pow + 31) / 32;
    a.words = (int)pps_dpps_mask_words(&p);
    a.kmax = pps_ctx_max_K(ctx);
    a.prm = p;
    a.best = out_best;
    a.mask = out_mask;
    a.dbg = out_dbg;
    pps_ctx_scratch(ctx, &a.keys, &a.counts);
    cudaStream_t st = pps_ctx_stream(ctx);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(a.keys, 0, sizeof(unsigned long long) * n_states, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.counts, 0, sizeof(int) * n_states, st);
    if (e == cudaSuccess && out_mask && (p.n_pow & 31) != 0)
        e = cudaMemsetAsync(out_mask, 0, sizeof(uint32_t) * (size_t)a.words * n_states, st);
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

// pps_run.cu -- running points (Sec. 5.1-5.2; include/pps.h, "Running
// points"): the attacking half rasterised at g, every grid point scored by
// the weighted sum of the five criteria (Eq. 4), the best point of each of
// the four ball-dependent zones, and the zones chosen for the supporters.
//
// One CTA per state (grid-stride over states).  A warp derives the state's
// constants first (validity, the guards inside the defence area, the
// nearest opponent's squared distance to the ball) into shared memory; then
// every thread scores points idx = tid, tid + 256, ... in row-major order
// (coalesced when the dense scores are written) and keeps, per zone, the
// 64-bit key (ordered score, ~idx); the keys meet in a warp shuffle
// reduction and one shared atomicMax per warp and zone.

#include <cuda_runtime.h>
#include <math_constants.h>

#include <cmath>
#include <cstring>

#include "pps.h"
#include "pps_internal.h"

namespace {

constexpr int kTPB = 256;
constexpr int kMaxSide = 32768;

__device__ __forceinline__ bool fin_(float x) { return fabsf(x) < CUDART_INF_F; }

// Order-preserving map of a float to an unsigned integer (larger float,
// larger integer); -0 and +0 are merged by the caller.
__device__ __forceinline__ uint32_t ordered(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// sqrt and 1/x from the SFU's approximations (a few ulp; the scores are
// compared with the FP64 oracle at 2e-5): sqrt(0) = 0.
__device__ __forceinline__ float sqrt_a(float x) {
    return x > 0.f ? __fmul_rn(x, rsqrtf(x)) : 0.f;
}

__device__ __forceinline__ float rcp_a(float x) { return __fdividef(1.f, x); }

__device__ __forceinline__ float unordered(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o);
}

// Bang-bang intercept time along the line to (px, py): accelerate at amax
// up to vmax from the projected speed w, arrival at any speed.
__device__ __forceinline__ float intercept_time(float ox, float oy, float ux,
                                                float uy, float px, float py,
                                                float vmax, float amax,
                                                float inv_amax, float inv_vmax) {
    const float dx = __fsub_rn(px, ox), dy = __fsub_rn(py, oy);
    const float d2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
    if (d2 <= 0.f) return 0.f;
    const float rd = rsqrtf(d2);
    const float d = __fmul_rn(d2, rd);
    float w = __fmul_rn(__fmaf_rn(ux, dx, __fmul_rn(uy, dy)), rd);
    w = fminf(fmaxf(w, -vmax), vmax);
    const float d_top = __fmul_rn(__fmaf_rn(-w, w, __fmul_rn(vmax, vmax)),
                                  __fmul_rn(0.5f, inv_amax));
    if (d <= d_top) {
        // w t + amax t^2 / 2 = d; the cancellation-free root for w >= 0
        const float r = sqrt_a(__fmaf_rn(w, w, __fmul_rn(2.f * amax, d)));
        return w >= 0.f ? __fdividef(__fmul_rn(2.f, d), __fadd_rn(w, r))
                        : __fmul_rn(__fsub_rn(r, w), inv_amax);
    }
    return __fmaf_rn(__fsub_rn(vmax, w), inv_amax, __fmul_rn(__fsub_rn(d, d_top), inv_vmax));
}

struct RShared {
    float gx[PPS_MAX_OPP], gy[PPS_MAX_OPP], gux[PPS_MAX_OPP], guy[PPS_MAX_OPP];
    unsigned long long key[4];
    float dmin2;  // the nearest opponent's squared distance to the ball
    int n_guard;
    int nx, ny;
    int valid;
};

struct RArgs {
    const pps_dstate* states;
    int n_states;
    pps_rparams p;
    const pps_dbest* pass;
    pps_rbest* out;
    float* scores;
    long long stride;
};

// The cuts are lowered by the edge tolerance tol = g / 1024: a point
// within it of a cut counts as on it (in front of it, or above it).
__device__ __forceinline__ int zone_of(float px, float py, float quarter_l,
                                       float ys, float tol) {
    return (px >= __fsub_rn(quarter_l, tol) ? 2 : 0) + (py >= __fsub_rn(ys, tol) ? 1 : 0);
}

// Warp 0: the state's constants.
__device__ void derive(const pps_dstate& st, const RArgs& a, RShared& sh,
                       float x0, float x1, float y1) {
    const int lane = threadIdx.x & 31;
    const float L = st.field_len, W = st.field_wid;
    bool ok = fin_(st.ball[0]) && fin_(st.ball[1]) && fin_(L) && L > 0.f &&
              fin_(W) && W > 0.f && fin_(st.goal_width) && st.goal_width > 0.f &&
              fin_(st.vmax) && st.vmax > 0.f && fin_(st.amax) && st.amax > 0.f &&
              st.n_opp >= 0 && st.n_opp <= PPS_MAX_OPP;
    int nx = 0, ny = 0;
    if (ok) {
        const float fx = rintf(__fdiv_rn(__fmul_rn(0.5f, L), a.p.spacing));
        const float fy = rintf(__fdiv_rn(W, a.p.spacing));
        ok = fx < (float)kMaxSide && fy < (float)kMaxSide;
        if (ok) {
            nx = (int)fx + 1;
            ny = (int)fy + 1;
            if (a.scores && (long long)nx * ny > a.stride) ok = false;
        }
    }
    const bool mine = ok && lane < st.n_opp;
    float ox = 0.f, oy = 0.f, ux = 0.f, uy = 0.f;
    if (mine) {
        ox = st.opp_pos[lane][0];
        oy = st.opp_pos[lane][1];
        ux = st.opp_vel[lane][0];
        uy = st.opp_vel[lane][1];
    }
    const bool bad = mine && !(fin_(ox) && fin_(oy) && fin_(ux) && fin_(uy));
    ok = ok && !__any_sync(0xffffffffu, bad);
    const bool guard = mine && ox >= x0 && ox <= x1 && oy >= -y1 && oy <= y1;
    const unsigned gm = __ballot_sync(0xffffffffu, guard);
    if (guard) {
        const int k = __popc(gm & ((1u << lane) - 1u));
        sh.gx[k] = ox;
        sh.gy[k] = oy;
        sh.gux[k] = ux;
        sh.guy[k] = uy;
    }
    float d2 = CUDART_INF_F;
    if (mine) {
        const float dx = __fsub_rn(ox, st.ball[0]), dy = __fsub_rn(oy, st.ball[1]);
        d2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d2 = fminf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    if (lane == 0) {
        sh.n_guard = __popc(gm);
        sh.dmin2 = d2;
        sh.nx = nx;
        sh.ny = ny;
        sh.valid = ok;
    }
    if (lane < 4) sh.key[lane] = 0ull;
}

__global__ void __launch_bounds__(kTPB, 4) run_kernel(const RArgs a) {
    __shared__ RShared sh;
    const pps_rparams& p = a.p;
    for (int s = blockIdx.x; s < a.n_states; s += gridDim.x) {
        const pps_dstate& st = a.states[s];
        const float L = st.field_len, W = st.field_wid;
        const float x1 = __fmul_rn(0.5f, L);
        const float x0 = __fsub_rn(x1, p.def_depth);
        const float y1 = __fmul_rn(0.5f, p.def_width);
        if (threadIdx.x < 32) derive(st, a, sh, x0, x1, y1);
        __syncthreads();
        if (sh.valid) {
            const int nx = sh.nx, n = sh.nx * sh.ny, ng = sh.n_guard;
            const float g = p.spacing, y_lo = __fmul_rn(-0.5f, W);
            const float y_hi = __fmul_rn(0.5f, W);
            // grid points on the defence area's edges or on a zone cut lie
            // within rounding of them: g / 1024 decides
            const float tol = __fmul_rn(g, 1.f / 1024.f);
            const float cx0 = __fadd_rn(x0, tol), cy1 = __fsub_rn(y1, tol);
            const float bx = st.ball[0], by = st.ball[1];
            const float quarter_l = __fmul_rn(0.25f, L);
            const float qw = __fmul_rn(0.25f, W);
            const float ys = fminf(fmaxf(by, -qw), qw);
            const float hw = __fmul_rn(0.5f, st.goal_width);
            const float inv_diag =
                __frcp_rn(__fsqrt_rn(__fmaf_rn(L, L, __fmul_rn(W, W))));
            const float inv_ref = __frcp_rn(p.ball_ref);
            const float inv_span = __frcp_rn(p.angle_span);
            const float inv_amax = __frcp_rn(st.amax);
            const float inv_2cap = __frcp_rn(__fmul_rn(2.f, p.guard_cap));
            const float vmax = st.vmax, inv_vmax = __frcp_rn(st.vmax);
            const float dmin2 = sh.dmin2;
            // per zone the best score and its first index (a thread meets its
            // points in increasing idx, so "greater" keeps the first on ties)
            float bsc[4] = {-CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F, -CUDART_INF_F};
            int bid[4] = {-1, -1, -1, -1};
            // row-major walk: idx = tid, tid + kTPB, ...; (j, i) advanced
            // incrementally
            const int step_j = kTPB / nx, step_i = kTPB - step_j * nx;
            int j = (int)threadIdx.x / nx, i = (int)threadIdx.x - j * nx;
            for (int idx = threadIdx.x; idx < n; idx += kTPB) {
                // the raster ends on the goal line and the touch line
                const float px = fminf(__fmul_rn((float)i, g), x1);
                const float py = fminf(__fmaf_rn((float)j, g, y_lo), y_hi);
                const bool cand = !(px > cx0 && py > -cy1 && py < cy1);
                float score = -CUDART_INF_F;
                if (cand) {
                    // 1. distance to the goal, 2. distance to the ball
                    const float gx = __fsub_rn(x1, px), gy = -py;
                    const float x_goal = __fmul_rn(
                        sqrt_a(__fmaf_rn(gx, gx, __fmul_rn(gy, gy))), inv_diag);
                    const float dbx = __fsub_rn(px, bx), dby = __fsub_rn(py, by);
                    const float db2 = __fmaf_rn(dbx, dbx, __fmul_rn(dby, dby));
                    const float db = sqrt_a(db2);
                    const float x_ball = __fmul_rn(fminf(db, p.ball_ref), inv_ref);
                    // 3. the angle band
                    const float alpha = fabsf(atan2f(gy, gx));
                    const float off = alpha < p.angle_lo ? __fsub_rn(p.angle_lo, alpha)
                                      : alpha > p.angle_hi ? __fsub_rn(alpha, p.angle_hi)
                                                           : 0.f;
                    const float x_angle = __fsub_rn(1.f, fminf(__fmul_rn(off, inv_span), 1.f));
                    // 4. the guards' time to P and Q.  The segment p + t (dx, dy),
                    // t in [0, 1], enters the area where it is inside both slabs
                    // (Liang-Barsky); dx = x1 - px >= 0 is the same for both
                    // posts, so the x slab's interval is shared.
                    const float dx = gx;
                    float tx0 = 0.f;
                    if (dx > 0.f) tx0 = fmaxf(0.f, __fmul_rn(__fsub_rn(x0, px), rcp_a(dx)));
                    float tsum = 0.f;
#pragma unroll
                    for (int side = 0; side < 2; ++side) {
                        const float dy = __fsub_rn(side ? hw : -hw, py);
                        float t0 = tx0, t1 = 1.f;
                        if (dy != 0.f) {
                            const float rdy = rcp_a(dy);
                            const float ra = __fmul_rn(__fsub_rn(-y1, py), rdy);
                            const float rb = __fmul_rn(__fsub_rn(y1, py), rdy);
                            t0 = fmaxf(t0, fminf(ra, rb));
                            t1 = fminf(t1, fmaxf(ra, rb));
                        } else if (py < -y1 || py > y1) {
                            t1 = -1.f;  // parallel to the y slab and outside it
                        }
                        float T = p.guard_cap;
                        if (t0 <= t1) {
                            const float ex = __fmaf_rn(t0, dx, px);
                            const float ey = __fmaf_rn(t0, dy, py);
                            for (int k = 0; k < ng; ++k)
                                T = fminf(T, intercept_time(sh.gx[k], sh.gy[k], sh.gux[k],
                                                            sh.guy[k], ex, ey, vmax,
                                                            st.amax, inv_amax, inv_vmax));
                        }
                        tsum = __fadd_rn(tsum, T);
                    }
                    const float x_guard = __fmul_rn(tsum, inv_2cap);
                    // 5. an opponent nearer the ball than p
                    const float x_avoid = dmin2 < db2 ? 1.f : 0.f;
                    score = __fmul_rn(-p.w_goal, x_goal);
                    score = __fmaf_rn(p.w_ball, x_ball, score);
                    score = __fmaf_rn(p.w_angle, x_angle, score);
                    score = __fmaf_rn(p.w_guard, x_guard, score);
                    score = __fmaf_rn(-p.w_avoid, x_avoid, score);
                    score = __fadd_rn(score, 0.f);  // -0 -> +0
                    const int z = zone_of(px, py, quarter_l, ys, tol);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const bool up = (q == z) && (score > bsc[q] || bid[q] < 0);
                        bsc[q] = up ? score : bsc[q];
                        bid[q] = up ? idx : bid[q];
                    }
                }
                if (a.scores) a.scores[(long long)s * a.stride + idx] = score;
                i += step_i;
                j += step_j;
                if (i >= nx) {
                    i -= nx;
                    ++j;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                unsigned long long k =
                    bid[q] < 0 ? 0ull
                               : ((unsigned long long)ordered(bsc[q]) << 32) |
                                     (unsigned long long)(0xFFFFFFFFu - (uint32_t)bid[q]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long v = __shfl_xor_sync(0xffffffffu, k, o);
                    k = v > k ? v : k;
                }
                if ((threadIdx.x & 31) == 0 && k) atomicMax(&sh.key[q], k);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            pps_rbest o;
            o.nx = sh.nx;
            o.ny = sh.ny;
            o.status = sh.valid ? PPS_STATE_OK : PPS_STATE_INVALID;
            o.avoided = -1;
            for (int q = 0; q < 4; ++q) {
                const unsigned long long k = sh.valid ? sh.key[q] : 0ull;
                o.chosen[q] = -1;
                if (k) {
                    const int idx = (int)(0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFull));
                    const int j = idx / sh.nx, i = idx - j * sh.nx;
                    o.idx[q] = idx;
                    o.score[q] = unordered((uint32_t)(k >> 32));
                    o.point[q][0] = fminf(__fmul_rn((float)i, p.spacing), __fmul_rn(0.5f, L));
                    o.point[q][1] = fminf(__fmaf_rn((float)j, p.spacing, __fmul_rn(-0.5f, W)),
                                          __fmul_rn(0.5f, W));
                } else {
                    o.idx[q] = -1;
                    o.score[q] = -CUDART_INF_F;
                    o.point[q][0] = o.point[q][1] = CUDART_NAN_F;
                }
            }
            if (sh.valid) {
                if (a.pass && a.pass[s].idx >= 0) {
                    const float rx = a.pass[s].recv[0], ry = a.pass[s].recv[1];
                    if (rx >= 0.f && rx <= __fmul_rn(0.5f, L) &&
                        fabsf(ry) <= __fmul_rn(0.5f, W)) {
                        const float qw = __fmul_rn(0.25f, W);
                        o.avoided = zone_of(rx, ry, __fmul_rn(0.25f, L),
                                            fminf(fmaxf(st.ball[1], -qw), qw),
                                            __fmul_rn(p.spacing, 1.f / 1024.f));
                    }
                }
                // III and IV first, then I and II, each pair by score
                int k = 0;
                for (int pair = 1; pair >= 0; --pair) {
                    const int za = 2 * pair, zb = za + 1;
                    const int first = o.score[zb] > o.score[za] ? zb : za;
                    const int order[2] = {first, first == za ? zb : za};
                    for (int t = 0; t < 2; ++t) {
                        const int z = order[t];
                        if (k < p.n_run && o.idx[z] >= 0 && z != o.avoided)
                            o.chosen[k++] = z;
                    }
                }
            }
            a.out[s] = o;
        }
        __syncthreads();  // the shared constants are rewritten next state
    }
}

bool fin(float x) { return std::isfinite(x); }

bool grid_of(float L, float W, float g, int* nx, int* ny) {
    if (!fin(L) || !fin(W) || !fin(g) || !(L > 0.f) || !(W > 0.f) || !(g > 0.f))
        return false;
    const float fx = std::nearbyint((0.5f * L) / g);
    const float fy = std::nearbyint(W / g);
    if (!(fx < (float)kMaxSide) || !(fy < (float)kMaxSide)) return false;
    *nx = (int)fx + 1;
    *ny = (int)fy + 1;
    return true;
}

}  // namespace

extern "C" pps_status pps_run_default_params(pps_rparams* out) {
    if (!out) return PPS_EINVAL;
    out->spacing = 0.1f;
    out->w_goal = out->w_ball = out->w_angle = out->w_guard = out->w_avoid = 1.f;
    out->ball_ref = 2.f;
    out->angle_lo = 0.25f;
    out->angle_hi = 0.75f;
    out->angle_span = 0.5f;
    out->def_depth = 1.2f;
    out->def_width = 2.4f;
    out->guard_cap = 2.f;
    out->n_run = 4;
    return PPS_OK;
}

extern "C" pps_status pps_run_grid(float field_len, float field_wid, float spacing,
                                   int* nx, int* ny) {
    if (!nx || !ny) return PPS_EINVAL;
    return grid_of(field_len, field_wid, spacing, nx, ny) ? PPS_OK : PPS_EINVAL;
}

extern "C" pps_status pps_run_points(pps_ctx* ctx, const pps_dstate* states,
                                     int n_states, const pps_rparams* params,
                                     const pps_dbest* pass, pps_rbest* out,
                                     float* out_scores, size_t score_stride) {
    PPS_RANGE("pps_run_points");
    if (!ctx) return PPS_EINVAL;
    if (pps_ctx_failed(ctx))
        return pps_ctx_error(ctx, PPS_ECUDA, "context failed earlier; call pps_reset");
    if (n_states == 0) return PPS_OK;
    if (n_states < 0 || !states || !out)
        return pps_ctx_error(ctx, PPS_EINVAL, "pps_run_points: bad buffers or counts");
    pps_rparams p;
    if (params)
        p = *params;
    else
        pps_run_default_params(&p);
    const float vals[] = {p.spacing, p.w_goal, p.w_ball, p.w_angle, p.w_guard,
                          p.w_avoid, p.ball_ref, p.angle_lo, p.angle_hi,
                          p.angle_span, p.def_depth, p.def_width, p.guard_cap};
    for (float x : vals)
        if (!fin(x))
            return pps_ctx_error(ctx, PPS_EINVAL, "pps_run_points: non-finite parameter");
    if (!(p.spacing > 0.f) || !(p.ball_ref > 0.f) || p.angle_lo < 0.f ||
        p.angle_hi < p.angle_lo || !(p.angle_span > 0.f) || !(p.def_depth > 0.f) ||
        !(p.def_width > 0.f) || !(p.guard_cap > 0.f) || p.n_run < 0 || p.n_run > 4 ||
        (out_scores && score_stride == 0))
        return pps_ctx_error(ctx, PPS_EINVAL, "pps_run_points: parameter out of range");
    cudaError_t e = cudaSetDevice(pps_ctx_device(ctx));
    RArgs a;
    std::memset(&a, 0, sizeof a);
    a.states = states;
    a.n_states = n_states;
    a.p = p;
    a.pass = pass;
    a.out = out;
    a.scores = out_scores;
    a.stride = out_scores ? (long long)score_stride : 0;
    if (e == cudaSuccess) {
        const int occ = pps_occupancy((const void*)run_kernel, kTPB, 0);
        long long grid = (long long)pps_ctx_num_sms(ctx) * occ;
        if (grid > n_states) grid = n_states;
        run_kernel<<<(unsigned)grid, kTPB, 0, pps_ctx_stream(ctx)>>>(a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return pps_ctx_cuda_error(ctx, e, "pps_run_points");
    return PPS_OK;
}

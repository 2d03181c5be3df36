// pps_lib.cu -- host side of the libpps C ABI (include/pps.h).
//
// Owns the context (device, stream, scratch, staging buffers), validates
// arguments, picks the kernel instance for the batch shape and launches it.
// All device work of a call is enqueued on the context's stream.

#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>

#include "pps.h"
#include "pps_internal.h"
#include "pps_search.cuh"

struct pps_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0, used = 0;
    int max_states = 0, max_points = 0, max_speeds = 0, max_K = 0;
    int max_opp = 0, jmax = 8;
    int num_sms = 0;
    unsigned long long* keys = nullptr;  // scratch, max_states entries and
                                         // a work-queue counter after them
    int* counts = nullptr;               // scratch, max_states entries
    struct Buf {
        void* p = nullptr;
        size_t cap = 0;
    } st, best, mask, dm, ds, dT;
    bool failed = false;
    char err[512] = {0};
};

namespace {

thread_local char g_create_err[512];

void set_err(pps_ctx* ctx, const char* fmt, ...) {
    char* dst = ctx ? ctx->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
}

pps_status cuda_fail(pps_ctx* ctx, cudaError_t e, const char* what) {
    set_err(ctx, "%s: %s", what, cudaGetErrorString(e));
    if (ctx) ctx->failed = true;
    return PPS_ECUDA;
}

pps_status dev_alloc(pps_ctx* ctx, void** p, size_t bytes, const char* what) {
    if (ctx->budget && ctx->used + bytes > ctx->budget) {
        set_err(ctx, "%s: %zu bytes exceed the memory budget (%zu of %zu used)",
                what, bytes, ctx->used, ctx->budget);
        return PPS_ENOMEM;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_err(ctx, "%s: cudaMalloc(%zu): %s", what, bytes,
                cudaGetErrorString(e));
        *p = nullptr;
        return PPS_ENOMEM;
    }
    ctx->used += bytes;
    return PPS_OK;
}

void dev_free(pps_ctx* ctx, void* p, size_t bytes) {
    if (p) {
        cudaFree(p);
        ctx->used -= bytes;
    }
}

// Grow a staging buffer to at least `bytes`.
pps_status ensure(pps_ctx* ctx, pps_ctx::Buf& b, size_t bytes,
                  const char* what) {
    if (b.cap >= bytes) return PPS_OK;
    dev_free(ctx, b.p, b.cap);
    b.p = nullptr;
    b.cap = 0;
    pps_status s = dev_alloc(ctx, &b.p, bytes, what);
    if (s == PPS_OK) b.cap = bytes;
    return s;
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.f; }

pps_status check_state(pps_ctx* ctx, const pps_state& s, int i) {
    if (s.n_opp < 0 || s.n_opp > ctx->max_opp) {
        set_err(ctx, "state %d: n_opp %d outside 0..%d", i, s.n_opp,
                ctx->max_opp);
        return PPS_EINVAL;
    }
    if (s.K < 1 || s.K > ctx->max_K) {
        set_err(ctx, "state %d: K %d outside 1..%d", i, s.K, ctx->max_K);
        return PPS_EINVAL;
    }
    if (!finite_pos(s.ball_decel) || !finite_pos(s.vmax) ||
        !finite_pos(s.amax) || !finite_pos(s.field_len) ||
        !finite_pos(s.field_wid) || !std::isfinite(s.goal_width) ||
        s.goal_width < 0.f) {
        set_err(ctx, "state %d: decel, vmax, amax, L, W must be finite and "
                     "> 0, goal width finite and >= 0", i);
        return PPS_EINVAL;
    }
    bool fin = std::isfinite(s.ball[0]) && std::isfinite(s.ball[1]);
    for (int j = 0; j < s.n_opp; ++j)
        fin = fin && std::isfinite(s.opp_pos[j][0]) &&
              std::isfinite(s.opp_pos[j][1]) &&
              std::isfinite(s.opp_vel[j][0]) && std::isfinite(s.opp_vel[j][1]);
    if (!fin) {
        set_err(ctx, "state %d: non-finite position or velocity", i);
        return PPS_EINVAL;
    }
    return PPS_OK;
}

template <int J, int V, bool EXT>
cudaError_t launch(const pps::SearchArgs& a, int num_sms, cudaStream_t st) {
    const int occ = pps_occupancy((const void*)pps::search_kernel<J, V, EXT>,
                                  pps::search_tpb<J, V>(), 0);
    // One warp per work item of 32 points; no more CTAs than items need.
    const long long items = (long long)a.n_states * a.words;
    long long grid = (long long)num_sms * occ;
    constexpr int tpb = pps::search_tpb<J, V>();
    const long long need = (items + tpb / 32 - 1) / (tpb / 32);
    if (grid > need) grid = need;
    pps::search_kernel<J, V, EXT><<<(unsigned)grid, tpb, 0, st>>>(a);
    pps::finalize_kernel<J, V><<<pps::finalize_blocks(a.n_states), 128, 0, st>>>(a);
    return cudaGetLastError();
}

template <int J, int V>
cudaError_t launch_e(const pps::SearchArgs& a, int num_sms, cudaStream_t st) {
    return a.dbg_point ? launch<J, V, true>(a, num_sms, st)
                       : launch<J, V, false>(a, num_sms, st);
}

template <int J>
cudaError_t launch_v(const pps::SearchArgs& a, int num_sms, cudaStream_t st) {
    if (a.V <= 1) return launch_e<J, 1>(a, num_sms, st);
    if (a.V <= 2) return launch_e<J, 2>(a, num_sms, st);
    if (a.V <= 4) return launch_e<J, 4>(a, num_sms, st);
    return launch_e<J, 8>(a, num_sms, st);
}

template <int J, int V>
int occupancy_of() {
    return pps_occupancy((const void*)pps::search_kernel<J, V>,
                         pps::search_tpb<J, V>(), 0);
}

std::mutex g_occ_mu;
std::map<std::tuple<int, const void*, int, size_t>, int> g_occ;

}  // namespace

int pps_occupancy(const void* func, int tpb, size_t smem) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    const auto key = std::make_tuple(dev, func, tpb, smem);
    std::lock_guard<std::mutex> lk(g_occ_mu);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) return it->second;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, func, tpb, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 1;  // not cached: the next call asks again
    }
    if (occ < 1) occ = 1;
    g_occ.emplace(key, occ);
    return occ;
}

// The calling thread's error buffer behind pps_last_error(NULL), shared with
// the no-allocation entry point in pps_noalloc.cu.
char* pps_thread_error_buffer() { return g_create_err; }

int pps_ctx_device(const pps_ctx* ctx) { return ctx->device; }
cudaStream_t pps_ctx_stream(const pps_ctx* ctx) { return ctx->stream; }
int pps_ctx_num_sms(const pps_ctx* ctx) { return ctx->num_sms; }
int pps_ctx_max_K(const pps_ctx* ctx) { return ctx->max_K; }
bool pps_ctx_failed(const pps_ctx* ctx) { return ctx->failed; }
void pps_ctx_scratch(pps_ctx* ctx, unsigned long long** keys, int** counts) {
    *keys = ctx->keys;
    *counts = ctx->counts;
}

unsigned long long* pps_ctx_work_counter(pps_ctx* ctx) {
    return ctx->keys + ctx->max_states;
}
int pps_ctx_max_states(const pps_ctx* ctx) { return ctx->max_states; }
int pps_ctx_jmax(const pps_ctx* ctx) { return ctx->jmax; }
int pps_ctx_max_opp(const pps_ctx* ctx) { return ctx->max_opp; }

pps_status pps_ctx_alloc(pps_ctx* ctx, void** p, size_t bytes,
                         const char* what) {
    return dev_alloc(ctx, p, bytes, what);
}

void pps_ctx_free(pps_ctx* ctx, void* p, size_t bytes) {
    dev_free(ctx, p, bytes);
}

pps_status pps_ctx_error(pps_ctx* ctx, pps_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof ctx->err, fmt, ap);
    va_end(ap);
    return s;
}

pps_status pps_ctx_cuda_error(pps_ctx* ctx, cudaError_t e, const char* what) {
    return cuda_fail(ctx, e, what);
}

extern "C" {

int pps_abi_version(void) { return PPS_ABI_VERSION; }

const char* pps_status_string(pps_status s) {
    switch (s) {
        case PPS_OK: return "PPS_OK";
        case PPS_EINVAL: return "PPS_EINVAL";
        case PPS_ENOMEM: return "PPS_ENOMEM";
        case PPS_ECUDA: return "PPS_ECUDA";
        case PPS_ETIMEOUT: return "PPS_ETIMEOUT";
        case PPS_ENOTIMPL: return "PPS_ENOTIMPL";
        default: return "PPS_UNKNOWN";
    }
}

const char* pps_last_error(const pps_ctx* ctx) {
    return ctx ? ctx->err : g_create_err;
}

pps_status pps_default_params(pps_params* out) {
    if (!out) return PPS_EINVAL;
    out->w_angle = 1.f;
    out->w_dist = 1.f;
    out->w_margin = 1.f;
    out->margin_cap = 1.f;
    out->tau_safe = 0.f;
    out->robot_radius = 0.09f;
    out->reach_radius = 0.f;
    out->min_pass_dist = 0.f;
    return PPS_OK;
}

pps_status pps_grid_from_field(float L, float W, float spacing,
                               pps_grid* out) {
    if (!out || !finite_pos(L) || !finite_pos(W) || !finite_pos(spacing))
        return PPS_EINVAL;
    const double nx = std::nearbyint((double)L / (double)spacing) + 1.0;
    const double ny = std::nearbyint((double)W / (double)spacing) + 1.0;
    if (nx * ny > (double)(1 << 24)) return PPS_EINVAL;
    out->spacing = spacing;
    out->nx = (int32_t)nx;
    out->ny = (int32_t)ny;
    out->x0 = -0.5f * L;
    out->y0 = -0.5f * W;
    return PPS_OK;
}

size_t pps_mask_words(const pps_grid* grid, int n_speeds) {
    if (!grid || grid->nx < 1 || grid->ny < 1 || n_speeds < 1) return 0;
    const size_t P = (size_t)grid->nx * (size_t)grid->ny;
    return (size_t)n_speeds * ((P + 31) / 32);
}

pps_status pps_create(pps_ctx** out, const pps_ctx_desc* desc) {
    if (!out) return PPS_EINVAL;
    *out = nullptr;
    if (!desc) {
        set_err(nullptr, "pps_create: desc is NULL");
        return PPS_EINVAL;
    }
    if (desc->max_states < 1 || desc->max_points < 0 ||
        desc->max_speeds < 0 || desc->max_speeds > PPS_MAX_SPEEDS ||
        desc->max_K < 0 || desc->max_K > PPS_MAX_K || desc->max_opp < 0 ||
        desc->max_opp > PPS_MAX_OPP) {
        set_err(nullptr, "pps_create: descriptor field out of range");
        return PPS_EINVAL;
    }
    pps_ctx* ctx = new (std::nothrow) pps_ctx();
    if (!ctx) return PPS_ENOMEM;
    ctx->device = desc->device;
    ctx->stream = (cudaStream_t)desc->stream;
    ctx->budget = desc->mem_budget_bytes;
    ctx->max_states = desc->max_states;
    ctx->max_points = desc->max_points ? desc->max_points : (1 << 24);
    ctx->max_speeds = desc->max_speeds ? desc->max_speeds : PPS_MAX_SPEEDS;
    ctx->max_K = desc->max_K ? desc->max_K : PPS_MAX_K;
    ctx->max_opp = desc->max_opp ? desc->max_opp : PPS_MAX_OPP;
    ctx->jmax = ctx->max_opp <= 8 ? 8 : 16;

    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount,
                                   ctx->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_err(nullptr, "pps_create: device %d unusable: %s", ctx->device,
                cudaGetErrorString(e));
        delete ctx;
        return PPS_ECUDA;
    }
    pps_status s = dev_alloc(ctx, (void**)&ctx->keys,
                             sizeof(unsigned long long) * (ctx->max_states + 1),
                             "argmax keys");
    if (s == PPS_OK)
        s = dev_alloc(ctx, (void**)&ctx->counts, sizeof(int) * ctx->max_states,
                      "feasible counts");
    if (s != PPS_OK) {
        std::snprintf(g_create_err, sizeof g_create_err, "pps_create: %s",
                      ctx->err);
        pps_destroy(ctx);
        return s;
    }
    *out = ctx;
    return PPS_OK;
}

void pps_destroy(pps_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, ctx->keys, sizeof(unsigned long long) * (ctx->max_states + 1));
    dev_free(ctx, ctx->counts, sizeof(int) * ctx->max_states);
    for (pps_ctx::Buf* b : {&ctx->st, &ctx->best, &ctx->mask, &ctx->dm,
                            &ctx->ds, &ctx->dT})
        dev_free(ctx, b->p, b->cap);
    cudaGetLastError();
    delete ctx;
}

pps_status pps_sync(pps_ctx* ctx) {
    if (!ctx) return PPS_EINVAL;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pps_sync");
    return ctx->failed ? PPS_ECUDA : PPS_OK;
}

pps_status pps_reset(pps_ctx* ctx) {
    if (!ctx) return PPS_EINVAL;
    cudaSetDevice(ctx->device);
    cudaGetLastError();
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pps_reset");
    ctx->failed = false;
    ctx->err[0] = 0;
    return PPS_OK;
}

pps_status pps_launch_info(const pps_ctx* ctx, int* num_sms,
                           int* ctas_per_sm) {
    if (!ctx || !num_sms || !ctas_per_sm) return PPS_EINVAL;
    *num_sms = ctx->num_sms;
    *ctas_per_sm = ctx->jmax == 8 ? occupancy_of<8, 4>() : occupancy_of<16, 4>();
    return PPS_OK;
}

pps_status pps_search(pps_ctx* ctx, const pps_state* states, int n_states,
                      const pps_grid* grid, const float* speeds, int n_speeds,
                      const pps_params* params, pps_best* out_best,
                      uint32_t* out_mask, const pps_debug_out* dbg,
                      unsigned flags) {
    PPS_RANGE("pps_search");
    if (!ctx) return PPS_EINVAL;
    ctx->err[0] = 0;
    if (ctx->failed) {
        set_err(ctx, "context failed earlier; call pps_reset");
        return PPS_ECUDA;
    }
    if (flags & ~PPS_DEVICE_PTRS) {
        set_err(ctx, "unknown flags 0x%x", flags);
        return PPS_EINVAL;
    }
    if (n_states < 0 || n_states > ctx->max_states) {
        set_err(ctx, "n_states %d outside 0..%d", n_states, ctx->max_states);
        return PPS_EINVAL;
    }
    if (!grid || !finite_pos(grid->spacing) || grid->nx < 1 || grid->ny < 1 ||
        !std::isfinite(grid->x0) || !std::isfinite(grid->y0) ||
        (long long)grid->nx * grid->ny > ctx->max_points) {
        set_err(ctx, "grid: spacing must be finite and > 0, 1 <= nx*ny <= %d",
                ctx->max_points);
        return PPS_EINVAL;
    }
    if (!speeds || n_speeds < 1 || n_speeds > ctx->max_speeds) {
        set_err(ctx, "n_speeds %d outside 1..%d", n_speeds, ctx->max_speeds);
        return PPS_EINVAL;
    }
    for (int v = 0; v < n_speeds; ++v)
        if (!finite_pos(speeds[v])) {
            set_err(ctx, "speed %d must be finite and > 0", v);
            return PPS_EINVAL;
        }
    pps_params prm;
    if (params)
        prm = *params;
    else
        pps_default_params(&prm);
    const float pv[] = {prm.w_angle, prm.w_dist, prm.w_margin,
                        prm.margin_cap, prm.tau_safe, prm.robot_radius,
                        prm.reach_radius, prm.min_pass_dist};
    for (float x : pv)
        if (!std::isfinite(x)) {
            set_err(ctx, "params must be finite");
            return PPS_EINVAL;
        }
    if (prm.robot_radius < 0.f || prm.reach_radius < 0.f ||
        prm.min_pass_dist < 0.f) {
        set_err(ctx, "radii and min_pass_dist must be >= 0");
        return PPS_EINVAL;
    }
    if (!out_best || (n_states > 0 && !states)) {
        set_err(ctx, "states and out_best are required");
        return PPS_EINVAL;
    }
    const bool on_dev = flags & PPS_DEVICE_PTRS;
    const long long P = (long long)grid->nx * grid->ny;
    if (dbg && dbg->point_best && !on_dev) {
        set_err(ctx, "dbg->point_best needs PPS_DEVICE_PTRS");
        return PPS_EINVAL;
    }
    if (dbg && dbg->T && dbg->T_stride < 1) {
        set_err(ctx, "dbg->T_stride must be >= 1");
        return PPS_EINVAL;
    }
    if (!on_dev) {
        for (int i = 0; i < n_states; ++i) {
            pps_status s = check_state(ctx, states[i], i);
            if (s != PPS_OK) return s;
            if (dbg && dbg->T && states[i].K > dbg->T_stride) {
                set_err(ctx, "state %d: K %d > dbg->T_stride %d", i,
                        states[i].K, dbg->T_stride);
                return PPS_EINVAL;
            }
        }
    }
    if (n_states == 0) return PPS_OK;
    if (P * n_speeds >= (1ll << 31)) {
        set_err(ctx, "n_speeds * P must be below 2^31");
        return PPS_EINVAL;
    }

    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    cudaStream_t st = ctx->stream;
    const size_t words = pps_mask_words(grid, n_speeds);
    const size_t nS = (size_t)n_states;

    pps::SearchArgs a;
    std::memset(&a, 0, sizeof a);
    a.n_states = n_states;
    a.nx = grid->nx;
    a.ny = grid->ny;
    a.P = (int)P;
    a.words = (int)((P + 31) / 32);
    a.g = grid->spacing;
    a.x0 = grid->x0;
    a.y0 = grid->y0;
    a.V = n_speeds;
    a.kmax = on_dev && dbg && dbg->T ? (dbg->T_stride < ctx->max_K
                                            ? dbg->T_stride
                                            : ctx->max_K)
                                     : ctx->max_K;
    // Unused speed slots repeat the last speed (their results are dropped).
    for (int v = 0; v < PPS_MAX_SPEEDS; ++v) {
        const float sv = speeds[v < n_speeds ? v : n_speeds - 1];
        a.speed[v] = sv;
        a.speed2[v] = sv * sv;
    }
    a.prm = prm;
    a.keys = ctx->keys;
    a.counts = ctx->counts;
    a.T_stride = dbg && dbg->T ? dbg->T_stride : 0;

    pps_status s = PPS_OK;
    if (on_dev) {
        a.states = states;
        a.best = out_best;
        a.mask = out_mask;
        if (dbg) {
            a.dbg_margin = dbg->margin;
            a.dbg_score = dbg->score;
            a.dbg_T = dbg->T;
            a.dbg_point = dbg->point_best;
        }
    } else {
        const size_t dbg_n = nS * n_speeds * (size_t)P;
        s = ensure(ctx, ctx->st, nS * sizeof(pps_state), "state staging");
        if (s == PPS_OK)
            s = ensure(ctx, ctx->best, nS * sizeof(pps_best), "result staging");
        if (s == PPS_OK && out_mask)
            s = ensure(ctx, ctx->mask, nS * words * 4, "mask staging");
        if (s == PPS_OK && dbg && dbg->margin)
            s = ensure(ctx, ctx->dm, dbg_n * 4, "margin staging");
        if (s == PPS_OK && dbg && dbg->score)
            s = ensure(ctx, ctx->ds, dbg_n * 4, "score staging");
        if (s == PPS_OK && dbg && dbg->T)
            s = ensure(ctx, ctx->dT, nS * (size_t)P * dbg->T_stride * 4,
                       "T staging");
        if (s != PPS_OK) return s;
        a.states = (const pps_state*)ctx->st.p;
        a.best = (pps_best*)ctx->best.p;
        a.mask = out_mask ? (uint32_t*)ctx->mask.p : nullptr;
        if (dbg) {
            a.dbg_margin = dbg->margin ? (float*)ctx->dm.p : nullptr;
            a.dbg_score = dbg->score ? (float*)ctx->ds.p : nullptr;
            a.dbg_T = dbg->T ? (float*)ctx->dT.p : nullptr;
        }
        e = cudaMemcpyAsync((void*)a.states, states, nS * sizeof(pps_state),
                            cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "state upload");
    }

    e = cudaMemsetAsync(ctx->keys, 0, nS * sizeof(unsigned long long), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ctx->counts, 0, nS * sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "scratch clear");

    e = ctx->jmax == 8 ? launch_v<8>(a, ctx->num_sms, st)
                       : launch_v<16>(a, ctx->num_sms, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "search launch");

    if (!on_dev) {
        e = cudaMemcpyAsync(out_best, a.best, nS * sizeof(pps_best),
                            cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && out_mask)
            e = cudaMemcpyAsync(out_mask, a.mask, nS * words * 4,
                                cudaMemcpyDeviceToHost, st);
        const size_t dbg_n = nS * n_speeds * (size_t)P;
        if (e == cudaSuccess && dbg && dbg->margin)
            e = cudaMemcpyAsync(dbg->margin, a.dbg_margin, dbg_n * 4,
                                cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && dbg && dbg->score)
            e = cudaMemcpyAsync(dbg->score, a.dbg_score, dbg_n * 4,
                                cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && dbg && dbg->T)
            e = cudaMemcpyAsync(dbg->T, a.dbg_T,
                                nS * (size_t)P * dbg->T_stride * 4,
                                cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "result download");
    }
    return PPS_OK;
}

}  // extern "C"

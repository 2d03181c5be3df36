// pps_plan.cu -- batched plans for uneven batches (include/pps.h, "Batched
// plans"): grouping by kernel instance, per-group work-item tables, the
// autotuner that picks each group's CTA size, and CUDA-graph replay.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "pps.h"
#include "pps_batch.cuh"
#include "pps_internal.h"

namespace {

// Candidates: (CTA size, samples a register block); every CTA size with
// one sample a block, the two smallest (registers to spare) also with two.
constexpr int kNumCand = 7;
constexpr int kCandTpb[kNumCand] = {128, 256, 512, 768, 1024, 128, 256};
constexpr int kCandKu[kNumCand] = {1, 1, 1, 1, 1, 2, 2};
constexpr int kMaxDevices = 64;

// Autotuner choices per (device, opponent slots, speed slots), shared by all
// plans of the process.
std::mutex g_tune_mu;
int g_tuned[kMaxDevices][4][4];  // candidate index + 1; 0 = not tuned yet

// Opponent-slot instances of the plan kernels.
int opp_slots(int max_opp) {
    return max_opp <= 6 ? 6 : max_opp <= 8 ? 8 : max_opp <= 12 ? 12 : 16;
}
int slot_of_j(int j) { return j == 6 ? 0 : j == 8 ? 1 : j == 12 ? 2 : 3; }
int slot_of_v(int v) { return v == 1 ? 0 : v == 2 ? 1 : v == 4 ? 2 : 3; }

int speed_slots(int n) { return n <= 1 ? 1 : n <= 2 ? 2 : n <= 4 ? 4 : 8; }

struct Group {
    int j = 8, v = 1;
    std::vector<int> states;      // state indices
    long long n_items = 0;
    int tpb = 512, ku = 1;
    float tuned_ms[kNumCand] = {0, 0, 0, 0, 0, 0, 0};
    long long states_off = 0;     // offset into the plan's bucket_states array
    long long start_off = 0;      // offset into the plan's item_start array
};

bool finite_pos(float x) { return std::isfinite(x) && x > 0.f; }

}  // namespace

struct pps_plan {
    pps_ctx* ctx = nullptr;
    int n = 0;
    unsigned flags = 0;
    pps_params prm{};
    std::vector<Group> groups;
    std::vector<long long> mask_off;  // n + 1
    // device tables
    pps_job* d_jobs = nullptr;
    int* d_bucket_states = nullptr;
    long long* d_item_start = nullptr;
    long long* d_mask_off = nullptr;
    unsigned long long* d_keys = nullptr;
    int* d_counts = nullptr;
    unsigned long long* d_next = nullptr;  // one work-queue counter per group
    unsigned char* d_recs = nullptr;       // per-state records (StateRec)
    size_t b_jobs = 0, b_states = 0, b_start = 0, b_mask = 0, b_keys = 0,
           b_counts = 0, b_next = 0, b_recs = 0;
    // autotuning and graph replay
    bool tuned = false;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* g_states = nullptr;
    const void* g_best = nullptr;
    const void* g_mask = nullptr;
};

namespace {

pps_status check_job(pps_ctx* ctx, const pps_job& j, int i) {
    const pps_grid& g = j.grid;
    if (!finite_pos(g.spacing) || g.nx < 1 || g.ny < 1 ||
        !std::isfinite(g.x0) || !std::isfinite(g.y0) ||
        (long long)g.nx * g.ny > (1 << 24))
        return pps_ctx_error(ctx, PPS_EINVAL, "job %d: bad grid", i);
    if (j.n_speeds < 1 || j.n_speeds > PPS_MAX_SPEEDS)
        return pps_ctx_error(ctx, PPS_EINVAL, "job %d: n_speeds %d outside 1..%d",
                             i, j.n_speeds, PPS_MAX_SPEEDS);
    for (int v = 0; v < j.n_speeds; ++v)
        if (!finite_pos(j.speeds[v]))
            return pps_ctx_error(ctx, PPS_EINVAL,
                                 "job %d: speed %d must be finite and > 0", i, v);
    if (j.max_opp < 0 || j.max_opp > PPS_MAX_OPP)
        return pps_ctx_error(ctx, PPS_EINVAL, "job %d: max_opp %d outside 0..%d",
                             i, j.max_opp, PPS_MAX_OPP);
    return PPS_OK;
}

pps_status check_params(pps_ctx* ctx, const pps_params& p) {
    const float v[] = {p.w_angle, p.w_dist, p.w_margin, p.margin_cap,
                       p.tau_safe, p.robot_radius, p.reach_radius,
                       p.min_pass_dist};
    for (float x : v)
        if (!std::isfinite(x))
            return pps_ctx_error(ctx, PPS_EINVAL, "params must be finite");
    if (p.robot_radius < 0.f || p.reach_radius < 0.f || p.min_pass_dist < 0.f)
        return pps_ctx_error(ctx, PPS_EINVAL,
                             "radii and min_pass_dist must be >= 0");
    return PPS_OK;
}

template <typename T>
pps_status upload(pps_plan* pl, T** dst, size_t* bytes, const T* src, size_t n,
                  const char* what) {
    *bytes = sizeof(T) * (n ? n : 1);
    pps_status s = pps_ctx_alloc(pl->ctx, (void**)dst, *bytes, what);
    if (s != PPS_OK) return s;
    if (n && src) {
        cudaError_t e = cudaMemcpy(*dst, src, sizeof(T) * n,
                                   cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return pps_ctx_cuda_error(pl->ctx, e, what);
    }
    return PPS_OK;
}

}  // namespace

extern "C" pps_status pps_plan_create(pps_ctx* ctx, const pps_job* jobs,
                                      int n_states, const pps_params* params,
                                      unsigned flags, pps_plan** out) {
    if (!out) return PPS_EINVAL;
    *out = nullptr;
    if (!ctx) return PPS_EINVAL;
    if (pps_ctx_failed(ctx))
        return pps_ctx_error(ctx, PPS_ECUDA,
                             "context failed earlier; call pps_reset");
    if (!jobs || n_states < 1 || n_states > (1 << 24))
        return pps_ctx_error(ctx, PPS_EINVAL, "n_states %d outside 1..2^24",
                             n_states);
    if (flags & ~(PPS_PLAN_AUTOTUNE | PPS_PLAN_GRAPH))
        return pps_ctx_error(ctx, PPS_EINVAL, "unknown plan flags 0x%x", flags);
    pps_params prm;
    if (params)
        prm = *params;
    else
        pps_default_params(&prm);
    pps_status s = check_params(ctx, prm);
    if (s != PPS_OK) return s;
    for (int i = 0; i < n_states; ++i)
        if ((s = check_job(ctx, jobs[i], i)) != PPS_OK) return s;

    pps_plan* pl = new (std::nothrow) pps_plan();
    if (!pl) return PPS_ENOMEM;
    pl->ctx = ctx;
    pl->n = n_states;
    pl->flags = flags;
    pl->prm = prm;

    // Group the states by kernel instance and lay out the mask.
    Group* by[4][4] = {};
    std::vector<Group> groups;
    groups.reserve(16);
    pl->mask_off.resize((size_t)n_states + 1);
    long long words = 0;
    for (int i = 0; i < n_states; ++i) {
        const pps_job& jb = jobs[i];
        const long long P = (long long)jb.grid.nx * jb.grid.ny;
        const long long w = (P + 31) / 32;
        pl->mask_off[i] = words;
        words += w * jb.n_speeds;
        const int J = opp_slots(jb.max_opp);
        const int V = speed_slots(jb.n_speeds);
        Group*& g = by[slot_of_j(J)][slot_of_v(V)];
        if (!g) {
            groups.emplace_back();
            g = &groups.back();
            g->j = J;
            g->v = V;
        }
        g->states.push_back(i);
    }
    pl->mask_off[n_states] = words;
    pl->groups = groups;

    // Per-group item tables: prefix sums of each state's 32-point items.
    std::vector<int> bucket_states;
    std::vector<long long> item_start;
    for (Group& g : pl->groups) {
        g.states_off = (long long)bucket_states.size();
        g.start_off = (long long)item_start.size();
        long long acc = 0;
        for (int st : g.states) {
            bucket_states.push_back(st);
            item_start.push_back(acc);
            const long long P = (long long)jobs[st].grid.nx * jobs[st].grid.ny;
            acc += (P + 31) / 32;
        }
        item_start.push_back(acc);
        g.n_items = acc;
    }
    cudaError_t e = cudaSetDevice(pps_ctx_device(ctx));
    if (e != cudaSuccess) {
        pps_plan_destroy(pl);
        return pps_ctx_cuda_error(ctx, e, "plan: cudaSetDevice");
    }
    if ((s = upload(pl, &pl->d_jobs, &pl->b_jobs, jobs, (size_t)n_states,
                    "plan jobs")) != PPS_OK ||
        (s = upload(pl, &pl->d_bucket_states, &pl->b_states,
                    bucket_states.data(), bucket_states.size(),
                    "plan states")) != PPS_OK ||
        (s = upload(pl, &pl->d_item_start, &pl->b_start, item_start.data(),
                    item_start.size(), "plan items")) != PPS_OK ||
        (s = upload(pl, &pl->d_mask_off, &pl->b_mask, pl->mask_off.data(),
                    pl->mask_off.size(), "plan mask offsets")) != PPS_OK ||
        (s = upload<unsigned long long>(pl, &pl->d_keys, &pl->b_keys, nullptr,
                                        (size_t)n_states, "plan keys")) !=
            PPS_OK ||
        (s = upload<int>(pl, &pl->d_counts, &pl->b_counts, nullptr,
                         (size_t)n_states, "plan counts")) != PPS_OK ||
        (s = upload<unsigned long long>(
             pl, &pl->d_next, &pl->b_next,
             std::vector<unsigned long long>(pl->groups.size(), 0ull).data(),
             pl->groups.size(), "plan queues")) != PPS_OK ||
        (s = upload<unsigned char>(pl, &pl->d_recs, &pl->b_recs, nullptr,
                                   (size_t)n_states * pps::kBatchRecStride,
                                   "plan state records")) != PPS_OK) {
        pps_plan_destroy(pl);
        return s;
    }
    if (flags & PPS_PLAN_GRAPH) {
        e = cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            pps_plan_destroy(pl);
            return pps_ctx_cuda_error(ctx, e, "plan: capture stream");
        }
    }
    // Groups whose instance this device has tuned before use that choice.
    const int dev = pps_ctx_device(ctx);
    if (dev >= 0 && dev < kMaxDevices) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        bool all = true;
        for (Group& g : pl->groups) {
            const int t = g_tuned[dev][slot_of_j(g.j)][slot_of_v(g.v)];
            if (t) {
                g.tpb = kCandTpb[t - 1];
                g.ku = kCandKu[t - 1];
            } else {
                all = false;
            }
        }
        pl->tuned = all;
    }
    *out = pl;
    return PPS_OK;
}

namespace {

pps::BatchArgs group_args(const pps_plan* pl, const Group& g,
                          const pps_state* states, pps_best* best,
                          uint32_t* mask) {
    pps::BatchArgs a;
    std::memset(&a, 0, sizeof a);
    a.states = states;
    a.jobs = pl->d_jobs;
    a.bucket_states = pl->d_bucket_states + g.states_off;
    a.item_start = pl->d_item_start + g.start_off;
    a.mask_off = pl->d_mask_off;
    a.n_bucket = (int)g.states.size();
    a.n_items = g.n_items;
    a.kmax = pps_ctx_max_K(pl->ctx);
    a.prm = pl->prm;
    a.best = best;
    a.mask = mask;
    a.keys = pl->d_keys;
    a.counts = pl->d_counts;
    a.next = pl->d_next + (&g - pl->groups.data());
    a.recs = pl->d_recs;
    return a;
}

// Persistent grid: CTAs resident on every SM, no more than the items need.
cudaError_t launch_group(const pps_plan* pl, const pps::BatchArgs& a,
                         const Group& g, int tpb, int ku, cudaStream_t st) {
    int occ = 1;
    switch (g.j) {
        case 6: occ = pps::batch_occupancy_j6(g.v, tpb, ku); break;
        case 8: occ = pps::batch_occupancy_j8(g.v, tpb, ku); break;
        case 12: occ = pps::batch_occupancy_j12(g.v, tpb, ku); break;
        default: occ = pps::batch_occupancy_j16(g.v, tpb, ku); break;
    }
    long long grid = (long long)pps_ctx_num_sms(pl->ctx) * occ;
    const long long need = (a.n_items + tpb / 32 - 1) / (tpb / 32);
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    switch (g.j) {
        case 6: return pps::batch_launch_j6(a, g.v, tpb, ku, (int)grid, st);
        case 8: return pps::batch_launch_j8(a, g.v, tpb, ku, (int)grid, st);
        case 12: return pps::batch_launch_j12(a, g.v, tpb, ku, (int)grid, st);
        default: return pps::batch_launch_j16(a, g.v, tpb, ku, (int)grid, st);
    }
}

cudaError_t enqueue_all(const pps_plan* pl, const pps_state* states,
                        pps_best* best, uint32_t* mask, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(pl->d_keys, 0, pl->b_keys, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->d_counts, 0, pl->b_counts, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->d_next, 0, pl->b_next, st);
    for (const Group& g : pl->groups) {
        if (e != cudaSuccess) break;
        e = launch_group(pl, group_args(pl, g, states, best, mask), g, g.tpb,
                         g.ku, st);
    }
    return e;
}

// Time each candidate (CTA size, samples a register block) on a prefix of
// every untuned group's items (enough items to fill the GPU several times
// over) and keep the fastest.
pps_status autotune(pps_plan* pl, const pps_state* states, pps_best* best,
                    uint32_t* mask) {
    pps_ctx* ctx = pl->ctx;
    const int dev = pps_ctx_device(ctx);
    cudaStream_t st = pps_ctx_stream(ctx);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const long long cap = (long long)pps_ctx_num_sms(ctx) * 16 * 24;
    for (Group& g : pl->groups) {
        if (e != cudaSuccess) break;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            const int t = g_tuned[dev][slot_of_j(g.j)][slot_of_v(g.v)];
            if (t) {
                g.tpb = kCandTpb[t - 1];
                g.ku = kCandKu[t - 1];
                continue;
            }
        }
        pps::BatchArgs a = group_args(pl, g, states, best, mask);
        a.n_items = std::min(a.n_items, cap);
        float best_ms = 1e30f;
        int best_c = 2;
        for (int c = 0; c < kNumCand && e == cudaSuccess; ++c) {
            const int tpb = kCandTpb[c], ku = kCandKu[c];
            e = launch_group(pl, a, g, tpb, ku, st);  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = launch_group(pl, a, g, tpb, ku, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) break;
            g.tuned_ms[c] = ms;
            if (ms < best_ms) {
                best_ms = ms;
                best_c = c;
            }
        }
        if (e != cudaSuccess) break;
        g.tpb = kCandTpb[best_c];
        g.ku = kCandKu[best_c];
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[dev][slot_of_j(g.j)][slot_of_v(g.v)] = best_c + 1;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return pps_ctx_cuda_error(ctx, e, "plan autotune");
    pl->tuned = true;
    return PPS_OK;
}

pps_status capture(pps_plan* pl, const pps_state* states, pps_best* best,
                   uint32_t* mask) {
    if (pl->exec) {
        cudaGraphExecDestroy(pl->exec);
        pl->exec = nullptr;
    }
    cudaError_t e = cudaStreamBeginCapture(pl->cap_stream,
                                           cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return pps_ctx_cuda_error(pl->ctx, e, "plan capture");
    cudaError_t le = enqueue_all(pl, states, best, mask, pl->cap_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(pl->cap_stream, &graph);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return pps_ctx_cuda_error(pl->ctx, le != cudaSuccess ? le : e,
                                  "plan capture");
    }
    e = cudaGraphInstantiate(&pl->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        pl->exec = nullptr;
        return pps_ctx_cuda_error(pl->ctx, e, "plan graph instantiate");
    }
    pl->g_states = states;
    pl->g_best = best;
    pl->g_mask = mask;
    return PPS_OK;
}

}  // namespace

extern "C" pps_status pps_plan_run(pps_plan* pl, const pps_state* states,
                                   pps_best* out_best, uint32_t* out_mask) {
    PPS_RANGE("pps_plan_run");
    if (!pl) return PPS_EINVAL;
    pps_ctx* ctx = pl->ctx;
    if (pps_ctx_failed(ctx))
        return pps_ctx_error(ctx, PPS_ECUDA,
                             "context failed earlier; call pps_reset");
    if (!states || !out_best)
        return pps_ctx_error(ctx, PPS_EINVAL,
                             "plan run: states and out_best are required");
    cudaError_t e = cudaSetDevice(pps_ctx_device(ctx));
    if (e != cudaSuccess) return pps_ctx_cuda_error(ctx, e, "cudaSetDevice");
    pps_status s;
    if ((pl->flags & PPS_PLAN_AUTOTUNE) && !pl->tuned &&
        (s = autotune(pl, states, out_best, out_mask)) != PPS_OK)
        return s;
    if (pl->flags & PPS_PLAN_GRAPH) {
        if (!pl->exec || pl->g_states != states || pl->g_best != out_best ||
            pl->g_mask != out_mask) {
            if ((s = capture(pl, states, out_best, out_mask)) != PPS_OK)
                return s;
        }
        e = cudaGraphLaunch(pl->exec, pps_ctx_stream(ctx));
        if (e != cudaSuccess) return pps_ctx_cuda_error(ctx, e, "plan graph launch");
        return PPS_OK;
    }
    e = enqueue_all(pl, states, out_best, out_mask, pps_ctx_stream(ctx));
    if (e != cudaSuccess) return pps_ctx_cuda_error(ctx, e, "plan launch");
    return PPS_OK;
}

extern "C" void pps_plan_destroy(pps_plan* pl) {
    if (!pl) return;
    pps_ctx* ctx = pl->ctx;
    cudaSetDevice(pps_ctx_device(ctx));
    cudaStreamSynchronize(pps_ctx_stream(ctx));
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    pps_ctx_free(ctx, pl->d_jobs, pl->b_jobs);
    pps_ctx_free(ctx, pl->d_bucket_states, pl->b_states);
    pps_ctx_free(ctx, pl->d_item_start, pl->b_start);
    pps_ctx_free(ctx, pl->d_mask_off, pl->b_mask);
    pps_ctx_free(ctx, pl->d_keys, pl->b_keys);
    pps_ctx_free(ctx, pl->d_counts, pl->b_counts);
    pps_ctx_free(ctx, pl->d_next, pl->b_next);
    pps_ctx_free(ctx, pl->d_recs, pl->b_recs);
    cudaGetLastError();
    delete pl;
}

extern "C" pps_status pps_plan_mask_offsets(const pps_plan* pl,
                                            int64_t* offsets) {
    if (!pl || !offsets) return PPS_EINVAL;
    for (size_t i = 0; i < pl->mask_off.size(); ++i)
        offsets[i] = (int64_t)pl->mask_off[i];
    return PPS_OK;
}

extern "C" pps_status pps_plan_groups(const pps_plan* pl, pps_plan_group* out,
                                      int cap, int* n) {
    if (!pl || !n || cap < 0 || (cap > 0 && !out)) return PPS_EINVAL;
    *n = (int)pl->groups.size();
    for (int i = 0; i < *n && i < cap; ++i) {
        const Group& g = pl->groups[i];
        out[i].opp_slots = g.j;
        out[i].speed_slots = g.v;
        out[i].n_states = (int32_t)g.states.size();
        out[i].cta_threads = g.tpb;
        out[i].sample_unroll = g.ku;
        out[i].n_items = g.n_items;
        for (int c = 0; c < kNumCand; ++c) out[i].tuned_ms[c] = g.tuned_ms[c];
    }
    return PPS_OK;
}

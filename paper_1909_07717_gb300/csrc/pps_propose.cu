// pps_propose.cu -- the proposal path (include/pps.h, "Learned proposal"):
// network prediction and top-k cells (pps_net.cu), then the exact search on
// the selected cells' fine grid points only, with the full-grid search as
// the fallback for states whose cells hold no feasible pass.

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>

#include "pps.h"
#include "pps_internal.h"
#include "pps_search.cuh"

char* pps_thread_error_buffer();

namespace {

constexpr int kMapW = PPS_NET_W, kMapPix = PPS_NET_H * PPS_NET_W;
constexpr int kFineNx = 481, kFineNy = 361;

// Exact search (eval_point) on the cells' fine points: a work item is half
// a cell (8 x 4 fine points centred on the map pixel's 8 x 8 block).  Items
// run rank-major -- every state's best-ranked cell first -- so that when a
// lower-ranked item starts, its state usually has a pass already; with
// `prune` an item whose score bound (score_bound: the whole mouth's angle
// and the last pass-line sample's margin, max over its points) falls below
// that pass's score is skipped: it cannot hold the best.
template <int JMAX, int VMAX>
__global__ void __launch_bounds__(pps::search_tpb<JMAX, VMAX>(), 1)
    refine_kernel(const pps::SearchArgs a, const int* __restrict__ cells,
                  int topk, bool prune) {
    constexpr int kWarps = pps::search_tpb<JMAX, VMAX>() / 32;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * kWarps;
    const long long gw = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const long long n_items = (long long)a.n_states * topk * 2;
    const pps::ItemGrid gr{a.g, a.x0, a.y0, a.V};
    for (long long item = gw; item < n_items; item += warps) {
        const int r = (int)(item / a.n_states);     // rank x 2 + half
        const int s = (int)(item - (long long)r * a.n_states);
        const int cell = cells[(long long)s * topk + (r >> 1)];
        const int cy = cell / kMapW, cx = cell - cy * kMapW;
        const int fx = 8 * cx - 4 + (lane & 7);
        const int fy = 8 * cy - 4 + (lane >> 3) + 4 * (r & 1);
        const bool active = fx >= 0 && fx < a.nx && fy >= 0 && fy < a.ny;
        const int ix = active ? fx : 0, iy = active ? fy : 0;
        const int p = iy * a.nx + ix;
        const pps_state& st = a.states[s];
        const pps::StateK sk = pps::derive_state(st, a.prm, JMAX, a.kmax);
        pps::OppRegs<JMAX> o;
        pps::load_opps<JMAX>(st, sk, o);
        if (prune) {
            // one read of the state's best so far, shared by the warp
            const unsigned long long cur =
                __shfl_sync(0xffffffffu, __ldcg(a.keys + s), 0);
            if (cur) {
                const float b =
                    active ? pps::score_bound<JMAX, VMAX>(a.prm, gr, a.speed,
                                                          a.speed2, sk, o, ix, iy)
                           : -CUDART_INF_F;
                // order_bits is monotone: compare the bound's key with the
                // score half of the best key
                const uint32_t bk =
                    __reduce_max_sync(0xffffffffu, pps::order_bits(b));
                if (bk < (uint32_t)(cur >> 32)) continue;
            }
        }
        pps::PointResult<JMAX, VMAX> res;
        pps::eval_point<JMAX, VMAX, false>(a.prm, gr, a.speed, a.speed2, st, sk,
                                           o, ix, iy, nullptr, res);
        int cnt = 0;
        unsigned long long key = 0ull;
#pragma unroll
        for (int v = 0; v < VMAX; ++v) {
            const bool f = active && v < a.V && res.feas[v];
            cnt += f;
            if (f) {
                const uint32_t idx = (uint32_t)(v * a.P + p);
                const unsigned long long k2 =
                    ((unsigned long long)pps::order_bits(res.score[v]) << 32) |
                    (unsigned long long)(~idx);
                key = k2 > key ? k2 : key;
            }
        }
        key = pps::warp_max_u64(key);
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0) {
            if (key) atomicMax(a.keys + s, key);
            if (cnt) atomicAdd(a.counts + s, cnt);
        }
    }
}

// After the refinement: skip[s] = 1 when the refined cells gave state s a
// pass (or the state is invalid); the others are appended to list.
__global__ void fallback_list_kernel(const pps_best* __restrict__ best, int n,
                                     int* __restrict__ skip,
                                     int* __restrict__ list,
                                     int* __restrict__ list_n) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const bool done = best[s].idx != -1;
    skip[s] = done;
    if (!done) list[atomicAdd(list_n, 1)] = s;
}

template <int J, int V>
int occupancy() {
    return pps_occupancy((const void*)refine_kernel<J, V>,
                         pps::search_tpb<J, V>(), 0);
}

template <int J, int V>
cudaError_t run(const pps::SearchArgs& base, const int* cells, int topk,
                bool fallback, bool prune, const pps_net_scratch& ns,
                int num_sms, cudaStream_t st) {
    const long long cap = (long long)num_sms * occupancy<J, V>();
    pps::SearchArgs a = base;
    cudaError_t e = cudaMemsetAsync(a.keys, 0, sizeof(unsigned long long) * a.n_states, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.counts, 0, sizeof(int) * a.n_states, st);
    if (e != cudaSuccess) return e;
    const long long items = (long long)a.n_states * topk * 2;
    constexpr int tpb = pps::search_tpb<J, V>();
    long long grid = (items + tpb / 32 - 1) / (tpb / 32);
    if (grid > cap) grid = cap;
    refine_kernel<J, V><<<(unsigned)grid, tpb, 0, st>>>(a, cells, topk, prune);
    pps::finalize_kernel<J, V><<<(a.n_states + 127) / 128, 128, 0, st>>>(a);
    if (!fallback) return cudaGetLastError();
    e = cudaMemsetAsync(ns.list_n, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    fallback_list_kernel<<<(a.n_states + 127) / 128, 128, 0, st>>>(
        a.best, a.n_states, ns.skip, ns.list, ns.list_n);
    e = cudaMemsetAsync(a.keys, 0, sizeof(unsigned long long) * a.n_states, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.counts, 0, sizeof(int) * a.n_states, st);
    if (e != cudaSuccess) return e;
    a.skip = ns.skip;
    a.list = ns.list;
    a.list_n = ns.list_n;
    // one CTA per SM at most: the list is usually empty or short
    pps::search_kernel<J, V, true>
        <<<(unsigned)num_sms, pps::search_tpb<J, V>(), 0, st>>>(a);
    pps::finalize_kernel<J, V><<<(a.n_states + 127) / 128, 128, 0, st>>>(a);
    return cudaGetLastError();
}

template <int J>
cudaError_t run_v(const pps::SearchArgs& a, const int* cells, int topk,
                  bool fb, bool pr, const pps_net_scratch& ns, int sms,
                  cudaStream_t st) {
    if (a.V <= 1) return run<J, 1>(a, cells, topk, fb, pr, ns, sms, st);
    if (a.V <= 2) return run<J, 2>(a, cells, topk, fb, pr, ns, sms, st);
    if (a.V <= 4) return run<J, 4>(a, cells, topk, fb, pr, ns, sms, st);
    return run<J, 8>(a, cells, topk, fb, pr, ns, sms, st);
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.f; }

}  // namespace

extern "C" pps_status pps_propose(pps_ctx* ctx, pps_net* net,
                                  const pps_state* states, int n,
                                  const pps_grid* fine, const float* speeds,
                                  int n_speeds, const pps_params* params,
                                  int topk, unsigned flags, pps_best* out_best,
                                  int32_t* out_cells) {
    PPS_RANGE("pps_propose");
    if (!ctx || !net) return PPS_EINVAL;
    if (pps_ctx_failed(ctx))
        return pps_ctx_error(ctx, PPS_ECUDA, "context failed earlier; call pps_reset");
    if (!states || !out_best || n < 1 || n > pps_ctx_max_states(ctx) ||
        n > pps_net_max_batch(net))
        return pps_ctx_error(ctx, PPS_EINVAL,
                             "pps_propose: n outside 1..min(max_states, max_batch)");
    if (!fine || fine->nx != kFineNx || fine->ny != kFineNy ||
        std::fabs(fine->spacing - 0.025f) > 1e-7f || fine->x0 != -6.f ||
        fine->y0 != -4.5f)
        return pps_ctx_error(ctx, PPS_EINVAL,
                             "pps_propose: fine grid must be 12x9 m at 0.025 m");
    if (topk < 1 || topk > kMapPix)
        return pps_ctx_error(ctx, PPS_EINVAL, "pps_propose: topk outside 1..2806");
    if (flags & ~(PPS_PROPOSE_FALLBACK | PPS_PROPOSE_NO_PRUNE))
        return pps_ctx_error(ctx, PPS_EINVAL, "pps_propose: unknown flags");
    if (!speeds || n_speeds < 1 || n_speeds > PPS_MAX_SPEEDS)
        return pps_ctx_error(ctx, PPS_EINVAL, "pps_propose: bad speeds");
    for (int v = 0; v < n_speeds; ++v)
        if (!finite_pos(speeds[v]))
            return pps_ctx_error(ctx, PPS_EINVAL, "pps_propose: bad speeds");
    pps_params prm;
    if (params)
        prm = *params;
    else
        pps_default_params(&prm);
    const float pv[] = {prm.w_angle, prm.w_dist, prm.w_margin, prm.margin_cap,
                        prm.tau_safe, prm.robot_radius, prm.reach_radius,
                        prm.min_pass_dist};
    for (float x : pv)
        if (!std::isfinite(x))
            return pps_ctx_error(ctx, PPS_EINVAL, "pps_propose: params must be finite");

    cudaError_t e = cudaSetDevice(pps_ctx_device(ctx));
    cudaStream_t nst = nullptr;
    float* scores = nullptr;
    int* cells = nullptr;
    pps_net_scratch ns{};
    if (e == cudaSuccess) e = pps_net_predict(net, states, n, &nst, &scores, &cells, &ns);
    if (out_cells) cells = out_cells;
    if (e == cudaSuccess) e = pps_net_topk(net, n, topk, cells);
    cudaStream_t st = pps_ctx_stream(ctx);
    if (e == cudaSuccess && nst != st) {
        // the exact refinement waits for the prediction on the net's stream
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, nst);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
        cudaEventDestroy(ev);
    }
    if (e != cudaSuccess) return pps_ctx_cuda_error(ctx, e, "pps_propose: predict");

    pps::SearchArgs a;
    std::memset(&a, 0, sizeof a);
    a.states = states;
    a.n_states = n;
    a.nx = fine->nx;
    a.ny = fine->ny;
    a.P = fine->nx * fine->ny;
    a.words = (a.P + 31) / 32;
    a.g = fine->spacing;
    a.x0 = fine->x0;
    a.y0 = fine->y0;
    a.V = n_speeds;
    a.kmax = pps_ctx_max_K(ctx);
    for (int v = 0; v < PPS_MAX_SPEEDS; ++v) {
        const float sv = speeds[v < n_speeds ? v : n_speeds - 1];
        a.speed[v] = sv;
        a.speed2[v] = sv * sv;
    }
    a.prm = prm;
    a.best = out_best;
    pps_ctx_scratch(ctx, &a.keys, &a.counts);
    const bool fb = flags & PPS_PROPOSE_FALLBACK;
    const bool prune = !(flags & PPS_PROPOSE_NO_PRUNE) && prm.w_angle >= 0.f &&
                       prm.w_margin >= 0.f;
    const int sms = pps_ctx_num_sms(ctx);
    e = pps_ctx_jmax(ctx) == 8
            ? run_v<8>(a, cells, topk, fb, prune, ns, sms, st)
            : run_v<16>(a, cells, topk, fb, prune, ns, sms, st);
    if (e != cudaSuccess) return pps_ctx_cuda_error(ctx, e, "pps_propose: refine");
    return PPS_OK;
}

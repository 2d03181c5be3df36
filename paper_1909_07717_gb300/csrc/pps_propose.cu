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
#include "pps_cells.cuh"
#include "pps_search.cuh"
#include "pps_staterec.cuh"
#include "pps_warpcopy.cuh"

char* pps_thread_error_buffer();

namespace {

constexpr int kMapW = PPS_NET_W, kMapPix = PPS_NET_H * PPS_NET_W;
constexpr int kFineNx = 481, kFineNy = 361;

// Exact search (eval_point) on the cells' fine points: a work item is half
// a cell (8 x 4 fine points centred on the map pixel's 8 x 8 block).  Items
// run rank-major -- every state's best-ranked cell first -- so that when a
// lower-ranked item starts, its state usually has a pass already; with
// `prune` an item whose score bound (score_bound: the whole mouth's angle
// and the margin over 4 of the pass-line samples, max over its points)
// falls below that pass's score is skipped: it cannot hold the best.
// Items are handed out one at a time from a work-queue counter (zero at
// launch): pruned items cost a small fraction of evaluated ones, so a
// static deal would leave most warps idle while a few finish theirs.
__device__ __forceinline__ long long next_item(unsigned long long* queue,
                                               int lane) {
    unsigned long long q = 0ull;
    if (lane == 0) q = atomicAdd(queue, 1ull);
    return (long long)__shfl_sync(0xffffffffu, q, 0);
}

// The large-batch refinement's items (half cells, rank-major) come from
// many states in turn; deriving each state per item took a fifth of its
// time, so the states' records are prepared once a call.
using pps::StateRec;
static_assert(sizeof(StateRec<PPS_MAX_OPP>) <= kPpsStateRecBytes,
              "the network's per-state scratch holds a record");

template <int JMAX>
__global__ void __launch_bounds__(128)
    prepare_states_kernel(const pps::SearchArgs a,
                          StateRec<JMAX>* __restrict__ recs) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.n_states) return;
    StateRec<JMAX> r;
    pps::make_state_rec<JMAX>(a.states[s], a.prm, a.kmax, r);
    recs[s] = r;
}

// SPLIT (small batches): a half cell is G items of 32 / G points, G lanes a
// point splitting its samples (G a power of two up to 32; the same bits, as
// in the per-job refinement below), each item deriving its state itself.
// Without SPLIT, G = 1 at compile time and the states' records come from
// prepare_states_kernel.
template <int JMAX, int VMAX, bool SPLIT>
__global__ void __launch_bounds__(pps::search_tpb<JMAX, VMAX>(), 1)
    refine_kernel(const pps::SearchArgs a, const int* __restrict__ cells,
                  int topk, int g, bool prune, unsigned long long* queue,
                  const StateRec<JMAX>* __restrict__ recs) {
    const int lane = threadIdx.x & 31;
    const int G = SPLIT ? g : 1;
    const long long n_items = (long long)a.n_states * topk * 2 * G;
    const pps::ItemGrid gr{a.g, a.x0, a.y0, a.V};
    for (long long item = next_item(queue, lane); item < n_items;
         item = next_item(queue, lane)) {
        const int rg = (int)(item / a.n_states);  // (rank x 2 + half) x G + sub
        const int s = (int)(item - (long long)rg * a.n_states);
        const int r = rg / G, pt = (rg - r * G) * (32 / G) + lane / G;
        const int cell = cells[(long long)s * topk + (r >> 1)];
        const int cy = cell / kMapW, cx = cell - cy * kMapW;
        const int fx = 8 * cx - 4 + (pt & 7);
        const int fy = 8 * cy - 4 + (pt >> 3) + 4 * (r & 1);
        const bool active = fx >= 0 && fx < a.nx && fy >= 0 && fy < a.ny;
        const int ix = active ? fx : 0, iy = active ? fy : 0;
        const int p = iy * a.nx + ix;
        const pps_state& st = a.states[s];
        pps::StateK sk;
        pps::OppRegs<JMAX> o;
        if constexpr (SPLIT) {
            sk = pps::derive_state(st, a.prm, JMAX, a.kmax);
            pps::load_opps<JMAX>(st, sk, o);
        } else {
            sk = recs[s].sk;
            o = recs[s].o;
        }
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
        pps::eval_point<JMAX, VMAX, false, pps::kKUnroll, SPLIT ? 0 : 1>(
            a.prm, gr, a.speed, a.speed2, st, sk, o, ix, iy, nullptr, res, G);
        const bool lead = (lane & (G - 1)) == 0;
        int cnt = 0;
        unsigned long long key = 0ull;
#pragma unroll
        for (int v = 0; v < VMAX; ++v) {
            const bool f = active && v < a.V && res.feas[v];
            cnt += f && lead;
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
    return pps_occupancy((const void*)refine_kernel<J, V, false>,
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
    constexpr int tpb = pps::search_tpb<J, V>();
    // lanes per point: doubled while the batch's items still fit in the
    // resident warps
    const long long halves = (long long)a.n_states * topk * 2;
    int G = 1;
    while (G < 32 && halves * 2 * G <= cap * (tpb / 32)) G *= 2;
    const long long items = halves * G;
    long long grid = (items + tpb / 32 - 1) / (tpb / 32);
    if (grid > cap) grid = cap;
    // the queue counter and the list's length (the next word) at once
    e = cudaMemsetAsync(ns.queue, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (G > 1) {
        refine_kernel<J, V, true><<<(unsigned)grid, tpb, 0, st>>>(
            a, cells, topk, G, prune, ns.queue, nullptr);
    } else {
        auto* recs = static_cast<StateRec<J>*>(ns.srec);
        prepare_states_kernel<J><<<(unsigned)((a.n_states + 127) / 128), 128, 0,
                                   st>>>(a, recs);
        refine_kernel<J, V, false><<<(unsigned)grid, tpb, 0, st>>>(
            a, cells, topk, 1, prune, ns.queue, recs);
    }
    pps::finalize_kernel<J, V><<<pps::finalize_blocks(a.n_states), 128, 0, st>>>(a);
    if (!fallback) return cudaGetLastError();
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
    pps::finalize_kernel<J, V><<<pps::finalize_blocks(a.n_states), 128, 0, st>>>(a);
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

// ------------------------------------------------ per-state fields and grids
// The proposal for states that each carry a job (grid and speeds), all
// grids of one spacing 0.2 / m on the map's cell lattice (cell_lattice):
// fields up to 12 x 9 m.  A state's work is its topk cells' m x m fine
// points, cut into items of 32 / G consecutive (cell rank, point) slots, a
// warp an item: G lanes share a point and split its samples (G = 1 for
// batches that fill the GPU; for small ones G grows, up to 32, until the
// items fill it, which cuts the latency of the call by up to G).  Items
// run rank-major: item q of every state before item q + 1 of any.
using pps::net::CellLattice;
using pps::net::cell_lattice;

struct JobsArgs {
    const pps_state* states;
    const pps_job* jobs;
    int n, kmax, m, vmax, topk, items_per_state;
    int lanes;  // G: lanes per point, a power of two up to 32
    pps_params prm;
    const int* cells;  // n x topk map pixels, best first
    pps_best* best;
    unsigned long long* keys;
    int* counts;
    int* list;    // fallback: the states to search on their full grid,
    int* list_n;  //   appended by the finalize
};

// A job's grid, speeds and cell lattice; valid = the state's grid has the
// call's spacing and lies on the lattice.
struct JobCells {
    pps::ItemGrid gr;
    int nx, ny, P, ox, oy;
    float sp[PPS_MAX_SPEEDS], sp2[PPS_MAX_SPEEDS];
    bool ok;
};

__device__ __forceinline__ void load_job_cells(const pps_job& j, int m,
                                               int vmax, JobCells& c) {
    const CellLattice cl = cell_lattice(j.grid);
    c.gr.g = j.grid.spacing;
    c.gr.x0 = j.grid.x0;
    c.gr.y0 = j.grid.y0;
    c.gr.V = j.n_speeds;
    c.nx = j.grid.nx;
    c.ny = j.grid.ny;
    c.P = c.nx * c.ny;
    c.ox = cl.ox;
    c.oy = cl.oy;
    c.ok = cl.ok && cl.m == m && j.n_speeds >= 1 && j.n_speeds <= vmax;
    const int nv = c.ok ? j.n_speeds : 1;
#pragma unroll
    for (int v = 0; v < PPS_MAX_SPEEDS; ++v) {
        const float x = j.speeds[v < nv ? v : nv - 1];
        c.sp[v] = x;
        c.sp2[v] = __fmul_rn(x, x);
    }
}

using pps::WarpStateJob;

__device__ __forceinline__ void load_state_job(WarpStateJob& d,
                                               const JobsArgs& a, int s,
                                               int lane) {
    pps::warp_load_state_job(d, a.states + s, a.jobs + s, lane);
}

// lead: the lane that counts its point's feasible passes (the first of the
// lanes that share the point; they all hold the same result).
template <int JMAX, int VMAX>
__device__ __forceinline__ void reduce_item(const JobsArgs& a, int s,
                                            int lane, bool active, bool lead,
                                            int p, int P, int V,
                                            const pps::PointResult<JMAX, VMAX>& r) {
    int cnt = 0;
    unsigned long long key = 0ull;
#pragma unroll
    for (int v = 0; v < VMAX; ++v) {
        const bool f = active && v < V && r.feas[v];
        cnt += f && lead;
        if (f) {
            const uint32_t idx = (uint32_t)(v * P + p);
            const unsigned long long k2 =
                ((unsigned long long)pps::order_bits(r.score[v]) << 32) |
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

template <int JMAX, int VMAX>
__global__ void __launch_bounds__(pps::search_tpb<JMAX, VMAX>(), 1)
    refine_jobs_kernel(const JobsArgs a, bool prune,
                       unsigned long long* queue) {
    const int lane = threadIdx.x & 31;
    const long long n_items = (long long)a.n * a.items_per_state;
    const int m2 = a.m * a.m;
    const int G = a.lanes, per = 32 / G;
    for (long long item = next_item(queue, lane); item < n_items;
         item = next_item(queue, lane)) {
        const int q = (int)(item / a.n);
        const int s = (int)(item - (long long)q * a.n);
        const int slot = q * per + lane / G;
        const int rank = slot / m2, within = slot - rank * m2;
        JobCells jc;
        load_job_cells(a.jobs[s], a.m, a.vmax, jc);
        bool active = jc.ok && rank < a.topk;
        int ix = 0, iy = 0;
        if (active) {
            const int cell = a.cells[(long long)s * a.topk + rank];
            const int cy = cell / kMapW, cx = cell - cy * kMapW;
            const int wy = within / a.m;
            ix = a.m * cx + jc.ox + (within - wy * a.m);
            iy = a.m * cy + jc.oy + wy;
            active = ix >= 0 && ix < jc.nx && iy >= 0 && iy < jc.ny;
        }
        if (__ballot_sync(0xffffffffu, active) == 0u) continue;
        if (!active) ix = iy = 0;
        const pps_state& st = a.states[s];
        const pps::StateK sk = pps::derive_state(st, a.prm, JMAX, a.kmax);
        pps::OppRegs<JMAX> o;
        pps::load_opps<JMAX>(st, sk, o);
        if (prune) {
            const unsigned long long cur =
                __shfl_sync(0xffffffffu, __ldcg(a.keys + s), 0);
            if (cur) {
                const float b =
                    active ? pps::score_bound<JMAX, VMAX>(a.prm, jc.gr, jc.sp,
                                                          jc.sp2, sk, o, ix, iy)
                           : -CUDART_INF_F;
                const uint32_t bk =
                    __reduce_max_sync(0xffffffffu, pps::order_bits(b));
                if (bk < (uint32_t)(cur >> 32)) continue;
            }
        }
        pps::PointResult<JMAX, VMAX> res;
        pps::eval_point<JMAX, VMAX, false, pps::kKUnroll, 0>(
            a.prm, jc.gr, jc.sp, jc.sp2, st, sk, o, ix, iy, nullptr, res, G);
        reduce_item<JMAX, VMAX>(a, s, lane, active, (lane & (G - 1)) == 0,
                                iy * jc.nx + ix, jc.P, jc.gr.V, res);
    }
}

// The finalize of state s by one warp (my: the warp's shared copy):
// decode the key, re-evaluate the winner for its margin and check that the
// score reproduces; clears the state's key and count for the next call.  A
// state whose job does not fit the call (another spacing, off the lattice,
// bad speeds) is invalid.  With `append`, a valid state without a pass is
// appended to the fallback list.  The key and count are read from L2 (the
// refinement's atomics complete there).
template <int JMAX, int VMAX>
__device__ __noinline__ void finalize_state(const JobsArgs& a, int s,
                                            int lane, WarpStateJob& my,
                                            bool append) {
    const unsigned long long key = __ldcg(a.keys + s);
    const int count = __ldcg(a.counts + s);
    load_state_job(my, a, s, lane);
    const pps_state& st = my.st;
    JobCells jc;
    load_job_cells(my.job, a.m, a.vmax, jc);
    pps::StateK sk = pps::derive_state(st, a.prm, JMAX, a.kmax);
    sk.valid = sk.valid && jc.ok;
    pps_best b;
    b.n_feasible = count;
    b.status = sk.valid ? PPS_STATE_OK : PPS_STATE_INVALID;
    if (!sk.valid || key == 0ull) {
        b.idx = sk.valid ? -1 : -2;
        b.ix = b.iy = b.speed_idx = -1;
        b.score = -CUDART_INF_F;
        b.margin = -CUDART_INF_F;
        b.n_feasible = sk.valid ? b.n_feasible : 0;
    } else {
        const uint32_t idx = ~(uint32_t)(key & 0xffffffffull);
        const int v = (int)(idx / (uint32_t)jc.P);
        const int p = (int)(idx - (uint32_t)v * (uint32_t)jc.P);
        b.idx = (int)idx;
        b.speed_idx = v;
        b.iy = p / jc.nx;
        b.ix = p - b.iy * jc.nx;
        b.score = pps::order_bits_inv((uint32_t)(key >> 32));
        pps::OppRegs<JMAX> o;
        pps::load_opps<JMAX>(st, sk, o);
        pps::PointResult<JMAX, VMAX> r;
        pps::eval_point<JMAX, VMAX, false, pps::kKUnroll, 32>(
            a.prm, jc.gr, jc.sp, jc.sp2, st, sk, o, b.ix, b.iy, nullptr, r);
        float mg = 0.f, sc = 0.f;
        bool f = false;
#pragma unroll
        for (int w = 0; w < VMAX; ++w)
            if (w == v) {
                mg = r.margin[w];
                sc = r.score[w];
                f = r.feas[w];
            }
        b.margin = mg;
        if (!f || __float_as_uint(sc) != __float_as_uint(b.score))
            b.status |= PPS_STATE_INCONSISTENT;
    }
    if (lane != 0) return;
    a.best[s] = b;
    a.keys[s] = 0ull;
    a.counts[s] = 0;
    if (append && b.idx == -1) a.list[atomicAdd(a.list_n, 1)] = s;
}

// One warp per state.
constexpr int kFinalizeTpb = 128;

template <int JMAX, int VMAX>
__global__ void __launch_bounds__(kFinalizeTpb)
    jobs_finalize_kernel(const JobsArgs a, bool append) {
    __shared__ WarpStateJob sh[kFinalizeTpb / 32];
    const int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (i >= a.n) return;
    finalize_state<JMAX, VMAX>(a, i, threadIdx.x & 31, sh[threadIdx.x >> 5],
                               append);
}

// Fallback: the listed states on their full grids.  A CTA takes a listed
// state at a time and its warps share that state's 32-point items; its
// first warp then finalizes the state.
template <int JMAX, int VMAX>
__global__ void __launch_bounds__(pps::search_tpb<JMAX, VMAX>(), 1)
    fallback_jobs_kernel(const JobsArgs a) {
    constexpr int kWarps = pps::search_tpb<JMAX, VMAX>() / 32;
    __shared__ WarpStateJob sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nl = *a.list_n;
    for (int li = blockIdx.x; li < nl; li += gridDim.x) {
        const int s = a.list[li];
        JobCells jc;
        load_job_cells(a.jobs[s], a.m, a.vmax, jc);
        if (!jc.ok) continue;
        const pps_state& st = a.states[s];
        const pps::StateK sk = pps::derive_state(st, a.prm, JMAX, a.kmax);
        pps::OppRegs<JMAX> o;
        pps::load_opps<JMAX>(st, sk, o);
        const int words = (jc.P + 31) / 32;
        for (int chunk = warp; chunk < words; chunk += kWarps) {
            const int p = chunk * 32 + lane;
            const bool active = p < jc.P;
            const int pc = active ? p : jc.P - 1;
            const int iy = pc / jc.nx, ix = pc - iy * jc.nx;
            pps::PointResult<JMAX, VMAX> res;
            pps::eval_point<JMAX, VMAX, false>(a.prm, jc.gr, jc.sp, jc.sp2, st,
                                               sk, o, ix, iy, nullptr, res);
            reduce_item<JMAX, VMAX>(a, s, lane, active, true, p, jc.P,
                                    jc.gr.V, res);
        }
        // the state is this CTA's alone: its first warp finalizes it once
        // every warp's atomics are done
        __syncthreads();
        if (warp == 0) finalize_state<JMAX, VMAX>(a, s, lane, sh, false);
    }
}

template <int J, int V>
cudaError_t run_jobs(JobsArgs a, bool fallback, bool prune,
                     const pps_net_scratch& ns, int num_sms, cudaStream_t st) {
    constexpr int tpb = pps::search_tpb<J, V>();
    cudaError_t e = cudaMemsetAsync(a.keys, 0, sizeof(unsigned long long) * a.n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.counts, 0, sizeof(int) * a.n, st);
    if (e != cudaSuccess) return e;
    const long long cap =
        (long long)num_sms *
        pps_occupancy((const void*)refine_jobs_kernel<J, V>, tpb, 0);
    // lanes per point: doubled while the batch's items still fit in the
    // resident warps
    const long long slots = (long long)a.topk * a.m * a.m;
    const long long warps = cap * (tpb / 32);
    int G = 1;
    while (G < 32 && (long long)a.n * ((slots * 2 * G + 31) / 32) <= warps)
        G *= 2;
    a.lanes = G;
    a.items_per_state = (int)((slots * G + 31) / 32);
    const long long items = (long long)a.n * a.items_per_state;
    long long grid = (items + tpb / 32 - 1) / (tpb / 32);
    if (grid > cap) grid = cap;
    // the queue counter and the list's length (the next word) at once
    e = cudaMemsetAsync(ns.queue, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (fallback) {
        a.list = ns.list;
        a.list_n = ns.list_n;
    }
    refine_jobs_kernel<J, V><<<(unsigned)grid, tpb, 0, st>>>(a, prune,
                                                             ns.queue);
    jobs_finalize_kernel<J, V>
        <<<(unsigned)((a.n + kFinalizeTpb / 32 - 1) / (kFinalizeTpb / 32)),
           kFinalizeTpb, 0, st>>>(a, fallback);
    if (!fallback) return cudaGetLastError();
    // the finalize left every key and count at zero and listed the states
    // without a pass
    fallback_jobs_kernel<J, V><<<(unsigned)num_sms, tpb, 0, st>>>(a);
    return cudaGetLastError();
}

template <int J>
cudaError_t run_jobs_v(const JobsArgs& a, int vslots, bool fb, bool pr,
                       const pps_net_scratch& ns, int sms, cudaStream_t st) {
    if (vslots <= 1) return run_jobs<J, 1>(a, fb, pr, ns, sms, st);
    if (vslots <= 2) return run_jobs<J, 2>(a, fb, pr, ns, sms, st);
    if (vslots <= 4) return run_jobs<J, 4>(a, fb, pr, ns, sms, st);
    return run_jobs<J, 8>(a, fb, pr, ns, sms, st);
}

}  // namespace

// Library-internal: the per-job proposal of n states (device states and
// jobs) on the network's stream, which must be `st` or ordered before it by
// the caller: prediction, top-k (off-grid cells last), refinement and the
// optional fallback.
cudaError_t pps_propose_jobs_enqueue(pps_net* net, const PpsProposeJobs& p,
                                     cudaStream_t st) {
    cudaStream_t nst = nullptr;
    float* scores = nullptr;
    int* cells = nullptr;
    pps_net_scratch ns{};
    cudaError_t e = pps_net_predict(net, p.states, p.n, &nst, &scores, &cells, &ns);
    if (p.out_cells) cells = p.out_cells;
    if (e == cudaSuccess) e = pps_net_topk(net, p.n, p.topk, cells, p.jobs);
    if (e == cudaSuccess && nst != st) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, nst);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
        cudaEventDestroy(ev);
    }
    if (e != cudaSuccess) return e;
    JobsArgs a;
    std::memset(&a, 0, sizeof a);
    a.states = p.states;
    a.jobs = p.jobs;
    a.n = p.n;
    a.kmax = p.kmax;
    a.m = p.m;
    a.vmax = p.vslots;
    a.topk = p.topk;
    a.prm = p.prm;
    a.cells = cells;
    a.best = p.best;
    a.keys = p.keys;
    a.counts = p.counts;
    const bool prune = p.prune && p.prm.w_angle >= 0.f && p.prm.w_margin >= 0.f;
    if (p.jslots <= 8)
        return run_jobs_v<8>(a, p.vslots, p.fallback, prune, ns, p.num_sms, st);
    if (p.jslots <= 12)
        return run_jobs_v<12>(a, p.vslots, p.fallback, prune, ns, p.num_sms, st);
    return run_jobs_v<16>(a, p.vslots, p.fallback, prune, ns, p.num_sms, st);
}

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

extern "C" pps_status pps_propose_jobs(pps_ctx* ctx, pps_net* net,
                                       const pps_state* states,
                                       const pps_job* jobs, int n,
                                       float spacing, int max_speeds,
                                       const pps_params* params, int topk,
                                       unsigned flags, pps_best* out_best,
                                       int32_t* out_cells) {
    PPS_RANGE("pps_propose_jobs");
    if (!ctx || !net) return PPS_EINVAL;
    if (pps_ctx_failed(ctx))
        return pps_ctx_error(ctx, PPS_ECUDA, "context failed earlier; call pps_reset");
    if (!states || !jobs || !out_best || n < 1 || n > pps_ctx_max_states(ctx) ||
        n > pps_net_max_batch(net))
        return pps_ctx_error(ctx, PPS_EINVAL,
                             "pps_propose_jobs: n outside 1..min(max_states, "
                             "max_batch), or a NULL buffer");
    pps_grid probe{spacing, 1, 1, -6.f, -4.5f};
    const CellLattice cl = cell_lattice(probe);
    if (!cl.ok)
        return pps_ctx_error(ctx, PPS_EINVAL,
                             "pps_propose_jobs: spacing must be 0.2, 0.1, "
                             "0.05 or 0.025 m");
    if (max_speeds < 1 || max_speeds > PPS_MAX_SPEEDS)
        return pps_ctx_error(ctx, PPS_EINVAL, "pps_propose_jobs: max_speeds "
                                              "outside 1..8");
    if (topk < 1 || topk > kMapPix)
        return pps_ctx_error(ctx, PPS_EINVAL, "pps_propose_jobs: topk outside 1..2806");
    if (flags & ~(PPS_PROPOSE_FALLBACK | PPS_PROPOSE_NO_PRUNE))
        return pps_ctx_error(ctx, PPS_EINVAL, "pps_propose_jobs: unknown flags");
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
            return pps_ctx_error(ctx, PPS_EINVAL, "pps_propose_jobs: params must be finite");
    cudaError_t e = cudaSetDevice(pps_ctx_device(ctx));
    PpsProposeJobs p;
    std::memset(&p, 0, sizeof p);
    p.states = states;
    p.jobs = jobs;
    p.n = n;
    const int mo = pps_ctx_max_opp(ctx);
    p.jslots = mo <= 8 ? 8 : mo <= 12 ? 12 : 16;
    p.vslots = max_speeds;
    p.m = cl.m;
    p.topk = topk;
    p.kmax = pps_ctx_max_K(ctx);
    p.fallback = flags & PPS_PROPOSE_FALLBACK;
    p.prune = !(flags & PPS_PROPOSE_NO_PRUNE);
    p.prm = prm;
    p.best = out_best;
    p.out_cells = out_cells;
    pps_ctx_scratch(ctx, &p.keys, &p.counts);
    p.num_sms = pps_ctx_num_sms(ctx);
    if (e == cudaSuccess)
        e = pps_propose_jobs_enqueue(net, p, pps_ctx_stream(ctx));
    if (e != cudaSuccess) return pps_ctx_cuda_error(ctx, e, "pps_propose_jobs");
    return PPS_OK;
}

// pps_batch.cuh -- device code of the batched plans (uneven batches).
//
// A plan searches states that each carry their own receive grid and kick
// speeds (pps_job).  The host groups the states into buckets by kernel
// instance (opponent slots JMAX, speed slots VMAX); within a bucket the work
// items are (state, 32 consecutive grid points) as in the single-grid
// search, numbered through a per-bucket prefix sum of each state's item
// count, so states of very different grid sizes share one persistent launch.
// The launch is persistent: every warp takes the next few items from an
// atomic counter (a work queue over the item range, so that warps whose
// items were cheap -- short pass lines, small K -- take more of them) and
// finds each item's state by binary search in the prefix sum.  The per-point arithmetic is eval_point, the same
// device code the single-grid search runs.
#pragma once

#include "pps_search.cuh"
#include "pps_staterec.cuh"
#include "pps_warpcopy.cuh"

namespace pps {

struct BatchArgs {
    const pps_state* states;      // every state of the plan
    const pps_job* jobs;          // per-state grid, speeds, opponent slots
    const int* bucket_states;     // state indices of this bucket
    const long long* item_start;  // n_bucket + 1 prefix sums of items
    const long long* mask_off;    // per state: its first mask word
    int n_bucket;
    long long n_items;
    int kmax;
    pps_params prm;
    pps_best* best;
    uint32_t* mask;               // may be null
    unsigned long long* keys;     // per state of the plan
    int* counts;                  // per state of the plan
    unsigned long long* next;     // the launch's work-queue counter: 0 when
                                  // it starts, left 0 by the finalize kernel
    unsigned char* recs;          // may be null: kBatchRecStride bytes per
                                  // state of the plan (StateRec)
};

// The states' records (StateRec), prepared once a run by
// batch_prepare_kernel for the plans, whose items (32 points of one state,
// one at a time) then load them instead of deriving them each; the serving
// loop's small launches pass none and derive them per item.
constexpr size_t kBatchRecStride = 336;
static_assert(sizeof(StateRec<PPS_MAX_OPP>) <= kBatchRecStride &&
                  kBatchRecStride % 16 == 0,
              "a record fits its 16-byte aligned slot");

// Items a warp takes from the work queue at a time.
constexpr unsigned long long kQueueRun = 4;

// A job's grid in the form the kernels use; speeds padded with the last one.
struct JobView {
    ItemGrid gr;
    int nx, P, words;
    float sp[PPS_MAX_SPEEDS], sp2[PPS_MAX_SPEEDS];
};

__device__ __forceinline__ void load_job(const pps_job& j, JobView& v) {
    v.gr.g = j.grid.spacing;
    v.gr.x0 = j.grid.x0;
    v.gr.y0 = j.grid.y0;
    v.gr.V = j.n_speeds;
    v.nx = j.grid.nx;
    v.P = j.grid.nx * j.grid.ny;
    v.words = (v.P + 31) >> 5;
#pragma unroll
    for (int s = 0; s < PPS_MAX_SPEEDS; ++s) {
        const float x = j.speeds[s < j.n_speeds ? s : j.n_speeds - 1];
        v.sp[s] = x;
        v.sp2[s] = __fmul_rn(x, x);
    }
}

// Largest b with item_start[b] <= item (item_start is non-decreasing).
__device__ __forceinline__ int find_bucket_slot(const long long* start, int n,
                                                long long item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// One work item: 32 consecutive grid points of one state (all lanes); KU
// samples a register block.
template <int JMAX, int VMAX, int KU>
__device__ __forceinline__ void batch_item(const BatchArgs& a, long long item,
                                           int lane) {
    {
        const int b = find_bucket_slot(a.item_start, a.n_bucket, item);
        const int s = __ldg(a.bucket_states + b);
        const int chunk = (int)(item - __ldg(a.item_start + b));
        JobView jv;
        load_job(a.jobs[s], jv);
        const pps_state& st = a.states[s];
        StateK sk;
        OppRegs<JMAX> o;
        if (a.recs) {
            const StateRec<JMAX>& r = *reinterpret_cast<const StateRec<JMAX>*>(
                a.recs + (size_t)s * kBatchRecStride);
            sk = r.sk;
            o = r.o;
        } else {
            sk = derive_state(st, a.prm, JMAX, a.kmax);
            load_opps<JMAX>(st, sk, o);
        }

        const int p = chunk * 32 + lane;
        const bool active = p < jv.P;
        const int pc = active ? p : jv.P - 1;
        const int iy = pc / jv.nx, ix = pc - iy * jv.nx;

        PointResult<JMAX, VMAX> r;
        eval_point<JMAX, VMAX, false, KU>(a.prm, jv.gr, jv.sp, jv.sp2, st, sk, o,
                                          ix, iy, nullptr, r);

        int cnt = 0;
        unsigned long long key = 0ull;
        const long long mbase = __ldg(a.mask_off + s);
#pragma unroll
        for (int v = 0; v < VMAX; ++v) {
            const bool f = active && v < jv.gr.V && r.feas[v];
            cnt += f;
            if (f) {
                const uint32_t idx = (uint32_t)(v * jv.P + p);
                const unsigned long long k2 =
                    ((unsigned long long)order_bits(r.score[v]) << 32) |
                    (unsigned long long)(~idx);
                key = k2 > key ? k2 : key;
            }
            if (v < jv.gr.V) {
                const uint32_t word = __ballot_sync(0xffffffffu, f);
                if (a.mask && lane == 0)
                    a.mask[mbase + (long long)v * jv.words + chunk] = word;
            }
        }
        key = warp_max_u64(key);
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0) {
            if (key) atomicMax(a.keys + s, key);
            if (cnt) atomicAdd(a.counts + s, cnt);
        }
    }
}

// The records of the bucket's states, a thread a state.
template <int JMAX>
__global__ void __launch_bounds__(128) batch_prepare_kernel(const BatchArgs a) {
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= a.n_bucket) return;
    const int s = a.bucket_states[i];
    StateRec<JMAX> r;
    make_state_rec<JMAX>(a.states[s], a.prm, a.kmax, r);
    *reinterpret_cast<StateRec<JMAX>*>(a.recs + (size_t)s * kBatchRecStride) = r;
}

template <int JMAX, int VMAX, int TPB, int KU>
__global__ void __launch_bounds__(TPB) batch_search_kernel(const BatchArgs a) {
    const int lane = threadIdx.x & 31;
    // several items a fetch only when there are many per warp: a small
    // launch (a serving batch) spreads its items one per warp
    const long long warps = (long long)gridDim.x * (TPB / 32);
    const unsigned long long run =
        a.n_items >= warps * 16 ? kQueueRun : 1ull;
    for (;;) {
        unsigned long long q = 0ull;
        if (lane == 0) q = atomicAdd(a.next, run);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= (unsigned long long)a.n_items) break;
        const long long end = (long long)(q + run) < a.n_items
                                  ? (long long)(q + run)
                                  : a.n_items;
        for (long long item = (long long)q; item < end; ++item)
            batch_item<JMAX, VMAX, KU>(a, item, lane);
    }
}

// One warp per state of the bucket (finalize_blocks(n) CTAs of 128): decode
// the key, re-evaluate the winning point for its margin (the lanes sharing
// its samples) and check that the score reproduces; lane 0 writes.
template <int JMAX, int VMAX>
__global__ void __launch_bounds__(128) batch_finalize_kernel(const BatchArgs a) {
    __shared__ WarpStateJob sh[128 / 32];  // the warp's state and job
    const int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const bool lead = lane == 0;
    if (i == 0 && lead) *a.next = 0ull;  // the queue is empty again for the next launch
    if (i >= a.n_bucket) return;
    const int s = a.bucket_states[i];
    const unsigned long long key = a.keys[s];
    const int count = a.counts[s];
    WarpStateJob& my = sh[threadIdx.x >> 5];
    warp_load_state_job(my, a.states + s, a.jobs + s, lane);
    const pps_state& st = my.st;
    const StateK sk = derive_state(st, a.prm, JMAX, a.kmax);
    JobView jv;
    load_job(my.job, jv);
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
        const int v = (int)(idx / (uint32_t)jv.P);
        const int p = (int)(idx - (uint32_t)v * (uint32_t)jv.P);
        b.idx = (int)idx;
        b.speed_idx = v;
        b.iy = p / jv.nx;
        b.ix = p - b.iy * jv.nx;
        b.score = order_bits_inv((uint32_t)(key >> 32));
        OppRegs<JMAX> o;
        load_opps<JMAX>(st, sk, o);
        PointResult<JMAX, VMAX> r;
        eval_point<JMAX, VMAX, false, kKUnroll, 32>(a.prm, jv.gr, jv.sp, jv.sp2, st,
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
    if (!lead) return;
    a.best[s] = b;
    // Leave the scratch cleared for the next launch that reuses it.
    a.keys[s] = 0ull;
    a.counts[s] = 0;
}

// Launch entry points, one translation unit per opponent-slot count
// (6, 8, 12, 16: the plan picks the smallest that holds a job's opponents).
// ku: samples a register block (1, or 2 at 128 and 256 threads).
#define PPS_BATCH_DECLARE(J)                                              \
    cudaError_t batch_launch_j##J(const BatchArgs& a, int vmax, int tpb, \
                                  int ku, int grid, cudaStream_t st);    \
    int batch_occupancy_j##J(int vmax, int tpb, int ku);
PPS_BATCH_DECLARE(6)
PPS_BATCH_DECLARE(8)
PPS_BATCH_DECLARE(12)
PPS_BATCH_DECLARE(16)
#undef PPS_BATCH_DECLARE

}  // namespace pps

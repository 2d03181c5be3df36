/*
 * pps.h -- C ABI of libpps, the GB300 (sm_103a) passing-point search.
 *
 * libpps computes the data-parallel core of the SBIP-based dynamic
 * passing-point search (DPPS) of the ZJUNlict 2019 team description paper:
 * for every game state, every candidate receive point of a field grid and
 * every kick speed it decides whether any opponent can intercept the pass
 * (Sec. 4.2), scores the feasible passes with the weighted-sum value
 * function (Sec. 4.3, Eq. 3) and returns the best pass per state.
 *
 * Model (the paper's prose, and the readings this library takes where the
 * paper is silent):
 *   ball     (Sec. 4.1, Eq. 1 read as d = v t - a t^2/2): rolls from the
 *            kick speed v with constant deceleration a (the short sliding
 *            phase neglected); it stops after v^2/(2a).
 *   samples  (Sec. 4.2): the ball is checked at K points spaced uniformly
 *            in distance along the pass line, k = 1..K, the receiver point
 *            being sample K.
 *   opponent (Sec. 4.2, SBIP): minimum time to bring its centre within
 *            reach_radius of a sample under a 1-D bang-bang motion along the
 *            line to it -- acceleration amax, speed cap vmax, starting from
 *            its velocity component toward the sample.
 *   feasible (Sec. 4.2): the ball reaches the receiver, the pass is at least
 *            min_pass_dist long, and margin > tau_safe, where
 *            margin = min_k (min_j t_opp_j(sample k) - t_ball(sample k)).
 *   score    (Sec. 4.3, Eq. 3; Sec. 4.4 shot angle):
 *            w_angle * theta / pi - w_dist * |receiver - goal| / diag
 *            + w_margin * min(margin, margin_cap), theta the largest
 *            opponent-free angular gap of the goal mouth (x = +L/2) seen from
 *            the receiver, opponents as discs of robot_radius; theta = 0 on
 *            or behind the goal line.
 *   best     (Sec. 1 item 1, Sec. 4.3): highest score; ties go to the
 *            smallest candidate index idx = v * P + iy * nx + ix.
 *
 * Conventions.  All functions return a pps_status and never abort or exit.
 * Floats are IEEE binary32, integers are int32 unless stated.  The caller
 * owns every input and output buffer and must keep them alive until the
 * work is complete (pps_sync, or a sync of the context's stream); the
 * library keeps no caller pointer past that point.  A context is used by
 * one host thread at a time.
 */
#ifndef PPS_H
#define PPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PPS_ABI_VERSION 2

#define PPS_MAX_OPP 16   /* opponents per state (the paper: up to 16 a side) */
#define PPS_MAX_SPEEDS 8 /* kick speeds per call */
#define PPS_MAX_K 4096   /* samples per pass line */

typedef int pps_status;
#define PPS_OK 0
#define PPS_EINVAL 1   /* an argument or an input value is out of range */
#define PPS_ENOMEM 2   /* device memory or the context's budget ran out */
#define PPS_ECUDA 3    /* a CUDA call failed; the context needs pps_reset */
#define PPS_ETIMEOUT 4 /* a bounded device wait gave up */
#define PPS_ENOTIMPL 5 /* not available in this library */

/* pps_search flag: every buffer argument is device memory (e.g. a torch
 * CUDA tensor's data pointer).  Without it they are host memory; the
 * library then stages them through its own device buffers and copies the
 * results back asynchronously on the context's stream (pinned host memory
 * makes those copies truly asynchronous). */
#define PPS_DEVICE_PTRS 1u

/* pps_best.status bits (per state). */
#define PPS_STATE_OK 0
#define PPS_STATE_INVALID 1      /* the state failed validation: no result */
#define PPS_STATE_INCONSISTENT 2 /* self-check: the best score could not be
                                    reproduced when re-evaluated (a library
                                    bug; please report) */

/* One game state.  296 bytes, 4-byte aligned, no padding.  Coordinates in
 * metres with the field centred on the origin, x toward the opponent goal,
 * velocities in m/s.  Opponent slots n_opp..PPS_MAX_OPP-1 are ignored. */
typedef struct pps_state {
    float ball[2];                  /* kick point (the passer's ball) */
    int32_t n_opp;                  /* 0..PPS_MAX_OPP opponents */
    float opp_pos[PPS_MAX_OPP][2];  /* opponent centres */
    float opp_vel[PPS_MAX_OPP][2];  /* opponent velocities */
    float ball_decel;               /* rolling deceleration a > 0, m/s^2 */
    float vmax;                     /* opponent speed limit > 0 */
    float amax;                     /* opponent acceleration limit > 0 */
    float field_len;                /* L > 0 (goal line at x = +L/2) */
    float field_wid;                /* W > 0 */
    float goal_width;               /* goal mouth width >= 0 */
    int32_t K;                      /* samples per pass line, 1..PPS_MAX_K */
} pps_state;

/* Candidate receive points: (x0 + ix * spacing, y0 + iy * spacing),
 * 0 <= ix < nx, 0 <= iy < ny; point index p = iy * nx + ix, P = nx * ny. */
typedef struct pps_grid {
    float spacing;
    int32_t nx, ny;
    float x0, y0;
} pps_grid;

/* Value-function weights and thresholds (Sec. 4.3: "adjustable"; the
 * paper gives no values -- pps_default_params gives the library's). */
typedef struct pps_params {
    float w_angle;       /* weight of theta / pi */
    float w_dist;        /* weight of -(receiver-to-goal distance) / diag */
    float w_margin;      /* weight of min(margin, margin_cap), in 1/s */
    float margin_cap;    /* s */
    float tau_safe;      /* feasibility threshold on the margin, s */
    float robot_radius;  /* opponent disc radius for shot blocking, m */
    float reach_radius;  /* opponent intercepts within this distance, m */
    float min_pass_dist; /* shortest pass considered, m */
} pps_params;

/* Result per state.  idx = -1 when no pass is feasible (score and margin
 * then -inf, ix = iy = speed_idx = -1); idx = -2 when the state was
 * invalid (status has PPS_STATE_INVALID). */
typedef struct pps_best {
    int32_t idx;        /* speed_idx * P + iy * nx + ix */
    int32_t ix, iy;
    int32_t speed_idx;
    float score;
    float margin;       /* margin of the best pass, s */
    int32_t n_feasible; /* feasible (point, speed) pairs of the state */
    int32_t status;     /* PPS_STATE_* bits */
} pps_best;

/* Optional per-candidate outputs, for inspection and parity testing.  Any
 * pointer may be NULL.  Same memory kind as the other buffers (flags).
 *   margin[s][v][p]   margin (s); -inf if the ball stops short, +inf with
 *                     no opponents
 *   score[s][v][p]    score, -inf when infeasible
 *   T[s][p][k]        min_j t_opp_j at sample k+1 (s), k < K_s; row stride
 *                     T_stride >= max K of the batch; +inf with no
 *                     opponents */
typedef struct pps_debug_out {
    float* margin;
    float* score;
    float* T;
    int32_t T_stride;
    float* point_best; /* [s][p]: best score over the speeds, -inf if no
                          speed is feasible (device memory only) */
} pps_debug_out;

/* Context creation parameters. */
typedef struct pps_ctx_desc {
    int32_t device;          /* CUDA device ordinal */
    void* stream;            /* cudaStream_t to run on; NULL = the legacy
                                default stream */
    size_t mem_budget_bytes; /* cap on the library's own device memory;
                                0 = no cap */
    int32_t max_states;      /* largest n_states per call (> 0) */
    int32_t max_points;      /* largest P per call; 0 = 1<<24 */
    int32_t max_speeds;      /* 0 = PPS_MAX_SPEEDS */
    int32_t max_K;           /* 0 = PPS_MAX_K */
    int32_t max_opp;         /* most opponents any state will have; 1..16,
                                0 = 16.  Sizes the kernel's opponent slots
                                (<= 8 runs the faster 8-slot kernel); a
                                state with more is invalid */
} pps_ctx_desc;

typedef struct pps_ctx pps_ctx;

/* Library ABI version (the PPS_ABI_VERSION it was compiled with). */
int pps_abi_version(void);

/* Human-readable name of a status code (static storage). */
const char* pps_status_string(pps_status s);

/* Last error message of a context ("" if none); valid until the next call
 * on the context.  ctx may be NULL (then: the calling thread's last
 * pps_create or pps_search_noalloc failure). */
const char* pps_last_error(const pps_ctx* ctx);

/* Library defaults: weights 1, margin_cap 1 s, tau_safe 0, robot_radius
 * 0.09 m, reach_radius 0, min_pass_dist 0. */
pps_status pps_default_params(pps_params* out);

/* Grid covering an L x W field at the given spacing with both edges
 * included: x0 = -L/2, y0 = -W/2, nx = round(L/spacing)+1,
 * ny = round(W/spacing)+1 (the paper rasterises at 0.1 m, Sec. 5.1).
 * EINVAL for non-finite or non-positive sizes or more than 2^24 points. */
pps_status pps_grid_from_field(float L, float W, float spacing,
                               pps_grid* out);

/* 32-bit words of feasibility mask per state: n_speeds * ceil(P / 32).
 * Mask layout: mask[s][v][w], bit b of word w is point p = 32 w + b
 * (p = iy * nx + ix); bits at p >= P are zero.  0 on bad arguments. */
size_t pps_mask_words(const pps_grid* grid, int n_speeds);

/* Create a context on desc->device: selects the device, allocates the
 * per-call scratch (max_states entries) and records the stream.
 * EINVAL on a bad descriptor, ENOMEM past the budget or on allocation
 * failure, ECUDA if the device cannot be used.  *out is NULL on error. */
pps_status pps_create(pps_ctx** out, const pps_ctx_desc* desc);

/* Free a context and everything it allocated.  NULL is accepted.  Waits
 * for the context's stream first. */
void pps_destroy(pps_ctx* ctx);

/* The exact search (Sec. 4.2-4.3) over n_states states sharing one grid
 * and one list of kick speeds.
 *   states     [n_states] pps_state
 *   grid       host pointer, always
 *   speeds     host pointer, always: n_speeds kick speeds > 0 (m/s),
 *              1 <= n_speeds <= min(PPS_MAX_SPEEDS, max_speeds)
 *   params     host pointer, always; NULL = pps_default_params
 *   out_best   [n_states] pps_best (required)
 *   out_mask   [n_states * pps_mask_words(grid, n_speeds)] uint32, or NULL
 *              to skip the mask
 *   dbg        host pointer to a pps_debug_out, or NULL
 *   flags      0 or PPS_DEVICE_PTRS
 * Enqueues the work on the context's stream and returns without waiting.
 * Host-memory states are validated before anything is enqueued (EINVAL on
 * n_opp outside 0..max_opp, K outside 1..max_K, a non-finite value, or a
 * non-positive decel, vmax, amax, L or W).  Device-memory states are
 * validated on the device: an invalid one gets idx -2 and
 * PPS_STATE_INVALID, the others are unaffected.  n_states == 0 is a no-op.
 * EINVAL for bad scalar arguments, ENOMEM if staging buffers for host
 * memory exceed the budget, ECUDA on a launch failure. */
pps_status pps_search(pps_ctx* ctx, const pps_state* states, int n_states,
                      const pps_grid* grid, const float* speeds,
                      int n_speeds, const pps_params* params,
                      pps_best* out_best, uint32_t* out_mask,
                      const pps_debug_out* dbg, unsigned flags);

/* Wait for the context's stream.  ECUDA if the device reported an error
 * (the context is then failed until pps_reset). */
pps_status pps_sync(pps_ctx* ctx);

/* Clear a failed context's error state after the caller has dealt with
 * the cause.  ECUDA if the device is still unusable. */
pps_status pps_reset(pps_ctx* ctx);

/* Largest n_states of one pps_search_noalloc call. */
#define PPS_NOALLOC_MAX_STATES 16384

/* The exact search without any device allocation.  The paper has no
 * counterpart: this is a deployment variant of pps_search.
 *
 * Some callers cannot call cudaMalloc: a robot's real-time decision loop
 * that forbids allocation once it is running (cudaMalloc can block and
 * synchronise the device), or a host whose device memory is already handed
 * out by another allocator.  They cannot create a context either, since
 * pps_create allocates the per-call scratch.  This entry point needs no
 * context: the scratch (an argmax key and a feasible count per state) is a
 * fixed array compiled into the library, PPS_NOALLOC_MAX_STATES * 12 bytes
 * (192 KiB), which every GPU that loads the library holds until the process
 * exits.  The call itself allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library routine.
 *
 *   device    CUDA device ordinal; made current by the call
 *   stream    cudaStream_t to run on (NULL = the legacy default stream)
 *   max_opp   1..16: <= 8 runs the 8-slot kernel; states with more
 *             opponents than the kernel's slots are marked invalid
 *   states, out_best, out_mask: DEVICE memory, as pps_search with
 *             PPS_DEVICE_PTRS (out_mask may be NULL); the records and mask
 *             are byte for byte those of pps_search on a context with the
 *             same opponent slots (max_opp <= 8 on both, or > 8 on both)
 *             for states whose K is within that context's max_K (this entry
 *             point accepts K up to PPS_MAX_K)
 *   grid, speeds, params: host memory, as pps_search
 * Returns EINVAL for n_states > PPS_NOALLOC_MAX_STATES or any argument
 * pps_search would reject (message in pps_last_error(NULL)), ECUDA on a
 * device error.  Enqueues the work on `stream` and returns without waiting.
 *
 * The first call on each device resolves the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it, and loads
 * every kernel instance this entry point can launch (8 or 16 opponent slots
 * x 1, 2, 4 or 8 speed slots) so that no later call loads code; make that
 * first call before any stream capture.  Every call on a device shares the
 * one array and clears the slots it uses before the search, so calls that
 * overlap on the GPU (concurrent streams, or several host threads) race on
 * it: order them on one stream or synchronise between them. */
pps_status pps_search_noalloc(int device, void* stream, int max_opp,
                              const pps_state* states, int n_states,
                              const pps_grid* grid, const float* speeds,
                              int n_speeds, const pps_params* params,
                              pps_best* out_best, uint32_t* out_mask);

/* ---- Batched plans: uneven batches, per-state grids and speeds ---------
 *
 * A plan searches n_states states that each have their own receive grid and
 * kick speeds (a field of 12x9 m at 0.025 m next to one of 9x6 m at 0.1 m,
 * one speed next to eight), with the same per-candidate definition as
 * pps_search (Sec. 4.2-4.3).  It is built once from the states' shapes; each
 * pps_plan_run then searches the current contents of a device buffer of
 * states.  The plan groups its states by kernel instance (6/8/12/16 opponent
 * slots, 1/2/4/8 speed slots) and runs each group as one persistent launch
 * whose work items are (state, 32 grid points), so states of very different
 * sizes balance across the GPU. */

/* One state's search shape.  60 bytes, 4-byte aligned. */
typedef struct pps_job {
    pps_grid grid;                 /* this state's receive points */
    int32_t n_speeds;              /* 1..PPS_MAX_SPEEDS */
    float speeds[PPS_MAX_SPEEDS];  /* kick speeds > 0, m/s (first n_speeds) */
    int32_t max_opp;               /* most opponents the state will have,
                                      0..16; picks the 6-, 8-, 12- or
                                      16-slot kernel */
} pps_job;

typedef struct pps_plan pps_plan;

/* pps_plan_create flags. */
#define PPS_PLAN_AUTOTUNE 1u /* time each group's candidate CTA sizes (128,
                                256, 512 threads) on the first run and keep
                                the fastest; choices are cached per device
                                and kernel instance for later plans */
#define PPS_PLAN_GRAPH 2u    /* capture the run's launches in a CUDA graph
                                and replay it while the buffers stay the
                                same (re-captured when they change) */

/* One kernel-instance group of a plan (pps_plan_groups). */
typedef struct pps_plan_group {
    int32_t opp_slots;    /* 6, 8, 12 or 16 */
    int32_t speed_slots;  /* 1, 2, 4 or 8 */
    int32_t n_states;
    int32_t cta_threads;  /* CTA size in use */
    int32_t sample_unroll;  /* samples a register block in use (1 or 2) */
    int32_t reserved;
    int64_t n_items;      /* (state, 32-point) work items */
    float tuned_ms[7];    /* autotuner's time per candidate (CTA threads,
                             samples a block): (128, 1), (256, 1), (512, 1),
                             (768, 1), (1024, 1), (128, 2), (256, 2); 0 when
                             not measured */
} pps_plan_group;

/* Build a plan on ctx for n_states (1..2^24) states shaped by jobs (host
 * memory; copied).  Mask layout: state s owns words
 * [offset[s], offset[s+1]) of out_mask (pps_plan_mask_offsets), speed-major
 * as in pps_search.  EINVAL on a bad job (grid or speeds as pps_search
 * requires, max_opp outside 0..16), ENOMEM past the context's budget. */
pps_status pps_plan_create(pps_ctx* ctx, const pps_job* jobs, int n_states,
                           const pps_params* params, unsigned flags,
                           pps_plan** out);

/* Free a plan (waits for the context's stream first).  NULL is accepted. */
void pps_plan_destroy(pps_plan* plan);

/* Mask word offsets: offsets[0..n_states] (host), offsets[n_states] is the
 * total number of words. */
pps_status pps_plan_mask_offsets(const pps_plan* plan, int64_t* offsets);

/* Search the states in `states` (DEVICE memory, n_states records in job
 * order; a state with more opponents than its job's max_opp is invalid, see
 * pps_best.status).  out_best (n_states records) and out_mask (total words,
 * or NULL) are DEVICE memory.  Enqueued on the context's stream; the first
 * run of an autotuned plan also times the candidates (synchronously). */
pps_status pps_plan_run(pps_plan* plan, const pps_state* states,
                        pps_best* out_best, uint32_t* out_mask);

/* The plan's groups: up to cap entries into out, the count into *n.  The
 * autotuner (PPS_PLAN_AUTOTUNE) picks each group's CTA size and samples a
 * register block (the unroll of the sample loop; results are the same bit
 * for bit either way) from the candidates tuned_ms lists. */
pps_status pps_plan_groups(const pps_plan* plan, pps_plan_group* out, int cap,
                           int* n);

/* ---- Serving: continuous batching of per-frame searches ----------------
 *
 * A server takes single-state requests (one vision frame of one match each,
 * any grid and speeds) from any thread and answers each with its pps_best
 * (and optionally its mask).  A scheduler thread forms batches
 * continuously: whenever one of the server's streams is free it launches
 * every queued request that fits -- at most max_batch, and only while the
 * device memory pool has room for the request's mask -- so requests that
 * arrive while others are on the GPU join the next launch, and launches on
 * different streams overlap on the device.  While a launch is in flight a
 * new one waits up to max_wait_us to gather more requests (one launch per
 * request would spend the host's time on launch overhead).  Results are those of pps_search
 * for the same state and shape, alone or in any mix. */

typedef struct pps_server pps_server;

/* Serving modes (pps_server_desc.mode). */
#define PPS_SERVE_EXACT 0    /* every frame on its full grid (pps_search) */
#define PPS_SERVE_PROPOSAL 1 /* every frame through the learned proposal
                                (pps_propose_jobs with the fallback): the
                                network ranks the map cells, the exact search
                                refines the topk best and searches the full
                                grid of a frame whose cells hold no feasible
                                pass; best records only (no masks) */

typedef struct pps_server_desc {
    int32_t device;
    int32_t n_streams;        /* batches in flight at once, 1..8 */
    int32_t max_batch;        /* requests per launch, 1..4096 */
    int32_t max_queue;        /* pending requests before submit refuses
                                 (PPS_ENOMEM), >= max_batch */
    size_t pool_bytes;        /* device memory for masks of in-flight
                                 requests (admission budget); 0 = masks off
                                 (and always off in the proposal mode) */
    int32_t max_opp;          /* most opponents of any request (<= 16) */
    int32_t max_wait_us;      /* with a launch already in flight, gather
                                 queued requests for up to this long before
                                 launching them (0 = launch at once) */
    pps_params params;        /* value-function parameters of every search */
    int32_t mode;             /* PPS_SERVE_EXACT or PPS_SERVE_PROPOSAL */
    int32_t topk;             /* proposal: map cells refined per frame,
                                 1..2806 */
    const float* net_weights; /* proposal: PPS_NET_PARAMS floats (host,
                                 copied at creation; one network per stream,
                                 its activations sized for max_batch frames);
                                 every request's grid must then lie on the
                                 map's cell lattice (see pps_propose_jobs) */
} pps_server_desc;

/* Per-request completion record. */
typedef struct pps_server_result {
    pps_best best;
    uint64_t ticket;
    int64_t latency_ns;       /* submit -> result available on the host */
    int64_t queue_ns;         /* submit -> its launch was enqueued */
    int32_t batch_size;       /* requests in the launch that served it */
    int32_t status;           /* PPS_OK, or why the request failed */
} pps_server_result;

/* Latency and throughput summary over the requests completed so far. */
typedef struct pps_server_stats {
    int64_t completed;
    int64_t batches;
    double mean_batch;
    double p50_us, p99_us, max_us, mean_us;
    double wall_s;            /* first submit -> last completion */
    double states_per_s;
} pps_server_stats;

/* Start a server (allocates its pools and streams, starts the scheduler
 * thread).  EINVAL on a bad descriptor, ENOMEM, ECUDA. */
pps_status pps_server_create(const pps_server_desc* desc, pps_server** out);

/* Stop the scheduler (after finishing in-flight work) and free everything.
 * NULL is accepted. */
void pps_server_destroy(pps_server* srv);

/* Queue one request: state and job in host memory (copied).  *ticket gets
 * its id.  EINVAL on a bad state or job, ENOMEM when max_queue requests are
 * pending or the request's mask can never fit the pool. */
pps_status pps_server_submit(pps_server* srv, const pps_state* state,
                             const pps_job* job, uint64_t* ticket);

/* Wait up to timeout_us (< 0: forever) for a ticket's result; ETIMEOUT if
 * it is not done.  If mask is not NULL and masks are on, the request's mask
 * words (job.n_speeds * ceil(P/32)) are copied there.  A result can be
 * taken once. */
pps_status pps_server_wait(pps_server* srv, uint64_t ticket,
                           int64_t timeout_us, pps_server_result* out,
                           uint32_t* mask);

/* Replay n_matches simulated matches of frames_per_match frames each at
 * `hz` frames per second per match (match m's frames at
 * t0 + (m / n_matches + f) / hz): frames[m * frames_per_match + f] with
 * jobs[m] (all host memory), submitted on schedule by one thread while the
 * scheduler serves them.  Results (n_matches * frames_per_match records,
 * host, may be NULL) and a summary of this replay. */
pps_status pps_server_replay(pps_server* srv, const pps_state* frames,
                             const pps_job* jobs, int n_matches,
                             int frames_per_match, double hz,
                             pps_server_result* results,
                             pps_server_stats* stats);

/* Summary over everything completed since the server started. */
pps_status pps_server_get_stats(pps_server* srv, pps_server_stats* out);

/* ---- Learned proposal -------------------------------------------------
 *
 * Not in the paper: a small network ranks coarse cells of the field so that
 * the exact search (Sec. 4.2-4.3) only has to run on the best of them.  The
 * network reads a 46 x 61 map of a 12 x 9 m field (0.2 m pixels, pixel
 * (y, x) centred at ((x - 30) / 5, (y - 22.5) / 5)) with 8 channels
 * rasterised from the state; c is the pixel centre, q the cell's four
 * sub-points c + (+-0.05, +-0.05) m (clamped into the field):
 *   0  opponent density at c, sum_j exp(-|c - o_j|^2 / (2 * 0.3^2))
 *   1  coarse score of the cell: the largest over q of the value function
 *      (Sec. 4.3) with the margin below, -1.2 where no speed is feasible
 *   2  |c - b| / diag
 *   3  margin of the cell: the largest over q and the feature kick speeds
 *      of the pass's safety margin (Sec. 4.2) with 16 pass-line samples,
 *      clamped to [-2, 1] (ball stopping short: -2; no opponents: 1)
 *   4  largest open shot angle over q (Sec. 4.3) / pi
 *   5  |goal centre - c| / diag
 *   6  c_x / (L / 2),  7  c_y / (W / 2)
 * and predicts, per pixel, the best exact score among the fine grid
 * points of that pixel's cell, as channel 1 plus a learned correction:
 * 4 layers of 3x3 convolutions
 * (8 -> 32 -> 32 -> 32 -> 1, ReLU between), bfloat16 weights and
 * activations with float32 accumulation, all on the tensor cores (tcgen05),
 * trained on the GPU with the library's own forward and backward kernels
 * (Adam). */

#define PPS_NET_H 46
#define PPS_NET_W 61
#define PPS_NET_PARAMS 21121 /* per layer W[3][3][cout][cin] then bias */

typedef struct pps_net pps_net;

/* A network on `device` for batches of up to max_batch states, with zero
 * weights (load them with pps_net_set_weights). */
pps_status pps_net_create(int device, void* stream, int max_batch,
                          pps_net** out);
void pps_net_destroy(pps_net* net);

/* Kick speeds (host, 1..8, each > 0) and value-function parameters (host,
 * NULL = pps_default_params) that channels 1, 3 and 4 of the input map are
 * computed for.  A new network uses speeds {2, 3.5, 5, 6.5} m/s and the
 * default parameters.  EINVAL on a bad speed or a non-finite parameter. */
pps_status pps_net_set_features(pps_net* net, const float* speeds,
                                int n_speeds, const pps_params* params);

/* The training loss of pps_net_grad and pps_net_train_step: the mean over
 * all map pixels of w (prediction - label)^2, where w = 1 for a pixel whose
 * label or prediction comes within top_band of its state's best label and
 * w = low_weight elsewhere, times under_weight where the prediction is
 * below the label (the weight is held constant in the gradient).  The
 * proposal only needs the best cells ranked high enough to be refined:
 * the band focuses the fit on them, and under_weight > 1 makes the
 * prediction err on the high side where a cell may or may not hold a
 * feasible pass.  A new network has top_band = +inf, low_weight = 1,
 * under_weight = 1 (plain mean squared error).  EINVAL unless top_band > 0,
 * 0 <= low_weight <= 1 and 1 <= under_weight <= 1000. */
pps_status pps_net_set_loss(pps_net* net, float top_band, float low_weight,
                            float under_weight);

/* Waits for the network's stream.  PPS_ETIMEOUT when a bounded wait of the
 * tensor-core inference kernel ran out since the last call (the outputs of
 * that pass are invalid; the flag is cleared). */
pps_status pps_net_sync(pps_net* net);

/* Self-test of those bounded waits: runs the inference kernel on n states
 * (device) with its tensor-core work withheld, so that no mbarrier ever
 * completes and every wait runs out after a short limit; the kernel then
 * releases its tensor memory and returns.  Returns what pps_net_sync then
 * reports -- PPS_ETIMEOUT when the timeout path works.  The output map of
 * that pass is garbage; the network stays usable. */
pps_status pps_net_selftest_timeout(pps_net* net, const pps_state* states,
                                    int n);

/* Weights as PPS_NET_PARAMS floats (host).  Setting them resets Adam. */
pps_status pps_net_set_weights(pps_net* net, const float* w);
pps_status pps_net_get_weights(pps_net* net, float* w);

/* The input map: out[n][46][61][8] bfloat16 bit patterns (device, 16-byte
 * aligned). */
pps_status pps_net_raster(pps_net* net, const pps_state* states, int n,
                          uint16_t* out);

/* Predicted cell scores, out[n][46][61] float (device).  States (device)
 * must be 12 x 9 m; n <= max_batch.  The four convolutions run in one
 * tcgen05 kernel (activations stay on the SM); enqueued on the network's
 * stream. */
pps_status pps_net_forward(pps_net* net, const pps_state* states, int n,
                           float* out);

/* The same prediction computed layer by layer on mma.sync (every activation
 * written to device memory), the forward pass of the PPS_NET_TRAIN_MMA_SYNC
 * training kernels.  It differs from pps_net_forward only by FP32 summation
 * order (and the bfloat16 roundings that order can flip). */
pps_status pps_net_forward_layers(pps_net* net, const pps_state* states,
                                  int n, float* out);

/* The prediction from a given input map instead of states: map[n][46][61][8]
 * bfloat16 bit patterns (device, 16-byte aligned; the layout pps_net_raster
 * writes).
 * layers = 0 runs the tcgen05 pass of pps_net_forward, layers != 0 the
 * layer-by-layer pass of pps_net_forward_layers.  For training or checking
 * the network on maps computed elsewhere. */
pps_status pps_net_forward_map(pps_net* net, const uint16_t* map, int n,
                               int layers, float* out);

/* The loss (pps_net_set_loss) of the prediction against labels[n][46][61]
 * (device) and its gradient with respect to the weights (grads:
 * PPS_NET_PARAMS floats, host, or NULL).  Waits for the result. */
pps_status pps_net_grad(pps_net* net, const pps_state* states,
                        const float* labels, int n, float* grads,
                        float* loss);

/* pps_net_grad from a given input map (device, as pps_net_forward_map). */
pps_status pps_net_grad_map(pps_net* net, const uint16_t* map,
                            const float* labels, int n, float* grads,
                            float* loss);

/* The kernels pps_net_grad and pps_net_train_step run on.
 *   PPS_NET_TRAIN_TCGEN05 (the default): the forward pass is the fused
 *     tcgen05 kernel of pps_net_forward, writing the hidden activations; the
 *     input gradients are tcgen05 convolutions; the weight and bias
 *     gradients a tcgen05 product over the batch's pixels, summed per CTA
 *     and then over the CTAs in a fixed order (the same gradient every run).
 *   PPS_NET_TRAIN_MMA_SYNC: the layer-by-layer mma.sync kernels (forward,
 *     input gradients, weight gradients with atomic sums).
 * EINVAL for another kind. */
#define PPS_NET_TRAIN_TCGEN05 0
#define PPS_NET_TRAIN_MMA_SYNC 1
pps_status pps_net_set_train_kernels(pps_net* net, int kind);

/* One Adam step (lr, beta 0.9/0.999) on a batch; *loss (host, may be NULL:
 * then the call does not wait) gets the batch's loss before the step. */
pps_status pps_net_train_step(pps_net* net, const pps_state* states,
                              const float* labels, int n, float lr,
                              float* loss);

/* Training labels from an exact search on the fine grid of the map (12 x 9 m
 * at 0.025 m: 481 x 361 points, 8 x 8 fine points per map pixel, centred on
 * it): point_best[n][361 * 481] (device; pps_debug_out.point_best) ->
 * labels[n][46][61] = max(cell maximum, floor). */
pps_status pps_net_labels(pps_net* net, const float* point_best, int n,
                          float floor_value, float* labels);

/* pps_net_labels for any fine grid on the map's cell lattice: the grid of
 * a field of at most 12 x 9 m centred on the origin (pps_grid_from_field)
 * at a spacing of 0.2 / m m, m = 1, 2, 4 or 8; pixel (cx, cy) then holds
 * the m x m fine points nearest its centre (-6 + 0.2 cx, -4.5 + 0.2 cy)
 * and a pixel without points gets floor_value.  EINVAL for another grid. */
pps_status pps_net_labels_grid(pps_net* net, const float* point_best, int n,
                               const pps_grid* fine, float floor_value,
                               float* labels);

/* pps_propose flags. */
#define PPS_PROPOSE_FALLBACK 1u /* states whose top-k cells hold no feasible
                                   pass are searched on the full grid */
#define PPS_PROPOSE_NO_PRUNE 2u /* evaluate every point of the top-k cells
                                   (n_feasible then counts them all) */

/* The proposal path: rasterise, predict, take each state's topk best map
 * pixels, and run the exact search only on their cells' fine grid points
 * (fine_grid must be the 481 x 361 grid of the 12 x 9 m field at 0.025 m).
 * states, out_best and out_cells (n x topk pixel indices y * 61 + x, or
 * NULL) are device memory; 1 <= topk <= 2806; n <= both the context's
 * max_states and the network's max_batch.  The network's input features
 * use its own speeds and parameters (pps_net_set_features); the exact
 * refinement uses speeds and params of this call.  Refinement items run
 * every state's best-ranked cells first.  Unless PPS_PROPOSE_NO_PRUNE is
 * set, and when w_angle >= 0 and w_margin >= 0, a half cell is skipped
 * when its score bound is below the state's best so far: the bound takes
 * the whole goal mouth's angle for the shot angle and the last pass-line
 * sample's term alone for each speed's margin.  Such a cell cannot hold
 * the best, so the result is the exact best over the top-k cells either
 * way.  out_best.n_feasible counts the feasible candidates
 * among the points evaluated (it depends on what was skipped; the whole
 * grid's count for a state that fell back).  The prediction runs on the
 * network's stream and the refinement on the context's (ordered by an
 * event); the call returns without waiting.  One network serves one
 * pps_propose at a time (it holds the call's scratch). */
pps_status pps_propose(pps_ctx* ctx, pps_net* net, const pps_state* states,
                       int n, const pps_grid* fine_grid, const float* speeds,
                       int n_speeds, const pps_params* params, int topk,
                       unsigned flags, pps_best* out_best, int32_t* out_cells);

/* The proposal path for states that each have their own field and grid:
 * jobs[i] (device, one pps_job per state) gives state i's receive grid and
 * kick speeds.  Every grid must have the same spacing `spacing` = 0.2 / m
 * (0.2, 0.1, 0.05 or 0.025 m) and lie on the map's cell lattice (the grid
 * pps_grid_from_field gives for a field of at most 12 x 9 m), so that map
 * pixel (cx, cy) holds its m x m nearest points; a state whose job does not
 * (another spacing, more than max_speeds speeds) gets PPS_STATE_INVALID.
 * The map of a smaller field is the same 46 x 61 map (the field in its
 * middle); pixels whose cell holds no point of the grid rank last in the
 * top-k.  The exact refinement runs on the topk cells' points with the
 * job's speeds; PPS_PROPOSE_FALLBACK searches a state whose cells hold no
 * feasible pass on its full grid.  Opponent slots follow the context's
 * max_opp (8, 12 or 16).  states, jobs, out_best and out_cells (n x topk,
 * or NULL) are device memory; limits, streams and pruning as pps_propose. */
pps_status pps_propose_jobs(pps_ctx* ctx, pps_net* net,
                            const pps_state* states, const pps_job* jobs,
                            int n, float spacing, int max_speeds,
                            const pps_params* params, int topk, unsigned flags,
                            pps_best* out_best, int32_t* out_cells);

/* Number of SMs and the CTAs per SM the search kernel runs with (for
 * benchmarks and the autotuner); EINVAL on NULL. */
pps_status pps_launch_info(const pps_ctx* ctx, int* num_sms,
                           int* ctas_per_sm);

/* ---- Directions x kick powers: the paper's own search (Sec. 4.2) -------
 *
 * From the ball holder, candidate passes are n_dir directions
 * (phi_i = 2 pi i / n_dir) x n_pow kick powers (v0_j uniform in
 * [v_lo, v_hi]; the paper: 128 x 64 over 1..6.5 m/s).  The ball rolls from
 * v = slide * v0 (Sec. 4.1: the kick speed drops to 5/7 in a short slide
 * whose distance is neglected) with the state's deceleration, until it
 * stops or reaches the field edge.  For every candidate the path is
 * searched, K samples uniform in distance, for the first sample a teammate
 * (receiver) can reach no later than the ball (SBIP, with the bang-bang
 * robot model of pps_search), and likewise for the opponents; at the stop
 * sample of a path that ends by stopping every robot gets the ball, at
 * max(its arrival, the stop time).  A candidate is feasible when a
 * teammate gets the ball and the first opponent comes more than tau_delta
 * later (the delta-time of Sec. 4.3).  Its score (Sec. 4.3 features):
 *   - w_time * t_team + w_angle * shot angle at the receive point / pi
 *   - w_dist * |goal - receive point| / diag
 *   - w_refr * refraction angle / pi   (the turn from the pass direction to
 *                                       the shot direction)
 *   + w_delta * min(t_opp - t_team, delta_cap).
 * The best candidate is the highest score; equal scores go to the smaller
 * idx = dir * n_pow + pow. */

#define PPS_MAX_TEAM 16

typedef struct pps_dstate {
    float ball[2];                   /* the ball, at the passer's feet (m) */
    int32_t n_team;                  /* receivers, 0..PPS_MAX_TEAM */
    int32_t n_opp;                   /* opponents, 0..PPS_MAX_OPP */
    float team_pos[PPS_MAX_TEAM][2]; /* receivers (the passer excluded) */
    float team_vel[PPS_MAX_TEAM][2];
    float opp_pos[PPS_MAX_OPP][2];
    float opp_vel[PPS_MAX_OPP][2];
    float ball_decel;                /* rolling deceleration (m/s^2) */
    float vmax, amax;                /* robot limits (both teams) */
    float field_len, field_wid, goal_width;
    int32_t K;                       /* samples per ball path, 1..PPS_MAX_K */
} pps_dstate;

typedef struct pps_dparams {
    int32_t n_dir, n_pow;  /* 1..1024 directions, 1..256 powers */
    float v_lo, v_hi;      /* kick power range (m/s), 0 < v_lo <= v_hi */
    float slide;           /* rolling speed / kick speed, in (0, 1] */
    float tau_delta;       /* delta-time threshold (s) */
    float delta_cap;       /* cap of the delta-time feature (s) */
    float w_time, w_angle, w_dist, w_refr, w_delta;
    float robot_radius;    /* disc radius for shot blocking (m) */
    float reach_radius;    /* intercept reach radius (m) */
} pps_dparams;

typedef struct pps_dbest {
    int32_t idx;           /* dir * n_pow + pow; -1: none feasible; -2:
                              invalid state */
    int32_t dir, pow;      /* -1 when idx < 0 */
    int32_t receiver;      /* index into team_pos of the first teammate */
    float score;           /* -inf when idx < 0 */
    float t_team, t_opp;   /* first teammate / opponent ball time (s);
                              t_opp = +inf when no opponent gets the ball */
    float recv[2];         /* receive point (m) */
    int32_t n_feasible;
    int32_t status;        /* PPS_STATE_* flags as in pps_best */
    int32_t reserved;
} pps_dbest;

/* Defaults: 128 x 64 over 1..6.5 m/s, slide 5/7, tau_delta 0, delta_cap
 * 1 s, all weights 1, robot radius 0.09 m, reach 0. */
pps_status pps_dpps_default_params(pps_dparams* out);

/* Mask words per state: ceil(n_dir * n_pow / 32); bit b of word w is the
 * candidate 32 w + b in idx order. */
size_t pps_dpps_mask_words(const pps_dparams* params);

/* The search over n_states states (n_states <= the context's max_states).
 * states, out_best (n_states records), out_mask (n_states x
 * pps_dpps_mask_words, or NULL) and out_dbg (NULL, or n_states x n_dir x
 * n_pow x 3 floats: t_team, t_opp, score of every candidate, for tests)
 * are device memory.  Enqueued on the context's stream.  EINVAL on bad
 * parameters; a state whose n_team or n_opp exceeds the context's max_opp,
 * or with values out of range, gets idx -2 and PPS_STATE_INVALID. */
pps_status pps_dpps_search(pps_ctx* ctx, const pps_dstate* states,
                           int n_states, const pps_dparams* params,
                           pps_dbest* out_best, uint32_t* out_mask,
                           float* out_dbg);

/* ---- Passing power and shooting decisions (Sec. 4.1, Sec. 4.4) --------- */

/* One passing-power query: receiver `receiver` (an index into team_pos) of
 * states[state] is to receive the ball at `target`. */
typedef struct pps_pass_query {
    int32_t state;
    int32_t receiver;
    float target[2];
} pps_pass_query;

typedef struct pps_pass_power {
    float v0;        /* kick power (m/s), within [v_lo, v_hi] */
    float v1;        /* rolling speed after the slide */
    float t_pass;    /* the ball's travel time: t_recv + buffer */
    float t_recv;    /* the receiver's arrival at the target (s) */
    int32_t clamped; /* 1 when v0 was limited to [v_lo, v_hi] */
    int32_t status;  /* PPS_STATE_OK, or PPS_STATE_INVALID (bad query or
                        state: the other fields are NaN) */
} pps_pass_power;

/* Sec. 4.1, Eq. 1-2: the pass takes the receiver's arrival time at the
 * target (bang-bang model) plus `buffer` seconds (the paper: 0.3); the
 * rolling speed covers the distance in that time (d = v1 t - a t^2 / 2,
 * the reading of the garbled Eq. 1; at least sqrt(2 a d), the slowest ball
 * that still reaches the target) and the kick power is v1 / slide (Eq. 2),
 * limited to [v_lo, v_hi].  params: slide, v_lo, v_hi, reach_radius
 * (NULL = pps_dpps_default_params).  states, queries and out are device
 * memory; enqueued on the context's stream. */
pps_status pps_pass_powers(pps_ctx* ctx, const pps_dstate* states,
                           int n_states, const pps_pass_query* queries,
                           int n_queries, float buffer,
                           const pps_dparams* params, pps_pass_power* out);

/* One shooting query: a shooter of states[state] at `from`. */
typedef struct pps_shot_query {
    int32_t state;
    float from[2];
} pps_shot_query;

typedef struct pps_shot {
    float theta;     /* the open shot angle (rad) */
    float dir;       /* shot direction: the middle of the largest gap */
    float t_line;    /* the ball's time to the goal line (+inf: stops short) */
    float t_opp;     /* first opponent interception on the way (+inf: none) */
    int32_t shoot;   /* 1: shoot */
    int32_t status;  /* PPS_STATE_OK or PPS_STATE_INVALID */
} pps_shot;

/* Sec. 4.4: shoot when the open angle is at least theta_min and the ball,
 * kicked at v_shot toward the middle of the largest open gap (rolling from
 * slide * v_shot), reaches the goal line with no opponent getting it first
 * (by more than tau_delta; opponents searched along the shot with the
 * state's K samples).  params: slide, tau_delta, robot_radius,
 * reach_radius.  Device memory; enqueued on the context's stream. */
pps_status pps_shoot(pps_ctx* ctx, const pps_dstate* states, int n_states,
                     const pps_shot_query* queries, int n_queries,
                     float v_shot, float theta_min, const pps_dparams* params,
                     pps_shot* out);

/* ---- Running points (Sec. 5.1-5.2) ----------------------------------------
 *
 * The attacking half of each state's field (the goal at x = +L/2) is
 * rasterised at `spacing` g: x = min(i g, L/2), i = 0..nx-1,
 * nx = round(L/2/g) + 1; y = min(-W/2 + j g, W/2), j = 0..ny-1,
 * ny = round(W/g) + 1 (rounding to nearest, ties to even, in float), so
 * the last column lies on the goal line and the last row on the touch
 * line.  Four zones (Sec. 5.1): I and II behind
 * x = L/4, III and IV in front of it, each pair split at the ball's y kept
 * within +-W/4 (I and III below the cut, II and IV on or above it; both
 * cuts inclusive upward), so the zones move with the ball.  Points inside
 * the opponent's defence area (x > L/2 - def_depth, |y| < def_width/2) are
 * no candidates.  A point within g / 1024 of a cut or of the area's edge
 * counts as on it (so grid lines that fall on them do not depend on the
 * rounding of i g).  Every other point p gets the weighted sum of Eq. 4 over
 * the five criteria of Sec. 5.2:
 *   - w_goal  * |goal - p| / sqrt(L^2 + W^2)           (closer is better)
 *   + w_ball  * min(|p - ball|, ball_ref) / ball_ref   (not too close)
 *   + w_angle * a(alpha)   alpha = |angle of goal - p off the x axis|;
 *                          a = 1 in [angle_lo, angle_hi], falling linearly
 *                          to 0 over angle_span on either side
 *   + w_guard * (T_P + T_Q) / (2 guard_cap)
 *                          P, Q: where the lines from p to the two goal
 *                          posts enter the defence area; T: the fastest
 *                          guard's arrival (guards: the opponents inside
 *                          the area; the bang-bang intercept time of the
 *                          pass search, reach 0), capped at guard_cap, and
 *                          guard_cap when no guard or no entry
 *   - w_avoid * [some opponent is nearer the ball than p]
 * The best point of each zone (the lowest j * nx + i on ties) is the
 * zone's running point.  Then the zones are chosen for n_run supporters:
 * zones without a candidate and the zone holding the best passing point
 * are left out; III and IV come before I and II, each pair by score (the
 * lower zone first on ties). */
typedef struct pps_rparams {
    float spacing;                          /* grid spacing g (m), > 0 */
    float w_goal, w_ball, w_angle, w_guard, w_avoid;  /* Eq. 4 weights */
    float ball_ref;                         /* m, > 0 */
    float angle_lo, angle_hi, angle_span;   /* rad: 0 <= lo <= hi, span > 0 */
    float def_depth, def_width;             /* defence area (m), > 0 */
    float guard_cap;                        /* s, > 0 */
    int32_t n_run;                          /* supporters, 0..4 */
} pps_rparams;

typedef struct pps_rbest {
    int32_t idx[4];       /* zones I..IV: grid index j * nx + i of the best
                             point; -1: no candidate in the zone */
    float score[4];       /* -inf when idx < 0 */
    float point[4][2];    /* (x, y) of the point (m); NaN when idx < 0 */
    int32_t chosen[4];    /* zones (0..3 = I..IV) for the supporters, in
                             order; -1 after the last */
    int32_t avoided;      /* zone of the best passing point; -1: none */
    int32_t nx, ny;       /* the state's grid */
    int32_t status;       /* PPS_STATE_OK or PPS_STATE_INVALID */
} pps_rbest;

/* Defaults: g = 0.1 m, weights 1, ball_ref 2 m, angles 0.25..0.75 rad with
 * span 0.5 rad, defence area 1.2 m x 2.4 m, guard_cap 2 s, n_run 4. */
pps_status pps_run_default_params(pps_rparams* out);

/* The grid of a field at spacing g, as the kernel forms it; PPS_EINVAL
 * for non-positive or non-finite sizes or a side above 32768 points. */
pps_status pps_run_grid(float field_len, float field_wid, float spacing,
                        int* nx, int* ny);

/* Running points of n_states states (their ball and opponents; receivers
 * and K unused).  pass: NULL, or n_states records of pps_dpps_search over
 * the same states, whose receive point (idx >= 0) names the zone to avoid.
 * out: n_states records.  out_scores: NULL, or n_states x score_stride
 * floats; state s writes its nx * ny scores (row j, column i at
 * s * score_stride + j * nx + i; -inf inside the defence area).  A state
 * that fails validation (non-finite ball or robot, non-positive field or
 * robot limits, n_opp outside 0..PPS_MAX_OPP, a grid side above 32768, or
 * nx * ny above score_stride when out_scores is given) gets
 * PPS_STATE_INVALID and idx -1.  Device memory, enqueued on the context's
 * stream; PPS_EINVAL for a NULL buffer, n_states < 0 or out-of-range
 * parameters. */
pps_status pps_run_points(pps_ctx* ctx, const pps_dstate* states,
                          int n_states, const pps_rparams* params,
                          const pps_dbest* pass, pps_rbest* out,
                          float* out_scores, size_t score_stride);

#ifdef __cplusplus
}
#endif
#endif /* PPS_H */

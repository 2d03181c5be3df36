// pps_server.cu -- continuous batching of per-frame searches (include/pps.h,
// "Serving").
//
// Requests (one state + its shape each) enter a FIFO queue from any thread.
// One scheduler thread owns every CUDA call of the server.  It keeps
// n_streams launch slots; whenever a slot is free and requests are queued it
// takes requests in order while the slot's batch has room (max_batch
// requests, and mask words within the slot's share of the device memory
// pool -- the admission budget), copies them in, launches the batched-plan
// kernels for the batch's kernel-instance groups, copies the results back
// and records an event.  Slots run on their own streams, so a batch launched
// while another is still on the GPU overlaps with it.  The scheduler polls
// the events, hands each finished request its result and latency, and frees
// the slot.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pps.h"
#include "pps_batch.cuh"
#include "pps_cells.cuh"
#include "pps_internal.h"

char* pps_thread_error_buffer();

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

int opp_slots(int m) { return m <= 6 ? 6 : m <= 8 ? 8 : m <= 12 ? 12 : 16; }
int speed_slots(int n) { return n <= 1 ? 1 : n <= 2 ? 2 : n <= 4 ? 4 : 8; }
// (opponent slots, speed slots) pairs: at most this many groups a launch
constexpr int kMaxGroups = 16;

struct Request {
    uint64_t ticket = 0;
    pps_state st;
    pps_job job;
    int64_t t_submit = 0;
    long long words = 0;  // mask words of this request
    long long items = 0;  // 32-point work items
};

struct Done {
    pps_server_result r;
    std::vector<uint32_t> mask;
};

// One launch slot: a stream, an event and the buffers of one batch.
struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    // One packed input buffer (states, jobs, group tables), copied in with
    // a single transfer; its sections are laid out per batch.
    unsigned char* d_in = nullptr;
    unsigned char* h_in = nullptr;
    size_t in_bytes = 0;
    pps_best* d_best = nullptr;
    pps_best* h_best = nullptr;
    unsigned long long* d_keys = nullptr;  // cleared by the finalize kernels
    int* d_counts = nullptr;
    unsigned long long* d_next = nullptr;  // a work-queue counter per group,
                                           // left 0 by the finalize kernels
    uint32_t* d_mask = nullptr;
    uint32_t* h_mask = nullptr;
    pps_net* net = nullptr;  // proposal mode: this slot's network
    // this batch's sections in the packed buffer
    size_t o_states = 0, o_jobs = 0, o_bucket = 0, o_start = 0, o_moff = 0;
    bool busy = false;
    int64_t t_launch = 0;
    std::vector<Request> reqs;
};

}  // namespace

struct pps_server {
    pps_server_desc d{};
    int num_sms = 0;
    long long mask_words_per_slot = 0;
    std::vector<Slot> slots;
    std::thread worker;
    std::atomic<bool> stop{false};
    std::mutex mu;                 // queue, done map, stats
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, Done> done;
    uint64_t next_ticket = 1;
    std::vector<int64_t> lat_ns;   // all completed latencies
    std::vector<int> batch_sizes;
    int64_t t_first = 0, t_last = 0;
    cudaError_t fatal = cudaSuccess;
};

namespace {

pps_status fail(pps_status s, const char* msg, cudaError_t e = cudaSuccess) {
    std::snprintf(pps_thread_error_buffer(), 512, "%s%s%s", msg,
                  e != cudaSuccess ? ": " : "",
                  e != cudaSuccess ? cudaGetErrorString(e) : "");
    return s;
}

void free_slot(Slot& s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    for (void* p : {(void*)s.d_in, (void*)s.d_best, (void*)s.d_keys,
                    (void*)s.d_counts, (void*)s.d_next, (void*)s.d_mask})
        if (p) cudaFree(p);
    for (void* p : {(void*)s.h_in, (void*)s.h_best, (void*)s.h_mask})
        if (p) cudaFreeHost(p);
    if (s.net) pps_net_destroy(s.net);
    if (s.done) cudaEventDestroy(s.done);
    if (s.stream) cudaStreamDestroy(s.stream);
    s = Slot();
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Sections of a packed input buffer for n requests: states, jobs, bucket
// list, item starts (n + one per group, at most 16 groups), mask offsets.
size_t layout(int n, size_t* st, size_t* jb, size_t* bk, size_t* sa,
              size_t* mo) {
    size_t o = 0;
    *st = o;
    o = align256(o + sizeof(pps_state) * n);
    *jb = o;
    o = align256(o + sizeof(pps_job) * n);
    *bk = o;
    o = align256(o + sizeof(int) * n);
    *sa = o;
    o = align256(o + sizeof(long long) * (n + 16));
    *mo = o;
    o = align256(o + sizeof(long long) * (n + 1));
    return o;
}

size_t packed_bytes(int n) {
    size_t a, b, c, d, e;
    return layout(n, &a, &b, &c, &d, &e);
}

template <typename T>
cudaError_t both(T** d, T** h, size_t n) {
    cudaError_t e = cudaMalloc((void**)d, sizeof(T) * n);
    if (e == cudaSuccess) e = cudaMallocHost((void**)h, sizeof(T) * n);
    return e;
}

cudaError_t alloc_slot(Slot& s, int max_batch, long long mask_words) {
    cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
    const size_t n = (size_t)max_batch;
    s.in_bytes = packed_bytes(max_batch);
    if (e == cudaSuccess) e = both(&s.d_in, &s.h_in, s.in_bytes);
    if (e == cudaSuccess) e = both(&s.d_best, &s.h_best, n);
    if (e == cudaSuccess)
        e = cudaMalloc((void**)&s.d_keys, sizeof(unsigned long long) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s.d_counts, sizeof(int) * n);
    if (e == cudaSuccess)
        e = cudaMemset(s.d_keys, 0, sizeof(unsigned long long) * n);
    if (e == cudaSuccess) e = cudaMemset(s.d_counts, 0, sizeof(int) * n);
    if (e == cudaSuccess)
        e = cudaMalloc((void**)&s.d_next, sizeof(unsigned long long) * kMaxGroups);
    if (e == cudaSuccess)
        e = cudaMemset(s.d_next, 0, sizeof(unsigned long long) * kMaxGroups);
    if (e == cudaSuccess && mask_words > 0)
        e = both(&s.d_mask, &s.h_mask, (size_t)mask_words);
    return e;
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.f; }

bool job_ok(const pps_job& j, int max_opp) {
    const pps_grid& g = j.grid;
    if (!finite_pos(g.spacing) || g.nx < 1 || g.ny < 1 || !std::isfinite(g.x0) ||
        !std::isfinite(g.y0) || (long long)g.nx * g.ny > (1 << 24))
        return false;
    if (j.n_speeds < 1 || j.n_speeds > PPS_MAX_SPEEDS) return false;
    for (int v = 0; v < j.n_speeds; ++v)
        if (!finite_pos(j.speeds[v])) return false;
    return j.max_opp >= 0 && j.max_opp <= max_opp;
}

bool state_ok(const pps_state& s, const pps_job& j) {
    if (s.n_opp < 0 || s.n_opp > j.max_opp || s.K < 1 || s.K > PPS_MAX_K)
        return false;
    if (!finite_pos(s.ball_decel) || !finite_pos(s.vmax) ||
        !finite_pos(s.amax) || !finite_pos(s.field_len) ||
        !finite_pos(s.field_wid) || !std::isfinite(s.goal_width) ||
        s.goal_width < 0.f || !std::isfinite(s.ball[0]) ||
        !std::isfinite(s.ball[1]))
        return false;
    for (int k = 0; k < s.n_opp; ++k)
        if (!std::isfinite(s.opp_pos[k][0]) || !std::isfinite(s.opp_pos[k][1]) ||
            !std::isfinite(s.opp_vel[k][0]) || !std::isfinite(s.opp_vel[k][1]))
            return false;
    return true;
}

void worker_main(pps_server* srv);

}  // namespace

extern "C" pps_status pps_server_create(const pps_server_desc* desc,
                                        pps_server** out) {
    if (!out) return PPS_EINVAL;
    *out = nullptr;
    if (!desc || desc->n_streams < 1 || desc->n_streams > 8 ||
        desc->max_batch < 1 || desc->max_batch > 4096 ||
        desc->max_queue < desc->max_batch || desc->max_opp < 0 ||
        desc->max_opp > PPS_MAX_OPP)
        return fail(PPS_EINVAL, "pps_server_create: descriptor out of range");
    const pps_params& p = desc->params;
    const float pv[] = {p.w_angle, p.w_dist, p.w_margin, p.margin_cap,
                        p.tau_safe, p.robot_radius, p.reach_radius,
                        p.min_pass_dist};
    for (float x : pv)
        if (!std::isfinite(x))
            return fail(PPS_EINVAL, "pps_server_create: params must be finite");
    if (p.robot_radius < 0.f || p.reach_radius < 0.f || p.min_pass_dist < 0.f)
        return fail(PPS_EINVAL, "pps_server_create: radii and min_pass_dist "
                                "must be >= 0");
    const bool proposal = desc->mode == PPS_SERVE_PROPOSAL;
    if (desc->mode != PPS_SERVE_EXACT && !proposal)
        return fail(PPS_EINVAL, "pps_server_create: unknown mode");
    if (proposal && (!desc->net_weights || desc->topk < 1 ||
                     desc->topk > PPS_NET_H * PPS_NET_W))
        return fail(PPS_EINVAL, "pps_server_create: the proposal mode needs "
                                "net_weights and topk in 1..2806");
    pps_server* srv = new (std::nothrow) pps_server();
    if (!srv) return PPS_ENOMEM;
    srv->d = *desc;
    srv->d.net_weights = nullptr;  // copied into each slot's network
    srv->mask_words_per_slot =
        proposal ? 0
                 : (long long)(desc->pool_bytes / 4 / (size_t)desc->n_streams);
    cudaError_t e = cudaSetDevice(desc->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&srv->num_sms,
                                   cudaDevAttrMultiProcessorCount, desc->device);
    srv->slots.resize((size_t)desc->n_streams);
    for (Slot& s : srv->slots)
        if (e == cudaSuccess)
            e = alloc_slot(s, desc->max_batch, srv->mask_words_per_slot);
    pps_status ns = PPS_OK;
    for (Slot& s : srv->slots) {
        if (e != cudaSuccess || ns != PPS_OK || !proposal) break;
        ns = pps_net_create(desc->device, s.stream, desc->max_batch, &s.net);
        if (ns == PPS_OK) ns = pps_net_set_weights(s.net, desc->net_weights);
    }
    if (e != cudaSuccess || ns != PPS_OK) {
        cudaGetLastError();
        for (Slot& s : srv->slots) free_slot(s);
        delete srv;
        if (ns != PPS_OK)
            return fail(ns, "pps_server_create: the slots' networks");
        return fail(e == cudaErrorMemoryAllocation ? PPS_ENOMEM : PPS_ECUDA,
                    "pps_server_create", e);
    }
    srv->worker = std::thread(worker_main, srv);
    *out = srv;
    return PPS_OK;
}

extern "C" void pps_server_destroy(pps_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    cudaSetDevice(srv->d.device);
    for (Slot& s : srv->slots) free_slot(s);
    cudaGetLastError();
    delete srv;
}

namespace {

// Proposal mode: the batch's requests ordered by their grids' cell size m
// (one pps_propose_jobs call per m), then each group enqueued.
void order_by_cells(Slot& s) {
    std::stable_sort(s.reqs.begin(), s.reqs.end(),
                     [](const Request& a, const Request& b) {
                         return pps::net::cell_lattice(a.job.grid).m <
                                pps::net::cell_lattice(b.job.grid).m;
                     });
}

cudaError_t launch_proposal(pps_server* srv, Slot& s, cudaStream_t st) {
    const int n = (int)s.reqs.size();
    int i0 = 0;
    cudaError_t e = cudaSuccess;
    while (i0 < n && e == cudaSuccess) {
        const int m = pps::net::cell_lattice(s.reqs[i0].job.grid).m;
        int i1 = i0, J = 8, V = 1;
        while (i1 < n && pps::net::cell_lattice(s.reqs[i1].job.grid).m == m) {
            J = std::max(J, opp_slots(s.reqs[i1].job.max_opp));
            V = std::max(V, speed_slots(s.reqs[i1].job.n_speeds));
            ++i1;
        }
        PpsProposeJobs p;
        std::memset(&p, 0, sizeof p);
        p.states = (const pps_state*)(s.d_in + s.o_states) + i0;
        p.jobs = (const pps_job*)(s.d_in + s.o_jobs) + i0;
        p.n = i1 - i0;
        p.jslots = J;
        p.vslots = V;
        p.m = m;
        p.topk = srv->d.topk;
        p.kmax = PPS_MAX_K;
        p.num_sms = srv->num_sms;
        p.fallback = true;
        p.prune = true;
        p.prm = srv->d.params;
        p.best = s.d_best + i0;
        p.keys = s.d_keys + i0;
        p.counts = s.d_counts + i0;
        e = pps_propose_jobs_enqueue(s.net, p, st);
        i0 = i1;
    }
    return e;
}

// Copy a batch in, launch its kernel-instance groups (or, in the proposal
// mode, its proposal calls), copy the results out and record the slot's
// event (all on the slot's stream).
cudaError_t launch_batch(pps_server* srv, Slot& s) {
    const bool proposal = srv->d.mode == PPS_SERVE_PROPOSAL;
    if (proposal) order_by_cells(s);
    const int n = (int)s.reqs.size();
    const size_t total = layout(n, &s.o_states, &s.o_jobs, &s.o_bucket,
                                &s.o_start, &s.o_moff);
    pps_state* h_states = (pps_state*)(s.h_in + s.o_states);
    pps_job* h_jobs = (pps_job*)(s.h_in + s.o_jobs);
    int* h_bucket = (int*)(s.h_in + s.o_bucket);
    long long* h_start = (long long*)(s.h_in + s.o_start);
    long long* h_moff = (long long*)(s.h_in + s.o_moff);
    struct G {
        int j, v;
        std::vector<int> idx;
        int boff = 0, soff = 0;
        long long items = 0;
    };
    std::vector<G> groups;
    long long moff = 0;
    for (int i = 0; i < n; ++i) {
        const Request& r = s.reqs[i];
        h_states[i] = r.st;
        h_jobs[i] = r.job;
        h_moff[i] = moff;
        moff += r.words;
        const int J = opp_slots(r.job.max_opp), V = speed_slots(r.job.n_speeds);
        G* g = nullptr;
        for (G& x : groups)
            if (x.j == J && x.v == V) g = &x;
        if (!g) {
            groups.push_back(G{J, V, {}});
            g = &groups.back();
        }
        g->idx.push_back(i);
    }
    h_moff[n] = moff;
    int bpos = 0, spos = 0;
    for (G& g : groups) {
        g.boff = bpos;
        g.soff = spos;
        long long acc = 0;
        for (int i : g.idx) {
            h_bucket[bpos++] = i;
            h_start[spos++] = acc;
            acc += s.reqs[i].items;
        }
        h_start[spos++] = acc;
        g.items = acc;
    }
    cudaStream_t st = s.stream;
    cudaError_t e = cudaMemcpyAsync(s.d_in, s.h_in, total,
                                    cudaMemcpyHostToDevice, st);
    const bool masks = srv->mask_words_per_slot > 0;
    constexpr int kTpb = 128;  // small batches: spread the items thinly
    if (proposal && e == cudaSuccess) e = launch_proposal(srv, s, st);
    for (const G& g : groups) {
        if (e != cudaSuccess || proposal) break;
        pps::BatchArgs a;
        std::memset(&a, 0, sizeof a);
        a.states = (const pps_state*)(s.d_in + s.o_states);
        a.jobs = (const pps_job*)(s.d_in + s.o_jobs);
        a.bucket_states = (const int*)(s.d_in + s.o_bucket) + g.boff;
        a.item_start = (const long long*)(s.d_in + s.o_start) + g.soff;
        a.mask_off = (const long long*)(s.d_in + s.o_moff);
        a.n_bucket = (int)g.idx.size();
        a.n_items = g.items;
        a.kmax = PPS_MAX_K;
        a.prm = srv->d.params;
        a.best = s.d_best;
        a.mask = masks ? s.d_mask : nullptr;
        a.keys = s.d_keys;
        a.counts = s.d_counts;
        a.next = s.d_next + (&g - groups.data());
        int occ = 1;
        switch (g.j) {
            case 6: occ = pps::batch_occupancy_j6(g.v, kTpb, 1); break;
            case 8: occ = pps::batch_occupancy_j8(g.v, kTpb, 1); break;
            case 12: occ = pps::batch_occupancy_j12(g.v, kTpb, 1); break;
            default: occ = pps::batch_occupancy_j16(g.v, kTpb, 1); break;
        }
        long long grid = (long long)srv->num_sms * occ;
        const long long need = (g.items + kTpb / 32 - 1) / (kTpb / 32);
        grid = std::max(1LL, std::min(grid, need));
        switch (g.j) {
            case 6: e = pps::batch_launch_j6(a, g.v, kTpb, 1, (int)grid, st); break;
            case 8: e = pps::batch_launch_j8(a, g.v, kTpb, 1, (int)grid, st); break;
            case 12: e = pps::batch_launch_j12(a, g.v, kTpb, 1, (int)grid, st); break;
            default: e = pps::batch_launch_j16(a, g.v, kTpb, 1, (int)grid, st); break;
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s.h_best, s.d_best, sizeof(pps_best) * n,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && masks && moff > 0)
        e = cudaMemcpyAsync(s.h_mask, s.d_mask, sizeof(uint32_t) * moff,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(s.done, st);
    s.t_launch = now_ns();
    return e;
}

// Hand every request of a finished slot its result.
void complete(pps_server* srv, Slot& s, int status) {
    const int64_t t = now_ns();
    const int n = (int)s.reqs.size();
    std::vector<Done> out((size_t)n);
    for (int i = 0; i < n; ++i) {
        const Request& r = s.reqs[i];
        Done& d = out[i];
        std::memset(&d.r, 0, sizeof d.r);
        d.r.best = s.h_best[i];
        d.r.ticket = r.ticket;
        d.r.latency_ns = t - r.t_submit;
        d.r.queue_ns = s.t_launch - r.t_submit;
        d.r.batch_size = n;
        d.r.status = status;
        const long long* h_moff = (const long long*)(s.h_in + s.o_moff);
        if (status == PPS_OK && srv->mask_words_per_slot > 0)
            d.mask.assign(s.h_mask + h_moff[i], s.h_mask + h_moff[i] + r.words);
    }
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        for (int i = 0; i < n; ++i) {
            srv->lat_ns.push_back(out[i].r.latency_ns);
            srv->done[out[i].r.ticket] = std::move(out[i]);
        }
        srv->batch_sizes.push_back(n);
        srv->t_last = t;
    }
    srv->cv_done.notify_all();
    s.reqs.clear();
    s.busy = false;
}

void worker_main(pps_server* srv) {
    cudaSetDevice(srv->d.device);
    const long long cap_words = srv->mask_words_per_slot;
    for (;;) {
        bool any_busy = false;
        for (Slot& s : srv->slots) {
            if (!s.busy) continue;
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaSuccess) {
                complete(srv, s, PPS_OK);
            } else if (q != cudaErrorNotReady) {
                srv->fatal = q;
                complete(srv, s, PPS_ECUDA);
            } else {
                any_busy = true;
            }
        }
        for (Slot& s : srv->slots) {
            if (s.busy) continue;
            {
                std::unique_lock<std::mutex> lk(srv->mu);
                if (srv->queue.empty()) break;
                // With a launch in flight, gather requests until the batch
                // is full or the oldest has waited max_wait_us.
                if (any_busy &&
                    (int)srv->queue.size() < srv->d.max_batch &&
                    now_ns() - srv->queue.front().t_submit <
                        (int64_t)srv->d.max_wait_us * 1000)
                    break;
                long long words = 0;
                while (!srv->queue.empty() &&
                       (int)s.reqs.size() < srv->d.max_batch) {
                    const Request& r = srv->queue.front();
                    if (cap_words > 0 && words + r.words > cap_words) break;
                    words += r.words;
                    s.reqs.push_back(r);
                    srv->queue.pop_front();
                }
            }
            if (s.reqs.empty()) break;
            const cudaError_t e = srv->fatal == cudaSuccess
                                      ? launch_batch(srv, s)
                                      : srv->fatal;
            if (e != cudaSuccess) {
                srv->fatal = e;
                complete(srv, s, PPS_ECUDA);
                continue;
            }
            s.busy = true;
            any_busy = true;
        }
        std::unique_lock<std::mutex> lk(srv->mu);
        if (!any_busy && srv->queue.empty()) {
            if (srv->stop) break;
            srv->cv_work.wait(lk, [&] { return srv->stop || !srv->queue.empty(); });
        }
    }
}

}  // namespace

namespace {

pps_status submit_at(pps_server* srv, const pps_state* state,
                     const pps_job* job, int64_t t_arrival, uint64_t* ticket) {
    if (!srv || !state || !job || !ticket)
        return fail(PPS_EINVAL, "pps_server_submit: NULL argument");
    if (!job_ok(*job, srv->d.max_opp) || !state_ok(*state, *job))
        return fail(PPS_EINVAL, "pps_server_submit: bad state or job");
    if (srv->d.mode == PPS_SERVE_PROPOSAL &&
        !pps::net::cell_lattice(job->grid).ok)
        return fail(PPS_EINVAL, "pps_server_submit: the proposal mode serves "
                                "grids on the map's cell lattice (a field of "
                                "at most 12 x 9 m at 0.2 / m m)");
    Request r;
    r.st = *state;
    r.job = *job;
    const long long P = (long long)job->grid.nx * job->grid.ny;
    r.items = (P + 31) / 32;
    r.words = srv->mask_words_per_slot > 0 ? r.items * job->n_speeds : 0;
    if (srv->mask_words_per_slot > 0 && r.words > srv->mask_words_per_slot)
        return fail(PPS_ENOMEM, "pps_server_submit: the request's mask is "
                                "larger than a stream's share of the pool");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->fatal != cudaSuccess)
            return fail(PPS_ECUDA, "pps_server_submit: server failed",
                        srv->fatal);
        if ((int)srv->queue.size() >= srv->d.max_queue)
            return fail(PPS_ENOMEM, "pps_server_submit: queue full");
        r.ticket = srv->next_ticket++;
        r.t_submit = t_arrival;
        if (srv->t_first == 0) srv->t_first = t_arrival;
        srv->queue.push_back(r);
        *ticket = r.ticket;
    }
    srv->cv_work.notify_one();
    return PPS_OK;
}

void summarize(std::vector<int64_t> lat, const std::vector<int>& batches,
               int64_t t0, int64_t t1, pps_server_stats* out) {
    std::memset(out, 0, sizeof *out);
    out->completed = (int64_t)lat.size();
    out->batches = (int64_t)batches.size();
    double bs = 0;
    for (int b : batches) bs += b;
    out->mean_batch = batches.empty() ? 0.0 : bs / batches.size();
    if (lat.empty()) return;
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double q) {
        size_t i = (size_t)std::ceil(q * lat.size()) - 1;
        return lat[std::min(i, lat.size() - 1)] / 1e3;
    };
    double sum = 0;
    for (int64_t x : lat) sum += (double)x;
    out->p50_us = pct(0.50);
    out->p99_us = pct(0.99);
    out->max_us = lat.back() / 1e3;
    out->mean_us = sum / lat.size() / 1e3;
    out->wall_s = (t1 - t0) / 1e9;
    out->states_per_s = out->wall_s > 0 ? lat.size() / out->wall_s : 0.0;
}

}  // namespace

extern "C" pps_status pps_server_submit(pps_server* srv, const pps_state* state,
                                        const pps_job* job, uint64_t* ticket) {
    return submit_at(srv, state, job, now_ns(), ticket);
}

extern "C" pps_status pps_server_wait(pps_server* srv, uint64_t ticket,
                                      int64_t timeout_us,
                                      pps_server_result* out, uint32_t* mask) {
    if (!srv || !out) return fail(PPS_EINVAL, "pps_server_wait: NULL argument");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto ready = [&] { return srv->done.count(ticket) > 0; };
    if (timeout_us < 0)
        srv->cv_done.wait(lk, ready);
    else if (!srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us),
                                    ready))
        return fail(PPS_ETIMEOUT, "pps_server_wait: not done");
    Done& d = srv->done[ticket];
    *out = d.r;
    if (mask && !d.mask.empty())
        std::memcpy(mask, d.mask.data(), d.mask.size() * sizeof(uint32_t));
    srv->done.erase(ticket);
    return out->status;
}

extern "C" pps_status pps_server_replay(pps_server* srv,
                                        const pps_state* frames,
                                        const pps_job* jobs, int n_matches,
                                        int frames_per_match, double hz,
                                        pps_server_result* results,
                                        pps_server_stats* stats) {
    if (!srv || !frames || !jobs || n_matches < 1 || frames_per_match < 1 ||
        !(hz > 0))
        return fail(PPS_EINVAL, "pps_server_replay: bad arguments");
    const size_t total = (size_t)n_matches * frames_per_match;
    std::vector<uint64_t> tickets(total);
    std::vector<int64_t> arrival(total);
    const double period_ns = 1e9 / hz;
    const int64_t t0 = now_ns() + 2000000;  // first frame 2 ms from now
    // Results are taken as they complete by a collector thread, in arrival
    // order, so finished requests do not pile up inside the server.
    std::vector<int64_t> lat(total);
    std::vector<int> sizes;
    int64_t t_last = 0;
    pps_status worst = PPS_OK;
    std::atomic<int> submit_status{PPS_OK};
    std::atomic<size_t> submitted{0};
    std::thread collector([&] {
        for (size_t k = 0; k < total; ++k) {
            const int f = (int)(k / n_matches), m = (int)(k % n_matches);
            const size_t i = (size_t)m * frames_per_match + f;
            while (submitted.load(std::memory_order_acquire) <= k) {
                if (submit_status != PPS_OK) return;
                std::this_thread::yield();
            }
            pps_server_result r;
            pps_status s = pps_server_wait(srv, tickets[i], -1, &r, nullptr);
            if (s != PPS_OK) worst = s;
            lat[i] = r.latency_ns;
            t_last = std::max(t_last, arrival[i] + r.latency_ns);
            if (results) results[i] = r;
        }
    });
    // Frames arrive in time order: frame f of every match, matches spread
    // evenly over the period.
    for (int f = 0; f < frames_per_match && submit_status == PPS_OK; ++f)
        for (int m = 0; m < n_matches; ++m) {
            const size_t i = (size_t)m * frames_per_match + f;
            const int64_t t =
                t0 + (int64_t)(((double)m / n_matches + f) * period_ns);
            for (;;) {
                const int64_t left = t - now_ns();
                if (left <= 0) break;
                if (left > 300000)
                    std::this_thread::sleep_for(
                        std::chrono::nanoseconds(left - 200000));
            }
            arrival[i] = t;
            pps_status s;
            while ((s = submit_at(srv, frames + i, jobs + m, t,
                                  &tickets[i])) == PPS_ENOMEM)
                std::this_thread::yield();  // queue full: back-pressure
            if (s != PPS_OK) {
                submit_status = s;
                break;
            }
            submitted.fetch_add(1, std::memory_order_release);
        }
    collector.join();
    if (submit_status.load() != PPS_OK) return submit_status.load();
    if (stats) {
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            sizes = srv->batch_sizes;
        }
        summarize(lat, sizes, t0, t_last, stats);
    }
    return worst;
}

extern "C" pps_status pps_server_get_stats(pps_server* srv,
                                           pps_server_stats* out) {
    if (!srv || !out) return PPS_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    summarize(srv->lat_ns, srv->batch_sizes, srv->t_first, srv->t_last, out);
    return PPS_OK;
}

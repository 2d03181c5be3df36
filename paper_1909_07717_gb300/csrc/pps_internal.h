// pps_internal.h -- library-internal access to a context (C++ linkage, not
// exported through the C ABI): device, stream, SM count, limits, budgeted
// device allocation and the context's error message.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>

#include "pps.h"

// An NVTX range over the host side of an entry point (enqueueing its
// work), for timelines in external profilers; free when none is attached.
struct PpsRange {
    explicit PpsRange(const char* name) { nvtxRangePushA(name); }
    ~PpsRange() { nvtxRangePop(); }
    PpsRange(const PpsRange&) = delete;
    PpsRange& operator=(const PpsRange&) = delete;
};
#define PPS_RANGE(name) PpsRange pps_range_(name)

int pps_ctx_device(const pps_ctx* ctx);
cudaStream_t pps_ctx_stream(const pps_ctx* ctx);
int pps_ctx_num_sms(const pps_ctx* ctx);
int pps_ctx_max_K(const pps_ctx* ctx);
bool pps_ctx_failed(const pps_ctx* ctx);
// Allocate `bytes` of device memory against the context's budget.
pps_status pps_ctx_alloc(pps_ctx* ctx, void** p, size_t bytes,
                         const char* what);
void pps_ctx_free(pps_ctx* ctx, void* p, size_t bytes);
// printf-style message into the context's error buffer; returns `s`.
pps_status pps_ctx_error(pps_ctx* ctx, pps_status s, const char* fmt, ...);
// Record a CUDA failure on the context (marks it failed).
pps_status pps_ctx_cuda_error(pps_ctx* ctx, cudaError_t e, const char* what);

// Context scratch and limits for the proposal path.
void pps_ctx_scratch(pps_ctx* ctx, unsigned long long** keys, int** counts);
// One device word for a kernel's work queue (zero it before the launch).
unsigned long long* pps_ctx_work_counter(pps_ctx* ctx);
int pps_ctx_max_states(const pps_ctx* ctx);
int pps_ctx_jmax(const pps_ctx* ctx);
int pps_ctx_max_opp(const pps_ctx* ctx);

// CTAs per SM of kernel `func` at `tpb` threads and `smem` bytes of dynamic
// shared memory on the calling thread's current device (at least 1).
// Cached per (device, kernel, CTA size, shared memory) under a lock, so
// concurrent callers and several devices each get their own figure.
int pps_occupancy(const void* func, int tpb, size_t smem);

// Network internals for the proposal path (pps_net.cu): the fallback's
// per-state skip flags, the list of states to re-search and its length,
// and kPpsStateRecBytes a state for the refinement's per-state records
// (pps_propose.cu).
constexpr size_t kPpsStateRecBytes = 384;
struct pps_net_scratch {
    int* skip;
    int* list;
    int* list_n;                // == (int*)(queue + 1)
    unsigned long long* queue;  // the refinement's work-queue counter
    void* srec;                 // max_batch x kPpsStateRecBytes
};
cudaError_t pps_net_predict(pps_net* net, const pps_state* states, int n,
                            cudaStream_t* st, float** scores, int** cells,
                            pps_net_scratch* scratch);
// Top-k map pixels per state into cells[n][k]; with jobs (device, one per
// state), pixels whose cell holds no point of the state's grid rank last.
cudaError_t pps_net_topk(pps_net* net, int n, int k, int* cells,
                         const pps_job* jobs = nullptr);
int pps_net_max_batch(const pps_net* net);

// The proposal for states with their own jobs (pps_propose_jobs), for the
// library's own callers (the serving loop) as well: every buffer is device
// memory; keys and counts are n entries of scratch, left zeroed.
struct PpsProposeJobs {
    const pps_state* states;
    const pps_job* jobs;
    int n;
    int jslots;  // opponent slots: 8, 12 or 16
    int vslots;  // speed slots: 1, 2, 4 or 8 (larger n_speeds: invalid)
    int m;       // fine points per map pixel side (0.2 m / spacing)
    int topk, kmax, num_sms;
    bool fallback, prune;
    pps_params prm;
    pps_best* best;
    int* out_cells;  // n x topk, or null (the network's own buffer)
    unsigned long long* keys;
    int* counts;
};
cudaError_t pps_propose_jobs_enqueue(pps_net* net, const PpsProposeJobs& p,
                                     cudaStream_t st);

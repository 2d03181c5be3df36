// pps_noalloc.cu -- pps_search_noalloc: the exact search without any device
// allocation, for callers that must not call cudaMalloc.
//
// The per-call scratch of the search (one packed argmax key and one feasible
// count per state) lives in a fixed file-scope __device__ array instead of a
// context's buffers.  Every GPU that loads this library holds that array
// (PPS_NOALLOC_MAX_STATES * 12 bytes) until the process exits.
//
// Host code cannot use the array's name as a device address (it names a
// host-side shadow), so the first call on each device, with that device
// current, asks the runtime for the device address once and caches it.
// That first call also loads every kernel instance the entry point can
// launch, so that a later call never loads code (which lazy module loading
// would otherwise do at an instance's first launch).

#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "pps.h"
#include "pps_internal.h"
#include "pps_search.cuh"

// Defined in pps_lib.cu: the thread's message buffer read by
// pps_last_error(NULL).
char* pps_thread_error_buffer();

namespace {

constexpr int kMaxStates = PPS_NOALLOC_MAX_STATES;
constexpr size_t kKeyBytes = sizeof(unsigned long long) * kMaxStates;
constexpr size_t kScratchBytes = kKeyBytes + sizeof(int) * kMaxStates;

// Scratch shared by every pps_search_noalloc call on a device: keys first,
// then counts.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
// The kernel instances this entry point launches: 8 or 16 opponent slots x
// 1, 2, 4 or 8 speed slots.
constexpr int kInstances = 8;
int instance_of(int J, int V) {
    return (J == 8 ? 0 : 4) + (V <= 1 ? 0 : V <= 2 ? 1 : V <= 4 ? 2 : 3);
}

std::mutex g_mu;
struct DeviceSetup {
    void* scratch = nullptr;  // device address of g_scratch on this device
    int num_sms = 0;
    int occ[kInstances] = {};  // CTAs per SM of each search-kernel instance
};
DeviceSetup g_dev[kMaxDevices];

pps_status fail(pps_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(pps_thread_error_buffer(), 512, fmt, ap);
    va_end(ap);
    return s;
}

// Load one instance's search and finalize kernels onto the current device
// (cudaFuncGetAttributes forces the module load that lazy loading would
// otherwise do at the first launch) and record its occupancy.
template <int J, int V>
cudaError_t load_instance(int* occ) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, pps::search_kernel<J, V>);
    if (e == cudaSuccess)
        e = cudaFuncGetAttributes(&fa, pps::finalize_kernel<J, V>);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            occ, pps::search_kernel<J, V>, pps::search_tpb<J, V>(), 0);
    if (*occ < 1) *occ = 1;
    return e;
}

template <int J>
cudaError_t load_instances(int* occ) {
    cudaError_t e = load_instance<J, 1>(occ + instance_of(J, 1));
    if (e == cudaSuccess) e = load_instance<J, 2>(occ + instance_of(J, 2));
    if (e == cudaSuccess) e = load_instance<J, 4>(occ + instance_of(J, 4));
    if (e == cudaSuccess) e = load_instance<J, 8>(occ + instance_of(J, 8));
    return e;
}

// Once per device, with that device current: resolve the scratch array's
// device address, the SM count, and load every kernel instance with its
// occupancy, so that no later call on the device loads code.
pps_status setup(int device, const DeviceSetup** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceSetup& d = g_dev[device];
    if (!d.scratch) {
        DeviceSetup n;
        cudaError_t e = cudaGetSymbolAddress(&n.scratch, g_scratch);
        if (e != cudaSuccess || !n.scratch) {
            cudaGetLastError();
            return fail(PPS_ECUDA,
                        "pps_search_noalloc: cudaGetSymbolAddress on device "
                        "%d: %s", device, cudaGetErrorString(e));
        }
        e = cudaDeviceGetAttribute(&n.num_sms, cudaDevAttrMultiProcessorCount,
                                   device);
        if (e == cudaSuccess) e = load_instances<8>(n.occ);
        if (e == cudaSuccess) e = load_instances<16>(n.occ);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(PPS_ECUDA, "pps_search_noalloc: device %d: %s",
                        device, cudaGetErrorString(e));
        }
        d = n;
    }
    *out = &d;
    return PPS_OK;
}

template <int J, int V>
cudaError_t launch(const pps::SearchArgs& a, const DeviceSetup& dv,
                   cudaStream_t st) {
    const int occ = dv.occ[instance_of(J, V)];
    // One warp per work item of 32 points; no more CTAs than items need.
    const long long items = (long long)a.n_states * a.words;
    long long grid = (long long)dv.num_sms * occ;
    constexpr int tpb = pps::search_tpb<J, V>();
    const long long need = (items + tpb / 32 - 1) / (tpb / 32);
    if (grid > need) grid = need;
    pps::search_kernel<J, V><<<(unsigned)grid, tpb, 0, st>>>(a);
    pps::finalize_kernel<J, V><<<pps::finalize_blocks(a.n_states), 128, 0, st>>>(a);
    return cudaGetLastError();
}

template <int J>
cudaError_t launch_v(const pps::SearchArgs& a, const DeviceSetup& dv,
                     cudaStream_t st) {
    if (a.V <= 1) return launch<J, 1>(a, dv, st);
    if (a.V <= 2) return launch<J, 2>(a, dv, st);
    if (a.V <= 4) return launch<J, 4>(a, dv, st);
    return launch<J, 8>(a, dv, st);
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.f; }

}  // namespace

extern "C" pps_status pps_search_noalloc(
    int device, void* stream, int max_opp, const pps_state* states,
    int n_states, const pps_grid* grid, const float* speeds, int n_speeds,
    const pps_params* params, pps_best* out_best, uint32_t* out_mask) {
    PPS_RANGE("pps_search_noalloc");
    pps_thread_error_buffer()[0] = 0;
    if (device < 0 || device >= kMaxDevices)
        return fail(PPS_EINVAL, "pps_search_noalloc: device %d outside 0..%d",
                    device, kMaxDevices - 1);
    if (max_opp < 1 || max_opp > PPS_MAX_OPP)
        return fail(PPS_EINVAL, "pps_search_noalloc: max_opp %d outside 1..%d",
                    max_opp, PPS_MAX_OPP);
    if (n_states < 0 || n_states > kMaxStates)
        return fail(PPS_EINVAL,
                    "pps_search_noalloc: n_states %d exceeds the limit of %d "
                    "states of the no-allocation entry point (use pps_search "
                    "with a context for larger batches)",
                    n_states, kMaxStates);
    if (!grid || !finite_pos(grid->spacing) || grid->nx < 1 || grid->ny < 1 ||
        !std::isfinite(grid->x0) || !std::isfinite(grid->y0) ||
        (long long)grid->nx * grid->ny > (1 << 24))
        return fail(PPS_EINVAL, "pps_search_noalloc: bad grid");
    if (!speeds || n_speeds < 1 || n_speeds > PPS_MAX_SPEEDS)
        return fail(PPS_EINVAL, "pps_search_noalloc: n_speeds %d outside 1..%d",
                    n_speeds, PPS_MAX_SPEEDS);
    for (int v = 0; v < n_speeds; ++v)
        if (!finite_pos(speeds[v]))
            return fail(PPS_EINVAL, "pps_search_noalloc: speed %d must be "
                                    "finite and > 0", v);
    pps_params prm;
    if (params)
        prm = *params;
    else
        pps_default_params(&prm);
    const float pv[] = {prm.w_angle, prm.w_dist, prm.w_margin,
                        prm.margin_cap, prm.tau_safe, prm.robot_radius,
                        prm.reach_radius, prm.min_pass_dist};
    for (float x : pv)
        if (!std::isfinite(x))
            return fail(PPS_EINVAL, "pps_search_noalloc: params must be finite");
    if (prm.robot_radius < 0.f || prm.reach_radius < 0.f ||
        prm.min_pass_dist < 0.f)
        return fail(PPS_EINVAL, "pps_search_noalloc: radii and min_pass_dist "
                                "must be >= 0");
    if (n_states > 0 && (!states || !out_best))
        return fail(PPS_EINVAL, "pps_search_noalloc: states and out_best are "
                                "required");
    const long long P = (long long)grid->nx * grid->ny;
    if (P * n_speeds >= (1ll << 31))
        return fail(PPS_EINVAL, "pps_search_noalloc: n_speeds * P must be "
                                "below 2^31");
    if (n_states == 0) return PPS_OK;

    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PPS_ECUDA, "pps_search_noalloc: cudaSetDevice(%d): %s",
                    device, cudaGetErrorString(e));
    }
    const DeviceSetup* dv = nullptr;
    pps_status s = setup(device, &dv);
    if (s != PPS_OK) return s;
    void* scratch = dv->scratch;

    cudaStream_t st = (cudaStream_t)stream;
    pps::SearchArgs a;
    std::memset(&a, 0, sizeof a);
    a.states = states;
    a.n_states = n_states;
    a.nx = grid->nx;
    a.ny = grid->ny;
    a.P = (int)P;
    a.words = (int)((P + 31) / 32);
    a.g = grid->spacing;
    a.x0 = grid->x0;
    a.y0 = grid->y0;
    a.V = n_speeds;
    a.kmax = PPS_MAX_K;
    // Unused speed slots repeat the last speed (their results are dropped).
    for (int v = 0; v < PPS_MAX_SPEEDS; ++v) {
        const float sv = speeds[v < n_speeds ? v : n_speeds - 1];
        a.speed[v] = sv;
        a.speed2[v] = sv * sv;
    }
    a.prm = prm;
    a.best = out_best;
    a.mask = out_mask;
    a.keys = (unsigned long long*)scratch;
    a.counts = (int*)((unsigned char*)scratch + kKeyBytes);

    // The array keeps the previous call's keys and counts: clear this call's
    // slots first (no allocation involved).
    e = cudaMemsetAsync(a.keys, 0, sizeof(unsigned long long) * n_states, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(a.counts, 0, sizeof(int) * n_states, st);
    if (e == cudaSuccess)
        e = max_opp <= 8 ? launch_v<8>(a, *dv, st)
                         : launch_v<16>(a, *dv, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PPS_ECUDA, "pps_search_noalloc: launch: %s",
                    cudaGetErrorString(e));
    }
    return PPS_OK;
}

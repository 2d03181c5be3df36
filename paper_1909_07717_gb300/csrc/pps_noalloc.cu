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
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices];  // device address of g_scratch per device
int g_num_sms[kMaxDevices];

pps_status fail(pps_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(pps_thread_error_buffer(), 512, fmt, ap);
    va_end(ap);
    return s;
}

// Once per device, with that device current: resolve the scratch array's
// device address (and the SM count for the persistent grid).
pps_status setup(int device, void** scratch, int* num_sms) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(PPS_ECUDA,
                        "pps_search_noalloc: cudaGetSymbolAddress on device "
                        "%d: %s", device, cudaGetErrorString(e));
        }
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount,
                                   device);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(PPS_ECUDA, "pps_search_noalloc: device %d: %s",
                        device, cudaGetErrorString(e));
        }
        g_num_sms[device] = sms;
        g_scratch_addr[device] = p;
    }
    *scratch = g_scratch_addr[device];
    *num_sms = g_num_sms[device];
    return PPS_OK;
}

template <int J, int V>
cudaError_t launch(const pps::SearchArgs& a, int num_sms, cudaStream_t st) {
    static int occ = 0;
    if (occ == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ, pps::search_kernel<J, V>, pps::search_tpb<J, V>(), 0);
        if (e != cudaSuccess) return e;
        if (occ < 1) occ = 1;
    }
    // One warp per work item of 32 points; no more CTAs than items need.
    const long long items = (long long)a.n_states * a.words;
    long long grid = (long long)num_sms * occ;
    constexpr int tpb = pps::search_tpb<J, V>();
    const long long need = (items + tpb / 32 - 1) / (tpb / 32);
    if (grid > need) grid = need;
    pps::search_kernel<J, V><<<(unsigned)grid, tpb, 0, st>>>(a);
    pps::finalize_kernel<J, V><<<(a.n_states + 127) / 128, 128, 0, st>>>(a);
    return cudaGetLastError();
}

template <int J>
cudaError_t launch_v(const pps::SearchArgs& a, int num_sms, cudaStream_t st) {
    if (a.V <= 1) return launch<J, 1>(a, num_sms, st);
    if (a.V <= 2) return launch<J, 2>(a, num_sms, st);
    if (a.V <= 4) return launch<J, 4>(a, num_sms, st);
    return launch<J, 8>(a, num_sms, st);
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
    void* scratch = nullptr;
    int num_sms = 0;
    pps_status s = setup(device, &scratch, &num_sms);
    if (s != PPS_OK) return s;

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
        e = max_opp <= 8 ? launch_v<8>(a, num_sms, st)
                         : launch_v<16>(a, num_sms, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PPS_ECUDA, "pps_search_noalloc: launch: %s",
                    cudaGetErrorString(e));
    }
    return PPS_OK;
}

// pps_warpcopy.cuh -- a warp's copy of one state and its job in shared
// memory, for the kernels that give a state to a single warp (the
// finalizes): every lane loads a few 32-bit words at once, one memory
// latency, instead of the chain of field loads the state's derivation
// would otherwise wait on, and the re-evaluation then reads the opponents
// from shared memory.
#pragma once

#include <stdint.h>

#include "pps.h"

namespace pps {

struct WarpStateJob {
    pps_state st;
    pps_job job;
};
static_assert(sizeof(pps_state) % 4 == 0 && sizeof(pps_job) % 4 == 0,
              "copied as 32-bit words");

template <int BYTES>
__device__ __forceinline__ void warp_copy(void* dst, const void* src,
                                          int lane) {
    constexpr int kWords = BYTES / 4, kPer = (kWords + 31) / 32;
    const uint32_t* from = static_cast<const uint32_t*>(src);
    uint32_t* to = static_cast<uint32_t*>(dst);
    uint32_t w[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i)
        if (i * 32 + lane < kWords) w[i] = __ldg(from + i * 32 + lane);
#pragma unroll
    for (int i = 0; i < kPer; ++i)
        if (i * 32 + lane < kWords) to[i * 32 + lane] = w[i];
}

// Every lane of the warp takes part; the copy is complete on return.
__device__ __forceinline__ void warp_load_state_job(WarpStateJob& d,
                                                    const pps_state* st,
                                                    const pps_job* job,
                                                    int lane) {
    __syncwarp();
    warp_copy<sizeof(pps_state)>(&d.st, st, lane);
    warp_copy<sizeof(pps_job)>(&d.job, job, lane);
    __syncwarp();
}

}  // namespace pps

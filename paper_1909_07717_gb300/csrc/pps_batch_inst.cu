// pps_batch_inst.cu -- instances of the batched-plan kernels for one
// opponent-slot count, PPS_BATCH_J (6, 8, 12 or 16): every speed-slot count
// and every (CTA size, samples a register block) the autotuner chooses from.  The build compiles this
// file once per slot count (-DPPS_BATCH_J=...), which keeps each instance
// set in its own object and the four compilations in parallel.
#include "pps_batch.cuh"
#include "pps_internal.h"

#ifndef PPS_BATCH_J
#error "compile with -DPPS_BATCH_J=6, 8, 12 or 16"
#endif

namespace pps {
namespace {

constexpr int J = PPS_BATCH_J;
static_assert(J == 6 || J == 8 || J == 12 || J == 16, "opponent slots");

template <int V, int T, int KU>
cudaError_t go(const BatchArgs& a, int grid, cudaStream_t st) {
    if (a.recs)
        batch_prepare_kernel<J><<<(a.n_bucket + 127) / 128, 128, 0, st>>>(a);
    batch_search_kernel<J, V, T, KU><<<grid, T, 0, st>>>(a);
    batch_finalize_kernel<J, V><<<finalize_blocks(a.n_bucket), 128, 0, st>>>(a);
    return cudaGetLastError();
}

// the autotuner's candidates: every CTA size with one sample a register
// block, the two smallest (registers to spare) also with two
template <int V>
cudaError_t go_t(const BatchArgs& a, int tpb, int ku, int grid, cudaStream_t st) {
    if (ku == 2 && tpb == 128) return go<V, 128, 2>(a, grid, st);
    if (ku == 2 && tpb == 256) return go<V, 256, 2>(a, grid, st);
    if (tpb == 128) return go<V, 128, 1>(a, grid, st);
    if (tpb == 256) return go<V, 256, 1>(a, grid, st);
    if (tpb == 512) return go<V, 512, 1>(a, grid, st);
    if (tpb == 768) return go<V, 768, 1>(a, grid, st);
    return go<V, 1024, 1>(a, grid, st);
}

template <int V, int T, int KU>
int occ() {
    return pps_occupancy((const void*)batch_search_kernel<J, V, T, KU>, T, 0);
}

template <int V>
int occ_t(int tpb, int ku) {
    if (ku == 2 && tpb == 128) return occ<V, 128, 2>();
    if (ku == 2 && tpb == 256) return occ<V, 256, 2>();
    if (tpb == 128) return occ<V, 128, 1>();
    if (tpb == 256) return occ<V, 256, 1>();
    if (tpb == 512) return occ<V, 512, 1>();
    if (tpb == 768) return occ<V, 768, 1>();
    return occ<V, 1024, 1>();
}

cudaError_t launch_any(const BatchArgs& a, int vmax, int tpb, int ku, int grid,
                       cudaStream_t st) {
    if (vmax <= 1) return go_t<1>(a, tpb, ku, grid, st);
    if (vmax <= 2) return go_t<2>(a, tpb, ku, grid, st);
    if (vmax <= 4) return go_t<4>(a, tpb, ku, grid, st);
    return go_t<8>(a, tpb, ku, grid, st);
}

int occupancy_any(int vmax, int tpb, int ku) {
    if (vmax <= 1) return occ_t<1>(tpb, ku);
    if (vmax <= 2) return occ_t<2>(tpb, ku);
    if (vmax <= 4) return occ_t<4>(tpb, ku);
    return occ_t<8>(tpb, ku);
}

}  // namespace

#define PPS_BATCH_DEFINE_(N)                                                 \
    cudaError_t batch_launch_j##N(const BatchArgs& a, int vmax, int tpb,    \
                                  int ku, int grid, cudaStream_t st) {      \
        return launch_any(a, vmax, tpb, ku, grid, st);                      \
    }                                                                       \
    int batch_occupancy_j##N(int vmax, int tpb, int ku) {                   \
        return occupancy_any(vmax, tpb, ku);                                \
    }
#define PPS_BATCH_DEFINE(N) PPS_BATCH_DEFINE_(N)
PPS_BATCH_DEFINE(PPS_BATCH_J)

}  // namespace pps

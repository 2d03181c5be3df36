// pps_batch_j12.cu -- instances of the batched-plan kernels with 12 opponent
// slots (all speed-slot counts and CTA sizes the autotuner chooses from).
#include "pps_batch.cuh"

namespace pps {
namespace {

template <int V, int T>
cudaError_t go(const BatchArgs& a, int grid, cudaStream_t st) {
    batch_search_kernel<12, V, T><<<grid, T, 0, st>>>(a);
    batch_finalize_kernel<12, V><<<(a.n_bucket + 127) / 128, 128, 0, st>>>(a);
    return cudaGetLastError();
}

template <int V>
cudaError_t go_t(const BatchArgs& a, int tpb, int grid, cudaStream_t st) {
    if (tpb == 128) return go<V, 128>(a, grid, st);
    if (tpb == 256) return go<V, 256>(a, grid, st);
    if (tpb == 512) return go<V, 512>(a, grid, st);
    if (tpb == 768) return go<V, 768>(a, grid, st);
    return go<V, 1024>(a, grid, st);
}

template <int V, int T>
int occ() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, batch_search_kernel<12, V, T>, T, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n < 1 ? 1 : n;
}

template <int V>
int occ_t(int tpb) {
    if (tpb == 128) return occ<V, 128>();
    if (tpb == 256) return occ<V, 256>();
    if (tpb == 512) return occ<V, 512>();
    if (tpb == 768) return occ<V, 768>();
    return occ<V, 1024>();
}

}  // namespace

cudaError_t batch_launch_j12(const BatchArgs& a, int vmax, int tpb, int grid,
                             cudaStream_t st) {
    if (vmax <= 1) return go_t<1>(a, tpb, grid, st);
    if (vmax <= 2) return go_t<2>(a, tpb, grid, st);
    if (vmax <= 4) return go_t<4>(a, tpb, grid, st);
    return go_t<8>(a, tpb, grid, st);
}

int batch_occupancy_j12(int vmax, int tpb) {
    if (vmax <= 1) return occ_t<1>(tpb);
    if (vmax <= 2) return occ_t<2>(tpb);
    if (vmax <= 4) return occ_t<4>(tpb);
    return occ_t<8>(tpb);
}

}  // namespace pps

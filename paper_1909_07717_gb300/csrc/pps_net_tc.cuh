// pps_net_tc.cuh -- the proposal network's inference pass on the 5th-
// generation tensor cores: the four 3x3 convolutions of one band of map
// rows as implicit GEMMs issued with tcgen05.mma (A = shifted activation
// windows and B = weights, both straight from shared memory through
// descriptors; D = FP32 accumulators in tensor memory), the bias / ReLU /
// bfloat16 epilogue read back with tcgen05.ld.  Activations never leave the
// SM; the next band's input rows stream in with cp.async while layers 2-4
// run.  For training the kernel also writes the hidden activations of each
// band's own rows to device memory.
//
// Layouts (all K-major, no swizzle: 8-row x 16-byte core matrices):
//   activations: one plane per 8 channels; a plane is a run of 16-byte
//     slots, slot = 8 + row * 64 + column (8 zero slots before row 0 and
//     after the last row); columns 61..63 of every row are zero, so a
//     column shift of -1 or +1 reads a zero at the map's edge -- the
//     previous row's column 63 serves as column -1.  A 128-row MMA tile is
//     two map rows; the tap (dy, dx) is a start-address offset of
//     (dy * 64 + dx) slots.  LBO (next 8 channels) = plane size, SBO = 128 B.
//   weights: [tap][8-channel chunk][output channel] x 16 B; LBO = cout x 16,
//     SBO = 128 B.
#pragma once

#include "pps_net.cuh"
#include "pps_tc.cuh"

namespace pps {
namespace net {
namespace tcf {

constexpr int kBand = 8;                            // output rows per unit
constexpr int kBands = (H + kBand - 1) / kBand;
constexpr int kLead = 8, kRow = 64;
constexpr int kInRows = kBand + 8, kARows = kBand + 6, kBRows = kBand + 4;
constexpr int kSlotsIn = kLead + kInRows * kRow + kLead;
constexpr int kSlotsA = kLead + kARows * kRow + kLead;
constexpr int kSlotsB = kLead + kBRows * kRow + kLead;
constexpr int kNOut = 16;  // output layer N (channel 0 used)
constexpr int kOffA = 2 * kSlotsIn * 16;
constexpr int kOffB = kOffA + 4 * kSlotsA * 16;
constexpr int kOffW0 = kOffB + 4 * kSlotsB * 16;
constexpr int kOffW1 = kOffW0 + 9 * 2 * CH * 16;
constexpr int kOffW2 = kOffW1 + 9 * 4 * CH * 16;
constexpr int kOffW3 = kOffW2 + 9 * 4 * CH * 16;
constexpr int kOffSkip = kOffW3 + 9 * 4 * kNOut * 16;
constexpr int kMaxTiles = kARows / 2;
constexpr int kOffBar = kOffSkip + kBand * W * 4;
constexpr int kOffTmem = kOffBar + 8 * kMaxTiles;
constexpr size_t kSmemBytes = kOffTmem + 8;
constexpr int kThreads = 512;
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kWaitPolls = 1u << 22;  // polls per mbarrier wait
constexpr uint32_t kTestPolls = 1u << 10;  // the self-test's short limit
static_assert(kSmemBytes <= 232448, "one CTA per SM");
static_assert(kARows / 2 * CH <= (int)kTmemCols, "accumulators fit");
static_assert(kOffBar % 8 == 0, "mbarrier alignment");

// Weights [tap][co][cin] (cout rows, the first cout_copy copied) ->
// [tap][cin / 8][cout_copy] x 16 B.
__device__ __forceinline__ void stage(uint8_t* dst, const __nv_bfloat16* src,
                                      int cout, int cout_copy, int cin) {
    const int chunks = cin / 8, total = 9 * chunks * cout_copy;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int co = i % cout_copy, rest = i / cout_copy;
        const int ch = rest % chunks, tap = rest / chunks;
        reinterpret_cast<uint4*>(dst)[(tap * chunks + ch) * cout_copy + co] =
            reinterpret_cast<const uint4*>(src)[(tap * cout + co) * chunks + ch];
    }
}

// Input rows y0 - 4 .. y0 + kBand + 3 of state s (16 channels = 2 planes),
// zero outside the map.
__device__ __forceinline__ void prefetch(const __nv_bfloat16* __restrict__ a0,
                                         long long u, uint8_t* in) {
    const int s = (int)(u / kBands);
    const int y0 = (int)(u - (long long)s * kBands) * kBand;
    const __nv_bfloat16* src = a0 + (long long)s * NPIX * C0;
    for (int i = threadIdx.x; i < kInRows * W * 2; i += blockDim.x) {
        const int half = i & 1, q = i >> 1;
        const int r = q / W, x = q - r * W;
        const int Y = y0 - 4 + r;
        const bool ok = Y >= 0 && Y < H;
        const __nv_bfloat16* g = src + ((ok ? Y : 0) * W + x) * C0 + half * 8;
        const uint32_t d =
            tc::smem_u32(in + (half * kSlotsIn + kLead + r * kRow + x) * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d),
                     "l"(g), "r"(ok ? 16 : 0));
    }
    asm volatile("cp.async.commit_group;");
}

// Issue one layer: ntiles 128-row tiles (two map rows each) of COUT
// accumulators, K = 9 taps x CIN, each tile's MMAs followed by a commit to
// its own mbarrier so that its epilogue can start while later tiles run.
// One thread.  Descriptors differ only in their start address: offsets in
// 16-byte units are added to a base descriptor.
template <int CIN, int COUT>
__device__ __forceinline__ void issue(uint32_t tmem, const uint8_t* in,
                                      int slots_in, const uint8_t* w,
                                      int ntiles, uint32_t bars) {
    constexpr uint32_t idesc = tc::idesc_bf16(128, COUT);
    const uint64_t a_base = tc::desc_kmajor(tc::smem_u32(in) + kLead * 16,
                                            slots_in * 16, 128);
    const uint64_t b_base = tc::desc_kmajor(tc::smem_u32(w), COUT * 16, 128);
    for (int j = 0; j < ntiles; ++j) {
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
#pragma unroll
            for (int kc = 0; kc < CIN / 16; ++kc) {
                const long long a_off =
                    (long long)(2 * kc) * slots_in + (2 * j + 1 + dy) * kRow + dx;
                const long long b_off = (long long)(tap * (CIN / 8) + 2 * kc) * COUT;
                tc::mma_bf16(tmem + j * COUT, a_base + (uint64_t)a_off,
                             b_base + (uint64_t)b_off, idesc, (tap | kc) != 0);
            }
        }
        tc::commit(bars + 8 * j);
    }
}

// Hidden-layer epilogue: bias, ReLU, bf16, into the next buffer (zero
// outside the map and in columns 61..63).  A warp serves one lane quarter
// of a tile as soon as that tile's accumulators are complete.
// With act (training), the band's own rows y0 .. y0 + kBand - 1 of the
// activations also go to act[s][y][x][32] in device memory for the
// backward pass (the halo rows are other bands' own rows).
template <bool KEEP>
__device__ __forceinline__ bool epi_hidden(uint32_t tmem, int ntiles,
                                           const float* __restrict__ bias,
                                           int y_first, uint8_t* out,
                                           int slots_out, uint32_t bars,
                                           uint32_t phases, uint32_t polls,
                                           __nv_bfloat16* __restrict__ act,
                                           int s, int y0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = warp & 3;
    bool ok = true;
    for (int j = warp >> 2; j < ntiles; j += kThreads / 128) {
        ok = ok && tc::mbar_wait(bars + 8 * j, (phases >> j) & 1u, polls);
        tc::fence_after_sync();
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + j * CH, v);
        const int r = 32 * q + lane, row = 2 * j + (r >> 6), col = r & 63;
        const int Y = y_first + row;
        const bool in_map = Y >= 0 && Y < H && col < W;
        const bool own = KEEP && in_map && Y >= y0 && Y < y0 + kBand;
        uint4* ga = own ? reinterpret_cast<uint4*>(
                              act + ((long long)s * NPIX + Y * W + col) * CH)
                        : nullptr;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint4 o;
            uint32_t* p = reinterpret_cast<uint32_t*>(&o);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = 8 * k + 2 * e;
                p[e] = in_map ? pack_bf16(fmaxf(v[c] + __ldg(bias + c), 0.f),
                                          fmaxf(v[c + 1] + __ldg(bias + c + 1), 0.f))
                              : 0u;
            }
            reinterpret_cast<uint4*>(out)[k * slots_out + kLead + row * kRow + col] = o;
            if (KEEP && own) ga[k] = o;
        }
    }
    return ok;
}

// KEEP (training): the hidden activations of each band's own rows also go
// to act1..act3; the inference instance carries none of that.
template <bool KEEP>
__global__ void __launch_bounds__(kThreads, 1)
    tc_forward_kernel(const __nv_bfloat16* __restrict__ a0, int n,
                      const __nv_bfloat16* __restrict__ Wf,
                      const float* __restrict__ w32, float* __restrict__ out,
                      int wf1, int wf2, int wf3, int b0, int b1, int b2, int b3,
                      int* __restrict__ err, int withhold,
                      __nv_bfloat16* __restrict__ act1,
                      __nv_bfloat16* __restrict__ act2,
                      __nv_bfloat16* __restrict__ act3) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t* bin = smem;
    uint8_t* ba = smem + kOffA;
    uint8_t* bb = smem + kOffB;
    float* skip = reinterpret_cast<float*>(smem + kOffSkip);
    const uint32_t bars = tc::smem_u32(smem + kOffBar);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + kOffTmem);
    const int warp = threadIdx.x >> 5;

    for (int i = threadIdx.x; i < kOffW0 / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    stage(smem + kOffW0, Wf, CH, CH, C0);
    stage(smem + kOffW1, Wf + wf1, CH, CH, CH);
    stage(smem + kOffW2, Wf + wf2, CH, CH, CH);
    stage(smem + kOffW3, Wf + wf3, CO, kNOut, CH);
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_holder), kTmemCols);
    if (threadIdx.x < kMaxTiles) tc::mbar_init(bars + 8 * threadIdx.x, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_holder;
    uint32_t phases = 0;  // bit j: parity of tile j's next completion
    bool bad = false;
    const long long units = (long long)n * kBands;
    if (blockIdx.x < units) prefetch(a0, blockIdx.x, bin);

    // make the layer's operands visible to the tensor cores and the last
    // epilogue's TMEM reads ordered before the barrier; then one thread
    // issues the layer
    auto start_layer = [&](auto issue_fn) -> bool {
        tc::fence_async_smem();
        tc::fence_before_sync();
        if (__syncthreads_or(bad)) return false;
        // withhold (self-test of the bounded waits): nothing is issued, no
        // mbarrier ever completes, every wait runs out
        if (threadIdx.x == 0 && !withhold) {
            tc::fence_after_sync();
            issue_fn();
        }
        return true;
    };
    auto end_layer = [&](int ntiles, bool ok) {
        if (!ok) {
            bad = true;
            atomicExch(err, 1);
        }
        phases ^= (1u << ntiles) - 1u;
    };

    const uint32_t polls = withhold ? kTestPolls : kWaitPolls;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const int s = (int)(u / kBands);
        const int y0 = (int)(u - (long long)s * kBands) * kBand;
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (__syncthreads_or(bad)) break;  // a wait ran out: stop everywhere
        for (int i = threadIdx.x; i < kBand * W; i += blockDim.x) {
            const int r = i / W, x = i - r * W;
            skip[i] = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(
                bin + (kLead + (r + 4) * kRow + x) * 16)[1]);
        }
        // layer 1: input -> A (kARows rows); once every tile is done the
        // input buffer is free for the next unit's rows
        constexpr int t1 = kARows / 2, t2 = kBRows / 2, t3 = (kBand + 2) / 2,
                      t4 = kBand / 2;
        if (!start_layer([&] { issue<C0, CH>(tmem, bin, kSlotsIn, smem + kOffW0, t1, bars); }))
            break;
        end_layer(t1, epi_hidden<KEEP>(tmem, t1, w32 + b0, y0 - 3, ba, kSlotsA, bars,
                                 phases, polls, act1, s, y0));
        if (!start_layer([&] { issue<CH, CH>(tmem, ba, kSlotsA, smem + kOffW1, t2, bars); }))
            break;
        if (u + gridDim.x < units) prefetch(a0, u + gridDim.x, bin);
        end_layer(t2, epi_hidden<KEEP>(tmem, t2, w32 + b1, y0 - 2, bb, kSlotsB, bars,
                                 phases, polls, act2, s, y0));
        if (!start_layer([&] { issue<CH, CH>(tmem, bb, kSlotsB, smem + kOffW2, t3, bars); }))
            break;
        end_layer(t3, epi_hidden<KEEP>(tmem, t3, w32 + b2, y0 - 1, ba, kSlotsA, bars,
                                 phases, polls, act3, s, y0));
        // layer 4: A -> the output map (+ the coarse-score input channel)
        if (!start_layer([&] { issue<CH, kNOut>(tmem, ba, kSlotsA, smem + kOffW3, t4, bars); }))
            break;
        bool ok = true;
        {
            const int lane = threadIdx.x & 31, q = warp & 3;
            for (int j = warp >> 2; j < t4; j += kThreads / 128) {
                ok = ok && tc::mbar_wait(bars + 8 * j, (phases >> j) & 1u, polls);
                tc::fence_after_sync();
                const float v = tc::tmem_ld1(tmem + ((uint32_t)(32 * q) << 16) + j * kNOut);
                const int r = 32 * q + lane, row = 2 * j + (r >> 6), col = r & 63;
                const int Y = y0 + row;
                if (Y < H && col < W)
                    out[(long long)s * NPIX + Y * W + col] =
                        v + __ldg(w32 + b3) + skip[row * W + col];
            }
        }
        end_layer(t4, ok);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace tcf
}  // namespace net
}  // namespace pps

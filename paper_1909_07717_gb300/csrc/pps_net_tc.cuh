// pps_net_tc.cuh -- the proposal network's inference pass on the 5th-
// generation tensor cores: the four 3x3 convolutions of one band of map
// rows as implicit GEMMs issued with tcgen05.mma (A = shifted activation
// windows and B = weights, both straight from shared memory through
// descriptors; D = FP32 accumulators in tensor memory), the bias / ReLU /
// bfloat16 epilogue read back with tcgen05.ld.  Activations never leave the
// SM.  For training the kernel also writes the hidden activations of each
// band's own rows to device memory.
//
// Roles (warp-specialised, one CTA per SM, persistent over bands):
//   * two issuer threads (tiles of even and odd index) issue the MMAs tile
//     by tile, and the first also loads each band's input rows with the
//     tensor memory accelerator (a 5-D tiled map of the 16-channel input,
//     rows outside the map and columns 61..63 filled with zeros by the copy
//     itself); tile j of layer L + 1 reads the output
//     rows of tiles j and j + 1 of layer L, so it is issued as soon as
//     those two tiles' epilogues are done -- the layers of a band, and
//     consecutive bands, overlap instead of running behind block barriers;
//   * 16 epilogue warps, four warpgroups taking the band's items in turn;
//     each group reads its tile's accumulators (each warp its lane
//     quarter), writes the next layer's input rows into shared memory and
//     arrives on the tile's "epilogue done" mbarrier.
//   The one-channel output layer is not a convolution of N = 16 MMAs
//   (15 wasted columns, 18 MMAs a tile): one pair of MMAs per layer-3
//   tile gives each pixel its 9 taps' partial sums (taps along N), and the
//   epilogue adds the 9 partials at the shifted pixels -- 10 MMAs a band
//   instead of 72.
//   Buffer reuse between the issuers: a commit tracks its own thread's
//   MMAs only.  Tile j of a layer waits for tiles j and j + 1 of the layer
//   below, one of each issuer, so every earlier MMA of both issuers has
//   completed before its epilogue overwrites a buffer; the next band's
//   layer-1 tile j waits for one tile only, and the rows its epilogue
//   overwrites are read by no other issuer's pending MMA (the partials of
//   tile j read only rows 2j, 2j + 1).
//   Tensor memory holds two halves of 256 columns, used by layers of
//   alternating parity, so a layer's accumulators can be written while the
//   previous layer's are still being read.  Every wait is bounded: a wait
//   that runs out sets the error flag and an abort flag the other roles
//   poll, the issuers wait (bounded) for their MMAs and copies in flight,
//   and the kernel returns.
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

#include <cuda.h>

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
constexpr int kMaxTiles = kARows / 2;
constexpr int kNOut = 16;  // output layer N (channel 0 used)
constexpr int kOffA = 2 * kSlotsIn * 16;
constexpr int kOffB = kOffA + 4 * kSlotsA * 16;
constexpr int kOffW0 = kOffB + 4 * kSlotsB * 16;
constexpr int kPairs = 5;  // layer 1: the 9 taps' 8 input channels in K pairs
constexpr int kOffW1 = kOffW0 + kPairs * 2 * CH * 16;
constexpr int kOffW2 = kOffW1 + 9 * 4 * CH * 16;
constexpr int kOffW3 = kOffW2 + 9 * 4 * CH * 16;
// Output layer (one channel): B = W3 with the 9 taps along N (16, 7 zero)
// and the 32 input channels along K; one tile's MMAs give every pixel of
// two layer-3 rows its 9 tap partials, which the epilogue adds up at the
// shifted pixels.  The partials of the band's 10 layer-3 rows wait in
// shared memory, [tap][1 + row x 64 + column] floats (a leading zero slot
// for column -1 of row 0; columns 61..63 are zero like the activations).
constexpr int kDSlots = 1 + (kBand + 2) * kRow;
constexpr int kDStride = (kDSlots + 3) & ~3;
constexpr int kOffBias = kOffW3 + 4 * kNOut * 16;           // 4 x 32 floats
constexpr int kOffPart = kOffBias + 4 * CH * 4;             // 9 x kDStride f32
constexpr int kOffBar = kOffPart + 9 * kDStride * 4;
// mbarriers: accumulators full [layer][tile], epilogue done [layer][tile]
// (layer 3 = the output layer's partials), output rows done [tile], input
// full, input free (both issuers), drain [issuer]
constexpr int kBarAcc = 0, kBarEpi = 4 * kMaxTiles, kBarOut = 8 * kMaxTiles,
              kBarInFull = kBarOut + kBand / 2, kBarInFree = kBarInFull + 1,
              kBarDrain = kBarInFree + 1, kNumBars = kBarDrain + 2;
constexpr int kOffTmem = kOffBar + 8 * kNumBars;
constexpr int kOffAbort = kOffTmem + 8;
constexpr size_t kSmemUsed = kOffAbort + 8;
constexpr size_t kSmemBytes = kSmemUsed + 128;  // slack to align the base to 128
constexpr int kEpiWarps = 16;
constexpr int kIssuers = 2;  // MMA-issuing threads (one a warp): tile j goes
                             // to issuer j mod 2 (one thread issues an MMA
                             // about every 55 cycles, two together every 40)
constexpr int kThreads = 32 * (kEpiWarps + kIssuers);
constexpr uint32_t kTmemCols = 512;                // two halves of 256
constexpr uint32_t kTmemHalf = 256;
constexpr uint32_t kInBytes = 2 * kInRows * kRow * 16;  // one band's input
constexpr uint32_t kWaitPolls = 1u << 22;  // polls per mbarrier wait
constexpr uint32_t kTestPolls = 1u << 10;  // the self-test's short limit
static_assert(kSmemBytes <= 232448, "one CTA per SM");
static_assert(kMaxTiles * 32 <= (int)kTmemHalf, "a layer's accumulators fit a half");
static_assert(kOffBar % 8 == 0, "mbarrier alignment");
static_assert((kSlotsIn * 16) % 128 == 0 && (kLead * 16) % 128 == 0,
              "the input planes start 128-byte aligned");

// Weights [tap][co][cin] (cout rows, the first cout_copy copied) ->
// [tap][cin / 8][cout_copy] x 16 B.
__device__ __forceinline__ void stage(uint8_t* dst, const __nv_bfloat16* src,
                                      int cout, int cout_copy, int cin, int tid,
                                      int nthreads) {
    const int chunks = cin / 8, total = 9 * chunks * cout_copy;
    for (int i = tid; i < total; i += nthreads) {
        const int co = i % cout_copy, rest = i / cout_copy;
        const int ch = rest % chunks, tap = rest / chunks;
        reinterpret_cast<uint4*>(dst)[(tap * chunks + ch) * cout_copy + co] =
            reinterpret_cast<const uint4*>(src)[(tap * cout + co) * chunks + ch];
    }
}

// Layer-1 weights [tap][co][16 cin] (channels 8..15 multiply the input's
// zero channels and are left out) -> [pair p][tap 2p, 2p + 1][co] x 16 B;
// the missing partner of tap 8 is zero.
__device__ __forceinline__ void stage_l1_pairs(uint8_t* dst, const __nv_bfloat16* src,
                                               int tid, int nthreads) {
    for (int i = tid; i < kPairs * 2 * CH; i += nthreads) {
        const int co = i % CH, h = (i / CH) & 1, p = i / (2 * CH);
        const int tap = 2 * p + h;
        reinterpret_cast<uint4*>(dst)[i] =
            tap < 9 ? reinterpret_cast<const uint4*>(src)[(tap * CH + co) * (C0 / 8)]
                    : make_uint4(0u, 0u, 0u, 0u);
    }
}

// Output-layer weights [tap][co][32 cin] (channel co = 0 used) -> [cin / 8]
// [n = tap, 16 rows, taps 9..15 zero] x 16 B: B of the partials' MMAs.
__device__ __forceinline__ void stage_out_taps(uint8_t* dst, const __nv_bfloat16* src,
                                               int tid, int nthreads) {
    for (int i = tid; i < (CH / 8) * kNOut; i += nthreads) {
        const int n = i % kNOut, c = i / kNOut;
        reinterpret_cast<uint4*>(dst)[i] =
            n < 9 ? reinterpret_cast<const uint4*>(src)[(n * CO) * (CH / 8) + c]
                  : make_uint4(0u, 0u, 0u, 0u);
    }
}

// Input rows y0 - 4 .. y0 + kBand + 3 of unit u's state into the input
// planes (one box a plane: 8 channels x 64 columns x kInRows rows; the map
// has 61 columns and H rows, the rest is filled with zeros), completing on
// the mbarrier.  One thread.
__device__ __forceinline__ void load_band(const CUtensorMap* map, long long u,
                                          uint32_t in, uint32_t bar) {
    const int s = (int)(u / kBands);
    const int y0 = (int)(u - (long long)s * kBands) * kBand;
    tc::mbar_expect_tx(bar, kInBytes);
#pragma unroll
    for (int h = 0; h < 2; ++h)
        tc::tma_load_5d(in + (uint32_t)(h * kSlotsIn + kLead) * 16u, map, 0, h, 0,
                        y0 - 4, s, bar);
}

// Issue tile j of one layer: 128 rows (two map rows) x COUT accumulators,
// K = 9 taps x CIN, then a commit to the tile's mbarrier.  One thread.
// Descriptors differ only in their start address: offsets in 16-byte units
// are added to a base descriptor.
template <int CIN, int COUT>
__device__ __forceinline__ void issue_tile(uint32_t d_tmem, const uint8_t* in,
                                           int slots_in, const uint8_t* w, int j,
                                           uint32_t bar) {
    constexpr uint32_t idesc = tc::idesc_bf16(128, COUT);
    const uint64_t a_base = tc::desc_kmajor(tc::smem_u32(in) + kLead * 16,
                                            slots_in * 16, 128);
    const uint64_t b_base = tc::desc_kmajor(tc::smem_u32(w), COUT * 16, 128);
    // the offsets only move the 14-bit start-address field (shared memory
    // addresses / 16 stay below 2^14), so they are added to the low words
    const uint32_t a_lo = (uint32_t)a_base + (uint32_t)((2 * j + 1) * kRow);
    const uint32_t a_hi = (uint32_t)(a_base >> 32);
    const uint32_t b_lo = (uint32_t)b_base, b_hi = (uint32_t)(b_base >> 32);
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
#pragma unroll
        for (int kc = 0; kc < CIN / 16; ++kc) {
            const uint32_t a_off = (uint32_t)(2 * kc * slots_in + dy * kRow + dx);
            const uint32_t b_off = (uint32_t)((tap * (CIN / 8) + 2 * kc) * COUT);
            tc::mma_bf16(d_tmem, ((uint64_t)a_hi << 32) | (a_lo + a_off),
                         ((uint64_t)b_hi << 32) | (b_lo + b_off), idesc,
                         (tap | kc) != 0);
        }
    }
    tc::commit(bar);
}

// Layer 1's tile j: K = 16 is two taps' 8 input channels.  The A
// descriptor's leading byte offset (the distance between its two K core
// matrices) is the slot distance between the two taps' windows, so one MMA
// reads both shifted windows; 5 MMAs instead of 9.
__device__ __forceinline__ void issue_tile_l1(uint32_t d_tmem, const uint8_t* in,
                                              const uint8_t* w, int j, uint32_t bar) {
    constexpr uint32_t idesc = tc::idesc_bf16(128, CH);
    const uint64_t a_base = tc::desc_kmajor(tc::smem_u32(in) + kLead * 16, 16, 128);
    const uint64_t b_base = tc::desc_kmajor(tc::smem_u32(w), CH * 16, 128);
    // start-address field only (the LBO field is set per pair below)
    const uint32_t a_lo = ((uint32_t)a_base & 0x3FFFu) + (uint32_t)((2 * j + 1) * kRow);
    const uint32_t a_hi = (uint32_t)(a_base >> 32);
    const uint32_t b_lo = (uint32_t)b_base, b_hi = (uint32_t)(b_base >> 32);
#pragma unroll
    for (int p = 0; p < kPairs; ++p) {
        const int ta = 2 * p, tb = 2 * p + 1;
        const int sa = (ta / 3 - 1) * kRow + (ta % 3 - 1);
        // tap 8 has no partner: its zero weights read the next slot
        const int sb = tb < 9 ? (tb / 3 - 1) * kRow + (tb % 3 - 1) : sa + 1;
        const uint32_t lo = (a_lo + (uint32_t)sa) | ((uint32_t)(sb - sa) << 16);
        tc::mma_bf16(d_tmem, ((uint64_t)a_hi << 32) | lo,
                     ((uint64_t)b_hi << 32) | (b_lo + (uint32_t)(p * 2 * CH)), idesc,
                     p != 0);
    }
    tc::commit(bar);
}

// The output layer's tap partials of layer-3 tile j (its rows 2j, 2j + 1 of
// buffer A, unshifted): D[pixel][tap] = sum over the 32 channels of
// W3[tap][c] act3[pixel][c], K = 32 in two MMAs of N = 16.
__device__ __forceinline__ void issue_out_taps(uint32_t d_tmem, const uint8_t* a3,
                                               const uint8_t* w, int j, uint32_t bar) {
    constexpr uint32_t idesc = tc::idesc_bf16(128, kNOut);
    const uint64_t a_base = tc::desc_kmajor(tc::smem_u32(a3) + kLead * 16,
                                            kSlotsA * 16, 128);
    const uint64_t b_base = tc::desc_kmajor(tc::smem_u32(w), kNOut * 16, 128);
    const uint32_t a_lo = (uint32_t)a_base + (uint32_t)(2 * j * kRow);
    const uint32_t a_hi = (uint32_t)(a_base >> 32);
    const uint32_t b_lo = (uint32_t)b_base, b_hi = (uint32_t)(b_base >> 32);
#pragma unroll
    for (int kc = 0; kc < CH / 16; ++kc)
        tc::mma_bf16(d_tmem, ((uint64_t)a_hi << 32) | (a_lo + (uint32_t)(2 * kc * kSlotsA)),
                     ((uint64_t)b_hi << 32) | (b_lo + (uint32_t)(2 * kc * kNOut)), idesc,
                     kc != 0);
    tc::commit(bar);
}

// Tiles (two map rows each) of the four layers: every layer's rows shrink
// by one at each side, down to the band's own rows.
__host__ __device__ constexpr int tiles_of(int layer) {
    return layer == 0 ? kARows / 2
                      : layer == 1 ? kBRows / 2 : layer == 2 ? (kBand + 2) / 2 : kBand / 2;
}
static_assert(tiles_of(0) == tiles_of(1) + 1 && tiles_of(1) == tiles_of(2) + 1 &&
                  tiles_of(2) == tiles_of(3) + 1 && tiles_of(0) == kMaxTiles,
              "tile j of a layer reads tiles j and j + 1 of the one before");

// Hidden-layer epilogue of tile j, one warp's lane quarter q: bias, ReLU,
// bf16, into the next layer's input rows (zero outside the map and in
// columns 61..63).  With KEEP (training) the band's own rows y0 .. y0 +
// kBand - 1 also go to act[s][y][x][32] in device memory for the backward
// pass (the halo rows are other bands' own rows).
template <bool KEEP>
__device__ __forceinline__ void epi_hidden_tile(uint32_t t_acc, const float* bias,
                                                int y_first, uint8_t* out,
                                                int slots_out, int j, int q, int lane,
                                                __nv_bfloat16* __restrict__ act,
                                                int s, int y0) {
    const int r = 32 * q + lane, row = 2 * j + (r >> 6), col = r & 63;
    const int Y = y_first + row;
    const bool in_map = Y >= 0 && Y < H && col < W;
    const bool own = KEEP && in_map && Y >= y0 && Y < y0 + kBand;
    uint4* ga = own ? reinterpret_cast<uint4*>(
                          act + ((long long)s * NPIX + Y * W + col) * CH)
                    : nullptr;
    // two halves of 16 columns (fewer live registers)
#pragma unroll
    for (int hlf = 0; hlf < 2; ++hlf) {
        float v[16];
        tc::tmem_ld16(t_acc + ((uint32_t)(32 * q) << 16) + 16 * hlf, v);
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const int k = 2 * hlf + kk;
            uint4 o;
            uint32_t* p = reinterpret_cast<uint32_t*>(&o);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = 8 * kk + 2 * e;
                p[e] = in_map ? pack_bf16(fmaxf(v[c] + bias[16 * hlf + c], 0.f),
                                          fmaxf(v[c + 1] + bias[16 * hlf + c + 1], 0.f))
                              : 0u;
            }
            reinterpret_cast<uint4*>(out)[k * slots_out + kLead + row * kRow + col] = o;
            if (KEEP && own) ga[k] = o;
        }
    }
}

// The partials' epilogue of layer-3 tile j, lane quarter q: the 9 tap
// partials of each of its pixels into shared memory.
__device__ __forceinline__ void epi_out_taps(uint32_t t_acc, float* part, int j, int q,
                                             int lane) {
    float v[16];
    tc::tmem_ld16(t_acc + ((uint32_t)(32 * q) << 16), v);
    const int r = 32 * q + lane, slot = 1 + (2 * j + (r >> 6)) * kRow + (r & 63);
#pragma unroll
    for (int t = 0; t < 9; ++t) part[t * kDStride + slot] = v[t];
}

// Output rows 2i, 2i + 1 of the band (layer-3 rows 2i .. 2i + 3): the 9
// partials at the shifted pixels, plus the bias and the coarse-score input
// channel (channel 1 of the input map).  One pixel a thread of the group.
__device__ __forceinline__ void epi_out_rows(const float* part, float b3,
                                             const __nv_bfloat16* __restrict__ a0,
                                             float* __restrict__ out, int i, int q,
                                             int lane, int s, int y0) {
    const int r = 32 * q + lane, row = 2 * i + (r >> 6), col = r & 63;
    const int Y = y0 + row;
    if (Y >= H || col >= W) return;
    float v = 0.f;
#pragma unroll
    for (int t = 0; t < 9; ++t)
        v += part[t * kDStride + 1 + (row + 1 + t / 3 - 1) * kRow + col + t % 3 - 1];
    const long long p = (long long)s * NPIX + Y * W + col;
    out[p] = v + b3 + __bfloat162float(a0[p * C0 + 1]);
}

// KEEP (training): the hidden activations of each band's own rows also go
// to act1..act3; the inference instance carries none of that.
template <bool KEEP>
__global__ void __launch_bounds__(kThreads, 1)
    tc_forward_kernel(const __grid_constant__ CUtensorMap in_map,
                      const __nv_bfloat16* __restrict__ a0, int n,
                      const __nv_bfloat16* __restrict__ Wf,
                      const float* __restrict__ w32, float* __restrict__ out,
                      int wf1, int wf2, int wf3, int b0, int b1, int b2, int b3,
                      int* __restrict__ err, int withhold,
                      __nv_bfloat16* __restrict__ act1,
                      __nv_bfloat16* __restrict__ act2,
                      __nv_bfloat16* __restrict__ act3) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
    uint8_t* bin = smem;
    uint8_t* ba = smem + kOffA;
    uint8_t* bb = smem + kOffB;
    float* bias = reinterpret_cast<float*>(smem + kOffBias);
    const uint32_t bars = tc::smem_u32(smem + kOffBar);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + kOffTmem);
    volatile int* abort = reinterpret_cast<volatile int*>(smem + kOffAbort);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    auto bar = [&](int i) { return bars + 8u * (uint32_t)i; };

    // activation buffers zeroed: the slots no copy and no epilogue writes
    // (the lead slots, the rows past a layer's last tile) stay zero
    for (int i = threadIdx.x; i < kOffW0 / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    stage_l1_pairs(smem + kOffW0, Wf, threadIdx.x, blockDim.x);
    stage(smem + kOffW1, Wf + wf1, CH, CH, CH, threadIdx.x, blockDim.x);
    stage(smem + kOffW2, Wf + wf2, CH, CH, CH, threadIdx.x, blockDim.x);
    stage_out_taps(smem + kOffW3, Wf + wf3, threadIdx.x, blockDim.x);
    for (int i = threadIdx.x; i < 9 * kDStride; i += blockDim.x)
        reinterpret_cast<float*>(smem + kOffPart)[i] = 0.f;
    for (int i = threadIdx.x; i < 4 * CH; i += blockDim.x) {
        const int l = i / CH, c = i - l * CH;
        const int off = l == 0 ? b0 : l == 1 ? b1 : l == 2 ? b2 : b3;
        bias[i] = (l < 3 || c == 0) ? w32[off + c] : 0.f;
    }
    if (threadIdx.x == 0) *abort = 0;
    if (warp == kEpiWarps) tc::tmem_alloc(tc::smem_u32(tmem_holder), kTmemCols);
    if (threadIdx.x < kNumBars)
        tc::mbar_init(bar(threadIdx.x),
                      threadIdx.x >= kBarEpi && threadIdx.x < kBarInFull ? 4u
                      : threadIdx.x == kBarInFree                       ? (uint32_t)kIssuers
                                                                         : 1u);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_holder;
    const long long units = (long long)n * kBands;
    const uint32_t polls = withhold ? kTestPolls : kWaitPolls;

    if (warp >= kEpiWarps) {
        // the issuers (lane 0 of the last two warps): issuer i issues the
        // tiles j = i, i + 2, ... of every layer, in the order the epilogue
        // warps take them; issuer 0 also loads the input.  withhold (self-
        // test of the bounded waits): nothing is issued, no mbarrier ever
        // completes, every epilogue wait runs out
        const int me = warp - kEpiWarps;
        if (lane == 0 && !withhold) {
            bool ok = true;
            auto wait = [&](int b, uint32_t par) {
                if (ok) ok = tc::mbar_wait_or_abort(bar(b), par, polls, abort);
                return ok;
            };
            auto acc = [&](int L, int j) { return kBarAcc + L * kMaxTiles + j; };
            auto epi = [&](int L, int j) { return kBarEpi + L * kMaxTiles + j; };
            const uint32_t in_s = tc::smem_u32(bin);
            bool tma_out = false;  // an input copy in flight not yet waited for
            uint32_t tma_par = 0;
            if (me == 0 && (long long)blockIdx.x < units) {
                load_band(&in_map, blockIdx.x, in_s, bar(kBarInFull));
                tma_out = true;
            }
            int k = 0;
            for (long long u = blockIdx.x; u < units; u += gridDim.x, ++k) {
                const uint32_t par = (uint32_t)k & 1u, prev = par ^ 1u;
                if (!wait(kBarInFull, par)) break;
                tma_out = false;
                tc::fence_after_sync();
                // layer 1 into half 0: tile j takes the columns of the last
                // band's layer-3 tile j
                for (int j = me; j < tiles_of(0); j += kIssuers) {
                    if (k > 0 && j < tiles_of(2) && !wait(epi(2, j), prev)) break;
                    tc::fence_after_sync();
                    issue_tile_l1(tmem + j * 32, bin, smem + kOffW0, j, bar(acc(0, j)));
                }
                if (!ok) break;
                tc::commit(bar(kBarInFree));  // the input is read once layer 1 is done
                // layer 2 into half 1: tile j reads layer-1 tiles j, j + 1 and
                // takes the columns of the last band's output partials of
                // layer-3 tile j
                for (int j = me; j < tiles_of(1); j += kIssuers) {
                    if (!wait(epi(0, j), par) || !wait(epi(0, j + 1), par)) break;
                    if (k > 0 && j < tiles_of(2) && !wait(epi(3, j), prev)) break;
                    tc::fence_after_sync();
                    issue_tile<CH, CH>(tmem + kTmemHalf + j * 32, ba, kSlotsA, smem + kOffW1,
                                       j, bar(acc(1, j)));
                }
                if (!ok) break;
                // the next band's input rows, once layer 1 (both issuers'
                // tiles) has read these
                if (me == 0 && u + gridDim.x < units) {
                    if (!wait(kBarInFree, par)) break;
                    load_band(&in_map, u + gridDim.x, in_s, bar(kBarInFull));
                    tma_out = true;
                    tma_par = prev;
                }
                // layer 3 into half 0 (the columns of this band's layer 1)
                for (int j = me; j < tiles_of(2); j += kIssuers) {
                    if (!wait(epi(1, j), par) || !wait(epi(1, j + 1), par)) break;
                    tc::fence_after_sync();
                    issue_tile<CH, CH>(tmem + j * 32, bb, kSlotsB, smem + kOffW2, j,
                                       bar(acc(2, j)));
                }
                if (!ok) break;
                // the output layer's tap partials of layer-3 tile j, into
                // half 1 (the columns of this band's layer 2)
                for (int j = me; j < tiles_of(2); j += kIssuers) {
                    if (!wait(epi(2, j), par)) break;
                    tc::fence_after_sync();
                    issue_out_taps(tmem + kTmemHalf + j * 32, ba, smem + kOffW3, j,
                                   bar(acc(3, j)));
                }
                if (!ok) break;
            }
            if (!ok) {
                atomicExch(err, 1);
                *abort = 1;
            }
            // drain: every MMA this thread issued, and an input copy nobody
            // waited for
            tc::commit(bar(kBarDrain + me));
            if (!tc::mbar_wait(bar(kBarDrain + me), 0u, polls)) atomicExch(err, 1);
            if (tma_out && !tc::mbar_wait(bar(kBarInFull), tma_par, polls))
                atomicExch(err, 1);
        }
    } else {
        // epilogue warpgroup g takes every fourth of the band's items, in
        // the order the issuers issue them (three hidden layers' tiles, the
        // output partials of the layer-3 tiles, the output row pairs);
        // warp q of the group reads TMEM lanes 32 q .. 32 q + 31
        const int g = warp >> 2, q = warp & 3;
        float* part = reinterpret_cast<float*>(smem + kOffPart);
        bool ok = true;
        int P = 0, k = 0;
        auto wt = [&](int b, uint32_t par) {
            if (ok) ok = tc::mbar_wait_or_abort(bar(b), par, polls, abort);
            return ok;
        };
        for (long long u = blockIdx.x; u < units && ok; u += gridDim.x, ++k) {
            const int s = (int)(u / kBands);
            const int y0 = (int)(u - (long long)s * kBands) * kBand;
            const uint32_t par = (uint32_t)k & 1u, prev = par ^ 1u;
            for (int L = 0; L < 5 && ok; ++L) {
                const int nt = L < 4 ? tiles_of(L < 3 ? L : 2) : tiles_of(3);
                for (int j = 0; j < nt; ++j, ++P) {
                    if ((P & 3) != g) continue;
                    if (L == 4) {
                        // output rows 2j, 2j + 1: partials of layer-3 tiles
                        // j and j + 1
                        if (!wt(kBarEpi + 3 * kMaxTiles + j, par) ||
                            !wt(kBarEpi + 3 * kMaxTiles + j + 1, par))
                            break;
                        epi_out_rows(part, bias[3 * CH], a0, out, j, q, lane, s, y0);
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(bar(kBarOut + j));
                        continue;
                    }
                    // the partials of tile j overwrite rows that the last
                    // band's output rows j - 1 and j read
                    if (L == 3 && k > 0 &&
                        ((j >= 1 && j - 1 < tiles_of(3) && !wt(kBarOut + j - 1, prev)) ||
                         (j < tiles_of(3) && !wt(kBarOut + j, prev))))
                        break;
                    if (!wt(kBarAcc + L * kMaxTiles + j, par)) break;
                    tc::fence_after_sync();
                    const uint32_t t_acc = tmem + (uint32_t)(L & 1) * kTmemHalf + j * 32;
                    if (L == 0)
                        epi_hidden_tile<KEEP>(t_acc, bias, y0 - 3, ba, kSlotsA, j, q, lane,
                                              act1, s, y0);
                    else if (L == 1)
                        epi_hidden_tile<KEEP>(t_acc, bias + CH, y0 - 2, bb, kSlotsB, j, q,
                                              lane, act2, s, y0);
                    else if (L == 2)
                        epi_hidden_tile<KEEP>(t_acc, bias + 2 * CH, y0 - 1, ba, kSlotsA, j,
                                              q, lane, act3, s, y0);
                    else
                        epi_out_taps(t_acc, part, j, q, lane);
                    // the rows written are the next layer's MMA operands
                    tc::fence_async_smem();
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(bar(kBarEpi + L * kMaxTiles + j));
                }
            }
        }
        if (!ok) {
            atomicExch(err, 1);
            *abort = 1;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == kEpiWarps) tc::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace tcf
}  // namespace net
}  // namespace pps

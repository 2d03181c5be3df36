// pps_net_tc_train.cuh -- the proposal network's training products on the
// 5th-generation tensor cores (tcgen05): the input gradient of a
// convolution (a masked single-layer convolution with the mirrored,
// channel-swapped weights) and the weight and bias gradients (a product
// over every pixel of the batch).  Operands are staged in shared memory in
// the K-major no-swizzle layout (8-row x 16-byte core matrices) and
// multiplied by one thread with tcgen05.mma into FP32 accumulators in
// tensor memory; every mbarrier wait is bounded and a timeout sets the
// network's error flag.
//
// Weight gradient.  dW[tap][co][ci] = sum_p g[p][co] x[p + off(tap)][ci]:
// the pixels are the K of the product, taken two map rows (128 slots of 64
// per row, columns 61..63 zero) at a time.  The tap's row shift dy is a
// start-address offset of 8 core matrices in a window of four rows of
// x^T; its column shift dx is carried by A, which stacks three copies of
// g^T shifted by dx in its rows: A[(dx, co)][q] = g[q - dx][co], so that
// D_dy[(dx, co)][ci] = sum_q g[q - dx][co] x[q + 64 dy][ci] is tap (dy, dx).
// B carries one more row of ones (the real pixels), so D_0[(0, co)][CIN]
// is the bias gradient sum_p g[p][co].  The 8 x 8 transposes from the
// pixel-major activations happen in registers while staging.  Each CTA
// accumulates over its share of the blocks and writes its partial sums; a
// second kernel adds the CTAs' partials in a fixed order, so the gradient
// does not depend on the schedule.
#pragma once

#include "pps_net.cuh"
#include "pps_tc.cuh"

namespace pps {
namespace net {
namespace tct {

constexpr int kThreads = 256;
constexpr int kRow = 64;                 // slots per map row
constexpr uint32_t kWaitPolls = 1u << 22;

// ------------------------------------------------------------ staging
// Transpose 8 pixels x 8 channels (in[i] = 8 channels of pixel i) into
// 8 channels x 8 pixels (out[c] = channel c of the 8 pixels).
__device__ __forceinline__ void transpose8(const uint4 (&in)[8],
                                           uint4 (&out)[8]) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t sel = (c & 1) ? 0x7632u : 0x5410u;
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint4& a = in[2 * j];
            const uint4& b = in[2 * j + 1];
            const uint32_t x = (c >> 1) == 0 ? a.x : (c >> 1) == 1 ? a.y
                               : (c >> 1) == 2 ? a.z : a.w;
            const uint32_t y = (c >> 1) == 0 ? b.x : (c >> 1) == 1 ? b.y
                               : (c >> 1) == 2 ? b.z : b.w;
            w[j] = __byte_perm(x, y, sel);
        }
        out[c] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// 8 channels [cg*8, cg*8+8) of pixel (Y, col) of state s from a
// pixel-major [n][H][W][C] bf16 tensor, zero outside the map.
template <int C>
__device__ __forceinline__ uint4 load8(const __nv_bfloat16* __restrict__ t,
                                       int s, int Y, int col, int cg) {
    if (Y < 0 || Y >= H || col < 0 || col >= W) return make_uint4(0u, 0u, 0u, 0u);
    const long long p = (long long)s * NPIX + Y * W + col;
    return __ldg(reinterpret_cast<const uint4*>(t + p * C) + cg);
}

// ------------------------------------------------------ weight gradient
// Core matrices sit kCm = 144 bytes apart along K (128 of data, 16 of
// padding): a warp's threads each write one core matrix's eight 16-byte
// rows at once, and the padding spreads those writes over all banks.
constexpr int kCm = 144;

template <int CIN, int COUT>
struct WgradShape {
    static constexpr int N = CIN + 16;           // + the ones column group
    static constexpr int kAChunks = 16;          // 128 slots / 8
    static constexpr int kXChunks = 32;          // 4 rows x 64 slots / 8
    static constexpr int kABytes = 16 * kAChunks * kCm;     // 128 rows
    static constexpr int kXBytes = (N / 8) * kXChunks * kCm;
    static constexpr int kStage = kABytes + kXBytes;
    static constexpr int kOffBar = 2 * kStage;
    static constexpr int kOffTmem = kOffBar + 16;
    static constexpr size_t kSmem = kOffTmem + 16;
    static constexpr uint32_t kTmemCols = 3 * N <= 128 ? 128 : 256;
    static_assert(3 * COUT <= 128, "three dx copies of g^T fit M = 128");
    static_assert(3 * N <= 256, "accumulators fit");
    static_assert(kSmem <= 232448, "shared memory");
};

// Stage block (s, yp) -- map rows 2 yp and 2 yp + 1 -- into one buffer.
template <int CIN, int COUT>
__device__ __forceinline__ void wgrad_stage(const __nv_bfloat16* __restrict__ g,
                                            const __nv_bfloat16* __restrict__ x,
                                            int s, int yp, uint8_t* buf) {
    using S = WgradShape<CIN, COUT>;
    constexpr int kCg = COUT / 8, kXg = CIN / 8;
    constexpr int kATasks = 3 * kCg * S::kAChunks;
    constexpr int kXTasks = kXg * S::kXChunks;
    constexpr int kOnes = S::kXChunks;            // the ones row group
    const int y0 = 2 * yp;
    uint8_t* A = buf;
    uint8_t* X = buf + S::kABytes;
    for (int t = threadIdx.x; t < kATasks + kXTasks + kOnes; t += blockDim.x) {
        uint4 in[8], out[8];
        uint8_t* dst;
        if (t < kATasks) {
            // A[(dx, co)][q] = g[q - dx][co], q = 8 c + i (two rows)
            const int c = t % S::kAChunks, r = t / S::kAChunks;
            const int cg = r % kCg, dxi = r / kCg;
            const int dx = dxi - 1;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int q = 8 * c + i - dx;
                const bool ok = q >= 0 && q < 2 * kRow;
                const int row = ok ? q / kRow : 0, col = ok ? q % kRow : W;
                in[i] = load8<COUT>(g, s, y0 + row, col, cg);
            }
            dst = A + ((dxi * kCg + cg) * S::kAChunks + c) * kCm;
        } else if (t < kATasks + kXTasks) {
            // X^T[ci][q], q = -64 + 8 c + i: rows y0 - 1 .. y0 + 2
            const int u = t - kATasks;
            const int c = u % S::kXChunks, cg = u / S::kXChunks;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int q = 8 * c + i;  // 0 .. 255 = row y0 - 1 + q / 64
                in[i] = load8<CIN>(x, s, y0 - 1 + q / kRow, q % kRow, cg);
            }
            dst = X + (cg * S::kXChunks + c) * kCm;
        } else {
            // the ones group: row CIN is 1 at real pixels, the rest 0
            const int c = t - kATasks - kXTasks;
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int q0 = 8 * c + 2 * j;
                const int Y = y0 - 1 + q0 / kRow;
                const int c0 = q0 % kRow, c1 = (q0 + 1) % kRow;
                const bool rowok = Y >= 0 && Y < H;
                const uint32_t lo = rowok && c0 < W ? 0x3F80u : 0u;
                const uint32_t hi = rowok && c1 < W ? 0x3F80u : 0u;
                w[j] = lo | (hi << 16);
            }
            uint4* d = reinterpret_cast<uint4*>(X + (kXg * S::kXChunks + c) * kCm);
            d[0] = make_uint4(w[0], w[1], w[2], w[3]);
#pragma unroll
            for (int k = 1; k < 8; ++k) d[k] = make_uint4(0u, 0u, 0u, 0u);
            continue;
        }
        transpose8(in, out);
        uint4* d = reinterpret_cast<uint4*>(dst);
#pragma unroll
        for (int k = 0; k < 8; ++k) d[k] = out[k];
    }
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads, 1)
    wgrad_tc_kernel(const __nv_bfloat16* __restrict__ g,
                    const __nv_bfloat16* __restrict__ x, int n,
                    float* __restrict__ part, int* __restrict__ err) {
    using S = WgradShape<CIN, COUT>;
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t bars = tc::smem_u32(smem + S::kOffBar);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + S::kOffTmem);
    const int warp = threadIdx.x >> 5;
    // A's rows past the three copies of g^T, and the second group past the
    // ones row, stay zero in both buffers
    for (int i = threadIdx.x; i < 2 * S::kStage / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_holder), S::kTmemCols);
    if (threadIdx.x < 2) tc::mbar_init(bars + 8 * threadIdx.x, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_holder;
    constexpr uint32_t idesc = tc::idesc_bf16(128, S::N);
    const long long blocks = (long long)n * (H / 2);
    uint32_t phase[2] = {0u, 0u};
    bool used[2] = {false, false}, first = true, bad = false;
    int it = 0;
    for (long long b = blockIdx.x; b < blocks; b += gridDim.x, ++it) {
        const int buf = it & 1;
        uint8_t* base = smem + buf * S::kStage;
        // the MMAs that read this buffer two blocks ago must be done
        if (used[buf]) {
            bool ok = true;
            if (threadIdx.x == 0)
                ok = tc::mbar_wait(bars + 8 * buf, phase[buf], kWaitPolls);
            phase[buf] ^= 1u;
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
            tc::fence_after_sync();
        }
        wgrad_stage<CIN, COUT>(g, x, (int)(b / (H / 2)), (int)(b % (H / 2)), base);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc::fence_after_sync();
            const uint64_t a0 = tc::desc_kmajor(tc::smem_u32(base), kCm,
                                                S::kAChunks * kCm);
            const uint64_t x0 = tc::desc_kmajor(tc::smem_u32(base + S::kABytes),
                                                kCm, S::kXChunks * kCm);
            constexpr int u = kCm / 16;   // a chunk in 16-byte units
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                for (int ks = 0; ks < 8; ++ks) {
                    // two chunks per K step of 16
                    const uint64_t a = a0 + (uint64_t)(2 * ks * u);
                    const uint64_t xb = x0 + (uint64_t)((8 + 8 * dy + 2 * ks) * u);
                    tc::mma_bf16(tmem + (uint32_t)((dy + 1) * S::N), a, xb, idesc,
                                 (first && ks == 0) ? 0u : 1u);
                }
            tc::commit(bars + 8 * buf);
        }
        first = false;
        used[buf] = true;
    }
    // wait for the last MMAs of both buffers, then read the accumulators
    bool ok = !bad;
    if (threadIdx.x == 0) {
        for (int k = 0; k < 2 && ok; ++k)
            if (used[k]) ok = tc::mbar_wait(bars + 8 * k, phase[k], kWaitPolls);
    }
    ok = !__syncthreads_or(!ok);
    tc::fence_after_sync();
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(err, 1);
    } else if (warp < 4 && it > 0) {
        // lane m = (dx index) * COUT + co of this warp's quarter
        const int m = 32 * warp + (threadIdx.x & 31);
        const int dxi = m / COUT, co = m - dxi * COUT;
        float* pw = part + (long long)blockIdx.x * (9 * COUT * CIN + COUT);
        for (int dy = 0; dy < 3; ++dy) {
            float v[32];
            for (int c0 = 0; c0 < CIN; c0 += 32) {
                tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) +
                                  (uint32_t)(dy * S::N + c0), v);
                if (dxi < 3) {
                    const int tap = dy * 3 + dxi;
                    for (int i = 0; i < 32 && c0 + i < CIN; ++i)
                        pw[(tap * COUT + co) * CIN + c0 + i] = v[i];
                }
            }
            if (dy == 1) {
                // the bias column (16-column alignment: columns CIN..CIN+15)
                float vb[32];
                tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) +
                                  (uint32_t)(dy * S::N + CIN - 16), vb);
                if (dxi == 1) pw[9 * COUT * CIN + co] = vb[16];
            }
        }
    }
    if (!ok || it == 0) {
        // no partials from this CTA: zeros keep the reduction exact
        float* pw = part + (long long)blockIdx.x * (9 * COUT * CIN + COUT);
        for (int i = threadIdx.x; i < 9 * COUT * CIN + COUT; i += blockDim.x)
            pw[i] = 0.f;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, S::kTmemCols);
}

// grad[layer weights] += sum over the CTAs' partials, in CTA order.
template <int CIN, int COUT>
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int ctas,
                                    float* __restrict__ gw,
                                    float* __restrict__ gb) {
    constexpr int kW = 9 * COUT * CIN, kAll = kW + COUT;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kAll) return;
    float acc = 0.f;
    for (int c = 0; c < ctas; ++c) acc += part[(long long)c * kAll + i];
    if (i < kW)
        gw[i] += acc;
    else
        gb[i - kW] += acc;
}

// ------------------------------------------------------ input gradient
// out[p][co] = (aux[p][co] > 0) ? sum_{tap, ci} Wt[tap][co][ci]
//              in[p + off(tap)][ci] : 0, in bfloat16: the input gradient of
// a layer through the mirrored, channel-swapped weights, masked by the
// ReLU of the layer's input.  Units are (state, band of 8 rows); a band's
// ten input rows sit in shared memory as one plane per 8 channels with 64
// slots per map row (columns 61..63 zero, so a column shift of -1 or +1
// reads a zero at the map's edge), the next unit's rows streaming in with
// cp.async into the other buffer while this one's MMAs run.  A 128-row
// tile is two map rows; the tap (dy, dx) is a start-address offset of
// dy * 64 + dx slots.
constexpr int kBand = 8;
constexpr int kBands = (H + kBand - 1) / kBand;
constexpr int kLead = 8;
constexpr int kInRows = kBand + 2;
constexpr int kSlots = kLead + kInRows * kRow + kLead;
constexpr int kTiles = kBand / 2;

template <int CIN, int COUT>
struct BconvShape {
    static constexpr int kPlanes = CIN / 8;
    static constexpr int kInBytes = kPlanes * kSlots * 16;
    static constexpr int kOffW = 2 * kInBytes;
    static constexpr int kWBytes = 9 * kPlanes * COUT * 16;
    static constexpr int kOffBar = kOffW + kWBytes;
    static constexpr int kOffTmem = kOffBar + 8 * kTiles;
    static constexpr size_t kSmem = kOffTmem + 16;
    static constexpr uint32_t kTmemCols = kTiles * COUT <= 64 ? 64 : 128;
    static_assert(kTiles * COUT <= 128, "accumulators fit");
    static_assert(kSmem <= 232448, "shared memory");
};

template <int CIN>
__device__ __forceinline__ void bconv_prefetch(const __nv_bfloat16* __restrict__ in,
                                               long long u, uint8_t* buf) {
    constexpr int kPlanes = CIN / 8;
    const int s = (int)(u / kBands);
    const int y0 = (int)(u - (long long)s * kBands) * kBand;
    const __nv_bfloat16* src = in + (long long)s * NPIX * CIN;
    for (int i = threadIdx.x; i < kInRows * W * kPlanes; i += blockDim.x) {
        const int pl = i % kPlanes, q = i / kPlanes;
        const int r = q / W, x = q - r * W;
        const int Y = y0 - 1 + r;
        const bool ok = Y >= 0 && Y < H;
        const __nv_bfloat16* gsrc = src + ((ok ? Y : 0) * W + x) * CIN + pl * 8;
        const uint32_t d =
            tc::smem_u32(buf + (pl * kSlots + kLead + r * kRow + x) * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d),
                     "l"(gsrc), "r"(ok ? 16 : 0));
    }
    asm volatile("cp.async.commit_group;");
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads, 1)
    bconv_tc_kernel(const __nv_bfloat16* __restrict__ in, int n,
                    const __nv_bfloat16* __restrict__ Wt,
                    const __nv_bfloat16* __restrict__ aux,
                    __nv_bfloat16* __restrict__ out, int* __restrict__ err) {
    using S = BconvShape<CIN, COUT>;
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t bars = tc::smem_u32(smem + S::kOffBar);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + S::kOffTmem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // both input buffers zero once: the lead and trail slots and columns
    // 61..63 are never written again
    for (int i = threadIdx.x; i < S::kOffW / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    {
        // weights [tap][co][ci] -> [tap][ci / 8][co] x 16 bytes
        constexpr int kChunks = CIN / 8, total = 9 * kChunks * COUT;
        for (int i = threadIdx.x; i < total; i += blockDim.x) {
            const int co = i % COUT, rest = i / COUT;
            const int ch = rest % kChunks, tap = rest / kChunks;
            reinterpret_cast<uint4*>(smem + S::kOffW)[(tap * kChunks + ch) * COUT + co] =
                reinterpret_cast<const uint4*>(Wt)[(tap * COUT + co) * kChunks + ch];
        }
    }
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_holder), S::kTmemCols);
    if (threadIdx.x < kTiles) tc::mbar_init(bars + 8 * threadIdx.x, 1);
    __syncthreads();   // the zeroing is done before any cp.async lands
    tc::fence_before_sync();
    const long long units = (long long)n * kBands;
    if (blockIdx.x < units) bconv_prefetch<CIN>(in, blockIdx.x, smem);
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_holder;
    constexpr uint32_t idesc = tc::idesc_bf16(128, COUT);
    uint32_t phase = 0;  // parity of the tiles' next completion (all tiles alike)
    bool bad = false;
    int it = 0;
    for (long long u = blockIdx.x; u < units; u += gridDim.x, ++it) {
        const int s = (int)(u / kBands);
        const int y0 = (int)(u - (long long)s * kBands) * kBand;
        uint8_t* cur = smem + (it & 1) * S::kInBytes;
        asm volatile("cp.async.wait_all;" ::: "memory");
        tc::fence_async_smem();
        tc::fence_before_sync();
        if (__syncthreads_or(bad)) break;
        if (threadIdx.x == 0) {
            tc::fence_after_sync();
            const uint64_t a_base = tc::desc_kmajor(
                tc::smem_u32(cur) + kLead * 16, kSlots * 16, 128);
            const uint64_t b_base =
                tc::desc_kmajor(tc::smem_u32(smem + S::kOffW), COUT * 16, 128);
            for (int j = 0; j < kTiles; ++j) {
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
#pragma unroll
                    for (int kc = 0; kc < CIN / 16; ++kc) {
                        const long long a_off = (long long)(2 * kc) * kSlots +
                                                (2 * j + 1 + dy) * kRow + dx;
                        const long long b_off =
                            (long long)(tap * (CIN / 8) + 2 * kc) * COUT;
                        tc::mma_bf16(tmem + j * COUT, a_base + (uint64_t)a_off,
                                     b_base + (uint64_t)b_off, idesc,
                                     (tap | kc) != 0);
                    }
                }
                tc::commit(bars + 8 * j);
            }
        }
        // the next unit's rows stream into the other buffer meanwhile (its
        // last readers, the previous unit's MMAs, completed before that
        // unit's epilogue ended)
        if (u + gridDim.x < units)
            bconv_prefetch<CIN>(in, u + gridDim.x,
                                smem + ((it + 1) & 1) * S::kInBytes);
        // epilogue: a warp serves one lane quarter of a tile once that
        // tile's accumulators are complete
        bool ok = true;
        const int q = warp & 3;
        for (int j = warp >> 2; j < kTiles; j += kThreads / 128) {
            ok = ok && tc::mbar_wait(bars + 8 * j, phase, kWaitPolls);
            tc::fence_after_sync();
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + j * COUT, v);
            const int r = 32 * q + lane, row = 2 * j + (r >> 6), col = r & 63;
            const int Y = y0 + row;
            if (!ok || Y >= H || col >= W) continue;
            const long long p = (long long)s * NPIX + Y * W + col;
            const uint4* m4 = reinterpret_cast<const uint4*>(aux + p * COUT);
            uint4* o4 = reinterpret_cast<uint4*>(out + p * COUT);
#pragma unroll
            for (int k = 0; k < COUT / 8; ++k) {
                const uint4 mk = __ldg(m4 + k);
                const uint32_t mw[4] = {mk.x, mk.y, mk.z, mk.w};
                uint32_t ow[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int c = 8 * k + 2 * e;
                    // a bfloat16 is > 0 when its sign bit is clear and it
                    // is not +0 (the activations are ReLU outputs)
                    const bool p0 = (mw[e] & 0xFFFFu) != 0u && !(mw[e] & 0x8000u);
                    const bool p1 = (mw[e] >> 16) != 0u && !(mw[e] & 0x80000000u);
                    ow[e] = pack_bf16(p0 ? v[c] : 0.f, p1 ? v[c + 1] : 0.f);
                }
                o4[k] = make_uint4(ow[0], ow[1], ow[2], ow[3]);
            }
        }
        phase ^= 1u;
        tc::fence_before_sync();
        if (__syncthreads_or(!ok)) {
            bad = true;
            if (threadIdx.x == 0) atomicExch(err, 1);
            break;
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, S::kTmemCols);
}

}  // namespace tct
}  // namespace net
}  // namespace pps

// pps_net.cuh -- device code of the learned proposal network.
//
// A 4-layer 3x3 convolutional network on the 46 x 61 map of a 12 x 9 m
// field (0.2 m pixels): 8 input channels -> 32 -> 32 -> 32 -> 1, ReLU after
// the hidden layers, bfloat16 weights and activations, float32
// accumulation.  Every convolution -- forward, input gradient and weight
// gradient -- is an implicit GEMM on the tensor cores (mma.sync m16n8k16,
// bf16 x bf16 -> f32).  Activations are stored pixel-major (NHWC) with the
// channel count padded to a multiple of 16 (the input map carries 8 zero
// channels; the output layer 15 zero channels), so one 32-bit load fetches
// the two consecutive channels an mma fragment register holds.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pps.h"
#include "pps_cells.cuh"
#include "pps_search.cuh"

namespace pps {
namespace net {

constexpr int H = 46, W = 61, NPIX = H * W;
constexpr int C0 = 16;  // padded input channels (8 used)
constexpr int CH = 32;  // hidden channels
constexpr int CO = 16;  // padded output channels (1 used)
constexpr float kSigOpp = 0.3f;

// Padded parameter layout (float32 master copy): per layer W[9][cout][cin]
// then bias[cout].
__host__ __device__ constexpr int lcin(int l) { return l == 0 ? C0 : CH; }
__host__ __device__ constexpr int lcout(int l) { return l == 3 ? CO : CH; }
__host__ __device__ constexpr int layer_size(int l) {
    return 9 * lcout(l) * lcin(l) + lcout(l);
}
__host__ __device__ constexpr int layer_off(int l) {
    return l == 0 ? 0 : layer_off(l - 1) + layer_size(l - 1);
}
constexpr int kPadParams = layer_off(4);

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0,
                                         uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ------------------------------------------------------------ rasteriser
// Kick speeds and value-function parameters the input features are
// computed for (the network is trained for one such set).
struct RasterCfg {
    float sp[PPS_MAX_SPEEDS], sp2[PPS_MAX_SPEEDS];
    int V;
    pps_params prm;
};
constexpr int kFeatK = 16;          // pass-line samples of the features
static_assert((kFeatK & (kFeatK - 1)) == 0, "1 / kFeatK must be exact");
constexpr float kScoreFloor = -1.2f;  // below every score of a 12 x 9 m field
constexpr float kSubOff = 0.05f;      // sub-points: the cell's quadrant centres

// The cell features of the pixel centred at (cx, cy), each the largest over
// its four sub-points (cx +- 0.05, cy +- 0.05) (clamped into the field);
// with LANES = 4 this lane takes sub-point sub0 alone and the caller takes
// the largest across the four lanes that share the pixel:
// f[0] the coarse score (the value function with the margin of kFeatK
// samples; kScoreFloor where no speed is feasible), f[1] the margin (best
// speed, clamped to [-2, 1]), f[2] the open shot angle / pi.
// The opponents' scaled pairs, read from the CTA's shared copy with 16-byte
// loads that stay inside the sample loop (two pairs a load; the same
// arithmetic and minimum tree as opp_min).
__device__ __forceinline__ float4 lds4(const void* p) {
    float4 v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(a));
    return v;
}

template <int J, bool GEN>
__device__ __forceinline__ float opp_min_shared(float f, float cbx, float cby,
                                                const OppRegs<J>& o, float reach) {
    static_assert(J % 4 == 0, "pairs are read two at a time");
    const float2 f2 = make_float2(f, f), cx2 = make_float2(cbx, cbx),
                 cy2 = make_float2(cby, cby);
    float t[J];
#pragma unroll
    for (int i = 0; i < J / 2; i += 2) {
        const float4 bx = lds4(&o.bx[i]), by = lds4(&o.by[i]);
        const float4 ux = lds4(&o.ux[i]), uy = lds4(&o.uy[i]);
        float2 r = sbip_num2<GEN>(f2, cx2, cy2, make_float2(bx.x, bx.y),
                                  make_float2(by.x, by.y), make_float2(ux.x, ux.y),
                                  make_float2(uy.x, uy.y), reach);
        t[2 * i] = r.x;
        t[2 * i + 1] = r.y;
        r = sbip_num2<GEN>(f2, cx2, cy2, make_float2(bx.z, bx.w),
                           make_float2(by.z, by.w), make_float2(ux.z, ux.w),
                           make_float2(uy.z, uy.w), reach);
        t[2 * i + 2] = r.x;
        t[2 * i + 3] = r.y;
    }
#pragma unroll
    for (int w = 1; w < J; w *= 2)
#pragma unroll
        for (int j = 0; j + w < J; j += 2 * w) t[j] = fminf(t[j], t[j + w]);
    return t[0];
}

// o: the state's opponents (OppRegs<J> as load_opps fills it), in the CTA's
// shared memory.
// VMAX: speed slots (4 or 8; the slots past cfg.V repeat the last speed
// and are left out of the margin), the ball terms of two speeds a packed
// f32x2 instruction.
template <int J, bool GEN, int VMAX, int LANES>
__device__ __forceinline__ void cell_features(const pps_state& st,
                                              const StateK& sk,
                                              const OppRegs<J>& o,
                                              const RasterCfg& cfg, float cx,
                                              float cy, int sub0, float (&f)[3]) {
    constexpr int VP = VMAX / 2;
    float2 s2[VP];
#pragma unroll
    for (int i = 0; i < VP; ++i)
        s2[i] = make_float2(cfg.sp2[2 * i], cfg.sp2[2 * i + 1]);  // padded already
    const float hw = 0.5f * st.field_wid;
    float mbest = -CUDART_INF_F, tbest = 0.f, sbest = kScoreFloor;
#pragma unroll 1
    for (int sub = sub0; sub < 4; sub += LANES) {
        const float qx =
            fminf(fmaxf(cx + ((sub & 1) ? kSubOff : -kSubOff), -sk.Lh), sk.Lh);
        const float qy =
            fminf(fmaxf(cy + ((sub & 2) ? kSubOff : -kSubOff), -hw), hw);
        const float dx = qx - sk.bx, dy = qy - sk.by;
        const float D = sqrtf(dx * dx + dy * dy);
        const float cbx = sk.kappa * dx, cby = sk.kappa * dy;
        const float twoabD = sk.two_ab * D;
        float2 mv2[VP];
#pragma unroll
        for (int i = 0; i < VP; ++i) mv2[i] = make_float2(CUDART_INF_F, CUDART_INF_F);
#pragma unroll 1
        for (int k = 1; k <= kFeatK; ++k) {
            const float fr = (float)k * (1.f / kFeatK);  // exact: kFeatK = 2^n
            const float aT =
                __fmul_rn(opp_min_shared<J, GEN>(fr, cbx, cby, o, sk.reach), sk.at_scale);
            const float nf = __fmul_rn(-fr, twoabD);
            const float2 nf2 = make_float2(nf, nf), aT2 = make_float2(aT, aT);
#pragma unroll
            for (int i = 0; i < VP; ++i) {
                const float2 a = __fadd2_rn(s2[i], nf2);
                const float2 t = __fadd2_rn(aT2, make_float2(sqrt_ball(fmaxf(a.x, 0.f)),
                                                              sqrt_ball(fmaxf(a.y, 0.f))));
                mv2[i] = make_float2(fminf(mv2[i].x, t.x), fminf(mv2[i].y, t.y));
            }
        }
        float mv[VMAX];
#pragma unroll
        for (int i = 0; i < VP; ++i) {
            mv[2 * i] = mv2[i].x;
            mv[2 * i + 1] = mv2[i].y;
        }
        float m = -CUDART_INF_F;
#pragma unroll
        for (int v = 0; v < VMAX; ++v) {
            if (v >= cfg.V) continue;
            float mm;
            if (cfg.sp2[v] - twoabD < 0.f)
                mm = -CUDART_INF_F;
            else if (sk.nopp == 0)
                mm = CUDART_INF_F;
            else
                mm = (mv[v] - cfg.sp[v]) / sk.ab;
            m = fmaxf(m, mm);
        }
        const float th = shot_angle<J>(st, sk, qx < sk.Lh, qx, qy, sk.Lh - qx,
                                       cfg.prm.robot_radius) *
                         0.318309886183790672f;
        const float gx = sk.Lh - qx;
        const float dg = sqrtf(gx * gx + qy * qy) * sk.inv_diag;
        const bool feas = m > cfg.prm.tau_safe && D >= cfg.prm.min_pass_dist;
        const float sc = feas ? cfg.prm.w_angle * th - cfg.prm.w_dist * dg +
                                    cfg.prm.w_margin * fminf(m, cfg.prm.margin_cap)
                              : kScoreFloor;
        mbest = fmaxf(mbest, m);
        tbest = fmaxf(tbest, th);
        sbest = fmaxf(sbest, sc);
    }
    f[0] = sbest;
    f[1] = fminf(fmaxf(mbest, -2.f), 1.f);
    f[2] = tbest;
}

// One thread a (state, pixel): the 8 input channels of the pixel centred
// at c = ((x - 30) / 5, (y - 22.5) / 5), bf16, written as 16-channel rows
// (channels 8..15 zero):
//   0  sum_j exp(-|c - o_j|^2 / (2 0.3^2))      opponent density
//   1  coarse score of the cell  (cell_features f[0])
//   2  |c - b| / diag
//   3  margin of the cell        (f[1])
//   4  shot angle of the cell    (f[2])
//   5  |goal centre - c| / diag
//   6  c_x / (L / 2),  7  c_y / (W / 2)
// Every CTA covers pixels of one state (kRasterCtas CTAs a state): one
// thread derives the state's constants and scales its opponents into
// shared memory, and the pixels read them from there (broadcasts) instead
// of each thread deriving them and holding the opponents in registers.
// LANES lanes a pixel: 1 (each lane the pixel's four sub-points in turn;
// the most work a CTA, for large batches) or 4 (a lane a sub-point, the
// features' maxima taken across the four: a quarter of the serial chain,
// for batches that leave most of the GPU idle).
constexpr int kRasterTpb = 128;
template <int LANES>
__host__ __device__ constexpr int raster_ctas() {
    return (NPIX + kRasterTpb / LANES - 1) / (kRasterTpb / LANES);
}

// A state's derived constants and scaled opponents as the rasteriser's CTAs
// hold them (the 8-slot layout when it has at most 8 opponents), prepared
// once a call by one thread a state for the large-batch instance: its 22
// CTAs a state otherwise each derived them on one thread while the other
// warps waited.
struct __align__(16) RasterRec {
    StateK sk;
    __align__(16) unsigned char opp[sizeof(OppRegs<PPS_MAX_OPP>)];
};
static_assert(sizeof(RasterRec) % 16 == 0, "copied 16 bytes a thread");

__device__ __forceinline__ void raster_derive(const pps_state& st,
                                              const RasterCfg& cfg,
                                              StateK& sk, unsigned char* opp) {
    sk = derive_state(st, cfg.prm, PPS_MAX_OPP, PPS_MAX_K);
    if (sk.nopp <= 8)
        load_opps<8>(st, sk, *reinterpret_cast<OppRegs<8>*>(opp));
    else
        load_opps<PPS_MAX_OPP>(st, sk, *reinterpret_cast<OppRegs<PPS_MAX_OPP>*>(opp));
}

__global__ void __launch_bounds__(128)
    raster_prepare_kernel(const pps_state* __restrict__ states, int n,
                          const RasterCfg cfg, RasterRec* __restrict__ recs) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    RasterRec r;
    raster_derive(states[s], cfg, r.sk, r.opp);
    recs[s] = r;
}

// recs (may be null): the states' records from raster_prepare_kernel.
template <int LANES>
__global__ void __launch_bounds__(kRasterTpb, 8)
    raster_kernel(const pps_state* __restrict__ states, int n,
                              const RasterCfg cfg,
                              __nv_bfloat16* __restrict__ out,
                              const RasterRec* __restrict__ recs) {
    constexpr int kPix = kRasterTpb / LANES, kCtas = raster_ctas<LANES>();
    constexpr int kStateWords = (int)(sizeof(pps_state) / 4);
    static_assert(sizeof(pps_state) % 4 == 0 && kStateWords <= kRasterTpb,
                  "the state is copied a 32-bit word a thread");
    __shared__ RasterRec s_rec;
    StateK& s_sk = s_rec.sk;
    unsigned char* s_opp = s_rec.opp;
    __shared__ __align__(16) pps_state s_st;
    const int s = (int)(blockIdx.x / kCtas);
    const int sub = LANES == 4 ? (int)(threadIdx.x & 3) : 0;
    const int q = (int)(blockIdx.x - (unsigned)s * kCtas) * kPix +
                  (int)(threadIdx.x / LANES);
    // the state in shared memory, a word a thread (one memory latency, not
    // the chain of field loads the derivation would wait on)
    constexpr int kRecChunks = (int)(sizeof(RasterRec) / 16);
    static_assert(kRecChunks <= kRasterTpb, "one 16-byte chunk a thread");
    if (threadIdx.x < kStateWords)
        reinterpret_cast<uint32_t*>(&s_st)[threadIdx.x] =
            __ldg(reinterpret_cast<const uint32_t*>(states + s) + threadIdx.x);
    if (recs && threadIdx.x < kRecChunks)
        reinterpret_cast<uint4*>(&s_rec)[threadIdx.x] =
            __ldg(reinterpret_cast<const uint4*>(recs + s) + threadIdx.x);
    __syncthreads();
    const pps_state& st = s_st;
    if (!recs) {
        if (threadIdx.x == 0) raster_derive(st, cfg, s_rec.sk, s_rec.opp);
        __syncthreads();
    }
    // lanes past the map's last pixel still take part in the shuffles below
    const bool active = q < NPIX;
    const int qa = active ? q : NPIX - 1;
    const long long i = (long long)s * NPIX + qa;
    const int y = qa / W, x = qa - y * W;
    const float cx = __fdiv_rn((float)(x - 30), 5.f);
    const float cy = __fdiv_rn(__fsub_rn((float)y, 22.5f), 5.f);
    const StateK& sk = s_sk;

    float f[3] = {kScoreFloor, -2.f, 0.f};
    if (sk.valid && active) {
        const auto& o8 = *reinterpret_cast<const OppRegs<8>*>(s_opp);
        const auto& o16 = *reinterpret_cast<const OppRegs<PPS_MAX_OPP>*>(s_opp);
        if (cfg.V <= 4) {
            if (sk.nopp <= 8)
                sk.general ? cell_features<8, true, 4, LANES>(st, sk, o8, cfg, cx, cy, sub, f)
                           : cell_features<8, false, 4, LANES>(st, sk, o8, cfg, cx, cy, sub, f);
            else
                sk.general ? cell_features<PPS_MAX_OPP, true, 4, LANES>(st, sk, o16, cfg, cx, cy, sub, f)
                           : cell_features<PPS_MAX_OPP, false, 4, LANES>(st, sk, o16, cfg, cx, cy, sub, f);
        } else {
            if (sk.nopp <= 8)
                sk.general ? cell_features<8, true, 8, LANES>(st, sk, o8, cfg, cx, cy, sub, f)
                           : cell_features<8, false, 8, LANES>(st, sk, o8, cfg, cx, cy, sub, f);
            else
                sk.general ? cell_features<PPS_MAX_OPP, true, 8, LANES>(st, sk, o16, cfg, cx, cy, sub, f)
                           : cell_features<PPS_MAX_OPP, false, 8, LANES>(st, sk, o16, cfg, cx, cy, sub, f);
        }
    }
    // the largest over the pixel's four sub-points (maxima are exact; the
    // margin's clamp is monotone, so the clamp of the largest is the largest
    // clamp)
    if (LANES == 4) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int off = 1; off < 4; off <<= 1)
                f[k] = fmaxf(f[k], __shfl_xor_sync(0xffffffffu, f[k], off));
    }
    if (!active || sub != 0) return;

    float dens = 0.f;
    for (int j = 0; j < sk.nopp; ++j) {
        const float dx = cx - st.opp_pos[j][0], dy = cy - st.opp_pos[j][1];
        dens += expf(-(dx * dx + dy * dy) / (2.f * kSigOpp * kSigOpp));
    }
    const float dxm = cx - sk.bx, dym = cy - sk.by;
    const float gx = sk.Lh - cx;
    float c[8];
    c[0] = dens;
    c[1] = f[0];
    c[2] = sqrtf(dxm * dxm + dym * dym) * sk.inv_diag;
    c[3] = f[1];
    c[4] = f[2];
    c[5] = sqrtf(gx * gx + cy * cy) * sk.inv_diag;
    c[6] = cx / (0.5f * st.field_len);
    c[7] = cy / (0.5f * st.field_wid);
    uint4 lo, hi;
    lo.x = pack_bf16(c[0], c[1]);
    lo.y = pack_bf16(c[2], c[3]);
    lo.z = pack_bf16(c[4], c[5]);
    lo.w = pack_bf16(c[6], c[7]);
    hi.x = hi.y = hi.z = hi.w = 0u;
    uint4* op = reinterpret_cast<uint4*>(out + i * C0);
    op[0] = lo;
    op[1] = hi;
}

// Input maps between the caller's 8-channel layout and the kernels'
// 16-channel rows (channels 8..15 zero): one thread per pixel, 16 bytes in,
// 32 out (or 32 in, 16 out).
__global__ void widen_map_kernel(const uint4* __restrict__ in8, long long n_pix,
                                 uint4* __restrict__ out16) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pix) return;
    out16[2 * i] = in8[i];
    out16[2 * i + 1] = make_uint4(0u, 0u, 0u, 0u);
}

__global__ void narrow_map_kernel(const uint4* __restrict__ in16,
                                  long long n_pix, uint4* __restrict__ out8) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pix) return;
    out8[i] = in16[2 * i];
}

// --------------------------------------------------------- convolution
// Epilogues of the implicit-GEMM convolution.
enum Epi {
    kHidden = 0,  // + bias, ReLU, bf16 out (hidden layers)
    kOutput = 1,  // + bias + the input map's coarse score (channel 1 of
                  // aux), channel 0 as float32 (output layer)
    kMaskedGrad = 2  // input gradient: bf16(acc) where aux (the layer's
                     // input) > 0
};

// out[p][co] = sum over taps and ci of Wt[tap][co][ci] * in[p + off(tap)][ci]
// for every pixel p of n images (aux: the layer input that masks an input
// gradient, or the input map whose coarse score the output adds); a CTA of 4 warps owns 64 consecutive
// pixels, each warp 16 of them across all COUT output channels.
template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(128)
    conv_kernel(const __nv_bfloat16* __restrict__ in,
                const __nv_bfloat16* __restrict__ Wt,
                const float* __restrict__ bias, long long n_pix,
                void* __restrict__ out,
                const __nv_bfloat16* __restrict__ aux) {
    static_assert(CIN % 16 == 0 && COUT % 8 == 0, "padded channel counts");
    __shared__ __align__(16) __nv_bfloat16 sw[9 * COUT * CIN];
    for (int i = threadIdx.x; i < 9 * COUT * CIN / 8; i += blockDim.x)
        reinterpret_cast<uint4*>(sw)[i] = reinterpret_cast<const uint4*>(Wt)[i];
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    const long long p0 = (long long)blockIdx.x * 64 + warp * 16;
    // the two pixel rows this thread's A fragments cover
    long long pr[2];
    int yy[2], xx[2];
    for (int h = 0; h < 2; ++h) {
        pr[h] = p0 + gid + 8 * h;
        const long long q = pr[h] < n_pix ? pr[h] % NPIX : 0;
        yy[h] = (int)(q / W);
        xx[h] = (int)(q - (long long)yy[h] * W);
    }
    constexpr int NT = COUT / 8;
    float acc[NT][4];
#pragma unroll
    for (int t = 0; t < NT; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;

#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        const uint32_t* src[2];
        bool ok[2];
        for (int h = 0; h < 2; ++h) {
            const int y2 = yy[h] + dy, x2 = xx[h] + dx;
            ok[h] = pr[h] < n_pix && y2 >= 0 && y2 < H && x2 >= 0 && x2 < W;
            const long long pn = pr[h] + dy * W + dx;
            src[h] = reinterpret_cast<const uint32_t*>(in + (ok[h] ? pn : 0) * CIN);
        }
#pragma unroll
        for (int kc = 0; kc < CIN / 16; ++kc) {
            const int k0 = kc * 16 + tig * 2;
            const uint32_t a0 = ok[0] ? __ldg(src[0] + k0 / 2) : 0u;
            const uint32_t a1 = ok[1] ? __ldg(src[1] + k0 / 2) : 0u;
            const uint32_t a2 = ok[0] ? __ldg(src[0] + k0 / 2 + 4) : 0u;
            const uint32_t a3 = ok[1] ? __ldg(src[1] + k0 / 2 + 4) : 0u;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const __nv_bfloat16* wrow = sw + (tap * COUT + t * 8 + gid) * CIN + k0;
                const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wrow);
                const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wrow + 8);
                mma_bf16(acc[t], a0, a1, a2, a3, b0, b1);
            }
        }
    }
    // epilogue: thread holds (row gid, cols 2tig, 2tig+1) and (row gid+8, ..)
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int c = t * 8 + tig * 2;
        for (int h = 0; h < 2; ++h) {
            const long long p = pr[h];
            if (p >= n_pix) continue;
            float v0 = acc[t][2 * h], v1 = acc[t][2 * h + 1];
            if (EPI == kHidden) {
                v0 = fmaxf(v0 + bias[c], 0.f);
                v1 = fmaxf(v1 + bias[c + 1], 0.f);
                reinterpret_cast<uint32_t*>(out)[(p * COUT + c) / 2] = pack_bf16(v0, v1);
            } else if (EPI == kOutput) {
                if (t == 0 && tig == 0)
                    reinterpret_cast<float*>(out)[p] =
                        v0 + bias[0] + __bfloat162float(aux[p * C0 + 1]);
            } else {
                const __nv_bfloat162 m = reinterpret_cast<const __nv_bfloat162*>(
                    aux)[(p * COUT + c) / 2];
                v0 = __bfloat162float(m.x) > 0.f ? v0 : 0.f;
                v1 = __bfloat162float(m.y) > 0.f ? v1 : 0.f;
                reinterpret_cast<uint32_t*>(out)[(p * COUT + c) / 2] = pack_bf16(v0, v1);
            }
        }
    }
}

// ------------------------------------------------------------ training
// Per state: the largest label of its map.
__global__ void __launch_bounds__(256)
    state_max_kernel(const float* __restrict__ label,
                     float* __restrict__ smax) {
    __shared__ float red[8];
    const float* l = label + (long long)blockIdx.x * NPIX;
    float m = -CUDART_INF_F;
    for (int i = threadIdx.x; i < NPIX; i += blockDim.x) m = fmaxf(m, l[i]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
        smax[blockIdx.x] = fmaxf(m, red[0]);
    }
}

// Top-focused, asymmetric mean squared error over n_pix pixels: pixel p of
// state s weighs 1 where its label or its prediction comes within top_band
// of the state's best label smax[s], low_w elsewhere, times under_w where
// the prediction is below the label (the weight is a constant of the
// gradient).  The loss (accumulated) and its gradient 2 w (out - label) /
// n_pix into channel 0 of a CO-channel bf16 map.
__global__ void loss_kernel(const float* __restrict__ out,
                            const float* __restrict__ label,
                            const float* __restrict__ smax, long long n_pix,
                            float inv_n, float top_band, float low_w,
                            float under_w, __nv_bfloat16* __restrict__ g,
                            float* __restrict__ loss_sum) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float sq = 0.f;
    if (i < n_pix) {
        const float o = out[i], l = label[i];
        const float cut = smax[i / NPIX] - top_band;
        const float d = o - l;
        const float w = ((l >= cut || o >= cut) ? 1.f : low_w) *
                        (d < 0.f ? under_w : 1.f);
        sq = w * d * d * inv_n;
        uint4 lo = {pack_bf16(2.f * w * d * inv_n, 0.f), 0u, 0u, 0u};
        uint4 z = {0u, 0u, 0u, 0u};
        uint4* op = reinterpret_cast<uint4*>(g + i * CO);
        op[0] = lo;
        op[1] = z;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss_sum, sq);
}

__device__ __forceinline__ uint32_t pair16(const __nv_bfloat16* base,
                                           long long i0, bool ok0,
                                           long long i1, bool ok1) {
    const unsigned short* b = reinterpret_cast<const unsigned short*>(base);
    const uint32_t lo = ok0 ? __ldg(b + i0) : 0u;
    const uint32_t hi = ok1 ? __ldg(b + i1) : 0u;
    return lo | (hi << 16);
}

// dW[tap][co][ci] += sum over pixels p of g[p][co] * x[p + off(tap)][ci]
// (x zero outside its image).  One warp per tap; the CTA owns `chunk`
// consecutive pixels; the warp's 16-pixel steps are the K of the mma
// (A = g transposed: co x pixels, B = shifted x: pixels x ci).
template <int CIN, int COUT>
__global__ void __launch_bounds__(288)
    wgrad_kernel(const __nv_bfloat16* __restrict__ g,
                 const __nv_bfloat16* __restrict__ x, long long n_pix,
                 int chunk, float* __restrict__ dW) {
    static_assert(CIN % 8 == 0 && COUT % 16 == 0, "padded channel counts");
    constexpr int MT = COUT / 16, NT = CIN / 8;
    const int lane = threadIdx.x & 31, tap = threadIdx.x >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const long long pbeg = (long long)blockIdx.x * chunk;
    const long long pend = pbeg + chunk < n_pix ? pbeg + chunk : n_pix;
    float acc[MT][NT][4];
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int t = 0; t < NT; ++t) acc[m][t][0] = acc[m][t][1] = acc[m][t][2] = acc[m][t][3] = 0.f;

    for (long long pk = pbeg; pk < pend; pk += 16) {
        // the four K positions (pixels) of this thread: 2tig, 2tig+1, +8, +9
        long long pp[4], nb[4];
        bool okg[4], okx[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            pp[e] = pk + 2 * tig + (e & 1) + 8 * (e >> 1);
            okg[e] = pp[e] < pend;
            const long long q = okg[e] ? pp[e] % NPIX : 0;
            const int y = (int)(q / W), xx = (int)(q - (long long)y * W);
            const int y2 = y + dy, x2 = xx + dx;
            okx[e] = okg[e] && y2 >= 0 && y2 < H && x2 >= 0 && x2 < W;
            nb[e] = okx[e] ? pp[e] + dy * W + dx : 0;
        }
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            const int co = m * 16 + gid;
            const uint32_t a0 = pair16(g, pp[0] * COUT + co, okg[0], pp[1] * COUT + co, okg[1]);
            const uint32_t a1 = pair16(g, pp[0] * COUT + co + 8, okg[0], pp[1] * COUT + co + 8, okg[1]);
            const uint32_t a2 = pair16(g, pp[2] * COUT + co, okg[2], pp[3] * COUT + co, okg[3]);
            const uint32_t a3 = pair16(g, pp[2] * COUT + co + 8, okg[2], pp[3] * COUT + co + 8, okg[3]);
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int ci = t * 8 + gid;
                const uint32_t b0 = pair16(x, nb[0] * CIN + ci, okx[0], nb[1] * CIN + ci, okx[1]);
                const uint32_t b1 = pair16(x, nb[2] * CIN + ci, okx[2], nb[3] * CIN + ci, okx[3]);
                mma_bf16(acc[m][t], a0, a1, a2, a3, b0, b1);
            }
        }
    }
    float* base = dW + (long long)tap * COUT * CIN;
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int r = m * 16 + gid, c = t * 8 + tig * 2;
            atomicAdd(base + r * CIN + c, acc[m][t][0]);
            atomicAdd(base + r * CIN + c + 1, acc[m][t][1]);
            atomicAdd(base + (r + 8) * CIN + c, acc[m][t][2]);
            atomicAdd(base + (r + 8) * CIN + c + 1, acc[m][t][3]);
        }
}

// db[c] += sum over pixels of g[p][c].
template <int C>
__global__ void bias_grad_kernel(const __nv_bfloat16* __restrict__ g,
                                 long long n_pix, float* __restrict__ db) {
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = 0.f;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n_pix;
         p += (long long)gridDim.x * blockDim.x) {
        const __nv_bfloat162* row = reinterpret_cast<const __nv_bfloat162*>(g + p * C);
#pragma unroll
        for (int c = 0; c < C / 2; ++c) {
            const float2 v = __bfloat1622float2(row[c]);
            acc[2 * c] += v.x;
            acc[2 * c + 1] += v.y;
        }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
        float v = acc[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) atomicAdd(db + c, v);
    }
}

// Adam on the padded float32 parameters; clears the gradient.
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ grad,
                            float* __restrict__ m, float* __restrict__ v,
                            int n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    grad[i] = 0.f;
}

// bf16 copies of the weights: Wf[l][tap][co][ci] for the forward pass and
// WT[l][8 - tap][ci][co] (taps mirrored, channels swapped) for the input
// gradient, which is the same convolution run backwards.
__global__ void cast_kernel(const float* __restrict__ w,
                            __nv_bfloat16* __restrict__ Wf,
                            __nv_bfloat16* __restrict__ WT) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int l = 0, base = 0, wbase = 0;
    int rem = i;
    for (l = 0; l < 4; ++l) {
        const int nw = 9 * lcout(l) * lcin(l);
        if (rem < nw) break;
        rem -= nw;
        base += layer_size(l);
        wbase += nw;
    }
    if (l == 4) return;
    const int cin = lcin(l), cout = lcout(l);
    const int tap = rem / (cout * cin);
    const int co = (rem / cin) % cout, ci = rem % cin;
    const __nv_bfloat16 b = __float2bfloat16_rn(w[base + rem]);
    Wf[wbase + rem] = b;
    WT[wbase + ((8 - tap) * cin + ci) * cout + co] = b;
}

// Labels: per map pixel, the best exact score of the fine grid points of
// its cell (cell_lattice), floored; cells without points get the floor.
__global__ void cell_label_kernel(const float* __restrict__ point_best,
                                  int n, int fnx, int fny, int m, int ox,
                                  int oy, float floor_v,
                                  float* __restrict__ labels) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * NPIX) return;
    const int s = (int)(i / NPIX), q = (int)(i - (long long)s * NPIX);
    const int cy = q / W, cx = q - cy * W;
    const float* pb = point_best + (long long)s * fnx * fny;
    float best = floor_v;
    for (int dy = 0; dy < m; ++dy) {
        const int fy = m * cy + oy + dy;
        if (fy < 0 || fy >= fny) continue;
        for (int dx = 0; dx < m; ++dx) {
            const int fx = m * cx + ox + dx;
            if (fx < 0 || fx >= fnx) continue;
            best = fmaxf(best, pb[(long long)fy * fnx + fx]);
        }
    }
    labels[i] = best;
}

// Top-k map pixels of every state (one CTA per state), best first; equal
// scores keep the smaller pixel.  Keys are (order-preserving score bits,
// ~pixel), all distinct: a radix select (8-bit digits, most significant
// first; it stops at the first digit whose keys are all needed) finds the
// k-th largest key T, the k keys >= T are compacted, and only those are
// ordered: up to 512 of them each go straight to its rank (the number of
// selected keys above it, counted by several threads a key), more are
// sorted by a bitonic network (next power of two).  1024 threads: a state
// alone on the GPU (one frame) is latency-bound, and each thread holds at
// most three pixels.
constexpr int kTopkThreads = 1024;
constexpr int kTopkIters = (NPIX + kTopkThreads - 1) / kTopkThreads;

__device__ __forceinline__ unsigned long long topk_key(const float* sc, int i) {
    uint32_t u = __float_as_uint(sc[i]);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (uint32_t)(~(uint32_t)i);
}

// With jobs, a pixel whose cell holds no point of the state's grid (a field
// smaller than the map's 12 x 9 m) ranks below every pixel that does: its
// key keeps only ~pixel, so it is taken only when k exceeds the cells that
// hold points.
__global__ void __launch_bounds__(kTopkThreads)
    topk_kernel(const float* __restrict__ scores, int k, int p2,
                int* __restrict__ cells, const pps_job* __restrict__ jobs) {
    extern __shared__ __align__(16) unsigned long long tk[];
    unsigned long long* key = tk;         // NPIX keys
    unsigned long long* sel = tk + NPIX;  // p2 selected keys
    __shared__ int hist[256];
    __shared__ int warp_sum[8];
    __shared__ unsigned long long s_prefix;
    __shared__ int s_need, s_count, s_done;
    const int s = blockIdx.x, t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const float* sc = scores + (long long)s * NPIX;
    // the pixels' keys (all loads in flight at once)
    if (jobs) {
        const pps_grid g = jobs[s].grid;
        const CellLattice cl = cell_lattice(g);
#pragma unroll
        for (int it = 0; it < kTopkIters; ++it) {
            const int i = it * kTopkThreads + t;
            if (i < NPIX) {
                const int cy = i / W, cx = i - cy * W;
                key[i] = cl.ok && cell_on_grid(cl, g, cx, cy)
                             ? topk_key(sc, i)
                             : (unsigned long long)(~(uint32_t)i);
            }
        }
    } else {
#pragma unroll
        for (int it = 0; it < kTopkIters; ++it) {
            const int i = it * kTopkThreads + t;
            if (i < NPIX) key[i] = topk_key(sc, i);
        }
    }
    if (t == 0) {
        s_prefix = 0ull;
        s_need = k;
        s_count = 0;
        s_done = 0;
    }
    __syncthreads();
    unsigned long long mask = 0ull;
    for (int shift = 56; shift >= 0 && k < NPIX; shift -= 8) {
        if (t < 256) hist[t] = 0;
        __syncthreads();
        const unsigned long long prefix = s_prefix;
#pragma unroll
        for (int it = 0; it < kTopkIters; ++it) {
            const int i = it * kTopkThreads + t;
            if (i < NPIX) {
                const unsigned long long v = key[i];
                if ((v & mask) == prefix)
                    atomicAdd(&hist[(v >> shift) & 255u], 1);
            }
        }
        __syncthreads();
        // counts of digits 255 - t, inclusive scan from the top digit down
        // (the first 256 threads)
        int own = 0, incl = 0;
        if (t < 256) {
            own = hist[255 - t];
            incl = own;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += y;
            }
            if (lane == 31) warp_sum[warp] = incl;
        }
        __syncthreads();
        const int need = s_need;
        if (t < 256) {
            for (int w = 0; w < warp; ++w) incl += warp_sum[w];
        }
        __syncthreads();
        if (t < 256 && incl >= need && incl - own < need) {  // exactly one thread
            s_prefix = prefix | ((unsigned long long)(255 - t) << shift);
            s_need = need - (incl - own);
            // every key of the new prefix is needed: the prefix (its lower
            // bits zero) is a threshold that selects exactly k keys
            s_done = s_need == own;
        }
        mask |= 0xFFull << shift;
        __syncthreads();
        if (s_done) break;
    }
    // the k-th largest key (or every key when k == NPIX)
    const unsigned long long T = k < NPIX ? s_prefix : 0ull;
    for (int i = t; i < p2; i += kTopkThreads) sel[i] = 0ull;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kTopkIters; ++it) {
        const int i = it * kTopkThreads + t;
        const unsigned long long v = i < NPIX ? key[i] : 0ull;
        const bool take = i < NPIX && v >= T;
        const unsigned b = __ballot_sync(0xffffffffu, take);
        int at = 0;
        if (lane == 0 && b) at = atomicAdd(&s_count, __popc(b));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (take) sel[at + __popc(b & ((1u << lane) - 1u))] = v;
    }
    __syncthreads();
    if (k <= 512) {
        // exactly k keys (all distinct): Q threads per key (Q a power of
        // two, k Q <= 1024) each count the keys above it among every Q-th
        // one, summed across the Q adjacent lanes
        int Q = 32;
        while (Q > 1 && Q * k > kTopkThreads) Q >>= 1;
        const int i = t / Q, part = t & (Q - 1);
        const unsigned long long v = i < k ? sel[i] : 0ull;
        int r = 0;
        if (i < k)
            for (int j = part; j < k; j += Q) r += sel[j] > v;
        for (int off = Q >> 1; off > 0; off >>= 1)
            r += __shfl_xor_sync(0xffffffffu, r, off);
        if (i < k && part == 0)
            cells[(long long)s * k + r] = (int)(~(uint32_t)(v & 0xffffffffull));
        return;
    }
    for (int size = 2; size <= p2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = t; i < p2; i += kTopkThreads) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool desc = (i & size) == 0;
                    const unsigned long long a = sel[i], b = sel[j];
                    if (desc ? a < b : a > b) {
                        sel[i] = b;
                        sel[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = t; i < k; i += kTopkThreads)
        cells[(long long)s * k + i] = (int)(~(uint32_t)(sel[i] & 0xffffffffull));
}

}  // namespace net
}  // namespace pps

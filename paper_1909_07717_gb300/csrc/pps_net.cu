// pps_net.cu -- host side of the learned proposal network (include/pps.h,
// "Learned proposal"): buffers, the weight layouts, forward, backward and
// the Adam step, all enqueued on the network's stream.

#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "pps.h"
#include "pps_internal.h"
#include "pps_net.cuh"
#include "pps_net_tc.cuh"
#include "pps_net_tc_train.cuh"

using namespace pps::net;
char* pps_thread_error_buffer();

struct pps_net {
    int device = 0;
    int num_sms = 1;
    cudaStream_t stream = nullptr;
    int max_batch = 0;
    int step = 0;
    float *w = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *Wf = nullptr, *WT = nullptr;
    __nv_bfloat16 *a0 = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr;
    __nv_bfloat16 *g1 = nullptr, *g2 = nullptr, *g3 = nullptr, *g4 = nullptr;
    float* out = nullptr;
    float* loss = nullptr;
    int* cells = nullptr;  // proposal scratch: max_batch x NPIX
    int* skip = nullptr;   // proposal scratch: max_batch
    void* srec = nullptr;  // proposal scratch: max_batch per-state records
    RasterRec* rrec = nullptr;  // the rasteriser's per-state records
    int* list = nullptr;   // proposal scratch: max_batch states to re-search
    // proposal scratch: the work queue's counter, then (in the next 8
    // bytes, so that one memset clears both) the list's length
    unsigned long long* queue = nullptr;
    int* list_n = nullptr;
    float* smax = nullptr; // training scratch: max_batch best labels
    int* err = nullptr;    // set by a kernel whose bounded wait ran out
    float* wpart = nullptr;  // weight-gradient partial sums, one row per CTA
    int train_kind = PPS_NET_TRAIN_TCGEN05;
    RasterCfg cfg{};       // speeds and parameters of the input features
    float top_band = 3.0e38f, low_w = 1.f, under_w = 1.f;  // the loss
    CUtensorMap in_map{};  // a0 as the forward kernel's tensor-memory-
                           // accelerator source (encoded once, at create)
};

namespace {

constexpr int kWeights = 9 * (C0 * CH + CH * CH + CH * CH + CH * CO);
// real (unpadded) channel counts of the flat host layout
constexpr int kRealIn[4] = {8, 32, 32, 32}, kRealOut[4] = {32, 32, 32, 1};

int wf_off(int l) {
    int o = 0;
    for (int i = 0; i < l; ++i) o += 9 * lcout(i) * lcin(i);
    return o;
}
int bias_off(int l) { return layer_off(l) + 9 * lcout(l) * lcin(l); }

pps_status fail(pps_status s, const char* msg, cudaError_t e = cudaSuccess) {
    std::snprintf(pps_thread_error_buffer(), 512, "%s%s%s", msg,
                  e != cudaSuccess ? ": " : "",
                  e != cudaSuccess ? cudaGetErrorString(e) : "");
    return s;
}

constexpr float kDefaultSpeeds[4] = {2.f, 3.5f, 5.f, 6.5f};

void set_cfg(RasterCfg& c, const float* speeds, int n, const pps_params* prm) {
    for (int v = 0; v < PPS_MAX_SPEEDS; ++v) {
        const float sv = speeds[v < n ? v : n - 1];
        c.sp[v] = sv;
        c.sp2[v] = sv * sv;
    }
    c.V = n;
    if (prm)
        c.prm = *prm;
    else
        pps_default_params(&c.prm);
}

unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t cast_weights(pps_net* nt) {
    cast_kernel<<<blocks(kWeights, 256), 256, 0, nt->stream>>>(nt->w, nt->Wf,
                                                               nt->WT);
    return cudaGetLastError();
}

// The input map of n states into nt->a0: rasterised from the states, or
// The rasteriser of n states into nt->a0: a lane a pixel when that fills a
// wave of the GPU's resident CTAs, else four lanes a pixel (a quarter of
// the serial chain for the small batches of serving; same results).
void launch_raster(pps_net* nt, const pps_state* states, int n, cudaStream_t st) {
    if ((long long)n * raster_ctas<1>() >= 8LL * nt->num_sms) {
        // large batches: the states' records prepared once a call
        raster_prepare_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
            states, n, nt->cfg, nt->rrec);
        raster_kernel<1><<<(unsigned)(n * raster_ctas<1>()), kRasterTpb, 0, st>>>(
            states, n, nt->cfg, nt->a0, nt->rrec);
    } else {
        raster_kernel<4><<<(unsigned)(n * raster_ctas<4>()), kRasterTpb, 0, st>>>(
            states, n, nt->cfg, nt->a0, nullptr);
    }
}

// (states NULL) copied from a caller's map[n][46][61][8] bf16 into the
// 16-channel rows the kernels read (channels 8..15 zero).
cudaError_t load_input(pps_net* nt, const pps_state* states,
                       const uint16_t* map, int n) {
    const long long P = (long long)n * NPIX;
    cudaStream_t st = nt->stream;
    if (states) {
        launch_raster(nt, states, n, st);
        return cudaGetLastError();
    }
    if ((reinterpret_cast<uintptr_t>(map) & 15) != 0)
        return cudaErrorMisalignedAddress;  // maps are read 16 bytes a pixel
    widen_map_kernel<<<blocks(P, 256), 256, 0, st>>>(
        reinterpret_cast<const uint4*>(map), P, reinterpret_cast<uint4*>(nt->a0));
    return cudaGetLastError();
}

// Forward pass of the map in nt->a0 into nt->out.  layers: layer by layer
// on mma.sync, every activation written to device memory; otherwise the
// fused tcgen05 kernel, which keeps the activations on the SM -- or, with
// keep (training), also writes them for the backward pass.
cudaError_t forward_loaded(pps_net* nt, int n, bool layers, bool keep = false,
                           bool withhold = false) {
    const long long P = (long long)n * NPIX;
    const unsigned g = blocks(P, 64);
    cudaStream_t st = nt->stream;
    if (!layers) {
        auto kernel = keep ? tcf::tc_forward_kernel<true>
                           : tcf::tc_forward_kernel<false>;
        cudaError_t e = cudaFuncSetAttribute(
            kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
            (int)tcf::kSmemBytes);
        if (e != cudaSuccess) return e;
        const long long units = (long long)n * tcf::kBands;
        const unsigned grid =
            (unsigned)(units < nt->num_sms ? units : nt->num_sms);
        kernel<<<grid, tcf::kThreads, tcf::kSmemBytes, st>>>(
            nt->in_map, nt->a0, n, nt->Wf, nt->w, nt->out, wf_off(1), wf_off(2), wf_off(3),
            bias_off(0), bias_off(1), bias_off(2), bias_off(3), nt->err,
            withhold ? 1 : 0, nt->a1, nt->a2, nt->a3);
        return cudaGetLastError();
    }
    conv_kernel<C0, CH, kHidden><<<g, 128, 0, st>>>(
        nt->a0, nt->Wf + wf_off(0), nt->w + bias_off(0), P, nt->a1, nullptr);
    conv_kernel<CH, CH, kHidden><<<g, 128, 0, st>>>(
        nt->a1, nt->Wf + wf_off(1), nt->w + bias_off(1), P, nt->a2, nullptr);
    conv_kernel<CH, CH, kHidden><<<g, 128, 0, st>>>(
        nt->a2, nt->Wf + wf_off(2), nt->w + bias_off(2), P, nt->a3, nullptr);
    conv_kernel<CH, CO, kOutput><<<g, 128, 0, st>>>(
        nt->a3, nt->Wf + wf_off(3), nt->w + bias_off(3), P, nt->out, nt->a0);
    return cudaGetLastError();
}

// Forward pass of n states (or, states NULL, of a caller's input map).
cudaError_t forward(pps_net* nt, const pps_state* states, int n, bool layers,
                    bool withhold = false, const uint16_t* map = nullptr) {
    cudaError_t e = load_input(nt, states, map, n);
    return e == cudaSuccess ? forward_loaded(nt, n, layers, false, withhold) : e;
}

// The forward pass of a training step: every activation kept for the
// backward pass, by the kernels of the network's training kind.
cudaError_t forward_train(pps_net* nt, const pps_state* states, int n,
                          const uint16_t* map = nullptr) {
    cudaError_t e = load_input(nt, states, map, n);
    if (e != cudaSuccess) return e;
    return nt->train_kind == PPS_NET_TRAIN_TCGEN05
               ? forward_loaded(nt, n, false, true)
               : forward_loaded(nt, n, true);
}

// The tcgen05 training products of one layer: weight and bias gradients of
// layer l from g (its output gradient) and x (its input), accumulated into
// nt->grad; and, for l > 0, the masked input gradient g_in.
template <int CIN, int COUT>
cudaError_t wgrad_tc(pps_net* nt, int l, const __nv_bfloat16* g,
                     const __nv_bfloat16* x, int n) {
    using S = tct::WgradShape<CIN, COUT>;
    cudaError_t e = cudaFuncSetAttribute(
        tct::wgrad_tc_kernel<CIN, COUT>,
        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kSmem);
    if (e != cudaSuccess) return e;
    const long long nb = (long long)n * (H / 2);
    const int grid = (int)(nb < nt->num_sms ? nb : nt->num_sms);
    tct::wgrad_tc_kernel<CIN, COUT><<<grid, tct::kThreads, S::kSmem,
                                      nt->stream>>>(g, x, n, nt->wpart,
                                                    nt->err);
    constexpr int kAll = 9 * COUT * CIN + COUT;
    tct::wgrad_reduce_kernel<CIN, COUT><<<blocks(kAll, 256), 256, 0,
                                          nt->stream>>>(
        nt->wpart, grid, nt->grad + layer_off(l), nt->grad + bias_off(l));
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t bconv_tc(pps_net* nt, const __nv_bfloat16* g,
                     const __nv_bfloat16* Wt, const __nv_bfloat16* aux,
                     __nv_bfloat16* out, int n) {
    using S = tct::BconvShape<CIN, COUT>;
    cudaError_t e = cudaFuncSetAttribute(
        tct::bconv_tc_kernel<CIN, COUT>,
        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kSmem);
    if (e != cudaSuccess) return e;
    const long long units = (long long)n * tct::kBands;
    const int grid = (int)(units < nt->num_sms ? units : nt->num_sms);
    tct::bconv_tc_kernel<CIN, COUT><<<grid, tct::kThreads, S::kSmem,
                                      nt->stream>>>(g, n, Wt, aux, out,
                                                    nt->err);
    return cudaGetLastError();
}

// The backward pass on tcgen05 (the loss gradient g4 already written).
cudaError_t backward_tc(pps_net* nt, int n) {
    cudaError_t e = wgrad_tc<CH, CO>(nt, 3, nt->g4, nt->a3, n);
    if (e == cudaSuccess)
        e = bconv_tc<CO, CH>(nt, nt->g4, nt->WT + wf_off(3), nt->a3, nt->g3, n);
    if (e == cudaSuccess) e = wgrad_tc<CH, CH>(nt, 2, nt->g3, nt->a2, n);
    if (e == cudaSuccess)
        e = bconv_tc<CH, CH>(nt, nt->g3, nt->WT + wf_off(2), nt->a2, nt->g2, n);
    if (e == cudaSuccess) e = wgrad_tc<CH, CH>(nt, 1, nt->g2, nt->a1, n);
    if (e == cudaSuccess)
        e = bconv_tc<CH, CH>(nt, nt->g2, nt->WT + wf_off(1), nt->a1, nt->g1, n);
    if (e == cudaSuccess) e = wgrad_tc<C0, CH>(nt, 0, nt->g1, nt->a0, n);
    return e;
}

// Gradients of the mean squared error into nt->grad (accumulated).
cudaError_t backward(pps_net* nt, const float* labels, int n) {
    const long long P = (long long)n * NPIX;
    const unsigned g = blocks(P, 64);
    const int chunk = 2048;
    const unsigned gw = blocks(P, chunk);
    cudaStream_t st = nt->stream;
    cudaError_t e = cudaMemsetAsync(nt->loss, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    state_max_kernel<<<n, 256, 0, st>>>(labels, nt->smax);
    loss_kernel<<<blocks(P, 256), 256, 0, st>>>(nt->out, labels, nt->smax, P,
                                                1.f / (float)P, nt->top_band,
                                                nt->low_w, nt->under_w, nt->g4,
                                                nt->loss);
    if (nt->train_kind == PPS_NET_TRAIN_TCGEN05) {
        e = cudaGetLastError();
        return e == cudaSuccess ? backward_tc(nt, n) : e;
    }
    // layer 4 (32 -> 1)
    wgrad_kernel<CH, CO><<<gw, 288, 0, st>>>(nt->g4, nt->a3, P, chunk,
                                              nt->grad + layer_off(3));
    bias_grad_kernel<CO><<<256, 256, 0, st>>>(nt->g4, P, nt->grad + bias_off(3));
    conv_kernel<CO, CH, kMaskedGrad><<<g, 128, 0, st>>>(
        nt->g4, nt->WT + wf_off(3), nullptr, P, nt->g3, nt->a3);
    // layer 3
    wgrad_kernel<CH, CH><<<gw, 288, 0, st>>>(nt->g3, nt->a2, P, chunk,
                                              nt->grad + layer_off(2));
    bias_grad_kernel<CH><<<256, 256, 0, st>>>(nt->g3, P, nt->grad + bias_off(2));
    conv_kernel<CH, CH, kMaskedGrad><<<g, 128, 0, st>>>(
        nt->g3, nt->WT + wf_off(2), nullptr, P, nt->g2, nt->a2);
    // layer 2
    wgrad_kernel<CH, CH><<<gw, 288, 0, st>>>(nt->g2, nt->a1, P, chunk,
                                              nt->grad + layer_off(1));
    bias_grad_kernel<CH><<<256, 256, 0, st>>>(nt->g2, P, nt->grad + bias_off(1));
    conv_kernel<CH, CH, kMaskedGrad><<<g, 128, 0, st>>>(
        nt->g2, nt->WT + wf_off(1), nullptr, P, nt->g1, nt->a1);
    // layer 1 (8 -> 32; the input needs no gradient)
    wgrad_kernel<C0, CH><<<gw, 288, 0, st>>>(nt->g1, nt->a0, P, chunk,
                                              nt->grad + layer_off(0));
    bias_grad_kernel<CH><<<256, 256, 0, st>>>(nt->g1, P, nt->grad + bias_off(0));
    return cudaGetLastError();
}

// flat host layout <-> padded device layout
void to_padded(const float* flat, std::vector<float>& pad) {
    pad.assign(kPadParams, 0.f);
    int k = 0;
    for (int l = 0; l < 4; ++l) {
        const int ci_r = kRealIn[l], co_r = kRealOut[l];
        const int cin = lcin(l), cout = lcout(l);
        for (int tap = 0; tap < 9; ++tap)
            for (int co = 0; co < co_r; ++co)
                for (int ci = 0; ci < ci_r; ++ci)
                    pad[layer_off(l) + (tap * cout + co) * cin + ci] = flat[k++];
        for (int co = 0; co < co_r; ++co) pad[bias_off(l) + co] = flat[k++];
    }
}

void from_padded(const std::vector<float>& pad, float* flat) {
    int k = 0;
    for (int l = 0; l < 4; ++l) {
        const int ci_r = kRealIn[l], co_r = kRealOut[l];
        const int cin = lcin(l), cout = lcout(l);
        for (int tap = 0; tap < 9; ++tap)
            for (int co = 0; co < co_r; ++co)
                for (int ci = 0; ci < ci_r; ++ci)
                    flat[k++] = pad[layer_off(l) + (tap * cout + co) * cin + ci];
        for (int co = 0; co < co_r; ++co) flat[k++] = pad[bias_off(l) + co];
    }
}

}  // namespace

static_assert(PPS_NET_PARAMS == 21121, "flat layout");

// Library-internal: predicted scores of n states (into the net's buffer),
// and the proposal scratch.
cudaError_t pps_net_predict(pps_net* nt, const pps_state* states, int n,
                            cudaStream_t* st, float** scores, int** cells,
                            pps_net_scratch* scratch) {
    *st = nt->stream;
    *scores = nt->out;
    *cells = nt->cells;
    scratch->skip = nt->skip;
    scratch->list = nt->list;
    scratch->list_n = nt->list_n;
    scratch->queue = nt->queue;
    scratch->srec = nt->srec;
    return forward(nt, states, n, false);
}

int pps_net_max_batch(const pps_net* nt) { return nt->max_batch; }

cudaError_t pps_net_topk(pps_net* nt, int n, int k, int* cells,
                         const pps_job* jobs) {
    int p2 = 1;
    while (p2 < k) p2 <<= 1;
    const size_t smem = sizeof(unsigned long long) * (size_t)(NPIX + p2);
    cudaError_t e = cudaFuncSetAttribute(
        topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    topk_kernel<<<n, kTopkThreads, smem, nt->stream>>>(nt->out, k, p2, cells,
                                                       jobs);
    return cudaGetLastError();
}

namespace {
// The input map a0 ([max_batch][H][W][16 channels] bf16) as a 5-D tiled
// tensor map: channels 0..7 (16 bytes), the two halves of 8 channels, the
// W columns, the H rows, the states.  The forward kernel copies one box of
// 8 channels x 64 columns x its band's input rows a plane; what lies
// outside the map (columns 61..63, rows above and below) reads as zero.
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*,
                                 const cuuint32_t*, const cuuint32_t*,
                                 CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t encode_input_map(pps_net* nt) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    const cuuint64_t dims[5] = {8, 2, (cuuint64_t)W, (cuuint64_t)H,
                                (cuuint64_t)nt->max_batch};
    const cuuint64_t strides[4] = {16, 2 * 16, (cuuint64_t)W * 32,
                                   (cuuint64_t)NPIX * 32};
    const cuuint32_t box[5] = {8, 1, (cuuint32_t)tcf::kRow, (cuuint32_t)tcf::kInRows, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = reinterpret_cast<EncodeTiled>(fn)(
        &nt->in_map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, nt->a0, dims, strides, box,
        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
        CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
}  // namespace

extern "C" pps_status pps_net_create(int device, void* stream, int max_batch,
                                     pps_net** out) {
    if (!out) return PPS_EINVAL;
    *out = nullptr;
    if (max_batch < 1 || max_batch > (1 << 16))
        return fail(PPS_EINVAL, "pps_net_create: max_batch outside 1..65536");
    pps_net* nt = new (std::nothrow) pps_net();
    if (!nt) return PPS_ENOMEM;
    nt->device = device;
    nt->stream = (cudaStream_t)stream;
    nt->max_batch = max_batch;
    set_cfg(nt->cfg, kDefaultSpeeds, 4, nullptr);
    const size_t P = (size_t)max_batch * NPIX;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&nt->num_sms, cudaDevAttrMultiProcessorCount,
                                   device);
    auto al = [&](auto** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc((void**)p, bytes);
        if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
    };
    al(&nt->w, sizeof(float) * kPadParams);
    al(&nt->grad, sizeof(float) * kPadParams);
    al(&nt->m, sizeof(float) * kPadParams);
    al(&nt->v, sizeof(float) * kPadParams);
    al(&nt->Wf, sizeof(__nv_bfloat16) * kWeights);
    al(&nt->WT, sizeof(__nv_bfloat16) * kWeights);
    al(&nt->a0, sizeof(__nv_bfloat16) * P * C0);
    al(&nt->a1, sizeof(__nv_bfloat16) * P * CH);
    al(&nt->a2, sizeof(__nv_bfloat16) * P * CH);
    al(&nt->a3, sizeof(__nv_bfloat16) * P * CH);
    al(&nt->g1, sizeof(__nv_bfloat16) * P * CH);
    al(&nt->g2, sizeof(__nv_bfloat16) * P * CH);
    al(&nt->g3, sizeof(__nv_bfloat16) * P * CH);
    al(&nt->g4, sizeof(__nv_bfloat16) * P * CO);
    al(&nt->out, sizeof(float) * P);
    al(&nt->loss, sizeof(float));
    al(&nt->cells, sizeof(int) * P);
    al(&nt->skip, sizeof(int) * (size_t)max_batch);
    al(&nt->srec, kPpsStateRecBytes * (size_t)max_batch);
    al(&nt->rrec, sizeof(RasterRec) * (size_t)max_batch);
    al(&nt->smax, sizeof(float) * (size_t)max_batch);
    al(&nt->list, sizeof(int) * (size_t)max_batch);
    al(&nt->queue, 2 * sizeof(unsigned long long));
    if (nt->queue) nt->list_n = reinterpret_cast<int*>(nt->queue + 1);
    al(&nt->err, sizeof(int));
    al(&nt->wpart, sizeof(float) * (size_t)(nt->num_sms > 0 ? nt->num_sms : 1) *
                       (9 * CH * CH + CH));
    if (e == cudaSuccess) e = encode_input_map(nt);
    if (e != cudaSuccess) {
        cudaGetLastError();
        pps_net_destroy(nt);
        return fail(e == cudaErrorMemoryAllocation ? PPS_ENOMEM : PPS_ECUDA,
                    "pps_net_create", e);
    }
    *out = nt;
    return PPS_OK;
}

extern "C" void pps_net_destroy(pps_net* nt) {
    if (!nt) return;
    cudaSetDevice(nt->device);
    cudaStreamSynchronize(nt->stream);
    for (void* p : {(void*)nt->w, (void*)nt->grad, (void*)nt->m, (void*)nt->v,
                    (void*)nt->Wf, (void*)nt->WT, (void*)nt->a0, (void*)nt->a1,
                    (void*)nt->a2, (void*)nt->a3, (void*)nt->g1, (void*)nt->g2,
                    (void*)nt->g3, (void*)nt->g4, (void*)nt->out,
                    (void*)nt->loss, (void*)nt->cells, (void*)nt->skip,
                    nt->srec, (void*)nt->rrec,
                    (void*)nt->smax, (void*)nt->list, (void*)nt->err,
                    (void*)nt->wpart, (void*)nt->queue})
        if (p) cudaFree(p);
    cudaGetLastError();
    delete nt;
}

extern "C" pps_status pps_net_set_weights(pps_net* nt, const float* w) {
    if (!nt || !w) return PPS_EINVAL;
    for (int i = 0; i < PPS_NET_PARAMS; ++i)
        if (!std::isfinite(w[i]))
            return fail(PPS_EINVAL, "pps_net_set_weights: non-finite weight");
    std::vector<float> pad;
    to_padded(w, pad);
    cudaSetDevice(nt->device);
    cudaError_t e = cudaMemcpyAsync(nt->w, pad.data(), sizeof(float) * kPadParams,
                                    cudaMemcpyHostToDevice, nt->stream);
    for (float* p : {nt->grad, nt->m, nt->v})
        if (e == cudaSuccess)
            e = cudaMemsetAsync(p, 0, sizeof(float) * kPadParams, nt->stream);
    if (e == cudaSuccess) e = cast_weights(nt);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nt->stream);
    nt->step = 0;
    return e == cudaSuccess ? PPS_OK : fail(PPS_ECUDA, "pps_net_set_weights", e);
}

extern "C" pps_status pps_net_sync(pps_net* nt) {
    if (!nt) return PPS_EINVAL;
    cudaSetDevice(nt->device);
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, nt->err, sizeof(int),
                                    cudaMemcpyDeviceToHost, nt->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nt->stream);
    if (e != cudaSuccess) return fail(PPS_ECUDA, "pps_net_sync", e);
    if (flag) {
        cudaMemsetAsync(nt->err, 0, sizeof(int), nt->stream);
        cudaStreamSynchronize(nt->stream);
        return fail(PPS_ETIMEOUT,
                    "pps_net_sync: a tensor-core wait ran out; outputs invalid");
    }
    return PPS_OK;
}

extern "C" pps_status pps_net_set_features(pps_net* nt, const float* speeds,
                                           int n_speeds,
                                           const pps_params* params) {
    if (!nt || !speeds || n_speeds < 1 || n_speeds > PPS_MAX_SPEEDS)
        return fail(PPS_EINVAL, "pps_net_set_features: 1..8 speeds");
    for (int v = 0; v < n_speeds; ++v)
        if (!std::isfinite(speeds[v]) || !(speeds[v] > 0.f))
            return fail(PPS_EINVAL, "pps_net_set_features: speeds must be > 0");
    if (params) {
        const float pv[] = {params->w_angle, params->w_dist, params->w_margin,
                            params->margin_cap, params->tau_safe,
                            params->robot_radius, params->reach_radius,
                            params->min_pass_dist};
        for (float x : pv)
            if (!std::isfinite(x))
                return fail(PPS_EINVAL, "pps_net_set_features: params must be finite");
        if (params->robot_radius < 0.f || params->reach_radius < 0.f)
            return fail(PPS_EINVAL, "pps_net_set_features: negative radius");
    }
    set_cfg(nt->cfg, speeds, n_speeds, params);
    return PPS_OK;
}

extern "C" pps_status pps_net_set_loss(pps_net* nt, float top_band,
                                       float low_weight, float under_weight) {
    if (!nt || !(top_band > 0.f) || !(low_weight >= 0.f && low_weight <= 1.f) ||
        !(under_weight >= 1.f && under_weight <= 1e3f))
        return fail(PPS_EINVAL,
                    "pps_net_set_loss: top_band > 0, low_weight in [0, 1], "
                    "under_weight in [1, 1000]");
    nt->top_band = std::isinf(top_band) ? 3.0e38f : top_band;
    nt->low_w = low_weight;
    nt->under_w = under_weight;
    return PPS_OK;
}

extern "C" pps_status pps_net_get_weights(pps_net* nt, float* w) {
    if (!nt || !w) return PPS_EINVAL;
    std::vector<float> pad(kPadParams);
    cudaSetDevice(nt->device);
    cudaError_t e = cudaMemcpyAsync(pad.data(), nt->w, sizeof(float) * kPadParams,
                                    cudaMemcpyDeviceToHost, nt->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nt->stream);
    if (e != cudaSuccess) return fail(PPS_ECUDA, "pps_net_get_weights", e);
    from_padded(pad, w);
    return PPS_OK;
}

namespace {
pps_status check_batch(const pps_net* nt, const void* states, int n) {
    if (!nt) return PPS_EINVAL;
    if (n < 1 || n > nt->max_batch)
        return fail(PPS_EINVAL, "pps_net: n outside 1..max_batch");
    if (!states) return fail(PPS_EINVAL, "pps_net: states is NULL");
    return PPS_OK;
}
}  // namespace

extern "C" pps_status pps_net_selftest_timeout(pps_net* nt,
                                               const pps_state* states, int n) {
    pps_status s = check_batch(nt, states, n);
    if (s != PPS_OK) return s;
    cudaSetDevice(nt->device);
    cudaError_t e = forward(nt, states, n, false, true);
    if (e != cudaSuccess) return fail(PPS_ECUDA, "pps_net_selftest_timeout", e);
    return pps_net_sync(nt);
}

extern "C" pps_status pps_net_raster(pps_net* nt, const pps_state* states,
                                     int n, uint16_t* out) {
    pps_status s = check_batch(nt, states, n);
    if (s != PPS_OK) return s;
    if (!out) return PPS_EINVAL;
    cudaSetDevice(nt->device);
    const long long P = (long long)n * NPIX;
    launch_raster(nt, states, n, nt->stream);
    if ((reinterpret_cast<uintptr_t>(out) & 15) != 0)
        return fail(PPS_EINVAL, "pps_net_raster: out must be 16-byte aligned");
    narrow_map_kernel<<<blocks(P, 256), 256, 0, nt->stream>>>(
        reinterpret_cast<const uint4*>(nt->a0), P, reinterpret_cast<uint4*>(out));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PPS_OK : fail(PPS_ECUDA, "pps_net_raster", e);
}

namespace {
pps_status forward_to(pps_net* nt, const pps_state* states, int n, float* out,
                      bool keep, const char* who,
                      const uint16_t* map = nullptr) {
    pps_status s = check_batch(nt, states ? (const void*)states : map, n);
    if (s != PPS_OK) return s;
    if (!out) return PPS_EINVAL;
    cudaSetDevice(nt->device);
    cudaError_t e = forward(nt, states, n, keep, false, map);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, nt->out, sizeof(float) * (size_t)n * NPIX,
                            cudaMemcpyDeviceToDevice, nt->stream);
    return e == cudaSuccess ? PPS_OK : fail(PPS_ECUDA, who, e);
}
}  // namespace

extern "C" pps_status pps_net_forward(pps_net* nt, const pps_state* states,
                                      int n, float* out) {
    PPS_RANGE("pps_net_forward");
    return forward_to(nt, states, n, out, false, "pps_net_forward");
}

extern "C" pps_status pps_net_forward_layers(pps_net* nt,
                                             const pps_state* states, int n,
                                             float* out) {
    return forward_to(nt, states, n, out, true, "pps_net_forward_layers");
}

extern "C" pps_status pps_net_forward_map(pps_net* nt, const uint16_t* map,
                                          int n, int layers, float* out) {
    if (!map || (reinterpret_cast<uintptr_t>(map) & 15) != 0)
        return fail(PPS_EINVAL, "pps_net_forward_map: map must be a 16-byte "
                                "aligned device pointer");
    return forward_to(nt, nullptr, n, out, layers != 0, "pps_net_forward_map",
                      map);
}

namespace {
pps_status grad_of(pps_net* nt, const pps_state* states, const uint16_t* map,
                   const float* labels, int n, float* grads, float* loss,
                   const char* who) {
    pps_status s = check_batch(nt, states ? (const void*)states : map, n);
    if (s != PPS_OK) return s;
    if (!labels) return PPS_EINVAL;
    cudaSetDevice(nt->device);
    cudaError_t e = cudaMemsetAsync(nt->grad, 0, sizeof(float) * kPadParams,
                                    nt->stream);
    if (e == cudaSuccess) e = forward_train(nt, states, n, map);
    if (e == cudaSuccess) e = backward(nt, labels, n);
    std::vector<float> pad(kPadParams);
    float l = 0.f;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pad.data(), nt->grad, sizeof(float) * kPadParams,
                            cudaMemcpyDeviceToHost, nt->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&l, nt->loss, sizeof(float), cudaMemcpyDeviceToHost,
                            nt->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nt->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(nt->grad, 0, sizeof(float) * kPadParams, nt->stream);
    if (e != cudaSuccess) return fail(PPS_ECUDA, who, e);
    if (grads) from_padded(pad, grads);
    if (loss) *loss = l;
    return PPS_OK;
}
}  // namespace

extern "C" pps_status pps_net_grad(pps_net* nt, const pps_state* states,
                                   const float* labels, int n, float* grads,
                                   float* loss) {
    if (!states) return PPS_EINVAL;
    return grad_of(nt, states, nullptr, labels, n, grads, loss, "pps_net_grad");
}

extern "C" pps_status pps_net_grad_map(pps_net* nt, const uint16_t* map,
                                       const float* labels, int n,
                                       float* grads, float* loss) {
    if (!map || (reinterpret_cast<uintptr_t>(map) & 15) != 0)
        return fail(PPS_EINVAL, "pps_net_grad_map: map must be a 16-byte "
                                "aligned device pointer");
    return grad_of(nt, nullptr, map, labels, n, grads, loss,
                   "pps_net_grad_map");
}

extern "C" pps_status pps_net_train_step(pps_net* nt, const pps_state* states,
                                         const float* labels, int n, float lr,
                                         float* loss) {
    PPS_RANGE("pps_net_train_step");
    pps_status s = check_batch(nt, states, n);
    if (s != PPS_OK) return s;
    if (!labels || !(lr > 0.f) || !std::isfinite(lr))
        return fail(PPS_EINVAL, "pps_net_train_step: labels and lr > 0");
    cudaSetDevice(nt->device);
    cudaError_t e = forward_train(nt, states, n);
    if (e == cudaSuccess) e = backward(nt, labels, n);
    ++nt->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - std::pow(b1, (float)nt->step));
    const float c2 = 1.f / (1.f - std::pow(b2, (float)nt->step));
    if (e == cudaSuccess) {
        adam_kernel<<<blocks(kPadParams, 256), 256, 0, nt->stream>>>(
            nt->w, nt->grad, nt->m, nt->v, kPadParams, lr, b1, b2, 1e-8f, c1,
            c2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cast_weights(nt);
    if (e == cudaSuccess && loss) {
        e = cudaMemcpyAsync(loss, nt->loss, sizeof(float),
                            cudaMemcpyDeviceToHost, nt->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(nt->stream);
    }
    return e == cudaSuccess ? PPS_OK : fail(PPS_ECUDA, "pps_net_train_step", e);
}

extern "C" pps_status pps_net_labels_grid(pps_net* nt,
                                          const float* point_best, int n,
                                          const pps_grid* fine,
                                          float floor_value, float* labels) {
    pps_status s = check_batch(nt, point_best, n);
    if (s != PPS_OK) return s;
    if (!labels || !fine || !std::isfinite(floor_value)) return PPS_EINVAL;
    const CellLattice cl = cell_lattice(*fine);
    if (!cl.ok)
        return fail(PPS_EINVAL, "pps_net_labels_grid: the grid is not on the "
                                "map's cell lattice");
    cudaSetDevice(nt->device);
    cell_label_kernel<<<blocks((long long)n * NPIX, 256), 256, 0, nt->stream>>>(
        point_best, n, fine->nx, fine->ny, cl.m, cl.ox, cl.oy, floor_value,
        labels);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PPS_OK : fail(PPS_ECUDA, "pps_net_labels", e);
}

extern "C" pps_status pps_net_labels(pps_net* nt, const float* point_best,
                                     int n, float floor_value, float* labels) {
    pps_grid fine;
    pps_grid_from_field(12.f, 9.f, 0.025f, &fine);
    return pps_net_labels_grid(nt, point_best, n, &fine, floor_value, labels);
}

extern "C" pps_status pps_net_set_train_kernels(pps_net* nt, int kind) {
    if (!nt || (kind != PPS_NET_TRAIN_TCGEN05 && kind != PPS_NET_TRAIN_MMA_SYNC))
        return fail(PPS_EINVAL, "pps_net_set_train_kernels: unknown kind");
    nt->train_kind = kind;
    return PPS_OK;
}

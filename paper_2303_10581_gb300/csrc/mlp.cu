// mlp.cu -- the learned proposal of the filter polygon: features of a point
// set and a small MLP that picks the direction count K in {8, 16, 32, 64}
// and the angular offsets of the K-direction polygon (kfilter.cu).  The
// paper filters with the fixed octagon; this is the extension its related
// work points to (more directions).  Whatever the MLP outputs, the polygon's
// vertices are extreme input points, so the filter stays exact.
//
// Features: a 32 x 32 occupancy grid of a 4096-point sample (evenly spaced
// indices) over the sample's bounding box, as fractions of the sample.
// MLP: 1024 -> 64 -> 64 -> 68 (4 K-logits, 64 offsets), ReLU between,
// BF16 weights, FP32 accumulation; one parameter array, row-major:
//   W1[64][1024] b1[64] W2[64][64] b2[64] W3[68][64] b3[68].
// Training kernels: forward (keeping the activations), the loss gradient
// (softmax cross-entropy on the K-logits; squared error on the offsets of
// samples that carry an offset label), backward through the activations,
// the weight gradients summed over the batch, and an Adam step on FP32
// master weights that also writes their BF16 copy.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "launch.h"
#include "mlp.cuh"

namespace ch {
namespace {

using namespace mlp;



// One block of 1024 threads per point set.
__global__ void __launch_bounds__(1024) features_kernel(const float *__restrict__ pts, int64_t n, float *__restrict__ feat)
{
    __shared__ float s_red[4][32];
    __shared__ uint32_t s_cnt[kIn];
    __shared__ float s_box[4];
    const int t = (int)threadIdx.x, lane = t & 31, warp = t >> 5;
    const int m = n < kSample ? (int)n : kSample;
    for (int c = t; c < kIn; c += 1024) s_cnt[c] = 0u;
    // the sample: points floor(j n / m), j < m
    float px[kSample / 1024], py[kSample / 1024];
    float x0 = __int_as_float(0x7f800000), x1 = -x0, y0 = x0, y1 = -x0;
#pragma unroll
    for (int r = 0; r < kSample / 1024; ++r) {
        const int j = r * 1024 + t;
        px[r] = py[r] = 0.0f;
        if (j < m) {
            const int64_t i = (int64_t)j * n / m;
            const float2 v = reinterpret_cast<const float2 *>(pts)[i];
            px[r] = v.x;
            py[r] = v.y;
            x0 = fminf(x0, v.x);
            x1 = fmaxf(x1, v.x);
            y0 = fminf(y0, v.y);
            y1 = fmaxf(y1, v.y);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x0 = fminf(x0, __shfl_xor_sync(0xffffffffu, x0, o));
        x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, o));
        y0 = fminf(y0, __shfl_xor_sync(0xffffffffu, y0, o));
        y1 = fmaxf(y1, __shfl_xor_sync(0xffffffffu, y1, o));
    }
    if (lane == 0) {
        s_red[0][warp] = x0;
        s_red[1][warp] = x1;
        s_red[2][warp] = y0;
        s_red[3][warp] = y1;
    }
    __syncthreads();
    if (t == 0) {
        float a = s_red[0][0], b = s_red[1][0], c = s_red[2][0], d = s_red[3][0];
        for (int w = 1; w < 32; ++w) {
            a = fminf(a, s_red[0][w]);
            b = fmaxf(b, s_red[1][w]);
            c = fminf(c, s_red[2][w]);
            d = fmaxf(d, s_red[3][w]);
        }
        s_box[0] = a;
        s_box[1] = b;
        s_box[2] = c;
        s_box[3] = d;
    }
    __syncthreads();
    const float w = __fsub_rn(s_box[1], s_box[0]), h = __fsub_rn(s_box[3], s_box[2]);
    const float sx = w > 0.0f ? 32.0f / w : 0.0f, sy = h > 0.0f ? 32.0f / h : 0.0f;
#pragma unroll
    for (int r = 0; r < kSample / 1024; ++r) {
        const int j = r * 1024 + t;
        if (j < m) {
            const int cx = min(kGrid - 1, (int)floorf(__fmul_rn(__fsub_rn(px[r], s_box[0]), sx)));
            const int cy = min(kGrid - 1, (int)floorf(__fmul_rn(__fsub_rn(py[r], s_box[2]), sy)));
            atomicAdd(&s_cnt[cy * kGrid + cx], 1u);
        }
    }
    __syncthreads();
    const float inv = 1.0f / (float)m;
    for (int c = t; c < kIn; c += 1024) feat[c] = (float)s_cnt[c] * inv;
}

// One block of 128 threads per sample: X[b] -> H1[b], H2[b], OUT[b].
__global__ void __launch_bounds__(128) forward_kernel(const float *__restrict__ X, int B, const __nv_bfloat16 *__restrict__ P,
                                                      float *__restrict__ H1, float *__restrict__ H2, float *__restrict__ OUT)
{
    __shared__ float s_x[kIn], s_h1[kHid], s_h2[kHid];
    const int b = blockIdx.x, t = (int)threadIdx.x;
    if (b >= B) return;
    for (int i = t; i < kIn; i += 128) s_x[i] = X[(int64_t)b * kIn + i];
    __syncthreads();
    if (t < kHid) {
        float acc = wf(P, oB1 + t);
        for (int i = 0; i < kIn; ++i) acc = __fmaf_rn(wf(P, oW1 + t * kIn + i), s_x[i], acc);
        s_h1[t] = fmaxf(acc, 0.0f);
        H1[b * kHid + t] = s_h1[t];
    }
    __syncthreads();
    if (t < kHid) {
        float acc = wf(P, oB2 + t);
        for (int i = 0; i < kHid; ++i) acc = __fmaf_rn(wf(P, oW2 + t * kHid + i), s_h1[i], acc);
        s_h2[t] = fmaxf(acc, 0.0f);
        H2[b * kHid + t] = s_h2[t];
    }
    __syncthreads();
    if (t < kOut) {
        float acc = wf(P, oB3 + t);
        for (int i = 0; i < kHid; ++i) acc = __fmaf_rn(wf(P, oW3 + t * kHid + i), s_h2[i], acc);
        OUT[b * kOut + t] = acc;
    }
}

// dOUT = d(loss) / d(OUT), loss = mean over the batch of
//   CE(softmax(OUT[0:4]), label) + lam * mask * mean_j (OUT[4+j] - off[j])^2.
__global__ void loss_grad_kernel(const float *__restrict__ OUT, int B, const int32_t *__restrict__ label,
                                 const float *__restrict__ off, const float *__restrict__ mask, float lam,
                                 float *__restrict__ dOUT, float *__restrict__ loss)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float *o = OUT + b * kOut;
    float mx = o[0];
    for (int k = 1; k < 4; ++k) mx = fmaxf(mx, o[k]);
    float e[4], z = 0.0f;
    for (int k = 0; k < 4; ++k) {
        e[k] = expf(o[k] - mx);
        z += e[k];
    }
    const int y = min(max(label[b], 0), 3);   // labels are 0..3; the clamp keeps a bad one in bounds
    float l = logf(z) + mx - o[y];
    const float invB = 1.0f / (float)B;
    for (int k = 0; k < 4; ++k) dOUT[b * kOut + k] = (e[k] / z - (k == y ? 1.0f : 0.0f)) * invB;
    const float w = lam * mask[b];
    for (int j = 0; j < 64; ++j) {
        const float d = o[4 + j] - off[b * 64 + j];
        l += w * d * d / 64.0f;
        dOUT[b * kOut + 4 + j] = w * 2.0f * d / 64.0f * invB;
    }
    loss[b] = l;
}

// Per sample: dH2 = (W3^T dOUT) * [H2 > 0], dH1 = (W2^T dH2) * [H1 > 0].
__global__ void __launch_bounds__(64) backward_kernel(const float *__restrict__ dOUT, int B, const __nv_bfloat16 *__restrict__ P,
                                                      const float *__restrict__ H1, const float *__restrict__ H2,
                                                      float *__restrict__ dH1, float *__restrict__ dH2)
{
    __shared__ float s_d[kOut], s_dh2[kHid];
    const int b = blockIdx.x, t = (int)threadIdx.x;
    if (b >= B) return;
    for (int j = t; j < kOut; j += 64) s_d[j] = dOUT[b * kOut + j];
    __syncthreads();
    float acc = 0.0f;
    for (int j = 0; j < kOut; ++j) acc = __fmaf_rn(wf(P, oW3 + j * kHid + t), s_d[j], acc);
    const float g2 = H2[b * kHid + t] > 0.0f ? acc : 0.0f;
    s_dh2[t] = g2;
    dH2[b * kHid + t] = g2;
    __syncthreads();
    acc = 0.0f;
    for (int j = 0; j < kHid; ++j) acc = __fmaf_rn(wf(P, oW2 + j * kHid + t), s_dh2[j], acc);
    dH1[b * kHid + t] = H1[b * kHid + t] > 0.0f ? acc : 0.0f;
}

// One thread per parameter: its gradient summed over the batch.
__global__ void wgrad_kernel(const float *__restrict__ X, int B, const float *__restrict__ H1, const float *__restrict__ H2,
                             const float *__restrict__ dH1, const float *__restrict__ dH2, const float *__restrict__ dOUT,
                             float *__restrict__ G)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    float acc = 0.0f;
    if (p < oB1) {
        const int j = p / kIn, i = p % kIn;
        for (int b = 0; b < B; ++b) acc = __fmaf_rn(dH1[b * kHid + j], X[(int64_t)b * kIn + i], acc);
    } else if (p < oW2) {
        for (int b = 0; b < B; ++b) acc += dH1[b * kHid + (p - oB1)];
    } else if (p < oB2) {
        const int j = (p - oW2) / kHid, i = (p - oW2) % kHid;
        for (int b = 0; b < B; ++b) acc = __fmaf_rn(dH2[b * kHid + j], H1[b * kHid + i], acc);
    } else if (p < oW3) {
        for (int b = 0; b < B; ++b) acc += dH2[b * kHid + (p - oB2)];
    } else if (p < oB3) {
        const int j = (p - oW3) / kHid, i = (p - oW3) % kHid;
        for (int b = 0; b < B; ++b) acc = __fmaf_rn(dOUT[b * kOut + j], H2[b * kHid + i], acc);
    } else {
        for (int b = 0; b < B; ++b) acc += dOUT[b * kOut + (p - oB3)];
    }
    G[p] = acc;
}

// Adam on the FP32 master weights; the BF16 copy is what the kernels read.
__global__ void adam_kernel(float *__restrict__ Wm, const float *__restrict__ G, float *__restrict__ M,
                            float *__restrict__ V, __nv_bfloat16 *__restrict__ P, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    const float g = G[p];
    const float m = b1 * M[p] + (1.0f - b1) * g;
    const float v = b2 * V[p] + (1.0f - b2) * g * g;
    M[p] = m;
    V[p] = v;
    const float w = Wm[p] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    Wm[p] = w;
    P[p] = __float2bfloat16_rn(w);
}

}  // namespace

namespace {

// ch_hull_learned's proposal in one block (mlp.cuh)
__global__ void __launch_bounds__(mlp::LT) learned_choice_kernel(const float *__restrict__ pts, int64_t n,
                                                                 const __nv_bfloat16 *__restrict__ P, LearnScratch *ls)
{
    mlp::learned_choice_block(pts, n, P, ls);
}

}  // namespace

cudaError_t launch_learned_choice(const float *pts, int64_t n, const void *params, void *ws, const Layout &L,
                                  cudaStream_t st)
{
    probe_before(CH_K_KGON, st);
    learned_choice_kernel<<<1, mlp::LT, 0, st>>>(pts, n, static_cast<const __nv_bfloat16 *>(params),
                                                at<LearnScratch>(ws, L.learn));
    note_kernels(CH_K_KGON, 1);
    probe_after(CH_K_KGON, st);
    return cudaGetLastError();
}

}  // namespace ch

using namespace ch;

extern "C" int32_t ch_mlp_param_count(void) { return mlp::kParams; }

extern "C" ch_status ch_kgon_features(const float *pts, int64_t n, float *feat, void *stream)
{
    if (!pts || !feat || n < 1 || (reinterpret_cast<uintptr_t>(pts) & 7u) || (reinterpret_cast<uintptr_t>(feat) & 3u))
        return CH_ERR_ARG;
    features_kernel<<<1, 1024, 0, reinterpret_cast<cudaStream_t>(stream)>>>(pts, n, feat);
    return cudaGetLastError() == cudaSuccess ? CH_OK : CH_ERR_CUDA;
}

extern "C" ch_status ch_mlp_forward(const float *X, int32_t B, const void *params, float *H1, float *H2, float *OUT,
                                    void *stream)
{
    if (!X || !params || !H1 || !H2 || !OUT || B < 1) return CH_ERR_ARG;
    forward_kernel<<<B, 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        X, B, static_cast<const __nv_bfloat16 *>(params), H1, H2, OUT);
    return cudaGetLastError() == cudaSuccess ? CH_OK : CH_ERR_CUDA;
}

extern "C" ch_status ch_mlp_train_step(const float *X, int32_t B, const int32_t *label, const float *off,
                                       const float *mask, float lam, void *params, float *master, float *adam_m,
                                       float *adam_v, int32_t step, float lr, float *scratch, float *loss, void *stream)
{
    if (!X || !label || !off || !mask || !params || !master || !adam_m || !adam_v || !scratch || !loss || B < 1 ||
        step < 1)
        return CH_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    __nv_bfloat16 *P = static_cast<__nv_bfloat16 *>(params);
    // scratch: H1, H2 (B x 64 each), OUT, dOUT (B x 68 each), dH1, dH2 (B x 64 each), G (params)
    float *H1 = scratch, *H2 = H1 + B * kHid, *OUT = H2 + B * kHid, *dOUT = OUT + B * kOut;
    float *dH1 = dOUT + B * kOut, *dH2 = dH1 + B * kHid, *G = dH2 + B * kHid;
    forward_kernel<<<B, 128, 0, st>>>(X, B, P, H1, H2, OUT);
    loss_grad_kernel<<<(B + 127) / 128, 128, 0, st>>>(OUT, B, label, off, mask, lam, dOUT, loss);
    backward_kernel<<<B, 64, 0, st>>>(dOUT, B, P, H1, H2, dH1, dH2);
    wgrad_kernel<<<(kParams + 255) / 256, 256, 0, st>>>(X, B, H1, H2, dH1, dH2, dOUT, G);
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    adam_kernel<<<(kParams + 255) / 256, 256, 0, st>>>(master, G, adam_m, adam_v, P, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError() == cudaSuccess ? CH_OK : CH_ERR_CUDA;
}

// Floats of scratch that ch_mlp_train_step needs for a batch of B.
extern "C" int64_t ch_mlp_scratch_floats(int32_t B)
{
    return (int64_t)B * (4 * kHid + 2 * kOut) + kParams;
}

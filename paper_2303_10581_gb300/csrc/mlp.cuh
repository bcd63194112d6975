// mlp.cuh -- the learned proposal's MLP shape and its one-block inference
// (features, the three layers, the choice of the polygon), shared by the
// MLP kernels (mlp.cu) and the extremes sweep, which can run it in an
// extra block beside its sweep (ch_hull_learned).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace ch {
namespace mlp {

constexpr int kGrid = 32;
constexpr int kIn = kGrid * kGrid;   // 1024
constexpr int kHid = 64;
constexpr int kOut = 4 + 64;         // K-logits, offsets
constexpr int kSample = 4096;

constexpr int oW1 = 0;
constexpr int oB1 = oW1 + kHid * kIn;
constexpr int oW2 = oB1 + kHid;
constexpr int oB2 = oW2 + kHid * kHid;
constexpr int oW3 = oB2 + kHid;
constexpr int oB3 = oW3 + kOut * kHid;
constexpr int kParams = oB3 + kOut;

__device__ __forceinline__ float wf(const __nv_bfloat16 *P, int i) { return __bfloat162float(P[i]); }

// The learned proposal for one point set in one block (ch_hull_learned):
// the features of features_kernel, the MLP of forward_kernel with each
// output's dot product spread over a warp (lanes take every 32nd input,
// then a shuffle sum), and the choice: K from the arg-max of the four
// K-logits (lowest on ties; a NaN logit never wins), the offsets (units of
// pi / K) clipped to +-0.45, the directions at angles 2 pi k / K +
// offset_k pi / K (cos and sin in binary64, rounded once; a multiple of
// pi / 4 with zero offset takes the octagon's integer direction).
constexpr int LT = 512;

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void learned_choice_block(const float *__restrict__ pts, int64_t n,
                                                     const __nv_bfloat16 *__restrict__ P, LearnScratch *ls,
                                                     float *dirs_out = nullptr, int32_t *k_out = nullptr)
{
    __shared__ float s_red[4][LT / 32];
    __shared__ uint32_t s_cnt[kIn];
    __shared__ float s_x[kIn], s_h1[kHid], s_h2[kHid], s_o[kOut];
    __shared__ float s_box[4];
    const int t = (int)threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int NWARP = LT / 32;
    const int m = n < kSample ? (int)n : kSample;
    for (int c = t; c < kIn; c += LT) s_cnt[c] = 0u;
    float px[kSample / LT], py[kSample / LT];
    float x0 = __int_as_float(0x7f800000), x1 = -x0, y0 = x0, y1 = -x0;
#pragma unroll
    for (int r = 0; r < kSample / LT; ++r) {
        const int j = r * LT + t;
        px[r] = py[r] = 0.0f;
        if (j < m) {
            const float2 v = reinterpret_cast<const float2 *>(pts)[(int64_t)j * n / m];
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
        for (int w = 1; w < NWARP; ++w) {
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
    for (int r = 0; r < kSample / LT; ++r) {
        const int j = r * LT + t;
        if (j < m) {
            const int cx = min(kGrid - 1, (int)floorf(__fmul_rn(__fsub_rn(px[r], s_box[0]), sx)));
            const int cy = min(kGrid - 1, (int)floorf(__fmul_rn(__fsub_rn(py[r], s_box[2]), sy)));
            atomicAdd(&s_cnt[cy * kGrid + cx], 1u);
        }
    }
    __syncthreads();
    const float inv = 1.0f / (float)m;
    for (int c = t; c < kIn; c += LT) {
        s_x[c] = (float)s_cnt[c] * inv;
        ls->feat[c] = s_x[c];
    }
    __syncthreads();
    for (int u = warp; u < kHid; u += NWARP) {   // layer 1: warp per unit
        float acc = 0.0f;
        for (int i = lane; i < kIn; i += 32) acc = __fmaf_rn(wf(P, oW1 + u * kIn + i), s_x[i], acc);
        acc = warp_sum(acc) + wf(P, oB1 + u);
        if (lane == 0) s_h1[u] = fmaxf(acc, 0.0f);
    }
    __syncthreads();
    for (int u = warp; u < kHid; u += NWARP) {
        float acc = 0.0f;
        for (int i = lane; i < kHid; i += 32) acc = __fmaf_rn(wf(P, oW2 + u * kHid + i), s_h1[i], acc);
        acc = warp_sum(acc) + wf(P, oB2 + u);
        if (lane == 0) s_h2[u] = fmaxf(acc, 0.0f);
    }
    __syncthreads();
    for (int u = warp; u < kOut; u += NWARP) {
        float acc = 0.0f;
        for (int i = lane; i < kHid; i += 32) acc = __fmaf_rn(wf(P, oW3 + u * kHid + i), s_h2[i], acc);
        acc = warp_sum(acc) + wf(P, oB3 + u);
        if (lane == 0) s_o[u] = acc;
    }
    __syncthreads();
    for (int i = t; i < kOut; i += LT) ls->out[i] = s_o[i];
    if (warp != 0) return;
    int best = 0;
    for (int i = 1; i < 4; ++i)
        if (s_o[i] > s_o[best]) best = i;   // a NaN logit never wins
    const int K = 8 << best;
    // (the caller's copy: the K directions, zeros after them)
    if (dirs_out)
        for (int k = K + lane; k < kMaxDirs; k += 32) dirs_out[2 * k] = dirs_out[2 * k + 1] = 0.0f;
    for (int k = lane; k < K; k += 32) {
        float u = fminf(fmaxf(s_o[4 + k], -0.45f), 0.45f);
        if (!(u == u)) u = 0.0f;
        float cx, cy;
        if (u == 0.0f && (8 * k) % K == 0) {
            const int o = 8 * k / K;
            cx = (float)((o == 0 || o == 1 || o == 7) ? 1 : ((o == 3 || o == 4 || o == 5) ? -1 : 0));
            cy = (float)((o == 1 || o == 2 || o == 3) ? 1 : ((o == 5 || o == 6 || o == 7) ? -1 : 0));
        } else {
            const double th = 2.0 * 3.141592653589793 * k / K + (double)u * 3.141592653589793 / K;
            cx = (float)cos(th);
            cy = (float)sin(th);
        }
        ls->dirs[2 * k] = cx;
        ls->dirs[2 * k + 1] = cy;
        if (dirs_out) {
            dirs_out[2 * k] = cx;
            dirs_out[2 * k + 1] = cy;
        }
    }
    if (lane == 0) {
        ls->K = K;
        if (k_out) *k_out = K;
    }
}


}  // namespace mlp
}  // namespace ch

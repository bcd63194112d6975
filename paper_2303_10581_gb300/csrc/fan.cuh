// fan.cuh -- the hull step's fan: angular bins around the centre and the
// order key of the farthest-point choice, shared by the filter's count
// pass (which gathers the first level's bin maxima on its sampled tiles)
// and the fan kernels (kgon.cu).
#pragma once

#include "common.cuh"

namespace ch {

// The first level's sample: every fan_sample_stride(tiles)-th 4096-point
// tile (at least every tile; about kFanBinTiles tiles, at most every 8th).
constexpr int64_t kFanBinTiles = 1536;
__host__ __device__ inline int64_t fan_sample_stride(int64_t tiles)
{
    const int64_t s = tiles / kFanBinTiles;
    return s < 1 ? 1 : (s > 8 ? 8 : s);
}

// Bin of the direction (dx, dy): a pseudo-angle in [0, 4) that grows with
// the angle counter-clockwise from +x, scaled to the bins.  Any value is
// safe (it only picks a triangle); the conversion saturates and the result
// is clamped.
template <int NB = kFanBins>
__device__ __forceinline__ int fan_bin(float dx, float dy)
{
    const float s = fabsf(dx) + fabsf(dy);
    float a = 0.0f;
    if (s > 0.0f) {
        const float t = __fdividef(dy, s);
        a = dx >= 0.0f ? (dy >= 0.0f ? t : 4.0f + t) : 2.0f - t;
    }
    // a is in [0, 4] (t in [-1, 1]; a NaN from an overflowed difference
    // converts to 0): only the top needs a clamp
    const int b = __float2int_rz(a * (NB / 4.0f));
    return min(b, NB - 1);
}

template <int NB = kFanBins>
__device__ __forceinline__ int next_bin(int b) { return b + 1 == NB ? 0 : b + 1; }
template <int NB = kFanBins>
__device__ __forceinline__ int prev_bin(int b) { return b == 0 ? NB - 1 : b - 1; }

// a - b = s + e and a + b = s + e exactly (Knuth's two-sum, binary32
// round to nearest; the intrinsics are never contracted into an FMA)
__device__ __forceinline__ void two_diff(float a, float b, float &s, float &e)
{
    s = __fsub_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fsub_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fadd_rn(b, bb));
}
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Order key for the farthest-point choice of a bin: |p - c|^2 - r2ref,
// from the differences p - c and their squares as exact pairs (two-sum,
// two-product by FMA), rounded once at the end.  The binary32 square
// |p - c|^2 itself resolves only 2^-23 of its value, while on the unit
// circle the radii of binary32 points differ by about 10^-7 and the top
// points of a bin by far less: the vertex would be any of its top points
// and the chords sag below the others.  Any key would keep the test exact
// (a vertex only has to be an input point); this one finds the farthest.
// r2ref: a squared distance of the set's scale (Sterbenz: the last
// difference is exact when the sum is within a factor 2 of it).
__device__ __forceinline__ uint32_t far_key(float px, float py, float cx, float cy, float r2ref)
{
    float dxh, dxl, dyh, dyl;
    two_diff(px, cx, dxh, dxl);
    two_diff(py, cy, dyh, dyl);
    const float sxh = __fmul_rn(dxh, dxh), sxl = __fmaf_rn(dxh, dxh, -sxh);
    const float syh = __fmul_rn(dyh, dyh), syl = __fmaf_rn(dyh, dyh, -syh);
    float sh, sl;
    two_sum(sxh, syh, sh, sl);
    const float cross = __fmul_rn(2.0f, __fmaf_rn(dxh, dxl, __fmul_rn(dyh, dyl)));
    const float lo = __fadd_rn(__fadd_rn(sl, __fadd_rn(sxl, syl)), cross);
    return ord_key(__fadd_rn(__fsub_rn(sh, r2ref), lo));
}

// r2ref of far_key for a polygon's set: the squared distance from its
// centre to its first vertex (binary32).
__device__ __forceinline__ float far_ref(const Octagon &o)
{
    const float ux = __fsub_rn(o.ax[0], o.cx), uy = __fsub_rn(o.ay[0], o.cy);
    return __fmaf_rn(ux, ux, __fmul_rn(uy, uy));
}

// Strictly inside a fan triangle (exact signs).  V: kFanBins vertices.
// With o = orient(c, v, p) = +1 the triangle is (c, v, w), w the next
// vertex, and p is inside iff orient(v, w, p) = orient(w, c, p) = +1; with
// o = -1 it is (c, w, v), w the previous vertex, and p is inside iff
// orient(w, v, p) = orient(c, w, p) = +1, i.e. orient(v, w, p) =
// orient(w, c, p) = -1.
//
// fan_signs_f32 takes the three signs in binary32 (branch-free, so a
// thread's items interleave): 1 inside, 0 outside, 2 undecided (a sign the
// binary32 bound does not prove, and that matters); fan_inside_exact
// settles the undecided ones.
// The two signs with c as a vertex are taken with c as the reference point
// (a cyclic shift of a triple keeps its orientation): orient(c, v, p) as
// orient(v, p, c) and orient(w, c, p) as orient(p, w, c), so that both use
// the differences p - c of the bin; orient_f32 certifies the sign of either
// form with the same bound.

}  // namespace ch

// kgon.cu -- a second throw-away step inside the device hull: a fan of
// triangles around an interior point, applied to the octagon filter's keep
// decisions before its survivors are written.
//
// The octagon filter (Sec. 3.1-3.2) removes almost nothing from points near
// a circle, and on a displaced circle 95 % survive it, although the hulls
// have a small fraction of the points as vertices.  The hull step repeats
// the throw-away idea of Sec. 3.1 on a much finer scale.  Let c be the
// centre of the bounding box, checked with exact signs to lie strictly
// inside the octagon, hence strictly inside the hull.  The plane around c
// is cut into kFanBins angular bins; the vertex of a bin is the input point
// farthest from c among a sample (the octagon survivors of about
// kFanBinTiles evenly spaced 4096-point tiles of the input, fan.cuh), and a
// bin the sample missed repeats the vertex before it.  For
// consecutive vertices v, w every point strictly inside the triangle
// (c, v, w) is a combination of c, v and w with positive weights, so it
// lies strictly inside the hull and is no vertex of it: it is dropped.
// This holds whatever the vertices are (they are input points), so nothing
// needs to be exact but the three orientation signs of the final test, and
// a triangle that comes out clockwise or flat drops nothing.
//
// The kernels run between the filter's count pass (which leaves keep bits,
// per-tile counts and per-block totals) and its scatter pass, so the
// scatter writes only the points that survive both tests:
//
//  (count pass)         per bin, the farthest sampled octagon survivor
//                       (atomicMax of (far_key << 32 | ~index) into global
//                       slots, on the sampled tiles, filter.cu)
//  fan_build_kernel     octagon survivor count; exact centre check against
//                       the octagon; the vertex of every bin
//  fan_estimate_kernel  exact test of an input sample: whether the fan drops
//                       at least an eighth of the octagon's survivors
//  fan_refine_kernel    per tile of the filter: the kept points' exact fan
//                       test, then new keep bits, tile counts and block totals
//
// Test of a point p: its bin b from a binary32 pseudo-angle (a hint only),
// v the vertex of b.  p strictly left of the ray c -> v: the triangle
// (c, v, next vertex); strictly right: (c, previous vertex, v); on it: kept.
#include <algorithm>

#include "common.cuh"
#include "fan.cuh"
#include "launch.h"

namespace ch {
namespace {

constexpr int FT = 512;                  // threads per block of the bins pass
constexpr int FITEMS = 8;                // points per thread per tile there
constexpr int CT = 1024;                 // threads per block of the refine pass: four
constexpr int CG = CT / kFiltThreads;    // groups of kFiltThreads, each with its own tiles
constexpr uint32_t kKgonMinS = 1u << 16; // fewer octagon survivors: not worth a pass
constexpr int kFanSmem = kFanBins * 8;   // bins or vertices, 224 KB
static_assert(kFiltItems == 16 && CT % kFiltThreads == 0, "refine pass: 16 keep bits per filter thread");

__device__ __forceinline__ float2 input_point(const float *pts, int64_t i)
{
    return __ldg(reinterpret_cast<const float2 *>(pts) + i);
}

// The signs orient_f32 certifies, as two flags (det > bound, -det > bound;
// neither when undecided or when the terms may have overflowed): the same
// arithmetic on the rounded differences a - c and b - c, without turning
// the flags into an integer.
struct Sgn {
    bool pos, neg;
};
__device__ __forceinline__ Sgn sgn_ref(float acx, float acy, float bcx, float bcy)
{
    const float detleft = __fmul_rn(acx, bcy);
    const float detright = __fmul_rn(acy, bcx);
    const float det = __fsub_rn(detleft, detright);
    const float detsum = __fadd_rn(fabsf(detleft), fabsf(detright));
    const float eb = __fmaf_ru(detsum, 2.384185791015625e-07f /* 2^-22 */, 7.174648137343064e-43f /* 2^-140 */);
    const bool ok = detsum <= 3.0e38f;
    return {ok && det > eb, ok && -det > eb};
}

template <int NB = kFanBins>
__device__ __forceinline__ int fan_signs_f32(const float2 *V, float cx, float cy, float px, float py)
{
    const float dx = __fsub_rn(px, cx), dy = __fsub_rn(py, cy);
    const int b = fan_bin<NB>(dx, dy);
    const float2 v = V[b];
    const Sgn o = sgn_ref(__fsub_rn(v.x, cx), __fsub_rn(v.y, cy), dx, dy);                   // (v, p, c)
    const float2 w = V[o.pos ? next_bin<NB>(b) : prev_bin<NB>(b)];
    const Sgn e1 = sgn_ref(__fsub_rn(v.x, px), __fsub_rn(v.y, py), __fsub_rn(w.x, px), __fsub_rn(w.y, py));   // (v, w, p)
    const Sgn e2 = sgn_ref(dx, dy, __fsub_rn(w.x, cx), __fsub_rn(w.y, cy));                   // (p, w, c)
    // inside: the three signs certified equal (strictly inside the triangle
    // on o's side); outside: one of the edges certified opposite to o
    const bool in = (o.pos && e1.pos && e2.pos) || (o.neg && e1.neg && e2.neg);
    const bool out = (o.pos && (e1.neg || e2.neg)) || (o.neg && (e1.pos || e2.pos));
    return in ? 1 : (out ? 0 : 2);
}

template <int NB = kFanBins>
__device__ __noinline__ bool fan_inside_exact(const float2 *V, float cx, float cy, float px, float py)
{
    const int b = fan_bin<NB>(px - cx, py - cy);
    const float2 v = V[b];
    const int o = orient(cx, cy, v.x, v.y, px, py);
    if (o == 0) return false;
    const float2 w = V[o > 0 ? next_bin<NB>(b) : prev_bin<NB>(b)];
    return orient(v.x, v.y, w.x, w.y, px, py) == o && orient(w.x, w.y, cx, cy, px, py) == o;
}

template <int NB = kFanBins>
__device__ __forceinline__ bool fan_inside(const float2 *V, float cx, float cy, float2 p)
{
    const int f = fan_signs_f32<NB>(V, cx, cy, p.x, p.y);
    return f != 2 ? f == 1 : fan_inside_exact<NB>(V, cx, cy, p.x, p.y);
}

// The fan runs when the octagon left at least kKgonMinS survivors and has
// an edge (otherwise it does nothing).
__device__ __forceinline__ bool fan_live(const KgonCtrl *kc, const Octagon *oct, uint32_t &s)
{
    s = oct->abort ? 0u : kc->s_oct;
    return s >= kKgonMinS && oct->has_edges && !oct->spec;   // spec: no keep bits to refine
}

// One thread per bin (kFanBins / BT blocks).  The vertex of bin b is the
// sampled point of the last non-empty bin at or before b, cyclically: a
// max-scan of "non-empty bin index" inside the block, and for the bins
// before the block's first non-empty one, the last non-empty bin of the
// nearest earlier range of BT bins that has one (searched range by range).
constexpr int BT = 1024;
static_assert(kFanBins % BT == 0, "bins split evenly over the blocks");

__device__ __forceinline__ int block_max(int v, int *s_w)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();   // s_w may still be read from an earlier call
    if (lane_id() == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    int m = -1;
    for (int w = 0; w < BT / 32; ++w) m = max(m, s_w[w]);
    return m;
}

// bc: the grid of the filter's count pass (its block totals are in
// filt_bsum[0, bc)); the count pass gathered the bins' farthest sampled
// points (filter.cu).
__global__ void __launch_bounds__(BT) fan_build_kernel(const float *__restrict__ pts, int64_t n, void *ws, Layout L,
                                                       int32_t bc)
{
    __shared__ int s_w[BT / 32];
    __shared__ int s_scan[BT / 32];
    __shared__ int s_ok;
    __shared__ uint32_t s_sum[BT / 32];
    const Octagon *oct = at<Octagon>(ws, L.oct);
    KgonCtrl *kc = at<KgonCtrl>(ws, L.kgon_ctrl);
    Kgon *g = at<Kgon>(ws, L.kgon);
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    // octagon survivors: the sum of the count pass's block totals (none
    // when the call was aborted: the count pass left no totals)
    uint32_t s = 0;
    if (!oct->abort) {
        const uint32_t *bsum = at<uint32_t>(ws, L.filt_bsum);
        uint32_t t = 0;
        for (int i = (int)tid; i < bc; i += BT) t += bsum[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) s_sum[warp] = t;
        __syncthreads();
        for (int w = 0; w < BT / 32; ++w) s += s_sum[w];
    }
    if (blockIdx.x == 0 && tid == 0) kc->s_oct = s;   // read by the later fan kernels
    if (!(s >= kKgonMinS && oct->has_edges && !oct->spec)) {   // (fan_live, before s_oct is visible)
        if (blockIdx.x == 0 && tid == 0) g->ok = 0u;
        return;
    }
    const float cx = oct->cx, cy = oct->cy;
    // c strictly left of every edge of non-zero length: the edges turn once
    // around c with every step counter-clockwise, so c lies strictly inside
    // the hull of the octagon's vertices
    if (tid == 0) s_ok = 1;
    __syncthreads();
    if (tid < 8 && ((oct->valid >> tid) & 1u) &&
        orient(oct->ax[tid], oct->ay[tid], oct->bx[tid], oct->by[tid], cx, cy) <= 0)
        s_ok = 0;
    const int b = (int)(blockIdx.x * BT + tid);
    const unsigned long long mine = kc->slot[b];
    int incl = mine != 0ull ? b : -1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl = max(incl, u);
    }
    if (lane == 31) s_scan[warp] = incl;
    __syncthreads();
    for (int w = 0; w < (int)warp; ++w) incl = max(incl, s_scan[w]);
    // the nearest earlier range with a non-empty bin (the block's own range
    // last, for the wrap-around)
    int prev = -1;
    for (uint32_t k = 1; k <= gridDim.x && prev < 0; ++k) {   // prev is block-uniform
        const uint32_t rb = (blockIdx.x + gridDim.x - k) % gridDim.x;
        const int j = (int)(rb * BT + tid);
        prev = block_max(kc->slot[j] != 0ull ? j : -1, s_w);
    }
    if (prev < 0 || !s_ok) {   // no sampled point at all, or c not inside
        if (blockIdx.x == 0 && tid == 0) g->ok = 0u;
        return;
    }
    const int cur = incl >= 0 ? incl : prev;
    const uint32_t i = ~(uint32_t)(cur == b ? mine : kc->slot[cur]);
    g->v[b] = input_point(pts, (int64_t)i < n ? i : 0u);
    if (blockIdx.x == 0 && tid == 0) {
        g->cx = cx;
        g->cy = cy;
        g->ok = 1u;
        g->disk_bad = 0u;
        g->disk_edges = 0u;
        g->rho2 = 0x7ff0000000000000ull;   // +inf until the estimate kernel bounds it
    }
}

// A disk around the centre inside the fan: the fan's triangles (c, v, w) of
// consecutive vertices turn counter-clockwise around c (bins in angular
// order), so when every triangle with v != w is proven strictly
// counter-clockwise their union is a polygon winding once around c, and
// the open disk of radius rho < the distance from c to each of its edges
// (segments [v, w], or the point v when v == w) lies in its interior,
// hence strictly inside the hull.  The distance to a segment is the
// distance to its nearer end when the foot of the perpendicular from c
// provably falls outside it, else at least the distance to its line.
// Binary64 with slack: cross and dot products lose at most 2^-50 of the
// sum of their terms' magnitudes, squares and the quotient 2^-40.  Returns
// the lower bound on the squared distance to edge (v, w), or -1 when the
// triangle is not proven counter-clockwise.
__device__ __forceinline__ double disk_bound(float cx, float cy, float2 v, float2 w)
{
    const double ux = (double)cx - v.x, uy = (double)cy - v.y;   // c - v
    const double dv = (ux * ux + uy * uy) * (1.0 - 0x1p-40);
    if (v.x == w.x && v.y == w.y) return dv;
    const double ex = (double)w.x - v.x, ey = (double)w.y - v.y;   // w - v
    const double t1 = ex * uy, t2 = ey * ux;
    const double lo = (t1 - t2) - (fabs(t1) + fabs(t2)) * 0x1p-50;   // c strictly left of v -> w
    if (!(lo > 0.0)) return -1.0;
    const double len2 = ex * ex + ey * ey;
    const double d1 = ex * ux, d2 = ey * uy;
    const double dot = d1 + d2, derr = (fabs(d1) + fabs(d2)) * 0x1p-50;   // (c - v) . (w - v)
    if (dot < -derr) return dv;   // the foot lies before v: v is the nearest point
    if (dot > len2 * (1.0 + 0x1p-40) + derr) {   // after w
        const double zx = (double)cx - w.x, zy = (double)cy - w.y;
        return (zx * zx + zy * zy) * (1.0 - 0x1p-40);
    }
    return lo * lo / (len2 * (1.0 + 0x1p-40)) * (1.0 - 0x1p-40);
}

// About 2^16 evenly spaced input points.  With f the share of them inside
// the fan and s of n points surviving the octagon, the fan drops at least
// f n - (n - s) of the survivors; the refine pass runs when that is at
// least s / 8.
__global__ void __launch_bounds__(256) fan_estimate_kernel(const float *__restrict__ pts, int64_t n, void *ws, Layout L)
{
    __shared__ uint32_t s_in[8], s_tot[8];
    KgonCtrl *kc = at<KgonCtrl>(ws, L.kgon_ctrl);
    uint32_t s;
    if (!fan_live(kc, at<Octagon>(ws, L.oct), s)) return;
    const Kgon *g = at<Kgon>(ws, L.kgon);
    if (!g->ok) return;
    const int64_t stride = std::max<int64_t>(1, n >> 16);
    const int64_t nsamp = (n - stride / 2 + stride - 1) / stride;
    uint32_t in = 0, tot = 0;
    for (int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x; k < nsamp; k += (int64_t)gridDim.x * 256) {
        in += fan_inside(g->v, g->cx, g->cy, input_point(pts, k * stride + stride / 2)) ? 1u : 0u;
        ++tot;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        in += __shfl_xor_sync(0xffffffffu, in, o);
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    const uint32_t warp = threadIdx.x >> 5;
    if (lane_id() == 0) {
        s_in[warp] = in;
        s_tot[warp] = tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t a = 0, b = 0;
        for (int w = 0; w < 8; ++w) {
            a += s_in[w];
            b += s_tot[w];
        }
        atomicAdd(&kc->inside, a);
        atomicAdd(&kc->sample, b);
    }
    // the disk around the centre (disk_bound), min over all bins
    Kgon *gw = at<Kgon>(ws, L.kgon);
    double mn = __longlong_as_double(0x7ff0000000000000ll);
    bool bad = false;
    uint32_t edges = 0;
    for (int b = (int)(blockIdx.x * 256 + threadIdx.x); b < kFanBins; b += (int)(gridDim.x * 256)) {
        const float2 v = g->v[b], w = g->v[next_bin(b)];
        const double d = disk_bound(g->cx, g->cy, v, w);
        if (d < 0.0) bad = true;
        else mn = fmin(mn, d);
        edges += (v.x != w.x || v.y != w.y) ? 1u : 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        edges += __shfl_xor_sync(0xffffffffu, edges, o);
    }
    bad = __any_sync(0xffffffffu, bad);
    if (lane_id() == 0) {
        atomicMin(&gw->rho2, (unsigned long long)__double_as_longlong(mn));   // >= 0: bits order as values
        if (bad) atomicOr(&gw->disk_bad, 1u);
        if (edges) atomicAdd(&gw->disk_edges, edges);
    }
}

__device__ __forceinline__ bool fan_worth(const KgonCtrl *kc, int64_t n, uint32_t s)
{
    const double f = kc->sample ? (double)kc->inside / (double)kc->sample : 0.0;
    return kc->sample > 0u && f * (double)n - (double)(n - s) >= (double)s / 8.0;
}

// Point of item q (of this thread's 16) of a filter tile; the layout is the
// count pass's: item q = r * G + h is point base + (r * kFiltThreads + t) * G + h.
template <int G>
__device__ __forceinline__ int64_t item_point(int64_t base, uint32_t t, int q)
{
    return base + (int64_t)((q / G) * kFiltThreads + t) * G + q % G;
}

// Fan test of one half (items 8 half .. 8 half + 7) of a filter thread's
// kept points.  Returns the bits (at item positions) of kept points strictly
// inside the fan.  The coordinates of the few undecided points are read
// again for the exact test, so none stay live across it.  Called by every
// lane of the warp (a warp-wide reduction picks the path).
template <int G>
__device__ __forceinline__ uint32_t refine_half(const float *__restrict__ pts, int64_t n, int64_t base, uint32_t t,
                                                uint32_t kb, int half, const float2 *sv, float cx, float cy,
                                                float rho2t, bool &use_disk)
{
    float px[8], py[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) px[k] = py[k] = 0.0f;
    if constexpr (G == 2) {
#pragma unroll
        for (int r4 = 0; r4 < 4; ++r4) {
            const int r = half * 4 + r4;
            if ((kb >> (2 * r)) & 3u) {
                const int64_t i = base + (int64_t)(r * kFiltThreads + t) * 2;
                float4 v;
                if (i + 1 < n) {
                    v = __ldcs(reinterpret_cast<const float4 *>(pts) + i / 2);
                } else {
                    const float2 a = reinterpret_cast<const float2 *>(pts)[i];
                    v = make_float4(a.x, a.y, 0.0f, 0.0f);
                }
                px[2 * r4] = v.x;
                py[2 * r4] = v.y;
                px[2 * r4 + 1] = v.z;
                py[2 * r4 + 1] = v.w;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int r = half * 8 + k;
            if ((kb >> r) & 1u) {
                const float2 v = __ldcs(reinterpret_cast<const float2 *>(pts) + base + r * kFiltThreads + t);
                px[k] = v.x;
                py[k] = v.y;
            }
        }
    }
    const uint32_t live = (kb >> (8 * half)) & 0xffu;
    // the disk around the centre first: r2 < rho2t proves |p - c|^2 < rho^2
    // (rho2t is rho^2 less 2^-20 of it, rounded down, which covers the
    // rounding of r2); when few of a lane's points lie outside the disk the
    // fan test visits only those
    // (use_disk, warp-uniform: a warp whose first half-tile finds fewer than
    // a quarter of its kept points in the disk stops testing it)
    uint32_t outd = live;
    if (use_disk) {
        outd = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float dx = __fsub_rn(px[k], cx), dy = __fsub_rn(py[k], cy);
            const float r2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
            outd |= (r2 < rho2t ? 0u : 1u) << k;
        }
        outd &= live;
        const unsigned hits = __reduce_add_sync(0xffffffffu, (unsigned)__popc(live & ~outd));
        const unsigned tried = __reduce_add_sync(0xffffffffu, (unsigned)__popc(live));
        if (4u * hits < tried) use_disk = false;
    }
    uint32_t in = live & ~outd;
    if (__reduce_max_sync(0xffffffffu, (unsigned)__popc(outd)) <= 2u) {
        for (uint32_t b = outd; b; b &= b - 1u) {
            const int k = __ffs(b) - 1;
            const float2 p = reinterpret_cast<const float2 *>(pts)[item_point<G>(base, t, 8 * half + k)];
            if (fan_inside(sv, cx, cy, p)) in |= 1u << k;
        }
        return in << (8 * half);
    }
    uint32_t und = 0;
    in = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int f = fan_signs_f32(sv, cx, cy, px[k], py[k]);
        in |= (f == 1 ? 1u : 0u) << k;
        und |= (f == 2 ? 1u : 0u) << k;
    }
    in = (in & live) | (live & ~outd);
    und &= outd;
    while (und) {
        const int k = __ffs(und) - 1;
        und &= und - 1u;
        const float2 p = reinterpret_cast<const float2 *>(pts)[item_point<G>(base, t, 8 * half + k)];
        if (fan_inside_exact(sv, cx, cy, p.x, p.y)) in |= 1u << k;
    }
    return in << (8 * half);
}

// The tiles of the filter go in contiguous ranges to groups of
// kFiltThreads threads (four per block); thread t of a group holds the 16
// keep bits of filter thread t.  Kept points strictly inside the fan lose
// their keep bit, and the tile's count and its count block's total drop by
// the number removed (atomics: no barrier in the loop), so the filter's
// scatter pass writes only the points that survive both tests.
template <int G>
__global__ void __launch_bounds__(CT, 1) fan_refine_kernel(const float *__restrict__ pts, int64_t n, void *ws,
                                                          Layout L, int32_t bc)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sv = reinterpret_cast<float2 *>(smem_raw);   // kFanBins vertices
    const Octagon *oct = at<Octagon>(ws, L.oct);
    KgonCtrl *kc = at<KgonCtrl>(ws, L.kgon_ctrl);
    uint32_t s;
    if (!fan_live(kc, oct, s)) return;
    const Kgon *g = at<Kgon>(ws, L.kgon);
    if (!g->ok || !fan_worth(kc, n, s)) return;
    {
        const float4 *src = reinterpret_cast<const float4 *>(g->v);
        float4 *dst = reinterpret_cast<float4 *>(sv);
        for (int i = threadIdx.x; i < kFanBins / 2; i += CT) dst[i] = __ldg(src + i);
    }
    const float cx = g->cx, cy = g->cy;
    // -1: no disk (the test never passes for r2 >= 0)
    // (the triangles wind around c only with three distinct vertices or more)
    const float rho2t = (g->disk_bad || g->disk_edges < 3u)
                            ? -1.0f
                            : __double2float_rd(__longlong_as_double((long long)g->rho2) * (1.0 - 0x1p-20));
    bool use_disk = rho2t > 0.0f;
    __syncthreads();
    uint16_t *bits = at<uint16_t>(ws, L.keep_bits);
    unsigned long long *status = at<unsigned long long>(ws, L.filt_status);
    uint32_t *bsum = at<uint32_t>(ws, L.filt_bsum);
    const int64_t ntiles = ceil_div(n, kFiltTile);
    const int64_t per_block = ceil_div(ntiles, (int64_t)bc);   // tiles per count block
    const uint32_t grp = threadIdx.x / kFiltThreads, t = threadIdx.x % kFiltThreads, lane = lane_id();
    const int64_t groups = (int64_t)gridDim.x * CG, gi = (int64_t)blockIdx.x * CG + grp;
    const int64_t per = ceil_div(ntiles, groups);
    const int64_t t1 = std::min<int64_t>(ntiles, (gi + 1) * per);
    for (int64_t tile = gi * per; tile < t1; ++tile) {
        const int64_t base = tile * kFiltTile;
        if (t == 0 && tile + 1 < t1) {   // the next tile streams into L2 meanwhile
            const uint32_t nn = (uint32_t)std::min<int64_t>(kFiltTile, n - base - kFiltTile);
            if (((reinterpret_cast<uintptr_t>(pts + 2 * (base + kFiltTile))) & 15u) == 0)
                bulk_prefetch_l2(pts + 2 * (base + kFiltTile), (nn * 8u) & ~15u);
        }
        const uint32_t kb = bits[tile * kFiltThreads + t];
        uint32_t in = 0;
        // every lane takes both halves (refine_half has a warp-wide
        // reduction; a half without kept points costs little)
#pragma unroll 1
        for (int half = 0; half < 2; ++half)
            in |= refine_half<G>(pts, n, base, t, kb, half, sv, cx, cy, rho2t, use_disk);
        if (in) bits[tile * kFiltThreads + t] = (uint16_t)(kb & ~in);
        uint32_t removed = __popc(in);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) removed += __shfl_xor_sync(0xffffffffu, removed, o);
        if (lane == 0 && removed) {
            atomicAdd(&status[tile], 0ull - (unsigned long long)removed);   // count - removed >= 0
            atomicSub(&bsum[tile / per_block], removed);
        }
    }
}

}  // namespace

cudaError_t launch_fan(const float *pts, int64_t n, bool vec, int64_t filter_blocks, void *ws, const Layout &L,
                       cudaStream_t st)
{
    const int sms = sm_count();
    static const bool attrs = [] {
        cudaFuncSetAttribute(fan_refine_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFanSmem);
        cudaFuncSetAttribute(fan_refine_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFanSmem);
        return true;
    }();
    (void)attrs;
    const int32_t bc = (int32_t)filter_blocks;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(sms, filter_blocks));
    probe_before(CH_K_KGON, st);
    fan_build_kernel<<<kFanBins / BT, BT, 0, st>>>(pts, n, ws, L, bc);
    fan_estimate_kernel<<<sms, 256, 0, st>>>(pts, n, ws, L);
    if (vec) fan_refine_kernel<2><<<(unsigned)grid, CT, kFanSmem, st>>>(pts, n, ws, L, bc);
    else fan_refine_kernel<1><<<(unsigned)grid, CT, kFanSmem, st>>>(pts, n, ws, L, bc);
    note_kernels(CH_K_KGON, 3);
    probe_after(CH_K_KGON, st);
    return cudaGetLastError();
}

namespace {

// ---------------------------------------------------------------------------
// second level, over the first level's survivors (the filter's scatter
// output: sort keys and payloads in point order).  On the unit circle the
// binary32 points scatter about 10^-7 around the circle while a chord of
// the first fan sags 6 10^-9 below it, so a fan vertex, the farthest
// sampled point of its bin, leaves the points near the top of that scatter
// outside its triangles: about a sixth of the points reach the sort.  The
// same test with kFan2Sub times as many bins, each vertex the farthest
// survivor of its sub-bin (every survivor, not a sample), drops most of
// those.  The vertices are again input points and the centre is the
// first level's, so the same argument holds: a survivor strictly inside a
// triangle (c, v, w) is no hull vertex.  Kernels (grid-wide passes, after
// the scatter):
//
//  fan2_max_kernel      whether the level runs (the first level's centre
//                       was proven inside and at least kFan2MinS points,
//                       or the tuned minimum, survived); per sub-bin the
//                       farthest survivor
//  fan2_build_kernel    the vertex of every sub-bin (the previous
//                       non-empty one for an empty sub-bin, cyclically)
//  fan2_test_kernel     per tile of 4096 survivors the exact test, keep bits
//                       and counts (in the filter's keep-bit, tile-count and
//                       block-total buffers, free by then)
//  fan2_scatter_kernel  the kept survivors, in their order, into the sort's
//                       second buffers; the sort then reads those
// ---------------------------------------------------------------------------
constexpr int F2T = 256;
static_assert(kFan2Bins % BT == 0, "sub-bins split evenly over the build blocks");
static_assert(F2T == kFiltThreads, "the test pass keeps the filter's keep-bit layout");

__device__ __forceinline__ float2 surv_point(const uint32_t *keys, const unsigned long long *pay, uint32_t i)
{
    return make_float2(key_float(keys[i]), key_float((uint32_t)(pay[i] >> 32)));
}

__global__ void __launch_bounds__(F2T) fan2_max_kernel(void *ws, Layout L, uint32_t min_s)
{
    const Octagon *oct = at<Octagon>(ws, L.oct);
    const Kgon *g = at<Kgon>(ws, L.kgon);
    const uint32_t m = at<Ctrl>(ws, L.ctrl)->surv_count;
    // g->ok is this call's: the fan kernels ran before (they clear it when
    // the fan does not run)
    const bool on = !oct->abort && g->ok && m >= min_s;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Fan2Ctrl *f2 = at<Fan2Ctrl>(ws, L.fan2);
        f2->on = on ? 1u : 0u;
        f2->count_in = on ? m : 0u;
    }
    if (!on) return;
    const uint32_t *keys = at<uint32_t>(ws, L.keys[0]);
    const unsigned long long *pay = at<unsigned long long>(ws, L.pay[0]);
    unsigned long long *slot = at<unsigned long long>(ws, L.fan2_slot);
    const float cx = g->cx, cy = g->cy, r2ref = far_ref(*oct);
    for (uint32_t i = blockIdx.x * F2T + threadIdx.x; i < m; i += gridDim.x * F2T) {
        const float2 p = surv_point(keys, pay, i);
        const float dx = __fsub_rn(p.x, cx), dy = __fsub_rn(p.y, cy);
        const int b = fan_bin<kFan2Bins>(dx, dy);
        const unsigned long long v = ((unsigned long long)far_key(p.x, p.y, cx, cy, r2ref) << 32) | (uint32_t)~i;
        if (v > __ldcg(&slot[b])) atomicMax(&slot[b], v);   // the read only saves atomics
    }
}

// One thread per sub-bin, as fan_build_kernel.
__global__ void __launch_bounds__(BT) fan2_build_kernel(void *ws, Layout L)
{
    __shared__ int s_w[BT / 32];
    __shared__ int s_scan[BT / 32];
    Fan2Ctrl *f2 = at<Fan2Ctrl>(ws, L.fan2);
    if (!f2->on) return;
    const unsigned long long *slot = at<unsigned long long>(ws, L.fan2_slot);
    const uint32_t *keys = at<uint32_t>(ws, L.keys[0]);
    const unsigned long long *pay = at<unsigned long long>(ws, L.pay[0]);
    float2 *V = at<float2>(ws, L.fan2_v);
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const int b = (int)(blockIdx.x * BT + tid);
    const unsigned long long mine = slot[b];
    int incl = mine != 0ull ? b : -1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl = max(incl, u);
    }
    if (lane == 31) s_scan[warp] = incl;
    __syncthreads();
    for (int w = 0; w < (int)warp; ++w) incl = max(incl, s_scan[w]);
    int prev = -1;
    for (uint32_t k = 1; k <= gridDim.x && prev < 0; ++k) {   // prev is block-uniform
        const uint32_t rb = (blockIdx.x + gridDim.x - k) % gridDim.x;
        const int j = (int)(rb * BT + tid);
        prev = block_max(slot[j] != 0ull ? j : -1, s_w);
    }
    if (prev < 0) {   // no survivor reached a slot: keep everything
        if (tid == 0) f2->bad = 1u;
        return;
    }
    const int cur = incl >= 0 ? incl : prev;
    const uint32_t i = ~(uint32_t)(cur == b ? mine : slot[cur]);
    V[b] = surv_point(keys, pay, i);
}

// Per-tile survivor counts of a window of tiles, added up in shared memory
// as the warps finish each tile (as in the filter's count pass).
constexpr int kF2Ring = 256;

__global__ void __launch_bounds__(F2T) fan2_test_kernel(void *ws, Layout L)
{
    __shared__ uint32_t s_cnt[kF2Ring];
    __shared__ uint32_t s_w[F2T / 32];
    const Fan2Ctrl *f2 = at<Fan2Ctrl>(ws, L.fan2);
    if (!f2->on) return;
    const uint32_t m = f2->count_in;
    const bool none = f2->bad != 0u;
    const Kgon *g = at<Kgon>(ws, L.kgon);
    const float cx = g->cx, cy = g->cy;
    const float2 *V = at<float2>(ws, L.fan2_v);
    const uint32_t *keys = at<uint32_t>(ws, L.keys[0]);
    const unsigned long long *pay = at<unsigned long long>(ws, L.pay[0]);
    uint16_t *bits = at<uint16_t>(ws, L.keep_bits);
    unsigned long long *status = at<unsigned long long>(ws, L.filt_status);
    for (int i = threadIdx.x; i < kF2Ring; i += F2T) s_cnt[i] = 0u;
    __syncthreads();
    const int64_t ntiles = ceil_div((int64_t)m, kFiltTile);
    const int64_t per = ceil_div(ntiles, (int64_t)gridDim.x);
    const int64_t t1 = std::min<int64_t>(ntiles, (int64_t)(blockIdx.x + 1) * per);
    uint32_t part = 0;
    for (int64_t w0 = (int64_t)blockIdx.x * per; w0 < t1; w0 += kF2Ring) {
        const int64_t w1 = std::min<int64_t>(t1, w0 + kF2Ring);
        for (int64_t tile = w0; tile < w1; ++tile) {
            const uint32_t base = (uint32_t)(tile * kFiltTile);
            uint32_t keep = 0;
            // eight survivors at a time: binary32 signs without branches (the
            // table loads of the eight overlap), then the exact tiers for
            // the undecided ones
#pragma unroll 1
            for (int h = 0; h < kFiltItems / 8; ++h) {
                float2 q[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t i = base + (8 * h + k) * F2T + threadIdx.x;
                    q[k] = i < m ? surv_point(keys, pay, i) : make_float2(cx, cy);
                }
                uint32_t live = 0, in = 0, und = 0;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    live |= (base + (8 * h + k) * F2T + threadIdx.x < m ? 1u : 0u) << k;
                    const int f = fan_signs_f32<kFan2Bins>(V, cx, cy, q[k].x, q[k].y);
                    in |= (f == 1 ? 1u : 0u) << k;
                    und |= (f == 2 ? 1u : 0u) << k;
                }
                und &= live;   // (positions past the list hold the centre: never read again)
                while (und) {
                    const int k = __ffs(und) - 1;
                    und &= und - 1u;
                    const float2 p = surv_point(keys, pay, base + (8 * h + k) * F2T + threadIdx.x);
                    if (fan_inside_exact<kFan2Bins>(V, cx, cy, p.x, p.y)) in |= 1u << k;
                }
                keep |= (live & (none ? 0xffu : ~in)) << (8 * h);
            }
            bits[tile * F2T + threadIdx.x] = (uint16_t)keep;
            uint32_t c = __popc(keep);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            if (lane_id() == 0 && c) atomicAdd(&s_cnt[tile - w0], c);
        }
        __syncthreads();
        for (int64_t i = threadIdx.x; i < w1 - w0; i += F2T) {
            const uint32_t v = s_cnt[i];
            status[w0 + i] = v;
            s_cnt[i] = 0u;
            part += v;
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane_id() == 0) s_w[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < F2T / 32; ++w) t += s_w[w];
        at<uint32_t>(ws, L.filt_bsum)[blockIdx.x] = t;
    }
}

// One warp writes the kept survivors of one tile in order (thread t of the
// test pass held items base + r * 256 + t, r < 16: eight groups of 32
// threads, each row's first output position from the warp's row counts).
__device__ __forceinline__ void fan2_scatter_tile(const uint32_t *__restrict__ keys,
                                                  const unsigned long long *__restrict__ pay,
                                                  const uint16_t *__restrict__ tbits, uint32_t base, uint32_t out_off,
                                                  uint32_t *out_keys, unsigned long long *out_pay)
{
    const uint32_t lane = lane_id(), lt = (1u << lane) - 1u;
    uint32_t kb[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) kb[k] = tbits[k * 32 + lane];
    uint32_t racc[kFiltItems];
    {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) w[j] = kb[2 * j] | (kb[2 * j + 1] << 16);
        uint32_t run = out_off;
#pragma unroll
        for (int r = 0; r < kFiltItems; ++r) {
            uint32_t c = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) c += __popc(w[j] & (0x10001u << r));
            racc[r] = run;
            run += __reduce_add_sync(0xffffffffu, c);
        }
    }
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
        const uint32_t kbk = tbits[k * 32 + lane];
        if (!__any_sync(0xffffffffu, kbk != 0u)) continue;
        const uint32_t t = k * 32 + lane;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t kv[8];
            unsigned long long pv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int r = 8 * h + q;
                kv[q] = 0u;
                pv[q] = 0ull;
                if ((kbk >> r) & 1u) {
                    kv[q] = keys[base + r * F2T + t];
                    pv[q] = pay[base + r * F2T + t];
                }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int r = 8 * h + q;
                const uint32_t mk = (kbk >> r) & 1u;
                const uint32_t b0 = __ballot_sync(0xffffffffu, mk);
                if (!b0) continue;
                const uint32_t pos = racc[r] + __popc(b0 & lt);
                racc[r] += __popc(b0);
                if (mk) {
                    out_keys[pos] = kv[q];
                    out_pay[pos] = pv[q];
                }
            }
        }
    }
}

// Launched with the test pass's grid: block b owns the same tile range, its
// output offset the earlier blocks' totals.  Block 0 hands the kept list to
// the sort (count, buffer 1).
__global__ void __launch_bounds__(F2T) fan2_scatter_kernel(void *ws, Layout L)
{
    __shared__ uint32_t s_red[2][F2T / 32];
    __shared__ uint32_t s_list[F2T];
    __shared__ uint32_t s_loff[F2T];
    __shared__ uint32_t s_nlist;
    const Fan2Ctrl *f2 = at<Fan2Ctrl>(ws, L.fan2);
    if (!f2->on) return;
    const uint32_t m = f2->count_in;
    const unsigned long long *status = at<unsigned long long>(ws, L.filt_status);
    const uint32_t *bsum = at<uint32_t>(ws, L.filt_bsum);
    const uint16_t *bits = at<uint16_t>(ws, L.keep_bits);
    const uint32_t *keys = at<uint32_t>(ws, L.keys[0]);
    const unsigned long long *pay = at<unsigned long long>(ws, L.pay[0]);
    uint32_t *out_keys = at<uint32_t>(ws, L.keys[1]);
    unsigned long long *out_pay = at<unsigned long long>(ws, L.pay[1]);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    constexpr int NWF = F2T / 32;
    uint32_t before = 0, total = 0;
    for (uint32_t i = tid; i < gridDim.x; i += F2T) {
        const uint32_t v = bsum[i];
        total += v;
        if (i < blockIdx.x) before += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        before += __shfl_xor_sync(0xffffffffu, before, o);
        total += __shfl_xor_sync(0xffffffffu, total, o);
    }
    if (lane == 0) {
        s_red[0][warp] = before;
        s_red[1][warp] = total;
    }
    __syncthreads();
    before = total = 0;
#pragma unroll
    for (int w = 0; w < NWF; ++w) {
        before += s_red[0][w];
        total += s_red[1][w];
    }
    if (blockIdx.x == 0 && tid == 0) {
        Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
        ctrl->surv_count = total;
        ctrl->sort_in = 1u;
    }
    __syncthreads();   // s_red is reused below
    const int64_t ntiles = ceil_div((int64_t)m, kFiltTile);
    const int64_t per = ceil_div(ntiles, (int64_t)gridDim.x);
    const int64_t r0 = (int64_t)blockIdx.x * per, r1 = std::min<int64_t>(ntiles, r0 + per);
    uint32_t run = before;
    for (int64_t c0 = r0; c0 < r1; c0 += F2T) {
        const int64_t t = c0 + tid;
        const uint32_t cnt = t < r1 ? (uint32_t)(status[t] & 0xffffffffull) : 0u;
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += u;
        }
        const uint32_t nz = __ballot_sync(0xffffffffu, cnt != 0u);
        if (lane == 31) {
            s_red[0][warp] = incl;
            s_red[1][warp] = __popc(nz);
        }
        __syncthreads();
        uint32_t wbefore = 0, chunk_total = 0, lbefore = 0, nlist = 0;
#pragma unroll
        for (int w = 0; w < NWF; ++w) {
            if (w < (int)warp) {
                wbefore += s_red[0][w];
                lbefore += s_red[1][w];
            }
            chunk_total += s_red[0][w];
            nlist += s_red[1][w];
        }
        if (cnt != 0u) {
            const uint32_t slot = lbefore + __popc(nz & ((1u << lane) - 1u));
            s_list[slot] = tid;
            s_loff[slot] = run + wbefore + incl - cnt;
        }
        if (tid == 0) s_nlist = nlist;
        __syncthreads();
        const uint32_t nl = s_nlist;
        for (uint32_t li = warp; li < nl; li += NWF) {
            const int64_t tile = c0 + s_list[li];
            fan2_scatter_tile(keys, pay, bits + tile * F2T, (uint32_t)(tile * kFiltTile), s_loff[li], out_keys,
                              out_pay);
        }
        __syncthreads();   // s_list, s_loff and s_red are rebuilt for the next chunk
        run += chunk_total;
    }
}

}  // namespace

cudaError_t launch_fan2(int64_t n, void *ws, const Layout &L, cudaStream_t st)
{
    if (L.fan2_bins == 0) return cudaSuccess;   // a set too small for the second level
    const int sms = sm_count();
    const int64_t tiles = ceil_div(n, kFiltTile);   // survivor tiles at most
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>((int64_t)sms * 4, kFiltMaxBlocks), tiles));
    probe_before(CH_K_KGON, st);
    const int lg = tune_value(CH_TUNE_FAN2_MIN_LOG2);
    const uint32_t min_s = lg ? (uint32_t)(1ull << lg) : kFan2MinS;
    fan2_max_kernel<<<sms * 8, F2T, 0, st>>>(ws, L, min_s);
    fan2_build_kernel<<<kFan2Bins / BT, BT, 0, st>>>(ws, L);
    fan2_test_kernel<<<(unsigned)grid, F2T, 0, st>>>(ws, L);
    fan2_scatter_kernel<<<(unsigned)grid, F2T, 0, st>>>(ws, L);
    note_kernels(CH_K_KGON, 4);
    probe_after(CH_K_KGON, st);
    return cudaGetLastError();
}

namespace {

// ---------------------------------------------------------------------------
// many sets (ch_hull_batched): the same fan for every set with at least
// kKgonMinS octagon survivors, between the batched count pass and its scan
// ---------------------------------------------------------------------------
constexpr int kBxBinStride = 2;   // built-in: the bins see every 2nd tile of a set (1 and 4 measured slower overall)

// One block: numbers the sets that get a fan and lays out the refine's
// work items (runs of up to kBxFanChunk tiles of one such set).
__global__ void __launch_bounds__(1024) bx_fan_select_kernel(void *ws, Layout L, BatchLayout BL, uint32_t chunk)
{
    __shared__ uint32_t s_w[2][32];
    BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    const SetInfo *sets = at<SetInfo>(ws, BL.sets);
    const Octagon *octs = at<Octagon>(ws, BL.octs);
    const uint32_t *soct = at<uint32_t>(ws, BL.soct);
    const uint32_t *nonfin = at<uint32_t>(ws, BL.nonfinite);
    int32_t *fan_id = at<int32_t>(ws, BL.fan_id);
    uint32_t *fan_set = at<uint32_t>(ws, BL.fan_set);
    uint2 *items = at<uint2>(ws, BL.fan_items);
    const int64_t B = BL.num_sets;
    const bool off = bc->abort != 0;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const int64_t per = ceil_div(B, (int64_t)blockDim.x);
    const int64_t b0 = min((int64_t)threadIdx.x * per, B), b1 = min(b0 + per, B);
    auto wants = [&](int64_t b) {
        return !off && soct[b] >= kKgonMinS && !octs[b].abort && octs[b].has_edges && nonfin[b] == 0u;
    };
    uint32_t nf = 0, ni = 0;
    for (int64_t b = b0; b < b1; ++b)
        if (wants(b)) {
            ++nf;
            ni += (uint32_t)ceil_div((int64_t)sets[b].ntiles, (int64_t)chunk);
        }
    uint32_t inf = nf, ini = ni;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t a = __shfl_up_sync(0xffffffffu, inf, o), c = __shfl_up_sync(0xffffffffu, ini, o);
        if (lane >= (uint32_t)o) {
            inf += a;
            ini += c;
        }
    }
    if (lane == 31) {
        s_w[0][warp] = inf;
        s_w[1][warp] = ini;
    }
    __syncthreads();
    uint32_t bf = 0, bi = 0, tf = 0, ti = 0;
    for (uint32_t w = 0; w < blockDim.x / 32; ++w) {
        if (w < warp) {
            bf += s_w[0][w];
            bi += s_w[1][w];
        }
        tf += s_w[0][w];
        ti += s_w[1][w];
    }
    uint32_t f = bf + inf - nf, it = bi + ini - ni;
    for (int64_t b = b0; b < b1; ++b) {
        if (wants(b) && f < (uint32_t)BL.max_fan) {
            fan_id[b] = (int32_t)f;
            fan_set[f] = (uint32_t)b;
            for (uint32_t c = 0; c < sets[b].ntiles; c += chunk) items[it++] = make_uint2(f, sets[b].tile_base + c);
            ++f;
        } else {
            fan_id[b] = -1;
        }
    }
    if (threadIdx.x == 0) {
        bc->nfan = min(tf, (uint32_t)BL.max_fan);
        bc->nitems = min(ti, (uint32_t)BL.max_items);
    }
}

// Per work item, every kBxBinStride-th tile (counted from the set's first):
// each point's bin around the set's box centre, packed (far_key << 32 |
// ~index) into the fan's global slots by atomicMax (the read first saves
// most atomics).
__global__ void __launch_bounds__(FT) bx_fan_bins_kernel(const float *__restrict__ pts, void *ws, Layout L,
                                                         BatchLayout BL, uint32_t chunk, uint32_t stride)
{
    const BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    const SetInfo *sets = at<SetInfo>(ws, BL.sets);
    const Octagon *octs = at<Octagon>(ws, BL.octs);
    const uint32_t *fan_set = at<uint32_t>(ws, BL.fan_set);
    const uint2 *items = at<uint2>(ws, BL.fan_items);
    unsigned long long *slots = at<unsigned long long>(ws, BL.fan_slot);
    const uint32_t nitems = bc->nitems;
    for (uint32_t w = blockIdx.x; w < nitems; w += gridDim.x) {
        const uint2 item = items[w];
        const uint32_t b = fan_set[item.x];
        const SetInfo &S = sets[b];
        const float cx = octs[b].cx, cy = octs[b].cy, r2ref = far_ref(octs[b]);
        const float2 *p2 = reinterpret_cast<const float2 *>(pts) + S.pt_begin;
        unsigned long long *sl = slots + (size_t)item.x * kFanBins;
        const uint32_t tend = min(item.y + chunk, S.tile_base + S.ntiles);
        for (uint32_t t = item.y; t < tend; ++t) {
            if ((t - S.tile_base) % stride) continue;
            const int64_t lo = (int64_t)(t - S.tile_base) * kFiltTile, hi = min(lo + kFiltTile, S.n);
            float2 p[FITEMS];
#pragma unroll
            for (int r = 0; r < FITEMS; ++r) {
                const int64_t i = lo + r * FT + threadIdx.x;
                p[r] = i < hi ? __ldg(p2 + i) : make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int r = 0; r < FITEMS; ++r) {
                const int64_t i = lo + r * FT + threadIdx.x;
                if (i < hi) {
                    const float dx = p[r].x - cx, dy = p[r].y - cy;
                    const int bin = fan_bin(dx, dy);
                    const unsigned long long v =
                        ((unsigned long long)far_key(p[r].x, p[r].y, cx, cy, r2ref) << 32) | (uint32_t)~(uint32_t)i;
                    if (v > __ldcg(sl + bin)) atomicMax(sl + bin, v);
                }
            }
        }
    }
}

// One block per fan (grid-stride): the exact centre check against the
// set's octagon, then every bin's vertex (the sampled point of the last
// non-empty bin at or before it, cyclically), and the slots are left zero
// for the next call.  Thread t owns the kBinsPerThread consecutive bins
// from t * kBinsPerThread: a scan in registers, one block scan of the
// threads' last non-empty bins.
constexpr int kBinsPerThread = kFanBins / BT;
static_assert(kFanBins % BT == 0, "bins split evenly over the threads");

__global__ void __launch_bounds__(BT) bx_fan_build_kernel(const float *__restrict__ pts, void *ws, Layout L,
                                                          BatchLayout BL)
{
    __shared__ int s_w[BT / 32];
    __shared__ int s_ok;
    const BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    const SetInfo *sets = at<SetInfo>(ws, BL.sets);
    const Octagon *octs = at<Octagon>(ws, BL.octs);
    const uint32_t *fan_set = at<uint32_t>(ws, BL.fan_set);
    uint32_t *fan_ok = at<uint32_t>(ws, BL.fan_ok);
    float2 *fan_c = at<float2>(ws, BL.fan_c);
    unsigned long long *slots = at<unsigned long long>(ws, BL.fan_slot);
    float2 *verts = at<float2>(ws, BL.fan_v);
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const uint32_t nfan = bc->nfan;
    for (uint32_t k = blockIdx.x; k < nfan; k += gridDim.x) {
        const uint32_t b = fan_set[k];
        const Octagon &oct = octs[b];
        const float cx = oct.cx, cy = oct.cy;
        unsigned long long *sl = slots + (size_t)k * kFanBins + (size_t)tid * kBinsPerThread;
        float2 *V = verts + (size_t)k * kFanBins + (size_t)tid * kBinsPerThread;
        const float2 *p2 = reinterpret_cast<const float2 *>(pts) + sets[b].pt_begin;
        const int64_t nb = sets[b].n;
        __syncthreads();   // shared words of the previous fan have been read
        if (tid == 0) s_ok = 1;
        __syncthreads();
        if (tid < 8 && ((oct.valid >> tid) & 1u) && orient(oct.ax[tid], oct.ay[tid], oct.bx[tid], oct.by[tid], cx, cy) <= 0)
            s_ok = 0;
        // this thread's bins: the point index of each non-empty one, ~0u empty
        uint32_t idx[kBinsPerThread];
        int mylast = -1;
#pragma unroll
        for (int j = 0; j < kBinsPerThread; ++j) {
            const unsigned long long v = __ldcg(sl + j);
            idx[j] = v != 0ull ? ~(uint32_t)v : ~0u;
            if (v != 0ull) mylast = j;
        }
        // the last non-empty bin of the threads before this one (exclusive
        // max-scan over thread order), and the last overall (wrap-around)
        int incl = mylast >= 0 ? (int)(tid * kBinsPerThread) + mylast : -1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl = max(incl, u);
        }
        int excl = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) excl = -1;
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        int before = -1, last = -1;
        for (uint32_t w = 0; w < BT / 32; ++w) {
            if (w < warp) before = max(before, s_w[w]);
            last = max(last, s_w[w]);
        }
        before = max(before, excl);
        const bool live = s_ok && last >= 0;
        if (live) {
            // the vertex index of a bin with no sample: that of the last
            // non-empty bin before it (cyclically); it lies in another
            // thread's range, read from the slots (not zeroed yet)
            int cur = before >= 0 ? before : last;
            uint32_t ci = ~(uint32_t)__ldcg(slots + (size_t)k * kFanBins + cur);
#pragma unroll
            for (int j = 0; j < kBinsPerThread; ++j) {
                if (idx[j] != ~0u) ci = idx[j];
                V[j] = __ldg(p2 + ((int64_t)ci < nb ? ci : 0u));
            }
        }
        __syncthreads();   // every read of the slots is done
#pragma unroll
        for (int j = 0; j < kBinsPerThread; ++j) sl[j] = 0ull;
        if (tid == 0) {
            fan_ok[k] = live ? 1u : 0u;
            fan_c[k] = make_float2(cx, cy);
        }
    }
}

// Persistent blocks take work items by ticket; the 28672 vertices of the
// item's fan are loaded into shared memory when the fan changes (items of
// one fan are consecutive).  The four groups of kFiltThreads threads share
// the item's tiles; thread t holds the 16 keep bits of count-pass thread t
// (point lo + r * 256 + t for bit r).  Kept points strictly inside the fan
// lose their bit, and the tile's count drops by the number removed.
__global__ void __launch_bounds__(CT, 1) bx_fan_refine_kernel(const float *__restrict__ pts, void *ws, Layout L,
                                                              BatchLayout BL, uint32_t chunk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sv = reinterpret_cast<float2 *>(smem_raw);   // kFanBins vertices
    __shared__ uint32_t s_item;
    BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    const SetInfo *sets = at<SetInfo>(ws, BL.sets);
    const uint32_t *fan_set = at<uint32_t>(ws, BL.fan_set);
    const uint32_t *fan_ok = at<uint32_t>(ws, BL.fan_ok);
    const float2 *fan_c = at<float2>(ws, BL.fan_c);
    const float2 *verts = at<float2>(ws, BL.fan_v);
    const uint2 *items = at<uint2>(ws, BL.fan_items);
    uint16_t *bits = at<uint16_t>(ws, L.keep_bits);
    unsigned long long *status = at<unsigned long long>(ws, L.filt_status);
    const uint32_t nitems = bc->nitems;
    const uint32_t grp = threadIdx.x / kFiltThreads, t = threadIdx.x % kFiltThreads, lane = lane_id();
    int64_t cur = -1;
    for (;;) {
        __syncthreads();   // s_item of the previous item has been read
        if (threadIdx.x == 0) s_item = atomicAdd(&bc->fan_ticket, 1u);
        __syncthreads();
        const uint32_t w = s_item;
        if (w >= nitems) break;
        const uint2 item = items[w];
        if (!fan_ok[item.x]) continue;   // block-uniform
        if ((int64_t)item.x != cur) {
            const float4 *src = reinterpret_cast<const float4 *>(verts + (size_t)item.x * kFanBins);
            float4 *dst = reinterpret_cast<float4 *>(sv);
            for (int i = threadIdx.x; i < kFanBins / 2; i += CT) dst[i] = __ldg(src + i);
            __syncthreads();
            cur = item.x;
        }
        const SetInfo &S = sets[fan_set[item.x]];
        const float2 c = fan_c[item.x];
        const float2 *p2 = reinterpret_cast<const float2 *>(pts) + S.pt_begin;
        const uint32_t tend = min(item.y + chunk, S.tile_base + S.ntiles);
        for (uint32_t tile = item.y + grp; tile < tend; tile += CG) {
            const int64_t lo = (int64_t)(tile - S.tile_base) * kFiltTile;
            const uint32_t kb = bits[(size_t)tile * kFiltThreads + t];
            uint32_t in = 0;
            if (kb) {
                float2 p[kFiltItems];
#pragma unroll
                for (int r = 0; r < kFiltItems; ++r)
                    p[r] = ((kb >> r) & 1u) ? __ldcs(p2 + lo + r * kFiltThreads + t) : make_float2(0.0f, 0.0f);
                uint32_t und = 0;
#pragma unroll
                for (int r = 0; r < kFiltItems; ++r) {
                    const int f = fan_signs_f32(sv, c.x, c.y, p[r].x, p[r].y);
                    in |= (f == 1 ? 1u : 0u) << r;
                    und |= (f == 2 ? 1u : 0u) << r;
                }
                in &= kb;
                und &= kb;
                while (und) {
                    const int r = __ffs(und) - 1;
                    und &= und - 1u;
                    const float2 q = p2[lo + r * kFiltThreads + t];
                    if (fan_inside_exact(sv, c.x, c.y, q.x, q.y)) in |= 1u << r;
                }
                if (in) bits[(size_t)tile * kFiltThreads + t] = (uint16_t)(kb & ~in);
            }
            uint32_t removed = __popc(in);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) removed += __shfl_xor_sync(0xffffffffu, removed, o);
            if (lane == 0 && removed) atomicAdd(&status[tile], 0ull - (unsigned long long)removed);
        }
    }
}

}  // namespace

cudaError_t launch_bx_fan(const float *pts, void *ws, const Layout &L, const BatchLayout &BL, cudaStream_t st)
{
    const int sms = sm_count();
    static const bool attrs = [] {
        cudaFuncSetAttribute(bx_fan_refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFanSmem);
        return true;
    }();
    (void)attrs;
    const uint32_t chunk = tune_value(CH_TUNE_BX_FAN_CHUNK) ? (uint32_t)tune_value(CH_TUNE_BX_FAN_CHUNK) : kBxFanChunk;
    const uint32_t stride = tune_value(CH_TUNE_BX_FAN_STRIDE) ? (uint32_t)tune_value(CH_TUNE_BX_FAN_STRIDE)
                                                              : kBxBinStride;
    probe_before(CH_K_KGON, st);
    bx_fan_select_kernel<<<1, 1024, 0, st>>>(ws, L, BL, chunk);
    bx_fan_bins_kernel<<<(unsigned)(sms * 4), FT, 0, st>>>(pts, ws, L, BL, chunk, stride);
    bx_fan_build_kernel<<<(unsigned)(sms * 2), BT, 0, st>>>(pts, ws, L, BL);
    bx_fan_refine_kernel<<<(unsigned)sms, CT, kFanSmem, st>>>(pts, ws, L, BL, chunk);
    note_kernels(CH_K_KGON, 4);
    probe_after(CH_K_KGON, st);
    return cudaGetLastError();
}

}  // namespace ch

// kgon.cu -- a second throw-away step inside the device hull: a fan of
// triangles around an interior point.
//
// The octagon filter (Sec. 3.1-3.2) removes almost nothing from points near
// a circle, and on a displaced circle 95 % survive it, although the hulls
// have a small fraction of the points as vertices.  Before sorting the
// survivors the hull step repeats the throw-away idea of Sec. 3.1 on a much
// finer scale.  Let c be the centre of the bounding box, checked with exact
// signs to lie strictly inside the octagon, hence strictly inside the hull.
// The plane around c is cut into kFanBins angular bins; the vertex of a bin
// is the survivor farthest from c among a sample (every 4th 4096-point tile
// of the survivors), and a bin the sample missed repeats the vertex before
// it.  For consecutive vertices v, w every point strictly inside the
// triangle (c, v, w) is a combination of c, v and w with positive weights,
// so it lies strictly inside the hull and is no vertex of it: it is
// dropped.  This holds whatever the vertices are (they are input points),
// so nothing needs to be exact but the three orientation signs of the
// final test, and a triangle that comes out clockwise or flat drops
// nothing.
//
//  kgon_bins_kernel      per bin, the farthest sampled survivor (atomicMax
//                        of (r^2 bits << 32 | ~position), in shared memory
//                        per block, then in global memory)
//  kgon_build_kernel     exact centre check against the octagon; the vertex
//                        of every bin
//  kgon_estimate_kernel  exact test of a second sample: the pass runs when
//                        it drops at least an eighth
//  kgon_count_kernel     per 4096-survivor tile: exact test, keep bits,
//                        counts (the fan in shared memory)
//  kgon_scatter_kernel   stable compaction into the other sort buffer; sets
//                        the survivor count and the sort's input buffer
//
// Test of a point p: its bin b from a binary32 pseudo-angle (a hint only),
// v the vertex of b.  p strictly left of the ray c -> v: the triangle
// (c, v, next vertex); strictly right: (c, previous vertex, v); on it: kept.
#include <algorithm>

#include "common.cuh"
#include "launch.h"

namespace ch {
namespace {

constexpr int FT = 512;                  // threads per block of the bins pass
constexpr int FITEMS = 8;                // survivors per thread per tile there
constexpr int FTILE = FT * FITEMS;       // 4096
constexpr int CT = 1024;                 // threads per block of the count and scatter passes
constexpr int CITEMS = FTILE / CT;       // 4 survivors per thread per tile
constexpr int CNW = CT / 32;
constexpr int kTileSample = 4;           // the bins see every 4th tile
constexpr uint32_t kKgonMinS = 1u << 16; // fewer survivors: not worth a pass
constexpr int kFanSmem = kFanBins * 8;   // bins or vertices, 128 KB
// keep words: per tile, per warp, per row r the ballot of "kept" over the
// warp's lanes (survivor base + r * CT + warp * 32 + lane), in the filter's
// per-tile keep-bit scratch (512 B per 4096-point tile)
static_assert(FTILE == kFiltTile && CNW * CITEMS * 4 == kFiltThreads * 2, "keep words fit the filter's scratch");

__device__ __forceinline__ float2 survivor(const uint32_t *keys, const unsigned long long *pay, int64_t q)
{
    return make_float2(key_float(__ldg(keys + q)), key_float((uint32_t)(__ldg(pay + q) >> 32)));
}

// Bin of the direction (dx, dy): a pseudo-angle in [0, 4) that grows with
// the angle counter-clockwise from +x, scaled to the bins.  Any value is
// safe (it only picks a triangle); the conversion saturates and the result
// is clamped.
__device__ __forceinline__ int fan_bin(float dx, float dy)
{
    const float s = fabsf(dx) + fabsf(dy);
    float a = 0.0f;
    if (s > 0.0f) {
        const float t = __fdividef(dy, s);
        a = dx >= 0.0f ? (dy >= 0.0f ? t : 4.0f + t) : 2.0f - t;
    }
    const int b = __float2int_rz(a * (kFanBins / 4.0f));
    return b < 0 ? 0 : (b >= kFanBins ? kFanBins - 1 : b);
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
__device__ __forceinline__ int fan_signs_f32(const float2 *V, float cx, float cy, float px, float py)
{
    const int b = fan_bin(px - cx, py - cy);
    const float2 v = V[b];
    const int o = orient_f32(cx, cy, v.x, v.y, px, py);
    const float2 w = V[(b + (o == 1 ? 1 : -1)) & (kFanBins - 1)];
    const int e1 = orient_f32(v.x, v.y, w.x, w.y, px, py);
    const int e2 = orient_f32(w.x, w.y, cx, cy, px, py);
    const bool out = (e1 != 2 && e1 != o) || (e2 != 2 && e2 != o);
    return o == 2 ? 2 : (out ? 0 : (e1 == o && e2 == o ? 1 : 2));
}

__device__ __noinline__ bool fan_inside_exact(const float2 *V, float cx, float cy, float px, float py)
{
    const int b = fan_bin(px - cx, py - cy);
    const float2 v = V[b];
    const int o = orient(cx, cy, v.x, v.y, px, py);
    if (o == 0) return false;
    const float2 w = V[(b + o) & (kFanBins - 1)];
    return orient(v.x, v.y, w.x, w.y, px, py) == o && orient(w.x, w.y, cx, cy, px, py) == o;
}

__device__ __forceinline__ bool fan_inside(const float2 *V, float cx, float cy, float2 p)
{
    const int f = fan_signs_f32(V, cx, cy, p.x, p.y);
    return f != 2 ? f == 1 : fan_inside_exact(V, cx, cy, p.x, p.y);
}

__device__ __forceinline__ bool kgon_live(const Ctrl *ctrl, const Octagon *oct, uint32_t &s)
{
    s = oct->abort ? 0u : ctrl->surv_count;
    return s >= kKgonMinS && oct->has_edges;
}

__global__ void __launch_bounds__(FT) kgon_bins_kernel(void *ws, Layout L)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long *s_best = reinterpret_cast<unsigned long long *>(smem_raw);   // kFanBins
    const Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    const Octagon *oct = at<Octagon>(ws, L.oct);
    uint32_t s;
    if (!kgon_live(ctrl, oct, s)) return;
    for (int i = threadIdx.x; i < kFanBins; i += FT) s_best[i] = 0ull;
    __syncthreads();
    const float cx = oct->cx, cy = oct->cy;
    const uint32_t *keys = at<uint32_t>(ws, L.keys[0]);
    const unsigned long long *pay = at<unsigned long long>(ws, L.pay[0]);
    const int64_t ntiles = ceil_div((int64_t)s, FTILE);
    const int64_t nsamp = ceil_div(ntiles, kTileSample);
    for (int64_t k = blockIdx.x; k < nsamp; k += gridDim.x) {
        const int64_t base = k * kTileSample * FTILE;
        float x[FITEMS], y[FITEMS];
#pragma unroll
        for (int r = 0; r < FITEMS; ++r) {
            const int64_t q = base + r * FT + threadIdx.x;
            x[r] = y[r] = 0.0f;
            if (q < s) {
                x[r] = key_float(__ldg(keys + q));
                y[r] = key_float(__ldg(reinterpret_cast<const uint2 *>(pay) + q).y);
            }
        }
#pragma unroll
        for (int r = 0; r < FITEMS; ++r) {
            const int64_t q = base + r * FT + threadIdx.x;
            if (q < s) {
                const float dx = x[r] - cx, dy = y[r] - cy;
                const int b = fan_bin(dx, dy);
                const float r2 = __fmaf_rn(dx, dx, dy * dy);   // >= +0
                const unsigned long long v = ((unsigned long long)__float_as_uint(r2) << 32) | (uint32_t)~(uint32_t)q;
                if (v > s_best[b]) atomicMax(&s_best[b], v);   // the read only saves atomics
            }
        }
    }
    __syncthreads();
    KgonCtrl *kc = at<KgonCtrl>(ws, L.kgon_ctrl);
    for (int i = threadIdx.x; i < kFanBins; i += FT) {
        const unsigned long long v = s_best[i];
        if (v != 0ull && v > __ldcg(&kc->slot[i])) atomicMax(&kc->slot[i], v);
    }
}

// One block: each thread owns PER consecutive bins.  The vertex of bin b is
// the sampled survivor of the last non-empty bin at or before b, cyclically
// (a max-scan of "last non-empty bin" over the threads).
constexpr int BT = 1024;

__global__ void __launch_bounds__(BT) kgon_build_kernel(void *ws, Layout L)
{
    constexpr int PER = kFanBins / BT;
    static_assert(kFanBins % BT == 0, "bins split evenly over the threads");
    __shared__ int s_w[BT / 32];
    __shared__ int s_ok;
    const Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    const Octagon *oct = at<Octagon>(ws, L.oct);
    Kgon *g = at<Kgon>(ws, L.kgon);
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    uint32_t s;
    if (!kgon_live(ctrl, oct, s)) {
        if (tid == 0) g->ok = 0u;
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
    const KgonCtrl *kc = at<KgonCtrl>(ws, L.kgon_ctrl);
    unsigned long long sl[PER];
    int last = -1;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        sl[k] = kc->slot[tid * PER + k];
        if (sl[k] != 0ull) last = (int)(tid * PER + k);
    }
    int incl = last;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl = max(incl, u);
    }
    int ex = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) ex = -1;
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    int before = -1, all = -1;
    for (int w = 0; w < BT / 32; ++w) {
        if (w < (int)warp) before = max(before, s_w[w]);
        all = max(all, s_w[w]);
    }
    if (all < 0 || !s_ok) {   // block-uniform
        if (tid == 0) g->ok = 0u;
        return;
    }
    int cur = max(before, ex);
    if (cur < 0) cur = all;   // before the first non-empty bin: wrap to the last one
    const uint32_t *keys = at<uint32_t>(ws, L.keys[0]);
    const unsigned long long *pay = at<unsigned long long>(ws, L.pay[0]);
    unsigned long long cv = kc->slot[cur];
    float2 pv[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {   // all loads before the stores
        if (sl[k] != 0ull) cv = sl[k];
        const uint32_t pos = ~(uint32_t)cv;
        pv[k] = survivor(keys, pay, pos < s ? pos : 0u);
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) g->v[tid * PER + k] = pv[k];
    if (tid == 0) {
        g->cx = cx;
        g->cy = cy;
        g->ok = 1u;
    }
}

__global__ void __launch_bounds__(256) kgon_estimate_kernel(void *ws, Layout L)
{
    __shared__ uint32_t s_in[8], s_tot[8];
    const Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    uint32_t s;
    if (!kgon_live(ctrl, at<Octagon>(ws, L.oct), s)) return;
    const Kgon *g = at<Kgon>(ws, L.kgon);
    if (!g->ok) return;
    KgonCtrl *kc = at<KgonCtrl>(ws, L.kgon_ctrl);
    const uint32_t *keys = at<uint32_t>(ws, L.keys[0]);
    const unsigned long long *pay = at<unsigned long long>(ws, L.pay[0]);
    // about 2^16 evenly spaced survivors
    const int64_t stride = std::max<int64_t>(1, (int64_t)s >> 16);
    const int64_t nsamp = ((int64_t)s - stride / 2 + stride - 1) / stride;
    uint32_t in = 0, tot = 0;
    for (int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x; k < nsamp; k += (int64_t)gridDim.x * 256) {
        in += fan_inside(g->v, g->cx, g->cy, survivor(keys, pay, k * stride + stride / 2)) ? 1u : 0u;
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
}

// The pass runs when the sample says it removes at least an eighth.
__device__ __forceinline__ bool kgon_worth(const KgonCtrl *kc) { return kc->sample > 0u && kc->inside * 8u >= kc->sample; }

// Block b owns a contiguous range of tiles (the scatter pass uses the same
// grid and ranges).  No barrier inside the loop: every warp writes its own
// keep words, and the block's total is reduced once at the end.
__global__ void __launch_bounds__(CT, 1) kgon_count_kernel(void *ws, Layout L)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sv = reinterpret_cast<float2 *>(smem_raw);   // kFanBins vertices
    __shared__ uint32_t s_w[CNW];
    const Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    uint32_t s;
    if (!kgon_live(ctrl, at<Octagon>(ws, L.oct), s)) return;
    KgonCtrl *kc = at<KgonCtrl>(ws, L.kgon_ctrl);
    const Kgon *g = at<Kgon>(ws, L.kgon);
    if (!g->ok || !kgon_worth(kc)) return;
    {
        const float4 *src = reinterpret_cast<const float4 *>(g->v);
        float4 *dst = reinterpret_cast<float4 *>(sv);
        for (int i = threadIdx.x; i < kFanBins / 2; i += CT) dst[i] = __ldg(src + i);
    }
    const float cx = g->cx, cy = g->cy;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) kc->s_in = s;
    const uint32_t *keys = at<uint32_t>(ws, L.keys[0]);
    const unsigned long long *pay = at<unsigned long long>(ws, L.pay[0]);
    uint32_t *kw = at<uint32_t>(ws, L.keep_bits);
    const int64_t ntiles = ceil_div((int64_t)s, FTILE);
    const int64_t per = ceil_div(ntiles, (int64_t)gridDim.x);
    const int64_t t1 = std::min<int64_t>(ntiles, (int64_t)(blockIdx.x + 1) * per);
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    uint32_t warp_total = 0;
    for (int64_t tile = (int64_t)blockIdx.x * per; tile < t1; ++tile) {
        const int64_t base = tile * FTILE;
        if (threadIdx.x == 0 && tile + 1 < t1) {   // the next tile streams into L2 meanwhile
            const uint32_t nn = (uint32_t)std::min<int64_t>(FTILE, (int64_t)s - base - FTILE);
            bulk_prefetch_l2(keys + base + FTILE, (nn * 4u) & ~15u);
            bulk_prefetch_l2(pay + base + FTILE, (nn * 8u) & ~15u);
        }
        float x[CITEMS], y[CITEMS];
        const int64_t left = (int64_t)s - base - threadIdx.x;   // item r exists iff r * CT < left
#pragma unroll
        for (int r = 0; r < CITEMS; ++r) {
            const int64_t q = base + r * CT + threadIdx.x;
            x[r] = y[r] = 0.0f;
            if ((int64_t)r * CT < left) {
                x[r] = key_float(__ldg(keys + q));
                y[r] = key_float(__ldg(reinterpret_cast<const uint2 *>(pay) + q).y);
            }
        }
        // binary32 signs for every item first, exact ones for the few
        // undecided (both paths give the exact answer on every item they
        // decide)
        uint32_t keep = 0, undecided = 0, live = 0;
#pragma unroll
        for (int r = 0; r < CITEMS; ++r) {
            const int f = fan_signs_f32(sv, cx, cy, x[r], y[r]);
            keep |= (f == 0 ? 1u : 0u) << r;
            undecided |= (f == 2 ? 1u : 0u) << r;
            live |= ((int64_t)r * CT < left ? 1u : 0u) << r;
        }
        keep &= live;
        undecided &= live;
#pragma unroll
        for (int r = 0; r < CITEMS; ++r)
            if (((undecided >> r) & 1u) && !fan_inside_exact(sv, cx, cy, x[r], y[r])) keep |= 1u << r;
        uint32_t word = 0;
#pragma unroll
        for (int r = 0; r < CITEMS; ++r) {
            const uint32_t m = __ballot_sync(0xffffffffu, (keep >> r) & 1u);
            if (lane == (uint32_t)r) word = m;
            warp_total += __popc(m);
        }
        if (lane < (uint32_t)CITEMS) kw[tile * (CNW * CITEMS) + warp * CITEMS + lane] = word;
    }
    if (lane == 0) s_w[warp] = warp_total;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < CNW; ++w) t += s_w[w];
        at<uint32_t>(ws, L.filt_bsum)[blockIdx.x] = t;
    }
}

// Same grid as the count pass (block b owns the same tile range).  Per tile:
// each warp reads its four keep words and starts the loads of its kept
// survivors, then one warp scans the 128 (row, warp) counts in element order.
__global__ void __launch_bounds__(CT, 1) kgon_scatter_kernel(void *ws, Layout L)
{
    __shared__ uint32_t s_red[2][CNW];
    __shared__ uint32_t s_cnt[CITEMS * CNW];   // [r][warp]
    __shared__ uint32_t s_off[CITEMS * CNW];
    __shared__ uint32_t s_tot;
    __shared__ uint32_t s_flag;
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    KgonCtrl *kc = at<KgonCtrl>(ws, L.kgon_ctrl);
    if (threadIdx.x == 0) s_flag = kc->s_in != 0u;   // set by the count pass when it ran
    __syncthreads();
    if (!s_flag) return;
    const uint32_t s = kc->s_in;
    const uint32_t *keys = at<uint32_t>(ws, L.keys[0]);
    const unsigned long long *pay = at<unsigned long long>(ws, L.pay[0]);
    uint32_t *okeys = at<uint32_t>(ws, L.keys[1]);
    unsigned long long *opay = at<unsigned long long>(ws, L.pay[1]);
    const uint32_t *bsum = at<uint32_t>(ws, L.filt_bsum);
    const uint4 *kw = at<uint4>(ws, L.keep_bits);   // one uint4 (rows 0..3) per (tile, warp)
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = lane_id(), lt = (1u << lane) - 1u;
    uint32_t before = 0, total = 0;
    for (uint32_t i = tid; i < gridDim.x; i += CT) {
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
    for (int w = 0; w < CNW; ++w) {
        before += s_red[0][w];
        total += s_red[1][w];
    }
    if (blockIdx.x == 0 && tid == 0) {
        ctrl->surv_count = total;
        ctrl->sort_in = 1u;
    }
    const int64_t ntiles = ceil_div((int64_t)s, FTILE);
    const int64_t per = ceil_div(ntiles, (int64_t)gridDim.x);
    const int64_t r0 = (int64_t)blockIdx.x * per, r1 = std::min<int64_t>(ntiles, r0 + per);
    uint64_t run = before;
    for (int64_t tile = r0; tile < r1; ++tile) {
        const int64_t base = tile * FTILE;
        if (tid == 0 && tile + 1 < r1) {
            const uint32_t nn = (uint32_t)std::min<int64_t>(FTILE, (int64_t)s - base - FTILE);
            bulk_prefetch_l2(keys + base + FTILE, (nn * 4u) & ~15u);
            bulk_prefetch_l2(pay + base + FTILE, (nn * 8u) & ~15u);
        }
        const uint4 w4 = kw[tile * CNW + warp];
        const uint32_t wd[CITEMS] = {w4.x, w4.y, w4.z, w4.w};
        uint32_t kk[CITEMS];
        unsigned long long kp[CITEMS];
#pragma unroll
        for (int r = 0; r < CITEMS; ++r) {
            kk[r] = 0u;
            kp[r] = 0ull;
            if ((wd[r] >> lane) & 1u) {
                const int64_t q = base + r * CT + tid;
                kk[r] = __ldg(keys + q);
                kp[r] = __ldg(pay + q);
            }
        }
        if (lane < (uint32_t)CITEMS) s_cnt[lane * CNW + warp] = __popc(wd[lane]);
        __syncthreads();
        if (warp == 0) {   // exclusive scan of the counts in (row, warp) order
            constexpr int PER = CITEMS * CNW / 32;
            uint32_t loc[PER], sum = 0;
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                loc[k] = s_cnt[lane * PER + k];
                sum += loc[k];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (uint32_t)o) incl += t;
            }
            uint32_t ex = incl - sum;
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                s_off[lane * PER + k] = ex;
                ex += loc[k];
            }
            if (lane == 31) s_tot = incl;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < CITEMS; ++r) {
            if ((wd[r] >> lane) & 1u) {
                const uint64_t pos = run + s_off[r * CNW + warp] + __popc(wd[r] & lt);
                okeys[pos] = kk[r];
                opay[pos] = kp[r];
            }
        }
        run += s_tot;
    }
}

}  // namespace

cudaError_t launch_kgon(void *ws, const Layout &L, cudaStream_t st)
{
    const int sms = sm_count();
    static int per_sm = [] {
        cudaFuncSetAttribute(kgon_bins_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFanSmem);
        cudaFuncSetAttribute(kgon_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFanSmem);
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kgon_count_kernel, CT, kFanSmem);
        return v > 0 ? v : 1;
    }();
    const int64_t tiles = ceil_div(L.n, FTILE);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>({tiles, (int64_t)sms * per_sm, kFiltMaxBlocks}));
    probe_before(CH_K_KGON, st);
    kgon_bins_kernel<<<sms, FT, kFanSmem, st>>>(ws, L);
    kgon_build_kernel<<<1, BT, 0, st>>>(ws, L);
    kgon_estimate_kernel<<<sms, 256, 0, st>>>(ws, L);
    kgon_count_kernel<<<(unsigned)grid, CT, kFanSmem, st>>>(ws, L);
    kgon_scatter_kernel<<<(unsigned)grid, CT, 0, st>>>(ws, L);
    note_kernels(CH_K_KGON, 5);
    probe_after(CH_K_KGON, st);
    return cudaGetLastError();
}

}  // namespace ch

// kgon.cu -- a second throw-away polygon inside the device hull.
//
// The octagon filter (Sec. 3.1-3.2) removes nothing from points near a
// circle; on a displaced circle 95 % of the points survive it although the
// hull has a few thousand vertices.  Before sorting the survivors, the hull
// step therefore repeats the idea of the filter with more directions
// (Sec. 3.1 uses 8): the extreme survivors of a sample along kKgonDirs
// directions span a convex polygon whose vertices are input points, so every
// point strictly inside it is strictly inside the hull and cannot be a hull
// vertex -- the hull of the remaining points is the hull of all points,
// whatever the sample.  A second sample estimates how much the polygon
// removes; the pass over all survivors runs only when that pays.
//
//  kgon_extremes_kernel  argmax along each direction over a sample of the
//                        survivors (binary32 dot products: any survivor is a
//                        valid vertex, so no exactness is needed here)
//  kgon_build_kernel     one warp: the vertices' exact convex hull (Andrew's
//                        chain, exact orientation), counter-clockwise
//  kgon_estimate_kernel  exact inside test of a second sample
//  kgon_count_kernel     per 4096-survivor tile: exact test, keep bits, counts
//  kgon_scatter_kernel   stable compaction into the other sort buffer; sets
//                        the survivor count and the sort's input buffer
//
// Strictly inside a strictly convex counter-clockwise polygon v[0..m):
// strictly left of v0->v1 and of v[m-1]->v0, and strictly left of the edge
// v[i]->v[i+1] of the fan wedge from v0 that contains the point (found by a
// binary search in binary32, then verified with exact signs; an exact
// search follows when the verification fails).
#include <algorithm>

#include "common.cuh"
#include "launch.h"

namespace ch {
namespace {

constexpr int KT = 256;                 // threads per block
constexpr int KITEMS = 16;              // survivors per thread per tile
constexpr int KTILE = KT * KITEMS;      // 4096
constexpr int KNW = KT / 32;
constexpr uint32_t kKgonMinS = 1u << 16;   // fewer survivors: not worth a pass
constexpr int kSampleLog2 = 20;            // about 2^20 sample points

__device__ __forceinline__ float2 survivor(const uint32_t *keys, const unsigned long long *pay, int64_t q)
{
    return make_float2(key_float(__ldg(keys + q)), key_float((uint32_t)(__ldg(pay + q) >> 32)));
}

__device__ __forceinline__ bool left_strict(float ax, float ay, float bx, float by, float2 p)
{
    return orient(ax, ay, bx, by, p.x, p.y) > 0;
}

// Exact test; g in shared memory.
__device__ __forceinline__ bool kgon_inside(const Kgon &g, float2 p)
{
    const int m = (int)g.m;
    if (!left_strict(g.vx[0], g.vy[0], g.vx[1], g.vy[1], p)) return false;
    if (!left_strict(g.vx[m - 1], g.vy[m - 1], g.vx[0], g.vy[0], p)) return false;
    // wedge: largest i in [1, m-2] with p on or left of the ray v0 -> v[i]
    const float ox = g.vx[0], oy = g.vy[0];
    int lo = 1, hi = m - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        const float c = (g.vx[mid] - ox) * (p.y - oy) - (g.vy[mid] - oy) * (p.x - ox);
        if (c >= 0.0f) lo = mid;
        else hi = mid;
    }
    const bool ok_lo = lo == 1 || orient(ox, oy, g.vx[lo], g.vy[lo], p.x, p.y) >= 0;
    const bool ok_hi = hi == m - 1 || orient(ox, oy, g.vx[hi], g.vy[hi], p.x, p.y) < 0;
    if (!(ok_lo && ok_hi)) {   // the binary32 search was fooled: exact search
        lo = 1;
        hi = m - 1;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (orient(ox, oy, g.vx[mid], g.vy[mid], p.x, p.y) >= 0) lo = mid;
            else hi = mid;
        }
    }
    return left_strict(g.vx[lo], g.vy[lo], g.vx[hi], g.vy[hi], p);
}

__device__ __forceinline__ bool kgon_live(const Ctrl *ctrl, const Octagon *oct, uint32_t &s)
{
    s = oct->abort ? 0u : ctrl->surv_count;
    return s >= kKgonMinS;
}

__global__ void __launch_bounds__(KT) kgon_extremes_kernel(void *ws, Layout L)
{
    __shared__ float s_c[kKgonDirs], s_s[kKgonDirs];
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    uint32_t s;
    if (!kgon_live(ctrl, at<Octagon>(ws, L.oct), s)) return;
    KgonCtrl *kc = at<KgonCtrl>(ws, L.kgon_ctrl);
    for (int j = threadIdx.x; j < kKgonDirs; j += KT) {
        float sn, cs;
        sincospif((float)j * (2.0f / kKgonDirs), &sn, &cs);
        s_c[j] = cs;
        s_s[j] = sn;
    }
    __syncthreads();
    const uint32_t *keys = at<uint32_t>(ws, L.keys[0]);
    const unsigned long long *pay = at<unsigned long long>(ws, L.pay[0]);
    const uint32_t lane = lane_id();
    const int64_t stride = std::max<int64_t>(1, (int64_t)s >> kSampleLog2);
    const int64_t nsamp = ((int64_t)s + stride - 1) / stride;
    constexpr int PER = kKgonDirs / 32;   // directions owned by each lane
    float best[PER];
    uint32_t bpos[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        best[k] = -__int_as_float(0x7f800000);
        bpos[k] = 0xffffffffu;
    }
    const int64_t wid = ((int64_t)blockIdx.x * KT + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * KT) >> 5;
    for (int64_t g0 = wid * 32; g0 < nsamp; g0 += nw * 32) {
        const int64_t k = g0 + lane;
        const bool ok = k < nsamp;
        const uint32_t q = ok ? (uint32_t)(k * stride) : 0u;
        const float2 p = ok ? survivor(keys, pay, q) : make_float2(0.0f, 0.0f);
#pragma unroll 4
        for (int j = 0; j < kKgonDirs; ++j) {
            float v = ok ? __fmaf_rn(p.x, s_c[j], p.y * s_s[j]) : -__int_as_float(0x7f800000);
            uint32_t pos = ok ? q : 0xffffffffu;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
                const uint32_t p2 = __shfl_xor_sync(0xffffffffu, pos, o);
                if (v2 > v || (v2 == v && p2 < pos)) {
                    v = v2;
                    pos = p2;
                }
            }
            if ((uint32_t)(j & 31) == lane) {
                const int kk = j >> 5;
                if (v > best[kk] || (v == best[kk] && pos < bpos[kk])) {
                    best[kk] = v;
                    bpos[kk] = pos;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k)
        if (bpos[k] != 0xffffffffu)
            atomicMax(&kc->slot[k * 32 + lane], ((unsigned long long)ord_key(best[k]) << 32) | (uint32_t)~bpos[k]);
}

// One warp.  Lane 0 runs Andrew's monotone chain over the (at most 128)
// vertices -- exact orientation, strict turns -- so the polygon is strictly
// convex and counter-clockwise whatever the sample gave.
__global__ void __launch_bounds__(32) kgon_build_kernel(void *ws, Layout L)
{
    __shared__ float px[kKgonDirs], py[kKgonDirs];
    __shared__ int hx[2 * kKgonDirs + 2];
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    Kgon *g = at<Kgon>(ws, L.kgon);
    uint32_t s;
    if (!kgon_live(ctrl, at<Octagon>(ws, L.oct), s)) {
        if (threadIdx.x == 0) g->m = 0;
        return;
    }
    const KgonCtrl *kc = at<KgonCtrl>(ws, L.kgon_ctrl);
    const uint32_t *keys = at<uint32_t>(ws, L.keys[0]);
    const unsigned long long *pay = at<unsigned long long>(ws, L.pay[0]);
    const uint32_t lane = lane_id();
    for (int j = lane; j < kKgonDirs; j += 32) {
        const unsigned long long v = kc->slot[j];
        const uint32_t pos = ~(uint32_t)v;
        const float2 p = (v != 0ull && pos < s) ? survivor(keys, pay, pos) : survivor(keys, pay, 0);
        px[j] = p.x;
        py[j] = p.y;
    }
    __syncwarp();
    if (lane != 0) return;
    // sort by (x, y): insertion sort of indices
    int idx[kKgonDirs];
    for (int j = 0; j < kKgonDirs; ++j) {
        int k = j;
        while (k > 0 && (px[idx[k - 1]] > px[j] || (px[idx[k - 1]] == px[j] && py[idx[k - 1]] > py[j]))) {
            idx[k] = idx[k - 1];
            --k;
        }
        idx[k] = j;
    }
    // dedupe equal points
    int u = 0;
    for (int j = 0; j < kKgonDirs; ++j)
        if (u == 0 || px[idx[j]] != px[idx[u - 1]] || py[idx[j]] != py[idx[u - 1]]) idx[u++] = idx[j];
    int h = 0;
    for (int j = 0; j < u; ++j) {   // lower chain
        while (h >= 2 && orient(px[hx[h - 2]], py[hx[h - 2]], px[hx[h - 1]], py[hx[h - 1]], px[idx[j]], py[idx[j]]) <= 0)
            --h;
        hx[h++] = idx[j];
    }
    const int lower = h;
    for (int j = u - 2; j >= 0; --j) {   // upper chain
        while (h > lower && orient(px[hx[h - 2]], py[hx[h - 2]], px[hx[h - 1]], py[hx[h - 1]], px[idx[j]], py[idx[j]]) <= 0)
            --h;
        hx[h++] = idx[j];
    }
    const int m = h - 1;   // the first point closes the cycle
    if (u < 3 || m < 3) {
        g->m = 0;
        return;
    }
    for (int j = 0; j < m; ++j) {
        g->vx[j] = px[hx[j]];
        g->vy[j] = py[hx[j]];
    }
    g->m = (uint32_t)m;
}

// Copies the polygon to shared memory; false when it is unusable.
__device__ __forceinline__ bool load_kgon(Kgon &sg, void *ws, const Layout &L)
{
    const Kgon *g = at<Kgon>(ws, L.kgon);
    const uint32_t m = g->m;
    if (threadIdx.x == 0) sg.m = m;
    for (uint32_t j = threadIdx.x; j < m; j += blockDim.x) {
        sg.vx[j] = g->vx[j];
        sg.vy[j] = g->vy[j];
    }
    __syncthreads();
    return m >= 3;
}

__global__ void __launch_bounds__(KT) kgon_estimate_kernel(void *ws, Layout L)
{
    __shared__ Kgon sg;
    __shared__ uint32_t s_in[KNW], s_tot[KNW];
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    uint32_t s;
    if (!kgon_live(ctrl, at<Octagon>(ws, L.oct), s)) return;
    if (!load_kgon(sg, ws, L)) return;
    KgonCtrl *kc = at<KgonCtrl>(ws, L.kgon_ctrl);
    const uint32_t *keys = at<uint32_t>(ws, L.keys[0]);
    const unsigned long long *pay = at<unsigned long long>(ws, L.pay[0]);
    // a second sample, offset from the first
    const int64_t stride = std::max<int64_t>(1, (int64_t)s >> 16);
    const int64_t nsamp = ((int64_t)s - stride / 2 + stride - 1) / stride;
    uint32_t in = 0, tot = 0;
    for (int64_t k = (int64_t)blockIdx.x * KT + threadIdx.x; k < nsamp; k += (int64_t)gridDim.x * KT) {
        const float2 p = survivor(keys, pay, k * stride + stride / 2);
        in += kgon_inside(sg, p) ? 1u : 0u;
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
        for (int w = 0; w < KNW; ++w) {
            a += s_in[w];
            b += s_tot[w];
        }
        atomicAdd(&kc->inside, a);
        atomicAdd(&kc->sample, b);
    }
}

// The pass runs when the sample says it removes at least an eighth.
__device__ __forceinline__ bool kgon_worth(const KgonCtrl *kc) { return kc->sample > 0u && kc->inside * 8u >= kc->sample; }

__global__ void __launch_bounds__(KT) kgon_count_kernel(void *ws, Layout L)
{
    __shared__ Kgon sg;
    __shared__ uint32_t s_w[KNW];
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    uint32_t s;
    if (!kgon_live(ctrl, at<Octagon>(ws, L.oct), s)) return;
    KgonCtrl *kc = at<KgonCtrl>(ws, L.kgon_ctrl);
    if (!kgon_worth(kc)) return;
    if (!load_kgon(sg, ws, L)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) kc->s_in = s;
    const uint32_t *keys = at<uint32_t>(ws, L.keys[0]);
    const unsigned long long *pay = at<unsigned long long>(ws, L.pay[0]);
    unsigned long long *status = at<unsigned long long>(ws, L.filt_status);
    uint16_t *bits = at<uint16_t>(ws, L.keep_bits);
    const int64_t ntiles = ceil_div((int64_t)s, KTILE);
    const int64_t per = ceil_div(ntiles, (int64_t)gridDim.x);
    const int64_t t1 = std::min<int64_t>(ntiles, (int64_t)(blockIdx.x + 1) * per);
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    uint32_t block_total = 0;
    for (int64_t tile = (int64_t)blockIdx.x * per; tile < t1; ++tile) {
        const int64_t base = tile * KTILE;
        uint32_t keep = 0;
#pragma unroll 4
        for (int r = 0; r < KITEMS; ++r) {
            const int64_t q = base + r * KT + threadIdx.x;
            if (q < s && !kgon_inside(sg, survivor(keys, pay, q))) keep |= 1u << r;
        }
        bits[tile * KT + threadIdx.x] = (uint16_t)keep;
        uint32_t c = __popc(keep);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) s_w[warp] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < KNW; ++w) t += s_w[w];
            status[tile] = t;
            block_total += t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) at<uint32_t>(ws, L.filt_bsum)[blockIdx.x] = block_total;
}

// Same grid as the count pass (block b owns the same tile range).
__global__ void __launch_bounds__(KT) kgon_scatter_kernel(void *ws, Layout L)
{
    __shared__ uint32_t s_red[2][KNW];
    __shared__ uint32_t s_off[KITEMS][KNW];
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
    const unsigned long long *status = at<unsigned long long>(ws, L.filt_status);
    const uint32_t *bsum = at<uint32_t>(ws, L.filt_bsum);
    const uint16_t *bits = at<uint16_t>(ws, L.keep_bits);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = lane_id(), lt = (1u << lane) - 1u;
    uint32_t before = 0, total = 0;
    for (uint32_t i = tid; i < gridDim.x; i += KT) {
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
    for (int w = 0; w < KNW; ++w) {
        before += s_red[0][w];
        total += s_red[1][w];
    }
    if (blockIdx.x == 0 && tid == 0) {
        ctrl->surv_count = total;
        ctrl->sort_in = 1u;
    }
    const int64_t ntiles = ceil_div((int64_t)s, KTILE);
    const int64_t per = ceil_div(ntiles, (int64_t)gridDim.x);
    const int64_t r0 = (int64_t)blockIdx.x * per, r1 = std::min<int64_t>(ntiles, r0 + per);
    uint64_t run = before;
    for (int64_t tile = r0; tile < r1; ++tile) {
        const uint32_t cnt = (uint32_t)(status[tile] & 0xffffffffull);
        if (cnt == 0u) continue;   // block-uniform
        const uint32_t keep = bits[tile * KT + tid];
        // offsets in element order: row r of warp w before everything of
        // later (row, warp) pairs
#pragma unroll
        for (int r = 0; r < KITEMS; ++r) {
            const uint32_t c = __popc(__ballot_sync(0xffffffffu, (keep >> r) & 1u));
            if (lane == 0) s_off[r][warp] = c;
        }
        __syncthreads();
        if (warp == 0) {
            constexpr int PER = KITEMS * KNW / 32;
            uint32_t *flat = &s_off[0][0];
            uint32_t loc[PER], sum = 0;
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                loc[k] = flat[lane * PER + k];
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
                flat[lane * PER + k] = ex;
                ex += loc[k];
            }
        }
        __syncthreads();
        const int64_t base = tile * KTILE;
#pragma unroll
        for (int r = 0; r < KITEMS; ++r) {
            const uint32_t m = __ballot_sync(0xffffffffu, (keep >> r) & 1u);
            if ((keep >> r) & 1u) {
                const int64_t q = base + r * KT + tid;
                const uint64_t pos = run + s_off[r][warp] + __popc(m & lt);
                okeys[pos] = __ldg(keys + q);
                opay[pos] = __ldg(pay + q);
            }
        }
        run += cnt;
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_kgon(void *ws, const Layout &L, cudaStream_t st)
{
    const int sms = sm_count();
    static int per_sm = [] {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kgon_count_kernel, KT, 0);
        return v > 0 ? v : 1;
    }();
    const int64_t tiles = ceil_div(L.n, KTILE);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>({tiles, (int64_t)sms * per_sm, kFiltMaxBlocks}));
    probe_before(CH_K_KGON, st);
    kgon_extremes_kernel<<<sms * 2, KT, 0, st>>>(ws, L);
    kgon_build_kernel<<<1, 32, 0, st>>>(ws, L);
    kgon_estimate_kernel<<<sms, KT, 0, st>>>(ws, L);
    kgon_count_kernel<<<(unsigned)grid, KT, 0, st>>>(ws, L);
    kgon_scatter_kernel<<<(unsigned)grid, KT, 0, st>>>(ws, L);
    note_kernels(CH_K_KGON, 5);
    probe_after(CH_K_KGON, st);
    return cudaGetLastError();
}

}  // namespace ch

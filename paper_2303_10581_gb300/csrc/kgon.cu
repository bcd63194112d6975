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
constexpr int kSampleLog2 = 16;            // about 2^16 sample points

__device__ __forceinline__ float2 survivor(const uint32_t *keys, const unsigned long long *pay, int64_t q)
{
    return make_float2(key_float(__ldg(keys + q)), key_float((uint32_t)(__ldg(pay + q) >> 32)));
}

__device__ __forceinline__ bool left_strict(float ax, float ay, float bx, float by, float2 p)
{
    return orient(ax, ay, bx, by, p.x, p.y) > 0;
}

// Exact test; g in shared memory.  Points strictly inside the polygon's
// inscribed circle around (cx, cy) -- radius shrunk so that binary32
// rounding of the squared distance cannot cross it -- are accepted at once.
__device__ __forceinline__ bool kgon_inside(const Kgon &g, float2 p)
{
    const float dx = p.x - g.cx, dy = p.y - g.cy;
    if (__fmaf_rn(dx, dx, dy * dy) < g.r2) return true;
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
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const int64_t stride = std::max<int64_t>(1, (int64_t)s >> kSampleLog2);
    const int64_t nsamp = ((int64_t)s + stride - 1) / stride;
    constexpr int PER = kKgonDirs / 32;   // lane owns directions lane + 32 k
    float best[PER], dc[PER], ds[PER];
    uint32_t bpos[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        best[k] = -__int_as_float(0x7f800000);
        bpos[k] = 0xffffffffu;
        dc[k] = s_c[lane + 32 * k];
        ds[k] = s_s[lane + 32 * k];
    }
    // each warp stages 32 sample points; every lane scans them for its directions
    __shared__ float2 s_p[KNW][32];
    __shared__ uint32_t s_q[KNW][32];
    const int64_t wid = ((int64_t)blockIdx.x * KT + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * KT) >> 5;
    for (int64_t g0 = wid * 32; g0 < nsamp; g0 += nw * 32) {
        const int64_t k = g0 + lane;
        const bool ok = k < nsamp;
        const uint32_t q = ok ? (uint32_t)(k * stride) : 0xffffffffu;
        s_p[warp][lane] = ok ? survivor(keys, pay, q) : make_float2(0.0f, 0.0f);
        s_q[warp][lane] = q;
        __syncwarp();
        const int cnt = (int)min((int64_t)32, nsamp - g0);
        for (int i = 0; i < cnt; ++i) {
            const float2 p = s_p[warp][i];
            const uint32_t pq = s_q[warp][i];
#pragma unroll
            for (int kk = 0; kk < PER; ++kk) {
                const float v = __fmaf_rn(p.x, dc[kk], p.y * ds[kk]);
                if (v > best[kk]) {   // sample positions increase: ties keep the first
                    best[kk] = v;
                    bpos[kk] = pq;
                }
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < PER; ++k)
        if (bpos[k] != 0xffffffffu)
            atomicMax(&kc->slot[k * 32 + lane], ((unsigned long long)ord_key(best[k]) << 32) | (uint32_t)~bpos[k]);
}

// One warp: the exact convex hull of the slots' points.  They are sorted by
// (x, y) (each lane ranks its slots against all), duplicates dropped, and
// the lower and the upper chain found by strict-turn elimination passes
// over the sorted sequence -- a sequence whose every turn is strict is its
// own chain, so this gives Andrew's chains (exact orientation) in parallel.
// The polygon is strictly convex and counter-clockwise.
__device__ __forceinline__ int warp_chain_pass(const float *px, const float *py, const uint8_t *src, uint8_t *dst,
                                               int len, int side, uint32_t lane)
{
    const uint32_t lt = (1u << lane) - 1u;
    int kept = 0;
    for (int c0 = 0; c0 < len; c0 += 32) {
        const int j = c0 + (int)lane;
        bool k = j < len;
        if (k && j > 0 && j < len - 1) {
            const int a = src[j - 1], b = src[j], c = src[j + 1];
            const int o = orient(px[a], py[a], px[b], py[b], px[c], py[c]);
            k = side == 0 ? o > 0 : o < 0;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, k);
        if (k) dst[kept + __popc(m & lt)] = src[j];
        kept += __popc(m);
    }
    __syncwarp();
    return kept;
}

__global__ void __launch_bounds__(32) kgon_build_kernel(void *ws, Layout L)
{
    constexpr int K = kKgonDirs;
    __shared__ float px[K], py[K];
    __shared__ uint8_t sorted[K];
    __shared__ uint8_t seq[2][2][K];   // [side][ping-pong]
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    Kgon *g = at<Kgon>(ws, L.kgon);
    const uint32_t lane = lane_id();
    uint32_t s;
    if (!kgon_live(ctrl, at<Octagon>(ws, L.oct), s)) {
        if (lane == 0) {
            g->m = 0;
            g->r2 = 0.0f;
        }
        return;
    }
    const KgonCtrl *kc = at<KgonCtrl>(ws, L.kgon_ctrl);
    const uint32_t *keys = at<uint32_t>(ws, L.keys[0]);
    const unsigned long long *pay = at<unsigned long long>(ws, L.pay[0]);
    for (int j = lane; j < K; j += 32) {
        const unsigned long long v = kc->slot[j];
        const uint32_t pos = ~(uint32_t)v;
        const float2 p = survivor(keys, pay, (v != 0ull && pos < s) ? pos : 0u);
        px[j] = p.x;
        py[j] = p.y;
    }
    __syncwarp();
    // rank by (x, y, slot)
    constexpr int PER = K / 32;
    int r[PER];
    float qx[PER], qy[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        r[k] = 0;
        qx[k] = px[lane + 32 * k];
        qy[k] = py[lane + 32 * k];
    }
    for (int i = 0; i < K; ++i) {
        const float ix = px[i], iy = py[i];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int j = (int)lane + 32 * k;
            r[k] += (ix < qx[k] || (ix == qx[k] && (iy < qy[k] || (iy == qy[k] && i < j)))) ? 1 : 0;
        }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) sorted[r[k]] = (uint8_t)(lane + 32 * k);
    __syncwarp();
    // drop equal points (keep the first of each run)
    int u = 0;
    for (int c0 = 0; c0 < K; c0 += 32) {
        const int j = c0 + (int)lane;
        const int a = sorted[j];
        const bool k = j == 0 || px[sorted[j - 1]] != px[a] || py[sorted[j - 1]] != py[a];
        const uint32_t m = __ballot_sync(0xffffffffu, k);
        if (k) {
            seq[0][0][u + __popc(m & ((1u << lane) - 1u))] = (uint8_t)a;
            seq[1][0][u + __popc(m & ((1u << lane) - 1u))] = (uint8_t)a;
        }
        u += __popc(m);
    }
    __syncwarp();
    int len[2] = {u, u}, cur[2] = {0, 0};
    for (int side = 0; side < 2; ++side) {
        for (int pass = 0; pass < K && len[side] > 2; ++pass) {
            const int kept = warp_chain_pass(px, py, seq[side][cur[side]], seq[side][cur[side] ^ 1], len[side], side, lane);
            cur[side] ^= 1;
            const bool done = kept == len[side];
            len[side] = kept;
            if (done) break;
        }
    }
    const int m = len[0] + len[1] - 2;
    if (u < 3 || m < 3) {
        if (lane == 0) {
            g->m = 0;
            g->r2 = 0.0f;
        }
        return;
    }
    // counter-clockwise: the lower chain left to right, then the upper chain
    // right to left without its two ends (shared with the lower one)
    const uint8_t *lo = seq[0][cur[0]], *up = seq[1][cur[1]];
    float sx = 0.0f, sy = 0.0f;
    for (int j = lane; j < m; j += 32) {
        const int a = j < len[0] ? lo[j] : up[len[1] - 2 - (j - len[0])];
        g->vx[j] = px[a];
        g->vy[j] = py[a];
        sx += px[a];
        sy += py[a];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    __syncwarp();   // the vertices in g are re-read below
    // quick-accept circle around the vertex centroid c: a lower bound of
    // c's distance to every edge line, from binary32 terms with a margin
    // of 1e-5 of their magnitudes (far above their rounding errors); zero
    // when c is not provably strictly inside
    const float cx = sx / (float)m, cy = sy / (float)m;
    float rmin = __int_as_float(0x7f800000);
    for (int j = lane; j < m; j += 32) {
        const int jn = j + 1 < m ? j + 1 : 0;
        const float ax = g->vx[j], ay = g->vy[j], ex = g->vx[jn] - ax, ey = g->vy[jn] - ay;
        const float t1 = ex * (cy - ay), t2 = ey * (cx - ax);
        const float cr = (t1 - t2) - 1e-5f * (fabsf(t1) + fabsf(t2));
        const float len_e = sqrtf(ex * ex + ey * ey) * (1.0f + 1e-5f);
        const float d = len_e > 0.0f ? cr / len_e : -1.0f;
        rmin = fminf(rmin, d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rmin = fminf(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
    if (lane == 0) {
        g->cx = cx;
        g->cy = cy;
        g->r2 = rmin > 0.0f && rmin < 1e18f ? rmin * rmin * (1.0f - 1e-4f) : 0.0f;
        g->m = (uint32_t)m;
    }
}

// Copies the polygon to shared memory; false when it is unusable.
__device__ __forceinline__ bool load_kgon(Kgon &sg, void *ws, const Layout &L)
{
    const Kgon *g = at<Kgon>(ws, L.kgon);
    const uint32_t m = g->m;
    if (threadIdx.x == 0) {
        sg.m = m;
        sg.cx = g->cx;
        sg.cy = g->cy;
        sg.r2 = g->r2;
    }
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
    __shared__ float2 s_qp[KNW][64];
    __shared__ uint16_t s_tag[KNW][64];
    __shared__ uint32_t s_res[KNW][32];
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
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id(), lt = (1u << lane) - 1u;
    uint32_t block_total = 0;
    for (int64_t tile = (int64_t)blockIdx.x * per; tile < t1; ++tile) {
        const int64_t base = tile * KTILE;
        if (threadIdx.x == 0 && tile + 1 < t1) {   // the next tile streams into L2 meanwhile
            const uint32_t nn = (uint32_t)std::min<int64_t>(KTILE, (int64_t)s - base - KTILE);
            bulk_prefetch_l2(keys + base + KTILE, (nn * 4u) & ~15u);
            bulk_prefetch_l2(pay + base + KTILE, (nn * 8u) & ~15u);
        }
        // all loads first (memory parallelism), then the quick test, then
        // the full test for the few points outside the quick circle
        float x[KITEMS], y[KITEMS];
        uint32_t live = 0;
#pragma unroll
        for (int r = 0; r < KITEMS; ++r) {
            const int64_t q = base + r * KT + threadIdx.x;
            x[r] = y[r] = 0.0f;
            if (q < s) {
                x[r] = key_float(__ldg(keys + q));
                y[r] = key_float(__ldg(reinterpret_cast<const uint2 *>(pay) + q).y);
                live |= 1u << r;
            }
        }
        uint32_t slow = 0;
#pragma unroll
        for (int r = 0; r < KITEMS; ++r) {
            const float dx = x[r] - sg.cx, dy = y[r] - sg.cy;
            if (!(__fmaf_rn(dx, dx, dy * dy) < sg.r2)) slow |= 1u << r;
        }
        slow &= live;
        // points outside the quick circle: queued per warp with their
        // coordinates and tested 32 at a time by all lanes as the queue
        // fills (kept bits come back per owner lane)
        uint32_t keep = 0;
        if (__any_sync(0xffffffffu, slow != 0u)) {
            s_res[warp][lane] = 0u;
            int cnt = 0;
#pragma unroll
            for (int r = 0; r < KITEMS; ++r) {
                const bool b = (slow >> r) & 1u;
                const uint32_t m = __ballot_sync(0xffffffffu, b);
                if (m == 0u) continue;
                if (b) {
                    const int at_ = cnt + __popc(m & lt);
                    s_qp[warp][at_] = make_float2(x[r], y[r]);
                    s_tag[warp][at_] = (uint16_t)((lane << 4) | (uint32_t)r);
                }
                cnt += __popc(m);
                if (cnt >= 32) {   // a full round; the overflow moves to the front
                    __syncwarp();
                    const uint32_t tg = s_tag[warp][lane];
                    if (!kgon_inside(sg, s_qp[warp][lane])) atomicOr(&s_res[warp][tg >> 4], 1u << (tg & 15u));
                    const bool more = (int)lane + 32 < cnt;
                    float2 pv = make_float2(0.0f, 0.0f);
                    uint16_t tv = 0;
                    if (more) {
                        pv = s_qp[warp][lane + 32];
                        tv = s_tag[warp][lane + 32];
                    }
                    __syncwarp();
                    if (more) {
                        s_qp[warp][lane] = pv;
                        s_tag[warp][lane] = tv;
                    }
                    cnt -= 32;
                    __syncwarp();
                }
            }
            __syncwarp();
            if ((int)lane < cnt) {
                const uint32_t tg = s_tag[warp][lane];
                if (!kgon_inside(sg, s_qp[warp][lane])) atomicOr(&s_res[warp][tg >> 4], 1u << (tg & 15u));
            }
            __syncwarp();
            keep = s_res[warp][lane];
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

// kfilter.cu -- the filter polygon generalised from the eight directions of
// Sec. 3.1 to K in {8, 16, 32, 64} directions: the polygon a learned
// proposal picks (the paper's related work cites a 16-direction filter as
// precedent).
//
// The directions (c_k, s_k) come from the caller (device array, counter-
// clockwise, |c_k|, |s_k| <= 1).  Vertex k is the point with the largest
// binary32 key fl(fl(c_k x) + fl(s_k y)), lowest index on ties; with the
// octagon's eight integer directions (1,0), (1,1), (0,1), (-1,1), ... these
// are exactly the keys of Sec. 3.1.  A point is discarded when it is
// strictly left of every edge of non-zero length of the closed vertex
// sequence (exact signs), as in Sec. 3.2; the vertices are input points, so
// no hull vertex is ever discarded.
//
//  kx_extremes_kernel<K>  tiles of 1024 points staged in shared memory;
//                         thread t keeps the best point of direction t mod K
//                         over its share of each tile; per-direction packed
//                         atomicMax (ord(key) << 32 | ~index); the last block
//                         decodes, resets the slots and builds the polygon
//                         (edges, an exact quick-discard rectangle)
//  kx_count_kernel<G>     the filter's count pass with this polygon: the
//                         rectangle, then the edges starting at the one
//                         facing the point; keep bits, tile counts and block
//                         totals in the filter's layout, so its scatter pass
//                         compacts the survivors
#include <algorithm>

#include "common.cuh"
#include "launch.h"

namespace ch {
namespace {

constexpr int XT = 512;       // threads per block of the sweep
constexpr int XTILE = 1024;   // points per tile of the sweep
constexpr uint32_t kSiteKxNonFinite = 50;

// Larger key, or equal key and lower index; index 0xffffffff: no candidate.
__device__ __forceinline__ void take_better(float &k, uint32_t &i, float ok, uint32_t oi)
{
    if (oi == 0xffffffffu) return;
    if (i == 0xffffffffu || ok > k || (ok == k && oi < i)) {
        k = ok;
        i = oi;
    }
}

// Last block: the polygon from the decoded vertices.  The rectangle is
// accepted when its four corners are strictly left of every edge of non-zero
// length (exact signs): that region is an intersection of open half-planes,
// hence convex, so the whole closed rectangle lies in it.
__device__ void build_kpoly(const float2 *p, int K, const uint32_t *s_ext, KPoly *kp)
{
    __shared__ float s_vx[kMaxDirs], s_vy[kMaxDirs];
    __shared__ unsigned s_vm[2];
    __shared__ float s_box[4];
    const int t = (int)threadIdx.x;
    if (t < K) {
        const float2 v = p[s_ext[t]];
        s_vx[t] = v.x;
        s_vy[t] = v.y;
    }
    __syncthreads();
    bool valid = false;
    if (t < K) {
        const int kn = t + 1 == K ? 0 : t + 1;
        const float ax = s_vx[t], ay = s_vy[t], bx = s_vx[kn], by = s_vy[kn];
        valid = !(ax == bx && ay == by);
        kp->ax[t] = ax;
        kp->ay[t] = ay;
        kp->bx[t] = bx;
        kp->by[t] = by;
    }
    if (t < 64) {
        const unsigned m = __ballot_sync(0xffffffffu, valid);
        if ((t & 31) == 0) s_vm[t >> 5] = m;
    }
    if (t == 0) {
        float x0 = s_vx[0], x1 = s_vx[0], y0 = s_vy[0], y1 = s_vy[0];
        for (int k = 1; k < K; ++k) {
            x0 = fminf(x0, s_vx[k]);
            x1 = fmaxf(x1, s_vx[k]);
            y0 = fminf(y0, s_vy[k]);
            y1 = fmaxf(y1, s_vy[k]);
        }
        s_box[0] = x0;
        s_box[1] = x1;
        s_box[2] = y0;
        s_box[3] = y1;
    }
    __syncthreads();
    const unsigned long long vmask = (unsigned long long)s_vm[0] | ((unsigned long long)s_vm[1] << 32);
    const unsigned long long kmask = K == 64 ? ~0ull : ((1ull << K) - 1ull);
    const unsigned long long valid_mask = vmask & kmask;
    const double cxd = 0.5 * ((double)s_box[0] + (double)s_box[1]);
    const double cyd = 0.5 * ((double)s_box[2] + (double)s_box[3]);
    const double hw = 0.5 * ((double)s_box[1] - (double)s_box[0]);
    const double hh = 0.5 * ((double)s_box[3] - (double)s_box[2]);
    float xl = 1.0f, xh = -1.0f, yl = 1.0f, yh = -1.0f;   // empty
    if (valid_mask != 0ull) {
        const double fr[8] = {0.90, 0.84, 0.78, 0.70, 0.60, 0.48, 0.35, 0.22};
        for (int j = 0; j < 8; ++j) {
            const float rxl = (float)(cxd - fr[j] * hw), rxh = (float)(cxd + fr[j] * hw);
            const float ryl = (float)(cyd - fr[j] * hh), ryh = (float)(cyd + fr[j] * hh);
            bool ok = rxl <= rxh && ryl <= ryh;
            if (t < 4 * K) {   // corner t / K against edge t % K
                const int c = t / K, e = t % K, en = e + 1 == K ? 0 : e + 1;
                const float px = (c == 0 || c == 3) ? rxl : rxh;
                const float py = (c < 2) ? ryl : ryh;
                if ((valid_mask >> e) & 1ull) ok = ok && orient(s_vx[e], s_vy[e], s_vx[en], s_vy[en], px, py) > 0;
            }
            if (__syncthreads_and(ok)) {
                xl = rxl;
                xh = rxh;
                yl = ryl;
                yh = ryh;
                break;
            }
        }
    }
    // convexity: every vertex on or left of every valid edge, and the centre
    // strictly left of all of them.  Then the vertices lie in every edge's
    // closed half-plane, the interior of their hull lies in every open one,
    // and a point strictly inside a triangle (centre, v_k, v_k+1) -- part of
    // that interior -- is strictly left of every edge.
    bool conv = valid_mask != 0ull;
    const float ccx = (float)cxd, ccy = (float)cyd;
    for (int pr = t; pr < K * (K + 1); pr += (int)blockDim.x) {   // (edge, vertex or centre) pairs
        const int e = pr / (K + 1), m = pr % (K + 1), en = e + 1 == K ? 0 : e + 1;
        if (!((valid_mask >> e) & 1ull)) continue;
        const float qx = m < K ? s_vx[m] : ccx, qy = m < K ? s_vy[m] : ccy;
        const int o = orient(s_vx[e], s_vy[e], s_vx[en], s_vy[en], qx, qy);
        if (m < K ? o < 0 : o <= 0) conv = false;
    }
    conv = __syncthreads_and(conv) != 0;
    if (t == 0) {
        kp->K = (uint32_t)K;
        kp->convex = conv ? 1u : 0u;
        kp->nvalid = (uint32_t)__popcll(valid_mask);
        kp->valid = valid_mask;
        kp->xl = xl;
        kp->xh = xh;
        kp->yl = yl;
        kp->yh = yh;
        kp->cx = (float)cxd;
        kp->cy = (float)cyd;
    }
}

template <int K>
__global__ void __launch_bounds__(XT) kx_extremes_kernel(const float *__restrict__ pts, int64_t n,
                                                         const float *__restrict__ dirs, uint32_t *ext_out, void *ws,
                                                         Layout L, unsigned long long *zero_ptr, int64_t zero_words)
{
    static_assert(K >= 8 && K <= kMaxDirs && XT % K == 0, "directions split the block evenly");
    constexpr int PARTS = XT / K;
    __shared__ float2 s_p[XTILE];
    __shared__ float s_bk[XT];
    __shared__ uint32_t s_bi[XT];
    __shared__ uint32_t s_ext[kMaxDirs];
    __shared__ int s_nf;
    __shared__ int s_last;
    KxCtrl *kc = at<KxCtrl>(ws, L.kxctrl);
    // clear what the following kernels of this call expect to be zero
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = gtid; w < zero_words; w += gthreads) zero_ptr[w] = 0ull;

    const int d = (int)threadIdx.x % K, part = (int)threadIdx.x / K;
    const float c = dirs[2 * d], sn = dirs[2 * d + 1];
    float best = __int_as_float(0x7fc00000);   // NaN: no candidate yet
    uint32_t bi = 0xffffffffu;
    float nf = 0.0f;                           // becomes NaN iff a coordinate is NaN or infinite
    const float2 *p2 = reinterpret_cast<const float2 *>(pts);
    const int64_t ntiles = ceil_div(n, (int64_t)XTILE);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t base = tile * XTILE;
        const int cnt = (int)std::min<int64_t>(XTILE, n - base);
        for (int j = (int)threadIdx.x; j < XTILE; j += XT) {
            float2 v = make_float2(0.0f, 0.0f);
            if (j < cnt) {
                v = __ldcs(p2 + base + j);
                nf = __fmaf_rn(v.x, 0.0f, nf);
                nf = __fmaf_rn(v.y, 0.0f, nf);
            }
            s_p[j] = v;
        }
        __syncthreads();
        for (int q = part; q < cnt; q += PARTS) {
            const float2 v = s_p[q];
            const float key = __fadd_rn(__fmul_rn(c, v.x), __fmul_rn(sn, v.y));
            // the first key is always taken (best starts as NaN); then only
            // a strictly larger one, so ties keep the lower index
            if (!(key <= best)) {
                best = key;
                bi = (uint32_t)(base + q);
            }
        }
        __syncthreads();
    }
    s_bk[threadIdx.x] = best;
    s_bi[threadIdx.x] = bi;
    if (threadIdx.x == 0) s_nf = 0;
    __syncthreads();
    if (nf != nf) s_nf = 1;
    if ((int)threadIdx.x < K) {
        float k = s_bk[threadIdx.x];
        uint32_t i = s_bi[threadIdx.x];
        for (int pp = 1; pp < PARTS; ++pp) take_better(k, i, s_bk[threadIdx.x + pp * K], s_bi[threadIdx.x + pp * K]);
        if (i != 0xffffffffu) atomicMax(&kc->slot[threadIdx.x], ((unsigned long long)ord_key(k) << 32) | (uint32_t)~i);
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_nf) atomicOr(&kc->nonfinite, 1u);
        __threadfence();
        s_last = atomicAdd(&kc->done, 1u) == gridDim.x - 1 ? 1 : 0;
    }
    __syncthreads();
    if (!s_last) return;

    // last block: decode, reset the slots for the next call, build the polygon
    __threadfence();
    if ((int)threadIdx.x < K) {
        const unsigned long long packed = atomicExch(&kc->slot[threadIdx.x], 0ull);
        uint32_t idx = ~(uint32_t)packed;
        if ((int64_t)idx >= n) idx = 0;   // every direction has a candidate; guards the loads below
        s_ext[threadIdx.x] = idx;
        if (ext_out) ext_out[threadIdx.x] = idx;
    }
    if (threadIdx.x == 0) {
        s_nf = atomicExch(&kc->nonfinite, 0u) != 0u ? 1 : 0;
        kc->done = 0;
    }
    __syncthreads();
    Octagon *oct = at<Octagon>(ws, L.oct);
    if (s_nf) {   // block-uniform
        if (threadIdx.x == 0) {
            set_error(ws, L, kErrNonFinite, kSiteKxNonFinite);
            oct->abort = 1;   // the later kernels of the call do nothing
        }
        return;
    }
    build_kpoly(p2, K, s_ext, at<KPoly>(ws, L.kpoly));
    if (threadIdx.x == 0) oct->abort = 0;
}

__device__ __forceinline__ int sign_exact(float ax, float ay, float bx, float by, float cx, float cy)
{
    const int o = orient_f32(ax, ay, bx, by, cx, cy);
    return o != 2 ? o : orient_rest(ax, ay, bx, by, cx, cy);
}

// keep(p) <=> NOT (p strictly left of every valid edge).  The edge facing
// p's angle around the centre (a binary32 hint) is tried first: p not
// strictly left of it is kept.  For a convex polygon, p strictly inside the
// triangle (centre, v_k, v_k+1) of that edge or a neighbour is discarded
// (it is strictly left of every edge).  Otherwise every edge is tried,
// alternating outwards from the hint; the answer does not depend on the
// order.
__device__ __forceinline__ bool kx_keep(const KPoly &sp, float x, float y)
{
    if (sp.xl <= x && x <= sp.xh && sp.yl <= y && y <= sp.yh) return false;
    if (sp.nvalid == 0u) return true;
    const int K = (int)sp.K;
    const float a = atan2f(y - sp.cy, x - sp.cx);
    int k0 = (int)floorf(a * ((float)K * 0.15915494f));   // angle / (2 pi / K)
    k0 = ((k0 % K) + K) % K;
    if (sp.convex) {
#pragma unroll 1
        for (int j = 0; j < 3; ++j) {   // k0, k0 - 1, k0 + 1
            int k = k0 + (j == 0 ? 0 : (j == 1 ? -1 : 1));
            k = k < 0 ? k + K : (k >= K ? k - K : k);
            if (!((sp.valid >> k) & 1ull)) continue;
            if (sign_exact(sp.ax[k], sp.ay[k], sp.bx[k], sp.by[k], x, y) <= 0) return true;
            if (sign_exact(sp.cx, sp.cy, sp.ax[k], sp.ay[k], x, y) > 0 &&
                sign_exact(sp.bx[k], sp.by[k], sp.cx, sp.cy, x, y) > 0)
                return false;
        }
    }
    for (int j = 0; j < K; ++j) {
        int k = k0 + ((j & 1) ? -((j + 1) >> 1) : (j >> 1));   // 0, -1, +1, -2, +2, ...
        k = k < 0 ? k + K : (k >= K ? k - K : k);
        if (!((sp.valid >> k) & 1ull)) continue;
        int o = orient_f32(sp.ax[k], sp.ay[k], sp.bx[k], sp.by[k], x, y);
        if (o == 2) o = orient_rest(sp.ax[k], sp.ay[k], sp.bx[k], sp.by[k], x, y);
        if (o <= 0) return true;
    }
    return false;
}

// The filter's count pass with the K-gon: each block a contiguous range of
// 4096-point tiles; thread t's items q = r * G + h are the points
// base + (r * kFiltThreads + t) * G + h (G = 2: 16-byte point pairs); 16
// keep bits per thread, the tile's count and the block's total.
template <int G>
__global__ void __launch_bounds__(kFiltThreads) kx_count_kernel(const float *__restrict__ pts, int64_t n, void *ws,
                                                               Layout L)
{
    constexpr int ROWS = kFiltItems / G;
    __shared__ KPoly sp;
    __shared__ uint32_t s_w[kFiltThreads / 32];
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = at<Octagon>(ws, L.oct)->abort ? 1 : 0;
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(at<KPoly>(ws, L.kpoly));
        uint32_t *dst = reinterpret_cast<uint32_t *>(&sp);
        for (uint32_t w = threadIdx.x; w < sizeof(KPoly) / 4; w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    if (s_abort) return;
    unsigned long long *status = at<unsigned long long>(ws, L.filt_status);
    uint16_t *bits = at<uint16_t>(ws, L.keep_bits);
    const int64_t ntiles = ceil_div(n, (int64_t)kFiltTile);
    const int64_t per = ceil_div(ntiles, (int64_t)gridDim.x);
    const int64_t t1 = std::min<int64_t>(ntiles, (int64_t)(blockIdx.x + 1) * per);
    const uint32_t t = threadIdx.x, warp = t >> 5, lane = lane_id();
    uint32_t block_total = 0;
    for (int64_t tile = (int64_t)blockIdx.x * per; tile < t1; ++tile) {
        const int64_t base = tile * kFiltTile;
        if (t == 0 && tile + 1 < t1) {   // the next tile streams into L2 meanwhile
            const int64_t nb = base + kFiltTile;
            const uint32_t nn = (uint32_t)std::min<int64_t>(kFiltTile, n - nb);
            if (((reinterpret_cast<uintptr_t>(pts + 2 * nb)) & 15u) == 0) bulk_prefetch_l2(pts + 2 * nb, (nn * 8u) & ~15u);
        }
        float px[kFiltItems], py[kFiltItems];
        uint32_t live = 0;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int64_t i = base + (int64_t)(r * kFiltThreads + t) * G;
            if constexpr (G == 2) {
                float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (i + 1 < n) {
                    v = __ldcs(reinterpret_cast<const float4 *>(pts) + i / 2);
                    live |= 3u << (2 * r);
                } else if (i < n) {
                    const float2 a = reinterpret_cast<const float2 *>(pts)[i];
                    v = make_float4(a.x, a.y, 0.0f, 0.0f);
                    live |= 1u << (2 * r);
                }
                px[2 * r] = v.x;
                py[2 * r] = v.y;
                px[2 * r + 1] = v.z;
                py[2 * r + 1] = v.w;
            } else {
                float2 v = make_float2(0.0f, 0.0f);
                if (i < n) {
                    v = __ldcs(reinterpret_cast<const float2 *>(pts) + i);
                    live |= 1u << r;
                }
                px[r] = v.x;
                py[r] = v.y;
            }
        }
        uint32_t keep = 0;
#pragma unroll
        for (int q = 0; q < kFiltItems; ++q)
            if (((live >> q) & 1u) && kx_keep(sp, px[q], py[q])) keep |= 1u << q;
        bits[tile * kFiltThreads + t] = (uint16_t)keep;
        uint32_t c = __popc(keep);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) s_w[warp] = c;
        __syncthreads();
        if (t == 0) {
            uint32_t tot = 0;
#pragma unroll
            for (int w = 0; w < kFiltThreads / 32; ++w) tot += s_w[w];
            status[tile] = tot;
            block_total += tot;
        }
        __syncthreads();
    }
    if (t == 0) at<uint32_t>(ws, L.filt_bsum)[blockIdx.x] = block_total;
}


// ---------------------------------------------------------------------------
// A K-direction polygon over the octagon's survivors (ch_hull_octagon_kgon,
// ch_hull_learned).  After the octagon's count pass, the vertex of
// direction k is the survivor with the largest key fl(fl(c_k x) + fl(s_k y)),
// lowest index on ties, and every survivor strictly left of every edge of
// non-zero length of that vertex sequence is dropped too.  Both polygons
// have input points as vertices, so what is dropped is strictly inside the
// hull (Sec. 3.2's argument, twice); a point survives when it is strictly
// inside neither.  The extremes of every direction survive the octagon
// (they lie on the hull's boundary), so up to rounding of the keys these
// are the polygon's vertices over all points; the survivors' extremes are
// what is computed.
// ---------------------------------------------------------------------------
constexpr int ST = 256;   // threads per block of the survivors' passes (one per count-pass thread)

// Whether the K-gon stage runs in this call: not aborted, the octagon's
// count pass left keep bits (no speculative sweep), and K is the stage's
// (kdev: the device's choice, when the host did not fix it).
__device__ __forceinline__ bool kx_stage_on(const Octagon *oct, const int32_t *kdev, int K)
{
    return !oct->abort && !oct->spec && (kdev == nullptr || *kdev == K);
}

template <int G>
__device__ __forceinline__ int64_t sv_point(int64_t base, uint32_t t, int q)
{
    return base + (int64_t)((q / G) * kFiltThreads + t) * G + q % G;
}

// Survivors of each tile are staged in shared memory (compacted), then
// thread t keeps the best of direction t mod K over its share of them.
struct SvSmem {
    float2 p[kFiltTile];
    uint16_t i[kFiltTile];   // index - base
    uint32_t w[ST / 32];
    float bk[ST];
    uint32_t bi[ST];
    uint32_t ext[kMaxDirs];
    int last;
};

template <int K, int G>
__device__ __forceinline__ void kx_sv_extremes_body(SvSmem &sm, const float *__restrict__ pts, int64_t n,
                                                    const float *__restrict__ dirs, const int32_t *kdev,
                                                    uint32_t *ext_out, void *ws, const Layout &L)
{
    static_assert(K >= 8 && K <= kMaxDirs && ST % K == 0 && ST == kFiltThreads, "directions split the block evenly");
    constexpr int PARTS = ST / K;
    float2 *s_p = sm.p;
    uint16_t *s_i = sm.i;
    uint32_t *s_w = sm.w;
    float *s_bk = sm.bk;
    uint32_t *s_bi = sm.bi;
    uint32_t *s_ext = sm.ext;
    int &s_last = sm.last;
    Octagon *oct = at<Octagon>(ws, L.oct);
    if (!kx_stage_on(oct, kdev, K)) return;
    KxCtrl *kc = at<KxCtrl>(ws, L.kxctrl);
    const uint16_t *bits = at<uint16_t>(ws, L.keep_bits);
    const float2 *p2 = reinterpret_cast<const float2 *>(pts);
    const uint32_t t = threadIdx.x, warp = t >> 5, lane = lane_id();
    const int d = (int)t % K, part = (int)t / K;
    const float c = dirs[2 * d], sn = dirs[2 * d + 1];
    float best = __int_as_float(0x7fc00000);   // NaN: no candidate yet
    uint32_t bi = 0xffffffffu;
    const int64_t ntiles = ceil_div(n, (int64_t)kFiltTile);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t base = tile * kFiltTile;
        const uint32_t kb = bits[tile * kFiltThreads + t];
        const uint32_t cnt = __popc(kb);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += u;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        uint32_t off = incl - cnt, total = 0;
#pragma unroll
        for (int w = 0; w < ST / 32; ++w) {
            if (w < (int)warp) off += s_w[w];
            total += s_w[w];
        }
        if (total == 0u) {   // block-uniform
            __syncthreads();
            continue;
        }
        for (uint32_t b = kb; b; b &= b - 1u) {
            const int q = __ffs(b) - 1;
            const int64_t i = sv_point<G>(base, t, q);
            s_p[off] = p2[i];
            s_i[off] = (uint16_t)(i - base);
            ++off;
        }
        __syncthreads();
        for (uint32_t q = part; q < total; q += PARTS) {
            const float2 v = s_p[q];
            const float key = __fadd_rn(__fmul_rn(c, v.x), __fmul_rn(sn, v.y));
            const uint32_t i = (uint32_t)(base + s_i[q]);
            // staged out of index order: equal keys keep the lower index
            if (!(key <= best) || (key == best && i < bi)) {
                best = key;
                bi = i;
            }
        }
        __syncthreads();
    }
    s_bk[t] = best;
    s_bi[t] = bi;
    __syncthreads();
    if ((int)t < K) {
        float k = s_bk[t];
        uint32_t i = s_bi[t];
        for (int pp = 1; pp < PARTS; ++pp) take_better(k, i, s_bk[t + pp * K], s_bi[t + pp * K]);
        if (i != 0xffffffffu) atomicMax(&kc->slot[t], ((unsigned long long)ord_key(k) << 32) | (uint32_t)~i);
        __threadfence();
    }
    __syncthreads();
    if (t == 0) {
        __threadfence();
        s_last = atomicAdd(&kc->done, 1u) == gridDim.x - 1 ? 1 : 0;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if ((int)t < K) {
        const unsigned long long packed = atomicExch(&kc->slot[t], 0ull);
        uint32_t idx = ~(uint32_t)packed;
        if ((int64_t)idx >= n) idx = 0;   // every direction has a survivor (the octagon's vertices survive)
        s_ext[t] = idx;
        if (ext_out) ext_out[t] = idx;
    }
    if (t == 0) kc->done = 0;
    __syncthreads();
    build_kpoly(p2, K, s_ext, at<KPoly>(ws, L.kpoly));
}

// KT: the host's K, or 0: the device's choice (*kdev), dispatched here so
// one launch serves every K.
template <int KT, int G>
__global__ void __launch_bounds__(ST) kx_sv_extremes_kernel(const float *__restrict__ pts, int64_t n,
                                                            const float *__restrict__ dirs, const int32_t *kdev,
                                                            uint32_t *ext_out, void *ws, Layout L)
{
    __shared__ SvSmem sm;
    if constexpr (KT == 0) {
        const int K = *kdev;   // uniform
        if (K == 16) kx_sv_extremes_body<16, G>(sm, pts, n, dirs, kdev, ext_out, ws, L);
        else if (K == 32) kx_sv_extremes_body<32, G>(sm, pts, n, dirs, kdev, ext_out, ws, L);
        else if (K == 64) kx_sv_extremes_body<64, G>(sm, pts, n, dirs, kdev, ext_out, ws, L);
    } else {
        kx_sv_extremes_body<KT, G>(sm, pts, n, dirs, kdev, ext_out, ws, L);
    }
}

// The survivors' exact test against the K-gon: bits of kept points strictly
// inside it are cleared, and the tile's count and its count block's total
// drop by the number removed (bc: the count pass's grid).
template <int G>
__global__ void __launch_bounds__(ST) kx_sv_refine_kernel(const float *__restrict__ pts, int64_t n,
                                                          const int32_t *kdev, int K, void *ws, Layout L, int32_t bc)
{
    __shared__ KPoly sp;
    const Octagon *oct = at<Octagon>(ws, L.oct);
    const int Kr = kdev ? *kdev : K;
    if (Kr == 8 || !kx_stage_on(oct, kdev, Kr)) return;
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(at<KPoly>(ws, L.kpoly));
        uint32_t *dst = reinterpret_cast<uint32_t *>(&sp);
        for (uint32_t w = threadIdx.x; w < sizeof(KPoly) / 4; w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    uint16_t *bits = at<uint16_t>(ws, L.keep_bits);
    unsigned long long *status = at<unsigned long long>(ws, L.filt_status);
    uint32_t *bsum = at<uint32_t>(ws, L.filt_bsum);
    const float2 *p2 = reinterpret_cast<const float2 *>(pts);
    const int64_t ntiles = ceil_div(n, (int64_t)kFiltTile);
    const int64_t per_block = ceil_div(ntiles, (int64_t)bc);
    const uint32_t t = threadIdx.x, lane = lane_id();
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t kb = bits[tile * kFiltThreads + t];
        uint32_t gone = 0;
        for (uint32_t b = kb; b; b &= b - 1u) {
            const int q = __ffs(b) - 1;
            const float2 v = p2[sv_point<G>(tile * kFiltTile, t, q)];
            if (!kx_keep(sp, v.x, v.y)) gone |= 1u << q;
        }
        if (gone) bits[tile * kFiltThreads + t] = (uint16_t)(kb & ~gone);
        uint32_t removed = __popc(gone);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) removed += __shfl_xor_sync(0xffffffffu, removed, o);
        if (lane == 0 && removed) {
            atomicAdd(&status[tile], 0ull - (unsigned long long)removed);
            atomicSub(&bsum[tile / per_block], removed);
        }
    }
}

template <int G>
cudaError_t launch_kx_sv_stage(const float *pts, int64_t n, const float *dirs, const int32_t *kdev, int K,
                               uint32_t *ext_out, void *ws, const Layout &L, int64_t bc, cudaStream_t st)
{
    const int64_t ntiles = ceil_div(n, (int64_t)kFiltTile);
    // the device's choice is mostly "no second polygon": a grid of one block
    // per SM keeps the two launches that then return at once short
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)sm_count() * (kdev ? 1 : 4)));
    const unsigned g = (unsigned)grid;
    probe_before(CH_K_KGON, st);
    if (kdev) kx_sv_extremes_kernel<0, G><<<g, ST, 0, st>>>(pts, n, dirs, kdev, ext_out, ws, L);
    else if (K == 16) kx_sv_extremes_kernel<16, G><<<g, ST, 0, st>>>(pts, n, dirs, kdev, ext_out, ws, L);
    else if (K == 32) kx_sv_extremes_kernel<32, G><<<g, ST, 0, st>>>(pts, n, dirs, kdev, ext_out, ws, L);
    else kx_sv_extremes_kernel<64, G><<<g, ST, 0, st>>>(pts, n, dirs, kdev, ext_out, ws, L);
    kx_sv_refine_kernel<G><<<g, ST, 0, st>>>(pts, n, kdev, K, ws, L, (int32_t)bc);
    note_kernels(CH_K_KGON, 2);
    probe_after(CH_K_KGON, st);
    return cudaGetLastError();
}

template <class Kern>
int resident(Kern k, int threads)
{
    int v = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k, threads, 0);
    return v > 0 ? v : 1;
}

template <int K>
cudaError_t launch_kx_extremes_k(const float *pts, int64_t n, const float *dirs, uint32_t *ext_out, void *ws,
                                 const Layout &L, cudaStream_t st)
{
    static const int per_sm = resident(kx_extremes_kernel<K>, XT);
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, (int64_t)XTILE), (int64_t)sm_count() * per_sm));
    kx_extremes_kernel<K><<<(unsigned)blocks, XT, 0, st>>>(pts, n, dirs, ext_out, ws, L,
                                                           at<unsigned long long>(ws, L.ctrl), (int64_t)L.zero_words);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_kx_extremes(const float *pts, int64_t n, const float *dirs, int K, uint32_t *ext_out, void *ws,
                               const Layout &L, cudaStream_t st)
{
    probe_before(CH_K_EXTREMES, st);
    cudaError_t e = cudaErrorInvalidValue;
    switch (K) {
    case 8: e = launch_kx_extremes_k<8>(pts, n, dirs, ext_out, ws, L, st); break;
    case 16: e = launch_kx_extremes_k<16>(pts, n, dirs, ext_out, ws, L, st); break;
    case 32: e = launch_kx_extremes_k<32>(pts, n, dirs, ext_out, ws, L, st); break;
    case 64: e = launch_kx_extremes_k<64>(pts, n, dirs, ext_out, ws, L, st); break;
    default: break;
    }
    note_kernels(CH_K_EXTREMES, 1);
    probe_after(CH_K_EXTREMES, st);
    return e;
}

cudaError_t launch_kx_count(const float *pts, int64_t n, int K, void *ws, const Layout &L, int64_t *grid,
                            cudaStream_t st)
{
    (void)K;   // the polygon in ws carries it
    const bool vec = (reinterpret_cast<uintptr_t>(pts) & 15u) == 0;
    static const int per_sm2 = resident(kx_count_kernel<2>, kFiltThreads);
    static const int per_sm1 = resident(kx_count_kernel<1>, kFiltThreads);
    const int64_t ntiles = ceil_div(n, (int64_t)kFiltTile);
    const int64_t bc = std::max<int64_t>(
        1, std::min<int64_t>({ntiles, (int64_t)sm_count() * (vec ? per_sm2 : per_sm1), (int64_t)kFiltMaxBlocks}));
    *grid = bc;
    probe_before(CH_K_FILTER, st);
    if (vec) kx_count_kernel<2><<<(unsigned)bc, kFiltThreads, 0, st>>>(pts, n, ws, L);
    else kx_count_kernel<1><<<(unsigned)bc, kFiltThreads, 0, st>>>(pts, n, ws, L);
    note_kernels(CH_K_FILTER, 1);
    probe_after(CH_K_FILTER, st);
    return cudaGetLastError();
}

cudaError_t launch_kx_sv(const float *pts, int64_t n, const float *dirs, const int32_t *kdev, int K, uint32_t *ext_out,
                        void *ws, const Layout &L, int64_t bc, cudaStream_t st)
{
    const bool vec = (reinterpret_cast<uintptr_t>(pts) & 15u) == 0;
    return vec ? launch_kx_sv_stage<2>(pts, n, dirs, kdev, K, ext_out, ws, L, bc, st)
               : launch_kx_sv_stage<1>(pts, n, dirs, kdev, K, ext_out, ws, L, bc, st);
}



}  // namespace ch

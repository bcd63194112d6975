// filter.cu -- Sec. 3.2 of Carrasco et al.: buildingFilter (is a point
// strictly inside the eight-vertex polygon?) and compactingFilteredPoints
// (stable compaction of the kept points).
//
// The paper writes an n-entry flag vector, scans it (tensor-core segmented
// scan, Thrust or CUB) and scatters.  Flags never reach memory here; two
// variants are built:
//
//  * two-pass (default): a streaming count pass tests 4096-point tiles and
//    writes keep bits and one survivor count per tile, each block over a
//    contiguous range of tiles, plus the block's total; a scatter pass with
//    the same grid finds each tile's output offset from the block totals
//    and an in-block scan of its range, visits only the tiles that have
//    survivors, loads only the kept points and writes them in ascending
//    index order.  No block waits on another, so both passes stream at
//    memory speed; when almost everything is discarded (normal data) the
//    points are read once, when nothing is (circle) they are read twice.
//  * single-pass: one persistent kernel takes tiles in ticket order, tests
//    them, publishes the tile count, gets its offset by decoupled look-back
//    and writes its survivors; points are read once, but each tile waits on
//    its predecessors.
//
// The test: the quick-discard rectangle, then the polygon edge facing the
// point's octant; a point strictly left of that edge is likely inside and
// needs every edge, so such points are queued per warp and tested 32 at a
// time (spread over the lanes they would hold whole warps in the edge
// loop).
//
// In the hull step the fan test of kgon.cu runs between the two passes and
// clears keep bits of points strictly inside the fan, so the scatter pass
// writes only the points that survive both tests.
//
// Memory traffic: 8 bytes per point read (twice for tiles with survivors in
// the two-pass variant), 12 bytes per kept point written.
#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "fan.cuh"
#include "launch.h"

namespace ch {

namespace {

// Outside the closed bounding box of the polygon's vertices: never strictly
// inside the polygon.  Only tested when the vertices were supplied by the
// caller (BOX); the data's own extremes span a box holding every point.
template <bool BOX>
__device__ __forceinline__ bool outside_box(const Octagon &o, float x, float y)
{
    if constexpr (BOX) return x < o.bxl || x > o.bxh || y < o.byl || y > o.byh;
    return false;
}

// keep(p) <=> NOT (p strictly left of every valid edge); see
// build_octagon_warp for the error bound of the binary32 test, which holds
// for points inside the vertices' bounding box.  The first edge tried is
// the one facing p's octant around the box centre, which settles points
// outside the polygon after one test; the order does not change the result.
template <bool BOX>
__device__ __forceinline__ bool keep_point(const Octagon &o, float x, float y)
{
    if (x >= o.xl && x <= o.xh && y >= o.yl && y <= o.yh) return false;
    if (!o.has_edges || outside_box<BOX>(o, x, y)) return true;
    const float ux = x - o.cx, uy = y - o.cy;
    int s;
    if (uy >= 0.0f) {
        if (ux >= 0.0f) s = ux >= uy ? 0 : 1;
        else s = uy >= -ux ? 2 : 3;
    } else {
        if (ux < 0.0f) s = -ux >= -uy ? 4 : 5;
        else s = -uy >= ux ? 6 : 7;
    }
#pragma unroll 1
    for (int j = 0; j < 8; ++j) {
        const int e = (s + j) & 7;
        if (!((o.valid >> e) & 1u)) continue;
        const float u = __fsub_rn(x, o.ax[e]);
        const float v = __fsub_rn(y, o.ay[e]);
        const float t = __fsub_rn(__fmul_rn(o.dx[e], v), __fmul_rn(o.dy[e], u));
        const float bnd = o.bound[e];
        if (t > bnd) continue;
        if (t < -bnd) return true;
        if (orient_d(o.ax[e], o.ay[e], o.bx[e], o.by[e], x, y) <= 0) return true;
    }
    return false;
}

constexpr int NW = kFiltThreads / 32;

// The polygon in shared memory, with the first look's per-edge data packed
// (one 16-byte and one 4-byte load per point): (ax, ay, dx, dy) and the
// bound of edge k; an edge of zero length gets zeros and +inf, which never
// proves a point outside it.
struct OctSmem : Octagon {
    float4 e4[8];
    float eb[8];
};

// Fills the packed edges of `so` from the polygon `o` (threads 0..7; the
// caller synchronises before they are read).
__device__ __forceinline__ void pack_edges(OctSmem &so, const Octagon &o)
{
    const uint32_t k = threadIdx.x;
    if (k < 8) {
        const bool v = (o.valid >> k) & 1u;
        so.e4[k] = v ? make_float4(o.ax[k], o.ay[k], o.dx[k], o.dy[k]) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        so.eb[k] = v ? o.bound[k] : __int_as_float(0x7f800000);
    }
}

// A point's first look: 0 discard (inside the quick-discard rectangle), 1
// keep (outside the vertices' box, or proven not strictly left of the edge
// facing it), 2 deferred (likely strictly inside: every edge must be
// tested).  The facing edge is the one of p's octant around the box centre,
// picked without branches (on a circle the lanes of a warp face every
// octant); any edge would give the same final decisions (a 1 is a proof, a
// 2 is tested in full).
template <bool BOX>
__device__ __forceinline__ uint32_t first_look(const OctSmem &o, float x, float y)
{
    // the rectangle first, as an early exit: it holds nearly every point of
    // a normal cloud (whole warps skip the rest) and none of a circle's
    if (x >= o.xl && x <= o.xh && y >= o.yl && y <= o.yh) return 0u;
    if (!o.has_edges || outside_box<BOX>(o, x, y)) return 1u;
    const float ux = x - o.cx, uy = y - o.cy;
    const float aux = fabsf(ux), auy = fabsf(uy);
    const uint32_t q = uy < 0.0f ? (ux < 0.0f ? 2u : 3u) : (ux < 0.0f ? 1u : 0u);   // quadrant
    const uint32_t e = 2u * q + ((q & 1u) ? (auy >= aux ? 0u : 1u) : (aux >= auy ? 0u : 1u));
    const float4 d = o.e4[e];
    const float u = __fsub_rn(x, d.x);
    const float v = __fsub_rn(y, d.y);
    const float t = __fsub_rn(__fmul_rn(d.z, v), __fmul_rn(d.w, u));
    return t < -o.eb[e] ? 1u : 2u;
}

// Deferred points, spread over the lanes, would hold whole warps in the
// edge loop; each warp queues them (lane, item) and tests them 32 at a
// time after its items' first look, re-reading each point (an L2 hit).
constexpr uint32_t kDeferCap = 32 * kFiltItems;   // every item of the warp

struct FiltQueue {
    uint16_t tag[kDeferCap];   // lane << 4 | item
    uint32_t res[32];          // kept item bits, per lane
};

__device__ __forceinline__ void queue_reset(FiltQueue &q)
{
    q.res[lane_id()] = 0u;
    __syncwarp();
}

// Tests this warp's deferred points (dm: this lane's deferred items, all
// lanes call): they are queued in lane order (an exclusive scan of the
// lanes' counts; the queue holds every item of the warp), tested 32 at a
// time, and this lane's keep bits among them are returned.  load(lane,
// item) reads a point of this warp.
template <bool BOX, class LoadPoint>
__device__ __forceinline__ uint32_t resolve_deferred(FiltQueue &q, const Octagon &so, uint32_t dm, LoadPoint load)
{
    const uint32_t c = __popc(dm);
    if (!__any_sync(0xffffffffu, c != 0u)) return 0u;   // the common case: nothing deferred
    const uint32_t lane = lane_id();
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    uint32_t slot = incl - c;
    for (uint32_t m = dm; m; m &= m - 1u) q.tag[slot++] = (uint16_t)((lane << 4) | (uint32_t)(__ffs(m) - 1));
    __syncwarp();
    for (uint32_t i = lane; i < total; i += 32) {
        const uint32_t tg = q.tag[i];
        const float2 v = load(tg >> 4, tg & 15u);
        if (keep_point<BOX>(so, v.x, v.y)) atomicOr(&q.res[tg >> 4], 1u << (tg & 15u));
    }
    __syncwarp();
    const uint32_t r = q.res[lane];
    q.res[lane] = 0u;   // only this lane touches its entry until the next call's barrier
    __syncwarp();
    return r;
}

// Copies the polygon to shared memory; false when the call was aborted
// (non-finite input or a bad vertex index).
__device__ __forceinline__ bool load_octagon(OctSmem &so, void *ws, const Layout &L)
{
    const Octagon *g = at<Octagon>(ws, L.oct);
    const uint32_t *src = reinterpret_cast<const uint32_t *>(g);
    uint32_t *dst = reinterpret_cast<uint32_t *>(static_cast<Octagon *>(&so));
    for (uint32_t w = threadIdx.x; w < sizeof(Octagon) / 4; w += blockDim.x) dst[w] = src[w];
    pack_edges(so, *g);
    __syncthreads();
    return !so.abort;
}

// Loads and tests one tile.  Thread t holds the points
// base + (r * 256 + t) * G + h, r < kFiltItems / G, h < G (G = 2: one
// 16-byte load per row; G = 1: one 8-byte load).  Returns the keep bits
// (bit r * G + h); positions past n are not kept.
template <int G, bool BOX>
__device__ __forceinline__ uint32_t load_test(const float *__restrict__ pts, int64_t n, int64_t base,
                                              const OctSmem &so, float (&px)[kFiltItems], float (&py)[kFiltItems],
                                              FiltQueue &fq)
{
    constexpr int ROWS = kFiltItems / G;
    const uint32_t tid = threadIdx.x;
    uint32_t keep = 0;
    if (base + kFiltTile <= n) {
        if constexpr (G == 2) {
            const float4 *p4 = reinterpret_cast<const float4 *>(pts) + base / 2;
            float4 v[ROWS];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) v[r] = __ldcs(p4 + r * kFiltThreads + tid);
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                px[2 * r] = v[r].x;
                py[2 * r] = v[r].y;
                px[2 * r + 1] = v[r].z;
                py[2 * r + 1] = v[r].w;
            }
        } else {
            const float2 *p2 = reinterpret_cast<const float2 *>(pts) + base;
            float2 v[ROWS];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) v[r] = __ldcs(p2 + r * kFiltThreads + tid);
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                px[r] = v[r].x;
                py[r] = v[r].y;
            }
        }
        uint32_t dm = 0;   // deferred items
#pragma unroll
        for (int q = 0; q < kFiltItems; ++q) {
            const uint32_t c = first_look<BOX>(so, px[q], py[q]);
            keep |= (c == 1u ? 1u : 0u) << q;
            dm |= (c == 2u ? 1u : 0u) << q;
        }
        const uint32_t wbase = tid & ~31u;
        keep |= resolve_deferred<BOX>(fq, so, dm, [&](uint32_t ln, uint32_t item) {
            const int64_t i = base + (int64_t)((item / G) * kFiltThreads + wbase + ln) * G + item % G;
            return reinterpret_cast<const float2 *>(pts)[i];
        });
    } else {
        const float2 *p2 = reinterpret_cast<const float2 *>(pts);
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
#pragma unroll
            for (int h = 0; h < G; ++h) {
                const int64_t i = base + (int64_t)(r * kFiltThreads + tid) * G + h;
                px[r * G + h] = 0.0f;
                py[r * G + h] = 0.0f;
                if (i < n) {
                    const float2 v = p2[i];
                    px[r * G + h] = v.x;
                    py[r * G + h] = v.y;
                    if (keep_point<BOX>(so, v.x, v.y)) keep |= 1u << (r * G + h);
                }
            }
        }
    }
    return keep;
}

// Kept points per (row, warp), turned into exclusive offsets in row-major
// order (the point order of the tile) in s_off by warp 0.  Returns the tile
// total to warp 0.  The caller synchronises before and after.
template <int G>
__device__ __forceinline__ void row_counts(uint32_t keep, uint32_t (&s_off)[kFiltItems / G][NW])
{
    constexpr int ROWS = kFiltItems / G;
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        uint32_t c = 0;
#pragma unroll
        for (int h = 0; h < G; ++h) c += __popc(__ballot_sync(0xffffffffu, (keep >> (r * G + h)) & 1u));
        if (lane == 0) s_off[r][warp] = c;
    }
}

template <int G>
__device__ __forceinline__ uint32_t scan_rows_warp0(uint32_t (&s_off)[kFiltItems / G][NW])
{
    constexpr int PER = (kFiltItems / G) * NW / 32;
    const uint32_t lane = lane_id();
    uint32_t *flat = &s_off[0][0];
    uint32_t loc[PER];
    uint32_t sum = 0;
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
    uint32_t run = incl - sum;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        flat[lane * PER + k] = run;
        run += loc[k];
    }
    return __shfl_sync(0xffffffffu, incl, 31);
}

// Writes the kept points of one tile; excl is the tile's output offset.
template <int G, bool KEYS>
__device__ __forceinline__ void scatter_tile(uint32_t keep, int64_t base, uint64_t excl,
                                             const uint32_t (&s_off)[kFiltItems / G][NW], const float (&px)[kFiltItems],
                                             const float (&py)[kFiltItems], uint32_t *surv_idx, float2 *surv_pts,
                                             uint32_t *out_keys, unsigned long long *out_pay)
{
    constexpr int ROWS = kFiltItems / G;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        uint32_t pre = s_off[r][warp];
#pragma unroll
        for (int h = 0; h < G; ++h) pre += __popc(__ballot_sync(0xffffffffu, (keep >> (r * G + h)) & 1u) & lt);
#pragma unroll
        for (int h = 0; h < G; ++h) {
            if ((keep >> (r * G + h)) & 1u) {
                const int64_t pos = (int64_t)excl + pre;
                const uint32_t idx = (uint32_t)(base + (int64_t)(r * kFiltThreads + tid) * G + h);
                if constexpr (KEYS) {
                    out_keys[pos] = ord_key(px[r * G + h]);
                    out_pay[pos] = ((unsigned long long)ord_key(py[r * G + h]) << 32) | idx;
                } else {
                    surv_idx[pos] = idx;
                    if (surv_pts) surv_pts[pos] = make_float2(px[r * G + h], py[r * G + h]);
                }
                ++pre;
            }
        }
    }
}

// One warp writes the kept points of one tile in point order, from the
// stored keep bits: the tile's 256 filter threads in eight groups of 32
// (group k holds threads 32 k + lane), each thread with kFiltItems / G rows
// of G points (point base + (r * 256 + t) * G + h).  The warp first counts
// every row's kept points (each row's first output position), asks L2 for
// all of its lanes' kept points at once, then per group loads the group's
// kept rows together and writes them (the warps of a block take different
// tiles and never wait on one another).
template <int G, bool KEYS>
__device__ __forceinline__ void scatter_tile_warp(const float *__restrict__ pts, int64_t n,
                                                  const uint16_t *__restrict__ tbits, int64_t base, uint32_t out_off,
                                                  uint32_t *surv_idx, float2 *surv_pts, uint32_t *out_keys,
                                                  unsigned long long *out_pay)
{
    constexpr int ROWS = kFiltItems / G;
    constexpr uint32_t RM = (1u << G) - 1u;   // a row's bits among a thread's 16
    const uint32_t lane = lane_id(), lt = (1u << lane) - 1u;
    uint32_t kb[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) kb[k] = tbits[k * 32 + lane];
    uint32_t racc[ROWS];   // next output position of row r
    {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) w[j] = kb[2 * j] | (kb[2 * j + 1] << 16);
        uint32_t run = out_off;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const uint32_t m = (RM << (r * G)) * 0x10001u;
            uint32_t c = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) c += __popc(w[j] & m);
            racc[r] = run;
            run += __reduce_add_sync(0xffffffffu, c);
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            if ((kb[k] >> (r * G)) & RM)
                prefetch_l2(pts + 2 * (base + (int64_t)(r * kFiltThreads + k * 32 + lane) * G));
        }
    }
    const auto put = [&](uint32_t pos, float x, float y, uint32_t idx) {
        if constexpr (KEYS) {
            out_keys[pos] = ord_key(x);
            out_pay[pos] = ((unsigned long long)ord_key(y) << 32) | idx;
        } else {
            surv_idx[pos] = idx;
            if (surv_pts) surv_pts[pos] = make_float2(x, y);
        }
    };
    // (one group at a time: its bits again from L1, so that the compiler
    // keeps one group's loads in registers, not all eight)
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
        const uint32_t kbk = tbits[k * 32 + lane];
        if (!__any_sync(0xffffffffu, kbk != 0u)) continue;
        const uint32_t t = k * 32 + lane;
        if constexpr (G == 2) {
            float4 v[ROWS];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                v[r] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if ((kbk >> (2 * r)) & 3u) {
                    const int64_t i = base + (int64_t)(r * kFiltThreads + t) * 2;
                    if (i + 1 < n) {
                        v[r] = __ldcs(reinterpret_cast<const float4 *>(pts) + i / 2);
                    } else {
                        const float2 a = reinterpret_cast<const float2 *>(pts)[i];
                        v[r] = make_float4(a.x, a.y, 0.0f, 0.0f);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const uint32_t m = (kbk >> (2 * r)) & 3u;
                const uint32_t b0 = __ballot_sync(0xffffffffu, m & 1u), b1 = __ballot_sync(0xffffffffu, m & 2u);
                if (!(b0 | b1)) continue;
                uint32_t pos = racc[r] + __popc(b0 & lt) + __popc(b1 & lt);
                racc[r] += __popc(b0) + __popc(b1);
                const uint32_t idx = (uint32_t)(base + (int64_t)(r * kFiltThreads + t) * 2);
                if (m & 1u) put(pos++, v[r].x, v[r].y, idx);
                if (m & 2u) put(pos, v[r].z, v[r].w, idx + 1u);
            }
        } else {   // 16 rows of one point: two halves of 8 loads
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float2 v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int r = 8 * h + q;
                    v[q] = make_float2(0.0f, 0.0f);
                    if ((kbk >> r) & 1u) v[q] = __ldcs(reinterpret_cast<const float2 *>(pts) + base + r * kFiltThreads + t);
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int r = 8 * h + q;
                    const uint32_t m = (kbk >> r) & 1u;
                    const uint32_t b0 = __ballot_sync(0xffffffffu, m);
                    if (!b0) continue;
                    const uint32_t pos = racc[r] + __popc(b0 & lt);
                    racc[r] += __popc(b0);
                    if (m) put(pos, v[q].x, v[q].y, (uint32_t)(base + r * kFiltThreads + t));
                }
            }
        }
    }
}

__device__ __forceinline__ void write_count(bool keys, Ctrl *ctrl, uint32_t *surv_count, uint32_t v)
{
    if (keys) ctrl->surv_count = v;
    else *surv_count = v;
}

// ---------------------------------------------------------------------------
// single pass: ticket-ordered tiles with decoupled look-back
// ---------------------------------------------------------------------------
template <int G, bool KEYS, bool BOX>
__global__ void __launch_bounds__(kFiltThreads) filter_kernel(const float *__restrict__ pts, int64_t n,
                                                              void *ws, Layout L, uint32_t *__restrict__ surv_idx,
                                                              float2 *__restrict__ surv_pts,
                                                              uint32_t *__restrict__ surv_count)
{
    __shared__ OctSmem so;
    __shared__ FiltQueue s_fq[NW];
    queue_reset(s_fq[threadIdx.x >> 5]);
    __shared__ uint32_t s_off[kFiltItems / G][NW];
    __shared__ uint32_t s_tile;
    __shared__ unsigned long long s_excl;
    __shared__ uint32_t s_total;

    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    unsigned long long *status = at<unsigned long long>(ws, L.filt_status);
    if (!load_octagon(so, ws, L)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) write_count(KEYS, ctrl, surv_count, 0);
        return;
    }
    const int64_t ntiles = ceil_div(n, kFiltTile);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&ctrl->filt_ticket, 1u);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= ntiles) break;
        const int64_t base = tile * kFiltTile;
        float px[kFiltItems], py[kFiltItems];
        const uint32_t keep = load_test<G, BOX>(pts, n, base, so, px, py, s_fq[threadIdx.x >> 5]);
        row_counts<G>(keep, s_off);
        __syncthreads();
        if (warp == 0) {
            const uint32_t total = scan_rows_warp0<G>(s_off);
            unsigned long long excl = 0;
            if (tile == 0) {
                if (lane == 0) st_release_u64(status, kFlagP | total);
            } else {
                if (lane == 0) st_release_u64(status + tile, kFlagA | total);
                excl = lookback_u64(status, tile, ws, L, 10);
                if (lane == 0) st_release_u64(status + tile, kFlagP | ((excl + total) & kValMask));
            }
            if (lane == 0) {
                s_excl = excl;
                s_total = total;
                if (tile == ntiles - 1) write_count(KEYS, ctrl, surv_count, (uint32_t)(excl + total));
            }
        }
        __syncthreads();
        if (s_total != 0)
            scatter_tile<G, KEYS>(keep, base, s_excl, s_off, px, py, surv_idx, surv_pts, at<uint32_t>(ws, L.keys[0]),
                                  at<unsigned long long>(ws, L.pay[0]));
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// the speculative sweep's candidates (extremes.cu): when the sweep proved
// every other point strictly inside the octagon (Octagon::spec), the count
// and scatter passes test and write only the candidates.  Segment j holds
// (unordered) the candidates of the j-th sweep block's contiguous index
// range, so segments in order, each sorted by index, give the survivors in
// ascending index order.
// ---------------------------------------------------------------------------
// Count pass: the exact test of every candidate; the slots of a segment's
// survivors go to utmp (unordered), their number to skept, and each count
// block's total to the block totals the fan reads.
__device__ void spec_count(const Octagon &so, void *ws, const Layout &L, uint32_t (&s_w)[NW])
{
    SpecCtrl *sc = at<SpecCtrl>(ws, L.spec);
    const float2 *cpt = at<float2>(ws, L.pay[1]);
    uint32_t *kept_slot = at<uint32_t>(ws, L.utmp);
    __shared__ uint32_t s_k;
    __shared__ uint32_t s_pre[kSpecWarps + 1];   // candidates before each slice of the segment
    const uint32_t nseg = sc->nseg, cap = sc->cap;
    uint32_t block_total = 0;
    for (uint32_t j = blockIdx.x; j < nseg; j += gridDim.x) {
        const size_t seg0 = (size_t)j * kSpecWarps * cap;
        __syncthreads();   // s_k and s_pre of the previous segment have been read
        if (threadIdx.x < 32) {
            const uint32_t c = threadIdx.x < (uint32_t)kSpecWarps ? min(sc->scnt[j * kSpecWarps + threadIdx.x], cap) : 0u;
            uint32_t incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (threadIdx.x >= (uint32_t)o) incl += t;
            }
            if (threadIdx.x < (uint32_t)kSpecWarps) s_pre[threadIdx.x + 1] = incl;
            if (threadIdx.x == 0) {
                s_pre[0] = 0u;
                s_k = 0u;
            }
        }
        __syncthreads();
        // the segment's candidates in one sweep: e-th candidate = candidate
        // e - s_pre[w] of the slice of warp w, at slot w * cap + that
        const uint32_t total = s_pre[kSpecWarps];
        for (uint32_t e = threadIdx.x; e < total; e += blockDim.x) {
            uint32_t w = 0;
            while (s_pre[w + 1] <= e) ++w;
            const uint32_t slot = w * cap + (e - s_pre[w]);
            const float2 p = cpt[seg0 + slot];
            if (keep_point<false>(so, p.x, p.y)) kept_slot[seg0 + atomicAdd(&s_k, 1u)] = slot;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            sc->skept[j] = s_k;
            block_total += s_k;
        }
    }
    (void)s_w;
    if (threadIdx.x == 0) at<uint32_t>(ws, L.filt_bsum)[blockIdx.x] = block_total;
}

struct SpecScatterSmem {
    uint32_t idx[kSpecKeptSmem];   // indices of a segment's survivors
    uint32_t red[NW];
};

// Scatter pass: each segment's survivors, ranked by index, at the segment's
// offset (the survivors of the segments before it); block 0 writes the
// count.  A segment with more survivors than shared memory holds is ranked
// from global memory (slower, same result).
template <bool KEYS>
__device__ void spec_scatter(SpecScatterSmem &sm, void *ws, const Layout &L, uint32_t *surv_idx, float2 *surv_pts,
                             uint32_t *surv_count, uint32_t *out_keys, unsigned long long *out_pay)
{
    const SpecCtrl *sc = at<SpecCtrl>(ws, L.spec);
    const uint32_t *cidx = at<uint32_t>(ws, L.keys[1]);
    const float2 *cpt = at<float2>(ws, L.pay[1]);
    const uint32_t *kept_slot = at<uint32_t>(ws, L.utmp);
    const uint32_t nseg = sc->nseg, cap = sc->cap, tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    if (blockIdx.x == 0) {
        uint32_t t = 0;
        for (uint32_t i = tid; i < nseg; i += blockDim.x) t += sc->skept[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sm.red[warp] = t;
        __syncthreads();
        if (tid == 0) {
            uint32_t total = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) total += sm.red[w];
            write_count(KEYS, at<Ctrl>(ws, L.ctrl), surv_count, total);
        }
    }
    for (uint32_t j = blockIdx.x; j < nseg; j += gridDim.x) {
        const uint32_t k = sc->skept[j];   // block-uniform
        if (k == 0u) continue;
        // offset: survivors of the segments before j
        uint32_t before = 0;
        for (uint32_t i = tid; i < j; i += blockDim.x) before += sc->skept[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
        __syncthreads();   // sm of the previous segment has been read
        if (lane == 0) sm.red[warp] = before;
        const size_t seg0 = (size_t)j * kSpecWarps * cap;
        const bool in_smem = k <= (uint32_t)kSpecKeptSmem;
        if (in_smem)
            for (uint32_t e = tid; e < k; e += blockDim.x) sm.idx[e] = cidx[seg0 + kept_slot[seg0 + e]];
        __syncthreads();
        uint32_t off = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) off += sm.red[w];
        for (uint32_t e = tid; e < k; e += blockDim.x) {
            const uint32_t slot = kept_slot[seg0 + e];
            const uint32_t mine = cidx[seg0 + slot];
            uint32_t r = 0;
            if (in_smem)
                for (uint32_t q = 0; q < k; ++q) r += sm.idx[q] < mine ? 1u : 0u;
            else
                for (uint32_t q = 0; q < k; ++q) r += cidx[seg0 + kept_slot[seg0 + q]] < mine ? 1u : 0u;
            const float2 p = cpt[seg0 + slot];
            const size_t pos = (size_t)off + r;
            if constexpr (KEYS) {
                out_keys[pos] = ord_key(p.x);
                out_pay[pos] = ((unsigned long long)ord_key(p.y) << 32) | mine;
            } else {
                surv_idx[pos] = mine;
                if (surv_pts) surv_pts[pos] = p;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// two passes: count -> scan -> scatter
// ---------------------------------------------------------------------------
// filt_status[t] receives the survivor count of tile t (low 32 bits); the
// scan turns it into (offset << 32 | count).  Each thread's 16 keep bits go
// to keep_bits, so the scatter pass does not test again.
// Per-tile survivor counts of a window of kCountRing tiles, added up in
// shared memory by the warps as they finish each tile, written to
// filt_status when the window is done.  Schedule, chosen by each block
// from its first tile: where it keeps under a quarter of its points (the
// rectangle settles most of them: bound by memory) the warps meet at a
// barrier after every tile, so that they read each tile together (a warp's
// share is 512 B of every 4 KB row; warps spread over tiles lose DRAM row
// locality: 0.66 against 0.89 of the copy peak on 10^9 normal points);
// elsewhere (every point takes the edge test: bound by issue) they run
// free and one warp's deferred points do not hold the others.
constexpr int kCountRing = 256;

// Block-wide sum to thread 0 (s_w: one slot per warp).
__device__ __forceinline__ uint32_t block_sum_to0(uint32_t v, uint32_t (&s_w)[NW])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane_id() == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    uint32_t t = 0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 0; w < NW; ++w) t += s_w[w];
    }
    return t;
}

// fan_slots (the hull step, else NULL): on every fan_stride-th tile the
// kept points' packed (far_key << 32 | ~index) go into the fan's bin slots
// by atomicMax (read first: most points do not raise their bin), the
// first level's farthest sampled point per bin without a pass of its own.
template <int G, bool BOX>
__global__ void __launch_bounds__(kFiltThreads, BOX ? 4 : 5) filter_count_kernel(const float *__restrict__ pts, int64_t n,
                                                                    void *ws, Layout L,
                                                                    unsigned long long *fan_slots,
                                                                    int32_t fan_stride)
{
    __shared__ OctSmem so;
    __shared__ FiltQueue s_fq[NW];
    __shared__ uint32_t s_cnt[kCountRing];
    queue_reset(s_fq[threadIdx.x >> 5]);
    __shared__ uint32_t s_w[NW];
    for (int i = threadIdx.x; i < kCountRing; i += kFiltThreads) s_cnt[i] = 0u;
    if (!load_octagon(so, ws, L)) return;   // (its barrier also covers s_cnt)
    if constexpr (!BOX) {
        if (so.spec) {   // the speculative sweep proved all but its candidates inside
            spec_count(so, ws, L, s_w);
            return;
        }
    }
    unsigned long long *status = at<unsigned long long>(ws, L.filt_status);
    uint16_t *bits = at<uint16_t>(ws, L.keep_bits);
    const int64_t ntiles = ceil_div(n, kFiltTile);
    const uint32_t lane = lane_id();
    // a contiguous range of tiles per block, so the scatter pass finds
    // every tile's output offset from the block totals and its own range
    const int64_t per = ceil_div(ntiles, (int64_t)gridDim.x);
    const int64_t t1 = min(ntiles, (int64_t)(blockIdx.x + 1) * per);
    uint32_t part = 0;   // this thread's share of the block total
    bool first = true, lockstep = true;
    for (int64_t w0 = (int64_t)blockIdx.x * per; w0 < t1; w0 += kCountRing) {
        const int64_t w1 = min(t1, w0 + kCountRing);
        for (int64_t tile = w0; tile < w1; ++tile) {
            if (threadIdx.x == 0 && tile + 1 < t1) {   // the next tile streams into L2 meanwhile
                const int64_t nb = (tile + 1) * kFiltTile;
                const uint32_t nn = (uint32_t)std::min<int64_t>(kFiltTile, n - nb);
                if (((reinterpret_cast<uintptr_t>(pts + 2 * nb)) & 15u) == 0)
                    bulk_prefetch_l2(pts + 2 * nb, (nn * 8u) & ~15u);
            }
            float px[kFiltItems], py[kFiltItems];
            const uint32_t keep = load_test<G, BOX>(pts, n, tile * kFiltTile, so, px, py, s_fq[threadIdx.x >> 5]);
            bits[tile * kFiltThreads + threadIdx.x] = (uint16_t)keep;
            if (!BOX && fan_slots && tile % fan_stride == 0) {   // block-uniform (the hull step only)
                // the kept points again from L2 (the tile was just read), so
                // that the test's registers are free here
                const float r2ref = far_ref(so);
#pragma unroll 1
                for (uint32_t m = keep; m; m &= m - 1u) {
                    const int q = __ffs(m) - 1;
                    const uint32_t i = (uint32_t)(tile * kFiltTile + ((q / G) * kFiltThreads + threadIdx.x) * G + q % G);
                    const float2 p = __ldcg(reinterpret_cast<const float2 *>(pts) + i);
                    const int b = fan_bin(__fsub_rn(p.x, so.cx), __fsub_rn(p.y, so.cy));
                    const unsigned long long v =
                        ((unsigned long long)far_key(p.x, p.y, so.cx, so.cy, r2ref) << 32) | (uint32_t)~i;
                    if (v > __ldcg(fan_slots + b)) atomicMax(fan_slots + b, v);
                }
            }
            uint32_t c = __popc(keep);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            if (lane == 0 && c) atomicAdd(&s_cnt[tile - w0], c);
            if (first) {   // the block's first tile decides (block-uniform: read after the barrier)
                __syncthreads();
                lockstep = s_cnt[tile - w0] < (uint32_t)(kFiltTile / 4);
                first = false;
            } else if (lockstep) {
                __syncthreads();
            }
        }
        __syncthreads();   // every warp's counts of the window are in
        for (int64_t i = threadIdx.x; i < w1 - w0; i += kFiltThreads) {
            const uint32_t v = s_cnt[i];
            status[w0 + i] = v;
            s_cnt[i] = 0u;
            part += v;
        }
        __syncthreads();
    }
    const uint32_t total = block_sum_to0(part, s_w);
    if (threadIdx.x == 0) at<uint32_t>(ws, L.filt_bsum)[blockIdx.x] = total;
}

// Second pass, launched with the count pass's grid: block b owns the same
// tile range.  Its output offset is the sum of the earlier blocks' totals;
// an in-block scan of its tiles' counts gives each tile's offset, and only
// tiles with survivors are visited.  Block 0 writes the survivor count.
template <int G, bool KEYS>
__global__ void __launch_bounds__(kFiltThreads, 3) filter_scatter_kernel(const float *__restrict__ pts, int64_t n,
                                                                      void *ws, Layout L,
                                                                      uint32_t *__restrict__ surv_idx,
                                                                      float2 *__restrict__ surv_pts,
                                                                      uint32_t *surv_count, int allow_spec)
{
    __shared__ uint32_t s_abort;
    __shared__ uint32_t s_red[2][NW];
    __shared__ uint32_t s_list[kFiltThreads];    // non-empty tiles of a chunk: offset in chunk
    __shared__ uint32_t s_loff[kFiltThreads];    // and their output offsets
    __shared__ uint32_t s_nlist;
    __shared__ uint32_t s_spec;
    __shared__ SpecScatterSmem s_sp;
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    if (threadIdx.x == 0) {
        const Octagon *oct = at<Octagon>(ws, L.oct);
        s_abort = oct->abort;
        s_spec = allow_spec ? oct->spec : 0u;   // a polygon the octagon record does not describe: never
    }
    __syncthreads();
    if (s_abort) {
        if (blockIdx.x == 0 && threadIdx.x == 0) write_count(KEYS, ctrl, surv_count, 0);
        return;
    }
    if (s_spec) {   // only the speculative sweep's candidates can survive
        spec_scatter<KEYS>(s_sp, ws, L, surv_idx, surv_pts, surv_count, at<uint32_t>(ws, L.keys[0]),
                           at<unsigned long long>(ws, L.pay[0]));
        return;
    }
    const unsigned long long *status = at<unsigned long long>(ws, L.filt_status);
    const uint32_t *bsum = at<uint32_t>(ws, L.filt_bsum);
    const uint16_t *bits = at<uint16_t>(ws, L.keep_bits);
    uint32_t *out_keys = at<uint32_t>(ws, L.keys[0]);
    unsigned long long *out_pay = at<unsigned long long>(ws, L.pay[0]);
    const int64_t ntiles = ceil_div(n, kFiltTile);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    // offset of this block's range, and the total
    uint32_t before = 0, total = 0;
    for (uint32_t i = tid; i < gridDim.x; i += kFiltThreads) {
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
    for (int w = 0; w < NW; ++w) {
        before += s_red[0][w];
        total += s_red[1][w];
    }
    if (blockIdx.x == 0 && tid == 0) write_count(KEYS, ctrl, surv_count, total);
    __syncthreads();   // s_red is reused below
    const int64_t per = ceil_div(ntiles, (int64_t)gridDim.x);
    const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(ntiles, r0 + per);
    uint32_t run = before;
    for (int64_t c0 = r0; c0 < r1; c0 += kFiltThreads) {
        // this chunk's tile counts: exclusive scan and the non-empty ones
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
        for (int w = 0; w < NW; ++w) {
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
        for (uint32_t li = warp; li < nl; li += NW)
            scatter_tile_warp<G, KEYS>(pts, n, bits + (c0 + s_list[li]) * kFiltThreads, (c0 + s_list[li]) * kFiltTile,
                                       s_loff[li], surv_idx, surv_pts, out_keys, out_pay);
        __syncthreads();   // s_list, s_loff and s_red are rebuilt for the next chunk
        run += chunk_total;
    }
}

// ---------------------------------------------------------------------------
// many sets (ch_hull_batched): the two passes over set-aligned 4096-point
// tiles, with 8-byte loads (sets start anywhere); indices are set-local
// ---------------------------------------------------------------------------
// Thread t tests points lo + r * 256 + t of the set (r < 16), below hi.
__device__ __forceinline__ uint32_t bx_load_test(const float2 *__restrict__ p2, int64_t lo, int64_t hi,
                                                 const OctSmem &so, float (&px)[kFiltItems],
                                                 float (&py)[kFiltItems], FiltQueue &fq)
{
    uint32_t keep = 0, dm = 0;
#pragma unroll
    for (int r = 0; r < kFiltItems; ++r) {
        const int64_t i = lo + r * kFiltThreads + threadIdx.x;
        px[r] = py[r] = 0.0f;
        if (i < hi) {
            const float2 v = __ldcs(p2 + i);
            px[r] = v.x;
            py[r] = v.y;
            const uint32_t c = first_look<false>(so, v.x, v.y);
            keep |= (c == 1u ? 1u : 0u) << r;
            dm |= (c == 2u ? 1u : 0u) << r;
        }
    }
    const uint32_t wbase = threadIdx.x & ~31u;
    return keep | resolve_deferred<false>(fq, so, dm, [&](uint32_t ln, uint32_t item) {
               return p2[lo + (int64_t)item * kFiltThreads + wbase + ln];
           });
}

// Copies set b's polygon to shared memory when the block moves to a new set.
__device__ __forceinline__ void bx_octagon_to_smem(OctSmem &so, int64_t &cur, int64_t b, const Octagon *octs)
{
    if (b == cur) return;   // block-uniform
    __syncthreads();
    const uint32_t *src = reinterpret_cast<const uint32_t *>(octs + b);
    uint32_t *dst = reinterpret_cast<uint32_t *>(static_cast<Octagon *>(&so));
    for (uint32_t w = threadIdx.x; w < sizeof(Octagon) / 4; w += blockDim.x) dst[w] = src[w];
    pack_edges(so, octs[b]);
    __syncthreads();
    cur = b;
}

__global__ void __launch_bounds__(kFiltThreads) bx_filter_count_kernel(const float *__restrict__ pts, void *ws,
                                                                       Layout L, BatchLayout BL)
{
    __shared__ OctSmem so;
    __shared__ FiltQueue s_fq[NW];
    __shared__ uint32_t s_cnt[kCountRing];
    queue_reset(s_fq[threadIdx.x >> 5]);
    const BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    if (bc->abort) return;
    for (int i = threadIdx.x; i < kCountRing; i += kFiltThreads) s_cnt[i] = 0u;   // (the first set's load syncs)
    const SetInfo *sets = at<SetInfo>(ws, BL.sets);
    const uint32_t *tile_set = at<uint32_t>(ws, BL.tile_set);
    const Octagon *octs = at<Octagon>(ws, BL.octs);
    unsigned long long *status = at<unsigned long long>(ws, L.filt_status);
    uint16_t *bits = at<uint16_t>(ws, L.keep_bits);
    uint32_t *soct = at<uint32_t>(ws, BL.soct);
    const uint32_t lane = lane_id();
    // a contiguous range of tiles per block: the polygon is loaded once per
    // set the range touches (a block-wide step; between two, the warps run
    // free and add their tile counts up in s_cnt)
    const int64_t T = bc->tiles;
    const int64_t per = ceil_div(T, (int64_t)gridDim.x);
    const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(T, t0 + per);
    int64_t cur = -1;
    for (int64_t w0 = t0; w0 < t1; w0 += kCountRing) {
        const int64_t w1 = min(t1, w0 + kCountRing);
        for (int64_t t = w0; t < w1; ++t) {
            const int64_t b = tile_set[t];
            bx_octagon_to_smem(so, cur, b, octs);
            if (threadIdx.x == 0 && t + 1 < t1) {   // the next tile streams into L2 meanwhile
                const int64_t nb = tile_set[t + 1];
                const int64_t nlo = (t + 1 - sets[nb].tile_base) * (int64_t)kFiltTile;
                const int64_t nhi = min(nlo + kFiltTile, sets[nb].n);
                const float2 *np = reinterpret_cast<const float2 *>(pts) + sets[nb].pt_begin;
                const uintptr_t a0 = (reinterpret_cast<uintptr_t>(np + nlo) + 15) & ~(uintptr_t)15;
                const uintptr_t a1 = reinterpret_cast<uintptr_t>(np + nhi) & ~(uintptr_t)15;
                if (a1 > a0) bulk_prefetch_l2(reinterpret_cast<const void *>(a0), (uint32_t)(a1 - a0));
            }
            uint32_t keep = 0;
            if (!so.abort) {
                const int64_t lo = (int64_t)(t - sets[b].tile_base) * kFiltTile;
                const int64_t hi = min(lo + kFiltTile, sets[b].n);
                float px[kFiltItems], py[kFiltItems];
                keep = bx_load_test(reinterpret_cast<const float2 *>(pts) + sets[b].pt_begin, lo, hi, so, px, py,
                                    s_fq[threadIdx.x >> 5]);
            }
            bits[(size_t)t * kFiltThreads + threadIdx.x] = (uint16_t)keep;
            uint32_t c = __popc(keep);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            if (lane == 0 && c) atomicAdd(&s_cnt[t - w0], c);
        }
        __syncthreads();
        for (int64_t i = threadIdx.x; i < w1 - w0; i += kFiltThreads) {
            const uint32_t v = s_cnt[i];
            status[w0 + i] = v;
            s_cnt[i] = 0u;
            if (v) atomicAdd(&soct[tile_set[w0 + i]], v);
        }
        __syncthreads();
    }
}

// One block: tile offsets (exclusive scan of the counts), each set's
// survivor range, and the layout of the later stages: each set's
// super-chunks (4096 survivors, also the sort tiles) and merge-tree nodes.
__global__ void __launch_bounds__(1024) bx_filter_scan_kernel(void *ws, Layout L, BatchLayout BL)
{
    __shared__ uint64_t s_w[32];
    __shared__ uint64_t s_w2[32];
    __shared__ uint64_t s_total;
    BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    if (bc->abort) return;
    SetInfo *sets = at<SetInfo>(ws, BL.sets);
    uint32_t *sc_set = at<uint32_t>(ws, BL.sc_set);
    unsigned long long *status = at<unsigned long long>(ws, L.filt_status);
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nthr = blockDim.x;
    // ---- 1. tiles
    {
        const int64_t T = bc->tiles;
        const int64_t per = ceil_div(T, (int64_t)nthr);
        const int64_t t0 = threadIdx.x * per, t1 = min(t0 + per, T);
        uint64_t sum = 0;
        for (int64_t t = t0; t < t1; ++t) sum += status[t] & 0xffffffffull;
        uint64_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += u;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        uint64_t before = 0, total = 0;
        for (uint32_t w = 0; w < nthr / 32; ++w) {
            if (w < warp) before += s_w[w];
            total += s_w[w];
        }
        uint64_t run = before + incl - sum;
        for (int64_t t = t0; t < t1; ++t) {
            const uint64_t c = status[t] & 0xffffffffull;
            status[t] = (run << 32) | c;
            run += c;
        }
        if (threadIdx.x == 0) s_total = total;
        __syncthreads();
    }
    // ---- 2. sets: survivors, super-chunks, tree nodes
    const int64_t B = BL.num_sets;
    const int64_t T = bc->tiles;
    const uint64_t total = s_total;
    auto off = [&](int64_t t) -> uint64_t { return t < T ? (status[t] >> 32) : total; };
    const int64_t per = ceil_div(B, (int64_t)nthr);
    const int64_t b0 = threadIdx.x * per, b1 = min(b0 + per, B);
    uint64_t sc_sum = 0, nd_sum = 0;
    for (int64_t b = b0; b < b1; ++b) {
        const uint64_t sb = off(sets[b].tile_base);
        const uint32_t s = (uint32_t)(off(sets[b].tile_base + sets[b].ntiles) - sb);
        sets[b].surv_base = sb;
        sets[b].s = s;
        const int64_t nsc = ceil_div((int64_t)s, kChainC);
        sets[b].nsc = (uint32_t)nsc;
        sc_sum += nsc;
        nd_sum += nsc > 0 ? tree_nodes(nsc) + 1 : 0;
    }
    uint64_t i1 = sc_sum, i2 = nd_sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t u1 = __shfl_up_sync(0xffffffffu, i1, o);
        const uint64_t u2 = __shfl_up_sync(0xffffffffu, i2, o);
        if (lane >= (uint32_t)o) {
            i1 += u1;
            i2 += u2;
        }
    }
    __syncthreads();
    if (lane == 31) {
        s_w[warp] = i1;
        s_w2[warp] = i2;
    }
    __syncthreads();
    uint64_t bsc = 0, bnd = 0, tsc = 0;
    for (uint32_t w = 0; w < nthr / 32; ++w) {
        if (w < warp) {
            bsc += s_w[w];
            bnd += s_w2[w];
        }
        tsc += s_w[w];
    }
    uint64_t rsc = bsc + i1 - sc_sum, rnd = bnd + i2 - nd_sum;
    for (int64_t b = b0; b < b1; ++b) {
        sets[b].sc_base = (uint32_t)rsc;
        sets[b].node_base = (uint32_t)rnd;
        for (uint32_t k = 0; k < sets[b].nsc; ++k) sc_set[rsc + k] = (uint32_t)b;
        rsc += sets[b].nsc;
        rnd += sets[b].nsc > 0 ? tree_nodes(sets[b].nsc) + 1 : 0;
    }
    if (threadIdx.x == 0) bc->nsc = (uint32_t)tsc;
}

// One warp per tile with survivors (warps of the whole grid in turn); the
// scan left each tile's output offset in the high half of filt_status.
__global__ void __launch_bounds__(kFiltThreads, 3) bx_filter_scatter_kernel(const float *__restrict__ pts, void *ws,
                                                                            Layout L, BatchLayout BL)
{
    const BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    if (bc->abort) return;
    const SetInfo *sets = at<SetInfo>(ws, BL.sets);
    const uint32_t *tile_set = at<uint32_t>(ws, BL.tile_set);
    const unsigned long long *status = at<unsigned long long>(ws, L.filt_status);
    const uint16_t *bits = at<uint16_t>(ws, L.keep_bits);
    uint32_t *out_keys = at<uint32_t>(ws, L.keys[0]);
    unsigned long long *out_pay = at<unsigned long long>(ws, L.pay[0]);
    const uint32_t T = bc->tiles;
    const uint32_t nwarps = gridDim.x * NW;
    for (uint32_t t = blockIdx.x * NW + (threadIdx.x >> 5); t < T; t += nwarps) {
        const unsigned long long st = status[t];
        if ((st & 0xffffffffull) == 0) continue;   // warp-uniform
        const int64_t b = tile_set[t];
        const int64_t lo = (int64_t)(t - sets[b].tile_base) * kFiltTile;
        const float *p = pts + 2 * sets[b].pt_begin;
        scatter_tile_warp<1, true>(p, sets[b].n, bits + (size_t)t * kFiltThreads, lo, (uint32_t)(st >> 32), nullptr,
                                   nullptr, out_keys, out_pay);
    }
}

template <class K>
int occupancy(K kernel, int threads)
{
    int v = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, 0);
    return v > 0 ? v : 1;
}

template <int G, bool KEYS>
cudaError_t launch_single(const float *pts, int64_t n, void *ws, const Layout &L, uint32_t *surv_idx,
                          float *surv_pts, uint32_t *surv_count, cudaStream_t st)
{
    // the hull step (KEYS) filters with the data's own extremes; ch_filter's
    // caller-supplied vertices need the bounding-box check
    static int per_sm = occupancy(filter_kernel<G, KEYS, !KEYS>, kFiltThreads);
    const int64_t ntiles = ceil_div(n, kFiltTile);
    int64_t blocks = std::min<int64_t>((int64_t)sm_count() * per_sm, ntiles);
    filter_kernel<G, KEYS, !KEYS><<<(unsigned)std::max<int64_t>(blocks, 1), kFiltThreads, 0, st>>>(
        pts, n, ws, L, surv_idx, reinterpret_cast<float2 *>(surv_pts), surv_count);
    note_kernels(CH_K_FILTER, 1);
    return cudaGetLastError();
}

// BOX: the polygon's vertices were supplied by the caller (ch_filter), so
// points outside their box must be kept first; otherwise they are the
// data's extremes, and the scatter may take the speculative sweep's
// candidates (Octagon::spec)
template <int G, bool KEYS, bool BOX>
cudaError_t launch_two_pass(const float *pts, int64_t n, void *ws, const Layout &L, uint32_t *surv_idx,
                            float *surv_pts, uint32_t *surv_count, cudaStream_t st, bool fan, const KgonStage *kg)
{
    // both passes use the same grid (block b owns the same tile range),
    // the count pass's resident blocks (the scatter pass's warps take
    // tiles on their own, so a second partial wave of it costs little)
    static const int per_sm = occupancy(filter_count_kernel<G, BOX>, kFiltThreads);
    const int64_t ntiles = ceil_div(n, kFiltTile);
    const int64_t bc = std::max<int64_t>(
        1, std::min<int64_t>(std::min<int64_t>((int64_t)sm_count() * per_sm, kFiltMaxBlocks), ntiles));
    // the hull step's fan gathers its bin maxima in this pass
    unsigned long long *fan_slots = (fan && !BOX) ? at<KgonCtrl>(ws, L.kgon_ctrl)->slot : nullptr;
    filter_count_kernel<G, BOX><<<(unsigned)bc, kFiltThreads, 0, st>>>(pts, n, ws, L, fan_slots,
                                                                       (int32_t)fan_sample_stride(ntiles));
    if (kg && (kg->kdev || kg->K != 8)) {   // the second polygon, over the octagon's survivors
        probe_after(CH_K_FILTER, st);
        const cudaError_t e = launch_kx_sv(pts, n, kg->dirs, kg->kdev, kg->K, kg->ext_out, ws, L, bc, st);
        if (e != cudaSuccess) return e;
        probe_before(CH_K_FILTER, st);
    }
    if (fan) {   // timed as its own group, between the filter's two
        probe_after(CH_K_FILTER, st);
        const cudaError_t e = launch_fan(pts, n, G == 2, bc, ws, L, st);
        if (e != cudaSuccess) return e;
        probe_before(CH_K_FILTER, st);
    }
    filter_scatter_kernel<G, KEYS><<<(unsigned)bc, kFiltThreads, 0, st>>>(
        pts, n, ws, L, surv_idx, reinterpret_cast<float2 *>(surv_pts), surv_count, BOX ? 0 : 1);
    note_kernels(CH_K_FILTER, 2);
    if (fan && KEYS) {   // the hull step: the fan's second level over the survivors just written
        probe_after(CH_K_FILTER, st);
        const cudaError_t e = launch_fan2(n, ws, L, st);
        if (e != cudaSuccess) return e;
        probe_before(CH_K_FILTER, st);
    }
    return cudaGetLastError();
}

// 0: two passes, 1: single pass with look-back; process-wide, read once per
// call when its kernels are enqueued (an atomic, so setting it from another
// host thread is not a data race)
std::atomic<int> g_filter_variant{0};

template <int G, bool KEYS>
cudaError_t launch_variant(const float *pts, int64_t n, void *ws, const Layout &L, uint32_t *surv_idx,
                           float *surv_pts, uint32_t *surv_count, cudaStream_t st, int variant, bool fan,
                           bool data_extremes, const KgonStage *kg)
{
    probe_before(CH_K_FILTER, st);
    cudaError_t e;
    if (variant == 1) e = launch_single<G, KEYS>(pts, n, ws, L, surv_idx, surv_pts, surv_count, st);
    else if (KEYS || data_extremes)
        e = launch_two_pass<G, KEYS, false>(pts, n, ws, L, surv_idx, surv_pts, surv_count, st, fan, kg);
    else e = launch_two_pass<G, false, true>(pts, n, ws, L, surv_idx, surv_pts, surv_count, st, fan, nullptr);
    probe_after(CH_K_FILTER, st);
    return e;
}

}  // namespace

int filter_variant() { return g_filter_variant.load(std::memory_order_relaxed); }

cudaError_t launch_filter(const float *pts, int64_t n, void *ws, const Layout &L, uint32_t *surv_idx,
                          float *surv_pts, uint32_t *surv_count, bool keys_mode, cudaStream_t st, int variant,
                          bool fan, bool data_extremes, const KgonStage *kg)
{
    const int v = variant < 0 ? g_filter_variant.load(std::memory_order_relaxed) : variant;
    const bool vec = (reinterpret_cast<uintptr_t>(pts) & 15u) == 0;
    if (keys_mode)
        return vec ? launch_variant<2, true>(pts, n, ws, L, nullptr, nullptr, nullptr, st, v, fan, true, kg)
                   : launch_variant<1, true>(pts, n, ws, L, nullptr, nullptr, nullptr, st, v, fan, true, kg);
    return vec ? launch_variant<2, false>(pts, n, ws, L, surv_idx, surv_pts, surv_count, st, v, false, data_extremes,
                                          nullptr)
               : launch_variant<1, false>(pts, n, ws, L, surv_idx, surv_pts, surv_count, st, v, false, data_extremes,
                                          nullptr);
}

cudaError_t launch_filter_scatter(const float *pts, int64_t n, int64_t grid, void *ws, const Layout &L,
                                  uint32_t *surv_idx, float *surv_pts, uint32_t *surv_count, bool keys_mode,
                                  cudaStream_t st)
{
    const bool vec = (reinterpret_cast<uintptr_t>(pts) & 15u) == 0;
    float2 *sp = reinterpret_cast<float2 *>(surv_pts);
    const unsigned g = (unsigned)std::max<int64_t>(1, grid);
    if (keys_mode) {
        if (vec) filter_scatter_kernel<2, true><<<g, kFiltThreads, 0, st>>>(pts, n, ws, L, nullptr, nullptr, nullptr, 0);
        else filter_scatter_kernel<1, true><<<g, kFiltThreads, 0, st>>>(pts, n, ws, L, nullptr, nullptr, nullptr, 0);
    } else {
        if (vec) filter_scatter_kernel<2, false><<<g, kFiltThreads, 0, st>>>(pts, n, ws, L, surv_idx, sp, surv_count, 0);
        else filter_scatter_kernel<1, false><<<g, kFiltThreads, 0, st>>>(pts, n, ws, L, surv_idx, sp, surv_count, 0);
    }
    note_kernels(CH_K_FILTER, 1);
    return cudaGetLastError();
}

cudaError_t launch_bx_filter(const float *pts, void *ws, const Layout &L, const BatchLayout &BL, cudaStream_t st)
{
    static int per_sm_c = occupancy(bx_filter_count_kernel, kFiltThreads);
    static int per_sm_s = occupancy(bx_filter_scatter_kernel, kFiltThreads);
    const int tuned = tune_value(CH_TUNE_BX_FILTER);
    const int64_t bc = std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * (tuned ? tuned : per_sm_c), BL.tiles_max));
    const int64_t bs = std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * (tuned ? tuned : per_sm_s), BL.tiles_max));
    probe_before(CH_K_FILTER, st);
    bx_filter_count_kernel<<<(unsigned)bc, kFiltThreads, 0, st>>>(pts, ws, L, BL);
    // the hull step's fan for the sets with many octagon survivors, timed
    // as its own group between the count pass and the scan
    probe_after(CH_K_FILTER, st);
    const cudaError_t e = launch_bx_fan(pts, ws, L, BL, st);
    if (e != cudaSuccess) return e;
    probe_before(CH_K_FILTER, st);
    bx_filter_scan_kernel<<<1, 1024, 0, st>>>(ws, L, BL);
    bx_filter_scatter_kernel<<<(unsigned)bs, kFiltThreads, 0, st>>>(pts, ws, L, BL);
    note_kernels(CH_K_FILTER, 3);
    probe_after(CH_K_FILTER, st);
    return cudaGetLastError();
}

}  // namespace ch

extern "C" ch_status ch_filter_variant(int32_t variant)
{
    if (variant != 0 && variant != 1) return CH_ERR_ARG;
    ch::g_filter_variant.store(variant, std::memory_order_relaxed);
    return CH_OK;
}

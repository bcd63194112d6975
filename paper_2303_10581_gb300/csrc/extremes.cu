// extremes.cu -- Sec. 3.1 of Carrasco et al. (findingPolygon): the eight
// polygon vertices in one sweep over the points, and the construction of
// the filter polygon used by the point test of Sec. 3.2.
//
// The paper finds the four axis extremes with a block-warp min/max
// reduction and then the four corner points with a second reduction of
// Manhattan distances to the bounding-box corners.  The Manhattan distance
// from (x, y) to the corner (xmax, ymax) is (xmax + ymax) - (x + y), so the
// closest point is the argmax of x + y, and similarly for the other three
// corners (argmin x + y, argmin x - y, argmax x - y).  All eight therefore
// come out of ONE sweep: each thread keeps eight running (key, index)
// pairs, a warp-shuffle reduction combines them, and the grid finishes with
// one 64-bit atomicMax per slot on (order-preserving key << 32 | ~index),
// which selects the largest key and, among equal keys, the lowest index.
// The last block to finish decodes the winners and builds the polygon.
#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "launch.h"
#include "mlp.cuh"

namespace ch {

namespace {

// slot order = polygon vertex order R, TR, T, TL, L, BL, B, BR; every slot
// maximises its key (a minimum is the maximum of the negated key, and
// binary32 negation is exact)
struct Best {
    float k[8];
    uint32_t i[8];
};

__device__ __forceinline__ void consider(Best &b, float x, float y, uint32_t idx)
{
    const float s = __fadd_rn(x, y);
    const float d = __fsub_rn(x, y);
    const float key[8] = {x, s, y, -d, -x, -s, -y, d};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        // running keys start as NaN, so the first point is always taken
        // (a key can legitimately be -inf when x + y overflows); after
        // that !(key <= best) is key > best, since keys of finite points are
        // never NaN
        if (!(key[j] <= b.k[j])) {
            b.k[j] = key[j];
            b.i[j] = idx;
        }
    }
}

// Strict "better": larger key, or equal key and lower index; index
// 0xffffffff marks an empty candidate.
__device__ __forceinline__ void combine(float &k, uint32_t &i, float ok, uint32_t oi)
{
    if (oi == 0xffffffffu) return;
    if (i == 0xffffffffu || ok > k || (ok == k && oi < i)) {
        k = ok;
        i = oi;
    }
}

}  // namespace

// Builds the filter polygon from the eight vertex indices.  Run by one full
// warp.  Edge k joins vertex k to vertex k+1 (mod 8); edges of zero length
// are disabled.  For each edge the binary32 test
//   t = fl(fl(dx * fl(py - ay)) - fl(dy * fl(px - ax)))
// is Shewchuk's orient2d expression for (b, p, a) with the edge differences
// precomputed; its rounding error is below (3 + 16 eps) eps * (|fl(dx*v)| +
// |fl(dy*u)|), eps = 2^-24.  Because |px - ax| <= W = xmax - xmin and
// |py - ay| <= H and rounding is monotone, that sum never exceeds
// M = (|dx| fl(H) + |dy| fl(W))(1 + 2^-20), so bound = 4 eps M + 2^-140
// (the last term covers products that underflow) is a static bound valid
// for every point: t > bound proves "strictly left", t < -bound proves
// "not left", anything else is decided exactly.  The edge test is disabled
// (bound = +inf) when the box extents overflow or M > 2^100.
//
// The box W x H is the closed bounding box of the eight vertices.  When
// they are the data's extremes (data_extremes: R, T, L, B really are the
// largest x, y and smallest x, y of all points) every point lies in it.
// For vertices chosen by the caller that need not hold, so the record asks
// the point test to keep every point outside the box first (box_check): a
// point strictly left of every edge has winding number >= 1 around the
// vertex sequence, so it lies in the vertices' convex hull and hence in
// their box; a point outside the box is never strictly inside.  The static
// bound then holds for every point that reaches the edge test.
//
// A closed axis-aligned rectangle whose four corners are, exactly, strictly
// left of every valid edge lies strictly inside the polygon (the region
// "strictly left of every edge" is an intersection of open half-planes,
// hence convex); points in it are discarded with four comparisons.  The
// largest of a few concentric candidates that passes is kept.
__device__ void build_octagon_warp(const float2 *pts, const uint32_t *ext8, Octagon *out, bool data_extremes)
{
    const uint32_t lane = lane_id();
    const uint32_t k = lane & 7u;
    const float2 a = pts[ext8[k]];
    const float2 b = pts[ext8[(k + 1) & 7u]];
    float xmax, ymax, xmin, ymin;
    if (data_extremes) {   // bounding box from R, T, L, B
        xmax = pts[ext8[0]].x;
        ymax = pts[ext8[2]].y;
        xmin = pts[ext8[4]].x;
        ymin = pts[ext8[6]].y;
    } else {               // bounding box of all eight vertices (lanes k, k ^ 1, ... of each group of 8)
        xmax = xmin = a.x;
        ymax = ymin = a.y;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
            xmin = fminf(xmin, __shfl_xor_sync(0xffffffffu, xmin, o));
            ymax = fmaxf(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
            ymin = fminf(ymin, __shfl_xor_sync(0xffffffffu, ymin, o));
        }
    }
    const bool valid = !(a.x == b.x && a.y == b.y);
    const float dx = __fsub_rn(b.x, a.x), dy = __fsub_rn(b.y, a.y);
    const float W = __fsub_rn(xmax, xmin), H = __fsub_rn(ymax, ymin);
    float bound = __int_as_float(0x7f800000);  // +inf: binary32 test off
    if (W <= 3.0e38f && H <= 3.0e38f) {
        double M = __dadd_ru(__dmul_ru(fabs((double)dx), (double)H), __dmul_ru(fabs((double)dy), (double)W));
        M = __dmul_ru(M, 1.0 + 0x1p-20);
        if (M <= 0x1p100) {
            double B = __dadd_ru(__dmul_ru(M, 0x1p-22), 0x1p-140);
            bound = __double2float_ru(B);
        }
    }
    const uint32_t vmask = __ballot_sync(0xffffffffu, valid) & 0xffu;
    if (lane < 8) {
        out->ax[k] = a.x;
        out->ay[k] = a.y;
        out->bx[k] = b.x;
        out->by[k] = b.y;
        out->dx[k] = dx;
        out->dy[k] = dy;
        out->bound[k] = bound;
    }
    const double cxd = 0.5 * ((double)xmin + (double)xmax);
    const double cyd = 0.5 * ((double)ymin + (double)ymax);
    const double hw = 0.5 * ((double)xmax - (double)xmin);
    const double hh = 0.5 * ((double)ymax - (double)ymin);
    // quick-discard rectangle: lane = (corner c = lane / 8, edge k)
    float xl = 1.0f, xh = -1.0f, yl = 1.0f, yh = -1.0f;  // empty
    if (vmask != 0) {
        const double fr[8] = {0.80, 0.74, 0.68, 0.62, 0.55, 0.45, 0.35, 0.25};
        for (int j = 0; j < 8; ++j) {
            const float rxl = (float)(cxd - fr[j] * hw), rxh = (float)(cxd + fr[j] * hw);
            const float ryl = (float)(cyd - fr[j] * hh), ryh = (float)(cyd + fr[j] * hh);
            const uint32_t c = lane >> 3;
            const float px = (c == 0 || c == 3) ? rxl : rxh;
            const float py = (c < 2) ? ryl : ryh;
            bool ok = !valid || orient(a.x, a.y, b.x, b.y, px, py) > 0;
            if (!(rxl <= rxh && ryl <= ryh)) ok = false;
            if (__all_sync(0xffffffffu, ok)) {
                xl = rxl;
                xh = rxh;
                yl = ryl;
                yh = ryh;
                break;
            }
        }
    }
    if (lane == 0) {
        out->valid = vmask;
        out->has_edges = vmask != 0;
        out->abort = 0;
        out->xl = xl;
        out->xh = xh;
        out->yl = yl;
        out->yh = yh;
        out->cx = (float)cxd;
        out->cy = (float)cyd;
        out->bxl = xmin;
        out->bxh = xmax;
        out->byl = ymin;
        out->byh = ymax;
        out->box_check = data_extremes ? 0u : 1u;
        out->spec = 0u;
    }
}

// ---------------------------------------------------------------------------
// the sweep
// ---------------------------------------------------------------------------
// NaN-propagating maximum (PTX max.NaN): the tile maxima of x and y become
// NaN when a coordinate is NaN, which is how the sweep notices NaN input.
// An infinite coordinate surfaces as an infinite R, T, L or B vertex.
__device__ __forceinline__ float max_nan(float a, float b)
{
    float d;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// The eight slot keys of a point (every slot maximises its key).
__device__ __forceinline__ void slot_keys(float x, float y, float (&k)[8])
{
    const float s = __fadd_rn(x, y);
    const float d = __fsub_rn(x, y);
    k[0] = x;
    k[1] = s;
    k[2] = y;
    k[3] = -d;
    k[4] = -x;
    k[5] = -s;
    k[6] = -y;
    k[7] = d;
}

// The speculative sweep's test region.  A is the octagon
//   xl <= x <= xh, yl <= y <= yh, sl <= x + y <= sh, dl <= x - y <= dh
// (exact arithmetic) with every bound a multiple of a power of two g
// chosen so that A's eight vertices are exact binary32 points.  The sweep
// compares x, y and the keys fl(x + y), fl(x - y) it computes anyway with
// the axis bounds and with diagonal bounds moved inwards by a margin m:
// since |x| + |y| <= M inside the box, |fl(x + y) - (x + y)| <= 2^-24 M <=
// m, so a point passing the test lies in A.  The last block checks exactly
// that every vertex of A is strictly left of every valid edge of the final
// octagon P; A is convex, so every point in A is strictly inside P, and
// the filter discards it.  Points failing the test are the candidates.
struct SpecBox {
    float xl, xh, yl, yh;   // axis bounds of A
    float slb, shb, dlb, dhb;   // diagonal bounds of the test (A's, moved in by the margin)
    float vx[8], vy[8];     // A's vertices, counter-clockwise from (xh, sh - xh)
    uint32_t ok;            // 0: no usable region this call
    uint32_t pad[7];
};
static_assert(sizeof(SpecBox) <= 256, "the layout's region for the speculative sweep's box");

__device__ __forceinline__ bool spec_inside(const SpecBox &b, float x, float y, float s, float d)
{
    return x >= b.xl && x <= b.xh && y >= b.yl && y <= b.yh && s >= b.slb && s <= b.shb && d >= b.dlb &&
           d <= b.dhb;
}

// Reserves c candidate slots for this lane in its warp's slice (all lanes
// call it; wcnt, warp-uniform, counts the slice's slots in use) and returns
// the lane's first slot, or ~0u when the slice would overflow: then the
// speculation is over for every block (fail) and wcnt is left past cap.
__device__ __forceinline__ uint32_t slice_reserve(uint32_t c, uint32_t &wcnt, uint32_t cap, SpecCtrl *sc)
{
    const uint32_t lane = lane_id();
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += t;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (wcnt + total > cap) {
        if (lane == 0) st_relaxed_u32(&sc->fail, 1u);
        wcnt = cap + 1u;
        return ~0u;
    }
    const uint32_t first = wcnt + incl - c;
    wcnt += total;
    return first;
}

// Whether the speculation is still on for this warp: its own slice has
// room and no slice anywhere overflowed (read only when the warp has
// candidates to write, so a set with few candidates rarely reads it).
__device__ __forceinline__ bool spec_still_live(uint32_t wcnt, uint32_t cap, SpecCtrl *sc)
{
    uint32_t f = 0;
    if (lane_id() == 0) f = ld_relaxed_u32(&sc->fail);
    return wcnt <= cap && __shfl_sync(0xffffffffu, f, 0) == 0u;
}

// One point per lane (valid: the lane has one): the warp appends the
// candidates among them.
__device__ __forceinline__ void spec_warp_point(const SpecBox &b, bool valid, uint32_t i, float x, float y,
                                                uint32_t &wcnt, uint32_t cap, SpecCtrl *sc, uint32_t *cidx,
                                                float2 *cpt, size_t slice0)
{
    const bool cand = valid && !spec_inside(b, x, y, __fadd_rn(x, y), __fsub_rn(x, y));
    if (!__any_sync(0xffffffffu, cand) || !spec_still_live(wcnt, cap, sc)) return;
    const uint32_t pos = slice_reserve(cand ? 1u : 0u, wcnt, cap, sc);
    if (cand && pos != ~0u) {
        cidx[slice0 + pos] = i;
        cpt[slice0 + pos] = make_float2(x, y);
    }
}

// One sweep: eight running extremes per thread (per tile, the maxima of the
// thread's points and the first tile reaching a larger key; the point in
// it is found at the end), warp + block reduction, grid finish by packed
// atomicMax, last block decodes and (optionally) builds the polygon.
// zero_* ranges are cleared on the way for the next kernel of the same
// call.
//
// SPEC (the speculative single sweep): every point the sweep cannot place
// in the region A of the sample kernel (SpecBox) is written to the block's
// candidate segment; the last block checks exactly that A lies strictly
// inside the final octagon.  Then every other point is discarded by the
// filter, whose count and scatter passes test only the candidates
// (Octagon::spec).  A full segment or a failed check leaves spec = 0 and
// the filter runs its two passes over all points.
//
// learn (ch_hull_learned): one more block than the sweep's runs the learned
// proposal (mlp.cuh) beside it -- features, MLP and the choice of the second
// polygon, ready long before the kernels that read it.
template <bool SPEC>
__global__ void __launch_bounds__(kExtThreads, 2) extremes_kernel(const float *__restrict__ pts, int64_t n,
                                                                  void *ws, Layout L, uint32_t *ext8_out,
                                                                  int build_polygon, unsigned long long *zero_ptr,
                                                                  int64_t zero_words, uint32_t cap,
                                                                  const __nv_bfloat16 *learn, float *learn_dirs,
                                                                  int32_t *learn_k)
{
    static_assert(kExtThreads == mlp::LT, "the learned block has the sweep's block size");
    const uint32_t nsweep = gridDim.x - (learn ? 1u : 0u);   // blocks of the sweep
    if (learn && blockIdx.x == nsweep) {
        mlp::learned_choice_block(pts, n, learn, at<LearnScratch>(ws, L.learn), learn_dirs, learn_k);
        return;
    }
    ExtCtrl *ctrl = at<ExtCtrl>(ws, L.extctrl);
    // clear what the following kernels of this call expect to be zero
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)nsweep * blockDim.x;
    for (int64_t w = gtid; w < zero_words; w += gthreads) zero_ptr[w] = 0ull;

    bool nan_seen = false;
    // full tiles: this thread's largest key per slot and (in shared memory)
    // the first tile reaching it (NaN, -1: none yet)
    float bk[8];
    __shared__ int32_t s_btile[8][kExtThreads];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        bk[j] = __int_as_float(0x7fc00000);
        s_btile[j][threadIdx.x] = -1;
    }

    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    // speculative sweep state
    __shared__ SpecBox s_box;
    SpecCtrl *sc = at<SpecCtrl>(ws, L.spec);
    uint32_t *cidx = at<uint32_t>(ws, L.keys[1]);
    float2 *cpt = at<float2>(ws, L.pay[1]);
    bool spec_live = false;
    uint32_t wcnt = 0;   // slots in use of this warp's slice
    const size_t slice0 = ((size_t)blockIdx.x * kSpecWarps + warp) * cap;
    if constexpr (SPEC) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(at<SpecBox>(ws, L.p0));
        uint32_t *dst = reinterpret_cast<uint32_t *>(&s_box);
        for (uint32_t w = threadIdx.x; w < sizeof(SpecBox) / 4; w += blockDim.x) dst[w] = src[w];
        __syncthreads();
        spec_live = s_box.ok != 0;
    }
    const SpecBox &box = s_box;

    const uintptr_t addr = reinterpret_cast<uintptr_t>(pts);
    const int64_t head = (addr & 15u) ? 1 : 0;  // points before the 16-byte boundary
    const int64_t npairs = (n - head) / 2;
    const float4 *p4 = reinterpret_cast<const float4 *>(pts + 2 * head);
    // each block a contiguous range of tiles of kExtPairs point pairs; the
    // next tile streams into L2 while this one is reduced
    constexpr int U = kExtPairs / kExtThreads;
    const int64_t ntiles = ceil_div(npairs, (int64_t)kExtPairs);
    const int64_t per = ceil_div(ntiles, (int64_t)nsweep);
    const int64_t t1 = min(ntiles, (int64_t)(blockIdx.x + 1) * per);
    const int64_t nfull = npairs / kExtPairs;   // the ragged last tile is taken point by point below
    const int64_t t1f = min(t1, nfull);
    for (int64_t tile = (int64_t)blockIdx.x * per; tile < t1f; ++tile) {
        const int64_t q0 = tile * kExtPairs;
        if (threadIdx.x == 0 && tile + 1 < t1) {
            const int64_t nq = min((int64_t)kExtPairs, npairs - q0 - kExtPairs);
            bulk_prefetch_l2(p4 + q0 + kExtPairs, (uint32_t)(nq * 16));
        }
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = __ldcs(p4 + q0 + u * kExtThreads + threadIdx.x);
        // the tile's maxima of the eight keys over this thread's points
        float tb[8];
#pragma unroll
        for (int p = 0; p < 2 * U; ++p) {
            const float x = (p & 1) ? v[p >> 1].z : v[p >> 1].x, y = (p & 1) ? v[p >> 1].w : v[p >> 1].y;
            float k[8];
            slot_keys(x, y, k);
            if (p == 0) {
#pragma unroll
                for (int j = 0; j < 8; ++j) tb[j] = k[j];
            } else {
                tb[0] = max_nan(tb[0], k[0]);
                tb[2] = max_nan(tb[2], k[2]);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j != 0 && j != 2) tb[j] = fmaxf(tb[j], k[j]);
            }
        }
        nan_seen |= (tb[0] != tb[0]) | (tb[2] != tb[2]);
        // a larger key: remember the tile (the point is found at the end)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (!(tb[j] <= bk[j])) {
                bk[j] = tb[j];
                s_btile[j][threadIdx.x] = (int32_t)tile;
            }
        }
        if constexpr (SPEC) {
            if (spec_live) {
                // the points outside the region A: candidates
                uint32_t cand = 0;
#pragma unroll
                for (int p = 0; p < 2 * U; ++p) {
                    const float x = (p & 1) ? v[p >> 1].z : v[p >> 1].x, y = (p & 1) ? v[p >> 1].w : v[p >> 1].y;
                    cand |= (spec_inside(box, x, y, __fadd_rn(x, y), __fsub_rn(x, y)) ? 0u : 1u) << p;
                }
                if (__any_sync(0xffffffffu, cand != 0u)) {
                    spec_live = spec_still_live(wcnt, cap, sc);
                    if (spec_live) {
                        uint32_t pos = slice_reserve(__popc(cand), wcnt, cap, sc);
                        spec_live = pos != ~0u;
                        if (spec_live) {
#pragma unroll
                            for (int p = 0; p < 2 * U; ++p) {
                                if (!((cand >> p) & 1u)) continue;
                                const float x = (p & 1) ? v[p >> 1].z : v[p >> 1].x;
                                const float y = (p & 1) ? v[p >> 1].w : v[p >> 1].y;
                                cidx[slice0 + pos] =
                                    (uint32_t)(head + 2 * (q0 + (p >> 1) * kExtThreads + threadIdx.x) + (p & 1));
                                cpt[slice0 + pos] = make_float2(x, y);
                                ++pos;
                            }
                        }
                    }
                }
            }
        }
    }
    Best b;   // the ragged tile and the unpaired points, point by point
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        b.k[j] = __int_as_float(0x7fc00000);  // NaN: no candidate yet
        b.i[j] = 0xffffffffu;
    }
    if ((int64_t)blockIdx.x * per <= nfull && nfull < t1) {   // this block holds the ragged last tile
        const int64_t q0 = nfull * kExtPairs;
        for (int u = 0; u < U; ++u) {   // warp-uniform trips: the warps append together
            const int64_t q = q0 + u * kExtThreads + threadIdx.x;
            const bool valid = q < npairs;
            const float4 v = valid ? __ldcs(p4 + q) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            const uint32_t i0 = (uint32_t)(head + 2 * q);
            if (valid) {
                nan_seen |= (v.x != v.x) | (v.y != v.y) | (v.z != v.z) | (v.w != v.w);
                consider(b, v.x, v.y, i0);
                consider(b, v.z, v.w, i0 + 1);
            }
            if constexpr (SPEC) {
                if (spec_live) {
                    spec_warp_point(box, valid, i0, v.x, v.y, wcnt, cap, sc, cidx, cpt, slice0);
                    spec_warp_point(box, valid, i0 + 1, v.z, v.w, wcnt, cap, sc, cidx, cpt, slice0);
                }
            }
        }
    }
    // the point before the aligned body (warp 0 of block 0, whose segment
    // comes first) and the odd point after it (warp 0 of the last block,
    // whose segment comes last)
    if (blockIdx.x == 0 && warp == 0 && head) {
        const bool mine = lane == 0;
        const float x = pts[0], y = pts[1];
        if (mine) {
            nan_seen |= (x != x) | (y != y);
            consider(b, x, y, 0);
        }
        if constexpr (SPEC)
            if (spec_live) spec_warp_point(box, mine, 0, x, y, wcnt, cap, sc, cidx, cpt, slice0);
    }
    if (blockIdx.x == nsweep - 1 && warp == 0 && (n - head) % 2 == 1) {
        const bool mine = lane == 0;
        const int64_t i = n - 1;
        const float x = pts[2 * i], y = pts[2 * i + 1];
        if (mine) {
            nan_seen |= (x != x) | (y != y);
            consider(b, x, y, (uint32_t)i);
        }
        if constexpr (SPEC)
            if (spec_live) spec_warp_point(box, mine, (uint32_t)i, x, y, wcnt, cap, sc, cidx, cpt, slice0);
    }
    if constexpr (SPEC)
        if (lane == 0) sc->scnt[blockIdx.x * kSpecWarps + warp] = min(wcnt, cap);

    // the full tiles' winners: per slot, the lanes holding the warp's
    // largest key re-read their tile and take its first point with that key
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float m = bk[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const int32_t bt = s_btile[j][threadIdx.x];
        if (bt >= 0 && bk[j] == m) {
            const int64_t q0 = (int64_t)bt * kExtPairs;
            uint32_t idx = 0xffffffffu;
#pragma unroll
            for (int u = U - 1; u >= 0; --u) {   // backwards: the last match is the first point
                const float4 w = p4[q0 + u * kExtThreads + threadIdx.x];
                float k[8];
                slot_keys(w.z, w.w, k);
                if (k[j] == bk[j]) idx = (uint32_t)(head + 2 * (q0 + u * kExtThreads + threadIdx.x) + 1);
                slot_keys(w.x, w.y, k);
                if (k[j] == bk[j]) idx = (uint32_t)(head + 2 * (q0 + u * kExtThreads + threadIdx.x));
            }
            if (idx != 0xffffffffu) combine(b.k[j], b.i[j], bk[j], idx);
        }
    }
    // warp reduction
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float ok = __shfl_xor_sync(0xffffffffu, b.k[j], o);
            const uint32_t oi = __shfl_xor_sync(0xffffffffu, b.i[j], o);
            combine(b.k[j], b.i[j], ok, oi);
        }
    }
    __shared__ float sk[kExtThreads / 32][8];
    __shared__ uint32_t si[kExtThreads / 32][8];
    __shared__ int s_nonfinite;
    __shared__ bool s_last;
    if (threadIdx.x == 0) s_nonfinite = 0;
    __syncthreads();
    if (nan_seen) s_nonfinite = 1;
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            sk[warp][j] = b.k[j];
            si[warp][j] = b.i[j];
        }
    }
    __syncthreads();
    if (warp == 0) {
        // lane j < 8 folds slot j over the block's warps
        if (lane < 8) {
            float k = sk[0][lane];
            uint32_t i = si[0][lane];
            for (int w = 1; w < kExtThreads / 32; ++w) combine(k, i, sk[w][lane], si[w][lane]);
            if (i != 0xffffffffu) {
                const unsigned long long packed = ((unsigned long long)ord_key(k) << 32) | (uint32_t)~i;
                atomicMax(&ctrl->ext_slot[lane], packed);
            }
        }
        if (lane == 0 && s_nonfinite) atomicOr(&ctrl->nonfinite, 1u);
        __threadfence();
        __syncwarp();
        if (lane == 0) s_last = atomicAdd(&ctrl->ext_done, 1u) == nsweep - 1;
    }
    __syncthreads();
    if (!s_last || warp != 0) return;

    // last block: decode, reset the slots for the next call, build polygon
    __threadfence();
    __shared__ uint32_t s_ext[8];
    if (lane < 8) {
        const unsigned long long packed = atomicExch(&ctrl->ext_slot[lane], 0ull);
        const uint32_t idx = ~(uint32_t)packed;
        s_ext[lane] = idx;
        ext8_out[lane] = idx;
    }
    uint32_t bad = lane == 0 ? atomicExch(&ctrl->nonfinite, 0u) : 0u;
    if (lane == 0) ctrl->ext_done = 0;
    __syncwarp();
    // an infinite coordinate makes an infinite R, T, L or B vertex (a slot
    // left without a point means its keys were all NaN, already flagged)
    if (lane < 4 && (int64_t)s_ext[2 * lane] < n) {
        const float c = pts[2 * (size_t)s_ext[2 * lane] + (lane & 1)];
        if (!(fabsf(c) <= 3.402823466e38f)) bad = 1u;
    }
    const bool nonfinite = __any_sync(0xffffffffu, bad != 0u);
    Octagon *oct = at<Octagon>(ws, L.oct);
    if (nonfinite) {
        if (lane == 0) {
            set_error(ws, L, kErrNonFinite, 1);
            if (build_polygon) oct->abort = 1;
        }
        return;
    }
    if (build_polygon) build_octagon_warp(reinterpret_cast<const float2 *>(pts), s_ext, oct, true);
    if constexpr (SPEC) {
        // A strictly inside P: every vertex of A strictly left of every
        // valid edge of P (exact signs); no full segment; P has an edge
        __syncwarp();
        const uint32_t vk = lane & 7u;
        bool ok = true;
        for (uint32_t e = lane >> 3; e < 8; e += 4)
            if ((oct->valid >> e) & 1u)
                ok = ok && orient(oct->ax[e], oct->ay[e], oct->bx[e], oct->by[e], box.vx[vk], box.vy[vk]) > 0;
        ok = __all_sync(0xffffffffu, ok);
        if (lane == 0)
            oct->spec = (ok && build_polygon && oct->has_edges && box.ok && ld_relaxed_u32(&sc->fail) == 0u) ? 1u : 0u;
    }
}

// The region A of the speculative sweep, from the eight key extremes of
// kSampleBlocks evenly spaced runs of kSampleRun points (the sample's
// bounding octagon), each bound moved towards the centre of the sample's
// box by the factor kP0Shrink, snapped inwards to multiples of g, the
// diagonal bounds clamped so that each cuts only its corner of the box
// (then A's vertices, computed below, are its corners in order).  Bounds
// and vertices are multiples of g, at most 2M in size with M = max|x| +
// max|y| over the box and g >= 2^-21 M, so they are exact in binary32.
// A usable region needs a box of non-zero size and vertices in order.
constexpr int kSampleBlocks = 32;
constexpr int kSampleThreads = 256;
constexpr int kSampleRun = kSampleThreads * 8;
constexpr double kP0Shrink = 0.9;
constexpr int kSpecProbe = 1024;   // points tested against A before the sweep

__device__ void build_spec_box(const float (&kmax)[8], SpecBox *out)
{
    // kmax in slot order: max x, max s, max y, max -d, max -x, max -s, max -y, max d
    double xh = kmax[0], sh = kmax[1], yh = kmax[2], dl = -(double)kmax[3];
    double xl = -(double)kmax[4], sl = -(double)kmax[5], yl = -(double)kmax[6], dh = kmax[7];
    SpecBox b{};
    b.ok = 0;
    const double M = fmax(fabs(xl), fabs(xh)) + fmax(fabs(yl), fabs(yh));
    bool ok = xl < xh && yl < yh && M < 1e37 && M > 1e-30;
    if (ok) {
        const double cx = 0.5 * (xl + xh), cy = 0.5 * (yl + yh), cs = cx + cy, cd = cx - cy;
        const double f = kP0Shrink;
        xh = cx + f * (xh - cx);
        xl = cx + f * (xl - cx);
        yh = cy + f * (yh - cy);
        yl = cy + f * (yl - cy);
        sh = cs + f * (sh - cs);
        sl = cs + f * (sl - cs);
        dh = cd + f * (dh - cd);
        dl = cd + f * (dl - cd);
        // grid: the smallest power of two >= 2^-21 M
        int ge = 0;
        frexp(M * 0x1p-21, &ge);   // M 2^-21 < 2^ge
        const double g = ldexp(1.0, ge);
        xh = floor(xh / g) * g;
        yh = floor(yh / g) * g;
        sh = floor(sh / g) * g;
        dh = floor(dh / g) * g;
        xl = ceil(xl / g) * g;
        yl = ceil(yl / g) * g;
        sl = ceil(sl / g) * g;
        dl = ceil(dl / g) * g;
        // each diagonal cuts its corner of the box, within the box's edges
        sh = fmax(fmin(sh, xh + yh), fmax(xh + yl, xl + yh));
        sl = fmin(fmax(sl, xl + yl), fmin(xh + yl, xl + yh));
        dh = fmax(fmin(dh, xh - yl), fmax(xh - yh, xl - yl));
        dl = fmin(fmax(dl, xl - yh), fmin(xh - yh, xl - yl));
        const double vx[8] = {xh, sh - yh, dl + yh, xl, xl, sl - yl, dh + yl, xh};
        const double vy[8] = {sh - xh, yh, yh, xl - dl, sl - xl, yl, yl, xh - dh};
        // in order around the box: right, top, left, bottom edges not inverted
        ok = xl < xh && yl < yh && vy[7] <= vy[0] && vx[2] <= vx[1] && vy[4] <= vy[3] && vx[5] <= vx[6];
        // the test's diagonal bounds, moved in by m = 2^-23 M' (M' = |x| + |y|
        // bound inside the snapped box), rounded inwards
        const double Mb = fmax(fabs(xl), fabs(xh)) + fmax(fabs(yl), fabs(yh));
        const double m = Mb * 0x1p-23;
        b.xl = (float)xl;
        b.xh = (float)xh;
        b.yl = (float)yl;
        b.yh = (float)yh;
        b.slb = __double2float_ru(sl + m);
        b.shb = __double2float_rd(sh - m);
        b.dlb = __double2float_ru(dl + m);
        b.dhb = __double2float_rd(dh - m);
        ok = ok && b.slb <= b.shb && b.dlb <= b.dhb;
        for (int k = 0; k < 8; ++k) {
            b.vx[k] = (float)vx[k];
            b.vy[k] = (float)vy[k];
        }
    }
    b.ok = ok ? 1u : 0u;
    *out = b;
}

__global__ void __launch_bounds__(kSampleThreads) spec_sample_kernel(const float *__restrict__ pts, int64_t n, void *ws,
                                                                     Layout L, uint32_t nseg, uint32_t cap)
{
    SpecCtrl *sc = at<SpecCtrl>(ws, L.spec);
    const float2 *p2 = reinterpret_cast<const float2 *>(pts);
    const int64_t start = (n - kSampleRun) * (int64_t)blockIdx.x / (gridDim.x - 1);
    float km[8];
    float2 pv[kSampleRun / kSampleThreads];
#pragma unroll
    for (int r = 0; r < kSampleRun / kSampleThreads; ++r) pv[r] = __ldg(p2 + start + r * kSampleThreads + threadIdx.x);
#pragma unroll
    for (int r = 0; r < kSampleRun / kSampleThreads; ++r) {
        float k[8];
        slot_keys(pv[r].x, pv[r].y, k);
#pragma unroll
        for (int j = 0; j < 8; ++j) km[j] = r == 0 ? k[j] : fmaxf(km[j], k[j]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int j = 0; j < 8; ++j) km[j] = fmaxf(km[j], __shfl_xor_sync(0xffffffffu, km[j], o));
    __shared__ float s_km[kSampleThreads / 32][8];
    __shared__ bool s_last;
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < 8; ++j) s_km[warp][j] = km[j];
    __syncthreads();
    if (warp != 0) return;
    if (lane < 8) {
        float m = s_km[0][lane];
        for (int w = 1; w < kSampleThreads / 32; ++w) m = fmaxf(m, s_km[w][lane]);
        atomicMax(&sc->kmax[lane], ord_key(m));
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) s_last = atomicAdd(&sc->sample_done, 1u) == gridDim.x - 1;
    __syncwarp();
    if (!s_last) return;
    __threadfence();
    __shared__ SpecBox s_box;
    if (lane == 0) {
        float kmax[8];
        for (int j = 0; j < 8; ++j) kmax[j] = key_float(atomicExch(&sc->kmax[j], 0u));
        sc->sample_done = 0u;
        sc->fail = 0u;
        sc->nseg = nseg;
        sc->cap = cap;
        build_spec_box(kmax, &s_box);
    }
    __syncwarp();
    // the share of kSpecProbe evenly spaced points outside A predicts the
    // candidates' share: above half the segments' capacity (1 / kSpecCapDiv
    // of the points) the sweep would most likely overflow them, so it does
    // not speculate (either way the outcome is checked, not assumed)
    uint32_t out = 0;
    if (s_box.ok) {
        const int64_t stride = n / kSpecProbe;
        for (int k = (int)lane; k < kSpecProbe; k += 32) {
            const float2 v = __ldg(p2 + (int64_t)k * stride);
            out += spec_inside(s_box, v.x, v.y, __fadd_rn(v.x, v.y), __fsub_rn(v.x, v.y)) ? 0u : 1u;
        }
    }
    out = __reduce_add_sync(0xffffffffu, out);
    if (lane == 0) {
        SpecBox b = s_box;
        if (2u * kSpecCapDiv * out > (uint32_t)kSpecProbe) b.ok = 0u;
        *at<SpecBox>(ws, L.p0) = b;
    }
}

// Polygon construction for a caller-supplied ext8 (ch_filter); also clears
// the control block and the look-back status of the filter.  An index
// >= n is reported as CH_ERR_ARG and the filter then does nothing.
__global__ void octagon_kernel(const float *__restrict__ pts, int64_t n, const uint32_t *ext8, void *ws,
                               Layout L, unsigned long long *zero_ptr, int64_t zero_words)
{
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = gtid; w < zero_words; w += gthreads) zero_ptr[w] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        __shared__ uint32_t s_ext[8];
        const uint32_t lane = lane_id();
        const uint32_t e = lane < 8 ? ext8[lane] : 0u;
        const bool bad = __any_sync(0xffffffffu, lane < 8 && (int64_t)e >= n);
        Octagon *oct = at<Octagon>(ws, L.oct);
        if (bad) {
            if (lane == 0) {
                set_error(ws, L, CH_ERR_ARG, 2);
                oct->abort = 1;
            }
            return;
        }
        if (lane < 8) s_ext[lane] = e;
        __syncwarp();
        build_octagon_warp(reinterpret_cast<const float2 *>(pts), s_ext, oct, false);
    }
}

// ---------------------------------------------------------------------------
// many sets (ch_hull_batched): the same reduction per 4096-point tile of one
// set, finished with per-set packed atomics; then one warp per set builds
// its polygon.  Indices are set-local.
// ---------------------------------------------------------------------------
// Each block takes a contiguous range of tiles; the running extremes are
// folded into the set's slots whenever the range moves on to another set
// (sets are contiguous in tile order, so a block flushes once per set it
// touches).
template <int NWARP>
__device__ __forceinline__ void bx_flush(Best &best, float &nf, int64_t b, unsigned long long *slots,
                                         uint32_t *nonfin, float (&sk)[NWARP][8], uint32_t (&si)[NWARP][8], int &s_bad)
{
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float ok = __shfl_xor_sync(0xffffffffu, best.k[j], o);
            const uint32_t oi = __shfl_xor_sync(0xffffffffu, best.i[j], o);
            combine(best.k[j], best.i[j], ok, oi);
        }
    }
    __syncthreads();   // sk, si and s_bad of the previous flush have been read
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    if (nf != nf) s_bad = 1;
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            sk[warp][j] = best.k[j];
            si[warp][j] = best.i[j];
        }
    __syncthreads();
    if (warp == 0 && lane < 8) {
        float k = sk[0][lane];
        uint32_t i = si[0][lane];
        for (int w = 1; w < NWARP; ++w) combine(k, i, sk[w][lane], si[w][lane]);
        if (i != 0xffffffffu)
            atomicMax(&slots[(size_t)b * 8 + lane], ((unsigned long long)ord_key(k) << 32) | (uint32_t)~i);
        if (lane == 0 && s_bad) atomicOr(&nonfin[b], 1u);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        best.k[j] = __int_as_float(0x7fc00000);
        best.i[j] = 0xffffffffu;
    }
    nf = 0.0f;
}

template <int T>   // threads per block: each holds kFiltTile / T points of a tile
__global__ void __launch_bounds__(T) bx_extremes_kernel(const float *__restrict__ pts, void *ws, Layout L,
                                                        BatchLayout BL)
{
    const BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    if (bc->abort) return;
    const SetInfo *sets = at<SetInfo>(ws, BL.sets);
    const uint32_t *tile_set = at<uint32_t>(ws, BL.tile_set);
    unsigned long long *slots = at<unsigned long long>(ws, BL.ext_slot);
    uint32_t *nonfin = at<uint32_t>(ws, BL.nonfinite);
    __shared__ float sk[T / 32][8];
    __shared__ uint32_t si_[T / 32][8];
    __shared__ int s_bad;
    const int64_t NT = bc->tiles;
    const int64_t per = ceil_div(NT, (int64_t)gridDim.x);
    const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(NT, t0 + per);
    constexpr int R = kFiltTile / T;   // points per thread per tile
    Best best;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        best.k[j] = __int_as_float(0x7fc00000);
        best.i[j] = 0xffffffffu;
    }
    float nf = 0.0f;
    int64_t cur = -1;
    for (int64_t t = t0; t < t1; ++t) {
        const int64_t b = tile_set[t];   // block-uniform
        if (b != cur) {
            if (cur >= 0) bx_flush(best, nf, cur, slots, nonfin, sk, si_, s_bad);
            cur = b;
        }
        const int64_t lo = (t - sets[b].tile_base) * (int64_t)kFiltTile;
        const int64_t hi = min(lo + kFiltTile, sets[b].n);
        const float2 *p2 = reinterpret_cast<const float2 *>(pts) + sets[b].pt_begin;
        if (threadIdx.x == 0 && t + 1 < t1) {   // the next tile streams into L2 meanwhile
            const int64_t nb = tile_set[t + 1];
            const int64_t nlo = (t + 1 - sets[nb].tile_base) * (int64_t)kFiltTile;
            const int64_t nhi = min(nlo + kFiltTile, sets[nb].n);
            const float2 *np = reinterpret_cast<const float2 *>(pts) + sets[nb].pt_begin;
            const uintptr_t a0 = (reinterpret_cast<uintptr_t>(np + nlo) + 15) & ~(uintptr_t)15;
            const uintptr_t a1 = reinterpret_cast<uintptr_t>(np + nhi) & ~(uintptr_t)15;
            if (a1 > a0) bulk_prefetch_l2(reinterpret_cast<const void *>(a0), (uint32_t)(a1 - a0));
        }
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t i = lo + r * T + threadIdx.x;
            v[r] = i < hi ? __ldcs(p2 + i) : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t i = lo + r * T + threadIdx.x;
            if (i < hi) {
                nf = __fmaf_rn(v[r].x, 0.0f, __fmaf_rn(v[r].y, 0.0f, nf));
                consider(best, v[r].x, v[r].y, (uint32_t)i);
            }
        }
    }
    if (cur >= 0) bx_flush(best, nf, cur, slots, nonfin, sk, si_, s_bad);
}

__global__ void __launch_bounds__(256) bx_octagon_kernel(const float *__restrict__ pts, void *ws, Layout L,
                                                         BatchLayout BL)
{
    const BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    const SetInfo *sets = at<SetInfo>(ws, BL.sets);
    const unsigned long long *slots = at<unsigned long long>(ws, BL.ext_slot);
    const uint32_t *nonfin = at<uint32_t>(ws, BL.nonfinite);
    Octagon *octs = at<Octagon>(ws, BL.octs);
    __shared__ uint32_t s_ext[8][8];
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    const int64_t b = (int64_t)blockIdx.x * 8 + warp;
    if (b >= BL.num_sets) return;
    Octagon *out = octs + b;
    if (bc->abort || sets[b].n == 0) {   // nothing to do: empty hull
        if (lane == 0) out->abort = 1;
        return;
    }
    if (nonfin[b]) {
        if (lane == 0) {
            out->abort = 1;
            set_error(ws, L, kErrNonFinite, 3);
        }
        return;
    }
    if (lane < 8) s_ext[warp][lane] = ~(uint32_t)slots[b * 8 + lane];
    __syncwarp();
    build_octagon_warp(reinterpret_cast<const float2 *>(pts) + sets[b].pt_begin, s_ext[warp], out, true);
}

cudaError_t launch_bx_extremes(const float *pts, void *ws, const Layout &L, const BatchLayout &BL, cudaStream_t st)
{
    const int per_sm = tune_value(CH_TUNE_BX_EXTREMES) ? tune_value(CH_TUNE_BX_EXTREMES) : 8;
    const int items = tune_value(CH_TUNE_BX_EXT_ITEMS) ? tune_value(CH_TUNE_BX_EXT_ITEMS) : 16;
    int64_t blocks = std::min<int64_t>(BL.tiles_max, (int64_t)sm_count() * per_sm);
    const unsigned g = (unsigned)std::max<int64_t>(blocks, 1);
    probe_before(CH_K_EXTREMES, st);
    if (items == 4) bx_extremes_kernel<1024><<<g, 1024, 0, st>>>(pts, ws, L, BL);
    else if (items == 8) bx_extremes_kernel<512><<<g, 512, 0, st>>>(pts, ws, L, BL);
    else bx_extremes_kernel<256><<<g, 256, 0, st>>>(pts, ws, L, BL);
    bx_octagon_kernel<<<(unsigned)ceil_div(BL.num_sets, 8), 256, 0, st>>>(pts, ws, L, BL);
    note_kernels(CH_K_EXTREMES, 2);
    probe_after(CH_K_EXTREMES, st);
    return cudaGetLastError();
}

int sm_count()
{
    static std::atomic<int> cached[64] = {};   // per device; several host threads may fill it
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int c = cached[dev].load(std::memory_order_relaxed);
    if (!c) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        c = v > 0 ? v : 1;
        cached[dev].store(c, std::memory_order_relaxed);
    }
    return c;
}

namespace {

template <bool SPEC>
int extremes_per_sm()
{
    static const int v = [] {
        int r = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, extremes_kernel<SPEC>, kExtThreads, 0);
        return r > 0 ? r : 1;
    }();
    return v;
}

}  // namespace

cudaError_t launch_extremes(const float *pts, int64_t n, void *ws, const Layout &L, uint32_t *ext8,
                            bool build_polygon, unsigned long long *zero_ptr, int64_t zero_words,
                            cudaStream_t st, bool spec, const void *learn_params, float *learn_dirs,
                            int32_t *learn_k)
{
    const __nv_bfloat16 *learn = static_cast<const __nv_bfloat16 *>(learn_params);
    const unsigned extra = learn ? 1u : 0u;
    const int64_t pairs = (n + 1) / 2;
    const int64_t tiles = ceil_div(pairs, (int64_t)kExtPairs);
    // the speculative sweep: large sets only, one candidate segment per
    // block inside the second sort buffers
    if (spec && build_polygon && n >= kSpecMinN) {
        // one wave with the learned block: it must not wait for a slot
        int64_t blocks = std::min<int64_t>(tiles, (int64_t)sm_count() * extremes_per_sm<true>() - extra);
        if (blocks < 1) blocks = 1;
        const int64_t cap = n / kSpecCapDiv / (blocks * kSpecWarps);   // candidate slots per warp slice
        if (blocks <= kSpecMaxSeg && cap >= 16) {
            probe_before(CH_K_EXTREMES, st);
            spec_sample_kernel<<<kSampleBlocks, kSampleThreads, 0, st>>>(pts, n, ws, L, (uint32_t)blocks,
                                                                         (uint32_t)cap);
            extremes_kernel<true><<<(unsigned)blocks + extra, kExtThreads, 0, st>>>(pts, n, ws, L, ext8, 1, zero_ptr,
                                                                                   zero_words, (uint32_t)cap, learn,
                                                                                   learn_dirs, learn_k);
            note_kernels(CH_K_EXTREMES, 2);
            probe_after(CH_K_EXTREMES, st);
            return cudaGetLastError();
        }
    }
    int64_t blocks = tiles;   // one wave: every block (and the learned one) resident
    const int64_t cap = (int64_t)sm_count() * extremes_per_sm<false>() - extra;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    probe_before(CH_K_EXTREMES, st);
    extremes_kernel<false><<<(unsigned)blocks + extra, kExtThreads, 0, st>>>(pts, n, ws, L, ext8, build_polygon ? 1 : 0,
                                                                             zero_ptr, zero_words, 0u, learn,
                                                                             learn_dirs, learn_k);
    note_kernels(CH_K_EXTREMES, 1);
    probe_after(CH_K_EXTREMES, st);
    return cudaGetLastError();
}

cudaError_t launch_octagon(const float *pts, int64_t n, const uint32_t *ext8, void *ws, const Layout &L,
                           unsigned long long *zero_ptr, int64_t zero_words, cudaStream_t st)
{
    int64_t blocks = ceil_div(zero_words, 256 * 4);
    const int64_t cap = (int64_t)sm_count() * 2;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    probe_before(CH_K_OCTAGON, st);
    octagon_kernel<<<(unsigned)blocks, 256, 0, st>>>(pts, n, ext8, ws, L, zero_ptr, zero_words);
    note_kernels(CH_K_OCTAGON, 1);
    probe_after(CH_K_OCTAGON, st);
    return cudaGetLastError();
}

}  // namespace ch

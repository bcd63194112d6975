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
    }
}

// One sweep: eight running extremes per thread, warp + block reduction,
// grid finish by packed atomicMax, last block decodes and (optionally)
// builds the polygon.  zero_* ranges are cleared on the way for the next
// kernel of the same call.
__global__ void __launch_bounds__(kExtThreads) extremes_kernel(const float *__restrict__ pts, int64_t n,
                                                               void *ws, Layout L, uint32_t *ext8_out,
                                                               int build_polygon, unsigned long long *zero_ptr,
                                                               int64_t zero_words)
{
    ExtCtrl *ctrl = at<ExtCtrl>(ws, L.extctrl);
    // clear what the following kernels of this call expect to be zero
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = gtid; w < zero_words; w += gthreads) zero_ptr[w] = 0ull;

    Best b;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        b.k[j] = __int_as_float(0x7fc00000);  // NaN: no candidate yet
        b.i[j] = 0xffffffffu;
    }
    float nf = 0.0f;   // becomes NaN iff some coordinate is NaN or infinite

    const uintptr_t addr = reinterpret_cast<uintptr_t>(pts);
    const int64_t head = (addr & 15u) ? 1 : 0;  // points before the 16-byte boundary
    const int64_t npairs = (n - head) / 2;
    const float4 *p4 = reinterpret_cast<const float4 *>(pts + 2 * head);
    // each block a contiguous range of tiles of kExtPairs point pairs; the
    // next tile streams into L2 while this one is reduced
    constexpr int U = kExtPairs / kExtThreads;
    const int64_t ntiles = ceil_div(npairs, (int64_t)kExtPairs);
    const int64_t per = ceil_div(ntiles, (int64_t)gridDim.x);
    const int64_t t1 = min(ntiles, (int64_t)(blockIdx.x + 1) * per);
    for (int64_t tile = (int64_t)blockIdx.x * per; tile < t1; ++tile) {
        const int64_t q0 = tile * kExtPairs;
        if (threadIdx.x == 0 && tile + 1 < t1) {
            const int64_t nq = min((int64_t)kExtPairs, npairs - q0 - kExtPairs);
            bulk_prefetch_l2(p4 + q0 + kExtPairs, (uint32_t)(nq * 16));
        }
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t q = q0 + u * kExtThreads + threadIdx.x;
            v[u] = q < npairs ? __ldcs(p4 + q) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t q = q0 + u * kExtThreads + threadIdx.x;
            if (q < npairs) {
                const uint32_t i0 = (uint32_t)(head + 2 * q);
                nf = __fmaf_rn(v[u].x, 0.0f, nf);
                nf = __fmaf_rn(v[u].y, 0.0f, nf);
                nf = __fmaf_rn(v[u].z, 0.0f, nf);
                nf = __fmaf_rn(v[u].w, 0.0f, nf);
                consider(b, v[u].x, v[u].y, i0);
                consider(b, v[u].z, v[u].w, i0 + 1);
            }
        }
    }
    // the point before the aligned body and the odd point after it
    if (gtid == 0 && head) {
        const float x = pts[0], y = pts[1];
        nf = __fmaf_rn(x, 0.0f, __fmaf_rn(y, 0.0f, nf));
        consider(b, x, y, 0);
    }
    if (gtid == 1 % gthreads && (n - head) % 2 == 1) {
        const int64_t i = n - 1;
        const float x = pts[2 * i], y = pts[2 * i + 1];
        nf = __fmaf_rn(x, 0.0f, __fmaf_rn(y, 0.0f, nf));
        consider(b, x, y, (uint32_t)i);
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
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    if (nf != nf) s_nonfinite = 1;
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
        if (lane == 0) s_last = atomicAdd(&ctrl->ext_done, 1u) == gridDim.x - 1;
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
    const uint32_t bad = lane == 0 ? atomicExch(&ctrl->nonfinite, 0u) : 0u;
    if (lane == 0) ctrl->ext_done = 0;
    const bool nonfinite = __shfl_sync(0xffffffffu, bad, 0) != 0;
    __syncwarp();
    Octagon *oct = at<Octagon>(ws, L.oct);
    if (nonfinite) {
        if (lane == 0) {
            set_error(ws, L, kErrNonFinite, 1);
            if (build_polygon) oct->abort = 1;
        }
        return;
    }
    if (build_polygon) build_octagon_warp(reinterpret_cast<const float2 *>(pts), s_ext, oct, true);
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
__global__ void __launch_bounds__(256) bx_extremes_kernel(const float *__restrict__ pts, void *ws, Layout L,
                                                          BatchLayout BL)
{
    const BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    if (bc->abort) return;
    const SetInfo *sets = at<SetInfo>(ws, BL.sets);
    const uint32_t *tile_set = at<uint32_t>(ws, BL.tile_set);
    unsigned long long *slots = at<unsigned long long>(ws, BL.ext_slot);
    uint32_t *nonfin = at<uint32_t>(ws, BL.nonfinite);
    __shared__ float sk[8][8];
    __shared__ uint32_t si_[8][8];
    __shared__ int s_bad;
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    const uint32_t T = bc->tiles;
    for (uint32_t t = blockIdx.x; t < T; t += gridDim.x) {
        const uint32_t b = tile_set[t];
        const int64_t lo = (int64_t)(t - sets[b].tile_base) * kFiltTile;
        const int64_t hi = min(lo + kFiltTile, sets[b].n);
        const float2 *p2 = reinterpret_cast<const float2 *>(pts) + sets[b].pt_begin;
        Best best;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            best.k[j] = __int_as_float(0x7fc00000);
            best.i[j] = 0xffffffffu;
        }
        float nf = 0.0f;
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const float2 v = __ldcs(p2 + i);
            nf = __fmaf_rn(v.x, 0.0f, __fmaf_rn(v.y, 0.0f, nf));
            consider(best, v.x, v.y, (uint32_t)i);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float ok = __shfl_xor_sync(0xffffffffu, best.k[j], o);
                const uint32_t oi = __shfl_xor_sync(0xffffffffu, best.i[j], o);
                combine(best.k[j], best.i[j], ok, oi);
            }
        }
        if (threadIdx.x == 0) s_bad = 0;
        __syncthreads();
        if (nf != nf) s_bad = 1;
        if (lane == 0)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                sk[warp][j] = best.k[j];
                si_[warp][j] = best.i[j];
            }
        __syncthreads();
        if (warp == 0 && lane < 8) {
            float k = sk[0][lane];
            uint32_t i = si_[0][lane];
            for (int w = 1; w < 8; ++w) combine(k, i, sk[w][lane], si_[w][lane]);
            if (i != 0xffffffffu)
                atomicMax(&slots[(size_t)b * 8 + lane], ((unsigned long long)ord_key(k) << 32) | (uint32_t)~i);
            if (lane == 0 && s_bad) atomicOr(&nonfin[b], 1u);
        }
        __syncthreads();
    }
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
    int64_t blocks = std::min<int64_t>(BL.tiles_max, (int64_t)sm_count() * per_sm);
    probe_before(CH_K_EXTREMES, st);
    bx_extremes_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(pts, ws, L, BL);
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

cudaError_t launch_extremes(const float *pts, int64_t n, void *ws, const Layout &L, uint32_t *ext8,
                            bool build_polygon, unsigned long long *zero_ptr, int64_t zero_words,
                            cudaStream_t st)
{
    static int per_sm = [] {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, extremes_kernel, kExtThreads, 0);
        return v > 0 ? v : 1;
    }();
    const int64_t pairs = (n + 1) / 2;
    int64_t blocks = ceil_div(pairs, (int64_t)kExtPairs);   // one wave: every block resident
    const int64_t cap = (int64_t)sm_count() * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    probe_before(CH_K_EXTREMES, st);
    extremes_kernel<<<(unsigned)blocks, kExtThreads, 0, st>>>(pts, n, ws, L, ext8, build_polygon ? 1 : 0,
                                                              zero_ptr, zero_words);
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

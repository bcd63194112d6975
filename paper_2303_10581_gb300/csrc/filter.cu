// filter.cu -- Sec. 3.2 of Carrasco et al.: buildingFilter (is a point
// strictly inside the eight-vertex polygon?) fused with
// compactingFilteredPoints (stable compaction of the kept points).
//
// The paper writes an n-entry flag vector, scans it (tensor-core segmented
// scan, Thrust or CUB) and scatters.  Here one persistent kernel does it in
// a single read of the points: each block takes 4096-point tiles in ticket
// order, tests them, counts the kept points per (row, warp) with ballots,
// publishes the tile count, obtains the tile's output offset with a
// decoupled look-back, and writes the kept points in ascending index
// order.  Flags never reach memory.  Memory traffic: 8 bytes per point read,
// 12 bytes per kept point written.
#include "common.cuh"
#include "launch.h"

namespace ch {

namespace {

// keep(p) <=> NOT (p strictly left of every valid edge); see
// build_octagon_warp for the error bound of the binary32 test.  The first
// edge tried is the one facing p's octant around the box centre, which
// settles points outside the polygon after one test; the order does not
// change the result.
__device__ __forceinline__ bool keep_point(const Octagon &o, float x, float y)
{
    if (x >= o.xl && x <= o.xh && y >= o.yl && y <= o.yh) return false;
    if (!o.has_edges) return true;
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

// G points per thread per row (2 with 16-byte vector loads, 1 with 8-byte).
template <int G, bool KEYS>
__global__ void __launch_bounds__(kFiltThreads) filter_kernel(const float *__restrict__ pts, int64_t n,
                                                              void *ws, Layout L, uint32_t *__restrict__ surv_idx,
                                                              float2 *__restrict__ surv_pts,
                                                              uint32_t *__restrict__ surv_count)
{
    constexpr int ROWS = kFiltItems / G;
    constexpr int NW = kFiltThreads / 32;
    __shared__ Octagon so;
    __shared__ uint32_t s_off[ROWS][NW];
    __shared__ uint32_t s_tile;
    __shared__ unsigned long long s_excl;
    __shared__ uint32_t s_total;

    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    unsigned long long *status = at<unsigned long long>(ws, L.filt_status);
    uint32_t *out_keys = at<uint32_t>(ws, L.keys[0]);
    unsigned long long *out_pay = at<unsigned long long>(ws, L.pay[0]);

    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(at<Octagon>(ws, L.oct));
        uint32_t *dst = reinterpret_cast<uint32_t *>(&so);
        for (uint32_t w = threadIdx.x; w < sizeof(Octagon) / 4; w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    if (so.abort) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (KEYS) ctrl->surv_count = 0;
            else if (surv_count) *surv_count = 0;
        }
        return;
    }

    const int64_t ntiles = ceil_div(n, kFiltTile);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    const uint32_t lt = (1u << lane) - 1u;

    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&ctrl->filt_ticket, 1u);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= ntiles) break;
        const int64_t base = tile * kFiltTile;

        float px[ROWS * G], py[ROWS * G];
        uint32_t keep = 0;
        if (base + kFiltTile <= n) {
            if constexpr (G == 2) {
                const float4 *p4 = reinterpret_cast<const float4 *>(pts) + base / 2;
                float4 v[ROWS];
#pragma unroll
                for (int r = 0; r < ROWS; ++r) v[r] = __ldcs(p4 + r * kFiltThreads + tid);
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    px[r * G] = v[r].x;
                    py[r * G] = v[r].y;
                    px[r * G + G - 1] = v[r].z;
                    py[r * G + G - 1] = v[r].w;
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
#pragma unroll
            for (int q = 0; q < ROWS * G; ++q)
                if (keep_point(so, px[q], py[q])) keep |= 1u << q;
        } else {
            const float2 *p2 = reinterpret_cast<const float2 *>(pts);
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
#pragma unroll
                for (int h = 0; h < G; ++h) {
                    const int64_t i = base + (int64_t)(r * kFiltThreads + tid) * G + h;
                    if (i < n) {
                        const float2 v = p2[i];
                        px[r * G + h] = v.x;
                        py[r * G + h] = v.y;
                        if (keep_point(so, v.x, v.y)) keep |= 1u << (r * G + h);
                    } else {
                        px[r * G + h] = 0.0f;
                        py[r * G + h] = 0.0f;
                    }
                }
            }
        }

        // counts per (row, warp)
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            uint32_t c = 0;
#pragma unroll
            for (int h = 0; h < G; ++h) c += __popc(__ballot_sync(0xffffffffu, (keep >> (r * G + h)) & 1u));
            if (lane == 0) s_off[r][warp] = c;
        }
        __syncthreads();
        if (warp == 0) {
            // exclusive scan over (row, warp) in row-major order
            constexpr int PER = ROWS * NW / 32;
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
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            // publish, look back, publish the inclusive prefix
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
                if (tile == ntiles - 1) {
                    if (KEYS) ctrl->surv_count = (uint32_t)(excl + total);
                    else *surv_count = (uint32_t)(excl + total);
                }
            }
        }
        __syncthreads();
        if (s_total != 0) {
            const unsigned long long excl = s_excl;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                uint32_t pre = s_off[r][warp];
                uint32_t b[G];
#pragma unroll
                for (int h = 0; h < G; ++h) {
                    b[h] = __ballot_sync(0xffffffffu, (keep >> (r * G + h)) & 1u);
                    pre += __popc(b[h] & lt);
                }
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
        __syncthreads();
    }
}

template <int G, bool KEYS>
int blocks_per_sm()
{
    static int cached = 0;
    if (!cached) {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, filter_kernel<G, KEYS>, kFiltThreads, 0);
        cached = v > 0 ? v : 1;
    }
    return cached;
}

template <int G, bool KEYS>
cudaError_t launch_t(const float *pts, int64_t n, void *ws, const Layout &L, uint32_t *surv_idx, float *surv_pts,
                     uint32_t *surv_count, cudaStream_t st)
{
    const int64_t ntiles = ceil_div(n, kFiltTile);
    int64_t blocks = (int64_t)sm_count() * blocks_per_sm<G, KEYS>();
    if (blocks > ntiles) blocks = ntiles;
    if (blocks < 1) blocks = 1;
    probe_before(CH_K_FILTER, st);
    filter_kernel<G, KEYS><<<(unsigned)blocks, kFiltThreads, 0, st>>>(
        pts, n, ws, L, surv_idx, reinterpret_cast<float2 *>(surv_pts), surv_count);
    probe_after(CH_K_FILTER, st);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_filter(const float *pts, int64_t n, void *ws, const Layout &L, uint32_t *surv_idx,
                          float *surv_pts, uint32_t *surv_count, bool keys_mode, cudaStream_t st)
{
    const bool vec = (reinterpret_cast<uintptr_t>(pts) & 15u) == 0;
    if (keys_mode)
        return vec ? launch_t<2, true>(pts, n, ws, L, nullptr, nullptr, nullptr, st)
                   : launch_t<1, true>(pts, n, ws, L, nullptr, nullptr, nullptr, st);
    return vec ? launch_t<2, false>(pts, n, ws, L, surv_idx, surv_pts, surv_count, st)
               : launch_t<1, false>(pts, n, ws, L, surv_idx, surv_pts, surv_count, st);
}

}  // namespace ch

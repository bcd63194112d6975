// sort.cu -- stable LSD radix sort of the survivors by (x, y) for the
// monotone chain of Sec. 3.3 (Andrew's algorithm starts from the points in
// lexicographic order; the paper leaves this step to a CPU library).
//
// Keys are (ord(x) << 32 | ord(y)) with ord() the order-preserving map of
// binary32 to uint32 (-0 mapped to +0), values are the original point
// indices.  The filter writes the pairs in ascending index order and every
// pass is stable, so equal points end up in ascending index order.
//
// Structure (one-sweep style, Adinets & Merrill 2022): one histogram kernel
// computes all eight 8-bit digit histograms in a single read and marks
// passes whose digit is constant (skipped); each remaining pass is one
// persistent kernel that ranks a 4096-key tile in shared memory (warp
// match_any ranking, stable), finds the tile's per-digit global offsets by
// a decoupled look-back over 256 digit counters, and writes the tile out
// digit-sorted, so stores are runs of consecutive addresses.
#include "common.cuh"
#include "launch.h"

namespace ch {

namespace {

constexpr int NW = kSortThreads / 32;

struct SortSmem {
    unsigned long long keys[kSortTile];
    uint32_t vals[kSortTile];
    uint32_t wh[NW][256];      // per-warp digit counts, then per-warp offsets
    uint32_t tstart[256];      // start of each digit inside the sorted tile
    uint32_t gbase[256];       // output position of the tile's digit run, minus tstart
    uint32_t dbase[256];       // global start of each digit (exclusive scan of the histogram)
    uint32_t warp_tot[NW];
    uint32_t tile;
};

// exclusive scan of v over the 256 threads of the block; returns the total
__device__ __forceinline__ uint32_t block_excl_scan256(uint32_t v, uint32_t &excl, uint32_t *warp_tot)
{
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const uint32_t t = warp_tot[w];
        if (w < (int)warp) before += t;
        total += t;
    }
    excl = before + incl - v;
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(256) sort_hist_kernel(void *ws, Layout L)
{
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    const Octagon *oct = at<Octagon>(ws, L.oct);
    const uint32_t s = oct->abort ? 0u : ctrl->surv_count;
    const int64_t ntiles = ceil_div((int64_t)s, kSortTile);
    uint32_t *status0 = at<uint32_t>(ws, L.sort_status[0]);
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = gtid; w < ntiles * 256; w += gthreads) status0[w] = 0u;

    __shared__ uint32_t sh[kSortPasses][256];
    __shared__ bool s_last;
    for (int i = threadIdx.x; i < kSortPasses * 256; i += blockDim.x) (&sh[0][0])[i] = 0u;
    __syncthreads();
    const unsigned long long *keys = at<unsigned long long>(ws, L.keys[0]);
    for (int64_t i = gtid; i < (int64_t)s; i += gthreads) {
        const unsigned long long k = keys[i];
#pragma unroll
        for (int p = 0; p < kSortPasses; ++p) atomicAdd(&sh[p][(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSortPasses * 256; i += blockDim.x) {
        const uint32_t c = (&sh[0][0])[i];
        if (c) atomicAdd(&(&ctrl->hist[0][0])[i], c);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ctrl->hist_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        uint32_t cur = 0;
        for (int p = 0; p < kSortPasses; ++p) {
            bool skip = true;
            for (int d = 0; d < 256; ++d) {
                const uint32_t c = *(volatile uint32_t *)&ctrl->hist[p][d];
                if (c != 0 && c != s) skip = false;
                if (c == s) break;
            }
            if (s <= 1) skip = true;
            ctrl->pass_skip[p] = skip;
            ctrl->pass_src[p] = cur;
            if (!skip) cur ^= 1u;
        }
        ctrl->final_buf = cur;
    }
}

__global__ void __launch_bounds__(kSortThreads) sort_pass_kernel(void *ws, Layout L, int p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem &sm = *reinterpret_cast<SortSmem *>(smem_raw);
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    const Octagon *oct = at<Octagon>(ws, L.oct);
    const uint32_t s = oct->abort ? 0u : ctrl->surv_count;
    if (s == 0 || ctrl->pass_skip[p]) return;
    const uint32_t src = ctrl->pass_src[p], dst = src ^ 1u;
    const int64_t ntiles = ceil_div((int64_t)s, kSortTile);
    const unsigned long long *kin = at<unsigned long long>(ws, L.keys[src]);
    const uint32_t *vin = at<uint32_t>(ws, L.vals[src]);
    unsigned long long *kout = at<unsigned long long>(ws, L.keys[dst]);
    uint32_t *vout = at<uint32_t>(ws, L.vals[dst]);
    uint32_t *status = at<uint32_t>(ws, L.sort_status[src]);
    uint32_t *status_next = at<uint32_t>(ws, L.sort_status[dst]);
    const int shift = 8 * p;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    const uint32_t lt = (1u << lane) - 1u;

    // clear the digit status of the next executed pass
    {
        const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid;
        const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
        for (int64_t w = gtid; w < ntiles * 256; w += gthreads) status_next[w] = 0u;
    }
    // global digit starts
    {
        uint32_t ex;
        block_excl_scan256(ctrl->hist[p][tid], ex, sm.warp_tot);
        sm.dbase[tid] = ex;
    }

    for (;;) {
        if (tid == 0) sm.tile = atomicAdd(&ctrl->sort_ticket[p], 1u);
        for (int d = lane; d < 256; d += 32) sm.wh[warp][d] = 0u;
        __syncthreads();
        const int64_t tile = sm.tile;
        if (tile >= ntiles) break;
        const int64_t base = tile * kSortTile;
        const uint32_t tile_n = (uint32_t)min((int64_t)kSortTile, (int64_t)s - base);

        unsigned long long k[kSortItems];
        uint32_t v[kSortItems];
        uint32_t rank[kSortItems];
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const uint32_t e = warp * (32 * kSortItems) + j * 32 + lane;
            if (e < tile_n) {
                k[j] = __ldcs(kin + base + e);
                v[j] = __ldcs(vin + base + e);
            } else {
                k[j] = ~0ull;
                v[j] = 0u;
            }
        }
        // stable rank inside the warp, items in element order (j, lane)
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const uint32_t e = warp * (32 * kSortItems) + j * 32 + lane;
            const bool ok = e < tile_n;
            const uint32_t d = ok ? (uint32_t)(k[j] >> shift) & 255u : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const uint32_t before = __popc(peers & lt);
            uint32_t cur = 0;
            if (ok) cur = sm.wh[warp][d];
            __syncwarp();
            if (ok && before == 0) sm.wh[warp][d] = cur + __popc(peers);
            __syncwarp();
            rank[j] = cur + before;
        }
        __syncthreads();
        // per digit: exclusive offsets across warps and the tile count
        uint32_t cnt = 0;
        {
            const uint32_t d = tid;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint32_t c = sm.wh[w][d];
                sm.wh[w][d] = cnt;
                cnt += c;
            }
        }
        uint32_t tstart;
        block_excl_scan256(cnt, tstart, sm.warp_tot);
        sm.tstart[tid] = tstart;
        // decoupled look-back per digit (thread tid owns digit tid)
        {
            const uint32_t d = tid;
            uint32_t *mine = status + tile * 256 + d;
            uint32_t excl = 0;
            if (tile == 0) {
                st_release_u32(mine, kFlagP32 | cnt);
            } else {
                st_release_u32(mine, kFlagA32 | cnt);
                int64_t t = tile - 1;
                uint32_t spins = 0;
                bool failed = false;
                while (t >= 0) {
                    uint32_t st = ld_acquire_u32(status + t * 256 + d);
                    while ((st >> 30) == 0u) {
                        if (++spins > kSpinLimit || (spins > 1024 && error_set(ws, L))) {
                            failed = true;
                            break;
                        }
                        if (spins > 64) __nanosleep(100);
                        st = ld_acquire_u32(status + t * 256 + d);
                    }
                    if (failed) break;
                    excl += st & kVal32;
                    if ((st >> 30) == 2u) break;
                    --t;
                }
                if (failed) set_error(ws, L, kErrTimeout, 20 + p);
                st_release_u32(mine, kFlagP32 | ((excl + cnt) & kVal32));
            }
            sm.gbase[d] = sm.dbase[d] + excl - tstart;
        }
        // stage the tile digit-sorted in shared memory
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const uint32_t e = warp * (32 * kSortItems) + j * 32 + lane;
            if (e < tile_n) {
                const uint32_t d = (uint32_t)(k[j] >> shift) & 255u;
                const uint32_t pos = sm.tstart[d] + sm.wh[warp][d] + rank[j];
                sm.keys[pos] = k[j];
                sm.vals[pos] = v[j];
            }
        }
        __syncthreads();
        for (uint32_t i = tid; i < tile_n; i += kSortThreads) {
            const unsigned long long key = sm.keys[i];
            const uint32_t d = (uint32_t)(key >> shift) & 255u;
            const uint32_t pos = sm.gbase[d] + i;
            if (pos < s) {   // always true unless a look-back wait gave up
                kout[pos] = key;
                vout[pos] = sm.vals[i];
            }
        }
        __syncthreads();
    }
}

int pass_blocks_per_sm()
{
    static int cached = 0;
    if (!cached) {
        cudaFuncSetAttribute(sort_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SortSmem));
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, sort_pass_kernel, kSortThreads, sizeof(SortSmem));
        cached = v > 0 ? v : 1;
    }
    return cached;
}

}  // namespace

cudaError_t launch_sort(void *ws, const Layout &L, cudaStream_t st)
{
    const int64_t cap = L.sort_tiles;
    int64_t hb = (int64_t)sm_count() * 4;
    if (hb > cap) hb = cap;
    if (hb < 1) hb = 1;
    probe_before(CH_K_SORT_HIST, st);
    sort_hist_kernel<<<(unsigned)hb, 256, 0, st>>>(ws, L);
    probe_after(CH_K_SORT_HIST, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int64_t pb = (int64_t)sm_count() * pass_blocks_per_sm();
    if (pb > cap) pb = cap;
    if (pb < 1) pb = 1;
    for (int p = 0; p < kSortPasses; ++p) {
        probe_before(CH_K_SORT_PASS, st);
        sort_pass_kernel<<<(unsigned)pb, kSortThreads, sizeof(SortSmem), st>>>(ws, L, p);
        probe_after(CH_K_SORT_PASS, st);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ch

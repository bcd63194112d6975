// sort.cu -- stable LSD radix sort of the survivors by x for the monotone
// chain of Sec. 3.3 (Andrew's algorithm starts from the points in
// lexicographic order; the paper leaves this step to a CPU library).
//
// Only x is sorted: the key is ord(x), the order-preserving map of binary32
// to uint32 (-0 mapped to +0), and the payload is (ord(y) << 32 | index).
// Among points of equal x only the lowest can be a lower-chain vertex and
// only the highest an upper-chain vertex (apart from the first and last x),
// so the chain kernel reduces each equal-x run itself and y never needs to
// be part of the sort order.  That makes four 8-bit passes instead of eight.
// The filter writes the pairs in ascending index order and every pass is
// stable, so each equal-x run stays in ascending index order.
//
// Structure (one-sweep style, Adinets & Merrill 2022): one histogram kernel
// computes all four digit histograms in a single read and marks passes
// whose digit is constant (skipped); each remaining pass is one persistent
// kernel that ranks a 4096-key tile in shared memory (warp match_any
// ranking, stable), finds the tile's per-digit global offsets by a
// decoupled look-back over 256 digit counters, and writes the tile out
// digit-sorted, so stores are runs of consecutive addresses.  The payload
// is staged in shared memory in element order and gathered through the
// tile's inverse permutation at write-out, so it never occupies registers.
// When a block takes a ticket it also asks the TMA unit to bring the tile
// one grid ahead into L2 (tickets go out in order, so that tile is taken
// about one tile-time later).  The survivors come from the buffer
// ctrl->sort_in names (the filter writes buffer 0).
#include <algorithm>

#include "common.cuh"
#include "launch.h"

namespace ch {

namespace {

constexpr int NW = kSortThreads / 32;

struct SortSmem {
    unsigned long long pay[kSortTile];   // payload, element order
    uint32_t keys[kSortTile];            // keys, digit-sorted order
    uint16_t inv[kSortTile];             // digit-sorted position -> element
    uint32_t wh[NW][256];                // per-warp digit counts, then per-warp offsets
    uint32_t tstart[256];                // start of each digit inside the sorted tile
    uint32_t gbase[256];                 // output position of the tile's digit run, minus tstart
    uint32_t dbase[256];                 // global start of each digit (exclusive scan of the histogram)
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
    const uint32_t s = hull_stage_count(ctrl, oct);
    const int64_t ntiles = ceil_div((int64_t)s, kSortTile);
    // the first executed pass reads the survivors' buffer and its status
    uint32_t *status0 = at<uint32_t>(ws, L.sort_status[ctrl->sort_in]);
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = gtid; w < ntiles * 256; w += gthreads) status0[w] = 0u;

    __shared__ uint32_t sh[kSortPasses][256];
    __shared__ bool s_last;
    for (int i = threadIdx.x; i < kSortPasses * 256; i += blockDim.x) (&sh[0][0])[i] = 0u;
    __syncthreads();
    const uint32_t *keys = at<uint32_t>(ws, L.keys[ctrl->sort_in]);
    const int64_t nq = (int64_t)s / 4;   // 16-byte vector loads
    const uint4 *k4 = reinterpret_cast<const uint4 *>(keys);
    for (int64_t i = gtid; i < nq; i += gthreads) {
        const uint4 v = __ldcs(k4 + i);
        const uint32_t kk[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int p = 0; p < kSortPasses; ++p) atomicAdd(&sh[p][(kk[q] >> (8 * p)) & 255u], 1u);
    }
    for (int64_t i = nq * 4 + gtid; i < (int64_t)s; i += gthreads) {
        const uint32_t k = keys[i];
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
    // a pass whose digit is the same for every key moves nothing: one
    // thread per digit checks all passes at once
    __shared__ int s_skip[kSortPasses];
    if (threadIdx.x < kSortPasses) s_skip[threadIdx.x] = s <= 1;
    __syncthreads();
    for (int i = threadIdx.x; i < kSortPasses * 256; i += blockDim.x)
        if (__ldcg(&(&ctrl->hist[0][0])[i]) == s) s_skip[i / 256] = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t cur = ctrl->sort_in;
        for (int p = 0; p < kSortPasses; ++p) {
            ctrl->pass_skip[p] = s_skip[p];
            ctrl->pass_src[p] = cur;
            if (!s_skip[p]) cur ^= 1u;
        }
        ctrl->final_buf = cur;
    }
}

// Exclusive prefix of digit d over the tiles before `tile` (within its
// segment): adds the published counts going back to the first inclusive
// prefix, kLookWin status words per round trip.  A status word carries its
// flag and count together and nothing else is published through it, so
// relaxed accesses suffice.
constexpr int kLookWin = 8;

__device__ __forceinline__ uint32_t digit_lookback(const uint32_t *status, int64_t tile, uint32_t d, void *ws,
                                                   const Layout &L, uint32_t site)
{
    uint32_t excl = 0, spins = 0;
    int64_t t = tile - 1;
    for (;;) {
        uint32_t v[kLookWin];
#pragma unroll
        for (int i = 0; i < kLookWin; ++i) v[i] = t - i >= 0 ? ld_relaxed_u32(status + (t - i) * 256 + d) : kFlagP32;
        bool stop = false, done = false;
        int used = 0;
#pragma unroll
        for (int i = 0; i < kLookWin; ++i) {
            if (!stop) {
                const uint32_t f = v[i] >> 30;
                if (f == 0u) {
                    stop = true;
                } else {
                    excl += v[i] & kVal32;
                    ++used;
                    if (f == 2u) stop = done = true;
                }
            }
        }
        if (done) return excl;
        t -= used;
        if (used < kLookWin) {   // the next tile has published nothing yet
            if (++spins > kSpinLimit || (spins > 1024 && error_set(ws, L))) {
                set_error(ws, L, kErrTimeout, site);
                return excl;
            }
            if (spins > 64) __nanosleep(100);
        }
    }
}

struct PassIO {
    const uint32_t *kin;
    const unsigned long long *pin;
    uint32_t *kout;
    unsigned long long *pout;
    uint32_t *status;   // 256 digit status words per tile
};

// One tile of a pass: tile_n <= 4096 (key, payload) pairs from element
// `base`, ranked stably by digit (key >> shift) & 255 and written to
// out_base + (segment digit start + rank in digit).  `first`: the
// segment's first tile (its prefix is its own count).  Expects sm.dbase
// (the segment's digit starts) set and sm.wh cleared, behind a barrier.
__device__ __forceinline__ void pass_tile(SortSmem &sm, const PassIO &io, int64_t tile, int64_t base,
                                          uint32_t tile_n, int64_t out_base, uint32_t out_n, int shift, bool first,
                                          void *ws, const Layout &L, uint32_t site)
{
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    const uint32_t lt = (1u << lane) - 1u;
    // keys to registers, payload to shared memory (element order)
    uint32_t k[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint32_t e = warp * (32 * kSortItems) + j * 32 + lane;
        if (e < tile_n) {
            k[j] = __ldcs(io.kin + base + e);
            sm.pay[e] = __ldcs(io.pin + base + e);
        } else {
            k[j] = 0u;
        }
    }
    // stable rank inside the warp, items in element order (j, lane)
    uint16_t rank[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint32_t e = warp * (32 * kSortItems) + j * 32 + lane;
        const bool ok = e < tile_n;
        const uint32_t d = ok ? (k[j] >> shift) & 255u : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = __popc(peers & lt);
        uint32_t cur = 0;
        if (ok) cur = sm.wh[warp][d];
        __syncwarp();
        if (ok && before == 0) sm.wh[warp][d] = cur + __popc(peers);
        __syncwarp();
        rank[j] = (uint16_t)(cur + before);
    }
    __syncthreads();
    // per digit: exclusive offsets across warps and the tile count
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const uint32_t c = sm.wh[w][tid];
        sm.wh[w][tid] = cnt;
        cnt += c;
    }
    uint32_t tstart;
    block_excl_scan256(cnt, tstart, sm.warp_tot);
    sm.tstart[tid] = tstart;
    // decoupled look-back per digit (thread tid owns digit tid)
    {
        const uint32_t d = tid;
        uint32_t *mine = io.status + tile * 256 + d;
        uint32_t excl = 0;
        if (first) {
            st_relaxed_u32(mine, kFlagP32 | cnt);
        } else {
            st_relaxed_u32(mine, kFlagA32 | cnt);
            excl = digit_lookback(io.status, tile, d, ws, L, site);
            st_relaxed_u32(mine, kFlagP32 | ((excl + cnt) & kVal32));
        }
        sm.gbase[d] = sm.dbase[d] + excl - tstart;
    }
    __syncthreads();   // every digit's tstart is read below (gbase after the next barrier)
    // digit-sorted keys and the inverse permutation
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const uint32_t e = warp * (32 * kSortItems) + j * 32 + lane;
        if (e < tile_n) {
            const uint32_t d = (k[j] >> shift) & 255u;
            const uint32_t pos = sm.tstart[d] + sm.wh[warp][d] + rank[j];
            sm.keys[pos] = k[j];
            sm.inv[pos] = (uint16_t)e;
        }
    }
    __syncthreads();
    // runs of equal digit go to consecutive addresses; the bound check only
    // matters after a look-back wait gave up
    if (tile_n == kSortTile) {
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const uint32_t i = j * kSortThreads + tid;
            const uint32_t key = sm.keys[i];
            const uint32_t pos = sm.gbase[(key >> shift) & 255u] + i;
            if (pos < out_n) {
                io.kout[out_base + pos] = key;
                io.pout[out_base + pos] = sm.pay[sm.inv[i]];
            }
        }
    } else {
        for (uint32_t i = tid; i < tile_n; i += kSortThreads) {
            const uint32_t key = sm.keys[i];
            const uint32_t pos = sm.gbase[(key >> shift) & 255u] + i;
            if (pos < out_n) {
                io.kout[out_base + pos] = key;
                io.pout[out_base + pos] = sm.pay[sm.inv[i]];
            }
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kSortThreads, 3) sort_pass_kernel(void *ws, Layout L, int p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem &sm = *reinterpret_cast<SortSmem *>(smem_raw);
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    const Octagon *oct = at<Octagon>(ws, L.oct);
    const uint32_t s = hull_stage_count(ctrl, oct);
    if (s == 0 || ctrl->pass_skip[p]) return;
    const uint32_t src = ctrl->pass_src[p], dst = src ^ 1u;
    const int64_t ntiles = ceil_div((int64_t)s, kSortTile);
    const PassIO io{at<uint32_t>(ws, L.keys[src]), at<unsigned long long>(ws, L.pay[src]),
                    at<uint32_t>(ws, L.keys[dst]), at<unsigned long long>(ws, L.pay[dst]),
                    at<uint32_t>(ws, L.sort_status[src])};
    uint32_t *status_next = at<uint32_t>(ws, L.sort_status[dst]);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = lane_id();

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
        if (tid == 0) {
            const uint32_t t = atomicAdd(&ctrl->sort_ticket[p], 1u);
            sm.tile = t;
            // tickets go out in order, one per block and tile: the tile one
            // grid ahead is taken about one tile-time from now (by whichever
            // block); stream it into L2 meanwhile
            const int64_t ahead = (int64_t)t + gridDim.x;
            if (ahead < ntiles) {
                const uint32_t nn = (uint32_t)min((int64_t)kSortTile, (int64_t)s - ahead * kSortTile);
                bulk_prefetch_l2(io.kin + ahead * kSortTile, (nn * 4u) & ~15u);
                bulk_prefetch_l2(io.pin + ahead * kSortTile, (nn * 8u) & ~15u);
            }
        }
        for (int d = lane; d < 256; d += 32) sm.wh[warp][d] = 0u;
        __syncthreads();
        const int64_t tile = sm.tile;
        if (tile >= ntiles) break;
        const int64_t base = tile * kSortTile;
        pass_tile(sm, io, tile, base, (uint32_t)min((int64_t)kSortTile, (int64_t)s - base), 0, s, 8 * p, tile == 0,
                  ws, L, 20 + p);
    }
}

// ---------------------------------------------------------------------------
// many sets (ch_hull_batched): every set's survivors form one contiguous
// segment, sorted on its own.  Sort tiles are the sets' super-chunks (a
// tile never spans two sets), digit histograms and digit starts are per
// set, and a look-back chain starts afresh at each set's first tile.  All
// four passes run (no skipping), so the result lands in buffer 0.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) bx_sort_hist_kernel(void *ws, Layout L, BatchLayout BL)
{
    const BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    if (bc->abort) return;
    const SetInfo *sets = at<SetInfo>(ws, BL.sets);
    const uint32_t *sc_set = at<uint32_t>(ws, BL.sc_set);
    uint32_t *hist = at<uint32_t>(ws, BL.hist);
    const uint32_t *keys = at<uint32_t>(ws, L.keys[0]);
    uint32_t *status0 = at<uint32_t>(ws, L.sort_status[0]);
    const uint32_t nsc = bc->nsc;
    {
        const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        for (int64_t w = gtid; w < (int64_t)nsc * 256; w += (int64_t)gridDim.x * blockDim.x) status0[w] = 0u;
    }
    __shared__ uint32_t sh[kSortPasses][256];
    for (uint32_t j = blockIdx.x; j < nsc; j += gridDim.x) {
        for (int i = threadIdx.x; i < kSortPasses * 256; i += blockDim.x) (&sh[0][0])[i] = 0u;
        __syncthreads();
        const uint32_t b = sc_set[j];
        const int64_t lo = (int64_t)(j - sets[b].sc_base) * kSortTile;
        const int64_t n_t = min((int64_t)kSortTile, (int64_t)sets[b].s - lo);
        const uint32_t *kt = keys + sets[b].surv_base + lo;
        for (int64_t i = threadIdx.x; i < n_t; i += blockDim.x) {
            const uint32_t k = kt[i];
#pragma unroll
            for (int p = 0; p < kSortPasses; ++p) atomicAdd(&sh[p][(k >> (8 * p)) & 255u], 1u);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kSortPasses * 256; i += blockDim.x) {
            const uint32_t c = (&sh[0][0])[i];
            if (c) atomicAdd(&hist[(size_t)b * kSortPasses * 256 + i], c);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kSortThreads, 3) bx_sort_pass_kernel(void *ws, Layout L, BatchLayout BL, int p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem &sm = *reinterpret_cast<SortSmem *>(smem_raw);
    BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    if (bc->abort) return;
    const SetInfo *sets = at<SetInfo>(ws, BL.sets);
    const uint32_t *sc_set = at<uint32_t>(ws, BL.sc_set);
    const uint32_t *hist = at<uint32_t>(ws, BL.hist);
    const int64_t ntiles = bc->nsc;
    const uint32_t src = (uint32_t)p & 1u, dst = src ^ 1u;
    const PassIO io{at<uint32_t>(ws, L.keys[src]), at<unsigned long long>(ws, L.pay[src]),
                    at<uint32_t>(ws, L.keys[dst]), at<unsigned long long>(ws, L.pay[dst]),
                    at<uint32_t>(ws, L.sort_status[src])};
    uint32_t *status_next = at<uint32_t>(ws, L.sort_status[dst]);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    {
        const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid;
        const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
        for (int64_t w = gtid; w < ntiles * 256; w += gthreads) status_next[w] = 0u;
    }
    for (;;) {
        if (tid == 0) sm.tile = atomicAdd(&bc->sort_ticket[p], 1u);
        for (int d = lane; d < 256; d += 32) sm.wh[warp][d] = 0u;
        __syncthreads();
        const int64_t tile = sm.tile;
        if (tile >= ntiles) break;
        const uint32_t b = sc_set[tile];
        const int64_t ltile = tile - sets[b].sc_base;
        const int64_t seg = (int64_t)sets[b].surv_base;
        const uint32_t seg_n = sets[b].s;
        {   // this set's digit starts (the scan's barriers also order sm.wh)
            uint32_t ex;
            block_excl_scan256(hist[((size_t)b * kSortPasses + p) * 256 + tid], ex, sm.warp_tot);
            sm.dbase[tid] = ex;
        }
        pass_tile(sm, io, tile, seg + ltile * kSortTile,
                  (uint32_t)min((int64_t)kSortTile, (int64_t)seg_n - ltile * kSortTile), seg, seg_n, 8 * p,
                  ltile == 0, ws, L, 40 + p);
    }
}

int pass_blocks_per_sm()
{
    static const int cached = [] {   // thread-safe one-time initialisation
        cudaFuncSetAttribute(sort_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SortSmem));
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, sort_pass_kernel, kSortThreads, sizeof(SortSmem));
        return v > 0 ? v : 1;
    }();
    return cached;
}

int bx_pass_blocks_per_sm()
{
    static const int cached = [] {
        cudaFuncSetAttribute(bx_sort_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SortSmem));
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, bx_sort_pass_kernel, kSortThreads, sizeof(SortSmem));
        return v > 0 ? v : 1;
    }();
    return cached;
}

}  // namespace

cudaError_t launch_bx_sort(void *ws, const Layout &L, const BatchLayout &BL, cudaStream_t st)
{
    const int64_t cap = BL.tiles_max;
    const int64_t hb = std::max<int64_t>(1, std::min<int64_t>(cap, (int64_t)sm_count() * 4));
    probe_before(CH_K_SORT_HIST, st);
    bx_sort_hist_kernel<<<(unsigned)hb, 256, 0, st>>>(ws, L, BL);
    note_kernels(CH_K_SORT_HIST, 1);
    probe_after(CH_K_SORT_HIST, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int tuned = tune_value(CH_TUNE_BX_SORT_PASS);
    const int64_t pb = std::max<int64_t>(
        1, std::min<int64_t>(cap, (int64_t)sm_count() * (tuned ? tuned : bx_pass_blocks_per_sm())));
    for (int p = 0; p < kSortPasses; ++p) {
        probe_before(CH_K_SORT_PASS, st);
        bx_sort_pass_kernel<<<(unsigned)pb, kSortThreads, sizeof(SortSmem), st>>>(ws, L, BL, p);
        note_kernels(CH_K_SORT_PASS, 1);
        probe_after(CH_K_SORT_PASS, st);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_sort(void *ws, const Layout &L, cudaStream_t st)
{
    const int64_t cap = L.sort_tiles;
    int64_t hb = (int64_t)sm_count() * 4;
    if (hb > cap) hb = cap;
    if (hb < 1) hb = 1;
    probe_before(CH_K_SORT_HIST, st);
    sort_hist_kernel<<<(unsigned)hb, 256, 0, st>>>(ws, L);
    note_kernels(CH_K_SORT_HIST, 1);
    probe_after(CH_K_SORT_HIST, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int64_t pb = (int64_t)sm_count() * pass_blocks_per_sm();
    if (pb > cap) pb = cap;
    if (pb < 1) pb = 1;
    for (int p = 0; p < kSortPasses; ++p) {
        probe_before(CH_K_SORT_PASS, st);
        sort_pass_kernel<<<(unsigned)pb, kSortThreads, sizeof(SortSmem), st>>>(ws, L, p);
        note_kernels(CH_K_SORT_PASS, 1);
        probe_after(CH_K_SORT_PASS, st);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ch

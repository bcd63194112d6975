// batched.cu -- the set bookkeeping of ch_hull_batched: validating the CSR
// offsets, the tile -> set map, and assembling the per-set hulls.  The
// per-set work itself (extremes, octagon, filter, sort, chains) runs in the
// batched kernels of the other translation units; every stage treats a set
// exactly as the single-set path treats its one input (Algorithm 1).
#include <algorithm>

#include "common.cuh"
#include "launch.h"

namespace ch {
namespace {

constexpr int kSetupThreads = 1024;
constexpr uint32_t kSiteOffsets = 40;

// One block: checks offsets (offsets[0] = 0, non-decreasing, offsets[B] <=
// n_cap) and fills each set's point range and first 4096-point tile.
__global__ void __launch_bounds__(kSetupThreads) bx_setup_kernel(const int64_t *__restrict__ offsets, void *ws,
                                                                 Layout L, BatchLayout BL, int64_t n_cap)
{
    __shared__ uint64_t s_w[kSetupThreads / 32];
    __shared__ int s_bad;
    BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    SetInfo *sets = at<SetInfo>(ws, BL.sets);
    const int64_t B = BL.num_sets;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    const int64_t per = ceil_div(B, (int64_t)kSetupThreads);
    const int64_t b0 = min((int64_t)threadIdx.x * per, B), b1 = min(b0 + per, B);
    int bad = 0;   // 1: the points do not fit the workspace, 2: malformed offsets
    uint64_t tiles = 0;
    for (int64_t b = b0; b < b1; ++b) {
        const int64_t lo = offsets[b], hi = offsets[b + 1];
        if (lo < 0 || hi < lo) bad = 2;
        else if (hi > n_cap) bad = max(bad, 1);
        else tiles += hi > lo ? (uint64_t)ceil_div(hi - lo, (int64_t)kFiltTile) : 0;
    }
    if (threadIdx.x == 0 && offsets[0] != 0) bad = 2;
    if (bad) atomicMax(&s_bad, bad);
    uint64_t incl = tiles;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += u;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (s_bad) {
        if (threadIdx.x == 0) {
            bc->abort = 1;
            set_error(ws, L, s_bad == 1 ? (uint32_t)CH_ERR_CAPACITY : (uint32_t)CH_ERR_ARG, kSiteOffsets);
        }
        return;
    }
    uint64_t before = 0, total = 0;
    for (uint32_t w = 0; w < kSetupThreads / 32; ++w) {
        if (w < warp) before += s_w[w];
        total += s_w[w];
    }
    uint64_t run = before + incl - tiles;
    for (int64_t b = b0; b < b1; ++b) {
        const int64_t lo = offsets[b], hi = offsets[b + 1];
        SetInfo &S = sets[b];
        S.pt_begin = lo;
        S.n = hi - lo;
        S.tile_base = (uint32_t)run;
        S.ntiles = (uint32_t)(hi > lo ? ceil_div(hi - lo, (int64_t)kFiltTile) : 0);
        S.s = 0;
        S.nsc = 0;
        S.hull = 0;
        run += S.ntiles;
    }
    if (threadIdx.x == 0) bc->tiles = (uint32_t)total;
}

// Largest i in [0, count) with key(i) <= v (-1 if none): binary search
// over a non-decreasing sequence.
template <class F>
__device__ __forceinline__ int64_t last_le(int64_t count, uint64_t v, F key)
{
    int64_t lo = 0, hi = count;   // first index with key > v lies in [lo, hi]
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (key(mid) <= v) lo = mid + 1;
        else hi = mid;
    }
    return lo - 1;
}

__global__ void __launch_bounds__(256) bx_tileset_kernel(void *ws, BatchLayout BL)
{
    const BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    if (bc->abort) return;
    const SetInfo *sets = at<SetInfo>(ws, BL.sets);
    uint32_t *tile_set = at<uint32_t>(ws, BL.tile_set);
    const int64_t T = bc->tiles, B = BL.num_sets;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x)
        tile_set[t] = (uint32_t)last_le(B, (uint64_t)t, [&](int64_t b) { return (uint64_t)sets[b].tile_base; });
}

// vertices of set b's hull: its lower chain, then its upper chain without
// the two ends it shares with the lower one
__device__ __forceinline__ void set_chain_sizes(const SetInfo &S, const uint32_t *off0, const uint32_t *off1,
                                                uint32_t &l0, uint32_t &hl, uint32_t &u0, uint32_t &hu)
{
    if (S.nsc == 0) {
        l0 = hl = u0 = hu = 0;
        return;
    }
    l0 = off0[S.sc_base];
    hl = off0[S.sc_base + S.nsc] - l0;
    u0 = off1[S.sc_base];
    hu = off1[S.sc_base + S.nsc] - u0;
}

// One block: hull sizes and their exclusive scan into hull_offsets[0..B].
__global__ void __launch_bounds__(kSetupThreads) bx_hullsize_kernel(void *ws, BatchLayout BL, int64_t *hull_offsets)
{
    __shared__ uint64_t s_w[kSetupThreads / 32];
    const BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    SetInfo *sets = at<SetInfo>(ws, BL.sets);
    const uint32_t *off0 = at<uint32_t>(ws, BL.sc_off[0]), *off1 = at<uint32_t>(ws, BL.sc_off[1]);
    const bool abort = bc->abort != 0;
    const int64_t B = BL.num_sets;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const int64_t per = ceil_div(B, (int64_t)kSetupThreads);
    const int64_t b0 = min((int64_t)threadIdx.x * per, B), b1 = min(b0 + per, B);
    uint64_t sum = 0;
    for (int64_t b = b0; b < b1 && !abort; ++b) {
        uint32_t l0, hl, u0, hu;
        set_chain_sizes(sets[b], off0, off1, l0, hl, u0, hu);
        const uint32_t h = hl == 0 ? 0u : hl + (hu >= 2 ? hu - 2 : 0u);
        sets[b].hull = h;
        sum += h;
    }
    uint64_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += u;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    uint64_t before = 0, total = 0;
    for (uint32_t w = 0; w < kSetupThreads / 32; ++w) {
        if (w < warp) before += s_w[w];
        total += s_w[w];
    }
    uint64_t run = before + incl - sum;
    for (int64_t b = b0; b < b1; ++b) {
        hull_offsets[b] = (int64_t)run;
        if (!abort) run += sets[b].hull;
    }
    if (threadIdx.x == 0) hull_offsets[B] = (int64_t)total;
}

// Output position p of the concatenated hulls -> its set (binary search over
// hull_offsets) -> the lower chain, or the upper chain read backwards.
__global__ void __launch_bounds__(256) bx_assemble_kernel(void *ws, Layout L, BatchLayout BL,
                                                          const int64_t *__restrict__ hull_offsets, uint32_t *hull_idx)
{
    const BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    if (bc->abort) return;
    const SetInfo *sets = at<SetInfo>(ws, BL.sets);
    const uint32_t *off0 = at<uint32_t>(ws, BL.sc_off[0]), *off1 = at<uint32_t>(ws, BL.sc_off[1]);
    const uint32_t *lower = at<uint32_t>(ws, BL.lower), *upper = at<uint32_t>(ws, L.utmp);
    const int64_t B = BL.num_sets;
    const int64_t H = hull_offsets[B];
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < H; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = last_le(B, (uint64_t)p, [&](int64_t i) { return (uint64_t)hull_offsets[i]; });
        uint32_t l0, hl, u0, hu;
        set_chain_sizes(sets[b], off0, off1, l0, hl, u0, hu);
        const int64_t k = p - hull_offsets[b];
        hull_idx[p] = k < hl ? lower[l0 + k] : upper[u0 + hu - 2 - (k - hl)];
    }
}

}  // namespace

cudaError_t launch_bx_setup(const int64_t *offsets, void *ws, const Layout &L, const BatchLayout &BL, int64_t n_cap,
                            cudaStream_t st)
{
    bx_setup_kernel<<<1, kSetupThreads, 0, st>>>(offsets, ws, L, BL, n_cap);
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ceil_div(BL.tiles_max, 256), sm_count() * 4));
    bx_tileset_kernel<<<(unsigned)blocks, 256, 0, st>>>(ws, BL);
    note_kernels(CH_K_EXTREMES, 2);
    return cudaGetLastError();
}

cudaError_t launch_bx_finish(void *ws, const Layout &L, const BatchLayout &BL, uint32_t *hull_idx,
                             int64_t *hull_offsets, cudaStream_t st)
{
    probe_before(CH_K_FINISH, st);
    bx_hullsize_kernel<<<1, kSetupThreads, 0, st>>>(ws, BL, hull_offsets);
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(ceil_div(L.n, 256), sm_count() * 4));
    bx_assemble_kernel<<<(unsigned)blocks, 256, 0, st>>>(ws, L, BL, hull_offsets, hull_idx);
    note_kernels(CH_K_FINISH, 2);
    probe_after(CH_K_FINISH, st);
    return cudaGetLastError();
}

}  // namespace ch

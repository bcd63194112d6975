// chain.cu -- Sec. 3.3 of Carrasco et al. (convexHull_algorithm), kept on
// the device: Andrew's monotone chain over the sorted survivors.
//
// The paper copies the candidates to the host and calls CGAL; its
// conclusion names a fully device-resident hull as the next step.  Here:
//
//  1. leaf chains: the sorted survivors are cut into chunks of kChainC
//     points; one thread runs the sequential monotone chain (lower and
//     upper) over its chunk, skipping repeats of the previous point.
//  2. merges: chunk chains are merged pairwise up a binary tree.  The
//     second child to finish merges the pair (no thread ever waits).  Two
//     x-ordered lower chains A | B merge by walking the common tangent:
//     the cursor b on B moves right while B's next vertex is on or below
//     line(a, b); the cursor a on A moves left while A's previous vertex is
//     on or below line(a, b); repeat until neither moves.  The merged
//     chain is A up to a followed by B from b, which is what the sequential
//     chain produces (same pops, same collinear exclusion).  Each chunk
//     keeps the surviving range [lo, hi] of its chain, and chunks whose
//     range empties are unlinked from a list of live chunks.  Upper chains
//     are handled the same way with the predicate mirrored.
//  3. emit: one pass compacts the live ranges (decoupled look-back over
//     chunk counts) into the lower chain and the upper chain, and the
//     final kernel appends the upper chain, reversed and without its end
//     points, behind the lower one: counter-clockwise from the
//     lexicographically smallest point.
#include "common.cuh"
#include "launch.h"

namespace ch {

namespace {

constexpr int C = kChainC;

struct ChainPtrs {
    const unsigned long long *keys;
    const uint32_t *vals;
    uint32_t *chain[2];      // lower, upper
    int32_t *lo[2], *hi[2], *prv[2], *nxt[2];
    int32_t *node;           // 4 ints per node: firstL lastL firstU lastU
    int32_t *node_cnt;       // arrivals per node (zeroed at the start of each call)
};

__device__ __forceinline__ ChainPtrs chain_ptrs(void *ws, const Layout &L, uint32_t buf)
{
    ChainPtrs P;
    P.keys = at<unsigned long long>(ws, L.keys[buf]);
    P.vals = at<uint32_t>(ws, L.vals[buf]);
    P.chain[0] = at<uint32_t>(ws, L.chainL);
    P.chain[1] = at<uint32_t>(ws, L.chainU);
    int32_t *ck = at<int32_t>(ws, L.chunk);
    const int64_t nc = L.n_chunks;
    P.lo[0] = ck + 0 * nc;
    P.hi[0] = ck + 1 * nc;
    P.lo[1] = ck + 2 * nc;
    P.hi[1] = ck + 3 * nc;
    P.prv[0] = ck + 4 * nc;
    P.nxt[0] = ck + 5 * nc;
    P.prv[1] = ck + 6 * nc;
    P.nxt[1] = ck + 7 * nc;
    P.node = at<int32_t>(ws, L.node);
    P.node_cnt = at<int32_t>(ws, L.node_cnt);
    return P;
}

__device__ __forceinline__ int32_t ldcg(const int32_t *p) { return __ldcg(p); }

__device__ __forceinline__ float2 vertex(const ChainPtrs &P, int side, int32_t c, int32_t k)
{
    const uint32_t pos = __ldcg(P.chain[side] + (int64_t)c * C + k);
    return key_point(__ldg(P.keys + pos));
}

// pop / advance test: lower chains drop a vertex when the turn is not
// strictly counter-clockwise, upper chains when it is not strictly clockwise
__device__ __forceinline__ bool drop(int side, const float2 &a, const float2 &b, const float2 &c)
{
    const int o = orient(a.x, a.y, b.x, b.y, c.x, c.y);
    return side == 0 ? o <= 0 : o >= 0;
}

// first / last live chunk of tree node (level, j); level 0 = chunk j
__device__ __forceinline__ void node_ends(const ChainPtrs &P, int level, int64_t nb, int64_t j, int side,
                                          int32_t &first, int32_t &last)
{
    if (level == 0) {
        const bool live = ldcg(P.hi[side] + j) >= ldcg(P.lo[side] + j);
        first = last = live ? (int32_t)j : -1;
    } else {
        first = ldcg(P.node + (nb + j) * 4 + 2 * side);
        last = ldcg(P.node + (nb + j) * 4 + 2 * side + 1);
    }
}

__device__ void merge_side(const ChainPtrs &P, int side, int32_t fa, int32_t la, int32_t fb, int32_t lb)
{
    int32_t *lo = P.lo[side], *hi = P.hi[side], *prv = P.prv[side], *nxt = P.nxt[side];
    int32_t ca = la, ka = ldcg(hi + ca);
    int32_t cb = fb, kb = ldcg(lo + cb);
    int32_t hia = ka, lob = kb;          // live range ends of the current chunks
    int32_t loa = ldcg(lo + ca), hib = ldcg(hi + cb);
    float2 pa = vertex(P, side, ca, ka);
    float2 pb = vertex(P, side, cb, kb);
    for (;;) {
        bool moved = false;
        for (;;) {   // advance b
            int32_t nc_ = cb, nk = kb + 1;
            int32_t nlo = lob, nhi = hib;
            if (kb >= hib) {
                if (cb == lb) break;
                nc_ = ldcg(nxt + cb);
                nlo = ldcg(lo + nc_);
                nhi = ldcg(hi + nc_);
                nk = nlo;
            }
            const float2 q = vertex(P, side, nc_, nk);
            if (!drop(side, pa, pb, q)) break;
            if (nc_ != cb) {          // chunk cb is now entirely removed
                lo[cb] = 1;
                hi[cb] = 0;
                cb = nc_;
                lob = nlo;
                hib = nhi;
            }
            kb = nk;
            pb = q;
            moved = true;
        }
        for (;;) {   // retreat a
            int32_t pc = ca, pk = ka - 1;
            int32_t plo = loa, phi = hia;
            if (ka <= loa) {
                if (ca == fa) break;
                pc = ldcg(prv + ca);
                plo = ldcg(lo + pc);
                phi = ldcg(hi + pc);
                pk = phi;
            }
            const float2 q = vertex(P, side, pc, pk);
            if (!drop(side, q, pa, pb)) break;
            if (pc != ca) {
                lo[ca] = 1;
                hi[ca] = 0;
                ca = pc;
                loa = plo;
                hia = phi;
            }
            ka = pk;
            pa = q;
            moved = true;
        }
        if (!moved) break;
    }
    hi[ca] = ka;
    lo[cb] = kb;
    nxt[ca] = cb;
    prv[cb] = ca;
}

__global__ void __launch_bounds__(kChainThreads) chain_kernel(void *ws, Layout L)
{
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    const Octagon *oct = at<Octagon>(ws, L.oct);
    const uint32_t s = oct->abort ? 0u : ctrl->surv_count;
    if (s == 0) return;
    const ChainPtrs P = chain_ptrs(ws, L, ctrl->final_buf);
    const int64_t nc = ceil_div((int64_t)s, C);
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gthreads) {
        // ---- leaf: sequential monotone chain over the chunk
        const int64_t begin = c * C;
        const int64_t end = min(begin + C, (int64_t)s);
        unsigned long long prev_key = begin > 0 ? __ldg(P.keys + begin - 1) : ~0ull;
        bool have_prev = begin > 0;
        int32_t h[2] = {0, 0};
        float2 t1[2], t2[2];   // top and second of each stack
        for (int64_t k = begin; k < end; ++k) {
            const unsigned long long key = __ldg(P.keys + k);
            if (have_prev && key == prev_key) continue;
            have_prev = true;
            prev_key = key;
            const float2 p = key_point(key);
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                uint32_t *st = P.chain[side] + begin;
                while (h[side] >= 2 && drop(side, t2[side], t1[side], p)) {
                    --h[side];
                    t1[side] = t2[side];
                    if (h[side] >= 2) t2[side] = key_point(__ldg(P.keys + st[h[side] - 2]));
                }
                st[h[side]] = (uint32_t)k;
                ++h[side];
                t2[side] = t1[side];
                t1[side] = p;
            }
        }
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            P.lo[side][c] = 0;
            P.hi[side][c] = h[side] - 1;
        }

        // ---- climb: the second child to arrive merges the pair
        int64_t node = c, w = nc, nb_child = 0, nb = 0;   // nb: base of the level above
        int level = 0;
        while (w > 1) {
            const int64_t parent = node >> 1, pw = (w + 1) / 2;
            const int64_t sib = node ^ 1;
            int32_t rec[4];
            if (sib >= w) {
                // no sibling: the parent is this node
#pragma unroll
                for (int side = 0; side < 2; ++side) node_ends(P, level, nb_child, node, side, rec[2 * side], rec[2 * side + 1]);
            } else {
                __threadfence();
                if (atomicAdd(P.node_cnt + nb + parent, 1) == 0) break;   // first to arrive: the sibling merges
                __threadfence();
                const int64_t a = parent * 2, b = a + 1;
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    int32_t fa, la, fb, lb;
                    node_ends(P, level, nb_child, a, side, fa, la);
                    node_ends(P, level, nb_child, b, side, fb, lb);
                    if (la < 0) {
                        rec[2 * side] = fb;
                        rec[2 * side + 1] = lb;
                    } else if (fb < 0) {
                        rec[2 * side] = fa;
                        rec[2 * side + 1] = la;
                    } else {
                        merge_side(P, side, fa, la, fb, lb);
                        rec[2 * side] = fa;
                        rec[2 * side + 1] = lb;
                    }
                }
            }
#pragma unroll
            for (int f = 0; f < 4; ++f) P.node[(nb + parent) * 4 + f] = rec[f];
            node = parent;
            nb_child = nb;
            nb += pw;
            w = pw;
            ++level;
        }
    }
}

// Compacts the live chain ranges: thread = chunk, look-back over chunk
// tiles, warp-cooperative copies.  Side 0 goes to hull_idx, side 1 to utmp.
__global__ void __launch_bounds__(kEmitThreads) emit_kernel(void *ws, Layout L, uint32_t *hull_idx)
{
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    const Octagon *oct = at<Octagon>(ws, L.oct);
    const uint32_t s = oct->abort ? 0u : ctrl->surv_count;
    if (s == 0) return;
    const ChainPtrs P = chain_ptrs(ws, L, ctrl->final_buf);
    const int64_t nc = ceil_div((int64_t)s, C);
    const int64_t ntiles = ceil_div(nc, kEmitThreads);
    uint32_t *utmp = at<uint32_t>(ws, L.utmp);
    unsigned long long *status[2] = {at<unsigned long long>(ws, L.emit_status[0]),
                                     at<unsigned long long>(ws, L.emit_status[1])};
    constexpr int NW = kEmitThreads / 32;
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_wsum[2][NW];
    __shared__ unsigned long long s_excl[2];
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&ctrl->emit_ticket[0], 1u);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= ntiles) break;
        const int64_t c = tile * kEmitThreads + tid;
        int32_t lo[2] = {0, 0}, cnt[2] = {0, 0};
        if (c < nc) {
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                lo[side] = ldcg(P.lo[side] + c);
                const int32_t hi = ldcg(P.hi[side] + c);
                cnt[side] = hi >= lo[side] ? hi - lo[side] + 1 : 0;
            }
        }
        uint32_t pre[2];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            uint32_t incl = (uint32_t)cnt[side];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (uint32_t)o) incl += t;
            }
            pre[side] = incl - (uint32_t)cnt[side];
            if (lane == 31) s_wsum[side][warp] = incl;
        }
        __syncthreads();
        if (warp < 2) {
            const int side = (int)warp;
            uint32_t wv = lane < (uint32_t)NW ? s_wsum[side][lane] : 0u;
            uint32_t incl = wv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (uint32_t)o) incl += t;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            if (lane < (uint32_t)NW) s_wsum[side][lane] = incl - wv;
            unsigned long long excl = 0;
            if (tile == 0) {
                if (lane == 0) st_release_u64(status[side], kFlagP | total);
            } else {
                if (lane == 0) st_release_u64(status[side] + tile, kFlagA | total);
                excl = lookback_u64(status[side], tile, ws, L, 30 + side);
                if (lane == 0) st_release_u64(status[side] + tile, kFlagP | ((excl + total) & kValMask));
            }
            if (lane == 0) {
                s_excl[side] = excl;
                if (tile == ntiles - 1) {
                    if (side == 0) ctrl->h_lower = (uint32_t)(excl + total);
                    else ctrl->h_upper = (uint32_t)(excl + total);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const uint64_t mypos = s_excl[side] + s_wsum[side][warp] + pre[side];
            uint32_t *out = side == 0 ? hull_idx : utmp;
            const uint32_t *chain = P.chain[side];
            for (int i = 0; i < 32; ++i) {
                const int32_t n_i = __shfl_sync(0xffffffffu, cnt[side], i);
                if (n_i == 0) continue;
                const int32_t lo_i = __shfl_sync(0xffffffffu, lo[side], i);
                const uint64_t pos_i = __shfl_sync(0xffffffffu, mypos, i);
                const int64_t ci = tile * kEmitThreads + warp * 32 + i;
                for (int32_t k = (int32_t)lane; k < n_i; k += 32) {
                    const uint32_t sp = __ldcg(chain + ci * C + lo_i + k);
                    if (pos_i + k < (uint64_t)s) out[pos_i + k] = __ldg(P.vals + sp);
                }
            }
        }
        __syncthreads();
    }
}

// hull = lower chain, then the upper chain reversed without its two ends
__global__ void finish_kernel(void *ws, Layout L, uint32_t *hull_idx, uint32_t *hull_count)
{
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    const uint32_t hl = ctrl->h_lower, hu = ctrl->h_upper;
    const uint32_t mid = hu >= 2 ? hu - 2 : 0;
    const uint32_t *utmp = at<uint32_t>(ws, L.utmp);
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < mid; m += gthreads)
        if (hl + m < L.n) hull_idx[hl + m] = utmp[hu - 2 - m];
    if (blockIdx.x == 0 && threadIdx.x == 0) *hull_count = hl == 0 ? 0u : hl + mid;
}

}  // namespace

cudaError_t launch_chain(void *ws, const Layout &L, uint32_t *hull_idx, uint32_t *hull_count, cudaStream_t st)
{
    const int sms = sm_count();
    int64_t cb = ceil_div(L.n_chunks, kChainThreads);
    if (cb > (int64_t)sms * 16) cb = (int64_t)sms * 16;
    if (cb < 1) cb = 1;
    probe_before(CH_K_CHAIN, st);
    chain_kernel<<<(unsigned)cb, kChainThreads, 0, st>>>(ws, L);
    probe_after(CH_K_CHAIN, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int64_t eb = L.emit_tiles;
    if (eb > (int64_t)sms * 4) eb = (int64_t)sms * 4;
    if (eb < 1) eb = 1;
    probe_before(CH_K_EMIT, st);
    emit_kernel<<<(unsigned)eb, kEmitThreads, 0, st>>>(ws, L, hull_idx);
    probe_after(CH_K_EMIT, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int64_t fb = ceil_div(L.n, 256 * 8);
    if (fb > (int64_t)sms * 4) fb = (int64_t)sms * 4;
    if (fb < 1) fb = 1;
    probe_before(CH_K_FINISH, st);
    finish_kernel<<<(unsigned)fb, 256, 0, st>>>(ws, L, hull_idx, hull_count);
    probe_after(CH_K_FINISH, st);
    return cudaGetLastError();
}

}  // namespace ch

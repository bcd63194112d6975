// chain.cu -- Sec. 3.3 of Carrasco et al. (convexHull_algorithm), kept on
// the device: Andrew's monotone chain over the survivors sorted by x.
//
// The paper copies the candidates to the host and calls CGAL; its
// conclusion names a fully device-resident hull as the next step.  Here:
//
//  0. runs: the survivors arrive sorted by x (equal x in ascending index
//     order).  In a run of equal x only the lowest point can be a vertex of
//     the lower chain and only the highest one of the upper chain, because
//     the others lie strictly above (below) it on the same vertical.  The
//     exceptions are the first x, whose lowest point starts both chains and
//     whose highest point follows it on the upper chain, and the last x,
//     whose highest point ends both chains after its lowest point on the
//     lower chain.  Each run is reduced to those representatives (first
//     occurrence on ties, i.e. the lowest index, which also collapses equal
//     points).  A block owns the runs starting in its 4096-point
//     super-chunk and looks ahead (block-parallel) when its last run
//     continues past the super-chunk.
//  1. elimination: per side, parallel passes over the representatives drop
//     every point whose turn with its current neighbours is not strict (for
//     the lower chain: on or above the segment joining them).  Such a point
//     lies on or above a segment between two points of the set, so it is
//     not a strict vertex of the lower hull and the sequential chain would
//     pop it too; a sequence where every turn is strict is its own monotone
//     chain.  Each warp first runs passes over its share of the sequence
//     (its two ends stay); then the warps' survivors are concatenated and
//     the passes continue over the whole super-chunk sequence (block-wide
//     while long, one warp once short) until nothing changes.  The
//     converged sequence is written out as the super-chunk's chain.
//  2. fallback, when the passes do not converge within their cap: what is
//     left is cut into leaves; one thread runs the sequential monotone
//     chain on each, and the leaf chains are merged pairwise up a binary
//     tree inside the block (shared memory, one level per barrier).
//     Across super-chunks a second kernel merges the chains up a tree in
//     global memory, where the second child to finish merges the pair (no
//     thread ever waits).  Two x-ordered lower chains A | B merge by walking
//     the common tangent: the cursor b on B moves right while B's next
//     vertex is on or below line(a, b); the cursor a on A moves left while
//     A's previous vertex is on or below line(a, b); repeat until neither
//     moves.  The merged chain is A up to a followed by B from b, which is
//     what the sequential chain produces (same pops, same collinear
//     exclusion).  Each chunk keeps the surviving range [lo, hi] of its
//     chain; chunks whose range empties are unlinked from a list of live
//     chunks.  Upper chains are handled the same way with the predicate
//     mirrored.
//  3. emit: one pass compacts the live ranges (decoupled look-back over
//     super-chunk counts) into the lower chain and the upper chain, and the
//     final kernel appends the upper chain, reversed and without its end
//     points, behind the lower one: counter-clockwise from the
//     lexicographically smallest point.
#include "common.cuh"
#include "launch.h"

namespace ch {

namespace {

constexpr int LT = kChainThreads;   // leaves per super-chunk
constexpr int SC = kChainC;         // points per super-chunk
constexpr int CS = kChainStride;    // chain slots per super-chunk
constexpr int NL = SC + 2;          // sequence capacity: SC points + 2 look-ahead slots
constexpr int NWB = LT / 32;        // warps per block
constexpr int LWMAX = ((NL + NWB - 1) / NWB + 31) / 32;   // longest leaf (17)

// pop / advance test: lower chains drop a vertex when the turn is not
// strictly counter-clockwise, upper chains when it is not strictly clockwise
__device__ __forceinline__ bool drop(int side, const float2 &a, const float2 &b, const float2 &c)
{
    const int o = orient(a.x, a.y, b.x, b.y, c.x, c.y);
    return side == 0 ? o <= 0 : o >= 0;
}

// One strict-turn elimination pass of a warp over the sequence
// src[0 .. len) of point indices (its two ends always stay): the kept
// entries go to dst in order; returns how many.  len >= 3.  Two 32-entry
// chunks per step, binary32 tier of both tests first, so their latencies
// overlap.
__device__ __forceinline__ int warp_elim_pass(const float2 *pts, const uint16_t *src, uint16_t *dst, int len,
                                              int side, int lane, uint32_t lt)
{
    int kept = 0;
    for (int c0 = 0; c0 < len; c0 += 64) {
        int j[2];
        bool test[2];
        float2 a[2], b[2], c[2];
        int o[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            j[u] = c0 + 32 * u + lane;
            test[u] = j[u] > 0 && j[u] < len - 1;
            const int jj = test[u] ? j[u] : 1;
            a[u] = pts[src[jj - 1]];
            b[u] = pts[src[jj]];
            c[u] = pts[src[jj + 1]];
            o[u] = orient_f32(a[u].x, a[u].y, b[u].x, b[u].y, c[u].x, c[u].y);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (test[u] && o[u] == 2) o[u] = orient_rest(a[u].x, a[u].y, b[u].x, b[u].y, c[u].x, c[u].y);
        uint32_t m[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const bool drop_it = test[u] && (side == 0 ? o[u] <= 0 : o[u] >= 0);
            const bool k = j[u] < len && !drop_it;
            m[u] = __ballot_sync(0xffffffffu, k);
            if (k) dst[kept + __popc(m[u] & lt)] = src[j[u]];
            kept += __popc(m[u]);
        }
    }
    __syncwarp();
    return kept;
}

// ---------------------------------------------------------------------------
// tangent walk, shared by the in-block and the global merge
// ---------------------------------------------------------------------------
// Acc provides lo/hi/prv/nxt get+set per chunk and point(side, chunk, k).
template <class Acc>
__device__ void merge_walk(Acc &A, int side, int fa, int la, int fb, int lb)
{
    int ca = la, ka = A.hi(side, ca);
    int cb = fb, kb = A.lo(side, cb);
    int loa = A.lo(side, ca), hib = A.hi(side, cb);
    float2 pa = A.point(side, ca, ka);
    float2 pb = A.point(side, cb, kb);
    for (;;) {
        bool moved = false;
        for (;;) {   // advance b
            int nc = cb, nk = kb + 1, nhi = hib;
            if (kb >= hib) {
                if (cb == lb) break;
                nc = A.nxt(side, cb);
                nk = A.lo(side, nc);
                nhi = A.hi(side, nc);
            }
            const float2 q = A.point(side, nc, nk);
            if (!drop(side, pa, pb, q)) break;
            if (nc != cb) {   // chunk cb is now entirely removed
                A.set_range(side, cb, 1, 0);
                cb = nc;
                hib = nhi;
            }
            kb = nk;
            pb = q;
            moved = true;
        }
        for (;;) {   // retreat a
            int pc = ca, pk = ka - 1, plo = loa;
            if (ka <= loa) {
                if (ca == fa) break;
                pc = A.prv(side, ca);
                plo = A.lo(side, pc);
                pk = A.hi(side, pc);
            }
            const float2 q = A.point(side, pc, pk);
            if (!drop(side, q, pa, pb)) break;
            if (pc != ca) {
                A.set_range(side, ca, 1, 0);
                ca = pc;
                loa = plo;
            }
            ka = pk;
            pa = q;
            moved = true;
        }
        if (!moved) break;
    }
    A.set_hi(side, ca, ka);
    A.set_lo(side, cb, kb);
    A.link(side, ca, cb);
}

// ---------------------------------------------------------------------------
// in-block state; one side (lower or upper) is processed at a time
// ---------------------------------------------------------------------------
struct ChainSmem {
    float2 pts[NL];               // staged points; [SC], [SC+1]: look-ahead lowest / highest
    uint16_t list[3][NL];         // run starts, sequences and elimination ping-pong
    uint8_t stk[LWMAX * LT];      // leaf stacks: entry j of leaf t at [j * LT + t]
    int16_t lb[LT];               // leaf t's first entry in the flat list array
    int16_t lo[LT], hi[LT], prv[LT], nxt[LT], first[LT], last[LT];
    uint32_t wsum[LT / 32];
    uint32_t total;
    float red_y[2][LT / 32];      // look-ahead reduction scratch
    uint32_t red_q[2][LT / 32];
    uint32_t ext_pos[2];          // global positions of the look-ahead lowest / highest
    float prev_x;
    int has_prev;
    int seq_len;
    int wcur, wdone;              // single-warp passes: buffer and convergence
};

// leaf c's entries start at flat[lb[c]]; its stack holds offsets from there
struct SmemAcc {
    ChainSmem &s;
    const uint16_t *flat;
    __device__ int lo(int, int c) const { return s.lo[c]; }
    __device__ int hi(int, int c) const { return s.hi[c]; }
    __device__ int prv(int, int c) const { return s.prv[c]; }
    __device__ int nxt(int, int c) const { return s.nxt[c]; }
    __device__ void set_range(int, int c, int l, int h) const
    {
        s.lo[c] = (int16_t)l;
        s.hi[c] = (int16_t)h;
    }
    __device__ void set_lo(int, int c, int l) const { s.lo[c] = (int16_t)l; }
    __device__ void set_hi(int, int c, int h) const { s.hi[c] = (int16_t)h; }
    __device__ void link(int, int a, int b) const
    {
        s.nxt[a] = (int16_t)b;
        s.prv[b] = (int16_t)a;
    }
    __device__ float2 point(int, int c, int k) const { return s.pts[flat[s.lb[c] + s.stk[k * LT + c]]]; }
};

// Exclusive scan of one count per thread over the block; the total goes to
// s.total.  Contains two barriers.
__device__ __forceinline__ uint32_t block_scan(ChainSmem &s, uint32_t v)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s.wsum[warp] = incl;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < LT / 32; ++w) {
        const uint32_t u = s.wsum[w];
        if (w < warp) before += u;
        total += u;
    }
    if (t == 0) s.total = total;
    __syncthreads();
    return before + incl - v;
}

// Stable compaction of positions [0, count).  Warp w owns the segment
// [w*S, w*S + S) and walks it 32 consecutive positions at a time, so lanes
// touch consecutive entries (no bank conflicts); keep(j) decides, out
// receives src(j) for the kept j.  Returns the number kept (all threads).
template <class Keep, class Src>
__device__ __forceinline__ int block_compact(ChainSmem &s, int count, Keep keep, Src src, uint16_t *out)
{
    constexpr int NWARP = LT / 32;
    constexpr int MAXC = (NL + NWARP * 32 - 1) / (NWARP * 32) + 1;   // 32-position chunks per warp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int S = (((count + NWARP - 1) / NWARP) + 31) & ~31;   // segment, a multiple of 32
    const int j0 = warp * S;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t masks[MAXC];
    int n = 0;
#pragma unroll
    for (int c = 0; c < MAXC; ++c) {
        uint32_t m = 0;
        if (c * 32 < S) {
            const int j = j0 + c * 32 + lane;
            m = __ballot_sync(0xffffffffu, j < count && keep(j));
        }
        masks[c] = m;
        n += __popc(m);
    }
    if (lane == 0) s.wsum[warp] = (uint32_t)n;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < NWARP; ++w) {
        const uint32_t u = s.wsum[w];
        if (w < warp) before += u;
        total += u;
    }
    uint32_t o = before;
#pragma unroll
    for (int c = 0; c < MAXC; ++c) {
        const uint32_t m = masks[c];
        if ((m >> lane) & 1u) out[o + __popc(m & lt)] = src(j0 + c * 32 + lane);
        o += __popc(m);
    }
    __syncthreads();
    return (int)total;
}

// ---------------------------------------------------------------------------
// global state (one "chunk" = one super-chunk)
// ---------------------------------------------------------------------------
struct ChainPtrs {
    const uint32_t *keys;             // sorted ord(x)
    const unsigned long long *pay;    // sorted ord(y) << 32 | index
    uint32_t *pos[2];                 // chain vertices: sorted positions, super-chunk c at [c * CS, ...)
    float2 *pt[2];                    // chain vertices: coordinates
    int32_t *lo[2], *hi[2], *prv[2], *nxt[2];
    int32_t *node;                    // 4 ints per tree node: firstL lastL firstU lastU
    int32_t *node_cnt;                // arrivals per node (zeroed at the start of each call)
};

__device__ __forceinline__ ChainPtrs chain_ptrs(void *ws, const Layout &L, uint32_t buf)
{
    ChainPtrs P;
    P.keys = at<uint32_t>(ws, L.keys[buf]);
    P.pay = at<unsigned long long>(ws, L.pay[buf]);
    for (int side = 0; side < 2; ++side) {
        P.pos[side] = at<uint32_t>(ws, L.chain_pos[side]);
        P.pt[side] = at<float2>(ws, L.chain_pt[side]);
    }
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

__device__ __forceinline__ float2 sorted_point(const ChainPtrs &P, int64_t q)
{
    return make_float2(key_float(__ldg(P.keys + q)), key_float((uint32_t)(__ldg(P.pay + q) >> 32)));
}

// Values written by other blocks are read through L2 (ld.cg): this
// thread's L1 may hold stale lines.
struct GlobalAcc {
    const ChainPtrs &P;
    __device__ int lo(int side, int c) const { return __ldcg(P.lo[side] + c); }
    __device__ int hi(int side, int c) const { return __ldcg(P.hi[side] + c); }
    __device__ int prv(int side, int c) const { return __ldcg(P.prv[side] + c); }
    __device__ int nxt(int side, int c) const { return __ldcg(P.nxt[side] + c); }
    __device__ void set_range(int side, int c, int l, int h) const
    {
        P.lo[side][c] = l;
        P.hi[side][c] = h;
    }
    __device__ void set_lo(int side, int c, int l) const { P.lo[side][c] = l; }
    __device__ void set_hi(int side, int c, int h) const { P.hi[side][c] = h; }
    __device__ void link(int side, int a, int b) const
    {
        P.nxt[side][a] = b;
        P.prv[side][b] = a;
    }
    __device__ float2 point(int side, int c, int k) const { return __ldcg(P.pt[side] + (int64_t)c * CS + k); }
};

// first / last live super-chunk (absolute index) of tree node (level, j)
// of a tree whose leaves are super-chunks coff + 0 .. and whose nodes start
// at node noff; level 0 = super-chunk coff + j
__device__ __forceinline__ void node_ends(const ChainPtrs &P, int level, int64_t coff, int64_t noff, int64_t nb,
                                          int64_t j, int side, int32_t &first, int32_t &last)
{
    if (level == 0) {
        const bool live = __ldcg(P.hi[side] + coff + j) >= __ldcg(P.lo[side] + coff + j);
        first = last = live ? (int32_t)(coff + j) : -1;
    } else {
        first = __ldcg(P.node + (noff + nb + j) * 4 + 2 * side);
        last = __ldcg(P.node + (noff + nb + j) * 4 + 2 * side + 1);
    }
}

// Climb the merge tree of one set from its super-chunk c (0 <= c < nsc;
// leaves at coff, nodes at noff): the second child to arrive at a node
// merges its two children and continues upward.
__device__ void climb(const ChainPtrs &P, int64_t c, int64_t nsc, int64_t coff, int64_t noff)
{
    GlobalAcc G{P};
    int64_t node = c, w = nsc, nb_child = 0, nb = 0;   // nb: base of the level above
    int level = 0;
    while (w > 1) {
        const int64_t parent = node >> 1, pw = (w + 1) / 2;
        const int64_t sib = node ^ 1;
        int32_t rec[4];
        if (sib >= w) {
#pragma unroll
            for (int side = 0; side < 2; ++side)
                node_ends(P, level, coff, noff, nb_child, node, side, rec[2 * side], rec[2 * side + 1]);
        } else {
            __threadfence();
            if (atomicAdd(P.node_cnt + noff + nb + parent, 1) == 0) return;   // first to arrive: the sibling merges
            __threadfence();
            const int64_t a = parent * 2, b = a + 1;
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                int32_t fa, la, fb, lb;
                node_ends(P, level, coff, noff, nb_child, a, side, fa, la);
                node_ends(P, level, coff, noff, nb_child, b, side, fb, lb);
                if (la < 0) {
                    rec[2 * side] = fb;
                    rec[2 * side + 1] = lb;
                } else if (fb < 0) {
                    rec[2 * side] = fa;
                    rec[2 * side + 1] = la;
                } else {
                    merge_walk(G, side, fa, la, fb, lb);
                    rec[2 * side] = fa;
                    rec[2 * side + 1] = lb;
                }
            }
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) P.node[(noff + nb + parent) * 4 + f] = rec[f];
        node = parent;
        nb_child = nb;
        nb += pw;
        w = pw;
        ++level;
    }
}

// Block reduction of (y, position) pairs: the lowest (highest) y, ties to the
// lowest position.  Contains two barriers.
__device__ __forceinline__ void block_extreme_y(ChainSmem &s, float ylo, uint32_t qlo, float yhi, uint32_t qhi,
                                                float &out_ylo, uint32_t &out_qlo, float &out_yhi, uint32_t &out_qhi)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float y1 = __shfl_xor_sync(0xffffffffu, ylo, o);
        const uint32_t q1 = __shfl_xor_sync(0xffffffffu, qlo, o);
        if (y1 < ylo || (y1 == ylo && q1 < qlo)) {
            ylo = y1;
            qlo = q1;
        }
        const float y2 = __shfl_xor_sync(0xffffffffu, yhi, o);
        const uint32_t q2 = __shfl_xor_sync(0xffffffffu, qhi, o);
        if (y2 > yhi || (y2 == yhi && q2 < qhi)) {
            yhi = y2;
            qhi = q2;
        }
    }
    if (lane == 0) {
        s.red_y[0][warp] = ylo;
        s.red_q[0][warp] = qlo;
        s.red_y[1][warp] = yhi;
        s.red_q[1][warp] = qhi;
    }
    __syncthreads();
    out_ylo = s.red_y[0][0];
    out_qlo = s.red_q[0][0];
    out_yhi = s.red_y[1][0];
    out_qhi = s.red_q[1][0];
    for (int w = 1; w < LT / 32; ++w) {
        if (s.red_y[0][w] < out_ylo || (s.red_y[0][w] == out_ylo && s.red_q[0][w] < out_qlo)) {
            out_ylo = s.red_y[0][w];
            out_qlo = s.red_q[0][w];
        }
        if (s.red_y[1][w] > out_yhi || (s.red_y[1][w] == out_yhi && s.red_q[1][w] < out_qhi)) {
            out_yhi = s.red_y[1][w];
            out_qhi = s.red_q[1][w];
        }
    }
    __syncthreads();
}

// The chains of one super-chunk: sorted positions [base, base + m) of a set
// occupying [sbeg, send); results go to chain slot j.  Called by all
// threads of the block.
__device__ void superchunk(ChainSmem &sm, const ChainPtrs &P, int64_t j, int64_t base, int m, int64_t sbeg,
                           int64_t send)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const float kInf = __int_as_float(0x7f800000);
    const int64_t sc = j;
    {
        // ---- stage the super-chunk (coalesced), decoded to points
        for (int i = t; i < m; i += LT) sm.pts[i] = sorted_point(P, base + i);
        if (t == 0) {
            sm.has_prev = base > sbeg;
            sm.prev_x = base > sbeg ? key_float(__ldg(P.keys + base - 1)) : 0.0f;
        }
        __syncthreads();

        // ---- runs of equal x that start in this super-chunk
        const int R = block_compact(
            sm, m,
            [&](int i) {
                return i == 0 ? !(sm.has_prev && sm.pts[0].x == sm.prev_x) : sm.pts[i].x != sm.pts[i - 1].x;
            },
            [](int i) { return (uint16_t)i; }, sm.list[2]);
        if (R == 0) {   // the whole super-chunk continues an earlier run
            if (t == 0)
                for (int side = 0; side < 2; ++side) {
                    P.lo[side][sc] = 0;
                    P.hi[side][sc] = -1;
                }
            __syncthreads();
            return;
        }
        // ---- look ahead when the last run continues past the super-chunk
        const float xr = sm.pts[m - 1].x;
        const bool ext = base + m < send && key_float(__ldg(P.keys + base + m)) == xr;
        int64_t run_end = base + m;
        if (ext) {
            float ylo = kInf, yhi = -kInf;
            uint32_t qlo = 0xffffffffu, qhi = 0xffffffffu;
            for (int64_t q0 = base + m;; q0 += LT) {
                const int64_t q = q0 + t;
                const bool in_run = q < send && key_float(__ldg(P.keys + q)) == xr;
                if (in_run) {
                    const float y = key_float((uint32_t)(__ldg(P.pay + q) >> 32));
                    if (y < ylo || (y == ylo && (uint32_t)q < qlo)) {
                        ylo = y;
                        qlo = (uint32_t)q;
                    }
                    if (y > yhi || (y == yhi && (uint32_t)q < qhi)) {
                        yhi = y;
                        qhi = (uint32_t)q;
                    }
                }
                // the keys are sorted, so the run's positions are contiguous
                const int n_in = __syncthreads_count(in_run);
                if (n_in < LT) {
                    run_end = q0 + n_in;
                    break;
                }
            }
            float oyl, oyh;
            uint32_t oql, oqh;
            block_extreme_y(sm, ylo, qlo, yhi, qhi, oyl, oql, oyh, oqh);
            if (t == 0) {
                sm.pts[SC] = make_float2(xr, oyl);
                sm.pts[SC + 1] = make_float2(xr, oyh);
                sm.ext_pos[0] = oql;
                sm.ext_pos[1] = oqh;
            }
        }
        const bool holds_last = run_end == send;
        __syncthreads();
        // ---- representatives: lowest (list[0]) and highest (list[1]) point of each run
        for (int k = t; k < R; k += LT) {
            const int r0 = sm.list[2][k];
            const int r1 = k + 1 < R ? sm.list[2][k + 1] : m;
            int lo = r0, hi = r0;
            float ylo = sm.pts[r0].y, yhi = ylo;
            for (int i = r0 + 1; i < r1; ++i) {
                const float y = sm.pts[i].y;
                if (y < ylo) {
                    ylo = y;
                    lo = i;
                }
                if (y > yhi) {
                    yhi = y;
                    hi = i;
                }
            }
            if (k == R - 1 && ext) {
                if (sm.pts[SC].y < ylo) lo = SC;
                if (sm.pts[SC + 1].y > yhi) hi = SC + 1;
            }
            sm.list[0][k] = (uint16_t)lo;
            sm.list[1][k] = (uint16_t)hi;
        }
        __syncthreads();
        const uint16_t first_lo = sm.list[0][0];
        const bool first_two = base == sbeg && sm.pts[sm.list[1][0]].y > sm.pts[first_lo].y;

        for (int side = 0; side < 2; ++side) {
            // ---- this side's sequence in list[0]
            if (side == 0) {
                // lowest of every run, then the highest of the very last run
                if (t == 0) {
                    int len = R;
                    if (holds_last && sm.pts[sm.list[1][R - 1]].y > sm.pts[sm.list[0][R - 1]].y)
                        sm.list[0][len++] = sm.list[1][R - 1];
                    sm.seq_len = len;
                }
            } else {
                // the lowest of the very first run, then the highest of every run
                const int off = first_two ? 1 : 0;
                for (int k = t; k < R; k += LT) sm.list[0][k + off] = sm.list[1][k];
                if (t == 0) {
                    if (first_two) sm.list[0][0] = first_lo;
                    sm.seq_len = R + off;
                }
            }
            __syncthreads();
            const int len = sm.seq_len;
            // ---- per warp: its share of the sequence, [warp * S, warp * S + S)
            const int S = (len + NWB - 1) / NWB;
            int w0 = warp * S;
            int wl = max(0, min(S, len - w0));   // this warp's live length
            uint16_t *flat = &sm.list[0][0];
            int cur = 0;                          // 0: list[0], 2: list[2]
            // elimination passes over the warp's segment; its two ends stay
            for (int pass = 0; pass < kElimPasses && wl > 2; ++pass) {
                const int kept = warp_elim_pass(sm.pts, flat + cur * NL + w0, flat + (2 - cur) * NL + w0, wl, side,
                                                lane, lt);
                cur = 2 - cur;
                const bool done = kept == wl;
                wl = kept;
                if (done) break;
            }
            // ---- block level: the warps' survivors concatenated in list[2],
            // then passes over the whole sequence.  A sequence whose every
            // turn is strict is its own chain: no leaves, no merges.
            if (cur == 2)
                for (int i = lane; i < wl; i += 32) flat[w0 + i] = flat[2 * NL + w0 + i];
            if (lane == 0) sm.wsum[warp] = (uint32_t)wl;
            __syncthreads();
            {
                int off = 0, tot = 0;
#pragma unroll
                for (int w = 0; w < NWB; ++w) {
                    const int u = (int)sm.wsum[w];
                    if (w < warp) off += u;
                    tot += u;
                }
                for (int i = lane; i < wl; i += 32) flat[2 * NL + off + i] = flat[w0 + i];
                __syncthreads();
                int blen = tot, bcur = 2;
                bool chain_done = blen <= 2;
                // long: all threads, block-wide compaction
                for (int bp = 0; bp < kBlockElimPasses && !chain_done && blen > kWarpSeqMax; ++bp) {
                    const uint16_t *src = flat + bcur * NL;
                    const int bl = blen;
                    const int kept = block_compact(
                        sm, bl,
                        [&](int j) {
                            return j == 0 || j == bl - 1 ||
                                   !drop(side, sm.pts[src[j - 1]], sm.pts[src[j]], sm.pts[src[j + 1]]);
                        },
                        [&](int j) { return src[j]; }, flat + (2 - bcur) * NL);
                    bcur = 2 - bcur;
                    chain_done = kept == bl || kept <= 2;
                    blen = kept;
                }
                if (!chain_done && blen <= kWarpSeqMax) {
                    // short: one warp runs the passes, no block barriers
                    if (warp == 0) {
                        int bl = blen, wc = bcur, done = 0;
                        for (int bp = 0; bp < kBlockElimPasses && !done; ++bp) {
                            const int kept =
                                warp_elim_pass(sm.pts, flat + wc * NL, flat + (2 - wc) * NL, bl, side, lane, lt);
                            wc = 2 - wc;
                            done = kept == bl || kept <= 2;
                            bl = kept;
                        }
                        if (lane == 0) {
                            sm.seq_len = bl;
                            sm.wcur = wc;
                            sm.wdone = done;
                        }
                    }
                    __syncthreads();
                    blen = sm.seq_len;
                    bcur = sm.wcur;
                    chain_done = sm.wdone != 0;
                }
                if (chain_done) {   // write the chain and go to the other side
                    uint32_t *dpos = P.pos[side] + sc * CS;
                    float2 *dpt = P.pt[side] + sc * CS;
                    for (int q = t; q < blen; q += LT) {
                        const int e = flat[bcur * NL + q];
                        dpos[q] = e < SC ? (uint32_t)(base + e) : sm.ext_pos[e - SC];
                        dpt[q] = sm.pts[e];
                    }
                    if (t == 0) {
                        P.lo[side][sc] = 0;
                        P.hi[side][sc] = blen - 1;
                    }
                    __syncthreads();
                    continue;
                }
                // not yet a chain: leaves and merges over the block's sequence
                const int S2 = (blen + NWB - 1) / NWB;
                w0 = warp * S2;
                wl = max(0, min(S2, blen - w0));
                cur = bcur;
            }
            // ---- leaf chains: lane l takes [l * LW, l * LW + LW) of the warp's list
            const int LW = (wl + 31) / 32;
            const int lbase = cur * NL + w0 + lane * LW;
            const int cnt = max(0, min(LW, wl - lane * LW));
            sm.lb[t] = (int16_t)lbase;
            int h = 0;
            float2 t1 = make_float2(0.0f, 0.0f), t2 = t1;   // top and second of the stack
            for (int k = 0; k < cnt; ++k) {
                const float2 p = sm.pts[flat[lbase + k]];
                while (h >= 2 && drop(side, t2, t1, p)) {
                    --h;
                    t1 = t2;
                    if (h >= 2) t2 = sm.pts[flat[lbase + sm.stk[(h - 2) * LT + t]]];
                }
                sm.stk[h * LT + t] = (uint8_t)k;
                ++h;
                t2 = t1;
                t1 = p;
            }
            sm.lo[t] = 0;
            sm.hi[t] = (int16_t)(h - 1);
            sm.first[t] = sm.last[t] = (int16_t)(h > 0 ? t : -1);
            __syncwarp();
            // ---- merge tree: five levels inside the warp, then three across warps
            SmemAcc A{sm, flat};
            for (int w = 1; w < 32; w *= 2) {
                if (lane < 32 / (2 * w)) {
                    const int a0 = warp * 32 + 2 * lane * w, b0 = a0 + w;
                    const int fa = sm.first[a0], la = sm.last[a0];
                    const int fb = sm.first[b0], lb = sm.last[b0];
                    if (la >= 0 && fb >= 0) merge_walk(A, side, fa, la, fb, lb);
                    sm.first[a0] = (int16_t)(la >= 0 ? fa : fb);
                    sm.last[a0] = (int16_t)(fb >= 0 ? lb : la);
                }
                __syncwarp();
            }
            __syncthreads();
            for (int w = 32; w < LT; w *= 2) {
                if (t < LT / (2 * w)) {
                    const int a0 = 2 * t * w, b0 = a0 + w;
                    const int fa = sm.first[a0], la = sm.last[a0];
                    const int fb = sm.first[b0], lb = sm.last[b0];
                    if (la >= 0 && fb >= 0) merge_walk(A, side, fa, la, fb, lb);
                    sm.first[a0] = (int16_t)(la >= 0 ? fa : fb);
                    sm.last[a0] = (int16_t)(fb >= 0 ? lb : la);
                }
                __syncthreads();
            }

            // ---- write the super-chunk's chain contiguously
            const int l = sm.lo[t], hh = sm.hi[t];
            const int c = hh >= l ? hh - l + 1 : 0;
            const int off = (int)block_scan(sm, (uint32_t)c);
            uint32_t *dpos = P.pos[side] + sc * CS + off;
            float2 *dpt = P.pt[side] + sc * CS + off;
            for (int q = 0; q < c; ++q) {
                const int e = flat[lbase + sm.stk[(l + q) * LT + t]];
                dpos[q] = e < SC ? (uint32_t)(base + e) : sm.ext_pos[e - SC];
                dpt[q] = sm.pts[e];
            }
            if (t == 0) {
                P.lo[side][sc] = 0;
                P.hi[side][sc] = (int)sm.total - 1;
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(LT) chain_kernel(void *ws, Layout L)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ChainSmem &sm = *reinterpret_cast<ChainSmem *>(smem_raw);
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    const Octagon *oct = at<Octagon>(ws, L.oct);
    const uint32_t s = hull_stage_count(ctrl, oct);
    if (s == 0) return;
    const ChainPtrs P = chain_ptrs(ws, L, ctrl->final_buf);
    const int64_t nsc = ceil_div((int64_t)s, SC);
    for (int64_t sc = blockIdx.x; sc < nsc; sc += gridDim.x) {
        // the block's next super-chunk streams into L2 meanwhile
        const int64_t nxt = sc + gridDim.x;
        if (threadIdx.x == 0 && nxt < nsc) {
            const uint32_t nn = (uint32_t)min((int64_t)SC, (int64_t)s - nxt * SC);
            bulk_prefetch_l2(P.keys + nxt * SC, (nn * 4u) & ~15u);
            bulk_prefetch_l2(P.pay + nxt * SC, (nn * 8u) & ~15u);
        }
        superchunk(sm, P, sc, sc * SC, (int)min((int64_t)SC, (int64_t)s - sc * SC), 0, s);
    }
}

// Global merge tree over the super-chunks: one thread per super-chunk
// climbs; the second child to reach a node merges the pair.
__global__ void __launch_bounds__(32) chain_merge_kernel(void *ws, Layout L)
{
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    const Octagon *oct = at<Octagon>(ws, L.oct);
    const uint32_t s = hull_stage_count(ctrl, oct);
    if (s == 0) return;
    const ChainPtrs P = chain_ptrs(ws, L, ctrl->final_buf);
    const int64_t nsc = ceil_div((int64_t)s, SC);
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nsc) climb(P, c, nsc, 0, 0);
}

// ---- many sets: super-chunks never span two sets; each set has its own
// merge tree; the sorted arrays end up in buffer 0 (four passes)
__global__ void __launch_bounds__(LT) bx_chain_kernel(void *ws, Layout L, BatchLayout BL)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ChainSmem &sm = *reinterpret_cast<ChainSmem *>(smem_raw);
    const BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    if (bc->abort) return;
    const SetInfo *sets = at<SetInfo>(ws, BL.sets);
    const uint32_t *sc_set = at<uint32_t>(ws, BL.sc_set);
    const ChainPtrs P = chain_ptrs(ws, L, 0);
    const int64_t nsc = bc->nsc;
    for (int64_t j = blockIdx.x; j < nsc; j += gridDim.x) {
        const uint32_t b = sc_set[j];
        const int64_t sb = (int64_t)sets[b].surv_base, n = sets[b].s;
        const int64_t local = j - sets[b].sc_base;
        superchunk(sm, P, j, sb + local * SC, (int)min((int64_t)SC, n - local * SC), sb, sb + n);
    }
}

__global__ void __launch_bounds__(32) bx_merge_kernel(void *ws, Layout L, BatchLayout BL)
{
    const BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    if (bc->abort) return;
    const SetInfo *sets = at<SetInfo>(ws, BL.sets);
    const uint32_t *sc_set = at<uint32_t>(ws, BL.sc_set);
    const ChainPtrs P = chain_ptrs(ws, L, 0);
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= (int64_t)bc->nsc) return;
    const uint32_t b = sc_set[j];
    climb(P, j - sets[b].sc_base, sets[b].nsc, sets[b].sc_base, sets[b].node_base);
}

// Compacts the live chain ranges of super-chunks [0, nc): thread =
// super-chunk, look-back over tiles of super-chunks, then the whole block
// copies the tile's ranges (the original indices: low half of the payload),
// each thread finding the super-chunk of an output position by binary
// search over the tile's offsets.  Side 0 goes to out0, side 1 to out1.
// With sc_off, each super-chunk's output offset per side is recorded too
// (sc_off[side][nc] = side total).
// copy = false: only the offsets (sc_off required); emit_copy_kernel then
// writes the ranges with the whole grid.
struct EmitArgs {
    uint32_t *out[2];
    uint32_t *sc_off[2];
    uint32_t *ticket;
    uint32_t *h_total[2];
    bool copy;
};

__device__ void emit_body(void *ws, const Layout &L, const ChainPtrs &P, int64_t nc, uint64_t s, const EmitArgs &E)
{
    const int64_t ntiles = ceil_div(nc, kEmitThreads);
    unsigned long long *status[2] = {at<unsigned long long>(ws, L.emit_status[0]),
                                     at<unsigned long long>(ws, L.emit_status[1])};
    constexpr int NW = kEmitThreads / 32;
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_wsum[2][NW];
    __shared__ unsigned long long s_excl[2];
    __shared__ uint32_t s_rel[2][kEmitThreads];   // offset of each super-chunk's range in the tile's output
    __shared__ int32_t s_lo[2][kEmitThreads];     // and its first chain slot
    __shared__ uint32_t s_tot[2];
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(E.ticket, 1u);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= ntiles) break;
        const int64_t c = tile * kEmitThreads + tid;
        int32_t lo[2] = {0, 0}, cnt[2] = {0, 0};
        if (c < nc) {
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                lo[side] = __ldcg(P.lo[side] + c);
                const int32_t hi = __ldcg(P.hi[side] + c);
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
                s_tot[side] = total;
                if (tile == ntiles - 1) {
                    *E.h_total[side] = (uint32_t)(excl + total);
                    if (E.sc_off[side]) E.sc_off[side][nc] = (uint32_t)(excl + total);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const uint32_t rel = s_wsum[side][warp] + pre[side];
            s_rel[side][tid] = rel;
            s_lo[side][tid] = lo[side];
            if (E.sc_off[side] && c < nc) E.sc_off[side][c] = (uint32_t)(s_excl[side] + rel);
        }
        __syncthreads();
        if (!E.copy) continue;   // (the loop's first barrier orders the next tile's shared writes)
        constexpr int B4 = 4;   // output positions per thread in flight
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const uint32_t T = s_tot[side];
            const uint64_t excl = s_excl[side];
            uint32_t *out = E.out[side];
            const uint32_t *chain = P.pos[side];
            for (uint32_t k0 = 0; k0 < T; k0 += B4 * kEmitThreads) {
                uint32_t sp[B4];
#pragma unroll
                for (int u = 0; u < B4; ++u) {
                    const uint32_t k = k0 + u * kEmitThreads + tid;
                    sp[u] = 0u;
                    if (k < T) {
                        // the last super-chunk whose range starts at or before k
                        // (empty ranges share their start with the next one)
                        int lo_j = 0, hi_j = kEmitThreads - 1;
                        while (lo_j < hi_j) {
                            const int mid = (lo_j + hi_j + 1) >> 1;
                            if (s_rel[side][mid] <= k) lo_j = mid;
                            else hi_j = mid - 1;
                        }
                        const int64_t ci = tile * kEmitThreads + lo_j;
                        sp[u] = __ldcg(chain + ci * CS + s_lo[side][lo_j] + (k - s_rel[side][lo_j]));
                    }
                }
#pragma unroll
                for (int u = 0; u < B4; ++u) {
                    const uint32_t k = k0 + u * kEmitThreads + tid;
                    if (k < T && excl + k < (uint64_t)s) out[excl + k] = (uint32_t)__ldg(P.pay + sp[u]);
                }
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kEmitThreads) emit_kernel(void *ws, Layout L, uint32_t *hull_idx)
{
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    const Octagon *oct = at<Octagon>(ws, L.oct);
    const uint32_t s = hull_stage_count(ctrl, oct);
    if (s == 0) return;
    const ChainPtrs P = chain_ptrs(ws, L, ctrl->final_buf);
    EmitArgs E{{hull_idx, at<uint32_t>(ws, L.utmp)},
               {at<uint32_t>(ws, L.emit_off[0]), at<uint32_t>(ws, L.emit_off[1])},
               &ctrl->emit_ticket[0],
               {&ctrl->h_lower, &ctrl->h_upper},
               false};
    emit_body(ws, L, P, ceil_div((int64_t)s, SC), s, E);
}

// The chains' surviving ranges into the outputs (lower chain to hull_idx,
// upper chain to utmp: original indices, the low half of the payload),
// every thread of the grid on its own output positions: the super-chunk
// of position k is the last one whose offset (emit_off) is at most k
// (binary search; an empty range shares its offset with the next one).
// A hull with many vertices on few super-chunks (the unit circle after
// the fan: about 2000 per super-chunk) is no longer copied by one block.
__global__ void __launch_bounds__(kEmitThreads) emit_copy_kernel(void *ws, Layout L, uint32_t *hull_idx)
{
    const Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    const Octagon *oct = at<Octagon>(ws, L.oct);
    const uint32_t s = hull_stage_count(ctrl, oct);
    if (s == 0) return;
    const ChainPtrs P = chain_ptrs(ws, L, ctrl->final_buf);
    const int32_t nc = (int32_t)ceil_div((int64_t)s, SC);
    const uint32_t gtid = blockIdx.x * kEmitThreads + threadIdx.x, gthreads = gridDim.x * kEmitThreads;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const uint32_t T = side ? ctrl->h_upper : ctrl->h_lower;
        const uint32_t *off = at<uint32_t>(ws, L.emit_off[side]);
        uint32_t *out = side ? at<uint32_t>(ws, L.utmp) : hull_idx;
        for (uint32_t k = gtid; k < T && k < s; k += gthreads) {
            int lo_j = 0, hi_j = nc - 1;
            while (lo_j < hi_j) {
                const int mid = (lo_j + hi_j + 1) >> 1;
                if (__ldg(off + mid) <= k) lo_j = mid;
                else hi_j = mid - 1;
            }
            const uint32_t sp =
                __ldcg(P.pos[side] + (int64_t)lo_j * CS + __ldcg(P.lo[side] + lo_j) + (k - __ldg(off + lo_j)));
            out[k] = (uint32_t)__ldg(P.pay + sp);
        }
    }
}

// all sets at once: lower chains to the batch's lower array, upper chains
// to utmp, each set's part delimited by the per-super-chunk offsets
__global__ void __launch_bounds__(kEmitThreads) bx_emit_kernel(void *ws, Layout L, BatchLayout BL)
{
    BatchCtrl *bc = at<BatchCtrl>(ws, BL.bctrl);
    if (bc->abort) return;
    const int64_t nc = bc->nsc;
    if (nc == 0) return;
    const ChainPtrs P = chain_ptrs(ws, L, 0);
    EmitArgs E{{at<uint32_t>(ws, BL.lower), at<uint32_t>(ws, L.utmp)},
               {at<uint32_t>(ws, BL.sc_off[0]), at<uint32_t>(ws, BL.sc_off[1])},
               &bc->emit_ticket,
               {&bc->h_lower, &bc->h_upper},
               true};
    emit_body(ws, L, P, nc, (uint64_t)L.n, E);
}

// hull = lower chain, then the upper chain reversed without its two ends
__global__ void finish_kernel(void *ws, Layout L, uint32_t *hull_idx, uint32_t *hull_count)
{
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    if (ctrl->small_done) return;
    const uint32_t hl = ctrl->h_lower, hu = ctrl->h_upper;
    const uint32_t mid = hu >= 2 ? hu - 2 : 0;
    const uint32_t *utmp = at<uint32_t>(ws, L.utmp);
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < mid; m += gthreads)
        if (hl + m < L.n) hull_idx[hl + m] = utmp[hu - 2 - m];
    if (blockIdx.x == 0 && threadIdx.x == 0) *hull_count = hl == 0 ? 0u : hl + mid;
}

// Few survivors (at most kSmallHull): one block sorts them by (x, y, index)
// in shared memory (bitonic network over the packed keys and indices),
// then one thread runs Andrew's monotone chain over them -- equal points
// collapse to the first, a turn that is not strictly counter-clockwise
// (exact sign) pops the middle point -- and writes the hull, counter-
// clockwise from the first point; the sort and chain kernels launched
// after it then stop at once.  More survivors: it does nothing.
constexpr int kSmallHull = 512;
constexpr int kSmallThreads = 256;

__global__ void __launch_bounds__(kSmallThreads) small_hull_kernel(void *ws, Layout L, uint32_t *hull_idx,
                                                                   uint32_t *hull_count)
{
    Ctrl *ctrl = at<Ctrl>(ws, L.ctrl);
    const Octagon *oct = at<Octagon>(ws, L.oct);
    const uint32_t s = hull_stage_count(ctrl, oct);
    if (s == 0 || s > (uint32_t)kSmallHull) return;
    __shared__ unsigned long long sk[kSmallHull];   // ord(x) << 32 | ord(y)
    __shared__ uint32_t si[kSmallHull];             // point index
    __shared__ uint16_t st[2 * kSmallHull + 2];     // chain stack: sorted positions
    const uint32_t *keys = at<uint32_t>(ws, L.keys[ctrl->sort_in]);
    const unsigned long long *pay = at<unsigned long long>(ws, L.pay[ctrl->sort_in]);
    uint32_t m = 32;
    while (m < s) m <<= 1;
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
        if (i < s) {
            const unsigned long long pv = pay[i];
            sk[i] = ((unsigned long long)keys[i] << 32) | (pv >> 32);
            si[i] = (uint32_t)pv;
        } else {
            sk[i] = ~0ull;   // after every point
            si[i] = ~0u;
        }
    }
    __syncthreads();
    for (uint32_t k = 2; k <= m; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
                const uint32_t l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const bool gt = sk[i] > sk[l] || (sk[i] == sk[l] && si[i] > si[l]);
                    if (gt == up) {
                        const unsigned long long tk = sk[i];
                        sk[i] = sk[l];
                        sk[l] = tk;
                        const uint32_t ti = si[i];
                        si[i] = si[l];
                        si[l] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x != 0) return;
    // equal points: the first (lowest index) stays
    uint32_t u = 0;
    for (uint32_t i = 0; i < s; ++i) {
        if (u > 0 && sk[i] == sk[u - 1]) continue;
        sk[u] = sk[i];
        si[u] = si[i];
        ++u;
    }
    auto px = [&](uint32_t k) { return key_float((uint32_t)(sk[k] >> 32)); };
    auto py = [&](uint32_t k) { return key_float((uint32_t)sk[k]); };
    uint32_t h = 0;
    if (u == 1) {
        hull_idx[0] = si[0];
        h = 1;
    } else {
        for (uint32_t k = 0; k < u; ++k) {   // lower chain, left to right
            while (h >= 2 && orient(px(st[h - 2]), py(st[h - 2]), px(st[h - 1]), py(st[h - 1]), px(k), py(k)) <= 0)
                --h;
            st[h++] = (uint16_t)k;
        }
        const uint32_t base = h + 1;
        for (int k = (int)u - 2; k >= 0; --k) {   // upper chain, right to left
            while (h >= base && orient(px(st[h - 2]), py(st[h - 2]), px(st[h - 1]), py(st[h - 1]), px(k), py(k)) <= 0)
                --h;
            st[h++] = (uint16_t)k;
        }
        --h;   // the last point is the first again
        for (uint32_t k = 0; k < h; ++k) hull_idx[k] = si[st[k]];
    }
    *hull_count = h;
    ctrl->small_done = 1u;
}

}  // namespace

cudaError_t launch_small_hull(void *ws, const Layout &L, uint32_t *hull_idx, uint32_t *hull_count, cudaStream_t st)
{
    probe_before(CH_K_CHAIN, st);
    small_hull_kernel<<<1, kSmallThreads, 0, st>>>(ws, L, hull_idx, hull_count);
    note_kernels(CH_K_CHAIN, 1);
    probe_after(CH_K_CHAIN, st);
    return cudaGetLastError();
}

cudaError_t launch_chain(void *ws, const Layout &L, uint32_t *hull_idx, uint32_t *hull_count, cudaStream_t st)
{
    const int sms = sm_count();
    int64_t cb = L.n_chunks;
    static const int per_sm = [] {   // thread-safe one-time initialisation
        cudaFuncSetAttribute(chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ChainSmem));
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, chain_kernel, LT, sizeof(ChainSmem));
        return v > 0 ? v : 1;
    }();
    if (cb > (int64_t)sms * per_sm) cb = (int64_t)sms * per_sm;
    if (cb < 1) cb = 1;
    probe_before(CH_K_CHAIN, st);
    chain_kernel<<<(unsigned)cb, LT, sizeof(ChainSmem), st>>>(ws, L);
    chain_merge_kernel<<<(unsigned)ceil_div(L.n_chunks, 32), 32, 0, st>>>(ws, L);
    note_kernels(CH_K_CHAIN, 2);
    probe_after(CH_K_CHAIN, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int64_t eb = L.emit_tiles;
    if (eb > (int64_t)sms * 4) eb = (int64_t)sms * 4;
    if (eb < 1) eb = 1;
    probe_before(CH_K_EMIT, st);
    emit_kernel<<<(unsigned)eb, kEmitThreads, 0, st>>>(ws, L, hull_idx);
    emit_copy_kernel<<<(unsigned)sms * 4, kEmitThreads, 0, st>>>(ws, L, hull_idx);
    note_kernels(CH_K_EMIT, 2);
    probe_after(CH_K_EMIT, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int64_t fb = ceil_div(L.n, 256 * 8);
    if (fb > (int64_t)sms * 4) fb = (int64_t)sms * 4;
    if (fb < 1) fb = 1;
    probe_before(CH_K_FINISH, st);
    finish_kernel<<<(unsigned)fb, 256, 0, st>>>(ws, L, hull_idx, hull_count);
    note_kernels(CH_K_FINISH, 1);
    probe_after(CH_K_FINISH, st);
    return cudaGetLastError();
}

cudaError_t launch_bx_chain(void *ws, const Layout &L, const BatchLayout &BL, cudaStream_t st)
{
    const int sms = sm_count();
    static const int per_sm = [] {   // thread-safe one-time initialisation
        cudaFuncSetAttribute(bx_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ChainSmem));
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, bx_chain_kernel, LT, sizeof(ChainSmem));
        return v > 0 ? v : 1;
    }();
    int64_t cb = BL.tiles_max;
    if (cb > (int64_t)sms * per_sm) cb = (int64_t)sms * per_sm;
    if (cb < 1) cb = 1;
    probe_before(CH_K_CHAIN, st);
    bx_chain_kernel<<<(unsigned)cb, LT, sizeof(ChainSmem), st>>>(ws, L, BL);
    bx_merge_kernel<<<(unsigned)ceil_div(BL.tiles_max, 32), 32, 0, st>>>(ws, L, BL);
    note_kernels(CH_K_CHAIN, 2);
    probe_after(CH_K_CHAIN, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int64_t eb = ceil_div(BL.tiles_max, kEmitThreads);
    const int emit_per_sm = tune_value(CH_TUNE_BX_EMIT) ? tune_value(CH_TUNE_BX_EMIT) : 4;
    if (eb > (int64_t)sms * emit_per_sm) eb = (int64_t)sms * emit_per_sm;
    if (eb < 1) eb = 1;
    probe_before(CH_K_EMIT, st);
    bx_emit_kernel<<<(unsigned)eb, kEmitThreads, 0, st>>>(ws, L, BL);
    note_kernels(CH_K_EMIT, 1);
    probe_after(CH_K_EMIT, st);
    return cudaGetLastError();
}

}  // namespace ch

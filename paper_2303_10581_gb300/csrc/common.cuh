// common.cuh -- shared device definitions of the octagon-filter hull path:
// workspace layout, order-preserving float keys, the exact orientation
// predicate and the bounded-wait helpers.
//
// Method: Carrasco et al., "An Evaluation of GPU Filters for Accelerating
// the 2D Convex Hull", Sec. 3 / Algorithm 1.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/convhull.h"

namespace ch {

// ---------------------------------------------------------------------------
// launch geometry
// ---------------------------------------------------------------------------
constexpr int kExtThreads = 512;      // extremes sweep
constexpr int kExtPairs = 2048;       // point pairs (16 B) per extremes tile: 32 KB
constexpr int kFiltThreads = 256;     // fused test + compaction
constexpr int kFiltItems = 16;        // points per thread per tile
constexpr int kFiltTile = kFiltThreads * kFiltItems;   // 4096 points = 32 KB
constexpr int kFiltMaxBlocks = 4096;                  // grid cap of the two-pass filter
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;   // 4096 keys
constexpr int kSortPasses = 4;        // 32-bit x keys, 8-bit digits
constexpr int kLeafC = 16;            // points per leaf chain (one thread)
constexpr int kChainThreads = 256;    // leaves per super-chunk (one block)
constexpr int kChainC = kLeafC * kChainThreads;   // 4096 points per super-chunk
constexpr int kChainStride = kChainC + 8;          // chain slots per super-chunk (up to kChainC + 1 used)
constexpr int kElimPasses = 12;       // cap on the per-warp elimination passes
constexpr int kBlockElimPasses = 24;  // cap on the passes over a super-chunk's whole sequence
constexpr int kWarpSeqMax = 256;      // whole-sequence passes run in one warp up to this length
constexpr int kEmitThreads = 256;     // chunks per emit tile (one per thread)
constexpr int64_t kMaxHullN = (int64_t)1 << 30;
constexpr int64_t kMaxN = ((int64_t)1 << 32) - 1;

// device error codes mirror ch_status
constexpr uint32_t kErrNonFinite = CH_ERR_NONFINITE;
constexpr uint32_t kErrTimeout = CH_ERR_TIMEOUT;
// bounded waits: polls before a look-back wait is declared dead (each poll
// is followed by a short nanosleep once the first few fail)
constexpr uint32_t kSpinLimit = 1u << 22;

// look-back status words: [flag:2 | value:62]
constexpr uint64_t kFlagA = 1ull << 62;   // tile aggregate published
constexpr uint64_t kFlagP = 2ull << 62;   // inclusive prefix published
constexpr uint64_t kValMask = (1ull << 62) - 1;
// 32-bit variant for the radix-sort digit status: [flag:2 | value:30]
constexpr uint32_t kFlagA32 = 1u << 30;
constexpr uint32_t kFlagP32 = 2u << 30;
constexpr uint32_t kVal32 = (1u << 30) - 1;

// ---------------------------------------------------------------------------
// filter polygon (Sec. 3.1 -> Sec. 3.2)
// ---------------------------------------------------------------------------
struct Octagon {
    // edge k runs from vertex k to vertex k+1 (mod 8), vertices in the
    // order R, TR, T, TL, L, BL, B, BR
    float ax[8], ay[8];     // edge start
    float bx[8], by[8];     // edge end
    float dx[8], dy[8];     // fl(b - a)
    float bound[8];         // static error bound of the binary32 test (+inf: off)
    uint32_t valid;         // bit k: edge k has non-zero length
    uint32_t has_edges;     // at least one valid edge
    uint32_t abort;         // non-finite input: later stages do nothing
    uint32_t spec;          // 1: the speculative sweep's candidates hold every survivor (spec.cu)
    float xl, xh, yl, yh;   // closed quick-discard rectangle (xl > xh: none)
    float cx, cy;           // bounding-box centre, for the edge order
    float bxl, bxh, byl, byh;   // closed bounding box of the eight vertices
    uint32_t box_check;     // 1: points may lie outside that box (caller-supplied vertices)
    uint32_t pad2;
};

// extremes reduction state: left zeroed by the last block of every sweep
struct ExtCtrl {
    unsigned long long ext_slot[8];   // packed (key, index) per extreme
    uint32_t ext_done;                // extremes blocks finished
    uint32_t nonfinite;               // a non-finite coordinate was seen
};

// second throw-away step of the hull step (kgon.cu): a fan of triangles
// around the bounding-box centre, one vertex per angular bin
// (28672 vertices of 8 bytes fill 224 KB: as many as one block's shared
// memory holds)
constexpr int kFanBins = 28672;

struct KgonCtrl {                          // zeroed with the control block
    unsigned long long slot[kFanBins];     // packed (far_key << 32 | ~index): farthest sampled input point per bin
    uint32_t sample, inside;               // the estimate's sample and how much of it is inside the fan
    uint32_t s_oct;                        // octagon survivors (0: the fan kernels did not run)
    uint32_t pad;
};

// second fan level (kgon.cu): over the first level's survivors, kFan2Sub
// sub-bins per bin, each vertex the farthest survivor of its sub-bin
constexpr int kFan2Sub = 8;
constexpr int kFan2Bins = kFanBins * kFan2Sub;   // 229376
constexpr uint32_t kFan2MinS = 1u << 19;         // fewer survivors of the first level: the sort takes them
constexpr int64_t kFan2MinN = 1 << 19;           // smaller sets get no tables

struct Fan2Ctrl {                          // zeroed with the control block
    uint32_t on;                           // 1: the second level runs this call
    uint32_t count_in;                     // survivors of the first level, its input
    uint32_t bad;                          // 1: no vertices (nothing is dropped)
    uint32_t pad;
};

struct Kgon {
    float cx, cy;                          // fan centre, strictly inside the hull
    uint32_t ok;                           // 0: no fan this call
    uint32_t disk_bad;                     // 1: no disk around the centre is proven inside the fan
    unsigned long long rho2;               // bits of a lower bound on the squared distance from
                                           // the centre to the fan's boundary (binary64 >= 0)
    uint32_t disk_edges;                   // consecutive vertex pairs with v != w
    uint32_t pad;
    float2 v[kFanBins];                    // vertex of every bin (input points)
};

// K-direction filter polygon (kfilter.cu; the learned proposal's filter)
constexpr int kMaxDirs = 64;

struct KxCtrl {                            // left zeroed by the last block of every sweep
    unsigned long long slot[kMaxDirs];     // packed (ord(key) << 32 | ~index) per direction
    uint32_t done;                         // sweep blocks finished
    uint32_t nonfinite;                    // a non-finite coordinate was seen
};

struct KPoly {
    uint32_t K;
    uint32_t nvalid;                       // edges of non-zero length
    unsigned long long valid;              // bit k: edge k (vertex k -> k+1) has non-zero length
    float xl, xh, yl, yh;                  // closed quick-discard rectangle (xl > xh: none)
    float cx, cy;                          // vertex bounding-box centre (facing-edge hint)
    uint32_t convex;                       // every vertex on or left of every valid edge, centre strictly inside
    uint32_t pad;
    float ax[kMaxDirs], ay[kMaxDirs];      // edge k: vertex k ...
    float bx[kMaxDirs], by[kMaxDirs];      // ... to vertex k + 1
};

// control block: zeroed at the start of every call (together with the
// filter's look-back status, which follows it)
struct Ctrl {
    uint32_t filt_ticket;             // tile tickets of the fused filter
    uint32_t surv_count;              // survivors
    uint32_t sort_ticket[kSortPasses];
    uint32_t hist[kSortPasses][256];  // digit histograms of the survivor keys
    uint32_t pass_src[kSortPasses];   // 0/1: buffer a pass reads
    uint32_t pass_skip[kSortPasses];  // pass is an identity (one digit only)
    uint32_t final_buf;               // buffer holding the sorted keys
    uint32_t hist_done;
    uint32_t emit_ticket[2];
    uint32_t h_lower, h_upper;
    uint32_t sort_in;                 // buffer holding the survivors for the sort (the filter writes buffer 0)
    uint32_t small_done;              // the one-block hull of few survivors wrote the hull: later kernels stop
};

// Points the sort and chain kernels of a single-set hull work on: none
// when the call was aborted or the one-block hull already finished it.
__device__ __forceinline__ uint32_t hull_stage_count(const Ctrl *ctrl, const Octagon *oct)
{
    return (oct->abort || ctrl->small_done) ? 0u : ctrl->surv_count;
}

// Speculative single sweep (extremes.cu, filter.cu): a test region from an
// input sample; the extremes sweep keeps the points it cannot prove inside
// it (the candidates: index in the second key buffer, point in the second
// payload buffer).  Segment j holds the candidates of sweep block j, in
// one slice of `cap` slots per warp.
constexpr int kSpecMaxSeg = 2048;         // sweep blocks (segments) at most
constexpr int kSpecWarps = kExtThreads / 32;   // slices per segment
constexpr int kSpecCapDiv = 32;           // all slices together hold n / 32 candidates
constexpr int kSpecKeptSmem = 2048;       // survivors per segment ranked in shared memory
constexpr int64_t kSpecMinN = 1 << 22;    // smaller sets: the plain two passes
struct SpecCtrl {
    uint32_t kmax[8];                     // ord_key of the sample's largest slot keys (self-resetting)
    uint32_t sample_done;                 // sample blocks finished
    uint32_t fail;                        // a slice overflowed: fall back (zeroed by the sample kernel)
    uint32_t nseg;                        // segments (sweep blocks) of this call
    uint32_t cap;                         // candidate slots per slice
    uint32_t scnt[kSpecMaxSeg * kSpecWarps];   // candidates written per slice
    uint32_t skept[kSpecMaxSeg];          // survivors of the octagon per segment (their slots in utmp)
};

// ch_hull_learned: features, activations and outputs of the MLP, and the
// polygon it picks (K and the directions)
struct LearnScratch {
    float feat[1024];
    float h1[64], h2[64];
    float out[68];
    float dirs[2 * kMaxDirs];
    int32_t K;
    int32_t pad[3];
};

// persistent words: survive calls, cleared by ch_last_error
struct Persist {
    uint32_t error;
    uint32_t error_site;
    uint32_t pad[62];
};

// Workspace layout for a problem of up to n points.
struct Layout {
    size_t persist, extctrl, oct, ext8;
    size_t kxctrl, kpoly;   // KxCtrl (self-resetting), KPoly
    size_t ctrl;            // Ctrl, immediately followed by
    size_t filt_status;     // u64[filt_tiles],
    size_t kgon_ctrl;       // KgonCtrl,
    size_t fan2;            // Fan2Ctrl,
    size_t fan2_slot;       // u64[fan2_bins]: per sub-bin the farthest survivor (far_key << 32 | ~position),
    size_t node_cnt;        // u32[n_nodes]: arrivals per merge-tree node, and
    size_t emit_status[2];  // u64[emit_tiles]: look-back of the chain compaction
    size_t zero_words;      // u64 words from ctrl to the end of emit_status[1]
    size_t keys[2];         // u32[n]: ord(x) of each survivor (sort key)
    size_t pay[2];          // u64[n]: ord(y) << 32 | point index (sort payload)
    size_t sort_status[2];  // u32[sort_tiles * 256]
    size_t chain_pos[2];    // u32[n_chunks * kChainStride]: sorted positions of chain vertices
    size_t chain_pt[2];     // float2[n_chunks * kChainStride]: their coordinates
    size_t chunk;           // int32[8 * n_chunks]: loL hiL loU hiU prvL nxtL prvU nxtU
    size_t node;            // int32[4 * n_nodes]: firstL lastL firstU lastU
    size_t emit_off[2];     // u32[n_chunks + 1]: output offset of each super-chunk's chain range, per side
    size_t keep_bits;       // u16[filt_tiles * kFiltThreads]: keep decisions of the count pass
    size_t filt_bsum;       // u32[kFiltMaxBlocks]: survivors per block of the count pass
    size_t kgon;            // Kgon
    size_t utmp;          // u32[n]
    size_t spec, p0;        // SpecCtrl, the speculative sweep's test region (SpecBox, extremes.cu)
    size_t learn;           // the learned proposal's scratch (LearnScratch)
    size_t fan2_v;          // float2[fan2_bins]: the second fan level's vertices
    size_t total;
    int64_t n, filt_tiles, sort_tiles, n_chunks, n_nodes, emit_tiles;
    int64_t fan2_bins;      // kFan2Bins for sets of at least kFan2MinN points, else 0 (no second level)
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

__host__ __device__ inline int64_t tree_nodes(int64_t nc)
{
    // nodes of all levels >= 1 of the binary merge tree over nc leaves
    int64_t total = 0, w = nc;
    while (w > 1) {
        w = (w + 1) / 2;
        total += w;
    }
    return total;
}

// Per-set bookkeeping of ch_hull_batched (all positions are global).
struct SetInfo {
    int64_t pt_begin;     // first point of the set in pts
    int64_t n;            // points in the set
    uint32_t tile_base;   // first 4096-point tile of the set
    uint32_t ntiles;
    uint32_t s;           // survivors of the filter
    uint32_t sc_base;     // first 4096-survivor super-chunk (= sort tile) of the set
    uint64_t surv_base;   // first survivor of the set in the sort arrays
    uint32_t nsc;         // super-chunks of the set
    uint32_t node_base;   // first merge-tree node of the set
    uint32_t hull;        // hull vertices of the set
    uint32_t pad[3];
};

// Batch-wide counters of ch_hull_batched (zeroed at the start of a call).
struct BatchCtrl {
    uint32_t tiles;       // point tiles over all sets
    uint32_t nsc;         // super-chunks over all sets
    uint32_t abort;       // bad offsets: nothing is computed
    uint32_t filt_ticket, emit_ticket, pad0;
    uint32_t sort_ticket[kSortPasses];
    uint32_t h_lower, h_upper;
    uint32_t nfan;        // sets that get the fan test (kgon.cu)
    uint32_t nitems;      // the fan refine's work items (a set's run of up to kBxFanChunk tiles)
    uint32_t fan_ticket;  // next work item of the fan refine
    uint32_t pad;
};
constexpr int kBxFanChunk = 64;       // tiles per work item of the batched fan refine (built-in)
constexpr int kBxFanChunkMin = 8;     // the smallest tunable one (sizes the work-item list)

// Extra workspace of ch_hull_batched, after the single-set regions.
struct BatchLayout {
    size_t sets;          // SetInfo[B]
    size_t octs;          // Octagon[B]
    size_t zero_begin;    // ---- zeroed by one memset per call:
    size_t bctrl;         // BatchCtrl
    size_t ext_slot;      // u64[B * 8]: packed extremes per set
    size_t nonfinite;     // u32[B]
    size_t hist;          // u32[B * kSortPasses * 256]
    size_t zero_end;      // ----
    size_t tile_set;      // u32[tiles_max]: set of each point tile
    size_t sc_set;        // u32[tiles_max]: set of each super-chunk
    size_t sc_off[2];     // u32[tiles_max + 1]: lower / upper chain offset of each super-chunk
    size_t lower;         // u32[n]: lower chains of all sets (set-local indices); aliases keys[1]
    // the fan of the hull step, per set with many octagon survivors (kgon.cu)
    size_t soct;          // u32[B]: octagon survivors per set (in the zeroed range)
    size_t fan_id;        // i32[B]: the set's fan number, -1: none
    size_t fan_set;       // u32[max_fan]: set of each fan
    size_t fan_ok;        // u32[max_fan]: the fan has vertices and its centre is inside
    size_t fan_c;         // float2[max_fan]: centre
    size_t fan_slot;      // u64[max_fan * kFanBins]: farthest sampled point per bin (left zeroed)
    size_t fan_v;         // float2[max_fan * kFanBins]: vertices
    size_t fan_items;     // uint2[max_items]: (fan, first tile) of each refine work item
    size_t total;
    int64_t num_sets, tiles_max, max_fan, max_items;
};

__host__ __device__ inline Layout make_layout(int64_t n, int64_t sets = 0)
{
    Layout L{};
    if (n < 1) n = 1;
    L.n = n;
    L.filt_tiles = ceil_div(n, kFiltTile);
    L.sort_tiles = ceil_div(n, kSortTile);
    L.n_chunks = ceil_div(n, kChainC);
    L.n_nodes = tree_nodes(L.n_chunks) + 1;
    if (sets > 0) {
        // every set adds at most one ragged tile / super-chunk, and each
        // set's merge tree has fewer than twice as many nodes as leaves
        L.filt_tiles = L.n_chunks = ceil_div(n, kChainC) + sets;
        L.sort_tiles = L.sort_tiles > L.n_chunks ? L.sort_tiles : L.n_chunks;
        L.n_nodes = 2 * L.n_chunks + sets;
    }
    L.emit_tiles = ceil_div(L.n_chunks, kEmitThreads);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    L.persist = take(sizeof(Persist));
    L.extctrl = take(sizeof(ExtCtrl));
    L.oct = take(sizeof(Octagon));
    L.ext8 = take(8 * sizeof(uint32_t));
    L.kxctrl = take(sizeof(KxCtrl));
    L.kpoly = take(sizeof(KPoly));
    L.ctrl = take(sizeof(Ctrl));
    L.filt_status = take((size_t)L.filt_tiles * 8);
    L.kgon_ctrl = take(sizeof(KgonCtrl));
    L.fan2_bins = (sets == 0 && n >= kFan2MinN) ? kFan2Bins : 0;
    L.fan2 = take(sizeof(Fan2Ctrl));
    L.fan2_slot = take((size_t)L.fan2_bins * 8);
    L.node_cnt = take((size_t)L.n_nodes * 4);
    L.emit_status[0] = take((size_t)L.emit_tiles * 8);
    L.emit_status[1] = take((size_t)L.emit_tiles * 8);
    L.zero_words = (L.emit_status[1] + (size_t)L.emit_tiles * 8 - L.ctrl + 7) / 8;
    L.keys[0] = take((size_t)n * 4);
    L.keys[1] = take((size_t)n * 4);
    L.pay[0] = take((size_t)n * 8);
    L.pay[1] = take((size_t)n * 8);
    L.sort_status[0] = take((size_t)L.sort_tiles * 256 * 4);
    L.sort_status[1] = take((size_t)L.sort_tiles * 256 * 4);
    for (int side = 0; side < 2; ++side) {
        L.chain_pos[side] = take((size_t)L.n_chunks * kChainStride * 4);
        L.chain_pt[side] = take((size_t)L.n_chunks * kChainStride * 8);
    }
    L.chunk = take((size_t)L.n_chunks * 8 * 4);
    L.node = take((size_t)L.n_nodes * 4 * 4);
    L.emit_off[0] = take((size_t)(L.n_chunks + 1) * 4);
    L.emit_off[1] = take((size_t)(L.n_chunks + 1) * 4);
    L.keep_bits = take((size_t)L.filt_tiles * kFiltThreads * 2);
    L.filt_bsum = take((size_t)kFiltMaxBlocks * 4);
    L.kgon = take(sizeof(Kgon));
    L.utmp = take((size_t)n * 4);
    L.spec = take(sizeof(SpecCtrl));
    L.p0 = take(256);
    L.learn = take(sizeof(LearnScratch));
    L.fan2_v = take((size_t)L.fan2_bins * 8);
    L.total = o;
    return L;
}

__host__ __device__ inline BatchLayout make_batch_layout(const Layout &L, int64_t sets)
{
    BatchLayout B{};
    B.num_sets = sets;
    B.tiles_max = L.n_chunks;
    size_t o = L.total;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    B.sets = take((size_t)sets * sizeof(SetInfo));
    B.octs = take((size_t)sets * sizeof(Octagon));
    B.zero_begin = o;
    B.bctrl = take(sizeof(BatchCtrl));
    B.ext_slot = take((size_t)sets * 8 * 8);
    B.nonfinite = take((size_t)sets * 4);
    B.hist = take((size_t)sets * kSortPasses * 256 * 4);
    B.soct = take((size_t)sets * 4);
    B.zero_end = o;
    B.tile_set = take((size_t)B.tiles_max * 4);
    B.sc_set = take((size_t)B.tiles_max * 4);
    B.sc_off[0] = take((size_t)(B.tiles_max + 1) * 4);
    B.sc_off[1] = take((size_t)(B.tiles_max + 1) * 4);
    B.lower = L.keys[1];   // the second sort buffer is free once the sort ends in buffer 0
    // a set with a fan has at least 2^16 points
    B.max_fan = sets < L.n / 65536 + 1 ? sets : L.n / 65536 + 1;
    B.max_items = B.tiles_max / kBxFanChunkMin + B.max_fan + 1;
    B.fan_id = take((size_t)sets * 4);
    B.fan_set = take((size_t)B.max_fan * 4);
    B.fan_ok = take((size_t)B.max_fan * 4);
    B.fan_c = take((size_t)B.max_fan * 8);
    B.fan_slot = take((size_t)B.max_fan * kFanBins * 8);
    B.fan_v = take((size_t)B.max_fan * kFanBins * 8);
    B.fan_items = take((size_t)B.max_items * 8);
    B.total = o;
    return B;
}

template <class T>
__host__ __device__ inline T *at(void *ws, size_t off)
{
    return reinterpret_cast<T *>(static_cast<char *>(ws) + off);
}

// ---------------------------------------------------------------------------
// order-preserving keys
// ---------------------------------------------------------------------------
// Map binary32 bits to uint32 so that unsigned order equals numeric order;
// -0 is first mapped to +0 so the two compare equal, as float compares do.
__device__ __forceinline__ uint32_t ord_key(float f)
{
    uint32_t b = __float_as_uint(f);
    if (b == 0x80000000u) b = 0;
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float key_float(uint32_t k)
{
    uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(b);
}

__device__ __forceinline__ unsigned long long point_key(float x, float y)
{
    return ((unsigned long long)ord_key(x) << 32) | ord_key(y);
}

__device__ __forceinline__ float2 key_point(unsigned long long k)
{
    return make_float2(key_float((uint32_t)(k >> 32)), key_float((uint32_t)k));
}

// ---------------------------------------------------------------------------
// exact orientation: sign of (b - a) x (c - a) for binary32 inputs
// ---------------------------------------------------------------------------
// Tier 3: the determinant expands into six products of two binary32 values
// (the a.x*a.y terms cancel); each is exact in binary64.  They are summed
// without error by Grow-Expansion with Two-Sum (Shewchuk, "Adaptive
// Precision Floating-Point Arithmetic and Fast Robust Geometric
// Predicates", 1997, Sec. 2); the sign of a non-overlapping expansion is
// the sign of its largest non-zero component.
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e)
{
    s = __dadd_rn(a, b);
    double bv = __dsub_rn(s, a);
    double av = __dsub_rn(s, bv);
    e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

static __device__ __noinline__ int orient_exact(float ax, float ay, float bx, float by, float cx, float cy)
{
    double t[6];
    t[0] = __dmul_rn((double)bx, (double)cy);
    t[1] = -__dmul_rn((double)bx, (double)ay);
    t[2] = -__dmul_rn((double)ax, (double)cy);
    t[3] = -__dmul_rn((double)by, (double)cx);
    t[4] = __dmul_rn((double)by, (double)ax);
    t[5] = __dmul_rn((double)ay, (double)cx);
    double e[6];
    int m = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double q = t[i];
        int k = 0;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            if (j < m) {
                double s, r;
                two_sum(q, e[j], s, r);
                q = s;
                if (r != 0.0) e[k++] = r;
            }
        }
        if (q != 0.0) e[k++] = q;
        m = k;
    }
    if (m == 0) return 0;
    return e[m - 1] > 0.0 ? 1 : -1;
}

// Tier 2: binary64 evaluation with Shewchuk's orient2d error bound
// ccwerrboundA = (3 + 16 eps) eps, eps = 2^-53.  Differences and products of
// binary32 values cannot underflow or overflow in binary64, so the bound
// holds; undecided cases go to tier 3.
static __device__ __noinline__ int orient_d(float ax, float ay, float bx, float by, float cx, float cy)
{
    // orient2d(pa = a, pb = b, pc = c)
    double detleft = __dmul_rn(__dsub_rn((double)ax, (double)cx), __dsub_rn((double)by, (double)cy));
    double detright = __dmul_rn(__dsub_rn((double)ay, (double)cy), __dsub_rn((double)bx, (double)cx));
    double det = __dsub_rn(detleft, detright);
    double detsum;
    if (detleft > 0.0) {
        if (detright <= 0.0) return det > 0.0 ? 1 : (det < 0.0 ? -1 : 0);
        detsum = __dadd_rn(detleft, detright);
    } else if (detleft < 0.0) {
        if (detright >= 0.0) return det > 0.0 ? 1 : (det < 0.0 ? -1 : 0);
        detsum = __dsub_rn(-detleft, detright);
    } else {
        return det > 0.0 ? 1 : (det < 0.0 ? -1 : 0);
    }
    const double errA = (3.0 + 16.0 * 0x1p-53) * 0x1p-53;   // exact in binary64
    double eb = __dmul_ru(errA, detsum);
    if (det >= eb) return 1;
    if (-det >= eb) return -1;
    return orient_exact(ax, ay, bx, by, cx, cy);
}

// Sterbenz: a - c is exact in binary32 when a and c have the same sign and
// are within a factor of two of each other.
__device__ __forceinline__ bool exact_diff(float a, float c)
{
    const float aa = fabsf(a), cc = fabsf(c);
    return ((a >= 0.0f) == (c >= 0.0f)) && aa <= 2.0f * cc && cc <= 2.0f * aa;
}

// Tier 1b: exact binary32 sign for nearby points.  When the four
// differences are exact, detleft = u1 v1 and detright = u2 v2 exactly; with
// p = fl(u v) and e = fma(u, v, -p) = u v - p (exact while |p| >= 2^-100 or
// a factor is zero, since then the product cannot underflow), rounding is
// monotone, so p1 > p2 implies u1 v1 > u2 v2, and when p1 == p2 the
// determinant is e1 - e2, whose sign survives the one rounding of
// fl(e1 - e2).  Returns 2 when the preconditions do not hold.
__device__ __forceinline__ int orient_near(float ax, float ay, float bx, float by, float cx, float cy)
{
    if (!(exact_diff(ax, cx) && exact_diff(by, cy) && exact_diff(ay, cy) && exact_diff(bx, cx))) return 2;
    const float u1 = __fsub_rn(ax, cx), v1 = __fsub_rn(by, cy);
    const float u2 = __fsub_rn(ay, cy), v2 = __fsub_rn(bx, cx);
    const float p1 = __fmul_rn(u1, v1), p2 = __fmul_rn(u2, v2);
    const bool ok1 = (u1 == 0.0f || v1 == 0.0f) || (fabsf(p1) >= 7.888609052210118e-31f /* 2^-100 */ &&
                                                    fabsf(p1) <= 3.0e38f);
    const bool ok2 = (u2 == 0.0f || v2 == 0.0f) || (fabsf(p2) >= 7.888609052210118e-31f && fabsf(p2) <= 3.0e38f);
    if (!(ok1 && ok2)) return 2;
    if (p1 != p2) return p1 > p2 ? 1 : -1;
    const float d = __fsub_rn(__fmaf_rn(u1, v1, -p1), __fmaf_rn(u2, v2, -p2));
    return d > 0.0f ? 1 : (d < 0.0f ? -1 : 0);
}

// Tier 1: binary32 evaluation with a dynamic bound.  The expression has
// Shewchuk's orient2d shape (four differences, two products, one
// subtraction), whose rounding error is below (3 + 16 eps) eps * detsum with
// eps = 2^-24 when nothing under- or overflows; 4 eps * detsum leaves room
// for the rounding of the bound itself, and 2^-140 absorbs the absolute
// error of products that fall into the subnormal range.  Undecided cases
// try tier 1b, then tier 2.
// The binary32 tier alone, branch-free: the sign when the bound proves it,
// 2 otherwise.
__device__ __forceinline__ int orient_f32(float ax, float ay, float bx, float by, float cx, float cy)
{
    float detleft = __fmul_rn(__fsub_rn(ax, cx), __fsub_rn(by, cy));
    float detright = __fmul_rn(__fsub_rn(ay, cy), __fsub_rn(bx, cx));
    float det = __fsub_rn(detleft, detright);
    float detsum = __fadd_rn(fabsf(detleft), fabsf(detright));
    float eb = __fmaf_ru(detsum, 2.384185791015625e-07f /* 2^-22 */, 7.174648137343064e-43f /* 2^-140 */);
    const int o = det > eb ? 1 : (-det > eb ? -1 : 2);
    return detsum <= 3.0e38f ? o : 2;
}

// orient_f32 of (a, b, c) given the rounded differences a - c = (acx, acy)
// and b - c = (bcx, bcy): the same arithmetic after the subtractions.
__device__ __forceinline__ int orient_f32_ref(float acx, float acy, float bcx, float bcy)
{
    float detleft = __fmul_rn(acx, bcy);
    float detright = __fmul_rn(acy, bcx);
    float det = __fsub_rn(detleft, detright);
    float detsum = __fadd_rn(fabsf(detleft), fabsf(detright));
    float eb = __fmaf_ru(detsum, 2.384185791015625e-07f /* 2^-22 */, 7.174648137343064e-43f /* 2^-140 */);
    const int o = det > eb ? 1 : (-det > eb ? -1 : 2);
    return detsum <= 3.0e38f ? o : 2;
}

// The tiers after binary32: exact differences, binary64, expansions.
__device__ __forceinline__ int orient_rest(float ax, float ay, float bx, float by, float cx, float cy)
{
    const int o = orient_near(ax, ay, bx, by, cx, cy);
    if (o != 2) return o;
    return orient_d(ax, ay, bx, by, cx, cy);
}

__device__ __forceinline__ int orient(float ax, float ay, float bx, float by, float cx, float cy)
{
    const int o = orient_f32(ax, ay, bx, by, cx, cy);
    return o != 2 ? o : orient_rest(ax, ay, bx, by, cx, cy);
}

// ---------------------------------------------------------------------------
// TMA bulk prefetch into L2
// ---------------------------------------------------------------------------
// Asks the TMA unit to bring `bytes` (a multiple of 16, from a 16-byte
// aligned address) into L2.  A hint: nothing waits on it.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// The line holding `p` into L2 (one lane's hint; nothing waits on it).
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// ---------------------------------------------------------------------------
// error reporting and bounded waits
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_error(void *ws, const Layout &L, uint32_t code, uint32_t site)
{
    Persist *p = at<Persist>(ws, L.persist);
    if (atomicCAS(&p->error, 0u, code) == 0u) atomicExch(&p->error_site, site);
}

__device__ __forceinline__ bool error_set(void *ws, const Layout &L)
{
    return *(volatile uint32_t *)&at<Persist>(ws, L.persist)->error != 0u;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Decoupled look-back (Merrill & Garland, "Single-pass Parallel Prefix Scan
// with Decoupled Look-back", 2016) over 64-bit status words, run by one
// full warp.  Returns the exclusive prefix of tile `tile`.  Waits are
// bounded: when a predecessor never publishes, the error word is set and
// the wait stops (the prefix is then meaningless, the call reports
// CH_ERR_TIMEOUT).
__device__ __forceinline__ unsigned long long lookback_u64(unsigned long long *status, int64_t tile,
                                                           void *ws, const Layout &L, uint32_t site)
{
    const uint32_t lane = lane_id();
    unsigned long long excl = 0;
    int64_t base = tile - 1;
    uint32_t spins = 0;
    while (base >= 0) {
        int64_t idx = base - (int64_t)lane;
        unsigned long long s = idx >= 0 ? ld_acquire_u64(status + idx) : kFlagP;
        while (__any_sync(0xffffffffu, (s >> 62) == 0)) {
            if (++spins > kSpinLimit || (spins > 1024 && error_set(ws, L))) {
                if (lane == 0) set_error(ws, L, kErrTimeout, site);
                return 0;
            }
            if (spins > 64) __nanosleep(100);
            if ((s >> 62) == 0) s = ld_acquire_u64(status + idx);
        }
        uint32_t pmask = __ballot_sync(0xffffffffu, (s >> 62) == 2);
        uint32_t stop = pmask ? (uint32_t)(__ffs(pmask) - 1) : 31u;
        unsigned long long v = lane <= stop ? (s & kValMask) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (pmask) break;
        base -= 32;
    }
    return excl;
}

}  // namespace ch

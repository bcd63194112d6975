/*
 * oracle.c -- plain, sequential CPU oracle for the octagon filter and the
 * monotone-chain hull of
 *   R. Carrasco, H. Ferrada, C. A. Navarro, N. Hitschfeld,
 *   "An Evaluation of GPU Filters for Accelerating the 2D Convex Hull"
 *   (arXiv 2303.10581).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the CUDA path is
 * compared against.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product library never
 * links, calls or falls back to it, and it shares no code, header, table or
 * helper with the CUDA sources.
 *
 * What it computes, in the paper's order (Sec. 3, Algorithm 1):
 *   1. findingPolygon (Sec. 3.1): the four axis extremes and the four
 *      bounding-box corner points.  A corner point minimises the Manhattan
 *      distance to a bounding-box corner; for the top-right corner
 *      (xmax, ymax) that distance is (xmax - x) + (ymax - y), so the closest
 *      point maximises x + y.  Likewise bottom-left minimises x + y,
 *      top-left minimises x - y and bottom-right maximises x - y.  The keys
 *      x + y and x - y are rounded to binary32 (the paper computes in FP32,
 *      Sec. 6).  Ties go to the lowest index.
 *   2. buildingFilter (Sec. 3.2): a point is discarded exactly when it lies
 *      strictly inside the polygon, i.e. strictly to the left of every
 *      non-degenerate edge of the closed vertex sequence
 *      R, TR, T, TL, L, BL, B, BR (counter-clockwise).  The orientation
 *      sign is exact.
 *   3. compactingFilteredPoints (Sec. 3.2, Sec. 4.1): survivors in
 *      ascending index order.
 *   4. convexHull (Sec. 3.3): Andrew's monotone chain over the survivors:
 *      lexicographic (x, y) order, duplicates collapsed to the lowest index,
 *      collinear points excluded, output counter-clockwise starting at the
 *      lexicographically smallest vertex.
 *
 * Exact orientation: for binary32 inputs the determinant
 *   (bx - ax)(cy - ay) - (by - ay)(cx - ax)
 * expands to six products of two binary32 numbers (the ax*ay terms cancel).
 * Each such product has at most 48 significant bits and a magnitude in
 * [2^-298, 2^256), so it is exact in binary64.  The six exact products are
 * summed in a fixed-point long accumulator (a 640-bit two's-complement
 * integer in units of 2^-352), whose sign is the exact sign.  Before the
 * accumulator, a plain recursive binary64 sum is accepted when it clears
 * the textbook bound for recursive summation of six terms (Higham,
 * "Accuracy and Stability of Numerical Algorithms", Eq. 4.4: error at most
 * gamma_5 * sum|x_i| < 8u * sum|x_i|, u = 2^-53); otherwise the
 * accumulator decides.  Setting oracle_set_force_exact(1) skips the
 * shortcut so the two can be checked against each other.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fast-math, no long
 * double), so binary32 expressions round exactly once per operation.
 *
 * Also the same filter with K directions in place of the eight (the
 * polygon a learned proposal picks): vertex k maximises the binary32 key
 * fl(fl(c_k x) + fl(s_k y)), lowest index on ties; the test and the
 * compaction are those of Sec. 3.2 (oracle_kgon_extremes,
 * oracle_kgon_filter).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NONFINITE 2

/* ------------------------------------------------------------------ */
/* exact orientation                                                   */
/* ------------------------------------------------------------------ */

#define ACC_LIMBS 10
#define ACC_UNIT_EXP 352 /* accumulator unit is 2^-352 */

typedef struct {
    uint64_t w[ACC_LIMBS];
} long_acc;

static int g_force_exact = 0;
static uint64_t g_exact_calls = 0;

void oracle_set_force_exact(int on) { g_force_exact = on ? 1 : 0; }
uint64_t oracle_exact_calls(void) { return g_exact_calls; }

/* Add (or subtract) mant * 2^pos units into the accumulator. */
static void acc_add(long_acc *a, uint64_t mant, int pos, int negative)
{
    int limb = pos / 64;
    int off = pos % 64;
    uint64_t lo = mant << off;
    uint64_t hi = off ? (mant >> (64 - off)) : 0;
    if (!negative) {
        uint64_t carry = 0;
        for (int k = limb; k < ACC_LIMBS; ++k) {
            uint64_t add = (k == limb) ? lo : (k == limb + 1 ? hi : 0);
            uint64_t s = a->w[k] + add;
            uint64_t c1 = s < add;
            uint64_t s2 = s + carry;
            uint64_t c2 = s2 < carry;
            a->w[k] = s2;
            carry = c1 | c2;
            if (k > limb + 1 && carry == 0) break;
        }
    } else {
        uint64_t borrow = 0;
        for (int k = limb; k < ACC_LIMBS; ++k) {
            uint64_t sub = (k == limb) ? lo : (k == limb + 1 ? hi : 0);
            uint64_t d = a->w[k] - sub;
            uint64_t b1 = a->w[k] < sub;
            uint64_t d2 = d - borrow;
            uint64_t b2 = d < borrow;
            a->w[k] = d2;
            borrow = b1 | b2;
            if (k > limb + 1 && borrow == 0) break;
        }
    }
}

/* Add the binary64 value v exactly.  v is a product of two binary32
 * numbers, so v == 0 or 2^-298 <= |v| < 2^256. */
static void acc_add_double(long_acc *a, double v)
{
    if (v == 0.0) return;
    int e;
    double m = frexp(fabs(v), &e);           /* |v| = m * 2^e, 0.5 <= m < 1 */
    uint64_t mant = (uint64_t)ldexp(m, 53);  /* exact 53-bit integer */
    int pos = e - 53 + ACC_UNIT_EXP;         /* |v| = mant * 2^(pos - 352) */
    acc_add(a, mant, pos, v < 0.0);
}

static int acc_sign(const long_acc *a)
{
    if (a->w[ACC_LIMBS - 1] >> 63) return -1;
    for (int k = 0; k < ACC_LIMBS; ++k)
        if (a->w[k]) return 1;
    return 0;
}

/* Exact sign of (b - a) x (c - a):  +1 = c strictly left of a->b
 * (counter-clockwise turn), 0 = collinear, -1 = clockwise. */
int oracle_orient(float ax, float ay, float bx, float by, float cx, float cy)
{
    double t[6];
    t[0] = (double)bx * (double)cy;
    t[1] = -((double)bx * (double)ay);
    t[2] = -((double)ax * (double)cy);
    t[3] = -((double)by * (double)cx);
    t[4] = (double)by * (double)ax;
    t[5] = (double)ay * (double)cx;
    if (!g_force_exact) {
        double s = 0.0, sa = 0.0;
        for (int k = 0; k < 6; ++k) {
            s += t[k];
            sa += fabs(t[k]);
        }
        if (fabs(s) > ldexp(sa, -50)) return s > 0.0 ? 1 : -1;
    }
    ++g_exact_calls;
    long_acc acc;
    memset(&acc, 0, sizeof acc);
    for (int k = 0; k < 6; ++k) acc_add_double(&acc, t[k]);
    return acc_sign(&acc);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.1: the eight polygon vertices                                */
/* ------------------------------------------------------------------ */

static int finite_point(float x, float y) { return isfinite(x) && isfinite(y); }

/* ext8 receives indices in counter-clockwise order
 *   R  = argmax x,      TR = argmax fl(x+y),  T = argmax y,
 *   TL = argmin fl(x-y), L = argmin x,        BL = argmin fl(x+y),
 *   B  = argmin y,      BR = argmax fl(x-y).
 * pts is packed (x, y) binary32, n >= 1.  Returns OR_ERR_NONFINITE if any
 * coordinate is NaN or infinite. */
int oracle_extremes(const float *pts, int64_t n, uint32_t *ext8)
{
    if (n < 1 || !pts || !ext8) return OR_ERR_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (!finite_point(pts[2 * i], pts[2 * i + 1])) return OR_ERR_NONFINITE;

    float bx_max = pts[0], bx_min = pts[0], by_max = pts[1], by_min = pts[1];
    float s0 = pts[0] + pts[1];
    float d0 = pts[0] - pts[1];
    float bs_max = s0, bs_min = s0, bd_max = d0, bd_min = d0;
    uint32_t iR = 0, iTR = 0, iT = 0, iTL = 0, iL = 0, iBL = 0, iB = 0, iBR = 0;
    for (int64_t i = 1; i < n; ++i) {
        float x = pts[2 * i], y = pts[2 * i + 1];
        float s = x + y;
        float d = x - y;
        if (x > bx_max) { bx_max = x; iR = (uint32_t)i; }
        if (x < bx_min) { bx_min = x; iL = (uint32_t)i; }
        if (y > by_max) { by_max = y; iT = (uint32_t)i; }
        if (y < by_min) { by_min = y; iB = (uint32_t)i; }
        if (s > bs_max) { bs_max = s; iTR = (uint32_t)i; }
        if (s < bs_min) { bs_min = s; iBL = (uint32_t)i; }
        if (d > bd_max) { bd_max = d; iBR = (uint32_t)i; }
        if (d < bd_min) { bd_min = d; iTL = (uint32_t)i; }
    }
    ext8[0] = iR;
    ext8[1] = iTR;
    ext8[2] = iT;
    ext8[3] = iTL;
    ext8[4] = iL;
    ext8[5] = iBL;
    ext8[6] = iB;
    ext8[7] = iBR;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.2: strict point-in-polygon test and stable compaction        */
/* ------------------------------------------------------------------ */

/* 1 if point i must be kept as a hull candidate, 0 if it lies strictly
 * inside the closed polygon v[0..7] (counter-clockwise).  Edges whose two
 * endpoints coincide are skipped; with no edge left nothing is inside. */
static int keep_point(const float *v, float px, float py)
{
    int edges = 0;
    for (int k = 0; k < 8; ++k) {
        float ax = v[2 * k], ay = v[2 * k + 1];
        float bx = v[2 * ((k + 1) % 8)], by = v[2 * ((k + 1) % 8) + 1];
        if (ax == bx && ay == by) continue;
        ++edges;
        if (oracle_orient(ax, ay, bx, by, px, py) <= 0) return 1;
    }
    return edges == 0;
}

/* Writes the ascending indices of the kept points to surv_idx (capacity n)
 * and returns their number, or -1 on bad arguments. */
int64_t oracle_filter(const float *pts, int64_t n, const uint32_t *ext8, uint32_t *surv_idx)
{
    if (n < 0 || (n > 0 && (!pts || !ext8 || !surv_idx))) return -1;
    if (n == 0) return 0;
    float v[16];
    for (int k = 0; k < 8; ++k) {
        if ((int64_t)ext8[k] >= n) return -1;
        v[2 * k] = pts[2 * (int64_t)ext8[k]];
        v[2 * k + 1] = pts[2 * (int64_t)ext8[k] + 1];
    }
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i)
        if (keep_point(v, pts[2 * i], pts[2 * i + 1])) surv_idx[s++] = (uint32_t)i;
    return s;
}

/* Keep flags, one byte per point (1 = kept); for sampled checks. */
int oracle_keep_flags(const float *pts, int64_t n, const uint32_t *ext8, const uint32_t *which,
                      int64_t m, uint8_t *flags)
{
    if (n < 1) return OR_ERR_ARG;
    float v[16];
    for (int k = 0; k < 8; ++k) {
        if ((int64_t)ext8[k] >= n) return OR_ERR_ARG;
        v[2 * k] = pts[2 * (int64_t)ext8[k]];
        v[2 * k + 1] = pts[2 * (int64_t)ext8[k] + 1];
    }
    for (int64_t j = 0; j < m; ++j) {
        int64_t i = which[j];
        if (i >= n) return OR_ERR_ARG;
        flags[j] = (uint8_t)keep_point(v, pts[2 * i], pts[2 * i + 1]);
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* K directions: the filter polygon of the learned proposal            */
/* ------------------------------------------------------------------ */

/* The polygon generalised from the eight directions of Sec. 3.1 to K
 * directions (c_k, s_k), k = 0 .. K-1 (dirs holds them as pairs, in
 * counter-clockwise order; |c_k|, |s_k| <= 1): vertex k is the point with
 * the largest binary32 key fl(fl(c_k x) + fl(s_k y)), ties to the lowest
 * index.  With the eight integer directions (1,0), (1,1), (0,1), (-1,1),
 * (-1,0), (-1,-1), (0,-1), (1,-1) the keys are x, fl(x+y), y, -fl(x-y), -x,
 * -fl(x+y), -y, fl(x-y) and the vertices are the octagon's R ... BR.
 * ext receives K indices.  Returns OR_ERR_NONFINITE for a NaN or infinite
 * coordinate. */
int oracle_kgon_extremes(const float *pts, int64_t n, int K, const float *dirs, uint32_t *ext)
{
    if (n < 1 || K < 3 || K > 64 || !pts || !dirs || !ext) return OR_ERR_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (!finite_point(pts[2 * i], pts[2 * i + 1])) return OR_ERR_NONFINITE;
    for (int k = 0; k < K; ++k) {
        const float c = dirs[2 * k], sn = dirs[2 * k + 1];
        float best = c * pts[0] + sn * pts[1];
        uint32_t at = 0;
        for (int64_t i = 1; i < n; ++i) {
            const float key = c * pts[2 * i] + sn * pts[2 * i + 1];
            if (key > best) {
                best = key;
                at = (uint32_t)i;
            }
        }
        ext[k] = at;
    }
    return OR_OK;
}

/* 1 if the point must be kept: not strictly to the left of every edge of
 * non-zero length of the closed vertex sequence v[0 .. K-1]. */
static int keep_point_k(const float *v, int K, float px, float py)
{
    int edges = 0;
    for (int k = 0; k < K; ++k) {
        float ax = v[2 * k], ay = v[2 * k + 1];
        float bx = v[2 * ((k + 1) % K)], by = v[2 * ((k + 1) % K) + 1];
        if (ax == bx && ay == by) continue;
        ++edges;
        if (oracle_orient(ax, ay, bx, by, px, py) <= 0) return 1;
    }
    return edges == 0;
}

/* Ascending indices of the points kept by the K-vertex polygon
 * pts[ext[0]], ..., pts[ext[K-1]]; returns their number, or -1 on bad
 * arguments. */
int64_t oracle_kgon_filter(const float *pts, int64_t n, int K, const uint32_t *ext, uint32_t *surv_idx)
{
    if (n < 0 || K < 3 || K > 64 || (n > 0 && (!pts || !ext || !surv_idx))) return -1;
    if (n == 0) return 0;
    float v[128];
    for (int k = 0; k < K; ++k) {
        if ((int64_t)ext[k] >= n) return -1;
        v[2 * k] = pts[2 * (int64_t)ext[k]];
        v[2 * k + 1] = pts[2 * (int64_t)ext[k] + 1];
    }
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i)
        if (keep_point_k(v, K, pts[2 * i], pts[2 * i + 1])) surv_idx[s++] = (uint32_t)i;
    return s;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.3: Andrew's monotone chain                                   */
/* ------------------------------------------------------------------ */

typedef struct {
    float x, y;
    uint32_t idx;
} hpt;

static int cmp_hpt(const void *pa, const void *pb)
{
    const hpt *a = (const hpt *)pa, *b = (const hpt *)pb;
    if (a->x < b->x) return -1;
    if (a->x > b->x) return 1;
    if (a->y < b->y) return -1;
    if (a->y > b->y) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* Hull of the points pts[idx[0..m-1]] (or of pts[0..m-1] when idx is NULL).
 * Writes original point indices, counter-clockwise from the lexicographically
 * smallest (x, y) vertex, to hull_out (capacity m) and returns the vertex
 * count, or -1 on bad arguments / allocation failure. */
int64_t oracle_hull(const float *pts, const uint32_t *idx, int64_t m, uint32_t *hull_out)
{
    if (m < 0) return -1;
    if (m == 0) return 0;
    hpt *p = (hpt *)malloc((size_t)m * sizeof(hpt));
    hpt *st = (hpt *)malloc((size_t)(2 * m + 2) * sizeof(hpt));
    if (!p || !st) {
        free(p);
        free(st);
        return -1;
    }
    for (int64_t k = 0; k < m; ++k) {
        uint32_t i = idx ? idx[k] : (uint32_t)k;
        p[k].x = pts[2 * (int64_t)i];
        p[k].y = pts[2 * (int64_t)i + 1];
        p[k].idx = i;
    }
    qsort(p, (size_t)m, sizeof(hpt), cmp_hpt);
    /* collapse equal points to the first (lowest index) */
    int64_t u = 0;
    for (int64_t k = 0; k < m; ++k) {
        if (u > 0 && p[k].x == p[u - 1].x && p[k].y == p[u - 1].y) continue;
        p[u++] = p[k];
    }
    if (u == 1) {
        hull_out[0] = p[0].idx;
        free(p);
        free(st);
        return 1;
    }
    int64_t h = 0;
    /* lower chain, left to right */
    for (int64_t k = 0; k < u; ++k) {
        while (h >= 2 && oracle_orient(st[h - 2].x, st[h - 2].y, st[h - 1].x, st[h - 1].y,
                                       p[k].x, p[k].y) <= 0)
            --h;
        st[h++] = p[k];
    }
    /* upper chain, right to left, on top of the lower one */
    int64_t base = h + 1;
    for (int64_t k = u - 2; k >= 0; --k) {
        while (h >= base && oracle_orient(st[h - 2].x, st[h - 2].y, st[h - 1].x, st[h - 1].y,
                                          p[k].x, p[k].y) <= 0)
            --h;
        st[h++] = p[k];
    }
    --h; /* the last point repeats the first */
    for (int64_t k = 0; k < h; ++k) hull_out[k] = st[k].idx;
    free(p);
    free(st);
    return h;
}

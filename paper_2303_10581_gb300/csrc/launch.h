// launch.h -- host-side launchers shared between the translation units of
// the library (internal; the public interface is include/convhull.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace ch {

int sm_count();

// instrumentation around every launch (probe.cu)
void probe_before(int kid, cudaStream_t st);
// counts `count` kernel launches of kernel id kid (every launcher calls it)
void note_kernels(int kid, int count);
void probe_after(int kid, cudaStream_t st);

// learn_params (the MLP's BF16 parameters, ch_hull_learned): one more block
// runs the learned proposal into the workspace's LearnScratch.
// spec (with build_polygon, on large sets): the speculative single sweep --
// a sample octagon first, then the sweep writes the points it cannot prove
// inside it as candidates; when its last block proves the sample octagon
// inside the final one (Octagon::spec), the filter's passes test only them
cudaError_t launch_extremes(const float *pts, int64_t n, void *ws, const Layout &L, uint32_t *ext8,
                            bool build_polygon, unsigned long long *zero_ptr, int64_t zero_words,
                            cudaStream_t st, bool spec = false, const void *learn_params = nullptr,
                            float *learn_dirs = nullptr, int32_t *learn_k = nullptr);

cudaError_t launch_octagon(const float *pts, int64_t n, const uint32_t *ext8, void *ws, const Layout &L,
                           unsigned long long *zero_ptr, int64_t zero_words, cudaStream_t st);

// point test + stable compaction.  keys_mode: write (x key, (y key, index))
// pairs into the sort buffers of ws instead of (index, point) outputs.
// variant: 0 two passes (needs keep_bits in L), 1 single pass, -1 the
// process-wide choice of ch_filter_variant.  fan (hull step, two passes
// only): launch_fan between the count and the scatter pass.  data_extremes:
// the polygon was built from the data's own extremes (ch_hull,
// ch_extremes_filter; always so in keys mode), which allows the speculative
// sweep's candidates; otherwise the vertices are the caller's (ch_filter).
// A second polygon between the count pass and the fan (two passes only):
// the K-direction polygon over the octagon's survivors (launch_kx_sv).
struct KgonStage {
    const float *dirs;       // device, K directions (cos, sin)
    const int32_t *kdev;     // device choice of K, or NULL: K below
    int K;                   // 16, 32 or 64 (8: no stage) when kdev is NULL
    uint32_t *ext_out;       // device, K vertex indices, or NULL
};
cudaError_t launch_filter(const float *pts, int64_t n, void *ws, const Layout &L, uint32_t *surv_idx,
                          float *surv_pts, uint32_t *surv_count, bool keys_mode, cudaStream_t st,
                          int variant = -1, bool fan = false, bool data_extremes = false,
                          const KgonStage *kgon = nullptr);

// the process-wide compaction schedule (ch_filter_variant)
int filter_variant();

// the filter's scatter pass alone, on keep bits, tile counts and block
// totals that a count pass of `grid` blocks (same layout as the filter's)
// left in ws
cudaError_t launch_filter_scatter(const float *pts, int64_t n, int64_t grid, void *ws, const Layout &L,
                                  uint32_t *surv_idx, float *surv_pts, uint32_t *surv_count, bool keys_mode,
                                  cudaStream_t st);

// blocks per SM set by ch_tune_set for a batched kernel (0: built-in choice)
int tune_value(int knob);

// K-direction filter polygon (kfilter.cu): extremes sweep + polygon, then
// the count pass; returns the count grid through *grid (for the scatter)
cudaError_t launch_kx_extremes(const float *pts, int64_t n, const float *dirs, int K, uint32_t *ext_out, void *ws,
                               const Layout &L, cudaStream_t st);
cudaError_t launch_kx_count(const float *pts, int64_t n, int K, void *ws, const Layout &L, int64_t *grid,
                            cudaStream_t st);

// a K-direction polygon over the octagon's survivors, refining the count
// pass's keep bits (bc blocks); K is the host's (16, 32, 64; 8: nothing)
// or, with kdev, the device's choice.  ext_out (nullable): its vertices.
cudaError_t launch_kx_sv(const float *pts, int64_t n, const float *dirs, const int32_t *kdev, int K, uint32_t *ext_out,
                        void *ws, const Layout &L, int64_t bc, cudaStream_t st);
// the learned proposal in one block (mlp.cu): features, the MLP, the choice
// of K and the directions, into the workspace's LearnScratch
cudaError_t launch_learned_choice(const float *pts, int64_t n, const void *params, void *ws, const Layout &L,
                                  cudaStream_t st);

// hull step: the fan test applied to the keep bits, tile counts and block
// totals that the filter's count pass (filter_blocks blocks) left in ws;
// may do nothing.  vec: the count pass used 16-byte point pairs.
// The second fan level over the survivors the filter's scatter wrote (sort
// keys and payloads in buffer 0): when it runs, the kept ones go to buffer 1
// and the sort reads those (Ctrl::sort_in).  After launch_fan and the
// scatter of the same call; does nothing for sets without its tables.
cudaError_t launch_fan2(int64_t n, void *ws, const Layout &L, cudaStream_t st);
cudaError_t launch_fan(const float *pts, int64_t n, bool vec, int64_t filter_blocks, void *ws, const Layout &L,
                       cudaStream_t st);

// the whole hull in one block when few points survived the filter (the
// sort and chain kernels then stop at once); otherwise nothing
cudaError_t launch_small_hull(void *ws, const Layout &L, uint32_t *hull_idx, uint32_t *hull_count, cudaStream_t st);

// stable LSD radix sort of the survivor (key, index) pairs held in ws
cudaError_t launch_sort(void *ws, const Layout &L, cudaStream_t st);

// monotone chain over the sorted survivors; writes the hull
cudaError_t launch_chain(void *ws, const Layout &L, uint32_t *hull_idx, uint32_t *hull_count, cudaStream_t st);

// ---- many sets (ch_hull_batched); every stage works per set
// validates offsets (points beyond n_cap: CH_ERR_CAPACITY) and maps tiles to sets
cudaError_t launch_bx_setup(const int64_t *offsets, void *ws, const Layout &L, const BatchLayout &BL,
                            int64_t n_cap, cudaStream_t st);
cudaError_t launch_bx_extremes(const float *pts, void *ws, const Layout &L, const BatchLayout &BL, cudaStream_t st);
cudaError_t launch_bx_filter(const float *pts, void *ws, const Layout &L, const BatchLayout &BL, cudaStream_t st);
// the fan test of the sets with many octagon survivors, on the batched
// count pass's keep bits and tile counts (kgon.cu)
cudaError_t launch_bx_fan(const float *pts, void *ws, const Layout &L, const BatchLayout &BL, cudaStream_t st);
cudaError_t launch_bx_sort(void *ws, const Layout &L, const BatchLayout &BL, cudaStream_t st);
cudaError_t launch_bx_chain(void *ws, const Layout &L, const BatchLayout &BL, cudaStream_t st);
cudaError_t launch_bx_finish(void *ws, const Layout &L, const BatchLayout &BL, uint32_t *hull_idx,
                             int64_t *hull_offsets, cudaStream_t st);

}  // namespace ch

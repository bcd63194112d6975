// api.cu -- the extern "C" entry points declared in include/convhull.h.
// Host code only: argument checks, workspace layout, launches.  No
// allocation, no host synchronisation (except ch_last_error), no host
// fallback: every step of Algorithm 1 runs in the kernels of this library.
#include <algorithm>
#include <atomic>
#include <cstring>

#include "common.cuh"
#include "launch.h"

using namespace ch;

namespace {

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

inline ch_status check_ws(void *ws, size_t ws_bytes, const Layout &L)
{
    if (!ws || !aligned(ws, 256)) return CH_ERR_ARG;
    if (ws_bytes < L.total) return CH_ERR_CAPACITY;
    return CH_OK;
}

inline ch_status cuda_status(cudaError_t e) { return e == cudaSuccess ? CH_OK : CH_ERR_CUDA; }

// Workspace bytes of a batched call over n points in B sets.
size_t batched_bytes(int64_t n, int64_t B) { return make_batch_layout(make_layout(n, B), B).total; }

}  // namespace

namespace ch {
namespace {
// process-wide knobs, read when a batched call enqueues its kernels
std::atomic<int> g_tune[CH_TUNE_COUNT] = {};
}
int tune_value(int knob)
{
    return knob >= 0 && knob < CH_TUNE_COUNT ? g_tune[knob].load(std::memory_order_relaxed) : 0;
}
}  // namespace ch

extern "C" ch_status ch_tune_set(int32_t knob, int32_t value)
{
    if (knob < 0 || knob >= CH_TUNE_COUNT || value < 0 || value > 64) return CH_ERR_ARG;
    if (knob == CH_TUNE_BX_FAN_CHUNK && value && value != 8 && value != 16 && value != 32 && value != 64)
        return CH_ERR_ARG;
    if (knob == CH_TUNE_BX_EXT_ITEMS && value && value != 4 && value != 8 && value != 16) return CH_ERR_ARG;
    if (knob == CH_TUNE_FAN2_MIN_LOG2 && value && (value < 10 || value > 31)) return CH_ERR_ARG;
    ch::g_tune[knob].store(value, std::memory_order_relaxed);
    return CH_OK;
}

extern "C" ch_status ch_tune_get(int32_t knob, int32_t *value)
{
    if (knob < 0 || knob >= CH_TUNE_COUNT || !value) return CH_ERR_ARG;
    *value = ch::g_tune[knob].load(std::memory_order_relaxed);
    return CH_OK;
}

extern "C" ch_status ch_workspace_size(int64_t n, int64_t num_sets, size_t *bytes)
{
    if (!bytes || n < 0 || num_sets < 1) return CH_ERR_ARG;
    if (n > kMaxN) return CH_ERR_CAPACITY;
    // room for either layout: the single-set one (ch_hull and the filters:
    // it has the second fan level's tables from kFan2MinN points) and the
    // batched one for num_sets sets
    *bytes = std::max(make_layout(n).total, batched_bytes(n, num_sets));
    return CH_OK;
}

extern "C" ch_status ch_workspace_init(void *ws, size_t ws_bytes, void *stream)
{
    if (!ws || !aligned(ws, 256) || ws_bytes < sizeof(Persist)) return CH_ERR_ARG;
    return cuda_status(cudaMemsetAsync(ws, 0, ws_bytes, as_stream(stream)));
}

extern "C" ch_status ch_extremes(const float *pts, int64_t n, uint32_t *ext8, void *ws, size_t ws_bytes,
                                 void *stream)
{
    if (!pts || !ext8 || n < 1 || !aligned(pts, 8) || !aligned(ext8, 4)) return CH_ERR_ARG;
    if (n > kMaxN) return CH_ERR_CAPACITY;
    const Layout L = make_layout(n);
    if (ch_status s = check_ws(ws, ws_bytes, L)) return s;
    return cuda_status(launch_extremes(pts, n, ws, L, ext8, false, nullptr, 0, as_stream(stream)));
}

extern "C" ch_status ch_filter(const float *pts, int64_t n, const uint32_t *ext8, uint32_t *surv_idx,
                               float *surv_pts, uint32_t *surv_count, void *ws, size_t ws_bytes, void *stream)
{
    if (!surv_count || n < 0 || !aligned(surv_count, 4)) return CH_ERR_ARG;
    if (n > kMaxN) return CH_ERR_CAPACITY;
    cudaStream_t st = as_stream(stream);
    if (n == 0) return cuda_status(cudaMemsetAsync(surv_count, 0, sizeof(uint32_t), st));
    if (!pts || !ext8 || !surv_idx || !aligned(pts, 8) || !aligned(ext8, 4) || !aligned(surv_idx, 4) ||
        (surv_pts && !aligned(surv_pts, 8)))
        return CH_ERR_ARG;
    const Layout L = make_layout(n);
    if (ch_status s = check_ws(ws, ws_bytes, L)) return s;
    cudaError_t e = launch_octagon(pts, n, ext8, ws, L, at<unsigned long long>(ws, L.ctrl),
                                   (int64_t)L.zero_words, st);
    if (e != cudaSuccess) return CH_ERR_CUDA;
    return cuda_status(launch_filter(pts, n, ws, L, surv_idx, surv_pts, surv_count, false, st));
}

extern "C" ch_status ch_extremes_filter(const float *pts, int64_t n, uint32_t *ext8, uint32_t *surv_idx,
                                        float *surv_pts, uint32_t *surv_count, void *ws, size_t ws_bytes,
                                        void *stream)
{
    if (!surv_count || n < 0 || !aligned(surv_count, 4)) return CH_ERR_ARG;
    if (n > kMaxN) return CH_ERR_CAPACITY;
    cudaStream_t st = as_stream(stream);
    if (n == 0) return cuda_status(cudaMemsetAsync(surv_count, 0, sizeof(uint32_t), st));
    if (!pts || !ext8 || !surv_idx || !aligned(pts, 8) || !aligned(ext8, 4) || !aligned(surv_idx, 4) ||
        (surv_pts && !aligned(surv_pts, 8)))
        return CH_ERR_ARG;
    const Layout L = make_layout(n);
    if (ch_status s = check_ws(ws, ws_bytes, L)) return s;
    const int variant = filter_variant();
    cudaError_t e = launch_extremes(pts, n, ws, L, ext8, true, at<unsigned long long>(ws, L.ctrl),
                                    (int64_t)L.zero_words, st, variant == 0);
    if (e == cudaSuccess)
        e = launch_filter(pts, n, ws, L, surv_idx, surv_pts, surv_count, false, st, variant, false, true);
    return cuda_status(e);
}

namespace {

inline bool kgon_k_ok(int32_t K) { return K == 8 || K == 16 || K == 32 || K == 64; }

}  // namespace

extern "C" ch_status ch_filter_kgon(const float *pts, int64_t n, const float *dirs, int32_t K, uint32_t *ext_out,
                                    uint32_t *surv_idx, float *surv_pts, uint32_t *surv_count, void *ws,
                                    size_t ws_bytes, void *stream)
{
    if (!surv_count || n < 0 || !aligned(surv_count, 4) || !kgon_k_ok(K)) return CH_ERR_ARG;
    if (n > kMaxN) return CH_ERR_CAPACITY;
    cudaStream_t st = as_stream(stream);
    if (n == 0) return cuda_status(cudaMemsetAsync(surv_count, 0, sizeof(uint32_t), st));
    if (!pts || !dirs || !surv_idx || !aligned(pts, 8) || !aligned(dirs, 4) || !aligned(surv_idx, 4) ||
        (surv_pts && !aligned(surv_pts, 8)) || (ext_out && !aligned(ext_out, 4)))
        return CH_ERR_ARG;
    const Layout L = make_layout(n);
    if (ch_status s = check_ws(ws, ws_bytes, L)) return s;
    int64_t grid = 0;
    cudaError_t e = launch_kx_extremes(pts, n, dirs, K, ext_out, ws, L, st);
    if (e == cudaSuccess) e = launch_kx_count(pts, n, K, ws, L, &grid, st);
    if (e == cudaSuccess) {
        probe_before(CH_K_FILTER, st);
        e = launch_filter_scatter(pts, n, grid, ws, L, surv_idx, surv_pts, surv_count, false, st);
        probe_after(CH_K_FILTER, st);
    }
    return cuda_status(e);
}

extern "C" ch_status ch_hull_kgon(const float *pts, int64_t n, const float *dirs, int32_t K, uint32_t *hull_idx,
                                  uint32_t *hull_count, void *ws, size_t ws_bytes, void *stream)
{
    if (!hull_count || n < 0 || !aligned(hull_count, 4) || !kgon_k_ok(K)) return CH_ERR_ARG;
    if (n >= kMaxHullN) return CH_ERR_CAPACITY;
    cudaStream_t st = as_stream(stream);
    if (n == 0) return cuda_status(cudaMemsetAsync(hull_count, 0, sizeof(uint32_t), st));
    if (!pts || !dirs || !hull_idx || !aligned(pts, 8) || !aligned(dirs, 4) || !aligned(hull_idx, 4))
        return CH_ERR_ARG;
    const Layout L = make_layout(n);
    if (ch_status s = check_ws(ws, ws_bytes, L)) return s;
    int64_t grid = 0;
    cudaError_t e = launch_kx_extremes(pts, n, dirs, K, nullptr, ws, L, st);
    if (e == cudaSuccess) e = launch_kx_count(pts, n, K, ws, L, &grid, st);
    if (e == cudaSuccess) {
        probe_before(CH_K_FILTER, st);
        e = launch_filter_scatter(pts, n, grid, ws, L, nullptr, nullptr, nullptr, true, st);
        probe_after(CH_K_FILTER, st);
    }
    if (e == cudaSuccess) e = launch_small_hull(ws, L, hull_idx, hull_count, st);
    if (e == cudaSuccess) e = launch_sort(ws, L, st);
    if (e == cudaSuccess) e = launch_chain(ws, L, hull_idx, hull_count, st);
    return cuda_status(e);
}

namespace {

// ch_hull's launches with an optional second polygon between the octagon's
// count pass and the fan
cudaError_t hull_pipeline(const float *pts, int64_t n, uint32_t *hull_idx, uint32_t *hull_count, void *ws,
                          const Layout &L, const KgonStage *kg, cudaStream_t st, const void *learn_params = nullptr,
                          float *learn_dirs = nullptr, int32_t *learn_k = nullptr)
{
    const int variant = filter_variant();
    cudaError_t e = launch_extremes(pts, n, ws, L, at<uint32_t>(ws, L.ext8), true,
                                    at<unsigned long long>(ws, L.ctrl), (int64_t)L.zero_words, st, variant == 0,
                                    learn_params, learn_dirs, learn_k);
    if (e == cudaSuccess) e = launch_filter(pts, n, ws, L, nullptr, nullptr, nullptr, true, st, variant, true, true, kg);
    if (e == cudaSuccess) e = launch_small_hull(ws, L, hull_idx, hull_count, st);
    if (e == cudaSuccess) e = launch_sort(ws, L, st);
    if (e == cudaSuccess) e = launch_chain(ws, L, hull_idx, hull_count, st);
    return e;
}

}  // namespace

extern "C" ch_status ch_hull(const float *pts, int64_t n, uint32_t *hull_idx, uint32_t *hull_count, void *ws,
                             size_t ws_bytes, void *stream)
{
    if (!hull_count || n < 0 || !aligned(hull_count, 4)) return CH_ERR_ARG;
    if (n >= kMaxHullN) return CH_ERR_CAPACITY;
    cudaStream_t st = as_stream(stream);
    if (n == 0) return cuda_status(cudaMemsetAsync(hull_count, 0, sizeof(uint32_t), st));
    if (!pts || !hull_idx || !aligned(pts, 8) || !aligned(hull_idx, 4)) return CH_ERR_ARG;
    const Layout L = make_layout(n);
    if (ch_status s = check_ws(ws, ws_bytes, L)) return s;
    // the two-pass schedule takes the speculative sweep's candidates
    return cuda_status(hull_pipeline(pts, n, hull_idx, hull_count, ws, L, nullptr, st));
}


extern "C" ch_status ch_hull_octagon_kgon(const float *pts, int64_t n, const float *dirs, int32_t K, uint32_t *ext_out,
                                          uint32_t *hull_idx, uint32_t *hull_count, void *ws, size_t ws_bytes,
                                          void *stream)
{
    if (!hull_count || n < 0 || !aligned(hull_count, 4) || !kgon_k_ok(K)) return CH_ERR_ARG;
    if (n >= kMaxHullN) return CH_ERR_CAPACITY;
    cudaStream_t st = as_stream(stream);
    if (n == 0) return cuda_status(cudaMemsetAsync(hull_count, 0, sizeof(uint32_t), st));
    if (!pts || !hull_idx || !aligned(pts, 8) || !aligned(hull_idx, 4) || (K != 8 && (!dirs || !aligned(dirs, 4))) ||
        (ext_out && !aligned(ext_out, 4)))
        return CH_ERR_ARG;
    const Layout L = make_layout(n);
    if (ch_status s = check_ws(ws, ws_bytes, L)) return s;
    const KgonStage kg{dirs, nullptr, K, ext_out};
    return cuda_status(hull_pipeline(pts, n, hull_idx, hull_count, ws, L, &kg, st));
}

extern "C" ch_status ch_hull_learned(const float *pts, int64_t n, const void *params, float *dirs_out, int32_t *k_out,
                                     uint32_t *hull_idx, uint32_t *hull_count, void *ws, size_t ws_bytes, void *stream)
{
    if (!hull_count || n < 0 || !aligned(hull_count, 4)) return CH_ERR_ARG;
    if (n >= kMaxHullN) return CH_ERR_CAPACITY;
    cudaStream_t st = as_stream(stream);
    if (n == 0) return cuda_status(cudaMemsetAsync(hull_count, 0, sizeof(uint32_t), st));
    if (!pts || !params || !hull_idx || !aligned(pts, 8) || !aligned(params, 4) || !aligned(hull_idx, 4) ||
        (dirs_out && !aligned(dirs_out, 4)) || (k_out && !aligned(k_out, 4)))
        return CH_ERR_ARG;
    const Layout L = make_layout(n);
    if (ch_status s = check_ws(ws, ws_bytes, L)) return s;
    // the proposal runs in one more block of the extremes sweep
    LearnScratch *ls = at<LearnScratch>(ws, L.learn);
    const KgonStage kg{ls->dirs, &ls->K, 0, nullptr};
    // (the learned block writes the choice to dirs_out and k_out itself)
    return cuda_status(hull_pipeline(pts, n, hull_idx, hull_count, ws, L, &kg, st, params, dirs_out, k_out));
}

extern "C" ch_status ch_hull_batched(const float *pts, const int64_t *offsets, int32_t num_sets, uint32_t *hull_idx,
                                     int64_t *hull_offsets, void *ws, size_t ws_bytes, void *stream)
{
    if (num_sets < 0 || !offsets || !hull_offsets || !aligned(offsets, 8) || !aligned(hull_offsets, 8))
        return CH_ERR_ARG;
    cudaStream_t st = as_stream(stream);
    if (num_sets == 0) return cuda_status(cudaMemsetAsync(hull_offsets, 0, sizeof(int64_t), st));
    if (!pts || !hull_idx || !aligned(pts, 8) || !aligned(hull_idx, 4)) return CH_ERR_ARG;
    if (!ws || !aligned(ws, 256)) return CH_ERR_ARG;
    // The total point count offsets[num_sets] is only known on the device:
    // the layout is built for the most points the workspace can hold, and
    // the device checks the offsets against that capacity.
    if (ws_bytes < batched_bytes(0, num_sets)) return CH_ERR_CAPACITY;
    int64_t lo = 0, hi = kMaxHullN - 1;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (batched_bytes(mid, num_sets) <= ws_bytes) lo = mid;
        else hi = mid - 1;
    }
    const int64_t n_cap = lo;
    const Layout L = make_layout(std::max<int64_t>(n_cap, 1), num_sets);
    const BatchLayout BL = make_batch_layout(L, num_sets);
    cudaError_t e = cudaMemsetAsync(at<char>(ws, L.ctrl), 0, L.zero_words * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(at<char>(ws, BL.zero_begin), 0, BL.zero_end - BL.zero_begin, st);
    if (e == cudaSuccess) e = launch_bx_setup(offsets, ws, L, BL, n_cap, st);
    if (e == cudaSuccess) e = launch_bx_extremes(pts, ws, L, BL, st);
    if (e == cudaSuccess) e = launch_bx_filter(pts, ws, L, BL, st);
    if (e == cudaSuccess) e = launch_bx_sort(ws, L, BL, st);
    if (e == cudaSuccess) e = launch_bx_chain(ws, L, BL, st);
    if (e == cudaSuccess) e = launch_bx_finish(ws, L, BL, hull_idx, hull_offsets, st);
    return cuda_status(e);
}

extern "C" ch_status ch_hull_counts(void *ws, size_t ws_bytes, int64_t n, uint32_t *counts, void *stream)
{
    if (!counts || n < 1) return CH_ERR_ARG;
    if (n >= kMaxHullN) return CH_ERR_CAPACITY;
    const Layout L = make_layout(n);
    if (ch_status s = check_ws(ws, ws_bytes, L)) return s;
    if (cudaStreamSynchronize(as_stream(stream)) != cudaSuccess) return CH_ERR_CUDA;
    uint32_t sorted = 0, s_oct = 0, spec = 0;
    Fan2Ctrl f2{};
    if (cudaMemcpy(&sorted, &at<Ctrl>(ws, L.ctrl)->surv_count, 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&s_oct, &at<KgonCtrl>(ws, L.kgon_ctrl)->s_oct, 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&spec, &at<Octagon>(ws, L.oct)->spec, 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&f2, at<Fan2Ctrl>(ws, L.fan2), sizeof f2, cudaMemcpyDeviceToHost) != cudaSuccess)
        return CH_ERR_CUDA;
    counts[0] = s_oct ? s_oct : sorted;
    counts[1] = sorted;
    counts[2] = spec;
    counts[3] = f2.on ? f2.count_in : sorted;
    return CH_OK;
}

extern "C" ch_status ch_last_error(void *ws, void *stream)
{
    if (!ws || !aligned(ws, 256)) return CH_ERR_ARG;
    cudaStream_t st = as_stream(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return CH_ERR_CUDA;
    Persist *p = at<Persist>(ws, 0);
    uint32_t code = 0;
    if (cudaMemcpy(&code, &p->error, sizeof code, cudaMemcpyDeviceToHost) != cudaSuccess) return CH_ERR_CUDA;
    if (code != 0 && cudaMemset(p, 0, 2 * sizeof(uint32_t)) != cudaSuccess) return CH_ERR_CUDA;
    return static_cast<ch_status>(code);
}

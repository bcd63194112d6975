// probe.cu -- launch counting and optional CUDA-event timing of each kernel
// of the path (instrumentation; see ch_probe_start / ch_probe_stop).
#include <atomic>
#include <vector>

#include "common.cuh"
#include "launch.h"

namespace ch {

namespace {

// Launch counts and the mask are atomics, so calls from several host threads
// do not race on them; the event lists are touched only while a probe is
// active, which is meant for one host thread at a time.
struct ProbeState {
    std::atomic<uint32_t> mask{0};
    int32_t cap = 0;
    std::atomic<int64_t> launches[CH_K_COUNT] = {};
    std::vector<cudaEvent_t> ev[CH_K_COUNT];   // begin/end pairs
    int32_t used[CH_K_COUNT] = {0};
    bool pending[CH_K_COUNT] = {false};
};

ProbeState g_probe;

}  // namespace

void note_kernels(int kid, int count) { g_probe.launches[kid].fetch_add(count, std::memory_order_relaxed); }

void probe_before(int kid, cudaStream_t st)
{
    if (!((g_probe.mask.load(std::memory_order_relaxed) >> kid) & 1u) || g_probe.used[kid] >= g_probe.cap) return;
    cudaEventRecord(g_probe.ev[kid][2 * g_probe.used[kid]], st);
    g_probe.pending[kid] = true;
}

void probe_after(int kid, cudaStream_t st)
{
    if (!g_probe.pending[kid]) return;
    cudaEventRecord(g_probe.ev[kid][2 * g_probe.used[kid] + 1], st);
    ++g_probe.used[kid];
    g_probe.pending[kid] = false;
}

}  // namespace ch

using namespace ch;

static void release_events()
{
    for (int k = 0; k < CH_K_COUNT; ++k) {
        for (cudaEvent_t e : g_probe.ev[k]) cudaEventDestroy(e);
        g_probe.ev[k].clear();
        g_probe.used[k] = 0;
        g_probe.pending[k] = false;
    }
}

extern "C" ch_status ch_probe_start(uint32_t kernel_mask, int32_t max_launches)
{
    if (max_launches < 0 || (kernel_mask && max_launches == 0)) return CH_ERR_ARG;
    release_events();
    const uint32_t mask = kernel_mask & ((1u << CH_K_COUNT) - 1u);
    g_probe.mask = 0;
    g_probe.cap = max_launches;
    for (int k = 0; k < CH_K_COUNT; ++k) {
        g_probe.launches[k] = 0;
        if ((mask >> k) & 1u) {
            g_probe.ev[k].resize(2 * (size_t)max_launches);
            for (auto &e : g_probe.ev[k])
                if (cudaEventCreate(&e) != cudaSuccess) {
                    e = nullptr;
                    release_events();
                    return CH_ERR_CUDA;
                }
        }
    }
    g_probe.mask = mask;   // events exist before any launch may record them
    return CH_OK;
}

extern "C" ch_status ch_probe_stop(double *ms, int64_t *launches)
{
    ch_status rc = CH_OK;
    for (int k = 0; k < CH_K_COUNT; ++k) {
        double total = 0.0;
        for (int32_t i = 0; i < g_probe.used[k]; ++i) {
            float t = 0.0f;
            if (cudaEventSynchronize(g_probe.ev[k][2 * i + 1]) != cudaSuccess ||
                cudaEventElapsedTime(&t, g_probe.ev[k][2 * i], g_probe.ev[k][2 * i + 1]) != cudaSuccess) {
                rc = CH_ERR_CUDA;
                break;
            }
            total += t;
        }
        if (ms) ms[k] = total;
        if (launches) launches[k] = g_probe.launches[k].load();
    }
    g_probe.mask = 0;
    release_events();
    return rc;
}

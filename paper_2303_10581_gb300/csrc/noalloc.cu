// noalloc.cu -- ch_filter_noalloc: the filter of ch_filter for callers that
// cannot allocate device memory and cannot hand the library a workspace
// either (for example a host framework that owns every device allocation,
// or a code path under a fixed memory budget or a latency budget that
// cudaMalloc's implicit synchronisation would break).
//
// The scratch the filter needs -- the polygon record, the tile tickets, the
// look-back status of every 4096-point tile and the error word -- lives in
// one file-scope device array, g_filter_scratch, of kNoAllocScratchBytes
// bytes.  Every GPU that loads this library keeps that array until the
// process exits.  It bounds n to kNoAllocMaxN points.
//
// In host code the name g_filter_scratch is only a host-side stand-in for
// the device array, not a device address: handing it to a kernel would
// fault, or on systems where the GPU can reach host memory silently use the
// wrong memory.  The first call on each device therefore looks up the real
// device address with cudaGetSymbolAddress (with that device current) and
// caches it; that first call should be made before any stream capture.  A
// cudaDeviceReset destroys the array with the context, and the cached
// address with it: after a reset this entry point must not be called again
// in the same process.
//
// All calls share the one array and it keeps whatever the last call left:
// each call clears the error word with cudaMemsetAsync and the polygon
// kernel clears the tickets and the look-back status before the filter
// runs.  Calls whose work overlaps on the GPU (different streams, or
// several host threads) race on the array and must be serialised by the
// caller.
//
// A caller of this entry point has no workspace to ask ch_last_error about,
// so device-side errors (a vertex index >= n, a look-back wait that gave
// up) come back in the count itself: a last one-thread kernel replaces
// *surv_count by kNoAllocFailed | code when the error word is set.
#include <mutex>

#include "common.cuh"
#include "launch.h"

namespace ch {

namespace {

constexpr int64_t kNoAllocMaxN = (int64_t)1 << 26;          // 67,108,864 points
constexpr size_t kNoAllocScratchBytes = 160 * 1024;         // 160 KiB per device

static __device__ __align__(256) unsigned char g_filter_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// The part of the workspace layout the polygon and filter kernels touch
// (error word, polygon, control block, filter look-back status); nothing
// after the look-back status is used, so the layout ends there.
Layout filter_only_layout(int64_t n)
{
    Layout L = make_layout(n);
    L.n_nodes = 0;
    L.node_cnt = L.filt_status + (size_t)L.filt_tiles * 8;
    L.zero_words = (L.node_cnt - L.ctrl + 7) / 8;
    L.total = align_up(L.node_cnt, 256);
    return L;
}

// Device address of g_filter_scratch on the current device (looked up once).
ch_status scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CH_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_filter_scratch) != cudaSuccess || !p) return CH_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return CH_OK;
}

inline bool aligned_to(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

constexpr uint32_t kNoAllocFailed = 0x80000000u;   // no valid count reaches 2^31 (n <= 2^26)

// Runs after the filter on the same stream: reports a device-side error of
// this call through the count.
__global__ void noalloc_status_kernel(void *scratch, Layout L, uint32_t *surv_count)
{
    const uint32_t code = at<Persist>(scratch, L.persist)->error;
    if (code != 0u) *surv_count = kNoAllocFailed | code;
}

}  // namespace

}  // namespace ch

using namespace ch;

extern "C" ch_status ch_filter_noalloc(const float *pts, int64_t n, const uint32_t *ext8, uint32_t *surv_idx,
                                       float *surv_pts, uint32_t *surv_count, void *stream)
{
    if (!surv_count || n < 0 || !aligned_to(surv_count, 4)) return CH_ERR_ARG;
    if (n > kNoAllocMaxN) return CH_ERR_CAPACITY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (n == 0) return cudaMemsetAsync(surv_count, 0, sizeof(uint32_t), st) == cudaSuccess ? CH_OK : CH_ERR_CUDA;
    if (!pts || !ext8 || !surv_idx || !aligned_to(pts, 8) || !aligned_to(ext8, 4) || !aligned_to(surv_idx, 4) ||
        (surv_pts && !aligned_to(surv_pts, 8)))
        return CH_ERR_ARG;
    const Layout L = filter_only_layout(n);
    if (L.total > kNoAllocScratchBytes) return CH_ERR_CAPACITY;
    void *scratch = nullptr;
    if (ch_status s = scratch_address(&scratch)) return s;
    // a stale error word would make look-back waits give up early
    if (cudaMemsetAsync(at<Persist>(scratch, L.persist), 0, sizeof(Persist), st) != cudaSuccess) return CH_ERR_CUDA;
    cudaError_t e = launch_octagon(pts, n, ext8, scratch, L, at<unsigned long long>(scratch, L.ctrl),
                                   (int64_t)L.zero_words, st);
    if (e != cudaSuccess) return CH_ERR_CUDA;
    // the single-pass schedule: its only scratch is the look-back status
    e = launch_filter(pts, n, scratch, L, surv_idx, surv_pts, surv_count, false, st, 1);
    if (e != cudaSuccess) return CH_ERR_CUDA;
    noalloc_status_kernel<<<1, 1, 0, st>>>(scratch, L, surv_count);
    return cudaGetLastError() == cudaSuccess ? CH_OK : CH_ERR_CUDA;
}

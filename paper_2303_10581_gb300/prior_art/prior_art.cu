// prior_art.cu -- the paper's library-based filter variants (Sec. 4:
// thrust-scan, thrust-copy, cub-flagged), built on Thrust and CUB, so that
// the hand-written path can be timed beside them on the same GPU and the
// same inputs.  Context only: nothing in libconvhull calls this library.
//
// Every variant: the eight extremes by library arg-reductions over key
// iterators (x, y, x + y, x - y), the polygon R, TR, T, TL, L, BL, B, BR, a
// flag per point from the plain binary32 test of Sec. 3.2 (kept unless
// strictly left of every edge of non-zero length; binary32 cross products,
// as the paper computes), then the library compaction of the point indices:
//   0 cub-flagged  cub::DeviceReduce::ArgMax/ArgMin, cub::DeviceSelect::Flagged
//   1 thrust-copy  thrust::max_element/min_element, thrust::copy_if
//   2 thrust-scan  thrust::max_element/min_element, thrust::exclusive_scan of
//                  the flags, then a scatter kernel
// Library scratch comes from the caller's buffer (a bump allocator), so no
// call allocates device memory.
#include <cstddef>
#include <cstdint>
#include <new>

#include <cub/device/device_reduce.cuh>
#include <cub/device/device_select.cuh>
#include <thrust/copy.h>
#include <thrust/execution_policy.h>
#include <thrust/extrema.h>
#include <thrust/functional.h>
#include <thrust/iterator/counting_iterator.h>
#include <thrust/iterator/transform_iterator.h>
#include <thrust/scan.h>
#include <thrust/system/cuda/execution_policy.h>

namespace {

struct Key {
    int which;   // 0 x, 1 y, 2 x + y, 3 x - y
    __host__ __device__ float operator()(const float2 &p) const
    {
        return which == 0 ? p.x : which == 1 ? p.y : which == 2 ? p.x + p.y : p.x - p.y;
    }
};

// vertex slot j (R, TR, T, TL, L, BL, B, BR): key and whether it is a maximum
__host__ __device__ inline Key slot_key(int j)
{
    const int w[8] = {0, 2, 1, 3, 0, 2, 1, 3};
    return Key{w[j]};
}
__host__ __device__ inline bool slot_max(int j) { return j == 0 || j == 1 || j == 2 || j == 7; }

struct Scratch {   // bump allocator over the caller's buffer
    using value_type = char;
    char *base;
    size_t cap;
    size_t *used;
    char *allocate(std::ptrdiff_t n)
    {
        const size_t at = (*used + 255) & ~size_t(255);
        if (at + (size_t)n > cap) throw std::bad_alloc();
        *used = at + (size_t)n;
        return base + at;
    }
    void deallocate(char *, size_t) {}
};

__global__ void flags_kernel(const float2 *__restrict__ p, int64_t n, const uint32_t *__restrict__ ext,
                             uint8_t *__restrict__ flag)
{
    __shared__ float2 v[8];
    if (threadIdx.x < 8) v[threadIdx.x] = p[ext[threadIdx.x]];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 q = p[i];
        bool inside = false, any = false;
        bool all_left = true;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float2 a = v[k], b = v[(k + 1) & 7];
            if (a.x == b.x && a.y == b.y) continue;
            any = true;
            const float c = (b.x - a.x) * (q.y - a.y) - (b.y - a.y) * (q.x - a.x);
            all_left = all_left && c > 0.0f;
        }
        inside = any && all_left;
        flag[i] = inside ? 0 : 1;
    }
}

__global__ void scatter_kernel(int64_t n, const uint8_t *__restrict__ flag, const uint32_t *__restrict__ pos,
                               uint32_t *__restrict__ out, uint32_t *count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (flag[i]) out[pos[i]] = (uint32_t)i;
        if (i == n - 1) *count = pos[i] + flag[i];
    }
}

__global__ void set_kernel(uint32_t *dst, uint32_t v) { *dst = v; }

struct NonZero {
    __host__ __device__ bool operator()(uint8_t f) const { return f != 0; }
};

struct Widen {   // flags summed as 32-bit counts
    __host__ __device__ uint32_t operator()(uint8_t f) const { return f; }
};

// layout of the caller's buffer: flags (n B), positions (4n B), ext (32 B),
// cub outputs, then library scratch
struct Layout {
    size_t flags, pos, ext, vals, scratch, total;
};

Layout layout(int64_t n)
{
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t b) { size_t at = o; o = (o + b + 255) & ~size_t(255); return at; };
    L.flags = take((size_t)n);
    L.pos = take((size_t)n * 4);
    L.ext = take(64);
    L.vals = take(64);
    L.scratch = o;
    L.total = o + ((size_t)64 << 20);   // library scratch
    return L;
}

int grid_for(int64_t n)
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t g = (n + 255) / 256;
    return (int)(g < (int64_t)sms * 8 ? (g > 0 ? g : 1) : (int64_t)sms * 8);
}

}  // namespace

extern "C" int pa_workspace_size(int64_t n, size_t *bytes)
{
    if (n < 1 || !bytes) return 1;
    *bytes = layout(n).total;
    return 0;
}

// Survivor indices (ascending) of pts[0, n) into out_idx, their number into
// *count (device).  variant 0, 1, 2 as above.  Returns 0, or 1 for bad
// arguments, 4 for a CUDA or library error.
extern "C" int pa_filter(const float *pts, int64_t n, int variant, uint32_t *out_idx, uint32_t *count, void *ws,
                         size_t ws_bytes, void *stream)
{
    if (!pts || !out_idx || !count || !ws || n < 1 || variant < 0 || variant > 2) return 1;
    const Layout L = layout(n);
    if (ws_bytes < L.total) return 1;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(ws);
    uint8_t *flags = reinterpret_cast<uint8_t *>(base + L.flags);
    uint32_t *pos = reinterpret_cast<uint32_t *>(base + L.pos);
    uint32_t *ext = reinterpret_cast<uint32_t *>(base + L.ext);
    float *vals = reinterpret_cast<float *>(base + L.vals);
    const float2 *p = reinterpret_cast<const float2 *>(pts);
    size_t used = 0;
    Scratch alloc{base + L.scratch, L.total - L.scratch, &used};
    try {
        // 1. the eight extremes
        for (int j = 0; j < 8; ++j) {
            const Key k = slot_key(j);
            if (variant == 0) {
                size_t tb = 0;
                if (slot_max(j)) {
                    auto it = thrust::make_transform_iterator(p, k);
                    cub::DeviceReduce::ArgMax(nullptr, tb, it, vals + j, ext + j, n, st);
                    used = 0;
                    void *t = alloc.allocate((std::ptrdiff_t)tb);
                    if (cub::DeviceReduce::ArgMax(t, tb, it, vals + j, ext + j, n, st) != cudaSuccess) return 4;
                } else {
                    auto it = thrust::make_transform_iterator(p, k);
                    cub::DeviceReduce::ArgMin(nullptr, tb, it, vals + j, ext + j, n, st);
                    used = 0;
                    void *t = alloc.allocate((std::ptrdiff_t)tb);
                    if (cub::DeviceReduce::ArgMin(t, tb, it, vals + j, ext + j, n, st) != cudaSuccess) return 4;
                }
            } else {
                used = 0;
                auto pol = thrust::cuda::par_nosync(alloc).on(st);
                auto it = thrust::make_transform_iterator(p, k);
                const auto e = slot_max(j) ? thrust::max_element(pol, it, it + n) : thrust::min_element(pol, it, it + n);
                set_kernel<<<1, 1, 0, st>>>(ext + j, (uint32_t)(e - it));
            }
        }
        // 2. flags
        flags_kernel<<<grid_for(n), 256, 0, st>>>(p, n, ext, flags);
        // 3. compaction
        used = 0;
        if (variant == 0) {
            size_t tb = 0;
            thrust::counting_iterator<uint32_t> idx(0);
            cub::DeviceSelect::Flagged(nullptr, tb, idx, flags, out_idx, count, n, st);
            void *t = alloc.allocate((std::ptrdiff_t)tb);
            if (cub::DeviceSelect::Flagged(t, tb, idx, flags, out_idx, count, n, st) != cudaSuccess) return 4;
        } else if (variant == 1) {
            auto pol = thrust::cuda::par(alloc).on(st);
            thrust::counting_iterator<uint32_t> idx(0);
            uint32_t *end = thrust::copy_if(pol, idx, idx + n, flags, out_idx, NonZero());
            set_kernel<<<1, 1, 0, st>>>(count, (uint32_t)(end - out_idx));
        } else {
            auto pol = thrust::cuda::par_nosync(alloc).on(st);
            auto wide = thrust::make_transform_iterator(flags, Widen());
            thrust::exclusive_scan(pol, wide, wide + n, pos, 0u);
            scatter_kernel<<<grid_for(n), 256, 0, st>>>(n, flags, pos, out_idx, count);
        }
    } catch (...) {
        return 4;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

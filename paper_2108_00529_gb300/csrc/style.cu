// style.cu -- supernode colour groups (Section 4.3).
//
// Communities are ordered by size (a stable radix sort of (size, id), so
// ties keep id order).  With alpha the total size, the longest prefix of
// that order whose sizes sum to at most alpha / 2 is group 0 (drawn brown);
// the remaining R communities get group 1 + floor(10 * rank / R), from small
// to big.  One block then walks the sorted sizes three times (sums, brown
// count, groups); prefix sums are 64-bit.
#include "bgv_internal.cuh"

namespace bgv {
namespace {
constexpr int kStyleThreads = 1024;

__global__ void k_size_keys(const uint32_t *__restrict__ size, int64_t K, unsigned long long *__restrict__ keys,
                            uint32_t *__restrict__ vals) {
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < K; k += int64_t(gridDim.x) * blockDim.x) {
        keys[k] = size[k];
        vals[k] = uint32_t(k);
    }
}

__device__ unsigned long long block_exclusive_u64(unsigned long long x, unsigned long long *total) {
    __shared__ unsigned long long warp_sums[kStyleThreads / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int w = 0; w < kStyleThreads / 32; ++w) {
            const unsigned long long t = warp_sums[w];
            warp_sums[w] = run;
            run += t;
        }
        warp_sums[kStyleThreads / 32] = run;
    }
    __syncthreads();
    const unsigned long long r = warp_sums[warp] + inc - x;
    *total = warp_sums[kStyleThreads / 32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kStyleThreads) k_colour_groups(const unsigned long long *__restrict__ sizes,
                                                                 const uint32_t *__restrict__ order, int64_t K,
                                                                 uint8_t *__restrict__ group) {
    const int64_t chunk = (K + kStyleThreads - 1) / kStyleThreads;
    const int64_t lo = int64_t(threadIdx.x) * chunk, hi = lo + chunk < K ? lo + chunk : K;
    unsigned long long mine = 0;
    for (int64_t r = lo; r < hi; ++r) mine += sizes[r];
    unsigned long long total;
    unsigned long long cum = block_exclusive_u64(mine, &total);
    // brown: the running size, this community included, stays within alpha/2
    unsigned long long brown = 0;
    for (int64_t r = lo; r < hi; ++r) {
        cum += sizes[r];
        brown += (2 * cum <= total) ? 1 : 0;
    }
    unsigned long long half;
    block_exclusive_u64(brown, &half);
    const int64_t rest = K - int64_t(half);
    for (int64_t r = lo; r < hi; ++r) {
        const int64_t k = order[r];
        group[k] = r < int64_t(half) ? uint8_t(0) : uint8_t(1 + (10 * (r - int64_t(half))) / rest);
    }
}

// Whole-graph drawing (Section 4.3): every node takes its supernode's colour.
__global__ void k_node_colours(int32_t n, const int32_t *__restrict__ node_map, int64_t K,
                               const uint8_t *__restrict__ group, uint8_t *__restrict__ node_colour) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        const int32_t k = node_map[v];
        node_colour[v] = (k >= 0 && k < K) ? group[k] : uint8_t(0);
    }
}
}  // namespace

}  // namespace bgv

using namespace bgv;

namespace {
void carve_style(Carver &c, int64_t K, SortBuffers &sort) { carve_sort(c, K > 0 ? K : 1, true, sort); }
}  // namespace

extern "C" size_t bgv_colour_groups_ws_size(int64_t K) {
    Carver c(nullptr, kHeaderBytes);
    SortBuffers sort;
    carve_style(c, K, sort);
    return c.used();
}

extern "C" int bgv_colour_groups(int64_t K, const uint32_t *sizes, uint8_t *group, int32_t n,
                                 const int32_t *node_map, uint8_t *node_colour, void *ws, size_t ws_bytes,
                                 void *stream) {
    if (K < 0 || K >= 0x7FFFFFFF || (K > 0 && (!sizes || !group))) return BGV_EINVAL;
    if (node_colour && (n < 0 || (n > 0 && !node_map))) return BGV_EINVAL;
    if (!ws || reinterpret_cast<uintptr_t>(ws) % kAlign) return BGV_EINVAL;
    if (ws_bytes < bgv_colour_groups_ws_size(K)) return BGV_ENOSPC;
    if (K == 0) return BGV_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Carver c(ws, kHeaderBytes);
    SortBuffers sort;
    carve_style(c, K, sort);
    note_launch(), k_size_keys<<<grid_for(K, 256, 152 * 8), 256, 0, st>>>(sizes, K, sort.keys[0], sort.vals[0]);
    BGV_TRY(launch_status());
    int res = 0;
    BGV_TRY(radix_sort(sort, K, nullptr, 32, st, &res, status_ptr(ws)));
    note_launch(), k_colour_groups<<<1, kStyleThreads, 0, st>>>(sort.keys[res], sort.vals[res], K, group);
    BGV_TRY(launch_status());
    if (node_colour && n > 0) {
        note_launch(), k_node_colours<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(n, node_map, K, group, node_colour);
        BGV_TRY(launch_status());
    }
    return BGV_OK;
}

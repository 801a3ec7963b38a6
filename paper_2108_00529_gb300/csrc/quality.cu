// quality.cu -- modularity of a labelling (the quality measure the paper
// reports for its communities, Table 1 column M).
//
// Q = sum over communities c of [ in_c / 2m - (vol_c / 2m)^2 ], with in_c
// twice the edges inside c and vol_c the endpoint count of c.  Everything is
// kept as exact integers: the intra-edge total in one counter, vol_c per
// label, sum vol_c^2 in 128 bits; Q = (2m * in - sum vol^2) / (2m)^2 is
// then one FP64 division of exact values, so the result does not depend on
// the order the threads ran in.
#include "bgv_internal.cuh"

namespace bgv {
namespace {
constexpr int kThreads = 256;
constexpr int kSqBlocks = 608;  // partial sums of vol^2 (a fixed count: sized into the workspace)
typedef unsigned __int128 u128;

__global__ void __launch_bounds__(kThreads) k_mod_count(const int32_t *__restrict__ edges, int64_t m, int32_t n,
                                                        const int32_t *__restrict__ labels, uint32_t *__restrict__ vol,
                                                        unsigned long long *intra, uint32_t *status) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e - lane < m; e += stride) {
        bool same = false;
        if (e < m) {
            const int32_t u = edges[2 * e], v = edges[2 * e + 1];
            if (static_cast<uint32_t>(u) < static_cast<uint32_t>(n) &&
                static_cast<uint32_t>(v) < static_cast<uint32_t>(n)) {
                const int32_t a = labels[u], b = labels[v];
                if (static_cast<uint32_t>(a) < static_cast<uint32_t>(n) &&
                    static_cast<uint32_t>(b) < static_cast<uint32_t>(n)) {
                    atomicAdd(&vol[a], 1u);
                    atomicAdd(&vol[b], 1u);
                    same = a == b;
                } else {
                    raise_status(status, BGV_DEV_BADLABEL);
                }
            } else {
                raise_status(status, BGV_DEV_BADEDGE);
            }
        }
        const unsigned mask = __ballot_sync(0xFFFFFFFFu, same);
        if (lane == 0 && mask) atomicAdd(intra, static_cast<unsigned long long>(__popc(mask)));
    }
}

// Per-block sums of vol^2 (each term < 2^64, the sums in 128 bits).
__global__ void __launch_bounds__(kThreads) k_mod_squares(const uint32_t *__restrict__ vol, int32_t n,
                                                          unsigned long long *__restrict__ part) {
    u128 acc = 0;
    for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < n; c += int64_t(gridDim.x) * blockDim.x) {
        const unsigned long long v = vol[c];
        acc += static_cast<u128>(v * v);
    }
    __shared__ unsigned long long lo[kThreads], hi[kThreads];
    lo[threadIdx.x] = static_cast<unsigned long long>(acc);
    hi[threadIdx.x] = static_cast<unsigned long long>(acc >> 64);
    __syncthreads();
    if (threadIdx.x == 0) {
        u128 s = 0;
        for (int t = 0; t < kThreads; ++t) s += (static_cast<u128>(hi[t]) << 64) | lo[t];
        part[2 * blockIdx.x] = static_cast<unsigned long long>(s);
        part[2 * blockIdx.x + 1] = static_cast<unsigned long long>(s >> 64);
    }
}
}  // namespace
}  // namespace bgv

using namespace bgv;

extern "C" size_t bgv_modularity_ws_size(int32_t n) {
    Carver c(nullptr, kHeaderBytes);
    c.take<uint32_t>(size_t(n > 0 ? n : 1));
    c.take<unsigned long long>(1);
    c.take<unsigned long long>(2 * kSqBlocks);
    return c.used();
}

extern "C" int bgv_modularity(const int32_t *edges, int64_t m, int32_t n, const int32_t *labels, double *q_out,
                              void *ws, size_t ws_bytes, void *stream) {
    if (n < 1 || n >= 0x7FFFFFFF || m < 0 || m >= (int64_t(1) << 31) || !q_out) return BGV_EINVAL;
    if ((m > 0 && !edges) || !labels || !ws || reinterpret_cast<uintptr_t>(ws) % kAlign) return BGV_EINVAL;
    if (ws_bytes < bgv_modularity_ws_size(n)) return BGV_ENOSPC;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    *q_out = 0.0;
    if (m == 0) return BGV_OK;
    Carver c(ws, kHeaderBytes);
    uint32_t *vol = c.take<uint32_t>(size_t(n));
    unsigned long long *intra = c.take<unsigned long long>(1);
    unsigned long long *part = c.take<unsigned long long>(2 * kSqBlocks);
    BGV_CUDA(cudaMemsetAsync(vol, 0, sizeof(uint32_t) * size_t(n), st));
    BGV_CUDA(cudaMemsetAsync(intra, 0, sizeof(unsigned long long), st));
    note_launch(), k_mod_count<<<grid_for(m, kThreads, sm_count() * 8), kThreads, 0, st>>>(edges, m, n, labels, vol, intra,
                                                                                   status_ptr(ws));
    BGV_TRY(launch_status());
    note_launch(), k_mod_squares<<<kSqBlocks, kThreads, 0, st>>>(vol, n, part);
    BGV_TRY(launch_status());
    unsigned long long h_intra = 0, h_part[2 * kSqBlocks];
    uint32_t dev_status = 0;
    BGV_CUDA(cudaMemcpyAsync(&h_intra, intra, sizeof(h_intra), cudaMemcpyDeviceToHost, st));
    BGV_CUDA(cudaMemcpyAsync(h_part, part, sizeof(h_part), cudaMemcpyDeviceToHost, st));
    BGV_CUDA(cudaMemcpyAsync(&dev_status, status_ptr(ws), sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    BGV_CUDA(cudaStreamSynchronize(st));
    if (dev_status) return BGV_EDEVICE;
    unsigned __int128 sq = 0;
    for (int b = 0; b < kSqBlocks; ++b)
        sq += (static_cast<unsigned __int128>(h_part[2 * b + 1]) << 64) | h_part[2 * b];
    // Q = (2m * 2 intra - sum vol^2) / (2m)^2; the numerator may be negative
    const unsigned __int128 two_m = 2 * static_cast<unsigned __int128>(m);
    const unsigned __int128 pos = two_m * 2 * h_intra;
    const double num = pos >= sq ? static_cast<double>(pos - sq) : -static_cast<double>(sq - pos);
    *q_out = num / (static_cast<double>(two_m) * static_cast<double>(two_m));
    return BGV_OK;
}

// primitives.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// Both take their element count either from the host or from a device
// scalar, so data-dependent sizes (cut edges, superedges) need no host round
// trip.  Grids are sized for the host-side upper bound; blocks past the
// device count do no work (the radix histogram still writes zeros for them so
// the digit offsets stay consistent).
#include <atomic>

#include "bgv_internal.cuh"

namespace bgv {

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launches_issued() { return g_launches.load(std::memory_order_relaxed); }

// ------------------------------------------------------------------- scan
namespace {
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096

__device__ __forceinline__ int64_t load_count(const int64_t *d_n, int64_t n_cap) {
    if (!d_n) return n_cap;
    int64_t n = *d_n;
    return n < n_cap ? n : n_cap;
}

// Thread-sequential load of kScanItems consecutive elements starting at i0.
__device__ __forceinline__ void load_items(const uint32_t *in, int64_t i0, int64_t n, uint32_t (&v)[kScanItems]) {
    if (i0 + kScanItems <= n && (reinterpret_cast<uintptr_t>(in + i0) & 15) == 0) {
        const uint4 *p = reinterpret_cast<const uint4 *>(in + i0);
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            uint4 t = p[q];
            v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) v[k] = (i0 + k < n) ? in[i0 + k] : 0u;
    }
}

// Block-wide exclusive scan of one value per thread; returns the exclusive
// prefix and writes the block total to *total.
__device__ __forceinline__ uint32_t block_exclusive(uint32_t x, uint32_t *total) {
    __shared__ uint32_t warp_sums[kScanThreads / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = wi - w;
        if (lane == kScanThreads / 32 - 1) warp_sums[kScanThreads / 32] = wi;
    }
    __syncthreads();
    uint32_t r = warp_sums[warp] + inc - x;
    *total = warp_sums[kScanThreads / 32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ in, int64_t n_cap,
                                                              const int64_t *d_n, uint32_t *__restrict__ partials) {
    const int64_t n = load_count(d_n, n_cap);
    const int64_t i0 = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
    uint32_t v[kScanItems];
    load_items(in, i0, n, v);
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s += v[k];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, d);
    __shared__ uint32_t ws[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
        partials[blockIdx.x] = t;
    }
}

// One block scans the tile partials in place (exclusive), looping over
// chunks with a running carry.  partials[nblocks] receives the total.
__global__ void __launch_bounds__(kScanThreads) k_scan_partials(uint32_t *partials, int64_t nblocks) {
    uint32_t carry = 0;
    for (int64_t base = 0; base < nblocks; base += kScanThreads) {
        int64_t i = base + threadIdx.x;
        uint32_t x = i < nblocks ? partials[i] : 0u;
        uint32_t tot;
        uint32_t ex = block_exclusive(x, &tot);
        if (i < nblocks) partials[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) partials[nblocks] = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t *in, uint32_t *out,  // may alias (in-place)
                                                           
                                                            int64_t n_cap, const int64_t *d_n,
                                                            const uint32_t *__restrict__ partials, int64_t nblocks,
                                                            unsigned long long *total_u64, int total_at_end) {
    const int64_t n = load_count(d_n, n_cap);
    const int64_t i0 = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
    uint32_t v[kScanItems];
    load_items(in, i0, n, v);
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s += v[k];
    uint32_t tot;
    uint32_t run = partials[blockIdx.x] + block_exclusive(s, &tot);
    if (i0 + kScanItems <= n && (reinterpret_cast<uintptr_t>(out + i0) & 15) == 0) {
        uint4 *p = reinterpret_cast<uint4 *>(out + i0);
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            uint4 t;
            t.x = run; run += v[4 * q];
            t.y = run; run += v[4 * q + 1];
            t.z = run; run += v[4 * q + 2];
            t.w = run; run += v[4 * q + 3];
            p[q] = t;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (i0 + k < n) out[i0 + k] = run;
            run += v[k];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        uint32_t total = partials[nblocks];
        if (total_u64) *total_u64 = total;
        if (total_at_end) out[n] = total;
    }
}
}  // namespace

size_t scan_tmp_bytes(int64_t n_cap) {
    int64_t nb = (n_cap + kScanTile - 1) / kScanTile;
    if (nb < 1) nb = 1;
    return size_t(nb + 1) * sizeof(uint32_t);
}

int scan_exclusive(const uint32_t *in, uint32_t *out, int64_t n_cap, const int64_t *d_n,
                   unsigned long long *total_u64, bool total_u32_at_end, void *tmp, cudaStream_t s) {
    int64_t nb = (n_cap + kScanTile - 1) / kScanTile;
    if (nb < 1) nb = 1;
    uint32_t *partials = static_cast<uint32_t *>(tmp);
    note_launch(), k_scan_reduce<<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(in, n_cap, d_n, partials);
    note_launch(), k_scan_partials<<<1, kScanThreads, 0, s>>>(partials, nb);
    note_launch(), k_scan_down<<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(in, out, n_cap, d_n, partials, nb, total_u64,
                                                                   total_u32_at_end ? 1 : 0);
    return launch_status();
}

// ------------------------------------------------------------- radix sort
namespace {
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys
constexpr int kBins = 256;
constexpr uint32_t kInvalidDigit = 0xFFFFu;

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const unsigned long long *__restrict__ keys, int64_t cap,
                                                            const int64_t *d_count, int shift,
                                                            uint32_t *__restrict__ hist, int64_t tiles) {
    __shared__ uint32_t h[kSortWarps][kBins];
    for (int i = threadIdx.x; i < kSortWarps * kBins; i += kSortThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const int64_t n = load_count(d_count, cap);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = int64_t(blockIdx.x) * kSortTile + int64_t(warp) * (32 * kSortItems);
    if (int64_t(blockIdx.x) * kSortTile < n) {
#pragma unroll 4
        for (int k = 0; k < kSortItems; ++k) {
            int64_t i = base + int64_t(k) * 32 + lane;
            if (i < n) {
                uint32_t d = static_cast<uint32_t>(keys[i] >> shift) & 0xFFu;
                atomicAdd(&h[warp][d], 1u);
            }
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kBins; d += kSortThreads) {
        uint32_t t = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) t += h[w][d];
        hist[int64_t(d) * tiles + blockIdx.x] = t;
    }
}

template <bool kVals>
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const unsigned long long *__restrict__ kin,
                                                               unsigned long long *__restrict__ kout,
                                                               const uint32_t *__restrict__ vin,
                                                               uint32_t *__restrict__ vout, int64_t cap,
                                                               const int64_t *d_count, int shift,
                                                               const uint32_t *__restrict__ offsets, int64_t tiles) {
    __shared__ uint32_t cnt[kSortWarps][kBins];
    const int64_t n = load_count(d_count, cap);
    if (int64_t(blockIdx.x) * kSortTile >= n) return;
    for (int i = threadIdx.x; i < kSortWarps * kBins; i += kSortThreads) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t base = int64_t(blockIdx.x) * kSortTile + int64_t(warp) * (32 * kSortItems);
    unsigned long long key[kSortItems];
    uint32_t val[kSortItems];
    uint32_t digit[kSortItems];
    uint32_t rank[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        int64_t i = base + int64_t(k) * 32 + lane;
        bool ok = i < n;
        key[k] = ok ? kin[i] : 0ull;
        if (kVals) val[k] = ok ? vin[i] : 0u;
        digit[k] = ok ? (static_cast<uint32_t>(key[k] >> shift) & 0xFFu) : kInvalidDigit;
    }
    // Stable rank within the warp, items in (k, lane) order.
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        uint32_t d = digit[k];
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        uint32_t before = 0;
        if (d != kInvalidDigit) before = cnt[warp][d];
        rank[k] = before + __popc(peers & lt_mask);
        __syncwarp();
        if (d != kInvalidDigit && (peers & lt_mask) == 0) cnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // Per digit: exclusive prefix over warps plus the global offset of this tile.
    for (int d = threadIdx.x; d < kBins; d += kSortThreads) {
        uint32_t run = offsets[int64_t(d) * tiles + blockIdx.x];
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            uint32_t c = cnt[w][d];
            cnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        uint32_t d = digit[k];
        if (d == kInvalidDigit) continue;
        uint32_t pos = cnt[warp][d] + rank[k];
        kout[pos] = key[k];
        if (kVals) vout[pos] = val[k];
    }
}
}  // namespace

int64_t sort_tiles(int64_t cap) {
    int64_t t = (cap + kSortTile - 1) / kSortTile;
    return t < 1 ? 1 : t;
}

size_t sort_hist_entries(int64_t cap) { return size_t(kBins) * size_t(sort_tiles(cap)) + 1; }

void carve_sort(Carver &c, int64_t cap, bool with_vals, SortBuffers &out) {
    out.keys[0] = c.take<unsigned long long>(size_t(cap));
    out.keys[1] = c.take<unsigned long long>(size_t(cap));
    out.vals[0] = with_vals ? c.take<uint32_t>(size_t(cap)) : nullptr;
    out.vals[1] = with_vals ? c.take<uint32_t>(size_t(cap)) : nullptr;
    out.hist = c.take<uint32_t>(sort_hist_entries(cap));
    out.scan_tmp = c.take<char>(scan_tmp_bytes(int64_t(sort_hist_entries(cap))));
}

int radix_sort(SortBuffers &b, int64_t cap, const int64_t *d_count, int end_bit, cudaStream_t s,
               int *result_buffer) {
    const int64_t tiles = sort_tiles(cap);
    const int64_t nh = int64_t(kBins) * tiles;
    int cur = 0;
    for (int shift = 0; shift < end_bit; shift += 8) {
        note_launch(), k_sort_hist<<<static_cast<unsigned>(tiles), kSortThreads, 0, s>>>(b.keys[cur], cap, d_count, shift, b.hist,
                                                                         tiles);
        BGV_TRY(scan_exclusive(b.hist, b.hist, nh, nullptr, nullptr, false, b.scan_tmp, s));
        if (b.vals[0]) {
            note_launch(), k_sort_scatter<true><<<static_cast<unsigned>(tiles), kSortThreads, 0, s>>>(
                b.keys[cur], b.keys[cur ^ 1], b.vals[cur], b.vals[cur ^ 1], cap, d_count, shift, b.hist, tiles);
        } else {
            note_launch(), k_sort_scatter<false><<<static_cast<unsigned>(tiles), kSortThreads, 0, s>>>(
                b.keys[cur], b.keys[cur ^ 1], nullptr, nullptr, cap, d_count, shift, b.hist, tiles);
        }
        BGV_TRY(launch_status());
        cur ^= 1;
    }
    *result_buffer = cur;
    return BGV_OK;
}

}  // namespace bgv

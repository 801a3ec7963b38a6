// hsort.cuh -- sort of (key, id) pairs into (key, id) order, given a hint:
// an order of the ids that is already close to the sorted one.
//
// ForceAtlas2 moves every body a little per iteration, so the previous
// iteration's Morton order of the bodies is such a hint for the next one:
// on the 3.2 M-body rmat22x supergraph, 98.3 % (first iterations) to 99.8 %
// (iteration 500) of the bodies end within 4,096 places of where the
// previous order had them.  The LSD radix sort ignores that; this sort uses
// it to cut the global passes to two (count, scatter) and to sort the rest
// in shared memory, with kernels that need no grid-wide residency.
//
// Method: a sample sort whose buckets follow the hint.
//   1. Samples: the ids at ns evenly spaced places of the hint and their
//      keys, ranked among themselves by counting (ns^2 comparisons spread
//      over many threads; equal pairs ranked by sample index) and stored in
//      (key, id) order.  Splitter u (1 <= u < nb) is sample u*s, with s
//      samples per bucket; bucket u holds the pairs x with
//      splitter(u) <= x < splitter(u+1), splitter(0) = -inf, splitter(nb) =
//      +inf.
//   2. Count: every pair's key and bucket (the search starts at the bucket
//      its place in the hint would have, so a good hint needs one or two
//      probes), counted per bucket with one atomic per bucket per warp; the
//      last block turns the counts into bucket starts.
//   3. Scatter: every pair to its bucket (one atomic per bucket per warp).
//   4. Bucket sort: one block per bucket.  Up to kHsCap pairs it sorts in
//      shared memory, as single words (key - min key) << idbits | id when the
//      bucket's keys span few enough bits, else as pairs: each thread's 4 or
//      8 through a sorting network in registers, then merges of sorted runs
//      by merge path.  A larger bucket (a poor hint) is sorted in chunks and
//      merged in global memory by the same block.
// The result is the (key, id) order for any hint: a poor hint only makes the
// buckets uneven.  A hint entry >= K raises BGV_DEV_BADHINT and is read as
// id 0 (a hint that is not a permutation gives an unspecified result but
// never an access outside the arrays).
#pragma once

#include "bgv_internal.cuh"

namespace bgv {

constexpr int kHsBucket = 1024;         // target pairs per bucket
constexpr int kHsMaxBuckets = 4096;     // so at most 4096 * 1024 pairs
constexpr int kHsMaxSamples = 4096;     // ns <= this
constexpr int kHsMaxPerBucket = 8;      // s <= this
constexpr int kHsThreads = 256;         // bucket-sort block
constexpr int kHsItems = 8;             // pairs (or words) per thread
constexpr int kHsPairCap = kHsThreads * kHsItems;  // 2048: a chunk of the pair sort
constexpr int kHsCap = kHsPairCap;      // larger buckets take the chunked path
constexpr int kHsRankSlices = 16;       // slices of the samples per ranking thread
constexpr int kHsSmem = kHsCap + kHsCap / 16;  // skewed shared-memory slots

inline int64_t hs_max_keys() { return int64_t(kHsMaxBuckets) * kHsBucket; }

// Small device arrays of the sort (the large ones are the caller's).
struct HsBuffers {
    unsigned long long *smp_key;  // [kHsMaxSamples] samples in hint order
    uint32_t *smp_id;             // [kHsMaxSamples]
    uint32_t *smp_rank;           // [kHsMaxSamples]
    unsigned long long *spl_key;  // [kHsMaxBuckets] splitter u at u - 1
    uint32_t *spl_id;             // [kHsMaxBuckets]
    uint32_t *count;              // [kHsMaxBuckets] pairs per bucket
    uint32_t *cursor;             // [kHsMaxBuckets] scatter cursors
    uint32_t *start;              // [kHsMaxBuckets + 1] bucket starts
    uint32_t *ticket;             // [2] last-block tickets
};

inline void carve_hs(Carver &c, HsBuffers &h) {
    h.smp_key = c.take<unsigned long long>(kHsMaxSamples);
    h.smp_id = c.take<uint32_t>(kHsMaxSamples);
    h.smp_rank = c.take<uint32_t>(kHsMaxSamples);
    h.spl_key = c.take<unsigned long long>(kHsMaxBuckets);
    h.spl_id = c.take<uint32_t>(kHsMaxBuckets);
    h.count = c.take<uint32_t>(kHsMaxBuckets);
    h.cursor = c.take<uint32_t>(kHsMaxBuckets);
    h.start = c.take<uint32_t>(kHsMaxBuckets + 1);
    h.ticket = c.take<uint32_t>(2);
}

// Buckets and samples per bucket for K pairs (nb = 1: no splitters).
struct HsShape {
    int nb, s, ns;
};
inline HsShape hs_shape(int64_t K) {
    HsShape h;
    h.nb = int((K + kHsBucket - 1) / kHsBucket);
    if (h.nb < 1) h.nb = 1;
    h.s = kHsMaxSamples / h.nb;
    if (h.s > kHsMaxPerBucket) h.s = kHsMaxPerBucket;
    if (h.s < 1) h.s = 1;
    h.ns = h.nb > 1 ? h.nb * h.s : 0;  // nb > 1 means K > 1024 >= 8 nb, so ns < K
    return h;
}

// Extra words the first kernel clears (for the kernels after the sort).
struct HsClears {
    unsigned long long *u64 = nullptr;
    int64_t n_u64 = 0;
    uint32_t *u32 = nullptr;
    int64_t n_u32 = 0;
};

// The kernels are private to each translation unit that includes this
// header (each instantiates its own key source).
namespace {

__device__ __forceinline__ bool hs_less(unsigned long long ak, uint32_t ai, unsigned long long bk, uint32_t bi) {
    return ak < bk || (ak == bk && ai < bi);
}

__device__ __forceinline__ uint32_t hs_id(const uint32_t *__restrict__ hint, int64_t p, int64_t K,
                                          uint32_t *status) {
    uint32_t id = hint[p];
    if (id >= uint64_t(K)) {
        raise_status(status, BGV_DEV_BADHINT);
        id = 0u;
    }
    return id;
}

// 1a. Sample keys; clears the counters of the later kernels.
template <class KeyOf>
__global__ void __launch_bounds__(256) k_hs_sample(KeyOf key_of, const uint32_t *__restrict__ hint, int64_t K, int nb,
                                                   int ns, HsBuffers h, HsClears clr, uint32_t *status) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t t0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    for (int64_t t = t0; t < ns; t += stride) {
        const int64_t p = ((2 * t + 1) * K) / (2 * int64_t(ns));
        const uint32_t id = hs_id(hint, p, K, status);
        h.smp_key[t] = key_of(id);
        h.smp_id[t] = id;
        h.smp_rank[t] = 0u;
    }
    for (int64_t t = t0; t < nb; t += stride) {
        h.count[t] = 0u;
        h.cursor[t] = 0u;
    }
    if (t0 < 2) h.ticket[t0] = 0u;
    for (int64_t t = t0; t < clr.n_u64; t += stride) clr.u64[t] = 0ull;
    for (int64_t t = t0; t < clr.n_u32; t += stride) clr.u32[t] = 0u;
}

// 1b. Ranks of the samples by counting, one slice of the others per block
// row; the last block places every s-th one as a splitter.
__global__ void __launch_bounds__(256) k_hs_rank(int ns, int s, HsBuffers h) {  // 256 threads
    __shared__ unsigned long long sk[(kHsMaxSamples + kHsRankSlices - 1) / kHsRankSlices];
    __shared__ uint32_t si[(kHsMaxSamples + kHsRankSlices - 1) / kHsRankSlices];
    __shared__ bool last;
    const int per = (ns + kHsRankSlices - 1) / kHsRankSlices;
    const int j0 = blockIdx.y * per;
    const int j1 = min(ns, j0 + per);
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        sk[j - j0] = h.smp_key[j];
        si[j - j0] = h.smp_id[j];
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ns) {
        const unsigned long long ki = h.smp_key[i];
        const uint32_t ii = h.smp_id[i];
        uint32_t c = 0;
        for (int j = j0; j < j1; ++j) {
            const unsigned long long kj = sk[j - j0];
            const uint32_t ij = si[j - j0];
            c += (hs_less(kj, ij, ki, ii) || (kj == ki && ij == ii && j < i)) ? 1u : 0u;
        }
        if (c) atomicAdd(&h.smp_rank[i], c);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&h.ticket[0], 1u) == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // every load first (one round trip to L2), then the placements
    constexpr int kPer = kHsMaxSamples / 256;
    uint32_t r[kPer], id[kPer];
    unsigned long long key[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int t = threadIdx.x + 256 * q;
        r[q] = t < ns ? __ldcg(&h.smp_rank[t]) : 0u;
        key[q] = t < ns ? __ldcg(&h.smp_key[t]) : 0ull;
        id[q] = t < ns ? __ldcg(&h.smp_id[t]) : 0u;
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        if (r[q] >= uint32_t(s) && r[q] % uint32_t(s) == 0u && r[q] < uint32_t(ns)) {
            const uint32_t u = r[q] / uint32_t(s);
            h.spl_key[u - 1] = key[q];
            h.spl_id[u - 1] = id[q];
        }
    }
}

// Bucket of pair x: the smallest u in [0, nb) with u == nb - 1 or
// x < splitter(u + 1) (stored at u), searched outwards from the guess g.
__device__ __forceinline__ int hs_bucket(unsigned long long xk, uint32_t xi, const unsigned long long *__restrict__ sk,
                                         const uint32_t *__restrict__ si, int nb, int g) {
    auto above = [&](int u) { return u >= nb - 1 || hs_less(xk, xi, __ldg(&sk[u]), __ldg(&si[u])); };
    int lo, hi;  // the answer is in [lo, hi]; above(hi); lo == 0 or !above(lo - 1)
    if (above(g)) {
        hi = g;
        for (int d = 1;; d <<= 1) {
            const int u = g - d;
            if (u < 0) {
                lo = 0;
                break;
            }
            if (!above(u)) {
                lo = u + 1;
                break;
            }
            hi = u;
        }
    } else {
        lo = g + 1;
        for (int d = 1;; d <<= 1) {
            const int u = g + d;
            if (u >= nb - 1) {
                hi = nb - 1;
                break;
            }
            if (above(u)) {
                hi = u;
                break;
            }
            lo = u + 1;
        }
    }
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (above(mid))
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// 2. Keys and buckets in hint order, counts per bucket; the last block
// writes the bucket starts.
template <class KeyOf>
__global__ void __launch_bounds__(256) k_hs_count(KeyOf key_of, const uint32_t *__restrict__ hint, int64_t K, int nb,
                                                  HsBuffers h, unsigned long long *__restrict__ tmp_key,
                                                  uint32_t *__restrict__ tmp_bucket, uint32_t *status) {
    __shared__ bool last;
    __shared__ uint32_t part[256];
    const int lane = threadIdx.x & 31;
    // the bucket a hint place would have if the buckets split the hint
    // evenly: the search starts there
    const float g_scale = float(nb) / float(K);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t p0 = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); p0 < K; p0 += stride) {
        const int64_t p = p0 + lane;
        int u = -1;
        if (p < K) {
            const uint32_t id = hs_id(hint, p, K, status);
            const unsigned long long k = key_of(id);
            const int g = min(nb - 1, int(float(p) * g_scale));
            u = nb > 1 ? hs_bucket(k, id, h.spl_key, h.spl_id, nb, g) : 0;
            tmp_key[p] = k;
            tmp_bucket[p] = uint32_t(u);
        }
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, u);
        if (u >= 0 && lane == __ffs(peers) - 1) atomicAdd(&h.count[u], uint32_t(__popc(peers)));
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&h.ticket[1], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // exclusive scan of the counts: a contiguous chunk per thread
    const int per = (nb + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
    uint32_t sum = 0;
    for (int b = b0; b < b1; ++b) sum += __ldcg(&h.count[b]);
    part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int t = 0; t < int(blockDim.x); ++t) {
            const uint32_t c = part[t];
            part[t] = run;
            run += c;
        }
    }
    __syncthreads();
    uint32_t run = part[threadIdx.x];
    for (int b = b0; b < b1; ++b) {
        h.start[b] = run;
        run += __ldcg(&h.count[b]);
    }
    if (threadIdx.x == 0) h.start[nb] = uint32_t(K);
}

// 3. Every pair to its bucket.
__global__ void __launch_bounds__(256) k_hs_scatter(const uint32_t *__restrict__ hint, int64_t K, HsBuffers h,
                                                    const unsigned long long *__restrict__ tmp_key,
                                                    const uint32_t *__restrict__ tmp_bucket,
                                                    unsigned long long *__restrict__ slot_key,
                                                    uint32_t *__restrict__ slot_id) {
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t p0 = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); p0 < K; p0 += stride) {
        const int64_t p = p0 + lane;
        int u = -1;
        unsigned long long k = 0ull;
        uint32_t id = 0u;
        if (p < K) {
            u = int(tmp_bucket[p]);
            k = tmp_key[p];
            id = hint[p];
            if (id >= uint64_t(K)) id = 0u;  // reported by the count kernel
        }
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, u);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0u;
        if (u >= 0 && lane == leader) base = atomicAdd(&h.cursor[u], uint32_t(__popc(peers)));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        if (u >= 0) {
            const uint32_t q = h.start[u] + base + uint32_t(__popc(peers & lt_mask));
            slot_key[q] = k;
            slot_id[q] = id;
        }
    }
}

// 4. Bucket sort.
__device__ __forceinline__ int hs_sw(int i) { return i + (i >> 4); }

__device__ __forceinline__ void hs_ce(unsigned long long (&k)[kHsItems], uint32_t (&v)[kHsItems], int a, int b) {
    if (hs_less(k[b], v[b], k[a], v[a])) {
        const unsigned long long tk = k[a];
        k[a] = k[b];
        k[b] = tk;
        const uint32_t tv = v[a];
        v[a] = v[b];
        v[b] = tv;
    }
}

// Sorts n <= kHsPairCap pairs from (ik, iv) into (ok, ov) (which may alias
// them); every thread of the block calls it.
__device__ void hs_block_sort(const unsigned long long *ik, const uint32_t *iv, int n, unsigned long long *ok,
                              uint32_t *ov, unsigned long long *shk, uint32_t *shv) {
    int P = kHsItems;
    while (P < n) P <<= 1;
    const int t = threadIdx.x;
    const bool act = kHsItems * t < P;
    unsigned long long k[kHsItems];
    uint32_t v[kHsItems];
#pragma unroll
    for (int j = 0; j < kHsItems; ++j) {
        const int q = kHsItems * t + j;
        const bool in = act && q < n;
        k[j] = in ? __ldcg(&ik[q]) : ~0ull;
        v[j] = in ? __ldcg(&iv[q]) : ~0u;
    }
    // Batcher's odd-even merge network for 8 inputs (19 comparators)
    hs_ce(k, v, 0, 1); hs_ce(k, v, 2, 3); hs_ce(k, v, 4, 5); hs_ce(k, v, 6, 7);
    hs_ce(k, v, 0, 2); hs_ce(k, v, 1, 3); hs_ce(k, v, 4, 6); hs_ce(k, v, 5, 7);
    hs_ce(k, v, 1, 2); hs_ce(k, v, 5, 6);
    hs_ce(k, v, 0, 4); hs_ce(k, v, 1, 5); hs_ce(k, v, 2, 6); hs_ce(k, v, 3, 7);
    hs_ce(k, v, 2, 4); hs_ce(k, v, 3, 5);
    hs_ce(k, v, 1, 2); hs_ce(k, v, 3, 4); hs_ce(k, v, 5, 6);
    for (int w = kHsItems; w < P; w <<= 1) {
        __syncthreads();  // the previous round's reads are done
        if (act) {
#pragma unroll
            for (int j = 0; j < kHsItems; ++j) {
                shk[hs_sw(kHsItems * t + j)] = k[j];
                shv[hs_sw(kHsItems * t + j)] = v[j];
            }
        }
        __syncthreads();
        if (act) {
            const int o0 = kHsItems * t;
            const int a0 = o0 & ~(2 * w - 1), b0 = a0 + w;
            const int o = o0 - a0;
            int lo = max(0, o - w), hi = min(o, w);
            while (lo < hi) {  // merge path: A's share of the first o outputs
                const int mid = (lo + hi) >> 1;
                const int bi = hs_sw(b0 + o - mid - 1), ai = hs_sw(a0 + mid);
                if (!hs_less(shk[bi], shv[bi], shk[ai], shv[ai]))
                    lo = mid + 1;
                else
                    hi = mid;
            }
            int ia = a0 + lo, ib = b0 + (o - lo);
            const int ae = a0 + w, be = b0 + w;
#pragma unroll
            for (int j = 0; j < kHsItems; ++j) {
                bool take_a;
                if (ia >= ae)
                    take_a = false;
                else if (ib >= be)
                    take_a = true;
                else
                    take_a = !hs_less(shk[hs_sw(ib)], shv[hs_sw(ib)], shk[hs_sw(ia)], shv[hs_sw(ia)]);
                const int q = hs_sw(take_a ? ia : ib);
                k[j] = shk[q];
                v[j] = shv[q];
                ia += take_a ? 1 : 0;
                ib += take_a ? 0 : 1;
            }
        }
    }
    __syncthreads();  // every read of (ik, iv) and of shared memory is done
    if (act) {
#pragma unroll
        for (int j = 0; j < kHsItems; ++j) {
            const int q = kHsItems * t + j;
            if (q < n) {
                ok[q] = k[j];
                ov[q] = v[j];
            }
        }
    }
    __syncthreads();
}

template <int I>
__device__ __forceinline__ void hs_ce64(unsigned long long (&c)[I], int a, int b) {
    const unsigned long long x = c[a], y = c[b];
    c[a] = x < y ? x : y;
    c[b] = x < y ? y : x;
}

// The same sort on single 64-bit words (no equal words but the padding):
// c holds the thread's I words of a P-word array (P a power of two >= I,
// at most I * blockDim.x); on return they are the thread's words of the
// sorted array.  The thread's words are sorted in registers, then merged.
template <int I>
__device__ void hs_sort_words(unsigned long long (&c)[I], int P, unsigned long long *sh) {
    static_assert(I == 4 || I == 8, "4 or 8 words a thread");
    const int t = threadIdx.x;
    const bool act = I * t < P;
    if constexpr (I == 4) {  // 5 comparators
        hs_ce64(c, 0, 1); hs_ce64(c, 2, 3);
        hs_ce64(c, 0, 2); hs_ce64(c, 1, 3);
        hs_ce64(c, 1, 2);
    } else {  // Batcher's odd-even merge network, 19 comparators
        hs_ce64(c, 0, 1); hs_ce64(c, 2, 3); hs_ce64(c, 4, 5); hs_ce64(c, 6, 7);
        hs_ce64(c, 0, 2); hs_ce64(c, 1, 3); hs_ce64(c, 4, 6); hs_ce64(c, 5, 7);
        hs_ce64(c, 1, 2); hs_ce64(c, 5, 6);
        hs_ce64(c, 0, 4); hs_ce64(c, 1, 5); hs_ce64(c, 2, 6); hs_ce64(c, 3, 7);
        hs_ce64(c, 2, 4); hs_ce64(c, 3, 5);
        hs_ce64(c, 1, 2); hs_ce64(c, 3, 4); hs_ce64(c, 5, 6);
    }
    for (int w = I; w < P; w <<= 1) {  // runs of w words; 2w > I, so a thread's outputs lie in one pair
        __syncthreads();  // the previous round's reads are done
        if (act) {
#pragma unroll
            for (int j = 0; j < I; ++j) sh[hs_sw(I * t + j)] = c[j];
        }
        __syncthreads();
        if (act) {
            const int o0 = I * t;
            const int a0 = o0 & ~(2 * w - 1), b0 = a0 + w;
            const int o = o0 - a0;
            int lo = max(0, o - w), hi = min(o, w);
            while (lo < hi) {  // merge path: A's share of the first o outputs
                const int mid = (lo + hi) >> 1;
                if (sh[hs_sw(a0 + mid)] <= sh[hs_sw(b0 + o - mid - 1)])
                    lo = mid + 1;
                else
                    hi = mid;
            }
            int ia = a0 + lo, ib = b0 + (o - lo);
            const int ae = a0 + w, be = b0 + w;
            unsigned long long va = ia < ae ? sh[hs_sw(ia)] : 0ull, vb = ib < be ? sh[hs_sw(ib)] : 0ull;
#pragma unroll
            for (int j = 0; j < I; ++j) {  // the heads stay in registers
                const bool take_a = ia < ae && (ib >= be || va <= vb);
                c[j] = take_a ? va : vb;
                if (take_a) {
                    ++ia;
                    va = ia < ae ? sh[hs_sw(ia)] : 0ull;
                } else {
                    ++ib;
                    vb = ib < be ? sh[hs_sw(ib)] : 0ull;
                }
            }
        }
    }
}

// n > kHsPairCap pairs (a wide or oversized bucket): chunks sorted in shared
// memory into (dk, dv), then merges of sorted runs in global memory,
// alternating between (dk, dv) and (sk, sv); the result ends in (dk, dv).
// Every thread of the block calls it.
__device__ void hs_pairs_chunked(unsigned long long *sk, uint32_t *sv, int64_t n, unsigned long long *dk,
                                 uint32_t *dv, unsigned long long *shk, uint32_t *shv) {
    for (int64_t c = 0; c < n; c += kHsPairCap)
        hs_block_sort(sk + c, sv + c, int(min(int64_t(kHsPairCap), n - c)), dk + c, dv + c, shk, shv);
    unsigned long long *srck = dk, *dstk = sk;
    uint32_t *srcv = dv, *dstv = sv;
    for (int64_t w = kHsPairCap; w < n; w <<= 1) {
        for (int64_t o0 = int64_t(threadIdx.x) * kHsItems; o0 < n; o0 += int64_t(blockDim.x) * kHsItems) {
            const int64_t a0 = o0 / (2 * w) * (2 * w), b0r = a0 + w;
            const int64_t alen = min(w, n - a0), blen = max(int64_t(0), min(w, n - b0r));
            const int64_t o = o0 - a0;
            int64_t lo = max(int64_t(0), o - blen), hi = min(o, alen);
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                const int64_t bi = b0r + o - mid - 1, ai = a0 + mid;
                if (!hs_less(__ldcg(&srck[bi]), __ldcg(&srcv[bi]), __ldcg(&srck[ai]), __ldcg(&srcv[ai])))
                    lo = mid + 1;
                else
                    hi = mid;
            }
            int64_t ia = a0 + lo, ib = b0r + (o - lo);
            const int64_t ae = a0 + alen, be = b0r + blen;
            for (int j = 0; j < kHsItems && o0 + j < n; ++j) {
                bool take_a;
                if (ia >= ae)
                    take_a = false;
                else if (ib >= be)
                    take_a = true;
                else
                    take_a = !hs_less(__ldcg(&srck[ib]), __ldcg(&srcv[ib]), __ldcg(&srck[ia]), __ldcg(&srcv[ia]));
                const int64_t q = take_a ? ia : ib;
                dstk[o0 + j] = __ldcg(&srck[q]);
                dstv[o0 + j] = __ldcg(&srcv[q]);
                ia += take_a ? 1 : 0;
                ib += take_a ? 0 : 1;
            }
        }
        __syncthreads();
        unsigned long long *tk = srck;
        srck = dstk;
        dstk = tk;
        uint32_t *tv = srcv;
        srcv = dstv;
        dstv = tv;
    }
    if (srck != dk) {
        for (int64_t q = threadIdx.x; q < n; q += blockDim.x) {
            dk[q] = __ldcg(&srck[q]);
            dv[q] = __ldcg(&srcv[q]);
        }
    }
}

// A bucket of n <= I * blockDim.x pairs: read coalesced through shared
// memory; if its keys span less than 2^(63 - idbits), the words
// (key - kmin) << idbits | id (ids < 2^idbits) order exactly as (key, id)
// and are sorted as single words, then written back coalesced; otherwise
// the pairs are sorted as pairs.  Every thread of the block calls it.
template <int I>
__device__ void hs_bucket_small(unsigned long long *sk, uint32_t *sv, int n, unsigned long long *dk,
                                uint32_t *dv, int idbits, unsigned long long *shk, uint32_t *shv,
                                unsigned long long *wmin, unsigned long long *wmax) {
    const int t = threadIdx.x;
    for (int q = t; q < n; q += blockDim.x) {
        shk[hs_sw(q)] = sk[q];
        shv[hs_sw(q)] = sv[q];
    }
    __syncthreads();
    unsigned long long c[I];
    unsigned long long kmin = ~0ull, kmax = 0ull;
#pragma unroll
    for (int j = 0; j < I; ++j) {
        const int q = I * t + j;
        c[j] = ~0ull;
        if (q < n) {
            const unsigned long long k = shk[hs_sw(q)];
            c[j] = k;
            kmin = k < kmin ? k : kmin;
            kmax = k > kmax ? k : kmax;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xFFFFFFFFu, kmin, d);
        const unsigned long long b = __shfl_xor_sync(0xFFFFFFFFu, kmax, d);
        kmin = a < kmin ? a : kmin;
        kmax = b > kmax ? b : kmax;
    }
    if ((t & 31) == 0) {
        wmin[t >> 5] = kmin;
        wmax[t >> 5] = kmax;
    }
    __syncthreads();
    kmin = wmin[0];
    kmax = wmax[0];
    for (int w = 1; w < int(blockDim.x >> 5); ++w) {
        kmin = wmin[w] < kmin ? wmin[w] : kmin;
        kmax = wmax[w] > kmax ? wmax[w] : kmax;
    }
    if (((kmax - kmin) >> (63 - idbits)) != 0ull) {  // too wide for one word
        __syncthreads();
        if (n <= kHsPairCap)
            hs_block_sort(sk, sv, n, dk, dv, shk, shv);
        else
            hs_pairs_chunked(sk, sv, n, dk, dv, shk, shv);
        return;
    }
#pragma unroll
    for (int j = 0; j < I; ++j) {
        const int q = I * t + j;
        if (q < n) c[j] = ((c[j] - kmin) << idbits) | shv[hs_sw(q)];
    }
    int P = I;
    while (P < n) P <<= 1;
    hs_sort_words<I>(c, P, shk);
    __syncthreads();  // the last round's reads are done
#pragma unroll
    for (int j = 0; j < I; ++j)
        if (I * t + j < n) shk[hs_sw(I * t + j)] = c[j];
    __syncthreads();
    const unsigned long long mask = (1ull << idbits) - 1ull;
    for (int q = t; q < n; q += blockDim.x) {
        const unsigned long long w = shk[hs_sw(q)];
        dk[q] = (w >> idbits) + kmin;
        dv[q] = uint32_t(w & mask);
    }
}

// One block per bucket: sorts its pairs from the slots into the output.
__global__ void __launch_bounds__(kHsThreads) k_hs_bucket(HsBuffers h, unsigned long long *__restrict__ slot_key,
                                                          uint32_t *__restrict__ slot_id,
                                                          unsigned long long *__restrict__ out_key,
                                                          uint32_t *__restrict__ out_id, int idbits) {
    __shared__ unsigned long long shk[kHsSmem];
    __shared__ uint32_t shv[kHsSmem];
    __shared__ unsigned long long wmin[kHsThreads / 32], wmax[kHsThreads / 32];
    const int u = blockIdx.x;
    const int64_t b0 = h.start[u];
    const int64_t n = int64_t(h.start[u + 1]) - b0;
    if (n <= 0) return;
    unsigned long long *sk = slot_key + b0, *dk = out_key + b0;
    uint32_t *sv = slot_id + b0, *dv = out_id + b0;
    if (n <= kHsCap / 2)  // every thread busy at 4 words
        hs_bucket_small<4>(sk, sv, int(n), dk, dv, idbits, shk, shv, wmin, wmax);
    else if (n <= kHsCap)
        hs_bucket_small<8>(sk, sv, int(n), dk, dv, idbits, shk, shv, wmin, wmax);
    else
        hs_pairs_chunked(sk, sv, n, dk, dv, shk, shv);
}

}  // namespace

// The sort on stream `st`, in two halves (the first ends once the samples
// are ranked, so a caller can time the two apart): K <= hs_max_keys()
// pairs; key_of(id) gives the key of id.  tmp_key/tmp_bucket and
// slot_key/slot_id hold K entries each and may not alias the hint or the
// output; the output may not alias the hint.
template <class KeyOf>
int hinted_sort_samples(KeyOf key_of, const uint32_t *hint, int64_t K, const HsBuffers &h, uint32_t *status,
                        cudaStream_t st, const HsClears &clr = HsClears()) {
    if (K <= 0) return BGV_OK;
    if (K > hs_max_keys()) return BGV_EINVAL;
    const HsShape sh = hs_shape(K);
    int64_t first_work = 2;
    for (const int64_t w : {int64_t(sh.ns), int64_t(sh.nb), clr.n_u64, clr.n_u32})
        if (w > first_work) first_work = w;
    note_launch(), k_hs_sample<KeyOf><<<grid_for(first_work, 256, sm_count() * 4), 256, 0, st>>>(
        key_of, hint, K, sh.nb, sh.ns, h, clr, status);
    BGV_TRY(launch_status());
    if (sh.ns > 0) {
        const dim3 g((sh.ns + 255) / 256, kHsRankSlices);
        note_launch(), k_hs_rank<<<g, 256, 0, st>>>(sh.ns, sh.s, h);
        BGV_TRY(launch_status());
    }
    return BGV_OK;
}

template <class KeyOf>
int hinted_sort_place(KeyOf key_of, const uint32_t *hint, int64_t K, const HsBuffers &h, unsigned long long *tmp_key,
                      uint32_t *tmp_bucket, unsigned long long *slot_key, uint32_t *slot_id,
                      unsigned long long *out_key, uint32_t *out_id, uint32_t *status, cudaStream_t st) {
    if (K <= 0) return BGV_OK;
    if (K > hs_max_keys()) return BGV_EINVAL;
    const HsShape sh = hs_shape(K);
    note_launch(), k_hs_count<KeyOf><<<grid_for(K, 256, sm_count() * 8), 256, 0, st>>>(key_of, hint, K, sh.nb, h,
                                                                                      tmp_key, tmp_bucket, status);
    BGV_TRY(launch_status());
    note_launch(), k_hs_scatter<<<grid_for(K, 256, sm_count() * 8), 256, 0, st>>>(hint, K, h, tmp_key, tmp_bucket,
                                                                                 slot_key, slot_id);
    BGV_TRY(launch_status());
    int idbits = 0;  // bits of the largest id
    while (idbits < 32 && (int64_t(1) << idbits) < K) ++idbits;
    note_launch(), k_hs_bucket<<<sh.nb, kHsThreads, 0, st>>>(h, slot_key, slot_id, out_key, out_id, idbits);
    return launch_status();
}

}  // namespace bgv

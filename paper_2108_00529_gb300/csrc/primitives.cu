// primitives.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// Both take their element count either from the host or from a device
// scalar, so data-dependent sizes (cut edges, superedges) need no host round
// trip.  Grids are sized for the host-side upper bound; blocks past the
// device count do no work (the radix histogram still writes zeros for them so
// the digit offsets stay consistent).
#include <algorithm>
#include <atomic>

#include "bgv_internal.cuh"

namespace bgv {

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launches_issued() { return g_launches.load(std::memory_order_relaxed); }

// Bound on the polling rounds of every decoupled look-back wait (process
// wide; the default ends a wait that cannot finish after a few seconds).
static std::atomic<int> g_spin_limit{1 << 22};
int spin_limit() { return g_spin_limit.load(std::memory_order_relaxed); }
int set_spin_limit(int limit) { return g_spin_limit.exchange(limit, std::memory_order_relaxed); }

int coop_blocks(const void *kernel, int threads, int want) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess) per_sm = 1;
    const int most = (per_sm > 0 ? per_sm : 1) * sm_count();
    const int b = want < most ? want : most;
    return b > 0 ? b : 1;
}

int launch_coop(const void *kernel, int blocks, int threads, void **args, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(blocks));
    cfg.blockDim = dim3(unsigned(threads));
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    note_launch();
    return cudaLaunchKernelExC(&cfg, kernel, args) == cudaSuccess ? BGV_OK : BGV_ECUDA;
}

int sm_count() {
    constexpr int kMaxDevices = 64;
    static std::atomic<int> cached[kMaxDevices];  // 0: not yet queried
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    if (dev < kMaxDevices) {
        const int c = cached[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
    if (dev < kMaxDevices) cached[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

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
// Stable LSD radix sort, 8-bit digits, in the one-sweep form: one kernel
// counts the digits of every pass at once; each pass is then a single
// kernel in which a block takes the next tile number from a counter, ranks
// its keys (warp match_any plus per-warp digit counters, in (item, lane)
// order, which keeps the sort stable), publishes its per-digit tile count,
// and looks back over the tiles before it to find its global offsets
// (decoupled look-back).  A block only ever waits for tiles with smaller
// numbers, which were handed to blocks that are already running, so the
// waits end; each wait is still bounded and reports BGV_DEV_TIMEOUT if the
// bound is hit.
namespace {
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
// Keys per thread: 8 up to a cutoff, 16 above it.  Measured on GB300 with
// 48-bit keys and values, 8 was faster at every size from 2^14 to 2^26
// keys (4.4 against 11.7 ms at 2^26), so the cutoff starts above any
// count; bgv_autotune_sort can set it from measurements on the GPU at hand.
constexpr int kSortItemsBig = 16, kSortItemsSmall = 8;
std::atomic<int64_t> g_small_sort_cutoff{int64_t(1) << 40};
inline int sort_items(int64_t cap) {
    return cap <= g_small_sort_cutoff.load(std::memory_order_relaxed) ? kSortItemsSmall : kSortItemsBig;
}
inline int64_t tiles_for(int64_t cap, int items) {
    const int64_t t = (cap + int64_t(kSortThreads) * items - 1) / (int64_t(kSortThreads) * items);
    return t < 1 ? 1 : t;
}
constexpr int kBins = 256;
constexpr int kMaxPasses = 8;
// Look-back words: 2 flag bits, the pass number (1..8) in bits 40..47 and a
// 40-bit count.  The words are cleared once per sort; a word written by an
// earlier pass carries another pass number and reads as "not yet published".
constexpr unsigned long long kFlagAgg = 1ull << 62, kFlagIncl = 2ull << 62, kFlagMask = 3ull << 62;
constexpr unsigned long long kCountMask = (1ull << 40) - 1;
constexpr int kTagShift = 40;
constexpr int kLookBack = 4;       // predecessors read per look-back round (16 keys per thread)
constexpr int kLookBackWide = 16;  // the same with 8 keys per thread (keys staged first)

// Digit counts of passes first..passes-1.  Each thread loads its kCountItems
// keys before counting, so their loads are in flight together.
constexpr int kCountItems = 8;
constexpr int kCountTile = kSortThreads * kCountItems;
__global__ void __launch_bounds__(kSortThreads) k_sort_count(const unsigned long long *__restrict__ keys, int64_t cap,
                                                             const int64_t *d_count, int first, int passes,
                                                             uint32_t *__restrict__ counts,
                                                             unsigned long long *__restrict__ status, int64_t tiles,
                                                             uint32_t *__restrict__ zero_words, int n_zero) {
    __shared__ uint32_t h[kMaxPasses][kBins];
    // clears what the passes after it start from: the look-back words of the
    // tiles (one tile's kBins words per block) and a few counters
    if (blockIdx.x < tiles) status[int64_t(blockIdx.x) * kBins + threadIdx.x] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x < n_zero) zero_words[threadIdx.x] = 0u;
    for (int i = threadIdx.x; i < kMaxPasses * kBins; i += kSortThreads) (&h[0][0])[i] = 0;
    const int64_t n = load_count(d_count, cap);
    const int64_t base = int64_t(blockIdx.x) * kCountTile;
    unsigned long long key[kCountItems];
#pragma unroll
    for (int k = 0; k < kCountItems; ++k) {
        const int64_t i = base + int64_t(k) * kSortThreads + threadIdx.x;
        key[k] = i < n ? keys[i] : 0ull;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kCountItems; ++k) {
        if (base + int64_t(k) * kSortThreads + threadIdx.x < n)
            for (int p = first; p < passes; ++p) atomicAdd(&h[p][uint32_t(key[k] >> (8 * p)) & 0xFFu], 1u);
    }
    __syncthreads();
    for (int i = first * kBins + threadIdx.x; i < passes * kBins; i += kSortThreads) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&counts[i], c);
    }
}

// Decoupled look-back of digit d for tile `tile`: adds the counts published
// by the tiles before it, kW at a time (independent loads in flight
// together), down to the nearest inclusive prefix; stops at a tile that has
// published nothing yet and waits for it.  Publishes the tile's inclusive
// count and returns the exclusive one.
template <int kW>
__device__ __forceinline__ unsigned long long look_back(volatile unsigned long long *st, int64_t tile, int d,
                                                        unsigned long long tag, uint32_t total, uint32_t *dev_status,
                                                        int spin_limit) {
    if (tile == 0) return 0ull;
    unsigned long long excl = 0;
    int64_t j = tile - 1;
    int spins = 0;
    while (true) {
        unsigned long long v[kW];
#pragma unroll
        for (int q = 0; q < kW; ++q) v[q] = j - q >= 0 ? st[(j - q) * kBins + d] : (kFlagIncl | tag);
        int q = 0;
        bool done = false;
        for (; q < kW; ++q) {
            const unsigned long long flag = (v[q] & ~(kFlagMask | kCountMask)) == tag ? (v[q] & kFlagMask) : 0ull;
            if (flag == 0) break;
            excl += v[q] & kCountMask;
            if (flag == kFlagIncl) {
                done = true;
                break;
            }
        }
        if (done) break;
        j -= q;
        if (q < kW) {
            if (++spins > spin_limit) {
                raise_status(dev_status, BGV_DEV_TIMEOUT);
                break;
            }
            __nanosleep(32);
        }
    }
    st[tile * kBins + d] = kFlagIncl | tag | (excl + total);
    return excl;
}

// With 8 keys per thread, 4 blocks fit on an SM (registers capped at 64), so
// the ~480 tiles of a million keys run in one wave, and the scatter goes
// through shared memory: keys are first placed in digit order inside the
// tile, then written out so that neighbouring threads write neighbouring
// addresses of one digit's run.
template <bool kVals, int kItems>
__global__ void __launch_bounds__(kSortThreads, kItems <= 8 ? 4 : 2) k_sort_onesweep(const unsigned long long *__restrict__ kin,
                                                                unsigned long long *__restrict__ kout,
                                                                const uint32_t *__restrict__ vin,
                                                                uint32_t *__restrict__ vout, int64_t cap,
                                                                const int64_t *d_count, int shift,
                                                                const uint32_t *__restrict__ pass_counts,
                                                                unsigned int *tile_counter,
                                                                unsigned long long *status, uint32_t *dev_status,
                                                                unsigned long long tag, int spin_limit) {
    // keys go through shared memory (coalesced digit runs on the way out)
    // with 8 keys per thread, and with 16 when there are no values (42 KB)
    constexpr bool kStage = kItems <= 8 || !kVals;
    constexpr int kTileKeys = kSortThreads * kItems;
    __shared__ uint32_t cnt[kSortWarps][kBins];
    __shared__ uint32_t tile_base[kBins];
    __shared__ uint32_t local_start[kBins];
    __shared__ unsigned long long skey[kStage ? kTileKeys : 1];
    __shared__ uint32_t sval[kStage && kVals ? kTileKeys : 1];
    __shared__ unsigned int tile_sh;
    if (threadIdx.x == 0) tile_sh = atomicAdd(tile_counter, 1u);
    for (int i = threadIdx.x; i < kSortWarps * kBins; i += kSortThreads) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t tile = tile_sh;
    const int64_t n = load_count(d_count, cap);
    if (tile * (kSortThreads * kItems) >= n) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t base = tile * (kSortThreads * kItems) + int64_t(warp) * (32 * kItems);
    // Keys are loaded up front, and with 8 keys per thread the values too
    // (their latency then overlaps the ranking; with 16 the registers would
    // halve the resident blocks).  Digits are recomputed from the keys.
    constexpr bool kEarlyVals = kVals && kItems <= 8;
    unsigned long long key[kItems];
    uint32_t val[kItems];
    uint32_t rank[kItems];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const int64_t i = base + int64_t(k) * 32 + lane;
        key[k] = i < n ? kin[i] : 0ull;
        if (kEarlyVals) val[k] = i < n ? vin[i] : 0u;
    }
    // Rank inside the warp: the lanes holding the same digit are found with
    // nine ballots (eight digit bits and validity); the lowest of them reads
    // and advances the warp's counter for that digit.
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const int64_t i = base + int64_t(k) * 32 + lane;
        const bool valid = i < n;
        const uint32_t d = static_cast<uint32_t>(key[k] >> shift) & 0xFFu;
        uint32_t peers = __ballot_sync(0xFFFFFFFFu, valid);
        if (!valid) peers = ~peers;
#pragma unroll
        for (int bit = 0; bit < 8; ++bit) {
            const uint32_t m = __ballot_sync(0xFFFFFFFFu, (d >> bit) & 1u);
            peers &= ((d >> bit) & 1u) ? m : ~m;
        }
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (valid && lane == leader) {
            before = cnt[warp][d];
            cnt[warp][d] = before + __popc(peers);
        }
        before = __shfl_sync(0xFFFFFFFFu, before, leader);
        rank[k] = before + __popc(peers & lt_mask);
        __syncwarp();
    }
    __syncthreads();
    // thread d owns digit d: warp prefixes and tile total, published at once
    const int d = threadIdx.x;
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t c = cnt[w][d];
        cnt[w][d] = total;
        total += c;
    }
    volatile unsigned long long *st = status;
    st[tile * kBins + d] = (tile == 0 ? kFlagIncl : kFlagAgg) | tag | total;
    // where digit d starts in the output: the exclusive scan of the pass's
    // digit counts (every block scans the 256 counts itself)
    uint32_t all_keys;
    const uint32_t digit_start = block_exclusive(pass_counts[d], &all_keys);
    if (kStage) {
        // keys go to their place in the tile before the look-back, which
        // frees their registers for a wider look-back window
        uint32_t all;
        local_start[d] = block_exclusive(total, &all);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const int64_t i = base + int64_t(k) * 32 + lane;
            if (i >= n) continue;
            const uint32_t dk = static_cast<uint32_t>(key[k] >> shift) & 0xFFu;
            const uint32_t slot = local_start[dk] + cnt[warp][dk] + rank[k];
            skey[slot] = key[k];
            if (kVals) sval[slot] = val[k];
        }
    }
    tile_base[d] = digit_start + uint32_t(look_back<kStage ? kLookBackWide : kLookBack>(st, tile, d, tag, total,
                                                                                         dev_status, spin_limit));
    __syncthreads();
    if constexpr (kStage) {
        const int64_t t0 = tile * kTileKeys;
        const int tile_n = n - t0 < kTileKeys ? int(n - t0) : kTileKeys;
        for (int slot = threadIdx.x; slot < tile_n; slot += kSortThreads) {
            const unsigned long long k = skey[slot];
            const uint32_t dk = static_cast<uint32_t>(k >> shift) & 0xFFu;
            const uint32_t pos = tile_base[dk] + uint32_t(slot) - local_start[dk];
            kout[pos] = k;
            if (kVals) vout[pos] = sval[slot];
        }
    } else {
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const int64_t i = base + int64_t(k) * 32 + lane;
            if (i >= n) continue;
            const uint32_t d = static_cast<uint32_t>(key[k] >> shift) & 0xFFu;
            const uint32_t pos = tile_base[d] + cnt[warp][d] + rank[k];
            kout[pos] = key[k];
            if (kVals) vout[pos] = kEarlyVals ? val[k] : vin[i];
        }
    }
}
}  // namespace

// ------------------------------------------------- cooperative radix sort
// All LSD passes in one persistent kernel (cooperative launch: every block
// resident), with no look-back.  Block b owns a contiguous chunk of tiles of
// 2,048 keys.  Per pass on the 8-bit digit at `shift`:
//   A  the block counts the digits of its chunk (shared-memory atomics);
//   -  grid barrier;
//   B  blocks 0..255 take one digit each and scan its counts over the chunks
//      (exclusive, in block order) and total them;
//   -  grid barrier;
//   C  the block turns the 256 totals into digit starts, then takes its
//      tiles in order: ranks each tile's keys stably (per-warp digit
//      counters in (item, lane) order, as in the onesweep pass), stages them
//      in shared memory in digit order and writes every digit's run at the
//      digit start + the chunk's prefix + what its earlier tiles wrote;
//   -  grid barrier before the next pass reads the output.
// Chunks in block order and tiles in order keep the passes stable.  The
// barrier waits are bounded (BGV_DEV_TIMEOUT).
template <bool kVals>
__global__ void __launch_bounds__(kSortThreads, kVals ? 3 : 4) k_sort_coop(unsigned long long *k0, unsigned long long *k1,
                                                                 uint32_t *v0, uint32_t *v1, int64_t cap,
                                                                 const int64_t *d_count, int first_pass, int passes,
                                                                 uint32_t *chunk_hist, uint32_t *chunk_pre,
                                                                 uint32_t *totals, GridBar *bar, uint32_t *dev_status,
                                                                 int spin_limit, const uint32_t *guard,
                                                                 uint32_t guard_min) {
    // guarded launch: runs only when *guard exceeds guard_min (every block
    // reads the same word, so all leave together, before any barrier)
    if (guard && *guard <= guard_min) return;
    constexpr int kItems = kSortItemsSmall;
    constexpr int kTileKeys = kSortThreads * kItems;
    __shared__ uint32_t cnt[kSortWarps][kBins];
    __shared__ uint32_t run[kBins];
    __shared__ uint32_t local_start[kBins];
    __shared__ unsigned long long skey[kTileKeys];
    __shared__ uint32_t sval[kVals ? kTileKeys : 1];
    const int64_t n = load_count(d_count, cap);
    const int64_t T = (n + kTileKeys - 1) / kTileKeys;
    const int64_t per = (T + gridDim.x - 1) / gridDim.x;
    const int64_t t_lo = int64_t(blockIdx.x) * per < T ? int64_t(blockIdx.x) * per : T;
    const int64_t t_hi = t_lo + per < T ? t_lo + per : T;
    const int64_t i_hi = t_hi * kTileKeys < n ? t_hi * kTileKeys : n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int d = threadIdx.x;  // the digit this thread owns in per-digit steps
    for (int p = first_pass; p < passes; ++p) {
        const int shift = 8 * p;
        const bool odd = ((p - first_pass) & 1) != 0;
        const unsigned long long *kin = odd ? k1 : k0;
        unsigned long long *kout = odd ? k0 : k1;
        const uint32_t *vin = odd ? v1 : v0;
        uint32_t *vout = odd ? v0 : v1;
        // A: digit counts of the chunk
        run[d] = 0u;
        __syncthreads();
        for (int64_t i = t_lo * kTileKeys + threadIdx.x; i < i_hi; i += kSortThreads)
            atomicAdd(&run[uint32_t(__ldcg(&kin[i]) >> shift) & 0xFFu], 1u);
        __syncthreads();
        chunk_hist[size_t(blockIdx.x) * kBins + d] = run[d];
        if (!grid_barrier(bar, spin_limit, dev_status)) return;
        // B: one digit per block, scanned over the chunks
        for (unsigned dd = blockIdx.x; dd < kBins; dd += gridDim.x) {
            uint32_t carry = 0u;
            for (unsigned b0 = 0; b0 < gridDim.x; b0 += kSortThreads) {
                const unsigned b = b0 + threadIdx.x;
                const uint32_t x = b < gridDim.x ? __ldcg(&chunk_hist[size_t(b) * kBins + dd]) : 0u;
                uint32_t tot;
                const uint32_t ex = block_exclusive(x, &tot);
                if (b < gridDim.x) chunk_pre[size_t(b) * kBins + dd] = carry + ex;
                carry += tot;
            }
            if (threadIdx.x == 0) totals[dd] = carry;
        }
        if (!grid_barrier(bar, spin_limit, dev_status)) return;
        // C: digit starts, then the chunk's tiles in order
        uint32_t all;
        const uint32_t dstart = block_exclusive(__ldcg(&totals[d]), &all);
        run[d] = dstart + __ldcg(&chunk_pre[size_t(blockIdx.x) * kBins + d]);
        for (int64_t tile = t_lo; tile < t_hi; ++tile) {
            for (int i = threadIdx.x; i < kSortWarps * kBins; i += kSortThreads) (&cnt[0][0])[i] = 0u;
            __syncthreads();
            const int64_t base = tile * kTileKeys + int64_t(warp) * (32 * kItems);
            unsigned long long key[kItems];
            uint32_t val[kItems], rank[kItems];
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                const int64_t i = base + int64_t(k) * 32 + lane;
                key[k] = i < n ? __ldcg(&kin[i]) : 0ull;
                if (kVals) val[k] = i < n ? __ldcg(&vin[i]) : 0u;
            }
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                const int64_t i = base + int64_t(k) * 32 + lane;
                const bool valid = i < n;
                const uint32_t dg = static_cast<uint32_t>(key[k] >> shift) & 0xFFu;
                uint32_t peers = __ballot_sync(0xFFFFFFFFu, valid);
                if (!valid) peers = ~peers;
#pragma unroll
                for (int bit = 0; bit < 8; ++bit) {
                    const uint32_t m = __ballot_sync(0xFFFFFFFFu, (dg >> bit) & 1u);
                    peers &= ((dg >> bit) & 1u) ? m : ~m;
                }
                const int leader = __ffs(peers) - 1;
                uint32_t before = 0;
                if (valid && lane == leader) {
                    before = cnt[warp][dg];
                    cnt[warp][dg] = before + __popc(peers);
                }
                before = __shfl_sync(0xFFFFFFFFu, before, leader);
                rank[k] = before + __popc(peers & lt_mask);
                __syncwarp();
            }
            __syncthreads();
            uint32_t total = 0u;
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                const uint32_t c = cnt[w][d];
                cnt[w][d] = total;
                total += c;
            }
            local_start[d] = block_exclusive(total, &all);
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                const int64_t i = base + int64_t(k) * 32 + lane;
                if (i >= n) continue;
                const uint32_t dk = static_cast<uint32_t>(key[k] >> shift) & 0xFFu;
                const uint32_t slot = local_start[dk] + cnt[warp][dk] + rank[k];
                skey[slot] = key[k];
                if (kVals) sval[slot] = val[k];
            }
            __syncthreads();
            const int64_t t0 = tile * kTileKeys;
            const int tile_n = n - t0 < kTileKeys ? int(n - t0) : kTileKeys;
            for (int slot = threadIdx.x; slot < tile_n; slot += kSortThreads) {
                const unsigned long long k = skey[slot];
                const uint32_t dk = static_cast<uint32_t>(k >> shift) & 0xFFu;
                const uint32_t pos = run[dk] + uint32_t(slot) - local_start[dk];
                kout[pos] = k;
                if (kVals) vout[pos] = sval[slot];
            }
            __syncthreads();
            run[d] += total;
        }
        if (p + 1 < passes && !grid_barrier(bar, spin_limit, dev_status)) return;
    }
}

// Which sort runs the passes: onesweep passes with decoupled look-back (0),
// the cooperative kernel (1), or by size (2, the default): cooperative for
// key counts in [g_coop_lo, g_coop_hi], where it measured faster on GB300
// (its three grid barriers per pass cost more than the look-back below that,
// its second read of the keys more above); process wide.
// Keys without values are sorted cooperatively from 2^21 keys up (68 M
// supergraph keys: 3.36 ms against 4.19 ms for onesweep at 8 keys per
// thread); the range applies to keys with values, where onesweep's single
// read of each pass wins above 2^23.
std::atomic<int> g_sort_method{2};
std::atomic<int64_t> g_coop_lo{int64_t(1) << 21}, g_coop_hi{int64_t(1) << 23};
inline bool use_coop(int64_t cap, bool with_vals) {
    const int m = g_sort_method.load(std::memory_order_relaxed);
    if (m != 2) return m == 1;
    const int64_t lo = g_coop_lo.load(std::memory_order_relaxed);
    return cap >= lo && (!with_vals || cap <= g_coop_hi.load(std::memory_order_relaxed));
}

// Launches the cooperative sort over passes first..passes-1 from buffer
// pair 0; the result is in pair (passes - first) % 2.  Its counter words
// (totals, barrier) must be zero: radix_sort clears them, the FA2 step's
// keys kernel clears them in its graph.
int coop_sort(SortBuffers &b, int64_t cap, const int64_t *d_count, int first, int passes, cudaStream_t s,
              uint32_t *dev_status, const uint32_t *guard = nullptr, uint32_t guard_min = 0) {
    const int64_t tiles = tiles_for(cap, kSortItemsSmall);
    const void *kernel = b.vals[0] ? reinterpret_cast<const void *>(k_sort_coop<true>)
                                   : reinterpret_cast<const void *>(k_sort_coop<false>);
    int blocks = coop_blocks(kernel, kSortThreads, sm_count() * 4);
    if (blocks > tiles) blocks = int(tiles);
    // per-chunk digit counts and prefixes live in the look-back words
    // (256 u64 per tile >= 2 x 256 u32 per block, as blocks <= tiles)
    uint32_t *chunk_hist = reinterpret_cast<uint32_t *>(b.status);
    uint32_t *chunk_pre = chunk_hist + size_t(blocks) * kBins;
    uint32_t *totals = b.counts;
    GridBar *bar = reinterpret_cast<GridBar *>(b.counts + kMaxPasses * kBins + kMaxPasses);
    unsigned long long *k0 = b.keys[0], *k1 = b.keys[1];
    uint32_t *v0 = b.vals[0], *v1 = b.vals[1];
    int limit = spin_limit();
    void *args[] = {&k0, &k1, &v0, &v1, &cap, &d_count, &first, &passes, &chunk_hist, &chunk_pre, &totals,
                    &bar, &dev_status, &limit, &guard, &guard_min};
    return launch_coop(kernel, blocks, kSortThreads, args, s);
}

// The look-back words are sized for the smaller tiles, so a workspace stays
// large enough whatever tile size the cutoff picks later.
int64_t sort_tiles(int64_t cap) {
    const int64_t tile = int64_t(kSortThreads) * kSortItemsSmall;
    int64_t t = (cap + tile - 1) / tile;
    return t < 1 ? 1 : t;
}

void carve_sort(Carver &c, int64_t cap, bool with_vals, SortBuffers &out) {
    out.keys[0] = c.take<unsigned long long>(size_t(cap));
    out.keys[1] = c.take<unsigned long long>(size_t(cap));
    out.vals[0] = with_vals ? c.take<uint32_t>(size_t(cap)) : nullptr;
    out.vals[1] = with_vals ? c.take<uint32_t>(size_t(cap)) : nullptr;
    out.status = c.take<unsigned long long>(size_t(kBins) * size_t(sort_tiles(cap)));
    out.counts = c.take<uint32_t>(size_t(sort_counter_words()));
}

namespace {
// One onesweep pass on the 8-bit digit at `shift`, from buffer pair `cur` to
// `cur ^ 1`.
int onesweep_pass(SortBuffers &b, int64_t cap, const int64_t *d_count, int cur, int shift, const uint32_t *base,
                  unsigned *tile_counter, unsigned long long tag, int items, cudaStream_t s, uint32_t *dev_status) {
    const bool small = items == kSortItemsSmall;
    const unsigned g = static_cast<unsigned>(tiles_for(cap, items));
    unsigned long long *ki = b.keys[cur], *ko = b.keys[cur ^ 1];
    uint32_t *vi = b.vals[cur], *vo = b.vals[cur ^ 1];
    if (b.vals[0] && small)
        note_launch(), k_sort_onesweep<true, kSortItemsSmall><<<g, kSortThreads, 0, s>>>(
            ki, ko, vi, vo, cap, d_count, shift, base, tile_counter, b.status, dev_status, tag, spin_limit());
    else if (b.vals[0])
        note_launch(), k_sort_onesweep<true, kSortItemsBig><<<g, kSortThreads, 0, s>>>(
            ki, ko, vi, vo, cap, d_count, shift, base, tile_counter, b.status, dev_status, tag, spin_limit());
    else if (small)
        note_launch(), k_sort_onesweep<false, kSortItemsSmall><<<g, kSortThreads, 0, s>>>(
            ki, ko, nullptr, nullptr, cap, d_count, shift, base, tile_counter, b.status, dev_status, tag, spin_limit());
    else
        note_launch(), k_sort_onesweep<false, kSortItemsBig><<<g, kSortThreads, 0, s>>>(
            ki, ko, nullptr, nullptr, cap, d_count, shift, base, tile_counter, b.status, dev_status, tag, spin_limit());
    return launch_status();
}

inline unsigned long long pass_tag(int p) { return static_cast<unsigned long long>(p + 1) << kTagShift; }
}  // namespace

int radix_sort(SortBuffers &b, int64_t cap, const int64_t *d_count, int end_bit, cudaStream_t s,
               int *result_buffer, uint32_t *dev_status, int items) {
    if (items != kSortItemsSmall && items != kSortItemsBig) items = sort_items(cap);
    const int64_t tiles = tiles_for(cap, items);
    const int passes = (end_bit + 7) / 8;
    if (passes > kMaxPasses) return BGV_EINVAL;
    uint32_t *tile_counters = b.counts + kMaxPasses * kBins;
    BGV_CUDA(cudaMemsetAsync(b.counts, 0, sizeof(uint32_t) * size_t(sort_counter_words()), s));
    if (use_coop(cap, b.vals[0] != nullptr)) {
        BGV_TRY(coop_sort(b, cap, d_count, 0, passes, s, dev_status));
        *result_buffer = passes & 1;
        return BGV_OK;
    }
    const int64_t count_blocks = (cap + kCountTile - 1) / kCountTile;  // >= tiles
    note_launch(), k_sort_count<<<static_cast<unsigned>(count_blocks > 0 ? count_blocks : 1), kSortThreads, 0, s>>>(
        b.keys[0], cap, d_count, 0, passes, b.counts, b.status, tiles, nullptr, 0);
    BGV_TRY(launch_status());
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        BGV_TRY(onesweep_pass(b, cap, d_count, cur, 8 * p, b.counts + p * kBins, tile_counters + p, pass_tag(p),
                              items, s, dev_status));
        cur ^= 1;
    }
    *result_buffer = cur;
    return BGV_OK;
}

// ----------------------------------------------- sort with a local finish
// For keys whose order is almost always decided above their lowest
// kLowBits = 24 bits (Morton keys of spread-out points: in rmat22x layouts
// at 1 to 500 FA2 iterations, 86 to 97 % of the bodies are alone in their
// cell of side 2^-12 of the frame and the longest run held 42 bodies): LSD
// passes on bits 24 and up only, which leave every run of equal high bits
// contiguous and in input order, then each run put in order of its low 24
// bits on its own, stably, so the result is the stable sort of the whole key.  A pass over all keys marks
// every 32-key chunk holding a descent (a key whose low bits are below its
// predecessor's in the same run) and sorts runs of up to kShortRun keys in
// registers; a warp skips the longer runs without a marked chunk (equal or
// already ordered keys: coincident bodies) and ranks those of up to
// kWarpRun keys; a block sorts each longer run by six 4-bit LSD passes
// through the idle half of the ping-pong buffers.
namespace {
constexpr int kShortRun = 8;
constexpr int kLowDigits = kLowBits / 4;  // 4-bit passes of the block finish (even: the run ends in place)
static_assert(kLowBits % 8 == 0 && kLowDigits % 2 == 0, "whole LSD passes above, an even count below");
constexpr unsigned long long kLowMask = (1ull << kLowBits) - 1ull;
constexpr int kWarpRun = 256;
constexpr int kFixThreads = 256;
// A run longer than this is not sorted by one block (its time would grow
// with the run, e.g. many bodies inside one cell of side 2^-12 of the
// frame): the whole array gets a full LSD sort instead.
constexpr uint32_t kFixGuard = 16384;

__device__ __forceinline__ unsigned long long run_key(unsigned long long k, int64_t pos) {
    return ((k & kLowMask) << 32) | static_cast<unsigned long long>(pos);
}

// End of the run of equal high bits that starts at `start` (the array is
// sorted on the high bits): galloping from the start (probes at +1, +2, +4,
// ... stay near the run), then a binary search inside the last step.
__device__ __forceinline__ int64_t run_end(const unsigned long long *keys, int64_t n, int64_t start) {
    const unsigned long long hi = keys[start] >> kLowBits;
    int64_t step = 1, lo = start + 1;  // keys[lo - 1] is in the run
    while (lo < n && (keys[lo] >> kLowBits) == hi) {
        lo += step;
        step <<= 1;
    }
    int64_t up = lo < n ? lo : n;  // first index past the run lies in (lo - step/2, up]
    lo = lo - (step >> 1);
    if (lo < start + 1) lo = start + 1;
    while (lo < up) {
        const int64_t mid = (lo + up) >> 1;
        if ((keys[mid] >> kLowBits) <= hi) lo = mid + 1; else up = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kFixThreads) k_fix_runs(unsigned long long *__restrict__ keys,
                                                          uint32_t *__restrict__ vals, int64_t cap,
                                                          const int64_t *d_count, uint8_t *__restrict__ descent,
                                                          uint32_t *__restrict__ runs, uint32_t *run_count) {
    const int64_t n = load_count(d_count, cap);
    const int lane = threadIdx.x & 31;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i - lane < n; i += stride) {
        bool head = false, desc = false;
        unsigned long long hi = 0;
        if (i < n) {
            const unsigned long long k = keys[i];
            hi = k >> kLowBits;
            if (i > 0) {
                const unsigned long long p = keys[i - 1];
                desc = (p >> kLowBits) == hi && (k & kLowMask) < (p & kLowMask);
                head = (p >> kLowBits) != hi;
            } else {
                head = true;
            }
            head = head && i + 1 < n && (keys[i + 1] >> kLowBits) == hi;  // runs of one need nothing
        }
        const unsigned mask = __ballot_sync(0xFFFFFFFFu, desc);
        if (lane == 0) descent[i >> 5] = mask != 0u;
        if (!head) continue;
        int r = 2;
        while (r <= kShortRun && i + r < n && (keys[i + r] >> kLowBits) == hi) ++r;
        if (r > kShortRun) {
            runs[atomicAdd(run_count, 1u)] = uint32_t(i);
            continue;
        }
        unsigned long long kk[kShortRun];
        uint32_t vv[kShortRun];
        bool ordered = true;
#pragma unroll
        for (int a = 0; a < kShortRun; ++a) {
            kk[a] = a < r ? run_key(keys[i + a], a) : ~0ull;
            vv[a] = (vals && a < r) ? vals[i + a] : 0u;
            if (a > 0) ordered = ordered && kk[a - 1] < kk[a];
        }
        if (ordered) continue;
#pragma unroll
        for (int a = 0; a < kShortRun; ++a) {
            if (a < r) {
                uint32_t rk = 0;
#pragma unroll
                for (int c = 0; c < kShortRun; ++c) rk += kk[c] < kk[a] ? 1u : 0u;
                keys[i + rk] = (hi << kLowBits) | (kk[a] >> 32);
                if (vals) vals[i + rk] = vv[a];
            }
        }
    }
}

// One warp per listed run: a run with no marked chunk is in order already;
// one of up to kWarpRun keys is ranked in registers (each lane holds up to
// 8 keys and counts the smaller ones through shuffles); longer ones go on
// to the block kernel's list.
__global__ void __launch_bounds__(kFixThreads) k_fix_warp(unsigned long long *__restrict__ keys,
                                                          uint32_t *__restrict__ vals, int64_t cap,
                                                          const int64_t *d_count, const uint8_t *__restrict__ descent,
                                                          const uint32_t *__restrict__ runs,
                                                          const uint32_t *run_count, uint32_t *__restrict__ big,
                                                          uint32_t *big_count) {
    constexpr int kPer = kWarpRun / 32;
    const int64_t n = load_count(d_count, cap);
    const int lane = threadIdx.x & 31;
    const uint32_t count = *run_count;
    const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t q = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; q < count; q += warps) {
        const int64_t start = runs[q];
        const int64_t end = __shfl_sync(0xFFFFFFFFu, lane == 0 ? run_end(keys, n, start) : 0, 0);
        const int64_t len = end - start;
        // chunks (start+1)/32 .. (end-1)/32 hold every descent of the run
        // (and maybe some of its neighbours': a needless sort at worst)
        bool marked = false;
        const int64_t c_lo = (start + 1) >> 5, c_hi = (end - 1) >> 5;
#pragma unroll 4
        for (int64_t w = (c_lo >> 4) + lane; w <= (c_hi >> 4); w += 32) {  // 16 chunk marks per load
            const uint4 m = reinterpret_cast<const uint4 *>(descent)[w];
            const uint32_t word[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
            for (int b = 0; b < 16; ++b) {
                const int64_t c = 16 * w + b;
                marked |= c >= c_lo && c <= c_hi && ((word[b >> 2] >> (8 * (b & 3))) & 0xFFu) != 0u;
            }
        }
        if (!__any_sync(0xFFFFFFFFu, marked)) continue;
        if (len > kWarpRun) {
            if (lane == 0) {
                big[atomicAdd(big_count, 1u)] = uint32_t(start);
                atomicMax(big_count + 1, uint32_t(len));
            }
            continue;
        }
        const unsigned long long hi = keys[start] >> kLowBits;
        unsigned long long kk[kPer];
        uint32_t vv[kPer], rank[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int64_t t = lane + 32 * j;
            kk[j] = t < len ? run_key(keys[start + t], t) : ~0ull;
            vv[j] = (vals && t < len) ? vals[start + t] : 0u;
            rank[j] = 0;
        }
#pragma unroll
        for (int jj = 0; jj < kPer; ++jj) {
            if (32 * jj >= len) break;
            for (int src = 0; src < 32; ++src) {
                const unsigned long long other = __shfl_sync(0xFFFFFFFFu, kk[jj], src);
#pragma unroll
                for (int j = 0; j < kPer; ++j) rank[j] += other < kk[j] ? 1u : 0u;
            }
        }
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int64_t t = lane + 32 * j;
            if (t < len) {
                keys[start + rank[j]] = (hi << kLowBits) | (kk[j] >> 32);
                if (vals) vals[start + rank[j]] = vv[j];
            }
        }
    }
}

// One block per listed run: six stable counting passes on 4-bit digits of
// the low 24 bits, from the run to the same range of the other ping-pong
// buffer and back.  The digit counts of all six passes come from one read
// (a stable pass does not change them).  A tile holds kBlockItems keys per
// thread; a key's place among equal digits comes from __match_any_sync in
// its warp and the counts of the (item, warp) groups before it, so input
// order is kept.
constexpr int kBlockItems = 8;
__global__ void __launch_bounds__(kFixThreads) k_fix_block(unsigned long long *__restrict__ keys,
                                                           uint32_t *__restrict__ vals,
                                                           unsigned long long *__restrict__ alt_keys,
                                                           uint32_t *__restrict__ alt_vals, int64_t cap,
                                                           const int64_t *d_count, const uint32_t *__restrict__ big,
                                                           const uint32_t *big_count) {
    if (big_count[1] > kFixGuard) return;  // the whole array was sorted again instead
    const int64_t n = load_count(d_count, cap);
    constexpr int kWarps = kFixThreads / 32;
    constexpr int kGroups = kBlockItems * kWarps;
    __shared__ uint32_t hist[kLowDigits][16];
    __shared__ uint32_t base[16];
    __shared__ uint32_t wcount[kGroups][17];
    __shared__ int64_t end_sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint32_t count = *big_count;
    for (uint32_t q = blockIdx.x; q < count; q += gridDim.x) {
        const int64_t start = big[q];
        if (threadIdx.x == 0) end_sh = run_end(keys, n, start);
        if (threadIdx.x < kLowDigits * 16) (&hist[0][0])[threadIdx.x] = 0;
        __syncthreads();
        const int64_t len = end_sh - start;
        unsigned long long *sk = keys + start, *dk = alt_keys + start;
        uint32_t *sv = vals ? vals + start : nullptr, *dv = alt_vals ? alt_vals + start : nullptr;
        for (int64_t t0 = 0; t0 < len; t0 += blockDim.x) {
            const int64_t t = t0 + threadIdx.x;
            const unsigned long long k = t < len ? sk[t] : 0ull;
#pragma unroll
            for (int p = 0; p < kLowDigits; ++p) {
                const int d = t < len ? int((k >> (4 * p)) & 15) : 16;
                const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
                if (d < 16 && (peers & lt_mask) == 0u) atomicAdd(&hist[p][d], __popc(peers));
            }
        }
        __syncthreads();
        for (int p = 0; p < kLowDigits; ++p) {
            const int shift = 4 * p;
            if (threadIdx.x == 0) {
                uint32_t run = 0;
                for (int d = 0; d < 16; ++d) {
                    base[d] = run;
                    run += hist[p][d];
                }
            }
            for (int64_t t0 = 0; t0 < len; t0 += int64_t(blockDim.x) * kBlockItems) {
                unsigned long long k[kBlockItems];
                uint32_t v[kBlockItems];
                int d[kBlockItems];
#pragma unroll
                for (int j = 0; j < kBlockItems; ++j) {
                    const int64_t t = t0 + int64_t(j) * blockDim.x + threadIdx.x;
                    k[j] = t < len ? sk[t] : 0ull;
                    v[j] = (sv && t < len) ? sv[t] : 0u;
                    d[j] = t < len ? int((k[j] >> shift) & 15) : 16;
                }
                for (int e = threadIdx.x; e < kGroups * 17; e += blockDim.x) (&wcount[0][0])[e] = 0;
                __syncthreads();
                unsigned peers[kBlockItems];
#pragma unroll
                for (int j = 0; j < kBlockItems; ++j) {
                    peers[j] = __match_any_sync(0xFFFFFFFFu, d[j]);
                    if ((peers[j] & lt_mask) == 0u) wcount[j * kWarps + warp][d[j]] = __popc(peers[j]);
                }
                __syncthreads();
                if (threadIdx.x < 16) {  // first place of each group's keys of digit threadIdx.x
                    uint32_t run = base[threadIdx.x];
                    for (int g = 0; g < kGroups; ++g) {
                        const uint32_t c = wcount[g][threadIdx.x];
                        wcount[g][threadIdx.x] = run;
                        run += c;
                    }
                    base[threadIdx.x] = run;
                }
                __syncthreads();
#pragma unroll
                for (int j = 0; j < kBlockItems; ++j) {
                    if (d[j] < 16) {
                        const uint32_t pos = wcount[j * kWarps + warp][d[j]] + __popc(peers[j] & lt_mask);
                        dk[pos] = k[j];
                        if (dv) dv[pos] = v[j];
                    }
                }
                __syncthreads();
            }
            unsigned long long *tk = sk;
            sk = dk;
            dk = tk;
            uint32_t *tv = sv;
            sv = dv;
            dv = tv;
        }
    }
}
}  // namespace

void carve_run_fix(Carver &c, int64_t cap, RunFixBuffers &r) {
    r.descent = c.take<uint8_t>(size_t((cap + 31) / 32 + 16));
    r.runs = c.take<uint32_t>(size_t(cap / (kShortRun + 1) + 1));
    r.big = c.take<uint32_t>(size_t(cap / (kWarpRun + 1) + 1));
    r.counts = c.take<uint32_t>(3);  // runs, big runs, longest big run
}

// digit counts of every pass, tile counters, then the grid-barrier words of
// the cooperative sort
int64_t sort_counter_words() { return int64_t(kMaxPasses) * kBins + kMaxPasses + 4; }

int radix_sort_high_result(int64_t cap, int end_bit) {
    const int passes = (end_bit + 7) / 8;
    if (end_bit <= kLowBits || passes > kMaxPasses || cap >= (int64_t(1) << 32)) return passes & 1;
    return (passes - kLowBits / 8) & 1;
}

int radix_sort_high(SortBuffers &b, const RunFixBuffers &r, int64_t cap, const int64_t *d_count, int end_bit,
                    cudaStream_t s, int *result_buffer, uint32_t *dev_status, bool counters_cleared) {
    const int passes = (end_bit + 7) / 8;
    if (end_bit <= kLowBits || passes > kMaxPasses || cap >= (int64_t(1) << 32))
        return radix_sort(b, cap, d_count, end_bit, s, result_buffer, dev_status);
    const int items = sort_items(cap);
    uint32_t *tile_counters = b.counts + kMaxPasses * kBins;
    if (!counters_cleared)
        BGV_CUDA(cudaMemsetAsync(b.counts, 0, sizeof(uint32_t) * size_t(sort_counter_words()), s));
    constexpr int first = kLowBits / 8;
    int cur = 0;
    if (use_coop(cap, b.vals[0] != nullptr)) {
        BGV_CUDA(cudaMemsetAsync(r.counts, 0, 3 * sizeof(uint32_t), s));
        BGV_TRY(coop_sort(b, cap, d_count, first, passes, s, dev_status));
        cur = (passes - first) & 1;
    } else {
        const int64_t count_blocks = (cap + kCountTile - 1) / kCountTile;  // >= tiles
        note_launch(), k_sort_count<<<static_cast<unsigned>(count_blocks > 0 ? count_blocks : 1), kSortThreads, 0,
                                      s>>>(b.keys[0], cap, d_count, first, passes, b.counts, b.status,
                                           tiles_for(cap, items), r.counts, 3);
        BGV_TRY(launch_status());
        for (int p = first; p < passes; ++p) {
            BGV_TRY(onesweep_pass(b, cap, d_count, cur, 8 * p, b.counts + p * kBins, tile_counters + p, pass_tag(p),
                                  items, s, dev_status));
            cur ^= 1;
        }
    }
    if (cap > 1) {
        note_launch(), k_fix_runs<<<grid_for(cap, kFixThreads, sm_count() * 64), kFixThreads, 0, s>>>(
            b.keys[cur], b.vals[cur], cap, d_count, r.descent, r.runs, r.counts);
        note_launch(), k_fix_warp<<<sm_count() * 8, kFixThreads, 0, s>>>(b.keys[cur], b.vals[cur], cap, d_count,
                                                                         r.descent, r.runs, r.counts, r.big,
                                                                         r.counts + 1);
        // the guard: a run too long for one block -> a full LSD sort of the
        // array (an even number of passes, so the result stays in `cur`)
        SortBuffers g = b;
        if (cur == 1) {
            std::swap(g.keys[0], g.keys[1]);
            std::swap(g.vals[0], g.vals[1]);
        }
        BGV_TRY(coop_sort(g, cap, d_count, 0, (passes + 1) & ~1, s, dev_status, r.counts + 2, kFixGuard));
        note_launch(), k_fix_block<<<sm_count() * 2, kFixThreads, 0, s>>>(b.keys[cur], b.vals[cur], b.keys[cur ^ 1],
                                                                          b.vals[cur ^ 1], cap, d_count, r.big,
                                                                          r.counts + 1);
        BGV_TRY(launch_status());
    }
    *result_buffer = cur;
    return BGV_OK;
}

// ------------------------------------------------ bounded-wait self check
// One onesweep block as tile 1 of a two-tile, all-zero key set whose tile 0
// never runs: its look-back finds nothing published and must give up at the
// spin limit (BGV_DEV_TIMEOUT).  Every digit offset is 0, so the block's
// writes stay inside its own tile's slots.
size_t wait_check_sort_bytes() {
    Carver c(nullptr, 0);
    SortBuffers b;
    carve_sort(c, 2 * int64_t(kSortThreads) * kSortItemsSmall, false, b);
    return c.used();
}

int wait_check_sort(void *scratch, uint32_t *dev_status, cudaStream_t s) {
    const int64_t cap = 2 * int64_t(kSortThreads) * kSortItemsSmall;
    Carver c(scratch, 0);
    SortBuffers b;
    carve_sort(c, cap, false, b);
    BGV_CUDA(cudaMemsetAsync(scratch, 0, wait_check_sort_bytes(), s));
    const uint32_t one = 1u;  // the tile counter: the launched block takes tile 1
    uint32_t *tile_counter = b.counts + kMaxPasses * kBins;
    BGV_CUDA(cudaMemcpyAsync(tile_counter, &one, sizeof(one), cudaMemcpyHostToDevice, s));
    note_launch(), k_sort_onesweep<false, kSortItemsSmall><<<1, kSortThreads, 0, s>>>(
        b.keys[0], b.keys[1], nullptr, nullptr, cap, nullptr, 0, b.counts, tile_counter, b.status, dev_status,
        pass_tag(0), spin_limit());
    BGV_TRY(launch_status());
    return cudaStreamSynchronize(s) == cudaSuccess ? BGV_OK : BGV_ECUDA;  // `one` lives on this stack
}

// ------------------------------------------------------------- autotuner
// Times the sort of 48-bit keys with values at 8 and at 16 keys per thread
// for sizes 2^14 .. max_keys (powers of four) and sets the cutoff to the
// largest size at which 8 was not slower.  Keys come from SplitMix64 of the
// index, so every GPU sees the same inputs.
namespace {
__global__ void k_tune_keys(unsigned long long *keys, uint32_t *vals, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        unsigned long long z = 0x5EEDull + static_cast<unsigned long long>(i) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        keys[i] = (z ^ (z >> 31)) & ((1ull << 48) - 1);
        vals[i] = uint32_t(i);
    }
}
}  // namespace

int64_t sort_cutoff() { return g_small_sort_cutoff.load(std::memory_order_relaxed); }
int64_t set_sort_cutoff(int64_t cutoff) { return g_small_sort_cutoff.exchange(cutoff, std::memory_order_relaxed); }
int set_sort_method(int method) { return g_sort_method.exchange(method, std::memory_order_relaxed); }
int sort_method() { return g_sort_method.load(std::memory_order_relaxed); }
void sort_coop_range(int64_t *lo, int64_t *hi) {
    *lo = g_coop_lo.load(std::memory_order_relaxed);
    *hi = g_coop_hi.load(std::memory_order_relaxed);
}

int autotune_sort(int64_t max_keys, SortBuffers &b, cudaStream_t s, uint32_t *dev_status, float *ms8, float *ms16,
                  float *ms_coop, int32_t *sizes_log2, int32_t *count, int32_t *method) {
    cudaEvent_t e0, e1;
    BGV_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return BGV_ECUDA;
    }
    const int method_before = g_sort_method.load(std::memory_order_relaxed);
    int rc = BGV_OK;
    int64_t cutoff = 0, coop_lo = -1, coop_hi = -1;
    int k = 0;
    for (int lg = 14; lg <= 30 && (int64_t(1) << lg) <= max_keys && rc == BGV_OK; lg += 2, ++k) {
        const int64_t n = int64_t(1) << lg;
        float best[3] = {0.0f, 0.0f, 0.0f};
        for (int v = 0; v < 3 && rc == BGV_OK; ++v) {
            // v 0, 1: onesweep passes at 8 and 16 keys per thread; v 2: cooperative
            const int items = v == 1 ? kSortItemsBig : kSortItemsSmall;
            g_sort_method.store(v == 2 ? 1 : 0, std::memory_order_relaxed);
            float times[3];
            for (int r = 0; r < 4 && rc == BGV_OK; ++r) {
                note_launch(), k_tune_keys<<<grid_for(n, 256, sm_count() * 8), 256, 0, s>>>(b.keys[0], b.vals[0], n);
                int res = 0;
                if (cudaEventRecord(e0, s) != cudaSuccess) rc = BGV_ECUDA;
                if (rc == BGV_OK) rc = radix_sort(b, n, nullptr, 48, s, &res, dev_status, items);
                if (rc == BGV_OK && cudaEventRecord(e1, s) != cudaSuccess) rc = BGV_ECUDA;
                if (rc == BGV_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = BGV_ECUDA;
                float ms = 0.0f;
                if (rc == BGV_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = BGV_ECUDA;
                if (r > 0) times[r - 1] = ms;  // the first run warms up
            }
            if (rc != BGV_OK) break;
            std::sort(times, times + 3);
            best[v] = times[1];
        }
        if (rc != BGV_OK) break;
        if (ms8) ms8[k] = best[0];
        if (ms16) ms16[k] = best[1];
        if (ms_coop) ms_coop[k] = best[2];
        if (sizes_log2) sizes_log2[k] = lg;
        if (best[0] <= best[1]) cutoff = n;
        if (best[2] < (best[0] < best[1] ? best[0] : best[1])) {  // cooperative faster at this size
            if (coop_lo < 0) coop_lo = n;
            coop_hi = n;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (count) *count = k;
    if (rc == BGV_OK) {
        // the cutoff of the onesweep passes, and the cooperative sort for the
        // span of sizes from the first to the last at which it was faster
        // (reaching halfway to the neighbouring sizes timed)
        g_small_sort_cutoff.store(cutoff, std::memory_order_relaxed);
        if (coop_lo > 0) {
            g_coop_lo.store(coop_lo - coop_lo / 2, std::memory_order_relaxed);
            g_coop_hi.store(coop_hi * 2 - 1, std::memory_order_relaxed);
            g_sort_method.store(2, std::memory_order_relaxed);
        } else {
            g_sort_method.store(0, std::memory_order_relaxed);
        }
    } else {
        g_sort_method.store(method_before, std::memory_order_relaxed);
    }
    if (method) *method = g_sort_method.load(std::memory_order_relaxed);
    return rc;
}

}  // namespace bgv

// bgv_internal.cuh -- shared internals of libbgv (GB300, sm_103a).
//
// Workspace carving, the hash family of the count-min sketches, the device
// status word, and the interfaces of the generic scan and radix sort used by
// the supergraph and ForceAtlas2 stages.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "bgv.h"

namespace bgv {

// ---------------------------------------------------------------- workspace
// Grid barrier words of a persistent kernel: arrivals (back to 0 after each
// barrier), generation, and an abort word set when a wait gave up (it stays
// set, and the barriers using these words fail at once, until cleared).
struct GridBar {
    unsigned int count, gen, abort, pad;
};

// Every public workspace starts with this header (kHeaderBytes bytes).
struct WsHeader {
    uint32_t status;        // BGV_DEV_* bits
    uint32_t pad0;
    // accumulated since bgv_ws_init
    unsigned long long interactions_total;  // FA2 terms over all steps
    unsigned long long steps_total;         // FA2 steps completed
    // per step (cleared at the start of every FA2 step)
    unsigned long long interactions;  // FA2: terms of the last step
    unsigned long long tree_nodes;    // FA2: quadtree internal nodes of the last step
    double S, T;                      // FA2: swing and traction of the last step
    unsigned int bbox_ticket;         // last-block tickets (reset by the last block)
    unsigned int node_ticket;
    // grid barrier of the persistent kernels (see GridBar)
    GridBar bar;
    unsigned long long reserved[20];
};
static_assert(sizeof(WsHeader) <= 256, "header must fit in 256 bytes");
constexpr size_t kHeaderBytes = 256;
constexpr size_t kAlign = 256;

// Sequential sub-allocator over a caller workspace.  With base == nullptr it
// only measures, which is how the *_ws_size queries are computed, so the two
// can never disagree.
struct Carver {
    char *base;
    size_t off;
    explicit Carver(void *b, size_t start = 0) : base(static_cast<char *>(b)), off(start) {}
    template <class T>
    T *take(size_t count) {
        off = (off + kAlign - 1) / kAlign * kAlign;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += (count ? count : 1) * sizeof(T);
        return p;
    }
    size_t used() const { return (off + kAlign - 1) / kAlign * kAlign; }
};

inline WsHeader *header(void *ws) { return static_cast<WsHeader *>(ws); }
inline uint32_t *status_ptr(void *ws) { return &header(ws)->status; }

#define BGV_TRY(expr)                         \
    do {                                      \
        int rc_ = (expr);                     \
        if (rc_ != BGV_OK) return rc_;        \
    } while (0)

#define BGV_CUDA(expr)                                   \
    do {                                                 \
        if ((expr) != cudaSuccess) return BGV_ECUDA;     \
    } while (0)

inline int launch_status() { return cudaGetLastError() == cudaSuccess ? BGV_OK : BGV_ECUDA; }

// Process-wide count of kernel launches issued by the library (every launch
// site calls note_launch; graph replays are added by the replay loop).
void note_launch();
void add_launches(unsigned long long n);
unsigned long long launches_issued();

// Polling rounds after which a decoupled look-back wait gives up and sets
// BGV_DEV_TIMEOUT (passed to the kernels at launch; process wide).
int spin_limit();
int set_spin_limit(int limit);  // returns the previous limit

// Multiprocessors of the current device (queried once per device and
// cached; 1 if the query fails, which keeps every grid-stride launch valid).
int sm_count();

// Blocks for `work` items of `threads` each, at most `cap_blocks` (default:
// 16 per multiprocessor); every kernel launched this way strides over the
// grid, so the cap only sets how many blocks share the work.
inline int grid_for(int64_t work, int threads, int64_t cap_blocks = -1) {
    if (cap_blocks < 1) cap_blocks = int64_t(sm_count()) * 16;
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap_blocks) b = cap_blocks;
    return static_cast<int>(b);
}

__device__ __forceinline__ void raise_status(uint32_t *status, uint32_t bits) { atomicOr(status, bits); }

// ------------------------------------------------------------- hash family
// h_i(x) = ((a_i x + b_i) mod (2^31 - 1)) mod width; coefficients from
// SplitMix64 (Steele, Lea, Flood 2014) at state seed + i.
constexpr int kMaxRows = 16;
struct HashFamily {
    unsigned long long a[kMaxRows];
    unsigned long long b[kMaxRows];
    int rows;
    uint32_t width;
};

HashFamily make_hash_family(uint64_t seed, int rows, uint32_t width);

__device__ __forceinline__ uint32_t mod_p31(unsigned long long t) {
    // t < 2^63; fold twice with 2^31 = 1 (mod 2^31 - 1), then one subtraction.
    unsigned long long y = (t & 0x7FFFFFFFull) + (t >> 31);
    y = (y & 0x7FFFFFFFull) + (y >> 31);
    return static_cast<uint32_t>(y >= 0x7FFFFFFFull ? y - 0x7FFFFFFFull : y);
}

__device__ __forceinline__ uint32_t hash_eval(unsigned long long a, unsigned long long b, uint32_t x,
                                              uint32_t width) {
    return mod_p31(a * static_cast<unsigned long long>(x) + b) % width;
}

// ------------------------------------------------------------------- scan
// Exclusive prefix sum of uint32 values.  The element count is `n_cap`, or
// *d_n when d_n != nullptr (then n_cap is an upper bound used for the grid).
// If `total_u64` is given it receives the sum; if `total_u32_at_end` the sum
// is also stored at out[n].  Sums must fit in 32 bits.
size_t scan_tmp_bytes(int64_t n_cap);
int scan_exclusive(const uint32_t *in, uint32_t *out, int64_t n_cap, const int64_t *d_n,
                   unsigned long long *total_u64, bool total_u32_at_end, void *tmp, cudaStream_t s);

// ------------------------------------------------------------- radix sort
// Stable LSD radix sort of uint64 keys (bits [0, end_bit), end_bit <= 64)
// with optional uint32 values.  Count = *d_count if given, else cap.
// keys[0]/vals[0] hold the input; *result_buffer receives the index (0 or 1)
// of the buffer pair holding the sorted output.  A look-back wait that hits
// its bound sets BGV_DEV_TIMEOUT in *dev_status.
struct SortBuffers {
    unsigned long long *keys[2];
    uint32_t *vals[2];               // both nullptr for keys only
    unsigned long long *status;      // 256 look-back words per tile
    uint32_t *counts;                // per-pass digit offsets, then tile counters
};
int64_t sort_tiles(int64_t cap);
void carve_sort(Carver &c, int64_t cap, bool with_vals, SortBuffers &out);
// `items` 8 or 16 forces the keys per thread; anything else follows the
// size cutoff (see autotune_sort).
int radix_sort(SortBuffers &b, int64_t cap, const int64_t *d_count, int end_bit, cudaStream_t s,
               int *result_buffer, uint32_t *dev_status, int items = 0);

// The same order (keys, with values when b.vals[0] is set) when the keys
// are nearly always told apart above their low kLowBits bits: LSD passes on
// the bits above them only, then every run of equal high bits sorted
// locally on its low bits.  Count = *d_count if given, else cap.
constexpr int kLowBits = 24;
struct RunFixBuffers {
    uint8_t *descent;   // per 32-key chunk: holds a key below its predecessor in the same run
    uint32_t *runs;     // starts of runs too long for one thread
    uint32_t *big;      // starts of runs too long for one warp
    uint32_t *counts;   // [0] runs, [1] big
};
void carve_run_fix(Carver &c, int64_t cap, RunFixBuffers &r);
// Words of SortBuffers::counts (digit counts and tile counters): cleared
// before a sort, by the sort itself unless its caller cleared them.
int64_t sort_counter_words();
int radix_sort_high(SortBuffers &b, const RunFixBuffers &r, int64_t cap, const int64_t *d_count, int end_bit,
                    cudaStream_t s, int *result_buffer, uint32_t *dev_status, bool counters_cleared = false);
// The buffer pair radix_sort_high(cap, end_bit) leaves its result in.
int radix_sort_high_result(int64_t cap, int end_bit);

// Sort autotuner: times the onesweep passes at 8 and at 16 keys per thread
// and the cooperative sort for 2^14, 2^16, ... up to max_keys; sets the
// cutoff between 8 and 16 (the largest size at which 8 was not slower) and
// the span of sizes where the cooperative sort was faster (method 2), or
// onesweep everywhere (method 0), for the whole process.  Per size k (count
// of them in *count): ms8[k], ms16[k], ms_coop[k], sizes_log2[k] (host
// arrays, may be NULL; 9 entries suffice).  b must hold max_keys pairs.
int autotune_sort(int64_t max_keys, SortBuffers &b, cudaStream_t s, uint32_t *dev_status, float *ms8, float *ms16,
                  float *ms_coop, int32_t *sizes_log2, int32_t *count, int32_t *method);
int64_t sort_cutoff();
int64_t set_sort_cutoff(int64_t cutoff);  // returns the previous cutoff
// 0: onesweep passes with decoupled look-back, 1: all passes in one
// cooperative kernel, 2 (default): cooperative for key counts in the range
// sort_coop_range gives, onesweep otherwise.  Process wide; returns the
// previous method.
int set_sort_method(int method);
int sort_method();
void sort_coop_range(int64_t *lo, int64_t *hi);



// Number of bits needed to hold values 0..n-1 (at least 1).
inline int bits_for(int64_t n) {
    int b = 1;
    while (b < 62 && (int64_t(1) << b) < n) ++b;
    return b;
}

// ------------------------------------------------- persistent kernels
// Grid-wide barrier for kernels launched cooperatively (all blocks resident
// at once).  The last block to arrive resets the count and advances the
// generation; the others poll the generation for at most spin_limit rounds,
// then set BGV_DEV_TIMEOUT and the abort word, and every later barrier of the
// workspace returns false at once.  Returns true when all blocks arrived.
__device__ __forceinline__ bool grid_barrier(GridBar *h, int spin_limit, uint32_t *status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = &h->gen, *abort = &h->abort;
        const unsigned int g = *gen;  // read before arriving
        __threadfence();
        int good = *abort == 0u;
        if (good) {
            if (atomicAdd(&h->count, 1u) + 1u == gridDim.x) {
                h->count = 0u;
                __threadfence();
                atomicAdd(&h->gen, 1u);
            } else {
                int spins = 0;
                while (*gen == g) {
                    if (*abort != 0u) {
                        good = 0;
                        break;
                    }
                    if (++spins > spin_limit) {
                        atomicOr(status, BGV_DEV_TIMEOUT);
                        atomicExch(&h->abort, 1u);
                        good = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Blocks of `threads` threads that a cooperative launch of `kernel` can keep
// resident at once, at most `want` (at least 1).
int coop_blocks(const void *kernel, int threads, int want);
// Cooperative launch on `st` (all blocks resident together).
int launch_coop(const void *kernel, int blocks, int threads, void **args, cudaStream_t st);

// --------------------------------------------------------- stage internals
// Enqueue-only stage bodies used by the public entry points and the
// pipeline; `status` points at the device status word.

// Batched form: G independent graphs laid side by side in one id space.
// Graph g owns nodes [node_off[g], node_off[g+1]); every stage keeps the
// graphs apart exactly as G separate calls would (own sketch matrices,
// hashing of local ids, own degree thresholds).  All arrays on the device.
struct BatchView {
    int32_t G;
    const int32_t *node_off;    // [G + 1]
    const int32_t *node_graph;  // [N] graph of each node
    const uint32_t *D0;         // [G] first-round degree threshold
};
struct SketchScratch {
    uint32_t *deg;
};
void carve_sketch(Carver &c, int64_t m, int32_t n, int32_t rows, int32_t width, SketchScratch &s);
// With `batch`, `sketch` holds G matrices of rows x width, one per graph.
int run_sketch(const int32_t *edges, int64_t m, int32_t n, const HashFamily &h, uint32_t *sketch,
               uint32_t *deg_est, const SketchScratch &s, uint32_t *status, cudaStream_t st,
               const BatchView *batch = nullptr);

struct CommScratch {
    uint2 *state;                   // (degree, label) per node
    uint4 *bstate;                  // batched form: (degree, label, threshold, first threshold)
    unsigned long long *best;       // packed (edge index, label) proposals
    uint32_t *jump;                 // labels after a pointer-jumping step
};
void carve_comm(Carver &c, int64_t m, int32_t n, CommScratch &s, bool batched = false);
// growth 0: the threshold is multiplied by its first value every round (the
// delta^i schedule).  `jumps` pointer-jumping steps follow every round.
// With `batch`, the threshold of every node starts at its graph's D0 and
// `threshold` is ignored.
// All rounds run in one persistent kernel whose grid barrier lives in `hdr`
// (the workspace header); its waits are bounded (BGV_DEV_TIMEOUT).
int run_communities(const int32_t *edges, int64_t m, int32_t n, const uint32_t *deg_est, int32_t passes,
                    uint32_t threshold, uint32_t growth, int32_t tie_mode, int32_t jumps, int32_t *labels,
                    uint32_t *deg_out, const CommScratch &s, uint32_t *status, cudaStream_t st,
                    const BatchView *batch, WsHeader *hdr);

// Mode degree: the most frequent nonzero value of deg (ties: the smaller),
// 0 if none; with `batch`, one per graph.  mode_dev: device, 1 or G values.
struct ModeScratch {
    SortBuffers sort;            // n keys (graph << 32 | degree)
    unsigned long long *best;    // per graph: (run length, ~degree)
};
void carve_mode(Carver &c, int32_t n, int32_t G, ModeScratch &s);
int run_mode_degree(const uint32_t *deg, int32_t n, const BatchView *batch, uint32_t *mode_dev,
                    const ModeScratch &s, uint32_t *status, cudaStream_t st);

struct SuperScratch {
    uint32_t *flags;        // [n+1] label present
    uint32_t *rank;         // [n+1]
    int32_t *label_of;      // [n]
    unsigned long long *nkeys;  // device count of (row, col) keys
    int64_t *nnz;           // device count of CSR entries
    unsigned long long *sketch;  // [rows * width], batched form: one per graph
    uint32_t *start;        // [2m + 1] first sorted key of every CSR entry
    int32_t *supidx;        // [2m] superedge of every CSR entry, -1 for col < row
    uint32_t *red_flags;    // look-back flags of the CSR pass, then its tile counter
    unsigned long long *red_agg, *red_incl;
    void *scan_tmp;
    SortBuffers sort_pairs;   // 2m keys
};
void carve_super(Carver &c, int64_t m, int32_t n, int32_t rows, int32_t width, SuperScratch &s, int32_t G = 1);
// With `batch`, community labels are node ids of their own graph, so the
// supernodes come out graph-major; the community-size sketch of graph g
// hashes local labels into its own matrix.
int run_supergraph(const int32_t *edges, int64_t m, int32_t n, const int32_t *labels, const uint32_t *deg_est,
                   const HashFamily &h, int32_t *node_map, int64_t *K_dev, int32_t *ssrc, int32_t *sdst,
                   uint32_t *sw, int64_t *Es_dev, uint32_t *mass, int32_t *csr_off, int32_t *csr_adj,
                   uint32_t *csr_w, uint64_t *vol, uint32_t *count, int32_t *comm_label,
                   const SuperScratch &s, uint32_t *status, cudaStream_t st, const BatchView *batch = nullptr);

// Launch shapes of a FA2 step (process wide; chosen by the autotuner): the
// longest rows the attraction sums one lane each (8, 16, 32; longer ones take
// a warp or a block), threads per block of the Barnes-Hut traversal (128,
// 256), blocks per SM of the persistent tail kernel (1..8, at most what
// stays resident).
struct Fa2Tune {
    int att_short, repulse_threads, tail_blocks_per_sm;
};
Fa2Tune fa2_tune();
int set_fa2_tune(const Fa2Tune &t);

// Scratch for one FA2 step over G graphs (G = 1: a single layout), carved
// from `scratch` (not counting a header).
size_t fa2_scratch_bytes(int64_t K, int64_t nnz, int32_t G = 1);
int fa2_check_params(const bgv_fa2_params *p);
// Batched form (G > 1): graph g owns bodies [koff[g], koff[g+1]) (koff on the
// device); speed then holds G values.  The sort keys put the graph id above
// the 2 max_depth Morton bits, so both must fit in 64 bits.
inline bool fa2_batch_fits(int32_t G, int max_depth) { return G <= 1 || 2 * max_depth + bits_for(G) <= 64; }
int run_fa2_init(int64_t K, const bgv_fa2_params &p, float *pos, float *Fprev, double *speed, cudaStream_t st,
                 int32_t G = 1, const int64_t *koff = nullptr);
// mode 0: forces only (Fr/Fa/Fg outputs, any may be null); mode 1: full step.
// `marks` (optional) receives kFa2Stages + 1 event records at the stage
// boundaries: frame+keys, sort, gather, tree, quad, repulsion, node, update.
// `build_plan` rebuilds the per-CSR attraction plan in the scratch; a loop
// over one CSR builds it on the first step only.
constexpr int kFa2Stages = 8;
int run_fa2(int mode, int64_t K, int64_t nnz, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
            const uint32_t *mass, const bgv_fa2_params &p, float *pos, float *F, float *Fprev, double *speed,
            float *Fr, float *Fa, float *Fg, WsHeader *hdr, void *scratch, cudaStream_t st,
            cudaEvent_t *marks = nullptr, bool build_plan = true, int32_t G = 1, const int64_t *koff = nullptr,
            bool hinted = false);
// `hinted`: the scratch holds the previous step's Morton order of the same
// bodies (the step before ran on this scratch with the same K and G), which
// then serves as the hint of the hinted sort (when fa2_order() is 1).
int fa2_order();
int set_fa2_order(int method);  // 0 or 1; returns the previous method, -1 for others

// Bounded-wait self checks: one block of a look-back kernel whose
// predecessor tile never publishes (sort pass, FA2 moment pass, CSR pass).
// Each synchronises `s`; the wait's timeout lands in *dev_status.
size_t wait_check_sort_bytes();
int wait_check_sort(void *scratch, uint32_t *dev_status, cudaStream_t s);
size_t wait_check_moments_bytes();
int wait_check_moments(void *scratch, uint32_t *dev_status, cudaStream_t s);
size_t wait_check_reduce_bytes();
int wait_check_reduce(void *scratch, uint32_t *dev_status, cudaStream_t s);

}  // namespace bgv

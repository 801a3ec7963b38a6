// sketch.cu -- degree count-min sketch (Algorithm 2, Section 3.3).
//
// Algorithm 2 adds 1 to M[i][h_i(x)] for every event x; the events here are
// the 2m edge endpoints.  Integer addition commutes, so the same matrix is
// built from exact per-node degrees: one edge pass counts degrees (L2
// atomics on an n-entry array, aggregated per warp over equal node ids),
// then every node with degree d adds d to its r cells.  That turns 2 r m
// scattered sketch updates into at most 2m + r n.
//
// Edges are read as int4 (two edges per 16-byte load) with a grid-stride
// loop over a grid sized to fill the GPU.
#include <mutex>

#include "bgv_internal.cuh"

namespace bgv {

HashFamily make_hash_family(uint64_t seed, int rows, uint32_t width) {
    HashFamily h{};
    const unsigned long long p = 2147483647ull;
    for (int i = 0; i < rows && i < kMaxRows; ++i) {
        unsigned long long st = seed + static_cast<unsigned long long>(i);
        unsigned long long z[2];
        for (int k = 0; k < 2; ++k) {
            st += 0x9E3779B97F4A7C15ull;
            unsigned long long x = st;
            x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
            x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
            z[k] = x ^ (x >> 31);
        }
        h.a[i] = 1 + z[0] % (p - 1);
        h.b[i] = z[1] % p;
    }
    h.rows = rows;
    h.width = width;
    return h;
}

namespace {
constexpr int kThreads = 256;

// One endpoint per lane: lanes holding the same node id are found with
// __match_any_sync and only the lowest of them adds their number, so a hub
// that shows up several times in a warp's 32 endpoints costs one atomic.
__device__ __forceinline__ void count_endpoints_warp(bool have, int32_t x, int32_t n, uint32_t *deg,
                                                     uint32_t *status) {
    const bool ok = have && static_cast<uint32_t>(x) < static_cast<uint32_t>(n);
    if (have && !ok) raise_status(status, BGV_DEV_BADEDGE);
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, ok ? x : -1);
    const int lane = threadIdx.x & 31;
    if (ok && (peers & ((1u << lane) - 1u)) == 0u) atomicAdd(&deg[x], uint32_t(__popc(peers)));
}

// Whole warps iterate together (the exit test uses the warp's first index)
// so every __match_any_sync sees all 32 lanes.  Each lane loads two int4
// (four edges) before counting, so the loads are in flight together.
constexpr int kDegLoads = 2;
__global__ void __launch_bounds__(kThreads) k_degree_count(const int32_t *__restrict__ edges, int64_t m, int32_t n,
                                                           uint32_t *__restrict__ deg, uint32_t *status) {
    const int4 *e2 = reinterpret_cast<const int4 *>(edges);
    const int64_t pairs = m >> 1;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t base = warp * 32 * kDegLoads; base < pairs; base += warps * 32 * kDegLoads) {
        int4 e[kDegLoads];
        bool have[kDegLoads];
#pragma unroll
        for (int r = 0; r < kDegLoads; ++r) {
            const int64_t p = base + int64_t(r) * 32 + lane;
            have[r] = p < pairs;
            e[r] = have[r] ? __ldcs(e2 + p) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int r = 0; r < kDegLoads; ++r) {
            count_endpoints_warp(have[r], e[r].x, n, deg, status);
            count_endpoints_warp(have[r], e[r].y, n, deg, status);
            count_endpoints_warp(have[r], e[r].z, n, deg, status);
            count_endpoints_warp(have[r], e[r].w, n, deg, status);
        }
    }
    if ((m & 1) && blockIdx.x == 0 && threadIdx.x < 32) {  // the odd last edge, one warp
        count_endpoints_warp(lane == 0, edges[2 * (m - 1)], n, deg, status);
        count_endpoints_warp(lane == 0, edges[2 * (m - 1) + 1], n, deg, status);
    }
}

// Batched form: node v of graph g = node_graph[v] hashes its local id
// v - node_off[g] into graph g's own rows x width matrix.
__device__ __forceinline__ uint32_t *sketch_of(uint32_t *sketch, const HashFamily &h, int64_t v,
                                               const int32_t *node_graph, const int32_t *node_off, uint32_t *x) {
    if (!node_graph) {
        *x = uint32_t(v);
        return sketch;
    }
    const int32_t g = node_graph[v];
    *x = uint32_t(v - node_off[g]);
    return sketch + size_t(g) * size_t(h.rows) * h.width;
}

__global__ void __launch_bounds__(kThreads) k_sketch_fill(const uint32_t *__restrict__ deg, int32_t n,
                                                          const __grid_constant__ HashFamily h,
                                                          uint32_t *__restrict__ sketch,
                                                          const int32_t *__restrict__ node_graph,
                                                          const int32_t *__restrict__ node_off) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint32_t d = deg[v];
        if (d == 0) continue;
        uint32_t x;
        uint32_t *M = sketch_of(sketch, h, v, node_graph, node_off, &x);
        for (int i = 0; i < h.rows; ++i) atomicAdd(&M[size_t(i) * h.width + hash_eval(h.a[i], h.b[i], x, h.width)], d);
    }
}

__global__ void __launch_bounds__(kThreads) k_sketch_query(const uint32_t *__restrict__ sketch, int32_t n,
                                                           const __grid_constant__ HashFamily h,
                                                           uint32_t *__restrict__ deg_est,
                                                           const int32_t *__restrict__ node_graph,
                                                           const int32_t *__restrict__ node_off) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint32_t x;
        const uint32_t *M = sketch_of(const_cast<uint32_t *>(sketch), h, v, node_graph, node_off, &x);
        uint32_t best = 0xFFFFFFFFu;
        for (int i = 0; i < h.rows; ++i) {
            uint32_t c = M[size_t(i) * h.width + hash_eval(h.a[i], h.b[i], x, h.width)];
            best = c < best ? c : best;
        }
        deg_est[v] = best;
    }
}
}  // namespace

void carve_sketch(Carver &c, int64_t m, int32_t n, int32_t rows, int32_t width, SketchScratch &s) {
    (void)m; (void)rows; (void)width;
    s.deg = c.take<uint32_t>(size_t(n));
}

int run_sketch(const int32_t *edges, int64_t m, int32_t n, const HashFamily &h, uint32_t *sketch,
               uint32_t *deg_est, const SketchScratch &s, uint32_t *status, cudaStream_t st, const BatchView *batch) {
    const int32_t *node_graph = batch ? batch->node_graph : nullptr;
    const int32_t *node_off = batch ? batch->node_off : nullptr;
    const size_t mats = batch ? size_t(batch->G) : 1;
    BGV_CUDA(cudaMemsetAsync(s.deg, 0, sizeof(uint32_t) * size_t(n), st));
    BGV_CUDA(cudaMemsetAsync(sketch, 0, sizeof(uint32_t) * size_t(h.rows) * h.width * mats, st));
    if (m > 0) {
        note_launch(), k_degree_count<<<grid_for((m / 2 + kDegLoads - 1) / kDegLoads, kThreads, sm_count() * 8), kThreads, 0, st>>>(edges, m, n, s.deg, status);
        BGV_TRY(launch_status());
    }
    note_launch(), k_sketch_fill<<<grid_for(n, kThreads, sm_count() * 8), kThreads, 0, st>>>(s.deg, n, h, sketch, node_graph,
                                                                                       node_off);
    BGV_TRY(launch_status());
    note_launch(), k_sketch_query<<<grid_for(n, kThreads, sm_count() * 8), kThreads, 0, st>>>(sketch, n, h, deg_est, node_graph,
                                                                                        node_off);
    return launch_status();
}

}  // namespace bgv

// ------------------------------------------------------------------------
// bgv_sketch_degrees_noalloc: the degree sketch for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc at all: a plugin running inside a
// host application whose device memory is owned by another allocator, code
// that runs while a stream is being captured (cudaMalloc is not allowed
// there), or real-time callers that must not allocate on their hot path.
// They cannot hand this library a workspace, so this entry point keeps the
// one scratch array the sketch needs -- the per-node degree counters -- in a
// fixed-size array of device memory that is part of the library image.  The
// caller still provides the edges, the sketch and the estimates.
//
// Size limit: n <= kNoAllocMaxNodes (4,194,304 nodes, 16 MiB of counters).
// Every GPU that loads the library holds that array until the process exits.
// All calls on a device share it and it keeps the last call's contents; the
// counters are cleared at the start of every call.  Calls whose work
// overlaps on the GPU (different streams, no ordering between them) race on
// the shared counters and give wrong results: order them on one stream.
namespace bgv {
namespace {
constexpr int32_t kNoAllocMaxNodes = 1 << 22;
constexpr int kNoAllocMaxDevices = 64;

// Degree counters followed by one status word used when the caller passes
// no status pointer (cleared by every such call and read back at its end).
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocMaxNodes + 64];

std::mutex g_noalloc_mutex;
uint32_t *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// The array's name is a host-side stand-in in host code, not a device
// address: the address a kernel may use is looked up once per device, with
// that device current, on the first call.
int noalloc_scratch(uint32_t **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return BGV_ECUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return BGV_ECUDA;
        g_noalloc_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return BGV_OK;
}
}  // namespace

}  // namespace bgv

extern "C" int bgv_sketch_degrees_noalloc(const int32_t *edges, int64_t m, int32_t n, int32_t rows, int32_t width,
                                          uint64_t seed, uint32_t *sketch, uint32_t *deg_est, uint32_t *status,
                                          void *stream) {
    using namespace bgv;
    if (n < 1 || m < 0 || m >= (int64_t(1) << 31)) return BGV_EINVAL;
    if (m > 0 && (!edges || reinterpret_cast<uintptr_t>(edges) % 16 != 0)) return BGV_EINVAL;
    if (rows < 1 || rows > kMaxRows || width < 1 || !sketch || !deg_est) return BGV_EINVAL;
    if (n > kNoAllocMaxNodes) return BGV_ELIMIT;
    uint32_t *scratch = nullptr;
    BGV_TRY(noalloc_scratch(&scratch));
    SketchScratch s;
    s.deg = scratch;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    const HashFamily h = make_hash_family(seed, rows, uint32_t(width));
    if (status) return run_sketch(edges, m, n, h, sketch, deg_est, s, status, cs);
    // No status word from the caller: use the one after the counters, cleared
    // on every call, and report what the device found before returning.
    uint32_t *own = scratch + kNoAllocMaxNodes;
    BGV_CUDA(cudaMemsetAsync(own, 0, sizeof(uint32_t), cs));
    BGV_TRY(run_sketch(edges, m, n, h, sketch, deg_est, s, own, cs));
    uint32_t seen = 0;
    BGV_CUDA(cudaMemcpyAsync(&seen, own, sizeof(uint32_t), cudaMemcpyDeviceToHost, cs));
    BGV_CUDA(cudaStreamSynchronize(cs));
    return seen ? BGV_EDEVICE : BGV_OK;
}


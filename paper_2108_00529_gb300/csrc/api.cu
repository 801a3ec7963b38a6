// api.cu -- the extern "C" entry points declared in include/bgv.h.
//
// Host-side validation, workspace sizing and carving, and the pipeline that
// chains the stages (Algorithm 3 end to end).  Everything on the data path
// runs in the kernels of sketch.cu, communities.cu, supergraph.cu and fa2.cu.
#include <algorithm>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "bgv_internal.cuh"

using namespace bgv;

namespace {

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int check_graph(const int32_t *edges, int64_t m, int32_t n) {
    if (n < 1 || n >= 0x7FFFFFFF || m < 0 || m >= (int64_t(1) << 31)) return BGV_EINVAL;
    if (m > 0 && (!edges || !aligned(edges, 16))) return BGV_EINVAL;
    return BGV_OK;
}

int check_sketch_shape(int32_t rows, int32_t width) {
    if (rows < 1 || rows > kMaxRows || width < 1) return BGV_EINVAL;
    return BGV_OK;
}

int check_ws(void *ws, size_t ws_bytes, size_t need) {
    if (!ws || !aligned(ws, kAlign)) return BGV_EINVAL;
    if (ws_bytes < need) return BGV_ENOSPC;
    return BGV_OK;
}

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

size_t sketch_ws(int64_t m, int32_t n, int32_t rows, int32_t width) {
    Carver c(nullptr, kHeaderBytes);
    SketchScratch s;
    carve_sketch(c, m, n, rows, width, s);
    return c.used();
}

size_t comm_ws(int64_t m, int32_t n) {
    Carver c(nullptr, kHeaderBytes);
    CommScratch s;
    carve_comm(c, m, n, s);
    return c.used();
}

size_t super_ws(int64_t m, int32_t n, int32_t rows, int32_t width) {
    Carver c(nullptr, kHeaderBytes);
    SuperScratch s;
    carve_super(c, m, n, rows, width, s);
    return c.used();
}

// ------------------------------------------------------------- pipeline
struct LayoutBuffers {
    uint32_t *sketch, *deg_est;
    uint32_t *mode;  // first-round threshold from the mode degree
    int32_t *labels;
    int64_t *K_dev, *Es_dev;
    int32_t *ssrc, *sdst;
    uint32_t *sw, *mass;
    int32_t *csr_off, *csr_adj;
    uint32_t *csr_w;
    float *F, *Fprev;
    double *speed;
    char *scratch;  // shared by the stages, which run one after another
};

size_t stage_scratch_bytes(int64_t m, int32_t n, const bgv_layout_params *p, int32_t G = 1) {
    size_t need = 0;
    {
        // the sketch's exact degree counters, then the mode degree from them
        Carver c(nullptr, 0);
        SketchScratch s;
        carve_sketch(c, m, n, p->rows, p->width, s);
        ModeScratch ms;
        carve_mode(c, n, G, ms);
        need = c.used() > need ? c.used() : need;
    }
    {
        Carver c(nullptr, 0);
        CommScratch s;
        carve_comm(c, m, n, s, G > 1);
        need = c.used() > need ? c.used() : need;
    }
    {
        Carver c(nullptr, 0);
        SuperScratch s;
        carve_super(c, m, n, p->rows, p->width, s, G);
        need = c.used() > need ? c.used() : need;
    }
    size_t f = fa2_scratch_bytes(n, 2 * m, G);
    return f > need ? f : need;
}

void carve_layout(Carver &c, int64_t m, int32_t n, const bgv_layout_params *p, LayoutBuffers &b, int32_t G = 1) {
    const size_t nn = size_t(n), mm = size_t(m > 0 ? m : 1), gg = size_t(G > 1 ? G : 1);
    b.sketch = c.take<uint32_t>(size_t(p->rows) * size_t(p->width) * gg);
    b.deg_est = c.take<uint32_t>(nn);
    b.mode = c.take<uint32_t>(1);
    b.labels = c.take<int32_t>(nn);
    b.K_dev = c.take<int64_t>(1);
    b.Es_dev = c.take<int64_t>(1);
    b.ssrc = c.take<int32_t>(mm);
    b.sdst = c.take<int32_t>(mm);
    b.sw = c.take<uint32_t>(mm);
    b.mass = c.take<uint32_t>(nn);
    b.csr_off = c.take<int32_t>(nn + 1);
    b.csr_adj = c.take<int32_t>(2 * mm);
    b.csr_w = c.take<uint32_t>(2 * mm);
    b.F = c.take<float>(2 * nn);
    b.Fprev = c.take<float>(2 * nn);
    b.speed = c.take<double>(gg);
    b.scratch = c.take<char>(stage_scratch_bytes(m, n, p, G));
}

int check_layout_params(const bgv_layout_params *p) {
    if (!p) return BGV_EINVAL;
    BGV_TRY(check_sketch_shape(p->rows, p->width));
    if (p->passes < 0 || (p->tie_mode != 0 && p->tie_mode != 1) || p->iterations < 0) return BGV_EINVAL;
    if ((p->threshold_mode != 0 && p->threshold_mode != 1) || p->jumps < 0 || p->jumps > 64) return BGV_EINVAL;
    return fa2_check_params(&p->fa2);
}

int fa2_loop(int64_t K, int64_t nnz, const int32_t *off, const int32_t *adj, const uint32_t *w, const uint32_t *mass,
             const bgv_fa2_params &p, int32_t iterations, int32_t use_graph, float *pos, float *F, float *Fprev,
             double *speed, WsHeader *hdr, void *scratch, cudaStream_t st, int32_t G = 1,
             const int64_t *koff = nullptr) {
    if (iterations <= 0 || K <= 0) return BGV_OK;
    if (!use_graph || st == nullptr || iterations < 2) {
        for (int32_t t = 0; t < iterations; ++t)
            BGV_TRY(run_fa2(1, K, nnz, off, adj, w, mass, p, pos, F, Fprev, speed, nullptr, nullptr, nullptr, hdr,
                            scratch, st, nullptr, t == 0, G, koff, t > 0));
        return BGV_OK;
    }
    // The first step runs outside the graph, builds the attraction plan and
    // sorts the bodies with the full radix sort; the captured step reuses the
    // plan and takes the previous step's order as its sort hint.
    BGV_TRY(run_fa2(1, K, nnz, off, adj, w, mass, p, pos, F, Fprev, speed, nullptr, nullptr, nullptr, hdr, scratch,
                    st, nullptr, true, G, koff));
    if (iterations == 1) return BGV_OK;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    BGV_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const unsigned long long before = launches_issued();
    int rc = run_fa2(1, K, nnz, off, adj, w, mass, p, pos, F, Fprev, speed, nullptr, nullptr, nullptr, hdr, scratch, st,
                     nullptr, false, G, koff, true);
    const unsigned long long per_step = launches_issued() - before;  // captured, not yet run
    cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (rc != BGV_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return rc != BGV_OK ? rc : BGV_ECUDA;
    }
    // the captured kernels keep the priorities of the streams they came from
    if (cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return BGV_ECUDA;
    }
    rc = BGV_OK;
    int32_t replays = 0;
    for (; replays < iterations - 1 && rc == BGV_OK; ++replays)
        if (cudaGraphLaunch(exec, st) != cudaSuccess) rc = BGV_ECUDA;
    add_launches(per_step * static_cast<unsigned long long>(replays) - per_step);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    return rc;
}

// Whole-graph CSR (ForceAtlas2 on the graph itself): the supergraph of the
// identity labelling is the graph with duplicate edges merged.
struct GraphCsrBuffers {
    int32_t *labels, *node_map;
    uint32_t *zero, *mass_tmp, *sw;
    int64_t *K_dev, *Es_dev;
    int32_t *ssrc, *sdst;
    SuperScratch super;
};

void carve_graph_csr(Carver &c, int64_t m, int32_t n, GraphCsrBuffers &b) {
    const size_t nn = size_t(n), mm = size_t(m > 0 ? m : 1);
    b.labels = c.take<int32_t>(nn);
    b.node_map = c.take<int32_t>(nn);
    b.zero = c.take<uint32_t>(nn);
    b.mass_tmp = c.take<uint32_t>(nn);
    b.K_dev = c.take<int64_t>(1);
    b.Es_dev = c.take<int64_t>(1);
    b.ssrc = c.take<int32_t>(mm);
    b.sdst = c.take<int32_t>(mm);
    b.sw = c.take<uint32_t>(mm);
    carve_super(c, m, n, 1, 1, b.super);
}

__global__ void k_identity_labels(int32_t n, int32_t *labels, uint32_t *zero) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        labels[v] = int32_t(v);
        zero[v] = 0u;
    }
}

// FA2 mass of a node of the whole graph: its degree (distinct neighbours)
// plus one.  Thread 0 also publishes nnz = csr_off[n].
__global__ void k_mass_from_degree(int32_t n, const int32_t *csr_off, uint32_t *mass, int64_t *nnz_dev) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x)
        mass[v] = uint32_t(csr_off[v + 1] - csr_off[v]) + 1u;
    if (blockIdx.x == 0 && threadIdx.x == 0) *nnz_dev = csr_off[n];
}

__global__ void k_radius(const uint32_t *mass, const int64_t *K_dev, float *radius) {
    const int64_t K = *K_dev;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < K; k += int64_t(gridDim.x) * blockDim.x)
        radius[k] = sqrtf(__uint2float_rn(mass[k]));
}

// First-round threshold from the mode of the sketched degrees (computed on
// the device, read back once).
int mode_threshold(const uint32_t *deg, int32_t n, uint32_t *mode_dev, void *scratch, uint32_t *status,
                   cudaStream_t st, uint32_t *D) {
    Carver c(scratch, 0);
    ModeScratch ms;
    carve_mode(c, n, 1, ms);
    BGV_TRY(run_mode_degree(deg, n, nullptr, mode_dev, ms, status, st));
    uint32_t h = 0;
    BGV_CUDA(cudaMemcpyAsync(&h, mode_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    BGV_CUDA(cudaStreamSynchronize(st));
    *D = h;
    return BGV_OK;
}

int layout_device(const int32_t *edges, int64_t m, int32_t n, const bgv_layout_params *p, int32_t *node_map,
                  float *xy, float *radius, int64_t *K_out, int64_t *Es_out, void *ws, cudaStream_t st,
                  LayoutBuffers &b) {
    WsHeader *hdr = header(ws);
    uint32_t *status = &hdr->status;
    const HashFamily h = make_hash_family(p->seed, p->rows, uint32_t(p->width));
    BGV_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), st));
    uint32_t D = p->threshold ? p->threshold : uint32_t((2 * m) / n);
    {
        Carver c(b.scratch, 0);
        SketchScratch s;
        carve_sketch(c, m, n, p->rows, p->width, s);
        BGV_TRY(run_sketch(edges, m, n, h, b.sketch, b.deg_est, s, status, st));
        if (!p->threshold && p->threshold_mode == 1) {
            // the most common degree of the graph (exact degrees, still in
            // the sketch's counters)
            ModeScratch ms;
            carve_mode(c, n, 1, ms);
            BGV_TRY(run_mode_degree(s.deg, n, nullptr, b.mode, ms, status, st));
            BGV_CUDA(cudaMemcpyAsync(&D, b.mode, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
            BGV_CUDA(cudaStreamSynchronize(st));
        }
    }
    {
        Carver c(b.scratch, 0);
        CommScratch s;
        carve_comm(c, m, n, s);
        BGV_TRY(run_communities(edges, m, n, b.deg_est, p->passes, D, p->growth, p->tie_mode, p->jumps, b.labels,
                                nullptr, s, status, st, nullptr, hdr));
    }
    {
        Carver c(b.scratch, 0);
        SuperScratch s;
        carve_super(c, m, n, p->rows, p->width, s);
        BGV_TRY(run_supergraph(edges, m, n, b.labels, b.deg_est, h, node_map, b.K_dev, b.ssrc, b.sdst, b.sw,
                               b.Es_dev, b.mass, b.csr_off, b.csr_adj, b.csr_w, nullptr, nullptr, nullptr, s, status,
                               st));
    }
    int64_t KE[2] = {0, 0};
    uint32_t dev_status = 0;
    BGV_CUDA(cudaMemcpyAsync(&KE[0], b.K_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    BGV_CUDA(cudaMemcpyAsync(&KE[1], b.Es_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    BGV_CUDA(cudaMemcpyAsync(&dev_status, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    BGV_CUDA(cudaStreamSynchronize(st));
    if (dev_status) return BGV_EDEVICE;
    const int64_t K = KE[0];
    if (K_out) *K_out = K;
    if (Es_out) *Es_out = KE[1];
    BGV_TRY(run_fa2_init(K, p->fa2, xy, b.Fprev, b.speed, st));
    BGV_TRY(fa2_loop(K, 2 * KE[1], b.csr_off, b.csr_adj, b.csr_w, b.mass, p->fa2, p->iterations, p->use_graph, xy, b.F,
                     b.Fprev, b.speed, hdr, b.scratch, st));
    if (radius) {
        note_launch(), k_radius<<<grid_for(K, 256, sm_count() * 8), 256, 0, st>>>(b.mass, b.K_dev, radius);
        BGV_TRY(launch_status());
    }
    return BGV_OK;
}

// ------------------------------------------------------------- batched form
// G independent graphs in one pass of every stage.  The caller's edge lists
// (local node ids, concatenated) are rewritten once into one id space in
// which graph g owns nodes [node_off[g], node_off[g+1]); every stage then
// runs over all graphs in the same launches and keeps them apart as
// BatchView describes.  Supernodes come out graph-major: graph g owns
// supernodes [K_off[g], K_off[g+1]) and superedges [Es_off[g], Es_off[g+1]).
struct BatchBuffers {
    int32_t *edges;        // [2m] global ids
    int32_t *node_off;     // [G + 1]
    int64_t *edge_off;     // [G + 1]
    int32_t *node_graph;   // [N]
    uint32_t *D0;          // [G]
    int64_t *koff;         // [G + 1] supernode offsets
    int64_t *Es_off;       // [G + 1] superedge offsets
    int32_t *node_map;     // [N] global supernode ids
};

void carve_batch(Carver &c, int64_t m, int32_t N, int32_t G, BatchBuffers &b) {
    const size_t gg = size_t(G) + 1;
    b.edges = c.take<int32_t>(2 * size_t(m > 0 ? m : 1));
    b.node_off = c.take<int32_t>(gg);
    b.edge_off = c.take<int64_t>(gg);
    b.node_graph = c.take<int32_t>(size_t(N));
    b.D0 = c.take<uint32_t>(gg);
    b.koff = c.take<int64_t>(gg);
    b.Es_off = c.take<int64_t>(gg);
    b.node_map = c.take<int32_t>(size_t(N));
}

// Largest g with off[g] <= x (off ascending, off[0] = 0 <= x).
template <class T>
__device__ __forceinline__ int32_t graph_of(const T *off, int32_t G, T x) {
    int32_t lo = 0, hi = G;  // off[lo] <= x < off[hi]
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= x) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_batch_nodes(int32_t N, int32_t G, const int32_t *node_off, int32_t *node_graph) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < N; v += int64_t(gridDim.x) * blockDim.x)
        node_graph[v] = graph_of(node_off, G, int32_t(v));
}

// Local -> global endpoint ids.  An endpoint outside its own graph becomes
// -1, which the stages report as BGV_DEV_BADEDGE.
__global__ void k_batch_edges(const int32_t *__restrict__ in, int64_t m, int32_t G, const int64_t *edge_off,
                              const int32_t *node_off, int32_t *__restrict__ out) {
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
        const int32_t g = graph_of(edge_off, G, e);
        const int32_t base = node_off[g], ng = node_off[g + 1] - base;
        const int2 uv = reinterpret_cast<const int2 *>(in)[e];
        const int32_t u = static_cast<uint32_t>(uv.x) < static_cast<uint32_t>(ng) ? uv.x + base : -1;
        const int32_t v = static_cast<uint32_t>(uv.y) < static_cast<uint32_t>(ng) ? uv.y + base : -1;
        reinterpret_cast<int2 *>(out)[e] = make_int2(u, v);
    }
}

// Supernode offsets (the dense rank of a graph's first node id, as labels
// are node ids of their own graph) and superedge offsets (superedges are
// sorted by source supernode).
__global__ void k_batch_offsets(int32_t G, const int32_t *node_off, const uint32_t *rank, const int64_t *K_dev,
                                const int32_t *ssrc, const int64_t *Es_dev, int64_t *koff, int64_t *Es_off) {
    const int64_t Es = *Es_dev;
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g <= G; g += gridDim.x * blockDim.x) {
        const int64_t k = g == G ? *K_dev : int64_t(rank[node_off[g]]);
        koff[g] = k;
        int64_t lo = 0, hi = Es;  // first superedge with source >= k
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (int64_t(ssrc[mid]) < k) lo = mid + 1; else hi = mid;
        }
        Es_off[g] = lo;
    }
}

__global__ void k_batch_local_map(int32_t N, const int32_t *node_map, const int32_t *node_graph, const int64_t *koff,
                                  int32_t *out) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < N; v += int64_t(gridDim.x) * blockDim.x)
        out[v] = int32_t(node_map[v] - koff[node_graph[v]]);
}

// Host-side check of the offsets; returns the totals.
int check_batch(int32_t G, const int64_t *edge_off, const int32_t *node_off, int64_t *m_out, int32_t *N_out) {
    if (G < 1 || G > (1 << 20) || !edge_off || !node_off) return BGV_EINVAL;
    if (edge_off[0] != 0 || node_off[0] != 0) return BGV_EINVAL;
    for (int32_t g = 0; g < G; ++g)
        if (node_off[g + 1] <= node_off[g] || edge_off[g + 1] < edge_off[g]) return BGV_EINVAL;
    if (node_off[G] >= 0x7FFFFFFF || edge_off[G] >= (int64_t(1) << 31)) return BGV_EINVAL;
    *m_out = edge_off[G];
    *N_out = node_off[G];
    return BGV_OK;
}

size_t layout_batched_ws(int64_t m, int32_t N, int32_t G, const bgv_layout_params *p) {
    Carver c(nullptr, kHeaderBytes);
    LayoutBuffers b;
    carve_layout(c, m, N, p, b, G);
    BatchBuffers bb;
    carve_batch(c, m, N, G, bb);
    return c.used();
}

int layout_batched_device(const int32_t *edges_local, const int64_t *edge_off, const int32_t *node_off, int32_t G,
                          int64_t m, int32_t N, const bgv_layout_params *p, int32_t *node_map, float *xy,
                          float *radius, int64_t *K_off, int64_t *Es_off, void *ws, cudaStream_t st) {
    Carver c(ws, kHeaderBytes);
    LayoutBuffers b;
    carve_layout(c, m, N, p, b, G);
    BatchBuffers bb;
    carve_batch(c, m, N, G, bb);
    WsHeader *hdr = header(ws);
    uint32_t *status = &hdr->status;
    const HashFamily h = make_hash_family(p->seed, p->rows, uint32_t(p->width));
    // first-round thresholds: the caller's, else floor(2 m_g / n_g) per graph
    uint32_t *D0 = static_cast<uint32_t *>(malloc(sizeof(uint32_t) * size_t(G)));
    if (!D0) return BGV_EINVAL;
    for (int32_t g = 0; g < G; ++g)
        D0[g] = p->threshold ? p->threshold
                             : uint32_t((2 * (edge_off[g + 1] - edge_off[g])) / (node_off[g + 1] - node_off[g]));
    cudaError_t ce = cudaMemcpyAsync(bb.D0, D0, sizeof(uint32_t) * size_t(G), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);  // D0 is freed next
    free(D0);
    BGV_CUDA(ce);
    BGV_CUDA(cudaMemcpyAsync(bb.node_off, node_off, sizeof(int32_t) * (size_t(G) + 1), cudaMemcpyHostToDevice, st));
    BGV_CUDA(cudaMemcpyAsync(bb.edge_off, edge_off, sizeof(int64_t) * (size_t(G) + 1), cudaMemcpyHostToDevice, st));
    BGV_CUDA(cudaMemsetAsync(status, 0, sizeof(uint32_t), st));
    note_launch(), k_batch_nodes<<<grid_for(N, 256, sm_count() * 8), 256, 0, st>>>(N, G, bb.node_off, bb.node_graph);
    BGV_TRY(launch_status());
    if (m > 0) {
        note_launch(), k_batch_edges<<<grid_for(m, 256, sm_count() * 16), 256, 0, st>>>(edges_local, m, G, bb.edge_off,
                                                                                  bb.node_off, bb.edges);
        BGV_TRY(launch_status());
    }
    const BatchView view{G, bb.node_off, bb.node_graph, bb.D0};
    {
        Carver sc(b.scratch, 0);
        SketchScratch s;
        carve_sketch(sc, m, N, p->rows, p->width, s);
        BGV_TRY(run_sketch(bb.edges, m, N, h, b.sketch, b.deg_est, s, status, st, &view));
        if (!p->threshold && p->threshold_mode == 1) {
            // each graph's most common degree, straight into D0
            ModeScratch ms;
            carve_mode(sc, N, G, ms);
            BGV_TRY(run_mode_degree(s.deg, N, &view, bb.D0, ms, status, st));
        }
    }
    {
        Carver sc(b.scratch, 0);
        CommScratch s;
        carve_comm(sc, m, N, s, true);
        BGV_TRY(run_communities(bb.edges, m, N, b.deg_est, p->passes, 0, p->growth, p->tie_mode, p->jumps, b.labels,
                                nullptr, s, status, st, &view, hdr));
    }
    {
        Carver sc(b.scratch, 0);
        SuperScratch s;
        carve_super(sc, m, N, p->rows, p->width, s, G);
        BGV_TRY(run_supergraph(bb.edges, m, N, b.labels, b.deg_est, h, bb.node_map, b.K_dev, b.ssrc, b.sdst, b.sw,
                               b.Es_dev, b.mass, b.csr_off, b.csr_adj, b.csr_w, nullptr, nullptr, nullptr, s, status,
                               st, &view));
        note_launch(), k_batch_offsets<<<grid_for(int64_t(G) + 1, 256, sm_count()), 256, 0, st>>>(
            G, bb.node_off, s.rank, b.K_dev, b.ssrc, b.Es_dev, bb.koff, bb.Es_off);
        BGV_TRY(launch_status());
    }
    note_launch(), k_batch_local_map<<<grid_for(N, 256, sm_count() * 8), 256, 0, st>>>(N, bb.node_map, bb.node_graph,
                                                                                  bb.koff, node_map);
    BGV_TRY(launch_status());
    uint32_t dev_status = 0;
    BGV_CUDA(cudaMemcpyAsync(K_off, bb.koff, sizeof(int64_t) * (size_t(G) + 1), cudaMemcpyDeviceToHost, st));
    BGV_CUDA(cudaMemcpyAsync(Es_off, bb.Es_off, sizeof(int64_t) * (size_t(G) + 1), cudaMemcpyDeviceToHost, st));
    BGV_CUDA(cudaMemcpyAsync(&dev_status, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    BGV_CUDA(cudaStreamSynchronize(st));
    if (dev_status) return BGV_EDEVICE;
    const int64_t K = K_off[G], Es = Es_off[G];
    BGV_TRY(run_fa2_init(K, p->fa2, xy, b.Fprev, b.speed, st, G, bb.koff));
    BGV_TRY(fa2_loop(K, 2 * Es, b.csr_off, b.csr_adj, b.csr_w, b.mass, p->fa2, p->iterations, p->use_graph, xy, b.F,
                     b.Fprev, b.speed, hdr, b.scratch, st, G, bb.koff));
    if (radius) {
        note_launch(), k_radius<<<grid_for(K, 256, sm_count() * 8), 256, 0, st>>>(b.mass, b.K_dev, radius);
        BGV_TRY(launch_status());
    }
    return BGV_OK;
}

// Batched FA2 on caller supergraphs: the graph offsets are validated on the
// host and copied into the workspace, right after the header.
size_t fa2_batched_ws(int64_t K, int64_t nnz, int32_t G) {
    Carver c(nullptr, kHeaderBytes);
    c.take<int64_t>(size_t(G) + 1);
    c.take<char>(fa2_scratch_bytes(K, nnz, G));
    return c.used();
}

int check_koff(int32_t G, const int64_t *koff, int64_t K, int max_depth) {
    if (G < 1 || G > (1 << 20) || !koff || koff[0] != 0 || koff[G] != K) return BGV_EINVAL;
    if (!fa2_batch_fits(G, max_depth)) return BGV_EINVAL;
    for (int32_t g = 0; g < G; ++g)
        if (koff[g + 1] <= koff[g]) return BGV_EINVAL;
    return BGV_OK;
}

int fa2_batched_setup(int32_t G, const int64_t *koff, int64_t K, int max_depth, void *ws, cudaStream_t st,
                      int64_t **dkoff, char **scratch) {
    BGV_TRY(check_koff(G, koff, K, max_depth));
    Carver c(ws, kHeaderBytes);
    *dkoff = c.take<int64_t>(size_t(G) + 1);
    *scratch = c.take<char>(0);
    BGV_CUDA(cudaMemcpyAsync(*dkoff, koff, sizeof(int64_t) * (size_t(G) + 1), cudaMemcpyHostToDevice, st));
    return BGV_OK;
}

}  // namespace

extern "C" {

int bgv_version(void) { return (0 << 16) | 1; }

const char *bgv_strerror(int code) {
    switch (code) {
        case BGV_OK: return "ok";
        case BGV_EINVAL: return "invalid argument";
        case BGV_ENOSPC: return "workspace too small";
        case BGV_EDEVICE: return "device reported an error (see the status word)";
        case BGV_ECUDA: return "CUDA error";
        case BGV_ELIMIT: return "size exceeds the fixed scratch of a no-allocation entry point";
        default: return "unknown error";
    }
}

int bgv_ws_init(void *ws, void *stream) {
    if (!ws || !aligned(ws, kAlign)) return BGV_EINVAL;
    BGV_CUDA(cudaMemsetAsync(ws, 0, kHeaderBytes, as_stream(stream)));
    return BGV_OK;
}

int bgv_status(void *ws, void *stream, uint32_t *out, int clear) {
    if (!ws || !out) return BGV_EINVAL;
    cudaStream_t st = as_stream(stream);
    BGV_CUDA(cudaMemcpyAsync(out, status_ptr(ws), sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    if (clear) BGV_CUDA(cudaMemsetAsync(status_ptr(ws), 0, sizeof(uint32_t), st));
    BGV_CUDA(cudaStreamSynchronize(st));
    return BGV_OK;
}

size_t bgv_sketch_degrees_ws_size(int64_t m, int32_t n, int32_t rows, int32_t width) {
    return sketch_ws(m, n, rows, width);
}

int bgv_sketch_degrees(const int32_t *edges, int64_t m, int32_t n, int32_t rows, int32_t width, uint64_t seed,
                       uint32_t *sketch, uint32_t *deg_est, void *ws, size_t ws_bytes, void *stream) {
    BGV_TRY(check_graph(edges, m, n));
    BGV_TRY(check_sketch_shape(rows, width));
    if (!sketch || !deg_est) return BGV_EINVAL;
    BGV_TRY(check_ws(ws, ws_bytes, sketch_ws(m, n, rows, width)));
    Carver c(ws, kHeaderBytes);
    SketchScratch s;
    carve_sketch(c, m, n, rows, width, s);
    const HashFamily h = make_hash_family(seed, rows, uint32_t(width));
    return run_sketch(edges, m, n, h, sketch, deg_est, s, status_ptr(ws), as_stream(stream));
}

size_t bgv_communities_ws_size(int64_t m, int32_t n) { return comm_ws(m, n); }

int bgv_communities(const int32_t *edges, int64_t m, int32_t n, const uint32_t *deg_est, int32_t passes,
                    uint32_t threshold, uint32_t growth, int32_t tie_mode, int32_t *labels, uint32_t *deg_out,
                    void *ws, size_t ws_bytes, void *stream) {
    BGV_TRY(check_graph(edges, m, n));
    if (!deg_est || !labels || passes < 0 || (tie_mode != 0 && tie_mode != 1)) return BGV_EINVAL;
    BGV_TRY(check_ws(ws, ws_bytes, comm_ws(m, n)));
    Carver c(ws, kHeaderBytes);
    CommScratch s;
    carve_comm(c, m, n, s);
    const uint32_t D = threshold ? threshold : uint32_t((2 * m) / n);
    return run_communities(edges, m, n, deg_est, passes, D, growth, tie_mode, 0, labels, deg_out, s, status_ptr(ws),
                           as_stream(stream), nullptr, header(ws));
}

size_t bgv_communities_ex_ws_size(int64_t m, int32_t n) {
    size_t comm = 0, mode = 0;
    {
        Carver c(nullptr, 0);
        CommScratch s;
        carve_comm(c, m, n, s);
        comm = c.used();
    }
    {
        Carver c(nullptr, 0);
        ModeScratch s;
        carve_mode(c, n, 1, s);
        mode = c.used();
    }
    Carver c(nullptr, kHeaderBytes);
    c.take<uint32_t>(1);
    c.take<char>(comm > mode ? comm : mode);
    return c.used();
}

int bgv_communities_ex(const int32_t *edges, int64_t m, int32_t n, const uint32_t *deg_est, int32_t passes,
                       uint32_t threshold, uint32_t growth, int32_t tie_mode, int32_t threshold_mode, int32_t jumps,
                       int32_t *labels, uint32_t *deg_out, uint32_t *threshold_out, void *ws, size_t ws_bytes,
                       void *stream) {
    BGV_TRY(check_graph(edges, m, n));
    if (!deg_est || !labels || passes < 0 || (tie_mode != 0 && tie_mode != 1)) return BGV_EINVAL;
    if ((threshold_mode != 0 && threshold_mode != 1) || jumps < 0 || jumps > 64) return BGV_EINVAL;
    BGV_TRY(check_ws(ws, ws_bytes, bgv_communities_ex_ws_size(m, n)));
    cudaStream_t st = as_stream(stream);
    Carver c(ws, kHeaderBytes);
    uint32_t *mode_dev = c.take<uint32_t>(1);
    char *region = c.take<char>(0);
    uint32_t D = threshold ? threshold : uint32_t((2 * m) / n);
    if (!threshold && threshold_mode == 1) BGV_TRY(mode_threshold(deg_est, n, mode_dev, region, status_ptr(ws), st, &D));
    if (threshold_out) *threshold_out = D;
    Carver rc(region, 0);
    CommScratch s;
    carve_comm(rc, m, n, s);
    return run_communities(edges, m, n, deg_est, passes, D, growth, tie_mode, jumps, labels, deg_out, s,
                           status_ptr(ws), st, nullptr, header(ws));
}

size_t bgv_mode_degree_ws_size(int32_t n) {
    Carver c(nullptr, kHeaderBytes);
    c.take<uint32_t>(1);
    ModeScratch s;
    carve_mode(c, n, 1, s);
    return c.used();
}

int bgv_mode_degree(const uint32_t *deg, int32_t n, uint32_t *mode_out, void *ws, size_t ws_bytes, void *stream) {
    if (n < 1 || n >= 0x7FFFFFFF || !deg || !mode_out) return BGV_EINVAL;
    BGV_TRY(check_ws(ws, ws_bytes, bgv_mode_degree_ws_size(n)));
    Carver c(ws, kHeaderBytes);
    uint32_t *mode_dev = c.take<uint32_t>(1);
    char *region = c.take<char>(0);
    return mode_threshold(deg, n, mode_dev, region, status_ptr(ws), as_stream(stream), mode_out);
}

size_t bgv_supergraph_ws_size(int64_t m, int32_t n, int32_t rows, int32_t width) {
    return super_ws(m, n, rows, width);
}

int bgv_supergraph(const int32_t *edges, int64_t m, int32_t n, const int32_t *labels, const uint32_t *deg_est,
                   int32_t rows, int32_t width, uint64_t seed, int32_t *node_map, int64_t *K_dev, int32_t *ssrc,
                   int32_t *sdst, uint32_t *sw, int64_t *Es_dev, uint32_t *mass, int32_t *csr_off, int32_t *csr_adj,
                   uint32_t *csr_w, uint64_t *vol, uint32_t *count, int32_t *comm_label, void *ws, size_t ws_bytes,
                   void *stream) {
    BGV_TRY(check_graph(edges, m, n));
    BGV_TRY(check_sketch_shape(rows, width));
    if (!labels || !deg_est || !node_map || !K_dev || !ssrc || !sdst || !sw || !Es_dev || !mass || !csr_off ||
        !csr_adj || !csr_w)
        return BGV_EINVAL;
    BGV_TRY(check_ws(ws, ws_bytes, super_ws(m, n, rows, width)));
    Carver c(ws, kHeaderBytes);
    SuperScratch s;
    carve_super(c, m, n, rows, width, s);
    const HashFamily h = make_hash_family(seed, rows, uint32_t(width));
    return run_supergraph(edges, m, n, labels, deg_est, h, node_map, K_dev, ssrc, sdst, sw, Es_dev, mass, csr_off,
                          csr_adj, csr_w, vol, count, comm_label, s, status_ptr(ws), as_stream(stream));
}

size_t bgv_graph_csr_ws_size(int64_t m, int32_t n) {
    Carver c(nullptr, kHeaderBytes);
    GraphCsrBuffers b;
    carve_graph_csr(c, m, n, b);
    return c.used();
}

int bgv_graph_csr(const int32_t *edges, int64_t m, int32_t n, int32_t *csr_off, int32_t *csr_adj, uint32_t *csr_w,
                  uint32_t *mass, int64_t *nnz_dev, void *ws, size_t ws_bytes, void *stream) {
    BGV_TRY(check_graph(edges, m, n));
    if (!csr_off || !csr_adj || !csr_w || !mass || !nnz_dev) return BGV_EINVAL;
    BGV_TRY(check_ws(ws, ws_bytes, bgv_graph_csr_ws_size(m, n)));
    Carver c(ws, kHeaderBytes);
    GraphCsrBuffers b;
    carve_graph_csr(c, m, n, b);
    cudaStream_t st = as_stream(stream);
    note_launch(), k_identity_labels<<<grid_for(n, 256, sm_count() * 8), 256, 0, st>>>(n, b.labels, b.zero);
    BGV_TRY(launch_status());
    const HashFamily h = make_hash_family(1, 1, 1);
    BGV_TRY(run_supergraph(edges, m, n, b.labels, b.zero, h, b.node_map, b.K_dev, b.ssrc, b.sdst, b.sw, b.Es_dev,
                           b.mass_tmp, csr_off, csr_adj, csr_w, nullptr, nullptr, nullptr, b.super, status_ptr(ws), st));
    note_launch(), k_mass_from_degree<<<grid_for(n, 256, sm_count() * 8), 256, 0, st>>>(n, csr_off, mass, nnz_dev);
    return launch_status();
}

void bgv_fa2_default_params(bgv_fa2_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->theta = 1.2f;
    p->kr = 2.0f;
    p->kg = 1.0f;
    p->tau = 1.0f;
    p->ks = 0.1f;
    p->ksmax = 10.0f;
    p->strong_gravity = 0;
    p->leaf_cap = 1;
    p->max_depth = 24;
    p->seed = 1;
}

int bgv_fa2_init(int64_t K, const bgv_fa2_params *p, float *pos, float *Fprev, double *speed, void *stream) {
    if (K < 0 || K >= 0x7FFFFFFF || !speed || (K > 0 && (!pos || !Fprev))) return BGV_EINVAL;
    BGV_TRY(fa2_check_params(p));
    return run_fa2_init(K, *p, pos, Fprev, speed, as_stream(stream));
}

size_t bgv_fa2_ws_size(int64_t K, int64_t nnz) { return kHeaderBytes + fa2_scratch_bytes(K, nnz); }

static int check_fa2_inputs(int64_t K, int64_t nnz, const int32_t *off, const int32_t *adj, const uint32_t *w,
                            const uint32_t *mass, const bgv_fa2_params *p, const float *pos) {
    if (K < 0 || K >= 0x7FFFFFFF || nnz < 0 || nnz >= (int64_t(1) << 31)) return BGV_EINVAL;
    BGV_TRY(fa2_check_params(p));
    if (K == 0) return BGV_OK;
    if (!off || !adj || !w || !mass || !pos || !aligned(pos, 8)) return BGV_EINVAL;
    return BGV_OK;
}

static int check_fa2_args(int64_t K, int64_t nnz, const int32_t *off, const int32_t *adj, const uint32_t *w,
                          const uint32_t *mass, const bgv_fa2_params *p, const float *pos, void *ws,
                          size_t ws_bytes) {
    BGV_TRY(check_fa2_inputs(K, nnz, off, adj, w, mass, p, pos));
    if (K == 0) return BGV_OK;
    return check_ws(ws, ws_bytes, bgv_fa2_ws_size(K, nnz));
}

int bgv_fa2_forces(int64_t K, int64_t nnz, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
                   const uint32_t *mass, const bgv_fa2_params *p, const float *pos, float *Fr, float *Fa, float *Fg,
                   void *ws, size_t ws_bytes, void *stream) {
    BGV_TRY(check_fa2_args(K, nnz, csr_off, csr_adj, csr_w, mass, p, pos, ws, ws_bytes));
    if (K == 0) return BGV_OK;
    return run_fa2(0, K, nnz, csr_off, csr_adj, csr_w, mass, *p, const_cast<float *>(pos), nullptr, nullptr, nullptr, Fr,
                   Fa, Fg, header(ws), static_cast<char *>(ws) + kHeaderBytes, as_stream(stream));
}

int bgv_fa2_step(int64_t K, int64_t nnz, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
                 const uint32_t *mass, const bgv_fa2_params *p, float *pos, float *F, float *Fprev, double *speed,
                 void *ws, size_t ws_bytes, void *stream) {
    BGV_TRY(check_fa2_args(K, nnz, csr_off, csr_adj, csr_w, mass, p, pos, ws, ws_bytes));
    if (K == 0) return BGV_OK;
    if (!F || !Fprev || !speed) return BGV_EINVAL;
    return run_fa2(1, K, nnz, csr_off, csr_adj, csr_w, mass, *p, pos, F, Fprev, speed, nullptr, nullptr, nullptr,
                   header(ws), static_cast<char *>(ws) + kHeaderBytes, as_stream(stream));
}

int bgv_fa2_run(int64_t K, int64_t nnz, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
                const uint32_t *mass, const bgv_fa2_params *p, int32_t iterations, int32_t use_graph, float *pos,
                float *F, float *Fprev, double *speed, void *ws, size_t ws_bytes, void *stream) {
    BGV_TRY(check_fa2_args(K, nnz, csr_off, csr_adj, csr_w, mass, p, pos, ws, ws_bytes));
    if (K == 0 || iterations <= 0) return iterations < 0 ? BGV_EINVAL : BGV_OK;
    if (!F || !Fprev || !speed) return BGV_EINVAL;
    return fa2_loop(K, nnz, csr_off, csr_adj, csr_w, mass, *p, iterations, use_graph, pos, F, Fprev, speed, header(ws),
                    static_cast<char *>(ws) + kHeaderBytes, as_stream(stream));
}

int bgv_fa2_run_timed(int64_t K, int64_t nnz, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
                      const uint32_t *mass, const bgv_fa2_params *p, int32_t iterations, float *pos, float *F,
                      float *Fprev, double *speed, void *ws, size_t ws_bytes, void *stream, float *stage_ms) {
    BGV_TRY(check_fa2_args(K, nnz, csr_off, csr_adj, csr_w, mass, p, pos, ws, ws_bytes));
    if (iterations < 0 || !stage_ms) return BGV_EINVAL;
    for (int i = 0; i < BGV_FA2_STAGES; ++i) stage_ms[i] = 0.0f;
    if (K == 0 || iterations == 0) return BGV_OK;
    if (!F || !Fprev || !speed) return BGV_EINVAL;
    cudaStream_t st = as_stream(stream);
    const int per = kFa2Stages + 1;
    const size_t nev = size_t(iterations) * per;
    cudaEvent_t *ev = static_cast<cudaEvent_t *>(calloc(nev, sizeof(cudaEvent_t)));
    if (!ev) return BGV_EINVAL;
    int rc = BGV_OK;
    size_t made = 0;
    for (; made < nev; ++made)
        if (cudaEventCreate(&ev[made]) != cudaSuccess) {
            rc = BGV_ECUDA;
            break;
        }
    for (int32_t t = 0; t < iterations && rc == BGV_OK; ++t)
        rc = run_fa2(1, K, nnz, csr_off, csr_adj, csr_w, mass, *p, pos, F, Fprev, speed, nullptr, nullptr, nullptr,
                     header(ws), static_cast<char *>(ws) + kHeaderBytes, st, ev + size_t(t) * per, t == 0, 1, nullptr,
                     t > 0);
    if (rc == BGV_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = BGV_ECUDA;
    for (int32_t t = 0; t < iterations && rc == BGV_OK; ++t)
        for (int k = 0; k < kFa2Stages; ++k) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, ev[size_t(t) * per + k], ev[size_t(t) * per + k + 1]) != cudaSuccess) {
                rc = BGV_ECUDA;
                break;
            }
            stage_ms[k] += ms;
        }
    for (size_t i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
    free(ev);
    return rc;
}

uint64_t bgv_launch_count(void) { return launches_issued(); }

int bgv_fa2_read_stats(void *ws, void *stream, bgv_fa2_stats *out) {
    if (!ws || !out) return BGV_EINVAL;
    WsHeader h;
    cudaStream_t st = as_stream(stream);
    BGV_CUDA(cudaMemcpyAsync(&h, ws, sizeof(WsHeader), cudaMemcpyDeviceToHost, st));
    BGV_CUDA(cudaStreamSynchronize(st));
    out->S = h.S;
    out->T = h.T;
    out->interactions = h.interactions;
    out->tree_nodes = h.tree_nodes;
    out->interactions_total = h.interactions_total;
    out->steps_total = h.steps_total;
    out->status = h.status;
    out->reserved = 0;
    return BGV_OK;
}

void bgv_layout_default_params(bgv_layout_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->rows = 4;
    p->width = 4096;
    p->seed = 1;
    p->passes = 3;
    p->threshold = 0;
    p->growth = 2;
    p->threshold_mode = 0;
    p->jumps = 0;
    p->tie_mode = 0;
    p->iterations = 200;
    p->use_graph = 1;
    bgv_fa2_default_params(&p->fa2);
}

size_t bgv_layout_ws_size(int64_t m, int32_t n, const bgv_layout_params *p) {
    if (check_layout_params(p) != BGV_OK || n < 1 || m < 0) return 0;
    Carver c(nullptr, kHeaderBytes);
    LayoutBuffers b;
    carve_layout(c, m, n, p, b);
    return c.used();
}

int bgv_layout(const int32_t *edges, int64_t m, int32_t n, const bgv_layout_params *p, int32_t *node_map, float *xy,
               float *radius, int64_t *K_out, int64_t *Es_out, void *ws, size_t ws_bytes, void *stream) {
    BGV_TRY(check_graph(edges, m, n));
    BGV_TRY(check_layout_params(p));
    if (!node_map || !xy || !aligned(xy, 8)) return BGV_EINVAL;
    BGV_TRY(check_ws(ws, ws_bytes, bgv_layout_ws_size(m, n, p)));
    Carver c(ws, kHeaderBytes);
    LayoutBuffers b;
    carve_layout(c, m, n, p, b);
    cudaStream_t st = as_stream(stream);
    BGV_TRY(layout_device(edges, m, n, p, node_map, xy, radius, K_out, Es_out, ws, st, b));
    uint32_t dev_status = 0;
    BGV_CUDA(cudaMemcpyAsync(&dev_status, status_ptr(ws), sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    BGV_CUDA(cudaStreamSynchronize(st));
    return dev_status ? BGV_EDEVICE : BGV_OK;
}

size_t bgv_layout_host_ws_size(int64_t m, int32_t n, const bgv_layout_params *p) {
    size_t base = bgv_layout_ws_size(m, n, p);
    if (!base) return 0;
    Carver c(nullptr, base);
    c.take<int32_t>(size_t(2 * (m > 0 ? m : 1)));
    c.take<int32_t>(size_t(n));
    c.take<float>(size_t(2) * size_t(n));
    c.take<float>(size_t(n));
    return c.used();
}

int bgv_layout_host(const int32_t *h_edges, int64_t m, int32_t n, const bgv_layout_params *p, int32_t *h_node_map,
                    float *h_xy, float *h_radius, int64_t *K_out, int64_t *Es_out, void *ws, size_t ws_bytes,
                    void *stream) {
    if (n < 1 || m < 0 || (m > 0 && !h_edges) || !h_node_map || !h_xy) return BGV_EINVAL;
    BGV_TRY(check_layout_params(p));
    BGV_TRY(check_ws(ws, ws_bytes, bgv_layout_host_ws_size(m, n, p)));
    cudaStream_t st = as_stream(stream);
    const size_t base = bgv_layout_ws_size(m, n, p);
    Carver io(ws, base);
    int32_t *d_edges = io.take<int32_t>(size_t(2 * (m > 0 ? m : 1)));
    int32_t *d_map = io.take<int32_t>(size_t(n));
    float *d_xy = io.take<float>(size_t(2) * size_t(n));
    float *d_rad = io.take<float>(size_t(n));
    if (m > 0) BGV_CUDA(cudaMemcpyAsync(d_edges, h_edges, sizeof(int32_t) * 2 * size_t(m), cudaMemcpyHostToDevice, st));
    Carver c(ws, kHeaderBytes);
    LayoutBuffers b;
    carve_layout(c, m, n, p, b);
    int64_t K = 0, Es = 0;
    BGV_TRY(layout_device(d_edges, m, n, p, d_map, d_xy, d_rad, &K, &Es, ws, st, b));
    BGV_CUDA(cudaMemcpyAsync(h_node_map, d_map, sizeof(int32_t) * size_t(n), cudaMemcpyDeviceToHost, st));
    if (K > 0) {
        BGV_CUDA(cudaMemcpyAsync(h_xy, d_xy, sizeof(float) * 2 * size_t(K), cudaMemcpyDeviceToHost, st));
        if (h_radius) BGV_CUDA(cudaMemcpyAsync(h_radius, d_rad, sizeof(float) * size_t(K), cudaMemcpyDeviceToHost, st));
    }
    uint32_t dev_status = 0;
    BGV_CUDA(cudaMemcpyAsync(&dev_status, status_ptr(ws), sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    BGV_CUDA(cudaStreamSynchronize(st));
    if (K_out) *K_out = K;
    if (Es_out) *Es_out = Es;
    return dev_status ? BGV_EDEVICE : BGV_OK;
}

size_t bgv_layout_batched_ws_size(int32_t G, const int64_t *edge_off, const int32_t *node_off,
                                  const bgv_layout_params *p) {
    int64_t m = 0;
    int32_t N = 0;
    if (check_layout_params(p) != BGV_OK || check_batch(G, edge_off, node_off, &m, &N) != BGV_OK) return 0;
    return layout_batched_ws(m, N, G, p);
}

int bgv_layout_batched(const int32_t *edges, int32_t G, const int64_t *edge_off, const int32_t *node_off,
                       const bgv_layout_params *p, int32_t *node_map, float *xy, float *radius, int64_t *K_off,
                       int64_t *Es_off, void *ws, size_t ws_bytes, void *stream) {
    int64_t m = 0;
    int32_t N = 0;
    BGV_TRY(check_batch(G, edge_off, node_off, &m, &N));
    BGV_TRY(check_layout_params(p));
    if (!fa2_batch_fits(G, p->fa2.max_depth)) return BGV_EINVAL;
    if ((m > 0 && (!edges || !aligned(edges, 8))) || !node_map || !xy || !aligned(xy, 8) || !K_off || !Es_off)
        return BGV_EINVAL;
    BGV_TRY(check_ws(ws, ws_bytes, layout_batched_ws(m, N, G, p)));
    cudaStream_t st = as_stream(stream);
    BGV_TRY(layout_batched_device(edges, edge_off, node_off, G, m, N, p, node_map, xy, radius, K_off, Es_off, ws, st));
    uint32_t dev_status = 0;
    BGV_CUDA(cudaMemcpyAsync(&dev_status, status_ptr(ws), sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    BGV_CUDA(cudaStreamSynchronize(st));
    return dev_status ? BGV_EDEVICE : BGV_OK;
}

size_t bgv_fa2_ws_size_batched(int32_t G, int64_t K, int64_t nnz) {
    if (G < 1 || G > (1 << 20)) return 0;
    return fa2_batched_ws(K, nnz, G);
}

int bgv_fa2_init_batched(int32_t G, const int64_t *koff, const bgv_fa2_params *p, float *pos, float *Fprev,
                         double *speed, void *ws, size_t ws_bytes, void *stream) {
    if (!koff || G < 1 || G > (1 << 20)) return BGV_EINVAL;
    const int64_t K = koff[G];
    if (K >= 0x7FFFFFFF || !pos || !Fprev || !speed || !aligned(pos, 8)) return BGV_EINVAL;
    BGV_TRY(fa2_check_params(p));
    BGV_TRY(check_ws(ws, ws_bytes, fa2_batched_ws(K, 0, G)));
    cudaStream_t st = as_stream(stream);
    int64_t *dkoff = nullptr;
    char *scratch = nullptr;
    BGV_TRY(fa2_batched_setup(G, koff, K, p->max_depth, ws, st, &dkoff, &scratch));
    return run_fa2_init(K, *p, pos, Fprev, speed, st, G, dkoff);
}

int bgv_fa2_forces_batched(int32_t G, const int64_t *koff, int64_t nnz, const int32_t *csr_off,
                           const int32_t *csr_adj, const uint32_t *csr_w, const uint32_t *mass,
                           const bgv_fa2_params *p, const float *pos, float *Fr, float *Fa, float *Fg, void *ws,
                           size_t ws_bytes, void *stream) {
    if (!koff || G < 1 || G > (1 << 20)) return BGV_EINVAL;
    const int64_t K = koff[G];
    BGV_TRY(check_fa2_inputs(K, nnz, csr_off, csr_adj, csr_w, mass, p, pos));
    BGV_TRY(check_ws(ws, ws_bytes, fa2_batched_ws(K, nnz, G)));
    cudaStream_t st = as_stream(stream);
    int64_t *dkoff = nullptr;
    char *scratch = nullptr;
    BGV_TRY(fa2_batched_setup(G, koff, K, p->max_depth, ws, st, &dkoff, &scratch));
    return run_fa2(0, K, nnz, csr_off, csr_adj, csr_w, mass, *p, const_cast<float *>(pos), nullptr, nullptr, nullptr,
                   Fr, Fa, Fg, header(ws), scratch, st, nullptr, true, G, dkoff);
}

int bgv_fa2_run_batched(int32_t G, const int64_t *koff, int64_t nnz, const int32_t *csr_off, const int32_t *csr_adj,
                        const uint32_t *csr_w, const uint32_t *mass, const bgv_fa2_params *p, int32_t iterations,
                        int32_t use_graph, float *pos, float *F, float *Fprev, double *speed, void *ws,
                        size_t ws_bytes, void *stream) {
    if (!koff || G < 1 || G > (1 << 20) || iterations < 0) return BGV_EINVAL;
    const int64_t K = koff[G];
    BGV_TRY(check_fa2_inputs(K, nnz, csr_off, csr_adj, csr_w, mass, p, pos));
    if (!F || !Fprev || !speed) return BGV_EINVAL;
    BGV_TRY(check_ws(ws, ws_bytes, fa2_batched_ws(K, nnz, G)));
    cudaStream_t st = as_stream(stream);
    int64_t *dkoff = nullptr;
    char *scratch = nullptr;
    BGV_TRY(fa2_batched_setup(G, koff, K, p->max_depth, ws, st, &dkoff, &scratch));
    return fa2_loop(K, nnz, csr_off, csr_adj, csr_w, mass, *p, iterations, use_graph, pos, F, Fprev, speed,
                    header(ws), scratch, st, G, dkoff);
}

size_t bgv_autotune_fa2_ws_size(int64_t K, int64_t nnz) {
    Carver c(nullptr, kHeaderBytes);
    const size_t k = size_t(K > 0 ? K : 1);
    c.take<float>(2 * k);  // positions
    c.take<float>(2 * k);  // F
    c.take<float>(2 * k);  // Fprev
    c.take<double>(1);     // speed
    c.take<char>(fa2_scratch_bytes(K, nnz));
    return c.used();
}

int bgv_set_fa2_tune(int32_t att_short, int32_t repulse_threads, int32_t tail_blocks_per_sm) {
    return set_fa2_tune(Fa2Tune{att_short, repulse_threads, tail_blocks_per_sm});
}

int bgv_autotune_fa2(int64_t K, int64_t nnz, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
                     const uint32_t *mass, const bgv_fa2_params *p, const float *pos, bgv_fa2_tune_report *out,
                     void *ws, size_t ws_bytes, void *stream) {
    if (K < 1 || K >= 0x7FFFFFFF || nnz < 0 || !csr_off || !mass || !pos || (nnz > 0 && (!csr_adj || !csr_w)))
        return BGV_EINVAL;
    BGV_TRY(fa2_check_params(p));
    BGV_TRY(check_ws(ws, ws_bytes, bgv_autotune_fa2_ws_size(K, nnz)));
    cudaStream_t st = as_stream(stream);
    Carver c(ws, kHeaderBytes);
    const size_t k = size_t(K);
    float *P = c.take<float>(2 * k), *F = c.take<float>(2 * k), *Fprev = c.take<float>(2 * k);
    double *speed = c.take<double>(1);
    void *scratch = c.take<char>(0);
    WsHeader *hdr = header(ws);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BGV_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return BGV_ECUDA;
    }
    const double one = 1.0;
    // median of three timed steps (after one warm-up step that builds the
    // attraction plan) from the caller's positions
    auto time_steps = [&](float *ms) -> int {
        BGV_CUDA(cudaMemcpyAsync(P, pos, sizeof(float) * 2 * k, cudaMemcpyDeviceToDevice, st));
        BGV_CUDA(cudaMemsetAsync(Fprev, 0, sizeof(float) * 2 * k, st));
        BGV_CUDA(cudaMemcpyAsync(speed, &one, sizeof(double), cudaMemcpyHostToDevice, st));
        float t[3];
        for (int r = 0; r < 4; ++r) {
            BGV_CUDA(cudaEventRecord(e0, st));
            BGV_TRY(run_fa2(1, K, nnz, csr_off, csr_adj, csr_w, mass, *p, P, F, Fprev, speed, nullptr, nullptr,
                            nullptr, hdr, scratch, st, nullptr, r == 0));
            BGV_CUDA(cudaEventRecord(e1, st));
            BGV_CUDA(cudaEventSynchronize(e1));
            float x = 0.0f;
            BGV_CUDA(cudaEventElapsedTime(&x, e0, e1));
            if (r > 0) t[r - 1] = x;
        }
        std::sort(t, t + 3);
        *ms = t[1];
        return BGV_OK;
    };
    bgv_fa2_tune_report r;
    memset(&r, 0, sizeof(r));
    Fa2Tune best = fa2_tune();
    const int shorts[3] = {8, 16, 32}, threads[2] = {128, 256}, tails[3] = {2, 4, 8};
    int rc = BGV_OK;
    float best_ms = 0.0f;
    for (int i = 0; i < 3 && rc == BGV_OK; ++i) {
        Fa2Tune t = best;
        t.att_short = shorts[i];
        set_fa2_tune(t);
        rc = time_steps(&r.ms_att_short[i]);
        if (rc == BGV_OK && (i == 0 || r.ms_att_short[i] < best_ms)) best_ms = r.ms_att_short[i], best.att_short = shorts[i];
    }
    for (int i = 0; i < 2 && rc == BGV_OK; ++i) {
        Fa2Tune t = best;
        t.repulse_threads = threads[i];
        set_fa2_tune(t);
        rc = time_steps(&r.ms_repulse_threads[i]);
        if (rc == BGV_OK && (i == 0 || r.ms_repulse_threads[i] < best_ms))
            best_ms = r.ms_repulse_threads[i], best.repulse_threads = threads[i];
    }
    for (int i = 0; i < 3 && rc == BGV_OK; ++i) {
        Fa2Tune t = best;
        t.tail_blocks_per_sm = tails[i];
        set_fa2_tune(t);
        rc = time_steps(&r.ms_tail_blocks[i]);
        if (rc == BGV_OK && (i == 0 || r.ms_tail_blocks[i] < best_ms))
            best_ms = r.ms_tail_blocks[i], best.tail_blocks_per_sm = tails[i];
    }
    set_fa2_tune(best);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BGV_TRY(rc);
    r.att_short = best.att_short;
    r.repulse_threads = best.repulse_threads;
    r.tail_blocks_per_sm = best.tail_blocks_per_sm;
    if (out) *out = r;
    return BGV_OK;
}

size_t bgv_autotune_sort_ws_size(int64_t max_keys) {
    Carver c(nullptr, kHeaderBytes);
    SortBuffers b;
    carve_sort(c, max_keys > 0 ? max_keys : 1, true, b);
    return c.used();
}

int bgv_autotune_sort(int64_t max_keys, bgv_tune_report *out, void *ws, size_t ws_bytes, void *stream) {
    if (max_keys < (int64_t(1) << 14) || max_keys >= (int64_t(1) << 31)) return BGV_EINVAL;
    BGV_TRY(check_ws(ws, ws_bytes, bgv_autotune_sort_ws_size(max_keys)));
    Carver c(ws, kHeaderBytes);
    SortBuffers b;
    carve_sort(c, max_keys, true, b);
    bgv_tune_report r;
    memset(&r, 0, sizeof(r));
    int32_t count = 0;
    int32_t method = 0;
    BGV_TRY(autotune_sort(max_keys, b, as_stream(stream), status_ptr(ws), r.ms8, r.ms16, r.ms_coop, r.sizes_log2,
                          &count, &method));
    r.count = count;
    r.method = method;
    sort_coop_range(&r.coop_lo, &r.coop_hi);
    r.cutoff = sort_cutoff();
    if (out) *out = r;
    return BGV_OK;
}

int64_t bgv_sort_cutoff(void) { return sort_cutoff(); }

int64_t bgv_set_sort_cutoff(int64_t cutoff) {
    if (cutoff < 0) return -1;
    return set_sort_cutoff(cutoff);
}

int32_t bgv_set_sort_method(int32_t method) {
    if (method < 0 || method > 2) return -1;
    return set_sort_method(method);
}

int32_t bgv_set_spin_limit(int32_t limit) {
    if (limit < 0) return -1;
    return set_spin_limit(limit);
}

size_t bgv_check_wait_timeout_ws_size(void) {
    size_t need = wait_check_sort_bytes();
    need = wait_check_moments_bytes() > need ? wait_check_moments_bytes() : need;
    need = wait_check_reduce_bytes() > need ? wait_check_reduce_bytes() : need;
    Carver c(nullptr, kHeaderBytes);
    c.take<char>(need);
    return c.used();
}

int bgv_check_wait_timeout(int32_t which, void *ws, size_t ws_bytes, void *stream) {
    BGV_TRY(check_ws(ws, ws_bytes, bgv_check_wait_timeout_ws_size()));
    Carver c(ws, kHeaderBytes);
    void *scratch = c.take<char>(0);
    cudaStream_t st = as_stream(stream);
    switch (which) {
        case 0: return wait_check_sort(scratch, status_ptr(ws), st);
        case 1: return wait_check_moments(scratch, status_ptr(ws), st);
        case 2: return wait_check_reduce(scratch, status_ptr(ws), st);
        default: return BGV_EINVAL;
    }
}

}  // extern "C"

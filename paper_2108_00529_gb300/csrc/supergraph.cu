// supergraph.cu -- supernodes, superedges, community sizes and the CSR that
// the ForceAtlas2 attraction reads (Section 4.1; Algorithm 3, "compute
// community sizes" and ForceAtlas2(Csrc, Cdst, Csize)).
//
// 1. Dense relabel: mark the labels in use, exclusive-scan the marks; the
//    rank of a label is its supernode id (ascending label order).
// 2. Cut edges: one edge pass emits (min, max) supernode pairs packed as
//    u64 keys (warp-aggregated compaction: one atomic per warp).
// 3. Stable LSD radix sort of the keys over 2 * bits(n) bits.
// 4. Reduce by key: run heads -> scan -> superedge endpoints and run lengths.
// 5. Community-size sketch: every node adds its sketched degree at the
//    hash of its label (u64 counters); mass = 1 + the row minimum.
// 6. Symmetric CSR with ascending neighbours: a stable sort of the
//    superedges by b orders them by (b, a); run boundaries in the two
//    orders give each row's in- and out-degree (no atomics), and every
//    entry's slot follows from its rank inside its run.
#include "bgv_internal.cuh"

namespace bgv {
namespace {
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_mark_labels(const int32_t *__restrict__ labels, int32_t n,
                                                          uint32_t *__restrict__ flags, uint32_t *status) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int32_t l = labels[v];
        if (static_cast<uint32_t>(l) < static_cast<uint32_t>(n))
            flags[l] = 1u;
        else
            raise_status(status, BGV_DEV_BADLABEL);
    }
}

__global__ void __launch_bounds__(kThreads) k_map_nodes(const int32_t *__restrict__ labels, int32_t n,
                                                        const uint32_t *__restrict__ flags,
                                                        const uint32_t *__restrict__ rank,
                                                        int32_t *__restrict__ node_map,
                                                        int32_t *__restrict__ label_of) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int32_t l = labels[v];
        node_map[v] = static_cast<uint32_t>(l) < static_cast<uint32_t>(n) ? int32_t(rank[l]) : 0;
        if (flags[v]) label_of[rank[v]] = int32_t(v);
    }
}

__device__ __forceinline__ void emit_cut(bool valid, unsigned long long key, unsigned long long *keys,
                                         int64_t *m_cut) {
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, valid);
    if (!mask) return;
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == __ffs(mask) - 1)
        base = atomicAdd(reinterpret_cast<unsigned long long *>(m_cut), static_cast<unsigned long long>(__popc(mask)));
    base = __shfl_sync(0xFFFFFFFFu, base, __ffs(mask) - 1);
    if (valid) keys[base + __popc(mask & ((1u << lane) - 1u))] = key;
}

__device__ __forceinline__ bool cut_key(int32_t u, int32_t v, int32_t n, const int32_t *node_map, int shift,
                                        unsigned long long *key, uint32_t *status) {
    if (static_cast<uint32_t>(u) >= static_cast<uint32_t>(n) || static_cast<uint32_t>(v) >= static_cast<uint32_t>(n)) {
        raise_status(status, BGV_DEV_BADEDGE);
        return false;
    }
    // node_map is one-to-one on labels, so equal supernodes = equal labels
    const uint32_t a = uint32_t(node_map[u]), b = uint32_t(node_map[v]);
    if (a == b) return false;
    const uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
    *key = (static_cast<unsigned long long>(lo) << shift) | hi;
    return true;
}

// Whole warps iterate together (the stride is a multiple of 32 and the exit
// test uses the warp's first index) so the ballot in emit_cut always sees all
// 32 lanes.
__global__ void __launch_bounds__(kThreads) k_cut_keys(const int32_t *__restrict__ edges, int64_t m, int32_t n,
                                                       const int32_t *__restrict__ node_map, int shift,
                                                       unsigned long long *__restrict__ keys, int64_t *m_cut,
                                                       uint32_t *status) {
    const int4 *e2 = reinterpret_cast<const int4 *>(edges);
    const int64_t full = m >> 1, pairs = (m + 1) >> 1;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p - lane < pairs; p += stride) {
        unsigned long long k0 = 0, k1 = 0;
        bool v0 = false, v1 = false;
        if (p < full) {
            const int4 e = __ldcs(e2 + p);
            v0 = cut_key(e.x, e.y, n, node_map, shift, &k0, status);
            v1 = cut_key(e.z, e.w, n, node_map, shift, &k1, status);
        } else if (p < pairs) {  // odd tail edge
            v0 = cut_key(edges[2 * (m - 1)], edges[2 * (m - 1) + 1], n, node_map, shift, &k0, status);
        }
        emit_cut(v0, k0, keys, m_cut);
        emit_cut(v1, k1, keys, m_cut);
    }
}

__global__ void __launch_bounds__(kThreads) k_run_heads(const unsigned long long *__restrict__ keys,
                                                        const int64_t *m_cut, int64_t cap,
                                                        uint32_t *__restrict__ heads) {
    int64_t mc = *m_cut;
    mc = mc < cap ? mc : cap;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < mc; i += stride)
        heads[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void __launch_bounds__(kThreads) k_emit_superedges(const unsigned long long *__restrict__ keys,
                                                              const int64_t *m_cut, int64_t cap,
                                                              const uint32_t *__restrict__ heads,
                                                              const uint32_t *__restrict__ segidx, int shift,
                                                              int32_t *__restrict__ ssrc, int32_t *__restrict__ sdst,
                                                              uint32_t *__restrict__ segstart) {
    int64_t mc = *m_cut;
    mc = mc < cap ? mc : cap;
    const unsigned long long lo_mask = (1ull << shift) - 1ull;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < mc; i += stride) {
        if (!heads[i]) continue;
        const uint32_t s = segidx[i];
        const unsigned long long k = keys[i];
        ssrc[s] = int32_t(k >> shift);
        sdst[s] = int32_t(k & lo_mask);
        segstart[s] = uint32_t(i);
    }
}

__global__ void __launch_bounds__(kThreads) k_weights(const uint32_t *__restrict__ segstart, const int64_t *Es_dev,
                                                      const int64_t *m_cut, uint32_t *__restrict__ sw) {
    const int64_t Es = *Es_dev, mc = *m_cut;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < Es; s += stride) {
        const int64_t next = (s + 1 < Es) ? int64_t(segstart[s + 1]) : mc;
        sw[s] = uint32_t(next - int64_t(segstart[s]));
    }
}

// Batched form: a label is a node id of its own graph g, hashed as its local
// id into graph g's matrix.
__device__ __forceinline__ size_t label_matrix(const HashFamily &h, int32_t l, const int32_t *node_graph,
                                               const int32_t *node_off, uint32_t *x) {
    if (!node_graph) {
        *x = uint32_t(l);
        return 0;
    }
    const int32_t g = node_graph[l];
    *x = uint32_t(l - node_off[g]);
    return size_t(g) * size_t(h.rows) * h.width;
}

__global__ void __launch_bounds__(kThreads) k_size_sketch(const int32_t *__restrict__ labels,
                                                          const uint32_t *__restrict__ deg_est,
                                                          const int32_t *__restrict__ node_map, int32_t n,
                                                          const __grid_constant__ HashFamily h,
                                                          unsigned long long *__restrict__ sketch,
                                                          unsigned long long *__restrict__ vol,
                                                          uint32_t *__restrict__ count,
                                                          const int32_t *__restrict__ node_graph,
                                                          const int32_t *__restrict__ node_off) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int32_t l = labels[v];
        if (static_cast<uint32_t>(l) >= static_cast<uint32_t>(n)) continue;
        const unsigned long long d = deg_est[v];
        if (d) {
            uint32_t x;
            unsigned long long *M = sketch + label_matrix(h, l, node_graph, node_off, &x);
            for (int i = 0; i < h.rows; ++i) atomicAdd(&M[size_t(i) * h.width + hash_eval(h.a[i], h.b[i], x, h.width)], d);
        }
        if (vol && d) atomicAdd(&vol[node_map[v]], d);
        if (count) atomicAdd(&count[node_map[v]], 1u);
    }
}

__global__ void __launch_bounds__(kThreads) k_mass(const int32_t *__restrict__ label_of, const int64_t *K_dev,
                                                   const __grid_constant__ HashFamily h,
                                                   const unsigned long long *__restrict__ sketch,
                                                   uint32_t *__restrict__ mass, int32_t *__restrict__ comm_label,
                                                   const int32_t *__restrict__ node_graph,
                                                   const int32_t *__restrict__ node_off) {
    const int64_t K = *K_dev;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < K; k += stride) {
        const uint32_t l = uint32_t(label_of[k]);
        uint32_t x;
        const unsigned long long *M = sketch + label_matrix(h, int32_t(l), node_graph, node_off, &x);
        unsigned long long best = ~0ull;
        for (int i = 0; i < h.rows; ++i) {
            const unsigned long long c = M[size_t(i) * h.width + hash_eval(h.a[i], h.b[i], x, h.width)];
            best = c < best ? c : best;
        }
        const unsigned long long ms = best + 1;
        mass[k] = ms > 0xFFFFFFFFull ? 0xFFFFFFFFu : uint32_t(ms);
        if (comm_label) comm_label[k] = int32_t(l);
    }
}

// Run boundaries of a sorted id sequence: first[id] and end[id] (both left
// at 0 for ids that do not occur), so the run length is end - first.
__global__ void __launch_bounds__(kThreads) k_runs_i32(const int32_t *__restrict__ ids, const int64_t *Es_dev,
                                                       uint32_t *__restrict__ first, uint32_t *__restrict__ end) {
    const int64_t Es = *Es_dev;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < Es; s += stride) {
        const int32_t a = ids[s];
        if (s == 0 || ids[s - 1] != a) first[a] = uint32_t(s);
        if (s == Es - 1 || ids[s + 1] != a) end[a] = uint32_t(s + 1);
    }
}

__global__ void __launch_bounds__(kThreads) k_runs_u64(const unsigned long long *__restrict__ ids,
                                                       const int64_t *Es_dev, uint32_t *__restrict__ first,
                                                       uint32_t *__restrict__ end) {
    const int64_t Es = *Es_dev;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < Es; s += stride) {
        const uint32_t a = uint32_t(ids[s]);
        if (s == 0 || uint32_t(ids[s - 1]) != a) first[a] = uint32_t(s);
        if (s == Es - 1 || uint32_t(ids[s + 1]) != a) end[a] = uint32_t(s + 1);
    }
}

// CSR row length = out-degree (run in the (src, dst) order) + in-degree (run
// in the (dst, src) order).
__global__ void __launch_bounds__(kThreads) k_row_lengths(int32_t n, const uint32_t *__restrict__ sf,
                                                          const uint32_t *__restrict__ se,
                                                          const uint32_t *__restrict__ df,
                                                          const uint32_t *__restrict__ de, uint32_t *__restrict__ cnt) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += stride)
        cnt[k] = (se[k] - sf[k]) + (de[k] - df[k]);
}

__global__ void __launch_bounds__(kThreads) k_dst_keys(const int32_t *__restrict__ sdst, const int64_t *Es_dev,
                                                       unsigned long long *__restrict__ keys,
                                                       uint32_t *__restrict__ vals) {
    const int64_t Es = *Es_dev;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < Es; s += stride) {
        keys[s] = static_cast<unsigned long long>(uint32_t(sdst[s]));
        vals[s] = uint32_t(s);
    }
}

// Row a lists its in-neighbours (smaller ids, from the (dst, src) order)
// first, then its out-neighbours (larger ids, from the (src, dst) order).
__global__ void __launch_bounds__(kThreads) k_csr_fill_src(const int32_t *__restrict__ ssrc,
                                                           const int32_t *__restrict__ sdst,
                                                           const uint32_t *__restrict__ sw, const int64_t *Es_dev,
                                                           const int32_t *__restrict__ csr_off,
                                                           const uint32_t *__restrict__ sf,
                                                           const uint32_t *__restrict__ df,
                                                           const uint32_t *__restrict__ de,
                                                           int32_t *__restrict__ csr_adj, uint32_t *__restrict__ csr_w) {
    const int64_t Es = *Es_dev;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < Es; s += stride) {
        const int32_t a = ssrc[s];
        const int64_t pos = int64_t(csr_off[a]) + (de[a] - df[a]) + (s - int64_t(sf[a]));
        csr_adj[pos] = sdst[s];
        csr_w[pos] = sw[s];
    }
}

__global__ void __launch_bounds__(kThreads) k_csr_fill_dst(const unsigned long long *__restrict__ bkeys,
                                                           const uint32_t *__restrict__ bvals, const int64_t *Es_dev,
                                                           const int32_t *__restrict__ ssrc,
                                                           const uint32_t *__restrict__ sw,
                                                           const int32_t *__restrict__ csr_off,
                                                           const uint32_t *__restrict__ df,
                                                           int32_t *__restrict__ csr_adj, uint32_t *__restrict__ csr_w) {
    const int64_t Es = *Es_dev;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < Es; t += stride) {
        const uint32_t b = uint32_t(bkeys[t]);
        const uint32_t s = bvals[t];
        const int64_t pos = int64_t(csr_off[b]) + (t - int64_t(df[b]));
        csr_adj[pos] = ssrc[s];
        csr_w[pos] = sw[s];
    }
}
}  // namespace

void carve_super(Carver &c, int64_t m, int32_t n, int32_t rows, int32_t width, SuperScratch &s, int32_t G) {
    s.flags = c.take<uint32_t>(size_t(n) + 1);
    s.rank = c.take<uint32_t>(size_t(n) + 1);
    s.label_of = c.take<int32_t>(size_t(n));
    s.src_first = c.take<uint32_t>(size_t(n));
    s.src_end = c.take<uint32_t>(size_t(n));
    s.dst_first = c.take<uint32_t>(size_t(n));
    s.dst_end = c.take<uint32_t>(size_t(n));
    s.m_cut = c.take<int64_t>(1);
    s.sketch = c.take<unsigned long long>(size_t(rows) * size_t(width) * size_t(G > 1 ? G : 1));
    s.heads = c.take<uint32_t>(size_t(m));
    s.segidx = c.take<uint32_t>(size_t(m) + 1);
    s.segstart = c.take<uint32_t>(size_t(m));
    int64_t big = int64_t(m) > int64_t(n) + 1 ? int64_t(m) : int64_t(n) + 1;
    s.scan_tmp = c.take<char>(scan_tmp_bytes(big));
    carve_sort(c, m, false, s.sort_cut);
    carve_sort(c, m, true, s.sort_dst);
}

int run_supergraph(const int32_t *edges, int64_t m, int32_t n, const int32_t *labels, const uint32_t *deg_est,
                   const HashFamily &h, int32_t *node_map, int64_t *K_dev, int32_t *ssrc, int32_t *sdst,
                   uint32_t *sw, int64_t *Es_dev, uint32_t *mass, int32_t *csr_off, int32_t *csr_adj,
                   uint32_t *csr_w, uint64_t *vol, uint32_t *count, int32_t *comm_label,
                   const SuperScratch &s, uint32_t *status, cudaStream_t st, const BatchView *batch) {
    const int32_t *node_graph = batch ? batch->node_graph : nullptr;
    const int32_t *node_off = batch ? batch->node_off : nullptr;
    const size_t mats = batch ? size_t(batch->G) : 1;
    const int gn = grid_for(n, kThreads, 152 * 8);
    const int gm = grid_for(m > 0 ? m : 1, kThreads, 152 * 8);
    const int shift = bits_for(n);  // supernode ids < K <= n fit in `shift` bits

    // 1. dense relabel
    BGV_CUDA(cudaMemsetAsync(s.flags, 0, sizeof(uint32_t) * (size_t(n) + 1), st));
    note_launch(), k_mark_labels<<<gn, kThreads, 0, st>>>(labels, n, s.flags, status);
    BGV_TRY(launch_status());
    BGV_TRY(scan_exclusive(s.flags, s.rank, n, nullptr, reinterpret_cast<unsigned long long *>(K_dev), false,
                           s.scan_tmp, st));
    note_launch(), k_map_nodes<<<gn, kThreads, 0, st>>>(labels, n, s.flags, s.rank, node_map, s.label_of);
    BGV_TRY(launch_status());

    // 2-4. cut edges -> sorted keys -> superedges with multiplicities
    BGV_CUDA(cudaMemsetAsync(s.m_cut, 0, sizeof(int64_t), st));
    SortBuffers cut = s.sort_cut;
    if (m > 0) {
        note_launch(), k_cut_keys<<<grid_for((m + 1) / 2, kThreads, 152 * 8), kThreads, 0, st>>>(edges, m, n, node_map,
                                                                                 shift, cut.keys[0], s.m_cut, status);
        BGV_TRY(launch_status());
    }
    int res = 0;
    BGV_TRY(radix_sort(cut, m > 0 ? m : 1, s.m_cut, 2 * shift, st, &res, status));
    const unsigned long long *sorted = cut.keys[res];
    note_launch(), k_run_heads<<<gm, kThreads, 0, st>>>(sorted, s.m_cut, m, s.heads);
    BGV_TRY(launch_status());
    BGV_TRY(scan_exclusive(s.heads, s.segidx, m > 0 ? m : 1, s.m_cut, reinterpret_cast<unsigned long long *>(Es_dev),
                           false, s.scan_tmp, st));
    note_launch(), k_emit_superedges<<<gm, kThreads, 0, st>>>(sorted, s.m_cut, m, s.heads, s.segidx, shift, ssrc, sdst,
                                                s.segstart);
    BGV_TRY(launch_status());
    note_launch(), k_weights<<<gm, kThreads, 0, st>>>(s.segstart, Es_dev, s.m_cut, sw);
    BGV_TRY(launch_status());

    // 5. community sizes
    BGV_CUDA(cudaMemsetAsync(s.sketch, 0, sizeof(unsigned long long) * size_t(h.rows) * h.width * mats, st));
    if (vol) BGV_CUDA(cudaMemsetAsync(vol, 0, sizeof(uint64_t) * size_t(n), st));
    if (count) BGV_CUDA(cudaMemsetAsync(count, 0, sizeof(uint32_t) * size_t(n), st));
    note_launch(), k_size_sketch<<<gn, kThreads, 0, st>>>(labels, deg_est, node_map, n, h, s.sketch,
                                                          reinterpret_cast<unsigned long long *>(vol), count,
                                                          node_graph, node_off);
    BGV_TRY(launch_status());
    note_launch(), k_mass<<<gn, kThreads, 0, st>>>(s.label_of, K_dev, h, s.sketch, mass, comm_label, node_graph,
                                                   node_off);
    BGV_TRY(launch_status());

    // 6. symmetric CSR: the superedges in (src, dst) order and, from a stable
    //    sort by dst, in (dst, src) order; run boundaries give the degrees.
    SortBuffers dsort = s.sort_dst;
    note_launch(), k_dst_keys<<<gm, kThreads, 0, st>>>(sdst, Es_dev, dsort.keys[0], dsort.vals[0]);
    BGV_TRY(launch_status());
    int dres = 0;
    BGV_TRY(radix_sort(dsort, m > 0 ? m : 1, Es_dev, shift, st, &dres, status));
    BGV_CUDA(cudaMemsetAsync(s.src_first, 0, sizeof(uint32_t) * size_t(n), st));
    BGV_CUDA(cudaMemsetAsync(s.src_end, 0, sizeof(uint32_t) * size_t(n), st));
    BGV_CUDA(cudaMemsetAsync(s.dst_first, 0, sizeof(uint32_t) * size_t(n), st));
    BGV_CUDA(cudaMemsetAsync(s.dst_end, 0, sizeof(uint32_t) * size_t(n), st));
    note_launch(), k_runs_i32<<<gm, kThreads, 0, st>>>(ssrc, Es_dev, s.src_first, s.src_end);
    note_launch(), k_runs_u64<<<gm, kThreads, 0, st>>>(dsort.keys[dres], Es_dev, s.dst_first, s.dst_end);
    note_launch(), k_row_lengths<<<gn, kThreads, 0, st>>>(n, s.src_first, s.src_end, s.dst_first, s.dst_end,
                                                          s.flags);
    BGV_TRY(launch_status());
    BGV_TRY(scan_exclusive(s.flags, reinterpret_cast<uint32_t *>(csr_off), n, nullptr, nullptr, true, s.scan_tmp,
                           st));
    note_launch(), k_csr_fill_src<<<gm, kThreads, 0, st>>>(ssrc, sdst, sw, Es_dev, csr_off, s.src_first,
                                                           s.dst_first, s.dst_end, csr_adj, csr_w);
    note_launch(), k_csr_fill_dst<<<gm, kThreads, 0, st>>>(dsort.keys[dres], dsort.vals[dres], Es_dev, ssrc, sw,
                                                           csr_off, s.dst_first, csr_adj, csr_w);
    return launch_status();
}

}  // namespace bgv

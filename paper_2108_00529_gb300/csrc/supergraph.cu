// supergraph.cu -- supernodes, superedges, community sizes and the CSR that
// the ForceAtlas2 attraction reads (Section 4.1; Algorithm 3, "compute
// community sizes" and ForceAtlas2(Csrc, Cdst, Csize)).
//
// 1. Dense relabel: mark the labels in use, exclusive-scan the marks; the
//    rank of a label is its supernode id (ascending label order).
// 2. Cut edges: one edge pass emits, for every edge whose endpoints lie in
//    different supernodes a != c, both directed pairs (a, c) and (c, a) as
//    u64 keys row << b | col.  Blocks compact their keys in shared memory
//    and take their output range with one atomic per 1,024 edges.
// 3. Stable LSD radix sort of the keys over 2 * bits(n) bits.  The sorted
//    keys are the symmetric CSR in row order with repeated pairs adjacent.
// 4. One pass over the sorted keys (decoupled look-back over tiles) collapses
//    repeated pairs: distinct pairs become CSR entries (ascending neighbours
//    per row, row offsets from the row changes) and the pairs with col > row
//    the superedges (src < dst, sorted ascending); a second pass turns run
//    starts into multiplicities (edge weights).
// 5. Community-size sketch: every node adds its sketched degree at the
//    hash of its label (u64 counters); mass = 1 + the row minimum.
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

// ------------------------------------------------------------- cut pairs
// A block takes chunks of kCutPairs int4 loads (two edges each): every thread
// emits up to 8 keys, the block scans the counts, stages the keys in shared
// memory in that order and writes them out in one coalesced run at an offset
// taken with a single atomic per chunk.
constexpr int kCutLoads = 2;                      // int4 loads per thread and chunk
constexpr int kCutPairs = kThreads * kCutLoads;   // int4 (edge pairs) per chunk
constexpr int kCutKeys = 4 * kCutPairs;           // keys per chunk at most

// The supernode pair (a, c) of edge (u, v); false for an edge inside one
// supernode (or a bad endpoint, which is reported).
__device__ __forceinline__ bool cut_pair(int32_t u, int32_t v, int32_t n, const int32_t *node_map, uint32_t *a,
                                         uint32_t *c, uint32_t *status) {
    if (static_cast<uint32_t>(u) >= static_cast<uint32_t>(n) || static_cast<uint32_t>(v) >= static_cast<uint32_t>(n)) {
        raise_status(status, BGV_DEV_BADEDGE);
        return false;
    }
    // node_map is one-to-one on labels, so equal supernodes = equal labels
    *a = uint32_t(node_map[u]);
    *c = uint32_t(node_map[v]);
    return *a != *c;
}

__device__ __forceinline__ uint32_t block_exclusive_u32(uint32_t x, uint32_t *total) {
    __shared__ uint32_t wsum[kThreads / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < kThreads / 32 ? wsum[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < kThreads / 32) wsum[lane] = wi - w;
        if (lane == kThreads / 32 - 1) wsum[kThreads / 32] = wi;
    }
    __syncthreads();
    const uint32_t r = wsum[warp] + inc - x;
    *total = wsum[kThreads / 32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kThreads) k_cut_pairs(const int32_t *__restrict__ edges, int64_t m, int32_t n,
                                                        const int32_t *__restrict__ node_map, int shift,
                                                        unsigned long long *__restrict__ keys,
                                                        unsigned long long *nkeys, uint32_t *status) {
    __shared__ unsigned long long stage[kCutKeys];
    __shared__ unsigned long long base_sh;
    const int4 *e2 = reinterpret_cast<const int4 *>(edges);
    const int64_t full = m >> 1, pairs = (m + 1) >> 1;
    const int64_t chunks = (pairs + kCutPairs - 1) / kCutPairs;
    for (int64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
        int4 e[kCutLoads];
#pragma unroll
        for (int r = 0; r < kCutLoads; ++r) {
            const int64_t p = c * kCutPairs + int64_t(r) * kThreads + threadIdx.x;
            e[r] = p < full ? __ldcs(e2 + p) : make_int4(0, 0, 0, 0);
        }
        uint32_t pa[2 * kCutLoads], pc[2 * kCutLoads];
        bool ok[2 * kCutLoads];
        uint32_t cnt = 0;
#pragma unroll
        for (int r = 0; r < kCutLoads; ++r) {
            const int64_t p = c * kCutPairs + int64_t(r) * kThreads + threadIdx.x;
            ok[2 * r] = ok[2 * r + 1] = false;
            if (p < full) {
                ok[2 * r] = cut_pair(e[r].x, e[r].y, n, node_map, &pa[2 * r], &pc[2 * r], status);
                ok[2 * r + 1] = cut_pair(e[r].z, e[r].w, n, node_map, &pa[2 * r + 1], &pc[2 * r + 1], status);
            } else if (p < pairs) {  // odd tail edge
                ok[2 * r] = cut_pair(edges[2 * (m - 1)], edges[2 * (m - 1) + 1], n, node_map, &pa[2 * r], &pc[2 * r],
                                     status);
            }
            cnt += (ok[2 * r] ? 2u : 0u) + (ok[2 * r + 1] ? 2u : 0u);
        }
        uint32_t total;
        uint32_t off = block_exclusive_u32(cnt, &total);
        if (threadIdx.x == 0) base_sh = total ? atomicAdd(nkeys, static_cast<unsigned long long>(total)) : 0ull;
#pragma unroll
        for (int j = 0; j < 2 * kCutLoads; ++j) {
            if (ok[j]) {
                stage[off] = (static_cast<unsigned long long>(pa[j]) << shift) | pc[j];
                stage[off + 1] = (static_cast<unsigned long long>(pc[j]) << shift) | pa[j];
                off += 2;
            }
        }
        __syncthreads();
        const unsigned long long base = base_sh;
        for (uint32_t j = threadIdx.x; j < total; j += kThreads) keys[base + j] = stage[j];
        __syncthreads();
    }
}

// --------------------------------------------------- pairs -> CSR, superedges
// Tiles of kRedTile sorted keys, taken in order from a counter.  A thread
// holds kRedItems consecutive keys (loaded through shared memory) and marks
// the distinct pairs (heads) and, among them, those with col > row (the
// superedges).  The tile's two counts are scanned as one u64 (heads in the
// low 32 bits: at most 2 m < 2^32 of them), then a decoupled look-back gives
// the tile's offsets.  Outputs are staged in shared memory and written in
// coalesced runs: csr_adj and the run start of every distinct pair, the
// superedge index of each CSR entry (or -1), ssrc/sdst of the superedges,
// and csr_off of every row that starts in the tile (and of the empty rows
// before it).  The last tile writes the totals, start[nnz] and the offsets of
// the rows after the last pair.
constexpr int kRedItems = 8;
constexpr int kRedTile = kThreads * kRedItems;
enum : uint32_t { kRedAgg = 1u, kRedIncl = 2u };

__device__ __forceinline__ int red_slot(int e) { return e + (e >> 3); }

__device__ __forceinline__ unsigned long long block_exclusive_u64(unsigned long long x, unsigned long long *total) {
    __shared__ unsigned long long wsum[kThreads / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long w = lane < kThreads / 32 ? wsum[lane] : 0ull;
        unsigned long long wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < kThreads / 32) wsum[lane] = wi - w;
        if (lane == kThreads / 32 - 1) wsum[kThreads / 32] = wi;
    }
    __syncthreads();
    const unsigned long long r = wsum[warp] + inc - x;
    *total = wsum[kThreads / 32];
    __syncthreads();
    return r;
}

constexpr int kRedGapList = 64;  // long runs of empty rows a tile fills with all its threads

__global__ void __launch_bounds__(kThreads) k_csr_reduce(const unsigned long long *__restrict__ keys,
                                                         const unsigned long long *nkeys_dev, int64_t cap, int shift,
                                                         const int64_t *K_dev, int32_t *__restrict__ csr_off,
                                                         int32_t *__restrict__ csr_adj, uint32_t *__restrict__ start,
                                                         int32_t *__restrict__ supidx, int32_t *__restrict__ ssrc,
                                                         int32_t *__restrict__ sdst, uint32_t *flags,
                                                         unsigned long long *agg, unsigned long long *incl,
                                                         int64_t *Es_dev, int64_t *nnz_dev, uint32_t *dev_status,
                                                         int spin_limit) {
    __shared__ unsigned long long skey[kRedTile + kRedTile / 8];
    __shared__ uint16_t ent_e[kRedTile];   // element of every distinct pair of the tile
    __shared__ uint16_t sup_e[kRedTile];   // element of every superedge of the tile
    __shared__ int32_t ssup[kRedTile];     // superedge index of every distinct pair, or -1
    __shared__ long long gap_lo[kRedGapList], gap_hi[kRedGapList];
    __shared__ int32_t gap_val[kRedGapList];
    __shared__ int gaps;
    __shared__ unsigned tile_sh;
    __shared__ unsigned long long excl_sh;
    int64_t nk = int64_t(*nkeys_dev);
    nk = nk < cap ? nk : cap;
    const int64_t K = *K_dev;
    const int64_t tiles = (nk + kRedTile - 1) / kRedTile;
    if (threadIdx.x == 0) {
        tile_sh = atomicAdd(&flags[tiles > 0 ? tiles : 1], 1u);
        gaps = 0;
    }
    __syncthreads();
    const int64_t tile = tile_sh;
    if (nk == 0) {  // no cut edges: every row is empty
        if (tile == 0)
            for (int64_t r = threadIdx.x; r <= K; r += kThreads) csr_off[r] = 0;
        if (tile == 0 && threadIdx.x == 0) {
            *Es_dev = 0;
            *nnz_dev = 0;
            start[0] = 0u;
        }
        return;
    }
    if (tile >= tiles) return;
    const int64_t t0 = tile * kRedTile;
    const int tn = nk - t0 < kRedTile ? int(nk - t0) : kRedTile;
    for (int e = threadIdx.x; e < tn; e += kThreads) skey[red_slot(e)] = keys[t0 + e];
    __syncthreads();
    const unsigned long long col_mask = (1ull << shift) - 1ull;
    const int e0 = threadIdx.x * kRedItems;
    const bool have_prev = e0 > 0 || t0 > 0;
    const unsigned long long before = e0 == 0 ? (t0 > 0 ? keys[t0 - 1] : 0ull) : skey[red_slot(e0 < tn ? e0 - 1 : 0)];
    unsigned long long prev = before;
    uint32_t heads = 0u, ups = 0u;  // bit j: item j is a head / a superedge
#pragma unroll
    for (int j = 0; j < kRedItems; ++j) {
        const int e = e0 + j;
        if (e < tn) {
            const unsigned long long k = skey[red_slot(e)];
            if ((j == 0 && !have_prev) || k != prev) {  // the first key of all, or a new pair
                heads |= 1u << j;
                if ((k & col_mask) > (k >> shift)) ups |= 1u << j;
            }
            prev = k;
        }
    }
    unsigned long long tile_tot;
    const unsigned long long mine = static_cast<unsigned long long>(__popc(heads)) |
                                    (static_cast<unsigned long long>(__popc(ups)) << 32);
    const unsigned long long local = block_exclusive_u64(mine, &tile_tot);
    // publish the tile total, then look back (warp 0) for the tile's offset
    if (threadIdx.x == 0) {
        if (tile == 0) {
            incl[0] = tile_tot;
        } else {
            agg[tile] = tile_tot;
        }
        __threadfence();
        atomicExch(&flags[tile], tile == 0 ? kRedIncl : kRedAgg);
    }
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        unsigned long long excl = 0ull;
        int64_t hi = tile - 1;
        int spins = 0;
        while (hi >= 0) {
            const int64_t idx = hi - lane;
            const uint32_t f = idx >= 0 ? *reinterpret_cast<volatile uint32_t *>(&flags[idx]) : kRedIncl;
            const unsigned inc_mask = __ballot_sync(0xFFFFFFFFu, f == kRedIncl);
            const int near = inc_mask ? __ffs(inc_mask) - 1 : 32;  // lowest lane = nearest tile
            if (__any_sync(0xFFFFFFFFu, lane < near && f == 0u)) {
                if (++spins > spin_limit) {
                    if (lane == 0) raise_status(dev_status, BGV_DEV_TIMEOUT);
                    break;
                }
                __nanosleep(32);
                continue;
            }
            __threadfence();
            unsigned long long v = 0ull;
            if (lane <= near && idx >= 0) v = __ldcg(f == kRedIncl ? &incl[idx] : &agg[idx]);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, d);
            excl += v;
            if (near < 32) break;
            hi -= 32;
        }
        if (lane == 0) {
            excl_sh = excl;
            if (tile > 0) {
                incl[tile] = excl + tile_tot;
                __threadfence();
                atomicExch(&flags[tile], kRedIncl);
            }
        }
    }
    __syncthreads();
    const unsigned long long excl = excl_sh;
    const uint32_t d_excl = uint32_t(excl), u_excl = uint32_t(excl >> 32);
    const uint32_t d_tile = uint32_t(tile_tot), u_tile = uint32_t(tile_tot >> 32);
    // Stage the tile's distinct pairs and superedges (by element), and write
    // the offsets of the rows that start here: rows prev_row + 1 .. row take
    // the index of the row's first pair (the ones before row are empty).
    uint32_t dl = uint32_t(local), ul = uint32_t(local >> 32);
    long long prev_row = have_prev ? static_cast<long long>(before >> shift) : -1ll;
#pragma unroll
    for (int j = 0; j < kRedItems; ++j) {
        const int e = e0 + j;
        if (e >= tn || !((heads >> j) & 1u)) continue;
        const unsigned long long k = skey[red_slot(e)];
        const long long row = static_cast<long long>(k >> shift);
        ent_e[dl] = uint16_t(e);
        if ((ups >> j) & 1u) {
            ssup[dl] = int32_t(u_excl + ul);
            sup_e[ul] = uint16_t(e);
            ++ul;
        } else {
            ssup[dl] = -1;
        }
        if (row > prev_row) {
            const int32_t v = int32_t(d_excl + dl);
            if (row - prev_row <= 32) {
                for (long long r = prev_row + 1; r <= row; ++r) csr_off[r] = v;
            } else {
                const int g = atomicAdd(&gaps, 1);
                if (g < kRedGapList) {
                    gap_lo[g] = prev_row + 1;
                    gap_hi[g] = row;
                    gap_val[g] = v;
                } else {
                    for (long long r = prev_row + 1; r <= row; ++r) csr_off[r] = v;
                }
            }
        }
        prev_row = row;
        ++dl;
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < d_tile; j += kThreads) {
        const int e = ent_e[j];
        csr_adj[d_excl + j] = int32_t(skey[red_slot(e)] & col_mask);
        start[d_excl + j] = uint32_t(t0 + e);
        supidx[d_excl + j] = ssup[j];
    }
    for (uint32_t j = threadIdx.x; j < u_tile; j += kThreads) {
        const unsigned long long k = skey[red_slot(sup_e[j])];
        ssrc[u_excl + j] = int32_t(k >> shift);
        sdst[u_excl + j] = int32_t(k & col_mask);
    }
    const int ng = gaps < kRedGapList ? gaps : kRedGapList;
    for (int g = 0; g < ng; ++g)
        for (long long r = gap_lo[g] + threadIdx.x; r <= gap_hi[g]; r += kThreads) csr_off[r] = gap_val[g];
    if (tile == tiles - 1) {  // the rows after the last pair, and the totals
        const uint32_t D = d_excl + d_tile, U = u_excl + u_tile;
        const long long last_row = static_cast<long long>(skey[red_slot(tn - 1)] >> shift);
        for (long long r = last_row + 1 + threadIdx.x; r <= K; r += kThreads) csr_off[r] = int32_t(D);
        if (threadIdx.x == 0) {
            start[D] = uint32_t(nk);
            *Es_dev = U;
            *nnz_dev = D;
        }
    }
}

// Multiplicities: CSR entry j covers sorted keys start[j] .. start[j+1].
__global__ void __launch_bounds__(kThreads) k_csr_weights(const uint32_t *__restrict__ start,
                                                          const int32_t *__restrict__ supidx, const int64_t *nnz_dev,
                                                          uint32_t *__restrict__ csr_w, uint32_t *__restrict__ sw) {
    const int64_t D = *nnz_dev;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < D; j += stride) {
        const uint32_t w = start[j + 1] - start[j];
        csr_w[j] = w;
        const int32_t u = supidx[j];
        if (u >= 0) sw[u] = w;
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

}  // namespace

void carve_super(Carver &c, int64_t m, int32_t n, int32_t rows, int32_t width, SuperScratch &s, int32_t G) {
    const int64_t keys = 2 * (m > 0 ? m : 1);  // both directions of every edge at most
    s.flags = c.take<uint32_t>(size_t(n) + 1);
    s.rank = c.take<uint32_t>(size_t(n) + 1);
    s.label_of = c.take<int32_t>(size_t(n));
    s.nkeys = c.take<unsigned long long>(1);
    s.nnz = c.take<int64_t>(1);
    s.sketch = c.take<unsigned long long>(size_t(rows) * size_t(width) * size_t(G > 1 ? G : 1));
    s.start = c.take<uint32_t>(size_t(keys) + 1);
    s.supidx = c.take<int32_t>(size_t(keys));
    const int64_t tiles = (keys + kRedTile - 1) / kRedTile;
    s.red_flags = c.take<uint32_t>(size_t(tiles) + 2);
    s.red_agg = c.take<unsigned long long>(size_t(tiles) + 1);
    s.red_incl = c.take<unsigned long long>(size_t(tiles) + 1);
    s.scan_tmp = c.take<char>(scan_tmp_bytes(int64_t(n) + 1));
    carve_sort(c, keys, false, s.sort_pairs);
}

int run_supergraph(const int32_t *edges, int64_t m, int32_t n, const int32_t *labels, const uint32_t *deg_est,
                   const HashFamily &h, int32_t *node_map, int64_t *K_dev, int32_t *ssrc, int32_t *sdst,
                   uint32_t *sw, int64_t *Es_dev, uint32_t *mass, int32_t *csr_off, int32_t *csr_adj,
                   uint32_t *csr_w, uint64_t *vol, uint32_t *count, int32_t *comm_label,
                   const SuperScratch &s, uint32_t *status, cudaStream_t st, const BatchView *batch) {
    const int32_t *node_graph = batch ? batch->node_graph : nullptr;
    const int32_t *node_off = batch ? batch->node_off : nullptr;
    const size_t mats = batch ? size_t(batch->G) : 1;
    const int gn = grid_for(n, kThreads, sm_count() * 8);
    const int shift = bits_for(n);  // supernode ids < K <= n fit in `shift` bits
    const int64_t cap = 2 * (m > 0 ? m : 1);

    // 1. dense relabel
    BGV_CUDA(cudaMemsetAsync(s.flags, 0, sizeof(uint32_t) * (size_t(n) + 1), st));
    note_launch(), k_mark_labels<<<gn, kThreads, 0, st>>>(labels, n, s.flags, status);
    BGV_TRY(launch_status());
    BGV_TRY(scan_exclusive(s.flags, s.rank, n, nullptr, reinterpret_cast<unsigned long long *>(K_dev), false,
                           s.scan_tmp, st));
    note_launch(), k_map_nodes<<<gn, kThreads, 0, st>>>(labels, n, s.flags, s.rank, node_map, s.label_of);
    BGV_TRY(launch_status());

    // 2-3. both directions of every cut edge -> sorted (row, col) keys
    BGV_CUDA(cudaMemsetAsync(s.nkeys, 0, sizeof(unsigned long long), st));
    SortBuffers pairs = s.sort_pairs;
    if (m > 0) {
        const int64_t chunks = ((m + 1) / 2 + kCutPairs - 1) / kCutPairs;
        note_launch(), k_cut_pairs<<<grid_for(chunks, 1, sm_count() * 8), kThreads, 0, st>>>(
            edges, m, n, node_map, shift, pairs.keys[0], s.nkeys, status);
        BGV_TRY(launch_status());
    }
    const int64_t *nkeys = reinterpret_cast<const int64_t *>(s.nkeys);
    // A row's pairs tie on their low 16 bits far too often for a local
    // finish on them (hub rows), so every digit gets an LSD pass.
    int res = 0;
    BGV_TRY(radix_sort(pairs, cap, nkeys, 2 * shift, st, &res, status));
    const unsigned long long *sorted = pairs.keys[res];

    // 4. distinct pairs -> CSR entries and superedges, then multiplicities
    const int64_t tiles = (cap + kRedTile - 1) / kRedTile;
    BGV_CUDA(cudaMemsetAsync(s.red_flags, 0, sizeof(uint32_t) * (size_t(tiles) + 2), st));
    note_launch(), k_csr_reduce<<<unsigned(tiles), kThreads, 0, st>>>(
        sorted, s.nkeys, cap, shift, K_dev, csr_off, csr_adj, s.start, s.supidx, ssrc, sdst, s.red_flags, s.red_agg,
        s.red_incl, Es_dev, s.nnz, status, spin_limit());
    BGV_TRY(launch_status());
    note_launch(), k_csr_weights<<<grid_for(cap, kThreads, sm_count() * 8), kThreads, 0, st>>>(s.start, s.supidx, s.nnz,
                                                                                             csr_w, sw);
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
    return launch_status();
}

// Bounded-wait self check of the CSR pass: one block as tile 1 of two tiles
// of equal keys (row 0, col 0; one supernode) whose tile 0 never runs, so
// its look-back must give up at the spin limit.  Equal keys make no CSR
// entries in tile 1, and the offsets of the single row stay in range.
namespace {
struct WaitCheckReduce {
    unsigned long long *keys, *nkeys, *agg, *incl;
    int64_t *K, *Es, *nnz;
    int32_t *csr_off, *csr_adj, *supidx, *ssrc, *sdst;
    uint32_t *start, *flags;
};
void carve_wait_check_reduce(Carver &c, WaitCheckReduce &w) {
    const size_t n = 2 * kRedTile;
    w.keys = c.take<unsigned long long>(n);
    w.nkeys = c.take<unsigned long long>(1);
    w.agg = c.take<unsigned long long>(2);
    w.incl = c.take<unsigned long long>(2);
    w.K = c.take<int64_t>(1);
    w.Es = c.take<int64_t>(1);
    w.nnz = c.take<int64_t>(1);
    w.csr_off = c.take<int32_t>(2);
    w.csr_adj = c.take<int32_t>(n);
    w.supidx = c.take<int32_t>(n);
    w.ssrc = c.take<int32_t>(n);
    w.sdst = c.take<int32_t>(n);
    w.start = c.take<uint32_t>(n + 1);
    w.flags = c.take<uint32_t>(3);
}
}  // namespace

size_t wait_check_reduce_bytes() {
    Carver c(nullptr, 0);
    WaitCheckReduce w;
    carve_wait_check_reduce(c, w);
    return c.used();
}

int wait_check_reduce(void *scratch, uint32_t *dev_status, cudaStream_t st) {
    Carver c(scratch, 0);
    WaitCheckReduce w;
    carve_wait_check_reduce(c, w);
    BGV_CUDA(cudaMemsetAsync(scratch, 0, wait_check_reduce_bytes(), st));
    const unsigned long long nk = 2 * kRedTile;
    const int64_t K = 1;
    const uint32_t one = 1u;  // the tile counter (after the two tiles' flags)
    BGV_CUDA(cudaMemcpyAsync(w.nkeys, &nk, sizeof(nk), cudaMemcpyHostToDevice, st));
    BGV_CUDA(cudaMemcpyAsync(w.K, &K, sizeof(K), cudaMemcpyHostToDevice, st));
    BGV_CUDA(cudaMemcpyAsync(w.flags + 2, &one, sizeof(one), cudaMemcpyHostToDevice, st));
    note_launch(), k_csr_reduce<<<1, kThreads, 0, st>>>(w.keys, w.nkeys, int64_t(nk), 1, w.K, w.csr_off, w.csr_adj,
                                                        w.start, w.supidx, w.ssrc, w.sdst, w.flags, w.agg, w.incl,
                                                        w.Es, w.nnz, dev_status, spin_limit());
    BGV_TRY(launch_status());
    return cudaStreamSynchronize(st) == cudaSuccess ? BGV_OK : BGV_ECUDA;
}

}  // namespace bgv

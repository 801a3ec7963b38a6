// communities.cu -- streaming community rounds (Algorithm 3, Section 3.2.1).
//
// Each round is two kernels.  The propose kernel streams the edge list
// (int4 loads, two edges per load), gathers the start-of-round (degree,
// label) pair of both endpoints as one 8-byte load each, applies the rule and
// offers the move to the joining node with a 64-bit atomicMin of
// (edge index << 32 | label): the lowest edge index wins whatever order the
// threads run in, so labels are bit-identical to the sequential oracle.  The
// apply kernel then updates every node that received a proposal and resets
// the proposal slot for the next round.  No state is written during a
// propose pass, so every edge reads the snapshot of the round.
//
// Batched form: each node also carries its graph's threshold, (degree,
// label, threshold) in one 16-byte word, so a propose still gathers one
// 32-byte sector per endpoint and graphs with different thresholds share a
// launch.  Edge indices and labels are global but ordered as inside each
// graph, so the winners are those of G separate runs.
#include "bgv_internal.cuh"

namespace bgv {
namespace {
constexpr int kThreads = 256;
constexpr unsigned long long kNone = ~0ull;


// The rule of one edge on the round's snapshot: returns the joining node w
// and the label it is offered, or -1 when the edge moves nothing.
__device__ __forceinline__ int32_t edge_rule(int32_t u, int32_t v, uint32_t du, uint32_t lu, uint32_t dv, uint32_t lv,
                                             uint32_t D, int tie_mode, uint32_t *lab) {
    if (du > D || dv > D) return -1;
    if (lu == lv) return -1;
    if (du > dv) {
        *lab = lu;
        return v;
    }
    if (dv > du) {
        *lab = lv;
        return u;
    }
    if (!tie_mode) return -1;
    *lab = u < v ? lv : lu;
    return u < v ? u : v;
}

__device__ __forceinline__ bool endpoints_ok(int32_t u, int32_t v, int32_t n, uint32_t *status) {
    if (static_cast<uint32_t>(u) >= static_cast<uint32_t>(n) || static_cast<uint32_t>(v) >= static_cast<uint32_t>(n)) {
        raise_status(status, BGV_DEV_BADEDGE);
        return false;
    }
    return u != v;
}

__device__ __forceinline__ void offer(unsigned long long *best, int32_t w, uint32_t e, uint32_t lab) {
    const unsigned long long cand = (static_cast<unsigned long long>(e) << 32) | lab;
    // The slot only decreases, so a stale read can only be larger than the
    // current value: skipping when cand is not below it is always safe.
    if (cand < __ldcg(&best[w])) atomicMin(&best[w], cand);
}

__device__ __forceinline__ void propose_edge(int32_t u, int32_t v, uint32_t e, int32_t n, const uint2 *state,
                                             unsigned long long *best, uint32_t D, int tie_mode,
                                             uint32_t *status) {
    if (!endpoints_ok(u, v, n, status)) return;
    // from L2: within the persistent kernel other blocks wrote them
    const uint2 su = __ldcg(&state[u]), sv = __ldcg(&state[v]);  // (degree, label)
    uint32_t lab;
    const int32_t w = edge_rule(u, v, su.x, su.y, sv.x, sv.y, D, tie_mode, &lab);
    if (w >= 0) offer(best, w, e, lab);
}

// Batched form: both endpoints belong to one graph, so the threshold
// carried by u is the graph's.
__device__ __forceinline__ void propose_edge_b(int32_t u, int32_t v, uint32_t e, int32_t n, const uint4 *state,
                                               unsigned long long *best, int tie_mode, uint32_t *status) {
    if (!endpoints_ok(u, v, n, status)) return;
    const uint4 su = __ldcg(&state[u]), sv = __ldcg(&state[v]);  // (degree, label, threshold, first threshold)
    uint32_t lab;
    const int32_t w = edge_rule(u, v, su.x, su.y, sv.x, sv.y, su.z, tie_mode, &lab);
    if (w >= 0) offer(best, w, e, lab);
}










// All rounds in one persistent kernel (cooperative launch, every block
// resident): initial state, then per round the proposals over the edge
// list, a grid barrier, the winning proposals applied (and the thresholds
// advanced), a barrier, the pointer-jumping steps (read, barrier, write,
// barrier), and at the end the labels.  The same per-edge and per-node rules
// as the kernels above, so the labels are the same bit for bit; the barrier
// waits are bounded and report BGV_DEV_TIMEOUT.  kB: the batched form (per
// node (degree, label, threshold, first threshold)).
template <bool kB>
__global__ void __launch_bounds__(kThreads) k_comm_rounds(const int32_t *__restrict__ edges, int64_t m, int32_t n,
                                                          const uint32_t *__restrict__ deg_est,
                                                          const int32_t *__restrict__ node_graph,
                                                          const uint32_t *__restrict__ D0, int32_t passes,
                                                          uint32_t threshold, uint32_t growth, int tie_mode,
                                                          int32_t jumps, uint2 *state, uint4 *bstate,
                                                          unsigned long long *best, uint32_t *jump,
                                                          int32_t *__restrict__ labels, uint32_t *__restrict__ deg_out,
                                                          uint32_t *status, WsHeader *hdr, int spin_limit) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t t0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    for (int64_t v = t0; v < n; v += stride) {
        if (kB) {
            const uint32_t d0 = D0[node_graph[v]];
            bstate[v] = make_uint4(deg_est[v], uint32_t(v), d0, d0);
        } else {
            state[v] = make_uint2(deg_est[v], uint32_t(v));
        }
        best[v] = kNone;
    }
    if (!grid_barrier(&hdr->bar, spin_limit, status)) return;
    const int4 *e2 = reinterpret_cast<const int4 *>(edges);
    const int64_t pairs = m >> 1;
    unsigned long long D = threshold;
    const unsigned long long factor = growth ? growth : threshold;
    for (int32_t p = 0; p < passes; ++p) {
        for (int64_t q = t0; q < pairs; q += stride) {
            const int4 e = __ldcs(e2 + q);
            if (kB) {
                propose_edge_b(e.x, e.y, uint32_t(2 * q), n, bstate, best, tie_mode, status);
                propose_edge_b(e.z, e.w, uint32_t(2 * q + 1), n, bstate, best, tie_mode, status);
            } else {
                propose_edge(e.x, e.y, uint32_t(2 * q), n, state, best, uint32_t(D), tie_mode, status);
                propose_edge(e.z, e.w, uint32_t(2 * q + 1), n, state, best, uint32_t(D), tie_mode, status);
            }
        }
        if ((m & 1) && t0 == 0) {
            if (kB)
                propose_edge_b(edges[2 * (m - 1)], edges[2 * (m - 1) + 1], uint32_t(m - 1), n, bstate, best, tie_mode,
                               status);
            else
                propose_edge(edges[2 * (m - 1)], edges[2 * (m - 1) + 1], uint32_t(m - 1), n, state, best, uint32_t(D),
                             tie_mode, status);
        }
        if (!grid_barrier(&hdr->bar, spin_limit, status)) return;
        for (int64_t v = t0; v < n; v += stride) {
            const unsigned long long b = __ldcg(&best[v]);
            if (kB) {
                uint4 st = bstate[v];
                if (b != kNone) {
                    st.y = static_cast<uint32_t>(b & 0xFFFFFFFFull);
                    if (st.x != 0xFFFFFFFFu) st.x += 1;
                    best[v] = kNone;
                }
                const unsigned long long nd = static_cast<unsigned long long>(st.z) * (growth ? growth : st.w);
                st.z = nd > 0xFFFFFFFFull ? 0xFFFFFFFFu : uint32_t(nd);
                bstate[v] = st;
            } else if (b != kNone) {
                uint2 st = state[v];
                st.y = static_cast<uint32_t>(b & 0xFFFFFFFFull);
                if (st.x != 0xFFFFFFFFu) st.x += 1;
                state[v] = st;
                best[v] = kNone;
            }
        }
        if (!grid_barrier(&hdr->bar, spin_limit, status)) return;
        for (int32_t j = 0; j < jumps; ++j) {
            for (int64_t v = t0; v < n; v += stride)
                jump[v] = kB ? __ldcg(&bstate[__ldcg(&bstate[v].y)].y) : __ldcg(&state[__ldcg(&state[v].y)].y);
            if (!grid_barrier(&hdr->bar, spin_limit, status)) return;
            for (int64_t v = t0; v < n; v += stride) {
                if (kB) bstate[v].y = __ldcg(&jump[v]);
                else state[v].y = __ldcg(&jump[v]);
            }
            if (!grid_barrier(&hdr->bar, spin_limit, status)) return;
        }
        D *= factor;
        if (D > 0xFFFFFFFFull) D = 0xFFFFFFFFull;
    }
    for (int64_t v = t0; v < n; v += stride) {
        const uint32_t d = kB ? __ldcg(&bstate[v].x) : __ldcg(&state[v].x);
        const uint32_t l = kB ? __ldcg(&bstate[v].y) : __ldcg(&state[v].y);
        labels[v] = int32_t(l);
        if (deg_out) deg_out[v] = d;
    }
}

// Mode degree (Section 4.2.2): the keys (graph << 32 | degree) are sorted;
// the end of every run of equal nonzero keys finds the run's start by binary
// search and offers (run length, complement of the degree) to its graph, so
// the longest run wins and ties go to the smaller degree.
__global__ void __launch_bounds__(kThreads) k_mode_keys(const uint32_t *__restrict__ deg, int32_t n,
                                                        const int32_t *__restrict__ node_graph,
                                                        unsigned long long *__restrict__ keys) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += stride) {
        const unsigned long long g = node_graph ? static_cast<unsigned long long>(node_graph[v]) : 0ull;
        keys[v] = (g << 32) | deg[v];
    }
}

__global__ void __launch_bounds__(kThreads) k_mode_runs(const unsigned long long *__restrict__ sorted, int32_t n,
                                                        unsigned long long *best) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long k = sorted[i];
        const uint32_t value = static_cast<uint32_t>(k & 0xFFFFFFFFull);
        if (value == 0 || (i + 1 < n && sorted[i + 1] == k)) continue;
        int64_t lo = 0, hi = i;  // first position holding k
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (sorted[mid] < k) lo = mid + 1; else hi = mid;
        }
        const unsigned long long len = static_cast<unsigned long long>(i - lo + 1);
        atomicMax(&best[k >> 32], (len << 32) | (0xFFFFFFFFull - value));
    }
}

__global__ void k_mode_out(const unsigned long long *__restrict__ best, int32_t G, uint32_t *__restrict__ mode) {
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
        mode[g] = best[g] ? uint32_t(0xFFFFFFFFull - (best[g] & 0xFFFFFFFFull)) : 0u;
}
}  // namespace

void carve_comm(Carver &c, int64_t m, int32_t n, CommScratch &s, bool batched) {
    (void)m;
    s.state = batched ? nullptr : c.take<uint2>(size_t(n));
    s.bstate = batched ? c.take<uint4>(size_t(n)) : nullptr;
    s.best = c.take<unsigned long long>(size_t(n));
    s.jump = c.take<uint32_t>(size_t(n));
}

void carve_mode(Carver &c, int32_t n, int32_t G, ModeScratch &s) {
    carve_sort(c, n, false, s.sort);
    s.best = c.take<unsigned long long>(size_t(G > 0 ? G : 1));
}

int run_mode_degree(const uint32_t *deg, int32_t n, const BatchView *batch, uint32_t *mode_dev,
                    const ModeScratch &s, uint32_t *status, cudaStream_t st) {
    const int32_t G = batch ? batch->G : 1;
    const int gn = grid_for(n, kThreads, sm_count() * 8);
    BGV_CUDA(cudaMemsetAsync(s.best, 0, sizeof(unsigned long long) * size_t(G), st));
    note_launch(), k_mode_keys<<<gn, kThreads, 0, st>>>(deg, n, batch ? batch->node_graph : nullptr,
                                                        s.sort.keys[0]);
    BGV_TRY(launch_status());
    SortBuffers sb = s.sort;
    int res = 0;
    BGV_TRY(radix_sort(sb, n, nullptr, 32 + (batch ? bits_for(G) : 0), st, &res, status));
    note_launch(), k_mode_runs<<<gn, kThreads, 0, st>>>(sb.keys[res], n, s.best);
    note_launch(), k_mode_out<<<grid_for(G, kThreads, sm_count()), kThreads, 0, st>>>(s.best, G, mode_dev);
    return launch_status();
}

int run_communities(const int32_t *edges, int64_t m, int32_t n, const uint32_t *deg_est, int32_t passes,
                    uint32_t threshold, uint32_t growth, int32_t tie_mode, int32_t jumps, int32_t *labels,
                    uint32_t *deg_out, const CommScratch &s, uint32_t *status, cudaStream_t st,
                    const BatchView *batch, WsHeader *hdr) {
    const int32_t *node_graph = batch ? batch->node_graph : nullptr;
    const uint32_t *D0 = batch ? batch->D0 : nullptr;
    uint2 *state = s.state;
    uint4 *bstate = s.bstate;
    unsigned long long *best = s.best;
    uint32_t *jump = s.jump;
    int tmode = tie_mode, limit = spin_limit();
    void *args[] = {&edges, &m, &n, &deg_est, &node_graph, &D0, &passes, &threshold, &growth, &tmode, &jumps,
                    &state, &bstate, &best, &jump, &labels, &deg_out, &status, &hdr, &limit};
    const void *kernel = batch ? reinterpret_cast<const void *>(k_comm_rounds<true>)
                               : reinterpret_cast<const void *>(k_comm_rounds<false>);
    const int blocks = coop_blocks(kernel, kThreads, sm_count() * 8);
    return launch_coop(kernel, blocks, kThreads, args, st);
}

}  // namespace bgv

// fa2.cu -- ForceAtlas2 on the supergraph (Section 3.1, Algorithm 1).
//
// One iteration is a fixed chain of kernels with no host round trip:
//   k_frame     bounding square of the positions (last-block finalise)
//   k_keys      fixed-point coordinates U and 2L-bit Morton keys
//   radix sort  (key, body) pairs -> Morton order
//   k_gather    bodies in Morton order (position, mass, fixed coords)
//   k_radix_tree binary radix tree over the sorted keys, one thread per
//               internal node (exponential + binary search on key prefixes)
//   k_mom_*     exact prefix sums of (m, m*Ux, m*Uy) in 64/128-bit integers
//               over the Morton order, so a node's moments are a difference
//   k_cells     quadtree cells: binary nodes whose 2-bit level exceeds their
//               parent's; FP32 centre of mass from the exact moments
//   k_preorder  cells and bodies laid out in depth-first pre-order with skip
//               indices (positions from a prefix count of cells per body)
//   k_repulse   Barnes-Hut repulsion: one warp per 32 Morton-consecutive
//               bodies walks the union of their traversals without a stack;
//               every lane takes its own opening decisions, so each body's
//               interaction set is exactly the one the definition gives
//   k_attract   attraction over fixed 8-entry chunks of the CSR (balanced
//               whatever the degrees), row pieces kept per chunk
//   k_node      per node: attraction pieces in chunk order, gravity, total
//               force, swing and traction (FP64, compensated); the last block
//               merges the block partials and updates the global speed
//   k_update    local speed, displacement, Fprev = F
//
// The opening test and the centre it uses are computed with explicit
// round-to-nearest FP32 operations (no contraction) from the exact integer
// moments, so the decisions do not depend on thread scheduling and equal
// the oracle's decisions on the same positions.
#include "bgv_internal.cuh"

namespace bgv {

namespace {
constexpr int kThreads = 256;
constexpr int kFrameBlocks = 304;      // 2 x 152 SMs
constexpr int kNodeBlocks = 152 * 8;  // node-kernel grid (rows are grid-strided)

typedef unsigned __int128 u128;


__device__ __forceinline__ unsigned long long spread_bits(uint32_t v) {
    unsigned long long x = v;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

// Exact power-of-two scale 2^-level for 0 <= level <= 126.
__device__ __forceinline__ float pow2_neg(int level) { return __int_as_float((127 - level) << 23); }

// ----------------------------------------------------------------- frame
__global__ void __launch_bounds__(kThreads) k_frame(const float2 *__restrict__ pos, int64_t K, float4 *part,
                                                    float4 *frame, unsigned int *ticket) {
    float lx = INFINITY, ly = INFINITY, hx = -INFINITY, hy = -INFINITY;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < K; i += stride) {
        const float2 p = pos[i];
        lx = fminf(lx, p.x); ly = fminf(ly, p.y);
        hx = fmaxf(hx, p.x); hy = fmaxf(hy, p.y);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        lx = fminf(lx, __shfl_xor_sync(0xFFFFFFFFu, lx, d));
        ly = fminf(ly, __shfl_xor_sync(0xFFFFFFFFu, ly, d));
        hx = fmaxf(hx, __shfl_xor_sync(0xFFFFFFFFu, hx, d));
        hy = fmaxf(hy, __shfl_xor_sync(0xFFFFFFFFu, hy, d));
    }
    __shared__ float4 wpart[kThreads / 32];
    __shared__ bool last;
    if ((threadIdx.x & 31) == 0) wpart[threadIdx.x >> 5] = make_float4(lx, ly, hx, hy);
    __syncthreads();
    if (threadIdx.x == 0) {
        float4 r = wpart[0];
        for (int w = 1; w < kThreads / 32; ++w) {
            r.x = fminf(r.x, wpart[w].x); r.y = fminf(r.y, wpart[w].y);
            r.z = fmaxf(r.z, wpart[w].z); r.w = fmaxf(r.w, wpart[w].w);
        }
        part[blockIdx.x] = r;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // the last block reduces the block partials, all threads at once
    // (min and max do not depend on the order)
    __threadfence();
    float4 r = make_float4(INFINITY, INFINITY, -INFINITY, -INFINITY);
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        const float4 q = __ldcg(&part[b]);
        r.x = fminf(r.x, q.x); r.y = fminf(r.y, q.y);
        r.z = fmaxf(r.z, q.z); r.w = fmaxf(r.w, q.w);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        r.x = fminf(r.x, __shfl_xor_sync(0xFFFFFFFFu, r.x, d));
        r.y = fminf(r.y, __shfl_xor_sync(0xFFFFFFFFu, r.y, d));
        r.z = fmaxf(r.z, __shfl_xor_sync(0xFFFFFFFFu, r.z, d));
        r.w = fmaxf(r.w, __shfl_xor_sync(0xFFFFFFFFu, r.w, d));
    }
    __syncthreads();  // wpart is reused
    if ((threadIdx.x & 31) == 0) wpart[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x != 0) return;
    r = wpart[0];
    for (int w = 1; w < kThreads / 32; ++w) {
        r.x = fminf(r.x, wpart[w].x); r.y = fminf(r.y, wpart[w].y);
        r.z = fmaxf(r.z, wpart[w].z); r.w = fmaxf(r.w, wpart[w].w);
    }
    const float ex = __fsub_rn(r.z, r.x), ey = __fsub_rn(r.w, r.y);
    const float ext = ex > ey ? ex : ey;
    float side = __fmul_rn(ext, 1.00000095367431640625f);  // 1 + 2^-20
    if (!(ext > 0.0f)) side = 1.0f;
    *frame = make_float4(r.x, r.y, side, 0.0f);
    *ticket = 0u;
}

// Batched form: one block per graph; graph g owns bodies [koff[g], koff[g+1]).
__global__ void __launch_bounds__(kThreads) k_frame_seg(const float2 *__restrict__ pos,
                                                        const int64_t *__restrict__ koff, float4 *__restrict__ frames,
                                                        int32_t *__restrict__ bgraph) {
    const int g = blockIdx.x;
    const int64_t a = koff[g], b = koff[g + 1];
    float lx = INFINITY, ly = INFINITY, hx = -INFINITY, hy = -INFINITY;
    for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
        const float2 p = pos[i];
        lx = fminf(lx, p.x); ly = fminf(ly, p.y);
        hx = fmaxf(hx, p.x); hy = fmaxf(hy, p.y);
        bgraph[i] = g;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        lx = fminf(lx, __shfl_xor_sync(0xFFFFFFFFu, lx, d));
        ly = fminf(ly, __shfl_xor_sync(0xFFFFFFFFu, ly, d));
        hx = fmaxf(hx, __shfl_xor_sync(0xFFFFFFFFu, hx, d));
        hy = fmaxf(hy, __shfl_xor_sync(0xFFFFFFFFu, hy, d));
    }
    __shared__ float4 wpart[kThreads / 32];
    if ((threadIdx.x & 31) == 0) wpart[threadIdx.x >> 5] = make_float4(lx, ly, hx, hy);
    __syncthreads();
    if (threadIdx.x != 0) return;
    float4 r = wpart[0];
    for (int w = 1; w < kThreads / 32; ++w) {
        r.x = fminf(r.x, wpart[w].x); r.y = fminf(r.y, wpart[w].y);
        r.z = fmaxf(r.z, wpart[w].z); r.w = fmaxf(r.w, wpart[w].w);
    }
    const float ex = __fsub_rn(r.z, r.x), ey = __fsub_rn(r.w, r.y);
    const float ext = ex > ey ? ex : ey;
    float side = __fmul_rn(ext, 1.00000095367431640625f);  // 1 + 2^-20
    if (!(ext > 0.0f)) side = 1.0f;
    frames[g] = make_float4(r.x, r.y, side, 0.0f);
}

// ------------------------------------------------------------------ keys
// Morton key of the body's fixed-point position in its graph's frame; in the
// batched form the graph id sits above the 2L Morton bits, so each graph's
// bodies stay together and form their own subtree.
__global__ void __launch_bounds__(kThreads) k_keys(const float2 *__restrict__ pos, int64_t K,
                                                   const float4 *__restrict__ frames,
                                                   const int32_t *__restrict__ bgraph, int L,
                                                   unsigned long long *__restrict__ keys,
                                                   uint32_t *__restrict__ vals, uint2 *__restrict__ U) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < K; i += stride) {
        const int g = bgraph ? bgraph[i] : 0;
        const float4 fr = frames[g];
        const float2 p = pos[i];
        const float ux = __fdiv_rn(__fsub_rn(p.x, fr.x), fr.z);
        const float uy = __fdiv_rn(__fsub_rn(p.y, fr.y), fr.z);
        const uint32_t Ux = __float2uint_rz(__fmul_rn(ux, 4294967296.0f));
        const uint32_t Uy = __float2uint_rz(__fmul_rn(uy, 4294967296.0f));
        const uint32_t qx = Ux >> (32 - L), qy = Uy >> (32 - L);
        keys[i] = (static_cast<unsigned long long>(g) << (2 * L)) | (spread_bits(qx) << 1) | spread_bits(qy);
        vals[i] = uint32_t(i);
        U[i] = make_uint2(Ux, Uy);
    }
}

__global__ void __launch_bounds__(kThreads) k_gather(const uint32_t *__restrict__ perm, int64_t K,
                                                     const float2 *__restrict__ pos,
                                                     const uint32_t *__restrict__ mass,
                                                     const uint2 *__restrict__ U, float4 *__restrict__ body,
                                                     uint2 *__restrict__ sU, uint32_t *__restrict__ smass) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < K; s += stride) {
        const uint32_t i = perm[s];
        const float2 p = pos[i];
        const uint32_t m = mass[i];
        body[s] = make_float4(p.x, p.y, __uint2float_rn(m), __int_as_float(int(i)));
        sU[s] = U[i];
        smass[s] = m;
    }
}

// ------------------------------------------------------------------ tree
// Binary radix tree over the Morton-sorted keys, built node-parallel: for
// internal node i (0 <= i < K-1) the direction, far end and split of its
// range are found by exponential and binary search on delta(i, j), the
// common-prefix length of keys i and j, with the positions breaking ties
// between equal keys (Karras, HPG 2012).  No node waits for another.
__device__ __forceinline__ int key_delta(const unsigned long long *__restrict__ keys, int64_t K, int keybits,
                                         int64_t i, unsigned long long ki, int64_t j) {
    if (j < 0 || j >= K) return -1;
    const unsigned long long kj = __ldg(&keys[j]);
    if (ki != kj) return __clzll(static_cast<long long>(ki ^ kj)) - (64 - keybits);
    return keybits + __clz(static_cast<int>(uint32_t(i) ^ uint32_t(j)));
}

__global__ void __launch_bounds__(kThreads) k_radix_tree(const unsigned long long *__restrict__ keys, int64_t K,
                                                         int L, int gbits, int32_t *__restrict__ left,
                                                         int32_t *__restrict__ right, int32_t *__restrict__ parent,
                                                         int2 *__restrict__ range, int8_t *__restrict__ level,
                                                         int32_t *__restrict__ root) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= K - 1) return;
    const int kb = 2 * L + gbits;
    const unsigned long long ki = __ldg(&keys[i]);
    const int d = key_delta(keys, K, kb, i, ki, i + 1) > key_delta(keys, K, kb, i, ki, i - 1) ? 1 : -1;
    const int dmin = key_delta(keys, K, kb, i, ki, i - d);
    int64_t lmax = 2;
    while (key_delta(keys, K, kb, i, ki, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (key_delta(keys, K, kb, i, ki, i + (l + t) * d) > dmin) l += t;
    const int64_t j = i + l * d;
    const int dnode = key_delta(keys, K, kb, i, ki, j);
    int64_t sp = 0;
    for (int64_t div = 2;; div <<= 1) {
        const int64_t t = (l + div - 1) / div;
        if (key_delta(keys, K, kb, i, ki, i + (sp + t) * d) > dnode) sp += t;
        if (t <= 1) break;
    }
    const int64_t gamma = i + sp * d + (d < 0 ? -1 : 0);
    const int64_t first = i < j ? i : j, last = i < j ? j : i;
    const int32_t lc = first == gamma ? ~int32_t(gamma) : int32_t(gamma);
    const int32_t rc = last == gamma + 1 ? ~int32_t(gamma + 1) : int32_t(gamma + 1);
    left[i] = lc;
    right[i] = rc;
    if (lc >= 0) parent[lc] = int32_t(i);
    if (rc >= 0) parent[rc] = int32_t(i);
    if (i == 0) {
        parent[0] = -1;
        *root = 0;
    }
    range[i] = make_int2(int32_t(first), int32_t(last));
    // 2-bit quadtree level below the graph bits; -1 above a graph's root
    level[i] = static_cast<int8_t>(dnode >= kb ? L : (dnode < gbits ? -1 : ((dnode - gbits) >> 1)));
}

// Exact moment prefix sums over the Morton order: P[s] = sum over bodies
// t < s of (m, m*Ux, m*Uy), in 64/128-bit integers, so every node's moments
// are P[last+1] - P[first] (exact, order-free).
constexpr int kMomItems = 8;
constexpr int kMomTile = kThreads * kMomItems;

struct Mom {
    unsigned long long M;
    u128 X, Y;
};
__device__ __forceinline__ Mom mom_add(Mom a, const Mom &b) {
    a.M += b.M;
    a.X += b.X;
    a.Y += b.Y;
    return a;
}
__device__ __forceinline__ Mom mom_shfl_up(const Mom &a, int d) {
    Mom r;
    r.M = __shfl_up_sync(0xFFFFFFFFu, a.M, d);
    const unsigned long long xl = __shfl_up_sync(0xFFFFFFFFu, static_cast<unsigned long long>(a.X), d);
    const unsigned long long xh = __shfl_up_sync(0xFFFFFFFFu, static_cast<unsigned long long>(a.X >> 64), d);
    const unsigned long long yl = __shfl_up_sync(0xFFFFFFFFu, static_cast<unsigned long long>(a.Y), d);
    const unsigned long long yh = __shfl_up_sync(0xFFFFFFFFu, static_cast<unsigned long long>(a.Y >> 64), d);
    r.X = (u128(xh) << 64) | xl;
    r.Y = (u128(yh) << 64) | yl;
    return r;
}
__device__ __forceinline__ Mom body_mom(const uint2 *sU, const uint32_t *smass, int64_t s, int64_t K) {
    Mom r{0ull, 0, 0};
    if (s < K) {
        const uint2 u = sU[s];
        const unsigned long long m = smass[s];
        r.M = m;
        r.X = u128(m) * u.x;
        r.Y = u128(m) * u.y;
    }
    return r;
}
__device__ __forceinline__ void mom_store(Mom v, unsigned long long *PM, ulonglong2 *PX, ulonglong2 *PY, int64_t s) {
    PM[s] = v.M;
    PX[s] = make_ulonglong2(static_cast<unsigned long long>(v.X), static_cast<unsigned long long>(v.X >> 64));
    PY[s] = make_ulonglong2(static_cast<unsigned long long>(v.Y), static_cast<unsigned long long>(v.Y >> 64));
}
__device__ __forceinline__ Mom mom_load(const unsigned long long *PM, const ulonglong2 *PX, const ulonglong2 *PY,
                                        int64_t s) {
    const ulonglong2 x = PX[s], y = PY[s];
    return Mom{PM[s], (u128(x.y) << 64) | x.x, (u128(y.y) << 64) | y.x};
}

// Block-wide exclusive scan of one Mom per thread; returns the prefix and
// the block total.
__device__ __forceinline__ Mom mom_block_exclusive(Mom v, Mom *total) {
    __shared__ unsigned long long sM[kThreads / 32];
    __shared__ ulonglong2 sX[kThreads / 32], sY[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Mom inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const Mom o = mom_shfl_up(inc, d);
        if (lane >= d) inc = mom_add(inc, o);
    }
    if (lane == 31) mom_store(inc, sM, sX, sY, warp);
    __syncthreads();
    Mom before{0ull, 0, 0}, all{0ull, 0, 0};
    for (int w = 0; w < kThreads / 32; ++w) {
        const Mom t = mom_load(sM, sX, sY, w);
        if (w < warp) before = mom_add(before, t);
        all = mom_add(all, t);
    }
    __syncthreads();
    *total = all;
    Mom ex = mom_add(before, inc);
    ex.M -= v.M;
    ex.X -= v.X;
    ex.Y -= v.Y;
    return ex;
}

__global__ void __launch_bounds__(kThreads) k_mom_reduce(const uint2 *__restrict__ sU,
                                                         const uint32_t *__restrict__ smass, int64_t K,
                                                         unsigned long long *__restrict__ TM,
                                                         ulonglong2 *__restrict__ TX, ulonglong2 *__restrict__ TY) {
    const int64_t s0 = int64_t(blockIdx.x) * kMomTile + int64_t(threadIdx.x) * kMomItems;
    Mom acc{0ull, 0, 0};
#pragma unroll
    for (int k = 0; k < kMomItems; ++k) acc = mom_add(acc, body_mom(sU, smass, s0 + k, K));
    Mom tot;
    mom_block_exclusive(acc, &tot);
    if (threadIdx.x == 0) mom_store(tot, TM, TX, TY, blockIdx.x);
}

__global__ void __launch_bounds__(kThreads) k_mom_tiles(unsigned long long *TM, ulonglong2 *TX, ulonglong2 *TY,
                                                        int64_t tiles) {
    Mom carry{0ull, 0, 0};
    for (int64_t base = 0; base < tiles; base += kThreads) {
        const int64_t t = base + threadIdx.x;
        const Mom v = t < tiles ? mom_load(TM, TX, TY, t) : Mom{0ull, 0, 0};
        Mom tot;
        const Mom ex = mom_block_exclusive(v, &tot);
        if (t < tiles) mom_store(mom_add(carry, ex), TM, TX, TY, t);
        carry = mom_add(carry, tot);
    }
}

__global__ void __launch_bounds__(kThreads) k_mom_down(const uint2 *__restrict__ sU,
                                                       const uint32_t *__restrict__ smass, int64_t K,
                                                       const unsigned long long *__restrict__ TM,
                                                       const ulonglong2 *__restrict__ TX,
                                                       const ulonglong2 *__restrict__ TY,
                                                       unsigned long long *__restrict__ PM,
                                                       ulonglong2 *__restrict__ PX, ulonglong2 *__restrict__ PY) {
    const int64_t s0 = int64_t(blockIdx.x) * kMomTile + int64_t(threadIdx.x) * kMomItems;
    Mom items[kMomItems];
    Mom acc{0ull, 0, 0};
#pragma unroll
    for (int k = 0; k < kMomItems; ++k) {
        items[k] = body_mom(sU, smass, s0 + k, K);
        acc = mom_add(acc, items[k]);
    }
    Mom tot;
    Mom run = mom_add(mom_load(TM, TX, TY, blockIdx.x), mom_block_exclusive(acc, &tot));
#pragma unroll
    for (int k = 0; k < kMomItems; ++k) {
        const int64_t s = s0 + k;
        if (s <= K) mom_store(run, PM, PX, PY, s);
        run = mom_add(run, items[k]);
    }
}

// Quadtree cells: the binary nodes whose 2-bit level exceeds their parent's
// (a chain of single-child cells collapses into its deepest cell, which
// takes the opening test for the whole chain).  For each cell: FP32 centre
// from the exact moments, mass, and the squared side used by the opening
// test (+inf for a leaf that is never accepted).  Cells are counted by their
// first body for the pre-order layout.
__global__ void __launch_bounds__(kThreads) k_cells(int64_t K, int L, int leaf_cap, const float4 *__restrict__ frames,
                                                    const int32_t *__restrict__ bgraph,
                                                    const int32_t *__restrict__ parent,
                                                    const int2 *__restrict__ range, const int8_t *__restrict__ level,
                                                    const unsigned long long *__restrict__ PM,
                                                    const ulonglong2 *__restrict__ PX,
                                                    const ulonglong2 *__restrict__ PY, float4 *__restrict__ cell,
                                                    int8_t *__restrict__ topflag, uint32_t *__restrict__ start_count,
                                                    unsigned long long *tree_nodes) {
    const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    bool top = false;
    if (p < K - 1) {
        const int lev = level[p];
        const int32_t par = parent[p];
        const int par_lev = (par < 0 || int64_t(par) >= K - 1) ? -1 : int(level[par]);
        top = par_lev < lev;
        topflag[p] = top ? 1 : 0;
        if (top) {
            const int2 rg = range[p];
            const int cnt = rg.y - rg.x + 1;
            const bool leaf = cnt <= leaf_cap || lev >= L;
            // A leaf made by the depth limit (coincident keys, more than
            // leaf_cap bodies) hides a chain of non-leaf cells with the same
            // bodies between its parent's level and L; the deepest of them,
            // at level L - 1, takes the opening test for the whole chain.
            const bool testable = leaf && cnt > leaf_cap && par_lev + 1 <= L - 1;
            // positions of graph g in Morton order are its index range too
            const float4 fr = frames[bgraph ? bgraph[rg.x] : 0];
            const Mom hi = mom_load(PM, PX, PY, rg.y + 1), lo = mom_load(PM, PX, PY, rg.x);
            const unsigned long long M = hi.M - lo.M;
            const u128 X = hi.X - lo.X, Y = hi.Y - lo.Y;
            const uint32_t qx = M ? uint32_t(X / M) : 0u, qy = M ? uint32_t(Y / M) : 0u;
            const float cx = __fadd_rn(fr.x, __fmul_rn(fr.z, __fmul_rn(__uint2float_rn(qx), 2.3283064365386963e-10f)));
            const float cy = __fadd_rn(fr.y, __fmul_rn(fr.z, __fmul_rn(__uint2float_rn(qy), 2.3283064365386963e-10f)));
            const float sl = __fmul_rn(fr.z, pow2_neg(testable ? L - 1 : lev));
            const float side2 = (leaf && !testable) ? INFINITY : __fmul_rn(sl, sl);
            cell[p] = make_float4(cx, cy, __ull2float_rn(M), side2);
            atomicAdd(&start_count[rg.x], 1u);
        }
    }
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, top);
    if ((threadIdx.x & 31) == 0 && mask) atomicAdd(tree_nodes, static_cast<unsigned long long>(__popc(mask)));
}

// Pre-order layout of cells and bodies.  With T[s] = number of cells whose
// first body precedes s (exclusive scan of the per-body counts):
//   body s           -> s + T[s+1]       (every cell starting at or before s
//                                          comes first)
//   cell [a, b]      -> a + T[a] + (its ancestors that also start at a)
//   skip(cell [a,b]) -> b + 1 + T[b+1]   (the element after its subtree)
// Elements are float4 (x, y, mass, side^2), side^2 = -1 for a body.
__global__ void __launch_bounds__(kThreads) k_preorder(int64_t K, const int32_t *__restrict__ parent,
                                                       const int2 *__restrict__ range,
                                                       const int8_t *__restrict__ topflag,
                                                       const float4 *__restrict__ cell,
                                                       const uint32_t *__restrict__ T,
                                                       const float4 *__restrict__ body, float4 *__restrict__ geo,
                                                       int32_t *__restrict__ skip) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t < K) {
        const int64_t pre = t + T[t + 1];
        const float4 b = body[t];
        geo[pre] = make_float4(b.x, b.y, b.z, -1.0f);
        skip[pre] = int32_t(pre + 1);
    }
    if (t < K - 1 && topflag[t]) {
        const int2 rg = range[t];
        int dep = 0;
        for (int32_t par = parent[t]; par >= 0 && int64_t(par) < K - 1; par = parent[par]) {
            if (range[par].x != rg.x) break;
            dep += topflag[par];
        }
        const int64_t pre = rg.x + int64_t(T[rg.x]) + dep;
        geo[pre] = cell[t];
        skip[pre] = int32_t(int64_t(rg.y) + 1 + T[rg.y + 1]);
    }
}

// -------------------------------------------------------------- repulsion
__device__ __forceinline__ void add_body(float xi, float yi, float kmi, float4 bj, float &fx, float &fy) {
    const float dx = xi - bj.x, dy = yi - bj.y;
    const float d2 = dx * dx + dy * dy;
    if (d2 > 0.0f) {
        const float f = __fdividef(kmi * bj.z, d2);
        fx += f * dx;
        fy += f * dy;
    }
}

// Barnes-Hut traversal without a stack.  A warp serves 32 * kBodiesPerLane
// Morton-consecutive bodies; each body keeps the pre-order index where its
// own traversal resumes.  Each step the warp takes the smallest resume index
// (one redux), loads that element once for all lanes, and only the bodies
// waiting at it act: a body is summed directly (not self) and passed; a cell
// holding the body is entered; any other cell is accepted (summed, resume
// after its subtree) or entered, by the FP32 opening test of the definition.
// Each body therefore sees exactly its own interaction set, in depth-first
// order.
constexpr int kBodiesPerLane = 1;

struct Walker {
    float xi, yi, kmi;
    uint32_t self, resume, end;
    float fx, fy;
    unsigned inter;
};

__device__ __forceinline__ void walker_step(Walker &b, uint32_t cur, float4 e, uint32_t sk, float theta2) {
    if (b.resume != cur) return;
    b.resume = cur + 1;
    if (e.w < 0.0f) {  // a body
        if (cur != b.self) {
            add_body(b.xi, b.yi, b.kmi, e, b.fx, b.fy);
            ++b.inter;
        }
    } else if (!(b.self > cur && b.self < sk)) {  // a cell not holding this body
        const float dx = __fsub_rn(b.xi, e.x), dy = __fsub_rn(b.yi, e.y);
        const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        if (e.w < __fmul_rn(theta2, d2)) {
            const float f = __fdividef(b.kmi * e.z, d2);
            b.fx += f * dx;
            b.fy += f * dy;
            ++b.inter;
            b.resume = sk;
        }
    }
    if (b.resume >= b.end) b.resume = 0xFFFFFFFFu;  // left its graph's subtree: done
}

__global__ void __launch_bounds__(kThreads) k_repulse(const float4 *__restrict__ geo, const int32_t *__restrict__ skip,
                                                      const uint32_t *__restrict__ T,
                                                      const int64_t *__restrict__ koff,
                                                      const int32_t *__restrict__ bgraph,
                                                      const float4 *__restrict__ body, int64_t K, float kr,
                                                      float theta2, float2 *__restrict__ Frep,
                                                      unsigned long long *inter_step,
                                                      unsigned long long *inter_total) {
    constexpr int kWarpBodies = 32 * kBodiesPerLane;
    const int lane = threadIdx.x & 31;
    const int64_t s0 = ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * kWarpBodies;
    if (s0 >= K) return;  // whole warp leaves together
    const uint32_t total = uint32_t(K + T[K]);
    Walker w[kBodiesPerLane];
#pragma unroll
    for (int q = 0; q < kBodiesPerLane; ++q) {
        const int64_t s = s0 + q * 32 + lane;
        const bool active = s < K;
        const float4 bi = active ? body[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        w[q].xi = bi.x;
        w[q].yi = bi.y;
        w[q].kmi = kr * bi.z;
        w[q].self = active ? uint32_t(s + T[s + 1]) : 0xFFFFFFFFu;
        // the body's own graph: its subtree spans [start, end) in pre-order
        uint32_t start = 0, end = total;
        if (active && bgraph) {
            const int g = bgraph[s];
            const int64_t a = koff[g], b = koff[g + 1];
            start = uint32_t(a + T[a]);
            end = uint32_t(b + T[b]);
        }
        w[q].end = end;
        w[q].resume = active ? start : 0xFFFFFFFFu;
        w[q].fx = 0.0f;
        w[q].fy = 0.0f;
        w[q].inter = 0;
    }
    while (true) {
        uint32_t mine = w[0].resume;
#pragma unroll
        for (int q = 1; q < kBodiesPerLane; ++q) mine = min(mine, w[q].resume);
        const uint32_t cur = __reduce_min_sync(0xFFFFFFFFu, mine);
        if (cur >= total) break;
        if (mine != cur) continue;
        const float4 e = geo[cur];
        const uint32_t sk = uint32_t(skip[cur]);
#pragma unroll
        for (int q = 0; q < kBodiesPerLane; ++q) walker_step(w[q], cur, e, sk, theta2);
    }
    unsigned inter = 0;
#pragma unroll
    for (int q = 0; q < kBodiesPerLane; ++q) {
        const int64_t s = s0 + q * 32 + lane;
        if (s < K) Frep[__float_as_int(body[s].w)] = make_float2(w[q].fx, w[q].fy);
        inter += w[q].inter;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) inter += __shfl_xor_sync(0xFFFFFFFFu, inter, d);
    if (lane == 0 && inter) {
        atomicAdd(inter_step, static_cast<unsigned long long>(inter));
        atomicAdd(inter_total, static_cast<unsigned long long>(inter));
    }
}

// ------------------------------------------------------------ attraction
// The CSR entries are cut into fixed chunks of kChunk consecutive entries,
// one chunk per thread whatever the row lengths (a hub row spreads over many
// threads, short rows share one).  A thread finds the row of its first entry
// by binary search on the offsets and walks its entries accumulating
// w_ij (p_j - p_i).  A row that starts and ends inside the chunk is written
// to `full`; the piece of a row that continues past the chunk goes to
// tail[chunk], the piece of a row that began before it to head[chunk].
// k_node adds a row's pieces in chunk order, so the sum order is fixed.
constexpr int kChunk = 8;

// The plan, written once per CSR:
//   chunk_row[g]   row of chunk g's first entry (the thread of row r writes r
//                  into every chunk that starts inside the row; a warp shares
//                  the writes of rows that cover many chunks);
//   chunk_meta[g]  byte k (1..7): row of entry k minus chunk_row[g]; byte 0:
//                  kMetaHead (the first row began in an earlier chunk),
//                  kMetaTail (the last row goes on into the next chunk),
//                  kMetaWalk (a row gap above 255: the chunk walks the
//                  offsets instead);
//   long_rows      the rows spread over more than kLongRowChunks chunks.
// With the rows of all 8 entries known up front, every load of a chunk is
// issued at once; no dependent walk over the row offsets.
constexpr int kLongRowChunks = 32;
constexpr unsigned kMetaHead = 1u, kMetaTail = 2u, kMetaWalk = 4u;

__global__ void __launch_bounds__(kThreads) k_chunk_rows(int64_t K, int64_t nnz, const int32_t *__restrict__ off,
                                                         int32_t *__restrict__ chunk_row, int32_t *__restrict__ long_rows,
                                                         int32_t *long_count) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t base = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) & ~int64_t(31); base < K; base += stride) {
        const int64_t r = base + lane;
        int64_t g0 = 0, g1 = 0;
        bool spread = false;
        if (r < K) {
            const int64_t b = off[r], e = off[r + 1] < nnz ? off[r + 1] : nnz;
            g0 = (b + kChunk - 1) / kChunk;
            g1 = (e + kChunk - 1) / kChunk;
            spread = e > b && (e - 1) / kChunk - b / kChunk > kLongRowChunks;
        }
        if (spread) long_rows[atomicAdd(long_count, 1)] = int32_t(r);
        const bool longrow = g1 - g0 > kLongRowChunks;
        if (!longrow)
            for (int64_t g = g0; g < g1; ++g) chunk_row[g] = int32_t(r);
        unsigned lm = __ballot_sync(0xFFFFFFFFu, longrow);
        while (lm) {
            const int src = __ffs(lm) - 1;
            lm &= lm - 1;
            const int64_t a = __shfl_sync(0xFFFFFFFFu, g0, src), z = __shfl_sync(0xFFFFFFFFu, g1, src);
            for (int64_t g = a + lane; g < z; g += 32) chunk_row[g] = int32_t(base + src);
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_chunk_meta(int64_t K, int64_t nnz, const int32_t *__restrict__ off,
                                                         const int32_t *__restrict__ chunk_row,
                                                         unsigned long long *__restrict__ chunk_meta) {
    const int64_t chunks = (nnz + kChunk - 1) / kChunk;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < chunks; g += stride) {
        const int64_t e0 = g * kChunk, e1 = e0 + kChunk < nnz ? e0 + kChunk : nnz;
        const int64_t r0 = chunk_row[g];
        unsigned long long meta = off[r0] < e0 ? kMetaHead : 0u;
        int64_t r = r0;
        for (int64_t e = e0 + 1; e < e1; ++e) {
            while (r + 1 < K && e >= off[r + 1]) ++r;
            const int64_t d = r - r0;
            if (d > 255) meta |= kMetaWalk;
            meta |= static_cast<unsigned long long>(d > 255 ? 255 : d) << (8 * (e - e0));
        }
        if (off[r + 1] > e1) meta |= kMetaTail;
        chunk_meta[g] = meta;
    }
}

// A row segment of a chunk goes to head[g] if it continues a row from an
// earlier chunk, to tail[g] if its row goes on past the chunk, else it is
// the whole row.
__device__ __forceinline__ void put_piece(bool first, bool last, unsigned flags, int64_t g, int64_t row, float ax,
                                          float ay, float2 *full, float2 *head, float2 *tail) {
    const float2 v = make_float2(ax, ay);
    if (first && (flags & kMetaHead)) head[g] = v;
    else if (last && (flags & kMetaTail)) tail[g] = v;
    else full[row] = v;
}

__global__ void __launch_bounds__(kThreads, 4) k_attract(int64_t K, int64_t nnz, const int32_t *__restrict__ off,
                                                      const int32_t *__restrict__ chunk_row,
                                                      const unsigned long long *__restrict__ chunk_meta,
                                                      const int32_t *__restrict__ adj,
                                                      const uint32_t *__restrict__ w, const float2 *__restrict__ pos,
                                                      float2 *__restrict__ full, float2 *__restrict__ head,
                                                      float2 *__restrict__ tail) {
    const int64_t chunks = (nnz + kChunk - 1) / kChunk;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(adj) | reinterpret_cast<uintptr_t>(w)) & 15) == 0;
    for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < chunks; g += stride) {
        const int64_t e0 = g * kChunk, e1 = e0 + kChunk < nnz ? e0 + kChunk : nnz;
        const int n = int(e1 - e0);
        const int64_t r0 = chunk_row[g];
        const unsigned long long meta = chunk_meta[g];
        const unsigned flags = unsigned(meta & 0xFFu);
        // All loads of the chunk first: 8 neighbour ids and weights (two
        // 16-byte loads each when aligned), then the 8 neighbour and 8 row
        // position gathers, so they are in flight together.
        int32_t jj[kChunk];
        uint32_t ww[kChunk];
        if (vec && n == kChunk) {
            const int4 a0 = __ldcs(reinterpret_cast<const int4 *>(adj + e0));
            const int4 a1 = __ldcs(reinterpret_cast<const int4 *>(adj + e0) + 1);
            const uint4 w0 = __ldcs(reinterpret_cast<const uint4 *>(w + e0));
            const uint4 w1 = __ldcs(reinterpret_cast<const uint4 *>(w + e0) + 1);
            jj[0] = a0.x; jj[1] = a0.y; jj[2] = a0.z; jj[3] = a0.w;
            jj[4] = a1.x; jj[5] = a1.y; jj[6] = a1.z; jj[7] = a1.w;
            ww[0] = w0.x; ww[1] = w0.y; ww[2] = w0.z; ww[3] = w0.w;
            ww[4] = w1.x; ww[5] = w1.y; ww[6] = w1.z; ww[7] = w1.w;
        } else {
#pragma unroll
            for (int k = 0; k < kChunk; ++k) {
                jj[k] = k < n ? adj[e0 + k] : -1;
                ww[k] = k < n ? w[e0 + k] : 0u;
            }
        }
        float2 pj[kChunk];
#pragma unroll
        for (int k = 0; k < kChunk; ++k)
            pj[k] = static_cast<uint64_t>(jj[k]) < static_cast<uint64_t>(K) ? pos[jj[k]] : make_float2(0.f, 0.f);
        if (!(flags & kMetaWalk)) {
            int32_t rk[kChunk];
            float2 pr[kChunk];
#pragma unroll
            for (int k = 0; k < kChunk; ++k) {
                rk[k] = int32_t(r0) + int32_t(k ? unsigned(meta >> (8 * k)) & 0xFFu : 0u);
                pr[k] = k < n ? pos[rk[k]] : make_float2(0.f, 0.f);
            }
            float ax = 0.0f, ay = 0.0f;
            bool first = true;
            int32_t row = rk[0];
#pragma unroll
            for (int k = 0; k < kChunk; ++k) {
                if (k < n) {
                    if (rk[k] != row) {
                        put_piece(first, false, flags, g, row, ax, ay, full, head, tail);
                        first = false;
                        row = rk[k];
                        ax = 0.0f;
                        ay = 0.0f;
                    }
                    if (static_cast<uint64_t>(jj[k]) < static_cast<uint64_t>(K)) {  // else an invalid CSR entry
                        const float wt = __uint2float_rn(ww[k]);
                        ax += wt * (pj[k].x - pr[k].x);
                        ay += wt * (pj[k].y - pr[k].y);
                    }
                }
            }
            put_piece(first, true, flags, g, row, ax, ay, full, head, tail);
            continue;
        }
        // Rows far apart (long runs of empty rows): walk the offsets.
        int64_t r = r0;
        int64_t rs = off[r], re = off[r + 1];
        float2 pi = pos[r];
        float ax = 0.0f, ay = 0.0f;
#pragma unroll
        for (int k = 0; k < kChunk; ++k) {
            if (k >= n) break;
            const int64_t e = e0 + k;
            while (e >= re && r + 1 < K) {  // row r ends before e: hand it over
                if (rs >= e0) full[r] = make_float2(ax, ay);  // started here: complete
                else head[g] = make_float2(ax, ay);
                ++r;
                rs = re;
                re = off[r + 1];
                pi = pos[r];
                ax = 0.0f;
                ay = 0.0f;
            }
            if (static_cast<uint64_t>(jj[k]) >= static_cast<uint64_t>(K)) continue;  // invalid CSR entry
            const float wt = __uint2float_rn(ww[k]);
            ax += wt * (pj[k].x - pi.x);
            ay += wt * (pj[k].y - pi.y);
        }
        if (rs >= e0 && re <= e1) full[r] = make_float2(ax, ay);
        else if (rs < e0) head[g] = make_float2(ax, ay);
        else tail[g] = make_float2(ax, ay);
    }
}

// Rows spread over more than kLongRowChunks chunks, one warp each: the
// lanes add strided subsets of the row's middle pieces in chunk order, then
// a fixed butterfly, then the row's first piece.  k_node reads the result
// from full[].
__global__ void __launch_bounds__(kThreads) k_long_rows(const int32_t *__restrict__ off,
                                                        const int32_t *__restrict__ long_rows,
                                                        const int32_t *__restrict__ long_count,
                                                        const float2 *__restrict__ head,
                                                        const float2 *__restrict__ tail, float2 *__restrict__ full) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int64_t count = *long_count;
    for (int64_t q = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; q < count; q += warps) {
        const int32_t r = long_rows[q];
        const int64_t a = off[r] / kChunk, z = (off[r + 1] - 1) / kChunk;
        float px = 0.0f, py = 0.0f;
#pragma unroll 4
        for (int64_t g = a + 1 + lane; g <= z; g += 32) {
            const float2 v = head[g];
            px += v.x;
            py += v.y;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            px += __shfl_xor_sync(0xFFFFFFFFu, px, d);
            py += __shfl_xor_sync(0xFFFFFFFFu, py, d);
        }
        if (lane == 0) {
            const float2 t = tail[a];
            full[r] = make_float2(t.x + px, t.y + py);
        }
    }
}

// --------------------------------------------- node forces, swing, speed
// Neumaier-compensated FP64 accumulation; merging two partial sums keeps
// both compensations.  Used in a fixed order, so results are reproducible.
struct Comp {
    double s, c;
};
__device__ __forceinline__ Comp comp_add(Comp a, double x) {
    const double t = a.s + x;
    const double e = fabs(a.s) >= fabs(x) ? (a.s - t) + x : (x - t) + a.s;
    return Comp{t, a.c + e};
}
__device__ __forceinline__ Comp comp_merge(Comp a, Comp b) {
    const double t = a.s + b.s;
    const double e = fabs(a.s) >= fabs(b.s) ? (a.s - t) + b.s : (b.s - t) + a.s;
    return Comp{t, a.c + b.c + e};
}
__device__ __forceinline__ Comp comp_shfl_down(Comp a, int d) {
    return Comp{__shfl_down_sync(0xFFFFFFFFu, a.s, d), __shfl_down_sync(0xFFFFFFFFu, a.c, d)};
}

// Block-wide merge of one (S, T) pair per thread, in a fixed tree; thread 0
// receives the result.
__device__ __forceinline__ void block_merge(Comp &S, Comp &T) {
    __shared__ Comp sS[kThreads / 32], sT[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const Comp oS = comp_shfl_down(S, d), oT = comp_shfl_down(T, d);
        S = comp_merge(S, oS);
        T = comp_merge(T, oT);
    }
    if (lane == 0) {
        sS[warp] = S;
        sT[warp] = T;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kThreads / 32; ++k) {
            S = comp_merge(S, sS[k]);
            T = comp_merge(T, sT[k]);
        }
    }
    __syncthreads();
}

// Block sum of one (S, T) pair per thread in plain FP64 (fixed tree);
// thread 0 receives it.  Compensation is applied where the block sums meet.
__device__ __forceinline__ void block_sum_plain(double &S, double &T) {
    __shared__ double sS[kThreads / 32], sT[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        S += __shfl_down_sync(0xFFFFFFFFu, S, d);
        T += __shfl_down_sync(0xFFFFFFFFu, T, d);
    }
    if (lane == 0) {
        sS[warp] = S;
        sT[warp] = T;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kThreads / 32; ++k) {
            S += sS[k];
            T += sT[k];
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads) k_node(int mode, int64_t K, const int32_t *__restrict__ off,
                                                   const float2 *__restrict__ full, const float2 *__restrict__ head,
                                                   const float2 *__restrict__ tail,
                                                   const uint32_t *__restrict__ mass, const float2 *__restrict__ pos,
                                                   const float2 *__restrict__ Frep, float kg, int strong,
                                                   float2 *__restrict__ F, const float2 *__restrict__ Fprev,
                                                   float2 *__restrict__ Fr_out, float2 *__restrict__ Fa_out,
                                                   float2 *__restrict__ Fg_out, double2 *part, double *speed,
                                                   float tau, WsHeader *hdr, float2 *__restrict__ rowst) {
    Comp S{0.0, 0.0}, T{0.0, 0.0};
    const int lane = threadIdx.x & 31;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t base = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) & ~int64_t(31); base < K; base += stride) {
        const int64_t i = base + lane;
        const bool valid = i < K;
        int64_t g1 = 0, g2 = -1;
        float ax = 0.0f, ay = 0.0f;
        // independent per-node loads first, so they overlap the piece sums
        float2 pi = make_float2(0.f, 0.f), fr = pi, fp = pi;
        uint32_t mi = 0;
        if (valid) {
            const int64_t b = off[i], e = off[i + 1];
            pi = pos[i];
            mi = mass[i];
            fr = Frep[i];
            if (mode != 0) fp = Fprev[i];
            if (e > b) {
                g1 = b / kChunk;
                g2 = (e - 1) / kChunk;
            }
        }
        // rows over many chunks were summed by k_long_rows into full[]
        if (valid && g2 >= g1) {
            if (g1 == g2 || g2 - g1 > kLongRowChunks) {
                const float2 v = full[i];
                ax = v.x;
                ay = v.y;
            } else {
                float2 v = tail[g1];
                ax = v.x;
                ay = v.y;
                for (int64_t g = g1 + 1; g <= g2; ++g) {
                    v = head[g];
                    ax += v.x;
                    ay += v.y;
                }
            }
        }
        if (!valid) continue;
        const float m = __uint2float_rn(mi);
        float gx, gy;
        if (strong) {
            gx = -kg * m * pi.x;
            gy = -kg * m * pi.y;
        } else {
            const float rr = sqrtf(pi.x * pi.x + pi.y * pi.y);
            gx = rr > 0.0f ? -kg * m * pi.x / rr : 0.0f;
            gy = rr > 0.0f ? -kg * m * pi.y / rr : 0.0f;
        }
        if (mode == 0) {
            if (Fr_out) Fr_out[i] = fr;
            if (Fa_out) Fa_out[i] = make_float2(ax, ay);
            if (Fg_out) Fg_out[i] = make_float2(gx, gy);
        } else {
            const float fx = fr.x + ax + gx, fy = fr.y + ay + gy;
            F[i] = make_float2(fx, fy);
            const float sx = fx - fp.x, sy = fy - fp.y, tx = fx + fp.x, ty = fy + fp.y;
            // per-node products in FP32; the sums over nodes are FP64
            const float msw = m * sqrtf(sx * sx + sy * sy), mtr = 0.5f * m * sqrtf(tx * tx + ty * ty);
            if (rowst) {
                rowst[i] = make_float2(msw, mtr);  // batched: summed per graph
            } else {
                S.s += double(msw);
                T.s += double(mtr);
            }
        }
    }
    if (mode == 0 || rowst) return;
    __shared__ bool last;
    block_sum_plain(S.s, T.s);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = make_double2(S.s, 0.0);
        part[2 * blockIdx.x + 1] = make_double2(T.s, 0.0);
        __threadfence();
        last = atomicAdd(&hdr->node_ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // The last block merges the block partials: each thread a strided subset
    // in block order, then the fixed block tree.
    Comp aS{0.0, 0.0}, aT{0.0, 0.0};
    for (unsigned bk = threadIdx.x; bk < gridDim.x; bk += blockDim.x) {
        const double2 ps = __ldcg(&part[2 * bk]), pt = __ldcg(&part[2 * bk + 1]);
        aS = comp_merge(aS, Comp{ps.x, ps.y});
        aT = comp_merge(aT, Comp{pt.x, pt.y});
    }
    block_merge(aS, aT);
    if (threadIdx.x != 0) return;
    const double Ssum = aS.s + aS.c, Tsum = aT.s + aT.c;
    double sp = *speed;
    if (Ssum > 0.0) {
        const double target = double(tau) * Tsum / Ssum;
        const double rise = target - sp, cap = 0.5 * sp;
        sp += rise < cap ? rise : cap;
    }
    *speed = sp;
    hdr->S = Ssum;
    hdr->T = Tsum;
    hdr->steps_total += 1;
    hdr->node_ticket = 0u;
}

// Batched form: one block per graph sums its rows' swing and traction (FP64,
// compensated, fixed order) and updates that graph's speed.
__global__ void __launch_bounds__(kThreads) k_speed_seg(const float2 *__restrict__ rowst,
                                                        const int64_t *__restrict__ koff, double *speed, float tau,
                                                        WsHeader *hdr) {
    const int g = blockIdx.x;
    const int64_t a = koff[g], b = koff[g + 1];
    Comp S{0.0, 0.0}, T{0.0, 0.0};
    for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
        const float2 v = rowst[i];
        S = comp_add(S, double(v.x));
        T = comp_add(T, double(v.y));
    }
    block_merge(S, T);
    if (threadIdx.x != 0) return;
    const double Ssum = S.s + S.c, Tsum = T.s + T.c;
    double sp = speed[g];
    if (Ssum > 0.0) {
        const double target = double(tau) * Tsum / Ssum;
        const double rise = target - sp, cap = 0.5 * sp;
        sp += rise < cap ? rise : cap;
    }
    speed[g] = sp;
    if (g == 0) {
        hdr->S = Ssum;
        hdr->T = Tsum;
        hdr->steps_total += 1;
    }
}

__global__ void __launch_bounds__(kThreads) k_update(int64_t K, const float2 *__restrict__ F, float2 *__restrict__ Fprev,
                                                     float2 *__restrict__ pos, const double *__restrict__ speed,
                                                     const int32_t *__restrict__ bgraph, float ks, float ksmax) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < K; i += stride) {
        const float sp = float(speed[bgraph ? bgraph[i] : 0]);
        const float2 f = F[i], fp = Fprev[i];
        const float sx = f.x - fp.x, sy = f.y - fp.y;
        const float swing = sqrtf(sx * sx + sy * sy);
        float s = ks * sp / (1.0f + sp * sqrtf(swing));
        const float fn = sqrtf(f.x * f.x + f.y * f.y);
        if (fn > 0.0f && s * fn > ksmax) s = ksmax / fn;
        float2 p = pos[i];
        p.x += s * f.x;
        p.y += s * f.y;
        pos[i] = p;
        Fprev[i] = f;
    }
}

// -------------------------------------------------------------------- init
__global__ void __launch_bounds__(kThreads) k_init(int64_t K, unsigned long long seed, float R, float2 *pos,
                                                   float2 *Fprev) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const float R2 = __fmul_rn(R, 2.0f);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < K; i += stride) {
        float c[2];
#pragma unroll
        for (int axis = 0; axis < 2; ++axis) {
            unsigned long long z = seed + 2ull * static_cast<unsigned long long>(i) + unsigned(axis);
            z += 0x9E3779B97F4A7C15ull;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            const float U = __fmul_rn(__uint2float_rn(uint32_t(z >> 40)), 5.9604644775390625e-08f);  // 2^-24
            c[axis] = __fsub_rn(__fmul_rn(U, R2), R);
        }
        pos[i] = make_float2(c[0], c[1]);
        Fprev[i] = make_float2(0.0f, 0.0f);
    }
}

__global__ void k_set_speed(double *speed) { *speed = 1.0; }

// Batched form: graph g starts exactly as it would alone (local index, its
// own square of side 2 sqrt(K_g)) with speed 1.
__global__ void __launch_bounds__(kThreads) k_init_seg(const int64_t *__restrict__ koff, unsigned long long seed,
                                                       float2 *pos, float2 *Fprev, double *speed) {
    const int g = blockIdx.x;
    const int64_t a = koff[g], b = koff[g + 1];
    const float R = sqrtf(float(b - a));
    const float R2 = __fmul_rn(R, 2.0f);
    for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
        const int64_t local = i - a;
        float c[2];
#pragma unroll
        for (int axis = 0; axis < 2; ++axis) {
            unsigned long long z = seed + 2ull * static_cast<unsigned long long>(local) + unsigned(axis);
            z += 0x9E3779B97F4A7C15ull;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            const float U = __fmul_rn(__uint2float_rn(uint32_t(z >> 40)), 5.9604644775390625e-08f);  // 2^-24
            c[axis] = __fsub_rn(__fmul_rn(U, R2), R);
        }
        pos[i] = make_float2(c[0], c[1]);
        Fprev[i] = make_float2(0.0f, 0.0f);
    }
    if (threadIdx.x == 0) speed[g] = 1.0;
}
}  // namespace

// ------------------------------------------------------------- scratch
struct Fa2Scratch {
    float4 *frame;         // frames: one per graph
    float4 *frame_part;
    int32_t *bgraph;       // batched form: graph of each body
    float2 *rowst;         // batched form: per-row swing, traction
    SortBuffers sort;
    uint2 *U;
    float4 *body;
    uint2 *sU;
    uint32_t *smass;
    int32_t *left, *right, *parent, *root;
    int2 *range;
    int8_t *level;
    unsigned long long *PM, *TM;   // moment prefix sums, per-tile sums
    ulonglong2 *PX, *PY, *TX, *TY;
    float4 *cell;          // per binary node: centre, mass, side^2 (cells only)
    int8_t *topflag;       // per binary node: is a quadtree cell
    uint32_t *start_count; // cells per first body
    uint32_t *T;           // exclusive scan of start_count, K + 1 entries
    void *scan_tmp;
    float4 *geo;           // pre-order elements (cells and bodies)
    int32_t *skip;         // pre-order index after each element's subtree
    float2 *Frep;
    float2 *full, *head, *tail;
    int32_t *chunk_row;   // plan: row of each chunk's first entry
    unsigned long long *chunk_meta;  // plan: rows of the chunk's entries, flags
    int32_t *long_rows;   // plan: rows over more than kLongRowChunks chunks
    int32_t *long_count;
    double2 *part;  // two per block: (S, comp), (T, comp)
};

static void carve_fa2(Carver &c, int64_t K, int64_t nnz, int32_t G, Fa2Scratch &s) {
    const size_t k = size_t(K > 0 ? K : 1);
    const size_t chunks = size_t((nnz > 0 ? nnz : 1) + kChunk - 1) / kChunk;
    const bool batched = G > 1;
    s.frame = c.take<float4>(size_t(G > 1 ? G : 1));
    s.frame_part = c.take<float4>(kFrameBlocks);
    s.bgraph = batched ? c.take<int32_t>(k) : nullptr;
    s.rowst = batched ? c.take<float2>(k) : nullptr;
    carve_sort(c, int64_t(k), true, s.sort);
    s.U = c.take<uint2>(k);
    s.body = c.take<float4>(k);
    s.sU = c.take<uint2>(k);
    s.smass = c.take<uint32_t>(k);
    const size_t tiles = (k + kMomTile - 1) / kMomTile;
    s.left = c.take<int32_t>(k);
    s.right = c.take<int32_t>(k);
    s.parent = c.take<int32_t>(k);
    s.root = c.take<int32_t>(1);
    s.range = c.take<int2>(k);
    s.level = c.take<int8_t>(k);
    s.PM = c.take<unsigned long long>(k + 1);
    s.PX = c.take<ulonglong2>(k + 1);
    s.PY = c.take<ulonglong2>(k + 1);
    s.TM = c.take<unsigned long long>(tiles);
    s.TX = c.take<ulonglong2>(tiles);
    s.TY = c.take<ulonglong2>(tiles);
    s.cell = c.take<float4>(k);
    s.topflag = c.take<int8_t>(k);
    s.start_count = c.take<uint32_t>(k + 1);
    s.T = c.take<uint32_t>(k + 1);
    s.scan_tmp = c.take<char>(scan_tmp_bytes(int64_t(k) + 1));
    s.geo = c.take<float4>(2 * k);
    s.skip = c.take<int32_t>(2 * k);
    s.Frep = c.take<float2>(k);
    s.full = c.take<float2>(k);
    s.head = c.take<float2>(chunks);
    s.tail = c.take<float2>(chunks);
    s.chunk_row = c.take<int32_t>(chunks);
    s.chunk_meta = c.take<unsigned long long>(chunks);
    s.long_rows = c.take<int32_t>(chunks / kLongRowChunks + 1);
    s.long_count = c.take<int32_t>(1);
    s.part = c.take<double2>(2 * kNodeBlocks);
}

size_t fa2_scratch_bytes(int64_t K, int64_t nnz, int32_t G) {
    Carver c(nullptr, 0);
    Fa2Scratch s;
    carve_fa2(c, K, nnz, G, s);
    return c.used();
}

int fa2_check_params(const bgv_fa2_params *p) {
    if (!p) return BGV_EINVAL;
    if (!(p->theta >= 0.0f) || !(p->kr >= 0.0f) || !(p->kg >= 0.0f) || !(p->tau > 0.0f) || !(p->ks >= 0.0f) ||
        !(p->ksmax > 0.0f))
        return BGV_EINVAL;
    if (p->strong_gravity != 0 && p->strong_gravity != 1) return BGV_EINVAL;
    if (p->leaf_cap < 1 || p->max_depth < 1 || p->max_depth > 24 || p->reserved != 0) return BGV_EINVAL;
    return BGV_OK;
}

int run_fa2_init(int64_t K, const bgv_fa2_params &p, float *pos, float *Fprev, double *speed, cudaStream_t st,
                 int32_t G, const int64_t *koff) {
    if (G > 1) {
        note_launch(), k_init_seg<<<G, kThreads, 0, st>>>(koff, p.seed, reinterpret_cast<float2 *>(pos),
                                                          reinterpret_cast<float2 *>(Fprev), speed);
        return launch_status();
    }
    if (K > 0) {
        const float R = __builtin_sqrtf(float(K));
        note_launch(), k_init<<<grid_for(K, kThreads, 152 * 8), kThreads, 0, st>>>(
            K, p.seed, R, reinterpret_cast<float2 *>(pos), reinterpret_cast<float2 *>(Fprev));
        BGV_TRY(launch_status());
    }
    note_launch(), k_set_speed<<<1, 1, 0, st>>>(speed);
    return launch_status();
}

int run_fa2(int mode, int64_t K, int64_t nnz, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
            const uint32_t *mass, const bgv_fa2_params &p, float *pos_f, float *F_f, float *Fprev_f, double *speed,
            float *Fr, float *Fa, float *Fg, WsHeader *hdr, void *scratch, cudaStream_t st, cudaEvent_t *marks,
            bool build_plan, int32_t G, const int64_t *koff) {
    if (K <= 0) return BGV_OK;
    const bool batched = G > 1;
    if (!fa2_batch_fits(G, p.max_depth)) return BGV_EINVAL;
    Carver c(scratch, 0);
    Fa2Scratch s;
    carve_fa2(c, K, nnz, G, s);
    float2 *pos = reinterpret_cast<float2 *>(pos_f);
    float2 *F = reinterpret_cast<float2 *>(F_f);
    float2 *Fprev = reinterpret_cast<float2 *>(Fprev_f);
    const int L = p.max_depth;
    const int gbits = batched ? bits_for(G) : 0;
    auto mark = [&](int i) -> int {
        if (marks && cudaEventRecord(marks[i], st) != cudaSuccess) return BGV_ECUDA;
        return BGV_OK;
    };

    // per-step counters and last-block tickets
    BGV_CUDA(cudaMemsetAsync(reinterpret_cast<char *>(hdr) + offsetof(WsHeader, interactions), 0,
                             offsetof(WsHeader, reserved) - offsetof(WsHeader, interactions), st));
    BGV_TRY(mark(0));
    if (batched)
        note_launch(), k_frame_seg<<<G, kThreads, 0, st>>>(pos, koff, s.frame, s.bgraph);
    else
        note_launch(), k_frame<<<kFrameBlocks, kThreads, 0, st>>>(pos, K, s.frame_part, s.frame, &hdr->bbox_ticket);
    BGV_TRY(launch_status());
    const int gk = grid_for(K, kThreads, 152 * 16);
    note_launch(), k_keys<<<gk, kThreads, 0, st>>>(pos, K, s.frame, s.bgraph, L, s.sort.keys[0], s.sort.vals[0],
                                                   s.U);
    BGV_TRY(launch_status());
    BGV_TRY(mark(1));
    int res = 0;
    BGV_TRY(radix_sort(s.sort, K, nullptr, 2 * L + gbits, st, &res, &hdr->status));
    BGV_TRY(mark(2));
    note_launch(), k_gather<<<gk, kThreads, 0, st>>>(s.sort.vals[res], K, pos, mass, s.U, s.body, s.sU, s.smass);
    BGV_TRY(launch_status());
    BGV_TRY(mark(3));
    if (K >= 2) {
        const unsigned gt = unsigned((K + kThreads - 1) / kThreads);
        const unsigned gi = unsigned((K - 1 + kThreads - 1) / kThreads);
        const unsigned tiles = unsigned((K + kMomTile - 1) / kMomTile);
        note_launch(), k_radix_tree<<<gi, kThreads, 0, st>>>(s.sort.keys[res], K, L, gbits, s.left, s.right,
                                                             s.parent, s.range, s.level, s.root);
        BGV_TRY(launch_status());
        note_launch(), k_mom_reduce<<<tiles, kThreads, 0, st>>>(s.sU, s.smass, K, s.TM, s.TX, s.TY);
        note_launch(), k_mom_tiles<<<1, kThreads, 0, st>>>(s.TM, s.TX, s.TY, tiles);
        note_launch(), k_mom_down<<<tiles, kThreads, 0, st>>>(s.sU, s.smass, K, s.TM, s.TX, s.TY, s.PM, s.PX, s.PY);
        BGV_TRY(launch_status());
        BGV_TRY(mark(4));
        BGV_CUDA(cudaMemsetAsync(s.start_count, 0, sizeof(uint32_t) * size_t(K), st));
        note_launch(), k_cells<<<gi, kThreads, 0, st>>>(K, L, p.leaf_cap, s.frame, s.bgraph, s.parent, s.range,
                                                        s.level, s.PM, s.PX, s.PY, s.cell, s.topflag, s.start_count,
                                                        &hdr->tree_nodes);
        BGV_TRY(launch_status());
        BGV_TRY(scan_exclusive(s.start_count, s.T, K, nullptr, nullptr, true, s.scan_tmp, st));
        note_launch(), k_preorder<<<gt, kThreads, 0, st>>>(K, s.parent, s.range, s.topflag, s.cell, s.T, s.body,
                                                           s.geo, s.skip);
        BGV_TRY(launch_status());
        BGV_TRY(mark(5));
        const float theta2 = p.theta * p.theta;
        const int64_t rwarps = (K + 32 * kBodiesPerLane - 1) / (32 * kBodiesPerLane);
        const unsigned gr = unsigned((rwarps * 32 + kThreads - 1) / kThreads);
        note_launch(), k_repulse<<<gr, kThreads, 0, st>>>(s.geo, s.skip, s.T, koff, s.bgraph, s.body, K, p.kr,
                                                          theta2, s.Frep, &hdr->interactions,
                                                          &hdr->interactions_total);
        BGV_TRY(launch_status());
    } else {
        BGV_CUDA(cudaMemsetAsync(s.Frep, 0, sizeof(float2), st));
        BGV_TRY(mark(4));
        BGV_TRY(mark(5));
    }
    BGV_TRY(mark(6));
    if (nnz > 0) {
        if (build_plan) {
            BGV_CUDA(cudaMemsetAsync(s.long_count, 0, sizeof(int32_t), st));
            note_launch(), k_chunk_rows<<<grid_for(K, kThreads, 152 * 16), kThreads, 0, st>>>(
                K, nnz, csr_off, s.chunk_row, s.long_rows, s.long_count);
            BGV_TRY(launch_status());
            note_launch(), k_chunk_meta<<<grid_for((nnz + kChunk - 1) / kChunk, kThreads, 152 * 16), kThreads, 0,
                                          st>>>(K, nnz, csr_off, s.chunk_row, s.chunk_meta);
            BGV_TRY(launch_status());
        }
        const int64_t nchunks = (nnz + kChunk - 1) / kChunk;
        note_launch(), k_attract<<<grid_for(nchunks, kThreads, (nchunks + kThreads - 1) / kThreads), kThreads, 0,
                                   st>>>(K, nnz, csr_off, s.chunk_row, s.chunk_meta, csr_adj, csr_w, pos, s.full,
                                         s.head, s.tail);
        BGV_TRY(launch_status());
        note_launch(), k_long_rows<<<152 * 4, kThreads, 0, st>>>(csr_off, s.long_rows, s.long_count, s.head, s.tail,
                                                                 s.full);
        BGV_TRY(launch_status());
    }
    note_launch(), k_node<<<grid_for(K, kThreads, kNodeBlocks), kThreads, 0, st>>>(
        mode, K, csr_off, s.full, s.head, s.tail, mass, pos, s.Frep, p.kg, p.strong_gravity, F, Fprev,
        reinterpret_cast<float2 *>(Fr), reinterpret_cast<float2 *>(Fa), reinterpret_cast<float2 *>(Fg), s.part, speed,
        p.tau, hdr, (batched && mode == 1) ? s.rowst : nullptr);
    BGV_TRY(launch_status());
    if (batched && mode == 1) {
        note_launch(), k_speed_seg<<<G, kThreads, 0, st>>>(s.rowst, koff, speed, p.tau, hdr);
        BGV_TRY(launch_status());
    }
    BGV_TRY(mark(7));
    if (mode == 1) {
        note_launch(), k_update<<<gk, kThreads, 0, st>>>(K, F, Fprev, pos, speed, s.bgraph, p.ks, p.ksmax);
        BGV_TRY(launch_status());
    }
    BGV_TRY(mark(8));
    return BGV_OK;
}

}  // namespace bgv

// fa2.cu -- ForceAtlas2 on the supergraph (Section 3.1, Algorithm 1).
//
// One iteration is a fixed chain of kernels with no host round trip:
//   k_frame     bounding square of the positions (last-block finalise)
//   k_keys      fixed-point coordinates U and 2L-bit Morton keys; clears the
//               step's counters (the captured step has no memset nodes)
//   radix sort  (key, body) pairs -> Morton order: LSD passes on the bits
//               above 24, then each run of equal high bits ordered locally
//   k_gather_moments
//               bodies in Morton order, and exact prefix sums of (m, m*Ux,
//               m*Uy) in 64/128-bit integers over that order (one pass,
//               decoupled look-back), so a node's moments are a difference
//   k_tree      binary radix tree over the sorted keys, one thread per
//               internal node (exponential + binary search on key prefixes),
//               and the quadtree cells: binary nodes whose 2-bit level
//               exceeds their parent's, FP32 centre of mass from the exact
//               moments
//   k_preorder  cells and bodies laid out in depth-first pre-order with skip
//               indices (positions from a prefix count of cells per body)
//   k_repulse   Barnes-Hut repulsion: one thread per body walks the
//               pre-order array without a stack (accept -> skip past the
//               subtree, open -> next element); every body takes its own
//               opening decisions, so its interaction set is exactly the
//               one the definition gives
//   k_att_*     attraction, rows by length class: short rows one lane
//               each, medium rows one warp each, long rows one block each
//               (the class lists are made once per CSR).  They run on a
//               second stream while the tree is built and walked.
//   k_tail      one persistent kernel (cooperative launch, bounded grid
//               barriers): per node gravity, total force, swing and
//               traction, summed exactly (integer accumulation); the global
//               speed (per graph in the batched form); per node the local
//               speed, the displacement and Fprev = F
//   (k_node gives the forces alone, without a step)
//
// The opening test and the centre it uses are computed with explicit
// round-to-nearest FP32 operations (no contraction) from the exact integer
// moments, so the decisions do not depend on thread scheduling and equal
// the oracle's decisions on the same positions.
#include <atomic>

#include "bgv_internal.cuh"
#include "hsort.cuh"

namespace bgv {

namespace {
constexpr int kThreads = 256;
constexpr int kMaxFrameBlocks = 1024;  // frame-kernel grid: 2 blocks per SM, at most this many
constexpr int kMaxNodeBlocks = 2048;   // node-kernel grid: 4 blocks per SM (measured best), at most this many
inline int frame_blocks() { return sm_count() * 2 < kMaxFrameBlocks ? sm_count() * 2 : kMaxFrameBlocks; }
inline int node_blocks() { return sm_count() * 4 < kMaxNodeBlocks ? sm_count() * 4 : kMaxNodeBlocks; }

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
// Fixed-point position of a body in its graph's frame: U = floor(2^32 (p -
// origin) / side) per axis, FP32 with round-to-nearest steps.
__device__ __forceinline__ uint2 fixed_point(float2 p, float4 fr) {
    const float ux = __fdiv_rn(__fsub_rn(p.x, fr.x), fr.z);
    const float uy = __fdiv_rn(__fsub_rn(p.y, fr.y), fr.z);
    return make_uint2(__float2uint_rz(__fmul_rn(ux, 4294967296.0f)), __float2uint_rz(__fmul_rn(uy, 4294967296.0f)));
}

// Morton key of the body's fixed-point position in its graph's frame; in the
// batched form the graph id sits above the 2L Morton bits, so each graph's
// bodies stay together and form their own subtree.
__device__ __forceinline__ unsigned long long morton_key(const float2 *__restrict__ pos,
                                                         const float4 *__restrict__ frames,
                                                         const int32_t *__restrict__ bgraph, int L, int64_t i) {
    const int g = bgraph ? bgraph[i] : 0;
    const uint2 U = fixed_point(pos[i], frames[g]);
    const uint32_t qx = U.x >> (32 - L), qy = U.y >> (32 - L);
    return (static_cast<unsigned long long>(g) << (2 * L)) | (spread_bits(qx) << 1) | spread_bits(qy);
}

// The same key by body id, for the hinted sort.
struct MortonOf {
    const float2 *pos;
    const float4 *frames;
    const int32_t *bgraph;
    int L;
    __device__ unsigned long long operator()(uint32_t id) const { return morton_key(pos, frames, bgraph, L, id); }
};

// Also clears, for the kernels after it, the step's counters (2 words), the
// moment look-back flags and the sort's digit counters: the launches that
// would otherwise clear them sit on the step's dependency chain.
__global__ void __launch_bounds__(kThreads) k_keys(const float2 *__restrict__ pos, int64_t K,
                                                   const float4 *__restrict__ frames,
                                                   const int32_t *__restrict__ bgraph, int L,
                                                   unsigned long long *__restrict__ keys,
                                                   uint32_t *__restrict__ vals,
                                                   unsigned long long *__restrict__ step_counters,
                                                   uint32_t *__restrict__ clear_a, int64_t n_a,
                                                   uint32_t *__restrict__ clear_b, int64_t n_b) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n_a || t < n_b || t < 2; t += stride) {
        if (t < 2) step_counters[t] = 0ull;
        if (t < n_a) clear_a[t] = 0u;
        if (t < n_b) clear_b[t] = 0u;
    }
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < K; i += stride) {
        keys[i] = morton_key(pos, frames, bgraph, L, i);
        vals[i] = uint32_t(i);
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

// Exact moment prefix sums over the Morton order: P[s] = sum over bodies
// t < s of (m, m*Ux, m*Uy), in 64/128-bit integers, so every node's moments
// are P[last+1] - P[first] (exact, order-free).
constexpr int kMomItems = 4;
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

// Moment prefix of one body in one 32-byte record (one sector per access):
// M in 64 bits, the coordinate sums in 96 (their totals stay below 2^95).
struct __align__(32) MomP {
    unsigned long long M, xl, yl;
    uint32_t xh, yh;
};
__device__ __forceinline__ uint4 momp_first_half(unsigned long long M, u128 X) {
    return make_uint4(uint32_t(M), uint32_t(M >> 32), uint32_t(X), uint32_t(X >> 32));
}
__device__ __forceinline__ uint4 momp_second_half(u128 X, u128 Y) {
    return make_uint4(uint32_t(Y), uint32_t(Y >> 32), uint32_t(X >> 64), uint32_t(Y >> 64));
}
__device__ __forceinline__ void momp_store(MomP *P, int64_t s, const Mom &v) {
    uint4 *p = reinterpret_cast<uint4 *>(P + s);
    p[0] = momp_first_half(v.M, v.X);
    p[1] = momp_second_half(v.X, v.Y);
}
__device__ __forceinline__ Mom momp_load(const MomP *P, int64_t s) {
    const uint4 *p = reinterpret_cast<const uint4 *>(P + s);
    const uint4 a = p[0], b = p[1];
    const unsigned long long xl = (static_cast<unsigned long long>(a.w) << 32) | a.z;
    const unsigned long long yl = (static_cast<unsigned long long>(b.y) << 32) | b.x;
    return Mom{(static_cast<unsigned long long>(a.y) << 32) | a.x, (u128(b.z) << 64) | xl, (u128(b.w) << 64) | yl};
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

// Sorted bodies and moment prefix sums in one pass, with a decoupled
// look-back across tiles.  Tiles of kMomTile sorted positions are taken in
// order from a counter (a tile waits only on tiles already taken, so the
// waits end); a thread gathers kMomItems consecutive positions: the body's
// position, mass and index (body[s]), and its fixed-point coordinates
// recomputed from the position as the keys were.  The tile publishes its
// total, the block adds the totals or inclusive prefixes of the tiles before
// it (up to kMomLookBack at a time), and the prefix records go out through
// shared memory so that every store is coalesced.  Also clears the
// per-body cell counters that k_tree fills.  P[K], the grand total, is
// written by the last tile.
struct MomTile {
    unsigned long long M, xl, xh, yl, yh, pad;
};
enum : uint32_t { kMomAgg = 1u, kMomIncl = 2u };  // look-back flags (0: nothing published)
constexpr int kMomLBItems = 4;                          // predecessors per thread and round
constexpr int kMomLookBack = kThreads * kMomLBItems;    // predecessors per round

__device__ __forceinline__ void mom_tile_store(MomTile *t, const Mom &v) {
    t->M = v.M;
    t->xl = static_cast<unsigned long long>(v.X);
    t->xh = static_cast<unsigned long long>(v.X >> 64);
    t->yl = static_cast<unsigned long long>(v.Y);
    t->yh = static_cast<unsigned long long>(v.Y >> 64);
}
__device__ __forceinline__ Mom mom_tile_load(const MomTile *t) {  // from L2: written by other blocks
    return Mom{__ldcg(&t->M), (u128(__ldcg(&t->xh)) << 64) | __ldcg(&t->xl),
               (u128(__ldcg(&t->yh)) << 64) | __ldcg(&t->yl)};
}
__device__ __forceinline__ Mom mom_warp_sum(Mom v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        Mom o;
        o.M = __shfl_xor_sync(0xFFFFFFFFu, v.M, d);
        const unsigned long long xl = __shfl_xor_sync(0xFFFFFFFFu, static_cast<unsigned long long>(v.X), d);
        const unsigned long long xh = __shfl_xor_sync(0xFFFFFFFFu, static_cast<unsigned long long>(v.X >> 64), d);
        const unsigned long long yl = __shfl_xor_sync(0xFFFFFFFFu, static_cast<unsigned long long>(v.Y), d);
        const unsigned long long yh = __shfl_xor_sync(0xFFFFFFFFu, static_cast<unsigned long long>(v.Y >> 64), d);
        o.X = (u128(xh) << 64) | xl;
        o.Y = (u128(yh) << 64) | yl;
        v = mom_add(v, o);
    }
    return v;
}
// Staging slot of tile element e: one 16-byte pad after every 8 elements, so
// the per-thread writes (stride 8) fall in different banks.
__device__ __forceinline__ int stage_slot(int e) { return e + (e >> 3); }
__global__ void __launch_bounds__(kThreads, 4) k_gather_moments(
    const uint32_t *__restrict__ perm, int64_t K, const float2 *__restrict__ pos, const uint32_t *__restrict__ mass,
    const float4 *__restrict__ frames, const int32_t *__restrict__ bgraph, float4 *__restrict__ body,
    MomP *__restrict__ P, uint32_t *__restrict__ start_count, uint32_t *__restrict__ start_levels, uint32_t *flags, MomTile *agg,
    MomTile *incl, uint32_t *dev_status, int spin_limit) {
    __shared__ uint4 stage[2 * (kMomTile + kMomTile / 8)];  // bodies, then two halves per prefix record
    __shared__ unsigned tile_sh;
    __shared__ int near_sh;
    __shared__ unsigned long long red_sh[kThreads / 32][5];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tiles = (K + kMomTile - 1) / kMomTile;
    if (threadIdx.x == 0) tile_sh = atomicAdd(&flags[tiles], 1u);
    __syncthreads();
    const int64_t tile = tile_sh;
    if (tile >= tiles) return;
    const int64_t t0 = tile * kMomTile;
    const int64_t s0 = t0 + int64_t(threadIdx.x) * kMomItems;
    // sorted position s holds body perm[s]
    uint32_t m[kMomItems], ux[kMomItems], uy[kMomItems];
    Mom acc{0ull, 0, 0};
#pragma unroll
    for (int k = 0; k < kMomItems; ++k) {
        const int64_t sk = s0 + k;
        uint4 b = make_uint4(0u, 0u, 0u, 0u);
        m[k] = 0u;
        ux[k] = 0u;
        uy[k] = 0u;
        if (sk < K) {
            const uint32_t i = perm[sk];
            const float2 p = pos[i];
            const uint2 U = fixed_point(p, frames[bgraph ? bgraph[i] : 0]);
            m[k] = mass[i];
            ux[k] = U.x;
            uy[k] = U.y;
            b = make_uint4(__float_as_uint(p.x), __float_as_uint(p.y), __float_as_uint(__uint2float_rn(m[k])), i);
        }
        stage[stage_slot(threadIdx.x * kMomItems + k)] = b;
        acc.M += m[k];
        acc.X += u128(m[k]) * ux[k];
        acc.Y += u128(m[k]) * uy[k];
    }
    Mom total;
    Mom run = mom_block_exclusive(acc, &total);  // synchronises: the staged bodies are complete
    if (threadIdx.x == 0) {
        mom_tile_store(tile == 0 ? &incl[0] : &agg[tile], total);
        __threadfence();
        atomicExch(&flags[tile], tile == 0 ? kMomIncl : kMomAgg);
    }
#pragma unroll
    for (int r = 0; r < kMomItems; ++r) {
        const int e = r * kThreads + threadIdx.x;
        const int64_t sk = t0 + e;
        if (sk < K) {
            const uint4 v = stage[stage_slot(e)];
            body[sk] = make_float4(__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z),
                                   __uint_as_float(v.w));
            start_count[sk] = 0u;
            start_levels[sk] = 0u;
        }
    }
    // Look-back by the whole block, kMomLookBack predecessors per round: the
    // nearest tile with an inclusive prefix in the window ends it; the tiles
    // after it must have published their totals.
    Mom excl{0ull, 0, 0};
    {
        int64_t hi = tile - 1;
        int spins = 0;
        while (hi >= 0) {
            if (threadIdx.x == 0) near_sh = -1;
            __syncthreads();
            uint32_t f[kMomLBItems];
#pragma unroll
            for (int r = 0; r < kMomLBItems; ++r) {
                const int64_t idx = hi - (r * kThreads + threadIdx.x);
                f[r] = idx >= 0 ? *reinterpret_cast<volatile uint32_t *>(&flags[idx]) : 0u;
                if (idx >= 0 && f[r] == kMomIncl) atomicMax(&near_sh, int(idx));
            }
            __syncthreads();
            const int64_t near = near_sh;
            const int64_t win_lo = hi - kMomLookBack + 1 > 0 ? hi - kMomLookBack + 1 : 0;
            const int64_t lo = near >= 0 ? near : win_lo;
            bool pending = false;
#pragma unroll
            for (int r = 0; r < kMomLBItems; ++r) {
                const int64_t idx = hi - (r * kThreads + threadIdx.x);
                pending |= idx >= lo && f[r] == 0u;
            }
            if (__syncthreads_or(pending)) {
                if (++spins > spin_limit) {
                    if (threadIdx.x == 0) raise_status(dev_status, BGV_DEV_TIMEOUT);
                    break;
                }
                __nanosleep(64);
                continue;
            }
            __threadfence();
            Mom v{0ull, 0, 0};
#pragma unroll
            for (int r = 0; r < kMomLBItems; ++r) {
                const int64_t idx = hi - (r * kThreads + threadIdx.x);
                if (idx >= lo) v = mom_add(v, mom_tile_load(f[r] == kMomIncl ? &incl[idx] : &agg[idx]));
            }
            v = mom_warp_sum(v);
            if (lane == 0) {
                red_sh[warp][0] = v.M;
                red_sh[warp][1] = static_cast<unsigned long long>(v.X);
                red_sh[warp][2] = static_cast<unsigned long long>(v.X >> 64);
                red_sh[warp][3] = static_cast<unsigned long long>(v.Y);
                red_sh[warp][4] = static_cast<unsigned long long>(v.Y >> 64);
            }
            __syncthreads();
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w)
                excl = mom_add(excl, Mom{red_sh[w][0], (u128(red_sh[w][2]) << 64) | red_sh[w][1],
                                         (u128(red_sh[w][4]) << 64) | red_sh[w][3]});
            if (near >= 0) break;
            hi = lo - 1;
        }
    }
    if (threadIdx.x == 0 && tile > 0) {
        mom_tile_store(&incl[tile], mom_add(excl, total));
        __threadfence();
        atomicExch(&flags[tile], kMomIncl);
    }
    const Mom tile_pre = excl;
    __syncthreads();  // the bodies have left the staging buffer
    run = mom_add(run, tile_pre);
    if (tile == tiles - 1 && threadIdx.x == 0) momp_store(P, K, mom_add(tile_pre, total));
    // the prefix records through the staging buffer (the bodies have left
    // it), then out with consecutive threads on consecutive 16-byte halves
    uint4 *stage2 = stage;
    {
        unsigned long long rm = run.M;
        u128 rx = run.X, ry = run.Y;
#pragma unroll
        for (int k = 0; k < kMomItems; ++k) {
            const int slot = 2 * stage_slot(threadIdx.x * kMomItems + k);
            stage2[slot] = momp_first_half(rm, rx);
            stage2[slot + 1] = momp_second_half(rx, ry);
            rm += m[k];
            rx += u128(m[k]) * ux[k];
            ry += u128(m[k]) * uy[k];
        }
    }
    __syncthreads();
    uint4 *P4 = reinterpret_cast<uint4 *>(P);
#pragma unroll
    for (int r = 0; r < 2 * kMomItems; ++r) {
        const int u = r * kThreads + threadIdx.x;  // 16-byte half u of the tile: record u / 2
        if (t0 + (u >> 1) < K) P4[2 * t0 + u] = stage2[2 * stage_slot(u >> 1) + (u & 1)];
    }
}

// 2-bit quadtree level of a binary node with split prefix length delta (the
// graph bits come first): -1 above a graph's root, L for coincident keys.
__device__ __forceinline__ int node_level(int delta, int kb, int L, int gbits) {
    return delta >= kb ? L : (delta < gbits ? -1 : ((delta - gbits) >> 1));
}

// Binary radix tree and quadtree cells in one pass, one thread per internal
// node (Karras, HPG 2012): the node's range and split prefix length come
// from an exponential and a binary search on key prefixes.  Its parent's
// split is the nearer of the two pairs just outside the range (the far one
// shares a shorter prefix), so the node knows its parent's level without
// waiting for anyone.  A node is a quadtree cell when its level exceeds its
// parent's (a chain of single-child cells collapses into its deepest cell,
// which takes the opening test for the whole chain).  For each cell: FP32
// centre from the exact moments, mass, and the squared side used by the
// opening test (+inf for a leaf that is never accepted); cells are counted
// per first body, and their levels recorded there, for the pre-order
// layout.
// A binary node can only be a quadtree cell if the split inside its range
// lies at a deeper 2-bit level than the split just outside it; both follow
// from the keys of the node and its two neighbours.  The test runs over all
// nodes (three coalesced key loads each) and lists the candidates, one
// atomic per block; the range searches then run densely over the list.
__global__ void __launch_bounds__(kThreads) k_tree_mark(const unsigned long long *__restrict__ keys, int64_t K,
                                                        int L, int gbits, int8_t *__restrict__ cell_level,
                                                        uint32_t *__restrict__ cand, uint32_t *cand_count) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    bool is_cand = false;
    if (i < K - 1) {
        const int kb = 2 * L + gbits;
        const unsigned long long ki = __ldg(&keys[i]);
        const int dnext = key_delta(keys, K, kb, i, ki, i + 1), dprev = key_delta(keys, K, kb, i, ki, i - 1);
        const int d = dnext > dprev ? 1 : -1;
        const int dmin = d > 0 ? dprev : dnext;
        // The node's split lies between its parent's (dmin) and that of the
        // pair (i, i + d) inside its range: when those two share a level,
        // the node shares it with its parent and is no cell.
        is_cand = node_level(d > 0 ? dnext : dprev, kb, L, gbits) != node_level(dmin, kb, L, gbits);
        if (!is_cand) cell_level[i] = -1;
    }
    // block-wide compaction: one atomic per block on the shared counter
    __shared__ uint32_t warp_n[kThreads / 32], block_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, is_cand);
    if (lane == 0) warp_n[warp] = uint32_t(__popc(mask));
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kThreads / 32; ++w) {
            const uint32_t c = warp_n[w];
            warp_n[w] = t;
            t += c;
        }
        block_base = t ? atomicAdd(cand_count, t) : 0u;
    }
    __syncthreads();
    if (is_cand) cand[block_base + warp_n[warp] + __popc(mask & ((1u << lane) - 1u))] = uint32_t(i);
}

// Binary radix tree and quadtree cells, one thread per listed candidate
// (Karras, HPG 2012): the node's range and split prefix length come from an
// exponential and a binary search on key prefixes.  Its parent's split is
// the nearer of the two pairs just outside the range (the far one shares a
// shorter prefix), so the node knows its parent's level without waiting for
// anyone.  A node is a quadtree cell when its level exceeds its parent's (a
// chain of single-child cells collapses into its deepest cell, which takes
// the opening test for the whole chain).  For each cell: FP32 centre from
// the exact moments, mass, and the squared side used by the opening test
// (+inf for a leaf that is never accepted); cells are counted per first
// body, and their levels recorded there, for the pre-order layout.
__global__ void __launch_bounds__(kThreads) k_tree(const unsigned long long *__restrict__ keys, int64_t K, int L,
                                                   int gbits, int leaf_cap, const float4 *__restrict__ frames,
                                                   const int32_t *__restrict__ bgraph,
                                                   const MomP *__restrict__ P, int2 *__restrict__ range,
                                                   int8_t *__restrict__ cell_level, float4 *__restrict__ cell,
                                                   uint32_t *__restrict__ start_count,
                                                   uint32_t *__restrict__ start_levels,
                                                   unsigned long long *tree_nodes, const uint32_t *__restrict__ cand,
                                                   const uint32_t *cand_count) {
    const int64_t count = *cand_count;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int kb = 2 * L + gbits;
    uint32_t tops = 0;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < count; q += stride) {
        const int64_t i = cand[q];
        const unsigned long long ki = __ldg(&keys[i]);
        const int dnext = key_delta(keys, K, kb, i, ki, i + 1), dprev = key_delta(keys, K, kb, i, ki, i - 1);
        const int d = dnext > dprev ? 1 : -1;
        const int dmin = d > 0 ? dprev : dnext;
        int64_t lmax = 2;
        while (key_delta(keys, K, kb, i, ki, i + lmax * d) > dmin) lmax <<= 1;
        int64_t l = 0;
        for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
            if (key_delta(keys, K, kb, i, ki, i + (l + t) * d) > dmin) l += t;
        const int64_t j = i + l * d;
        const int dnode = key_delta(keys, K, kb, i, ki, j);
        const int64_t first = i < j ? i : j, last = i < j ? j : i;
        const int lev = node_level(dnode, kb, L, gbits);
        const int par_lev = node_level(dmin, kb, L, gbits);
        const bool top = par_lev < lev;
        cell_level[i] = static_cast<int8_t>(top ? lev : -1);
        if (top) {
            ++tops;
            range[i] = make_int2(int32_t(first), int32_t(last));
            const int cnt = int(last - first) + 1;
            const bool leaf = cnt <= leaf_cap || lev >= L;
            // A leaf made by the depth limit (coincident keys, more than
            // leaf_cap bodies) hides a chain of non-leaf cells with the same
            // bodies between its parent's level and L; the deepest of them,
            // at level L - 1, takes the opening test for the whole chain.
            const bool testable = leaf && cnt > leaf_cap && par_lev + 1 <= L - 1;
            // positions of graph g in Morton order are its index range too
            const float4 fr = frames[bgraph ? bgraph[first] : 0];
            const Mom hi = momp_load(P, last + 1), lo = momp_load(P, first);
            const unsigned long long M = hi.M - lo.M;
            const u128 X = hi.X - lo.X, Y = hi.Y - lo.Y;
            const uint32_t qx = M ? uint32_t(X / M) : 0u, qy = M ? uint32_t(Y / M) : 0u;
            const float two_m32 = 2.3283064365386963e-10f;  // 2^-32
            const float cx = __fadd_rn(fr.x, __fmul_rn(fr.z, __fmul_rn(__uint2float_rn(qx), two_m32)));
            const float cy = __fadd_rn(fr.y, __fmul_rn(fr.z, __fmul_rn(__uint2float_rn(qy), two_m32)));
            const float sl = __fmul_rn(fr.z, pow2_neg(testable ? L - 1 : lev));
            const float side2 = (leaf && !testable) ? INFINITY : __fmul_rn(sl, sl);
            cell[i] = make_float4(cx, cy, __ull2float_rn(M), side2);
            atomicAdd(&start_count[first], 1u);
            atomicOr(&start_levels[first], 1u << lev);
        }
    }
#pragma unroll
    for (int dd = 16; dd > 0; dd >>= 1) tops += __shfl_xor_sync(0xFFFFFFFFu, tops, dd);
    if ((threadIdx.x & 31) == 0 && tops) atomicAdd(tree_nodes, static_cast<unsigned long long>(tops));
}

// Pre-order layout of cells and bodies.  With T[s] = number of cells whose
// first body precedes s (exclusive scan of the per-body counts):
//   body s           -> s + T[s+1]       (every cell starting at or before s
//                                          comes first)
//   cell [a, b]      -> a + T[a] + (its ancestors that also start at a)
//   skip(cell [a,b]) -> b + 1 + T[b+1]   (the element after its subtree)
// The cells starting at body a are nested with strictly increasing levels,
// so a cell's ancestors among them are those of a lower level in
// start_levels[a].  Elements are float4 (x, y, mass, side^2), side^2 = -1
// for a body.
__global__ void __launch_bounds__(kThreads) k_preorder(int64_t K, const int2 *__restrict__ range,
                                                       const int8_t *__restrict__ cell_level,
                                                       const uint32_t *__restrict__ start_levels,
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
    if (t < K - 1) {
        const int lev = cell_level[t];
        if (lev >= 0) {
            const int2 rg = range[t];
            const int dep = __popc(start_levels[rg.x] & ((1u << lev) - 1u));
            const int64_t pre = rg.x + int64_t(T[rg.x]) + dep;
            geo[pre] = cell[t];
            skip[pre] = int32_t(int64_t(rg.y) + 1 + T[rg.y + 1]);
        }
    }
}

// -------------------------------------------------------------- repulsion
// Barnes-Hut traversal without a stack, one body per thread, over the
// pre-order array.  At element `cur` (a cell or a body) the thread accepts it
// -- sums its monopole and moves to skip[cur], past its subtree -- or enters
// it (cur + 1).  A body is always accepted except the thread's own (its
// side^2 is -1); a cell holding the thread's body is always entered; any
// other cell is accepted by the FP32 opening test of the definition.  Each
// body sees exactly its own interaction set in depth-first order; threads of
// a warp are Morton neighbours, so they mostly read the same elements.
template <int kRT>
__global__ void __launch_bounds__(kRT) k_repulse(const float4 *__restrict__ geo, const int32_t *__restrict__ skip,
                                                      const uint32_t *__restrict__ T,
                                                      const int64_t *__restrict__ koff,
                                                      const int32_t *__restrict__ bgraph,
                                                      const float4 *__restrict__ body, int64_t K, float kr,
                                                      float theta2, float2 *__restrict__ Frep,
                                                      unsigned long long *inter_step,
                                                      unsigned long long *inter_total) {
    const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    unsigned inter = 0;
    if (s < K) {
        const float4 bi = body[s];
        const float kmi = kr * bi.z;
        const uint32_t self = uint32_t(s + T[s + 1]);
        // the body's own graph: its subtree spans [start, end) in pre-order
        uint32_t cur = 0, end = uint32_t(K + T[K]);
        if (bgraph) {
            const int g = bgraph[s];
            const int64_t a = koff[g], b = koff[g + 1];
            cur = uint32_t(a + T[a]);
            end = uint32_t(b + T[b]);
        }
        float fx = 0.0f, fy = 0.0f;
        while (cur < end) {
            const float4 e = geo[cur];
            const uint32_t sk = uint32_t(skip[cur]);
            const float dx = __fsub_rn(bi.x, e.x), dy = __fsub_rn(bi.y, e.y);
            const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
            // accepted: not an element holding the body (cur <= self < sk) and
            // the opening test passes; no branch, so lanes stay converged
            const bool accept = self - cur >= sk - cur && e.w < __fmul_rn(theta2, d2);
            const float f = accept && d2 > 0.0f ? __fdividef(kmi * e.z, d2) : 0.0f;
            fx += f * dx;
            fy += f * dy;
            inter += accept ? 1u : 0u;
            cur = accept ? sk : cur + 1;
        }
        Frep[__float_as_int(bi.w)] = make_float2(fx, fy);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) inter += __shfl_xor_sync(0xFFFFFFFFu, inter, d);
    if ((threadIdx.x & 31) == 0 && inter) {
        atomicAdd(inter_step, static_cast<unsigned long long>(inter));
        atomicAdd(inter_total, static_cast<unsigned long long>(inter));
    }
}

// ------------------------------------------------------------ attraction
// F^a_i = sum over row i's CSR entries (j, w) of w (p_j - p_i), in FP32.
// Every row is summed by one worker in an order that depends only on the
// row's own entries (deterministic, and the same whatever else the CSR
// holds).  The plan, made once per CSR, lists the rows by length: short rows
// (at most `att_short` entries) take one lane each, 32 rows to a warp, and
// add their entries in order; medium rows (up to kAttMedium entries) take
// one warp each, two rows at a time: lane l adds entries l, l + 32, ... in order, then a fixed
// butterfly; long rows take one block each (thread t adds t, t + 256, ...,
// then a fixed tree).  Every worker first issues kAttIn loads of neighbour
// ids and weights, then their position gathers, so they are in flight
// together.  An empty row is a short row of sum 0.
constexpr int kAttMedium = 4096;
// loads in flight per worker; with 5 blocks of 256 per SM (at most 51
// registers) that is 320 outstanding gathers per SM
constexpr int kAttIn = 8;

// Block-aggregated append of row r to the list of class c (one atomic per
// class per block).
__global__ void __launch_bounds__(kThreads) k_att_plan(int64_t K, const int32_t *__restrict__ off, int att_short,
                                                       int32_t *__restrict__ rows_short, int32_t *__restrict__ rows_med,
                                                       int32_t *__restrict__ rows_long, uint32_t *counts) {
    __shared__ uint32_t wn[3][kThreads / 32], base[3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t r0 = int64_t(blockIdx.x) * blockDim.x; r0 < K; r0 += int64_t(gridDim.x) * blockDim.x) {
        const int64_t r = r0 + threadIdx.x;
        int c = -1;
        if (r < K) {
            const int64_t len = int64_t(off[r + 1]) - off[r];
            c = len <= att_short ? 0 : (len <= kAttMedium ? 1 : 2);
        }
        unsigned m[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            m[k] = __ballot_sync(0xFFFFFFFFu, c == k);
            if (lane == 0) wn[k][warp] = uint32_t(__popc(m[k]));
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            const int k = threadIdx.x;
            uint32_t t = 0;
            for (int w = 0; w < kThreads / 32; ++w) {
                const uint32_t x = wn[k][w];
                wn[k][w] = t;
                t += x;
            }
            base[k] = t ? atomicAdd(&counts[k], t) : 0u;
        }
        __syncthreads();
        if (c >= 0) {
            int32_t *list = c == 0 ? rows_short : (c == 1 ? rows_med : rows_long);
            list[base[c] + wn[c][warp] + __popc(m[c] & ((1u << lane) - 1u))] = int32_t(r);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ bool valid_row(int32_t j, int64_t K) {
    return static_cast<uint64_t>(int64_t(j)) < static_cast<uint64_t>(K);  // an invalid entry adds nothing
}

// Short rows: one lane each.
__global__ void __launch_bounds__(kThreads, 5) k_att_short(int64_t K, const int32_t *__restrict__ off,
                                                        const int32_t *__restrict__ adj,
                                                        const uint32_t *__restrict__ w,
                                                        const float2 *__restrict__ pos,
                                                        const int32_t *__restrict__ rows, const uint32_t *counts,
                                                        float2 *__restrict__ full) {
    const int64_t count = counts[0];
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < count; q += stride) {
        const int32_t r = rows[q];
        const int64_t b = off[r], e = off[r + 1];
        const float2 pi = pos[r];
        float ax = 0.0f, ay = 0.0f;
        for (int64_t e0 = b; e0 < e; e0 += kAttIn) {
            int32_t j[kAttIn];
            uint32_t wt[kAttIn];
#pragma unroll
            for (int k = 0; k < kAttIn; ++k) {
                j[k] = e0 + k < e ? __ldcs(adj + e0 + k) : -1;
                wt[k] = e0 + k < e ? __ldcs(w + e0 + k) : 0u;
            }
            float2 pj[kAttIn];
#pragma unroll
            for (int k = 0; k < kAttIn; ++k) pj[k] = valid_row(j[k], K) ? pos[j[k]] : pi;
#pragma unroll
            for (int k = 0; k < kAttIn; ++k) {
                const float wf = valid_row(j[k], K) ? __uint2float_rn(wt[k]) : 0.0f;
                ax += wf * (pj[k].x - pi.x);
                ay += wf * (pj[k].y - pi.y);
            }
        }
        full[r] = make_float2(ax, ay);
    }
}

// Medium rows: one warp each, two rows at a time (each lane keeps
// kAttIn / 2 loads in flight per row, so a warp waits on two rows' round
// trips at once).  Lane l adds entries l, l + 32, ... of a row in order, then
// a fixed butterfly: the sums do not depend on how the rows are paired.
__global__ void __launch_bounds__(kThreads, 4) k_att_medium(int64_t K, const int32_t *__restrict__ off,
                                                         const int32_t *__restrict__ adj,
                                                         const uint32_t *__restrict__ w,
                                                         const float2 *__restrict__ pos,
                                                         const int32_t *__restrict__ rows, const uint32_t *counts,
                                                         float2 *__restrict__ full) {
    constexpr int kIn = kAttIn / 2;
    const int lane = threadIdx.x & 31;
    const int64_t count = counts[1];
    const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t q = ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * 2; q < count; q += warps * 2) {
        const bool two = q + 1 < count;
        const int32_t r0 = rows[q], r1 = two ? rows[q + 1] : r0;
        const int64_t b0 = off[r0], len0 = int64_t(off[r0 + 1]) - b0;
        const int64_t b1 = off[r1], len1 = two ? int64_t(off[r1 + 1]) - b1 : 0;
        const float2 p0 = pos[r0], p1 = pos[r1];
        float ax0 = 0.0f, ay0 = 0.0f, ax1 = 0.0f, ay1 = 0.0f;
        const int64_t len = len0 > len1 ? len0 : len1;
        for (int64_t t0 = lane; t0 < len; t0 += 32 * kIn) {
            int32_t j0[kIn], j1[kIn];
            uint32_t w0[kIn], w1[kIn];
#pragma unroll
            for (int k = 0; k < kIn; ++k) {
                const int64_t t = t0 + 32 * k;
                j0[k] = t < len0 ? __ldcs(adj + b0 + t) : -1;
                w0[k] = t < len0 ? __ldcs(w + b0 + t) : 0u;
                j1[k] = t < len1 ? __ldcs(adj + b1 + t) : -1;
                w1[k] = t < len1 ? __ldcs(w + b1 + t) : 0u;
            }
            float2 q0[kIn], q1[kIn];
#pragma unroll
            for (int k = 0; k < kIn; ++k) {
                q0[k] = valid_row(j0[k], K) ? pos[j0[k]] : p0;
                q1[k] = valid_row(j1[k], K) ? pos[j1[k]] : p1;
            }
#pragma unroll
            for (int k = 0; k < kIn; ++k) {
                const float wf0 = valid_row(j0[k], K) ? __uint2float_rn(w0[k]) : 0.0f;
                const float wf1 = valid_row(j1[k], K) ? __uint2float_rn(w1[k]) : 0.0f;
                ax0 += wf0 * (q0[k].x - p0.x);
                ay0 += wf0 * (q0[k].y - p0.y);
                ax1 += wf1 * (q1[k].x - p1.x);
                ay1 += wf1 * (q1[k].y - p1.y);
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            ax0 += __shfl_xor_sync(0xFFFFFFFFu, ax0, d);
            ay0 += __shfl_xor_sync(0xFFFFFFFFu, ay0, d);
            ax1 += __shfl_xor_sync(0xFFFFFFFFu, ax1, d);
            ay1 += __shfl_xor_sync(0xFFFFFFFFu, ay1, d);
        }
        if (lane == 0) {
            full[r0] = make_float2(ax0, ay0);
            if (two) full[r1] = make_float2(ax1, ay1);
        }
    }
}

// Long rows: one block each.
__global__ void __launch_bounds__(kThreads) k_att_long(int64_t K, const int32_t *__restrict__ off,
                                                       const int32_t *__restrict__ adj, const uint32_t *__restrict__ w,
                                                       const float2 *__restrict__ pos, const int32_t *__restrict__ rows,
                                                       const uint32_t *counts, float2 *__restrict__ full) {
    __shared__ float2 wsum[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t count = counts[2];
    for (int64_t q = blockIdx.x; q < count; q += gridDim.x) {
        const int32_t r = rows[q];
        const int64_t b = off[r], e = off[r + 1];
        const float2 pi = pos[r];
        float ax = 0.0f, ay = 0.0f;
        for (int64_t e0 = b + threadIdx.x; e0 < e; e0 += int64_t(kThreads) * kAttIn) {
            int32_t j[kAttIn];
            uint32_t wt[kAttIn];
#pragma unroll
            for (int k = 0; k < kAttIn; ++k) {
                const int64_t x = e0 + int64_t(kThreads) * k;
                j[k] = x < e ? __ldcs(adj + x) : -1;
                wt[k] = x < e ? __ldcs(w + x) : 0u;
            }
            float2 pj[kAttIn];
#pragma unroll
            for (int k = 0; k < kAttIn; ++k) pj[k] = valid_row(j[k], K) ? pos[j[k]] : pi;
#pragma unroll
            for (int k = 0; k < kAttIn; ++k) {
                const float wf = valid_row(j[k], K) ? __uint2float_rn(wt[k]) : 0.0f;
                ax += wf * (pj[k].x - pi.x);
                ay += wf * (pj[k].y - pi.y);
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            ax += __shfl_xor_sync(0xFFFFFFFFu, ax, d);
            ay += __shfl_xor_sync(0xFFFFFFFFu, ay, d);
        }
        if (lane == 0) wsum[warp] = make_float2(ax, ay);
        __syncthreads();
        if (threadIdx.x == 0) {
            float2 t = wsum[0];
            for (int k = 1; k < kThreads / 32; ++k) {
                t.x += wsum[k].x;
                t.y += wsum[k].y;
            }
            full[r] = t;
        }
        __syncthreads();
    }
}

// --------------------------------------------- node forces, swing, speed
// Global swing and traction (the sums that set the adaptive speed):
// S = sum m_i swing_i and T = sum m_i traction_i over FP32 per-node products,
// which are non-negative.  They are summed EXACTLY: each product f * 2^q
// (f its 24-bit significand) is added as a fixed-point integer into a
// 128-bit accumulator V whose unit 2^q0 sits kXHead binary places below the
// largest term seen so far (q0 moves up, with V shifted down, when a larger
// term arrives).  A term below the unit loses only its bits under 2^q0, less
// than 2^-95 of the largest term, so the accumulated value equals the exact
// sum to about 2^-64 relative even over 2^31 terms; integer addition does not
// depend on the order of the merges.  The total is rounded once to FP64, so S
// and T are the correctly rounded sums of the products (Kahan or Neumaier
// compensation in FP64 would leave about two units in the last place, and
// FP64 arithmetic runs at a small fraction of the integer rate on this GPU).
constexpr int kXHead = 72;          // each term < 2^(24 + 72): 2^31 terms fit in 127 bits
constexpr int kXNoAnchor = -100000; // anchor of an empty accumulator
struct XSum {
    u128 V;
    int q0;
    int bad;  // 1: an infinite term, 2: a NaN term
};
__device__ __forceinline__ XSum xsum_zero() { return XSum{0, kXNoAnchor, 0}; }

__device__ __forceinline__ void xsum_add(XSum &a, float x) {
    const uint32_t b = __float_as_uint(x) & 0x7FFFFFFFu;  // terms are >= 0 (a -0 adds nothing)
    const int e = int(b >> 23);
    if (e == 255) {
        a.bad |= (b & 0x7FFFFFu) ? 2 : 1;
        return;
    }
    const uint32_t f = e ? ((b & 0x7FFFFFu) | 0x800000u) : b;
    const int q = (e ? e : 1) - 150;  // x = f * 2^q
    if (f == 0u) return;
    if (q - kXHead > a.q0) {  // a new largest term: move the anchor up
        const int d = q - kXHead - a.q0;
        a.V = d >= 128 ? u128(0) : (a.V >> d);
        a.q0 = q - kXHead;
    }
    const int sh = q - a.q0;  // <= kXHead
    if (sh >= 0)
        a.V += u128(f) << sh;
    else if (sh > -24)
        a.V += u128(f >> -sh);
}

__device__ __forceinline__ XSum xsum_merge(XSum a, XSum b) {
    if (b.q0 > a.q0) {
        const XSum t = a;
        a = b;
        b = t;
    }
    const int d = a.q0 - b.q0;
    if (d < 128) a.V += b.V >> d;
    a.bad |= b.bad;
    return a;
}

__device__ __forceinline__ XSum xsum_shfl_down(const XSum &a, int d) {
    XSum r;
    r.V = (u128(__shfl_down_sync(0xFFFFFFFFu, static_cast<unsigned long long>(a.V >> 64), d)) << 64) |
          __shfl_down_sync(0xFFFFFFFFu, static_cast<unsigned long long>(a.V), d);
    r.q0 = __shfl_down_sync(0xFFFFFFFFu, a.q0, d);
    r.bad = __shfl_down_sync(0xFFFFFFFFu, a.bad, d);
    return r;
}

// The accumulated value rounded once to FP64 (round to nearest even): the top
// 64 bits of V, with a sticky bit for the rest, converted, then scaled.
__device__ __forceinline__ double xsum_value(const XSum &a) {
    if (a.bad) return (a.bad & 2) ? __longlong_as_double(0x7FF8000000000000ll) : __longlong_as_double(0x7FF0000000000000ll);
    const unsigned long long hi = static_cast<unsigned long long>(a.V >> 64);
    if (!hi) return ldexp(__ull2double_rn(static_cast<unsigned long long>(a.V)), a.q0);
    const int sh = 64 - __clzll(static_cast<long long>(hi));  // bits of V above its top 64
    unsigned long long t = static_cast<unsigned long long>(a.V >> sh);
    if (a.V & ((u128(1) << sh) - 1)) t |= 1ull;  // sticky: far below the rounding position
    return ldexp(__ull2double_rn(t), a.q0 + sh);
}

// Stored form of one accumulator (per-block partials).
struct XPart {
    unsigned long long lo, hi;
    int q0, bad;
};
__device__ __forceinline__ XPart xsum_pack(const XSum &a) {
    return XPart{static_cast<unsigned long long>(a.V), static_cast<unsigned long long>(a.V >> 64), a.q0, a.bad};
}
__device__ __forceinline__ XSum xsum_unpack(const XPart *p) {  // from L2: written by other blocks
    const unsigned long long lo = __ldcg(&p->lo), hi = __ldcg(&p->hi);
    return XSum{(u128(hi) << 64) | lo, __ldcg(&p->q0), __ldcg(&p->bad)};
}

// Block-wide merge of one (S, T) pair per thread in a fixed tree; thread 0
// receives the result.
__device__ __forceinline__ void xsum_block(XSum &S, XSum &T) {
    __shared__ XPart sS[kThreads / 32], sT[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const XSum oS = xsum_shfl_down(S, d), oT = xsum_shfl_down(T, d);
        S = xsum_merge(S, oS);
        T = xsum_merge(T, oT);
    }
    if (lane == 0) {
        sS[warp] = xsum_pack(S);
        sT[warp] = xsum_pack(T);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kThreads / 32; ++k) {
            S = xsum_merge(S, XSum{(u128(sS[k].hi) << 64) | sS[k].lo, sS[k].q0, sS[k].bad});
            T = xsum_merge(T, XSum{(u128(sT[k].hi) << 64) | sT[k].lo, sT[k].q0, sT[k].bad});
        }
    }
    __syncthreads();
}

__device__ __forceinline__ double speed_update(double sp, double Ssum, double Tsum, float tau) {
    if (Ssum > 0.0) {
        const double target = double(tau) * Tsum / Ssum;
        const double rise = target - sp, cap = 0.5 * sp;
        sp += rise < cap ? rise : cap;
    }
    return sp;
}

// Per-node swing and traction products, FP32 with every rounding explicit
// (no contraction), so they can be recomputed bit for bit from F, Fprev and
// the mass: m |F - Fprev| and (m / 2) |F + Fprev|.
__device__ __forceinline__ float2 swing_traction(float m, float fx, float fy, float px, float py) {
    const float sx = __fsub_rn(fx, px), sy = __fsub_rn(fy, py), tx = __fadd_rn(fx, px), ty = __fadd_rn(fy, py);
    const float sw = sqrtf(__fadd_rn(__fmul_rn(sx, sx), __fmul_rn(sy, sy)));
    const float tr = sqrtf(__fadd_rn(__fmul_rn(tx, tx), __fmul_rn(ty, ty)));
    return make_float2(__fmul_rn(m, sw), __fmul_rn(__fmul_rn(0.5f, m), tr));
}

// The step's tail in one persistent kernel (all blocks resident at once,
// cooperative launch): per node the total force and the swing and traction
// products; a grid barrier; the global speed (every block merges the block
// partials in block order, so all blocks hold the same value; batched: one
// block per graph sums that graph's rows, then a second barrier); then per
// node the local speed and the displacement, Fprev = F.  The barrier waits
// are bounded and report BGV_DEV_TIMEOUT.
// full == nullptr: no CSR entries, no attraction.
__device__ __forceinline__ float2 force_sum(float2 fa, float m, float2 pi, float2 fr, float kg, int strong) {
    float gx, gy;
    if (strong) {
        gx = -kg * m * pi.x;
        gy = -kg * m * pi.y;
    } else {
        const float rr = sqrtf(pi.x * pi.x + pi.y * pi.y);
        gx = rr > 0.0f ? -kg * m * pi.x / rr : 0.0f;
        gy = rr > 0.0f ? -kg * m * pi.y / rr : 0.0f;
    }
    return make_float2(fr.x + fa.x + gx, fr.y + fa.y + gy);
}

// Total force on node i: repulsion fr, attraction full[i] (none if null),
// gravity.
__device__ __forceinline__ float2 node_force(int64_t i, const float2 *__restrict__ full, float m, float2 pi, float2 fr,
                                             float kg, int strong) {
    return force_sum(full ? full[i] : make_float2(0.0f, 0.0f), m, pi, fr, kg, strong);
}

__device__ __forceinline__ float2 displaced(float2 p, float2 f, float2 fp, float sp, float ks, float ksmax) {
    const float sx = f.x - fp.x, sy = f.y - fp.y;
    const float swing = sqrtf(sx * sx + sy * sy);
    float s = ks * sp / (1.0f + sp * sqrtf(swing));
    const float fn = sqrtf(f.x * f.x + f.y * f.y);
    if (fn > 0.0f && s * fn > ksmax) s = ksmax / fn;
    p.x += s * f.x;
    p.y += s * f.y;
    return p;
}

// Forces only (no state change): repulsion, attraction and gravity per node.
__global__ void __launch_bounds__(kThreads) k_node(int64_t K, const float2 *__restrict__ att,
                                                   const uint32_t *__restrict__ mass, const float2 *__restrict__ pos,
                                                   const float2 *__restrict__ Frep, float kg, int strong,
                                                   float2 *__restrict__ Fr_out, float2 *__restrict__ Fa_out,
                                                   float2 *__restrict__ Fg_out) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < K; i += stride) {
        const float m = __uint2float_rn(mass[i]);
        const float2 pi = pos[i];
        if (Fr_out) Fr_out[i] = Frep[i];
        if (Fa_out) Fa_out[i] = att ? att[i] : make_float2(0.0f, 0.0f);
        if (Fg_out) Fg_out[i] = node_force(i, nullptr, m, pi, make_float2(0.0f, 0.0f), kg, strong);
    }
}

constexpr int kTailItems = 4;  // nodes a thread takes per pass
__global__ void __launch_bounds__(kThreads) k_tail(int64_t K, const float2 *__restrict__ att,
                                                   const uint32_t *__restrict__ mass, float2 *__restrict__ pos,
                                                   const float2 *__restrict__ Frep, float kg, int strong,
                                                   float2 *__restrict__ F, float2 *__restrict__ Fprev, XPart *part,
                                                   double *speed, float tau, float ks, float ksmax, WsHeader *hdr,
                                                   float2 *__restrict__ rowst, const int64_t *__restrict__ koff,
                                                   const int32_t *__restrict__ bgraph, int32_t G, int spin_limit) {
    __shared__ double sp_sh;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t t0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const bool batched = rowst != nullptr;
    const double sp_old = batched ? 0.0 : *speed;  // read by every block before anyone writes it
    XSum S = xsum_zero(), T = xsum_zero();
    // kTailItems nodes per pass, every load issued before the arithmetic (the
    // exact sums do not depend on the order of the terms)
    for (int64_t i0 = t0; i0 < K; i0 += stride * kTailItems) {
        uint32_t mk[kTailItems];
        float2 pk[kTailItems], rk[kTailItems], ak[kTailItems], qk[kTailItems];
#pragma unroll
        for (int k = 0; k < kTailItems; ++k) {
            const int64_t i = i0 + stride * k;
            const bool in = i < K;
            const float2 z = make_float2(0.0f, 0.0f);
            mk[k] = in ? mass[i] : 0u;
            pk[k] = in ? pos[i] : z;
            rk[k] = in ? Frep[i] : z;
            ak[k] = in && att ? att[i] : z;
            qk[k] = in ? Fprev[i] : z;
        }
#pragma unroll
        for (int k = 0; k < kTailItems; ++k) {
            const int64_t i = i0 + stride * k;
            if (i >= K) continue;
            const float m = __uint2float_rn(mk[k]);
            const float2 f = force_sum(ak[k], m, pk[k], rk[k], kg, strong);
            F[i] = f;
            const float2 st = swing_traction(m, f.x, f.y, qk[k].x, qk[k].y);
            if (batched) {
                rowst[i] = st;
            } else {
                xsum_add(S, st.x);
                xsum_add(T, st.y);
            }
        }
    }
    if (!batched) {
        xsum_block(S, T);
        if (threadIdx.x == 0) {
            part[2 * blockIdx.x] = xsum_pack(S);
            part[2 * blockIdx.x + 1] = xsum_pack(T);
        }
        if (!grid_barrier(&hdr->bar, spin_limit, &hdr->status)) return;
        S = xsum_zero();
        T = xsum_zero();
        for (unsigned bk = threadIdx.x; bk < gridDim.x; bk += blockDim.x) {
            S = xsum_merge(S, xsum_unpack(&part[2 * bk]));
            T = xsum_merge(T, xsum_unpack(&part[2 * bk + 1]));
        }
        xsum_block(S, T);
        if (threadIdx.x == 0) {
            const double Ssum = xsum_value(S), Tsum = xsum_value(T);
            sp_sh = speed_update(sp_old, Ssum, Tsum, tau);
            if (blockIdx.x == 0) {
                *speed = sp_sh;
                hdr->S = Ssum;
                hdr->T = Tsum;
                hdr->steps_total += 1;
            }
        }
        __syncthreads();
    } else {
        if (!grid_barrier(&hdr->bar, spin_limit, &hdr->status)) return;
        for (int32_t g = blockIdx.x; g < G; g += gridDim.x) {  // one block per graph
            const int64_t a = koff[g], b = koff[g + 1];
            XSum Sg = xsum_zero(), Tg = xsum_zero();
            for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) {
                const float2 v = __ldcg(&rowst[i]);
                xsum_add(Sg, v.x);
                xsum_add(Tg, v.y);
            }
            xsum_block(Sg, Tg);
            if (threadIdx.x == 0) {
                const double Ssum = xsum_value(Sg), Tsum = xsum_value(Tg);
                speed[g] = speed_update(speed[g], Ssum, Tsum, tau);
                if (g == 0) {
                    hdr->S = Ssum;
                    hdr->T = Tsum;
                    hdr->steps_total += 1;
                }
            }
        }
        if (!grid_barrier(&hdr->bar, spin_limit, &hdr->status)) return;
    }
    const float sp_all = float(sp_sh);
    for (int64_t i0 = t0; i0 < K; i0 += stride * kTailItems) {
        float2 fk[kTailItems], qk[kTailItems], pk[kTailItems];
        float sk[kTailItems];
#pragma unroll
        for (int k = 0; k < kTailItems; ++k) {
            const int64_t i = i0 + stride * k;
            const bool in = i < K;
            const float2 z = make_float2(0.0f, 0.0f);
            fk[k] = in ? __ldcg(&F[i]) : z;  // written by this kernel before the barrier
            qk[k] = in ? Fprev[i] : z;
            pk[k] = in ? pos[i] : z;
            sk[k] = in && batched ? float(__ldcg(&speed[bgraph[i]])) : sp_all;
        }
#pragma unroll
        for (int k = 0; k < kTailItems; ++k) {
            const int64_t i = i0 + stride * k;
            if (i >= K) continue;
            pos[i] = displaced(pk[k], fk[k], qk[k], sk[k], ks, ksmax);
            Fprev[i] = fk[k];
        }
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
    RunFixBuffers runfix;
    float4 *body;          // sorted bodies: x, y, mass, index
    int2 *range;           // per binary node that is a cell: its bodies
    int8_t *cell_level;    // per binary node: its level if a cell, else -1
    MomP *P;               // moment prefix sums, K + 1 records
    uint32_t *mom_flags;   // look-back flags per tile, the tile counter, the tree candidate count
    uint32_t *cand;        // binary nodes that may be quadtree cells
    MomTile *mom_agg, *mom_incl;
    float4 *cell;          // per binary node: centre, mass, side^2 (cells only)
    uint32_t *start_count; // cells per first body
    uint32_t *start_levels;  // levels of the cells per first body (bit mask)
    uint32_t *T;           // exclusive scan of start_count, K + 1 entries
    void *scan_tmp;
    float4 *geo;           // pre-order elements (cells and bodies)
    int32_t *skip;         // pre-order index after each element's subtree
    float2 *Frep;
    float2 *full;          // attraction per row
    int32_t *rows_short, *rows_med, *rows_long;  // plan: rows by length class
    uint32_t *att_counts;  // plan: the three list lengths
    XPart *part;  // per node-kernel block: exact S and T partials
    HsBuffers hs;  // hinted sort of the Morton keys
};

static void carve_fa2(Carver &c, int64_t K, int64_t nnz, int32_t G, Fa2Scratch &s) {
    const size_t k = size_t(K > 0 ? K : 1);
    const bool batched = G > 1;
    s.frame = c.take<float4>(size_t(G > 1 ? G : 1));
    s.frame_part = c.take<float4>(kMaxFrameBlocks);
    s.bgraph = batched ? c.take<int32_t>(k) : nullptr;
    s.rowst = batched ? c.take<float2>(k) : nullptr;
    carve_sort(c, int64_t(k), true, s.sort);
    carve_run_fix(c, int64_t(k), s.runfix);
    s.body = c.take<float4>(k);
    const size_t tiles = (k + kMomTile - 1) / kMomTile;
    s.range = c.take<int2>(k);
    s.cell_level = c.take<int8_t>(k);
    s.P = c.take<MomP>(k + 1);
    s.mom_flags = c.take<uint32_t>(tiles + 2);  // look-back flags, tile counter, tree candidate count
    s.mom_agg = c.take<MomTile>(tiles);
    s.mom_incl = c.take<MomTile>(tiles);
    s.cell = c.take<float4>(k);
    s.cand = c.take<uint32_t>(k);
    s.start_count = c.take<uint32_t>(k + 1);
    s.start_levels = c.take<uint32_t>(k);
    s.T = c.take<uint32_t>(k + 1);
    s.scan_tmp = c.take<char>(scan_tmp_bytes(int64_t(k) + 1));
    s.geo = c.take<float4>(2 * k);
    s.skip = c.take<int32_t>(2 * k);
    s.Frep = c.take<float2>(k);
    s.full = c.take<float2>(k);
    s.rows_short = c.take<int32_t>(k);
    s.rows_med = c.take<int32_t>(k);
    s.rows_long = c.take<int32_t>(k);
    s.att_counts = c.take<uint32_t>(4);
    s.part = c.take<XPart>(2 * size_t(kMaxNodeBlocks));
    carve_hs(c, s.hs);
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
        note_launch(), k_init<<<grid_for(K, kThreads, sm_count() * 8), kThreads, 0, st>>>(
            K, p.seed, R, reinterpret_cast<float2 *>(pos), reinterpret_cast<float2 *>(Fprev));
        BGV_TRY(launch_status());
    }
    note_launch(), k_set_speed<<<1, 1, 0, st>>>(speed);
    return launch_status();
}

// Bounded-wait self check of the moment pass: one block as tile 1 of two
// tiles of bodies (all at the origin, body 0 everywhere, mass 0, frame side
// 1) whose tile 0 never runs, so its look-back must give up at the spin
// limit.  Writes stay within the two tiles' bodies and prefix records.
namespace {
struct WaitCheckMoments {
    uint32_t *perm, *mass, *start_count, *start_levels, *flags;
    float2 *pos;
    float4 *frame, *body;
    MomP *P;
    MomTile *agg, *incl;
};
void carve_wait_check_moments(Carver &c, WaitCheckMoments &w) {
    const size_t K = 2 * kMomTile;
    w.perm = c.take<uint32_t>(K);
    w.mass = c.take<uint32_t>(K);
    w.start_count = c.take<uint32_t>(K);
    w.start_levels = c.take<uint32_t>(K);
    w.flags = c.take<uint32_t>(3);
    w.pos = c.take<float2>(K);
    w.frame = c.take<float4>(1);
    w.body = c.take<float4>(K);
    w.P = c.take<MomP>(K + 1);
    w.agg = c.take<MomTile>(2);
    w.incl = c.take<MomTile>(2);
}
}  // namespace

size_t wait_check_moments_bytes() {
    Carver c(nullptr, 0);
    WaitCheckMoments w;
    carve_wait_check_moments(c, w);
    return c.used();
}

int wait_check_moments(void *scratch, uint32_t *dev_status, cudaStream_t st) {
    Carver c(scratch, 0);
    WaitCheckMoments w;
    carve_wait_check_moments(c, w);
    BGV_CUDA(cudaMemsetAsync(scratch, 0, wait_check_moments_bytes(), st));
    const float4 frame = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
    const uint32_t one = 1u;  // the tile counter (after the two tiles' flags)
    BGV_CUDA(cudaMemcpyAsync(w.frame, &frame, sizeof(frame), cudaMemcpyHostToDevice, st));
    BGV_CUDA(cudaMemcpyAsync(w.flags + 2, &one, sizeof(one), cudaMemcpyHostToDevice, st));
    note_launch(), k_gather_moments<<<1, kThreads, 0, st>>>(w.perm, 2 * kMomTile, w.pos, w.mass, w.frame, nullptr,
                                                            w.body, w.P, w.start_count, w.start_levels, w.flags,
                                                            w.agg, w.incl, dev_status, spin_limit());
    BGV_TRY(launch_status());
    return cudaStreamSynchronize(st) == cudaSuccess ? BGV_OK : BGV_ECUDA;
}

// Launch shapes of the step, process wide (bgv_autotune_fa2 picks them):
// the longest rows the attraction sums one lane each, threads per block of
// the traversal, blocks per SM of the persistent tail.  Packed in one word so a
// step reads a consistent set.
static std::atomic<uint32_t> g_fa2_tune{(32u << 16) | (128u << 4) | 4u};  // measured best on GB300 (rmat22x)
Fa2Tune fa2_tune() {
    const uint32_t w = g_fa2_tune.load(std::memory_order_relaxed);
    return Fa2Tune{int(w >> 16), int((w >> 4) & 0xFFFu), int(w & 0xFu)};
}
int set_fa2_tune(const Fa2Tune &t) {
    if ((t.att_short != 8 && t.att_short != 16 && t.att_short != 32) ||
        (t.repulse_threads != 128 && t.repulse_threads != 256) || t.tail_blocks_per_sm < 1 ||
        t.tail_blocks_per_sm > 8)
        return BGV_EINVAL;
    g_fa2_tune.store((uint32_t(t.att_short) << 16) | (uint32_t(t.repulse_threads) << 4) | uint32_t(t.tail_blocks_per_sm),
                     std::memory_order_relaxed);
    return BGV_OK;
}

// How a step after the first of a run finds the Morton order, process
// wide: 1 (default) the hinted sort from the previous step's order, 0 the
// full radix sort every step.  Both give the same order.
static std::atomic<int> g_fa2_order{1};
int fa2_order() { return g_fa2_order.load(std::memory_order_relaxed); }
int set_fa2_order(int method) {
    if (method != 0 && method != 1) return -1;
    return g_fa2_order.exchange(method, std::memory_order_relaxed);
}

// A second stream per host thread and device, made on first use.
cudaStream_t aux_stream() {
    static thread_local cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
        streams[dev] = nullptr;
    return streams[dev];
}

// A stream at the device's highest priority per host thread and device,
// made on first use.
cudaStream_t priority_stream() {
    static thread_local cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!streams[dev]) {
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&streams[dev], cudaStreamNonBlocking, greatest) != cudaSuccess)
            streams[dev] = nullptr;
    }
    return streams[dev];
}

// The two events of a fork onto the second stream and the join back,
// destroyed when the step's work has been enqueued (work already enqueued
// keeps them valid).
struct ForkJoin {
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaError_t make() {
        cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
        return e;
    }
    ~ForkJoin() {
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
    }
};

static int run_fa2_body(int mode, int64_t K, int64_t nnz, const int32_t *csr_off, const int32_t *csr_adj,
                        const uint32_t *csr_w, const uint32_t *mass, const bgv_fa2_params &p, float *pos_f, float *F_f,
                        float *Fprev_f, double *speed, float *Fr, float *Fa, float *Fg, WsHeader *hdr, void *scratch,
                        cudaStream_t st, cudaEvent_t *marks, bool build_plan, int32_t G, const int64_t *koff,
                        bool hinted) {
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
    const Fa2Tune tune = fa2_tune();
    auto mark = [&](int i) -> int {
        if (marks && cudaEventRecord(marks[i], st) != cudaSuccess) return BGV_ECUDA;
        return BGV_OK;
    };

    // The per-step counters are cleared by k_keys; S and T are written whole
    // by the node kernels; the last-block tickets are reset by their last
    // blocks (the header starts zeroed, see bgv_ws_init).
    BGV_TRY(mark(0));
    ForkJoin ev;
    cudaStream_t aux = nullptr;
    if (nnz > 0) {
        aux = aux_stream();
        if (!aux || ev.make() != cudaSuccess) return BGV_ECUDA;
    }
    // Once the second stream is forked, every way out of this function joins
    // it back into `st` (so `st` stays ordered after the attraction, and a
    // capture never ends with an unjoined fork).
    struct JoinGuard {
        cudaEvent_t ev = nullptr;
        cudaStream_t from = nullptr, into = nullptr;
        int join() {
            if (!ev) return BGV_OK;
            const cudaError_t a = cudaEventRecord(ev, from);
            const cudaError_t b = cudaStreamWaitEvent(into, ev, 0);
            ev = nullptr;
            return a == cudaSuccess && b == cudaSuccess ? BGV_OK : BGV_ECUDA;
        }
        ~JoinGuard() { join(); }
    } guard;
    // The attraction needs only the positions and the CSR: it runs on a
    // second stream while the tree is built and traversed, and k_node waits
    // for it.
    if (nnz > 0) {
        BGV_CUDA(cudaEventRecord(ev.fork, st));
        BGV_CUDA(cudaStreamWaitEvent(aux, ev.fork, 0));
        guard.ev = ev.join;
        guard.from = aux;
        guard.into = st;
        if (build_plan) {
            BGV_CUDA(cudaMemsetAsync(s.att_counts, 0, 4 * sizeof(uint32_t), aux));
            note_launch(), k_att_plan<<<grid_for(K, kThreads), kThreads, 0, aux>>>(
                K, csr_off, tune.att_short, s.rows_short, s.rows_med, s.rows_long, s.att_counts);
            BGV_TRY(launch_status());
        }
        note_launch(), k_att_short<<<grid_for(K, kThreads), kThreads, 0, aux>>>(K, csr_off, csr_adj, csr_w, pos,
                                                                                s.rows_short, s.att_counts, s.full);
        BGV_TRY(launch_status());
        note_launch(), k_att_medium<<<grid_for(K * 32, kThreads), kThreads, 0, aux>>>(
            K, csr_off, csr_adj, csr_w, pos, s.rows_med, s.att_counts, s.full);
        BGV_TRY(launch_status());
        note_launch(), k_att_long<<<sm_count() * 2, kThreads, 0, aux>>>(K, csr_off, csr_adj, csr_w, pos, s.rows_long,
                                                                        s.att_counts, s.full);
        BGV_TRY(launch_status());
    }
    if (batched)
        note_launch(), k_frame_seg<<<G, kThreads, 0, st>>>(pos, koff, s.frame, s.bgraph);
    else
        note_launch(), k_frame<<<frame_blocks(), kThreads, 0, st>>>(pos, K, s.frame_part, s.frame, &hdr->bbox_ticket);
    BGV_TRY(launch_status());
    const int64_t mom_tiles = (K + kMomTile - 1) / kMomTile;
    // the sorted order lands in the buffer pair the radix sort ends in, so
    // the next iteration finds its hint there whichever sort made it
    const int res = radix_sort_high_result(K, 2 * L + gbits);
    if (hinted && fa2_order() == 1 && K <= hs_max_keys()) {
        // the previous iteration's sorted ids are the hint; the sort also
        // clears the step counters and the moment flags, as k_keys does
        const MortonOf key_of{pos, s.frame, s.bgraph, L};
        HsClears clr;
        clr.u64 = &hdr->interactions;  // interactions, tree_nodes
        clr.n_u64 = 2;
        clr.u32 = s.mom_flags;
        clr.n_u32 = mom_tiles + 2;
        const uint32_t *hint = s.sort.vals[res];
        BGV_TRY(hinted_sort_samples(key_of, hint, K, s.hs, &hdr->status, st, clr));
        BGV_TRY(mark(1));
        // the pre-order arrays are free until k_preorder: the buckets' slots
        unsigned long long *slot_key = reinterpret_cast<unsigned long long *>(s.geo);
        uint32_t *slot_id = reinterpret_cast<uint32_t *>(slot_key + K);
        BGV_TRY(hinted_sort_place(key_of, hint, K, s.hs, s.sort.keys[res ^ 1], s.sort.vals[res ^ 1], slot_key, slot_id,
                                  s.sort.keys[res], s.sort.vals[res], &hdr->status, st));
    } else {
        const int gk = grid_for(K, kThreads, sm_count() * 16);
        note_launch(), k_keys<<<gk, kThreads, 0, st>>>(pos, K, s.frame, s.bgraph, L, s.sort.keys[0], s.sort.vals[0],
                                                       &hdr->interactions, s.mom_flags, mom_tiles + 2, s.sort.counts,
                                                       sort_counter_words());
        BGV_TRY(launch_status());
        BGV_TRY(mark(1));
        int got = 0;
        BGV_TRY(radix_sort_high(s.sort, s.runfix, K, nullptr, 2 * L + gbits, st, &got, &hdr->status, true));
        if (got != res) return BGV_EINVAL;  // radix_sort_high_result disagrees with the sort
    }
    BGV_TRY(mark(2));
    {
        note_launch(), k_gather_moments<<<unsigned(mom_tiles), kThreads, 0, st>>>(
            s.sort.vals[res], K, pos, mass, s.frame, s.bgraph, s.body, s.P, s.start_count,
            s.start_levels, s.mom_flags, s.mom_agg, s.mom_incl, &hdr->status, spin_limit());
        BGV_TRY(launch_status());
    }
    BGV_TRY(mark(3));
    if (K >= 2) {
        const unsigned gt = unsigned((K + kThreads - 1) / kThreads);
        const unsigned gi = unsigned((K - 1 + kThreads - 1) / kThreads);
        uint32_t *cand_count = s.mom_flags + mom_tiles + 1;  // cleared by k_keys
        note_launch(), k_tree_mark<<<gi, kThreads, 0, st>>>(s.sort.keys[res], K, L, gbits, s.cell_level, s.cand,
                                                            cand_count);
        BGV_TRY(launch_status());
        note_launch(), k_tree<<<grid_for(K, kThreads, sm_count() * 8), kThreads, 0, st>>>(
            s.sort.keys[res], K, L, gbits, p.leaf_cap, s.frame, s.bgraph, s.P, s.range, s.cell_level, s.cell,
            s.start_count, s.start_levels, &hdr->tree_nodes, s.cand, cand_count);
        BGV_TRY(launch_status());
        BGV_TRY(mark(4));
        BGV_TRY(scan_exclusive(s.start_count, s.T, K, nullptr, nullptr, true, s.scan_tmp, st));
        note_launch(), k_preorder<<<gt, kThreads, 0, st>>>(K, s.range, s.cell_level, s.start_levels, s.cell, s.T,
                                                           s.body, s.geo, s.skip);
        BGV_TRY(launch_status());
        BGV_TRY(mark(5));
        const float theta2 = p.theta * p.theta;
        if (tune.repulse_threads == 128) {
            const unsigned gr = unsigned((K + 127) / 128);
            note_launch(), k_repulse<128><<<gr, 128, 0, st>>>(s.geo, s.skip, s.T, koff, s.bgraph, s.body, K, p.kr,
                                                              theta2, s.Frep, &hdr->interactions,
                                                              &hdr->interactions_total);
        } else {
            const unsigned gr = unsigned((K + kThreads - 1) / kThreads);
            note_launch(), k_repulse<kThreads><<<gr, kThreads, 0, st>>>(s.geo, s.skip, s.T, koff, s.bgraph, s.body, K,
                                                                        p.kr, theta2, s.Frep, &hdr->interactions,
                                                                        &hdr->interactions_total);
        }
        BGV_TRY(launch_status());
    } else {
        BGV_CUDA(cudaMemsetAsync(s.Frep, 0, sizeof(float2), st));
        BGV_TRY(mark(4));
        BGV_TRY(mark(5));
    }
    BGV_TRY(mark(6));
    BGV_TRY(guard.join());  // the attraction ran alongside on the second stream
    BGV_TRY(mark(7));
    const float2 *att = nnz > 0 ? s.full : nullptr;
    if (mode == 0) {
        note_launch(), k_node<<<grid_for(K, kThreads, node_blocks()), kThreads, 0, st>>>(
            K, att, mass, pos, s.Frep, p.kg, p.strong_gravity, reinterpret_cast<float2 *>(Fr),
            reinterpret_cast<float2 *>(Fa), reinterpret_cast<float2 *>(Fg));
        BGV_TRY(launch_status());
    } else {
        float2 *rowst = batched ? s.rowst : nullptr;
        const int64_t *koff_d = batched ? koff : nullptr;
        const int32_t *bgraph = s.bgraph;
        int32_t g_count = G;
        float kg = p.kg, tau = p.tau, ks = p.ks, ksmax = p.ksmax;
        int strong = p.strong_gravity, limit = spin_limit();
        int64_t k_count = K;
        XPart *part = s.part;
        const float2 *frep = s.Frep;
        void *args[] = {&k_count, &att, &mass, &pos, &frep, &kg, &strong, &F, &Fprev, &part, &speed, &tau, &ks,
                        &ksmax, &hdr, &rowst, &koff_d, &bgraph, &g_count, &limit};
        const int blocks = coop_blocks(reinterpret_cast<const void *>(k_tail), kThreads,
                                       sm_count() * tune.tail_blocks_per_sm);
        BGV_TRY(launch_coop(reinterpret_cast<const void *>(k_tail), blocks, kThreads, args, st));
    }
    BGV_TRY(mark(8));
    return BGV_OK;
}

// The iteration's main chain runs on a high-priority stream forked from the
// caller's and joined back at the end: when SMs free up, its blocks go before
// those of the attraction, which runs beside it at the default priority.
int run_fa2(int mode, int64_t K, int64_t nnz, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
            const uint32_t *mass, const bgv_fa2_params &p, float *pos_f, float *F_f, float *Fprev_f, double *speed,
            float *Fr, float *Fa, float *Fg, WsHeader *hdr, void *scratch, cudaStream_t st, cudaEvent_t *marks,
            bool build_plan, int32_t G, const int64_t *koff, bool hinted) {
    if (K <= 0) return BGV_OK;
    cudaStream_t hp = priority_stream();
    ForkJoin ev;
    if (!hp || ev.make() != cudaSuccess) return BGV_ECUDA;
    BGV_CUDA(cudaEventRecord(ev.fork, st));
    BGV_CUDA(cudaStreamWaitEvent(hp, ev.fork, 0));
    const int rc = run_fa2_body(mode, K, nnz, csr_off, csr_adj, csr_w, mass, p, pos_f, F_f, Fprev_f, speed, Fr, Fa, Fg,
                                hdr, scratch, hp, marks, build_plan, G, koff, hinted);
    BGV_CUDA(cudaEventRecord(ev.join, hp));
    BGV_CUDA(cudaStreamWaitEvent(st, ev.join, 0));
    return rc;
}

}  // namespace bgv

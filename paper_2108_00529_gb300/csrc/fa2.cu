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
//   k_quad      quadtree nodes: binary nodes whose 2-bit level exceeds their
//               parent's; up to four children each; FP32 centre of mass from
//               the exact moments; leaf flags
//   k_repulse   Barnes-Hut repulsion: one warp per 32 Morton-consecutive
//               bodies walks the union of their traversals with a shared
//               stack of (node, lane mask) entries; every lane takes its own
//               opening decisions, so each body's interaction set is exactly
//               the one the sequential definition gives
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
constexpr int kNodeBlocks = 152 * 4;
constexpr int kStack = 96;             // >= 3 * (24 + 1) + 1
constexpr int kNone = INT32_MIN;       // empty child slot

typedef unsigned __int128 u128;

struct __align__(16) QNode {
    float4 a;    // decision/force centre x, y; mass; (cell side)^2
    int4 info;   // first body, last body (Morton positions), leaf flag, level
    int4 ch;     // children: >= 0 node id, < 0 ~body position, kNone empty
    int4 pad;
};

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
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    float4 r = __ldcg(&part[0]);
    for (unsigned b = 1; b < gridDim.x; ++b) {
        const float4 q = __ldcg(&part[b]);
        r.x = fminf(r.x, q.x); r.y = fminf(r.y, q.y);
        r.z = fmaxf(r.z, q.z); r.w = fmaxf(r.w, q.w);
    }
    const float ex = __fsub_rn(r.z, r.x), ey = __fsub_rn(r.w, r.y);
    const float ext = ex > ey ? ex : ey;
    float side = __fmul_rn(ext, 1.00000095367431640625f);  // 1 + 2^-20
    if (!(ext > 0.0f)) side = 1.0f;
    *frame = make_float4(r.x, r.y, side, 0.0f);
    *ticket = 0u;
}

// ------------------------------------------------------------------ keys
__global__ void __launch_bounds__(kThreads) k_keys(const float2 *__restrict__ pos, int64_t K,
                                                   const float4 *__restrict__ frame, int L,
                                                   unsigned long long *__restrict__ keys,
                                                   uint32_t *__restrict__ vals, uint2 *__restrict__ U) {
    const float4 fr = *frame;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < K; i += stride) {
        const float2 p = pos[i];
        const float ux = __fdiv_rn(__fsub_rn(p.x, fr.x), fr.z);
        const float uy = __fdiv_rn(__fsub_rn(p.y, fr.y), fr.z);
        const uint32_t Ux = __float2uint_rz(__fmul_rn(ux, 4294967296.0f));
        const uint32_t Uy = __float2uint_rz(__fmul_rn(uy, 4294967296.0f));
        const uint32_t qx = Ux >> (32 - L), qy = Uy >> (32 - L);
        keys[i] = (spread_bits(qx) << 1) | spread_bits(qy);
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
                                                         int L, int32_t *__restrict__ left,
                                                         int32_t *__restrict__ right, int32_t *__restrict__ parent,
                                                         int2 *__restrict__ range, int8_t *__restrict__ level,
                                                         int32_t *__restrict__ root) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= K - 1) return;
    const int kb = 2 * L;
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
    level[i] = static_cast<int8_t>(dnode >= kb ? L : (dnode >> 1));
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

__global__ void __launch_bounds__(kThreads) k_quad(int64_t K, int L, int leaf_cap, const float4 *__restrict__ frame,
                                                   const int32_t *__restrict__ left, const int32_t *__restrict__ right,
                                                   const int32_t *__restrict__ parent, const int2 *__restrict__ range,
                                                   const int8_t *__restrict__ level,
                                                   const unsigned long long *__restrict__ PM,
                                                   const ulonglong2 *__restrict__ PX,
                                                   const ulonglong2 *__restrict__ PY, QNode *__restrict__ q,
                                                   unsigned long long *tree_nodes) {
    const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    bool top = false;
    if (p < K - 1) {
        const int lev = level[p];
        const int32_t par = parent[p];
        const int par_lev = (par < 0 || int64_t(par) >= K - 1) ? -1 : int(level[par]);
        top = par_lev < lev;
        if (top) {
            const int2 rg = range[p];
            const int cnt = rg.y - rg.x + 1;
            const bool leaf = cnt <= leaf_cap || lev >= L;
            // A leaf made by the depth limit (coincident keys, more than
            // leaf_cap bodies) hides a chain of non-leaf cells with the same
            // bodies between its parent's level and L; the deepest of them,
            // at level L - 1, takes the opening test for the whole chain.
            const bool testable = leaf && cnt > leaf_cap && par_lev + 1 <= L - 1;
            int4 ch = make_int4(kNone, kNone, kNone, kNone);
            if (!leaf) {
                int refs[4];
                int nref = 0;
                const int32_t kids[2] = {left[p], right[p]};
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int32_t k = kids[c];
                    if (k < 0 || int(level[k]) > lev) {
                        refs[nref++] = k;
                    } else {  // same 2-bit level: part of this quadtree node
                        refs[nref++] = left[k];
                        refs[nref++] = right[k];
                    }
                }
                ch.x = refs[0];
                ch.y = nref > 1 ? refs[1] : kNone;
                ch.z = nref > 2 ? refs[2] : kNone;
                ch.w = nref > 3 ? refs[3] : kNone;
            }
            const float4 fr = *frame;
            const Mom hi = mom_load(PM, PX, PY, rg.y + 1), lo = mom_load(PM, PX, PY, rg.x);
            const unsigned long long M = hi.M - lo.M;
            const u128 X = hi.X - lo.X, Y = hi.Y - lo.Y;
            const uint32_t qx = M ? uint32_t(X / M) : 0u, qy = M ? uint32_t(Y / M) : 0u;
            const float cx = __fadd_rn(fr.x, __fmul_rn(fr.z, __fmul_rn(__uint2float_rn(qx), 2.3283064365386963e-10f)));
            const float cy = __fadd_rn(fr.y, __fmul_rn(fr.z, __fmul_rn(__uint2float_rn(qy), 2.3283064365386963e-10f)));
            const float sl = __fmul_rn(fr.z, pow2_neg(testable ? L - 1 : lev));
            QNode nd;
            nd.a = make_float4(cx, cy, __ull2float_rn(M), __fmul_rn(sl, sl));
            nd.info = make_int4(rg.x, rg.y, testable ? 2 : (leaf ? 1 : 0), lev);
            nd.ch = ch;
            nd.pad = make_int4(0, 0, 0, 0);
            q[p] = nd;
        }
    }
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, top);
    if ((threadIdx.x & 31) == 0 && mask) atomicAdd(tree_nodes, static_cast<unsigned long long>(__popc(mask)));
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

// Opening test of the quadtree definition, operation by operation in FP32
// round-to-nearest (no contraction), so it decides exactly as the oracle.
__device__ __forceinline__ bool accept_cell(float xi, float yi, float4 a, float theta2, float &dx, float &dy,
                                            float &d2) {
    dx = __fsub_rn(xi, a.x);
    dy = __fsub_rn(yi, a.y);
    d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    return a.w < __fmul_rn(theta2, d2);
}

__global__ void __launch_bounds__(kThreads) k_repulse(const QNode *__restrict__ q, const int32_t *__restrict__ root_p,
                                                      const float4 *__restrict__ body, int64_t K, float kr,
                                                      float theta2, float2 *__restrict__ Frep,
                                                      unsigned long long *inter_step,
                                                      unsigned long long *inter_total, uint32_t *status) {
    __shared__ int2 stack[kThreads / 32][kStack];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t s0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) & ~int64_t(31);
    if (s0 >= K) return;  // whole warp leaves together
    const int64_t s = s0 + lane;
    const bool active = s < K;
    const float4 bi = active ? body[s] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float xi = bi.x, yi = bi.y, kmi = kr * bi.z;
    const int si = int(s);
    float fx = 0.0f, fy = 0.0f;
    unsigned inter = 0;
    int2 *stk = stack[warp];
    const unsigned am = __ballot_sync(0xFFFFFFFFu, active);
    const int root = *root_p;
    if (root < 0 || int64_t(root) >= K - 1) {  // the tree build did not finish
        if (lane == 0) raise_status(status, BGV_DEV_STACK);
        return;
    }
    if (lane == 0) stk[0] = make_int2(root, int(am));
    int sp = 1;
    __syncwarp();
    while (sp > 0) {
        --sp;
        const int2 e = stk[sp];
        __syncwarp();
        const QNode *nd = q + e.x;
        const int4 info = nd->info;
        const float4 a = nd->a;
        const int4 ch = nd->ch;
        const bool mine = (unsigned(e.y) >> lane) & 1u;
        const bool own = si >= info.x && si <= info.y;
        if (info.z) {  // leaf: every body except self (a depth leaf may be accepted whole)
            bool direct = mine;
            if (mine && info.z == 2 && !own) {
                float dx, dy, d2;
                if (accept_cell(xi, yi, a, theta2, dx, dy, d2)) {
                    const float f = __fdividef(kmi * a.z, d2);
                    fx += f * dx;
                    fy += f * dy;
                    ++inter;
                    direct = false;
                }
            }
            if (__any_sync(0xFFFFFFFFu, direct)) {
                for (int t = info.x; t <= info.y; ++t) {
                    const float4 bj = body[t];
                    if (direct && t != si) {
                        add_body(xi, yi, kmi, bj, fx, fy);
                        ++inter;
                    }
                }
            }
            continue;
        }
        bool open = false;
        if (mine) {
            if (own) {
                open = true;  // the cell holds this body
            } else {
                float dx, dy, d2;
                if (accept_cell(xi, yi, a, theta2, dx, dy, d2)) {
                    const float f = __fdividef(kmi * a.z, d2);
                    fx += f * dx;
                    fy += f * dy;
                    ++inter;
                } else {
                    open = true;
                }
            }
        }
        const unsigned om = __ballot_sync(0xFFFFFFFFu, open);
        if (!om) continue;
        // Children in order; single bodies are summed at once, cells pushed
        // (last child first, so the first child is visited next).
        const int kids[4] = {ch.x, ch.y, ch.z, ch.w};
        int npush = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int k = kids[c];
            if (k == kNone) continue;
            if (k < 0) {
                const int b = ~k;
                const float4 bj = body[b];
                if (open && b != si) {
                    add_body(xi, yi, kmi, bj, fx, fy);
                    ++inter;
                }
            } else {
                ++npush;
            }
        }
        if (sp + npush > kStack) {
            if (lane == 0) raise_status(status, BGV_DEV_STACK);
            break;
        }
        if (lane == 0) {
#pragma unroll
            for (int c = 3; c >= 0; --c)
                if (kids[c] >= 0) stk[sp++] = make_int2(kids[c], int(om));
        } else {
            sp += npush;
        }
        __syncwarp();
    }
    if (active) {
        const int orig = __float_as_int(bi.w);
        Frep[orig] = make_float2(fx, fy);
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

__device__ __forceinline__ int64_t row_containing(const int32_t *__restrict__ off, int64_t K, int64_t e) {
    int64_t lo = 0, hi = K;  // off[lo] <= e < off[hi]
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (int64_t(__ldg(&off[mid])) <= e) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kThreads) k_attract(int64_t K, int64_t nnz, const int32_t *__restrict__ off,
                                                      const int32_t *__restrict__ adj,
                                                      const uint32_t *__restrict__ w, const float2 *__restrict__ pos,
                                                      float2 *__restrict__ full, float2 *__restrict__ head,
                                                      float2 *__restrict__ tail) {
    const int64_t chunks = (nnz + kChunk - 1) / kChunk;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < chunks; g += stride) {
        const int64_t e0 = g * kChunk, e1 = e0 + kChunk < nnz ? e0 + kChunk : nnz;
        int64_t r = row_containing(off, K, e0);
        int64_t rs = off[r], re = off[r + 1];
        float2 pi = pos[r];
        float ax = 0.0f, ay = 0.0f;
        for (int64_t e = e0; e < e1; ++e) {
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
            const int32_t j = adj[e];
            if (static_cast<uint64_t>(j) >= static_cast<uint64_t>(K)) continue;  // invalid CSR entry
            const float2 pj = pos[j];
            const float wt = __uint2float_rn(w[e]);
            ax += wt * (pj.x - pi.x);
            ay += wt * (pj.y - pi.y);
        }
        if (rs >= e0 && re <= e1) full[r] = make_float2(ax, ay);
        else if (rs < e0) head[g] = make_float2(ax, ay);
        else tail[g] = make_float2(ax, ay);
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

__global__ void __launch_bounds__(kThreads) k_node(int mode, int64_t K, const int32_t *__restrict__ off,
                                                   const float2 *__restrict__ full, const float2 *__restrict__ head,
                                                   const float2 *__restrict__ tail,
                                                   const uint32_t *__restrict__ mass, const float2 *__restrict__ pos,
                                                   const float2 *__restrict__ Frep, float kg, int strong,
                                                   float2 *__restrict__ F, const float2 *__restrict__ Fprev,
                                                   float2 *__restrict__ Fr_out, float2 *__restrict__ Fa_out,
                                                   float2 *__restrict__ Fg_out, double2 *part, double *speed,
                                                   float tau, WsHeader *hdr) {
    Comp S{0.0, 0.0}, T{0.0, 0.0};
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < K; i += stride) {
        const int64_t b = off[i], e = off[i + 1];
        float ax = 0.0f, ay = 0.0f;
        if (e > b) {
            const int64_t g1 = b / kChunk, g2 = (e - 1) / kChunk;
            if (g1 == g2) {
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
        const float2 pi = pos[i];
        const float m = __uint2float_rn(mass[i]);
        float gx, gy;
        if (strong) {
            gx = -kg * m * pi.x;
            gy = -kg * m * pi.y;
        } else {
            const float rr = sqrtf(pi.x * pi.x + pi.y * pi.y);
            gx = rr > 0.0f ? -kg * m * pi.x / rr : 0.0f;
            gy = rr > 0.0f ? -kg * m * pi.y / rr : 0.0f;
        }
        const float2 fr = Frep[i];
        if (mode == 0) {
            if (Fr_out) Fr_out[i] = fr;
            if (Fa_out) Fa_out[i] = make_float2(ax, ay);
            if (Fg_out) Fg_out[i] = make_float2(gx, gy);
        } else {
            const float fx = fr.x + ax + gx, fy = fr.y + ay + gy;
            F[i] = make_float2(fx, fy);
            const float2 fp = Fprev[i];
            const float sx = fx - fp.x, sy = fy - fp.y, tx = fx + fp.x, ty = fy + fp.y;
            const double md = double(mass[i]);
            S = comp_add(S, md * double(sqrtf(sx * sx + sy * sy)));
            T = comp_add(T, md * 0.5 * double(sqrtf(tx * tx + ty * ty)));
        }
    }
    if (mode == 0) return;
    __shared__ bool last;
    block_merge(S, T);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = make_double2(S.s, S.c);
        part[2 * blockIdx.x + 1] = make_double2(T.s, T.c);
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

__global__ void __launch_bounds__(kThreads) k_update(int64_t K, const float2 *__restrict__ F, float2 *__restrict__ Fprev,
                                                     float2 *__restrict__ pos, const double *__restrict__ speed,
                                                     float ks, float ksmax) {
    const float sp = float(*speed);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < K; i += stride) {
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
}  // namespace

// ------------------------------------------------------------- scratch
struct Fa2Scratch {
    float4 *frame;
    float4 *frame_part;
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
    QNode *q;
    float2 *Frep;
    float2 *full, *head, *tail;
    double2 *part;  // two per block: (S, comp), (T, comp)
};

static void carve_fa2(Carver &c, int64_t K, int64_t nnz, Fa2Scratch &s) {
    const size_t k = size_t(K > 0 ? K : 1);
    const size_t chunks = size_t((nnz > 0 ? nnz : 1) + kChunk - 1) / kChunk;
    s.frame = c.take<float4>(1);
    s.frame_part = c.take<float4>(kFrameBlocks);
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
    s.q = c.take<QNode>(k);
    s.Frep = c.take<float2>(k);
    s.full = c.take<float2>(k);
    s.head = c.take<float2>(chunks);
    s.tail = c.take<float2>(chunks);
    s.part = c.take<double2>(2 * kNodeBlocks);
}

size_t fa2_scratch_bytes(int64_t K, int64_t nnz) {
    Carver c(nullptr, 0);
    Fa2Scratch s;
    carve_fa2(c, K, nnz, s);
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

int run_fa2_init(int64_t K, const bgv_fa2_params &p, float *pos, float *Fprev, double *speed, cudaStream_t st) {
    if (K > 0) {
        const float R = __builtin_sqrtf(float(K));
        note_launch(), k_init<<<grid_for(K, kThreads, 152 * 8), kThreads, 0, st>>>(K, p.seed, R, reinterpret_cast<float2 *>(pos),
                                                                   reinterpret_cast<float2 *>(Fprev));
        BGV_TRY(launch_status());
    }
    note_launch(), k_set_speed<<<1, 1, 0, st>>>(speed);
    return launch_status();
}

int run_fa2(int mode, int64_t K, int64_t nnz, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
            const uint32_t *mass, const bgv_fa2_params &p, float *pos_f, float *F_f, float *Fprev_f, double *speed,
            float *Fr, float *Fa, float *Fg, WsHeader *hdr, void *scratch, cudaStream_t st, cudaEvent_t *marks) {
    if (K <= 0) return BGV_OK;
    Carver c(scratch, 0);
    Fa2Scratch s;
    carve_fa2(c, K, nnz, s);
    float2 *pos = reinterpret_cast<float2 *>(pos_f);
    float2 *F = reinterpret_cast<float2 *>(F_f);
    float2 *Fprev = reinterpret_cast<float2 *>(Fprev_f);
    const int L = p.max_depth;
    auto mark = [&](int i) -> int {
        if (marks && cudaEventRecord(marks[i], st) != cudaSuccess) return BGV_ECUDA;
        return BGV_OK;
    };

    // per-step counters and last-block tickets
    BGV_CUDA(cudaMemsetAsync(reinterpret_cast<char *>(hdr) + offsetof(WsHeader, interactions), 0,
                             offsetof(WsHeader, reserved) - offsetof(WsHeader, interactions), st));
    BGV_TRY(mark(0));
    note_launch(), k_frame<<<kFrameBlocks, kThreads, 0, st>>>(pos, K, s.frame_part, s.frame, &hdr->bbox_ticket);
    BGV_TRY(launch_status());
    const int gk = grid_for(K, kThreads, 152 * 16);
    note_launch(), k_keys<<<gk, kThreads, 0, st>>>(pos, K, s.frame, L, s.sort.keys[0], s.sort.vals[0], s.U);
    BGV_TRY(launch_status());
    BGV_TRY(mark(1));
    int res = 0;
    BGV_TRY(radix_sort(s.sort, K, nullptr, 2 * L, st, &res, &hdr->status));
    BGV_TRY(mark(2));
    note_launch(), k_gather<<<gk, kThreads, 0, st>>>(s.sort.vals[res], K, pos, mass, s.U, s.body, s.sU, s.smass);
    BGV_TRY(launch_status());
    BGV_TRY(mark(3));
    if (K >= 2) {
        const unsigned gt = unsigned((K + kThreads - 1) / kThreads);
        const unsigned gi = unsigned((K - 1 + kThreads - 1) / kThreads);
        const unsigned tiles = unsigned((K + kMomTile - 1) / kMomTile);
        note_launch(), k_radix_tree<<<gi, kThreads, 0, st>>>(s.sort.keys[res], K, L, s.left, s.right, s.parent,
                                                             s.range, s.level, s.root);
        BGV_TRY(launch_status());
        note_launch(), k_mom_reduce<<<tiles, kThreads, 0, st>>>(s.sU, s.smass, K, s.TM, s.TX, s.TY);
        note_launch(), k_mom_tiles<<<1, kThreads, 0, st>>>(s.TM, s.TX, s.TY, tiles);
        note_launch(), k_mom_down<<<tiles, kThreads, 0, st>>>(s.sU, s.smass, K, s.TM, s.TX, s.TY, s.PM, s.PX, s.PY);
        BGV_TRY(launch_status());
        BGV_TRY(mark(4));
        note_launch(), k_quad<<<gi, kThreads, 0, st>>>(K, L, p.leaf_cap, s.frame, s.left, s.right, s.parent, s.range,
                                                       s.level, s.PM, s.PX, s.PY, s.q, &hdr->tree_nodes);
        BGV_TRY(launch_status());
        BGV_TRY(mark(5));
        const float theta2 = p.theta * p.theta;
        note_launch(), k_repulse<<<gt, kThreads, 0, st>>>(s.q, s.root, s.body, K, p.kr, theta2, s.Frep,
                                                          &hdr->interactions, &hdr->interactions_total,
                                                          &hdr->status);
        BGV_TRY(launch_status());
    } else {
        BGV_CUDA(cudaMemsetAsync(s.Frep, 0, sizeof(float2), st));
        BGV_TRY(mark(4));
        BGV_TRY(mark(5));
    }
    BGV_TRY(mark(6));
    if (nnz > 0) {
        note_launch(), k_attract<<<grid_for((nnz + kChunk - 1) / kChunk, kThreads, 152 * 16), kThreads, 0, st>>>(
            K, nnz, csr_off, csr_adj, csr_w, pos, s.full, s.head, s.tail);
        BGV_TRY(launch_status());
    }
    note_launch(), k_node<<<kNodeBlocks, kThreads, 0, st>>>(mode, K, csr_off, s.full, s.head, s.tail, mass, pos,
                                                            s.Frep, p.kg, p.strong_gravity, F, Fprev,
                                                            reinterpret_cast<float2 *>(Fr),
                                                            reinterpret_cast<float2 *>(Fa),
                                                            reinterpret_cast<float2 *>(Fg), s.part, speed, p.tau, hdr);
    BGV_TRY(launch_status());
    BGV_TRY(mark(7));
    if (mode == 1) {
        note_launch(), k_update<<<gk, kThreads, 0, st>>>(K, F, Fprev, pos, speed, p.ks, p.ksmax);
        BGV_TRY(launch_status());
    }
    BGV_TRY(mark(8));
    return BGV_OK;
}

}  // namespace bgv

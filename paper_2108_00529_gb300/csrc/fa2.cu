// fa2.cu -- ForceAtlas2 on the supergraph (Section 3.1, Algorithm 1).
//
// One iteration is a fixed chain of kernels with no host round trip:
//   k_frame     bounding square of the positions (last-block finalise)
//   k_keys      fixed-point coordinates U and 2L-bit Morton keys
//   radix sort  (key, body) pairs -> Morton order
//   k_gather    bodies in Morton order (position, mass, fixed coords)
//   k_tree      bottom-up binary radix tree over the sorted keys: each leaf
//               climbs, the second child to reach a parent merges the two
//               (one atomicExch per node), carrying exact integer moments
//               (sum m, sum m*Ux, sum m*Uy in 64/128-bit integers)
//   k_quad      quadtree nodes: binary nodes whose 2-bit level exceeds their
//               parent's; up to four children each; FP32 centre of mass from
//               the exact moments; leaf flags
//   k_repulse   Barnes-Hut repulsion: one warp per 32 Morton-consecutive
//               bodies walks the union of their traversals with a shared
//               stack of (node, lane mask) entries; every lane takes its own
//               opening decisions, so each body's interaction set is exactly
//               the one the sequential definition gives
//   k_node      attraction (one warp per CSR row), gravity, total force,
//               swing and traction (FP64 block partials); the last block sums
//               the partials with Kahan compensation and updates the speed
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
                                                     uint2 *__restrict__ sU, uint32_t *__restrict__ smass,
                                                     int32_t *__restrict__ other) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; s < K; s += stride) {
        const uint32_t i = perm[s];
        const float2 p = pos[i];
        const uint32_t m = mass[i];
        body[s] = make_float4(p.x, p.y, __uint2float_rn(m), __int_as_float(int(i)));
        sU[s] = U[i];
        smass[s] = m;
        other[s] = -1;
    }
}

// ------------------------------------------------------------------ tree
// Distance between Morton neighbours j and j+1: the highest differing key
// bit (as bit position + 1, shifted up), or for equal keys the index bits,
// which always compare below any key difference.  Smaller = more similar.
__device__ __forceinline__ unsigned long long sep_dist(const unsigned long long *keys, int64_t j) {
    const unsigned long long x = __ldg(&keys[j]) ^ __ldg(&keys[j + 1]);
    if (x) return static_cast<unsigned long long>(64 - __clzll(static_cast<long long>(x))) << 32;
    return static_cast<unsigned long long>(uint32_t(j) ^ uint32_t(j + 1));
}

// Quadtree level (2-bit prefix length) of the binary node split at j.
__device__ __forceinline__ int sep_level(const unsigned long long *keys, int64_t j, int L) {
    const unsigned long long x = __ldg(&keys[j]) ^ __ldg(&keys[j + 1]);
    if (!x) return L;
    const int hb = 63 - __clzll(static_cast<long long>(x));
    return (2 * L - 1 - hb) >> 1;
}

struct Moments {
    unsigned long long M;
    u128 X, Y;
};

__global__ void __launch_bounds__(kThreads) k_tree(const unsigned long long *__restrict__ keys, int64_t K,
                                                   const uint2 *__restrict__ sU, const uint32_t *__restrict__ smass,
                                                   int32_t *other, int32_t *left, int32_t *right, int32_t *parent,
                                                   int2 *range, unsigned long long *nM, ulonglong2 *nX,
                                                   ulonglong2 *nY, int32_t *root) {
    const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= K) return;
    int64_t l = s, r = s;
    int32_t cur = ~int32_t(s);
    Moments mo;
    {
        const uint2 u = sU[s];
        const unsigned long long m = smass[s];
        mo.M = m;
        mo.X = u128(m) * u.x;
        mo.Y = u128(m) * u.y;
    }
    while (true) {
        bool as_left;
        if (l == 0) as_left = true;
        else if (r == K - 1) as_left = false;
        else as_left = sep_dist(keys, r) < sep_dist(keys, l - 1);
        const int64_t p = as_left ? r : l - 1;
        if (as_left) left[p] = cur; else right[p] = cur;
        if (cur >= 0) parent[cur] = int32_t(p);
        __threadfence();
        const int32_t prev = atomicExch(&other[p], as_left ? int32_t(l) : int32_t(r));
        if (prev < 0) return;  // the sibling is still climbing; it finishes p
        __threadfence();
        if (as_left) r = prev; else l = prev;
        const int32_t sib = __ldcg(as_left ? &right[p] : &left[p]);
        if (sib < 0) {
            const int32_t b = ~sib;
            const uint2 u = sU[b];
            const unsigned long long m = smass[b];
            mo.M += m;
            mo.X += u128(m) * u.x;
            mo.Y += u128(m) * u.y;
        } else {
            const ulonglong2 x = __ldcg(&nX[sib]), y = __ldcg(&nY[sib]);
            mo.M += __ldcg(&nM[sib]);
            mo.X += (u128(x.y) << 64) | x.x;
            mo.Y += (u128(y.y) << 64) | y.x;
        }
        nM[p] = mo.M;
        nX[p] = make_ulonglong2(static_cast<unsigned long long>(mo.X), static_cast<unsigned long long>(mo.X >> 64));
        nY[p] = make_ulonglong2(static_cast<unsigned long long>(mo.Y), static_cast<unsigned long long>(mo.Y >> 64));
        range[p] = make_int2(int32_t(l), int32_t(r));
        cur = int32_t(p);
        if (l == 0 && r == K - 1) {
            parent[p] = -1;
            *root = int32_t(p);
            return;
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_quad(const unsigned long long *__restrict__ keys, int64_t K, int L,
                                                   int leaf_cap, const float4 *__restrict__ frame,
                                                   const int32_t *__restrict__ left, const int32_t *__restrict__ right,
                                                   const int32_t *__restrict__ parent, const int2 *__restrict__ range,
                                                   const unsigned long long *__restrict__ nM,
                                                   const ulonglong2 *__restrict__ nX,
                                                   const ulonglong2 *__restrict__ nY, QNode *__restrict__ q,
                                                   unsigned long long *tree_nodes) {
    const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    bool top = false;
    if (p < K - 1) {
        const int lev = sep_level(keys, p, L);
        const int32_t par = parent[p];
        top = par < 0 || int64_t(par) >= K - 1 || sep_level(keys, par, L) < lev;
        if (top) {
            const int2 rg = range[p];
            const int cnt = rg.y - rg.x + 1;
            const bool leaf = cnt <= leaf_cap || lev >= L;
            // A leaf made by the depth limit (coincident keys, more than
            // leaf_cap bodies) hides a chain of non-leaf cells with the same
            // bodies between its parent's level and L; the deepest of them,
            // at level L - 1, takes the opening test for the whole chain.
            const int par_lev = (par < 0 || int64_t(par) >= K - 1) ? -1 : sep_level(keys, par, L);
            const bool testable = leaf && cnt > leaf_cap && par_lev + 1 <= L - 1;
            int4 ch = make_int4(kNone, kNone, kNone, kNone);
            if (!leaf) {
                int refs[4];
                int nref = 0;
                const int32_t kids[2] = {left[p], right[p]};
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int32_t k = kids[c];
                    if (k < 0 || sep_level(keys, k, L) > lev) {
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
            const unsigned long long M = nM[p];
            const ulonglong2 x = nX[p], y = nY[p];
            const u128 X = (u128(x.y) << 64) | x.x, Y = (u128(y.y) << 64) | y.x;
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
        const float f = kmi * bj.z / d2;
        fx += f * dx;
        fy += f * dy;
    }
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
    int sp = 0;
    const unsigned am = __ballot_sync(0xFFFFFFFFu, active);
    const int root = *root_p;
    if (root < 0 || int64_t(root) >= K - 1) {  // the tree build did not finish
        if (lane == 0) raise_status(status, BGV_DEV_STACK);
        return;
    }
    if (lane == 0) stk[0] = make_int2(root, int(am));
    sp = 1;
    __syncwarp();
    while (sp > 0) {
        --sp;
        const int2 e = stk[sp];
        __syncwarp();
        const bool mine = (unsigned(e.y) >> lane) & 1u;
        if (e.x < 0) {  // a single body
            const int b = ~e.x;
            if (mine && b != si) {
                add_body(xi, yi, kmi, body[b], fx, fy);
                ++inter;
            }
            continue;
        }
        const QNode *nd = q + e.x;
        const int4 info = nd->info;
        if (info.z) {  // leaf: every body except self (a depth leaf may be accepted whole)
            bool direct = mine;
            if (mine && info.z == 2 && !(si >= info.x && si <= info.y)) {
                const float4 a = nd->a;
                const float dx = __fsub_rn(xi, a.x), dy = __fsub_rn(yi, a.y);
                const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                if (a.w < __fmul_rn(theta2, d2)) {
                    const float f = kmi * a.z / d2;
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
            if (si >= info.x && si <= info.y) {
                open = true;  // the cell holds this body
            } else {
                const float4 a = nd->a;
                const float dx = __fsub_rn(xi, a.x), dy = __fsub_rn(yi, a.y);
                const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                if (a.w < __fmul_rn(theta2, d2)) {
                    const float f = kmi * a.z / d2;
                    fx += f * dx;
                    fy += f * dy;
                    ++inter;
                } else {
                    open = true;
                }
            }
        }
        const unsigned om = __ballot_sync(0xFFFFFFFFu, open);
        if (om) {
            const int4 ch = nd->ch;
            const int nch = 1 + (ch.y != kNone) + (ch.z != kNone) + (ch.w != kNone);
            if (sp + nch > kStack) {
                if (lane == 0) raise_status(status, BGV_DEV_STACK);
                break;
            }
            if (lane == 0) {
                int t = sp + nch;
                if (ch.w != kNone) stk[--t] = make_int2(ch.w, int(om));
                if (ch.z != kNone) stk[--t] = make_int2(ch.z, int(om));
                if (ch.y != kNone) stk[--t] = make_int2(ch.y, int(om));
                stk[--t] = make_int2(ch.x, int(om));
            }
            sp += nch;
            __syncwarp();
        }
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

// ------------------------------------------------------ node forces, speed
__global__ void __launch_bounds__(kThreads) k_node(int mode, int64_t K, const int32_t *__restrict__ csr_off,
                                                   const int32_t *__restrict__ csr_adj,
                                                   const uint32_t *__restrict__ csr_w,
                                                   const uint32_t *__restrict__ mass, const float2 *__restrict__ pos,
                                                   const float2 *__restrict__ Frep, float kg, int strong,
                                                   float2 *__restrict__ F, const float2 *__restrict__ Fprev,
                                                   float2 *__restrict__ Fr_out, float2 *__restrict__ Fa_out,
                                                   float2 *__restrict__ Fg_out, double2 *part, double *speed,
                                                   float tau, WsHeader *hdr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t gwarp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    double sw_acc = 0.0, tr_acc = 0.0;  // lane 0 only
    for (int64_t i = gwarp; i < K; i += nwarps) {
        const float2 pi = pos[i];
        const int32_t b = csr_off[i], e = csr_off[i + 1];
        float ax = 0.0f, ay = 0.0f;
        for (int32_t t = b + lane; t < e; t += 32) {
            const int32_t j = csr_adj[t];
            if (static_cast<uint64_t>(j) >= static_cast<uint64_t>(K)) continue;  // invalid CSR entry
            const float2 pj = pos[j];
            const float w = __uint2float_rn(csr_w[t]);
            ax += w * (pj.x - pi.x);
            ay += w * (pj.y - pi.y);
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            ax += __shfl_xor_sync(0xFFFFFFFFu, ax, d);
            ay += __shfl_xor_sync(0xFFFFFFFFu, ay, d);
        }
        if (lane == 0) {
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
                sw_acc += md * double(sqrtf(sx * sx + sy * sy));
                tr_acc += md * 0.5 * double(sqrtf(tx * tx + ty * ty));
            }
        }
    }
    if (mode == 0) return;
    __shared__ double2 wsum[kThreads / 32];
    __shared__ bool last;
    if (lane == 0) wsum[warp] = make_double2(sw_acc, tr_acc);
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            a += wsum[w].x;
            c += wsum[w].y;
        }
        part[blockIdx.x] = make_double2(a, c);
        __threadfence();
        last = atomicAdd(&hdr->node_ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    // Kahan-compensated sums over the block partials, in block order.
    double S = 0.0, cS = 0.0, T = 0.0, cT = 0.0;
    for (unsigned bk = 0; bk < gridDim.x; ++bk) {
        const double2 pv = __ldcg(&part[bk]);
        const double yS = pv.x - cS, tS = S + yS;
        cS = (tS - S) - yS;
        S = tS;
        const double yT = pv.y - cT, tT = T + yT;
        cT = (tT - T) - yT;
        T = tT;
    }
    double sp = *speed;
    if (S > 0.0) {
        const double target = double(tau) * T / S;
        const double rise = target - sp, cap = 0.5 * sp;
        sp += rise < cap ? rise : cap;
    }
    *speed = sp;
    hdr->S = S;
    hdr->T = T;
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
    int32_t *other, *left, *right, *parent, *root;
    int2 *range;
    unsigned long long *nM;
    ulonglong2 *nX, *nY;
    QNode *q;
    float2 *Frep;
    double2 *part;
};

static void carve_fa2(Carver &c, int64_t K, Fa2Scratch &s) {
    const size_t k = size_t(K > 0 ? K : 1);
    s.frame = c.take<float4>(1);
    s.frame_part = c.take<float4>(kFrameBlocks);
    carve_sort(c, int64_t(k), true, s.sort);
    s.U = c.take<uint2>(k);
    s.body = c.take<float4>(k);
    s.sU = c.take<uint2>(k);
    s.smass = c.take<uint32_t>(k);
    s.other = c.take<int32_t>(k);
    s.left = c.take<int32_t>(k);
    s.right = c.take<int32_t>(k);
    s.parent = c.take<int32_t>(k);
    s.root = c.take<int32_t>(1);
    s.range = c.take<int2>(k);
    s.nM = c.take<unsigned long long>(k);
    s.nX = c.take<ulonglong2>(k);
    s.nY = c.take<ulonglong2>(k);
    s.q = c.take<QNode>(k);
    s.Frep = c.take<float2>(k);
    s.part = c.take<double2>(kNodeBlocks);
}

size_t fa2_scratch_bytes(int64_t K, int64_t nnz) {
    (void)nnz;
    Carver c(nullptr, 0);
    Fa2Scratch s;
    carve_fa2(c, K, s);
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

int run_fa2(int mode, int64_t K, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
            const uint32_t *mass, const bgv_fa2_params &p, float *pos_f, float *F_f, float *Fprev_f, double *speed,
            float *Fr, float *Fa, float *Fg, WsHeader *hdr, void *scratch, cudaStream_t st, cudaEvent_t *marks) {
    if (K <= 0) return BGV_OK;
    Carver c(scratch, 0);
    Fa2Scratch s;
    carve_fa2(c, K, s);
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
    BGV_TRY(radix_sort(s.sort, K, nullptr, 2 * L, st, &res));
    BGV_TRY(mark(2));
    note_launch(), k_gather<<<gk, kThreads, 0, st>>>(s.sort.vals[res], K, pos, mass, s.U, s.body, s.sU, s.smass,
                                                     s.other);
    BGV_TRY(launch_status());
    BGV_TRY(mark(3));
    if (K >= 2) {
        const unsigned gt = unsigned((K + kThreads - 1) / kThreads);
        BGV_CUDA(cudaMemsetAsync(s.root, 0xFF, sizeof(int32_t), st));
        note_launch(), k_tree<<<gt, kThreads, 0, st>>>(s.sort.keys[res], K, s.sU, s.smass, s.other, s.left, s.right,
                                                       s.parent, s.range, s.nM, s.nX, s.nY, s.root);
        BGV_TRY(launch_status());
        BGV_TRY(mark(4));
        note_launch(), k_quad<<<unsigned((K - 1 + kThreads - 1) / kThreads), kThreads, 0, st>>>(
            s.sort.keys[res], K, L, p.leaf_cap, s.frame, s.left, s.right, s.parent, s.range, s.nM, s.nX, s.nY, s.q,
            &hdr->tree_nodes);
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
    note_launch(), k_node<<<kNodeBlocks, kThreads, 0, st>>>(mode, K, csr_off, csr_adj, csr_w, mass, pos, s.Frep, p.kg,
                                                            p.strong_gravity, F, Fprev, reinterpret_cast<float2 *>(Fr),
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

// style.cu -- supernode colour groups (Section 4.3) and drawing the discs
// into an image (Section 4.1 radii, Section 4.3 colours).
//
// Communities are ordered by size (a stable radix sort of (size, id), so
// ties keep id order).  With alpha the total size, the longest prefix of
// that order whose sizes sum to at most alpha / 2 is group 0 (drawn brown);
// the remaining R communities get group 1 + floor(10 * rank / R), from small
// to big.  One block then walks the sorted sizes three times (sums, brown
// count, groups); prefix sums are 64-bit.
#include "bgv_internal.cuh"

namespace bgv {
namespace {
constexpr int kStyleThreads = 1024;

__global__ void k_size_keys(const uint32_t *__restrict__ size, int64_t K, unsigned long long *__restrict__ keys,
                            uint32_t *__restrict__ vals) {
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < K; k += int64_t(gridDim.x) * blockDim.x) {
        keys[k] = size[k];
        vals[k] = uint32_t(k);
    }
}

__device__ unsigned long long block_exclusive_u64(unsigned long long x, unsigned long long *total) {
    __shared__ unsigned long long warp_sums[kStyleThreads / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int w = 0; w < kStyleThreads / 32; ++w) {
            const unsigned long long t = warp_sums[w];
            warp_sums[w] = run;
            run += t;
        }
        warp_sums[kStyleThreads / 32] = run;
    }
    __syncthreads();
    const unsigned long long r = warp_sums[warp] + inc - x;
    *total = warp_sums[kStyleThreads / 32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kStyleThreads) k_colour_groups(const unsigned long long *__restrict__ sizes,
                                                                 const uint32_t *__restrict__ order, int64_t K,
                                                                 uint8_t *__restrict__ group) {
    const int64_t chunk = (K + kStyleThreads - 1) / kStyleThreads;
    const int64_t lo = int64_t(threadIdx.x) * chunk, hi = lo + chunk < K ? lo + chunk : K;
    unsigned long long mine = 0;
    for (int64_t r = lo; r < hi; ++r) mine += sizes[r];
    unsigned long long total;
    unsigned long long cum = block_exclusive_u64(mine, &total);
    // brown: the running size, this community included, stays within alpha/2
    unsigned long long brown = 0;
    for (int64_t r = lo; r < hi; ++r) {
        cum += sizes[r];
        brown += (2 * cum <= total) ? 1 : 0;
    }
    unsigned long long half;
    block_exclusive_u64(brown, &half);
    const int64_t rest = K - int64_t(half);
    for (int64_t r = lo; r < hi; ++r) {
        const int64_t k = order[r];
        group[k] = r < int64_t(half) ? uint8_t(0) : uint8_t(1 + (10 * (r - int64_t(half))) / rest);
    }
}

// Whole-graph drawing (Section 4.3): every node takes its supernode's colour.
__global__ void k_node_colours(int32_t n, const int32_t *__restrict__ node_map, int64_t K,
                               const uint8_t *__restrict__ group, uint8_t *__restrict__ node_colour) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        const int32_t k = node_map[v];
        node_colour[v] = (k >= 0 && k < K) ? group[k] : uint8_t(0);
    }
}
}  // namespace

}  // namespace bgv

using namespace bgv;

namespace {
void carve_style(Carver &c, int64_t K, SortBuffers &sort) { carve_sort(c, K > 0 ? K : 1, true, sort); }
}  // namespace

extern "C" size_t bgv_colour_groups_ws_size(int64_t K) {
    Carver c(nullptr, kHeaderBytes);
    SortBuffers sort;
    carve_style(c, K, sort);
    return c.used();
}

extern "C" int bgv_colour_groups(int64_t K, const uint32_t *sizes, uint8_t *group, int32_t n,
                                 const int32_t *node_map, uint8_t *node_colour, void *ws, size_t ws_bytes,
                                 void *stream) {
    if (K < 0 || K >= 0x7FFFFFFF || (K > 0 && (!sizes || !group))) return BGV_EINVAL;
    if (node_colour && (n < 0 || (n > 0 && !node_map))) return BGV_EINVAL;
    if (!ws || reinterpret_cast<uintptr_t>(ws) % kAlign) return BGV_EINVAL;
    if (ws_bytes < bgv_colour_groups_ws_size(K)) return BGV_ENOSPC;
    if (K == 0) return BGV_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Carver c(ws, kHeaderBytes);
    SortBuffers sort;
    carve_style(c, K, sort);
    note_launch(), k_size_keys<<<grid_for(K, 256, sm_count() * 8), 256, 0, st>>>(sizes, K, sort.keys[0], sort.vals[0]);
    BGV_TRY(launch_status());
    int res = 0;
    BGV_TRY(radix_sort(sort, K, nullptr, 32, st, &res, status_ptr(ws)));
    note_launch(), k_colour_groups<<<1, kStyleThreads, 0, st>>>(sort.keys[res], sort.vals[res], K, group);
    BGV_TRY(launch_status());
    if (node_colour && n > 0) {
        note_launch(), k_node_colours<<<grid_for(n, 256, sm_count() * 8), 256, 0, st>>>(n, node_map, K, group, node_colour);
        BGV_TRY(launch_status());
    }
    return BGV_OK;
}

// ------------------------------------------------------------- drawing
// Discs of radius r (sqrt of the size, Section 4.1) in the colour of their
// group (Section 4.3), splatted into an RGBA image: the discs' bounding box
// maps to the pixels with one scale s = min(W, H) / largest extent; pixel
// (px, py) shows the disc whose scaled circle covers its centre (px + 0.5,
// py + 0.5); overlaps keep the smaller radius, then the smaller id.  One
// warp per disc marks the covered pixels with an atomicMax of (priority,
// id); a second pass shades.  FP32 with explicit round-to-nearest
// operations, so the coverage equals the plain definition's.
namespace bgv {
namespace {
__constant__ uint8_t c_palette[11][3] = {
    {177, 89, 40},   {202, 178, 214}, {106, 61, 154}, {253, 191, 111}, {255, 127, 0}, {251, 154, 153},
    {227, 26, 28},   {178, 223, 138}, {51, 160, 44},  {166, 206, 227}, {31, 120, 180}};

__global__ void __launch_bounds__(kStyleThreads) k_render_frame(const float2 *__restrict__ xy,
                                                                const float *__restrict__ radius, int64_t K,
                                                                int32_t W, int32_t H, float4 *frame) {
    float lx = INFINITY, ly = INFINITY, hx = -INFINITY, hy = -INFINITY;
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x) {
        const float2 p = xy[k];
        const float r = radius[k];
        lx = fminf(lx, __fsub_rn(p.x, r)); ly = fminf(ly, __fsub_rn(p.y, r));
        hx = fmaxf(hx, __fadd_rn(p.x, r)); hy = fmaxf(hy, __fadd_rn(p.y, r));
    }
    __shared__ float4 part[kStyleThreads / 32];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        lx = fminf(lx, __shfl_xor_sync(0xFFFFFFFFu, lx, d)); ly = fminf(ly, __shfl_xor_sync(0xFFFFFFFFu, ly, d));
        hx = fmaxf(hx, __shfl_xor_sync(0xFFFFFFFFu, hx, d)); hy = fmaxf(hy, __shfl_xor_sync(0xFFFFFFFFu, hy, d));
    }
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = make_float4(lx, ly, hx, hy);
    __syncthreads();
    if (threadIdx.x != 0) return;
    float4 b = part[0];
    for (int w = 1; w < kStyleThreads / 32; ++w) {
        b.x = fminf(b.x, part[w].x); b.y = fminf(b.y, part[w].y);
        b.z = fmaxf(b.z, part[w].z); b.w = fmaxf(b.w, part[w].w);
    }
    const float ex = __fsub_rn(b.z, b.x), ey = __fsub_rn(b.w, b.y);
    const float ext = ex > ey ? ex : ey;
    const float s = (K > 0 && ext > 0.0f) ? __fdiv_rn(float(W < H ? W : H), ext) : 1.0f;
    *frame = make_float4(b.x, b.y, s, 0.0f);
}

__global__ void __launch_bounds__(kStyleThreads) k_render_splat(const float2 *__restrict__ xy,
                                                                const float *__restrict__ radius, int64_t K,
                                                                int32_t W, int32_t H, const float4 *frame,
                                                                unsigned long long *__restrict__ zbuf) {
    const int lane = threadIdx.x & 31;
    const float4 f = *frame;
    const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t k = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; k < K; k += warps) {
        const float2 p = xy[k];
        const float r = radius[k];
        const float u = __fmul_rn(__fsub_rn(p.x, f.x), f.z), v = __fmul_rn(__fsub_rn(p.y, f.y), f.z);
        const float rs = __fmul_rn(r, f.z), rs2 = __fmul_rn(rs, rs);
        // pixels whose centre can lie within rs of (u, v), one pixel of slack
        const int x0 = max(0, int(floorf(u - rs)) - 1), x1 = min(W - 1, int(ceilf(u + rs)) + 1);
        const int y0 = max(0, int(floorf(v - rs)) - 1), y1 = min(H - 1, int(ceilf(v + rs)) + 1);
        if (!(rs >= 0.0f) || x0 > x1 || y0 > y1) continue;
        const unsigned long long key =
            (static_cast<unsigned long long>(0xFFFFFFFFu - __float_as_uint(r)) << 32) | (0xFFFFFFFFull - uint64_t(k));
        const int bw = x1 - x0 + 1;
        const int64_t cells = int64_t(bw) * (y1 - y0 + 1);
        for (int64_t c = lane; c < cells; c += 32) {
            const int px = x0 + int(c % bw), py = y0 + int(c / bw);
            const float dx = __fsub_rn(__fadd_rn(float(px), 0.5f), u), dy = __fsub_rn(__fadd_rn(float(py), 0.5f), v);
            const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
            if (d2 <= rs2) atomicMax(&zbuf[size_t(py) * W + px], key);
        }
    }
}

__global__ void __launch_bounds__(kStyleThreads) k_render_shade(const unsigned long long *__restrict__ zbuf,
                                                                int64_t pixels, int64_t K,
                                                                const uint8_t *__restrict__ group,
                                                                uchar4 *__restrict__ rgba) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < pixels;
         i += int64_t(gridDim.x) * blockDim.x) {
        const unsigned long long z = zbuf[i];
        uchar4 o = make_uchar4(255, 255, 255, 255);
        if (z) {
            const int64_t k = int64_t(0xFFFFFFFFull - (z & 0xFFFFFFFFull));
            const uint8_t g = k < K ? group[k] : 0;
            const int c = g <= 10 ? g : 0;
            o = make_uchar4(c_palette[c][0], c_palette[c][1], c_palette[c][2], 255);
        }
        rgba[i] = o;
    }
}
}  // namespace
}  // namespace bgv

extern "C" size_t bgv_render_ws_size(int32_t W, int32_t H) {
    Carver c(nullptr, kHeaderBytes);
    c.take<float4>(1);
    c.take<unsigned long long>(size_t(W > 0 ? W : 1) * size_t(H > 0 ? H : 1));
    return c.used();
}

extern "C" int bgv_render(int64_t K, const float *xy, const float *radius, const uint8_t *group, int32_t W, int32_t H,
                          uint8_t *rgba, void *ws, size_t ws_bytes, void *stream) {
    if (K < 0 || K >= 0xFFFFFFFFll || W < 1 || H < 1 || W > 32768 || H > 32768 || !rgba) return BGV_EINVAL;
    if (K > 0 && (!xy || !radius || !group || reinterpret_cast<uintptr_t>(xy) % 8)) return BGV_EINVAL;
    if (reinterpret_cast<uintptr_t>(rgba) % 4) return BGV_EINVAL;
    if (!ws || reinterpret_cast<uintptr_t>(ws) % kAlign) return BGV_EINVAL;
    if (ws_bytes < bgv_render_ws_size(W, H)) return BGV_ENOSPC;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Carver c(ws, kHeaderBytes);
    float4 *frame = c.take<float4>(1);
    const int64_t pixels = int64_t(W) * H;
    unsigned long long *zbuf = c.take<unsigned long long>(size_t(pixels));
    BGV_CUDA(cudaMemsetAsync(zbuf, 0, sizeof(unsigned long long) * size_t(pixels), st));
    const float2 *p = reinterpret_cast<const float2 *>(xy);
    note_launch(), k_render_frame<<<1, kStyleThreads, 0, st>>>(p, radius, K, W, H, frame);
    BGV_TRY(launch_status());
    if (K > 0) {
        note_launch(), k_render_splat<<<grid_for(K * 32, kStyleThreads, sm_count() * 16), kStyleThreads, 0, st>>>(
            p, radius, K, W, H, frame, zbuf);
        BGV_TRY(launch_status());
    }
    note_launch(), k_render_shade<<<grid_for(pixels, kStyleThreads, sm_count() * 8), kStyleThreads, 0, st>>>(
        zbuf, pixels, K, group, reinterpret_cast<uchar4 *>(rgba));
    return launch_status();
}

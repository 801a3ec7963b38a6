// hsort.cu -- the hinted sort as a public entry point (keys from an array):
// the same kernels the ForceAtlas2 step runs on its Morton keys.
#include "hsort.cuh"

namespace bgv {
namespace {

struct KeyArray {
    const unsigned long long *keys;
    __device__ unsigned long long operator()(uint32_t id) const { return __ldg(&keys[id]); }
};

struct HsWs {
    HsBuffers h;
    unsigned long long *tmp_key, *slot_key;
    uint32_t *tmp_bucket, *slot_id;
};

void carve_hs_ws(Carver &c, int64_t K, HsWs &w) {
    const size_t k = size_t(K > 0 ? K : 1);
    carve_hs(c, w.h);
    w.tmp_key = c.take<unsigned long long>(k);
    w.tmp_bucket = c.take<uint32_t>(k);
    w.slot_key = c.take<unsigned long long>(k);
    w.slot_id = c.take<uint32_t>(k);
}

bool aligned_to(const void *p, size_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; }

bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
    const char *x = static_cast<const char *>(a), *y = static_cast<const char *>(b);
    return x < y + nb && y < x + na;
}

}  // namespace
}  // namespace bgv

using namespace bgv;

extern "C" {

int64_t bgv_sort_hinted_max_keys(void) { return hs_max_keys(); }

size_t bgv_sort_hinted_ws_size(int64_t K) {
    if (K < 0 || K > hs_max_keys()) return 0;
    Carver c(nullptr, kHeaderBytes);
    HsWs w;
    carve_hs_ws(c, K, w);
    return c.used();
}

int bgv_sort_hinted(const uint64_t *keys, const uint32_t *hint, int64_t K, uint64_t *out_keys, uint32_t *out_ids,
                    void *ws, size_t ws_bytes, void *stream) {
    if (K < 0 || K > hs_max_keys() || !ws || !aligned_to(ws, kAlign)) return BGV_EINVAL;
    if (ws_bytes < bgv_sort_hinted_ws_size(K)) return BGV_ENOSPC;
    if (K == 0) return BGV_OK;
    if (!keys || !hint || !out_keys || !out_ids) return BGV_EINVAL;
    if (!aligned_to(keys, 8) || !aligned_to(out_keys, 8) || !aligned_to(hint, 4) || !aligned_to(out_ids, 4))
        return BGV_EINVAL;
    const size_t kb = sizeof(uint64_t) * size_t(K), ib = sizeof(uint32_t) * size_t(K);
    if (overlaps(out_keys, kb, keys, kb) || overlaps(out_keys, kb, hint, ib) || overlaps(out_ids, ib, keys, kb) ||
        overlaps(out_ids, ib, hint, ib) || overlaps(out_keys, kb, out_ids, ib))
        return BGV_EINVAL;
    Carver c(ws, kHeaderBytes);
    HsWs w;
    carve_hs_ws(c, K, w);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t *status = status_ptr(ws);
    const KeyArray key_of{reinterpret_cast<const unsigned long long *>(keys)};
    BGV_TRY(hinted_sort_samples(key_of, hint, K, w.h, status, st));
    BGV_TRY(hinted_sort_place(key_of, hint, K, w.h, w.tmp_key, w.tmp_bucket, w.slot_key, w.slot_id,
                              reinterpret_cast<unsigned long long *>(out_keys), out_ids, status, st));
    uint32_t dev_status = 0;
    BGV_CUDA(cudaMemcpyAsync(&dev_status, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    BGV_CUDA(cudaStreamSynchronize(st));
    return dev_status ? BGV_EDEVICE : BGV_OK;
}

int32_t bgv_set_fa2_order(int32_t method) { return set_fa2_order(method); }

}  // extern "C"

// tsqs_wide.cu -- large elements (Section VIII.G-H).
//
// The paper sorts an array of pointers when elements are large and then moves each
// element once along the cycles of the permutation ("late swapping").  On the GPU the
// pointer array becomes 16-byte records (order-preserving image of the key, original
// index), sorted by the record path of the hot path; equal keys are then ordered by
// their index, so the result is the stable order and unique.  One gather pass moves
// every element to its place in a scratch array, and a copy brings it back.
#include <cuda_runtime.h>

#include "tsqs.h"
#include "tsqs_kernels.cuh"

namespace tsqs {

namespace {

// records[i] = (order-preserving image of element i's key, i)
template <int KIND>
__global__ void k_wide_keys(const unsigned char *__restrict__ base, uint64_t n, uint64_t es,
                            uint64_t key_off, Rec16 *__restrict__ rec) {
    using K = Key<KIND>;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const typename K::S k = *reinterpret_cast<const typename K::S *>(base + i * es + key_off);
        Rec16 r;
        r.key = (unsigned long long)K::canon(k);      // canonical keys are unsigned: zero-extend
        r.pay = i;
        rec[i] = r;
    }
}

// dst element i = src element rec[i].pay; a group of 2^lg lanes copies one element,
// word by word (W = 4 or 16 bytes)
template <class W>
__global__ void k_wide_gather(const W *__restrict__ src, uint64_t n, uint32_t words, uint32_t lg,
                              const Rec16 *__restrict__ rec, W *__restrict__ dst) {
    const uint64_t gt = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint32_t lane = (uint32_t)(gt & ((1u << lg) - 1u));
    const uint64_t groups = ((uint64_t)gridDim.x * blockDim.x) >> lg;
    for (uint64_t i = gt >> lg; i < n; i += groups) {
        const uint64_t j = rec[i].pay;
        const W *s = src + j * words;
        W *d = dst + i * words;
        for (uint32_t w = lane; w < words; w += 1u << lg) d[w] = s[w];
    }
}

}  // namespace

int wide_keys(int kind, const void *base, uint64_t n, uint64_t es, uint64_t key_off, void *rec,
              int sms, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned char *b = (const unsigned char *)base;
    Rec16 *r = (Rec16 *)rec;
    const dim3 grid(sms * 4), block(256);
    switch (kind) {
    case TSQS_I32: k_wide_keys<TSQS_I32><<<grid, block, 0, s>>>(b, n, es, key_off, r); break;
    case TSQS_U32: k_wide_keys<TSQS_U32><<<grid, block, 0, s>>>(b, n, es, key_off, r); break;
    case TSQS_F32: k_wide_keys<TSQS_F32><<<grid, block, 0, s>>>(b, n, es, key_off, r); break;
    case TSQS_I64: k_wide_keys<TSQS_I64><<<grid, block, 0, s>>>(b, n, es, key_off, r); break;
    case TSQS_U64: k_wide_keys<TSQS_U64><<<grid, block, 0, s>>>(b, n, es, key_off, r); break;
    case TSQS_F64: k_wide_keys<TSQS_F64><<<grid, block, 0, s>>>(b, n, es, key_off, r); break;
    default: return TSQS_EINVAL;
    }
    return cudaGetLastError() == cudaSuccess ? TSQS_OK : TSQS_ECUDA;
}

int wide_gather(const void *src, uint64_t n, uint64_t es, const void *rec, void *dst, int sms,
                void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const bool vec = es % 16 == 0 && ((uintptr_t)src & 15u) == 0 && ((uintptr_t)dst & 15u) == 0;
    const uint64_t words = vec ? es / 16 : es / 4;
    uint32_t lg = 0;                                  // lanes per element: up to 32
    while ((1ull << lg) < words && lg < 5) lg++;
    const dim3 grid(sms * 8), block(256);
    if (vec)
        k_wide_gather<uint4><<<grid, block, 0, s>>>((const uint4 *)src, n, (uint32_t)words, lg,
                                                    (const Rec16 *)rec, (uint4 *)dst);
    else
        k_wide_gather<unsigned int><<<grid, block, 0, s>>>((const unsigned int *)src, n, (uint32_t)words,
                                                           lg, (const Rec16 *)rec, (unsigned int *)dst);
    return cudaGetLastError() == cudaSuccess ? TSQS_OK : TSQS_ECUDA;
}

}  // namespace tsqs

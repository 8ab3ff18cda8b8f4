// Device helpers shared by the kernels: typed loads, calibration, candidate append.
#pragma once

#include "hs_internal.cuh"

namespace hs {

// Read element i of a spectrum stored as T and widen it to FP32 (exact for FP16 and BF16).
template <typename T>
__device__ __forceinline__ float ldx(const T* p, uint32_t i);
template <>
__device__ __forceinline__ float ldx<float>(const float* p, uint32_t i) {
    return __ldg(p + i);
}
template <>
__device__ __forceinline__ float ldx<__half>(const __half* p, uint32_t i) {
    return __half2float(__ldg(p + i));
}
template <>
__device__ __forceinline__ float ldx<__nv_bfloat16>(const __nv_bfloat16* p, uint32_t i) {
    return __bfloat162float(__ldg(p + i));
}

template <typename T>
__device__ __forceinline__ float widen(T v);
template <>
__device__ __forceinline__ float widen<float>(float v) {
    return v;
}
template <>
__device__ __forceinline__ float widen<__half>(__half v) {
    return __half2float(v);
}
template <>
__device__ __forceinline__ float widen<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

// snr_H = (S * c_H - mu_H) * isig_H, each operation rounded separately (no contraction).
__device__ __forceinline__ float calibrate(const Tables& t, float S, int H) {
    return __fmul_rn(__fsub_rn(__fmul_rn(S, t.c[H]), t.mu[H]), t.isig[H]);
}

// Two FP32 sums per instruction: each half is rounded exactly as a separate add would be.
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 r;
    asm("add.rn.f32x2 %0, %1, %2;"
        : "=l"(*reinterpret_cast<unsigned long long*>(&r))
        : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)));
    return r;
}

// Running best over H: replaced only on a strictly larger snr, so the smallest H wins ties.
__device__ __forceinline__ void keep_best(float snr, int H, float& best, int& bh) {
    if (snr > best) {
        best = snr;
        bh = H;
    }
}

// Merge of two first-largest reductions over disjoint sets of H: the larger snr, or on equal snr the
// smaller H, which is what one scan over H = 1, 2, .. with strict > would keep.
__device__ __forceinline__ void merge_best(float p, int q, float& best, int& bh) {
    if (p > best || (p == best && q < bh)) {
        best = p;
        bh = q;
    }
}

// Warp-aggregated append of at most one candidate per lane.  Must be reached by all 32 lanes.
__device__ __forceinline__ void append_candidate(bool hit, hs_candidate* cand, unsigned long long* count,
                                                 long long cap, unsigned* status, uint32_t spec, uint32_t bin,
                                                 float snr, int z, int h, int variant) {
    unsigned mask = __ballot_sync(0xffffffffu, hit);
    if (mask == 0u) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (hit) {
        unsigned long long pos = base + (unsigned long long)__popc(mask & ((1u << lane) - 1u));
        if (pos < (unsigned long long)cap) {
            uint4 v;
            v.x = spec;
            v.y = bin;
            v.z = __float_as_uint(snr);
            v.w = (uint32_t)(uint16_t)(int16_t)z | ((uint32_t)h << 16) | ((uint32_t)variant << 24);
            reinterpret_cast<uint4*>(cand)[pos] = v;
        } else {
            atomicOr(status, kStatusOverflow);
        }
    }
}

// Last spectrum s with prefix[s] <= item (spectra with no tiles are skipped over).
__device__ __forceinline__ int find_spectrum(const int64_t* prefix, int n_spectra, unsigned long long item) {
    int lo = 0, hi = n_spectra - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if ((unsigned long long)__ldg(prefix + mid) <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace hs

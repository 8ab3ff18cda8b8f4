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

// ---- Eq. 2 windows (the 1-D kernels and the row-wise 2-D form) ----
// Largest of the elements [w0, w1] (inclusive, w0 <= w1 <= N-1), read in aligned 16-byte chunks so a
// window of i bins costs about i/4 + 1 loads.
template <typename T>
__device__ __forceinline__ float window_max16(const T* x, uint32_t N, uint32_t w0, uint32_t w1) {
    constexpr uint32_t E = 16 / sizeof(T);  // elements per chunk
    const uint32_t c0 = w0 / E, c1 = w1 / E;
    if (c1 >= N / E) {  // the window reaches the partial chunk at the end: plain loads
        float m = -INFINITY;
        for (uint32_t k = w0; k <= w1; ++k) m = fmaxf(m, ldx(x, k));
        return m;
    }
    const uint4* cx = reinterpret_cast<const uint4*>(x);
    float m = -INFINITY;
    {
        uint4 raw = __ldg(cx + c0);
        const T* e = reinterpret_cast<const T*>(&raw);
#pragma unroll
        for (uint32_t k = 0; k < E; ++k) {
            uint32_t pos = c0 * E + k;
            if (pos >= w0 && pos <= w1) m = fmaxf(m, widen<T>(e[k]));
        }
    }
    for (uint32_t c = c0 + 1; c < c1; ++c) {
        uint4 raw = __ldg(cx + c);
        const T* e = reinterpret_cast<const T*>(&raw);
#pragma unroll
        for (uint32_t k = 0; k < E; ++k) m = fmaxf(m, widen<T>(e[k]));
    }
    if (c1 > c0) {
        uint4 raw = __ldg(cx + c1);
        const T* e = reinterpret_cast<const T*>(&raw);
#pragma unroll
        for (uint32_t k = 0; k < E; ++k)
            if (c1 * E + k <= w1) m = fmaxf(m, widen<T>(e[k]));
    }
    return m;
}

// One aligned 32-byte chunk through the non-coherent path in a single 256-bit load (sm_100 and later).
struct Chunk32 {
    uint32_t w[8];
};
__device__ __forceinline__ Chunk32 ld_chunk32(const void* p) {
    Chunk32 c;
    asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(c.w[0]), "=r"(c.w[1]), "=r"(c.w[2]), "=r"(c.w[3]), "=r"(c.w[4]), "=r"(c.w[5]), "=r"(c.w[6]),
          "=r"(c.w[7])
        : "l"(p));
    return c;
}
template <typename T>
__device__ __forceinline__ float chunk_elem(const Chunk32& c, uint32_t k);  // element k of the chunk
template <>
__device__ __forceinline__ float chunk_elem<float>(const Chunk32& c, uint32_t k) {
    return __uint_as_float(c.w[k]);
}
template <>
__device__ __forceinline__ float chunk_elem<__half>(const Chunk32& c, uint32_t k) {
    return __half2float(__ushort_as_half((unsigned short)(c.w[k >> 1] >> (16 * (k & 1)))));
}
template <>
__device__ __forceinline__ float chunk_elem<__nv_bfloat16>(const Chunk32& c, uint32_t k) {
    return __uint_as_float((c.w[k >> 1] >> (16 * (k & 1))) << 16);  // a bfloat16 is the high half of a float
}

// The same in 32-byte chunks aligned on the address (a spectrum starts 16-byte aligned, so chunk
// boundaries are taken from x rounded down to 32 bytes), about i/8 + 1 loads for a window of i bins.
// A window whose chunks would reach before the spectrum's first element or past its last is read
// element by element instead.
template <typename T>
__device__ __forceinline__ float window_max32(const T* x, uint32_t N, uint32_t w0, uint32_t w1) {
    constexpr uint32_t E = 32 / sizeof(T);  // elements per chunk
    const uint32_t sh = (uint32_t)(reinterpret_cast<uintptr_t>(x) & 31u) / (uint32_t)sizeof(T);
    const uint32_t a0 = w0 + sh, a1 = w1 + sh;  // positions from x - sh, which is 32-byte aligned
    const uint32_t c0 = a0 / E, c1 = a1 / E;
    float m = -INFINITY;
    if (c0 * E < sh || (c1 + 1u) * E > N + sh) {
        for (uint32_t k = w0; k <= w1; ++k) m = fmaxf(m, ldx(x, k));
        return m;
    }
    const T* xa = x - sh;
    {
        const Chunk32 c = ld_chunk32(xa + c0 * E);
#pragma unroll
        for (uint32_t k = 0; k < E; ++k) {
            const uint32_t pos = c0 * E + k;
            if (pos >= a0 && pos <= a1) m = fmaxf(m, chunk_elem<T>(c, k));
        }
    }
    for (uint32_t cc = c0 + 1; cc < c1; ++cc) {
        const Chunk32 c = ld_chunk32(xa + cc * E);
#pragma unroll
        for (uint32_t k = 0; k < E; ++k) m = fmaxf(m, chunk_elem<T>(c, k));
    }
    if (c1 > c0) {
        const Chunk32 c = ld_chunk32(xa + c1 * E);
#pragma unroll
        for (uint32_t k = 0; k < E; ++k)
            if (c1 * E + k <= a1) m = fmaxf(m, chunk_elem<T>(c, k));
    }
    return m;
}

// Largest of the elements [w0, w1] of a window of i bins.  FP32 windows of kWide32 or more bins take
// 32-byte chunks (half the load requests: Eq. 2 4-7% faster on the DM-trial batch than 16-byte
// chunks, and faster than starting them at 9 bins); 16-bit storage keeps 16-byte chunks (32-byte
// ones measured 26% slower there: unpacking 16 halves per chunk costs more than the requests saved).
// The maximum is exact, so the order of comparison does not change its value (and inputs carry no
// NaN).
constexpr int kWide32 = 5;
template <typename T>
__device__ __forceinline__ float window_max(const T* x, uint32_t N, uint32_t w0, uint32_t w1, int i) {
    if constexpr (sizeof(T) == 4) {
        if (i >= kWide32) return window_max32(x, N, w0, w1);
    }
    return window_max16(x, N, w0, w1);
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

// The Farey sequence of order 32 and the exact fixed-point form of the Eq. 1 index, shared by the
// 1-D kernels.
#pragma once

#include <initializer_list>
#include <utility>

#include "hs_common.cuh"

namespace hs {

// Eq. 1.  The index of harmonic i of H at output bin n, round-half-up(n*i/H), depends only on the
// reduced fraction i/H, so each of the 324 distinct fractions of F_32 (the Farey sequence of order
// 32) is read once and added to every S_H it belongs to.  Visiting the fractions in increasing
// order adds the terms of each S_H in the order i = 1..H, as the definition does.
struct Frac {
    int p, q;
};
__host__ __device__ constexpr Frac farey_at(int k) {  // k-th term of F_32 after 0/1: 1/32, 1/31, ..., 1/1
    Frac a{0, 1}, b{1, 32};
    for (int i = 0; i < k; ++i) {
        int m = (32 + a.q) / b.q;
        Frac c{m * b.p - a.p, m * b.q - a.q};
        a = b;
        b = c;
    }
    return b;
}
constexpr int kNumFrac = 324;
static_assert(farey_at(kNumFrac - 1).p == 1 && farey_at(kNumFrac - 1).q == 1, "F_32 has 324 terms after 0/1");

// round-half-up(n*p/q) = floor((n*F + 2^31) / 2^32) with F = ceil(2^32 p/q): the error n*(F - 2^32 p/q)
// / 2^32 < 2^-6 <= 1/(2q) for n < 2^26 never reaches the next multiple of 1/(2q), so this is exact.
// It is evaluated in 32-bit pieces: high word of n*F plus the carry of (low word + 2^31).
template <int P, int Q>
struct FracConst {
    static constexpr uint32_t F = (uint32_t)((((uint64_t)P << 32) + Q - 1) / Q);
};

template <int P, int Q>
__device__ __forceinline__ uint32_t frac_index(uint32_t n) {
    if (Q == 1) return n;
    constexpr uint32_t F = FracConst<P, Q>::F;
    return __umulhi(n, F) + ((n * F) >> 31);
}

// Power-of-two stages (HS_FLAG_POW2_STAGES): only H = 1, 2, 4, .. are searched.  A stage H = m q
// of fraction p/q needs q and m to be powers of two, so Eq. 1 then reads only the fractions i/32.
__host__ __device__ constexpr bool is_pow2(int v) {
    return (v & (v - 1)) == 0;
}

// Generic hmax: one output per call, harmonics beyond hmax skipped (and, with P2, every H that is
// not a stage).
template <typename T, int K, bool P2 = false>
__device__ __forceinline__ void farey_step(const T* x, uint32_t n, int hmax, float (&S)[kHmax + 1]) {
    constexpr Frac f = farey_at(K);
    if constexpr (!P2 || is_pow2(f.q)) {
        const float v = widen<T>(__ldg(x + frac_index<f.p, f.q>(n)));
#pragma unroll
        for (int m = 1; m * f.q <= kHmax; ++m)
            if ((!P2 || is_pow2(m)) && m * f.q <= hmax) S[m * f.q] = __fadd_rn(S[m * f.q], v);
    }
}

template <typename T, bool P2 = false, int... K>
__device__ __forceinline__ void farey_all(const T* x, uint32_t n, int hmax, float (&S)[kHmax + 1],
                                          std::integer_sequence<int, K...>) {
    (farey_step<T, K, P2>(x, n, hmax, S), ...);  // in increasing fraction order
}


// Sets of H as bit masks (bit H-1), for sweeps that keep only some of the sums S_H live at a time: a
// reduced fraction p/q is read by a set when the set holds a multiple of q.
__host__ __device__ constexpr bool in_hset(uint32_t M, int H) { return H >= 1 && H <= 32 && ((M >> (H - 1)) & 1u); }
__host__ __device__ constexpr int hslot(uint32_t M, int H) {  // position of H among the set's members
    int s = 0;
    for (int h = 1; h < H; ++h) s += in_hset(M, h) ? 1 : 0;
    return s;
}
__host__ __device__ constexpr int hset_size(uint32_t M) { return hslot(M, 33); }
__host__ __device__ constexpr bool frac_in_hset(uint32_t M, int q) {
    for (int m = 1; m * q <= 32; ++m)
        if (in_hset(M, m * q)) return true;
    return false;
}
__host__ __device__ constexpr uint32_t hset(std::initializer_list<int> hs) {
    uint32_t m = 0;
    for (int h : hs) m |= 1u << (h - 1);
    return m;
}

}  // namespace hs

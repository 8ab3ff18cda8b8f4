// 1-D harmonic-sum kernels: the four variants of Section 2 (Eq. 1-4), one spectrum per launch or a
// packed batch of spectra walked by one persistent launch over a (spectrum, tile) work queue.
#include <algorithm>
#include <type_traits>
#include <utility>

#include "hs_common.cuh"
#include "hs_farey.cuh"

namespace hs {

// ------------------------------------------------------------------------------------------
// Per-bin evaluation of one variant.  Writes best snr / H (and the Eq. 4 path) of output bin n,
// and, when all_h is set, the snr of every H (-inf where H is not valid).
// ------------------------------------------------------------------------------------------

template <int V, typename T>
struct Bin;

// ------------------------------------------------------------------------------------------
// Eq. 1 with hmax = 32 and no every-H table: outputs n and n+1 together, H = 1..32 in passes.
//
// Pairs: for a fraction f <= 1 the bins of outputs n and n+1 differ by 0 or 1.  With W = n F + 2^31,
// bin(n) = W >> 32 and bin(n+1) = (W + F) >> 32, one more exactly when the low word of W carries on
// adding F.  Both candidates are loaded and the carry picks one.  The low word of W is lo + 2^31
// (lo = low word of n F), and an unsigned compare of lo + 2^31 is a signed compare of lo itself:
// (lo + 2^31 mod 2^32) >u ~F  <=>  (int)lo > (int)(~F ^ 2^31).  The two sums of a pair share one
// packed add.
//
// Passes: the 32 packed sums of a pair would stay live through the whole Farey sweep (64
// registers).  H = 1..32 is instead split into three sets of 10-11 sums, each swept over the
// fractions it needs in increasing order (so every S_H still adds its terms in the order i = 1..H),
// which halves the registers and doubles the warps an SM holds.  A fraction p/q is read by every pass
// holding a multiple of q; these sets (from a local search over splits) repeat only 10 of the 324
// fractions.  Each pass reduces its own H with the first-largest rule and the passes merge with
// "larger snr, or equal snr and smaller H", which gives the same best H as one scan over H = 1..32.
// ------------------------------------------------------------------------------------------
constexpr uint32_t kEq1Pass0 = hset({3, 5, 7, 10, 14, 15, 20, 21, 25, 28, 30});
constexpr uint32_t kEq1Pass1 = hset({4, 6, 8, 9, 12, 16, 18, 24, 27, 29, 32});
constexpr uint32_t kEq1Pass2 = hset({1, 2, 11, 13, 17, 19, 22, 23, 26, 31});
constexpr uint32_t kPow2Stages = hset({1, 2, 4, 8, 16, 32});
static_assert((kEq1Pass0 | kEq1Pass1 | kEq1Pass2) == 0xFFFFFFFFu &&
                  (kEq1Pass0 & kEq1Pass1) == 0u && (kEq1Pass0 & kEq1Pass2) == 0u && (kEq1Pass1 & kEq1Pass2) == 0u,
              "the passes cover H = 1..32 once each");

template <uint32_t F>
struct CarryBound {
    static constexpr int32_t value = (int32_t)(~F ^ 0x80000000u);
};

template <typename T, int P, int Q>
__device__ __forceinline__ float2 pair_values(const T* x, uint32_t n) {
    float2 v;
    if constexpr (Q == 1) {
        v.x = widen<T>(__ldg(x + n));
        v.y = widen<T>(__ldg(x + n + 1));
    } else {
        constexpr uint32_t F = FracConst<P, Q>::F;
        const uint32_t lo = n * F;
        const uint32_t k = __umulhi(n, F) + (lo >> 31);
        const T* p = x + k;
        const float a = widen<T>(__ldg(p)), b = widen<T>(__ldg(p + 1));
        v.x = a;
        v.y = ((int32_t)lo > CarryBound<F>::value) ? b : a;
    }
    return v;
}

template <uint32_t M, int H>
__device__ __forceinline__ void pair_add(float2* S, float2 v) {
    if constexpr (in_hset(M, H)) {
        constexpr int s = hslot(M, H);
        S[s] = add2(S[s], v);
    }
}
template <uint32_t M, int Q, int... Ms>
__device__ __forceinline__ void pair_add_multiples(float2* S, float2 v, std::integer_sequence<int, Ms...>) {
    (pair_add<M, (Ms + 1) * Q>(S, v), ...);
}
template <typename T, uint32_t M, int K>
__device__ __forceinline__ void pair_step(const T* x, uint32_t n, float2* S) {
    constexpr Frac f = farey_at(K);
    if constexpr (frac_in_hset(M, f.q))
        pair_add_multiples<M, f.q>(S, pair_values<T, f.p, f.q>(x, n), std::make_integer_sequence<int, 32 / f.q>{});
}
template <uint32_t M, int H>
__device__ __forceinline__ void pair_keep(const Tables& tb, const float2* S, float& pa, int& qa, float& pb, int& qb) {
    if constexpr (in_hset(M, H)) {
        constexpr int s = hslot(M, H);
        keep_best(calibrate(tb, S[s].x, H), H, pa, qa);
        keep_best(calibrate(tb, S[s].y, H), H, pb, qb);
    }
}
template <uint32_t M, int... Hs>
__device__ __forceinline__ void pair_keep_all(const Tables& tb, const float2* S, float& pa, int& qa, float& pb,
                                              int& qb, std::integer_sequence<int, Hs...>) {
    (pair_keep<M, Hs + 1>(tb, S, pa, qa, pb, qb), ...);
}
template <typename T, uint32_t M, int... K>
__device__ __forceinline__ void pair_pass(const T* x, uint32_t n, const Tables& tb, float& ba, int& ha, float& bb,
                                          int& hb, std::integer_sequence<int, K...>) {
    float2 S[hset_size(M)];
#pragma unroll
    for (int i = 0; i < hset_size(M); ++i) S[i] = make_float2(0.f, 0.f);
    (pair_step<T, M, K>(x, n, S), ...);  // fractions in increasing order
    float pa = -INFINITY, pb = -INFINITY;
    int qa = 0, qb = 0;
    pair_keep_all<M>(tb, S, pa, qa, pb, qb, std::make_integer_sequence<int, 32>{});
    merge_best(pa, qa, ba, ha);
    merge_best(pb, qb, bb, hb);
}
// Passes per storage type: FP32 runs the three passes at four CTAs per SM; FP16/BF16 spend two more
// instructions per fraction on widening and measured faster as one pass over all 32 sums at two CTAs
// per SM (369 against 501 ms on 4096 x 2^20 bins).  Batched calls with a workspace do not use the
// 16-bit kernel at all: they widen groups of spectra and run the FP32 one (launch_eq1_widened).
template <typename T>
struct Eq1Passes {
    static constexpr bool split = std::is_same<T, float>::value;
    static constexpr int min_blocks = split ? 4 : 2;
};

// best snr / H of outputs n and n+1 (n + 1 < N); the power-of-two stages are one pass over i/32
template <typename T, bool P2>
__device__ __forceinline__ void eq1_pair(const T* x, uint32_t n, const Tables& tb, float& ba, int& ha, float& bb,
                                         int& hb) {
    constexpr auto K = std::make_integer_sequence<int, kNumFrac>{};
    if constexpr (P2) {
        pair_pass<T, kPow2Stages>(x, n, tb, ba, ha, bb, hb, K);
    } else if constexpr (!Eq1Passes<T>::split) {
        pair_pass<T, 0xFFFFFFFFu>(x, n, tb, ba, ha, bb, hb, K);
    } else {
        pair_pass<T, kEq1Pass0>(x, n, tb, ba, ha, bb, hb, K);
        pair_pass<T, kEq1Pass1>(x, n, tb, ba, ha, bb, hb, K);
        pair_pass<T, kEq1Pass2>(x, n, tb, ba, ha, bb, hb, K);
    }
}

template <typename T>
struct Bin<HS_STD, T> {
    template <bool P2>
    static __device__ __forceinline__ void eval(const T* x, uint32_t N, uint32_t n, int hmax, int hv, const Tables& tb,
                                                float* all_h, uint32_t all_stride, float& best, int& bh,
                                                uint32_t& path, uint32_t flags) {
        float S[kHmax + 1];
#pragma unroll
        for (int H = 0; H <= kHmax; ++H) S[H] = 0.f;
        farey_all<T, P2>(x, n, hmax, S, std::make_integer_sequence<int, kNumFrac>{});
#pragma unroll
        for (int H = 1; H <= kHmax; ++H) {
            if (H <= hmax) {
                if (P2 && !is_pow2(H)) {
                    if (all_h) all_h[(size_t)(H - 1) * all_stride + n] = -INFINITY;  // not a stage
                    continue;
                }
                float snr = calibrate(tb, S[H], H);
                if (all_h) all_h[(size_t)(H - 1) * all_stride + n] = snr;
                keep_best(snr, H, best, bh);
            }
        }
    }
};

// Eq. 2: harmonic i adds the largest of x(i*n+j0) .. x(i*n+i), j0 = 1 as written (0 under
// HS_FLAG_MAX_WINDOW0).
template <typename T>
struct Bin<HS_MAX, T> {
    template <bool P2>
    static __device__ __forceinline__ void eval(const T* x, uint32_t N, uint32_t n, int hmax, int hv, const Tables& tb,
                                                float* all_h, uint32_t all_stride, float& best, int& bh,
                                                uint32_t& path, uint32_t flags) {
        const uint32_t j0 = (flags & HS_FLAG_MAX_WINDOW0) ? 0u : 1u;
        float S = 0.f;
        auto add = [&](int i, float m) {
            S = __fadd_rn(S, m);
            const bool stage = !P2 || is_pow2(i);
            const float snr = stage ? calibrate(tb, S, i) : -INFINITY;
            if (stage) keep_best(snr, i, best, bh);
            if (all_h) all_h[(size_t)(i - 1) * all_stride + n] = snr;
        };
        // Harmonics 1 to 4 span at most five elements, read with plain loads (coalesced across the
        // warp) instead of masked 16-byte chunks; valid H means H n + H <= N - 1.
        if (hv >= 1) {
            const T* p = x + n;  // [n + j0, n + 1]
            float m = widen<T>(__ldg(p + 1));
            if (j0 == 0) m = fmaxf(m, widen<T>(__ldg(p)));
            add(1, m);
        }
        if (hv >= 2) {
            const T* p = x + 2 * n;  // [2n + j0, 2n + 2]
            float m = fmaxf(widen<T>(__ldg(p + 1)), widen<T>(__ldg(p + 2)));
            if (j0 == 0) m = fmaxf(m, widen<T>(__ldg(p)));
            add(2, m);
        }
        if (hv >= 3) {
            const T* p = x + 3 * n;  // [3n + j0, 3n + 3]
            float m = fmaxf(fmaxf(widen<T>(__ldg(p + 1)), widen<T>(__ldg(p + 2))), widen<T>(__ldg(p + 3)));
            if (j0 == 0) m = fmaxf(m, widen<T>(__ldg(p)));
            add(3, m);
        }
        if (hv >= 4) {
            const T* p = x + 4 * n;  // [4n + j0, 4n + 4]
            float m = fmaxf(fmaxf(widen<T>(__ldg(p + 1)), widen<T>(__ldg(p + 2))),
                            fmaxf(widen<T>(__ldg(p + 3)), widen<T>(__ldg(p + 4))));
            if (j0 == 0) m = fmaxf(m, widen<T>(__ldg(p)));
            add(4, m);
        }
        for (int i = 5; i <= hv; ++i) {
            const uint32_t base = (uint32_t)i * n;
            add(i, window_max(x, N, base + j0, base + (uint32_t)i, i));
        }
        if (all_h)
            for (int i = hv + 1; i <= hmax; ++i) all_h[(size_t)(i - 1) * all_stride + n] = -INFINITY;
    }
};

// Eq. 3: harmonic i adds x(i*n).  Harmonics run up to the bin's own valid count, four loads at a time;
// the loop is unrolled, so each harmonic's calibration constants are compile-time operands.
template <typename T>
struct Bin<HS_FBIN, T> {
    template <bool P2>
    static __device__ __forceinline__ void eval(const T* x, uint32_t N, uint32_t n, int hmax, int hv, const Tables& tb,
                                                float* all_h, uint32_t all_stride, float& best, int& bh,
                                                uint32_t& path, uint32_t flags) {
        float S = 0.f;
#pragma unroll
        for (int i0 = 1; i0 <= kHmax; i0 += 4) {
            if (i0 > hv) break;
            float v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = (i0 + k <= hv) ? ldx(x, (uint32_t)(i0 + k) * n) : 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (i0 + k <= hv) {
                    S = __fadd_rn(S, v[k]);
                    const bool stage = !P2 || is_pow2(i0 + k);
                    const float snr = stage ? calibrate(tb, S, i0 + k) : -INFINITY;
                    if (stage) keep_best(snr, i0 + k, best, bh);
                    if (all_h) all_h[(size_t)(i0 + k - 1) * all_stride + n] = snr;
                }
            }
        }
        if (all_h)
            for (int i = hv + 1; i <= hmax; ++i) all_h[(size_t)(i - 1) * all_stride + n] = -INFINITY;
    }
};

// Eq. 4: harmonic i compares x(i*n+j) with x(i*n+j+1); the right bin wins only if strictly larger,
// and then j grows by one.  Under HS_FLAG_GREEDY_FIXED1 the first term is x(n) itself and the pairs
// start at harmonic 2; the furthest read is then H*n+H-1, so H is valid while H*(n+1) <= N.
template <typename T>
struct Bin<HS_GREEDY, T> {
    template <bool P2>
    static __device__ __forceinline__ void eval(const T* x, uint32_t N, uint32_t n, int hmax, int hv, const Tables& tb,
                                                float* all_h, uint32_t all_stride, float& best, int& bh,
                                                uint32_t& path, uint32_t flags) {
        const bool fixed1 = (flags & HS_FLAG_GREEDY_FIXED1) != 0;
        float S = 0.f;
        uint32_t j = 0, p = 0;
#pragma unroll
        for (int i = 1; i <= kHmax; ++i) {
            if (i > hv) break;
            if (fixed1 && i == 1) {
                S = __fadd_rn(S, ldx(x, n));
            } else {
                const T* q = x + ((uint32_t)i * n + j);  // r through q + 1: no address of its own
                const float l = widen<T>(__ldg(q)), r = widen<T>(__ldg(q + 1));
                const bool right = r > l;
                p |= (right ? 1u : 0u) << (i - 1);
                j += right ? 1u : 0u;
                S = __fadd_rn(S, right ? r : l);
            }
            const bool stage = !P2 || is_pow2(i);
            const float snr = stage ? calibrate(tb, S, i) : -INFINITY;
            if (stage) keep_best(snr, i, best, bh);
            if (all_h) all_h[(size_t)(i - 1) * all_stride + n] = snr;
        }
        if (all_h)
            for (int i = hv + 1; i <= hmax; ++i) all_h[(size_t)(i - 1) * all_stride + n] = -INFINITY;
        path = p;
    }
    // Two bins of the same valid count, their chains interleaved: the reads of one bin's next harmonic
    // wait on that bin's choice only, so two chains keep twice the loads in flight.  No every-H table.
    template <bool P2>
    static __device__ __forceinline__ void eval2(const T* x, uint32_t n1, uint32_t n2, int hv, const Tables& tb,
                                                 float& b1, int& h1, uint32_t& path1, float& b2, int& h2,
                                                 uint32_t& path2, uint32_t flags) {
        const bool fixed1 = (flags & HS_FLAG_GREEDY_FIXED1) != 0;
        float S1 = 0.f, S2 = 0.f;
        uint32_t j1 = 0, j2 = 0, q1 = 0, q2 = 0;
#pragma unroll
        for (int i = 1; i <= kHmax; ++i) {
            if (i > hv) break;
            if (fixed1 && i == 1) {
                S1 = __fadd_rn(S1, ldx(x, n1));
                S2 = __fadd_rn(S2, ldx(x, n2));
            } else {
                const T* a = x + ((uint32_t)i * n1 + j1);
                const T* b = x + ((uint32_t)i * n2 + j2);
                const float l1 = widen<T>(__ldg(a)), r1 = widen<T>(__ldg(a + 1));
                const float l2 = widen<T>(__ldg(b)), r2 = widen<T>(__ldg(b + 1));
                const bool g1 = r1 > l1, g2 = r2 > l2;
                q1 |= (g1 ? 1u : 0u) << (i - 1);
                q2 |= (g2 ? 1u : 0u) << (i - 1);
                j1 += g1 ? 1u : 0u;
                j2 += g2 ? 1u : 0u;
                S1 = __fadd_rn(S1, g1 ? r1 : l1);
                S2 = __fadd_rn(S2, g2 ? r2 : l2);
            }
            if (!P2 || is_pow2(i)) {
                keep_best(calibrate(tb, S1, i), i, b1, h1);
                keep_best(calibrate(tb, S2, i), i, b2, h2);
            }
        }
        path1 = q1;
        path2 = q2;
    }
};

// ------------------------------------------------------------------------------------------
// Valid harmonic count of output bin n (N >= 1): the largest H <= hmax whose reads stay inside the
// spectrum.  Eq. 2: H (n+1) <= N-1; Eq. 3: H n <= N-1 (every H at n = 0); Eq. 4: H (n+1) <= N-1, or
// <= N under the fixed first term; Eq. 1: always hmax.  It never grows with n, so for Eq. 3 and 4 a
// thread divides once for its first bin of a tile and then steps it down as its bins advance (Eq. 2,
// bound by load latency, ran slower that way and divides for every bin).
// ------------------------------------------------------------------------------------------
template <int V>
struct ValidH {
    static __device__ __forceinline__ uint32_t limit(uint32_t N, uint32_t flags) {
        return (V == HS_GREEDY && (flags & HS_FLAG_GREEDY_FIXED1)) ? N : N - 1;
    }
    static __device__ __forceinline__ uint32_t span(uint32_t n) {
        return V == HS_FBIN ? n : n + 1;
    }
    static __device__ __forceinline__ int first(uint32_t N, uint32_t n, int hmax, uint32_t flags) {
        if (V == HS_STD) return hmax;
        const uint32_t d = span(n);
        return d == 0 ? hmax : (int)min((uint32_t)hmax, limit(N, flags) / d);
    }
    static __device__ __forceinline__ int step(int hv, uint32_t N, uint32_t n, uint32_t flags) {
        if (V == HS_MAX) return (int)min((uint32_t)hv, limit(N, flags) / span(n));
        if (V != HS_STD) {
            const uint32_t a = limit(N, flags), d = span(n);  // hv * d <= 2^31: n < N <= 2^26
            while (hv > 0 && (uint32_t)hv * d > a) --hv;
        }
        return hv;
    }
};

// ------------------------------------------------------------------------------------------
// One tile of output bins [t0, t1) of one spectrum; the whole block walks it in steps of kBlock.
// ------------------------------------------------------------------------------------------
template <int V, typename T, bool P2>
__device__ __forceinline__ void run_tile(const T* x, uint32_t N, uint32_t t0, uint32_t t1, const Tables& tb,
                                         const Work1d& w, const Out1d& o, size_t out_off, uint32_t spec,
                                         unsigned* status) {
    uint32_t base = t0;
    int hv = ValidH<V>::first(N, base + threadIdx.x, w.hmax, (uint32_t)w.flags);
    for (; base < t1; base += kBlock) {
        uint32_t n = base + threadIdx.x;
        bool active = n < t1;
        float best = -INFINITY;
        int bh = 0;
        uint32_t path = 0;
        if (active) {
            hv = ValidH<V>::step(hv, N, n, (uint32_t)w.flags);
            Bin<V, T>::template eval<P2>(x, N, n, w.hmax, hv, tb, o.all_h, N, best, bh, path, (uint32_t)w.flags);
            o.best_snr[out_off + n] = best;
            o.best_h[out_off + n] = (uint8_t)bh;
            if (V == HS_GREEDY && o.path) o.path[out_off + n] = path;
        }
        if (o.cand)
            append_candidate(active && best > w.threshold, o.cand, o.cand_count, o.cand_cap, status, spec, n, best,
                             0, bh, V);
    }
}

// Eq. 1 over output pairs ([t0, t1) of one spectrum, N >= 1): thread t owns outputs n = base + 2t and
// n + 1.  A lone last output n (n + 1 == t1) is taken as the second output of the pair (n - 1, n), so
// every read stays at or below n.  A one-bin spectrum reads x(0) for every term: S_H is then the
// running sum of H copies of x(0).
template <typename T, bool P2>
__device__ __forceinline__ void eq1_pair_tile(const T* x, uint32_t N, uint32_t t0, uint32_t t1, const Tables& tb,
                                              const Work1d& w, const Out1d& o, size_t out_off, uint32_t spec,
                                              unsigned* status) {
    for (uint32_t base = t0; base < t1; base += 2 * kBlock) {
        const uint32_t n = base + 2 * threadIdx.x;
        const bool va = n < t1, vb = n + 1 < t1;
        float ba = -INFINITY, bb = -INFINITY;
        int ha = 0, hb = 0;
        if (va) {
            if (N == 1) {
                const float x0 = widen<T>(__ldg(x));
                float r = 0.f;
#pragma unroll
                for (int H = 1; H <= kHmax; ++H) {
                    r = __fadd_rn(r, x0);
                    if (!P2 || is_pow2(H)) keep_best(calibrate(tb, r, H), H, ba, ha);
                }
            } else {
                const uint32_t ne = vb ? n : n - 1;  // one inlined sweep serves both cases
                float pa = -INFINITY, pb = -INFINITY;
                int qa = 0, qb = 0;
                eq1_pair<T, P2>(x, ne, tb, pa, qa, pb, qb);
                if (vb) {
                    ba = pa;
                    ha = qa;
                    bb = pb;
                    hb = qb;
                } else {
                    ba = pb;
                    ha = qb;
                }
            }
            o.best_snr[out_off + n] = ba;
            o.best_h[out_off + n] = (uint8_t)ha;
            if (vb) {
                o.best_snr[out_off + n + 1] = bb;
                o.best_h[out_off + n + 1] = (uint8_t)hb;
            }
        }
        if (o.cand) {
            append_candidate(va && ba > w.threshold, o.cand, o.cand_count, o.cand_cap, status, spec, n, ba, 0, ha,
                             HS_STD);
            append_candidate(vb && bb > w.threshold, o.cand, o.cand_count, o.cand_cap, status, spec, n + 1, bb, 0, hb,
                             HS_STD);
        }
    }
}

template <int V>
struct MinBlocks {
    static constexpr int value = V == HS_STD ? 2 : 6;
};


// the zoned kernels carry one copy of the bin loop per unrolled count.  Eq. 3 runs at full occupancy
// (32 registers, a few spilled): its loads are independent and latency-bound, and eight CTAs per SM
// measured 3-7% faster than six.  Eq. 2 at five CTAs per SM (48 registers) measured 8% faster than
// at four for FP32, whose six-CTA build spills heavily; 16-bit storage gains 3% more at six.  Eq. 4
// is fastest at five (six and eight measured slower).
template <int V, typename T>
struct ZonedMinBlocks {
    static constexpr int value = V == HS_MAX ? (sizeof(T) == 2 ? 6 : 5) : (V == HS_FBIN ? 8 : 5);
};

// Eq. 2 indexes the calibration tables by a runtime H, which is cheaper from shared memory than
// from the kernel-parameter bank; Eq. 1, 3 and 4 unroll H (the loop leaves at the bin's valid count)
// and read the parameter bank directly.
template <int V>
__device__ __forceinline__ const Tables& stage_tables(const Tables& tb, Tables& smem) {
    if (V == HS_MAX) {
        for (int k = threadIdx.x; k < 3 * (kHmax + 1); k += blockDim.x)
            reinterpret_cast<float*>(&smem)[k] = reinterpret_cast<const float*>(&tb)[k];
        __syncthreads();
        return smem;
    }
    return tb;
}

// ------------------------------------------------------------------------------------------
// Zones of constant valid-harmonic count (Eq. 2-4).  The valid count of output bin n never grows
// with n: Eq. 3 keeps H while H n <= L, Eq. 2 and 4 while H (n + 1) <= L (L = N - 1, or N for Eq. 4
// with its first term fixed).  So the bins whose count is exactly h form one contiguous zone
// [edge(h + 1), edge(h)), edge(h) being the first bin whose count is below h, and half of all bins
// lie in zone 1.  A spectrum is cut into its zones and each zone into tiles whose bin count is
// inversely proportional to the cost of a bin there: every work item then costs about the same, so
// the persistent CTAs advance through the batch together and only one or two spectra are being read
// at any time (their spans stay in L2).  An item runs with its zone's count fixed, unrolled at
// compile time up to kZoneUnrolled harmonics.
// ------------------------------------------------------------------------------------------
constexpr int kZoneUnrolled = 8;

__host__ __device__ inline uint32_t zone_limit(int v, uint32_t N, int flags) {
    return (v == HS_GREEDY && (flags & HS_FLAG_GREEDY_FIXED1)) ? N : N - 1u;
}
// the first bin whose valid count is below h (h >= 1), at most N
__host__ __device__ inline uint32_t zone_edge(int v, uint32_t N, uint32_t L, int h) {
    const uint32_t e = v == HS_FBIN ? L / (uint32_t)h + 1u : L / (uint32_t)h;
    return e < N ? e : N;
}
// relative cost of one bin whose valid count is h (loads and adds; Eq. 2 windows grow with i)
__host__ __device__ inline uint32_t zone_cost(int v, int h) {
    const uint32_t u = (uint32_t)h;
    return v == HS_MAX ? 8u + 2u * u + u * (u + 1u) / 4u : (v == HS_GREEDY ? 4u + 2u * u : 4u + u);
}
// bins per tile of zone h: opt * kBlock in zone 1, scaled down by the cost ratio, a multiple of kBlock
__host__ __device__ inline uint32_t zone_tile(int v, int h, int opt) {
    const uint32_t c1 = zone_cost(v, 1), ch = zone_cost(v, h);
    const uint32_t k = ((uint32_t)opt * c1 + ch / 2u) / ch;
    return (uint32_t)kBlock * (k > 0u ? k : 1u);
}
// [lo, hi) of zone h; zone 1 runs on to N (its last bins may have no valid H at all)
__host__ __device__ inline void zone_range(const ZoneSpec& z, uint32_t N, int h, uint32_t& lo, uint32_t& hi) {
    const uint32_t L = zone_limit(z.v, N, z.flags);
    lo = h >= z.hmax ? 0u : zone_edge(z.v, N, L, h + 1);
    hi = h <= 1 ? N : zone_edge(z.v, N, L, h);
    if (hi < lo) hi = lo;  // edges never increase with h; kept as a guard
}
__host__ __device__ inline uint32_t zone_items(const ZoneSpec& z, uint32_t N, int h) {
    uint32_t lo, hi;
    zone_range(z, N, h, lo, hi);
    const uint32_t B = zone_tile(z.v, h, z.opt);
    return (hi - lo + B - 1u) / B;
}
__host__ __device__ inline int64_t zone_item_count(const ZoneSpec& z, uint32_t N) {
    if (N == 0) return 0;
    int64_t t = 0;
    for (int h = 1; h <= z.hmax; ++h) t += zone_items(z, N, h);
    return t;
}

// Work item k of a spectrum of N bins: its zone h and bin range [lo, hi).  All 32 lanes of one warp
// call it; lane j looks at zone hmax - j (zones in increasing bin order).
__device__ inline void zone_lookup(const ZoneSpec& z, uint32_t N, uint32_t k, int& h, uint32_t& lo, uint32_t& hi) {
    const int lane = threadIdx.x & 31;
    const int hz = z.hmax - lane;
    uint32_t zlo = 0, zhi = 0, B = 1, T = 0;
    if (hz >= 1) {
        zone_range(z, N, hz, zlo, zhi);
        B = zone_tile(z.v, hz, z.opt);
        T = (zhi - zlo + B - 1u) / B;
    }
    uint32_t incl = T;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += u;
    }
    const unsigned m = __ballot_sync(0xffffffffu, incl > k);
    const int owner = m ? __ffs(m) - 1 : 0;
    const uint32_t a = zlo + (k - (incl - T)) * B;
    h = m ? __shfl_sync(0xffffffffu, hz, owner) : 0;
    lo = m ? __shfl_sync(0xffffffffu, a, owner) : 0u;
    hi = m ? __shfl_sync(0xffffffffu, min(zhi, a + B), owner) : 0u;
}

// The bins [lo, hi) of one zone, whose valid count is H (a compile-time count) or h (H = 0).
template <int V, typename T, bool P2, int H>
__device__ __forceinline__ void zone_run(const T* x, uint32_t N, uint32_t lo, uint32_t hi, int h, const Tables& tb,
                                         const Work1d& w, const Out1d& o, size_t out_off, uint32_t spec,
                                         unsigned* status) {
    const int hv = H > 0 ? H : h;
    if constexpr (V == HS_GREEDY && H != 1) {
        // Eq. 4: thread t takes the bins base + t and base + kBlock + t together
        for (uint32_t base = lo; base < hi; base += 2 * kBlock) {
            const uint32_t n1 = base + threadIdx.x, n2 = n1 + kBlock;
            const bool a1 = n1 < hi, a2 = n2 < hi;
            float b1 = -INFINITY, b2 = -INFINITY;
            int h1 = 0, h2 = 0;
            uint32_t p1 = 0, p2 = 0;
            if (a1) {
                Bin<V, T>::template eval2<P2>(x, n1, a2 ? n2 : n1, hv, tb, b1, h1, p1, b2, h2, p2,
                                              (uint32_t)w.flags);
                o.best_snr[out_off + n1] = b1;
                o.best_h[out_off + n1] = (uint8_t)h1;
                if (o.path) o.path[out_off + n1] = p1;
            }
            if (a2) {
                o.best_snr[out_off + n2] = b2;
                o.best_h[out_off + n2] = (uint8_t)h2;
                if (o.path) o.path[out_off + n2] = p2;
            }
            if (o.cand) {
                append_candidate(a1 && b1 > w.threshold, o.cand, o.cand_count, o.cand_cap, status, spec, n1, b1, 0,
                                 h1, V);
                append_candidate(a2 && b2 > w.threshold, o.cand, o.cand_count, o.cand_cap, status, spec, n2, b2, 0,
                                 h2, V);
            }
        }
        return;
    }
    // zone 1 also holds the bins with no valid H at all (from edge(1) on): they keep -inf, 0
    const uint32_t e1 = H == 1 ? zone_edge(V, N, zone_limit(V, N, w.flags), 1) : 0u;
    for (uint32_t base = lo; base < hi; base += kBlock) {
        const uint32_t n = base + threadIdx.x;
        const bool active = n < hi;
        float best = -INFINITY;
        int bh = 0;
        uint32_t path = 0;
        if (active) {
            if (H != 1 || n < e1)
                Bin<V, T>::template eval<P2>(x, N, n, w.hmax, hv, tb, nullptr, 0u, best, bh, path, (uint32_t)w.flags);
            o.best_snr[out_off + n] = best;
            o.best_h[out_off + n] = (uint8_t)bh;
            if (V == HS_GREEDY && o.path) o.path[out_off + n] = path;
        }
        if (o.cand)
            append_candidate(active && best > w.threshold, o.cand, o.cand_count, o.cand_cap, status, spec, n, best,
                             0, bh, V);
    }
}

template <int V, typename T, bool P2>
__device__ __forceinline__ void zone_dispatch(const T* x, uint32_t N, uint32_t lo, uint32_t hi, int h,
                                              const Tables& tb, const Work1d& w, const Out1d& o, size_t out_off,
                                              uint32_t spec, unsigned* status) {
    static_assert(kZoneUnrolled == 8, "one case per unrolled count");
    switch (h) {
        case 1: zone_run<V, T, P2, 1>(x, N, lo, hi, h, tb, w, o, out_off, spec, status); break;
        case 2: zone_run<V, T, P2, 2>(x, N, lo, hi, h, tb, w, o, out_off, spec, status); break;
        case 3: zone_run<V, T, P2, 3>(x, N, lo, hi, h, tb, w, o, out_off, spec, status); break;
        case 4: zone_run<V, T, P2, 4>(x, N, lo, hi, h, tb, w, o, out_off, spec, status); break;
        case 5: zone_run<V, T, P2, 5>(x, N, lo, hi, h, tb, w, o, out_off, spec, status); break;
        case 6: zone_run<V, T, P2, 6>(x, N, lo, hi, h, tb, w, o, out_off, spec, status); break;
        case 7: zone_run<V, T, P2, 7>(x, N, lo, hi, h, tb, w, o, out_off, spec, status); break;
        case 8: zone_run<V, T, P2, 8>(x, N, lo, hi, h, tb, w, o, out_off, spec, status); break;
        default: zone_run<V, T, P2, 0>(x, N, lo, hi, h, tb, w, o, out_off, spec, status); break;
    }
}

// One spectrum: CTA b runs work item b.
template <int V, typename T, bool P2>
__global__ void __launch_bounds__(kBlock, ZonedMinBlocks<V, T>::value) k_hs1d_zoned_single(const __grid_constant__ Tables tb_param,
                                                                                  const Work1d w, const Out1d o,
                                                                                  WsControl* ctl) {
    __shared__ Tables s_tb;
    const Tables& tb = stage_tables<V>(tb_param, s_tb);
    __shared__ int s_h;
    __shared__ uint32_t s_lo, s_hi;
    const uint32_t N = (uint32_t)w.n_bins;
    if (threadIdx.x < 32) {
        int h;
        uint32_t lo, hi;
        zone_lookup(ZoneSpec{V, w.hmax, w.flags, w.opt}, N, blockIdx.x, h, lo, hi);
        if (threadIdx.x == 0) {
            s_h = h;
            s_lo = lo;
            s_hi = hi;
        }
    }
    __syncthreads();
    zone_dispatch<V, T, P2>((const T*)w.x, N, s_lo, s_hi, s_h, tb, w, o, 0, w.first_id, &ctl->status);
}

// Warp 0 resolves a claimed work item (held by thread 0) into spectrum, zone and bin range.  Items
// increase along each CTA's sequence, so the search starts from the spectrum of the CTA's last item.
struct ZoneSlot {
    unsigned long long item;
    int spec, h;
    uint32_t lo, hi;
};
__device__ __forceinline__ int spectrum_from(const int64_t* prefix, int n_spectra, int s, unsigned long long item) {
    for (int k = 0; k < 2; ++k) {
        if (s + 1 >= n_spectra || (unsigned long long)__ldg(prefix + s + 1) > item) return s;
        ++s;
    }
    return find_spectrum(prefix, n_spectra, item);
}
__device__ __forceinline__ void zone_resolve(const ZoneSpec& z, const Work1d& w, const int64_t* prefix,
                                             unsigned long long total, unsigned long long claimed, int hint,
                                             ZoneSlot& slot) {
    const unsigned long long item = __shfl_sync(0xffffffffu, claimed, 0);
    int s = 0, h = 0;
    uint32_t lo = 0, hi = 0;
    if (item < total) {
        if ((threadIdx.x & 31) == 0) s = spectrum_from(prefix, w.n_spectra, hint, item);
        s = __shfl_sync(0xffffffffu, s, 0);
        const uint32_t N = (uint32_t)(w.offsets[s + 1] - w.offsets[s]);
        zone_lookup(z, N, (uint32_t)(item - (unsigned long long)prefix[s]), h, lo, hi);
    }
    if (threadIdx.x == 0) {
        slot.item = item;
        slot.spec = s;
        slot.h = h;
        slot.lo = lo;
        slot.hi = hi;
    }
}

// Persistent kernel over a batch: CTAs pop (spectrum, zone, tile) items in order.  Warp 0 claims and
// resolves the next item at the start of the current one (into the other of two slots), so the
// lookup's memory latency overlaps the other warps' work on the current item.
template <int V, typename T, bool P2>
__global__ void __launch_bounds__(kBlock, ZonedMinBlocks<V, T>::value) k_hs1d_zoned(const __grid_constant__ Tables tb_param,
                                                                                const Work1d w, const Out1d o,
                                                                                WsControl* ctl, const int64_t* prefix) {
    __shared__ Tables s_tb;
    const Tables& tb = stage_tables<V>(tb_param, s_tb);
    __shared__ ZoneSlot s_slot[2];
    const unsigned long long total = *(volatile unsigned long long*)&ctl->total_items;
    const ZoneSpec z{V, w.hmax, w.flags, w.opt};
    unsigned long long claimed = 0;
    if (threadIdx.x == 0) claimed = atomicAdd(&ctl->queue, 1u);
    if (threadIdx.x < 32) zone_resolve(z, w, prefix, total, claimed, 0, s_slot[0]);
    __syncthreads();
    for (int b = 0;; b ^= 1) {
        const ZoneSlot cur = s_slot[b];
        if (cur.item >= total) break;
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0) claimed = atomicAdd(&ctl->queue, 1u);
            zone_resolve(z, w, prefix, total, claimed, cur.spec, s_slot[b ^ 1]);
        }
        const int64_t off = w.offsets[cur.spec];
        const uint32_t N = (uint32_t)(w.offsets[cur.spec + 1] - off);
        zone_dispatch<V, T, P2>((const T*)w.x + off, N, cur.lo, cur.hi, cur.h, tb, w, o, (size_t)off,
                                w.first_id + (uint32_t)cur.spec, &ctl->status);
        __syncthreads();  // the next slot is written and every thread has read this one
    }
}

template <int V, typename T, bool P2>
__global__ void __launch_bounds__(kBlock, MinBlocks<V>::value) k_hs1d_single(const __grid_constant__ Tables tb_param,
                                                                            const Work1d w, const Out1d o,
                                                                            WsControl* ctl) {
    __shared__ Tables s_tb;
    const Tables& tb = stage_tables<V>(tb_param, s_tb);
    uint32_t N = (uint32_t)w.n_bins;
    uint32_t tile = (uint32_t)(kBlock * w.opt);
    uint32_t t0 = blockIdx.x * tile;
    uint32_t t1 = min(N, t0 + tile);
    run_tile<V, T, P2>((const T*)w.x, N, t0, t1, tb, w, o, 0, w.first_id, &ctl->status);
}

// Tile prefix sums of a batch and reset of the work queue.  One block.  Offsets are absolute
// element indices into the input (a batch may be a slice of a larger one).  A spectrum that breaks
// the layout contract (negative or oversized length, misaligned start) is given zero tiles and
// flagged in the status word.
__global__ void __launch_bounds__(1024) k_tile_scan(const int64_t* offsets, int n, int64_t tile, int64_t max_bins,
                                                    int elem_bytes, ZoneSpec zs, int64_t* prefix, WsControl* ctl) {
    __shared__ int64_t warp_sum[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) {
        carry = 0;
        ctl->queue = 0u;
    }
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        int s = base + threadIdx.x;
        int64_t t = 0;
        if (s < n) {
            int64_t a = offsets[s], b = offsets[s + 1], len = b - a;
            bool bad = a < 0 || len < 0 || len > max_bins || ((a * elem_bytes) & 15) != 0;
            if (bad) atomicOr(&ctl->status, kStatusBadInput);
            t = bad ? 0 : (zs.v ? zone_item_count(zs, (uint32_t)len) : (len + tile - 1) / tile);
        }
        // inclusive scan over the block
        int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        int64_t v = t;
        for (int d = 1; d < 32; d <<= 1) {
            int64_t u = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v += u;
        }
        if (lane == 31) warp_sum[wid] = v;
        __syncthreads();
        if (wid == 0) {
            int nw = blockDim.x >> 5;
            int64_t ws = lane < nw ? warp_sum[lane] : 0;
            for (int d = 1; d < 32; d <<= 1) {
                int64_t u = __shfl_up_sync(0xffffffffu, ws, d);
                if (lane >= d) ws += u;
            }
            if (lane < nw) warp_sum[lane] = ws;
        }
        __syncthreads();
        int64_t excl = carry + (wid ? warp_sum[wid - 1] : 0) + v - t;
        if (s < n) prefix[s] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + t;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        prefix[n] = carry;
        ctl->total_items = (unsigned long long)carry;
    }
}

// Persistent kernel: CTAs pop (spectrum, tile) items in order from the queue.  The next item is
// claimed while the current one is processed, so the atomic's round trip is off the critical path.
template <int V, typename T, bool P2>
__global__ void __launch_bounds__(kBlock, MinBlocks<V>::value) k_hs1d_batched(const __grid_constant__ Tables tb_param,
                                                                             const Work1d w, const Out1d o,
                                                                             WsControl* ctl, const int64_t* prefix) {
    __shared__ Tables s_tb;
    const Tables& tb = stage_tables<V>(tb_param, s_tb);
    __shared__ unsigned long long s_item;
    __shared__ int s_spec;
    const unsigned long long total = *(volatile unsigned long long*)&ctl->total_items;
    const uint32_t tile = (uint32_t)(kBlock * w.opt);
    if (threadIdx.x == 0) {
        unsigned long long item = atomicAdd(&ctl->queue, 1u);
        s_item = item;
        s_spec = item < total ? find_spectrum(prefix, w.n_spectra, item) : 0;
    }
    __syncthreads();
    for (;;) {
        const unsigned long long item = s_item;
        const int s = s_spec;
        if (item >= total) break;
        unsigned long long next = 0;
        if (threadIdx.x == 0) next = atomicAdd(&ctl->queue, 1u);  // result consumed after the tile
        const int64_t off = w.offsets[s];
        const uint32_t N = (uint32_t)(w.offsets[s + 1] - off);
        const uint32_t t0 = (uint32_t)(item - (unsigned long long)prefix[s]) * tile;
        const uint32_t t1 = min(N, t0 + tile);
        run_tile<V, T, P2>((const T*)w.x + off, N, t0, t1, tb, w, o, (size_t)off, w.first_id + (uint32_t)s,
                           &ctl->status);
        __syncthreads();  // every thread has read s_item / s_spec
        if (threadIdx.x == 0) {
            s_item = next;
            s_spec = next < total ? find_spectrum(prefix, w.n_spectra, next) : 0;
        }
        __syncthreads();
    }
}

// Eq. 1 over output pairs: one spectrum (a tile per CTA) and the persistent batch walk.
template <typename T, bool P2>
__global__ void __launch_bounds__(kBlock, Eq1Passes<T>::min_blocks) k_eq1_pairs_single(const __grid_constant__ Tables tb,
                                                                               const Work1d w, const Out1d o,
                                                                               WsControl* ctl) {
    const uint32_t N = (uint32_t)w.n_bins;
    const uint32_t tile = (uint32_t)(kBlock * w.opt);
    const uint32_t t0 = blockIdx.x * tile;
    eq1_pair_tile<T, P2>((const T*)w.x, N, t0, min(N, t0 + tile), tb, w, o, 0, w.first_id, &ctl->status);
}

// REBASE: w.x holds elements offsets[0] .. of the batch rather than the batch itself (a group of
// spectra widened into FP32); outputs keep the batch's absolute positions.
template <typename T, bool P2, bool REBASE = false>
__global__ void __launch_bounds__(kBlock, Eq1Passes<T>::min_blocks) k_eq1_pairs_batched(const __grid_constant__ Tables tb,
                                                                                const Work1d w, const Out1d o,
                                                                                WsControl* ctl, const int64_t* prefix) {
    __shared__ unsigned long long s_item;
    __shared__ int s_spec;
    const unsigned long long total = *(volatile unsigned long long*)&ctl->total_items;
    const uint32_t tile = (uint32_t)(kBlock * w.opt);
    if (threadIdx.x == 0) {
        const unsigned long long item = atomicAdd(&ctl->queue, 1u);
        s_item = item;
        s_spec = item < total ? find_spectrum(prefix, w.n_spectra, item) : 0;
    }
    __syncthreads();
    for (;;) {
        const unsigned long long item = s_item;
        const int s = s_spec;
        if (item >= total) break;
        unsigned long long next = 0;
        if (threadIdx.x == 0) next = atomicAdd(&ctl->queue, 1u);  // result consumed after the tile
        const int64_t off = w.offsets[s];
        const uint32_t N = (uint32_t)(w.offsets[s + 1] - off);
        const uint32_t t0 = (uint32_t)(item - (unsigned long long)prefix[s]) * tile;
        int64_t in_off = off;
        bool inside = true;
        if constexpr (REBASE) {
            // the spectrum must lie in the widened range, and the range must have fit (offsets that
            // are not monotone can give a spectrum of valid length outside it)
            const int64_t base = w.offsets[0], end = w.offsets[w.n_spectra];
            inside = off >= base && off + (int64_t)N <= end && end - base <= (int64_t)w.n_spectra * w.max_bins;
            in_off = off - base;
            if (!inside && threadIdx.x == 0) atomicOr(&ctl->status, kStatusBadInput);
        }
        if (inside)
            eq1_pair_tile<T, P2>((const T*)w.x + in_off, N, t0, min(N, t0 + tile), tb, w, o, (size_t)off,
                                 w.first_id + (uint32_t)s, &ctl->status);
        __syncthreads();  // every thread has read s_item / s_spec
        if (threadIdx.x == 0) {
            s_item = next;
            s_spec = next < total ? find_spectrum(prefix, w.n_spectra, next) : 0;
        }
        __syncthreads();
    }
}

// Elements offsets[0] .. offsets[n] of a 16-bit batch widened to FP32 (exactly) at out[0 ..), eight
// per thread and step when the range starts 16-byte aligned.  A range that is reversed or longer than
// cap elements is left alone (the tile scan reports the bad layout; its spectra get no work).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_widen(const T* x, const int64_t* offsets, int n, int64_t cap,
                                                  float* out) {
    static_assert(sizeof(T) == 2, "16-bit storage: eight elements per 16-byte load");
    const int64_t base = offsets[0], end = offsets[n];
    if (base < 0 || end < base || end - base > cap) return;
    const int64_t len = end - base;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const T* src = x + base;
    int64_t done = 0;
    if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
        const int64_t n8 = len / 8;
        for (int64_t i = t; i < n8; i += stride) {
            const uint4 raw = __ldg(reinterpret_cast<const uint4*>(src) + i);
            const T* e = reinterpret_cast<const T*>(&raw);
            float4 lo, hi;
            lo.x = widen<T>(e[0]);
            lo.y = widen<T>(e[1]);
            lo.z = widen<T>(e[2]);
            lo.w = widen<T>(e[3]);
            hi.x = widen<T>(e[4]);
            hi.y = widen<T>(e[5]);
            hi.z = widen<T>(e[6]);
            hi.w = widen<T>(e[7]);
            reinterpret_cast<float4*>(out)[2 * i] = lo;
            reinterpret_cast<float4*>(out)[2 * i + 1] = hi;
        }
        done = n8 * 8;
    }
    for (int64_t i = done + t; i < len; i += stride) out[i] = widen<T>(src[i]);
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
void launch_tile_scan(const int64_t* offsets, int n_spectra, int64_t tile, int64_t max_bins, int elem_bytes,
                      int64_t* prefix, WsControl* ctl, cudaStream_t s) {
    k_tile_scan<<<1, 1024, 0, s>>>(offsets, n_spectra, tile, max_bins, elem_bytes, ZoneSpec{0, 0, 0, 0}, prefix, ctl);
}

template <int V, typename T, bool P2>
static int& occupancy_slot() {
    static int occ[kMaxDevices] = {};  // resident CTAs per SM of the persistent kernel, per device
    return occ[device_slot()];
}

template <int V, typename T, bool P2>
static int occupancy() {
    int& oc = occupancy_slot<V, T, P2>();
    if (oc == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oc, k_hs1d_batched<V, T, P2>, kBlock, 0);
        if (e != cudaSuccess || oc < 1) oc = 1;
    }
    return oc;
}

template <int V, typename T, bool P2>
static int& zoned_occupancy_slot() {
    static int occ[kMaxDevices] = {};  // resident CTAs per SM of the persistent zoned kernel, per device
    return occ[device_slot()];
}

template <int V, typename T, bool P2>
static int zoned_occupancy() {
    int& oc = zoned_occupancy_slot<V, T, P2>();
    if (oc == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oc, k_hs1d_zoned<V, T, P2>, kBlock, 0);
        if (e != cudaSuccess || oc < 1) oc = 1;
    }
    return oc;
}

template <int V, typename T, bool P2>
static cudaError_t launch_zoned(const Tables& tab, const Work1d& w, const Out1d& o, WsControl* ctl, int64_t* prefix,
                                int sm_count, cudaStream_t s) {
    const ZoneSpec z{V, w.hmax, w.flags, w.opt};
    if (w.offsets == nullptr) {
        const int64_t items = zone_item_count(z, (uint32_t)w.n_bins);
        if (items == 0) return cudaSuccess;
        k_hs1d_zoned_single<V, T, P2><<<(unsigned)items, kBlock, 0, s>>>(tab, w, o, ctl);
        return cudaGetLastError();
    }
    k_tile_scan<<<1, 1024, 0, s>>>(w.offsets, w.n_spectra, 0, w.max_bins, (int)sizeof(T), z, prefix, ctl);
    const int occ = zoned_occupancy<V, T, P2>();
    const unsigned grid = persistent_grid(sm_count, occ, w.ctas_per_sm);
    k_hs1d_zoned<V, T, P2><<<grid, kBlock, 0, s>>>(tab, w, o, ctl, prefix);
    return cudaGetLastError();
}

template <typename T, bool P2, bool REBASE>
static int& pair_occupancy_slot() {
    static int occ[kMaxDevices] = {};  // resident CTAs per SM of the persistent Eq. 1 pair kernel, per device
    return occ[device_slot()];
}

template <typename T, bool P2, bool REBASE = false>
static int pair_occupancy() {
    int& oc = pair_occupancy_slot<T, P2, REBASE>();
    if (oc == 0) {
        cudaError_t e =
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oc, k_eq1_pairs_batched<T, P2, REBASE>, kBlock, 0);
        if (e != cudaSuccess || oc < 1) oc = 1;
    }
    return oc;
}

// A 16-bit batch with a staging region: groups of up to kStageSpectra consecutive spectra (one
// contiguous range of the batch) are widened into the region and summed by the FP32 kernel, which
// reads them rebased and writes the batch's output positions.  Bit-identical to the 16-bit kernel
// (widening is exact and the sums are the same FP32 operations in the same order).
template <typename T, bool P2>
static cudaError_t launch_eq1_widened(const Tables& tab, const Work1d& w, const Out1d& o, WsControl* ctl,
                                      int64_t* prefix, int sm_count, cudaStream_t s) {
    const int64_t tile = (int64_t)kBlock * w.opt;
    const unsigned grid = persistent_grid(sm_count, pair_occupancy<float, P2, true>(), w.ctas_per_sm);
    Work1d g = w;
    g.x = w.stage;
    for (int g0 = 0; g0 < w.n_spectra; g0 += kStageSpectra) {
        const int ng = std::min(kStageSpectra, w.n_spectra - g0);
        k_widen<T><<<(unsigned)(sm_count * 8), kBlock, 0, s>>>((const T*)w.x, w.offsets + g0, ng,
                                                              (int64_t)ng * w.max_bins, w.stage);
        g.offsets = w.offsets + g0;
        g.n_spectra = ng;
        g.first_id = w.first_id + (uint32_t)g0;
        // the layout checks use the storage type's alignment, so a spectrum the 16-bit kernel would
        // refuse is refused here too
        launch_tile_scan(g.offsets, ng, tile, w.max_bins, (int)sizeof(T), prefix, ctl, s);
        k_eq1_pairs_batched<float, P2, true><<<grid, kBlock, 0, s>>>(tab, g, o, ctl, prefix);
    }
    return cudaGetLastError();
}

template <typename T, bool P2>
static cudaError_t launch_eq1_pairs(const Tables& tab, const Work1d& w, const Out1d& o, WsControl* ctl,
                                    int64_t* prefix, int sm_count, cudaStream_t s) {
    if constexpr (sizeof(T) == 2)
        if (w.offsets != nullptr && w.stage != nullptr) return launch_eq1_widened<T, P2>(tab, w, o, ctl, prefix, sm_count, s);
    const int64_t tile = (int64_t)kBlock * w.opt;
    if (w.offsets == nullptr) {
        if (w.n_bins == 0) return cudaSuccess;
        k_eq1_pairs_single<T, P2><<<(unsigned)((w.n_bins + tile - 1) / tile), kBlock, 0, s>>>(tab, w, o, ctl);
        return cudaGetLastError();
    }
    launch_tile_scan(w.offsets, w.n_spectra, tile, w.max_bins, (int)sizeof(T), prefix, ctl, s);
    const unsigned grid = persistent_grid(sm_count, pair_occupancy<T, P2>(), w.ctas_per_sm);
    k_eq1_pairs_batched<T, P2><<<grid, kBlock, 0, s>>>(tab, w, o, ctl, prefix);
    return cudaGetLastError();
}

template <int V, typename T, bool P2>
static cudaError_t launch_typed(const Tables& tab, const Work1d& w, const Out1d& o, WsControl* ctl,
                                int64_t* prefix, int sm_count, cudaStream_t s) {
    // Eq. 1 with hmax 32 and no every-H table runs over output pairs in passes
    if constexpr (V == HS_STD)
        if (w.hmax == kHmax && o.all_h == nullptr) return launch_eq1_pairs<T, P2>(tab, w, o, ctl, prefix, sm_count, s);
    // Eq. 2-4 run zone by zone; the every-H table (hs_sum_1d debug output) keeps the per-bin kernel
    if constexpr (V != HS_STD)
        if (o.all_h == nullptr) return launch_zoned<V, T, P2>(tab, w, o, ctl, prefix, sm_count, s);
    const int64_t tile = (int64_t)kBlock * w.opt;
    if (w.offsets == nullptr) {
        if (w.n_bins == 0) return cudaSuccess;
        unsigned grid = (unsigned)((w.n_bins + tile - 1) / tile);
        k_hs1d_single<V, T, P2><<<grid, kBlock, 0, s>>>(tab, w, o, ctl);
        return cudaGetLastError();
    }
    launch_tile_scan(w.offsets, w.n_spectra, tile, w.max_bins, (int)sizeof(T), prefix, ctl, s);
    const unsigned pgrid = persistent_grid(sm_count, occupancy<V, T, P2>(), w.ctas_per_sm);
    k_hs1d_batched<V, T, P2><<<pgrid, kBlock, 0, s>>>(tab, w, o, ctl, prefix);
    return cudaGetLastError();
}

template <int V>
static cudaError_t launch_dtype(hs_dtype dt, const Tables& tab, const Work1d& w, const Out1d& o, WsControl* ctl,
                                int64_t* prefix, int sm_count, cudaStream_t s) {
    const bool p2 = (w.flags & HS_FLAG_POW2_STAGES) != 0;
    switch (dt) {
        case HS_F32:
            return p2 ? launch_typed<V, float, true>(tab, w, o, ctl, prefix, sm_count, s)
                      : launch_typed<V, float, false>(tab, w, o, ctl, prefix, sm_count, s);
        case HS_F16:
            return p2 ? launch_typed<V, __half, true>(tab, w, o, ctl, prefix, sm_count, s)
                      : launch_typed<V, __half, false>(tab, w, o, ctl, prefix, sm_count, s);
        case HS_BF16:
            return p2 ? launch_typed<V, __nv_bfloat16, true>(tab, w, o, ctl, prefix, sm_count, s)
                      : launch_typed<V, __nv_bfloat16, false>(tab, w, o, ctl, prefix, sm_count, s);
    }
    return cudaErrorInvalidValue;
}

template <int V, typename T, bool P2>
static void warm_t() {
    if constexpr (V == HS_STD) {
        occupancy<V, T, P2>();
        pair_occupancy<T, P2>();
        if constexpr (sizeof(T) == 2) pair_occupancy<float, P2, true>();  // 16-bit batches via FP32 groups
    } else {
        zoned_occupancy<V, T, P2>();
    }
}

template <int V, bool P2>
static void warm_p(hs_dtype dt) {
    if (dt == HS_F32) warm_t<V, float, P2>();
    if (dt == HS_F16) warm_t<V, __half, P2>();
    if (dt == HS_BF16) warm_t<V, __nv_bfloat16, P2>();
}

template <int V>
static void warm_v(hs_dtype dt) {
    warm_p<V, false>(dt);
    warm_p<V, true>(dt);
}

// Query occupancy outside any stream capture.
void warm_1d(hs_variant v, hs_dtype dt) {
    if (v == HS_STD) {
        warm_v<HS_STD>(dt);
        warm_eq1_staged(dt);
    }
    if (v == HS_MAX) warm_v<HS_MAX>(dt);
    if (v == HS_FBIN) warm_v<HS_FBIN>(dt);
    if (v == HS_GREEDY) warm_v<HS_GREEDY>(dt);
}

cudaError_t launch_1d(hs_variant v, hs_dtype dt, const Tables& tab, const Work1d& w, const Out1d& o,
                      WsControl* ctl, int64_t* prefix, int sm_count, cudaStream_t s) {
    if (v == HS_STD && (w.flags & HS_FLAG_STAGED_SPANS) && eq1_staged_applies(w, o))
        return launch_eq1_staged(dt, tab, w, o, ctl, prefix, sm_count, s);
    switch (v) {
        case HS_STD: return launch_dtype<HS_STD>(dt, tab, w, o, ctl, prefix, sm_count, s);
        case HS_MAX: return launch_dtype<HS_MAX>(dt, tab, w, o, ctl, prefix, sm_count, s);
        case HS_FBIN: return launch_dtype<HS_FBIN>(dt, tab, w, o, ctl, prefix, sm_count, s);
        case HS_GREEDY: return launch_dtype<HS_GREEDY>(dt, tab, w, o, ctl, prefix, sm_count, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace hs

// 1-D harmonic-sum kernels: the four variants of Section 2 (Eq. 1-4), one spectrum per launch or a
// packed batch of spectra walked by one persistent launch over a (spectrum, tile) work queue.
#include <algorithm>
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

// hmax = 32, outputs n and n+1 together.  For fraction f <= 1 their bins differ by 0 or 1: with
// W = n*F + 2^31, bin(n) = W >> 32 and bin(n+1) = (W + F) >> 32, which is one more exactly when
// the low word of W carries on adding F.  Both candidates are loaded and the carry picks one.  The
// low word of W is lo + 2^31 (lo = low word of n*F), and an unsigned compare of lo + 2^31 is a signed
// compare of lo itself, so the carry test needs no add.
// (lo + 2^31 mod 2^32) >u ~F  <=>  (int)lo > (int)(~F ^ 2^31): flipping the top bit maps unsigned
// order onto signed order.
template <uint32_t F>
struct CarryBound {
    static constexpr int32_t value = (int32_t)(~F ^ 0x80000000u);
};

template <typename T, int K, bool P2>
__device__ __forceinline__ void farey_pair_step(const T* x, uint32_t n, float2 (&S)[kHmax + 1]) {
    constexpr Frac f = farey_at(K);
    if constexpr (P2 && !is_pow2(f.q)) return;  // not read by any power-of-two stage
    float2 v;
    if (f.q == 1) {
        const T* p = x + n;
        v.x = widen<T>(__ldg(p));
        v.y = widen<T>(__ldg(p + 1));
    } else {
        constexpr uint32_t F = FracConst<f.p, f.q>::F;
        const uint32_t lo = n * F;
        const uint32_t k = __umulhi(n, F) + (lo >> 31);
        const T* p = x + k;
        const float a = widen<T>(__ldg(p)), b = widen<T>(__ldg(p + 1));
        v.x = a;
        v.y = ((int32_t)lo > CarryBound<F>::value) ? b : a;
    }
#pragma unroll
    for (int m = 1; m * f.q <= kHmax; ++m)
        if (!P2 || is_pow2(m)) S[m * f.q] = add2(S[m * f.q], v);
}

template <typename T, bool P2, int... K>
__device__ __forceinline__ void farey_pair_all(const T* x, uint32_t n, float2 (&S)[kHmax + 1],
                                               std::integer_sequence<int, K...>) {
    (farey_pair_step<T, K, P2>(x, n, S), ...);
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
    // outputs n and n+1 (both < N); hmax == 32; no every-H table
    template <bool P2>
    static __device__ __forceinline__ void eval_pair(const T* x, uint32_t n, const Tables& tb, float& best_a,
                                                     int& bh_a, float& best_b, int& bh_b) {
        float2 S[kHmax + 1];
#pragma unroll
        for (int H = 0; H <= kHmax; ++H) S[H] = make_float2(0.f, 0.f);
        farey_pair_all<T, P2>(x, n, S, std::make_integer_sequence<int, kNumFrac>{});
#pragma unroll
        for (int H = 1; H <= kHmax; ++H) {
            if (P2 && !is_pow2(H)) continue;
            keep_best(calibrate(tb, S[H].x, H), H, best_a, bh_a);
            keep_best(calibrate(tb, S[H].y, H), H, best_b, bh_b);
        }
    }
};

// Largest of the elements [w0, w1] (inclusive, w0 <= w1 <= N-1), read in aligned 16-byte chunks so a
// window of i bins costs about i/4 + 1 loads.  The maximum is exact, so the order of comparison does
// not change its value (and inputs carry no NaN).
template <typename T>
__device__ __forceinline__ float window_max(const T* x, uint32_t N, uint32_t w0, uint32_t w1) {
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
            add(i, window_max(x, N, base + j0, base + (uint32_t)i));
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
    if (V == HS_STD && w.hmax == kHmax && o.all_h == nullptr) {
        // consecutive output pairs: thread t owns bins base + 2t and base + 2t + 1
        for (; base + 2 * kBlock <= t1; base += 2 * kBlock) {
            const uint32_t n = base + 2 * threadIdx.x;
            float ba = -INFINITY, bb = -INFINITY;
            int ha = 0, hb = 0;
            Bin<HS_STD, T>::template eval_pair<P2>(x, n, tb, ba, ha, bb, hb);
            o.best_snr[out_off + n] = ba;
            o.best_h[out_off + n] = (uint8_t)ha;
            o.best_snr[out_off + n + 1] = bb;
            o.best_h[out_off + n + 1] = (uint8_t)hb;
            if (o.cand) {
                append_candidate(ba > w.threshold, o.cand, o.cand_count, o.cand_cap, status, spec, n, ba, 0, ha, V);
                append_candidate(bb > w.threshold, o.cand, o.cand_count, o.cand_cap, status, spec, n + 1, bb, 0, hb,
                                 V);
            }
        }
    }
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

template <int V>
struct MinBlocks {
    static constexpr int value = V == HS_STD ? 2 : 6;
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
                                                    int elem_bytes, int64_t* prefix, WsControl* ctl) {
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
            t = bad ? 0 : (len + tile - 1) / tile;
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

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
void launch_tile_scan(const int64_t* offsets, int n_spectra, int64_t tile, int64_t max_bins, int elem_bytes,
                      int64_t* prefix, WsControl* ctl, cudaStream_t s) {
    k_tile_scan<<<1, 1024, 0, s>>>(offsets, n_spectra, tile, max_bins, elem_bytes, prefix, ctl);
}

template <int V, typename T, bool P2>
static int& occupancy_slot() {
    static int occ = 0;  // resident CTAs per SM of the persistent kernel
    return occ;
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
static cudaError_t launch_typed(const Tables& tab, const Work1d& w, const Out1d& o, WsControl* ctl,
                                int64_t* prefix, int sm_count, cudaStream_t s) {
    const int64_t tile = (int64_t)kBlock * w.opt;
    if (w.offsets == nullptr) {
        if (w.n_bins == 0) return cudaSuccess;
        unsigned grid = (unsigned)((w.n_bins + tile - 1) / tile);
        k_hs1d_single<V, T, P2><<<grid, kBlock, 0, s>>>(tab, w, o, ctl);
        return cudaGetLastError();
    }
    launch_tile_scan(w.offsets, w.n_spectra, tile, w.max_bins, (int)sizeof(T), prefix, ctl, s);
    k_hs1d_batched<V, T, P2><<<(unsigned)(sm_count * occupancy<V, T, P2>()), kBlock, 0, s>>>(tab, w, o, ctl,
                                                                                          prefix);
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

template <int V, bool P2>
static void warm_p(hs_dtype dt) {
    if (dt == HS_F32) occupancy<V, float, P2>();
    if (dt == HS_F16) occupancy<V, __half, P2>();
    if (dt == HS_BF16) occupancy<V, __nv_bfloat16, P2>();
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

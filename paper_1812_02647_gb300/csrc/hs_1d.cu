// 1-D harmonic-sum kernels: the four variants of Section 2 (Eq. 1-4), one spectrum per launch or a
// packed batch of spectra walked by one persistent launch over a (spectrum, tile) work queue.
#include <algorithm>

#include "hs_common.cuh"

namespace hs {

// ------------------------------------------------------------------------------------------
// Per-bin evaluation of one variant.  Writes best snr / H (and the Eq. 4 path) of output bin n,
// and, when all_h is set, the snr of every H (-inf where H is not valid).
// ------------------------------------------------------------------------------------------

template <int V, typename T>
struct Bin;

// Eq. 1: a fresh sum of x(round-half-up(n*i/H)) for every H; every index is <= n.
template <typename T>
struct Bin<HS_STD, T> {
    static __device__ __forceinline__ void eval(const T* x, uint32_t N, uint32_t n, int hmax, const Tables& tb,
                                                float* all_h, uint32_t all_stride, float& best, int& bh,
                                                uint32_t& path) {
#pragma unroll
        for (int H = 1; H <= kHmax; ++H) {
            if (H <= hmax) {
                float S = 0.f;
#pragma unroll
                for (int i = 1; i <= H; ++i) {
                    uint32_t idx = (2u * n * (uint32_t)i + (uint32_t)H) / (2u * (uint32_t)H);
                    S = __fadd_rn(S, ldx(x, idx));
                }
                float snr = calibrate(tb, S, H);
                if (all_h) all_h[(size_t)(H - 1) * all_stride + n] = snr;
                keep_best(snr, H, best, bh);
            }
        }
    }
};

// Eq. 2: harmonic i adds the largest of x(i*n+1) .. x(i*n+i) (first maximum).
template <typename T>
struct Bin<HS_MAX, T> {
    static __device__ __forceinline__ void eval(const T* x, uint32_t N, uint32_t n, int hmax, const Tables& tb,
                                                float* all_h, uint32_t all_stride, float& best, int& bh,
                                                uint32_t& path) {
        int hv = N >= 1 ? (int)min((uint32_t)hmax, (N - 1) / (n + 1)) : 0;
        float S = 0.f;
#pragma unroll 1
        for (int i = 1; i <= hmax; ++i) {
            float snr = -INFINITY;
            if (i <= hv) {
                uint32_t base = (uint32_t)i * n;
                float m = ldx(x, base + 1);
                for (int j = 2; j <= i; ++j) {
                    float v = ldx(x, base + j);
                    m = (v > m) ? v : m;
                }
                S = __fadd_rn(S, m);
                snr = calibrate(tb, S, i);
                keep_best(snr, i, best, bh);
            }
            if (all_h) all_h[(size_t)(i - 1) * all_stride + n] = snr;
        }
    }
};

// Eq. 3: harmonic i adds x(i*n).
template <typename T>
struct Bin<HS_FBIN, T> {
    static __device__ __forceinline__ void eval(const T* x, uint32_t N, uint32_t n, int hmax, const Tables& tb,
                                                float* all_h, uint32_t all_stride, float& best, int& bh,
                                                uint32_t& path) {
        int hv = (n == 0) ? hmax : (int)min((uint32_t)hmax, (N - 1) / n);
        float S = 0.f;
#pragma unroll
        for (int i = 1; i <= kHmax; ++i) {
            if (i <= hmax) {
                float snr = -INFINITY;
                if (i <= hv) {
                    S = __fadd_rn(S, ldx(x, (uint32_t)i * n));
                    snr = calibrate(tb, S, i);
                    keep_best(snr, i, best, bh);
                }
                if (all_h) all_h[(size_t)(i - 1) * all_stride + n] = snr;
            }
        }
    }
};

// Eq. 4: harmonic i compares x(i*n+j) with x(i*n+j+1); the right bin wins only if strictly larger,
// and then j grows by one.
template <typename T>
struct Bin<HS_GREEDY, T> {
    static __device__ __forceinline__ void eval(const T* x, uint32_t N, uint32_t n, int hmax, const Tables& tb,
                                                float* all_h, uint32_t all_stride, float& best, int& bh,
                                                uint32_t& path) {
        int hv = N >= 1 ? (int)min((uint32_t)hmax, (N - 1) / (n + 1)) : 0;
        float S = 0.f;
        uint32_t j = 0, p = 0;
#pragma unroll
        for (int i = 1; i <= kHmax; ++i) {
            if (i <= hmax) {
                float snr = -INFINITY;
                if (i <= hv) {
                    uint32_t b = (uint32_t)i * n + j;
                    float l = ldx(x, b), r = ldx(x, b + 1), t;
                    if (r > l) {
                        t = r;
                        p |= 1u << (i - 1);
                        j += 1;
                    } else {
                        t = l;
                    }
                    S = __fadd_rn(S, t);
                    snr = calibrate(tb, S, i);
                    keep_best(snr, i, best, bh);
                }
                if (all_h) all_h[(size_t)(i - 1) * all_stride + n] = snr;
            }
        }
        path = p;
    }
};

// ------------------------------------------------------------------------------------------
// One tile of output bins [t0, t1) of one spectrum; the whole block walks it in steps of kBlock.
// ------------------------------------------------------------------------------------------
template <int V, typename T>
__device__ __forceinline__ void run_tile(const T* x, uint32_t N, uint32_t t0, uint32_t t1, const Tables& tb,
                                         const Work1d& w, const Out1d& o, size_t out_off, uint32_t spec,
                                         unsigned* status) {
    for (uint32_t base = t0; base < t1; base += kBlock) {
        uint32_t n = base + threadIdx.x;
        bool active = n < t1;
        float best = -INFINITY;
        int bh = 0;
        uint32_t path = 0;
        if (active) {
            Bin<V, T>::eval(x, N, n, w.hmax, tb, o.all_h, N, best, bh, path);
            o.best_snr[out_off + n] = best;
            o.best_h[out_off + n] = (uint8_t)bh;
            if (V == HS_GREEDY && o.path) o.path[out_off + n] = path;
        }
        if (o.cand)
            append_candidate(active && best > w.threshold, o.cand, o.cand_count, o.cand_cap, status, spec, n, best,
                             0, bh, V);
    }
}

template <int V, typename T>
__global__ void __launch_bounds__(kBlock) k_hs1d_single(const __grid_constant__ Tables tb, const Work1d w,
                                                        const Out1d o, WsControl* ctl) {
    uint32_t N = (uint32_t)w.n_bins;
    uint32_t tile = (uint32_t)(kBlock * w.opt);
    uint32_t t0 = blockIdx.x * tile;
    uint32_t t1 = min(N, t0 + tile);
    run_tile<V, T>((const T*)w.x, N, t0, t1, tb, w, o, 0, w.first_id, &ctl->status);
}

// Tile prefix sums of a batch and reset of the work queue.  One block.  A spectrum that breaks
// the layout contract (negative or oversized length, offsets[0] != 0, misaligned start) is given
// zero tiles and flagged in the status word.
__global__ void __launch_bounds__(1024) k_tile_scan(const int64_t* offsets, int n, int64_t tile, int64_t max_bins,
                                                    int elem_bytes, int64_t* prefix, WsControl* ctl) {
    __shared__ int64_t warp_sum[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) {
        carry = 0;
        ctl->queue = 0u;
        if (offsets[0] != 0) atomicOr(&ctl->status, kStatusBadInput);
    }
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        int s = base + threadIdx.x;
        int64_t t = 0;
        if (s < n) {
            int64_t a = offsets[s], b = offsets[s + 1], len = b - a;
            bool bad = len < 0 || len > max_bins || ((a * elem_bytes) & 15) != 0;
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

template <int V, typename T>
__global__ void __launch_bounds__(kBlock) k_hs1d_batched(const __grid_constant__ Tables tb, const Work1d w,
                                                         const Out1d o, WsControl* ctl, const int64_t* prefix) {
    __shared__ unsigned long long s_item;
    __shared__ int s_spec;
    const unsigned long long total = *(volatile unsigned long long*)&ctl->total_items;
    const uint32_t tile = (uint32_t)(kBlock * w.opt);
    for (;;) {
        if (threadIdx.x == 0) {
            unsigned long long item = atomicAdd(&ctl->queue, 1u);
            int s = 0;
            if (item < total) {
                int lo = 0, hi = w.n_spectra - 1;  // last s with prefix[s] <= item
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if ((unsigned long long)prefix[mid] <= item) lo = mid; else hi = mid - 1;
                }
                s = lo;
            }
            s_item = item;
            s_spec = s;
        }
        __syncthreads();
        unsigned long long item = s_item;
        int s = s_spec;
        __syncthreads();
        if (item >= total) break;
        int64_t off = w.offsets[s];
        uint32_t N = (uint32_t)(w.offsets[s + 1] - off);
        uint32_t t0 = (uint32_t)(item - (unsigned long long)prefix[s]) * tile;
        uint32_t t1 = min(N, t0 + tile);
        run_tile<V, T>((const T*)w.x + off, N, t0, t1, tb, w, o, (size_t)off, w.first_id + (uint32_t)s,
                       &ctl->status);
    }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
template <int V, typename T>
static int& occupancy_slot() {
    static int occ = 0;  // resident CTAs per SM of the persistent kernel
    return occ;
}

template <int V, typename T>
static int occupancy() {
    int& oc = occupancy_slot<V, T>();
    if (oc == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oc, k_hs1d_batched<V, T>, kBlock, 0);
        if (e != cudaSuccess || oc < 1) oc = 1;
    }
    return oc;
}

template <int V, typename T>
static cudaError_t launch_typed(const Tables& tab, const Work1d& w, const Out1d& o, WsControl* ctl,
                                int64_t* prefix, int sm_count, cudaStream_t s) {
    const int64_t tile = (int64_t)kBlock * w.opt;
    if (w.offsets == nullptr) {
        if (w.n_bins == 0) return cudaSuccess;
        unsigned grid = (unsigned)((w.n_bins + tile - 1) / tile);
        k_hs1d_single<V, T><<<grid, kBlock, 0, s>>>(tab, w, o, ctl);
        return cudaGetLastError();
    }
    k_tile_scan<<<1, 1024, 0, s>>>(w.offsets, w.n_spectra, tile, w.max_bins, (int)sizeof(T), prefix, ctl);
    k_hs1d_batched<V, T><<<(unsigned)(sm_count * occupancy<V, T>()), kBlock, 0, s>>>(tab, w, o, ctl, prefix);
    return cudaGetLastError();
}

template <int V>
static cudaError_t launch_dtype(hs_dtype dt, const Tables& tab, const Work1d& w, const Out1d& o, WsControl* ctl,
                                int64_t* prefix, int sm_count, cudaStream_t s) {
    switch (dt) {
        case HS_F32: return launch_typed<V, float>(tab, w, o, ctl, prefix, sm_count, s);
        case HS_F16: return launch_typed<V, __half>(tab, w, o, ctl, prefix, sm_count, s);
        case HS_BF16: return launch_typed<V, __nv_bfloat16>(tab, w, o, ctl, prefix, sm_count, s);
    }
    return cudaErrorInvalidValue;
}

template <int V>
static void warm_v(hs_dtype dt) {
    if (dt == HS_F32) occupancy<V, float>();
    if (dt == HS_F16) occupancy<V, __half>();
    if (dt == HS_BF16) occupancy<V, __nv_bfloat16>();
}

// Query occupancy outside any stream capture.
void warm_1d(hs_variant v, hs_dtype dt) {
    if (v == HS_STD) warm_v<HS_STD>(dt);
    if (v == HS_MAX) warm_v<HS_MAX>(dt);
    if (v == HS_FBIN) warm_v<HS_FBIN>(dt);
    if (v == HS_GREEDY) warm_v<HS_GREEDY>(dt);
}

cudaError_t launch_1d(hs_variant v, hs_dtype dt, const Tables& tab, const Work1d& w, const Out1d& o,
                      WsControl* ctl, int64_t* prefix, int sm_count, cudaStream_t s) {
    switch (v) {
        case HS_STD: return launch_dtype<HS_STD>(dt, tab, w, o, ctl, prefix, sm_count, s);
        case HS_MAX: return launch_dtype<HS_MAX>(dt, tab, w, o, ctl, prefix, sm_count, s);
        case HS_FBIN: return launch_dtype<HS_FBIN>(dt, tab, w, o, ctl, prefix, sm_count, s);
        case HS_GREEDY: return launch_dtype<HS_GREEDY>(dt, tab, w, o, ctl, prefix, sm_count, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace hs

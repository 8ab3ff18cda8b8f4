// Auxiliary device steps: standardise + cast to FP16/BF16 storage, and a stable LSD radix sort of
// the candidate list by (variant, spectrum, z, bin).
#include <algorithm>

#include "hs_common.cuh"

namespace hs {

// ------------------------------------------------------------------------------------------
// y = (p - mu_s) / sigma_s in FP32 (IEEE division), rounded to nearest even FP16 / BF16.
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T narrow(float y);
template <>
__device__ __forceinline__ __half narrow<__half>(float y) {
    return __float2half_rn(y);
}
template <>
__device__ __forceinline__ __nv_bfloat16 narrow<__nv_bfloat16>(float y) {
    return __float2bfloat16_rn(y);
}

// Streaming kernel: blockIdx.y walks spectra, the x-blocks of a row stride over the spectrum with
// 16-byte loads of four values (8-byte stores of four FP16/BF16 results); a spectrum whose start or
// length is not a multiple of four takes the element-wise path for its head and tail.
template <typename T>
struct Pack4;
template <>
struct Pack4<__half> {
    static __device__ __forceinline__ uint2 make(float a, float b, float c, float d) {
        __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, d);
        return make_uint2(*reinterpret_cast<unsigned*>(&lo), *reinterpret_cast<unsigned*>(&hi));
    }
};
template <>
struct Pack4<__nv_bfloat16> {
    static __device__ __forceinline__ uint2 make(float a, float b, float c, float d) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
        return make_uint2(*reinterpret_cast<unsigned*>(&lo), *reinterpret_cast<unsigned*>(&hi));
    }
};

template <typename T>
__global__ void __launch_bounds__(256) k_standardize_cast(const float* p, const int64_t* offsets, int n_spectra,
                                                          int64_t n_bins, const float* mu, const float* sigma, T* out) {
    for (int s = blockIdx.y; s < n_spectra; s += gridDim.y) {
        const int64_t off = offsets ? offsets[s] : 0;
        const int64_t N = offsets ? offsets[s + 1] - off : n_bins;
        const float m = mu[s], sd = sigma[s];
        const int64_t step = (int64_t)gridDim.x * blockDim.x;
        const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        // elements before the first 16-byte boundary of the input, and after the last
        const int64_t head = ((4 - (off & 3)) & 3) < N ? ((4 - (off & 3)) & 3) : N;
        const int64_t nvec = (N - head) / 4;
        if (t0 < head) out[off + t0] = narrow<T>(__fdiv_rn(__fsub_rn(p[off + t0], m), sd));
        const float4* pv = reinterpret_cast<const float4*>(p + off + head);
        uint2* ov = reinterpret_cast<uint2*>(out + off + head);
        for (int64_t k = t0; k < nvec; k += step) {
            const float4 v = __ldg(pv + k);
            ov[k] = Pack4<T>::make(__fdiv_rn(__fsub_rn(v.x, m), sd), __fdiv_rn(__fsub_rn(v.y, m), sd),
                                   __fdiv_rn(__fsub_rn(v.z, m), sd), __fdiv_rn(__fsub_rn(v.w, m), sd));
        }
        for (int64_t k = head + 4 * nvec + t0; k < N; k += step)
            out[off + k] = narrow<T>(__fdiv_rn(__fsub_rn(p[off + k], m), sd));
    }
}

cudaError_t launch_standardize_cast(const float* p, const int64_t* offsets, int n_spectra, int64_t n_bins,
                                    const float* mu, const float* sigma, hs_dtype dt, void* out, cudaStream_t s) {
    if (n_spectra == 0 || n_bins == 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // about eight resident blocks per SM in total, spread over spectra
    const int64_t cap = std::max<int64_t>(64, (int64_t)sms * 8 / n_spectra);
    const int64_t per_spec = std::max<int64_t>(1, std::min<int64_t>((n_bins / 4 + 255) / 256, cap));
    const int64_t ys = std::max<int64_t>(1, std::min<int64_t>(n_spectra, (int64_t)sms * 8 / per_spec + 1));
    dim3 grid((unsigned)per_spec, (unsigned)std::min<int64_t>(ys, 65535));
    if (dt == HS_F16)
        k_standardize_cast<__half><<<grid, 256, 0, s>>>(p, offsets, n_spectra, n_bins, mu, sigma, (__half*)out);
    else
        k_standardize_cast<__nv_bfloat16>
            <<<grid, 256, 0, s>>>(p, offsets, n_spectra, n_bins, mu, sigma, (__nv_bfloat16*)out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Candidate sort.  Key digits, least significant first: bin (4 bytes), z (2 bytes, offset by
// 2^15), spectrum (4 bytes), variant (1 byte).  A digit that is the same for every candidate is
// copied through instead of scattered.  The count is read on the device, so the launch shapes
// cover the capacity and blocks beyond the count exit.
// ------------------------------------------------------------------------------------------
constexpr int kSortBlock = 256;
constexpr int kSortPer = 16;
constexpr int kSortChunk = kSortBlock * kSortPer;
constexpr int kSortPasses = 11;

__device__ __forceinline__ unsigned cand_digit(const uint4& c, int pass) {
    switch (pass) {
        case 0: case 1: case 2: case 3: return (c.y >> (8 * pass)) & 0xffu;             // bin
        case 4: case 5: return (((c.w & 0xffffu) ^ 0x8000u) >> (8 * (pass - 4))) & 0xffu;  // z, biased
        case 6: case 7: case 8: case 9: return (c.x >> (8 * (pass - 6))) & 0xffu;        // spectrum
        default: return (c.w >> 24) & 0xffu;                                              // variant
    }
}

struct SortCtl {
    unsigned long long n;     // number of candidates to sort
    unsigned nb;              // blocks that hold candidates: the histogram's row stride
    unsigned dig_or[kSortPasses];
    unsigned dig_and[kSortPasses];
};

__global__ void k_sort_init(const unsigned long long* count, long long cap, SortCtl* sc) {
    if (threadIdx.x == 0) {
        unsigned long long c = *count;
        sc->n = c < (unsigned long long)cap ? c : (unsigned long long)cap;
        sc->nb = (unsigned)((sc->n + kSortChunk - 1) / kSortChunk);
    }
    if (threadIdx.x < kSortPasses) {
        sc->dig_or[threadIdx.x] = 0u;
        sc->dig_and[threadIdx.x] = 0xffu;
    }
}

__global__ void __launch_bounds__(kSortBlock) k_sort_digits(const uint4* c, SortCtl* sc) {
    const unsigned long long n = sc->n;
    unsigned o[kSortPasses], a[kSortPasses];
    for (int p = 0; p < kSortPasses; ++p) {
        o[p] = 0u;
        a[p] = 0xffu;
    }
    for (unsigned long long k = (unsigned long long)blockIdx.x * kSortBlock + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * kSortBlock) {
        uint4 v = c[k];
        for (int p = 0; p < kSortPasses; ++p) {
            unsigned d = cand_digit(v, p);
            o[p] |= d;
            a[p] &= d;
        }
    }
    for (int p = 0; p < kSortPasses; ++p) {
        atomicOr(&sc->dig_or[p], o[p]);
        atomicAnd(&sc->dig_and[p], a[p]);
    }
}

__device__ __forceinline__ bool pass_skipped(const SortCtl* sc, int pass) {
    return (sc->dig_or[pass] ^ sc->dig_and[pass]) == 0u;
}

// per-block digit histograms, stored digit-major: hist[d * nblocks + block]
__global__ void __launch_bounds__(kSortBlock) k_sort_hist(const uint4* src, const SortCtl* sc, int pass,
                                                          unsigned* hist) {
    __shared__ unsigned h[256];
    if (pass_skipped(sc, pass) || blockIdx.x >= sc->nb) return;
    const unsigned long long n = sc->n;
    const unsigned nblocks = sc->nb;
    h[threadIdx.x] = 0u;
    __syncthreads();
    const unsigned long long c0 = (unsigned long long)blockIdx.x * kSortChunk;
    for (int k = threadIdx.x; k < kSortChunk; k += kSortBlock) {
        unsigned long long i = c0 + k;
        if (i < n) atomicAdd(&h[cand_digit(src[i], pass)], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of hist (256 * nb entries) in place, one block; four consecutive entries per thread
__global__ void __launch_bounds__(1024) k_sort_scan(const SortCtl* sc, int pass, unsigned* hist) {
    __shared__ unsigned ws[32];
    __shared__ unsigned carry;
    if (pass_skipped(sc, pass)) return;
    const int total = 256 * (int)sc->nb;
    if (threadIdx.x == 0) carry = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < total; base += 4096) {
        const int i0 = base + 4 * threadIdx.x;
        unsigned e[4], t = 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            e[k] = i0 + k < total ? hist[i0 + k] : 0u;
            t += e[k];
        }
        unsigned v = t;
        for (int d = 1; d < 32; d <<= 1) {
            unsigned u = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v += u;
        }
        if (lane == 31) ws[wid] = v;
        __syncthreads();
        if (wid == 0) {
            unsigned x = ws[lane];
            for (int d = 1; d < 32; d <<= 1) {
                unsigned u = __shfl_up_sync(0xffffffffu, x, d);
                if (lane >= d) x += u;
            }
            ws[lane] = x;
        }
        __syncthreads();
        unsigned run = carry + (wid ? ws[wid - 1] : 0u) + v - t;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k < total) hist[i0 + k] = run;
            run += e[k];
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry = run;
        __syncthreads();
    }
}

// stable scatter: warp w of a block owns the w-th contiguous slice of the block's chunk
__global__ void __launch_bounds__(kSortBlock) k_sort_scatter(const uint4* src, uint4* dst, const SortCtl* sc,
                                                             int pass, const unsigned* hist) {
    constexpr int kWarps = kSortBlock / 32;
    constexpr int kSlice = kSortChunk / kWarps;
    __shared__ unsigned wbase[kWarps][256];
    const unsigned long long n = sc->n;
    const unsigned long long c0 = (unsigned long long)blockIdx.x * kSortChunk;
    if (c0 >= n) return;
    const unsigned nblocks = sc->nb;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (pass_skipped(sc, pass)) {
        for (int k = threadIdx.x; k < kSortChunk; k += kSortBlock) {
            unsigned long long i = c0 + k;
            if (i < n) dst[i] = src[i];
        }
        return;
    }
    for (int d = lane; d < 256; d += 32) wbase[w][d] = 0u;
    __syncwarp();
    const unsigned long long s0 = c0 + (unsigned long long)w * kSlice;
    for (int k = 0; k < kSlice; k += 32) {  // count this warp's digits
        unsigned long long i = s0 + k + lane;
        if (i < n) atomicAdd(&wbase[w][cand_digit(src[i], pass)], 1u);
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, plus the block's global base
    for (int d = threadIdx.x; d < 256; d += kSortBlock) {
        unsigned run = hist[(size_t)d * nblocks + blockIdx.x];
        for (int k = 0; k < kWarps; ++k) {
            unsigned c = wbase[k][d];
            wbase[k][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int k = 0; k < kSlice; k += 32) {
        unsigned long long i = s0 + k + lane;
        bool ok = i < n;
        uint4 v = ok ? src[i] : make_uint4(0, 0, 0, 0);
        unsigned d = ok ? cand_digit(v, pass) : 0xffffffffu;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank = __popc(peers & ((1u << lane) - 1u));
        if (ok) dst[wbase[w][d] + rank] = v;
        __syncwarp();
        if (ok && rank == 0) wbase[w][d] += __popc(peers);
        __syncwarp();
    }
}

__global__ void k_copy_cand(const uint4* src, uint4* dst, const SortCtl* sc) {
    const unsigned long long n = sc->n;
    for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * blockDim.x)
        dst[k] = src[k];
}

size_t sort_scratch_bytes(int64_t capacity) {
    int64_t nb = (capacity + kSortChunk - 1) / kSortChunk;
    return 256 + sizeof(unsigned) * 256 * (size_t)std::max<int64_t>(nb, 1);
}

cudaError_t launch_sort_candidates(hs_candidate* cand, const unsigned long long* count, int64_t capacity,
                                   hs_candidate* tmp, WsControl* ctl, cudaStream_t s) {
    if (capacity <= 0) return cudaSuccess;
    SortCtl* sc = reinterpret_cast<SortCtl*>(reinterpret_cast<char*>(ctl) + 64);
    unsigned* hist = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(ctl) + kWsControlBytes);
    const int nblocks = (int)((capacity + kSortChunk - 1) / kSortChunk);
    k_sort_init<<<1, 32, 0, s>>>(count, capacity, sc);
    k_sort_digits<<<std::min(nblocks * 4, 1024), kSortBlock, 0, s>>>(reinterpret_cast<const uint4*>(cand), sc);
    uint4* a = reinterpret_cast<uint4*>(cand);
    uint4* b = reinterpret_cast<uint4*>(tmp);
    for (int p = 0; p < kSortPasses; ++p) {
        k_sort_hist<<<nblocks, kSortBlock, 0, s>>>(a, sc, p, hist);
        k_sort_scan<<<1, 1024, 0, s>>>(sc, p, hist);
        k_sort_scatter<<<nblocks, kSortBlock, 0, s>>>(a, b, sc, p, hist);
        std::swap(a, b);
    }
    // an odd number of passes leaves the result in tmp
    k_copy_cand<<<std::min(nblocks * 4, 1024), 256, 0, s>>>(a, reinterpret_cast<uint4*>(cand), sc);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Candidate sifting.  In a list sorted by (variant, spectrum, z, bin), a candidate is dropped when a
// stronger candidate of its (variant, spectrum) group is related to it: some k = 1..kmax puts the
// higher fundamental within k*tol bins (and k*tol_z drift rows) of k times the lower one.  The
// fundamental is (bin / H, z / H) for Eq. 1 and its 2-D form, which report the H-th harmonic, and
// the bin itself for Eq. 2-4.  Stronger: larger snr, or equal snr and earlier in the list.  Every
// comparison is taken in FP32 with each operation rounded, in the order written.
// ------------------------------------------------------------------------------------------
namespace {

struct Fund {
    float f, z, snr;
    unsigned long long key;  // (variant, spectrum)
};

__device__ __forceinline__ Fund fundamental(const uint4 c) {
    Fund r;
    const float bin = (float)c.y;
    const float z = (float)(int16_t)(c.w & 0xFFFFu);
    const unsigned h = max((c.w >> 16) & 0xFFu, 1u), v = c.w >> 24;
    if (v == (unsigned)HS_STD) {
        r.f = __fdiv_rn(bin, (float)h);
        r.z = __fdiv_rn(z, (float)h);
    } else {
        r.f = bin;
        r.z = z;
    }
    r.snr = __uint_as_float(c.z);
    r.key = ((unsigned long long)v << 32) | c.x;
    return r;
}

__device__ __forceinline__ bool related_k(float fl, float zl, float fh, float zh, float tol, float tol_z, int k) {
    const float kf = (float)k;
    return fabsf(__fsub_rn(fh, __fmul_rn(kf, fl))) <= __fmul_rn(kf, tol) &&
           fabsf(__fsub_rn(zh, __fmul_rn(kf, zl))) <= __fmul_rn(kf, tol_z);
}

// Whether some k = 1..kmax relates the two fundamentals.  Without drift, g(k) = |fh - k fl| - k tol
// is convex in k with its kink at fh / fl, falling before it and, when fl > tol, rising after it; so
// if any k <= kmax has g(k) <= 0, so does the integer minimiser of g over 1..kmax, which lies next to
// fh / fl (clamped to 1..kmax).  The integers around it are tested, one further on each side for the
// rounding of the quotient, each with the exact test.  With drift, or fl <= tol, every k is tested.
__device__ __forceinline__ bool related(float4 a, float4 b, float tol, float tol_z, int kmax) {
    const bool al = a.x <= b.x;
    const float fl = al ? a.x : b.x, zl = al ? a.y : b.y, fh = al ? b.x : a.x, zh = al ? b.y : a.y;
    int k0 = 1, k1 = kmax;
    if (zl == 0.f && zh == 0.f && fl > tol) {
        const float kc = __fdiv_rn(fh, fl);
        const int kf = kc < (float)kmax ? (int)kc : kmax;  // floor of a non-negative quotient, capped
        k0 = max(1, kf - 1);
        k1 = min(kmax, kf + 2);
    }
    for (int k = k0; k <= k1; ++k)
        if (related_k(fl, zl, fh, zh, tol, tol_z, k)) return true;
    return false;
}

__device__ __forceinline__ unsigned long long cand_key(const uint4* c, uint32_t i) {
    const uint4 v = c[i];
    return ((unsigned long long)(v.w >> 24) << 32) | v.x;
}

__device__ __forceinline__ uint32_t sift_count(const unsigned long long* count, long long cap) {
    const unsigned long long cnt = *count;
    return (uint32_t)(cnt < (unsigned long long)cap ? cnt : (unsigned long long)cap);
}

// (fundamental frequency, drift, snr) of every candidate, once
__global__ void __launch_bounds__(256) k_sift_fund(const uint4* cand, const unsigned long long* count, long long cap,
                                                   float4* fund) {
    const uint32_t n = sift_count(count, cap);
    for (uint32_t i = blockIdx.x * 256u + threadIdx.x; i < n; i += gridDim.x * 256u) {
        const Fund r = fundamental(cand[i]);
        fund[i] = make_float4(r.f, r.z, r.snr, 0.f);
    }
}

__global__ void __launch_bounds__(256) k_sift(const uint4* cand, const float4* fund, const unsigned long long* count,
                                              long long cap, float tol, float tol_z, int kmax, uint4* out,
                                              unsigned long long* out_count) {
    const uint32_t n = sift_count(count, cap);
    for (uint32_t base = blockIdx.x * 256u; base < n; base += gridDim.x * 256u) {
        const uint32_t i = base + threadIdx.x;
        bool keep = false;
        uint4 ci = make_uint4(0u, 0u, 0u, 0u);
        if (i < n) {
            ci = cand[i];
            const unsigned long long key = ((unsigned long long)(ci.w >> 24) << 32) | ci.x;
            const float4 a = fund[i];
            // the group [lo, end) of this (variant, spectrum) in the sorted list
            uint32_t lo = 0, hi = i;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (cand_key(cand, mid) < key) lo = mid + 1; else hi = mid;
            }
            uint32_t end = i + 1, top = n;
            while (end < top) {
                const uint32_t mid = (end + top) >> 1;
                if (cand_key(cand, mid) <= key) end = mid + 1; else top = mid;
            }
            keep = true;
            for (uint32_t j = lo; j < end && keep; ++j) {
                if (j == i) continue;
                const float4 b = fund[j];
                const bool stronger = b.z > a.z || (b.z == a.z && j < i);
                if (stronger && related(b, a, tol, tol_z, kmax)) keep = false;
            }
        }
        // warp-aggregated append of the kept candidates (unordered; sorted afterwards)
        const unsigned mask = __ballot_sync(0xffffffffu, keep);
        if (mask) {
            const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
            unsigned long long pos = 0;
            if (lane == leader) pos = atomicAdd(out_count, (unsigned long long)__popc(mask));
            pos = __shfl_sync(0xffffffffu, pos, leader);
            if (keep) out[pos + __popc(mask & ((1u << lane) - 1u))] = ci;
        }
    }
}

}  // namespace

cudaError_t launch_sift_candidates(const hs_candidate* cand, const unsigned long long* count, int64_t capacity,
                                   float tol, float tol_z, int kmax, hs_candidate* out,
                                   unsigned long long* out_count, hs_candidate* tmp, WsControl* ctl,
                                   cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out_count, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || capacity <= 0) return e;
    const int nb = (int)std::min<int64_t>((capacity + 255) / 256, 4096);
    float4* fund = reinterpret_cast<float4*>(tmp);  // scratch until the final sort
    k_sift_fund<<<nb, 256, 0, s>>>(reinterpret_cast<const uint4*>(cand), count, capacity, fund);
    k_sift<<<nb, 256, 0, s>>>(reinterpret_cast<const uint4*>(cand), fund, count, capacity, tol, tol_z, kmax,
                              reinterpret_cast<uint4*>(out), out_count);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_sort_candidates(out, out_count, capacity, tmp, ctl, s);
}

}  // namespace hs

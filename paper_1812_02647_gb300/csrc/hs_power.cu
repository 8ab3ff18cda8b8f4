// The step before the harmonic sums: power of a complex spectrum, dereddened by interpolated block
// medians, standardised and stored in the plan's storage type (the input of Section 2's sums).
//   P_k = re_k re_k + im_k im_k                                   FP32, each operation rounded
//   m_j = lower median of P over block j (rank floor((size_j - 1)/2))
//   base_k = m_a + t (m_b - m_a), linear between the centres of neighbouring blocks (flat before the
//            first centre and after the last); Exp-distributed power has mean median / ln 2
//   x_k = (P_k ln2) / base_k - 1, or 0 where base_k <= 0
// Kernels: a warp sorts each block of B bins with a bitonic network (exact min/max) and keeps the
// lower median; a streaming pass computes x from the medians of a bin's block and its neighbour.
#include <algorithm>

#include "hs_common.cuh"

namespace hs {

namespace {

constexpr int kPowBlock = 256;  // threads per CTA

__device__ __forceinline__ float power_of(const float2* spec, uint32_t k) {
    const float2 z = __ldg(spec + k);
    return __fadd_rn(__fmul_rn(z.x, z.x), __fmul_rn(z.y, z.y));
}

// Bitonic sort of the B values of one warp, value r*32 + lane held in v[r]; ascending.
template <int B>
__device__ __forceinline__ void warp_bitonic(float (&v)[B / 32], uint32_t lane) {
    constexpr int R = B / 32;
#pragma unroll
    for (int k = 2; k <= B; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {  // partner in another register of the same lane
                const int jr = j / 32;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int rp = r ^ jr;
                    if (rp > r) {
                        const bool up = (((r * 32 + (int)lane) & k) == 0);
                        const float a = v[r], b = v[rp];
                        const float lo = fminf(a, b), hi = fmaxf(a, b);
                        v[r] = up ? lo : hi;
                        v[rp] = up ? hi : lo;
                    }
                }
            } else {  // partner in lane ^ j, same register
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float o = __shfl_xor_sync(0xffffffffu, v[r], j);
                    const int i = r * 32 + (int)lane;
                    const bool up = ((i & k) == 0);
                    const bool lower = ((int)lane & j) == 0;  // this element has the smaller index
                    const float lo = fminf(v[r], o), hi = fmaxf(v[r], o);
                    v[r] = (lower == up) ? lo : hi;
                }
            }
        }
    }
}

struct PowWork {
    const float2* spec;
    const int64_t* offsets;  // nullptr: one spectrum of n_bins
    const int64_t* prefix;   // median-block prefix per spectrum (batched)
    int64_t n_bins;
    float* medians;
    long long med_cap;
};

// Spectrum s of the work: 1 to process, 0 to skip (empty, or rejected by the layout check, which
// flags it), -1 when its medians would not fit the caller's array.
__device__ __forceinline__ int pow_spectrum(const PowWork& w, int s, int B, int64_t& off, uint32_t& N,
                                            int64_t& moff) {
    if (w.offsets) {
        off = w.offsets[s];
        moff = w.prefix[s];
        if (w.prefix[s + 1] == moff) return 0;
        N = (uint32_t)(w.offsets[s + 1] - off);
    } else {
        off = 0;
        N = (uint32_t)w.n_bins;
        moff = 0;
        if (N == 0) return 0;
    }
    return moff + (int64_t)((N + B - 1) / B) <= w.med_cap ? 1 : -1;
}

template <int B>
__global__ void __launch_bounds__(kPowBlock) k_block_median(const PowWork w, WsControl* ctl) {
    int64_t off, moff;
    uint32_t N;
    const int use = pow_spectrum(w, blockIdx.y, B, off, N, moff);
    if (use != 1) {
        if (use < 0 && threadIdx.x == 0 && blockIdx.x == 0) atomicOr(&ctl->status, kStatusBadInput);
        return;
    }
    const float2* spec = w.spec + off;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nblk = (N + B - 1) / B;
    const uint32_t warps = kPowBlock / 32;
    for (uint32_t jb = blockIdx.x * warps + (threadIdx.x >> 5); jb < nblk; jb += gridDim.x * warps) {
        const uint32_t lo = jb * B, size = min((uint32_t)B, N - lo);
        float v[B / 32];
#pragma unroll
        for (int r = 0; r < B / 32; ++r) {
            const uint32_t e = (uint32_t)r * 32u + lane;
            v[r] = e < size ? power_of(spec, lo + e) : INFINITY;  // padding sorts to the end
        }
        warp_bitonic<B>(v, lane);
        const uint32_t rank = (size - 1u) / 2u;
#pragma unroll
        for (int r = 0; r < B / 32; ++r)
            if (rank == (uint32_t)r * 32u + lane) w.medians[moff + jb] = v[r];
    }
}

template <typename T>
__device__ __forceinline__ void store_as(T* out, uint32_t k, float x);
template <>
__device__ __forceinline__ void store_as<float>(float* out, uint32_t k, float x) {
    out[k] = x;
}
template <>
__device__ __forceinline__ void store_as<__half>(__half* out, uint32_t k, float x) {
    out[k] = __float2half_rn(x);
}
template <>
__device__ __forceinline__ void store_as<__nv_bfloat16>(__nv_bfloat16* out, uint32_t k, float x) {
    out[k] = __float2bfloat16_rn(x);
}

template <typename T>
__global__ void __launch_bounds__(kPowBlock) k_power_normalize(const PowWork w, int B, T* out) {
    int64_t off, moff;
    uint32_t N;
    if (pow_spectrum(w, blockIdx.y, B, off, N, moff) != 1) return;
    const float2* spec = w.spec + off;
    const float* m = w.medians + moff;
    T* o = out + off;
    const uint32_t nblk = (N + B - 1) / B;
    const float ln2 = 0.693147180559945309417232f;
    const float fB = (float)B, hfull = 0.5f * (float)(B - 1);
    for (uint32_t k = blockIdx.x * kPowBlock + threadIdx.x; k < N; k += gridDim.x * kPowBlock) {
        const uint32_t j = k / (uint32_t)B;
        const float d = (float)(k - j * (uint32_t)B);
        const float hj = 0.5f * (float)(min((uint32_t)B, N - j * B) - 1u);
        float base;
        if (d >= hj && j + 1 < nblk) {
            const float hn = 0.5f * (float)(min((uint32_t)B, N - (j + 1) * B) - 1u);
            const float t = __fdiv_rn(__fsub_rn(d, hj), __fadd_rn(__fsub_rn(fB, hj), hn));
            const float a = __ldg(m + j), b = __ldg(m + j + 1);
            base = __fadd_rn(a, __fmul_rn(t, __fsub_rn(b, a)));
        } else if (d < hj && j > 0) {
            const float t = __fdiv_rn(__fsub_rn(__fadd_rn(d, fB), hfull), __fadd_rn(__fsub_rn(fB, hfull), hj));
            const float a = __ldg(m + j - 1), b = __ldg(m + j);
            base = __fadd_rn(a, __fmul_rn(t, __fsub_rn(b, a)));
        } else {
            base = __ldg(m + j);
        }
        const float P = power_of(spec, k);
        const float x = base > 0.f ? __fsub_rn(__fdiv_rn(__fmul_rn(P, ln2), base), 1.0f) : 0.f;
        store_as<T>(o, k, x);
    }
}

// CTAs per spectrum: enough to cover its blocks, and about eight CTAs per SM over the whole batch.
inline unsigned ctas_per_spectrum(int64_t units, int64_t per_cta, int n_spectra, int sms) {
    const int64_t need = std::max<int64_t>(1, (units + per_cta - 1) / per_cta);
    return (unsigned)std::min<int64_t>(need, std::max(1, sms * 8 / std::max(1, n_spectra)));
}

template <int B>
cudaError_t launch_median(const PowWork& w, int n_spectra, int64_t longest, int sms, WsControl* ctl, cudaStream_t s) {
    const unsigned gx = ctas_per_spectrum((longest + B - 1) / B, kPowBlock / 32, n_spectra, sms);
    k_block_median<B><<<dim3(gx, (unsigned)n_spectra), kPowBlock, 0, s>>>(w, ctl);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_power_normalize(const float* spec, const int64_t* offsets, int n_spectra, int64_t n_bins, int block,
                                   float* medians, long long med_cap, hs_dtype dt, void* out, int64_t max_bins,
                                   int sm_count, int64_t* prefix, WsControl* ctl, cudaStream_t s) {
    PowWork w{reinterpret_cast<const float2*>(spec), offsets, prefix, n_bins, medians, med_cap};
    if (offsets) launch_tile_scan(offsets, n_spectra, block, max_bins, 8, prefix, ctl, s);
    const int64_t longest = offsets ? max_bins : n_bins;
    cudaError_t e = cudaSuccess;
    switch (block) {
        case 32: e = launch_median<32>(w, n_spectra, longest, sm_count, ctl, s); break;
        case 64: e = launch_median<64>(w, n_spectra, longest, sm_count, ctl, s); break;
        case 128: e = launch_median<128>(w, n_spectra, longest, sm_count, ctl, s); break;
        case 256: e = launch_median<256>(w, n_spectra, longest, sm_count, ctl, s); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const dim3 grid(ctas_per_spectrum(longest, kPowBlock, n_spectra, sm_count), (unsigned)n_spectra);
    switch (dt) {
        case HS_F32: k_power_normalize<float><<<grid, kPowBlock, 0, s>>>(w, block, (float*)out); break;
        case HS_F16: k_power_normalize<__half><<<grid, kPowBlock, 0, s>>>(w, block, (__half*)out); break;
        case HS_BF16: k_power_normalize<__nv_bfloat16><<<grid, kPowBlock, 0, s>>>(w, block, (__nv_bfloat16*)out); break;
    }
    return cudaGetLastError();
}

}  // namespace hs

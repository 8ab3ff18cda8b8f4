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
#include <type_traits>

#include "hs_common.cuh"

namespace hs {

namespace {

constexpr int kPowBlock = 256;  // threads per CTA

__device__ __forceinline__ float power_of(const float2* spec, uint32_t k) {
    const float2 z = __ldg(spec + k);
    return __fadd_rn(__fmul_rn(z.x, z.x), __fmul_rn(z.y, z.y));
}

// Bitonic sorts (ascending) of the B values of one warp, value lane*R + r held in v[r] (R = B/32).
// Pairs closer than R are exchanged inside a lane's registers, farther ones across lanes.
// Two independent sorts, stage by stage, so the latencies of their shuffles overlap.
template <int B>
__device__ __forceinline__ void warp_bitonic2(float (&v)[B / 32], float (&u)[B / 32], uint32_t lane) {
    constexpr int R = B / 32;
#pragma unroll
    for (int k = 2; k <= B; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < R) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int rp = r ^ j;
                    if (rp > r) {
                        const bool up = ((((int)lane * R + r) & k) == 0);
                        const float a = v[r], b = v[rp], c = u[r], d = u[rp];
                        const float lo = fminf(a, b), hi = fmaxf(a, b), lo2 = fminf(c, d), hi2 = fmaxf(c, d);
                        v[r] = up ? lo : hi;
                        v[rp] = up ? hi : lo;
                        u[r] = up ? lo2 : hi2;
                        u[rp] = up ? hi2 : lo2;
                    }
                }
            } else {
                const int jl = j / R;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float o = __shfl_xor_sync(0xffffffffu, v[r], jl);
                    const float o2 = __shfl_xor_sync(0xffffffffu, u[r], jl);
                    const bool up = ((((int)lane * R + r) & k) == 0);
                    const bool lower = ((int)lane & jl) == 0;
                    const bool take_min = lower == up;
                    v[r] = take_min ? fminf(v[r], o) : fmaxf(v[r], o);
                    u[r] = take_min ? fminf(u[r], o2) : fmaxf(u[r], o2);
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

// The powers of block jb (bins lane*R .. lane*R + R-1 of it per lane, R = B/32), padded with +inf.
template <int B>
__device__ __forceinline__ void load_block(const float2* spec, uint32_t N, uint32_t jb, uint32_t lane,
                                           float (&v)[B / 32]) {
    constexpr uint32_t R = B / 32;
    const uint32_t lo = jb * B, size = min((uint32_t)B, N - lo);
    if (R >= 2 && size == (uint32_t)B) {  // a full block: 16-byte loads (lo and lane * R are even and
                                          // the spectrum starts 16-byte aligned)
        const float4* q = reinterpret_cast<const float4*>(spec + lo + lane * R);
#pragma unroll
        for (uint32_t r = 0; r + 1 < R; r += 2) {
            const float4 z = __ldg(q + r / 2);
            v[r] = __fadd_rn(__fmul_rn(z.x, z.x), __fmul_rn(z.y, z.y));
            v[r + 1] = __fadd_rn(__fmul_rn(z.z, z.z), __fmul_rn(z.w, z.w));
        }
    } else {
#pragma unroll
        for (uint32_t r = 0; r < R; ++r) {
            const uint32_t e = lane * R + r;
            v[r] = e < size ? power_of(spec, lo + e) : INFINITY;  // padding sorts to the end
        }
    }
}

// After sorting: the lane holding rank floor((size - 1)/2) writes the block's lower median.
template <int B>
__device__ __forceinline__ void keep_median(float* med, uint32_t N, uint32_t jb, uint32_t lane, const float (&v)[B / 32]) {
    constexpr uint32_t R = B / 32;
    const uint32_t size = min((uint32_t)B, N - jb * B);
    const uint32_t rank = (size - 1u) / 2u;
#pragma unroll
    for (uint32_t r = 0; r < R; ++r)
        if (rank == lane * R + r) med[jb] = v[r];
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
    const uint32_t stride = gridDim.x * warps;
    // two blocks per warp at a time: their loads and sorting networks are independent
    for (uint32_t jb = blockIdx.x * warps + (threadIdx.x >> 5); jb < nblk; jb += 2 * stride) {
        constexpr uint32_t R = B / 32;
        float v[R], u[R];
        const uint32_t jb2 = jb + stride;
        const bool two = jb2 < nblk;  // uniform over the warp
        load_block<B>(spec, N, jb, lane, v);
        if (two) {
            load_block<B>(spec, N, jb2, lane, u);
        } else {
#pragma unroll
            for (uint32_t r = 0; r < R; ++r) u[r] = INFINITY;
        }
        warp_bitonic2<B>(v, u, lane);  // both networks in one straight-line sequence
        keep_median<B>(w.medians + moff, N, jb, lane, v);
        if (two) keep_median<B>(w.medians + moff, N, jb2, lane, u);
    }
}

// x of bin k from its power P and the medians m of its spectrum
template <int B>
__device__ __forceinline__ float pow_norm(const float* m, uint32_t N, uint32_t nblk, uint32_t k, float P) {
    const float ln2 = 0.693147180559945309417232f;
    const float fB = (float)B, hfull = 0.5f * (float)(B - 1);
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
    return base > 0.f ? __fsub_rn(__fdiv_rn(__fmul_rn(P, ln2), base), 1.0f) : 0.f;
}

// Two neighbouring outputs (k even; the spectrum's start is even, so the pair is 4- or 8-byte aligned).
template <typename T>
__device__ __forceinline__ void store_pair(T* out, uint32_t k, float a, float b);
template <>
__device__ __forceinline__ void store_pair<float>(float* out, uint32_t k, float a, float b) {
    *reinterpret_cast<float2*>(out + k) = make_float2(a, b);
}
template <>
__device__ __forceinline__ void store_pair<__half>(__half* out, uint32_t k, float a, float b) {
    *reinterpret_cast<__half2*>(out + k) = __floats2half2_rn(a, b);
}
template <>
__device__ __forceinline__ void store_pair<__nv_bfloat16>(__nv_bfloat16* out, uint32_t k, float a, float b) {
    *reinterpret_cast<__nv_bfloat162*>(out + k) = __floats2bfloat162_rn(a, b);
}
template <typename T>
__device__ __forceinline__ void store_one(T* out, uint32_t k, float x) {
    if constexpr (sizeof(T) == 4)
        out[k] = x;
    else if constexpr (std::is_same<T, __half>::value)
        out[k] = __float2half_rn(x);
    else
        out[k] = __float2bfloat16_rn(x);
}

template <int B>
__device__ __forceinline__ void norm_quad(const float* m, uint32_t N, uint32_t nblk, uint32_t k,
                                          const float4& z0, const float4& z1, float (&x)[4]) {
    x[0] = pow_norm<B>(m, N, nblk, k, __fadd_rn(__fmul_rn(z0.x, z0.x), __fmul_rn(z0.y, z0.y)));
    x[1] = pow_norm<B>(m, N, nblk, k + 1, __fadd_rn(__fmul_rn(z0.z, z0.z), __fmul_rn(z0.w, z0.w)));
    x[2] = pow_norm<B>(m, N, nblk, k + 2, __fadd_rn(__fmul_rn(z1.x, z1.x), __fmul_rn(z1.y, z1.y)));
    x[3] = pow_norm<B>(m, N, nblk, k + 3, __fadd_rn(__fmul_rn(z1.z, z1.z), __fmul_rn(z1.w, z1.w)));
}

// Four consecutive bins per thread: two 16-byte loads of (re, im) pairs, two paired stores.
template <int B, typename T>
__global__ void __launch_bounds__(kPowBlock) k_power_normalize(const PowWork w, T* out) {
    int64_t off, moff;
    uint32_t N;
    if (pow_spectrum(w, blockIdx.y, B, off, N, moff) != 1) return;
    const float2* spec = w.spec + off;
    const float* m = w.medians + moff;
    T* o = out + off;
    const uint32_t nblk = (N + B - 1) / B;
    const uint32_t n4 = N / 4u;
    const uint32_t stride = gridDim.x * kPowBlock;
    for (uint32_t q = blockIdx.x * kPowBlock + threadIdx.x; q < n4; q += 2 * stride) {
        // two quads per iteration, loaded before either is used
        const bool two = q + stride < n4;
        const uint32_t q2 = two ? q + stride : q;  // a second quad, or the first again (not stored)
        const float4* p = reinterpret_cast<const float4*>(spec + 4u * q);
        const float4* p2 = reinterpret_cast<const float4*>(spec + 4u * q2);
        const float4 z0 = __ldg(p), z1 = __ldg(p + 1), y0 = __ldg(p2), y1 = __ldg(p2 + 1);
        float a[4], b[4];
        norm_quad<B>(m, N, nblk, 4u * q, z0, z1, a);
        norm_quad<B>(m, N, nblk, 4u * q2, y0, y1, b);
        store_pair<T>(o, 4u * q, a[0], a[1]);
        store_pair<T>(o, 4u * q + 2, a[2], a[3]);
        if (two) {
            store_pair<T>(o, 4u * q2, b[0], b[1]);
            store_pair<T>(o, 4u * q2 + 2, b[2], b[3]);
        }
    }
    if (blockIdx.x == 0)  // the last N mod 4 bins
        for (uint32_t k = 4u * n4 + threadIdx.x; k < N; k += kPowBlock) store_one<T>(o, k, pow_norm<B>(m, N, nblk, k, power_of(spec, k)));
}

// CTAs per spectrum: enough to cover its blocks, at least four, and about 32 CTAs per SM over the
// whole batch, so that every SM holds its full eight CTAs with work to balance.
inline unsigned ctas_per_spectrum(int64_t units, int64_t per_cta, int n_spectra, int sms) {
    const int64_t need = std::max<int64_t>(1, (units + per_cta - 1) / per_cta);
    return (unsigned)std::min<int64_t>(need, std::max(4, sms * 32 / std::max(1, n_spectra)));
}

template <int B>
cudaError_t launch_block(const PowWork& w, int n_spectra, int64_t longest, int sms, WsControl* ctl, hs_dtype dt,
                         void* out, cudaStream_t s) {
    const unsigned gm = ctas_per_spectrum((longest + B - 1) / B, kPowBlock / 32, n_spectra, sms);
    k_block_median<B><<<dim3(gm, (unsigned)n_spectra), kPowBlock, 0, s>>>(w, ctl);
    const dim3 grid(ctas_per_spectrum((longest + 3) / 4, kPowBlock, n_spectra, sms), (unsigned)n_spectra);
    switch (dt) {
        case HS_F32: k_power_normalize<B, float><<<grid, kPowBlock, 0, s>>>(w, (float*)out); break;
        case HS_F16: k_power_normalize<B, __half><<<grid, kPowBlock, 0, s>>>(w, (__half*)out); break;
        case HS_BF16: k_power_normalize<B, __nv_bfloat16><<<grid, kPowBlock, 0, s>>>(w, (__nv_bfloat16*)out); break;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_power_normalize(const float* spec, const int64_t* offsets, int n_spectra, int64_t n_bins, int block,
                                   float* medians, long long med_cap, hs_dtype dt, void* out, int64_t max_bins,
                                   int sm_count, int64_t* prefix, WsControl* ctl, cudaStream_t s) {
    PowWork w{reinterpret_cast<const float2*>(spec), offsets, prefix, n_bins, medians, med_cap};
    if (offsets) launch_tile_scan(offsets, n_spectra, block, max_bins, 8, prefix, ctl, s);
    const int64_t longest = offsets ? max_bins : n_bins;
    switch (block) {
        case 32: return launch_block<32>(w, n_spectra, longest, sm_count, ctl, dt, out, s);
        case 64: return launch_block<64>(w, n_spectra, longest, sm_count, ctl, dt, out, s);
        case 128: return launch_block<128>(w, n_spectra, longest, sm_count, ctl, dt, out, s);
        case 256: return launch_block<256>(w, n_spectra, longest, sm_count, ctl, dt, out, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace hs

// Adjoint of the per-bin best snr: a scatter-add transpose of the forward gather, routed through
// the saved best H of every bin (and, for Eq. 4, the saved left/right choices; for Eq. 2 the
// window's first maximum, recomputed from the spectrum; the window starts at j0 = 1 as written, or
// at j0 = 0 under HS_FLAG_MAX_WINDOW0; under HS_FLAG_GREEDY_FIXED1 harmonic 1 reads bin n).
//   grad_x[m] += g[n] * c_H* * isig_H*   for every term of S_H*(n) that reads bin m.
#include "hs_common.cuh"

namespace hs {

constexpr int kAdjBlock = 256;

template <int V, typename T>
__global__ void __launch_bounds__(kAdjBlock) k_backward(const __grid_constant__ Tables tb, const T* x,
                                                        const int64_t* offsets, int64_t n_bins, int hmax, uint32_t flags,
                                                        const float* g, const uint8_t* best_h, const uint32_t* path,
                                                        float* grad) {
    const int s = blockIdx.y;
    const int64_t off = offsets ? offsets[s] : 0;
    const uint32_t N = (uint32_t)(offsets ? offsets[s + 1] - off : n_bins);
    const T* xs = x + off;
    float* gs = grad + off;
    for (uint32_t n = blockIdx.x * kAdjBlock + threadIdx.x; n < N; n += gridDim.x * kAdjBlock) {
        const int Hs = best_h[off + n];
        const float gn = g[off + n];
        // a best H the bin cannot have (corrupt routing) is skipped rather than read out of range
        const bool fixed1 = V == HS_GREEDY && (flags & HS_FLAG_GREEDY_FIXED1) != 0;
        const uint32_t j0 = (flags & HS_FLAG_MAX_WINDOW0) ? 0u : 1u;
        int hv = hmax;
        if (V == HS_MAX || V == HS_GREEDY) hv = (int)min((uint32_t)hmax, (fixed1 ? N : N - 1) / (n + 1));
        if (V == HS_FBIN && n > 0) hv = (int)min((uint32_t)hmax, (N - 1) / n);
        if (Hs == 0 || Hs > hv || gn == 0.f) continue;
        const float wgt = __fmul_rn(__fmul_rn(gn, tb.c[Hs]), tb.isig[Hs]);
        uint32_t p = (V == HS_GREEDY) ? path[off + n] : 0u;
        uint32_t j = 0;
        for (int i = 1; i <= Hs; ++i) {
            uint32_t m;
            if (V == HS_STD) {
                m = (2u * n * (uint32_t)i + (uint32_t)Hs) / (2u * (uint32_t)Hs);
            } else if (V == HS_FBIN) {
                m = (uint32_t)i * n;
            } else if (V == HS_MAX) {
                uint32_t base = (uint32_t)i * n;
                m = base + j0;
                float mv = ldx(xs, m);
                for (int jj = (int)j0 + 1; jj <= i; ++jj) {
                    float v = ldx(xs, base + jj);
                    if (v > mv) {
                        mv = v;
                        m = base + jj;
                    }
                }
            } else if (fixed1 && i == 1) {
                m = n;  // the fixed first term
            } else {
                j += (p >> (i - 1)) & 1u;
                m = (uint32_t)i * n + j;
            }
            atomicAdd(gs + m, wgt);
        }
    }
}

template <int V>
static cudaError_t launch_v(hs_dtype dt, const Tables& tab, const void* x, const int64_t* offsets, int n_spectra,
                            int64_t n_bins, int hmax, uint32_t flags, const float* g, const uint8_t* bh, const uint32_t* path,
                            float* grad, cudaStream_t s) {
    unsigned gx = (unsigned)std::min<int64_t>((n_bins + kAdjBlock - 1) / kAdjBlock, 2048);
    if (gx == 0) return cudaSuccess;
    dim3 grid(gx, (unsigned)n_spectra);
    switch (dt) {
        case HS_F32:
            k_backward<V, float><<<grid, kAdjBlock, 0, s>>>(tab, (const float*)x, offsets, n_bins, hmax, flags, g, bh, path, grad);
            break;
        case HS_F16:
            k_backward<V, __half><<<grid, kAdjBlock, 0, s>>>(tab, (const __half*)x, offsets, n_bins, hmax, flags, g, bh, path, grad);
            break;
        case HS_BF16:
            k_backward<V, __nv_bfloat16>
                <<<grid, kAdjBlock, 0, s>>>(tab, (const __nv_bfloat16*)x, offsets, n_bins, hmax, flags, g, bh, path, grad);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_backward(hs_variant v, hs_dtype dt, const Tables& tab, const void* x, const int64_t* offsets,
                            int n_spectra, int64_t n_bins, int hmax, int flags, const float* g, const uint8_t* best_h,
                            const uint32_t* path, float* grad, cudaStream_t s) {
    switch (v) {
        case HS_STD: return launch_v<HS_STD>(dt, tab, x, offsets, n_spectra, n_bins, hmax, (uint32_t)flags, g, best_h, path, grad, s);
        case HS_MAX: return launch_v<HS_MAX>(dt, tab, x, offsets, n_spectra, n_bins, hmax, (uint32_t)flags, g, best_h, path, grad, s);
        case HS_FBIN: return launch_v<HS_FBIN>(dt, tab, x, offsets, n_spectra, n_bins, hmax, (uint32_t)flags, g, best_h, path, grad, s);
        case HS_GREEDY:
            return launch_v<HS_GREEDY>(dt, tab, x, offsets, n_spectra, n_bins, hmax, (uint32_t)flags, g, best_h, path, grad, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace hs

// 2-D harmonic sum over an FDAS plane: Eq. 1 applied to the frequency bin n and the drift row z,
//   h(n, z)_H = H^-1/2 sum_{i=1..H} x(round(n*i/H), round(z*i/H)),  rounded half up, H = 1..16.
// A CTA owns 32 consecutive bins and every row; warp g walks rows g, g+8, ...  Each cell's best
// (snr, H) is written, and the per-bin best over rows is reduced in shared memory in row order.
#include "hs_common.cuh"

namespace hs {

constexpr int k2dBins = 32;    // bins per CTA
constexpr int k2dGroups = 8;   // warps per CTA, each a set of rows

// floor((2*z*i + H) / (2*H)) with a compile-time denominator and any sign of z.
template <int H, int I>
__device__ __forceinline__ int zround(int z) {
    int a = 2 * z * I + H;
    return a >= 0 ? a / (2 * H) : -((-a + 2 * H - 1) / (2 * H));
}

template <int H, int I>
struct Term2d {
    static __device__ __forceinline__ float sum(const float* plane, int64_t stride, int z, int z_min, uint32_t n) {
        uint32_t ni = (2u * n * (uint32_t)I + (uint32_t)H) / (2u * (uint32_t)H);
        int zi = zround<H, I>(z);
        float v = __ldg(plane + (int64_t)(zi - z_min) * stride + ni);
        return __fadd_rn(Term2d<H, I - 1>::sum(plane, stride, z, z_min, n), v);
    }
};
template <int H>
struct Term2d<H, 0> {
    static __device__ __forceinline__ float sum(const float*, int64_t, int, int, uint32_t) { return 0.f; }
};

template <int H>
__device__ __forceinline__ void cell_h(const float* plane, int64_t stride, int z, int z_min, uint32_t n, int hmax,
                                       const Tables& tb, float& best, int& bh) {
    if (H <= hmax) {
        float S = Term2d<H, H>::sum(plane, stride, z, z_min, n);  // terms added in order i = 1..H
        keep_best(calibrate(tb, S, H), H, best, bh);
    }
}

template <int... Hs>
struct CellAll;
template <int H, int... Rest>
struct CellAll<H, Rest...> {
    static __device__ __forceinline__ void run(const float* p, int64_t st, int z, int zm, uint32_t n, int hmax,
                                               const Tables& tb, float& best, int& bh) {
        cell_h<H>(p, st, z, zm, n, hmax, tb, best, bh);
        CellAll<Rest...>::run(p, st, z, zm, n, hmax, tb, best, bh);
    }
};
template <>
struct CellAll<> {
    static __device__ __forceinline__ void run(const float*, int64_t, int, int, uint32_t, int, const Tables&, float&,
                                               int&) {}
};

__global__ void __launch_bounds__(k2dBins* k2dGroups) k_hs2d(const __grid_constant__ Tables tb, const Work2d w,
                                                            const hs_out2d o, long long cand_cap, WsControl* ctl) {
    __shared__ float s_snr[k2dGroups][k2dBins];
    __shared__ int s_row[k2dGroups][k2dBins];
    __shared__ int s_h[k2dGroups][k2dBins];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const uint32_t n = blockIdx.x * k2dBins + lane;
    const bool active = n < (uint32_t)w.n_bins;
    float rbest = -INFINITY;
    int rrow = 0, rh = 0;
    for (int r = g; r < w.nz; r += k2dGroups) {
        const int z = w.z_min + r;
        float best = -INFINITY;
        int bh = 0;
        if (active) {
            CellAll<1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16>::run(w.plane, w.row_stride, z, w.z_min, n,
                                                                                 w.hmax, tb, best, bh);
            size_t cell = (size_t)r * (size_t)w.n_bins + n;
            o.best_snr[cell] = best;
            o.best_h[cell] = (uint8_t)bh;
            if (best > rbest) {  // rows visited in increasing order: the lowest row keeps ties
                rbest = best;
                rrow = r;
                rh = bh;
            }
        }
        if (o.cand)
            append_candidate(active && best > w.threshold, o.cand, o.cand_count, cand_cap, &ctl->status, w.plane_id,
                             n, best, z, bh, HS_STD);
    }
    s_snr[g][lane] = rbest;
    s_row[g][lane] = rbest == -INFINITY ? 0x7fffffff : rrow;
    s_h[g][lane] = rh;
    __syncthreads();
    if (g == 0 && active) {
        float b = s_snr[0][lane];
        int br = s_row[0][lane], bhh = s_h[0][lane];
        for (int k = 1; k < k2dGroups; ++k) {
            float v = s_snr[k][lane];
            int rr = s_row[k][lane];
            if (v > b || (v == b && rr < br)) {
                b = v;
                br = rr;
                bhh = s_h[k][lane];
            }
        }
        o.best_snr_n[n] = b;
        o.best_h_n[n] = (uint8_t)bhh;
        o.best_z_n[n] = (int16_t)(w.z_min + (br == 0x7fffffff ? 0 : br));
    }
}

cudaError_t launch_2d(const Tables& tab, const Work2d& w, const hs_out2d& o, long long cand_cap, WsControl* ctl,
                      cudaStream_t s) {
    if (w.n_bins == 0) return cudaSuccess;
    unsigned grid = (unsigned)((w.n_bins + k2dBins - 1) / k2dBins);
    k_hs2d<<<grid, k2dBins * k2dGroups, 0, s>>>(tab, w, o, cand_cap, ctl);
    return cudaGetLastError();
}

}  // namespace hs

// 2-D harmonic sum over an FDAS plane: Eq. 1 applied to the frequency bin n and the drift row z,
//   h(n, z)_H = H^-1/2 sum_{i=1..H} x(round(n*i/H), round(z*i/H)),  rounded half up, H = 1..16.
// A CTA owns 32 consecutive bins and every row; warp g walks rows g, g+8, ...  Each cell's best
// (snr, H) is written, and the per-bin best over rows is reduced in shared memory in row order.
#include <utility>

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

__global__ void __launch_bounds__(k2dBins * k2dGroups, 2) k_hs2d(const __grid_constant__ Tables tb, const Work2d w,
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

// ------------------------------------------------------------------------------------------
// H = 1..16 fast path.  Both rounded indices of harmonic i of H depend only on the reduced fraction
// i/H, so each of the 80 fractions of F_16 is read once per cell and added to every S_H it serves,
// visiting fractions in increasing order (which keeps each S_H's terms in the order i = 1..H).  A
// warp walks one row at a time, so the row index round(z*p/q) is the same for all its lanes; each
// lane owns two neighbouring bins n, n+1, whose column indices differ by the carry of the
// fixed-point low word (as in the 1-D Eq. 1 kernel).
// ------------------------------------------------------------------------------------------
struct Frac16 {
    int p, q;
};
__host__ __device__ constexpr Frac16 farey16_at(int k) {  // k-th term of F_16 after 0/1: 1/16 .. 1/1
    Frac16 a{0, 1}, b{1, 16};
    for (int i = 0; i < k; ++i) {
        int m = (16 + a.q) / b.q;
        Frac16 c{m * b.p - a.p, m * b.q - a.q};
        a = b;
        b = c;
    }
    return b;
}
constexpr int kNumFrac16 = 80;
static_assert(farey16_at(kNumFrac16 - 1).p == 1 && farey16_at(kNumFrac16 - 1).q == 1, "F_16 has 80 terms after 0/1");

constexpr int k2dPairBins = 64;  // bins per CTA on the fast path (32 lanes x 2)



// The row of fraction p/q at drift z, round-half-up(z*p/q) = floor((2zp + q) / (2q)) for any sign of z,
// in unsigned arithmetic: with a = 2zp + 65537q (= 2zp + q + 2q*32768, positive for |z| <= 32767 and
// below 2^21), floor(a / 2q) = umulhi(a, ceil(2^32 / 2q)) exactly (the error a / 2^32 stays below
// 1/(2q)), and the row is that minus 32768.  Its element offset in the plane is
// umulhi(...) * stride + base, base = -(32768 + z_min) * stride (the plane holds fewer than 2^32
// elements, so the offset is exact modulo 2^32).
template <int P, int Q>
__device__ __forceinline__ uint32_t row_offset16(int z, uint32_t stride, uint32_t base) {
    constexpr uint32_t R = (uint32_t)(((1ull << 32) + 2 * Q - 1) / (2 * Q));
    const uint32_t a = (uint32_t)(z * (2 * P) + 65537 * Q);
    return __umulhi(a, R) * stride + base;
}

// n even and n+1 < row length, so both reads of every fraction stay inside the row (k(n) + 1 <= n + 1).
template <int K>
__device__ __forceinline__ void farey16_pair_step(const float* plane, int z, uint32_t stride, uint32_t base, uint32_t n,
                                                  float2 (&S)[HS_HMAX_2D + 1]) {
    constexpr Frac16 f = farey16_at(K);
    const uint32_t roff = row_offset16<f.p, f.q>(z, stride, base);
    // the second read goes through the pointer (p + 1), so it shares the first read's address
    float2 v;
    if (f.q == 1) {
        const float* p = plane + (roff + n);
        v.x = __ldg(p);
        v.y = __ldg(p + 1);
    } else {
        constexpr uint32_t F = (uint32_t)((((uint64_t)f.p << 32) + f.q - 1) / f.q);
        const uint32_t lo = n * F;
        const uint32_t k = __umulhi(n, F) + (lo >> 31);
        const float* p = plane + (roff + k);
        const float a = __ldg(p), b = __ldg(p + 1);
        v.x = a;
        v.y = ((int32_t)lo > (int32_t)(~F ^ 0x80000000u)) ? b : a;  // (lo + 2^31) >u ~F as a signed compare
    }
#pragma unroll
    for (int m = 1; m * f.q <= HS_HMAX_2D; ++m) S[m * f.q] = add2(S[m * f.q], v);
}

template <int... K>
__device__ __forceinline__ void farey16_pair_all(const float* plane, int z, uint32_t stride, uint32_t base, uint32_t n,
                                                 float2 (&S)[HS_HMAX_2D + 1], std::integer_sequence<int, K...>) {
    (farey16_pair_step<K>(plane, z, stride, base, n, S), ...);
}

// Four CTAs per SM (64 registers, some spilled) measured 3% faster than two (128 registers, none
// spilled); three (80 registers, none spilled) measured 40% slower.
__global__ void __launch_bounds__(k2dGroups * 32, 4) k_hs2d_pairs(const __grid_constant__ Tables tb, const Work2d w,
                                                               const hs_out2d o, long long cand_cap, WsControl* ctl) {
    __shared__ float s_snr[k2dGroups][k2dPairBins];
    __shared__ int s_row[k2dGroups][k2dPairBins];
    __shared__ int s_h[k2dGroups][k2dPairBins];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const uint32_t nb = (uint32_t)w.n_bins;  // even and >= 2 on this path
    const uint32_t n = blockIdx.x * k2dPairBins + 2 * lane;  // this lane's bins n and n+1
    const bool act0 = n < nb, act1 = n + 1 < nb;
    const uint32_t nq = act0 ? n : nb - 2;  // idle lanes evaluate the last pair of the row
    const uint32_t stride = (uint32_t)w.row_stride;
    const uint32_t base = (uint32_t)(-(32768 + w.z_min)) * stride;
    float rb[2] = {-INFINITY, -INFINITY};
    int rr[2] = {0x7fffffff, 0x7fffffff}, rh[2] = {0, 0};
    for (int r = g; r < w.nz; r += k2dGroups) {
        const int z = w.z_min + r;
        float2 S[HS_HMAX_2D + 1];
#pragma unroll
        for (int H = 0; H <= HS_HMAX_2D; ++H) S[H] = make_float2(0.f, 0.f);
        farey16_pair_all(w.plane, z, stride, base, nq, S, std::make_integer_sequence<int, kNumFrac16>{});
        float b0 = -INFINITY, b1 = -INFINITY;
        int h0 = 0, h1 = 0;
#pragma unroll
        for (int H = 1; H <= HS_HMAX_2D; ++H) {
            keep_best(calibrate(tb, S[H].x, H), H, b0, h0);
            keep_best(calibrate(tb, S[H].y, H), H, b1, h1);
        }
        const size_t cell = (size_t)r * nb + n;
        if (act1) {
            *reinterpret_cast<float2*>(o.best_snr + cell) = make_float2(b0, b1);
            o.best_h[cell] = (uint8_t)h0;
            o.best_h[cell + 1] = (uint8_t)h1;
        } else if (act0) {
            o.best_snr[cell] = b0;
            o.best_h[cell] = (uint8_t)h0;
        }
        if (act0 && b0 > rb[0]) {  // rows visited in increasing order: the lowest row keeps ties
            rb[0] = b0;
            rr[0] = r;
            rh[0] = h0;
        }
        if (act1 && b1 > rb[1]) {
            rb[1] = b1;
            rr[1] = r;
            rh[1] = h1;
        }
        if (o.cand) {
            append_candidate(act0 && b0 > w.threshold, o.cand, o.cand_count, cand_cap, &ctl->status, w.plane_id, n,
                             b0, z, h0, HS_STD);
            append_candidate(act1 && b1 > w.threshold, o.cand, o.cand_count, cand_cap, &ctl->status, w.plane_id,
                             n + 1, b1, z, h1, HS_STD);
        }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        s_snr[g][2 * lane + k] = rb[k];
        s_row[g][2 * lane + k] = rr[k];
        s_h[g][2 * lane + k] = rh[k];
    }
    __syncthreads();
    if (threadIdx.x < k2dPairBins) {
        const int c = threadIdx.x;
        const uint32_t nn = blockIdx.x * k2dPairBins + c;
        if (nn < nb) {
            float b = s_snr[0][c];
            int br = s_row[0][c], bh = s_h[0][c];
            for (int k = 1; k < k2dGroups; ++k) {
                const float v = s_snr[k][c];
                const int rw = s_row[k][c];
                if (v > b || (v == b && rw < br)) {
                    b = v;
                    br = rw;
                    bh = s_h[k][c];
                }
            }
            o.best_snr_n[nn] = b;
            o.best_h_n[nn] = (uint8_t)bh;
            o.best_z_n[nn] = (int16_t)(w.z_min + (br == 0x7fffffff ? 0 : br));
        }
    }
}

// ------------------------------------------------------------------------------------------
// Row-wise 2-D forms of Eq. 2-4: harmonic i of the cell (n, z) lies on the row i*z and is taken there
// exactly as the 1-D equation takes it: Eq. 3 x(i n, i z); Eq. 2 the largest of x(i n + j0 .. i n + i,
// i z) (j0 = 1, or 0 under HS_FLAG_MAX_WINDOW0); Eq. 4 the choice between x(i n + j, i z) and
// x(i n + j + 1, i z), the right one only when strictly larger, j carried from harmonic to harmonic
// (HS_FLAG_GREEDY_FIXED1: the first term is x(n, z)).  Terms are a running sum in the order i = 1..H.
// H is valid while the 1-D rule holds for n (Eq. 3: H n <= N-1, every H at n = 0; Eq. 2 and 4:
// H (n+1) <= N-1, or <= N under the fixed first term) and H z stays within the plane's rows.  The
// paper writes Eq. 2-4 in 1-D only; taking the drift of harmonic i as i z follows the 2-D form of
// Eq. 1.  Same CTA layout and per-bin reduction as k_hs2d.
// ------------------------------------------------------------------------------------------
template <int V>
__device__ __forceinline__ float rowwise_term(const float* row, uint32_t n, int i, uint32_t& j, int flags) {
    const uint32_t base = (uint32_t)i * n;
    if (V == HS_FBIN) return __ldg(row + base);
    if (V == HS_MAX) {
        const int j0 = (flags & HS_FLAG_MAX_WINDOW0) ? 0 : 1;
        float m = __ldg(row + base + j0);
        for (int jj = j0 + 1; jj <= i; ++jj) m = fmaxf(m, __ldg(row + base + jj));
        return m;
    }
    if ((flags & HS_FLAG_GREEDY_FIXED1) && i == 1) return __ldg(row + n);
    const float l = __ldg(row + base + j), r = __ldg(row + base + j + 1);
    if (r > l) {
        ++j;
        return r;
    }
    return l;
}

template <int V>
__global__ void __launch_bounds__(k2dBins * k2dGroups) k_hs2d_rowwise(const __grid_constant__ Tables tb, const Work2d w,
                                                                     const hs_out2d o, long long cand_cap,
                                                                     WsControl* ctl) {
    __shared__ float s_snr[k2dGroups][k2dBins];
    __shared__ int s_row[k2dGroups][k2dBins];
    __shared__ int s_h[k2dGroups][k2dBins];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const uint32_t n = blockIdx.x * k2dBins + lane;
    const uint32_t N = (uint32_t)w.n_bins;
    const bool active = n < N;
    const int z_max = w.z_min + w.nz - 1;
    // valid H from the bin alone (the 1-D rule)
    int hn = w.hmax;
    if (active) {
        if (V == HS_FBIN) {
            if (n > 0) hn = min(hn, (int)((N - 1) / n));
        } else {
            const uint32_t L = (V == HS_GREEDY && (w.flags & HS_FLAG_GREEDY_FIXED1)) ? N : N - 1;
            hn = min(hn, (int)(L / (n + 1)));
        }
    }
    float rbest = -INFINITY;
    int rrow = 0, rh = 0;
    for (int r = g; r < w.nz; r += k2dGroups) {
        const int z = w.z_min + r;
        float best = -INFINITY;
        int bh = 0;
        if (active) {
            int hv = hn;
            if (z > 0) hv = min(hv, z_max / z);
            if (z < 0) hv = min(hv, w.z_min / z);  // both negative: the quotient floors towards zero
            float S = 0.f;
            uint32_t j = 0;
            for (int i = 1; i <= hv; ++i) {
                const float* row = w.plane + (int64_t)(i * z - w.z_min) * w.row_stride;
                S = __fadd_rn(S, rowwise_term<V>(row, n, i, j, w.flags));
                keep_best(calibrate(tb, S, i), i, best, bh);
            }
            const size_t cell = (size_t)r * (size_t)w.n_bins + n;
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
                             n, best, z, bh, V);
    }
    s_snr[g][lane] = rbest;
    s_row[g][lane] = rbest == -INFINITY ? 0x7fffffff : rrow;
    s_h[g][lane] = rh;
    __syncthreads();
    if (g == 0 && active) {
        float b = s_snr[0][lane];
        int br = s_row[0][lane], bhh = s_h[0][lane];
        for (int k = 1; k < k2dGroups; ++k) {
            const float v = s_snr[k][lane];
            const int rr = s_row[k][lane];
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

cudaError_t launch_2d(hs_variant v, const Tables& tab, const Work2d& w, const hs_out2d& o, long long cand_cap,
                      WsControl* ctl, cudaStream_t s) {
    if (w.n_bins == 0) return cudaSuccess;
    if (v != HS_STD) {
        const unsigned grid = (unsigned)((w.n_bins + k2dBins - 1) / k2dBins);
        if (v == HS_FBIN) k_hs2d_rowwise<HS_FBIN><<<grid, k2dBins * k2dGroups, 0, s>>>(tab, w, o, cand_cap, ctl);
        if (v == HS_MAX) k_hs2d_rowwise<HS_MAX><<<grid, k2dBins * k2dGroups, 0, s>>>(tab, w, o, cand_cap, ctl);
        if (v == HS_GREEDY) k_hs2d_rowwise<HS_GREEDY><<<grid, k2dBins * k2dGroups, 0, s>>>(tab, w, o, cand_cap, ctl);
        return cudaGetLastError();
    }
    // float2 stores of the cell pair (n, n+1) need an even row length and an 8-byte aligned output
    const bool cells_aligned = (w.n_bins % 2) == 0 && (reinterpret_cast<uintptr_t>(o.best_snr) & 7) == 0;
    const bool small_plane = (uint64_t)w.nz * (uint64_t)w.row_stride < (1ull << 32);
    if (w.hmax == HS_HMAX_2D && cells_aligned && small_plane) {
        unsigned grid = (unsigned)((w.n_bins + k2dPairBins - 1) / k2dPairBins);
        k_hs2d_pairs<<<grid, k2dGroups * 32, 0, s>>>(tab, w, o, cand_cap, ctl);
    } else {
        unsigned grid = (unsigned)((w.n_bins + k2dBins - 1) / k2dBins);
        k_hs2d<<<grid, k2dBins * k2dGroups, 0, s>>>(tab, w, o, cand_cap, ctl);
    }
    return cudaGetLastError();
}

}  // namespace hs

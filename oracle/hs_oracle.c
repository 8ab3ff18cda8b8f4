/*
 * CPU oracle for the incoherent harmonic sum of Adamek & Armour, "A GPU implementation of the
 * harmonic sum algorithm" (arXiv:1812.02647).
 *
 * TEST INFRASTRUCTURE.  Plain, slow, obviously correct C: a direct evaluation of Eq. 1-4 for
 * every output bin, in two modes (FP64, and FP32 with every operation rounded in the written
 * order; build with -ffp-contract=off and no fast-math).  Only the tests, the package smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code with the GPU
 * library and includes none of its headers.
 *
 * Range reading (the paper gives none): harmonics are truncated, never zero-padded.  The number
 * of valid harmonics at output bin n of an N-bin spectrum is the largest H <= hmax whose reads
 * all lie in [0, N):
 *     Eq. 1 (STD)            always hmax (every index is <= n)
 *     Eq. 2, 4 (MAX, MAX0, GREEDY) H*(n+1) <= N-1   (the furthest read is H*n+H)
 *     GREEDY1                    H*(n+1) <= N     (the furthest read is H*n+H-1: j <= H-2)
 *     Eq. 3 (FBIN)           H*n <= N-1        (n = 0 reads x(0) for every H)
 * A bin with no valid H gets snr = -inf and H = 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define HS_O_STD 1
#define HS_O_MAX 2
#define HS_O_FBIN 4
#define HS_O_GREEDY 8
#define HS_O_MAX0 16 /* Eq. 2 with the window j = 0..i (a variant flag; the paper writes j = 1..i) */
#define HS_O_GREEDY1 32 /* Eq. 4 with the first term fixed at x(n) and the first pair at 2n (a variant flag) */
#define HS_O_POW2 64 /* flag bit OR'ed into a variant: only H = 1, 2, 4, .. are stages of the search */
#define HS_O_HMAX 32

int hs_oracle_hvalid(int variant, int64_t n, int64_t N, int hmax) {
    variant &= ~HS_O_POW2;
    if (variant == HS_O_STD) return hmax;
    int64_t lim;
    if (variant == HS_O_FBIN) {
        if (n == 0) return N >= 1 ? hmax : 0;
        lim = (N - 1) / n; /* H*n <= N-1 */
    } else if (variant == HS_O_GREEDY1) {
        lim = N / (n + 1); /* H*(n+1) <= N */
        if (N < 1) lim = 0;
    } else {
        lim = (N - 1) / (n + 1); /* H*(n+1) <= N-1 */
        if (N < 1) lim = 0;
    }
    return lim < hmax ? (int)lim : hmax;
}

/* Eq. 1 index: n*i/H rounded half up, in exact integer arithmetic. */
static inline int64_t hs_oracle_eq1_index(int64_t n, int i, int H) {
    return (2 * n * (int64_t)i + H) / (2 * (int64_t)H);
}

/* floor(a / b) for b > 0 and any sign of a. */
static inline int64_t hs_oracle_floor_div(int64_t a, int64_t b) {
    int64_t q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

#define REAL float
#define SFX f32
#include "hs_oracle_body.h"
#undef REAL
#undef SFX

#define REAL double
#define SFX f64
#include "hs_oracle_body.h"
#undef REAL
#undef SFX

/*
 * Adjoint of the per-bin best snr with respect to the spectrum, in FP64.
 * best_snr(n) = (S_{H*}(n) * c_{H*} - mu) * isig with H* = best_h[n] held fixed, and S a sum of
 * single bins, so d best_snr(n) / d x(m) = c_{H*} * isig_{H*} * (number of terms of S_{H*}(n)
 * that read bin m).  The read bins are those of Eq. 1-4 above; for Eq. 2 the bin of each window
 * maximum (first maximum), for Eq. 4 the bin the recursion chose.  Both are recomputed here from
 * x.  grad_x is accumulated into (the caller zeroes it).
 */
void hs_oracle_grad_f64(int variant, const double* x, int64_t N, int hmax, const double* isig_in,
                        const double* g, const uint8_t* best_h, double* grad_x) {
    variant &= ~HS_O_POW2; /* the routing is the saved best H either way */
    for (int64_t n = 0; n < N; ++n) {
        int Hs = best_h[n];
        if (Hs <= 0 || Hs > hmax || g[n] == 0.0) continue;
        double isig = isig_in ? isig_in[Hs] : 1.0;
        double w = g[n] * (1.0 / sqrt((double)Hs)) * isig;
        int64_t j = 0;
        for (int i = 1; i <= Hs; ++i) {
            int64_t m;
            if (variant == HS_O_STD) {
                m = hs_oracle_eq1_index(n, i, Hs);
            } else if (variant == HS_O_FBIN) {
                m = (int64_t)i * n;
            } else if (variant == HS_O_MAX || variant == HS_O_MAX0) {
                int64_t base = (int64_t)i * n;
                int j0 = variant == HS_O_MAX0 ? 0 : 1;
                m = base + j0;
                for (int jj = j0 + 1; jj <= i; ++jj)
                    if (x[base + jj] > x[m]) m = base + jj;
            } else if (variant == HS_O_GREEDY1 && i == 1) {
                m = n; /* the fixed first term */
            } else {
                int64_t base = (int64_t)i * n + j;
                if (x[base + 1] > x[base]) {
                    m = base + 1;
                    j += 1;
                } else {
                    m = base;
                }
            }
            grad_x[m] += w;
        }
    }
}

/*
 * Standardise and store at reduced precision: y = (p - mu) / sigma in FP32 (IEEE division),
 * then rounded to nearest-even FP16 (dtype 1) or BF16 (dtype 2).  The conversions are written
 * out from the IEEE 754 binary16 / bfloat16 formats.
 */
static uint16_t f32_to_f16_rne(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    uint32_t sign = (u >> 16) & 0x8000u, a = u & 0x7FFFFFFFu;
    if (a > 0x7F800000u) return (uint16_t)(sign | 0x7E00u);  /* NaN */
    if (a >= 0x477FF000u) return (uint16_t)(sign | 0x7C00u); /* >= 65520 rounds to infinity */
    if (a < 0x38800000u) {                                   /* below 2^-14: binary16 subnormal */
        int e = (int)(a >> 23);
        int shift = 126 - e; /* value = m * 2^(e-150) = (m >> shift) units of 2^-24 */
        if (e == 0 || shift > 24) return (uint16_t)sign;
        uint32_t m = (a & 0x7FFFFFu) | 0x800000u;
        uint32_t q = m >> shift, rem = m & ((1u << shift) - 1u), half = 1u << (shift - 1);
        if (rem > half || (rem == half && (q & 1u))) q += 1;
        return (uint16_t)(sign | q);
    }
    uint32_t r = a - 0x38000000u; /* exponent bias 127 -> 15 */
    uint32_t h = (r + 0x0FFFu + ((r >> 13) & 1u)) >> 13;
    return (uint16_t)(sign | h);
}

static uint16_t f32_to_bf16_rne(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7FFFFFFFu) > 0x7F800000u) return (uint16_t)((u >> 16) | 0x40u);
    return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

void hs_oracle_standardize_cast(const float* p, int64_t n, float mu, float sigma, int dtype, uint16_t* out) {
    for (int64_t k = 0; k < n; ++k) {
        float y = (p[k] - mu) / sigma;
        out[k] = (dtype == 1) ? f32_to_f16_rne(y) : f32_to_bf16_rne(y);
    }
}

/*
 * The step before the harmonic sum (the sums of Section 2 run on a power spectrum): the power of a
 * complex spectrum, divided by a running estimate of its local mean, standardised, and stored as
 * FP32 (dtype 0), FP16 (1) or BF16 (2).  Reading (the paper does not describe its normalisation):
 * block medians, robust to the pulsar's own harmonics, as in PRESTO-style dereddening.
 *   P_k = re_k re_k + im_k im_k                             FP32, each operation rounded
 *   m_j = the lower median of P over block j = [jB, min(N, jB + B)): rank floor((size_j - 1)/2)
 *   Exp-distributed power has mean median / ln 2; between block centres c_j = jB + h_j,
 *   h_j = (size_j - 1)/2, the median is interpolated linearly.  For bin k in block j, d = k - jB:
 *     d >= h_j, j + 1 < J:  t = (d - h_j) / (B - h_j + h_{j+1}),      a = m_j,     b = m_{j+1}
 *     d <  h_j, j > 0:      t = (d + B - h_{j-1}) / (B - h_{j-1} + h_j), a = m_{j-1}, b = m_j
 *     otherwise (before the first centre, after the last): base = m_j
 *     base = a + t (b - a)
 *   x_k = (P_k ln2) / base - 1, and 0 where base <= 0 (a block with no power).
 * medians (optional) receives m_j, j = 0..ceil(N/B)-1.
 */
static int hs_oracle_cmp_float(const void* a, const void* b) {
    float x = *(const float*)a, y = *(const float*)b;
    return (x > y) - (x < y);
}

void hs_oracle_power_normalize(const float* spec, int64_t n, int block, int dtype, void* out, float* medians) {
    const float ln2 = 0.693147180559945309417232f;
    int64_t nblk = (n + block - 1) / block;
    float* P = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    float* m = (float*)malloc(sizeof(float) * (size_t)(nblk > 0 ? nblk : 1));
    float* tmp = (float*)malloc(sizeof(float) * (size_t)block);
    for (int64_t k = 0; k < n; ++k) {
        float re = spec[2 * k], im = spec[2 * k + 1];
        float a = re * re;
        float b = im * im;
        P[k] = a + b;
    }
    for (int64_t j = 0; j < nblk; ++j) {
        int64_t lo = j * block, size = (n - lo < block) ? n - lo : block;
        memcpy(tmp, P + lo, sizeof(float) * (size_t)size);
        qsort(tmp, (size_t)size, sizeof(float), hs_oracle_cmp_float);
        m[j] = tmp[(size - 1) / 2];
        if (medians) medians[j] = m[j];
    }
    for (int64_t k = 0; k < n; ++k) {
        int64_t j = k / block;
        float d = (float)(k - j * block);
        int64_t size_j = (n - j * block < block) ? n - j * block : block;
        float hj = 0.5f * (float)(size_j - 1);
        float base;
        if (d >= hj && j + 1 < nblk) {
            int64_t size_n = (n - (j + 1) * block < block) ? n - (j + 1) * block : block;
            float hn = 0.5f * (float)(size_n - 1);
            float t = (d - hj) / ((float)block - hj + hn);
            base = m[j] + t * (m[j + 1] - m[j]);
        } else if (d < hj && j > 0) {
            float hp = 0.5f * (float)(block - 1); /* block j-1 is full */
            float t = (d + (float)block - hp) / ((float)block - hp + hj);
            base = m[j - 1] + t * (m[j] - m[j - 1]);
        } else {
            base = m[j];
        }
        float x = base > 0.0f ? (P[k] * ln2) / base - 1.0f : 0.0f;
        if (dtype == 0)
            ((float*)out)[k] = x;
        else
            ((uint16_t*)out)[k] = dtype == 1 ? f32_to_f16_rne(x) : f32_to_bf16_rne(x);
    }
    free(P);
    free(m);
    free(tmp);
}

/*
 * Mean and standard deviation of h_H for standardised exponential noise (x = p - 1, p ~ Exp(1)),
 * at bins far enough from 0 that all reads are distinct (n >= H):
 *   STD, FBIN: h is a scaled sum of H independent unit-variance terms -> (0, 1).
 *   MAX: the max of i iid Exp(1) has mean sum_{k<=i} 1/k and variance sum_{k<=i} 1/k^2, so
 *        mu_H = sum_{i<=H} (Hn(i) - 1) / sqrt(H),  sigma_H^2 = sum_{i<=H} sum_{k<=i} k^-2 / H.
 *   MAX0: windows of i + 1 bins: the same with Hn(i+1) and k <= i+1 (windows of one bin n are
 *        disjoint for n >= H, since (i+1) n > i n + i).
 *   GREEDY: each step is the max of two fresh iid Exp(1) bins: mean 1/2, variance 5/4, so
 *        mu_H = sqrt(H)/2, sigma_H = sqrt(5/4).
 *   GREEDY1: the first term is one standardised bin (0, 1), the H - 1 others as above, so
 *        mu_H = (H - 1) / (2 sqrt(H)), sigma_H^2 = (1 + 5/4 (H - 1)) / H.
 * mu[0], sigma[0] are set to (0, 1).
 */
void hs_oracle_noise_moments(int variant, int hmax, double* mu, double* sigma) {
    mu[0] = 0.0;
    sigma[0] = 1.0;
    double m_acc = 0.0, v_acc = 0.0, harm = 0.0, harm2 = 0.0;
    for (int H = 1; H <= hmax; ++H) {
        if (variant == HS_O_MAX || variant == HS_O_MAX0) {
            int w = variant == HS_O_MAX0 ? H + 1 : H; /* bins in harmonic H's window */
            if (H == 1 && variant == HS_O_MAX0) {
                harm = 1.0;
                harm2 = 1.0;
            }
            harm += 1.0 / w;
            harm2 += 1.0 / ((double)w * w);
            m_acc += harm - 1.0;
            v_acc += harm2;
            mu[H] = m_acc / sqrt((double)H);
            sigma[H] = sqrt(v_acc / H);
        } else if (variant == HS_O_GREEDY) {
            mu[H] = 0.5 * sqrt((double)H);
            sigma[H] = sqrt(1.25);
        } else if (variant == HS_O_GREEDY1) {
            mu[H] = 0.5 * (H - 1) / sqrt((double)H);
            sigma[H] = sqrt((1.0 + 1.25 * (H - 1)) / H);
        } else {
            mu[H] = 0.0;
            sigma[H] = 1.0;
        }
    }
}

int hs_oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

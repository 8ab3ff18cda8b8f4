/*
 * Seeded, counter-based synthetic inputs for the harmonic sum: power spectra of
 * exponential(1) noise standardised to mean 0 / variance 1, with optional injected
 * pulsar harmonics, and 2-D FDAS-like planes.
 *
 * This module holds no harmonic-sum arithmetic. It is shared, as data only, by the
 * CPU oracle, the tests and the benchmark; every element is a pure function of
 * (seed, stream, spectrum or plane row, bin), so any subset of a very large input
 * can be regenerated on its own.
 *
 * Value of bin m (all in double, rounded to float once):
 *     p(m)  = -log(u),  u in (0,1) from the counter generator   (Exp(1) power)
 *     v(m)  = p(m) - 1 + signal(m)        (standardised: Exp(1) has mean 1, sd 1)
 *     raw   = p(m) + signal(m)            (when the raw flag is set)
 * signal(m) = sum_k a_k * profile(m - k*f0), a_k = A/k, k = 1..K, where the profile is
 *     sinc^2(d) = (sin(pi d)/(pi d))^2 for |d| <= 8            (shape 0: scalloping across a bin)
 *     exp(-d^2/(2 w^2))                 for |d| <= 8 w         (shape 1: broadened harmonic)
 * The pulsar experiment of the paper (Section 3) uses a pulse train whose harmonics land
 * between Fourier bins; shape 0 reproduces that in the spectral domain directly.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t shape;  /* -1: no pulsar, 0: sinc^2, 1: gaussian */
    int32_t n_harm; /* K */
    double f0;      /* fundamental, in bins */
    double amp;     /* A; harmonic k has amplitude A/k */
    double width;   /* gaussian sigma in bins (shape 1) */
    double z0;      /* 2-D only: drift of the fundamental in z rows; harmonic k sits at row k*z0 */
} hs_pulsar;

/* SplitMix64 finaliser (Steele, Lea, Flood 2014). */
static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t word3(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b) {
    uint64_t k1 = mix64(seed + 0x9E3779B97F4A7C15ULL * (stream + 1));
    uint64_t k2 = mix64(k1 + 0xD1B54A32D192ED03ULL * (a + 1));
    return mix64(k2 + 0x9E3779B97F4A7C15ULL * (b + 1));
}

/* u in the open interval (0,1) with 53 random bits. */
static inline double u01(uint64_t w) { return ((double)(w >> 11) + 0.5) * 0x1.0p-53; }

double hs_synth_uniform(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b) {
    return u01(word3(seed, stream, a, b));
}

#define STREAM_NOISE 1ULL

static double profile(const hs_pulsar* p, double d) {
    if (p->shape == 0) {
        if (fabs(d) > 8.0) return 0.0;
        if (d == 0.0) return 1.0;
        double s = sin(M_PI * d) / (M_PI * d);
        return s * s;
    }
    double w = p->width;
    if (fabs(d) > 8.0 * w) return 0.0;
    return exp(-(d * d) / (2.0 * w * w));
}

static double signal_at(const hs_pulsar* p, double m) {
    if (!p || p->shape < 0 || p->n_harm <= 0 || p->f0 <= 0.0) return 0.0;
    double reach = (p->shape == 0) ? 8.0 : 8.0 * p->width;
    long k_lo = (long)floor((m - reach) / p->f0);
    long k_hi = (long)ceil((m + reach) / p->f0);
    if (k_lo < 1) k_lo = 1;
    if (k_hi > p->n_harm) k_hi = p->n_harm;
    double s = 0.0;
    for (long k = k_lo; k <= k_hi; ++k) s += (p->amp / (double)k) * profile(p, m - (double)k * p->f0);
    return s;
}

static inline float bin_value(uint64_t seed, uint64_t row_id, int64_t m, const hs_pulsar* p, int raw) {
    double pw = -log(u01(word3(seed, STREAM_NOISE, row_id, (uint64_t)m)));
    double v = raw ? pw : pw - 1.0;
    return (float)(v + signal_at(p, (double)m));
}

/* One spectrum (row_id names its noise stream), bins [m0, m0+count). */
void hs_synth_spectrum(uint64_t seed, uint64_t row_id, int64_t m0, int64_t count, const hs_pulsar* p,
                       int raw, float* out, int nthreads) {
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1) if (count > 65536)
    for (int64_t k = 0; k < count; ++k) out[k] = bin_value(seed, row_id, m0 + k, p, raw);
}

/* A packed batch: spectrum s occupies out[offsets[s] .. offsets[s+1]) and uses noise
 * stream row_id = first_id + s; pulsars[s].shape < 0 means noise only. */
void hs_synth_batch(uint64_t seed, uint64_t first_id, int32_t n_spec, const int64_t* offsets,
                    const hs_pulsar* pulsars, int raw, float* out, int nthreads) {
    const int64_t chunk = 1 << 16;
    int64_t total = offsets[n_spec] - offsets[0];
    int64_t n_chunks = (total + chunk - 1) / chunk;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t c = 0; c < n_chunks; ++c) {
        int64_t g0 = offsets[0] + c * chunk, g1 = g0 + chunk;
        if (g1 > offsets[n_spec]) g1 = offsets[n_spec];
        /* locate the spectrum holding g0 (offsets are sorted) */
        int32_t lo = 0, hi = n_spec - 1;
        while (lo < hi) {
            int32_t mid = (lo + hi + 1) / 2;
            if (offsets[mid] <= g0) lo = mid; else hi = mid - 1;
        }
        for (int32_t s = lo; s < n_spec && offsets[s] < g1; ++s) {
            int64_t a = g0 > offsets[s] ? g0 : offsets[s];
            int64_t b = g1 < offsets[s + 1] ? g1 : offsets[s + 1];
            const hs_pulsar* p = pulsars ? &pulsars[s] : NULL;
            for (int64_t g = a; g < b; ++g)
                out[g - offsets[0]] = bin_value(seed, first_id + (uint64_t)s, g - offsets[s], p, raw);
        }
    }
}

/* A 2-D plane of nz rows (row r holds z = z_min + r) by n_bins, rows row_stride floats apart.
 * Pulsar j puts harmonic k at bin k*f0 on the row nearest to k*z0 (gaussian across bins). */
void hs_synth_plane(uint64_t seed, uint64_t plane_id, int32_t nz, int32_t z_min, int64_t n_bins,
                    int64_t row_stride, const hs_pulsar* pulsars, int32_t n_pulsars, float* out,
                    int nthreads) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int32_t r = 0; r < nz; ++r) {
        int32_t z = z_min + r;
        uint64_t row_id = plane_id * 4096ULL + (uint64_t)r;
        float* row = out + (int64_t)r * row_stride;
        for (int64_t m = 0; m < n_bins; ++m) {
            double pw = -log(u01(word3(seed, STREAM_NOISE, row_id, (uint64_t)m)));
            row[m] = (float)(pw - 1.0);
        }
        /* add harmonics that land on this row; recompute the whole bin value so it is rounded once */
        for (int32_t j = 0; j < n_pulsars; ++j) {
            const hs_pulsar* p = &pulsars[j];
            if (p->shape < 0) continue;
            for (int32_t k = 1; k <= p->n_harm; ++k) {
                double zk = (double)k * p->z0;
                int32_t zr = (int32_t)floor(zk + 0.5);
                if (zr != z) continue;
                double c = (double)k * p->f0, reach = 8.0 * p->width;
                int64_t m_lo = (int64_t)floor(c - reach), m_hi = (int64_t)ceil(c + reach);
                if (m_lo < 0) m_lo = 0;
                if (m_hi > n_bins - 1) m_hi = n_bins - 1;
                for (int64_t m = m_lo; m <= m_hi; ++m) {
                    double pw = -log(u01(word3(seed, STREAM_NOISE, row_id, (uint64_t)m)));
                    double s = 0.0;
                    for (int32_t jj = 0; jj < n_pulsars; ++jj) {
                        const hs_pulsar* q = &pulsars[jj];
                        if (q->shape < 0) continue;
                        for (int32_t kk = 1; kk <= q->n_harm; ++kk) {
                            if ((int32_t)floor((double)kk * q->z0 + 0.5) != z) continue;
                            double d = (double)m - (double)kk * q->f0;
                            if (fabs(d) > 8.0 * q->width) continue;
                            s += (q->amp / (double)kk) * exp(-(d * d) / (2.0 * q->width * q->width));
                        }
                    }
                    row[m] = (float)(pw - 1.0 + s);
                }
            }
        }
    }
}

/*
 * Per-bin harmonic-sum definitions, written once and instantiated for REAL = float (the FP32
 * mode, every operation rounded to float in the order written) and REAL = double (the FP64
 * mode).  Included twice by hs_oracle.c with REAL and SFX defined.  TEST INFRASTRUCTURE.
 *
 * Readings of the paper used here (Section 2 of arXiv:1812.02647):
 *   Eq. 1  index of harmonic i of H at output bin n is round-half-up(n*i/H) = (2*n*i + H) div (2*H).
 *   Eq. 2  the max runs over the literal window j = 1..i, i.e. bins i*n+1 .. i*n+i; first max wins.
 *          Variant flag MAX0: the window j = 0..i, bins i*n .. i*n+i.
 *   Eq. 3  bins i*n.
 *   Eq. 4  start with S = 0, j = 0; harmonic i compares x(i*n+j) (left) with x(i*n+j+1) (right);
 *          the right bin is taken only when strictly larger, and then j grows by one.
 *          Variant flag GREEDY1: the first term is x(n) and the pairs start at harmonic 2 (j = 0).
 *   Terms are summed in the order i = 1..H; h = S * c_H with c_H = 1/sqrt(H);
 *   snr = (h - mu_H) * isig_H; the best H is the first H with the largest snr.
 *   Variant flag POW2 (the stages of SIGPROC/PRESTO-style searches): only H = 1, 2, 4, 8, .. are
 *   searched; the other H report snr = -inf (Eq. 2-4 still add their terms to the running sum).
 */
#define CAT2_(a, b) a##b
#define CAT2(a, b) CAT2_(a, b)
#define FN(name) CAT2(name, SFX)

/* All four variants for one output bin n of a spectrum x[0..N). */
static void FN(hs_bin_)(int variant, const REAL* x, int64_t N, int64_t n, int hmax, const REAL* cs,
                        const REAL* mu, const REAL* isig, REAL* best_out, uint8_t* h_out,
                        uint32_t* path_out, REAL* all_h, int64_t all_h_stride) {
    const int pow2 = (variant & HS_O_POW2) != 0; /* stages H = 1, 2, 4, ..: other H are not searched */
    variant &= ~HS_O_POW2;
    int hv = hs_oracle_hvalid(variant, n, N, hmax);
    REAL best = -INFINITY;
    int best_h = 0;
    REAL S = 0;        /* running partial sum for Eq. 2-4 (harmonic H adds one term) */
    int64_t j = 0;     /* Eq. 4 neighbour offset */
    uint32_t path = 0; /* Eq. 4 choices: bit i-1 set when harmonic i took the right bin */
    for (int H = 1; H <= hmax; ++H) {
        REAL snr = -INFINITY;
        const int stage = !pow2 || (H & (H - 1)) == 0;
        /* Eq. 1 sums are independent per H, so its non-stage H are not computed at all */
        if (H <= hv && (stage || variant != HS_O_STD)) {
            REAL sum = 0;
            if (variant == HS_O_STD) {
                /* Eq. 1: a fresh sum of H terms for every H */
                for (int i = 1; i <= H; ++i) sum = sum + x[hs_oracle_eq1_index(n, i, H)];
            } else if (variant == HS_O_MAX || variant == HS_O_MAX0) {
                /* Eq. 2: harmonic H contributes the largest of x(H*n+j0) .. x(H*n+H), with j0 = 1 as
                 * written (the MAX0 variant flag starts the window at j0 = 0) */
                int64_t base = (int64_t)H * n;
                int j0 = variant == HS_O_MAX0 ? 0 : 1;
                REAL m = x[base + j0];
                for (int jj = j0 + 1; jj <= H; ++jj) {
                    REAL v = x[base + jj];
                    m = (v > m) ? v : m;
                }
                S = S + m;
                sum = S;
            } else if (variant == HS_O_FBIN) {
                /* Eq. 3 */
                S = S + x[(int64_t)H * n];
                sum = S;
            } else if (variant == HS_O_GREEDY1 && H == 1) {
                /* Eq. 4 variant flag: the first term is x(n) itself; pairs start at harmonic 2 */
                S = S + x[n];
                sum = S;
            } else { /* HS_O_GREEDY, Eq. 4 (and GREEDY1 from H = 2 on) */
                int64_t base = (int64_t)H * n + j;
                REAL l = x[base], r = x[base + 1], t;
                if (r > l) {
                    t = r;
                    path |= 1u << (H - 1);
                    j += 1;
                } else {
                    t = l;
                }
                S = S + t;
                sum = S;
            }
            if (stage) {
                REAL h = sum * cs[H];
                snr = (h - mu[H]) * isig[H];
                if (snr > best) {
                    best = snr;
                    best_h = H;
                }
            }
        }
        if (all_h) all_h[(int64_t)(H - 1) * all_h_stride + n] = snr;
    }
    *best_out = best;
    *h_out = (uint8_t)best_h;
    if (path_out) *path_out = path;
}

/* One spectrum, every bin; bins are independent, so they may run on several threads. */
void FN(hs_oracle_1d_)(int variant, const REAL* x, int64_t N, int hmax, const REAL* mu_in,
                       const REAL* isig_in, REAL* best_snr, uint8_t* best_h, uint32_t* path, REAL* all_h,
                       int nthreads) {
    REAL cs[HS_O_HMAX + 1], mu[HS_O_HMAX + 1], isig[HS_O_HMAX + 1];
    for (int H = 0; H <= hmax; ++H) {
        cs[H] = (H == 0) ? (REAL)0 : (REAL)(1.0 / sqrt((double)H));
        mu[H] = mu_in ? mu_in[H] : (REAL)0;
        isig[H] = isig_in ? isig_in[H] : (REAL)1;
    }
#pragma omp parallel for schedule(dynamic, 2048) num_threads(nthreads > 0 ? nthreads : 1) if (nthreads > 1)
    for (int64_t n = 0; n < N; ++n)
        FN(hs_bin_)(variant, x, N, n, hmax, cs, mu, isig, &best_snr[n], &best_h[n], path ? &path[n] : NULL, all_h, N);
}

/* Only the listed output bins of one spectrum (for spot checks of very large inputs). */
void FN(hs_oracle_bins_)(int variant, const REAL* x, int64_t N, int hmax, const REAL* mu_in, const REAL* isig_in,
                         const int64_t* bins, int64_t count, REAL* best_snr, uint8_t* best_h, uint32_t* path) {
    REAL cs[HS_O_HMAX + 1], mu[HS_O_HMAX + 1], isig[HS_O_HMAX + 1];
    for (int H = 0; H <= hmax; ++H) {
        cs[H] = (H == 0) ? (REAL)0 : (REAL)(1.0 / sqrt((double)H));
        mu[H] = mu_in ? mu_in[H] : (REAL)0;
        isig[H] = isig_in ? isig_in[H] : (REAL)1;
    }
    for (int64_t k = 0; k < count; ++k) {
        uint32_t pth = 0;
        FN(hs_bin_)(variant, x, N, bins[k], hmax, cs, mu, isig, &best_snr[k], &best_h[k], &pth, NULL, N);
        if (path) path[k] = pth;
    }
}

/* A packed batch: spectrum s is x[offsets[s] .. offsets[s+1]); outputs use the same packing.
 * Spectra are handed to threads one at a time, as in the paper's CPU versions (Section 2). */
void FN(hs_oracle_batched_)(int variant, const REAL* x, const int64_t* offsets, int n_spec, int hmax,
                            const REAL* mu, const REAL* isig, REAL* best_snr, uint8_t* best_h, uint32_t* path,
                            int nthreads) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) if (nthreads > 1)
    for (int s = 0; s < n_spec; ++s) {
        int64_t o = offsets[s], len = offsets[s + 1] - offsets[s];
        FN(hs_oracle_1d_)(variant, x + o, len, hmax, mu, isig, best_snr + o, best_h + o, path ? path + o : NULL,
                          NULL, 1);
    }
}

/* 2-D Eq. 1 over an FDAS plane: row r holds z = z_min + r, bins along the row.
 *   h(n, z)_H = c_H * sum_{i=1..H} x(round(n*i/H), round(z*i/H)), both rounded half up.
 * Outputs: per cell (r, n) the best snr and H; per bin n the best over rows (lowest row on ties).
 * Requires z_min <= 0 <= z_min + nz - 1 so every rounded row lies in the plane. */
void FN(hs_oracle_2d_)(const REAL* plane, int nz, int z_min, int64_t n_bins, int64_t row_stride, int hmax,
                       const REAL* mu_in, const REAL* isig_in, REAL* best_snr, uint8_t* best_h, REAL* best_snr_n,
                       uint8_t* best_h_n, int32_t* best_z_n, REAL* all_h, int nthreads) {
    REAL cs[HS_O_HMAX + 1], mu[HS_O_HMAX + 1], isig[HS_O_HMAX + 1];
    for (int H = 0; H <= hmax; ++H) {
        cs[H] = (H == 0) ? (REAL)0 : (REAL)(1.0 / sqrt((double)H));
        mu[H] = mu_in ? mu_in[H] : (REAL)0;
        isig[H] = isig_in ? isig_in[H] : (REAL)1;
    }
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) if (nthreads > 1)
    for (int r = 0; r < nz; ++r) {
        int64_t z = (int64_t)z_min + r;
        for (int64_t n = 0; n < n_bins; ++n) {
            REAL best = -INFINITY;
            int bh = 0;
            for (int H = 1; H <= hmax; ++H) {
                REAL sum = 0;
                for (int i = 1; i <= H; ++i) {
                    int64_t zi = hs_oracle_floor_div(2 * z * i + H, 2 * (int64_t)H);
                    int64_t ni = hs_oracle_eq1_index(n, i, H);
                    sum = sum + plane[(zi - z_min) * row_stride + ni];
                }
                REAL h = sum * cs[H];
                REAL snr = (h - mu[H]) * isig[H];
                if (all_h) all_h[((int64_t)(H - 1) * nz + r) * n_bins + n] = snr;
                if (snr > best) {
                    best = snr;
                    bh = H;
                }
            }
            best_snr[(int64_t)r * n_bins + n] = best;
            best_h[(int64_t)r * n_bins + n] = (uint8_t)bh;
        }
    }
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1) if (nthreads > 1)
    for (int64_t n = 0; n < n_bins; ++n) {
        REAL best = -INFINITY;
        int br = 0;
        for (int r = 0; r < nz; ++r) {
            REAL v = best_snr[(int64_t)r * n_bins + n];
            if (v > best) {
                best = v;
                br = r;
            }
        }
        best_snr_n[n] = best;
        best_h_n[n] = best_h[(int64_t)br * n_bins + n];
        best_z_n[n] = z_min + br;
    }
}

/* Only the listed cells (row rows[k], bin bins[k]) of a 2-D plane, same definition as above. */
/*
 * 2-D form of Eq. 3 (a variant of the 2-D sums): the output cell (n, z) is the fundamental and
 * harmonic i reads x(i*n, i*z), added in the order i = 1..H as a running sum.  H is valid while
 * H*n <= N-1 (every H at n = 0) and H*z stays within the plane's rows.
 */
void FN(hs_oracle_2d_fbin_)(const REAL* plane, int nz, int z_min, int64_t n_bins, int64_t row_stride, int hmax,
                            const REAL* mu_in, const REAL* isig_in, REAL* best_snr, uint8_t* best_h, REAL* best_snr_n,
                            uint8_t* best_h_n, int32_t* best_z_n, REAL* all_h, int nthreads) {
    REAL cs[HS_O_HMAX + 1], mu[HS_O_HMAX + 1], isig[HS_O_HMAX + 1];
    for (int H = 0; H <= hmax; ++H) {
        cs[H] = (H == 0) ? (REAL)0 : (REAL)(1.0 / sqrt((double)H));
        mu[H] = mu_in ? mu_in[H] : (REAL)0;
        isig[H] = isig_in ? isig_in[H] : (REAL)1;
    }
    const int64_t z_max = (int64_t)z_min + nz - 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) if (nthreads > 1)
    for (int r = 0; r < nz; ++r) {
        int64_t z = (int64_t)z_min + r;
        for (int64_t n = 0; n < n_bins; ++n) {
            REAL best = -INFINITY, S = 0;
            int bh = 0;
            for (int H = 1; H <= hmax; ++H) {
                REAL snr = -INFINITY;
                int valid = (H * n <= n_bins - 1) && (H * z >= z_min) && (H * z <= z_max);
                if (valid) {
                    S = S + plane[(H * z - z_min) * row_stride + H * n];
                    REAL h = S * cs[H];
                    snr = (h - mu[H]) * isig[H];
                    if (snr > best) {
                        best = snr;
                        bh = H;
                    }
                }
                if (all_h) all_h[((int64_t)(H - 1) * nz + r) * n_bins + n] = snr;
                if (!valid) { /* later H are invalid too: reads move further out */
                    for (int H2 = H + 1; H2 <= hmax; ++H2)
                        if (all_h) all_h[((int64_t)(H2 - 1) * nz + r) * n_bins + n] = -INFINITY;
                    break;
                }
            }
            best_snr[(int64_t)r * n_bins + n] = best;
            best_h[(int64_t)r * n_bins + n] = (uint8_t)bh;
        }
    }
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1) if (nthreads > 1)
    for (int64_t n = 0; n < n_bins; ++n) {
        REAL best = -INFINITY;
        int br = 0;
        for (int r = 0; r < nz; ++r) {
            REAL v = best_snr[(int64_t)r * n_bins + n];
            if (v > best) {
                best = v;
                br = r;
            }
        }
        best_snr_n[n] = best;
        best_h_n[n] = best_h[(int64_t)br * n_bins + n];
        best_z_n[n] = z_min + br;
    }
}

/*
 * 2-D forms of Eq. 2 and Eq. 4 (a reading: the paper writes these two sums in 1-D only).  As in the
 * 2-D form of Eq. 3, harmonic i of the cell (n, z) lies on the row i*z, and within that row it is
 * taken exactly as the 1-D equation takes it: Eq. 2 the largest of x(i*n+j0 .. i*n+i, i*z) (j0 = 1,
 * or 0 under MAX0), first maximum; Eq. 4 the choice between x(i*n+j, i*z) and x(i*n+j+1, i*z), the
 * right one only when strictly larger, j carried from harmonic to harmonic (GREEDY1: the first term
 * is x(n, z) and the pairs start at harmonic 2).  Terms are added in the order i = 1..H.  H is valid
 * while the 1-D rule holds for n (H*(n+1) <= N-1, or <= N under GREEDY1) and H*z stays within the
 * plane's rows.  Per bin n the best over rows keeps the lowest row on ties.
 */
void FN(hs_oracle_2d_rowwise_)(int variant, const REAL* plane, int nz, int z_min, int64_t n_bins,
                               int64_t row_stride, int hmax, const REAL* mu_in, const REAL* isig_in, REAL* best_snr,
                               uint8_t* best_h, REAL* best_snr_n, uint8_t* best_h_n, int32_t* best_z_n, REAL* all_h,
                               int nthreads) {
    REAL cs[HS_O_HMAX + 1], mu[HS_O_HMAX + 1], isig[HS_O_HMAX + 1];
    for (int H = 0; H <= hmax; ++H) {
        cs[H] = (H == 0) ? (REAL)0 : (REAL)(1.0 / sqrt((double)H));
        mu[H] = mu_in ? mu_in[H] : (REAL)0;
        isig[H] = isig_in ? isig_in[H] : (REAL)1;
    }
    const int64_t z_max = (int64_t)z_min + nz - 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) if (nthreads > 1)
    for (int r = 0; r < nz; ++r) {
        const int64_t z = (int64_t)z_min + r;
        for (int64_t n = 0; n < n_bins; ++n) {
            const int hv = hs_oracle_hvalid(variant, n, n_bins, hmax);
            REAL best = -INFINITY, S = 0;
            int bh = 0;
            int64_t j = 0;
            for (int H = 1; H <= hmax; ++H) {
                REAL snr = -INFINITY;
                const int valid = H <= hv && H * z >= z_min && H * z <= z_max;
                if (valid) {
                    const REAL* row = plane + (H * z - z_min) * row_stride;
                    REAL t;
                    if (variant == HS_O_MAX || variant == HS_O_MAX0) {
                        const int64_t base = (int64_t)H * n;
                        const int jfirst = (variant == HS_O_MAX0) ? 0 : 1;
                        t = row[base + jfirst];
                        for (int jw = jfirst + 1; jw <= H; ++jw) {
                            REAL v = row[base + jw];
                            t = (v > t) ? v : t;
                        }
                    } else if (H == 1 && variant == HS_O_GREEDY1) { /* first term fixed at x(n, z) */
                        t = row[n];
                    } else { /* HS_O_GREEDY (and GREEDY1 from H = 2 on) */
                        const int64_t base = (int64_t)H * n + j;
                        REAL lft = row[base], rgt = row[base + 1];
                        if (rgt > lft) {
                            t = rgt;
                            j += 1;
                        } else {
                            t = lft;
                        }
                    }
                    S = S + t;
                    REAL h = S * cs[H];
                    snr = (h - mu[H]) * isig[H];
                    if (snr > best) {
                        best = snr;
                        bh = H;
                    }
                }
                if (all_h) all_h[((int64_t)(H - 1) * nz + r) * n_bins + n] = snr;
                if (!valid) { /* later H are invalid too: the rows H*z move further out */
                    for (int H2 = H + 1; H2 <= hmax; ++H2)
                        if (all_h) all_h[((int64_t)(H2 - 1) * nz + r) * n_bins + n] = -INFINITY;
                    break;
                }
            }
            best_snr[(int64_t)r * n_bins + n] = best;
            best_h[(int64_t)r * n_bins + n] = (uint8_t)bh;
        }
    }
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1) if (nthreads > 1)
    for (int64_t n = 0; n < n_bins; ++n) {
        REAL best = -INFINITY;
        int br = 0;
        for (int r = 0; r < nz; ++r) {
            REAL v = best_snr[(int64_t)r * n_bins + n];
            if (v > best) {
                best = v;
                br = r;
            }
        }
        best_snr_n[n] = best;
        best_h_n[n] = best_h[(int64_t)br * n_bins + n];
        best_z_n[n] = z_min + br;
    }
}

void FN(hs_oracle_2d_cells_)(const REAL* plane, int nz, int z_min, int64_t n_bins, int64_t row_stride, int hmax,
                             const REAL* mu_in, const REAL* isig_in, const int32_t* rows, const int64_t* bins,
                             int64_t count, REAL* best_snr, uint8_t* best_h) {
    REAL cs[HS_O_HMAX + 1], mu[HS_O_HMAX + 1], isig[HS_O_HMAX + 1];
    for (int H = 0; H <= hmax; ++H) {
        cs[H] = (H == 0) ? (REAL)0 : (REAL)(1.0 / sqrt((double)H));
        mu[H] = mu_in ? mu_in[H] : (REAL)0;
        isig[H] = isig_in ? isig_in[H] : (REAL)1;
    }
    (void)nz;
    (void)n_bins;
    for (int64_t k = 0; k < count; ++k) {
        int64_t z = (int64_t)z_min + rows[k], n = bins[k];
        REAL best = -INFINITY;
        int bh = 0;
        for (int H = 1; H <= hmax; ++H) {
            REAL sum = 0;
            for (int i = 1; i <= H; ++i) {
                int64_t zi = hs_oracle_floor_div(2 * z * i + H, 2 * (int64_t)H);
                sum = sum + plane[(zi - z_min) * row_stride + hs_oracle_eq1_index(n, i, H)];
            }
            REAL snr = (sum * cs[H] - mu[H]) * isig[H];
            if (snr > best) {
                best = snr;
                bh = H;
            }
        }
        best_snr[k] = best;
        best_h[k] = (uint8_t)bh;
    }
}

#undef FN
#undef CAT2
#undef CAT2_

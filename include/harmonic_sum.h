/*
 * harmonic_sum.h -- C ABI of the GB300 (sm_103a) incoherent harmonic-sum library.
 *
 * The operation is the incoherent harmonic sum of Adamek & Armour, "A GPU implementation of the
 * harmonic sum algorithm" (arXiv:1812.02647), Section 2: for every output bin n of a power
 * spectrum x and every number of harmonics H = 1..hmax, a sum of H terms scaled by 1/sqrt(H),
 * reduced per bin to the best signal-to-noise ratio and the H that gives it.  Four variants:
 *
 *   HS_STD     Eq. 1   h(n)_H = H^-1/2 sum_{i=1..H} x(round(n*i/H)),  rounded half up
 *   HS_MAX     Eq. 2   h(n)_H = H^-1/2 sum_{i=1..H} max_{1<=j<=i} x(i*n + j)
 *   HS_FBIN    Eq. 3   h(n)_H = H^-1/2 sum_{i=1..H} x(i*n)
 *   HS_GREEDY  Eq. 4   h(n)_H = H^-1/2 sum_{i=1..H} max(x(i*n + j), x(i*n + j + 1)), j grows by
 *                      one each time the right bin is strictly larger (j starts at 0)
 *
 * and the 2-D form of Eq. 1 over an FDAS plane (abstract and Section 1): h(n, z)_H =
 * H^-1/2 sum_i x(round(n*i/H), round(z*i/H)).
 *
 * Arithmetic contract (FP32 path): terms are read as FP32 (FP16/BF16 storage is widened exactly),
 * summed in the order i = 1..H with no fused multiply-add, h = S * c_H with c_H = float(1/sqrt(H))
 * (computed in double, rounded once), snr = (h - mu_H) * isig_H with per-variant calibration
 * tables (identity by default), best H = the first H with the largest snr.  Harmonics whose reads
 * would leave [0, N) are not summed (truncation): Eq. 1 keeps every H; Eq. 2 and 4 need
 * H*(n+1) <= N-1; Eq. 3 needs H*n <= N-1.  A bin with no valid H reports snr = -inf, H = 0.
 *
 * Conventions for every entry point:
 *   - Device buffers are owned by the caller; the library never frees them.  A plan owns host
 *     state only.  Scratch memory comes from the caller as a workspace (hs_plan_workspace_size).
 *   - Calls enqueue work on the caller's stream and return immediately; argument errors are
 *     detected on the host and returned before anything is enqueued.  Errors found on the device
 *     (candidate overflow, a bounded wait that gave up) are recorded in a status word inside the
 *     workspace and returned by hs_sync_status.
 *   - Device input pointers must be 16-byte aligned (HS_ERR_ALIGN otherwise).
 *   - No C++ exception crosses this interface.
 */
#ifndef HARMONIC_SUM_H
#define HARMONIC_SUM_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HS_HMAX_1D 32 /* largest number of harmonics in 1-D */
#define HS_HMAX_2D 16 /* largest number of harmonics in 2-D */
#define HS_MAX_BINS_1D (1LL << 26) /* longest 1-D spectrum (indices stay in 32 bits) */

typedef enum hs_status {
    HS_OK = 0,
    HS_ERR_INVALID = 1,    /* bad argument: null pointer, size out of range, variant not in plan */
    HS_ERR_ALIGN = 2,      /* a device pointer is not 16-byte aligned */
    HS_ERR_CUDA = 3,       /* a CUDA runtime call failed (launch error, etc.) */
    HS_ERR_NOMEM = 4,      /* host allocation failed, or the workspace is smaller than required */
    HS_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up (recorded in the status word) */
    HS_ERR_UNSUPPORTED = 6, /* valid request this build does not implement (e.g. dtype for 2-D) */
    HS_WARN_CAND_OVERFLOW = 100 /* more candidates than capacity; the true count is still stored */
} hs_status;

typedef enum hs_variant { HS_STD = 1, HS_MAX = 2, HS_FBIN = 4, HS_GREEDY = 8 } hs_variant;

typedef enum hs_dtype { HS_F32 = 0, HS_F16 = 1, HS_BF16 = 2 } hs_dtype;

/* plan flags */
#define HS_FLAG_OUT_ALL_H 1 /* hs_sum_1d may write the snr of every H (debug table) */
/* Eq. 1 over a batch (hs_sum_batched, hmax 32, no every-H table): stage each Farey fraction's input
 * span of a tile in shared memory with bulk copies and read it from there, the span-per-harmonic
 * access pattern of Section 2 made explicit.  Results are bit-identical to the default path, which
 * gathers through L1 and is faster on GB300; the flag exists for comparison. */
#define HS_FLAG_STAGED_SPANS 2
/* Eq. 2 with the window j = 0..i: harmonic i adds the largest of x(i n) .. x(i n + i) (i + 1 bins)
 * instead of x(i n + 1) .. x(i n + i) as written in Section 2, so that a pulsar between two bins is
 * seen by its lower neighbour too.  Applies to the forward sums and the adjoint; the valid H are
 * unchanged (H (n + 1) <= N - 1).  Calibrate with hs_noise_calibration_flags. */
#define HS_FLAG_MAX_WINDOW0 4
/* 1-D plans: search only the power-of-two stages H = 1, 2, 4, 8, 16, 32 (as SIGPROC and PRESTO do)
 * instead of every H = 1..hmax.  Eq. 1 then reads only the 32 fractions i/32 and adds 63 terms per
 * bin; Eq. 2-4 still add every harmonic to their running sums.  The every-H table reads -inf for
 * H that are not stages. */
#define HS_FLAG_POW2_STAGES 8
/* Eq. 4 with its first term fixed: h_1 = x(n) and the pairwise choice starts at harmonic 2 with j = 0
 * (the form with h_1 = x(n) and the first pair at 2n), instead of max(x(n), x(n+1)) as written.  H is
 * valid while H (n + 1) <= N (the furthest read is H n + H - 1).  Forward sums and adjoint;
 * calibrate with hs_noise_calibration_flags. */
#define HS_FLAG_GREEDY_FIXED1 16
/* Diagnostic, for testing the error path of the bounded device waits: with HS_FLAG_STAGED_SPANS,
 * the work item holding the first tile of the batch arms its first shared-memory slot for 16 bytes
 * more than it copies, so that slot never fills.  The consumer warps of that CTA give up after
 * their bounded wait (about a second), the CTA stops, the launch still ends, and hs_sync_status
 * returns HS_ERR_TIMEOUT; the outputs of that CTA's tiles are left unwritten.  No other path reads
 * the flag. */
#define HS_FLAG_CHECK_TIMEOUT 32

typedef struct hs_plan hs_plan; /* opaque; host memory only */

typedef struct hs_plan_desc {
    int variants;          /* bitmask of hs_variant this plan may run */
    int hmax;              /* 1..32 for 1-D plans, 1..16 for 2-D plans */
    hs_dtype dtype;        /* storage type of the input spectra */
    int64_t max_bins;      /* longest spectrum (1-D) or row (2-D) this plan accepts */
    int nz;                /* 2-D: rows of the plane (0 for a 1-D plan) */
    int z_min;             /* 2-D: z of row 0; rows cover z_min..z_min+nz-1, which must contain 0 */
    float threshold;       /* candidates are bins whose best snr is strictly above this */
    int64_t cand_capacity; /* entries in the caller's candidate buffer (0: no candidate list) */
    int flags;             /* HS_FLAG_* */
} hs_plan_desc;

/* One candidate: 16 bytes, written with one 128-bit store. */
typedef struct hs_candidate {
    uint32_t spectrum; /* spectrum (1-D) or plane (2-D) id */
    uint32_t bin;      /* output bin n; for Eq. 1 the fundamental frequency is n/H bins */
    float snr;         /* best calibrated snr of the bin */
    int16_t z;         /* drift row value z (2-D), 0 for 1-D */
    uint8_t h;         /* H that gave snr */
    uint8_t variant;   /* hs_variant that produced it */
} hs_candidate;

/* Per-bin outputs of a 1-D call (caller-owned device memory).  For a batch every array is packed
 * exactly like the input: spectrum s occupies [offsets[s], offsets[s+1]). */
typedef struct hs_out {
    float* best_snr;        /* [bins] required */
    uint8_t* best_h;        /* [bins] required */
    uint32_t* path;         /* [bins] Eq. 4 choices (bit i-1 = harmonic i took the right bin); NULL to skip */
    float* all_h;           /* [hmax][bins] snr of every H (-inf where H is not valid); needs
                               HS_FLAG_OUT_ALL_H and hs_sum_1d; NULL to skip */
    hs_candidate* cand;     /* [cand_capacity] appended to, in no particular order; NULL to skip */
    unsigned long long* cand_count; /* device counter, incremented by the number of candidates
                                       found (also beyond capacity); the caller zeroes it */
} hs_out;

/* Outputs of a 2-D call; plane cells are [nz][n_bins] with the same row order as the input. */
typedef struct hs_out2d {
    float* best_snr;   /* [nz][n_bins] best snr of each (z, n) cell */
    uint8_t* best_h;   /* [nz][n_bins] */
    float* best_snr_n; /* [n_bins] best over z of each bin (lowest row wins ties) */
    uint8_t* best_h_n; /* [n_bins] */
    int16_t* best_z_n; /* [n_bins] z value (not the row index) of that best */
    hs_candidate* cand; /* cells whose best snr is above the threshold; NULL to skip */
    unsigned long long* cand_count;
} hs_out2d;

/* ---- plan ------------------------------------------------------------------------------- */

/* Validate *desc and create a plan (host allocation only).  HS_ERR_INVALID for an out-of-range
 * field; HS_ERR_NOMEM if the host allocation fails. */
hs_status hs_plan_create(hs_plan** plan, const hs_plan_desc* desc);

/* Free a plan (NULL is accepted). */
hs_status hs_plan_destroy(hs_plan* plan);

/* Replace the calibration tables of one variant: mu[H], isig[H] for H = 0..hmax (host arrays,
 * copied; entry 0 unused).  NULL for both restores the identity (mu = 0, isig = 1), under which
 * snr equals the scaled sum h of Section 2 bit for bit. */
hs_status hs_plan_set_calibration(hs_plan* plan, hs_variant v, const float* mu, const float* isig);

/* Closed-form noise calibration for standardised Exp(1) spectra (bins n >= H): for Eq. 1 and 3
 * (0, 1); for Eq. 2 mu_H = sum_{i<=H}(Hn(i)-1)/sqrt(H), sigma_H^2 = sum_{i<=H} sum_{k<=i} k^-2 / H
 * (Hn = harmonic number); for Eq. 4 mu_H = sqrt(H)/2, sigma_H = sqrt(5/4).  Writes hmax+1 floats
 * to each host array (isig = 1/sigma), computed in double and rounded once. */
hs_status hs_noise_calibration(hs_variant v, int hmax, float* mu, float* isig);

/* The same for the sums a plan with these flags computes: with HS_FLAG_MAX_WINDOW0, Eq. 2 windows
 * hold i + 1 bins, so Hn(i+1) and k <= i+1 replace Hn(i) and k <= i above; with
 * HS_FLAG_GREEDY_FIXED1, Eq. 4 has mu_H = (H - 1) / (2 sqrt(H)), sigma_H^2 = (1 + 5/4 (H - 1)) / H.
 * flags = 0 gives hs_noise_calibration. */
hs_status hs_noise_calibration_flags(hs_variant v, int hmax, int flags, float* mu, float* isig);

/* Bytes of device workspace a call needs for up to n_spectra spectra (1 for hs_sum_1d / 2-D).
 * The workspace holds the status word, the work queue and tile prefix sums; it must be 256-byte
 * aligned, must not be shared by calls that may overlap on the GPU, and is zeroed by
 * hs_workspace_init.  A plan with FP16/BF16 storage, Eq. 1 and hmax 32 (without
 * HS_FLAG_STAGED_SPANS) also reserves min(n_spectra, 64) * max_bins * 4 bytes: batched Eq. 1 widens
 * up to 64 consecutive spectra at a time into FP32 there and sums them with the FP32 kernel (exact:
 * the same values and operations), which requires non-decreasing offsets (a spectrum outside its
 * group's range is skipped and reported as HS_ERR_INVALID by hs_sync_status). */
hs_status hs_plan_workspace_size(const hs_plan* plan, int n_spectra, size_t* bytes);

/* Zero the workspace status word on the stream (call once after allocating the workspace and
 * after reading a failure from hs_sync_status). */
hs_status hs_workspace_init(const hs_plan* plan, void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* ---- forward ---------------------------------------------------------------------------- */

/* One spectrum: d_x holds n_bins values of the plan's dtype (device, 16-byte aligned).
 * spectrum_id is copied into candidates.  Section 2, Eq. 1-4. */
hs_status hs_sum_1d(const hs_plan* plan, hs_variant v, const void* d_x, int64_t n_bins, uint32_t spectrum_id,
                    const hs_out* out, void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* A batch of spectra of uneven length packed back to back: spectrum s is
 * d_x[d_offsets[s] .. d_offsets[s+1]) (offsets: device int64[n_spectra+1], absolute element indices
 * into d_x, non-decreasing, each length <= plan max_bins, each start 16-byte aligned, i.e.
 * d_offsets[s] * element size a multiple of 16).  Outputs are indexed by the same absolute
 * positions, so a batch may be any slice of a larger packed array.  One persistent launch walks a
 * work queue of (spectrum, tile) items; candidate spectrum ids are first_id + s.
 * hs_graph_create_batched captures this call in a CUDA graph for replay.
 * The library sees only the pointer: d_x must hold elements of the plan's dtype up to the last
 * offset, or the kernels read past the caller's buffer (the Python binding checks this). */
hs_status hs_sum_batched(const hs_plan* plan, hs_variant v, const void* d_x, const int64_t* d_offsets,
                         int n_spectra, uint32_t first_id, const hs_out* out, void* d_ws, size_t ws_bytes,
                         cudaStream_t stream);

/* A batch that lives in host memory, streamed to the device in n_chunks pieces: the copy of piece
 * c+1 (host to device, on an internal stream) overlaps the harmonic sums of piece c (every variant
 * bit set in variant_mask, in the order STD, MAX, FBIN, GREEDY, each writing to outs[k] for the k-th
 * set bit) on the caller's stream.  h_x must be page-locked (cudaHostAlloc / pinned) for the copies
 * to overlap; h_offsets is a host int64[n_spectra+1] array with h_offsets[0] = 0.  d_x (device, at
 * least h_offsets[n_spectra] elements) and d_offsets (device int64[n_spectra+1]) are caller-owned
 * staging buffers that receive the batch.  Everything is enqueued asynchronously; the call returns
 * before the data has moved, so h_x must stay valid until the stream has been synchronised. */
hs_status hs_sum_batched_host(const hs_plan* plan, int variant_mask, const void* h_x, const int64_t* h_offsets,
                              int n_spectra, uint32_t first_id, void* d_x, int64_t* d_offsets, const hs_out* outs,
                              int n_chunks, void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* Same as hs_sum_batched, but without a workspace: for callers that cannot allocate device memory
 * when they call, such as a real-time search pipeline that reserves all of its GPU memory at
 * start-up and forbids allocation in its processing loop (an allocation there can stall or fail in
 * the middle of an observation), or a plugin whose host application owns the device memory pool.
 * (The paper has no counterpart to this; it is a deployment convenience.)
 *   - Its scratch memory is an array of about 128 KiB compiled into the library; every GPU that
 *     loads the library holds one copy until the process exits.  Nothing is allocated or freed.
 *   - At most HS_NOALLOC_MAX_SPECTRA spectra per call; a larger n_spectra returns HS_ERR_INVALID.
 *   - The first call on each device looks up the array's device address (once per device, with
 *     that device current); make that first call before any stream capture.
 *   - Every call on a device shares the one array: calls that may overlap on the GPU (different
 *     streams, or different host threads) race and must be serialised by the caller.
 *   - There is no status word to read back: a candidate overflow shows as *cand_count > capacity,
 *     a spectrum that breaks the layout contract is skipped (its outputs are not written), and a
 *     launch whose bounded device waits gave up (only the HS_FLAG_STAGED_SPANS kernel waits) leaves
 *     the outputs of the affected tiles unwritten.  Callers that need these signals use
 *     hs_sum_batched and hs_sync_status.
 * Outputs, inputs and their layout are exactly those of hs_sum_batched. */
#define HS_NOALLOC_MAX_SPECTRA 16384
hs_status hs_sum_batched_noalloc(const hs_plan* plan, hs_variant v, const void* d_x, const int64_t* d_offsets,
                                 int n_spectra, uint32_t first_id, const hs_out* out, cudaStream_t stream);

/* 2-D Eq. 1 over an FDAS plane of plan->nz rows (row r holds z = z_min + r) by n_bins bins,
 * rows row_stride elements apart (FP32 only in this build).  H = 1..hmax (<= 16). */
hs_status hs_sum_2d(const hs_plan* plan, const void* d_plane, int64_t n_bins, int64_t row_stride,
                    uint32_t plane_id, const hs_out2d* out, void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* The same plane with a chosen variant: HS_STD is hs_sum_2d; the other three are row-wise 2-D forms
 * of Section 2's Eq. 2-4, in which the cell (n, z) is the fundamental and harmonic i lies on the row
 * i z, taken there as the 1-D equation takes it:
 *   HS_FBIN    x(i n, i z)
 *   HS_MAX     the largest of x(i n + j, i z), j = 1..i (j = 0..i under HS_FLAG_MAX_WINDOW0)
 *   HS_GREEDY  the larger of x(i n + j, i z) and x(i n + j + 1, i z), the right one only when
 *              strictly larger (then j grows by one); HS_FLAG_GREEDY_FIXED1 takes x(n, z) first
 * summed in the order i = 1..H.  H is valid while the 1-D rule holds for n (H n <= n_bins - 1 for
 * HS_FBIN, every H at n = 0; H (n + 1) <= n_bins - 1 for HS_MAX and HS_GREEDY, <= n_bins under
 * HS_FLAG_GREEDY_FIXED1) and H z lies within the plane's rows.  The paper writes Eq. 2-4 in 1-D only;
 * the drift i z of harmonic i follows the 2-D form of Eq. 1.  Calibrate with hs_noise_calibration
 * (the per-row statistics are the 1-D ones).  The plan must include v. */
hs_status hs_sum_2d_variant(const hs_plan* plan, hs_variant v, const void* d_plane, int64_t n_bins,
                            int64_t row_stride, uint32_t plane_id, const hs_out2d* out, void* d_ws, size_t ws_bytes,
                            cudaStream_t stream);

/* ---- adjoint ---------------------------------------------------------------------------- */

/* Adjoint of best_snr with respect to x, with each bin's best H held fixed (the routing of the
 * forward pass):  d_grad_x[m] += sum_n d_grad_snr[n] * c_H* * isig_H* * #{terms of S_H*(n)
 * reading bin m}.  Eq. 1 and 3 read fixed bins; Eq. 2 the first maximum of each window
 * (recomputed from d_x); Eq. 4 the bins recorded in d_path (required for HS_GREEDY).
 * d_offsets NULL means one spectrum of n_bins; otherwise a packed batch as in hs_sum_batched.
 * d_grad_x is FP32, packed like d_x, and accumulated into with atomics (the caller zeroes it;
 * summation order, hence the last bits, is not deterministic). */
hs_status hs_backward(const hs_plan* plan, hs_variant v, const void* d_x, const int64_t* d_offsets,
                      int n_spectra, int64_t n_bins, const float* d_grad_snr, const uint8_t* d_best_h,
                      const uint32_t* d_path, float* d_grad_x, cudaStream_t stream);

/* ---- reduced-precision storage ---------------------------------------------------------- */

/* y = (p - mu_s) / sigma_s in FP32 (IEEE division), stored as FP16 or BF16 rounded to nearest
 * even.  d_mu / d_sigma: device float[n_spectra] (per spectrum of the packed batch described by
 * d_offsets; d_offsets NULL means one spectrum of n_bins).  dst_dtype is HS_F16 or HS_BF16. */
hs_status hs_standardize_cast(const float* d_p, const int64_t* d_offsets, int n_spectra, int64_t n_bins,
                              const float* d_mu, const float* d_sigma, hs_dtype dst_dtype, void* d_out,
                              cudaStream_t stream);

/* ---- the step before the sums: power, dereddening, standardisation -------------------------- */

/* The input of the sums from a complex spectrum (the paper sums a power spectrum and does not say how
 * it is normalised; this is the block-median reading):
 *   P_k = re_k^2 + im_k^2 (FP32);  m_j = the lower median of P over block j of `block` bins (rank
 *   floor((size - 1)/2)); base_k = the straight line between the centres of the two nearest blocks
 *   (flat before the first centre and after the last); x_k = P_k ln2 / base_k - 1 (Exp-distributed
 *   power has mean median / ln 2), 0 where base_k <= 0; stored in the plan's dtype (RNE).
 * d_spec: device float pairs (re, im); spectrum s holds complex bins [offsets[s], offsets[s+1]) of
 * the packed batch (16-byte aligned starts: even offsets), or, with d_offsets NULL, one spectrum of
 * n_bins.  block: 32, 64, 128 or 256.  d_medians: device float[medians_capacity] receiving the
 * block medians, spectrum s's from sum_{r<s} ceil(len_r / block) on; a batch whose medians do not
 * fit is reported by hs_sync_status (HS_ERR_INVALID) and its spectra left unwritten.  d_out: the
 * plan's dtype, packed like d_spec (one value per complex bin), ready for hs_sum_batched.  The
 * workspace is the plan's (hs_plan_workspace_size for n_spectra). */
hs_status hs_power_normalize(const hs_plan* plan, const float* d_spec, const int64_t* d_offsets, int n_spectra,
                             int64_t n_bins, int block, float* d_medians, int64_t medians_capacity, void* d_out,
                             void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* ---- candidates ------------------------------------------------------------------------- */

/* Sort the first min(count, capacity) candidates in place by (variant, spectrum, z, bin), on the
 * device.  d_count is read on the device; d_tmp must hold capacity candidates. */
hs_status hs_sort_candidates(hs_candidate* d_cand, const unsigned long long* d_count, int64_t capacity,
                             hs_candidate* d_tmp, void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* Sift a sorted candidate list (the step after the sums): within each (variant, spectrum) group, drop
 * every candidate to which a stronger candidate of the group is related.  A candidate's fundamental
 * is (bin / H, z / H) for Eq. 1 and its 2-D form (they report the H-th harmonic) and (bin, z) for
 * Eq. 2-4; two candidates are related when, for some k = 1..kmax, the higher fundamental lies within
 * k*tol_bins bins and k*tol_z drift rows of k times the lower one (harmonics and neighbouring bins).
 * Stronger: larger snr, or equal snr and earlier in the list.  Comparisons in FP32, each operation
 * rounded.  d_cand: min(count, capacity) candidates sorted by hs_sort_candidates; the kept ones go
 * to d_out, sorted the same way, and their number to d_out_count (set on the device).  d_out and
 * d_tmp hold capacity candidates; the workspace is the sort's.  O(g^2) comparisons per group of g. */
hs_status hs_sift_candidates(const hs_candidate* d_cand, const unsigned long long* d_count, int64_t capacity,
                             float tol_bins, float tol_z, int kmax, hs_candidate* d_out,
                             unsigned long long* d_out_count, hs_candidate* d_tmp, void* d_ws, size_t ws_bytes,
                             cudaStream_t stream);

/* ---- CUDA graphs -------------------------------------------------------------------------- */

typedef struct hs_graph hs_graph; /* an instantiated CUDA graph plus the arguments it was built for */

/* Capture hs_sum_batched (for every variant bit set in variant_mask, in the order STD, MAX,
 * FBIN, GREEDY, each writing to outs[k] for the k-th set bit) into a CUDA graph on the stream.
 * Pointers are baked in: replaying reads the current contents of the same buffers. */
hs_status hs_graph_create_batched(const hs_plan* plan, int variant_mask, const void* d_x, const int64_t* d_offsets,
                                  int n_spectra, uint32_t first_id, const hs_out* outs, void* d_ws, size_t ws_bytes,
                                  cudaStream_t stream, hs_graph** graph);
hs_status hs_graph_launch(hs_graph* graph, cudaStream_t stream);
hs_status hs_graph_destroy(hs_graph* graph);

/* ---- tuning and status ------------------------------------------------------------------ */

/* Time the tile shapes of one variant and keep the fastest in the plan.  d_scratch (caller-owned)
 * starts with one spectrum of n_bins elements of the plan's dtype; the tuner replicates it into a
 * batch of 8 spectra and times hs_sum_batched on it, so d_scratch must hold 8 * n_bins * (element
 * size + 9) bytes plus 1 KiB, and the workspace must be sized for 8 spectra.  Results are cached in
 * the JSON file named by HS_AUTOTUNE_CACHE (if set); a cached entry is used without timing. */
hs_status hs_autotune(hs_plan* plan, hs_variant v, int64_t n_bins, void* d_scratch, size_t scratch_bytes,
                      void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* Tune on the caller's own batch (same arguments as hs_sum_batched, outputs overwritten, candidates
 * untouched): each tile shape is timed twice on exactly this work and the fastest kept in the plan.
 * Synchronises the stream. */
hs_status hs_autotune_batched(hs_plan* plan, hs_variant v, const void* d_x, const int64_t* d_offsets, int n_spectra,
                              const hs_out* out, void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* Output bins per work item (tile) the plan currently uses for a variant (0 for a bad argument). */
int hs_plan_tile_bins(const hs_plan* plan, hs_variant v);

/* Set the tile of a variant to tile_bins output bins (a multiple of 256, at most 16384), e.g. a value
 * an earlier tuning run reported.  HS_ERR_INVALID otherwise. */
hs_status hs_plan_set_tile_bins(hs_plan* plan, hs_variant v, int tile_bins);

/* Batched calls run one persistent launch per variant, by default with as many 256-thread CTAs per SM
 * as fit, so launches on other streams wait for its end.  A cap of 1..HS_MAX_CTAS_PER_SM CTAs per SM
 * (0 restores the default) leaves room on every SM for a launch on another stream, e.g. Eq. 3 or 4
 * beside Eq. 1; the results do not depend on it.  hs_plan_ctas_per_sm returns the cap (-1 for a bad
 * argument); the setter returns HS_ERR_INVALID outside 0..HS_MAX_CTAS_PER_SM. */
#define HS_MAX_CTAS_PER_SM 8
int hs_plan_ctas_per_sm(const hs_plan* plan, hs_variant v);
hs_status hs_plan_set_ctas_per_sm(hs_plan* plan, hs_variant v, int ctas_per_sm);

/* Synchronise the stream and return the device status word of the workspace: HS_OK,
 * HS_WARN_CAND_OVERFLOW or HS_ERR_TIMEOUT.  Also reports a pending CUDA error as HS_ERR_CUDA. */
hs_status hs_sync_status(const hs_plan* plan, const void* d_ws, cudaStream_t stream);

/* Human-readable name of a status code (static string). */
const char* hs_status_string(hs_status s);

/* Library version, as major*10000 + minor*100 + patch. */
int hs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HARMONIC_SUM_H */

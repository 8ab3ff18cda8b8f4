// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/harmonic_sum.h"

namespace hs {

constexpr int kHmax = HS_HMAX_1D;
constexpr int kBlock = 256;  // threads per CTA of the 1-D kernels

// status-word bits (device, in the workspace)
constexpr unsigned kStatusOverflow = 1u;
constexpr unsigned kStatusTimeout = 2u;
constexpr unsigned kStatusBadInput = 4u;

// Workspace layout: [0, 256) control words, then tile prefix sums (int64[n_spectra + 1]).
struct WsControl {
    unsigned int status;
    unsigned int queue;  // next work item of the persistent kernel
    unsigned long long total_items;
};
constexpr size_t kWsControlBytes = 256;

inline size_t ws_bytes_for(int n_spectra) {
    return kWsControlBytes + sizeof(int64_t) * (size_t)(n_spectra + 2);
}

// Eq. 1 over 16-bit storage in a batch widens up to kStageSpectra spectra at a time into FP32 in the
// workspace, after the prefix sums, and runs the FP32 kernel on them.
constexpr int kStageSpectra = 64;
inline size_t stage_offset(int n_spectra) {
    return (ws_bytes_for(n_spectra) + 255) & ~(size_t)255;
}
inline size_t stage_bytes(int n_spectra, int64_t max_bins) {
    const int g = n_spectra < kStageSpectra ? n_spectra : kStageSpectra;
    return (size_t)(g < 1 ? 1 : g) * (size_t)max_bins * sizeof(float);
}

// Scale and calibration of one variant: snr_H = (S_H * c[H] - mu[H]) * isig[H].
struct Tables {
    float c[kHmax + 1];
    float mu[kHmax + 1];
    float isig[kHmax + 1];
};

struct Out1d {
    float* best_snr;
    uint8_t* best_h;
    uint32_t* path;
    float* all_h;
    hs_candidate* cand;
    unsigned long long* cand_count;
    long long cand_cap;
};

// What one launch works on: either a single spectrum (offsets == nullptr, n_bins) or a batch.
struct Work1d {
    const void* x;
    const int64_t* offsets;  // device, n_spectra + 1 (batched) or nullptr
    int64_t n_bins;          // single spectrum length
    int n_spectra;
    uint32_t first_id;
    int hmax;
    float threshold;
    int opt;        // outputs per thread; a tile is kBlock * opt output bins
    int64_t max_bins;
    int flags;        // plan flags (HS_FLAG_*)
    int ctas_per_sm;  // persistent batched launches: CTAs per SM (0: as many as fit)
    float* stage;     // FP32 staging of 16-bit spectra for Eq. 1 (batched calls), or nullptr
};

struct Launch {
    int opt;          // outputs per thread
    int ctas_per_sm;  // 0: as many as fit
};

// Grid of a persistent launch: occ CTAs fit on an SM; a plan may ask for fewer, so that launches on
// other streams find room beside it.
inline unsigned persistent_grid(int sm_count, int occ, int ctas_per_sm) {
    const int k = ctas_per_sm > 0 && ctas_per_sm < occ ? ctas_per_sm : occ;
    return (unsigned)(sm_count * (k > 0 ? k : 1));
}

// Values worth computing once per device (occupancies, function attributes): slot d of an array of
// kMaxDevices belongs to device ordinal d.  A device ordinal beyond the table shares slot 0.
constexpr int kMaxDevices = 64;
inline int device_slot() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) d = 0;
    return d;
}

// Zone tiling of Eq. 2-4 (hs_1d.cu): variant (0 = plain tiles), hmax, plan flags, tile parameter.
struct ZoneSpec {
    int v, hmax, flags, opt;
};

}  // namespace hs

struct hs_plan {
    hs_plan_desc d;
    hs::Tables tab[4];  // indexed by variant bit position (STD, MAX, FBIN, GREEDY)
    hs::Launch launch[4];
    int sm_count;
};

namespace hs {

inline int vindex(hs_variant v) {
    switch (v) {
        case HS_STD: return 0;
        case HS_MAX: return 1;
        case HS_FBIN: return 2;
        case HS_GREEDY: return 3;
    }
    return -1;
}

// kernels (hs_1d.cu)
cudaError_t launch_1d(hs_variant v, hs_dtype dt, const Tables& tab, const Work1d& w, const Out1d& o,
                      WsControl* ctl, int64_t* tile_prefix, int sm_count, cudaStream_t s);

void warm_1d(hs_variant v, hs_dtype dt);

// tile prefix sums of a batch and reset of its work queue (hs_1d.cu)
void launch_tile_scan(const int64_t* offsets, int n_spectra, int64_t tile, int64_t max_bins, int elem_bytes,
                      int64_t* prefix, WsControl* ctl, cudaStream_t s);

// Eq. 1 over a batch with the input spans staged in shared memory (hs_1d_staged.cu): taken under
// HS_FLAG_STAGED_SPANS for hmax = 32 without the every-H table
bool eq1_staged_applies(const Work1d& w, const Out1d& o);
cudaError_t launch_eq1_staged(hs_dtype dt, const Tables& tab, const Work1d& w, const Out1d& o, WsControl* ctl,
                              int64_t* prefix, int sm_count, cudaStream_t s);
void warm_eq1_staged(hs_dtype dt);

// 2-D (hs_2d.cu)
struct Work2d {
    const float* plane;
    int64_t n_bins, row_stride;
    int nz, z_min, hmax;
    uint32_t plane_id;
    float threshold;
    int flags;  // plan flags (HS_FLAG_MAX_WINDOW0, HS_FLAG_GREEDY_FIXED1 for the row-wise forms)
};
cudaError_t launch_2d(hs_variant v, const Tables& tab, const Work2d& w, const hs_out2d& o, long long cand_cap,
                      WsControl* ctl, cudaStream_t s);

// adjoint (hs_adjoint.cu)
cudaError_t launch_backward(hs_variant v, hs_dtype dt, const Tables& tab, const void* x, const int64_t* offsets,
                            int n_spectra, int64_t n_bins, int hmax, int flags, const float* g, const uint8_t* best_h,
                            const uint32_t* path, float* grad, cudaStream_t s);

// auxiliaries (hs_aux.cu)
cudaError_t launch_standardize_cast(const float* p, const int64_t* offsets, int n_spectra, int64_t n_bins,
                                    const float* mu, const float* sigma, hs_dtype dt, void* out, cudaStream_t s);
cudaError_t launch_power_normalize(const float* spec, const int64_t* offsets, int n_spectra, int64_t n_bins, int block,
                                   float* medians, long long med_cap, hs_dtype dt, void* out, int64_t max_bins,
                                   int sm_count, int64_t* prefix, WsControl* ctl, cudaStream_t s);
cudaError_t launch_sift_candidates(const hs_candidate* cand, const unsigned long long* count, int64_t capacity,
                                   float tol, float tol_z, int kmax, hs_candidate* out,
                                   unsigned long long* out_count, hs_candidate* tmp, WsControl* ctl,
                                   cudaStream_t s);
cudaError_t launch_sort_candidates(hs_candidate* cand, const unsigned long long* count, int64_t capacity,
                                   hs_candidate* tmp, WsControl* ctl, cudaStream_t s);

}  // namespace hs

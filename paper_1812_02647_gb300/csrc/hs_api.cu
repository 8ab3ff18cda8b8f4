// The C ABI: plan, validation, workspace, dispatch to the kernels, CUDA-graph capture, status.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hs_internal.cuh"

namespace hs {
size_t sort_scratch_bytes(int64_t capacity);
}

using namespace hs;

namespace {

constexpr int kPlanFlags = HS_FLAG_OUT_ALL_H | HS_FLAG_STAGED_SPANS | HS_FLAG_MAX_WINDOW0 | HS_FLAG_POW2_STAGES |
                           HS_FLAG_GREEDY_FIXED1 | HS_FLAG_CHECK_TIMEOUT;

bool single_variant(int v) { return v == HS_STD || v == HS_MAX || v == HS_FBIN || v == HS_GREEDY; }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

int current_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

hs_status check_cuda(cudaError_t e) { return e == cudaSuccess ? HS_OK : HS_ERR_CUDA; }

hs_status check_ws(const hs_plan* p, int n_spectra, const void* d_ws, size_t ws_bytes) {
    size_t need = 0;
    hs_plan_workspace_size(p, n_spectra, &need);
    if (!d_ws) return HS_ERR_INVALID;
    if (!aligned(d_ws, 256)) return HS_ERR_ALIGN;
    if (ws_bytes < need) return HS_ERR_NOMEM;
    return HS_OK;
}

hs_status check_out(const hs_plan* p, hs_variant v, const hs_out* o, bool batched) {
    if (!o || !o->best_snr || !o->best_h) return HS_ERR_INVALID;
    if (!aligned(o->best_snr, 4)) return HS_ERR_ALIGN;
    if (o->path && !aligned(o->path, 4)) return HS_ERR_ALIGN;
    if (o->all_h) {
        if (batched || !(p->d.flags & HS_FLAG_OUT_ALL_H)) return HS_ERR_INVALID;
        if (!aligned(o->all_h, 4)) return HS_ERR_ALIGN;
    }
    if (o->cand) {
        if (!o->cand_count || p->d.cand_capacity <= 0) return HS_ERR_INVALID;
        if (!aligned(o->cand, 16) || !aligned(o->cand_count, 8)) return HS_ERR_ALIGN;
    }
    (void)v;
    return HS_OK;
}

Out1d make_out(const hs_plan* p, hs_variant v, const hs_out* o) {
    Out1d r;
    r.best_snr = o->best_snr;
    r.best_h = o->best_h;
    r.path = v == HS_GREEDY ? o->path : nullptr;
    r.all_h = o->all_h;
    r.cand = o->cand;
    r.cand_count = o->cand_count;
    r.cand_cap = p->d.cand_capacity;
    return r;
}

}  // namespace

extern "C" {

const char* hs_status_string(hs_status s) {
    switch (s) {
        case HS_OK: return "HS_OK";
        case HS_ERR_INVALID: return "HS_ERR_INVALID: invalid argument";
        case HS_ERR_ALIGN: return "HS_ERR_ALIGN: pointer not aligned";
        case HS_ERR_CUDA: return "HS_ERR_CUDA: CUDA runtime error";
        case HS_ERR_NOMEM: return "HS_ERR_NOMEM: out of memory or workspace too small";
        case HS_ERR_TIMEOUT: return "HS_ERR_TIMEOUT: a bounded device wait gave up";
        case HS_ERR_UNSUPPORTED: return "HS_ERR_UNSUPPORTED: not implemented for these arguments";
        case HS_WARN_CAND_OVERFLOW: return "HS_WARN_CAND_OVERFLOW: more candidates than capacity";
    }
    return "unknown hs_status";
}

int hs_version(void) { return 100; }

hs_status hs_plan_create(hs_plan** plan, const hs_plan_desc* d) {
    if (!plan || !d) return HS_ERR_INVALID;
    *plan = nullptr;
    if (d->variants <= 0 || (d->variants & ~0xF) != 0) return HS_ERR_INVALID;
    if (d->dtype != HS_F32 && d->dtype != HS_F16 && d->dtype != HS_BF16) return HS_ERR_INVALID;
    if (d->nz < 0) return HS_ERR_INVALID;
    const int hcap = d->nz > 0 ? HS_HMAX_2D : HS_HMAX_1D;
    if (d->hmax < 1 || d->hmax > hcap) return HS_ERR_INVALID;
    if (d->max_bins < 0 || d->max_bins > HS_MAX_BINS_1D) return HS_ERR_INVALID;
    if (d->nz > 0 && (d->z_min > 0 || d->z_min + d->nz - 1 < 0 || d->nz > 32767)) return HS_ERR_INVALID;
    if (d->cand_capacity < 0 || (d->flags & ~kPlanFlags) != 0 || (d->nz != 0 && (d->flags & HS_FLAG_POW2_STAGES))) return HS_ERR_INVALID;
    if (std::isnan(d->threshold)) return HS_ERR_INVALID;
    hs_plan* p = new (std::nothrow) hs_plan;
    if (!p) return HS_ERR_NOMEM;
    p->d = *d;
    for (int k = 0; k < 4; ++k) {
        for (int H = 0; H <= kHmax; ++H) {
            p->tab[k].c[H] = H == 0 ? 0.f : (float)(1.0 / std::sqrt((double)H));
            p->tab[k].mu[H] = 0.f;
            p->tab[k].isig[H] = 1.f;
        }
    }
    p->launch[0].opt = 4;  // Eq. 1
    p->launch[1].opt = 4;  // Eq. 2
    p->launch[2].opt = 8;  // Eq. 3
    p->launch[3].opt = 8;  // Eq. 4
    for (int k = 0; k < 4; ++k) p->launch[k].ctas_per_sm = 0;  // as many CTAs per SM as fit
    p->sm_count = 0;
    *plan = p;
    return HS_OK;
}

hs_status hs_plan_destroy(hs_plan* plan) {
    delete plan;
    return HS_OK;
}

hs_status hs_plan_set_calibration(hs_plan* p, hs_variant v, const float* mu, const float* isig) {
    if (!p || !single_variant(v)) return HS_ERR_INVALID;
    if ((mu == nullptr) != (isig == nullptr)) return HS_ERR_INVALID;
    Tables& t = p->tab[vindex(v)];
    for (int H = 0; H <= kHmax; ++H) {
        bool have = mu && H <= p->d.hmax;
        t.mu[H] = have ? mu[H] : 0.f;
        t.isig[H] = have ? isig[H] : 1.f;
        if (have && (!std::isfinite(t.mu[H]) || !std::isfinite(t.isig[H]))) {
            for (int k = 0; k <= kHmax; ++k) {
                t.mu[k] = 0.f;
                t.isig[k] = 1.f;
            }
            return HS_ERR_INVALID;
        }
    }
    return HS_OK;
}

hs_status hs_noise_calibration(hs_variant v, int hmax, float* mu, float* isig) {
    return hs_noise_calibration_flags(v, hmax, 0, mu, isig);
}

hs_status hs_noise_calibration_flags(hs_variant v, int hmax, int flags, float* mu, float* isig) {
    if (!single_variant(v) || !mu || !isig || hmax < 1 || hmax > HS_HMAX_1D) return HS_ERR_INVALID;
    if ((flags & ~kPlanFlags) != 0) return HS_ERR_INVALID;
    const int extra = (flags & HS_FLAG_MAX_WINDOW0) ? 1 : 0;  // Eq. 2 window of i + extra bins
    // standardised Exp(1) noise, bins far enough from 0 that every read is a distinct bin
    double hn = 0.0, hn2 = 0.0, mean_sum = 0.0, var_sum = 0.0;
    mu[0] = 0.f;
    isig[0] = 1.f;
    for (int H = 1; H <= hmax; ++H) {
        double m = 0.0, sd = 1.0;
        if (v == HS_MAX) {
            // mean and variance of the max of w = H + extra unit exponentials: Hn(w), sum_{k<=w} k^-2
            if (H == 1 && extra) {
                hn = 1.0;
                hn2 = 1.0;
            }
            const double wn = H + extra;
            hn += 1.0 / wn;
            hn2 += 1.0 / (wn * wn);
            mean_sum += hn - 1.0;
            var_sum += hn2;
            m = mean_sum / std::sqrt((double)H);
            sd = std::sqrt(var_sum / H);
        } else if (v == HS_GREEDY && (flags & HS_FLAG_GREEDY_FIXED1)) {
            m = 0.5 * (H - 1) / std::sqrt((double)H);  // one bin, then H - 1 maxima of two
            sd = std::sqrt((1.0 + 1.25 * (H - 1)) / H);
        } else if (v == HS_GREEDY) {
            m = 0.5 * std::sqrt((double)H);  // max of two unit exponentials: mean 3/2, variance 5/4
            sd = std::sqrt(1.25);
        }
        mu[H] = (float)m;
        isig[H] = (float)(1.0 / sd);
    }
    return HS_OK;
}

// Eq. 1 of a 16-bit plan runs batches through an FP32 copy of up to kStageSpectra spectra at a time
// (the FP32 pair kernel is faster than any 16-bit form of it measured), held in the workspace.
static bool stages_eq1(const hs_plan* p) {
    return p->d.dtype != HS_F32 && (p->d.variants & HS_STD) && p->d.hmax == kHmax &&
           !(p->d.flags & HS_FLAG_STAGED_SPANS);
}

hs_status hs_plan_workspace_size(const hs_plan* p, int n_spectra, size_t* bytes) {
    if (!p || !bytes || n_spectra < 0) return HS_ERR_INVALID;
    const int ns = n_spectra < 1 ? 1 : n_spectra;
    size_t a = ws_bytes_for(ns);
    if (stages_eq1(p)) a = stage_offset(ns) + stage_bytes(ns, p->d.max_bins);
    size_t b = sort_scratch_bytes(p->d.cand_capacity);
    *bytes = (a > b ? a : b + 0);
    *bytes = (*bytes + 255) & ~(size_t)255;
    return HS_OK;
}

hs_status hs_workspace_init(const hs_plan* p, void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (!p || !d_ws || ws_bytes < kWsControlBytes) return HS_ERR_INVALID;
    if (!aligned(d_ws, 256)) return HS_ERR_ALIGN;
    return check_cuda(cudaMemsetAsync(d_ws, 0, kWsControlBytes, stream));
}

static hs_status ensure_sm_count(const hs_plan* p) {
    if (p->sm_count <= 0) {
        int n = current_sm_count();
        if (n <= 0) return HS_ERR_CUDA;
        const_cast<hs_plan*>(p)->sm_count = n;
    }
    return HS_OK;
}

hs_status hs_sum_1d(const hs_plan* p, hs_variant v, const void* d_x, int64_t n_bins, uint32_t spectrum_id,
                    const hs_out* out, void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (!p || !single_variant(v) || !(p->d.variants & v) || p->d.nz != 0) return HS_ERR_INVALID;
    if (n_bins < 0 || n_bins > p->d.max_bins) return HS_ERR_INVALID;
    if (!d_x) return HS_ERR_INVALID;
    if (!aligned(d_x, 16)) return HS_ERR_ALIGN;
    hs_status st = check_out(p, v, out, false);
    if (st != HS_OK) return st;
    if ((st = check_ws(p, 1, d_ws, ws_bytes)) != HS_OK) return st;
    if ((st = ensure_sm_count(p)) != HS_OK) return st;
    Work1d w{};
    w.x = d_x;
    w.offsets = nullptr;
    w.n_bins = n_bins;
    w.n_spectra = 1;
    w.first_id = spectrum_id;
    w.hmax = p->d.hmax;
    w.threshold = p->d.threshold;
    w.opt = p->launch[vindex(v)].opt;
    w.ctas_per_sm = p->launch[vindex(v)].ctas_per_sm;
    w.max_bins = p->d.max_bins;
    w.flags = p->d.flags;
    WsControl* ctl = reinterpret_cast<WsControl*>(d_ws);
    int64_t* prefix = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(d_ws) + kWsControlBytes);
    return check_cuda(launch_1d(v, p->d.dtype, p->tab[vindex(v)], w, make_out(p, v, out), ctl, prefix,
                                p->sm_count, stream));
}

hs_status hs_sum_batched(const hs_plan* p, hs_variant v, const void* d_x, const int64_t* d_offsets, int n_spectra,
                         uint32_t first_id, const hs_out* out, void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (!p || !single_variant(v) || !(p->d.variants & v) || p->d.nz != 0) return HS_ERR_INVALID;
    if (n_spectra < 0 || !d_x || !d_offsets) return HS_ERR_INVALID;
    if (!aligned(d_x, 16) || !aligned(d_offsets, 8)) return HS_ERR_ALIGN;
    hs_status st = check_out(p, v, out, true);
    if (st != HS_OK) return st;
    if ((st = check_ws(p, n_spectra, d_ws, ws_bytes)) != HS_OK) return st;
    if (n_spectra == 0) return HS_OK;
    if ((st = ensure_sm_count(p)) != HS_OK) return st;
    Work1d w{};
    w.x = d_x;
    w.offsets = d_offsets;
    w.n_bins = 0;
    w.n_spectra = n_spectra;
    w.first_id = first_id;
    w.hmax = p->d.hmax;
    w.threshold = p->d.threshold;
    w.opt = p->launch[vindex(v)].opt;
    w.ctas_per_sm = p->launch[vindex(v)].ctas_per_sm;
    w.max_bins = p->d.max_bins;
    w.flags = p->d.flags;
    w.stage = (v == HS_STD && stages_eq1(p))
                  ? reinterpret_cast<float*>(reinterpret_cast<char*>(d_ws) + stage_offset(n_spectra))
                  : nullptr;
    WsControl* ctl = reinterpret_cast<WsControl*>(d_ws);
    int64_t* prefix = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(d_ws) + kWsControlBytes);
    return check_cuda(launch_1d(v, p->d.dtype, p->tab[vindex(v)], w, make_out(p, v, out), ctl, prefix,
                                p->sm_count, stream));
}

hs_status hs_sum_2d(const hs_plan* p, const void* d_plane, int64_t n_bins, int64_t row_stride, uint32_t plane_id,
                    const hs_out2d* out, void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    return hs_sum_2d_variant(p, HS_STD, d_plane, n_bins, row_stride, plane_id, out, d_ws, ws_bytes, stream);
}

hs_status hs_sum_2d_variant(const hs_plan* p, hs_variant v, const void* d_plane, int64_t n_bins, int64_t row_stride,
                            uint32_t plane_id, const hs_out2d* out, void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (!p || p->d.nz <= 0 || !single_variant(v) || !(p->d.variants & v)) return HS_ERR_INVALID;
    if (p->d.dtype != HS_F32) return HS_ERR_UNSUPPORTED;
    if (!d_plane || n_bins < 0 || n_bins > p->d.max_bins || row_stride < n_bins) return HS_ERR_INVALID;
    if (!aligned(d_plane, 16) || (row_stride * 4) % 16 != 0) return HS_ERR_ALIGN;
    if (!out || !out->best_snr || !out->best_h || !out->best_snr_n || !out->best_h_n || !out->best_z_n)
        return HS_ERR_INVALID;
    if (out->cand && (!out->cand_count || p->d.cand_capacity <= 0)) return HS_ERR_INVALID;
    if (out->cand && (!aligned(out->cand, 16) || !aligned(out->cand_count, 8))) return HS_ERR_ALIGN;
    hs_status st = check_ws(p, 1, d_ws, ws_bytes);
    if (st != HS_OK) return st;
    Work2d w{};
    w.plane = reinterpret_cast<const float*>(d_plane);
    w.n_bins = n_bins;
    w.row_stride = row_stride;
    w.nz = p->d.nz;
    w.z_min = p->d.z_min;
    w.hmax = p->d.hmax;
    w.plane_id = plane_id;
    w.threshold = p->d.threshold;
    w.flags = p->d.flags;
    return check_cuda(launch_2d(v, p->tab[vindex(v)], w, *out, p->d.cand_capacity, reinterpret_cast<WsControl*>(d_ws),
                                stream));
}

hs_status hs_backward(const hs_plan* p, hs_variant v, const void* d_x, const int64_t* d_offsets, int n_spectra,
                      int64_t n_bins, const float* d_grad_snr, const uint8_t* d_best_h, const uint32_t* d_path,
                      float* d_grad_x, cudaStream_t stream) {
    if (!p || !single_variant(v) || !(p->d.variants & v) || p->d.nz != 0) return HS_ERR_INVALID;
    if (!d_x || !d_grad_snr || !d_best_h || !d_grad_x || (v == HS_GREEDY && !d_path)) return HS_ERR_INVALID;
    if (!aligned(d_x, 16) || !aligned(d_grad_snr, 4) || !aligned(d_grad_x, 4)) return HS_ERR_ALIGN;
    if (d_offsets) {
        if (n_spectra < 0 || n_spectra > 65535) return HS_ERR_INVALID;
        n_bins = p->d.max_bins;
    } else {
        if (n_bins < 0 || n_bins > p->d.max_bins) return HS_ERR_INVALID;
        n_spectra = 1;
    }
    if (n_spectra == 0) return HS_OK;
    return check_cuda(launch_backward(v, p->d.dtype, p->tab[vindex(v)], d_x, d_offsets, n_spectra, n_bins,
                                      p->d.hmax, p->d.flags, d_grad_snr, d_best_h, d_path, d_grad_x, stream));
}

hs_status hs_power_normalize(const hs_plan* p, const float* d_spec, const int64_t* d_offsets, int n_spectra,
                             int64_t n_bins, int block, float* d_medians, int64_t medians_capacity, void* d_out,
                             void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (!p || p->d.nz != 0 || !d_spec || !d_medians || !d_out || medians_capacity < 0) return HS_ERR_INVALID;
    if (block != 32 && block != 64 && block != 128 && block != 256) return HS_ERR_INVALID;
    if (!aligned(d_spec, 16) || !aligned(d_medians, 4) || !aligned(d_out, 16)) return HS_ERR_ALIGN;
    if (d_offsets) {
        if (n_spectra < 0 || n_spectra > 65535 || !aligned(d_offsets, 8)) return HS_ERR_INVALID;
    } else {
        if (n_bins < 0 || n_bins > p->d.max_bins) return HS_ERR_INVALID;
        n_spectra = 1;
    }
    hs_status st = check_ws(p, n_spectra, d_ws, ws_bytes);
    if (st != HS_OK) return st;
    if (n_spectra == 0 || (!d_offsets && n_bins == 0)) return HS_OK;
    if ((st = ensure_sm_count(p)) != HS_OK) return st;
    WsControl* ctl = reinterpret_cast<WsControl*>(d_ws);
    int64_t* prefix = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(d_ws) + kWsControlBytes);
    return check_cuda(launch_power_normalize(d_spec, d_offsets, n_spectra, n_bins, block, d_medians,
                                             (long long)medians_capacity, p->d.dtype, d_out, p->d.max_bins,
                                             p->sm_count, prefix, ctl, stream));
}

hs_status hs_standardize_cast(const float* d_p, const int64_t* d_offsets, int n_spectra, int64_t n_bins,
                              const float* d_mu, const float* d_sigma, hs_dtype dst, void* d_out,
                              cudaStream_t stream) {
    if (!d_p || !d_mu || !d_sigma || !d_out || (dst != HS_F16 && dst != HS_BF16)) return HS_ERR_INVALID;
    if (!aligned(d_p, 16) || !aligned(d_out, 16)) return HS_ERR_ALIGN;
    if (d_offsets) {
        if (n_spectra < 0 || n_spectra > 65535 || n_bins < 0) return HS_ERR_INVALID;
    } else {
        if (n_bins < 0) return HS_ERR_INVALID;
        n_spectra = 1;
    }
    return check_cuda(launch_standardize_cast(d_p, d_offsets, n_spectra, n_bins, d_mu, d_sigma, dst, d_out, stream));
}

hs_status hs_sort_candidates(hs_candidate* d_cand, const unsigned long long* d_count, int64_t capacity,
                             hs_candidate* d_tmp, void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (!d_cand || !d_count || !d_tmp || capacity < 0 || !d_ws) return HS_ERR_INVALID;
    if (!aligned(d_cand, 16) || !aligned(d_tmp, 16) || !aligned(d_ws, 256)) return HS_ERR_ALIGN;
    if (ws_bytes < sort_scratch_bytes(capacity)) return HS_ERR_NOMEM;
    return check_cuda(launch_sort_candidates(d_cand, d_count, capacity, d_tmp, reinterpret_cast<WsControl*>(d_ws),
                                             stream));
}

hs_status hs_sift_candidates(const hs_candidate* d_cand, const unsigned long long* d_count, int64_t capacity,
                             float tol_bins, float tol_z, int kmax, hs_candidate* d_out,
                             unsigned long long* d_out_count, hs_candidate* d_tmp, void* d_ws, size_t ws_bytes,
                             cudaStream_t stream) {
    if (!d_cand || !d_count || !d_out || !d_out_count || !d_tmp || !d_ws || capacity < 0) return HS_ERR_INVALID;
    if (!(tol_bins >= 0.f) || !(tol_z >= 0.f) || !std::isfinite(tol_bins) || !std::isfinite(tol_z) || kmax < 1 ||
        kmax > 64 || d_out == d_cand)
        return HS_ERR_INVALID;
    if (!aligned(d_cand, 16) || !aligned(d_out, 16) || !aligned(d_tmp, 16) || !aligned(d_ws, 256)) return HS_ERR_ALIGN;
    if (ws_bytes < sort_scratch_bytes(capacity)) return HS_ERR_NOMEM;
    return check_cuda(launch_sift_candidates(d_cand, d_count, capacity, tol_bins, tol_z, kmax, d_out, d_out_count,
                                             d_tmp, reinterpret_cast<WsControl*>(d_ws), stream));
}

struct hs_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

hs_status hs_graph_create_batched(const hs_plan* p, int variant_mask, const void* d_x, const int64_t* d_offsets,
                                  int n_spectra, uint32_t first_id, const hs_out* outs, void* d_ws, size_t ws_bytes,
                                  cudaStream_t stream, hs_graph** graph) {
    if (!graph) return HS_ERR_INVALID;
    *graph = nullptr;
    if (!p || variant_mask <= 0 || (variant_mask & ~p->d.variants) != 0 || !outs) return HS_ERR_INVALID;
    // validate every call before capturing anything
    int k = 0;
    for (int b = 0; b < 4; ++b) {
        hs_variant v = (hs_variant)(1 << b);
        if (!(variant_mask & v)) continue;
        hs_status st = check_out(p, v, &outs[k++], true);
        if (st != HS_OK) return st;
    }
    hs_status st = ensure_sm_count(p);
    if (st != HS_OK) return st;
    for (int b = 0; b < 4; ++b)
        if (variant_mask & (1 << b)) warm_1d((hs_variant)(1 << b), p->d.dtype);
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return HS_ERR_CUDA;
    // captured on a private stream; the graph runs where hs_graph_launch puts it
    (void)stream;
    hs_graph* g = new (std::nothrow) hs_graph;
    if (!g) {
        cudaStreamDestroy(cs);
        return HS_ERR_NOMEM;
    }
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        delete g;
        cudaStreamDestroy(cs);
        return HS_ERR_CUDA;
    }
    k = 0;
    hs_status cst = HS_OK;
    for (int b = 0; b < 4 && cst == HS_OK; ++b) {
        hs_variant v = (hs_variant)(1 << b);
        if (!(variant_mask & v)) continue;
        cst = hs_sum_batched(p, v, d_x, d_offsets, n_spectra, first_id, &outs[k++], d_ws, ws_bytes, cs);
    }
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &gr);
    cudaStreamDestroy(cs);
    if (cst != HS_OK || e != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        delete g;
        return cst != HS_OK ? cst : HS_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&g->exec, gr, 0) != cudaSuccess) {
        cudaGraphDestroy(gr);
        delete g;
        return HS_ERR_CUDA;
    }
    g->graph = gr;
    *graph = g;
    return HS_OK;
}

hs_status hs_graph_launch(hs_graph* g, cudaStream_t stream) {
    if (!g) return HS_ERR_INVALID;
    return check_cuda(cudaGraphLaunch(g->exec, stream));
}

hs_status hs_graph_destroy(hs_graph* g) {
    if (!g) return HS_OK;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return HS_OK;
}

hs_status hs_sync_status(const hs_plan* p, const void* d_ws, cudaStream_t stream) {
    if (!p || !d_ws) return HS_ERR_INVALID;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return HS_ERR_CUDA;
    unsigned status = 0;
    if (cudaMemcpy(&status, d_ws, sizeof(status), cudaMemcpyDeviceToHost) != cudaSuccess) return HS_ERR_CUDA;
    if (status & kStatusTimeout) return HS_ERR_TIMEOUT;
    if (status & kStatusBadInput) return HS_ERR_INVALID;
    if (status & kStatusOverflow) return HS_WARN_CAND_OVERFLOW;
    return HS_OK;
}

}  // extern "C"

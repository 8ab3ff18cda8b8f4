// Autotuner: times the tile shapes of one variant on the persistent batched launch and keeps the
// fastest in the plan.  Results are cached in a flat JSON object, keyed by (variant, dtype, hmax,
// log2 bins, SM count), in the file named by the HS_AUTOTUNE_CACHE environment variable.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <string>

#include "hs_internal.cuh"

using namespace hs;

namespace {

std::map<std::string, int> read_cache(const char* path) {
    std::map<std::string, int> m;
    FILE* f = path ? std::fopen(path, "r") : nullptr;
    if (!f) return m;
    char key[256];
    int val;
    int c;
    while ((c = std::fgetc(f)) != EOF) {
        if (c != '"') continue;
        int k = 0;
        while ((c = std::fgetc(f)) != EOF && c != '"' && k < 255) key[k++] = (char)c;
        key[k] = 0;
        if (std::fscanf(f, " : %d", &val) == 1) m[key] = val;
    }
    std::fclose(f);
    return m;
}

void write_cache(const char* path, const std::map<std::string, int>& m) {
    if (!path) return;
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "{\n");
    size_t i = 0;
    for (auto& kv : m) std::fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++i < m.size() ? "," : "");
    std::fprintf(f, "}\n");
    std::fclose(f);
    std::rename(tmp.c_str(), path);
}

}  // namespace

extern "C" hs_status hs_autotune(hs_plan* p, hs_variant v, int64_t n_bins, void* d_scratch, size_t scratch_bytes,
                                 void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (!p || vindex(v) < 0 || !(p->d.variants & v) || p->d.nz != 0) return HS_ERR_INVALID;
    if (n_bins < 1 || n_bins > p->d.max_bins || !d_scratch || !d_ws) return HS_ERR_INVALID;
    const size_t es = p->d.dtype == HS_F32 ? 4 : 2;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t x_b = (size_t)n_bins * es;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    char key[160];
    std::snprintf(key, sizeof key, "v%d_d%d_h%d_b%d_sm%d", (int)v, (int)p->d.dtype, p->d.hmax,
                  (int)std::ceil(std::log2((double)n_bins)), sms);
    const char* cache = std::getenv("HS_AUTOTUNE_CACHE");
    std::map<std::string, int> m = read_cache(cache);
    auto it = m.find(key);
    if (it != m.end() && it->second >= 1 && it->second <= 64) {
        p->launch[vindex(v)].opt = it->second;
        return HS_OK;
    }
    // Tune on the launch the batched entry points use: the spectrum at the start of d_scratch is
    // replicated into a batch of kTuneReplicas spectra, timed through hs_sum_batched.
    constexpr int kTuneReplicas = 8;
    const size_t xr_b = up(x_b * kTuneReplicas), o4_b = up((size_t)n_bins * 4 * kTuneReplicas),
                 o1_b = up((size_t)n_bins * kTuneReplicas), off_b = up(sizeof(int64_t) * (kTuneReplicas + 1));
    if (scratch_bytes < xr_b + 2 * o4_b + o1_b + off_b) return HS_ERR_NOMEM;
    size_t ws_need = 0;
    hs_plan_workspace_size(p, kTuneReplicas, &ws_need);
    if (ws_bytes < ws_need) return HS_ERR_NOMEM;
    char* base = reinterpret_cast<char*>(d_scratch);
    for (int r = 1; r < kTuneReplicas; ++r)
        if (cudaMemcpyAsync(base + (size_t)r * n_bins * es, base, (size_t)n_bins * es, cudaMemcpyDeviceToDevice,
                            stream) != cudaSuccess)
            return HS_ERR_CUDA;
    int64_t offs[kTuneReplicas + 1];
    for (int r = 0; r <= kTuneReplicas; ++r) offs[r] = (int64_t)r * n_bins;
    int64_t* d_offs = reinterpret_cast<int64_t*>(base + xr_b + 2 * o4_b + o1_b);
    if (cudaStreamSynchronize(stream) != cudaSuccess ||
        cudaMemcpy(d_offs, offs, sizeof(offs), cudaMemcpyHostToDevice) != cudaSuccess)
        return HS_ERR_CUDA;
    hs_out o{};
    o.best_snr = reinterpret_cast<float*>(base + xr_b);
    o.path = reinterpret_cast<uint32_t*>(base + xr_b + o4_b);
    o.best_h = reinterpret_cast<uint8_t*>(base + xr_b + 2 * o4_b);
    const int old_opt = p->launch[vindex(v)].opt;
    const int choices[] = {2, 4, 8, 16, 32, 64};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HS_ERR_CUDA;
    float best_ms = 1e30f;
    int best_opt = old_opt;
    hs_status st = HS_OK;
    for (int opt : choices) {
        p->launch[vindex(v)].opt = opt;
        if ((st = hs_sum_batched(p, v, d_scratch, d_offs, kTuneReplicas, 0, &o, d_ws, ws_bytes, stream)) != HS_OK)
            break;
        cudaEventRecord(e0, stream);
        for (int r = 0; r < 3; ++r) hs_sum_batched(p, v, d_scratch, d_offs, kTuneReplicas, 0, &o, d_ws, ws_bytes, stream);
        cudaEventRecord(e1, stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = HS_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best_opt = opt;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->launch[vindex(v)].opt = st == HS_OK ? best_opt : old_opt;
    if (st == HS_OK && cache) {
        m[key] = best_opt;
        write_cache(cache, m);
    }
    return st;
}

// Tune on the caller's own batch: every tile shape is timed with hs_sum_batched on exactly the work
// that will later be run (outputs are overwritten), twice, and the fastest kept in the plan.
extern "C" hs_status hs_autotune_batched(hs_plan* p, hs_variant v, const void* d_x, const int64_t* d_offsets,
                                         int n_spectra, const hs_out* out, void* d_ws, size_t ws_bytes,
                                         cudaStream_t stream) {
    if (!p || vindex(v) < 0 || !(p->d.variants & v) || p->d.nz != 0 || !out || n_spectra <= 0) return HS_ERR_INVALID;
    hs_out o = *out;
    o.cand = nullptr;  // timing runs do not touch the caller's candidate list
    o.cand_count = nullptr;
    const int old_opt = p->launch[vindex(v)].opt;
    const int choices[] = {2, 4, 8, 16, 32, 64};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HS_ERR_CUDA;
    float best_ms = 1e30f;
    int best_opt = old_opt;
    hs_status st = HS_OK;
    for (int opt : choices) {
        p->launch[vindex(v)].opt = opt;
        if ((st = hs_sum_batched(p, v, d_x, d_offsets, n_spectra, 0, &o, d_ws, ws_bytes, stream)) != HS_OK) break;
        for (int rep = 0; rep < 2 && st == HS_OK; ++rep) {
            cudaEventRecord(e0, stream);
            hs_sum_batched(p, v, d_x, d_offsets, n_spectra, 0, &o, d_ws, ws_bytes, stream);
            cudaEventRecord(e1, stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = HS_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best_opt = opt;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->launch[vindex(v)].opt = st == HS_OK ? best_opt : old_opt;
    return st;
}

extern "C" int hs_plan_tile_bins(const hs_plan* p, hs_variant v) {
    if (!p || vindex(v) < 0) return 0;
    return kBlock * p->launch[vindex(v)].opt;
}

extern "C" int hs_plan_ctas_per_sm(const hs_plan* p, hs_variant v) {
    if (!p || vindex(v) < 0) return -1;
    return p->launch[vindex(v)].ctas_per_sm;
}

extern "C" hs_status hs_plan_set_ctas_per_sm(hs_plan* p, hs_variant v, int ctas_per_sm) {
    if (!p || vindex(v) < 0 || ctas_per_sm < 0 || ctas_per_sm > HS_MAX_CTAS_PER_SM) return HS_ERR_INVALID;
    p->launch[vindex(v)].ctas_per_sm = ctas_per_sm;
    return HS_OK;
}

extern "C" hs_status hs_plan_set_tile_bins(hs_plan* p, hs_variant v, int tile_bins) {
    if (!p || vindex(v) < 0 || tile_bins < kBlock || tile_bins > 64 * kBlock || tile_bins % kBlock != 0)
        return HS_ERR_INVALID;
    p->launch[vindex(v)].opt = tile_bins / kBlock;
    return HS_OK;
}

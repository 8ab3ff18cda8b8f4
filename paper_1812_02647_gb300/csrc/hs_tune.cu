// Autotuner: times the tile shapes of one variant and keeps the fastest in the plan.  Results are
// cached in a flat JSON object, keyed by (variant, dtype, hmax, log2 bins, SM count), in the file
// named by the HS_AUTOTUNE_CACHE environment variable.
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
    const size_t x_b = up(n_bins * es), snr_b = up(n_bins * 4), h_b = up(n_bins), path_b = up(n_bins * 4);
    if (scratch_bytes < x_b + snr_b + h_b + path_b) return HS_ERR_NOMEM;
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
    char* base = reinterpret_cast<char*>(d_scratch);
    hs_out o{};
    o.best_snr = reinterpret_cast<float*>(base + x_b);
    o.best_h = reinterpret_cast<uint8_t*>(base + x_b + snr_b);
    o.path = reinterpret_cast<uint32_t*>(base + x_b + snr_b + h_b);
    const int old_opt = p->launch[vindex(v)].opt;
    const int choices[] = {1, 2, 4, 8, 16, 32};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HS_ERR_CUDA;
    float best_ms = 1e30f;
    int best_opt = old_opt;
    hs_status st = HS_OK;
    for (int opt : choices) {
        p->launch[vindex(v)].opt = opt;
        if ((st = hs_sum_1d(p, v, d_scratch, n_bins, 0, &o, d_ws, ws_bytes, stream)) != HS_OK) break;
        cudaEventRecord(e0, stream);
        for (int r = 0; r < 3; ++r) hs_sum_1d(p, v, d_scratch, n_bins, 0, &o, d_ws, ws_bytes, stream);
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

// hs_sum_batched_noalloc: the batched harmonic sum for callers that cannot allocate device memory.
//
// The batched launch needs a little scratch memory (a status word, the work-queue counter and one
// tile prefix sum per spectrum).  hs_sum_batched takes it from a caller-allocated workspace.  This
// entry point instead uses a fixed array compiled into the library, so a caller can run the batched
// sum without ever allocating: for example a real-time search pipeline that reserves all of its GPU
// memory at start-up and does not allow allocations inside its processing loop (an allocation there
// can stall or fail in the middle of an observation), or a plugin whose host application owns the
// device memory pool.
#include <cstring>
#include <mutex>

#include "hs_internal.cuh"

using namespace hs;

namespace {

// Largest batch this entry point accepts, and the scratch it needs for that many spectra.
constexpr int kNoallocMaxSpectra = HS_NOALLOC_MAX_SPECTRA;
constexpr size_t kNoallocBytes = (kWsControlBytes + sizeof(int64_t) * (size_t)(kNoallocMaxSpectra + 2) + 255) &
                                 ~(size_t)255;

// One copy per device that loads the library; it lives until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per device.  In host code
// the name g_noalloc_scratch only stands for the device array; it is not an address a kernel can use.
hs_status scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return HS_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HS_OK;
}

bool is_aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

}  // namespace

extern "C" hs_status hs_sum_batched_noalloc(const hs_plan* p, hs_variant v, const void* d_x,
                                            const int64_t* d_offsets, int n_spectra, uint32_t first_id,
                                            const hs_out* out, cudaStream_t stream) {
    if (!p || vindex(v) < 0 || !(p->d.variants & v) || p->d.nz != 0) return HS_ERR_INVALID;
    if (n_spectra < 0 || n_spectra > kNoallocMaxSpectra) return HS_ERR_INVALID;  // beyond the fixed scratch
    if (!d_x || !d_offsets || !out || !out->best_snr || !out->best_h) return HS_ERR_INVALID;
    if (!is_aligned(d_x, 16) || !is_aligned(d_offsets, 8) || !is_aligned(out->best_snr, 4)) return HS_ERR_ALIGN;
    if (out->all_h) return HS_ERR_INVALID;
    if (out->path && !is_aligned(out->path, 4)) return HS_ERR_ALIGN;
    if (out->cand) {
        if (!out->cand_count || p->d.cand_capacity <= 0) return HS_ERR_INVALID;
        if (!is_aligned(out->cand, 16) || !is_aligned(out->cand_count, 8)) return HS_ERR_ALIGN;
    }
    if (n_spectra == 0) return HS_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return HS_ERR_CUDA;
    void* scratch = nullptr;
    hs_status st = scratch_address(&scratch);
    if (st != HS_OK) return st;
    // the array keeps whatever the previous call left: the status word must start at zero (the
    // queue counter and prefix sums are rewritten by the launch itself)
    if (cudaMemsetAsync(scratch, 0, kWsControlBytes, stream) != cudaSuccess) return HS_ERR_CUDA;
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
    Out1d o;
    o.best_snr = out->best_snr;
    o.best_h = out->best_h;
    o.path = v == HS_GREEDY ? out->path : nullptr;
    o.all_h = nullptr;
    o.cand = out->cand;
    o.cand_count = out->cand_count;
    o.cand_cap = p->d.cand_capacity;
    WsControl* ctl = reinterpret_cast<WsControl*>(scratch);
    int64_t* prefix = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(scratch) + kWsControlBytes);
    cudaError_t e = launch_1d(v, p->d.dtype, p->tab[vindex(v)], w, o, ctl, prefix, sms, stream);
    return e == cudaSuccess ? HS_OK : HS_ERR_CUDA;
}

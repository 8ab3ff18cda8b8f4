// Host-resident batches: the host-to-device copy of each piece of the batch overlaps the harmonic
// sums of the previous piece.  On GB300 the host link and the SMs are independent resources, so a
// batch that starts in host memory costs about max(copy, compute) instead of their sum.
#include <vector>

#include "hs_internal.cuh"

using namespace hs;

extern "C" hs_status hs_sum_batched_host(const hs_plan* p, int variant_mask, const void* h_x,
                                         const int64_t* h_offsets, int n_spectra, uint32_t first_id, void* d_x,
                                         int64_t* d_offsets, const hs_out* outs, int n_chunks, void* d_ws,
                                         size_t ws_bytes, cudaStream_t stream) {
    if (!p || variant_mask <= 0 || (variant_mask & ~p->d.variants) != 0 || p->d.nz != 0) return HS_ERR_INVALID;
    if (!h_x || !h_offsets || !d_x || !d_offsets || !outs || n_spectra < 0 || n_chunks < 1) return HS_ERR_INVALID;
    if (n_spectra == 0) return HS_OK;
    if (h_offsets[0] != 0) return HS_ERR_INVALID;
    for (int s = 0; s < n_spectra; ++s)
        if (h_offsets[s + 1] < h_offsets[s] || h_offsets[s + 1] - h_offsets[s] > p->d.max_bins) return HS_ERR_INVALID;
    const size_t es = p->d.dtype == HS_F32 ? 4 : 2;
    const int64_t total = h_offsets[n_spectra];
    if (n_chunks > n_spectra) n_chunks = n_spectra;
    // piece boundaries: the first spectrum at or past each equal share of the bins
    std::vector<int> cut(n_chunks + 1, n_spectra);
    cut[0] = 0;
    for (int c = 1, s = 0; c < n_chunks; ++c) {
        const int64_t goal = total * c / n_chunks;
        while (s < n_spectra && h_offsets[s] < goal) ++s;
        cut[c] = s < cut[c - 1] ? cut[c - 1] : s;
    }
    cudaStream_t cs = nullptr;
    std::vector<cudaEvent_t> ev(n_chunks, nullptr);
    hs_status st = HS_OK;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return HS_ERR_CUDA;
    for (auto& e : ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) st = HS_ERR_CUDA;
    // the copy stream starts after the caller's stream reaches this point (buffers may be in use)
    cudaEvent_t start = nullptr;
    if (st == HS_OK && cudaEventCreateWithFlags(&start, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(start, stream);
        cudaStreamWaitEvent(cs, start, 0);
    } else {
        st = HS_ERR_CUDA;
    }
    if (st == HS_OK &&
        cudaMemcpyAsync(d_offsets, h_offsets, sizeof(int64_t) * (n_spectra + 1), cudaMemcpyHostToDevice, cs) !=
            cudaSuccess)
        st = HS_ERR_CUDA;
    for (int c = 0; c < n_chunks && st == HS_OK; ++c) {
        const int s0 = cut[c], s1 = cut[c + 1];
        const int64_t a = h_offsets[s0], b = h_offsets[s1];
        if (b > a &&
            cudaMemcpyAsync(static_cast<char*>(d_x) + a * es, static_cast<const char*>(h_x) + a * es, (b - a) * es,
                            cudaMemcpyHostToDevice, cs) != cudaSuccess) {
            st = HS_ERR_CUDA;
            break;
        }
        cudaEventRecord(ev[c], cs);
        cudaStreamWaitEvent(stream, ev[c], 0);
        if (s1 == s0) continue;
        int k = 0;
        for (int bit = 0; bit < 4 && st == HS_OK; ++bit) {
            const hs_variant v = (hs_variant)(1 << bit);
            if (!(variant_mask & v)) continue;
            st = hs_sum_batched(p, v, d_x, d_offsets + s0, s1 - s0, first_id + (uint32_t)s0, &outs[k++], d_ws,
                                ws_bytes, stream);
        }
    }
    // the resources are released once the enqueued work that uses them has finished
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (start) cudaEventDestroy(start);
    cudaStreamDestroy(cs);
    return st;
}

// Eq. 1 over a packed batch with the input spans staged in shared memory by the bulk-copy engine.
//
// Section 2 (Eq. 1): S_H(n) = sum_{i=1..H} x(round(n i / H)).  For an output tile [n0, n0 + B) the
// reads of one reduced fraction f = p/q of F_32 all fall in [round(n0 f), round((n0 + B - 1) f)], a
// span of about B f elements, so a tile needs about 162.5 B input elements in all (the 324 fractions'
// values sum to 162.5).  Each CTA runs one producer warp and eight consumer warps:
//   - the producer claims work items from the batch queue and, fraction group by fraction group,
//     copies each fraction's span (start rounded down to 16 bytes) into a ring of shared-memory slots
//     with cp.async.bulk, completing an mbarrier per slot;
//   - consumer thread d owns the outputs n0 + d + 512 r (r = 0, 1) of every tile, so a warp's 32 lanes
//     read 32 consecutive outputs, whose indices for one fraction lie within 32 consecutive elements:
//     every shared-memory load is one conflict-free wavefront.
// The index inside a span is exact: with F = ceil(2^32 p/q) and W0 = n0 F + 2^31, the absolute index
// of output n0 + d is (W0 + d F) >> 32; the span starts at b = (W0 >> 32) rounded down to the copy
// granule, so the offset is (d F + (W0 - b 2^32)) >> 32, one 32x32->64-bit multiply-add.
// Fractions are visited in increasing order, so every S_H still adds its terms in the order
// i = 1..H and the results are bit-identical to the per-bin definition.
#include <algorithm>

#include "hs_async.cuh"
#include "hs_farey.cuh"

namespace hs {

namespace {

// Shape measured best among 8/16 consumer warps, 2/4 outputs per thread, 6-12 slots of 12-24 KB and
// one or two CTAs per SM.
constexpr int kStConsWarps = 16;
constexpr int kStCons = kStConsWarps * 32;        // consumer threads
constexpr int kStR = 2;                           // outputs per consumer thread (even)
constexpr int kStB = kStCons * kStR;              // output bins per tile
constexpr int kStThreads = kStCons + 32;          // + one producer warp
constexpr int kStSlots = 8;                       // ring of shared-memory slots
constexpr int kStSlotBytes = 24 * 1024;
constexpr int kStCtas = 1;                        // resident CTAs per SM
constexpr int kStDescs = 4;                       // tile descriptors in flight

// Where each fraction's span lives: group g of consecutive fractions fills one slot; a fraction's
// region holds up to cap elements, enough for any tile (derivation at region_cap).
struct StLayout {
    int group[kNumFrac];
    int off[kNumFrac];   // element offset of the region inside its slot
    int cap[kNumFrac];   // region capacity, elements (a multiple of the 16-byte granule)
    uint32_t F[kNumFrac];
    int p[kNumFrac], q[kNumFrac];
    int gfirst[kNumFrac + 1];
    int ngroups;
};

// Elements one tile can need from fraction p/q, for E elements per 16 bytes:
//   idx(n0 + B - 1) - idx(n0) <= ceil((B - 1) p/q) (round-half-up is monotone and moves by at most
//   the ceiling of the argument's change), and idx(n0) - b <= E - 1 for the rounded-down start b,
//   so the copy [b, b + cnt) with cnt = roundup_E(idx(n0 + B - 1) - b + 1) has
//   cnt <= roundup_E(ceil((B - 1) p/q) + E).
constexpr int region_cap(int p, int q, int E) {
    const int span = ((kStB - 1) * p + q - 1) / q;
    return (span + E + E - 1) / E * E;
}

constexpr StLayout make_layout(int esize) {
    StLayout L{};
    const int E = 16 / esize, slot_elems = kStSlotBytes / esize;
    int g = 0, off = 0, cnt = 0;
    L.gfirst[0] = 0;
    Frac a{0, 1}, b{1, 32};  // walk F_32 in increasing order, as farey_at does
    for (int j = 0; j < kNumFrac; ++j) {
        const int cap = region_cap(b.p, b.q, E);
        if (off + cap > slot_elems || cnt == 32) {  // a group is one slot and at most one producer lane each
            ++g;
            off = 0;
            cnt = 0;
            L.gfirst[g] = j;
        }
        L.group[j] = g;
        L.off[j] = off;
        L.cap[j] = cap;
        L.p[j] = b.p;
        L.q[j] = b.q;
        L.F[j] = b.q == 1 ? 0u : (uint32_t)((((uint64_t)b.p << 32) + b.q - 1) / b.q);
        off += cap;
        ++cnt;
        const int m = (32 + a.q) / b.q;
        const Frac c{m * b.p - a.p, m * b.q - a.q};
        a = b;
        b = c;
    }
    L.ngroups = g + 1;
    for (int k = g + 1; k <= kNumFrac; ++k) L.gfirst[k] = kNumFrac;
    return L;
}

template <int ES>
struct StLayoutOf {
    static constexpr StLayout value = make_layout(ES);
};

// the producer indexes the layout by lane at run time: a device-memory copy of the same tables
__device__ const StLayout kStLayout4 = make_layout(4);
__device__ const StLayout kStLayout2 = make_layout(2);

constexpr bool layout_fits(const StLayout& L, int esize) {
    for (int j = 0; j < kNumFrac; ++j)
        if (L.off[j] + L.cap[j] > kStSlotBytes / esize) return false;
    return true;
}
static_assert(layout_fits(StLayoutOf<4>::value, 4) && layout_fits(StLayoutOf<2>::value, 2),
              "every fraction's region fits its slot");
// The producer writes tile t's descriptor once every consumer warp has released the group armed
// kStSlots groups earlier, so consumers are at most ceil(kStSlots / ngroups) tiles behind: with
// kStDescs = 4 entries a descriptor is never overwritten before it is read.
static_assert(kStSlots <= 3 * StLayoutOf<4>::value.ngroups && kStSlots <= 3 * StLayoutOf<2>::value.ngroups,
              "descriptor ring too short for the slot ring");

struct StDesc {
    const void* x;                // spectrum start
    unsigned long long out_off;   // output offset of the spectrum
    uint32_t n0, N, spec, flags;
};
constexpr uint32_t kStDirect = 1u;  // tile within one granule of the spectrum end: no staging
constexpr uint32_t kStEnd = 2u;     // no more work

constexpr size_t kStSmemBytes = (size_t)kStSlots * kStSlotBytes + 2 * kStSlots * sizeof(uint64_t) +
                                kStDescs * sizeof(StDesc) + 16;

struct StShared {
    unsigned char* slots;
    uint32_t full0, empty0;  // shared addresses of the barrier arrays
    StDesc* desc;
    volatile int* abort_flag;
};

__device__ __forceinline__ void st_fail(const StShared& sh, unsigned* status) {
    *sh.abort_flag = 1;
    atomicOr(status, kStatusTimeout);
}

// Items increase along each CTA's sequence, so the next spectrum is usually the same or the next one.
__device__ __forceinline__ int next_spectrum(const int64_t* prefix, int n_spectra, int s, unsigned long long item) {
    for (int k = 0; k < 2; ++k) {
        if (s + 1 >= n_spectra || (unsigned long long)__ldg(prefix + s + 1) > item) return s;
        ++s;
    }
    return find_spectrum(prefix, n_spectra, item);
}

// ---- producer warp ----
template <typename T>
__device__ void st_producer(const Work1d& w, WsControl* ctl, const int64_t* prefix, uint32_t item_tiles,
                            const StShared& sh) {
    constexpr uint32_t E = 16 / sizeof(T);
    const StLayout& L = sizeof(T) == 4 ? kStLayout4 : kStLayout2;
    const int lane = threadIdx.x & 31;
    const unsigned long long total = *(volatile unsigned long long*)&ctl->total_items;
    uint32_t slot = 0, eparity = 1;  // a fresh barrier counts its preceding (odd) phase as complete
    uint32_t armed = 0, armed_parity = 0, fparity = 0;
    uint32_t tile_seq = 0;
    bool ok = true;

    unsigned long long item = 0;
    int s = 0;
    if (lane == 0) {
        item = atomicAdd(&ctl->queue, 1u);
        if (item < total) s = find_spectrum(prefix, w.n_spectra, item);
    }
    item = __shfl_sync(0xffffffffu, item, 0);
    s = __shfl_sync(0xffffffffu, s, 0);

    // HS_FLAG_CHECK_TIMEOUT: the item holding the batch's first tile arms its first slot for more
    // bytes than it copies, so the consumers' bounded waits run out (tests the error path)
    bool withhold = (w.flags & HS_FLAG_CHECK_TIMEOUT) != 0 && item == 0;
    while (ok && item < total) {
        unsigned long long next = 0;
        if (lane == 0) next = atomicAdd(&ctl->queue, 1u);  // consumed after this item's copies are queued
        const int64_t off = w.offsets[s];
        const uint32_t N = (uint32_t)(w.offsets[s + 1] - off);
        const T* xs = (const T*)w.x + off;
        const uint32_t base = (uint32_t)(item - (unsigned long long)prefix[s]) * (item_tiles * (uint32_t)kStB);
        for (uint32_t t = 0; ok && t < item_tiles; ++t) {
            const uint32_t n0 = base + t * (uint32_t)kStB;
            if (n0 >= N) break;
            const bool direct = (uint64_t)n0 + kStB + E > N;
            for (int g = 0; g < L.ngroups; ++g) {
                if (!mbar_wait(sh.empty0 + 8 * slot, eparity, sh.abort_flag)) {
                    if (lane == 0) st_fail(sh, &ctl->status);
                    ok = false;
                    break;
                }
                const int j = L.gfirst[g] + lane;
                uint32_t bytes = 0, dst = 0;
                const T* src = xs;
                if (!direct && j < L.gfirst[g + 1]) {
                    uint32_t b, last;
                    if (L.q[j] == 1) {
                        b = n0 & ~(E - 1);
                        last = n0 + kStB - 1;
                    } else {
                        const uint64_t F = L.F[j];
                        b = (uint32_t)(((uint64_t)n0 * F + 0x80000000ull) >> 32) & ~(E - 1);
                        last = (uint32_t)(((uint64_t)(n0 + kStB - 1) * F + 0x80000000ull) >> 32);
                    }
                    uint32_t cnt = (last - b + E) & ~(E - 1);
                    if (cnt > (uint32_t)L.cap[j]) {  // excluded by region_cap's bound; kept as a guard
                        cnt = (uint32_t)L.cap[j];
                        atomicOr(&ctl->status, kStatusBadInput);
                    }
                    bytes = cnt * (uint32_t)sizeof(T);
                    src = xs + b;
                    dst = smem_addr(sh.slots + (size_t)slot * kStSlotBytes) + (uint32_t)L.off[j] * (uint32_t)sizeof(T);
                }
                uint32_t tot = bytes;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
                if (lane == 0) {
                    if (g == 0) {
                        StDesc dsc;
                        dsc.x = xs;
                        dsc.out_off = (unsigned long long)off;
                        dsc.n0 = n0;
                        dsc.N = N;
                        dsc.spec = w.first_id + (uint32_t)s;
                        dsc.flags = direct ? kStDirect : 0u;
                        sh.desc[tile_seq % kStDescs] = dsc;
                    }
                    mbar_arrive_expect_tx(sh.full0 + 8 * slot, withhold ? tot + 16u : tot);  // releases the descriptor store
                }
                withhold = false;
                __syncwarp();
                if (bytes != 0u) bulk_copy_g2s(dst, src, bytes, sh.full0 + 8 * slot);
                armed |= 1u << slot;
                armed_parity = (armed_parity & ~(1u << slot)) | (fparity << slot);
                if (++slot == kStSlots) {
                    slot = 0;
                    eparity ^= 1u;
                    fparity ^= 1u;
                }
            }
            ++tile_seq;
        }
        if (lane == 0) {
            item = next;
            if (item < total) s = next_spectrum(prefix, w.n_spectra, s, item);
        }
        item = __shfl_sync(0xffffffffu, item, 0);
        s = __shfl_sync(0xffffffffu, s, 0);
    }
    if (ok) {  // end marker in the next slot
        if (mbar_wait(sh.empty0 + 8 * slot, eparity, sh.abort_flag)) {
            if (lane == 0) {
                StDesc dsc{};
                dsc.flags = kStEnd;
                sh.desc[tile_seq % kStDescs] = dsc;
                mbar_arrive_expect_tx(sh.full0 + 8 * slot, 0u);
            }
            armed |= 1u << slot;
            armed_parity = (armed_parity & ~(1u << slot)) | (fparity << slot);
        } else if (lane == 0) {
            st_fail(sh, &ctl->status);
        }
    }
    // No copy may still be writing shared memory when the CTA retires: wait (bounded) for the last
    // phase armed on every slot.
    if (lane == 0) {
        for (int k = 0; k < kStSlots; ++k)
            if (armed & (1u << k))
                if (!mbar_wait(sh.full0 + 8 * k, (armed_parity >> k) & 1u, nullptr)) atomicOr(&ctl->status, kStatusTimeout);
    }
    __syncwarp();
}

// ---- consumer warps ----
struct StCons {
    const StShared* sh;
    unsigned* status;
    const unsigned char* base;  // current slot
    uint32_t slot, parity;
    bool ok;

    __device__ __forceinline__ void wait_full() {
        if (ok && !mbar_wait(sh->full0 + 8 * slot, parity, sh->abort_flag)) {
            ok = false;
            st_fail(*sh, status);
        }
    }
    __device__ __forceinline__ void release() {
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(sh->empty0 + 8 * slot);
        if (++slot == kStSlots) {
            slot = 0;
            parity ^= 1u;
        }
        base = sh->slots + (size_t)slot * kStSlotBytes;
    }
};

// Fraction K of F_32 for the outputs n0 + d + kStCons r (r < kStR), added to every S_H it belongs to.
// acc[k] holds outputs r = 2k and 2k + 1, two sums per packed add.
template <typename T, int K>
__device__ __forceinline__ void st_term(StCons& c, uint32_t n0, uint32_t d, float2 (&acc)[kStR / 2][kHmax + 1]) {
    using LO = StLayoutOf<sizeof(T)>;
    constexpr uint32_t E = 16 / sizeof(T);
    constexpr int g = LO::value.group[K];
    constexpr bool first = LO::value.gfirst[g] == K;
    constexpr bool last = LO::value.gfirst[g + 1] == K + 1;
    constexpr int off = LO::value.off[K];
    constexpr Frac f = farey_at(K);
    if constexpr (first && g > 0) c.wait_full();
    const T* reg = reinterpret_cast<const T*>(c.base) + off;
    float v[kStR];
    if constexpr (f.q == 1) {
        const T* p = reg + (n0 & (E - 1)) + d;
#pragma unroll
        for (int r = 0; r < kStR; ++r) v[r] = widen<T>(p[kStCons * r]);
    } else {
        constexpr uint32_t F = FracConst<f.p, f.q>::F;
        const uint64_t W0 = (uint64_t)n0 * F + 0x80000000ull;
        const uint64_t cw = W0 & ((((uint64_t)E - 1) << 32) | 0xFFFFFFFFull);  // W0 - b 2^32
#pragma unroll
        for (int r = 0; r < kStR; ++r)
            v[r] = widen<T>(reg[(uint32_t)(((uint64_t)(d + kStCons * r) * F + cw) >> 32)]);
    }
#pragma unroll
    for (int k = 0; k < kStR / 2; ++k) {
        const float2 u = make_float2(v[2 * k], v[2 * k + 1]);
#pragma unroll
        for (int m = 1; m * f.q <= kHmax; ++m) acc[k][m * f.q] = add2(acc[k][m * f.q], u);
    }
    if constexpr (last) c.release();
}

template <typename T, int... K>
__device__ __forceinline__ void st_sweep(StCons& c, uint32_t n0, uint32_t d, float2 (&acc)[kStR / 2][kHmax + 1],
                                         std::integer_sequence<int, K...>) {
    (st_term<T, K>(c, n0, d, acc), ...);
}

__device__ __forceinline__ void st_store(const Work1d& w, const Out1d& o, const StDesc& ds, uint32_t n, float best,
                                         int bh, unsigned* status) {
    o.best_snr[ds.out_off + n] = best;
    o.best_h[ds.out_off + n] = (uint8_t)bh;
    if (o.cand) append_candidate(best > w.threshold, o.cand, o.cand_count, o.cand_cap, status, ds.spec, n, best, 0, bh,
                                 HS_STD);
}

template <typename T>
__device__ void st_consumer(const Tables& tb, const Work1d& w, const Out1d& o, WsControl* ctl, const StShared& sh) {
    constexpr int G = StLayoutOf<sizeof(T)>::value.ngroups;
    const uint32_t d = threadIdx.x;  // 0 .. kStCons - 1
    StCons c{&sh, &ctl->status, sh.slots, 0u, 0u, true};
    uint32_t tile_seq = 0;
    for (;;) {
        c.wait_full();  // group 0 of the next tile carries its descriptor
        if (!c.ok) break;
        const StDesc ds = sh.desc[tile_seq % kStDescs];
        if (ds.flags & kStEnd) break;
        if (ds.flags & kStDirect) {
            c.release();
            for (int g = 1; g < G; ++g) {
                c.wait_full();
                c.release();
            }
            if (!c.ok) break;
            const T* xs = (const T*)ds.x;
#pragma unroll 1
            for (int r = 0; r < kStR; ++r) {
                const uint32_t n = ds.n0 + d + (uint32_t)kStCons * r;
                float best = -INFINITY;
                int bh = 0;
                const bool active = n < ds.N;
                if (active) {
                    float S[kHmax + 1];
#pragma unroll
                    for (int H = 0; H <= kHmax; ++H) S[H] = 0.f;
                    farey_all<T>(xs, n, kHmax, S, std::make_integer_sequence<int, kNumFrac>{});
#pragma unroll
                    for (int H = 1; H <= kHmax; ++H) keep_best(calibrate(tb, S[H], H), H, best, bh);
                    o.best_snr[ds.out_off + n] = best;
                    o.best_h[ds.out_off + n] = (uint8_t)bh;
                }
                if (o.cand)
                    append_candidate(active && best > w.threshold, o.cand, o.cand_count, o.cand_cap, &ctl->status,
                                     ds.spec, n, best, 0, bh, HS_STD);
            }
        } else {
            float2 acc[kStR / 2][kHmax + 1];
#pragma unroll
            for (int k = 0; k < kStR / 2; ++k)
#pragma unroll
                for (int H = 0; H <= kHmax; ++H) acc[k][H] = make_float2(0.f, 0.f);
            st_sweep<T>(c, ds.n0, d, acc, std::make_integer_sequence<int, kNumFrac>{});
            if (!c.ok) break;
#pragma unroll
            for (int k = 0; k < kStR / 2; ++k) {
                float b0 = -INFINITY, b1 = -INFINITY;
                int h0 = 0, h1 = 0;
#pragma unroll
                for (int H = 1; H <= kHmax; ++H) {
                    keep_best(calibrate(tb, acc[k][H].x, H), H, b0, h0);
                    keep_best(calibrate(tb, acc[k][H].y, H), H, b1, h1);
                }
                st_store(w, o, ds, ds.n0 + d + kStCons * (2 * k), b0, h0, &ctl->status);
                st_store(w, o, ds, ds.n0 + d + kStCons * (2 * k + 1), b1, h1, &ctl->status);
            }
        }
        ++tile_seq;
    }
}

template <typename T>
__global__ void __launch_bounds__(kStThreads, kStCtas)
    k_hs1d_eq1_staged(const __grid_constant__ Tables tb, const Work1d w, const Out1d o, WsControl* ctl,
                      const int64_t* prefix, uint32_t item_tiles) {
    extern __shared__ __align__(128) unsigned char st_smem[];
    StShared sh;
    sh.slots = st_smem;
    uint64_t* bars = reinterpret_cast<uint64_t*>(st_smem + (size_t)kStSlots * kStSlotBytes);
    sh.full0 = smem_addr(bars);
    sh.empty0 = smem_addr(bars + kStSlots);
    sh.desc = reinterpret_cast<StDesc*>(bars + 2 * kStSlots);
    sh.abort_flag = reinterpret_cast<volatile int*>(sh.desc + kStDescs);
    if (threadIdx.x == 0) {
        for (int k = 0; k < kStSlots; ++k) {
            mbar_init(sh.full0 + 8 * k, 1u);
            mbar_init(sh.empty0 + 8 * k, (uint32_t)kStConsWarps);
        }
        *sh.abort_flag = 0;
        fence_mbarrier_init();
        fence_proxy_async_shared();
    }
    __syncthreads();
    if (threadIdx.x >= kStCons)
        st_producer<T>(w, ctl, prefix, item_tiles, sh);
    else
        st_consumer<T>(tb, w, o, ctl, sh);
}

template <typename T>
cudaError_t set_smem_attr() {
    // the attribute belongs to the device context: set once per device
    static bool done[kMaxDevices] = {};
    static cudaError_t err[kMaxDevices] = {};
    const int d = device_slot();
    if (!done[d]) {
        err[d] = cudaFuncSetAttribute(k_hs1d_eq1_staged<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kStSmemBytes);
        done[d] = true;
    }
    return err[d];
}

template <typename T>
cudaError_t launch_typed(const Tables& tab, const Work1d& w, const Out1d& o, WsControl* ctl, int64_t* prefix,
                         int sm_count, cudaStream_t s) {
    cudaError_t e = set_smem_attr<T>();
    if (e != cudaSuccess) return e;
    const uint32_t item_tiles = (uint32_t)std::max(1, w.opt * kBlock / kStB);
    launch_tile_scan(w.offsets, w.n_spectra, (int64_t)item_tiles * kStB, w.max_bins, (int)sizeof(T), prefix, ctl, s);
    const unsigned grid = persistent_grid(sm_count, kStCtas, w.ctas_per_sm);
    k_hs1d_eq1_staged<T><<<grid, kStThreads, kStSmemBytes, s>>>(tab, w, o, ctl, prefix, item_tiles);
    return cudaGetLastError();
}

}  // namespace

bool eq1_staged_applies(const Work1d& w, const Out1d& o) {
    return w.offsets != nullptr && w.hmax == kHmax && o.all_h == nullptr && o.path == nullptr &&
           (w.flags & HS_FLAG_POW2_STAGES) == 0;
}

void warm_eq1_staged(hs_dtype dt) {
    if (dt == HS_F32) set_smem_attr<float>();
    if (dt == HS_F16) set_smem_attr<__half>();
    if (dt == HS_BF16) set_smem_attr<__nv_bfloat16>();
}

cudaError_t launch_eq1_staged(hs_dtype dt, const Tables& tab, const Work1d& w, const Out1d& o, WsControl* ctl,
                              int64_t* prefix, int sm_count, cudaStream_t s) {
    switch (dt) {
        case HS_F32: return launch_typed<float>(tab, w, o, ctl, prefix, sm_count, s);
        case HS_F16: return launch_typed<__half>(tab, w, o, ctl, prefix, sm_count, s);
        case HS_BF16: return launch_typed<__nv_bfloat16>(tab, w, o, ctl, prefix, sm_count, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace hs

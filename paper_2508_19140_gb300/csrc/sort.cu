// K4: stable LSD radix sort of (u32 key, u32 value) pairs.
//
// The split sort of Sec. 3.2 ("Tiled Rendering") runs this twice: first over
// the points by depth key, then over the point-tile copies by tile id. Both
// sorts must be stable: stability is what makes ties in depth fall back to
// point index, and what keeps the depth order inside every tile after the
// second sort.
//
// One pass per digit of up to 9 bits, three kernels per pass
// (reduce-then-scan):
//   hist    per 4096-key tile, a digit histogram -> hist[digit][tile], and the
//           per-digit totals (integer atomics, order-free);
//   scan    one block per digit: exclusive scan over tiles, offset by the
//           totals of all smaller digits;
//   scatter per tile: stable in-tile rank (warp match + per-warp counters in
//           ascending warp order), staged in shared memory in digit order, then
//           written out in runs so consecutive threads write consecutive
//           addresses.
// The element count may live on the device (copies are counted on the GPU);
// the kernels are persistent over tiles so one launch shape serves any count up
// to the capacity, with no host synchronisation.
#include "rast_internal.cuh"

namespace rast {
namespace {

constexpr int kThreads = 256;
constexpr int kIPT = 16;
constexpr int kSortTile = kThreads * kIPT;  // 4096 keys per tile
constexpr int kWarpItems = 32 * kIPT;       // 512 keys per warp

int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

__device__ __forceinline__ int64_t read_count(int64_t n_host, const uint32_t* d_n) {
    return d_n ? (int64_t)(*d_n) : n_host;
}

template <int BITS>
__global__ void __launch_bounds__(kThreads) k_radix_hist(const uint32_t* __restrict__ keys,
                                                         int64_t n_host, const uint32_t* d_n,
                                                         int shift, uint32_t* __restrict__ hist,
                                                         int64_t hist_tiles,
                                                         uint32_t* __restrict__ bin_total) {
    constexpr int BINS = 1 << BITS;
    __shared__ uint32_t s_h[8 * BINS];
    const int64_t n = read_count(n_host, d_n);
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    const int warp = threadIdx.x >> 5;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        for (int i = threadIdx.x; i < 8 * BINS; i += kThreads) s_h[i] = 0;
        __syncthreads();
        const int64_t base = tile * kSortTile;
        if (base + kSortTile <= n) {
            const uint4* k4 = reinterpret_cast<const uint4*>(keys + base);
#pragma unroll
            for (int j = 0; j < kIPT / 4; ++j) {
                const uint4 q = k4[j * kThreads + threadIdx.x];
                atomicAdd(&s_h[warp * BINS + ((q.x >> shift) & (BINS - 1))], 1u);
                atomicAdd(&s_h[warp * BINS + ((q.y >> shift) & (BINS - 1))], 1u);
                atomicAdd(&s_h[warp * BINS + ((q.z >> shift) & (BINS - 1))], 1u);
                atomicAdd(&s_h[warp * BINS + ((q.w >> shift) & (BINS - 1))], 1u);
            }
        } else {
            for (int j = 0; j < kIPT; ++j) {
                const int64_t idx = base + (int64_t)j * kThreads + threadIdx.x;
                if (idx < n) atomicAdd(&s_h[warp * BINS + ((keys[idx] >> shift) & (BINS - 1))], 1u);
            }
        }
        __syncthreads();
        for (int bin = threadIdx.x; bin < BINS; bin += kThreads) {
            uint32_t c = 0;
#pragma unroll
            for (int w = 0; w < 8; ++w) c += s_h[w * BINS + bin];
            hist[(int64_t)bin * hist_tiles + tile] = c;
            if (c) atomicAdd(&bin_total[bin], c);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive scan across a block of NT threads (NT <= 1024); returns the
// thread's exclusive prefix, `total` gets the block sum. Uses s_warp[33]:
// [0, 32) the warps' exclusive prefixes, [32] the total (kept apart so a
// 32-warp block does not overwrite warp 31's prefix with it).
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* s_warp, uint32_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = NT / 32;
    const uint32_t inc = warp_incl_scan(x);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NW ? s_warp[lane] : 0u;
        const uint32_t wi = warp_incl_scan(w);
        if (lane < NW) s_warp[lane] = wi - w;
        if (lane == NW - 1) s_warp[32] = wi;
    }
    __syncthreads();
    const uint32_t res = s_warp[warp] + inc - x;
    total = s_warp[32];
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(1024) k_radix_scan(uint32_t* __restrict__ hist, int64_t hist_tiles,
                                                     const uint32_t* __restrict__ bin_total,
                                                     int64_t n_host, const uint32_t* d_n) {
    __shared__ uint32_t s_warp[33];
    const int bin = blockIdx.x;
    const int64_t n = read_count(n_host, d_n);
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    uint32_t part = 0;
    for (int b = threadIdx.x; b < bin; b += 1024) part += bin_total[b];
    uint32_t base;
    block_excl_scan<1024>(part, s_warp, base);
    const int64_t per = (ntiles + 1023) / 1024;
    const int64_t lo = threadIdx.x * per;
    const int64_t hi = lo + per < ntiles ? lo + per : ntiles;
    uint32_t* row = hist + (int64_t)bin * hist_tiles;
    uint32_t s = 0;
    for (int64_t t = lo; t < hi; ++t) s += row[t];
    uint32_t tot;
    uint32_t run = base + block_excl_scan<1024>(s, s_warp, tot);
    for (int64_t t = lo; t < hi; ++t) {
        const uint32_t c = row[t];
        row[t] = run;
        run += c;
    }
}

template <int BITS>
__global__ void __launch_bounds__(kThreads) k_radix_scatter(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n_host, const uint32_t* d_n, int shift,
    const uint32_t* __restrict__ hist, int64_t hist_tiles) {
    constexpr int BINS = 1 << BITS;
    constexpr int VPT = BINS > kThreads ? BINS / kThreads : 1;
    extern __shared__ uint32_t smem[];
    uint32_t* s_keys = smem;                       // kSortTile
    uint32_t* s_vals = s_keys + kSortTile;         // kSortTile
    uint32_t* s_whist = s_vals + kSortTile;        // 8 * BINS: per-warp counts, then prefixes
    uint32_t* s_excl = s_whist + 8 * BINS;         // BINS: tile-local digit starts
    uint32_t* s_gbase = s_excl + BINS;             // BINS: global digit starts of this tile
    uint32_t* s_warp = s_gbase + BINS;             // 33
    const int64_t n = read_count(n_host, d_n);
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t base = tile * kSortTile;
        const int64_t wbase = base + warp * kWarpItems;
        uint32_t k[kIPT], v[kIPT];
#pragma unroll
        for (int r = 0; r < kIPT; ++r) {
            const int64_t idx = wbase + r * 32 + lane;
            const bool ok = idx < n;
            k[r] = ok ? kin[idx] : 0u;
            v[r] = ok ? vin[idx] : 0u;
        }
        for (int i = threadIdx.x; i < 8 * BINS; i += kThreads) s_whist[i] = 0;
        for (int b = threadIdx.x; b < BINS; b += kThreads) s_gbase[b] = hist[(int64_t)b * hist_tiles + tile];
        __syncthreads();

        // Stable rank inside the warp's 512 keys: rounds in input order, lanes
        // in order within a round.
        uint32_t lp[kIPT];
#pragma unroll
        for (int r = 0; r < kIPT; ++r) {
            const int64_t idx = wbase + r * 32 + lane;
            const bool ok = idx < n;
            const uint32_t d = ok ? ((k[r] >> shift) & (BINS - 1)) : 0u;
            // Lanes holding the same digit: one ballot per digit bit (and one
            // for validity) instead of a match instruction.
            uint32_t peers = __ballot_sync(0xffffffffu, ok);
            if (!ok) peers = ~peers;
#pragma unroll
            for (int bb = 0; bb < BITS; ++bb) {
                const bool set = (d >> bb) & 1u;
                const uint32_t m = __ballot_sync(0xffffffffu, set);
                peers &= set ? m : ~m;
            }
            uint32_t pre = 0;
            if (ok) pre = s_whist[warp * BINS + d];
            __syncwarp();
            if (ok && (peers & lt) == 0) s_whist[warp * BINS + d] = pre + __popc(peers);
            __syncwarp();
            lp[r] = pre + __popc(peers & lt);
        }
        __syncthreads();

        // Per digit: warp prefixes (ascending warp = ascending input order) and totals.
        uint32_t tot[VPT];
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            const int bin = threadIdx.x * VPT + q;
            uint32_t run = 0;
            if (bin < BINS) {
#pragma unroll
                for (int w = 0; w < 8; ++w) {
                    const uint32_t c = s_whist[w * BINS + bin];
                    s_whist[w * BINS + bin] = run;
                    run += c;
                }
            }
            tot[q] = run;
        }
        uint32_t local = 0;
#pragma unroll
        for (int q = 0; q < VPT; ++q) local += tot[q];
        uint32_t all;
        uint32_t ex = block_excl_scan<kThreads>(local, s_warp, all);
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            const int bin = threadIdx.x * VPT + q;
            if (bin < BINS) s_excl[bin] = ex;
            ex += tot[q];
        }
        __syncthreads();

#pragma unroll
        for (int r = 0; r < kIPT; ++r) {
            const int64_t idx = wbase + r * 32 + lane;
            if (idx < n) {
                const uint32_t d = (k[r] >> shift) & (BINS - 1);
                const uint32_t pos = s_excl[d] + s_whist[warp * BINS + d] + lp[r];
                s_keys[pos] = k[r];
                s_vals[pos] = v[r];
            }
        }
        __syncthreads();

        const int cntv = (int)(n - base < kSortTile ? n - base : kSortTile);
        for (int j = threadIdx.x; j < cntv; j += kThreads) {
            const uint32_t key = s_keys[j];
            const uint32_t d = (key >> shift) & (BINS - 1);
            const uint32_t dst = s_gbase[d] + ((uint32_t)j - s_excl[d]);
            kout[dst] = key;
            vout[dst] = s_vals[j];
        }
        __syncthreads();
    }
}

template <int BITS>
size_t scatter_smem() {
    constexpr int BINS = 1 << BITS;
    return sizeof(uint32_t) * (2 * kSortTile + 8 * BINS + 2 * BINS + 33);
}

template <int BITS>
cudaError_t sort_pass(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout,
                      int64_t n, const uint32_t* d_n, int64_t cap, int shift, uint32_t* hist,
                      int64_t hist_tiles, uint32_t* bin_total, cudaStream_t s,
                      const char* const names[3]) {
    static bool attr_set = false;
    const size_t smem = scatter_smem<BITS>();
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_radix_scatter<BITS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int64_t tiles_cap = (cap + kSortTile - 1) / kSortTile;
    if (tiles_cap == 0) return cudaSuccess;
    const int sms = num_sms();
    const unsigned gh = (unsigned)(tiles_cap < (int64_t)sms * 8 ? tiles_cap : (int64_t)sms * 8);
    const unsigned gs = (unsigned)(tiles_cap < (int64_t)sms * 4 ? tiles_cap : (int64_t)sms * 4);
    {
        ProfScope ps(names[0], s);
        k_radix_hist<BITS><<<gh, kThreads, 0, s>>>(kin, n, d_n, shift, hist, hist_tiles, bin_total);
    }
    {
        ProfScope ps(names[1], s);
        k_radix_scan<<<1 << BITS, 1024, 0, s>>>(hist, hist_tiles, bin_total, n, d_n);
    }
    {
        ProfScope ps(names[2], s);
        k_radix_scatter<BITS><<<gs, kThreads, smem, s>>>(kin, vin, kout, vout, n, d_n, shift, hist,
                                                          hist_tiles);
    }
    return cudaGetLastError();
}

}  // namespace

SortPlan make_sort_plan(int bits) {
    SortPlan p{};
    if (bits <= 0) {
        p.passes = 0;
        return p;
    }
    int passes = (bits + 8) / 9;
    int per = (bits + passes - 1) / passes;
    if (per < 4) per = 4;
    int shift = 0;
    for (int k = 0; k < passes; ++k) {
        p.digit_bits[k] = per;
        p.shift[k] = shift;
        shift += per;
    }
    p.passes = passes;
    return p;
}

int64_t sort_hist_tiles(int64_t cap) { return (cap + kSortTile - 1) / kSortTile; }

cudaError_t radix_sort(uint32_t* keys[2], uint32_t* vals[2], int64_t n, const uint32_t* d_n,
                       int64_t cap, const SortPlan& plan, uint32_t* hist, int64_t hist_tiles,
                       uint32_t* bin_total, cudaStream_t s, int* result_buf,
                       const char* const names[3]) {
    int cur = 0;
    *result_buf = 0;
    if (plan.passes == 0 || cap == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(bin_total, 0, sizeof(uint32_t) * 512 * plan.passes, s);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < plan.passes; ++k) {
        uint32_t* bt = bin_total + 512 * k;
        const int nb = plan.digit_bits[k];
        switch (nb) {
#define RAST_PASS(B)                                                                              \
    case B:                                                                                       \
        e = sort_pass<B>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n, d_n, cap,         \
                         plan.shift[k], hist, hist_tiles, bt, s, names);                          \
        break;
            RAST_PASS(4)
            RAST_PASS(5)
            RAST_PASS(6)
            RAST_PASS(7)
            RAST_PASS(8)
            RAST_PASS(9)
#undef RAST_PASS
            default:
                return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    *result_buf = cur;
    return cudaSuccess;
}

}  // namespace rast

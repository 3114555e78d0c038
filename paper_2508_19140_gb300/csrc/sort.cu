// K4: stable LSD radix sort of (u32 key, u32 value) pairs, one kernel per digit.
//
// The split sort of Sec. 3.2 ("Tiled Rendering") runs this twice: first over
// the points by depth key, then over the point-tile copies by tile id. Both
// sorts must be stable: stability is what makes ties in depth fall back to
// point index, and what keeps the depth order inside every tile after the
// second sort.
//
// Structure (single-sweep LSD with decoupled look-back):
//   k_digit_hist  one read of all keys counts the digits of every pass at once
//                 (digit counts do not depend on the order), and clears the
//                 per-pass tile counters and look-back status words;
//   k_sweep       per pass, persistent CTAs take 4096-key tiles in input order
//                 from an atomic counter, rank each key stably inside the tile
//                 (one ballot per digit bit, or one match instruction for
//                 9-bit digits, gives each lane the mask of lanes holding the
//                 same digit; warps counted in ascending order),
//                 publish the tile's per-digit counts, and add the counts of
//                 all earlier tiles by looking back over their published words
//                 eight at a time (a tile whose whole prefix is known publishes
//                 it, so walks are short). Keys are then staged in shared
//                 memory in digit order and written out in runs.
// A tile only waits on tiles that running CTAs took before it, so the waits
// always end; each wait is still bounded, and on expiry the kernel raises the
// timeout bit of the workspace error word and carries on with the partial
// prefix instead of spinning on. The element count may live on the device (copies
// are counted on the GPU): launch shapes depend only on the capacity.
#include <cuda/atomic>

#include "rast_internal.cuh"

namespace rast {
namespace {

constexpr int kThreads = 256;
constexpr int kIPT = 16;
constexpr int kSortTile = kThreads * kIPT;  // 4096 keys per tile
constexpr int kWarpItems = 32 * kIPT;       // 512 keys per warp
constexpr uint32_t kFlagAgg = 1u << 30;     // tile count published
constexpr uint32_t kFlagPrefix = 2u << 30;  // inclusive prefix over tiles 0..t published
constexpr uint32_t kValueMask = (1u << 30) - 1;
constexpr int kLookback = 8;               // predecessor tiles read per look-back step

__device__ __forceinline__ int64_t read_count(int64_t n_host, const uint32_t* d_n) {
    return d_n ? (int64_t)(*d_n) : n_host;
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

// Digit counts of every pass with one read of the keys; clears the tile
// counters and the look-back words the passes will use.
template <int BITS>
__global__ void __launch_bounds__(kThreads) k_digit_hist(const uint32_t* __restrict__ keys, int64_t n_host,
                                                         const uint32_t* d_n, int passes,
                                                         uint32_t* __restrict__ ghist,
                                                         uint32_t* __restrict__ counters,
                                                         uint32_t* __restrict__ status, int64_t tiles_cap) {
    constexpr int BINS = 1 << BITS;
    __shared__ uint32_t s_h[kMaxSortPasses * BINS];
    const int64_t n = read_count(n_host, d_n);
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    for (int i = threadIdx.x; i < passes * BINS; i += kThreads) s_h[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x < kMaxSortPasses) counters[threadIdx.x] = 0;
    for (int p = 0; p < passes; ++p) {
        uint32_t* st = status + (int64_t)p * tiles_cap * BINS;
        const int64_t words = ntiles * BINS;
        for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < words; i += (int64_t)gridDim.x * kThreads)
            st[i] = 0;
    }
    __syncthreads();
    // Eight independent loads in flight per thread before the shared-memory
    // counting (one load at a time leaves the kernel waiting on latency).
    constexpr int U = 8;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t i0 = (int64_t)blockIdx.x * kThreads + threadIdx.x; i0 < n; i0 += U * stride) {
        uint32_t k[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * stride;
            k[u] = i < n ? keys[i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (i0 + u * stride >= n) break;
            for (int p = 0; p < passes; ++p)
                atomicAdd(&s_h[p * BINS + ((k[u] >> (p * BITS)) & (BINS - 1))], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * BINS; i += kThreads)
        if (s_h[i]) atomicAdd(&ghist[i], s_h[i]);
}

// IDV: the input values are their positions (not read from memory).
template <int BITS, bool IDV>
__global__ void __launch_bounds__(kThreads, 3) k_sweep(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n_host, const uint32_t* d_n, int shift,
    const uint32_t* __restrict__ ghist_pass, uint32_t* __restrict__ counter, uint32_t* __restrict__ status,
    uint32_t* __restrict__ err, int stall_test) {
    constexpr int BINS = 1 << BITS;
    constexpr int VPT = BINS > kThreads ? BINS / kThreads : 1;
    extern __shared__ uint32_t smem[];
    uint32_t* s_keys = smem;                       // kSortTile: keys in digit order
    uint32_t* s_vals = s_keys + kSortTile;         // kSortTile: values in digit order
    uint32_t* s_vin = s_vals + kSortTile;          // kSortTile: values in input order
    uint32_t* s_whist = s_vin + kSortTile;         // 8 * BINS: per-warp counts, then prefixes
    uint32_t* s_excl = s_whist + 8 * BINS;         // BINS: tile-local digit starts
    uint32_t* s_gbase = s_excl + BINS;             // BINS: global digit starts of this tile
    uint32_t* s_goff = s_gbase + BINS;             // BINS: global digit starts of the pass
    uint32_t* s_thist = s_goff + BINS;             // BINS: the tile's digit counts
    uint32_t* s_warp = s_thist + BINS;             // 33
    uint32_t* s_tile = s_warp + 33;                // 1
    // A pass after one whose look-back wait ran out does nothing: its input
    // is a partial order whose digit counts no longer match the histogram,
    // so its scatter positions could leave the buffers. (Within the pass that
    // gave up, a partial prefix only lowers positions: they stay in [0, n).)
    if (*err & kErrTimeout) return;
    const int64_t n = read_count(n_host, d_n);
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();

    // Global start of every digit in this pass.
    {
        uint32_t tot[VPT];
        uint32_t local = 0;
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            const int bin = threadIdx.x * VPT + q;
            tot[q] = bin < BINS ? ghist_pass[bin] : 0u;
            local += tot[q];
        }
        uint32_t all;
        uint32_t ex = block_excl_scan<kThreads>(local, s_warp, all);
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            const int bin = threadIdx.x * VPT + q;
            if (bin < BINS) s_goff[bin] = ex;
            ex += tot[q];
        }
    }

    // The next tile is taken from the counter during the previous tile's last
    // phase, so the loop spends no barrier on it. (A CTA holds the next tile
    // only while finishing one it took earlier, which never waits on it: every
    // look-back still ends.)
    for (int i = threadIdx.x; i < BINS; i += kThreads) s_thist[i] = 0;
    if (threadIdx.x == 0) *s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    for (;;) {
        const int64_t tile = *s_tile;
        if (tile >= ntiles) break;
        const int64_t base = tile * kSortTile;
        const int64_t wbase = base + warp * kWarpItems;
        // Keys to registers; values straight to shared memory in input order
        // (they are only moved, never inspected).
        uint32_t k[kIPT];
#pragma unroll
        for (int r = 0; r < kIPT; ++r) {
            const int64_t idx = wbase + r * 32 + lane;
            const bool ok = idx < n;
            k[r] = ok ? kin[idx] : 0u;
            s_vin[warp * kWarpItems + r * 32 + lane] = ok ? (IDV ? (uint32_t)idx : vin[idx]) : 0u;
        }
        // The tile's digit counts first (shared-memory adds), so they are
        // published before the ranking: a successor's look-back then rarely
        // finds this tile unpublished.
#pragma unroll
        for (int r = 0; r < kIPT; ++r)
            if (wbase + r * 32 + lane < n) atomicAdd(&s_thist[(k[r] >> shift) & (BINS - 1)], 1u);
        for (int i = threadIdx.x; i < 8 * BINS; i += kThreads) s_whist[i] = 0;
        __syncthreads();
        // Publish the tile's counts (test hook: with stall_test the first
        // tile publishes nothing, so its successor's wait runs out).
        uint32_t* my = status + tile * BINS;
        const bool withhold = stall_test && tile == 0;
        const uint32_t spin_limit = stall_test ? 64u : (1u << 22);
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            const int bin = threadIdx.x * VPT + q;
            if (bin < BINS && !withhold) {
                cuda::atomic_ref<uint32_t, cuda::thread_scope_device> w(my[bin]);
                w.store((tile == 0 ? kFlagPrefix : kFlagAgg) | s_thist[bin], cuda::memory_order_relaxed);
            }
        }

        // Stable rank inside the warp's 512 keys: rounds in input order, lanes
        // in order within a round. Ranks (< 512) are kept two to a register.
        uint32_t lp[kIPT / 2];
#pragma unroll
        for (int r = 0; r < kIPT / 2; ++r) lp[r] = 0;
#pragma unroll
        for (int r = 0; r < kIPT; ++r) {
            const int64_t idx = wbase + r * 32 + lane;
            const bool ok = idx < n;
            const uint32_t d = ok ? ((k[r] >> shift) & (BINS - 1)) : 0u;
            // Lanes holding the same digit. Up to 8-bit digits: one ballot per
            // digit bit (and one for validity); 9-bit digits: one match
            // instruction, measured faster there (lanes past the end share a
            // digit value of their own).
            uint32_t peers;
            if constexpr (BITS >= 9) {
                peers = __match_any_sync(0xffffffffu, ok ? d : (uint32_t)BINS);
            } else {
                peers = __ballot_sync(0xffffffffu, ok);
                if (!ok) peers = ~peers;
#pragma unroll
                for (int bb = 0; bb < BITS; ++bb) {
                    const bool set = (d >> bb) & 1u;
                    const uint32_t m = __ballot_sync(0xffffffffu, set);
                    peers &= set ? m : ~m;
                }
            }
            // The first lane of each digit group adds the group to the warp's
            // counter (atomics of one warp to one address apply in program
            // order, so rounds need no barrier) and hands the old value on.
            const int leader = __ffs(peers) - 1;
            uint32_t pre = 0;
            if (ok && lane == leader) pre = atomicAdd(&s_whist[warp * BINS + d], (uint32_t)__popc(peers));
            pre = __shfl_sync(0xffffffffu, pre, leader);
            lp[r >> 1] |= (pre + __popc(peers & lt)) << ((r & 1) * 16);
        }
        __syncthreads();

        // Per digit: warp prefixes (ascending warp = ascending input order) and
        // the tile's count.
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
        // Look back for the counts of all earlier tiles and publish the
        // inclusive prefix.
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            const int bin = threadIdx.x * VPT + q;
            if (bin < BINS) s_excl[bin] = tot[q];  // tile-local digit counts, scanned in place below
        }
        __syncthreads();
        // Tile-local digit starts: warp 0 scans the BINS counts in place (each
        // lane a run of consecutive bins) while the other warps look back.
        if (warp == 0) {
            constexpr int PER = BINS >= 32 ? BINS / 32 : 1;
            uint32_t c[PER], sum = 0;
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int bin = lane * PER + q;
                c[q] = bin < BINS ? s_excl[bin] : 0u;
                sum += c[q];
            }
            uint32_t run = warp_incl_scan(sum) - sum;
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int bin = lane * PER + q;
                if (bin < BINS) s_excl[bin] = run;
                run += c[q];
            }
        }
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            const int bin = threadIdx.x * VPT + q;
            if (bin >= BINS) continue;
            // Look back over windows of kLookback predecessors: the window's
            // loads are independent and in flight together, so a walk over
            // many tiles that only published their own counts costs one load
            // latency per window instead of one per tile.
            uint32_t excl = 0;
            int64_t t = tile - 1;
            uint32_t spins = 0;
            while (t >= 0) {
                uint32_t w[kLookback];
#pragma unroll
                for (int j = 0; j < kLookback; ++j) {
                    w[j] = kFlagPrefix;  // before tile 0: an empty prefix
                    if (t - j >= 0) {
                        cuda::atomic_ref<uint32_t, cuda::thread_scope_device> a(status[(t - j) * BINS + bin]);
                        w[j] = a.load(cuda::memory_order_relaxed);
                    }
                }
                int j = 0;
                bool found = false;
                for (; j < kLookback; ++j) {
                    if ((w[j] >> 30) == 0u) break;  // not published yet: poll again from here
                    excl += w[j] & kValueMask;
                    if ((w[j] & kFlagPrefix) != 0u) {
                        found = true;
                        break;
                    }
                }
                if (found) break;
                t -= j;
                if (j < kLookback) {
                    if (++spins > spin_limit) {  // a predecessor never published: give up
                        atomicOr(err, kErrTimeout);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            if (tile != 0) {
                cuda::atomic_ref<uint32_t, cuda::thread_scope_device> w(my[bin]);
                w.store(kFlagPrefix | (excl + tot[q]), cuda::memory_order_relaxed);
            }
            s_gbase[bin] = s_goff[bin] + excl;
        }
        __syncthreads();

#pragma unroll
        for (int r = 0; r < kIPT; ++r) {
            const int64_t idx = wbase + r * 32 + lane;
            if (idx < n) {
                const uint32_t d = (k[r] >> shift) & (BINS - 1);
                const uint32_t rank = (lp[r >> 1] >> ((r & 1) * 16)) & 0xffffu;
                const uint32_t pos = s_excl[d] + s_whist[warp * BINS + d] + rank;
                s_keys[pos] = k[r];
                s_vals[pos] = s_vin[warp * kWarpItems + r * 32 + lane];
            }
        }
        __syncthreads();

        const int cntv = (int)(n - base < kSortTile ? n - base : kSortTile);
        for (int j = threadIdx.x; j < cntv; j += kThreads) {
            const uint32_t key = s_keys[j];
            const uint32_t d = (key >> shift) & (BINS - 1);
            const uint32_t dst = s_gbase[d] + ((uint32_t)j - s_excl[d]);
            if (kout) kout[dst] = key;
            vout[dst] = s_vals[j];
        }
        for (int i = threadIdx.x; i < BINS; i += kThreads) s_thist[i] = 0;  // read before the look-back barrier
        if (threadIdx.x == 0) *s_tile = atomicAdd(counter, 1u);  // every thread has read this tile's index
        __syncthreads();
    }
}

template <int BITS>
size_t sweep_smem() {
    constexpr int BINS = 1 << BITS;
    return sizeof(uint32_t) * (3 * kSortTile + 8 * BINS + 4 * BINS + 33 + 1);
}

template <int BITS>
cudaError_t sort_t(uint32_t* keys[2], uint32_t* vals[2], int64_t n, const uint32_t* d_n, int64_t cap,
                   const SortPlan& plan, const SortScratch& sc, cudaStream_t s, int* result_buf,
                   const char* const names[2], bool identity_vals, bool keys_out) {
    constexpr int BINS = 1 << BITS;
    // Launch attributes and the resident CTAs per SM of the sweep, once per
    // device: persistent grid = as many CTAs as fit on the GPU at once (every
    // CTA resident, so a look-back never waits on a tile no running CTA holds).
    static PerDevice setup;
    const size_t smem = sweep_smem<BITS>();
    int per_sm = 1;
    cudaError_t e = per_device(setup, &per_sm, [smem](int, int* v) {
        *v = 1;
        cudaError_t r =
            cudaFuncSetAttribute(k_sweep<BITS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_sweep<BITS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r != cudaSuccess) return r;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sweep<BITS, false>, kThreads, smem) ==
                cudaSuccess && occ >= 1)
            *v = occ;
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    const int64_t tiles_cap = (cap + kSortTile - 1) / kSortTile;
    const int sms = device_sm_count();
    e = cudaMemsetAsync(sc.ghist, 0, sizeof(uint32_t) * plan.passes * BINS, s);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps(names[0], s);
        int64_t g = (cap + kThreads * 16 - 1) / (kThreads * 16);
        if (g > (int64_t)sms * 4) g = (int64_t)sms * 4;
        if (g < 1) g = 1;
        k_digit_hist<BITS><<<(unsigned)g, kThreads, 0, s>>>(keys[0], n, d_n, plan.passes, sc.ghist,
                                                           sc.counters, sc.status, tiles_cap);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int64_t resident = (int64_t)sms * per_sm;
    const unsigned gs = (unsigned)(tiles_cap < resident ? tiles_cap : resident);
    int cur = 0;
    for (int k = 0; k < plan.passes; ++k) {
        ProfScope ps(names[1], s);
        auto kern = (k == 0 && identity_vals) ? k_sweep<BITS, true> : k_sweep<BITS, false>;
        uint32_t* kout = (k + 1 == plan.passes && !keys_out) ? nullptr : keys[cur ^ 1];
        kern<<<gs, kThreads, smem, s>>>(keys[cur], vals[cur], kout, vals[cur ^ 1], n, d_n,
                                                 plan.shift[k], sc.ghist + k * BINS, sc.counters + k,
                                                 sc.status + (int64_t)k * tiles_cap * BINS, sc.err,
                                                 (k == 0 && sc.stall_test) ? 1 : 0);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    *result_buf = cur;
    return cudaSuccess;
}

}  // namespace

SortPlan make_sort_plan(int bits) {
    SortPlan p{};
    if (bits <= 0) {
        p.passes = 0;
        return p;
    }
    // Up to 9-bit digits for short keys (tile ids); 7-bit digits for long keys
    // (depth): measured, four 7-bit passes over 27-bit depth keys beat three
    // 9-bit ones (fewer ballots and bins per pass, more CTAs per SM).
    // Keys wider than 28 bits (a far/near ratio beyond about 2^29) take four
    // wider digits: the scratch buffers hold at most kMaxSortPasses passes.
    int passes = bits > 18 ? (bits + 6) / 7 : (bits + 8) / 9;
    if (passes > kMaxSortPasses) passes = kMaxSortPasses;
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

int64_t sort_status_words(const SortPlan& plan, int64_t cap) {
    if (plan.passes == 0) return 0;
    return (int64_t)plan.passes * ((cap + kSortTile - 1) / kSortTile) * (1 << plan.digit_bits[0]);
}

cudaError_t radix_sort(uint32_t* keys[2], uint32_t* vals[2], int64_t n, const uint32_t* d_n, int64_t cap,
                       const SortPlan& plan, const SortScratch& sc, cudaStream_t s, int* result_buf,
                       const char* const names[2], bool identity_vals, bool keys_out) {
    *result_buf = 0;
    if (plan.passes == 0 || cap == 0) return cudaSuccess;
    if (plan.passes > kMaxSortPasses) return cudaErrorInvalidValue;
    switch (plan.digit_bits[0]) {
        case 4: return sort_t<4>(keys, vals, n, d_n, cap, plan, sc, s, result_buf, names, identity_vals, keys_out);
        case 5: return sort_t<5>(keys, vals, n, d_n, cap, plan, sc, s, result_buf, names, identity_vals, keys_out);
        case 6: return sort_t<6>(keys, vals, n, d_n, cap, plan, sc, s, result_buf, names, identity_vals, keys_out);
        case 7: return sort_t<7>(keys, vals, n, d_n, cap, plan, sc, s, result_buf, names, identity_vals, keys_out);
        case 8: return sort_t<8>(keys, vals, n, d_n, cap, plan, sc, s, result_buf, names, identity_vals, keys_out);
        case 9: return sort_t<9>(keys, vals, n, d_n, cap, plan, sc, s, result_buf, names, identity_vals, keys_out);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rast

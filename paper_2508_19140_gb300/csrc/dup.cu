// K2 + K3 + K5: copies of each point per touched tile, and per-tile ranges.
//
// Second half of the split sort of Sec. 3.2 ("Tiled Rendering"): after the
// points are sorted by depth, each point (in depth order) writes one copy per
// tile its footprint touches, keyed by the global tile id. Writing the copies
// in depth order and sorting them stably by tile id afterwards yields the
// (tile, depth, point index) order. The copy offsets come from an exclusive
// scan of the per-point tile counts in depth order; the total D stays on the
// device and is clamped to the workspace capacity (overflow sets the
// capacity bit of the error word; no write ever leaves the buffers).
#include "rast_internal.cuh"

namespace rast {
namespace {

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

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

constexpr int kT = 256;
constexpr int kPer = kScanItems / kT;  // consecutive items per thread
static_assert(kPer % 4 == 0, "items move as 16-byte vectors");

// kPer consecutive u32 / uint2 items starting at s0 (vector loads and stores
// when the whole run is in range; `fill` past the end).
__device__ __forceinline__ void load_u32s(const uint32_t* __restrict__ p, int64_t s0, int64_t n, uint32_t v[kPer],
                                          uint32_t fill) {
    if (s0 + kPer <= n) {
#pragma unroll
        for (int j = 0; j < kPer; j += 4) {
            const uint4 q = *reinterpret_cast<const uint4*>(p + s0 + j);
            v[j] = q.x; v[j + 1] = q.y; v[j + 2] = q.z; v[j + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kPer; ++j) v[j] = s0 + j < n ? p[s0 + j] : fill;
    }
}

__device__ __forceinline__ void store_rects(uint2* __restrict__ p, int64_t s0, int64_t n, const uint2 r[kPer]) {
    if (s0 + kPer <= n) {
#pragma unroll
        for (int j = 0; j < kPer; j += 2)
            *reinterpret_cast<uint4*>(p + s0 + j) = make_uint4(r[j].x, r[j].y, r[j + 1].x, r[j + 1].y);
    } else {
#pragma unroll
        for (int j = 0; j < kPer; ++j)
            if (s0 + j < n) p[s0 + j] = r[j];
    }
}

// Sorted-order rects of a block of kScanItems points (gathered once, kept for
// k_dup_write) and the block's copy count. If the depth sort failed (its
// look-back wait ran out: the error word is set before this kernel starts),
// every point counts as empty, so no copy is made from a partial order; an
// index outside [0, n) is treated the same way. P4: bilinear packed 4-byte
// rects (the gather's array is half the size).
template <bool P4>
__global__ void __launch_bounds__(kT) k_dup_count(const uint32_t* __restrict__ sorted_pts,
                                                  const void* __restrict__ rect, void* __restrict__ rectS,
                                                  int64_t n, uint32_t* __restrict__ blk,
                                                  const WsHeader* __restrict__ hdr) {
    __shared__ uint32_t s_warp[33];
    const int64_t s0 = (int64_t)blockIdx.x * kScanItems + (int64_t)threadIdx.x * kPer;
    const bool failed = (hdr->error & kErrTimeout) != 0u;
    uint32_t gi[kPer];
    load_u32s(sorted_pts, s0, n, gi, 0xffffffffu);
    uint32_t c = 0;
    if constexpr (P4) {
        const uint32_t* r4 = static_cast<const uint32_t*>(rect);
        uint32_t r[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) r[j] = (!failed && (int64_t)gi[j] < n) ? r4[gi[j]] : kRect4Empty;
#pragma unroll
        for (int j = 0; j < kPer; ++j) c += rect4_count(r[j]);
        uint32_t* out = static_cast<uint32_t*>(rectS);
        if (s0 + kPer <= n) {
#pragma unroll
            for (int j = 0; j < kPer; j += 4)
                *reinterpret_cast<uint4*>(out + s0 + j) = make_uint4(r[j], r[j + 1], r[j + 2], r[j + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < kPer; ++j)
                if (s0 + j < n) out[s0 + j] = r[j];
        }
    } else {
        const uint2* r8 = static_cast<const uint2*>(rect);
        uint2 r[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) r[j] = (!failed && (int64_t)gi[j] < n) ? r8[gi[j]] : make_uint2(1u, 0u);
#pragma unroll
        for (int j = 0; j < kPer; ++j) c += rect_count(r[j]);
        store_rects(static_cast<uint2*>(rectS), s0, n, r);
    }
    uint32_t tot;
    block_excl_scan<kT>(c, s_warp, tot);
    if (threadIdx.x == 0) blk[blockIdx.x] = tot;
}

// Per-point copy counts, kPer consecutive points from s0: the count array
// (Gaussian), or the packed bilinear rects (P4; an empty rect counts 0).
template <bool P4>
__device__ __forceinline__ void load_counts(const uint32_t* __restrict__ p, int64_t s0, int64_t n, uint32_t v[kPer]) {
    load_u32s(p, s0, n, v, P4 ? kRect4Empty : 0u);
    if constexpr (P4) {
#pragma unroll
        for (int j = 0; j < kPer; ++j) v[j] = rect4_count(v[j]);
    }
}

template <bool P4>
__global__ void __launch_bounds__(kT) k_count_blocks(const uint32_t* __restrict__ cnt, int64_t n,
                                                     uint32_t* __restrict__ blk) {
    __shared__ uint32_t s_warp[33];
    const int64_t s0 = (int64_t)blockIdx.x * kScanItems + (int64_t)threadIdx.x * kPer;
    uint32_t v[kPer];
    load_counts<P4>(cnt, s0, n, v);
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) sum += v[j];
    uint32_t tot;
    block_excl_scan<kT>(sum, s_warp, tot);
    if (threadIdx.x == 0) blk[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_blocks(uint32_t* __restrict__ blk, int64_t nb,
                                                      WsHeader* hdr, int64_t cap) {
    __shared__ uint32_t s_warp[33];
    __shared__ unsigned long long s_wtot[32];
    const int64_t per = (nb + 1023) / 1024;
    const int64_t lo = threadIdx.x * per;
    const int64_t hi = lo + per < nb ? lo + per : nb;
    unsigned long long s = 0;
    for (int64_t t = lo; t < hi; ++t) s += blk[t];
    // 64-bit total: warp shuffle reduction, then one value per warp
    unsigned long long ws = s;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, o);
    if ((threadIdx.x & 31) == 0) s_wtot[threadIdx.x >> 5] = ws;
    uint32_t tot;
    uint32_t run = block_excl_scan<1024>((uint32_t)s, s_warp, tot);  // exact whenever total <= cap
    for (int64_t t = lo; t < hi; ++t) {
        const uint32_t c = blk[t];
        blk[t] = run;
        run += c;
    }
    if (hdr && threadIdx.x == 0) {
        unsigned long long total = 0;
        for (int w = 0; w < 32; ++w) total += s_wtot[w];
        const bool over = total > (unsigned long long)cap;
        hdr->n_copies_raw = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
        hdr->n_copies = over ? 0u : (uint32_t)total;
        if (over) atomicOr(&hdr->error, kErrCapacity);
    }
}

// Writes the copies: key = global tile id, value = global point index.
// Copies of a block of kScanItems depth-ordered points: 2 * kT threads with
// half as many items each as the counting kernels (the per-item copy loops
// are the long part here, so more threads beat more items per thread).
constexpr int kTW = 2 * kT;
constexpr int kPerW = kScanItems / kTW;
static_assert(kPerW == 4, "the packed-rect path loads four rects as one 16-byte vector");
// Gaussian copies a block stages in shared memory before writing them out
// (four a point on average fit; a block with more writes its copies
// directly). Bilinear points make at most four copies each, in runs of one
// to four per thread, and write them directly: measured, staging them costs
// more occupancy than the scattered stores do.
constexpr int kStageCap = 4 * kScanItems;
constexpr size_t kDupWriteSmem = sizeof(uint32_t) * 2 * kStageCap;

template <bool P4>
__global__ void __launch_bounds__(kTW) k_dup_write(const ViewTable vt, const uint32_t* __restrict__ sorted_pts,
                                                   const void* __restrict__ rectS, int64_t n,
                                                   const uint32_t* __restrict__ blk,
                                                   uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                   int64_t cap) {
    __shared__ uint32_t s_warp[33];
    extern __shared__ uint32_t s_copy[];  // [kStageCap] tile ids, then [kStageCap] point indices
    const int64_t s0 = (int64_t)blockIdx.x * kScanItems + (int64_t)threadIdx.x * kPerW;
    uint2 r[kPerW];
    uint32_t gi[kPerW];
    if (s0 + kPerW <= n) {
        if constexpr (P4) {
            const uint4 q = *reinterpret_cast<const uint4*>(static_cast<const uint32_t*>(rectS) + s0);
            r[0] = rect4_unpack(q.x); r[1] = rect4_unpack(q.y); r[2] = rect4_unpack(q.z); r[3] = rect4_unpack(q.w);
        } else {
            const uint2* rs = static_cast<const uint2*>(rectS);
#pragma unroll
            for (int j = 0; j < kPerW; j += 2) {
                const uint4 q = *reinterpret_cast<const uint4*>(rs + s0 + j);
                r[j] = make_uint2(q.x, q.y);
                r[j + 1] = make_uint2(q.z, q.w);
            }
        }
#pragma unroll
        for (int j = 0; j < kPerW; j += 4) {
            const uint4 q = *reinterpret_cast<const uint4*>(sorted_pts + s0 + j);
            gi[j] = q.x; gi[j + 1] = q.y; gi[j + 2] = q.z; gi[j + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kPerW; ++j) {
            const bool ok = s0 + j < n;
            if constexpr (P4) r[j] = ok ? rect4_unpack(static_cast<const uint32_t*>(rectS)[s0 + j]) : make_uint2(1u, 0u);
            else r[j] = ok ? static_cast<const uint2*>(rectS)[s0 + j] : make_uint2(1u, 0u);
            gi[j] = ok ? sorted_pts[s0 + j] : 0u;
        }
    }
    uint32_t c[kPerW], sum = 0;
#pragma unroll
    for (int j = 0; j < kPerW; ++j) {
        c[j] = rect_count(r[j]);
        sum += c[j];
    }
    uint32_t tot;
    const uint32_t ex = block_excl_scan<kTW>(sum, s_warp, tot);
    const uint32_t blk0 = blk[blockIdx.x];
    // The block's copies fill one contiguous range of the output: staged in
    // shared memory, they leave in coalesced runs instead of one scattered
    // 4-byte store per copy and array.
    const bool staged = !P4 && tot <= (uint32_t)kStageCap;
    uint32_t o = staged ? ex : blk0 + ex;
#pragma unroll
    for (int j = 0; j < kPerW; ++j) {
        if (c[j] == 0) continue;
        const ViewDev& V = vt.v[view_of_point(vt, gi[j])];
        const int tx0 = r[j].x & 0xffff, ty0 = r[j].x >> 16, tx1 = r[j].y & 0xffff, ty1 = r[j].y >> 16;
        for (int ty = ty0; ty <= ty1; ++ty) {
            const uint32_t row = (uint32_t)(V.tile_off + (int64_t)ty * V.tiles_x);
            for (int tx = tx0; tx <= tx1; ++tx) {
                if (staged) {
                    s_copy[o] = row + (uint32_t)tx;
                    s_copy[kStageCap + o] = gi[j];
                } else if ((int64_t)o < cap) {
                    keys[o] = row + (uint32_t)tx;
                    vals[o] = gi[j];
                }
                ++o;
            }
        }
    }
    if (!staged) return;  // block-uniform
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < tot; i += kTW) {
        const int64_t g = (int64_t)blk0 + i;
        if (g < cap) {
            keys[g] = s_copy[i];
            vals[g] = s_copy[kStageCap + i];
        }
    }
}

template <bool P4>
__global__ void __launch_bounds__(kT) k_scan_apply(const uint32_t* __restrict__ cnt, int64_t n,
                                                   const uint32_t* __restrict__ blk,
                                                   uint32_t* __restrict__ base) {
    __shared__ uint32_t s_warp[33];
    const int64_t s0 = (int64_t)blockIdx.x * kScanItems + (int64_t)threadIdx.x * kPer;
    uint32_t v[kPer];
    load_counts<P4>(cnt, s0, n, v);
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) sum += v[j];
    uint32_t tot;
    uint32_t o = blk[blockIdx.x] + block_excl_scan<kT>(sum, s_warp, tot);
    uint32_t r[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        r[j] = o;
        o += v[j];
    }
    if (s0 + kPer <= n) {
#pragma unroll
        for (int j = 0; j < kPer; j += 4)
            *reinterpret_cast<uint4*>(base + s0 + j) = make_uint4(r[j], r[j + 1], r[j + 2], r[j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < kPer; ++j)
            if (s0 + j < n) base[s0 + j] = r[j];
    }
}

// Tile ranges from the sorted tile keys. If the tile sort's look-back wait ran
// out, the keys are a partial order: the ranges are left empty (cleared before
// this kernel), so the blends read no copy of it.
__global__ void __launch_bounds__(kT) k_ranges(const uint32_t* __restrict__ keys,
                                               const WsHeader* __restrict__ hdr,
                                               uint2* __restrict__ ranges) {
    if (hdr->error & kErrTimeout) return;
    const int64_t D = hdr->n_copies;
    // Four consecutive keys per thread (one 16-byte load) plus the keys just
    // before and after them; a range starts or ends where neighbours differ.
    for (int64_t p0 = ((int64_t)blockIdx.x * kT + threadIdx.x) * 4; p0 < D; p0 += (int64_t)gridDim.x * kT * 4) {
        uint32_t k[6];  // keys p0-1 .. p0+4 (sentinels outside [0, D))
        k[0] = p0 > 0 ? keys[p0 - 1] : 0xffffffffu;
        if (p0 + 4 <= D) {
            const uint4 q = *reinterpret_cast<const uint4*>(keys + p0);
            k[1] = q.x; k[2] = q.y; k[3] = q.z; k[4] = q.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) k[1 + j] = p0 + j < D ? keys[p0 + j] : 0xffffffffu;
        }
        k[5] = p0 + 4 < D ? keys[p0 + 4] : 0xffffffffu;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t p = p0 + j;
            if (p >= D) break;
            const uint32_t t = k[1 + j];
            if (p == 0 || k[j] != t) ranges[t].x = (uint32_t)p;
            if (p + 1 == D || k[2 + j] != t) ranges[t].y = (uint32_t)(p + 1);
        }
    }
}

// ---- untiled baseline with one 64-bit-key sort (the arrangement Sec. 3.2
// "Tiled Rendering" starts from) ------------------------------------------
// Copies in POINT order, one per in-image pixel of the point's 2x2 box (the
// projection's rect with one-pixel tiles): the low key word is the point's
// depth key, the high word its pixel id; the point index goes with them. A
// stable LSD radix sort over the 64-bit key [pixel | depth] then yields the
// per-pixel lists in (depth, point index) order, ties falling back to the
// point order the copies were written in.
__global__ void __launch_bounds__(kT) k_untiled_copies(const ViewTable vt, const uint32_t* __restrict__ rect4,
                                                       const uint32_t* __restrict__ dkey,
                                                       const uint32_t* __restrict__ base,
                                                       uint32_t* __restrict__ key_lo, uint32_t* __restrict__ key_hi,
                                                       uint32_t* __restrict__ pt, int64_t cap) {
    const int64_t gi = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (gi >= vt.n_total) return;
    const uint2 r = rect4_unpack(rect4[gi]);  // bilinear only: packed rects
    if (rect_count(r) == 0) return;
    const ViewDev& V = vt.v[view_of_point(vt, gi)];
    const int x0 = r.x & 0xffff, y0 = r.x >> 16, x1 = r.y & 0xffff, y1 = r.y >> 16;
    const uint32_t k = dkey[gi];
    int64_t o = base[gi];
    for (int y = y0; y <= y1; ++y)
        for (int x = x0; x <= x1; ++x, ++o) {
            if (o >= cap) return;
            key_lo[o] = k;
            key_hi[o] = (uint32_t)(V.tile_off + (int64_t)y * V.tiles_x + x);
            pt[o] = (uint32_t)gi;
        }
}

// Between the low-word and high-word digit passes of the 64-bit sort: the
// high key word and the point index of every copy, fetched by the copy id the
// low-word passes carried (a copy id outside [0, D) yields an empty key past
// every pixel; after a timed-out pass the count is treated as zero).
__global__ void __launch_bounds__(kT) k_gather_hi(const uint32_t* __restrict__ cid,
                                                  const uint32_t* __restrict__ key_hi,
                                                  const uint32_t* __restrict__ pt,
                                                  const WsHeader* __restrict__ hdr,
                                                  uint32_t* __restrict__ kout, uint32_t* __restrict__ vout) {
    if (hdr->error & kErrTimeout) return;
    const int64_t D = hdr->n_copies;
    for (int64_t j = (int64_t)blockIdx.x * kT + threadIdx.x; j < D; j += (int64_t)gridDim.x * kT) {
        const uint32_t c = cid[j];
        const bool ok = (int64_t)c < D;
        kout[j] = ok ? key_hi[c] : 0xffffffffu;
        vout[j] = ok ? pt[c] : 0u;
    }
}

}  // namespace

cudaError_t launch_untiled_copies(const ViewTable& vt, const Bufs& b, const uint32_t* dkey, uint32_t* key_lo,
                                  uint32_t* key_hi, uint32_t* pt, cudaStream_t s) {
    const int64_t n = vt.n_total;
    const int64_t nb = (n + kScanItems - 1) / kScanItems;
    if (nb == 0) return cudaSuccess;
    {
        ProfScope ps("dup.count", s);
        k_count_blocks<true><<<(unsigned)nb, kT, 0, s>>>(b.rect4, n, b.blk);
    }
    {
        ProfScope ps("dup.scan", s);
        k_scan_blocks<<<1, 1024, 0, s>>>(b.blk, nb, b.hdr, b.copy_cap);
        k_scan_apply<true><<<(unsigned)nb, kT, 0, s>>>(b.rect4, n, b.blk, b.base);
    }
    {
        ProfScope ps("dup.write", s);
        k_untiled_copies<<<(unsigned)((n + kT - 1) / kT), kT, 0, s>>>(vt, b.rect4, dkey, b.base, key_lo, key_hi, pt,
                                                                      b.copy_cap);
    }
    return cudaGetLastError();
}

cudaError_t launch_gather_hi(const Bufs& b, const uint32_t* cid, const uint32_t* key_hi, const uint32_t* pt,
                             uint32_t* kout, uint32_t* vout, cudaStream_t s) {
    if (b.copy_cap == 0) return cudaSuccess;
    int64_t g = (b.copy_cap + kT - 1) / kT;
    const int64_t gmax = (int64_t)device_sm_count() * 16;
    if (g > gmax) g = gmax;
    ProfScope ps("sort64.gather_hi", s);
    k_gather_hi<<<(unsigned)g, kT, 0, s>>>(cid, key_hi, pt, b.hdr, kout, vout);
    return cudaGetLastError();
}

cudaError_t launch_duplicate(const ViewTable& vt, const Bufs& b, const uint32_t* sorted_pts,
                             cudaStream_t s) {
    const int64_t n = vt.n_total;
    const int64_t nb = (n + kScanItems - 1) / kScanItems;
    if (nb == 0) return cudaSuccess;  // the header was zeroed at the start of the pass
    {
        ProfScope ps("dup.count", s);
        if (vt.mode == 0) k_dup_count<true><<<(unsigned)nb, kT, 0, s>>>(sorted_pts, b.rect4, b.rect4S, n, b.blk, b.hdr);
        else k_dup_count<false><<<(unsigned)nb, kT, 0, s>>>(sorted_pts, b.rect, b.rectS, n, b.blk, b.hdr);
    }
    {
        ProfScope ps("dup.scan", s);
        k_scan_blocks<<<1, 1024, 0, s>>>(b.blk, nb, b.hdr, b.copy_cap);
    }
    {
        static PerDevice attr;
        const cudaError_t e = per_device(attr, nullptr, [](int, int*) {
            return cudaFuncSetAttribute(k_dup_write<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kDupWriteSmem);
        });
        if (e != cudaSuccess) return e;
        ProfScope ps("dup.write", s);
        if (vt.mode == 0)
            k_dup_write<true><<<(unsigned)nb, kTW, 0, s>>>(vt, sorted_pts, b.rect4S, n, b.blk, b.keyC[0],
                                                         b.valC[0], b.copy_cap);
        else
            k_dup_write<false><<<(unsigned)nb, kTW, kDupWriteSmem, s>>>(vt, sorted_pts, b.rectS, n, b.blk,
                                                                      b.keyC[0], b.valC[0], b.copy_cap);
    }
    return cudaGetLastError();
}

cudaError_t launch_ranges(const ViewTable& vt, const Bufs& b, const uint32_t* sorted_tiles,
                          cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b.ranges, 0, sizeof(uint2) * vt.tiles_total, s);
    if (e != cudaSuccess || b.copy_cap == 0) return e;
    int64_t g = (b.copy_cap + kT - 1) / kT;
    const int64_t gmax = (int64_t)device_sm_count() * 8;
    if (g > gmax) g = gmax;
    ProfScope ps("ranges", s);
    k_ranges<<<(unsigned)g, kT, 0, s>>>(sorted_tiles, b.hdr, b.ranges);
    return cudaGetLastError();
}

cudaError_t launch_point_scan(const ViewTable& vt, const Bufs& b, cudaStream_t s) {
    const int64_t n = vt.n_total;
    const int64_t nb = (n + kScanItems - 1) / kScanItems;
    if (nb == 0) return cudaSuccess;
    {
        ProfScope ps("point_scan.count", s);
        if (vt.mode == 0) k_count_blocks<true><<<(unsigned)nb, kT, 0, s>>>(b.rect4, n, b.blk);
        else k_count_blocks<false><<<(unsigned)nb, kT, 0, s>>>(b.cnt, n, b.blk);
    }
    {
        ProfScope ps("point_scan.scan", s);
        k_scan_blocks<<<1, 1024, 0, s>>>(b.blk, nb, nullptr, 0);
    }
    {
        ProfScope ps("point_scan.apply", s);
        if (vt.mode == 0) k_scan_apply<true><<<(unsigned)nb, kT, 0, s>>>(b.rect4, n, b.blk, b.base);
        else k_scan_apply<false><<<(unsigned)nb, kT, 0, s>>>(b.cnt, n, b.blk, b.base);
    }
    return cudaGetLastError();
}

}  // namespace rast

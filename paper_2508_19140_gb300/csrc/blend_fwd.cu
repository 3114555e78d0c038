// K6: front-to-back blend per tile (Eq. 1), one CTA per tile (16x16 or 8x8
// pixels), one thread per pixel.
//
// F = sum_i T_i a_i f_i, T_i = prod_{j<i} (1 - a_j), over the pixel's covering
// fragments in (depth, point index) order, stopping before the first fragment
// that would take T below t_min. Each CTA walks its tile's sorted list in
// batches of D records (the blend depth: tile^2 x RPT): every thread gathers
// its RPT records with 16-byte cp.async copies into a shared-memory ring (two
// or three batches deep, padded stride against bank conflicts), and each pixel
// composites the records of the batch that cover it, in list order. The copies
// of the next batches (and the point indices of the ones after) are in flight
// while a batch is composited, so the gather latency overlaps the compositing
// instead of adding to every batch of the tile's serial chain.
//
// Bilinear splats touch at most 4 pixels, so testing every record against
// every pixel would make the kernel ALU-bound. Instead the record's thread
// computes its four slot alphas once (the oracle's FP32 operations) and sets
// one bit per covered pixel in a per-pixel D-bit mask (shared-memory atomicOr,
// order-free and therefore deterministic); each pixel visits only its set bits
// in ascending order = list order.
//
// Gaussian splats cover many pixels; there each warp owns an 8x4 sub-tile,
// ballots the batch's records whose pixel box overlaps the sub-tile, and
// composites only those, all 32 lanes in lockstep.
//
// Tiles are visited heaviest first (k_tile_buckets / k_tile_scatter): the
// blend's duration is bounded below by its longest tile list, so that list
// must start at once. The CTA stops reading as soon as every in-image pixel
// has terminated (__syncthreads_count), which is where early termination saves
// HBM traffic. Saved for the backward pass: T_final and the 1-based list
// position of the last blended fragment per pixel. The per-tile count of
// records the method had to read (every record if some pixel never terminated,
// else up to the last terminating fragment) is summed into the workspace
// header. The untiled baseline's per-pixel kernel (k_blend_fwd_pixel) is at
// the end of the file.
#include "blend_common.cuh"

namespace rast {
namespace {

// Tiles in descending order of list length, bucketed by floor(log2(len)),
// over the whole grid: k_tile_buckets counts the tiles of every bucket
// (block-local counts, then one global add per bucket), k_tile_scatter turns
// the 33 counts into bucket starts (heaviest bucket first) and places each
// tile at its bucket's next free position. The order inside a bucket depends
// on timing and only affects scheduling: every tile is blended the same way.
__device__ __forceinline__ int len_bucket(uint2 r) {
    const uint32_t len = r.y - r.x;
    return len ? 32 - __clz(len) : 0;  // 0..32
}

__global__ void __launch_bounds__(256) k_tile_buckets(const uint2* __restrict__ ranges, int64_t P,
                                                      uint32_t* __restrict__ counts) {
    __shared__ uint32_t s_cnt[33];
    if (threadIdx.x < 33) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P; t += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&s_cnt[len_bucket(ranges[t])], 1u);
    __syncthreads();
    if (threadIdx.x < 33 && s_cnt[threadIdx.x]) atomicAdd(&counts[threadIdx.x], s_cnt[threadIdx.x]);
}

__global__ void __launch_bounds__(256) k_tile_scatter(const uint2* __restrict__ ranges, int64_t P,
                                                      const uint32_t* __restrict__ counts,
                                                      uint32_t* __restrict__ cursor, uint32_t* __restrict__ order) {
    __shared__ uint32_t s_start[33];  // global start of each bucket
    __shared__ uint32_t s_cnt[33];    // this block's tiles per bucket, then its next free slot
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int bk = 32; bk >= 0; --bk) {
            s_start[bk] = run;
            run += counts[bk];
        }
    }
    if (threadIdx.x < 33) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    // This block's contiguous chunk of tiles: count, reserve one range per
    // bucket with a single global atomic, then place.
    const int64_t chunk = (P + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * chunk, hi = lo + chunk < P ? lo + chunk : P;
    for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) atomicAdd(&s_cnt[len_bucket(ranges[t])], 1u);
    __syncthreads();
    if (threadIdx.x < 33) {
        const uint32_t c = s_cnt[threadIdx.x];
        s_cnt[threadIdx.x] = s_start[threadIdx.x] + (c ? atomicAdd(&cursor[threadIdx.x], c) : 0u);
    }
    __syncthreads();
    for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x)
        order[atomicAdd(&s_cnt[len_bucket(ranges[t])], 1u)] = (uint32_t)t;
}

// cp.async ring depth (batches in flight per CTA): three batches for 16x16
// tiles with one record per thread; two otherwise (deeper batches hide more
// latency each, and 8x8 tiles gain more from the extra CTAs per SM that a
// smaller ring leaves room for).
template <int TS, int RPT>
constexpr int stages_for() { return TS == 16 && RPT == 1 ? 3 : 2; }

template <int TS, int RPT, int C, bool BF16>
constexpr size_t bilinear_fwd_smem() {
    return sizeof(uint32_t) * stages_for<TS, RPT>() * TS * TS * RPT * ring_stride(RecLayout<0, C, BF16>::words) + 128;
}

// RPT = records each thread stages per batch: the batch ("blend depth") is
// D = TS * TS * RPT records; every pixel composites the records of a batch
// that cover it between two barriers, so a deeper batch spends fewer barriers
// per record and evens out the pixels' per-batch fragment counts.
template <int TS, int RPT, int C, bool BF16>
__global__ void __launch_bounds__(TS * TS) k_blend_fwd_bilinear(
    const ViewTable vt, const uint2* __restrict__ ranges, const uint32_t* __restrict__ order,
    const uint32_t* __restrict__ pts, const uint32_t* __restrict__ rec, uint32_t* __restrict__ rec_tile,
    float* __restrict__ t_final, uint32_t* __restrict__ last_out, WsHeader* __restrict__ hdr,
    unsigned long long* __restrict__ trace) {
    constexpr int NT = TS * TS;     // threads = pixels
    constexpr int D = NT * RPT;     // records per batch
    constexpr int MW = D / 32;      // mask words per pixel
    constexpr int kStages = stages_for<TS, RPT>();
    const unsigned long long t_start = global_ns();
    const long long c_start = clock64();
    constexpr int RW = RecLayout<0, C, BF16>::words;
    constexpr int RS = ring_stride(RW);
    constexpr int FW = RecLayout<0, C, BF16>::feat_word;
    extern __shared__ __align__(128) uint32_t s_dyn[];
    uint32_t* const s_ring = align128(s_dyn);  // [kStages][D][RS] raw records
    __shared__ uint32_t s_mask[NT][MW + 1];    // MW words + 1 pad: conflict-free row reads
    // Per record: the alphas of its 2x2 slots (FP32, pinned ops) and (tile-local
    // anchor (X0 + 1) | (Y0 + 1) << 8, depth bits). A fragment reads both with
    // two independent vector loads and picks its slot's alpha in registers, so
    // no shared-memory load waits on another one.
    __shared__ float4 s_alpha4[D];
    __shared__ uint2 s_az[D];
    __shared__ uint32_t s_maxstop;

    const int64_t tile = order[blockIdx.x];
    const ViewDev& V = vt.v[view_of_tile(vt, tile)];
    const int64_t lt = tile - V.tile_off;
    const int tx = (int)(lt % V.tiles_x), ty = (int)(lt / V.tiles_x);
    const int tid = threadIdx.x, lane = tid & 31;
    const int lx = tid & (TS - 1), ly = tid / TS;
    const int px = tx * TS + lx, py = ty * TS + ly;
    const bool inside = px < V.W && py < V.H;
    const uint2 rg = ranges[tile];
    const uint32_t len = rg.y - rg.x;
    const uint32_t nbatch = (len + D - 1) / D;
    const float amax = vt.alpha_max, tmin = vt.t_min;

    float T = 1.f, A = 0.f, Dp = 0.f;
    float F[C];
#pragma unroll
    for (int c = 0; c < C; ++c) F[c] = 0.f;
    uint32_t last = 0, stop = 0;
    bool done = !inside;
#pragma unroll
    for (int w = 0; w < MW; ++w) s_mask[tid][w] = 0;
    if (tid == 0) s_maxstop = 0;
    // Every row must be clear before any record thread sets bits in another
    // pixel's row (the first batch's atomicOr).
    __syncthreads();

    // Thread t copies records t, t + NT, ... of every batch. idx[s] = point
    // indices of batch j + kStages + s while batch j is processed (the copies
    // are issued kStages batches ahead, the indices read kStages further).
    auto point_of = [&](uint32_t j, int k) -> uint32_t {
        const uint32_t r = j * D + k * NT + tid;
        return r < len ? pts[rg.x + r] : 0xffffffffu;
    };
    auto issue = [&](uint32_t j, const uint32_t (&gi)[RPT]) {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (gi[k] != 0xffffffffu) {
                uint32_t* dst = s_ring + ((size_t)(j % kStages) * D + k * NT + tid) * RS;
                const uint32_t* src = rec + (size_t)gi[k] * RW;
#pragma unroll
                for (int q = 0; q < RW; q += 4) cp_async16(dst + q, src + q);
            }
        }
        cp_async_commit();
    };
    uint32_t idx[kStages][RPT];
#pragma unroll
    for (int st = 0; st < kStages; ++st)
#pragma unroll
        for (int k = 0; k < RPT; ++k) idx[st][k] = point_of(st, k);
#pragma unroll
    for (int st = 0; st < kStages; ++st) {
        issue(st, idx[st]);
#pragma unroll
        for (int k = 0; k < RPT; ++k) idx[st][k] = point_of(st + kStages, k);
    }

    for (uint32_t j = 0; j < nbatch; ++j) {
        const uint32_t* ring = s_ring + (size_t)(j % kStages) * D * RS;
        cp_async_wait<kStages - 1>();  // this thread's copies of batch j have landed
        const uint32_t rel0 = j * D;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = k * NT + tid;
            if (rel0 + r < len) {
                // Per record: the four fragment alphas of its 2x2 box (the ops of
                // bilin_weight and the clamp, so every pixel sees the same FP32
                // bits) and one mask bit per covered pixel of this tile.
                const uint4 g = *reinterpret_cast<const uint4*>(ring + r * RS);
                if (rec_tile) {
                    // The record, in list order, for the backward's sequential reads
                    // (coalesced: consecutive threads write consecutive records).
                    uint4* dst = reinterpret_cast<uint4*>(rec_tile + (size_t)(rg.x + rel0 + r) * RW);
                    dst[0] = g;
#pragma unroll
                    for (int q = 1; q < RW / 4; ++q)
                        dst[q] = *reinterpret_cast<const uint4*>(ring + r * RS + 4 * q);
                }
                const BilinGeom bg = bilin_geom(__uint_as_float(g.x), __uint_as_float(g.y));
                const float o = __uint_as_float(g.w);
                const float ax = __fsub_rn(1.f, bg.a), by = __fsub_rn(1.f, bg.b);
                s_alpha4[r] = make_float4(fminf(__fmul_rn(o, __fmul_rn(ax, by)), amax),
                                          fminf(__fmul_rn(o, __fmul_rn(bg.a, by)), amax),
                                          fminf(__fmul_rn(o, __fmul_rn(ax, bg.b)), amax),
                                          fminf(__fmul_rn(o, __fmul_rn(bg.a, bg.b)), amax));
                const int X0 = bg.i0 - tx * TS, Y0 = bg.j0 - ty * TS;
                s_az[r] = make_uint2((uint32_t)(X0 + 1) | ((uint32_t)(Y0 + 1) << 8), g.z);
                const uint32_t bit = 1u << lane;
                const int word = r >> 5;
#pragma unroll
                for (int dy = 0; dy < 2; ++dy) {
                    const int Y = Y0 + dy;
                    if ((unsigned)Y >= (unsigned)TS) continue;
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx) {
                        const int X = X0 + dx;
                        if ((unsigned)X < (unsigned)TS) atomicOr(&s_mask[Y * TS + X][word], bit);
                    }
                }
            }
        }
        if (__syncthreads_count(!done) == 0) break;
        if (!done) {
            // One loop over every set bit of the pixel's D-bit mask, in order.
            int w = 0;
            uint32_t m = s_mask[tid][0];
#pragma unroll 1
            while (true) {
                while (m == 0 && w < MW - 1) m = s_mask[tid][++w];
                if (m == 0) break;
                const int r = w * 32 + __ffs(m) - 1;
                m &= m - 1;
                const uint2 az = s_az[r];
                const float4 a4 = s_alpha4[r];
                const bool sx = lx + 1 != (int)(az.x & 0xffu), sy = ly + 1 != (int)(az.x >> 8);
                const float alpha = sy ? (sx ? a4.w : a4.z) : (sx ? a4.y : a4.x);
                const float nT = __fmul_rn(T, __fsub_rn(1.f, alpha));
                if (nT < tmin) {
                    done = true;
                    stop = rel0 + r + 1;
                    break;
                }
                const uint32_t* rp = ring + r * RS;
                float f[C];
                load_features<C, BF16>(rp + FW, f);
                const float ta = T * alpha;
#pragma unroll
                for (int c = 0; c < C; ++c) F[c] = fmaf(ta, f[c], F[c]);
                Dp = fmaf(ta, __uint_as_float(az.y), Dp);
                A += ta;
                T = nT;
                last = rel0 + r + 1;
            }
        }
#pragma unroll
        for (int w = 0; w < MW; ++w) s_mask[tid][w] = 0;
        __syncthreads();
        // Slot j % kStages is free: refill it with batch j + kStages.
        issue(j + kStages, idx[0]);
#pragma unroll
        for (int st = 0; st + 1 < kStages; ++st)
#pragma unroll
            for (int k = 0; k < RPT; ++k) idx[st][k] = idx[st + 1][k];
#pragma unroll
        for (int k = 0; k < RPT; ++k) idx[kStages - 1][k] = point_of(j + 2 * kStages, k);
    }
    cp_async_wait<0>();  // no copy may land after the CTA has exited

    if (inside) {
        const int64_t pix = (int64_t)py * V.W + px;
        float* of = V.out_feat + pix * C;
        if (C % 4 == 0) {
#pragma unroll
            for (int c = 0; c < C; c += 4)
                *reinterpret_cast<float4*>(of + c) = make_float4(F[c], F[c + 1], F[c + 2], F[c + 3]);
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) of[c] = F[c];
        }
        if (V.out_alpha) V.out_alpha[pix] = A;
        if (V.out_depth) V.out_depth[pix] = Dp;
        t_final[V.pix_off + pix] = T;
        last_out[V.pix_off + pix] = last;
    }
    const int open = __syncthreads_or(inside && stop == 0);
    if (stop) atomicMax(&s_maxstop, stop);
    __syncthreads();
    if (tid == 0) {
        atomicAdd(&hdr->needed, (unsigned long long)(open ? (rg.y - rg.x) : s_maxstop));
        trace_tile(trace, tile, 0, t_start, c_start);
    }
}

// Gaussian: every warp owns an 8x4 sub-tile and walks the tile's list on its
// own, 32 records at a time, with no CTA-wide barrier: each lane gathers one
// record (the CTA's warps read the same records, so all but the first find
// them in L1), stages it in the warp's own shared-memory rows as three
// 16-byte words (screen position, opacity and depth; conic; pixel box) plus
// FP32 features, and the warp ballots the records whose box meets its
// sub-tile and composites those, all 32 lanes in lockstep. A warp stops as
// soon as its own 32 pixels have terminated, and never waits for the other
// sub-tiles of the tile. The next chunk's records are loaded while this one is
// composited.
template <int TS, int C, bool BF16>
__global__ void __launch_bounds__(TS * TS) k_blend_fwd_gauss(
    const ViewTable vt, const uint2* __restrict__ ranges, const uint32_t* __restrict__ order,
    const uint32_t* __restrict__ pts, const uint32_t* __restrict__ rec, float* __restrict__ t_final,
    uint32_t* __restrict__ last_out, WsHeader* __restrict__ hdr) {
    constexpr int NT = TS * TS;
    constexpr int NW = NT / 32;      // warps = 8x4 sub-tiles
    constexpr int WPR = TS / 8;      // warps per row of 8x4 sub-tiles
    __shared__ float4 s_a[NW][32];   // (u - 1/2, v - 1/2, opacity, depth)
    __shared__ float4 s_c[NW][32];   // conic (a, b, c), unused
    __shared__ int4 s_box[NW][32];   // pixel box (x0, x1, y0, y1)
    __shared__ __align__(16) float s_f[NW][32 * C];
    __shared__ uint32_t s_maxstop;

    const int64_t tile = order[blockIdx.x];
    const ViewDev& V = vt.v[view_of_tile(vt, tile)];
    const int64_t lt = tile - V.tile_off;
    const int tx = (int)(lt % V.tiles_x), ty = (int)(lt / V.tiles_x);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sx0 = tx * TS + (warp % WPR) * 8, sy0 = ty * TS + (warp / WPR) * 4;
    const int px = sx0 + (lane & 7), py = sy0 + (lane >> 3);
    const bool inside = px < V.W && py < V.H;
    const uint2 rg = ranges[tile];
    const int RW = vt.rec_words, FW = vt.feat_word;
    const float amax = vt.alpha_max, tmin = vt.t_min;
    const float fpx = (float)px, fpy = (float)py;
    float4* const wa = s_a[warp];
    float4* const wc = s_c[warp];
    int4* const wbox = s_box[warp];
    float* const wf = s_f[warp];

    float T = 1.f, A = 0.f, Dp = 0.f;
    float F[C];
#pragma unroll
    for (int c = 0; c < C; ++c) F[c] = 0.f;
    uint32_t last = 0, stop = 0;
    bool done = !inside;
    if (tid == 0) s_maxstop = 0;

    uint4 g = make_uint4(0u, 0u, 0u, 0u), h = make_uint4(0u, 0u, 0u, 0u);
    float f[C];
#pragma unroll
    for (int c = 0; c < C; ++c) f[c] = 0.f;
    if (rg.x + lane < rg.y) {
        const uint32_t* rp = rec + (size_t)pts[rg.x + lane] * RW;
        g = *reinterpret_cast<const uint4*>(rp);
        h = *reinterpret_cast<const uint4*>(rp + 4);
        load_features<C, BF16>(rp + FW, f);
    }
    uint32_t gi_next = (rg.x + 32 + lane < rg.y) ? pts[rg.x + 32 + lane] : 0u;

#pragma unroll 1
    for (uint32_t q0 = rg.x; q0 < rg.y; q0 += 32) {
        if (__all_sync(0xffffffffu, done)) break;  // this sub-tile is finished
        bool hit = false;
        if (q0 + lane < rg.y) {
            const float um = __fsub_rn(__uint_as_float(g.x), 0.5f);
            const float vm = __fsub_rn(__uint_as_float(g.y), 0.5f);
            const GaussBox bx = gauss_box(um, vm, __uint_as_float(h.w));
            wa[lane] = make_float4(um, vm, __uint_as_float(g.w), __uint_as_float(g.z));
            wc[lane] = make_float4(__uint_as_float(h.x), __uint_as_float(h.y), __uint_as_float(h.z), 0.f);
            wbox[lane] = make_int4(bx.x0, bx.x1, bx.y0, bx.y1);
            store_row<C>(wf + lane * C, f);
            hit = bx.x0 <= sx0 + 7 && bx.x1 >= sx0 && bx.y0 <= sy0 + 3 && bx.y1 >= sy0;
        }
        uint32_t m = __ballot_sync(0xffffffffu, hit);
        __syncwarp();
        {
            // the next chunk's record (and the point index of the one after)
            const uint32_t qn = q0 + 32 + lane;
            if (qn < rg.y) {
                const uint32_t* rp = rec + (size_t)gi_next * RW;
                g = *reinterpret_cast<const uint4*>(rp);
                h = *reinterpret_cast<const uint4*>(rp + 4);
                load_features<C, BF16>(rp + FW, f);
            }
            gi_next = (qn + 32 < rg.y) ? pts[qn + 32] : 0u;
        }
        const uint32_t rel0 = q0 - rg.x;
        while (m) {
            const int r = __ffs(m) - 1;
            m &= m - 1;
            if (done) continue;
            const int4 bb = wbox[r];
            if (px < bb.x || px > bb.y || py < bb.z || py > bb.w) continue;
            const float4 ra = wa[r];
            const float4 rc = wc[r];
            const float dx = __fsub_rn(fpx, ra.x), dy = __fsub_rn(fpy, ra.y);
            const float mm = gauss_m(dx, dy, rc.x, rc.y, rc.z);
            if (!(mm <= 9.f)) continue;
            const float alpha = fminf(__fmul_rn(ra.z, gauss_value(mm)), amax);
            const float nT = __fmul_rn(T, __fsub_rn(1.f, alpha));
            if (nT < tmin) {
                done = true;
                stop = rel0 + r + 1;
                continue;
            }
            float fr[C];
            load_features<C, false>(reinterpret_cast<const uint32_t*>(wf + r * C), fr);
            const float ta = T * alpha;
#pragma unroll
            for (int c = 0; c < C; ++c) F[c] = fmaf(ta, fr[c], F[c]);
            Dp = fmaf(ta, ra.w, Dp);
            A += ta;
            T = nT;
            last = rel0 + r + 1;
        }
        __syncwarp();  // the warp's rows are refilled by the next chunk
    }

    if (inside) {
        const int64_t pix = (int64_t)py * V.W + px;
        store_row<C>(V.out_feat + pix * C, F);
        if (V.out_alpha) V.out_alpha[pix] = A;
        if (V.out_depth) V.out_depth[pix] = Dp;
        t_final[V.pix_off + pix] = T;
        last_out[V.pix_off + pix] = last;
    }
    const int open = __syncthreads_or(inside && stop == 0);
    if (stop) atomicMax(&s_maxstop, stop);
    __syncthreads();
    if (tid == 0)
        atomicAdd(&hdr->needed, (unsigned long long)(open ? (rg.y - rg.x) : s_maxstop));
}

template <int TS, int RPT, int C, bool BF16>
cudaError_t launch_fwd_t(const ViewTable& vt, const Bufs& b, const uint32_t* pts, cudaStream_t s) {
    const unsigned grid = (unsigned)vt.tiles_total;
    if (vt.mode == 0) {
        constexpr size_t smem = bilinear_fwd_smem<TS, RPT, C, BF16>();
        static PerDevice attr;
        const cudaError_t e = per_device(attr, nullptr, [](int, int*) {
            return cudaFuncSetAttribute(k_blend_fwd_bilinear<TS, RPT, C, BF16>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        });
        if (e != cudaSuccess) return e;
        ProfScope ps("blend_fwd", s);
        k_blend_fwd_bilinear<TS, RPT, C, BF16><<<grid, TS * TS, smem, s>>>(
            vt, b.ranges, b.order, pts, b.rec, b.rec_tile, b.t_final, b.last, b.hdr, b.trace);
        return cudaGetLastError();
    }
    ProfScope ps("blend_fwd", s);
    k_blend_fwd_gauss<TS, C, BF16><<<grid, TS * TS, 0, s>>>(vt, b.ranges, b.order, pts, b.rec, b.t_final,
                                                        b.last, b.hdr);
    return cudaGetLastError();
}

template <int TS, int C, bool BF16>
cudaError_t launch_fwd_d(const ViewTable& vt, const Bufs& b, const uint32_t* pts, cudaStream_t s) {
    const int rpt = vt.mode == 0 ? vt.blend_depth / (TS * TS) : 1;
    if constexpr (TS == 8) {
        if (rpt == 4) return launch_fwd_t<TS, 4, C, BF16>(vt, b, pts, s);
    }
    if (rpt == 2) return launch_fwd_t<TS, 2, C, BF16>(vt, b, pts, s);
    return launch_fwd_t<TS, 1, C, BF16>(vt, b, pts, s);
}

template <int C>
cudaError_t launch_fwd_c(const ViewTable& vt, const Bufs& b, const uint32_t* pts, cudaStream_t s) {
    if (vt.tile == 8)
        return vt.bf16 ? launch_fwd_d<8, C, true>(vt, b, pts, s) : launch_fwd_d<8, C, false>(vt, b, pts, s);
    return vt.bf16 ? launch_fwd_d<16, C, true>(vt, b, pts, s) : launch_fwd_d<16, C, false>(vt, b, pts, s);
}

}  // namespace

bool channels_supported(int C) {
    return C == 1 || C == 2 || C == 3 || C == 4 || C == 8 || C == 16;
}

cudaError_t launch_tile_order(const ViewTable& vt, const Bufs& b, cudaStream_t s) {
    const int64_t P = vt.tiles_total;
    if (P == 0) return cudaSuccess;
    uint32_t* counts = b.order + P;  // 33 bucket counts, then 33 cursors
    cudaError_t e = cudaMemsetAsync(counts, 0, 66 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const int64_t want = (P + 255) / 256;
    const unsigned grid = (unsigned)(want < 1024 ? want : 1024);
    {
        ProfScope ps("tile_order.count", s);
        k_tile_buckets<<<grid, 256, 0, s>>>(b.ranges, P, counts);
    }
    {
        ProfScope ps("tile_order.scatter", s);
        k_tile_scatter<<<grid, 256, 0, s>>>(b.ranges, P, counts, counts + 33, b.order);
    }
    return cudaGetLastError();
}

namespace {

// Untiled baseline (the per-pixel lists of the original INPC rasterizer that
// Sec. 3.2 "Tiled Rendering" replaces): the copies are per-pixel fragments
// sorted by (pixel, depth, point index), and one thread composites its
// pixel's list front to back, gathering every fragment's record from memory.
// Same FP32 operations as the tiled kernel, so the images are identical.
template <int C, bool BF16>
__global__ void __launch_bounds__(256) k_blend_fwd_pixel(const ViewTable vt, const uint2* __restrict__ ranges,
                                                         const uint32_t* __restrict__ pts,
                                                         const uint32_t* __restrict__ rec,
                                                         float* __restrict__ t_final, uint32_t* __restrict__ last_out,
                                                         WsHeader* __restrict__ hdr) {
    constexpr int RW = RecLayout<0, C, BF16>::words;
    constexpr int FW = RecLayout<0, C, BF16>::feat_word;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // global pixel ("tile") id
    const bool valid = p < vt.tiles_total;
    uint32_t need = 0;
    if (valid) {
        const ViewDev& V = vt.v[view_of_tile(vt, p)];
        const int64_t lp = p - V.tile_off;
        const int px = (int)(lp % V.W), py = (int)(lp / V.W);
        const uint2 rg = ranges[p];
        const float amax = vt.alpha_max, tmin = vt.t_min;
        float T = 1.f, A = 0.f, Dp = 0.f;
        float F[C];
#pragma unroll
        for (int c = 0; c < C; ++c) F[c] = 0.f;
        uint32_t last = 0, stop = 0;
#pragma unroll 1
        for (uint32_t q = rg.x; q < rg.y; ++q) {
            const uint32_t* rp = rec + (size_t)pts[q] * RW;
            const uint4 g = *reinterpret_cast<const uint4*>(rp);
            const BilinGeom bg = bilin_geom(__uint_as_float(g.x), __uint_as_float(g.y));
            const float o = __uint_as_float(g.w);
            const float wx = px == bg.i0 ? __fsub_rn(1.f, bg.a) : bg.a;
            const float wy = py == bg.j0 ? __fsub_rn(1.f, bg.b) : bg.b;
            const float alpha = fminf(__fmul_rn(o, __fmul_rn(wx, wy)), amax);
            const float nT = __fmul_rn(T, __fsub_rn(1.f, alpha));
            if (nT < tmin) {
                stop = q - rg.x + 1;
                break;
            }
            float f[C];
            load_features<C, BF16>(rp + FW, f);
            const float ta = T * alpha;
#pragma unroll
            for (int c = 0; c < C; ++c) F[c] = fmaf(ta, f[c], F[c]);
            Dp = fmaf(ta, __uint_as_float(g.z), Dp);
            A += ta;
            T = nT;
            last = q - rg.x + 1;
        }
        const int64_t pix = (int64_t)py * V.W + px;
        float* of = V.out_feat + pix * C;
#pragma unroll
        for (int c = 0; c < C; ++c) of[c] = F[c];
        if (V.out_alpha) V.out_alpha[pix] = A;
        if (V.out_depth) V.out_depth[pix] = Dp;
        t_final[V.pix_off + pix] = T;
        last_out[V.pix_off + pix] = last;
        need = stop ? stop : rg.y - rg.x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) need += __shfl_xor_sync(0xffffffffu, need, o);
    if ((threadIdx.x & 31) == 0 && need) atomicAdd(&hdr->needed, (unsigned long long)need);
}

// The same per-pixel lists composited by one warp per pixel (the layout of
// the untiled rasterizer Sec. 3.2 starts from): the lanes gather 32
// consecutive fragments' records at once and compute their alphas; the
// transmittance then steps through the 32 alphas in list order with the
// per-thread walk's FP32 operations (every lane runs the same serial chain on
// shuffled alphas, so the termination decision and T_final are those of the
// serial walk bit for bit); the chunk's F, depth and alpha sums are warp
// reductions (tree order: within FP32 rounding of the serial sums, not bit
// for bit).
__device__ __forceinline__ float warp_sum_f(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <int C, bool BF16>
__global__ void __launch_bounds__(256) k_blend_fwd_pixel_warp(const ViewTable vt, const uint2* __restrict__ ranges,
                                                              const uint32_t* __restrict__ pts,
                                                              const uint32_t* __restrict__ rec,
                                                              float* __restrict__ t_final,
                                                              uint32_t* __restrict__ last_out,
                                                              WsHeader* __restrict__ hdr) {
    constexpr int RW = RecLayout<0, C, BF16>::words;
    constexpr int FW = RecLayout<0, C, BF16>::feat_word;
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // global pixel ("tile") id
    const int lane = threadIdx.x & 31;
    if (p >= vt.tiles_total) return;  // uniform per warp
    const ViewDev& V = vt.v[view_of_tile(vt, p)];
    const int64_t lp = p - V.tile_off;
    const int px = (int)(lp % V.W), py = (int)(lp / V.W);
    const uint2 rg = ranges[p];
    const float amax = vt.alpha_max, tmin = vt.t_min;
    float T = 1.f, A = 0.f, Dp = 0.f;
    float F[C];
#pragma unroll
    for (int c = 0; c < C; ++c) F[c] = 0.f;
    uint32_t last = 0, stop = 0;
#pragma unroll 1
    for (uint32_t q0 = rg.x; q0 < rg.y; q0 += 32) {
        const uint32_t q = q0 + lane;
        const int nv = (int)min(32u, rg.y - q0);
        float alpha = 0.f, z = 0.f;
        float f[C];
#pragma unroll
        for (int c = 0; c < C; ++c) f[c] = 0.f;
        if (q < rg.y) {
            const uint32_t* rp = rec + (size_t)pts[q] * RW;
            const uint4 g = *reinterpret_cast<const uint4*>(rp);
            const BilinGeom bg = bilin_geom(__uint_as_float(g.x), __uint_as_float(g.y));
            const float o = __uint_as_float(g.w);
            const float wx = px == bg.i0 ? __fsub_rn(1.f, bg.a) : bg.a;
            const float wy = py == bg.j0 ? __fsub_rn(1.f, bg.b) : bg.b;
            alpha = fminf(__fmul_rn(o, __fmul_rn(wx, wy)), amax);
            load_features<C, BF16>(rp + FW, f);
            z = __uint_as_float(g.z);
        }
        // Serial transmittance over the chunk: T_k before fragment k in lane k.
        float Tk = 0.f;
        int kstop = nv;
        for (int k = 0; k < nv; ++k) {
            const float ak = __shfl_sync(0xffffffffu, alpha, k);
            const float nT = __fmul_rn(T, __fsub_rn(1.f, ak));
            if (nT < tmin) {
                kstop = k;
                break;
            }
            if (lane == k) Tk = T;
            T = nT;
        }
        const float ta = lane < kstop ? Tk * alpha : 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) F[c] += warp_sum_f(ta * f[c]);
        Dp += warp_sum_f(ta * z);
        A += warp_sum_f(ta);
        if (kstop > 0) last = q0 - rg.x + (uint32_t)kstop;
        if (kstop < nv) {
            stop = q0 - rg.x + (uint32_t)kstop + 1;
            break;
        }
    }
    if (lane == 0) {
        const int64_t pix = (int64_t)py * V.W + px;
        store_row<C>(V.out_feat + pix * C, F);
        if (V.out_alpha) V.out_alpha[pix] = A;
        if (V.out_depth) V.out_depth[pix] = Dp;
        t_final[V.pix_off + pix] = T;
        last_out[V.pix_off + pix] = last;
        const uint32_t need = stop ? stop : rg.y - rg.x;
        if (need) atomicAdd(&hdr->needed, (unsigned long long)need);
    }
}

template <int C>
cudaError_t launch_pixel_warp_c(const ViewTable& vt, const Bufs& b, const uint32_t* pts, cudaStream_t s) {
    const unsigned grid = (unsigned)((vt.tiles_total * 32 + 255) / 256);
    ProfScope ps("blend_fwd_pixel_warp", s);
    if (vt.bf16)
        k_blend_fwd_pixel_warp<C, true><<<grid, 256, 0, s>>>(vt, b.ranges, pts, b.rec, b.t_final, b.last, b.hdr);
    else
        k_blend_fwd_pixel_warp<C, false><<<grid, 256, 0, s>>>(vt, b.ranges, pts, b.rec, b.t_final, b.last, b.hdr);
    return cudaGetLastError();
}

template <int C>
cudaError_t launch_pixel_c(const ViewTable& vt, const Bufs& b, const uint32_t* pts, cudaStream_t s) {
    const unsigned grid = (unsigned)((vt.tiles_total + 255) / 256);
    ProfScope ps("blend_fwd_pixel", s);
    if (vt.bf16) k_blend_fwd_pixel<C, true><<<grid, 256, 0, s>>>(vt, b.ranges, pts, b.rec, b.t_final, b.last, b.hdr);
    else k_blend_fwd_pixel<C, false><<<grid, 256, 0, s>>>(vt, b.ranges, pts, b.rec, b.t_final, b.last, b.hdr);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blend_fwd_pixel(const ViewTable& vt, const Bufs& b, const uint32_t* pts, cudaStream_t s) {
    if (vt.tiles_total == 0) return cudaSuccess;
    switch (vt.C) {
        case 1: return launch_pixel_c<1>(vt, b, pts, s);
        case 2: return launch_pixel_c<2>(vt, b, pts, s);
        case 3: return launch_pixel_c<3>(vt, b, pts, s);
        case 4: return launch_pixel_c<4>(vt, b, pts, s);
        case 8: return launch_pixel_c<8>(vt, b, pts, s);
        case 16: return launch_pixel_c<16>(vt, b, pts, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_blend_fwd_pixel_warp(const ViewTable& vt, const Bufs& b, const uint32_t* pts, cudaStream_t s) {
    if (vt.tiles_total == 0) return cudaSuccess;
    switch (vt.C) {
        case 1: return launch_pixel_warp_c<1>(vt, b, pts, s);
        case 2: return launch_pixel_warp_c<2>(vt, b, pts, s);
        case 3: return launch_pixel_warp_c<3>(vt, b, pts, s);
        case 4: return launch_pixel_warp_c<4>(vt, b, pts, s);
        case 8: return launch_pixel_warp_c<8>(vt, b, pts, s);
        case 16: return launch_pixel_warp_c<16>(vt, b, pts, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_blend_fwd(const ViewTable& vt, const Bufs& b, const uint32_t* pts, cudaStream_t s) {
    if (vt.tiles_total == 0) return cudaSuccess;
    switch (vt.C) {
        case 1: return launch_fwd_c<1>(vt, b, pts, s);
        case 2: return launch_fwd_c<2>(vt, b, pts, s);
        case 3: return launch_fwd_c<3>(vt, b, pts, s);
        case 4: return launch_fwd_c<4>(vt, b, pts, s);
        case 8: return launch_fwd_c<8>(vt, b, pts, s);
        case 16: return launch_fwd_c<16>(vt, b, pts, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rast

// K7 + K8: backward pass (appendix, corrected Eq. 2).
//
// K7 replays each tile's list back to front, per pixel, from the saved final
// transmittance T_{K+1} and the position of the last blended fragment:
//   T_k     = T_{k+1} / (1 - a_k)
//   dL/da_k = T_k (g_F . f_k + g_D z_k) - (S_k + g_D SD_k - g_A T_{K+1}) / (1 - a_k)
//   S_k     = sum_{i>k} a_i T_i (g_F . f_i),  SD_k = sum_{i>k} a_i T_i z_i
//   dL/df_k = T_k a_k g_F,  dL/dz_k = T_k a_k g_D,
// where g_A is dL/dalpha of the alpha output 1 - T_{K+1} (the background term
// of Eq. 2 arrives through it). Fragments with a_k = 0 are not skipped.
// Chain: bilinear dL/do = w dL/da; Gaussian dL/do = G dL/da and, through
// G = exp(-m/2), dL/d(u, v) and dL/d(conic); nothing flows through a clamped
// alpha. The FP32 alpha of every fragment is recomputed with the forward's
// exact operations.
//
// Determinism without float atomics: the contributions of all pixels of a tile
// to one copy are combined in a fixed order inside the CTA (bilinear: the copy
// owns four slots, one per pixel of its 2x2 box; Gaussian: one slot per warp,
// filled by a fixed-order shuffle reduction), and written to the copy's own
// slot base[i] + (rank of the tile in the point's tile rect); a bilinear point
// with a single copy writes its row to a per-point array instead (whole
// sectors, no slot base needed), or, when its FP32 dL/df row is itself whole
// sectors (C a multiple of 8), writes dL/df to the output and keeps only dL/do
// in the per-point array (one whole sector per point). K8 then sums a point's
// slots in rect order and writes the outputs with coalesced stores. A per-tile cutoff (depth bits and
// point index of the last record the replay touched) tells K8 which slots were
// written.
#include "blend_common.cuh"

namespace rast {
namespace {

__device__ __forceinline__ uint32_t block_max_u32(uint32_t x, uint32_t* s) {
    if (threadIdx.x == 0) *s = 0;
    __syncthreads();
    atomicMax(s, x);
    __syncthreads();
    const uint32_t r = *s;
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------- bilinear

// On 16x16 tiles a bilinear point with one copy and C a multiple of 8 (its
// FP32 dL/df row is then whole 32-byte sectors) has dL/df written straight to
// the output by the blend and only dL/do kept for K8, alone in a 32-byte
// sector of its own (a 4-byte scattered store leaves a partial sector, which
// HBM must read-modify-write). 8x8 tiles keep the whole per-point row
// (measured faster there). Either layout fits the grow_stride(C + 1) rows.
__host__ __device__ constexpr bool direct_feat_grads(int C, int tile) { return C % 8 == 0 && tile == 16; }
constexpr int kOpRow = 8;  // floats per point of the dL/do sectors

// cp.async ring depth (batches in flight per CTA): three batches for 16x16
// tiles with one record per thread; two otherwise (deeper batches hide more
// latency each, and 8x8 tiles gain more from the extra CTAs per SM that a
// smaller ring leaves room for).
template <int TS, int RPT>
constexpr int stages_for() { return TS == 16 && RPT == 1 ? 3 : 2; }

// Ring stride (words) of a staged record: padded against bank conflicts when
// every thread copies its own record; the record stride itself when a batch
// arrives as one bulk copy of contiguous records (TSRC).
template <int C, bool BF16, bool TSRC>
constexpr int bwd_ring_stride() {
    return TSRC ? RecLayout<0, C, BF16>::words : ring_stride(RecLayout<0, C, BF16>::words);
}

template <int TS, int RPT, int C, bool BF16, bool TSRC>
constexpr size_t bilinear_bwd_smem() {
    constexpr int D = TS * TS * RPT;
    return sizeof(uint32_t) * stages_for<TS, RPT>() * D * bwd_ring_stride<C, BF16, TSRC>()  // record ring
           + sizeof(float) * 4 * 2 * D                                              // (T a, w dL/da) per slot
           + sizeof(float) * TS * TS * C                                            // upstream dL/dF per pixel
           + 128;
}

// RPT = records each thread stages per batch (blend depth D = TS * TS * RPT).
// 8x8 tiles with one record per thread: held to 64 registers, so the 16 CTAs
// per SM that shared memory allows stay resident (no spills at that bound).
// TSRC: the workspace holds the forward's tile-ordered record copy, so each
// batch is one contiguous run of records, staged by ONE TMA bulk copy
// (cp.async.bulk, completed on a per-stage mbarrier) issued by thread 0; if
// the last forward did not write the copy (header flag), the threads gather
// the records by point index into the same ring instead.
template <int TS, int RPT, int C, bool BF16, bool TSRC>
__global__ void __launch_bounds__(TS * TS, TS == 8 && RPT == 1 ? 16 : 1) k_blend_bwd_bilinear(
    const ViewTable vt, const uint2* __restrict__ ranges, const uint32_t* __restrict__ order,
    const uint32_t* __restrict__ pts, const uint32_t* __restrict__ rec, const uint32_t* __restrict__ rec_tile,
    const float* __restrict__ t_final, const uint32_t* __restrict__ last_in,
    const uint32_t* __restrict__ base, float* __restrict__ partial, float* __restrict__ grow,
    uint2* __restrict__ cutoff, WsHeader* __restrict__ hdr, unsigned long long* __restrict__ trace) {
    constexpr int NT = TS * TS;  // threads = pixels
    constexpr int D = NT * RPT;  // records per batch
    constexpr int MW = D / 32;   // mask words per pixel
    constexpr int kStages = stages_for<TS, RPT>();
    const unsigned long long t_start = global_ns();
    const long long c_start = clock64();
    constexpr int P = C + 1;  // dfeat[C], dopacity
    constexpr int PS = partial_stride(P);
    constexpr int GS = grow_stride(P);
    constexpr int RW = RecLayout<0, C, BF16>::words;
    constexpr int RS = bwd_ring_stride<C, BF16, TSRC>();
    constexpr int FW = RecLayout<0, C, BF16>::feat_word;
    extern __shared__ __align__(128) uint32_t s_dyn[];
    uint32_t* const s_ring = align128(s_dyn);                                 // [kStages][D][RS]
    float* const s_ta = reinterpret_cast<float*>(s_ring + kStages * D * RS);  // [4][D]
    float* const s_da = s_ta + 4 * D;                                         // [4][D]
    float* const s_gF = s_da + 4 * D;                                         // [NT][C]
    __shared__ uint32_t s_mask[NT][MW + 1];
    // Per record: the bilinear weights and the 1 / (1 - alpha) of its 2x2
    // slots, and (tile-local anchor, depth bits, opacity bits). A fragment
    // reads the three with independent vector loads and picks its slot in
    // registers, so no shared-memory load waits on another one.
    __shared__ float4 s_w4[D];
    __shared__ float4 s_inv4[D];
    __shared__ uint4 s_azo[D];
    __shared__ uint32_t s_red;
    __shared__ __align__(8) uint64_t s_mbar[kStages];  // TSRC: one bulk-copy barrier per ring stage

    const int64_t tile = order[blockIdx.x];
    const ViewDev& V = vt.v[view_of_tile(vt, tile)];
    const int64_t lt = tile - V.tile_off;
    const int tx = (int)(lt % V.tiles_x), ty = (int)(lt / V.tiles_x);
    const int tid = threadIdx.x, lane = tid & 31;
    const int lx = tid & (TS - 1), ly = tid / TS;
    const int px = tx * TS + lx, py = ty * TS + ly;
    const bool inside = px < V.W && py < V.H;
    const uint2 rg = ranges[tile];
    const float amax = vt.alpha_max;

    float T = 1.f, Tfin = 1.f, gA = 0.f, gD = 0.f;
    float gF[C];
    uint32_t last = 0;
#pragma unroll
    for (int c = 0; c < C; ++c) gF[c] = 0.f;
    if (inside) {
        const int64_t pix = (int64_t)py * V.W + px;
        T = Tfin = t_final[V.pix_off + pix];
        last = last_in[V.pix_off + pix];
#pragma unroll
        for (int c = 0; c < C; ++c) gF[c] = V.g_feat[pix * C + c];
        if (V.g_alpha) gA = V.g_alpha[pix];
        if (V.g_depth) gD = V.g_depth[pix];
    }
#pragma unroll
    for (int c = 0; c < C; ++c) s_gF[tid * C + c] = gF[c];
    // Each thread clears its own mask row; the barriers inside block_max_u32
    // order these stores before any thread sets bits in another pixel's row
    // (and the bulk-copy barriers' initialisation before the first copy).
#pragma unroll
    for (int w = 0; w < MW; ++w) s_mask[tid][w] = 0;
    if (TSRC && tid == 0) {
#pragma unroll
        for (int st = 0; st < kStages; ++st) mbar_init(&s_mbar[st], 1);
        mbar_init_fence();
    }
    const uint32_t maxlast = block_max_u32(last, &s_red);
    if (tid == 0 && maxlast) atomicAdd(&hdr->needed_bwd, (unsigned long long)maxlast);
    if (maxlast == 0) {
        if (tid == 0) {
            cutoff[tile] = make_uint2(0u, 0u);
            trace_tile(trace, tile, 1, t_start, c_start);
        }
        return;
    }
    float Sg = 0.f, SD = 0.f;
    const float Kd = -gA * Tfin;  // constant part of the 1/(1-a) term
    const uint32_t end = rg.x + maxlast;
    const uint32_t nb = (maxlast - 1) / D + 1;  // batches, processed last to first

    // Iteration j handles batch nb-1-j. Thread t copies records t, t + NT, ...
    // of each batch; idx[s] = points of iteration j + kStages + s.
    auto point_of = [&](uint32_t j, int k) -> uint32_t {
        if (j >= nb) return 0xffffffffu;
        const uint32_t q = rg.x + (nb - 1 - j) * D + k * NT + tid;
        return q < end ? pts[q] : 0xffffffffu;
    };
    // TSRC with the copy written: one bulk copy per batch. Otherwise every
    // thread gathers its records by point index (cp.async).
    const bool bulk = TSRC && hdr->rec_tile_valid != 0u;
    uint32_t phase = 0;        // bulk: parity bit per ring stage
    uint32_t outstanding = 0;  // bulk: stages with a copy not yet waited for
    auto issue = [&](uint32_t j, const uint32_t (&gi)[RPT]) {
        const int st = (int)(j % kStages);
        if (bulk) {
            if (j < nb) {
                const uint32_t b0 = rg.x + (nb - 1 - j) * D;
                const uint32_t nrec = end - b0 < (uint32_t)D ? end - b0 : (uint32_t)D;
                if (tid == 0)
                    bulk_copy_g2s(s_ring + (size_t)st * D * RS, rec_tile + (size_t)b0 * RW, nrec * RW * 4u,
                                  &s_mbar[st]);
                outstanding |= 1u << st;
            }
            return;
        }
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (gi[k] != 0xffffffffu) {
                uint32_t* dst = s_ring + ((size_t)st * D + k * NT + tid) * RS;
                const uint32_t* src = rec + (size_t)gi[k] * RW;
#pragma unroll
                for (int q = 0; q < RW; q += 4) cp_async16(dst + q, src + q);
            }
        }
        cp_async_commit();
    };
    bool failed = false;       // bulk: a copy did not arrive within the poll bound
    uint32_t idx[kStages][RPT];
    uint32_t gi_cur[kStages][RPT];  // point indices per ring slot
#pragma unroll
    for (int st = 0; st < kStages; ++st)
#pragma unroll
        for (int k = 0; k < RPT; ++k) idx[st][k] = point_of(st, k);
#pragma unroll
    for (int st = 0; st < kStages; ++st) {
        issue(st, idx[st]);
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            gi_cur[st][k] = idx[st][k];
            idx[st][k] = point_of(st + kStages, k);
        }
    }

    for (uint32_t j = 0; j < nb; ++j) {
        const uint32_t bi = nb - 1 - j;
        const int st = (int)(j % kStages);
        const uint32_t* ring = s_ring + (size_t)st * D * RS;
        const uint32_t rel0 = bi * D;
#pragma unroll
        for (int k = 0; k < 4 * RPT; ++k) {
            s_ta[k * NT + tid] = 0.f;
            s_da[k * NT + tid] = 0.f;
        }
        if (bulk) {
            if (mbar_wait(&s_mbar[st], (phase >> st) & 1u)) {
                phase ^= 1u << st;
                outstanding &= ~(1u << st);
            } else {
                failed = true;  // records of this batch may be missing: stop after this barrier round
            }
        } else {
            cp_async_wait<kStages - 1>();
        }
        // Per staged record: slot rank, anchor, and where its gradient goes.
        int slot_base[RPT], anchor[RPT];
        bool single[RPT];      // the point has this one copy: its gradient is final here
        uint32_t my_base[RPT]; // first partial slot of a point with several copies
        uint32_t gi_rec[RPT];  // the record's point index
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            slot_base[k] = 0;
            anchor[k] = 0;
            single[k] = false;
            my_base[k] = 0;
            gi_rec[k] = 0xffffffffu;
            const int r = k * NT + tid;
            const uint32_t q = rg.x + rel0 + r;
            if (q >= end) continue;
            const uint4 g = *reinterpret_cast<const uint4*>(ring + r * RS);
            const BilinGeom bg = bilin_geom(__uint_as_float(g.x), __uint_as_float(g.y));
            const float o = __uint_as_float(g.w);
            const float ax = __fsub_rn(1.f, bg.a), by = __fsub_rn(1.f, bg.b);
            const float w0 = __fmul_rn(ax, by), w1 = __fmul_rn(bg.a, by);
            const float w2 = __fmul_rn(ax, bg.b), w3 = __fmul_rn(bg.a, bg.b);
            s_w4[r] = make_float4(w0, w1, w2, w3);
            // 1 / (1 - alpha) of each slot, alpha = min(o w, amax) exactly as the forward has it
            s_inv4[r] = make_float4(rcp_fast(__fsub_rn(1.f, fminf(__fmul_rn(o, w0), amax))),
                                    rcp_fast(__fsub_rn(1.f, fminf(__fmul_rn(o, w1), amax))),
                                    rcp_fast(__fsub_rn(1.f, fminf(__fmul_rn(o, w2), amax))),
                                    rcp_fast(__fsub_rn(1.f, fminf(__fmul_rn(o, w3), amax))));
            const int X0 = bg.i0 - tx * TS, Y0 = bg.j0 - ty * TS;
            anchor[k] = (X0 + 1) | ((Y0 + 1) << 8);
            s_azo[r] = make_uint4((uint32_t)anchor[k], g.z, g.w, 0u);
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
            // The point's tile rect (as the projection computed it) and this tile's rank in it.
            const int tx0 = max(bg.i0, 0) / TS, tx1 = min(bg.i0 + 1, V.W - 1) / TS;
            const int ty0 = max(bg.j0, 0) / TS, ty1 = min(bg.j0 + 1, V.H - 1) / TS;
            slot_base[k] = (ty - ty0) * (tx1 - tx0 + 1) + (tx - tx0);
            single[k] = tx0 == tx1 && ty0 == ty1;
            uint32_t gi = gi_cur[0][k];
#pragma unroll
            for (int s2 = 1; s2 < kStages; ++s2)
                if (st == s2) gi = gi_cur[s2][k];
            gi_rec[k] = gi;
            // Only points with several copies need a partial slot; the load is
            // consumed after the compositing loop, which hides its latency.
            if (!single[k]) my_base[k] = base[gi];
            if (q + 1 == end) cutoff[tile] = make_uint2(g.z, gi);
        }
        __syncthreads();
        if (inside && last > rel0) {
            // One loop over the set bits of the pixel's mask, last to first.
            int w = MW - 1;
            uint32_t m = s_mask[tid][MW - 1];
#pragma unroll 1
            while (true) {
                while (m == 0 && w > 0) m = s_mask[tid][--w];
                if (m == 0) break;
                const int bit = 31 - __clz(m);
                m &= ~(1u << bit);
                const int r = w * 32 + bit;
                if (rel0 + r >= last) continue;
                const uint4 azo = s_azo[r];
                const float4 w4 = s_w4[r];
                const float4 i4 = s_inv4[r];
                const bool sx = lx + 1 != (int)(azo.x & 0xffu), sy = ly + 1 != (int)(azo.x >> 8);
                const int slot = (int)sx + 2 * (int)sy;
                const float wgt = sy ? (sx ? w4.w : w4.z) : (sx ? w4.y : w4.x);
                const float inv = sy ? (sx ? i4.w : i4.z) : (sx ? i4.y : i4.x);
                const float ow = __fmul_rn(__uint_as_float(azo.z), wgt);
                const float alpha = fminf(ow, amax);
                const float Tk = T * inv;  // T_k = T_{k+1} / (1 - alpha_k)
                const uint32_t* rp = ring + r * RS;
                float f[C];
                load_features<C, BF16>(rp + FW, f);
                float fdot = 0.f;
#pragma unroll
                for (int c = 0; c < C; ++c) fdot = fmaf(gF[c], f[c], fdot);
                const float z = __uint_as_float(azo.y);
                const float dalpha = Tk * (fdot + gD * z) - (Sg + gD * SD + Kd) * inv;
                const float ta = Tk * alpha;
                Sg = fmaf(ta, fdot, Sg);
                SD = fmaf(ta, z, SD);
                T = Tk;
                s_ta[slot * D + r] = ta;
                s_da[slot * D + r] = (ow <= amax) ? wgt * dalpha : 0.f;
            }
        }
#pragma unroll
        for (int w = 0; w < MW; ++w) s_mask[tid][w] = 0;
        if (__syncthreads_or(failed)) {
            // A bulk copy did not arrive in time: report it and stop (every
            // thread leaves here together; nothing is written from this batch).
            if (tid == 0) atomicOr(&hdr->error, kErrTimeout);
            break;
        }
        // Slot st is free (every pixel is done with it): refill it with iteration j + kStages.
        issue(j + kStages, idx[0]);
#pragma unroll
        for (int s2 = 0; s2 < kStages; ++s2)
            if (st == s2) {
#pragma unroll
                for (int k = 0; k < RPT; ++k) gi_cur[s2][k] = idx[0][k];
            }
#pragma unroll
        for (int s2 = 0; s2 + 1 < kStages; ++s2)
#pragma unroll
            for (int k = 0; k < RPT; ++k) idx[s2][k] = idx[s2 + 1][k];
#pragma unroll
        for (int k = 0; k < RPT; ++k) idx[kStages - 1][k] = point_of(j + 2 * kStages, k);
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (gi_rec[k] == 0xffffffffu) continue;
            const int r = k * NT + tid;
            const int X0 = (anchor[k] & 0xff) - 1, Y0 = (anchor[k] >> 8) - 1;
            // dL/df = sum over the 2x2 slots (fixed order) of T a times the pixel's dL/dF.
            float acc[P];
#pragma unroll
            for (int q = 0; q < P; ++q) acc[q] = 0.f;
#pragma unroll
            for (int sl = 0; sl < 4; ++sl) {
                const int X = X0 + (sl & 1), Y = Y0 + (sl >> 1);
                const float ta = s_ta[sl * D + r];
                if ((unsigned)X < (unsigned)TS && (unsigned)Y < (unsigned)TS) {
                    const float* gp = s_gF + (Y * TS + X) * C;
#pragma unroll
                    for (int c = 0; c < C; ++c) acc[c] += ta * gp[c];
                }
                acc[C] += s_da[sl * D + r];
            }
            if (single[k]) {
                if constexpr (direct_feat_grads(C, TS)) {
                    // Sole copy, dL/df rows of whole sectors: final, straight to
                    // the output; dL/do waits for K8 in a whole sector of its own.
                    const ViewDev& Vp = vt.shared_tiles ? vt.v[view_of_point(vt, gi_rec[k])] : V;
                    if (Vp.d_feat) store_row<C>(Vp.d_feat + ((int64_t)gi_rec[k] - Vp.pt_off) * C, acc);
                    float row[kOpRow];
#pragma unroll
                    for (int q = 0; q < kOpRow; ++q) row[q] = q == 0 ? acc[C] : 0.f;
                    store_row<kOpRow>(grow + (size_t)gi_rec[k] * kOpRow, row);
                } else {
                    // Sole copy: the point's gradient, in a whole-sector row of its
                    // own (K8 copies it to the outputs with coalesced writes).
                    float row[GS];
#pragma unroll
                    for (int q = 0; q < GS; ++q) row[q] = q < P ? acc[q] : 0.f;
                    store_row<GS>(grow + (size_t)gi_rec[k] * GS, row);
                }
            } else {
                float row[PS];
#pragma unroll
                for (int q = 0; q < PS; ++q) row[q] = q < P ? acc[q] : 0.f;
                store_row<PS>(partial + (size_t)(my_base[k] + (uint32_t)slot_base[k]) * PS, row);
            }
        }
        // No third barrier: the next iteration's writes to shared memory (this
        // thread's own contribution columns, the staging arrays and mask bits)
        // come after its first barrier, which every reader here precedes.
    }
    cp_async_wait<0>();
    // No bulk copy may land after the CTA has exited: wait (bounded) for any
    // the loop did not consume (only after a timeout).
#pragma unroll
    for (int st = 0; st < kStages; ++st)
        if ((outstanding >> st) & 1u) mbar_wait(&s_mbar[st], (phase >> st) & 1u);
    if (tid == 0) trace_tile(trace, tile, 1, t_start, c_start);
}

// ---------------------------------------------------------------- Gaussian

// Warp sums of N values per lane by recursive halving: at each level a lane
// keeps one half of its values (the upper half, ceil(N/2) slots with the
// missing ones zero, on lanes with the level's offset bit set) and adds the
// partner lane's copy of that half, so N values cost about N shuffles in all
// instead of five per value; scatter_index() says which value a lane ends up
// holding. Each sum is formed over the same pairing tree as an xor butterfly
// over offsets 16, 8, 4, 2, 1, so its bits do not depend on which lane holds
// it, on timing, or on how the values are split into halves.
template <int N, int OFF>
__device__ __forceinline__ float warp_reduce_scatter(const float (&v)[N], int lane) {
    if constexpr (N == 1) {
        float x = v[0];
#pragma unroll
        for (int o = OFF; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        return x;
    } else {
        static_assert(OFF > 0, "at most 32 values");
        constexpr int H = (N + 1) / 2;
        float w[H];
        const bool up = (lane & OFF) != 0;
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float lo = v[k], hi = k + H < N ? v[k + H] : 0.f;
            w[k] = (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, up ? lo : hi, OFF);
        }
        return warp_reduce_scatter<H, OFF / 2>(w, lane);
    }
}

// The value whose sum warp_reduce_scatter<N, OFF> returns on `lane`, or -1 if
// the lane holds a padding slot or a copy that a lower lane also holds.
template <int N, int OFF>
__device__ __forceinline__ int scatter_index(int lane) {
    if constexpr (N == 1) {
        return OFF == 0 || (lane & (2 * OFF - 1)) == 0 ? 0 : -1;
    } else {
        constexpr int H = (N + 1) / 2;
        const int sub = scatter_index<H, OFF / 2>(lane);
        if (sub < 0) return -1;
        const int idx = ((lane & OFF) ? H : 0) + sub;
        return idx < N ? idx : -1;
    }
}

// Gaussian backward: records per batch, batches in flight, padded rows.
constexpr int kGaussBatch = 32;   // records per batch: one ballot per warp and batch
constexpr int kGaussStages = 4;   // batches staged at once (how far warps may drift apart)
__host__ __device__ constexpr int gauss_contrib_stride(int P) { return P | 1; }  // odd: conflict-free rows
// Staged words of a record: the used prefix (u, v, z, o, conic, radius,
// features) rounded to 16 bytes. A stride of 12 words keeps the lane-parallel
// reads of the ballot step free of bank conflicts.
template <int C, bool BF16>
__host__ __device__ constexpr int gauss_ring_stride() {
    return (RecLayout<1, C, BF16>::need + 3) & ~3;
}
template <int TS, int C, bool BF16>
constexpr size_t gauss_bwd_smem() {
    return 128 + sizeof(uint32_t) * kGaussStages * kGaussBatch * gauss_ring_stride<C, BF16>() +
           sizeof(float) * kGaussStages * (TS * TS / 32) * kGaussBatch * gauss_contrib_stride(C + 7);
}

// Polls `bar` for the phase of this parity, giving up after `polls` polls or
// once another warp of the CTA has given up (abort flag).
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, const volatile uint32_t* abort,
                                                   uint32_t polls) {
    const uint32_t b = smem_addr(bar);
    for (uint32_t i = 0; i < polls; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(b), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((i & 63u) == 63u && *abort) return false;
    }
    return false;
}

// The warps of a tile (8x4 sub-tiles) run through the tile's batches without
// CTA barriers. A batch of kGaussBatch records sits in one of kGaussStages
// ring stages; one warp stages it with per-lane cp.async copies (record, point
// index, partial-slot base) that complete on the stage's mbarrier, and every
// warp waits on that barrier's phases in order. Per batch a warp ballots the
// records whose pixel box meets its sub-tile; for each one that some lane
// really blended (inside its box, m <= 9, before the pixel's last fragment)
// the lanes compute their P contributions, sum them over the warp with one
// reduce-scatter, and the lanes holding the sums write the record's row of
// the warp's contribution table (rows of odd stride: conflict-free) and a hit
// bit. The warp then counts itself done with the batch; the last of the NW
// warps adds the rows of the warps that hit each record, in warp order (the
// sum does not depend on which warp comes last), writes the copies' partial
// rows, clears the stage and stages the batch kGaussStages further on. Warps
// may thus drift apart by up to kGaussStages - 1 batches: a tile costs about
// its slowest warp's work, not the sum over batches of each batch's slowest.
template <int TS, int C, bool BF16>
__global__ void __launch_bounds__(TS * TS) k_blend_bwd_gauss(
    const ViewTable vt, const uint2* __restrict__ ranges, const uint32_t* __restrict__ order,
    const uint32_t* __restrict__ pts, const uint32_t* __restrict__ rec,
    const float* __restrict__ t_final, const uint32_t* __restrict__ last_in,
    const uint32_t* __restrict__ base, float* __restrict__ partial, uint2* __restrict__ cutoff,
    WsHeader* __restrict__ hdr) {
    constexpr int NT = TS * TS;
    constexpr int NW = NT / 32;                    // warps = 8x4 sub-tiles
    constexpr int WPR = TS / 8;                    // sub-tiles per row
    constexpr int GB = kGaussBatch;
    constexpr int R = kGaussStages;
    constexpr int NG = GB / 32;                    // ballot groups per batch
    constexpr int P = C + 7;  // dfeat[C], do, du, dv, dca, dcb, dcc, dz
    constexpr int PO = gauss_contrib_stride(P);
    constexpr int PS = partial_stride(P);
    constexpr int RW = RecLayout<1, C, BF16>::words;
    constexpr int RS = gauss_ring_stride<C, BF16>();
    constexpr int FW = RecLayout<1, C, BF16>::feat_word;
    extern __shared__ __align__(128) uint32_t s_dyn[];
    uint32_t* const s_ring = align128(s_dyn);                                     // [R][GB][RS]
    float* const s_contrib = reinterpret_cast<float*>(s_ring + R * GB * RS);      // [R][NW][GB][PO]
    __shared__ uint32_t s_gi[R][GB];               // point index of each staged record
    __shared__ uint32_t s_base[R][GB];             // its first partial slot
    __shared__ uint32_t s_pnext[R][GB];            // point indices of the batch a stage takes next
    __shared__ uint32_t s_hit[R][NW * NG];         // records each warp contributed to
    __shared__ uint32_t s_done[R];                 // warps done with the stage's batch
    __shared__ __align__(8) uint64_t s_mbar[R];    // stage filled (32 arrivals: the staging lanes)
    __shared__ int4 s_box[NW][GB];                 // per warp: pixel boxes of the batch's records
    __shared__ uint32_t s_red;
    __shared__ uint32_t s_abort;

    const int64_t tile = order[blockIdx.x];
    const ViewDev& V = vt.v[view_of_tile(vt, tile)];
    const int64_t lt = tile - V.tile_off;
    const int tx = (int)(lt % V.tiles_x), ty = (int)(lt / V.tiles_x);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sx0 = tx * TS + (warp % WPR) * 8, sy0 = ty * TS + (warp / WPR) * 4;
    const int px = sx0 + (lane & 7), py = sy0 + (lane >> 3);
    const bool inside = px < V.W && py < V.H;
    const uint2 rg = ranges[tile];
    const float amax = vt.alpha_max;
    const float fpx = (float)px, fpy = (float)py;

    float T = 1.f, Tfin = 1.f, gA = 0.f, gD = 0.f;
    float gF[C];
    uint32_t last = 0;
#pragma unroll
    for (int c = 0; c < C; ++c) gF[c] = 0.f;
    if (inside) {
        const int64_t pix = (int64_t)py * V.W + px;
        T = Tfin = t_final[V.pix_off + pix];
        last = last_in[V.pix_off + pix];
#pragma unroll
        for (int c = 0; c < C; ++c) gF[c] = V.g_feat[pix * C + c];
        if (V.g_alpha) gA = V.g_alpha[pix];
        if (V.g_depth) gD = V.g_depth[pix];
    }
    if (tid < R) s_done[tid] = 0;
    for (int i = tid; i < R * NW * NG; i += NT) (&s_hit[0][0])[i] = 0;
    if (tid == 0) {
        s_abort = 0;
#pragma unroll
        for (int st = 0; st < R; ++st) mbar_init(&s_mbar[st], 32);
        mbar_init_fence();
    }
    // The barriers inside block_max_u32 also order the initialisation above
    // before any copy or wait.
    const uint32_t maxlast = block_max_u32(last, &s_red);
    if (tid == 0 && maxlast) atomicAdd(&hdr->needed_bwd, (unsigned long long)maxlast);
    if (maxlast == 0) {
        if (tid == 0) cutoff[tile] = make_uint2(0u, 0u);
        return;
    }
    float Sg = 0.f, SD = 0.f;
    const float Kd = -gA * Tfin;
    const uint32_t end = rg.x + maxlast;
    const uint32_t nb = (maxlast - 1) / GB + 1;  // batches; iteration j handles batch nb - 1 - j
    const uint32_t wlast = __reduce_max_sync(0xffffffffu, last);
    const int my_k = scatter_index<P, 16>(lane);  // the warp sum this lane writes, if any
    // Test hook (RAST_FLAG_TEST_BLEND_STALL): iteration 1 is never staged and
    // every wait gives up after 64 polls.
    const bool stall_test = (vt.flags & RAST_FLAG_TEST_BLEND_STALL) != 0;
    const uint32_t polls = stall_test ? 64u : kMbarPolls;

    // Stages iteration j (all 32 lanes of one warp): lane l copies record l of
    // the batch, its point index and its partial-slot base, then arrives on
    // the stage's barrier once its copies have landed.
    // Iterations j >= R take their point indices from s_pnext (loaded by one
    // warp while it worked on iteration j - R, off the staging warp's path).
    auto stage = [&](uint32_t j) {
        if (stall_test && j == 1) return;  // nothing arrives: the waits on this phase run out
        const int st = (int)(j % R);
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            const int rr = g * 32 + lane;
            const uint32_t q = rg.x + (nb - 1 - j) * GB + rr;
            if (q < end) {
                const uint32_t gi = j < (uint32_t)R ? pts[q] : s_pnext[st][rr];
                uint32_t* dst = s_ring + ((size_t)st * GB + rr) * RS;
                const uint32_t* src = rec + (size_t)gi * RW;
#pragma unroll
                for (int w = 0; w < RS; w += 4) cp_async16(dst + w, src + w);
                cp_async4(&s_gi[st][rr], pts + q);
                cp_async4(&s_base[st][rr], base + gi);
            }
        }
        cp_async_mbar_arrive_noinc(&s_mbar[st]);
    };
    if (warp == 0) {
        for (uint32_t j = 0; j < (uint32_t)R && j < nb; ++j) stage(j);
    }

    uint32_t phase = 0;  // parity of the next phase to wait for, per stage
    for (uint32_t j = 0; j < nb; ++j) {
        const int st = (int)(j % R);
        const uint32_t rel0 = (nb - 1 - j) * GB;
        const uint32_t b0 = rg.x + rel0;
        const int nrec = (int)(end - b0 < (uint32_t)GB ? end - b0 : (uint32_t)GB);
        // Every warp waits on every phase, in order, so a parity always refers
        // to the current or the immediately preceding phase. The lanes poll
        // independently; the warp goes on only if all of them saw the phase.
        if (!__all_sync(0xffffffffu, mbar_wait_or_abort(&s_mbar[st], (phase >> st) & 1u, &s_abort, polls))) {
            if (lane == 0) {
                s_abort = 1u;
                atomicOr(&hdr->error, kErrTimeout);
            }
            break;
        }
        phase ^= 1u << st;
        // One warp per iteration loads the point indices of iteration j + R
        // now and stores them before it counts itself done, so the load's
        // latency overlaps its own work on this batch.
        const bool pref = warp == (int)(j % NW) && j + R < nb;
        uint32_t pnext[NG];
        if (pref) {
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                const uint32_t q = rg.x + (nb - 1 - (j + R)) * GB + g * 32 + lane;
                pnext[g] = q < end ? pts[q] : 0u;
            }
        }
        const uint32_t* ring = s_ring + (size_t)st * GB * RS;
        float* contrib = s_contrib + (size_t)(st * NW + warp) * GB * PO;
        // (Hit words start cleared: the batch's last warp clears them.)
#pragma unroll 1
        for (int grp = NG - 1; grp >= 0 && wlast > rel0; --grp) {
            const int r0 = grp * 32;
            bool hit = false;
            if (r0 + lane < nrec) {
                const uint32_t* rp = ring + (r0 + lane) * RS;
                const float um = __fsub_rn(__uint_as_float(rp[0]), 0.5f);
                const float vm = __fsub_rn(__uint_as_float(rp[1]), 0.5f);
                const GaussBox bx = gauss_box(um, vm, __uint_as_float(rp[7]));
                s_box[warp][r0 + lane] = make_int4(bx.x0, bx.x1, bx.y0, bx.y1);
                hit = bx.x0 <= sx0 + 7 && bx.x1 >= sx0 && bx.y0 <= sy0 + 3 && bx.y1 >= sy0;
            }
            uint32_t m = __ballot_sync(0xffffffffu, hit);
            __syncwarp();
            uint32_t written = 0;
            while (m) {
                const int bit = 31 - __clz(m);
                m &= ~(1u << bit);
                const int r = r0 + bit;
                const int4 bb = s_box[warp][r];
                bool act = inside && rel0 + r < last && px >= bb.x && px <= bb.y && py >= bb.z && py <= bb.w;
                const uint32_t* rp = ring + r * RS;
                float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rc = ra;
                float dx = 0.f, dy = 0.f, mm = 0.f;
                if (act) {
                    const uint4 g = *reinterpret_cast<const uint4*>(rp);
                    const uint4 h = *reinterpret_cast<const uint4*>(rp + 4);
                    ra = make_float4(__fsub_rn(__uint_as_float(g.x), 0.5f), __fsub_rn(__uint_as_float(g.y), 0.5f),
                                     __uint_as_float(g.w), __uint_as_float(g.z));
                    rc = make_float4(__uint_as_float(h.x), __uint_as_float(h.y), __uint_as_float(h.z), 0.f);
                    dx = __fsub_rn(fpx, ra.x);
                    dy = __fsub_rn(fpy, ra.y);
                    mm = gauss_m(dx, dy, rc.x, rc.y, rc.z);
                    act = mm <= 9.f;
                }
                if (!__any_sync(0xffffffffu, act)) continue;  // no lane blended this record
                written |= 1u << bit;
                float v[P];
#pragma unroll
                for (int k = 0; k < P; ++k) v[k] = 0.f;
                if (act) {
                    const float G = gauss_value(mm);
                    const float o = ra.z;
                    const float og = __fmul_rn(o, G);
                    const float alpha = fminf(og, amax);
                    const float inv = rcp_fast(__fsub_rn(1.f, alpha));
                    const float Tk = T * inv;  // T_k = T_{k+1} / (1 - alpha_k)
                    float fr[C];
                    load_features<C, BF16>(rp + FW, fr);
                    float fdot = 0.f;
#pragma unroll
                    for (int c = 0; c < C; ++c) fdot = fmaf(gF[c], fr[c], fdot);
                    const float z = ra.w;
                    const float dalpha = Tk * (fdot + gD * z) - (Sg + gD * SD + Kd) * inv;
                    const float ta = Tk * alpha;
                    Sg = fmaf(ta, fdot, Sg);
                    SD = fmaf(ta, z, SD);
                    T = Tk;
#pragma unroll
                    for (int c = 0; c < C; ++c) v[c] = ta * gF[c];
                    v[C + 6] = ta * gD;
                    if (og <= amax) {
                        const float dm = -0.5f * o * G * dalpha;
                        v[C] = G * dalpha;
                        v[C + 1] = -dm * (2.f * rc.x * dx + 2.f * rc.y * dy);
                        v[C + 2] = -dm * (2.f * rc.y * dx + 2.f * rc.z * dy);
                        v[C + 3] = dm * dx * dx;
                        v[C + 4] = dm * 2.f * dx * dy;
                        v[C + 5] = dm * dy * dy;
                    }
                }
                const float sum = warp_reduce_scatter<P, 16>(v, lane);
                if (my_k >= 0) contrib[r * PO + my_k] = sum;
            }
            if (lane == 0) s_hit[st][warp * NG + grp] = written;
        }
        if (pref) {
#pragma unroll
            for (int g = 0; g < NG; ++g) s_pnext[st][g * 32 + lane] = pnext[g];
        }
        // Done with the batch (its rows and hit bits written, its records read).
        __syncwarp();
        __threadfence_block();
        uint32_t prev = 0;
        if (lane == 0) prev = atomicAdd(&s_done[st], 1u);
        prev = __shfl_sync(0xffffffffu, prev, 0);
        if (prev != (uint32_t)(NW - 1)) continue;
        // Last warp of the batch: a lane sums a record's rows in warp order.
        __threadfence_block();
#pragma unroll 1
        for (int g = 0; g < NG; ++g) {
            const int rr = g * 32 + lane;
            if (rr >= nrec) continue;
            float row[PS];
#pragma unroll
            for (int k = 0; k < PS; ++k) row[k] = 0.f;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                if ((s_hit[st][w * NG + g] >> lane) & 1u) {
                    const float* cp = s_contrib + ((size_t)(st * NW + w) * GB + rr) * PO;
#pragma unroll
                    for (int k = 0; k < P; ++k) row[k] += cp[k];
                }
            }
            // The copy's rank in the point's tile rect (the projection's rect
            // of the in-image box) picks its partial slot.
            const uint32_t* rp = ring + rr * RS;
            const float um = __fsub_rn(__uint_as_float(rp[0]), 0.5f);
            const float vm = __fsub_rn(__uint_as_float(rp[1]), 0.5f);
            const GaussBox bx = gauss_box(um, vm, __uint_as_float(rp[7]));
            const int tx0 = max(bx.x0, 0) / TS, tx1 = min(bx.x1, V.W - 1) / TS;
            const int ty0 = max(bx.y0, 0) / TS;
            const int slot = (ty - ty0) * (tx1 - tx0 + 1) + (tx - tx0);
            store_row<PS>(partial + (size_t)(s_base[st][rr] + (uint32_t)slot) * PS, row);
            if (b0 + rr + 1 == end) cutoff[tile] = make_uint2(rp[2], s_gi[st][rr]);
        }
        __syncwarp();  // every lane has read the hit words before they are cleared
        for (int i = lane; i < NW * NG; i += 32) s_hit[st][i] = 0;
        if (lane == 0) s_done[st] = 0;
        // Everything of this batch is read and the stage is clear: refill it.
        __syncwarp();
        __threadfence_block();
        if (j + R < nb) stage(j + R);
    }
    // No copy may land after the CTA has exited (only after a timeout can one
    // still be in flight here).
    cp_async_wait_all();
}

// ---------------------------------------------------------------- K8 reduce

template <int C, int MODE>
__global__ void __launch_bounds__(256, 6) k_reduce_grads(const ViewTable vt, const uint32_t* __restrict__ zbits,
                                                      const uint2* __restrict__ rect,
                                                      const uint32_t* __restrict__ rect4,
                                                      const uint32_t* __restrict__ base,
                                                      const uint2* __restrict__ cutoff,
                                                      const float* __restrict__ partial,
                                                      const float* __restrict__ grow) {
    constexpr int P = MODE == 0 ? C + 1 : C + 7;
    constexpr int PS = partial_stride(P);
    constexpr int GS = grow_stride(P);
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= vt.n_total) return;
    const ViewDev& V = vt.v[view_of_point(vt, gi)];
    const int64_t i = gi - V.pt_off;
    float acc[P];
#pragma unroll
    for (int k = 0; k < P; ++k) acc[k] = 0.f;
    // Independent loads first: one memory round trip for all three.
    const uint2 rc = MODE == 0 ? rect4_unpack(rect4[gi]) : rect[gi];
    const uint32_t zb = zbits[gi];
    const uint32_t pbase = base[gi];
    const uint32_t cnt = rect_count(rc);
    if constexpr (MODE == 0 && direct_feat_grads(C, 16)) {
        if (cnt == 1 && vt.tile == 16) {
            // One copy: the blend wrote dL/df itself if its replay reached the
            // point; dL/do waits in the per-point array.
            const uint2 co = cutoff[V.tile_off + (int64_t)(rc.x >> 16) * V.tiles_x + (rc.x & 0xffff)];
            const bool done = zb < co.x || (zb == co.x && (uint32_t)gi <= co.y);
            if (V.d_opacity) V.d_opacity[i] = done ? grow[(size_t)gi * kOpRow] : 0.f;
            if (!done && V.d_feat) store_row<C>(V.d_feat + i * C, acc);
            if (V.d_xyz) {
                V.d_xyz[3 * i] = 0.f;
                V.d_xyz[3 * i + 1] = 0.f;
                V.d_xyz[3 * i + 2] = 0.f;
            }
            if (V.d_scale) V.d_scale[i] = 0.f;
            return;
        }
    }
    if (MODE == 0 && cnt) {
        // Bilinear: one, two or four tiles. The cutoffs of all of them first,
        // then the rows (two at a time for C <= 11), so a point waits on two
        // memory round trips rather than two per tile; rows still add up in
        // rect order.
        const int tx0 = rc.x & 0xffff, ty0 = rc.x >> 16, tx1 = rc.y & 0xffff;
        const int w = tx1 - tx0 + 1;
        bool dn[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            dn[k] = false;
            if (k < (int)cnt) {
                const uint2 co = cutoff[V.tile_off + (int64_t)(ty0 + k / w) * V.tiles_x + (tx0 + k % w)];
                dn[k] = zb < co.x || (zb == co.x && (uint32_t)gi <= co.y);
            }
        }
        // A point with one copy has its row indexed by point.
        const float* pp = cnt == 1 ? grow + (size_t)gi * GS : partial + (size_t)pbase * PS;
        constexpr int KB = PS <= 12 ? 2 : 1;  // rows in flight (wide rows one at a time: no spills)
#pragma unroll
        for (int k0 = 0; k0 < 4; k0 += KB) {
            if (k0 >= (int)cnt) break;
            float4 x[KB][PS / 4];
#pragma unroll
            for (int h = 0; h < KB; ++h)
#pragma unroll
                for (int j = 0; j < PS / 4; ++j)
                    x[h][j] = dn[k0 + h] ? reinterpret_cast<const float4*>(pp + (size_t)(k0 + h) * PS)[j]
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int h = 0; h < KB; ++h) {
                if (!dn[k0 + h]) continue;
#pragma unroll
                for (int j = 0; j < PS / 4; ++j) {
                    if (4 * j + 0 < P) acc[4 * j + 0] += x[h][j].x;
                    if (4 * j + 1 < P) acc[4 * j + 1] += x[h][j].y;
                    if (4 * j + 2 < P) acc[4 * j + 2] += x[h][j].z;
                    if (4 * j + 3 < P) acc[4 * j + 3] += x[h][j].w;
                }
            }
        }
    } else if (cnt) {
        const int tx0 = rc.x & 0xffff, ty0 = rc.x >> 16, tx1 = rc.y & 0xffff, ty1 = rc.y >> 16;
        const float* pp = partial + (size_t)pbase * PS;
        int k = 0;
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx, ++k) {
                const uint2 co = cutoff[V.tile_off + (int64_t)ty * V.tiles_x + tx];
                const bool done = zb < co.x || (zb == co.x && (uint32_t)gi <= co.y);
                if (!done) continue;
                // Bilinear points with one copy have their row indexed by point.
                const bool own = MODE == 0 && cnt == 1;
                const float4* row = reinterpret_cast<const float4*>(own ? grow + (size_t)gi * GS : pp + (size_t)k * PS);
#pragma unroll
                for (int j = 0; j < PS / 4; ++j) {
                    const float4 x = row[j];
                    if (4 * j + 0 < P) acc[4 * j + 0] += x.x;
                    if (4 * j + 1 < P) acc[4 * j + 1] += x.y;
                    if (4 * j + 2 < P) acc[4 * j + 2] += x.z;
                    if (4 * j + 3 < P) acc[4 * j + 3] += x.w;
                }
            }
    }
    if (V.d_feat) store_row<C>(V.d_feat + i * C, acc);
    if (V.d_opacity) V.d_opacity[i] = acc[C];
    if (MODE == 0) {
        if (V.d_xyz) {
            V.d_xyz[3 * i] = 0.f;
            V.d_xyz[3 * i + 1] = 0.f;
            V.d_xyz[3 * i + 2] = 0.f;
        }
        if (V.d_scale) V.d_scale[i] = 0.f;
        return;
    }
    float gx = 0.f, gy = 0.f, gz = 0.f, gs = 0.f;
    if (cnt) {
        // Camera-space position (same operation order as the projection).
        const float x = V.xyz[3 * i], y = V.xyz[3 * i + 1], zw = V.xyz[3 * i + 2];
        float xc = __fmul_rn(V.R[0], x);
        xc = __fadd_rn(xc, __fmul_rn(V.R[1], y));
        xc = __fadd_rn(xc, __fmul_rn(V.R[2], zw));
        xc = __fadd_rn(xc, V.t[0]);
        float yc = __fmul_rn(V.R[3], x);
        yc = __fadd_rn(yc, __fmul_rn(V.R[4], y));
        yc = __fadd_rn(yc, __fmul_rn(V.R[5], zw));
        yc = __fadd_rn(yc, V.t[1]);
        float zc = __fmul_rn(V.R[6], x);
        zc = __fadd_rn(zc, __fmul_rn(V.R[7], y));
        zc = __fadd_rn(zc, __fmul_rn(V.R[8], zw));
        zc = __fadd_rn(zc, V.t[2]);
        const float fx = V.fx, fy = V.fy;
        const float s = V.scale ? V.scale[i] : __fdiv_rn(__fmul_rn(5.f, V.near_z), fx);
        const float s2 = s * s;
        const float iz = 1.f / zc, iz2 = iz * iz, iz3 = iz2 * iz, iz4 = iz2 * iz2, iz5 = iz4 * iz;
        float S00, S01, S11;
        if (vt.gauss_cov == 0) {
            S00 = s2 * (fx * fx * iz2 + fx * fx * xc * xc * iz4) + vt.dilation;
            S01 = s2 * (fx * fy * xc * yc * iz4);
            S11 = s2 * (fy * fy * iz2 + fy * fy * yc * yc * iz4) + vt.dilation;
        } else {
            S00 = s2 * fx * fy * iz2 + vt.dilation;
            S11 = S00;
            S01 = 0.f;
        }
        const float det = S00 * S11 - S01 * S01;
        const float idet = 1.f / det, idet2 = idet * idet;
        const float dca = acc[C + 3], dcb = acc[C + 4], dcc = acc[C + 5];
        // conic a = S11/det, b = -S01/det, c = S00/det
        const float dS00 = dca * (-S11 * S11 * idet2) + dcb * (S01 * S11 * idet2) +
                           dcc * (idet - S00 * S11 * idet2);
        const float dS11 = dca * (idet - S11 * S00 * idet2) + dcb * (S01 * S00 * idet2) +
                           dcc * (-S00 * S00 * idet2);
        const float dS01 = dca * (2.f * S11 * S01 * idet2) + dcb * (-idet - 2.f * S01 * S01 * idet2) +
                           dcc * (2.f * S00 * S01 * idet2);
        const float du = acc[C + 1], dv = acc[C + 2];
        gx = du * fx * iz;
        gy = dv * fy * iz;
        gz = acc[C + 6] - du * fx * xc * iz2 - dv * fy * yc * iz2;
        if (vt.gauss_cov == 0) {
            gx += dS00 * s2 * fx * fx * 2.f * xc * iz4 + dS01 * s2 * fx * fy * yc * iz4;
            gy += dS11 * s2 * fy * fy * 2.f * yc * iz4 + dS01 * s2 * fx * fy * xc * iz4;
            gz += dS00 * s2 * (-2.f * fx * fx * iz3 - 4.f * fx * fx * xc * xc * iz5) +
                  dS11 * s2 * (-2.f * fy * fy * iz3 - 4.f * fy * fy * yc * yc * iz5) +
                  dS01 * s2 * (-4.f * fx * fy * xc * yc * iz5);
            gs = dS00 * 2.f * s * (fx * fx * iz2 + fx * fx * xc * xc * iz4) +
                 dS11 * 2.f * s * (fy * fy * iz2 + fy * fy * yc * yc * iz4) +
                 dS01 * 2.f * s * (fx * fy * xc * yc * iz4);
        } else {
            const float dS = dS00 + dS11;
            gz += dS * s2 * fx * fy * (-2.f * iz3);
            gs = dS * 2.f * s * fx * fy * iz2;
        }
    }
    if (V.d_xyz) {
        const float* R = V.R;
        V.d_xyz[3 * i + 0] = R[0] * gx + R[3] * gy + R[6] * gz;
        V.d_xyz[3 * i + 1] = R[1] * gx + R[4] * gy + R[7] * gz;
        V.d_xyz[3 * i + 2] = R[2] * gx + R[5] * gy + R[8] * gz;
    }
    if (V.d_scale) V.d_scale[i] = V.scale ? gs : 0.f;
}

template <int TS, int RPT, int C, bool BF16, bool TSRC>
cudaError_t launch_bwd_bilinear(const ViewTable& vt, const Bufs& b, const uint32_t* pts, cudaStream_t s) {
    const unsigned grid = (unsigned)vt.tiles_total;
    constexpr size_t smem = bilinear_bwd_smem<TS, RPT, C, BF16, TSRC>();
    static PerDevice attr;
    const cudaError_t e = per_device(attr, nullptr, [](int, int*) {
        return cudaFuncSetAttribute(k_blend_bwd_bilinear<TS, RPT, C, BF16, TSRC>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (e != cudaSuccess) return e;
    ProfScope ps("blend_bwd", s);
    k_blend_bwd_bilinear<TS, RPT, C, BF16, TSRC><<<grid, TS * TS, smem, s>>>(
        vt, b.ranges, b.order, pts, b.rec, b.rec_tile, b.t_final, b.last, b.base, b.partial, b.grow, b.cutoff,
        b.hdr, b.trace);
    return cudaGetLastError();
}

template <int TS, int C, bool BF16>
cudaError_t launch_gauss_bwd(const ViewTable& vt, const Bufs& b, const uint32_t* pts, cudaStream_t s) {
    const unsigned grid = (unsigned)vt.tiles_total;
    constexpr size_t smem = gauss_bwd_smem<TS, C, BF16>();
    static PerDevice attr;
    const cudaError_t e = per_device(attr, nullptr, [](int, int*) {
        return cudaFuncSetAttribute(k_blend_bwd_gauss<TS, C, BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    });
    if (e != cudaSuccess) return e;
    ProfScope ps("blend_bwd", s);
    k_blend_bwd_gauss<TS, C, BF16><<<grid, TS * TS, smem, s>>>(
        vt, b.ranges, b.order, pts, b.rec, b.t_final, b.last, b.base, b.partial, b.cutoff, b.hdr);
    return cudaGetLastError();
}

template <int TS, int RPT, int C, bool BF16>
cudaError_t launch_bwd_t(const ViewTable& vt, const Bufs& b, const uint32_t* pts, cudaStream_t s) {
    const unsigned grid = (unsigned)vt.tiles_total;
    if (vt.mode == 0) {
        // With the forward's tile-ordered record copy in the workspace, the
        // batches are staged by bulk copies.
        if (b.rec_tile) return launch_bwd_bilinear<TS, RPT, C, BF16, true>(vt, b, pts, s);
        return launch_bwd_bilinear<TS, RPT, C, BF16, false>(vt, b, pts, s);
    } else {
        return launch_gauss_bwd<TS, C, BF16>(vt, b, pts, s);
    }
    return cudaGetLastError();
}

template <int TS, int C, bool BF16>
cudaError_t launch_bwd_d(const ViewTable& vt, const Bufs& b, const uint32_t* pts, cudaStream_t s) {
    const int rpt = vt.mode == 0 ? vt.blend_depth / (TS * TS) : 1;
    if constexpr (TS == 8) {
        if (rpt == 4) return launch_bwd_t<TS, 4, C, BF16>(vt, b, pts, s);
    }
    if (rpt == 2) return launch_bwd_t<TS, 2, C, BF16>(vt, b, pts, s);
    return launch_bwd_t<TS, 1, C, BF16>(vt, b, pts, s);
}

template <int C>
cudaError_t launch_bwd_c(const ViewTable& vt, const Bufs& b, const uint32_t* pts, cudaStream_t s) {
    if (vt.tile == 8)
        return vt.bf16 ? launch_bwd_d<8, C, true>(vt, b, pts, s) : launch_bwd_d<8, C, false>(vt, b, pts, s);
    return vt.bf16 ? launch_bwd_d<16, C, true>(vt, b, pts, s) : launch_bwd_d<16, C, false>(vt, b, pts, s);
}

template <int C>
cudaError_t launch_reduce_c(const ViewTable& vt, const Bufs& b, cudaStream_t s) {
    const unsigned grid = (unsigned)((vt.n_total + 255) / 256);
    ProfScope ps("reduce_grads", s);
    if (vt.mode == 0)
        k_reduce_grads<C, 0><<<grid, 256, 0, s>>>(vt, b.zbits, b.rect, b.rect4, b.base, b.cutoff, b.partial, b.grow);
    else
        k_reduce_grads<C, 1><<<grid, 256, 0, s>>>(vt, b.zbits, b.rect, b.rect4, b.base, b.cutoff, b.partial, b.grow);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blend_bwd(const ViewTable& vt, const Bufs& b, const uint32_t* pts, cudaStream_t s) {
    if (vt.tiles_total == 0) return cudaSuccess;
    switch (vt.C) {
        case 1: return launch_bwd_c<1>(vt, b, pts, s);
        case 2: return launch_bwd_c<2>(vt, b, pts, s);
        case 3: return launch_bwd_c<3>(vt, b, pts, s);
        case 4: return launch_bwd_c<4>(vt, b, pts, s);
        case 8: return launch_bwd_c<8>(vt, b, pts, s);
        case 16: return launch_bwd_c<16>(vt, b, pts, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_reduce_grads(const ViewTable& vt, const Bufs& b, cudaStream_t s) {
    if (vt.n_total == 0) return cudaSuccess;
    switch (vt.C) {
        case 1: return launch_reduce_c<1>(vt, b, s);
        case 2: return launch_reduce_c<2>(vt, b, s);
        case 3: return launch_reduce_c<3>(vt, b, s);
        case 4: return launch_reduce_c<4>(vt, b, s);
        case 8: return launch_reduce_c<8>(vt, b, s);
        case 16: return launch_reduce_c<16>(vt, b, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rast

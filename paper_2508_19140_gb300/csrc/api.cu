// C ABI of the tiled point rasterizer (declared in include/inpc_rast.h).
//
// Host side only: argument checks, the workspace layout, the view table the
// kernels receive by value, and the order of the stages. No stage
// synchronises with the host, so a whole rasterize_batch call can be captured
// in a CUDA graph.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rast_internal.cuh"

namespace rast {
namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

uint32_t f32_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}

int bit_length(uint64_t x) {
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

enum Slot {
    S_HDR, S_REC, S_RECT, S_CNT, S_ZBITS, S_KEYA0, S_KEYA1, S_VALA0, S_VALA1, S_RECTS, S_BASE, S_BLK,
    S_KEYC0, S_KEYC1, S_VALC0, S_VALC1, S_PARTIAL, S_GROW, S_SGHIST, S_SCOUNT, S_SSTATUS, S_RANGES, S_ORDER, S_CUTOFF, S_TRACE,
    S_TFINAL, S_LAST, S_PIXC, S_PTC, S_RECTILE, S_COUNT
};
const char* kSlotNames[S_COUNT] = {
    "header", "records", "rect", "count", "zbits", "keys_a0", "keys_a1", "vals_a0", "vals_a1",
    "rect_sorted", "base", "block_sums", "keys_c0", "keys_c1", "vals_c0", "vals_c1",
    "partial", "grad_rows", "sort_hist", "sort_counters", "sort_status", "ranges", "tile_order", "cutoff", "tile_trace", "t_final", "last",
    "copy_pixel", "copy_point", "records_tiled"};

// Arrangements of the pipeline.
enum Arrangement {
    kTiled = 0,        // tiles of opts->tile pixels, split sort (the paper's method)
    kUntiledSplit = 1, // one-pixel tiles through the split sort, one thread per pixel
    kUntiledKey64 = 2  // one-pixel tiles, one 64-bit [pixel | depth] key sort of copies, one warp per pixel
};

struct Plan {
    ViewTable vt;
    size_t off[S_COUNT];
    size_t bytes[S_COUNT];
    size_t total;
    int64_t copy_cap, blk_cap;
    SortPlan planA, planC;
    int partial_floats;
    int arrangement;
    bool save_tiled;  // the forward writes the tile-ordered record copy
};

int32_t write_layout(const Plan& pl, int keys_slot, int vals_slot, rast_ws_entry_t* out, int32_t max);

rast_status_t check_view(const rast_view_t& v, int pass, int T) {
    const rast_points_t& p = v.pts;
    const rast_camera_t& c = v.cam;
    if (p.n < 0) return RAST_ERR_ARG;
    if (p.n > 0 && (!p.xyz || !p.opacity || !p.feat)) return RAST_ERR_ARG;
    if (c.width < 1 || c.height < 1 || c.width > 65535 * T || c.height > 65535 * T)
        return RAST_ERR_ARG;
    if (!(c.near_z > 0.f) || !(c.far_z > c.near_z) || !std::isfinite(c.far_z)) return RAST_ERR_ARG;
    const float* cf = &c.fx;
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(cf[k])) return RAST_ERR_ARG;
    if ((pass & RAST_PASS_FWD) && !v.out.feat) return RAST_ERR_ARG;
    if ((pass & RAST_PASS_BWD) && !v.grad.g_feat) return RAST_ERR_ARG;
    return RAST_OK;
}

// Compiled blend depths (records per blend batch): bilinear tile^2 x {1, 2},
// and x 4 for 8x8 tiles; Gaussian tile^2.
bool blend_depth_supported(int mode, int tile, int depth) {
    const int nt = tile * tile;
    if (depth == nt) return true;
    if (mode != RAST_SPLAT_BILINEAR) return false;
    return depth == 2 * nt || (tile == 8 && depth == 4 * nt);
}

// cont[k] != 0: view k is another point cloud of view k - 1's image (same
// camera, outputs and image gradients; its points join the same tile lists).
// arrangement: see Arrangement (the untiled ones have one "tile" per pixel:
// per-pixel lists, the untiled baselines).
rast_status_t make_plan(const rast_view_t* views, int32_t n_views, const rast_opts_t* o, int pass,
                        Plan& pl, const uint8_t* cont = nullptr, int arrangement = kTiled) {
    const bool untiled = arrangement != kTiled;
    if (!views || !o || n_views < 1 || n_views > kMaxViews) return RAST_ERR_ARG;
    if (o->mode != RAST_SPLAT_BILINEAR && o->mode != RAST_SPLAT_GAUSSIAN) return RAST_ERR_ARG;
    if (o->gauss_cov != RAST_GAUSS_EWA && o->gauss_cov != RAST_GAUSS_ISO_SCREEN) return RAST_ERR_ARG;
    const int T = untiled ? 1 : o->tile;
    if (untiled && (o->mode != RAST_SPLAT_BILINEAR || (pass & RAST_PASS_BWD))) return RAST_ERR_NOT_SUPPORTED;
    if (!untiled && o->tile != 8 && o->tile != 16) return RAST_ERR_NOT_SUPPORTED;
    const int depth = untiled ? 1 : (o->blend_depth == 0 ? o->tile * o->tile : o->blend_depth);
    if (!untiled && !blend_depth_supported(o->mode, o->tile, depth)) return RAST_ERR_NOT_SUPPORTED;
    if (!(o->t_min >= 0.f) || !(o->alpha_max > 0.f && o->alpha_max < 1.f)) return RAST_ERR_ARG;
    if (!(o->dilation >= 0.f) || o->max_copies < 0) return RAST_ERR_ARG;
    if ((o->flags & ~(RAST_FLAG_TEST_SORT_STALL | RAST_FLAG_SAVE_FOR_BWD | RAST_FLAG_TEST_BLEND_STALL)) != 0)
        return RAST_ERR_ARG;
    const int C = views[0].pts.channels;
    const int dt = views[0].pts.feat_dtype;
    if (dt != RAST_F32 && dt != RAST_BF16) return RAST_ERR_ARG;
    if (C < 1) return RAST_ERR_ARG;
    if (!channels_supported(C)) return RAST_ERR_NOT_SUPPORTED;
    std::memset(&pl, 0, sizeof(pl));
    pl.arrangement = arrangement;
    ViewTable& vt = pl.vt;
    vt.n_views = n_views;
    vt.C = C;
    vt.bf16 = dt == RAST_BF16;
    vt.mode = o->mode;
    vt.gauss_cov = o->gauss_cov;
    vt.tile = T;
    vt.blend_depth = depth;
    vt.t_min = o->t_min;
    vt.alpha_max = o->alpha_max;
    vt.dilation = o->dilation;
    vt.flags = o->flags;
    vt.feat_word = o->mode == RAST_SPLAT_GAUSSIAN ? 8 : 4;
    // Power-of-two record stride of at least 8 words (see RecLayout).
    const int fwords = vt.bf16 ? (C + 1) / 2 : C;
    const int need = vt.feat_word + fwords;
    vt.rec_words = need <= 8 ? 8 : (need <= 16 ? 16 : 32);
    int64_t npt = 0, ntile = 0, npix = 0;
    uint32_t max_cull = 1;
    int prim = 0;  // the view that owns the image of view k
    for (int k = 0; k < n_views; ++k) {
        const rast_view_t& v = views[k];
        if (v.pts.channels != C || v.pts.feat_dtype != dt) return RAST_ERR_ARG;
        const bool joins = cont && cont[k] && k > 0;
        if (!joins) prim = k;
        if (joins) vt.shared_tiles = 1;
        rast_status_t st = check_view(v, pass, T);
        if (st != RAST_OK) return st;
        ViewDev& d = vt.v[k];
        const rast_camera_t& c = v.cam;
        d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
        for (int j = 0; j < 9; ++j) d.R[j] = c.R[j];
        for (int j = 0; j < 3; ++j) d.t[j] = c.t[j];
        d.near_z = c.near_z;
        d.far_z = c.far_z;
        d.W = c.width;
        d.H = c.height;
        d.tiles_x = (c.width + T - 1) / T;
        d.tiles_y = (c.height + T - 1) / T;
        // Bilinear rects are packed into 32 bits (14 bits of tile row).
        if (o->mode == RAST_SPLAT_BILINEAR && d.tiles_y > kRect4MaxTilesY) return RAST_ERR_NOT_SUPPORTED;
        d.key_base = f32_bits(c.near_z);
        d.key_cull = f32_bits(c.far_z) - f32_bits(c.near_z);
        if (d.key_cull > max_cull) max_cull = d.key_cull;
        d.pt_off = npt;
        d.n = v.pts.n;
        d.tile_off = joins ? vt.v[prim].tile_off : ntile;
        d.pix_off = joins ? vt.v[prim].pix_off : npix;
        d.xyz = v.pts.xyz;
        d.opacity = v.pts.opacity;
        d.feat = v.pts.feat;
        d.scale = v.pts.scale;
        d.out_feat = v.out.feat;
        d.out_alpha = v.out.alpha;
        d.out_depth = v.out.depth;
        d.g_feat = v.grad.g_feat;
        d.g_alpha = v.grad.g_alpha;
        d.g_depth = v.grad.g_depth;
        d.d_feat = v.grad.d_feat;
        d.d_opacity = v.grad.d_opacity;
        d.d_xyz = v.grad.d_xyz;
        d.d_scale = v.grad.d_scale;
        if (joins) {
            // Same image as the owning view: its outputs and image gradients.
            const ViewDev& P = vt.v[prim];
            d.out_feat = P.out_feat;
            d.out_alpha = P.out_alpha;
            d.out_depth = P.out_depth;
            d.g_feat = P.g_feat;
            d.g_alpha = P.g_alpha;
            d.g_depth = P.g_depth;
        }
        npt += v.pts.n;
        if (!joins) {
            ntile += (int64_t)d.tiles_x * d.tiles_y;
            npix += (int64_t)c.width * c.height;
        }
    }
    if (npt >= ((int64_t)1 << 30) || ntile >= ((int64_t)1 << 30) || npix >= ((int64_t)1 << 40))
        return RAST_ERR_ARG;
    vt.n_total = npt;
    vt.tiles_total = ntile;
    vt.pix_total = npix;

    const int64_t per_pt = o->max_copies > 0 ? o->max_copies : (o->mode == RAST_SPLAT_BILINEAR ? 4 : 16);
    // Copy capacity: sort prefixes are 30-bit values, so at most 2^30 - 1 copies
    // (beyond that the forward reports RAST_ERR_CAPACITY).
    pl.copy_cap = npt * per_pt;
    if (pl.copy_cap >= ((int64_t)1 << 30)) pl.copy_cap = ((int64_t)1 << 30) - 1;
    pl.blk_cap = (npt + kScanItems - 1) / kScanItems + 1;
    // Depth keys of a batch with several images carry the image index above
    // the depth bits, so the depth order is image-major (views joined into
    // one image keep one depth order). The copies of one tile all belong to
    // one image, so the tile lists are unchanged; the duplication pass then
    // reads each image's packed rects as a contiguous slice rather than
    // gathering over the whole batch.
    uint64_t key_max = max_cull;
    {
        const int db = bit_length(max_cull);
        int nimg = 0;
        for (int k = 0; k < n_views; ++k)
            if (!(cont && cont[k] && k > 0)) ++nimg;
        const int ib = bit_length((uint64_t)(nimg - 1));
        if (ib > 0 && db + ib <= 32) {
            int img = -1;
            for (int k = 0; k < n_views; ++k) {
                if (!(cont && cont[k] && k > 0)) ++img;
                const uint32_t hi = (uint32_t)img << db;
                vt.v[k].key_base -= hi;  // bits(z) - key_base = (bits(z) - bits(near)) + hi (mod 2^32)
                vt.v[k].key_cull += hi;
            }
            key_max = ((uint64_t)(nimg - 1) << db) | max_cull;
        }
    }
    pl.planA = make_sort_plan(bit_length(key_max));
    pl.planC = make_sort_plan(bit_length((uint64_t)(ntile > 0 ? ntile - 1 : 0)));
    pl.partial_floats = partial_stride(o->mode == RAST_SPLAT_BILINEAR ? C + 1 : C + 7);

    const int64_t N = npt, D = pl.copy_cap;
    pl.bytes[S_HDR] = sizeof(WsHeader);
    pl.bytes[S_REC] = (size_t)N * vt.rec_words * 4;
    pl.bytes[S_RECT] = (size_t)N * 8;
    pl.bytes[S_CNT] = (size_t)N * 4;
    pl.bytes[S_ZBITS] = (size_t)N * 4;
    pl.bytes[S_KEYA0] = pl.bytes[S_KEYA1] = pl.bytes[S_VALA0] = pl.bytes[S_VALA1] = (size_t)N * 4;
    pl.bytes[S_RECTS] = (size_t)N * 8;
    pl.bytes[S_BASE] = (size_t)N * 4;
    pl.bytes[S_BLK] = (size_t)pl.blk_cap * 4;
    pl.bytes[S_KEYC0] = pl.bytes[S_KEYC1] = pl.bytes[S_VALC0] = pl.bytes[S_VALC1] = (size_t)D * 4;
    pl.bytes[S_PARTIAL] = (size_t)D * pl.partial_floats * 4;
    pl.bytes[S_GROW] = o->mode == RAST_SPLAT_BILINEAR ? (size_t)N * grow_stride(C + 1) * 4 : 0;
    pl.bytes[S_SGHIST] = (size_t)kMaxSortPasses * 512 * 4;
    pl.bytes[S_SCOUNT] = (size_t)kMaxSortPasses * 4;
    {
        // The 64-bit-key arrangement sorts copies, not points, by depth.
        const int64_t na = arrangement == kUntiledKey64 ? pl.copy_cap : npt;
        const int64_t wa = sort_status_words(pl.planA, na), wc = sort_status_words(pl.planC, pl.copy_cap);
        pl.bytes[S_SSTATUS] = (size_t)(wa > wc ? wa : wc) * 4;
    }
    pl.bytes[S_PIXC] = pl.bytes[S_PTC] = arrangement == kUntiledKey64 ? (size_t)D * 4 : 0;
    // Bilinear tiled: the forward blend writes every record it reads, in
    // tile-list order, so the backward reads its batches sequentially.
    pl.save_tiled = arrangement == kTiled && o->mode == RAST_SPLAT_BILINEAR &&
                    (o->flags & RAST_FLAG_SAVE_FOR_BWD) != 0;
    pl.bytes[S_RECTILE] = pl.save_tiled ? (size_t)D * vt.rec_words * 4 : 0;
    pl.bytes[S_RANGES] = (size_t)ntile * 8;
    pl.bytes[S_ORDER] = (size_t)(ntile + 66) * 4;  // heavy-first order + bucket counts and cursors
    pl.bytes[S_CUTOFF] = (size_t)ntile * 8;
    pl.bytes[S_TRACE] = (size_t)ntile * 2 * 4 * 8;
    pl.bytes[S_TFINAL] = (size_t)npix * 4;
    pl.bytes[S_LAST] = (size_t)npix * 4;
    size_t off = 0;
    for (int k = 0; k < S_COUNT; ++k) {
        pl.off[k] = off;
        off += align_up(pl.bytes[k] ? pl.bytes[k] : 1);
    }
    pl.total = off;
    return RAST_OK;
}

}  // namespace

namespace {

Bufs make_bufs(const Plan& pl, void* ws) {
    char* w = static_cast<char*>(ws);
    auto at = [&](int s) { return (void*)(w + pl.off[s]); };
    Bufs b;
    std::memset(&b, 0, sizeof(b));
    b.hdr = (WsHeader*)at(S_HDR);
    b.rec = (uint32_t*)at(S_REC);
    b.rect = (uint2*)at(S_RECT);
    b.rect4 = (uint32_t*)at(S_RECT);
    b.cnt = (uint32_t*)at(S_CNT);
    b.zbits = (uint32_t*)at(S_ZBITS);
    b.keyA[0] = (uint32_t*)at(S_KEYA0);
    b.keyA[1] = (uint32_t*)at(S_KEYA1);
    b.valA[0] = (uint32_t*)at(S_VALA0);
    b.valA[1] = (uint32_t*)at(S_VALA1);
    b.rectS = (uint2*)at(S_RECTS);
    b.rect4S = (uint32_t*)at(S_RECTS);
    b.base = (uint32_t*)at(S_BASE);
    b.blk = (uint32_t*)at(S_BLK);
    b.keyC[0] = (uint32_t*)at(S_KEYC0);
    b.keyC[1] = (uint32_t*)at(S_KEYC1);
    b.valC[0] = (uint32_t*)at(S_VALC0);
    b.valC[1] = (uint32_t*)at(S_VALC1);
    b.partial = (float*)at(S_PARTIAL);
    b.grow = (float*)at(S_GROW);
    b.sort_ghist = (uint32_t*)at(S_SGHIST);
    b.sort_counters = (uint32_t*)at(S_SCOUNT);
    b.sort_status = (uint32_t*)at(S_SSTATUS);
    b.ranges = (uint2*)at(S_RANGES);
    b.order = (uint32_t*)at(S_ORDER);
    b.cutoff = (uint2*)at(S_CUTOFF);
    b.trace = (unsigned long long*)at(S_TRACE);
    b.t_final = (float*)at(S_TFINAL);
    b.last = (uint32_t*)at(S_LAST);
    b.pixC = (uint32_t*)at(S_PIXC);
    b.ptC = (uint32_t*)at(S_PTC);
    b.rec_tile = pl.save_tiled ? (uint32_t*)at(S_RECTILE) : nullptr;
    b.copy_cap = pl.copy_cap;
    b.blk_cap = pl.blk_cap;
    return b;
}

__global__ void k_init_header(WsHeader* h, int32_t n_views, long long n_points, long long cap,
                              long long n_tiles, long long n_pixels, uint32_t rec_tile_valid) {
    h->rec_tile_valid = rec_tile_valid;
    h->error = 0u;
    h->n_copies = 0u;
    h->n_copies_raw = 0u;
    h->n_views = (uint32_t)n_views;
    h->needed = 0ull;
    h->needed_bwd = 0ull;
    h->n_points = n_points;
    h->copy_cap = cap;
    h->n_tiles = n_tiles;
    h->n_pixels = n_pixels;
}

// ---- per-stage profiling ---------------------------------------------------

struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
};

struct Profiler {
    std::mutex mu;
    bool on = false;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;

    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};
Profiler g_prof;

}  // namespace

int device_sm_count() {
    static PerDevice pd;
    int n = 1;
    const cudaError_t e = per_device(pd, &n, [](int dev, int* v) {
        *v = 1;
        int c = 0;
        const cudaError_t r = cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        if (r == cudaSuccess && c > 0) *v = c;
        return cudaSuccess;
    });
    return e == cudaSuccess && n > 0 ? n : 1;
}

ProfScope::ProfScope(const char* name, cudaStream_t st) : idx(-1), s(st) {
    nvtxRangePushA(name);  // a no-op unless a profiler is attached
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (!g_prof.on) return;
    ProfRec r{name, g_prof.get(), g_prof.get()};
    cudaEventRecord(r.a, s);
    g_prof.recs.push_back(r);
    idx = (int)g_prof.recs.size() - 1;
}

ProfScope::~ProfScope() {
    nvtxRangePop();
    if (idx < 0) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (idx < (int)g_prof.recs.size()) cudaEventRecord(g_prof.recs[idx].b, s);
}

namespace {

#define RAST_TRY(expr)                      \
    do {                                    \
        cudaError_t e_ = (expr);            \
        if (e_ != cudaSuccess) return e_;   \
    } while (0)

const char* const kDepthSortNames[2] = {"depth_sort.hist", "depth_sort.sweep"};
const char* const kTileSortNames[2] = {"tile_sort.hist", "tile_sort.sweep"};

cudaError_t run_fwd(const Plan& pl, const Bufs& b, cudaStream_t s) {
    const ViewTable& vt = pl.vt;
    {
        ProfScope ps("init_header", s);
        k_init_header<<<1, 1, 0, s>>>(b.hdr, vt.n_views, vt.n_total, pl.copy_cap, vt.tiles_total,
                                      vt.pix_total, pl.save_tiled ? 1u : 0u);
        RAST_TRY(cudaGetLastError());
    }
    // The depth sort's first pass generates the point indices itself.
    RAST_TRY(launch_project(vt, b, pl.planA.passes == 0, s));
    int ra = 0, rc = 0;
    {
        uint32_t* k[2] = {b.keyA[0], b.keyA[1]};
        uint32_t* v[2] = {b.valA[0], b.valA[1]};
        const SortScratch sc{b.sort_ghist, b.sort_counters, b.sort_status, &b.hdr->error,
                             (vt.flags & RAST_FLAG_TEST_SORT_STALL) != 0};
        // Only the depth order of the point indices is used after this sort.
        RAST_TRY(radix_sort(k, v, vt.n_total, nullptr, vt.n_total, pl.planA, sc, s, &ra, kDepthSortNames,
                            true, false));
    }
    const uint32_t* depth_sorted = b.valA[ra];
    // A depth sort whose look-back wait ran out leaves a partial order: the
    // duplication then sees the error bit and writes no copies.
    RAST_TRY(launch_duplicate(vt, b, depth_sorted, s));
    {
        uint32_t* k[2] = {b.keyC[0], b.keyC[1]};
        uint32_t* v[2] = {b.valC[0], b.valC[1]};
        const SortScratch sc{b.sort_ghist, b.sort_counters, b.sort_status, &b.hdr->error};
        RAST_TRY(radix_sort(k, v, 0, &b.hdr->n_copies, pl.copy_cap, pl.planC, sc, s, &rc, kTileSortNames));
    }
    RAST_TRY(launch_ranges(vt, b, b.keyC[rc], s));
    if (vt.tile == 1) return launch_blend_fwd_pixel(vt, b, b.valC[rc], s);  // untiled baseline
    RAST_TRY(launch_tile_order(vt, b, s));
    RAST_TRY(launch_blend_fwd(vt, b, b.valC[rc], s));
    return cudaSuccess;
}

// Untiled baseline with ONE stable LSD radix sort over the copies' 64-bit key
// [pixel id | depth key] (ties: point index), the arrangement whose cost
// Sec. 3.2 "Tiled Rendering" counts as 28n: every point makes a copy per
// in-image pixel of its 2x2 box (about 4n copies), written in point order.
// The LSD passes over the low word (depth digits) carry the copy id; before
// the passes over the high word (pixel digits) each copy's high word and point
// index are fetched by that id, and those passes carry the point index. The
// key the passes see is the same 64-bit key digit for digit; only its high
// word is read when its digits are reached. Result: (pixel, point) pairs in
// (pixel, depth, point index) order in keys/vals[result_pair(pl)].
int key64_result_pair(const Plan& pl) {
    const int ga = pl.planA.passes & 1;  // pair holding the low-word passes' copy ids
    const int g = ga ^ 1;                // the free pair the gather fills
    return g ^ (pl.planC.passes & 1);
}

cudaError_t run_fwd_key64(const Plan& pl, const Bufs& b, cudaStream_t s) {
    const ViewTable& vt = pl.vt;
    {
        ProfScope ps("init_header", s);
        k_init_header<<<1, 1, 0, s>>>(b.hdr, vt.n_views, vt.n_total, pl.copy_cap, vt.tiles_total,
                                      vt.pix_total, pl.save_tiled ? 1u : 0u);
        RAST_TRY(cudaGetLastError());
    }
    RAST_TRY(launch_project(vt, b, false, s));
    RAST_TRY(launch_untiled_copies(vt, b, b.keyA[0], b.keyC[0], b.pixC, b.ptC, s));
    const SortScratch sc{b.sort_ghist, b.sort_counters, b.sort_status, &b.hdr->error,
                         (vt.flags & RAST_FLAG_TEST_SORT_STALL) != 0};
    static const char* const kLoNames[2] = {"sort64.lo.hist", "sort64.lo.sweep"};
    static const char* const kHiNames[2] = {"sort64.hi.hist", "sort64.hi.sweep"};
    int ra = 0, rb = 0;
    {
        uint32_t* k[2] = {b.keyC[0], b.keyC[1]};
        uint32_t* v[2] = {b.valC[0], b.valC[1]};
        // Low word: the values are the copy ids (generated by the first pass).
        RAST_TRY(radix_sort(k, v, 0, &b.hdr->n_copies, pl.copy_cap, pl.planA, sc, s, &ra, kLoNames, true, false));
    }
    const int g = ra ^ 1;
    RAST_TRY(launch_gather_hi(b, b.valC[ra], b.pixC, b.ptC, b.keyC[g], b.valC[g], s));
    {
        uint32_t* k[2] = {b.keyC[g], b.keyC[ra]};
        uint32_t* v[2] = {b.valC[g], b.valC[ra]};
        SortScratch sc2 = sc;
        sc2.stall_test = false;
        RAST_TRY(radix_sort(k, v, 0, &b.hdr->n_copies, pl.copy_cap, pl.planC, sc2, s, &rb, kHiNames));
    }
    const int r = key64_result_pair(pl);
    RAST_TRY(launch_ranges(vt, b, b.keyC[r], s));
    return launch_blend_fwd_pixel_warp(vt, b, b.valC[r], s);
}

cudaError_t run_bwd(const Plan& pl, const Bufs& b, cudaStream_t s) {
    const ViewTable& vt = pl.vt;
    const int rc = pl.planC.passes & 1;
    RAST_TRY(cudaMemsetAsync(&b.hdr->needed_bwd, 0, sizeof(unsigned long long), s));
    RAST_TRY(launch_point_scan(vt, b, s));
    RAST_TRY(launch_blend_bwd(vt, b, b.valC[rc], s));
    RAST_TRY(launch_reduce_grads(vt, b, s));
    return cudaSuccess;
}

rast_view_t single_view(const rast_points_t* pts, const rast_camera_t* cam, const rast_images_t* out,
                        const rast_grads_t* grads) {
    rast_view_t v;
    std::memset(&v, 0, sizeof(v));
    v.pts = *pts;
    v.cam = *cam;
    if (out) v.out = *out;
    if (grads) v.grad = *grads;
    return v;
}

// One launch sequence over the views (cont: see make_plan).
rast_status_t run_views(const rast_view_t* views, int32_t n_views, int32_t pass, const rast_opts_t* opts,
                        void* workspace, size_t ws_bytes, void* stream, const uint8_t* cont,
                        int arrangement = kTiled) {
    if (pass < 1 || pass > 3) return RAST_ERR_ARG;
    Plan pl;
    const rast_status_t st = make_plan(views, n_views, opts, pass, pl, cont, arrangement);
    if (st != RAST_OK) return st;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) return RAST_ERR_ARG;
    if (ws_bytes < pl.total) return RAST_ERR_CAPACITY;
    Bufs b = make_bufs(pl, workspace);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (pass & RAST_PASS_FWD) {
        const cudaError_t e = arrangement == kUntiledKey64 ? run_fwd_key64(pl, b, s) : run_fwd(pl, b, s);
        if (e != cudaSuccess) return RAST_ERR_CUDA;
    }
    if (pass & RAST_PASS_BWD) {
        if (run_bwd(pl, b, s) != cudaSuccess) return RAST_ERR_CUDA;
    }
    return RAST_OK;
}

}  // namespace
}  // namespace rast

using namespace rast;

extern "C" {

void rast_default_opts(rast_opts_t* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->mode = RAST_SPLAT_BILINEAR;
    o->gauss_cov = RAST_GAUSS_EWA;
    o->tile = kTileDefault;
    o->blend_depth = 0;
    o->t_min = 1e-4f;
    o->alpha_max = 0.99f;
    o->dilation = 0.16f;
    o->max_copies = 0;
    o->flags = 0;
}

size_t rasterize_workspace_size(const rast_view_t* views, int32_t n_views, const rast_opts_t* opts) {
    Plan pl;
    if (make_plan(views, n_views, opts, 0, pl) != RAST_OK) return 0;
    return pl.total;
}

int32_t rasterize_workspace_layout(const rast_view_t* views, int32_t n_views, const rast_opts_t* opts,
                                   rast_ws_entry_t* out, int32_t max) {
    Plan pl;
    if (make_plan(views, n_views, opts, 0, pl) != RAST_OK) return -1;
    const int rc = pl.planC.passes & 1;
    return write_layout(pl, rc ? S_KEYC1 : S_KEYC0, rc ? S_VALC1 : S_VALC0, out, max);
}

}  // extern "C"

namespace rast {
namespace {

// Every workspace array as (name, offset, bytes), then the aliases of the
// sort results: "depth_sorted" (point indices in depth order), "sorted_keys"
// and "sorted_vals" (the slots given).
int32_t write_layout(const Plan& pl, int keys_slot, int vals_slot, rast_ws_entry_t* out, int32_t max) {
    const int ra = pl.planA.passes & 1;
    struct Alias { const char* name; int slot; };
    const Alias extra[] = {{"depth_sorted", ra ? S_VALA1 : S_VALA0},
                           {"sorted_keys", keys_slot},
                           {"sorted_vals", vals_slot}};
    int n = 0;
    for (int k = 0; k < S_COUNT; ++k, ++n) {
        if (out && n < max) {
            std::snprintf(out[n].name, sizeof(out[n].name), "%s", kSlotNames[k]);
            out[n].offset = (int64_t)pl.off[k];
            out[n].bytes = (int64_t)pl.bytes[k];
        }
    }
    for (const Alias& a : extra) {
        if (out && n < max) {
            std::snprintf(out[n].name, sizeof(out[n].name), "%s", a.name);
            out[n].offset = (int64_t)pl.off[a.slot];
            out[n].bytes = (int64_t)pl.bytes[a.slot];
        }
        ++n;
    }
    return n;
}

}  // namespace
}  // namespace rast

extern "C" {

rast_status_t rasterize_batch(const rast_view_t* views, int32_t n_views, int32_t pass,
                              const rast_opts_t* opts, void* workspace, size_t ws_bytes,
                              void* stream) {
    return run_views(views, n_views, pass, opts, workspace, ws_bytes, stream, nullptr);
}

}  // extern "C"

namespace {

// Builds the view list of a multi-cloud image: cloud k becomes view k, views
// 1.. join view 0's image.
rast_status_t cloud_views(const rast_points_t* clouds, const rast_grads_t* grads, int32_t n_clouds,
                          const rast_camera_t* cam, const rast_images_t* out, rast_view_t* views,
                          uint8_t* cont) {
    if (!clouds || !cam || !out || n_clouds < 1 || n_clouds > kMaxViews) return RAST_ERR_ARG;
    for (int k = 0; k < n_clouds; ++k) {
        std::memset(&views[k], 0, sizeof(rast_view_t));
        views[k].pts = clouds[k];
        views[k].cam = *cam;
        views[k].out = *out;
        if (grads) {
            views[k].grad = grads[k];
            views[k].grad.g_feat = grads[0].g_feat;
            views[k].grad.g_alpha = grads[0].g_alpha;
            views[k].grad.g_depth = grads[0].g_depth;
        }
        cont[k] = k > 0;
    }
    return RAST_OK;
}

}  // namespace

extern "C" {

size_t rasterize_clouds_workspace_size(const rast_points_t* clouds, int32_t n_clouds, const rast_camera_t* cam,
                                       const rast_opts_t* opts) {
    rast_view_t views[kMaxViews];
    uint8_t cont[kMaxViews];
    rast_images_t dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    if (cloud_views(clouds, nullptr, n_clouds, cam, &dummy, views, cont) != RAST_OK) return 0;
    Plan pl;
    if (make_plan(views, n_clouds, opts, 0, pl, cont) != RAST_OK) return 0;
    return pl.total;
}

rast_status_t rasterize_clouds(const rast_points_t* clouds, const rast_grads_t* grads, int32_t n_clouds,
                               const rast_camera_t* cam, const rast_images_t* out, int32_t pass,
                               const rast_opts_t* opts, void* workspace, size_t ws_bytes, void* stream) {
    rast_view_t views[kMaxViews];
    uint8_t cont[kMaxViews];
    if ((pass & RAST_PASS_BWD) && !grads) return RAST_ERR_ARG;
    const rast_status_t st = cloud_views(clouds, grads, n_clouds, cam, out, views, cont);
    if (st != RAST_OK) return st;
    return run_views(views, n_clouds, pass, opts, workspace, ws_bytes, stream, cont);
}

}  // extern "C"

extern "C" {

size_t rasterize_untiled_workspace_size(const rast_points_t* pts, const rast_camera_t* cam,
                                        const rast_opts_t* opts) {
    if (!pts || !cam) return 0;
    rast_images_t dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    const rast_view_t v = single_view(pts, cam, &dummy, nullptr);
    Plan pl;
    if (make_plan(&v, 1, opts, 0, pl, nullptr, kUntiledSplit) != RAST_OK) return 0;
    return pl.total;
}

rast_status_t rasterize_fwd_untiled(const rast_points_t* pts, const rast_camera_t* cam, const rast_opts_t* opts,
                                    void* workspace, size_t ws_bytes, const rast_images_t* out, void* stream) {
    if (!pts || !cam || !out) return RAST_ERR_ARG;
    const rast_view_t v = single_view(pts, cam, out, nullptr);
    return run_views(&v, 1, RAST_PASS_FWD, opts, workspace, ws_bytes, stream, nullptr, kUntiledSplit);
}

size_t rasterize_untiled64_workspace_size(const rast_points_t* pts, const rast_camera_t* cam,
                                          const rast_opts_t* opts) {
    if (!pts || !cam) return 0;
    rast_images_t dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    const rast_view_t v = single_view(pts, cam, &dummy, nullptr);
    Plan pl;
    if (make_plan(&v, 1, opts, 0, pl, nullptr, kUntiledKey64) != RAST_OK) return 0;
    return pl.total;
}

int32_t rasterize_untiled64_workspace_layout(const rast_points_t* pts, const rast_camera_t* cam,
                                             const rast_opts_t* opts, rast_ws_entry_t* out, int32_t max) {
    if (!pts || !cam) return -1;
    rast_images_t dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    const rast_view_t v = single_view(pts, cam, &dummy, nullptr);
    Plan pl;
    if (make_plan(&v, 1, opts, 0, pl, nullptr, kUntiledKey64) != RAST_OK) return -1;
    const int r = key64_result_pair(pl);
    return write_layout(pl, r ? S_KEYC1 : S_KEYC0, r ? S_VALC1 : S_VALC0, out, max);
}

rast_status_t rasterize_fwd_untiled64(const rast_points_t* pts, const rast_camera_t* cam, const rast_opts_t* opts,
                                      void* workspace, size_t ws_bytes, const rast_images_t* out, void* stream) {
    if (!pts || !cam || !out) return RAST_ERR_ARG;
    const rast_view_t v = single_view(pts, cam, out, nullptr);
    return run_views(&v, 1, RAST_PASS_FWD, opts, workspace, ws_bytes, stream, nullptr, kUntiledKey64);
}

rast_status_t rasterize_fwd(const rast_points_t* pts, const rast_camera_t* cam, const rast_opts_t* opts,
                            void* workspace, size_t ws_bytes, const rast_images_t* out, void* stream) {
    if (!pts || !cam || !out) return RAST_ERR_ARG;
    const rast_view_t v = single_view(pts, cam, out, nullptr);
    return rasterize_batch(&v, 1, RAST_PASS_FWD, opts, workspace, ws_bytes, stream);
}

rast_status_t rasterize_bwd(const rast_points_t* pts, const rast_camera_t* cam, const rast_opts_t* opts,
                            void* workspace, size_t ws_bytes, const rast_grads_t* grads, void* stream) {
    if (!pts || !cam || !grads) return RAST_ERR_ARG;
    const rast_view_t v = single_view(pts, cam, nullptr, grads);
    return rasterize_batch(&v, 1, RAST_PASS_BWD, opts, workspace, ws_bytes, stream);
}

rast_status_t rasterize_get_status(const void* workspace, size_t ws_bytes, void* stream,
                                   rast_stats_t* stats) {
    if (!workspace || ws_bytes < sizeof(WsHeader)) return RAST_ERR_ARG;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return RAST_ERR_CUDA;
    WsHeader h;
    if (cudaMemcpy(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return RAST_ERR_CUDA;
    rast_status_t r = RAST_OK;
    if (h.error & kErrCapacity) r = RAST_ERR_CAPACITY;
    else if (h.error & kErrTimeout) r = RAST_ERR_TIMEOUT;
    if (stats) {
        stats->status = r;
        stats->n_views = (int32_t)h.n_views;
        stats->n_points = h.n_points;
        stats->n_copies = h.n_copies_raw;
        stats->copy_capacity = h.copy_cap;
        stats->needed_records = (int64_t)h.needed;
        stats->n_tiles = h.n_tiles;
        stats->n_pixels = h.n_pixels;
        stats->needed_records_bwd = (int64_t)h.needed_bwd;
    }
    return r;
}

const char* rasterize_status_string(rast_status_t s) {
    switch (s) {
        case RAST_OK: return "ok";
        case RAST_ERR_ARG: return "invalid argument";
        case RAST_ERR_CAPACITY: return "capacity exceeded";
        case RAST_ERR_CUDA: return "CUDA error";
        case RAST_ERR_TIMEOUT: return "device wait timed out";
        case RAST_ERR_NOT_SUPPORTED: return "not supported";
    }
    return "unknown status";
}

void rasterize_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    for (auto& r : g_prof.recs) {
        g_prof.pool.push_back(r.a);
        g_prof.pool.push_back(r.b);
    }
    g_prof.recs.clear();
    g_prof.on = on != 0;
}

int32_t rasterize_profile_read(rast_profile_entry_t* out, int32_t max) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    std::vector<rast_profile_entry_t> agg;
    for (auto& r : g_prof.recs) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) ms = 0.f;
        rast_profile_entry_t* e = nullptr;
        for (auto& x : agg)
            if (r.name == x.name) e = &x;
        if (!e) {
            rast_profile_entry_t z;
            std::memset(&z, 0, sizeof(z));
            std::snprintf(z.name, sizeof(z.name), "%s", r.name.c_str());
            agg.push_back(z);
            e = &agg.back();
        }
        e->launches += 1;
        e->total_ms += ms;
    }
    const int n = (int)agg.size();
    for (int k = 0; k < n && k < max; ++k) out[k] = agg[k];
    return n;
}

int32_t rasterize_tune_candidates(int32_t mode, int32_t* tiles, int32_t* depths, int32_t max) {
    if (mode != RAST_SPLAT_BILINEAR && mode != RAST_SPLAT_GAUSSIAN) return -1;
    static const int32_t kPairs[][2] = {{16, 256}, {16, 512}, {8, 64}, {8, 128}, {8, 256}};
    int32_t n = 0;
    for (const auto& pr : kPairs) {
        if (!blend_depth_supported(mode, pr[0], pr[1])) continue;
        if (n < max) {
            if (tiles) tiles[n] = pr[0];
            if (depths) depths[n] = pr[1];
        }
        ++n;
    }
    return n;
}

const char* rasterize_version(void) { return "inpc-rast-gb300 0.1 (sm_103a)"; }

}  // extern "C"

// Internal declarations of the GB300 tiled point rasterizer (sm_103a).
// Shared by the kernel translation units and the C-ABI layer in api.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "inpc_rast.h"

namespace rast {

constexpr int kMaxViews = 16;
constexpr int kTileDefault = 16;     // tile edge (pixels); 8 is the other compiled size
constexpr int kTileMax = 16;

// Status bits in the workspace header's error word.
constexpr uint32_t kErrCapacity = 1u;
constexpr uint32_t kErrTimeout = 2u;

// One view as the kernels see it (passed by value inside ViewTable).
struct ViewDev {
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float near_z, far_z;
    int32_t W, H, tiles_x, tiles_y;
    uint32_t key_base;   // FP32 bits of near_z: depth key = bits(z) - key_base
    uint32_t key_cull;   // key of culled points: bits(far) - bits(near) (> every visible key)
    int64_t pt_off;      // first global point index
    int64_t n;
    int64_t tile_off;    // first global tile id
    int64_t pix_off;     // first global pixel
    const float* xyz;
    const float* opacity;
    const void* feat;
    const float* scale;
    float* out_feat;
    float* out_alpha;
    float* out_depth;
    const float* g_feat;
    const float* g_alpha;
    const float* g_depth;
    float* d_feat;
    float* d_opacity;
    float* d_xyz;
    float* d_scale;
};

struct ViewTable {
    int32_t n_views;
    int32_t C;
    int32_t bf16;        // features stored as bf16
    int32_t mode;        // 0 bilinear, 1 Gaussian
    int32_t gauss_cov;   // 0 EWA, 1 isotropic screen
    int32_t tile;        // tile edge in pixels (8 or 16)
    int32_t blend_depth; // records per blend batch: tile^2 x {1, 2} (x 4 for tile 8); Gaussian: tile^2
    int32_t rec_words;   // record stride in 32-bit words (multiple of 4)
    int32_t feat_word;   // first feature word in a record
    int32_t shared_tiles; // some view blends into another view's tiles (point clouds of one image)
    int32_t flags;        // rast_opts_t::flags
    float t_min, alpha_max, dilation;
    int64_t n_total, tiles_total, pix_total;
    ViewDev v[kMaxViews];
};

// Device header at the start of the workspace.
struct WsHeader {
    uint32_t error;
    uint32_t n_copies;        // D after the dup scan (clamped to capacity)
    uint32_t n_copies_raw;    // D before clamping
    uint32_t n_views;
    unsigned long long needed;      // records the forward blend had to read
    unsigned long long needed_bwd;  // records the backward replay read
    long long n_points, copy_cap, n_tiles, n_pixels;
    uint32_t rec_tile_valid;  // the last forward wrote the tile-ordered record copy
    uint32_t pad0;
    long long pad1;
};

// ---- small device helpers --------------------------------------------------

// View of a global point index: views hold consecutive point ranges (pt_off
// ascending); the loop runs n_views - 1 uniform iterations (none for one view).
__device__ __forceinline__ int view_of_point(const ViewTable& vt, int64_t gi) {
    int v = 0;
    for (int k = 1; k < vt.n_views; ++k)
        if (gi >= vt.v[k].pt_off) v = k;
    return v;
}

__device__ __forceinline__ int view_of_tile(const ViewTable& vt, int64_t t) {
    int v = 0;
#pragma unroll 1
    for (int k = 1; k < vt.n_views; ++k)
        if (t >= vt.v[k].tile_off) v = k;
    return v;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t sm_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

// Per-tile trace record written by one thread of a blend CTA.
__device__ __forceinline__ void trace_tile(unsigned long long* tr, int64_t tile, int pass,
                                           unsigned long long t0, long long c0) {
    unsigned long long* e = tr + (tile * 2 + pass) * 4;
    e[0] = t0;
    e[1] = global_ns();
    e[2] = (unsigned long long)(clock64() - c0);
    e[3] = sm_id();
}

__device__ __forceinline__ float bf16lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// Packed tile rect of a point: (tx0 | ty0 << 16, tx1 | ty1 << 16), inclusive;
// an empty rect is (1, 0) (tx0 > tx1).
// Row stride (floats) of the per-copy gradient partials: P rounded up to a
// multiple of 4 so every row is written and read as 16-byte vectors.
__host__ __device__ constexpr int partial_stride(int P) { return (P + 3) & ~3; }

// Row stride (floats) of the per-point gradient rows of single-copy points:
// a power of two >= P, so each row is whole 32-byte sectors (C <= 7) or whole
// 64-byte bursts (8 <= C <= 15) and a scattered row write never merges with a
// neighbour's bytes.
__host__ __device__ constexpr int grow_stride(int P) { return P <= 4 ? 4 : (P <= 8 ? 8 : (P <= 16 ? 16 : 32)); }

// Bilinear footprints (2x2 pixels) touch at most 2x2 tiles, so their rect
// packs into 32 bits: tx0 (16 bits) | ty0 (14 bits) << 16 | (tx1 - tx0) << 30
// | (ty1 - ty0) << 31; empty = all ones (tx0 = 0xffff is never a tile
// column: tiles_x <= 65535). Half the bytes of the gather in depth order that
// the duplication makes, so twice as much of the array stays in L2.
constexpr uint32_t kRect4Empty = 0xffffffffu;
constexpr int kRect4MaxTilesY = 1 << 14;

__device__ __forceinline__ uint32_t rect4_pack(int tx0, int ty0, int tx1, int ty1) {
    return (uint32_t)tx0 | ((uint32_t)ty0 << 16) | ((uint32_t)(tx1 - tx0) << 30) | ((uint32_t)(ty1 - ty0) << 31);
}

__device__ __forceinline__ uint2 rect4_unpack(uint32_t p) {
    if (p == kRect4Empty) return make_uint2(1u, 0u);
    const uint32_t tx0 = p & 0xffffu, ty0 = (p >> 16) & 0x3fffu;
    const uint32_t tx1 = tx0 + ((p >> 30) & 1u), ty1 = ty0 + (p >> 31);
    return make_uint2(tx0 | (ty0 << 16), tx1 | (ty1 << 16));
}

__device__ __forceinline__ uint32_t rect4_count(uint32_t p) {
    return p == kRect4Empty ? 0u : (1u + ((p >> 30) & 1u)) * (1u + (p >> 31));
}

__device__ __forceinline__ uint32_t rect_count(uint2 r) {
    const int tx0 = r.x & 0xffff, ty0 = r.x >> 16, tx1 = r.y & 0xffff, ty1 = r.y >> 16;
    if (tx1 < tx0 || ty1 < ty0) return 0;
    return (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
}

// ---- per-device, thread-safe one-time set-up ------------------------------
// Launch attributes (cudaFuncSetAttribute), SM counts and occupancy belong to
// a device, not to the process: one process may drive several GPUs, from
// several host threads. A PerDevice slot runs its set-up once per device
// (with that device current, under std::call_once, so concurrent first calls
// wait for one another) and keeps the result and the status of the set-up.
constexpr int kMaxDevices = 64;

struct PerDevice {
    std::once_flag flag[kMaxDevices];
    int value[kMaxDevices] = {};
    cudaError_t err[kMaxDevices] = {};
};

// fn(int device, int* value) -> cudaError_t. Returns the set-up's status and
// stores its value in *out (if non-null).
template <typename F>
cudaError_t per_device(PerDevice& pd, int* out, F&& fn) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(pd.flag[dev], [&] { pd.err[dev] = fn(dev, &pd.value[dev]); });
    if (out) *out = pd.value[dev];
    return pd.err[dev];
}

// Multiprocessor count of the current device (1 if the query fails).
int device_sm_count();

// ---- per-kernel profiling (defined in api.cu) ------------------------------
// Opens an NVTX range named `name` for the scope (host-side, so profilers can
// group the launches by stage; free when no profiler is attached). While
// profiling is enabled it also records a CUDA event pair on `s` around the
// scope; rasterize_profile_read() sums the times per name. `name` must have
// static storage duration.
struct ProfScope {
    ProfScope(const char* name, cudaStream_t s);
    ~ProfScope();
    int idx;
    cudaStream_t s;
};

// ---- launchers (each defined in its own translation unit) ------------------

struct Bufs {
    // per point
    uint32_t* rec;        // records, rec_words per point
    uint32_t* rec_tile;   // bilinear: the records the forward blend read, in tile-list order (per copy)
    uint2* rect;          // tile rect per point (Gaussian; bilinear: rect4)
    uint32_t* rect4;      // bilinear: packed tile rect per point (same memory as rect)
    uint32_t* cnt;        // copies per point (point order; Gaussian only: bilinear counts come from rect4)
    uint32_t* zbits;      // FP32 bits of the view depth per point (backward bookkeeping)
    uint32_t* keyA[2];    // depth sort ping-pong
    uint32_t* valA[2];
    uint2* rectS;         // rects in depth order (Gaussian; bilinear: rect4S)
    uint32_t* rect4S;     // bilinear: packed rects in depth order (same memory as rectS)
    uint32_t* blk;        // block sums for scans
    uint32_t* base;       // point-order exclusive scan of cnt (backward)
    // per copy
    uint32_t* keyC[2];
    uint32_t* valC[2];
    uint32_t* pixC;       // untiled 64-bit-key sort: pixel id per copy (point order)
    uint32_t* ptC;        // untiled 64-bit-key sort: point index per copy (point order)
    float* partial;       // backward per-copy partial gradients (points with several copies)
    float* grow;          // backward gradient rows of single-copy points, indexed by point
    // radix sort scratch
    uint32_t* sort_ghist;     // [passes][bins] digit counts
    uint32_t* sort_counters;  // [kMaxSortPasses] tile counters of the passes
    uint32_t* sort_status;    // [passes][tiles][bins] look-back words
    // per tile / pixel
    uint2* ranges;
    uint32_t* order;      // tiles, heaviest list first
    uint2* cutoff;        // backward: (depth bits, point) of the last record processed per tile
    unsigned long long* trace;  // per tile x {fwd, bwd}: start ns, end ns, cycles, SM id
    float* t_final;
    uint32_t* last;
    WsHeader* hdr;
    int64_t copy_cap;
    int64_t blk_cap;
};

// Sort plan for one radix sort: digit passes over [0, bits).
// Most digit passes one radix sort runs: the digit counts, the per-pass tile
// counters and the histogram kernel's shared counts are sized for this many.
constexpr int kMaxSortPasses = 4;

struct SortPlan {
    int passes;
    int digit_bits[8];
    int shift[8];
};
SortPlan make_sort_plan(int bits);
// Look-back words one sort with this plan needs for `cap` elements.
int64_t sort_status_words(const SortPlan& plan, int64_t cap);

struct SortScratch {
    uint32_t* ghist;     // [kMaxSortPasses][512]
    uint32_t* counters;  // [kMaxSortPasses]
    uint32_t* status;    // sort_status_words()
    uint32_t* err;       // workspace error word
    bool stall_test = false;  // RAST_FLAG_TEST_SORT_STALL: the first pass's first tile never publishes
};

// write_vals: also write the identity point values into valA[0] (needed only
// when the depth sort makes no pass).
cudaError_t launch_project(const ViewTable& vt, const Bufs& b, bool write_vals, cudaStream_t s);
// Stable LSD radix sort of (key, val) pairs in keys[0]/vals[0] using keys[1]/vals[1]
// as scratch; count from d_n (device) if non-null else n (at most cap). Sets
// *result_buf to the index (0/1) of the buffer that holds the result.
// names: profiling names of the digit-count kernel and of the sweep passes.
// identity_vals: the input values are their own positions (0, 1, 2, ...);
// vals[0] is then not read. keys_out = false: only the values are wanted, the
// last pass does not write keys (keys[*result_buf] is left stale).
cudaError_t radix_sort(uint32_t* keys[2], uint32_t* vals[2], int64_t n, const uint32_t* d_n, int64_t cap,
                       const SortPlan& plan, const SortScratch& sc, cudaStream_t s, int* result_buf,
                       const char* const names[2], bool identity_vals = false, bool keys_out = true);
cudaError_t launch_duplicate(const ViewTable& vt, const Bufs& b, const uint32_t* sorted_pts,
                             cudaStream_t s);
cudaError_t launch_ranges(const ViewTable& vt, const Bufs& b, const uint32_t* sorted_tiles,
                          cudaStream_t s);
cudaError_t launch_tile_order(const ViewTable& vt, const Bufs& b, cudaStream_t s);
cudaError_t launch_blend_fwd(const ViewTable& vt, const Bufs& b, const uint32_t* sorted_pts,
                             cudaStream_t s);
// Untiled baseline: one thread per pixel walks its per-pixel fragment list.
cudaError_t launch_blend_fwd_pixel(const ViewTable& vt, const Bufs& b, const uint32_t* pts, cudaStream_t s);
// Untiled baseline with the 64-bit-key sort: copies in point order
// (low key word: depth key, high word: pixel id, plus the point index), the
// gather of the high word between the low-word and high-word digit passes,
// and one warp per pixel in the blend.
cudaError_t launch_untiled_copies(const ViewTable& vt, const Bufs& b, const uint32_t* dkey, uint32_t* key_lo,
                                  uint32_t* key_hi, uint32_t* pt, cudaStream_t s);
cudaError_t launch_gather_hi(const Bufs& b, const uint32_t* cid, const uint32_t* key_hi, const uint32_t* pt,
                             uint32_t* kout, uint32_t* vout, cudaStream_t s);
cudaError_t launch_blend_fwd_pixel_warp(const ViewTable& vt, const Bufs& b, const uint32_t* pts, cudaStream_t s);
cudaError_t launch_point_scan(const ViewTable& vt, const Bufs& b, cudaStream_t s);
cudaError_t launch_blend_bwd(const ViewTable& vt, const Bufs& b, const uint32_t* sorted_pts,
                             cudaStream_t s);
cudaError_t launch_reduce_grads(const ViewTable& vt, const Bufs& b, cudaStream_t s);

bool channels_supported(int C);


constexpr int kScanItems = 2048;   // items per block in the dup / point scans (8 per thread)

}  // namespace rast

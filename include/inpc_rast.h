/*
 * inpc_rast.h -- C ABI of the GB300 tiled point rasterizer.
 *
 * The rasterizer of "A Bag of Tricks for Efficient Implicit Neural Point
 * Clouds" (arXiv 2508.19140): N points (position p_i, opacity o_i, an
 * n_w-channel feature f_i; Sec. 2 "Rendering Feature Maps") are projected
 * through a pinhole camera, splatted as bilinear 2x2 footprints or as small
 * isotropic Gaussians (Sec. 3.2 "Rendering Points as Small Gaussians"), binned
 * into 16x16 (or 8x8) tiles and sorted by (tile, depth, point index) (Sec. 3.2 "Tiled
 * Rendering", split sort), then alpha-blended front to back by Eq. 1 into a
 * feature image F (H x W x n_w), an alpha image and a depth image. The
 * backward pass implements the corrected gradient of the appendix (Eq. 2,
 * "Addressing Gradient Approximations"), fragments with alpha = 0 included.
 *
 * Conventions
 *   - All pointers inside the structs below are DEVICE pointers owned by the
 *     caller unless stated otherwise; the library never allocates, frees or
 *     retains them beyond the call. The `rast_*_t` structs themselves live in
 *     host memory and are read during the call only.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Compute entry points enqueue work and return without a host
 *     synchronisation; argument errors are reported synchronously.
 *   - Camera: x_c = R x_w + t (R row-major), u = fx x_c / z_c + cx,
 *     v = fy y_c / z_c + cy; pixel (i, j) has its centre at (i + 1/2, j + 1/2).
 *     Points with z_c <= near_z or z_c >= far_z are culled.
 *   - Layouts: xyz [n][3] f32, opacity [n] f32, scale [n] f32, feat [n][C]
 *     f32 or bf16 (row-major), images [H][W][C] f32 (HWC, as F in Sec. 2),
 *     alpha and depth [H][W] f32.
 *   - Errors: no C++ exception crosses this ABI and no kernel traps. A
 *     device-side capacity overflow, or a bounded device-side wait that ran
 *     out, is recorded in the workspace and reported by
 *     rasterize_get_status(); the stages after it then see an empty copy list,
 *     so no kernel reads a partial sort result.
 */
#ifndef INPC_RAST_H
#define INPC_RAST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RAST_OK = 0,
    RAST_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, bad enum) */
    RAST_ERR_CAPACITY = 2,       /* workspace too small, or copies exceeded max_copies */
    RAST_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    RAST_ERR_TIMEOUT = 4,        /* a bounded device-side wait gave up */
    RAST_ERR_NOT_SUPPORTED = 5   /* channel count, tile size, blend depth or mode not compiled in */
} rast_status_t;

typedef enum { RAST_SPLAT_BILINEAR = 0, RAST_SPLAT_GAUSSIAN = 1 } rast_mode_t;

/* EWA: Sigma_2D = s^2 J J^T + dilation I with J the affine (Jacobian)
 * approximation of the perspective projection (Sec. 3.2, small Gaussians).
 * ISO_SCREEN: Sigma_2D = (s^2 fx fy / z^2 + dilation) I. */
typedef enum { RAST_GAUSS_EWA = 0, RAST_GAUSS_ISO_SCREEN = 1 } rast_gauss_cov_t;

typedef enum { RAST_F32 = 0, RAST_BF16 = 1 } rast_dtype_t;

typedef enum { RAST_PASS_FWD = 1, RAST_PASS_BWD = 2 } rast_pass_t;

typedef struct {
    float fx, fy, cx, cy;
    float R[9];          /* world -> camera rotation, row-major */
    float t[3];
    float near_z, far_z;
    int32_t width, height;
} rast_camera_t;

typedef struct {
    int64_t n;             /* number of points (>= 0) */
    const float* xyz;      /* [n][3] */
    const float* opacity;  /* [n] */
    const void* feat;      /* [n][channels], element type feat_dtype */
    int32_t feat_dtype;    /* rast_dtype_t */
    int32_t channels;      /* C: 1, 2, 3, 4, 8 or 16 */
    const float* scale;    /* [n] world-space Gaussian scale; NULL: 5 px at the near plane */
} rast_points_t;

typedef struct {
    int32_t mode;          /* rast_mode_t */
    int32_t gauss_cov;     /* rast_gauss_cov_t */
    int32_t tile;          /* tile edge in pixels: 16 (default) or 8; the images and gradients
                              do not depend on it, only the work split does */
    int32_t blend_depth;   /* records staged per blend batch: 0 = tile * tile (default);
                              bilinear also 2 * tile * tile, and 4 * tile * tile for 8x8
                              tiles; Gaussian tile * tile only. Results do not depend on it */
    float t_min;           /* early termination: stop before T (1 - a) < t_min (1e-4) */
    float alpha_max;       /* alpha clamp (0.99) */
    float dilation;        /* screen-space dilation variance, Gaussian mode (0.16) */
    int32_t max_copies;    /* capacity: point-tile copies per point (0 = 4 bilinear, 16 Gaussian) */
    int32_t flags;         /* 0 or an OR of RAST_FLAG_SAVE_FOR_BWD, RAST_FLAG_TEST_SORT_STALL and
                              RAST_FLAG_TEST_BLEND_STALL */
} rast_opts_t;

/* The forward blend also writes a copy of every point record it reads, in
 * tile-list order, into the workspace (bilinear mode, tiled calls; the
 * workspace grows by one record per copy of the capacity), so that a backward
 * pass on the same workspace reads its records as sequential runs instead of
 * gathering them by point index. Results are identical either way; a backward
 * after a forward without the flag gathers. Set it when a backward will
 * follow (training), leave it out for inference. Pass the same flags to
 * rasterize_workspace_size and to every call on that workspace. */
#define RAST_FLAG_SAVE_FOR_BWD 2

/* Test hook for the bounded device-side waits (failure detection). With this
 * flag the first digit pass of the depth sort withholds the look-back word of
 * its first 4096-key tile, so the tile after it waits on a word nothing will
 * ever set, and that wait is limited to 64 polls instead of 2^22. The wait
 * runs out, the kernel sets the timeout bit of the workspace error word and
 * returns normally; every later stage sees the bit and produces an empty copy
 * list (images of zero coverage, zero point gradients), and
 * rasterize_get_status() returns RAST_ERR_TIMEOUT. Needs more than 4096
 * points. Never set outside tests. */
#define RAST_FLAG_TEST_SORT_STALL 1

/* Test hook for the bounded waits of the Gaussian backward blend (failure
 * detection). With this flag in the opts of a Gaussian backward pass, the
 * second batch of every tile with more than 32 replayed records is never
 * staged, so the warps' waits on its staging barrier can never succeed, and
 * each wait is limited to 64 polls instead of 2^20. The waits run out, the
 * kernel sets the timeout bit of the workspace error word and returns
 * normally (the point gradients are then incomplete), and
 * rasterize_get_status() returns RAST_ERR_TIMEOUT. Never set outside tests. */
#define RAST_FLAG_TEST_BLEND_STALL 4

typedef struct {
    float* feat;    /* [H][W][C] out */
    float* alpha;   /* [H][W] out: 1 - T_final; may be NULL */
    float* depth;   /* [H][W] out: sum_i T_i a_i z_i; may be NULL */
} rast_images_t;

typedef struct {
    const float* g_feat;   /* [H][W][C] dL/dF (required for BWD) */
    const float* g_alpha;  /* [H][W] dL/dalpha, NULL = 0 */
    const float* g_depth;  /* [H][W] dL/ddepth, NULL = 0 */
    float* d_feat;         /* [n][C] out, f32 whatever feat_dtype is */
    float* d_opacity;      /* [n] out */
    float* d_xyz;          /* [n][3] out, Gaussian mode only (NULL allowed) */
    float* d_scale;        /* [n] out, Gaussian mode with scale != NULL (NULL allowed) */
} rast_grads_t;

typedef struct {
    rast_points_t pts;
    rast_camera_t cam;
    rast_images_t out;
    rast_grads_t grad;     /* read by BWD only */
} rast_view_t;

/* Counters read back by rasterize_get_status(). */
typedef struct {
    int32_t status;          /* rast_status_t recorded on the device */
    int32_t n_views;
    int64_t n_points;        /* total points over all views */
    int64_t n_copies;        /* D: point-tile copies created by the last forward */
    int64_t copy_capacity;   /* copies the workspace can hold */
    int64_t needed_records;  /* records the blend had to read (after early termination) */
    int64_t n_tiles;
    int64_t n_pixels;
    int64_t needed_records_bwd; /* records the backward replay read (last backward) */
} rast_stats_t;

/* One workspace array: name, byte offset, bytes (rasterize_workspace_layout). */
typedef struct { char name[24]; int64_t offset; int64_t bytes; } rast_ws_entry_t;

/* One row of the per-stage timing profile. */
typedef struct {
    char name[32];
    int32_t launches;
    double total_ms;
} rast_profile_entry_t;

/* Fill `opts` with the defaults stated above. */
void rast_default_opts(rast_opts_t* opts);

/* Bytes of device workspace rasterize_batch() needs for these views and
 * options (0 on invalid arguments). The workspace carries the forward's state
 * (records, sorted tile lists, per-pixel final T and last contributor) to the
 * backward pass, so one workspace must outlive the fwd/bwd pair. */
size_t rasterize_workspace_size(const rast_view_t* views, int32_t n_views, const rast_opts_t* opts);

/* Forward pass of ONE view (Eq. 1): projection + footprint count, split
 * radix sort by (tile, depth, index), tile ranges, front-to-back blend.
 * Writes out->feat, out->alpha, out->depth. Equivalent to rasterize_batch
 * with one view and RAST_PASS_FWD. */
rast_status_t rasterize_fwd(const rast_points_t* pts, const rast_camera_t* cam,
                            const rast_opts_t* opts, void* workspace, size_t ws_bytes,
                            const rast_images_t* out, void* stream);

/* Forward pass of ONE view like rasterize_fwd, but allocating nothing and
 * taking no workspace: for callers that cannot allocate device memory where
 * they render (a plug-in inside an application that owns all GPU
 * allocations, or a path that must not allocate during stream capture). No
 * counterpart in the paper: it is a deployment convenience.
 * The intermediate arrays live in one static device array of 16 MiB
 * (1 << 24 bytes) that every GPU loading the library keeps until exit;
 * problems whose rasterize_workspace_size() exceeds it return
 * RAST_ERR_CAPACITY before any device work (e.g. up to 53,888 points at
 * 256x256 with 4 f32 features fit). The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture. Every call reuses the same array and
 * finds the previous call's contents there (the forward clears what it needs
 * zeroed); calls whose GPU work overlaps race on it and must be serialised by
 * the caller. Writes out->feat, out->alpha, out->depth; no backward state is
 * kept for the caller. Outside stream capture every call looks the array's
 * address up again (a context torn down and created again gets the new one);
 * during capture the address found by the last call outside it is used.
 * Errors the GPU raises during the pass (copies beyond max_copies, a bounded
 * wait that ran out) are not in the return value, which comes before the GPU
 * work: read them with rasterize_noalloc_get_status. */
rast_status_t rasterize_fwd_noalloc(const rast_points_t* pts, const rast_camera_t* cam,
                                   const rast_opts_t* opts, const rast_images_t* out,
                                   void* stream);

/* Synchronises `stream`, then reads the device-side status word and counters
 * that the last rasterize_fwd_noalloc call on the current device left in the
 * static array (stats may be NULL), as rasterize_get_status does for a
 * caller's workspace. No counterpart in the paper. Before any
 * rasterize_fwd_noalloc call on the device it returns RAST_OK with zero
 * counters. */
rast_status_t rasterize_noalloc_get_status(void* stream, rast_stats_t* stats);

/* Backward pass of ONE view (appendix Eq. 2, corrected). `workspace` must
 * hold the state of the matching rasterize_fwd on the same inputs. Writes
 * every element of the d_* outputs given (zeros for culled points). */
rast_status_t rasterize_bwd(const rast_points_t* pts, const rast_camera_t* cam,
                            const rast_opts_t* opts, void* workspace, size_t ws_bytes,
                            const rast_grads_t* grads, void* stream);

/* Several views (each with its own points, camera, outputs and gradients)
 * in one launch sequence: global tile ids concatenate the views' tiles, so
 * one sort and one blend launch serve all views. pass = RAST_PASS_FWD,
 * RAST_PASS_BWD or both OR-ed. No host synchronisation: capturable in a CUDA
 * graph. n_views <= 16. */
rast_status_t rasterize_batch(const rast_view_t* views, int32_t n_views, int32_t pass,
                              const rast_opts_t* opts, void* workspace, size_t ws_bytes,
                              void* stream);

/* Untiled baseline, forward only, bilinear only: the original INPC
 * arrangement that Sec. 3.2 "Tiled Rendering" replaces. Every point makes one
 * copy per pixel of its 2x2 footprint inside the image (about 4 per point
 * instead of ~1.1 per 16x16 tile), the copies are sorted by (pixel, depth,
 * point index) with the same split sort, and each pixel's list is composited
 * by its own thread, gathering every fragment's record. Outputs are identical
 * to rasterize_fwd (same per-pixel order and FP32 operations); it exists to
 * measure what tiling saves on this GPU. opts->tile and blend_depth are
 * ignored; RAST_ERR_NOT_SUPPORTED for Gaussian mode. */
size_t rasterize_untiled_workspace_size(const rast_points_t* pts, const rast_camera_t* cam,
                                        const rast_opts_t* opts);
rast_status_t rasterize_fwd_untiled(const rast_points_t* pts, const rast_camera_t* cam, const rast_opts_t* opts,
                                    void* workspace, size_t ws_bytes, const rast_images_t* out, void* stream);

/* Untiled baseline in the arrangement whose sort cost Sec. 3.2 "Tiled
 * Rendering" counts as 28n: every point makes one copy per in-image pixel of
 * its 2x2 footprint (about 4n copies), written in point order, and ONE stable
 * LSD radix sort orders the copies by a 64-bit key [pixel id | depth key]
 * (pixel id in the high word, the FP32 depth bits minus those of near_z in
 * the low word; ties fall back to point index). The digit passes over the low
 * word carry each copy's id; before the passes over the high word, each
 * copy's pixel id and point index are fetched by that id (the key's high word
 * is only read once its digits are reached). Each pixel's list is then
 * composited by one warp: 32 fragments' records gathered and their alphas
 * computed at once, the transmittance stepped through them in list order with
 * the same FP32 operations as the per-thread walk (so the per-pixel lists,
 * last-contributor positions and termination decisions equal
 * rasterize_fwd_untiled's bit for bit), the sums of the chunk reduced across
 * the warp (images within FP32 rounding of the serial sums). Forward only,
 * bilinear only (RAST_ERR_NOT_SUPPORTED otherwise); opts->tile and
 * blend_depth are ignored. Workspace, stream and errors as rasterize_fwd.
 * rasterize_untiled64_workspace_layout lists the workspace arrays like
 * rasterize_workspace_layout ("sorted_keys" = pixel ids, "sorted_vals" =
 * point indices in (pixel, depth, point index) order). */
size_t rasterize_untiled64_workspace_size(const rast_points_t* pts, const rast_camera_t* cam,
                                          const rast_opts_t* opts);
int32_t rasterize_untiled64_workspace_layout(const rast_points_t* pts, const rast_camera_t* cam,
                                             const rast_opts_t* opts, rast_ws_entry_t* out, int32_t max);
rast_status_t rasterize_fwd_untiled64(const rast_points_t* pts, const rast_camera_t* cam, const rast_opts_t* opts,
                                      void* workspace, size_t ws_bytes, const rast_images_t* out, void* stream);

/* Several point clouds rendered into ONE image (the ring buffer of
 * view-specific clouds of Sec. 3.1 "Fast and Stable View-Specific Sampling
 * during Inference": the clouds sampled for the last frames are reused and
 * rendered together). The result is exactly that of one cloud holding
 * clouds[0], clouds[1], ... concatenated in this order (equal depths fall
 * back to that order), without copying them. clouds[k] and grads[k] are cloud
 * k's points and point gradients (d_feat, d_opacity, d_xyz, d_scale); the
 * image gradients g_feat, g_alpha, g_depth are taken from grads[0]; grads may
 * be NULL for a forward-only pass. 1 <= n_clouds <= 16; same channel count and
 * feature dtype in every cloud. Workspace, stream and errors as
 * rasterize_batch; the workspace size comes from
 * rasterize_clouds_workspace_size (0 for invalid arguments). */
size_t rasterize_clouds_workspace_size(const rast_points_t* clouds, int32_t n_clouds, const rast_camera_t* cam,
                                       const rast_opts_t* opts);
rast_status_t rasterize_clouds(const rast_points_t* clouds, const rast_grads_t* grads, int32_t n_clouds,
                               const rast_camera_t* cam, const rast_images_t* out, int32_t pass,
                               const rast_opts_t* opts, void* workspace, size_t ws_bytes, void* stream);

/* Synchronises `stream`, then reads the device-side status word and counters
 * of `workspace` (stats may be NULL). Returns the recorded status. */
rast_status_t rasterize_get_status(const void* workspace, size_t ws_bytes, void* stream,
                                   rast_stats_t* stats);

/* Human-readable name of a status code (static storage). */
const char* rasterize_status_string(rast_status_t status);

/* Byte offsets of the workspace arrays, for inspection by tests: one entry
 * per internal array ("header", "records", "rect", "count", "ranges",
 * "t_final", "last", ...) plus three aliases of the sort results:
 * "depth_sorted" (point indices in depth order), "sorted_keys" and
 * "sorted_vals" (tile id and point index of every copy, in (tile, depth bits,
 * point index) order). Writes up to `max` (name, offset, bytes) triples and
 * returns how many exist. Layout only: no device access. */
int32_t rasterize_workspace_layout(const rast_view_t* views, int32_t n_views,
                                   const rast_opts_t* opts, rast_ws_entry_t* out, int32_t max);

/* Per-stage timing with CUDA events recorded on the launch stream around each
 * stage. enable(1) clears and starts recording, enable(0) stops. read()
 * waits for the recorded events, writes up to `max` entries and returns how
 * many stages were seen. */
void rasterize_profile_enable(int32_t on);
int32_t rasterize_profile_read(rast_profile_entry_t* out, int32_t max);

/* Compiled (tile edge, blend depth) pairs for splat mode `mode`, in the
 * order an autotuner should try them (the default first). Writes up to `max`
 * pairs to tiles[] / depths[] (either may be NULL to only count) and returns
 * how many exist; -1 for an unknown mode. Host only, no device access. The
 * paper fixes 16x16 tiles (Sec. 3.2); the other pairs change only the work
 * split, never the images (gradients agree to FP32 rounding). */
int32_t rasterize_tune_candidates(int32_t mode, int32_t* tiles, int32_t* depths, int32_t max);

/* ---------------------------------------------------------------------------
 * Distilled background model (Sec. 3.2 "Faster Background Model Evaluation"):
 * the background behind the points is a spherical environment map
 * F_bg (H_b x W_b x C; the paper's is 1024 x 2048 x 4) read by bilinear
 * interpolation along each pixel's viewing direction and composited with the
 * transmittance the blend leaves (the T_{K+1} f_bg term of Eq. 2):
 *     out = feat + (1 - alpha) * f_bg(d).
 * Directions: d_c = ((x + 1/2 - cx) / fx, (y + 1/2 - cy) / fy, 1) normalised
 * (camera space), rotated to world space with R^T. Map: longitude
 * atan2(d_x, d_z) -> column (lambda / 2 pi + 1/2) W_b - 1/2, polar angle
 * acos(d_y) -> row (theta / pi) H_b - 1/2; texel centres at integer + 1/2;
 * columns wrap, rows clamp at the poles. All pointers are caller-owned device
 * memory; calls are asynchronous on `stream`; argument errors return
 * synchronously. ------------------------------------------------------------ */
typedef struct {
    const float* map;      /* [height][width][channels] FP32, row-major; 16-byte aligned
                              when channels is a multiple of 4 */
    int32_t height;        /* H_b (rows, polar angle) */
    int32_t width;         /* W_b (columns, longitude) */
    int32_t channels;      /* C: equal to the image's channels (1, 2, 3, 4, 8 or 16) */
} rast_envmap_t;

/* Camera-space unit viewing directions of every pixel ([height][width][3]
 * FP32). They depend only on the intrinsics and the image size, so they can be
 * computed once and passed to the calls below for every frame (the paper
 * caches them). */
rast_status_t rasterize_view_dirs(const rast_camera_t* cam, float* dirs, void* stream);

/* out = feat + (1 - alpha) * f_bg for every pixel ([height][width][C]).
 * `dirs`: cached directions from rasterize_view_dirs, or NULL to compute them
 * from the intrinsics. `out` may equal `feat`. RAST_ERR_NOT_SUPPORTED for a
 * channel count that is not compiled in. */
rast_status_t rasterize_bg_composite(const rast_camera_t* cam, const rast_envmap_t* env, const float* dirs,
                                     const float* feat, const float* alpha, float* out, void* stream);

/* Bytes of device scratch rasterize_bg_composite_bwd needs (8 bytes per map
 * element); 0 for an invalid map. */
size_t rasterize_bg_scratch_size(const rast_envmap_t* env);

/* Backward of rasterize_bg_composite for g = dL/dout ([height][width][C]):
 *   g_alpha[p] += -(g[p] . f_bg[p])   (in place; NULL to skip; it is the
 *                                      blend's dL/dalpha input),
 *   d_map      = dL/dF_bg             ([H_b][W_b][C], overwritten),
 * and dL/dfeat is g itself. The map gradient is summed as 64-bit fixed-point
 * integers with resolution 2^-32 in `scratch` (rasterize_bg_scratch_size bytes,
 * 8-byte aligned, contents overwritten), so it is bit-identical from run to run;
 * each sum must stay below 2^31 in magnitude. RAST_ERR_CAPACITY if the scratch
 * is too small. */
rast_status_t rasterize_bg_composite_bwd(const rast_camera_t* cam, const rast_envmap_t* env, const float* dirs,
                                         const float* alpha, const float* g, float* g_alpha, float* d_map,
                                         void* scratch, size_t scratch_bytes, void* stream);

/* Spherical contraction of n positions (Sec. 3.4 "Implementation
 * Improvements"; the contraction of Mip-NeRF 360 that INPC applies to sampled
 * points before its appearance field), in one kernel:
 *     out_i = x_i                           if |x_i| <= 1
 *           = (2 - 1/|x_i|) x_i / |x_i|     otherwise  (|out_i| < 2).
 * xyz, out: device [n][3] FP32; out may equal xyz (in place). */
rast_status_t rasterize_contract(const float* xyz, float* out, int64_t n, void* stream);

/* Library version string. */
const char* rasterize_version(void);

#ifdef __cplusplus
}
#endif

#endif /* INPC_RAST_H */

// rasterize_fwd_noalloc: the forward pass of one view with no device
// allocation anywhere, for callers that cannot allocate GPU memory.
//
// Some callers of this library cannot call cudaMalloc at the point where they
// render: a plug-in hosted by an application that owns every device
// allocation (interactive viewers and compositors with a fixed memory budget
// per frame), or code on a path that must not allocate because it runs while a
// stream is being captured into a CUDA graph. They still own their inputs and
// outputs, but have nowhere to put the forward pass's intermediate arrays
// (projected records, sort buffers, tile ranges, per-pixel state).
//
// This entry point keeps those arrays in one file-scope device array of
// kNoAllocBytes (16 MiB), which every GPU that loads the library holds until
// the process exits. Problems whose workspace would not fit are rejected with
// RAST_ERR_CAPACITY before any device work. Errors the GPU itself raises
// during the pass (more copies than max_copies allows, a bounded wait that ran
// out) land in the scratch's header like in a caller's workspace, and
// rasterize_noalloc_get_status reads them back. All calls share the array and
// it keeps the previous call's contents; the forward pass initialises
// everything it reads (its header, tile ranges and sort bin totals are cleared
// on the stream before use), so stale contents are harmless. Calls whose GPU
// work overlaps (different streams, or different host threads, without
// ordering) race on the array and must be serialised by the caller.
#include <cstring>
#include <mutex>

#include "rast_internal.cuh"

namespace rast {
namespace {

constexpr size_t kNoAllocBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

// The scratch. In host code this name is only a host-side stand-in for the
// device symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up with that
// device current). Outside stream capture it is looked up on every call and
// the cache refreshed, so a context torn down and created again (after
// cudaDeviceReset, say) never leaves a stale address behind; while `stream`
// is being captured the cached address is used, which is why the first call
// on a device must come before any capture.
rast_status_t scratch_address(cudaStream_t stream, void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RAST_ERR_CUDA;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return RAST_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cap == cudaStreamCaptureStatusNone || !g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RAST_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return RAST_OK;
}

}  // namespace
}  // namespace rast

extern "C" rast_status_t rasterize_fwd_noalloc(const rast_points_t* pts, const rast_camera_t* cam,
                                               const rast_opts_t* opts, const rast_images_t* out,
                                               void* stream) {
    if (!pts || !cam || !opts || !out) return RAST_ERR_ARG;
    rast_view_t v;
    std::memset(&v, 0, sizeof(v));
    v.pts = *pts;
    v.cam = *cam;
    v.out = *out;
    const size_t need = rasterize_workspace_size(&v, 1, opts);
    if (need == 0) return RAST_ERR_ARG;
    if (need > rast::kNoAllocBytes) return RAST_ERR_CAPACITY;  // too large for the static scratch
    void* ws = nullptr;
    const rast_status_t st = rast::scratch_address(static_cast<cudaStream_t>(stream), &ws);
    if (st != RAST_OK) return st;
    return rasterize_batch(&v, 1, RAST_PASS_FWD, opts, ws, rast::kNoAllocBytes, stream);
}

// Device-side status of the last rasterize_fwd_noalloc call on the current
// device: the same header rasterize_get_status reads from a caller's
// workspace, read here from the static scratch.
extern "C" rast_status_t rasterize_noalloc_get_status(void* stream, rast_stats_t* stats) {
    void* ws = nullptr;
    const rast_status_t st = rast::scratch_address(static_cast<cudaStream_t>(stream), &ws);
    if (st != RAST_OK) return st;
    return rasterize_get_status(ws, rast::kNoAllocBytes, stream, stats);
}

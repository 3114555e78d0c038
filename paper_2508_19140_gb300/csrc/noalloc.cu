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
// RAST_ERR_CAPACITY before any device work. All calls share the array and it
// keeps the previous call's contents; the forward pass initialises everything
// it reads (its header, tile ranges and sort bin totals are cleared on the
// stream before use), so stale contents are harmless. Calls whose GPU work
// overlaps (different streams, or different host threads, without ordering)
// race on the array and must be serialised by the caller.
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

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.
rast_status_t scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RAST_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
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
    const rast_status_t st = rast::scratch_address(&ws);
    if (st != RAST_OK) return st;
    return rasterize_batch(&v, 1, RAST_PASS_FWD, opts, ws, rast::kNoAllocBytes, stream);
}

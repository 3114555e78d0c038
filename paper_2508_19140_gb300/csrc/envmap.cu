// Distilled background model (Sec. 3.2, "Faster Background Model
// Evaluation"): the background behind the blended points is read from a
// spherical environment map (H_b x W_b x C, the paper's is 1024 x 2048 x 4) by
// bilinear interpolation along each pixel's viewing direction, and composited
// with the transmittance the blend leaves (the T_{K+1} f_bg term of Eq. 2):
//   out = F + (1 - alpha) f_bg(d).
// Viewing directions depend only on the intrinsics and can be cached across
// frames (the paper caches them); they are rotated to world space per frame.
// Mapping: longitude atan2(d_x, d_z) -> column, polar angle acos(d_y) -> row,
// texel centres at integer + 1/2, columns wrap, rows clamp at the poles.
//
// Backward: dL/dF = g (the caller passes g on to the blend's backward),
// dL/dalpha += -g . f_bg, dL/dmap[texel] = sum over pixels of w (1 - alpha) g.
// The map gradient is a scatter of four taps per pixel; it is accumulated as
// 64-bit fixed-point integers (resolution 2^-32) with integer atomics, which
// are exact and order-free, so reruns are bit-identical, then converted.
#include <cstdint>
#include <type_traits>

#include "blend_common.cuh"

namespace rast {
namespace {

struct EnvCam {
    float fx, fy, cx, cy;
    float R[9];
    int32_t W, H;
};

struct Taps {
    uint32_t idx[4];  // texel index (row * W_b + col)
    float w[4];
};

__device__ __forceinline__ void pixel_dir(const EnvCam& c, const float* __restrict__ dirs, int64_t p, int x,
                                          int y, float d[3]) {
    if (dirs) {
        d[0] = dirs[3 * p];
        d[1] = dirs[3 * p + 1];
        d[2] = dirs[3 * p + 2];
        return;
    }
    const float a = ((float)x + 0.5f - c.cx) / c.fx, b = ((float)y + 0.5f - c.cy) / c.fy;
    const float inv = rsqrtf(a * a + b * b + 1.f);
    d[0] = a * inv;
    d[1] = b * inv;
    d[2] = inv;
}

__device__ __forceinline__ Taps taps_of(const EnvCam& c, const float d[3], int Hb, int Wb) {
    // world direction R^T d
    const float wx = c.R[0] * d[0] + c.R[3] * d[1] + c.R[6] * d[2];
    const float wy = c.R[1] * d[0] + c.R[4] * d[1] + c.R[7] * d[2];
    const float wz = c.R[2] * d[0] + c.R[5] * d[1] + c.R[8] * d[2];
    constexpr float kInv2Pi = 0.15915494309189535f, kInvPi = 0.3183098861837907f;
    const float lam = atan2f(wx, wz);
    const float th = acosf(fminf(1.f, fmaxf(-1.f, wy)));
    const float X = (lam * kInv2Pi + 0.5f) * (float)Wb - 0.5f;
    const float Y = th * kInvPi * (float)Hb - 0.5f;
    const float fx0 = floorf(X), fy0 = floorf(Y);
    const float a = X - fx0, b = Y - fy0;
    int x0 = (int)fx0, y0 = (int)fy0;
    int x1 = x0 + 1;
    x0 = x0 < 0 ? x0 + Wb : (x0 >= Wb ? x0 - Wb : x0);
    x1 = x1 < 0 ? x1 + Wb : (x1 >= Wb ? x1 - Wb : x1);
    const int r0 = min(max(y0, 0), Hb - 1), r1 = min(max(y0 + 1, 0), Hb - 1);
    Taps t;
    t.idx[0] = (uint32_t)(r0 * Wb + x0); t.w[0] = (1.f - a) * (1.f - b);
    t.idx[1] = (uint32_t)(r0 * Wb + x1); t.w[1] = a * (1.f - b);
    t.idx[2] = (uint32_t)(r1 * Wb + x0); t.w[2] = (1.f - a) * b;
    t.idx[3] = (uint32_t)(r1 * Wb + x1); t.w[3] = a * b;
    return t;
}

template <int C>
__device__ __forceinline__ void lookup(const float* __restrict__ map, const Taps& t, float bg[C]) {
#pragma unroll
    for (int c = 0; c < C; ++c) bg[c] = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float* m = map + (size_t)t.idx[k] * C;
        if constexpr (C % 4 == 0) {
#pragma unroll
            for (int c = 0; c < C; c += 4) {
                const float4 v = __ldg(reinterpret_cast<const float4*>(m + c));
                bg[c] = fmaf(t.w[k], v.x, bg[c]);
                bg[c + 1] = fmaf(t.w[k], v.y, bg[c + 1]);
                bg[c + 2] = fmaf(t.w[k], v.z, bg[c + 2]);
                bg[c + 3] = fmaf(t.w[k], v.w, bg[c + 3]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) bg[c] = fmaf(t.w[k], __ldg(m + c), bg[c]);
        }
    }
}

__global__ void __launch_bounds__(256) k_view_dirs(const EnvCam c, float* __restrict__ dirs) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)c.W * c.H) return;
    float d[3];
    pixel_dir(c, nullptr, p, (int)(p % c.W), (int)(p / c.W), d);
    dirs[3 * p] = d[0];
    dirs[3 * p + 1] = d[1];
    dirs[3 * p + 2] = d[2];
}

template <int C>
__global__ void __launch_bounds__(256) k_bg_fwd(const EnvCam c, const float* __restrict__ map, int Hb, int Wb,
                                                const float* __restrict__ dirs, const float* feat,
                                                const float* __restrict__ alpha, float* out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)c.W * c.H) return;
    float d[3];
    pixel_dir(c, dirs, p, (int)(p % c.W), (int)(p / c.W), d);
    const Taps t = taps_of(c, d, Hb, Wb);
    float bg[C];
    lookup<C>(map, t, bg);
    const float tr = 1.f - alpha[p];
    float v[C];
#pragma unroll
    for (int k = 0; k < C; ++k) v[k] = fmaf(tr, bg[k], feat[p * C + k]);
    store_row<C>(out + p * C, v);
}

template <int C>
__global__ void __launch_bounds__(256) k_bg_bwd(const EnvCam c, const float* __restrict__ map, int Hb, int Wb,
                                                const float* __restrict__ dirs, const float* __restrict__ alpha,
                                                const float* __restrict__ g, float* __restrict__ g_alpha,
                                                unsigned long long* __restrict__ acc) {
    const int64_t n = (int64_t)c.W * c.H;
    const int64_t p0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) >= n) return;  // whole warp past the end
    // Lanes past the end (last warp only) take part in the shuffles with zero
    // contributions to their neighbour's texels.
    const bool valid = p0 < n;
    const int64_t p = valid ? p0 : n - 1;
    float d[3];
    pixel_dir(c, dirs, p, (int)(p % c.W), (int)(p / c.W), d);
    const Taps t = taps_of(c, d, Hb, Wb);
    float bg[C];
    lookup<C>(map, t, bg);
    const float tr = valid ? 1.f - alpha[p] : 0.f;
    float gv[C];
    float ga = 0.f;
#pragma unroll
    for (int k = 0; k < C; ++k) {
        gv[k] = valid ? g[p * C + k] : 0.f;
        ga = fmaf(-gv[k], bg[k], ga);
    }
    if (g_alpha && valid) g_alpha[p] += ga;
    constexpr float kScale = 4294967296.f;  // 2^32
    // Neighbouring pixels of a row mostly share texels: lanes with the same
    // texel form contiguous runs; each run's fixed-point sum is formed with a
    // warp prefix sum and added by the run's last lane (integer sums: exact,
    // so the grouping does not change the result).
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float s = t.w[k] * tr;
        const uint32_t id = t.idx[k];
        const uint32_t prev = __shfl_up_sync(0xffffffffu, id, 1);
        const uint32_t next = __shfl_down_sync(0xffffffffu, id, 1);
        const bool head = lane == 0 || prev != id;
        const bool tail = lane == 31 || next != id;
        const uint32_t heads = __ballot_sync(0xffffffffu, head);
        const int start = 31 - __clz(heads & (lt | (1u << lane)));  // first lane of this run
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            long long x = __float2ll_rn(s * gv[ch] * kScale);
            // inclusive prefix sum over the warp
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            const long long before = __shfl_sync(0xffffffffu, x, start > 0 ? start - 1 : 0);
            const long long run = start > 0 ? x - before : x;
            if (tail && run != 0) atomicAdd(acc + (size_t)id * C + ch, (unsigned long long)run);
        }
    }
}

__global__ void __launch_bounds__(256) k_fixed_to_float(const unsigned long long* __restrict__ acc, int64_t n,
                                                        float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = __ll2float_rn((long long)acc[i]) * 2.3283064365386963e-10f;  // * 2^-32
}

EnvCam env_cam(const rast_camera_t& c) {
    EnvCam e;
    e.fx = c.fx; e.fy = c.fy; e.cx = c.cx; e.cy = c.cy;
    for (int k = 0; k < 9; ++k) e.R[k] = c.R[k];
    e.W = c.width;
    e.H = c.height;
    return e;
}

bool env_ok(const rast_envmap_t* env) {
    return env && env->map && env->height > 0 && env->width > 0 && channels_supported(env->channels) &&
           (int64_t)env->height * env->width < ((int64_t)1 << 32) / 16;
}

// Texels are read as 16-byte vectors when C is a multiple of 4.
bool env_aligned(const rast_envmap_t* env) {
    return env->channels % 4 != 0 || (reinterpret_cast<uintptr_t>(env->map) & 15) == 0;
}

bool cam_ok(const rast_camera_t* c) {
    return c && c->width > 0 && c->height > 0 && c->fx != 0.f && c->fy != 0.f;
}

template <typename F>
cudaError_t dispatch_c(int C, F&& f) {
    switch (C) {
        case 1: return f(std::integral_constant<int, 1>());
        case 2: return f(std::integral_constant<int, 2>());
        case 3: return f(std::integral_constant<int, 3>());
        case 4: return f(std::integral_constant<int, 4>());
        case 8: return f(std::integral_constant<int, 8>());
        case 16: return f(std::integral_constant<int, 16>());
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace rast

using namespace rast;

extern "C" {

rast_status_t rasterize_view_dirs(const rast_camera_t* cam, float* dirs, void* stream) {
    if (!cam_ok(cam) || !dirs) return RAST_ERR_ARG;
    const int64_t n = (int64_t)cam->width * cam->height;
    cudaStream_t s = (cudaStream_t)stream;
    {
        ProfScope ps("bg.dirs", s);
        k_view_dirs<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(env_cam(*cam), dirs);
    }
    return cudaGetLastError() == cudaSuccess ? RAST_OK : RAST_ERR_CUDA;
}

rast_status_t rasterize_bg_composite(const rast_camera_t* cam, const rast_envmap_t* env, const float* dirs,
                                     const float* feat, const float* alpha, float* out, void* stream) {
    if (!cam_ok(cam) || !feat || !alpha || !out) return RAST_ERR_ARG;
    if (!env || !env->map || env->height <= 0 || env->width <= 0) return RAST_ERR_ARG;
    if (!env_ok(env)) return RAST_ERR_NOT_SUPPORTED;
    if (!env_aligned(env)) return RAST_ERR_ARG;
    const int64_t n = (int64_t)cam->width * cam->height;
    cudaStream_t s = (cudaStream_t)stream;
    const EnvCam ec = env_cam(*cam);
    cudaError_t e = dispatch_c(env->channels, [&](auto cc) {
        constexpr int C = decltype(cc)::value;
        ProfScope ps("bg.fwd", s);
        k_bg_fwd<C><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ec, env->map, env->height, env->width, dirs,
                                                                 feat, alpha, out);
        return cudaGetLastError();
    });
    return e == cudaSuccess ? RAST_OK : RAST_ERR_CUDA;
}

size_t rasterize_bg_scratch_size(const rast_envmap_t* env) {
    if (!env_ok(env)) return 0;
    return ((size_t)env->height * env->width * env->channels * 8 + 255) & ~(size_t)255;
}

rast_status_t rasterize_bg_composite_bwd(const rast_camera_t* cam, const rast_envmap_t* env, const float* dirs,
                                         const float* alpha, const float* g, float* g_alpha, float* d_map,
                                         void* scratch, size_t scratch_bytes, void* stream) {
    if (!cam_ok(cam) || !alpha || !g || !d_map || !scratch) return RAST_ERR_ARG;
    if (!env || !env->map || env->height <= 0 || env->width <= 0) return RAST_ERR_ARG;
    if (!env_ok(env)) return RAST_ERR_NOT_SUPPORTED;
    if (!env_aligned(env)) return RAST_ERR_ARG;
    if (scratch_bytes < rasterize_bg_scratch_size(env)) return RAST_ERR_CAPACITY;
    if ((reinterpret_cast<uintptr_t>(scratch) & 7) != 0) return RAST_ERR_ARG;
    const int64_t n = (int64_t)cam->width * cam->height;
    const int64_t m = (int64_t)env->height * env->width * env->channels;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* acc = static_cast<unsigned long long*>(scratch);
    if (cudaMemsetAsync(acc, 0, (size_t)m * 8, s) != cudaSuccess) return RAST_ERR_CUDA;
    const EnvCam ec = env_cam(*cam);
    cudaError_t e = dispatch_c(env->channels, [&](auto cc) {
        constexpr int C = decltype(cc)::value;
        ProfScope ps("bg.bwd", s);
        k_bg_bwd<C><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ec, env->map, env->height, env->width, dirs,
                                                                 alpha, g, g_alpha, acc);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return RAST_ERR_CUDA;
    {
        ProfScope ps("bg.map_grad", s);
        k_fixed_to_float<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(acc, m, d_map);
    }
    return cudaGetLastError() == cudaSuccess ? RAST_OK : RAST_ERR_CUDA;
}

}  // extern "C"

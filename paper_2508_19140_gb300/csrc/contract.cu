// Spherical contraction of sampled positions in one kernel (Sec. 3.4,
// "Implementation Improvements": the contraction of Mip-NeRF 360 that INPC
// applies to the points before the appearance field, fused instead of a chain
// of framework kernels):
//   c(x) = x                      if |x| <= 1
//        = (2 - 1/|x|) x / |x|    otherwise.
// Memory-bound: 12 bytes in, 12 bytes out per point. Each thread handles four
// points as three 16-byte loads and stores when the arrays are 16-byte
// aligned; IEEE-rounded square root and divisions.
#include "rast_internal.cuh"

namespace rast {
namespace {

__device__ __forceinline__ void contract3(float& a, float& b, float& c) {
    const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b)), __fmul_rn(c, c));
    if (r2 <= 1.f) return;
    float r;
    if (r2 < 3.0e38f) {
        r = __fsqrt_rn(r2);
    } else {  // |x| beyond ~1.7e19: scale so the squares do not overflow
        const float m = fmaxf(fabsf(a), fmaxf(fabsf(b), fabsf(c)));
        const float p = __fdiv_rn(a, m), q = __fdiv_rn(b, m), t = __fdiv_rn(c, m);
        r = __fmul_rn(m, __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(p, p), __fmul_rn(q, q)), __fmul_rn(t, t))));
    }
    const float k = __fsub_rn(2.f, __fdiv_rn(1.f, r));  // contracted radius
    a = __fmul_rn(__fdiv_rn(a, r), k);
    b = __fmul_rn(__fdiv_rn(b, r), k);
    c = __fmul_rn(__fdiv_rn(c, r), k);
}

__global__ void __launch_bounds__(256) k_contract_vec4(const float4* __restrict__ in, float4* __restrict__ out,
                                                       int64_t groups) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= groups) return;
    float4 v0 = in[3 * g], v1 = in[3 * g + 1], v2 = in[3 * g + 2];
    // points: (v0.x v0.y v0.z) (v0.w v1.x v1.y) (v1.z v1.w v2.x) (v2.y v2.z v2.w)
    contract3(v0.x, v0.y, v0.z);
    contract3(v0.w, v1.x, v1.y);
    contract3(v1.z, v1.w, v2.x);
    contract3(v2.y, v2.z, v2.w);
    out[3 * g] = v0;
    out[3 * g + 1] = v1;
    out[3 * g + 2] = v2;
}

__global__ void __launch_bounds__(256) k_contract(const float* __restrict__ in, float* __restrict__ out,
                                                  int64_t first, int64_t n) {
    const int64_t i = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float a = in[3 * i], b = in[3 * i + 1], c = in[3 * i + 2];
    contract3(a, b, c);
    out[3 * i] = a;
    out[3 * i + 1] = b;
    out[3 * i + 2] = c;
}

}  // namespace
}  // namespace rast

using namespace rast;

extern "C" rast_status_t rasterize_contract(const float* xyz, float* out, int64_t n, void* stream) {
    if (n < 0 || (n > 0 && (!xyz || !out))) return RAST_ERR_ARG;
    if (n == 0) return RAST_OK;
    cudaStream_t s = (cudaStream_t)stream;
    ProfScope ps("contract", s);
    const bool vec = ((reinterpret_cast<uintptr_t>(xyz) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    int64_t done = 0;
    if (vec) {
        const int64_t groups = n / 4;
        if (groups > 0)
            k_contract_vec4<<<(unsigned)((groups + 255) / 256), 256, 0, s>>>(
                reinterpret_cast<const float4*>(xyz), reinterpret_cast<float4*>(out), groups);
        done = groups * 4;
    }
    if (done < n)
        k_contract<<<(unsigned)((n - done + 255) / 256), 256, 0, s>>>(xyz, out, done, n);
    return cudaGetLastError() == cudaSuccess ? RAST_OK : RAST_ERR_CUDA;
}

// K1: projection + footprint + tile count, one thread per point.
//
// Pinhole projection of Sec. 2 ("Rendering Feature Maps"); footprints of
// Sec. 3.2: a bilinear 2x2 splat, or an isotropic world-space Gaussian
// projected with the affine approximation, dilated by variance 0.16 and
// truncated at 3 sigma ("Rendering Points as Small Gaussians"). Every value
// that decides a discrete outcome (culling, pixel box, tile rect, depth key)
// is computed in FP32 with round-to-nearest intrinsics in one fixed order, so
// the result does not depend on FMA contraction:
//   x_c = ((R0 x + R1 y) + R2 z) + t0,  u = fx (x_c / z_c) + cx,
//   bilinear box {floor(u - 1/2), +1} x {floor(v - 1/2), +1},
//   Gaussian box [ceil(u - 1/2 - r), floor(u - 1/2 + r)], r = ceil(3 sqrt(lambda_max)).
// Output per point: a record (u, v, z, o[, conic a b c, r], features) with a
// power-of-two stride of 32-128 bytes (one DRAM burst per gather, 16-byte
// chunks for the blends' cp.async copies), the depth key
// bits(z) - bits(near) for the split sort's first stage, the tile rect and the
// number of tiles it touches.
#include "rast_internal.cuh"

namespace rast {
namespace {

// Inputs of one point, loaded before any of the block's points is computed.
struct PointIn {
    float x, y, z, o, s;
    uint4 f[2];      // the features' raw words when they fit in 32 aligned bytes
    int nf;          // feature words in f as 16-byte vectors: 1 or 2; -1 = one 8-byte pair
                     // (BF16, C = 4); 0 = not loaded (the body copies the features itself)
};

// Loads a point's inputs (features as raw words on the aligned paths: FP32 with
// C a multiple of 4 up to 8, BF16 with C 4, 8 or 16).
template <int MODE>
__device__ __forceinline__ void load_point(const ViewTable& vt, const ViewDev& V, int64_t i, PointIn& in) {
    in.x = V.xyz[3 * i + 0];
    in.y = V.xyz[3 * i + 1];
    in.z = V.xyz[3 * i + 2];
    in.o = V.opacity[i];
    in.s = 0.f;
    if (MODE == 1) in.s = V.scale ? V.scale[i] : __fdiv_rn(__fmul_rn(5.f, V.near_z), V.fx);
    in.nf = 0;
    const int C = vt.C;
    if (!vt.bf16) {
        // FP32: C = 4 is one 16-byte vector, C = 8 two.
        const float* f = static_cast<const float*>(V.feat) + i * C;
        if ((C == 4 || C == 8) && (reinterpret_cast<uintptr_t>(f) & 15) == 0) {
            in.f[0] = *reinterpret_cast<const uint4*>(f);
            if (C == 8) in.f[1] = *reinterpret_cast<const uint4*>(f + 4);
            in.nf = C / 4;
        }
    } else {
        // BF16: C = 8 is one 16-byte vector, C = 16 two, C = 4 one 8-byte pair.
        const unsigned short* f = static_cast<const unsigned short*>(V.feat) + i * C;
        const uintptr_t fa = reinterpret_cast<uintptr_t>(f);
        if ((C == 8 || C == 16) && (fa & 15) == 0) {
            in.f[0] = *reinterpret_cast<const uint4*>(f);
            if (C == 16) in.f[1] = *reinterpret_cast<const uint4*>(f + 8);
            in.nf = C / 8;
        } else if (C == 4 && (fa & 7) == 0) {
            const uint2 q = *reinterpret_cast<const uint2*>(f);
            in.f[0] = make_uint4(q.x, q.y, 0u, 0u);
            in.nf = -1;
        }
    }
}

template <int MODE>
__device__ __forceinline__ void project_point(const ViewTable& vt, const Bufs& b, bool write_vals, int64_t gi,
                                              const ViewDev& V, int64_t i, const PointIn& in) {
    const float x = in.x, y = in.y, z = in.z;
    float xc = __fmul_rn(V.R[0], x);
    xc = __fadd_rn(xc, __fmul_rn(V.R[1], y));
    xc = __fadd_rn(xc, __fmul_rn(V.R[2], z));
    xc = __fadd_rn(xc, V.t[0]);
    float yc = __fmul_rn(V.R[3], x);
    yc = __fadd_rn(yc, __fmul_rn(V.R[4], y));
    yc = __fadd_rn(yc, __fmul_rn(V.R[5], z));
    yc = __fadd_rn(yc, V.t[1]);
    float zc = __fmul_rn(V.R[6], x);
    zc = __fadd_rn(zc, __fmul_rn(V.R[7], y));
    zc = __fadd_rn(zc, __fmul_rn(V.R[8], z));
    zc = __fadd_rn(zc, V.t[2]);

    bool vis = (zc > V.near_z) && (zc < V.far_z);
    float u = 0.f, v = 0.f, ca = 0.f, cb = 0.f, cc = 0.f, r = 0.f;
    int bx0 = 0, bx1 = -1, by0 = 0, by1 = -1;
    if (vis) {
        u = __fadd_rn(__fmul_rn(V.fx, __fdiv_rn(xc, zc)), V.cx);
        v = __fadd_rn(__fmul_rn(V.fy, __fdiv_rn(yc, zc)), V.cy);
        const float um = __fsub_rn(u, 0.5f), vm = __fsub_rn(v, 0.5f);
        const float Wm1 = (float)(V.W - 1), Hm1 = (float)(V.H - 1);
        if (MODE == 0) {
            const float fi = floorf(um), fj = floorf(vm);
            vis = (fi >= -1.f) && (fi <= Wm1) && (fj >= -1.f) && (fj <= Hm1);
            if (vis) {
                const int i0 = (int)fi, j0 = (int)fj;
                bx0 = max(i0, 0);
                bx1 = min(i0 + 1, V.W - 1);
                by0 = max(j0, 0);
                by1 = min(j0 + 1, V.H - 1);
            }
        } else {
            const float s = in.s;
            const float s2 = __fmul_rn(s, s);
            const float zz = __fmul_rn(zc, zc);
            float S00, S01, S11;
            if (vt.gauss_cov == 0) {
                const float j00 = __fdiv_rn(V.fx, zc), j11 = __fdiv_rn(V.fy, zc);
                const float j02 = -__fdiv_rn(__fmul_rn(V.fx, xc), zz);
                const float j12 = -__fdiv_rn(__fmul_rn(V.fy, yc), zz);
                const float d0 = __fadd_rn(__fmul_rn(j00, j00), __fmul_rn(j02, j02));
                const float d1 = __fadd_rn(__fmul_rn(j11, j11), __fmul_rn(j12, j12));
                const float e = __fmul_rn(j02, j12);
                S00 = __fadd_rn(__fmul_rn(s2, d0), vt.dilation);
                S01 = __fmul_rn(s2, e);
                S11 = __fadd_rn(__fmul_rn(s2, d1), vt.dilation);
            } else {
                const float ff = __fdiv_rn(__fmul_rn(V.fx, V.fy), zz);
                S00 = __fadd_rn(__fmul_rn(s2, ff), vt.dilation);
                S11 = S00;
                S01 = 0.f;
            }
            const float det = __fsub_rn(__fmul_rn(S00, S11), __fmul_rn(S01, S01));
            ca = __fdiv_rn(S11, det);
            cb = -__fdiv_rn(S01, det);
            cc = __fdiv_rn(S00, det);
            const float mid = __fmul_rn(0.5f, __fadd_rn(S00, S11));
            const float hd = __fmul_rn(0.5f, __fsub_rn(S00, S11));
            const float disc = __fsqrt_rn(__fadd_rn(__fmul_rn(hd, hd), __fmul_rn(S01, S01)));
            const float lmax = __fadd_rn(mid, disc);
            r = ceilf(__fmul_rn(3.f, __fsqrt_rn(lmax)));
            float lox = ceilf(__fsub_rn(um, r)), hix = floorf(__fadd_rn(um, r));
            float loy = ceilf(__fsub_rn(vm, r)), hiy = floorf(__fadd_rn(vm, r));
            lox = fmaxf(lox, 0.f);
            loy = fmaxf(loy, 0.f);
            hix = fminf(hix, Wm1);
            hiy = fminf(hiy, Hm1);
            vis = (lox <= hix) && (loy <= hiy);
            if (vis) {
                bx0 = (int)lox; bx1 = (int)hix; by0 = (int)loy; by1 = (int)hiy;
            }
        }
    }

    uint2 rect = make_uint2(1u, 0u);
    uint32_t count = 0;
    uint32_t key = V.key_cull;
    if (vis) {
        const int sh = __ffs(vt.tile) - 1;  // tile edges are powers of two (1, 8, 16)
        const int tx0 = bx0 >> sh, tx1 = bx1 >> sh, ty0 = by0 >> sh, ty1 = by1 >> sh;
        rect = make_uint2((uint32_t)tx0 | ((uint32_t)ty0 << 16), (uint32_t)tx1 | ((uint32_t)ty1 << 16));
        count = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
        key = __float_as_uint(zc) - V.key_base;

        // Record: u, v, z, o [, a, b, c, r], features.
        uint32_t* rec = b.rec + gi * vt.rec_words;
        const float o = in.o;
        *reinterpret_cast<uint4*>(rec) =
            make_uint4(__float_as_uint(u), __float_as_uint(v), __float_as_uint(zc), __float_as_uint(o));
        if (MODE == 1)
            *reinterpret_cast<uint4*>(rec + 4) = make_uint4(__float_as_uint(ca), __float_as_uint(cb),
                                                            __float_as_uint(cc), __float_as_uint(r));
        uint32_t* fw = rec + vt.feat_word;
        const int C = vt.C;
        if (in.nf != 0) {
            // exactly the feature words of the record: 8 bytes, or 16 / 32 bytes
            if (in.nf < 0) {
                *reinterpret_cast<uint2*>(fw) = make_uint2(in.f[0].x, in.f[0].y);
            } else {
                *reinterpret_cast<uint4*>(fw) = in.f[0];
                if (in.nf == 2) *reinterpret_cast<uint4*>(fw + 4) = in.f[1];
            }
        } else if (!vt.bf16) {
            const float* f = static_cast<const float*>(V.feat) + i * C;
            if ((C & 3) == 0 && ((reinterpret_cast<uintptr_t>(f) & 15) == 0)) {
                for (int c = 0; c < C; c += 4)
                    *reinterpret_cast<float4*>(fw + c) = *reinterpret_cast<const float4*>(f + c);
            } else {
                for (int c = 0; c < C; ++c) fw[c] = __float_as_uint(f[c]);
            }
        } else {
            const unsigned short* f = static_cast<const unsigned short*>(V.feat) + i * C;
            const uintptr_t fa = reinterpret_cast<uintptr_t>(f);
            if ((C & 7) == 0 && (fa & 15) == 0) {
                for (int c = 0; c < C; c += 8)
                    *reinterpret_cast<uint4*>(fw + (c >> 1)) = *reinterpret_cast<const uint4*>(f + c);
            } else if ((C & 3) == 0 && (fa & 7) == 0) {
                for (int c = 0; c < C; c += 4)
                    *reinterpret_cast<uint2*>(fw + (c >> 1)) = *reinterpret_cast<const uint2*>(f + c);
            } else {
                for (int c = 0; c < C; c += 2) {
                    const uint32_t lo = f[c];
                    const uint32_t hi = (c + 1 < C) ? f[c + 1] : 0u;
                    fw[c >> 1] = lo | (hi << 16);
                }
            }
        }
    }
    b.keyA[0][gi] = key;
    if (write_vals) b.valA[0][gi] = (uint32_t)gi;
    if (MODE == 0)
        b.rect4[gi] = vis ? rect4_pack((int)(rect.x & 0xffffu), (int)(rect.x >> 16), (int)(rect.y & 0xffffu),
                                       (int)(rect.y >> 16))
                          : kRect4Empty;
    else
        b.rect[gi] = rect;
    if (MODE == 1) b.cnt[gi] = count;  // bilinear counts come from the packed rect (rect4_count)
    b.zbits[gi] = __float_as_uint(zc);
}

// kPointsPerThread points per thread, all their loads issued before any is
// computed: the kernel waits on one memory round trip per thread instead of
// two per point (inputs, then features).
constexpr int kPointsPerThread = 2;

template <int MODE>
__global__ void __launch_bounds__(256) k_project(const ViewTable vt, const Bufs b, bool write_vals) {
    constexpr int K = kPointsPerThread;
    const int64_t g0 = (int64_t)blockIdx.x * (256 * K) + threadIdx.x;
    PointIn in[K];
    int vi[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t gi = g0 + k * 256;
        vi[k] = 0;
        if (gi < vt.n_total) {
            vi[k] = view_of_point(vt, gi);
            const ViewDev& V = vt.v[vi[k]];
            load_point<MODE>(vt, V, gi - V.pt_off, in[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t gi = g0 + k * 256;
        if (gi < vt.n_total) {
            const ViewDev& V = vt.v[vi[k]];
            project_point<MODE>(vt, b, write_vals, gi, V, gi - V.pt_off, in[k]);
        }
    }
}

}  // namespace

cudaError_t launch_project(const ViewTable& vt, const Bufs& b, bool write_vals, cudaStream_t s) {
    if (vt.n_total == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((vt.n_total + 256 * kPointsPerThread - 1) / (256 * kPointsPerThread));
    ProfScope ps("project", s);
    if (vt.mode == 0) k_project<0><<<grid, 256, 0, s>>>(vt, b, write_vals);
    else k_project<1><<<grid, 256, 0, s>>>(vt, b, write_vals);
    return cudaGetLastError();
}

}  // namespace rast

// Shared pieces of the blend kernels (K6 forward, K7 backward).
//
// A record is gathered once per (tile, batch) by one thread and staged in
// shared memory; the per-pixel work then reads only shared memory. The
// per-fragment alpha and the coverage test are single device functions used
// by both passes, so the backward replays the forward's FP32 decisions bit for
// bit (round-to-nearest intrinsics, no contraction):
//   bilinear:  a = (u - 1/2) - floor(u - 1/2), w = wx * wy with wx = 1 - a at
//              the anchor column and a at the next one, alpha = min(o w, amax);
//   Gaussian:  d = (px - (u - 1/2), py - (v - 1/2)),
//              m = ((a dx) dx + 2 (b dx) dy) + (c dy) dy, covered iff the pixel
//              is in the box of radius r and m <= 9, alpha = min(o exp(-m/2), amax);
//   step:      T' = T (1 - alpha); the fragment is excluded and the pixel stops
//              once T' < t_min.
#pragma once

#include "rast_internal.cuh"

namespace rast {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---- cp.async (LDGSTS) staging ----------------------------------------------
// Each thread copies its own record into a shared-memory ring slot; copies are
// grouped per batch and retired with wait_group, so several batches are in
// flight per CTA without any spin-wait.

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem_dst)), "l"(gmem_src)
                 : "memory");
}

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(smem_dst)), "l"(gmem_src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Arrives on `bar` once every cp.async this thread has issued so far has
// landed (counted as one of the barrier's expected arrivals).
__device__ __forceinline__ void cp_async_mbar_arrive_noinc(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// 1 / x with the hardware reciprocal (rcp.approx: at most 1 ulp off, where an
// IEEE-rounded reciprocal is a multi-instruction sequence). The backward's
// replay T_k = T_{k+1} / (1 - alpha_k) uses it: 1 - alpha >= 1 - alpha_max
// = 0.01, so x is never tiny, and each replay step then carries about 1.5 ulp
// instead of 1 (the gradients' tolerance covers replays of thousands of steps).
__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---- TMA bulk copies completed on an mbarrier ---------------------------------
// One thread arms the barrier with the batch's byte count and issues a single
// global -> shared bulk copy of a contiguous run of records; every thread then
// waits on the barrier's phase. Each wait is bounded: after kMbarPolls polls
// it reports failure (the caller raises the timeout bit of the error word and
// stops) instead of spinning on.

constexpr uint32_t kMbarPolls = 1u << 20;

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes the barriers' initialisation visible to the copy engine (follow with
// a CTA barrier before the first copy).
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arms `bar` for `bytes` and copies them from global `src` to shared `dst`
// (both 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    const uint32_t b = smem_addr(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(b)
                 : "memory");
}

// Waits until the phase of `bar` with this parity has completed; false if it
// did not within kMbarPolls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t b = smem_addr(bar);
    for (uint32_t i = 0; i < kMbarPolls; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(b), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Record stride (u32 words) for a mode, channel count and feature type; the
// host computes the same value (rec_words). A power of two of at least 8
// words (32 bytes): every record is 16-byte aligned for cp.async and no record
// straddles a 64-byte DRAM burst, so each gather costs one burst.
template <int MODE, int C, bool BF16>
struct RecLayout {
    static constexpr int feat_word = MODE == 0 ? 4 : 8;
    static constexpr int feat_words = BF16 ? (C + 1) / 2 : C;
    static constexpr int need = feat_word + feat_words;
    static constexpr int words = need <= 8 ? 8 : (need <= 16 ? 16 : 32);
};

// Shared-memory stride (words) of a staged record: 4 words more than its
// global stride, so consecutive records start in 8 different 4-bank groups
// (a stride of 8, 16 or 32 words would start them in at most 4) and the
// per-fragment reads of random records conflict less; still a multiple of 16
// bytes for cp.async.
__host__ __device__ constexpr int ring_stride(int rw) { return rw + 4; }

// 128-byte aligned view of a dynamic shared-memory buffer (allocated with
// 128 spare bytes).
__device__ __forceinline__ uint32_t* align128(uint32_t* p) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uint32_t sa = smem_addr(p);
    return reinterpret_cast<uint32_t*>(a + ((128u - (sa & 127u)) & 127u));
}

// Stores N floats at dst: 16-byte vector stores when N is a multiple of 4 and
// dst is 16-byte aligned, scalar stores otherwise.
template <int N>
__device__ __forceinline__ void store_row(float* dst, const float* v) {
    if constexpr (N % 4 == 0) {
        if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
#pragma unroll
            for (int k = 0; k < N; k += 4)
                *reinterpret_cast<float4*>(dst + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < N; ++k) dst[k] = v[k];
}

// Features of one record as FP32 registers.
template <int C, bool BF16>
__device__ __forceinline__ void load_features(const uint32_t* __restrict__ rp, float (&f)[C]) {
    if (!BF16) {
        if (C % 4 == 0) {
#pragma unroll
            for (int c = 0; c < C; c += 4) {
                const uint4 q = *reinterpret_cast<const uint4*>(rp + c);
                f[c] = __uint_as_float(q.x);
                f[c + 1] = __uint_as_float(q.y);
                f[c + 2] = __uint_as_float(q.z);
                f[c + 3] = __uint_as_float(q.w);
            }
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) f[c] = __uint_as_float(rp[c]);
        }
    } else {
        if (C % 8 == 0) {
#pragma unroll
            for (int c = 0; c < C; c += 8) {
                const uint4 q = *reinterpret_cast<const uint4*>(rp + c / 2);
                f[c] = bf16lo(q.x); f[c + 1] = bf16hi(q.x);
                f[c + 2] = bf16lo(q.y); f[c + 3] = bf16hi(q.y);
                f[c + 4] = bf16lo(q.z); f[c + 5] = bf16hi(q.z);
                f[c + 6] = bf16lo(q.w); f[c + 7] = bf16hi(q.w);
            }
        } else {
#pragma unroll
            for (int c = 0; c < C; c += 2) {
                const uint32_t w = rp[c / 2];
                f[c] = bf16lo(w);
                if (c + 1 < C) f[c + 1] = bf16hi(w);
            }
        }
    }
}

// Bilinear anchor and fractions from the screen position (exact in FP32).
struct BilinGeom {
    int i0, j0;
    float a, b;
};

__device__ __forceinline__ BilinGeom bilin_geom(float u, float v) {
    const float um = __fsub_rn(u, 0.5f), vm = __fsub_rn(v, 0.5f);
    const float fi = floorf(um), fj = floorf(vm);
    BilinGeom g;
    g.i0 = (int)fi;
    g.j0 = (int)fj;
    g.a = __fsub_rn(um, fi);
    g.b = __fsub_rn(vm, fj);
    return g;
}

// Bilinear weight of the fragment at pixel (px, py) (a pixel of the 2x2 box).
__device__ __forceinline__ float bilin_weight(int px, int py, int i0, int j0, float a, float b) {
    const float wx = (px == i0) ? __fsub_rn(1.f, a) : a;
    const float wy = (py == j0) ? __fsub_rn(1.f, b) : b;
    return __fmul_rn(wx, wy);
}

// Gaussian pixel box from the record's radius r (inclusive, unclipped).
struct GaussBox {
    int x0, x1, y0, y1;
};

__device__ __forceinline__ GaussBox gauss_box(float um, float vm, float r) {
    GaussBox bx;
    bx.x0 = (int)ceilf(__fsub_rn(um, r));
    bx.x1 = (int)floorf(__fadd_rn(um, r));
    bx.y0 = (int)ceilf(__fsub_rn(vm, r));
    bx.y1 = (int)floorf(__fadd_rn(vm, r));
    return bx;
}

// Mahalanobis distance squared of pixel (px, py) (FP32, fixed order).
__device__ __forceinline__ float gauss_m(float dx, float dy, float ca, float cb, float cc) {
    const float t0 = __fmul_rn(__fmul_rn(ca, dx), dx);
    const float t1 = __fmul_rn(__fmul_rn(cb, dx), dy);
    const float t2 = __fmul_rn(__fmul_rn(cc, dy), dy);
    return __fadd_rn(__fadd_rn(t0, __fadd_rn(t1, t1)), t2);
}

__device__ __forceinline__ float gauss_value(float m) { return expf(__fmul_rn(-0.5f, m)); }

}  // namespace rast

// CPU ORACLE for the differentiable tiled point rasterizer.
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call
// this file; only the tests, the package's smoke check and the benchmark's CPU
// baseline leg do. It shares no code, header, table or helper with the CUDA
// path.
//
// What it computes is the plain definition, in the paper's order, one point and
// one pixel at a time:
//   (1) project each point through a pinhole camera (Sec. 2 "Rendering Feature
//       Maps": points p_i rendered to a feature image F in R^{H x W x n_w});
//   (2) give it a footprint: a bilinear 2x2 splat whose weights sum to one
//       (Sec. 3.2, "Rendering Points as Small Gaussians", first paragraph), or
//       an isotropic world-space Gaussian projected with the affine (EWA)
//       approximation, dilated by a 2D Gaussian of variance 0.16 and truncated
//       at 3 sigma (same paragraph);
//   (3) list, per pixel, every covering fragment and sort the list by depth
//       (Sec. 2, "Rendering Feature Maps": depth-sorted per-pixel lists);
//   (4) alpha-blend front to back by Eq. 1, F = sum_i T_i a_i f_i with
//       T_i = prod_{j<i} (1 - a_j);
//   (5) differentiate by the corrected Eq. 2 of the appendix ("Addressing
//       Gradient Approximations"), including fragments whose alpha is zero.
// The tile lists of Sec. 3.2 "Tiled Rendering" (per-tile copies ordered by
// depth, then by point index) are built separately and only serve to check the
// sort order bit for bit; the image never depends on them.
//
// Precision. Values (alpha, T, F, depth, all gradients) are FP64. Every
// discrete decision -- visibility, the pixel box, the bilinear anchor,
// Gaussian coverage, the alpha clamp and early termination -- is taken in the
// precision selected by `pin32`: with pin32 = 1 the projection is evaluated in
// FP32 with one fixed operation order (no fused multiply-add) and the decisions
// run in FP32, which is the arithmetic the GPU kernels use for them; with
// pin32 = 0 everything, decisions included, is FP64 (used by the finite
// difference checks). The operation order is stated in `project()` below.
//
// Readings where the paper is silent (each one also listed in the design
// notes): pixel centres at (i + 1/2, j + 1/2); bilinear anchor floor(u - 1/2);
// fragment alpha = min(o * w, alpha_max) with alpha_max = 0.99; depth key =
// FP32 bits of the view-space z; equal depths ordered by point index; stop
// before a fragment once T * (1 - alpha) < t_min (the fragment is excluded);
// no small-alpha skip; the Gaussian covers a pixel iff its Mahalanobis
// distance squared is <= 9 and the pixel lies in the box of radius
// r = ceil(3 sqrt(lambda_max)); depth output D = sum_i T_i a_i z_i.
//
// Parity: pinned by closed forms, invariants, brute force on tiny inputs and
// FP64 central finite differences (tests/test_oracle_pins.py). The paper
// prints no numeric output of the rasterizer, so whole-path accuracy against
// the paper itself is unpinned.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

typedef struct {
    float fx, fy, cx, cy;
    float R[9];      // row-major, x_c = R x_w + t
    float t[3];
    float near_z, far_z;
    int32_t width, height;
} orc_camera_t;

typedef struct {
    int32_t mode;       // 0 = bilinear 2x2 splat, 1 = Gaussian
    int32_t gauss_cov;  // 0 = EWA affine projection, 1 = isotropic in screen space
    int32_t tile;       // tile edge in pixels (tile lists only)
    int32_t pin32;      // 1 = FP32 pinned decisions, 0 = all FP64
    float t_min;        // early termination threshold on T (1e-4)
    float alpha_max;    // alpha clamp (0.99)
    float dilation;     // screen-space dilation variance (0.16)
    int32_t n_threads;  // OpenMP threads, <= 0: library default
} orc_opts_t;

}  // extern "C"

namespace {

// One projected point. Values are FP64 copies of what the decision precision
// produced (exact promotions when pin32 = 1).
struct Splat {
    bool vis = false;       // in front of near, before far, non-empty in-image box
    uint32_t zbits = 0;     // FP32 bit pattern of z_c (sort key)
    double xc = 0, yc = 0, zc = 0;  // camera space
    double u = 0, v = 0;    // screen position
    double s = 0;           // world-space Gaussian scale
    double ca = 0, cb = 0, cc = 0;  // conic = inverse 2D covariance
    double S00 = 0, S01 = 0, S11 = 0;  // 2D covariance
    double um = 0, vm = 0;  // u - 1/2, v - 1/2
    int i0 = 0, j0 = 0;     // bilinear anchor
    double a = 0, b = 0;    // bilinear fractions
    int bx0 = 0, bx1 = -1, by0 = 0, by1 = -1;  // inclusive in-image pixel box
};

uint32_t f32_bits(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    return b;
}

// Projection of point p in precision T (float: pinned FP32 order; double: FP64).
//   x_c = ((R0 x + R1 y) + R2 z) + t0   (likewise y_c, z_c)
//   u   = fx * (x_c / z_c) + cx          (likewise v)
// Bilinear: um = u - 1/2, i0 = floor(um), a = um - i0 (exact), box {i0, i0+1}.
// Gaussian (EWA): J = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]],
//   Sigma = s^2 J J^T + dil I; conic = Sigma^{-1};
//   lambda_max = (S00+S11)/2 + sqrt(((S00-S11)/2)^2 + S01^2);
//   r = ceil(3 sqrt(lambda_max)); box = [ceil(um - r), floor(um + r)].
template <typename T>
Splat project(const double* p, double scale, bool has_scale, const orc_camera_t& cam,
              const orc_opts_t& o) {
    Splat sp;
    const T x = (T)p[0], y = (T)p[1], z = (T)p[2];
    T R[9], t[3];
    for (int k = 0; k < 9; ++k) R[k] = (T)cam.R[k];
    for (int k = 0; k < 3; ++k) t[k] = (T)cam.t[k];
    T xc = R[0] * x; xc = xc + R[1] * y; xc = xc + R[2] * z; xc = xc + t[0];
    T yc = R[3] * x; yc = yc + R[4] * y; yc = yc + R[5] * z; yc = yc + t[1];
    T zc = R[6] * x; zc = zc + R[7] * y; zc = zc + R[8] * z; zc = zc + t[2];
    sp.xc = (double)xc; sp.yc = (double)yc; sp.zc = (double)zc;
    sp.zbits = f32_bits((float)zc);
    const T nearT = (T)cam.near_z, farT = (T)cam.far_z;
    if (!(zc > nearT && zc < farT)) return sp;
    const T fx = (T)cam.fx, fy = (T)cam.fy, cx = (T)cam.cx, cy = (T)cam.cy;
    T qx = xc / zc; T u = fx * qx; u = u + cx;
    T qy = yc / zc; T v = fy * qy; v = v + cy;
    sp.u = (double)u; sp.v = (double)v;
    const T half = (T)0.5;
    const T um = u - half, vm = v - half;
    sp.um = (double)um; sp.vm = (double)vm;
    const T Wm1 = (T)(cam.width - 1), Hm1 = (T)(cam.height - 1);
    if (o.mode == 0) {
        const T fi = std::floor(um), fj = std::floor(vm);
        if (!(fi >= (T)-1 && fi <= Wm1 && fj >= (T)-1 && fj <= Hm1)) return sp;
        sp.i0 = (int)fi; sp.j0 = (int)fj;
        const T a = um - fi, b = vm - fj;
        sp.a = (double)a; sp.b = (double)b;
        sp.bx0 = std::max(sp.i0, 0); sp.bx1 = std::min(sp.i0 + 1, cam.width - 1);
        sp.by0 = std::max(sp.j0, 0); sp.by1 = std::min(sp.j0 + 1, cam.height - 1);
        sp.vis = true;
        return sp;
    }
    // Gaussian footprint.
    T s = has_scale ? (T)scale : (T)((T)5 * nearT / fx);
    sp.s = (double)s;
    const T s2 = s * s;
    const T dil = (T)o.dilation;
    const T zz = zc * zc;
    T S00, S01, S11;
    if (o.gauss_cov == 0) {
        const T j00 = fx / zc, j11 = fy / zc;
        T j02 = fx * xc; j02 = j02 / zz; j02 = -j02;
        T j12 = fy * yc; j12 = j12 / zz; j12 = -j12;
        T d0 = j00 * j00; d0 = d0 + j02 * j02;
        T d1 = j11 * j11; d1 = d1 + j12 * j12;
        T e = j02 * j12;
        S00 = s2 * d0; S00 = S00 + dil;
        S01 = s2 * e;
        S11 = s2 * d1; S11 = S11 + dil;
    } else {
        T ff = fx * fy; ff = ff / zz;
        S00 = s2 * ff; S00 = S00 + dil;
        S11 = S00;
        S01 = (T)0;
    }
    sp.S00 = (double)S00; sp.S01 = (double)S01; sp.S11 = (double)S11;
    T det = S00 * S11; det = det - S01 * S01;
    const T ca = S11 / det, cb = -(S01 / det), cc = S00 / det;
    sp.ca = (double)ca; sp.cb = (double)cb; sp.cc = (double)cc;
    T mid = S00 + S11; mid = half * mid;
    T hd = S00 - S11; hd = half * hd;
    T disc = hd * hd; disc = disc + S01 * S01; disc = std::sqrt(disc);
    const T lmax = mid + disc;
    T r = std::sqrt(lmax); r = (T)3 * r; r = std::ceil(r);
    T lox = std::ceil(um - r), hix = std::floor(um + r);
    T loy = std::ceil(vm - r), hiy = std::floor(vm + r);
    lox = std::max(lox, (T)0); loy = std::max(loy, (T)0);
    hix = std::min(hix, Wm1); hiy = std::min(hiy, Hm1);
    if (!(lox <= hix && loy <= hiy)) return sp;
    sp.bx0 = (int)lox; sp.bx1 = (int)hix; sp.by0 = (int)loy; sp.by1 = (int)hiy;
    sp.vis = true;
    return sp;
}

Splat project_any(const double* p, double scale, bool has_scale, const orc_camera_t& cam,
                  const orc_opts_t& o) {
    return o.pin32 ? project<float>(p, scale, has_scale, cam, o)
                   : project<double>(p, scale, has_scale, cam, o);
}

// One fragment of splat `sp` at pixel (px, py). Returns false if it does not
// cover the pixel. `alpha_dec` is the alpha in decision precision (widened to
// double), `alpha` the FP64 value, `w_or_g` the bilinear weight or Gaussian
// value G = exp(-m/2) in FP64, `unclamped` whether o*w <= alpha_max.
struct Frag {
    double alpha_dec, alpha, w_or_g, m, dx, dy;
    bool unclamped;
};

template <typename T>
bool fragment(const Splat& sp, double opac, int px, int py, const orc_opts_t& o, Frag& fr) {
    if (px < sp.bx0 || px > sp.bx1 || py < sp.by0 || py > sp.by1) return false;
    const T oT = (T)opac;
    const T amax = (T)o.alpha_max;
    if (o.mode == 0) {
        // Bilinear weights: (1-a)(1-b), a(1-b), (1-a)b, ab.
        const T aT = (T)sp.a, bT = (T)sp.b;
        const T wx = (px == sp.i0) ? (T)1 - aT : aT;
        const T wy = (py == sp.j0) ? (T)1 - bT : bT;
        const T w = wx * wy;
        const T ow = oT * w;
        fr.unclamped = ow <= amax;
        fr.alpha_dec = (double)std::min(ow, amax);
        const double wx64 = (px == sp.i0) ? 1.0 - sp.a : sp.a;
        const double wy64 = (py == sp.j0) ? 1.0 - sp.b : sp.b;
        fr.w_or_g = wx64 * wy64;
        fr.alpha = fr.unclamped ? opac * fr.w_or_g : (double)o.alpha_max;
        fr.m = 0; fr.dx = 0; fr.dy = 0;
        return true;
    }
    // Gaussian: m = d^T conic d, d = pixel centre - (u, v); covered iff m <= 9.
    const T dx = (T)px - (T)sp.um, dy = (T)py - (T)sp.vm;
    const T ca = (T)sp.ca, cb = (T)sp.cb, cc = (T)sp.cc;
    T t0 = ca * dx; t0 = t0 * dx;
    T t1 = cb * dx; t1 = t1 * dy;
    T t2 = cc * dy; t2 = t2 * dy;
    T m = t0 + (t1 + t1); m = m + t2;
    if (!(m <= (T)9)) return false;
    const T g = std::exp((T)-0.5 * m);
    const T og = oT * g;
    fr.unclamped = og <= amax;
    fr.alpha_dec = (double)std::min(og, amax);
    const double dx64 = (double)px - sp.um, dy64 = (double)py - sp.vm;
    const double m64 = sp.ca * dx64 * dx64 + 2.0 * sp.cb * dx64 * dy64 + sp.cc * dy64 * dy64;
    fr.dx = dx64; fr.dy = dy64; fr.m = m64;
    fr.w_or_g = std::exp(-0.5 * m64);
    fr.alpha = fr.unclamped ? opac * fr.w_or_g : (double)o.alpha_max;
    return true;
}

struct Ctx {
    int64_t n;
    const double* xyz;
    const double* opacity;
    const double* scale;
    const double* feat;
    int C;
    orc_camera_t cam;
    orc_opts_t opt;
    std::vector<Splat> sp;
};

void project_all(Ctx& c) {
    c.sp.resize((size_t)c.n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c.n; ++i)
        c.sp[i] = project_any(c.xyz + 3 * i, c.scale ? c.scale[i] : 0.0, c.scale != nullptr,
                              c.cam, c.opt);
}

// Per-pixel fragment lists for the requested pixels (slot >= 0), each sorted
// by (FP32 depth bits, point index). CSR over slots.
void pixel_lists(const Ctx& c, const std::vector<int32_t>& slot_of_pixel, int64_t n_slots,
                 std::vector<int64_t>& start, std::vector<int32_t>& pts) {
    const int W = c.cam.width;
    std::vector<int64_t> cnt((size_t)n_slots + 1, 0);
    for (int64_t i = 0; i < c.n; ++i) {
        const Splat& s = c.sp[i];
        if (!s.vis) continue;
        for (int py = s.by0; py <= s.by1; ++py)
            for (int px = s.bx0; px <= s.bx1; ++px) {
                const int32_t sl = slot_of_pixel[(size_t)py * W + px];
                if (sl >= 0) cnt[sl + 1]++;
            }
    }
    for (int64_t k = 0; k < n_slots; ++k) cnt[k + 1] += cnt[k];
    start = cnt;
    pts.assign((size_t)start[n_slots], 0);
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t i = 0; i < c.n; ++i) {  // ascending index: ties stay in index order
        const Splat& s = c.sp[i];
        if (!s.vis) continue;
        for (int py = s.by0; py <= s.by1; ++py)
            for (int px = s.bx0; px <= s.bx1; ++px) {
                const int32_t sl = slot_of_pixel[(size_t)py * W + px];
                if (sl >= 0) pts[fill[sl]++] = (int32_t)i;
            }
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t k = 0; k < n_slots; ++k) {
        std::stable_sort(pts.begin() + start[k], pts.begin() + start[k + 1],
                         [&](int32_t p, int32_t q) { return c.sp[p].zbits < c.sp[q].zbits; });
    }
}

// Compositing of one pixel by Eq. 1 with early termination. Fills the blended
// fragments (in order) and returns the number blended.
struct PixOut {
    int32_t n_blend = 0, n_cover = 0, term_idx = -1;  // term_idx: list index of the stopping fragment
    double T = 1.0, D = 0.0;
    double margin = 1e300;  // min |T(1-a) - t_min| / t_min over tested steps (decision precision)
};

struct Blended {
    int32_t pt;
    Frag fr;
    double T;  // T_k before this fragment
};

template <typename T>
void composite_pixel_t(const Ctx& c, int px, int py, const int32_t* lst, int64_t len,
                       double* F, PixOut& po, std::vector<Blended>* keep) {
    const T tmin = (T)c.opt.t_min;
    T Tdec = (T)1;
    double T64 = 1.0, D = 0.0;
    for (int k = 0; k < c.C; ++k) F[k] = 0.0;
    int32_t ncov = 0, nbl = 0;
    for (int64_t q = 0; q < len; ++q) {
        const int32_t i = lst[q];
        Frag fr;
        if (!fragment<T>(c.sp[i], c.opacity[i], px, py, c.opt, fr)) continue;
        ++ncov;
        if (po.term_idx >= 0) continue;  // only counting coverage past termination
        const T aT = (T)fr.alpha_dec;
        const T nxt = Tdec * ((T)1 - aT);
        const double mg = std::fabs((double)nxt - (double)tmin) / (double)tmin;
        if (mg < po.margin) po.margin = mg;
        if (nxt < tmin) {
            po.term_idx = (int32_t)q;
            continue;
        }
        if (keep) keep->push_back(Blended{i, fr, T64});
        const double w = T64 * fr.alpha;
        for (int k = 0; k < c.C; ++k) F[k] += w * c.feat[(size_t)i * c.C + k];
        D += w * c.sp[i].zc;
        T64 *= (1.0 - fr.alpha);
        Tdec = nxt;
        ++nbl;
    }
    po.n_blend = nbl; po.n_cover = ncov; po.T = T64; po.D = D;
}

void composite_pixel(const Ctx& c, int px, int py, const int32_t* lst, int64_t len, double* F,
                     PixOut& po, std::vector<Blended>* keep) {
    if (c.opt.pin32) composite_pixel_t<float>(c, px, py, lst, len, F, po, keep);
    else composite_pixel_t<double>(c, px, py, lst, len, F, po, keep);
}

// Tile of pixel (px, py) and the position of point i in that tile's list.
struct TileLists {
    int tiles_x = 0, tiles_y = 0;
    std::vector<int64_t> start;    // per tile
    std::vector<int32_t> pts;      // sorted by (zbits, index)
};

void tile_lists(const Ctx& c, const std::vector<char>& want, TileLists& tl) {
    const int Ts = c.opt.tile;
    tl.tiles_x = (c.cam.width + Ts - 1) / Ts;
    tl.tiles_y = (c.cam.height + Ts - 1) / Ts;
    const int64_t P = (int64_t)tl.tiles_x * tl.tiles_y;
    std::vector<int64_t> cnt((size_t)P + 1, 0);
    for (int64_t i = 0; i < c.n; ++i) {
        const Splat& s = c.sp[i];
        if (!s.vis) continue;
        for (int ty = s.by0 / Ts; ty <= s.by1 / Ts; ++ty)
            for (int tx = s.bx0 / Ts; tx <= s.bx1 / Ts; ++tx) {
                const int64_t t = (int64_t)ty * tl.tiles_x + tx;
                if (want[t]) cnt[t + 1]++;
            }
    }
    for (int64_t t = 0; t < P; ++t) cnt[t + 1] += cnt[t];
    tl.start = cnt;
    tl.pts.assign((size_t)cnt[P], 0);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t i = 0; i < c.n; ++i) {
        const Splat& s = c.sp[i];
        if (!s.vis) continue;
        for (int ty = s.by0 / Ts; ty <= s.by1 / Ts; ++ty)
            for (int tx = s.bx0 / Ts; tx <= s.bx1 / Ts; ++tx) {
                const int64_t t = (int64_t)ty * tl.tiles_x + tx;
                if (want[t]) tl.pts[fill[t]++] = (int32_t)i;
            }
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < P; ++t)
        std::stable_sort(tl.pts.begin() + tl.start[t], tl.pts.begin() + tl.start[t + 1],
                         [&](int32_t p, int32_t q) { return c.sp[p].zbits < c.sp[q].zbits; });
}

int64_t position_in_tile(const Ctx& c, const TileLists& tl, int64_t t, int32_t i) {
    const auto b = tl.pts.begin() + tl.start[t], e = tl.pts.begin() + tl.start[t + 1];
    auto it = std::lower_bound(b, e, i, [&](int32_t p, int32_t q) {
        if (c.sp[p].zbits != c.sp[q].zbits) return c.sp[p].zbits < c.sp[q].zbits;
        return p < q;
    });
    return (int64_t)(it - b);
}

void set_threads(const orc_opts_t* o) {
#ifdef _OPENMP
    if (o->n_threads > 0) omp_set_num_threads(o->n_threads);
#else
    (void)o;
#endif
}

Ctx make_ctx(int64_t n, const double* xyz, const double* opacity, const double* scale,
             const double* feat, int32_t C, const orc_camera_t* cam, const orc_opts_t* opt) {
    Ctx c;
    c.n = n; c.xyz = xyz; c.opacity = opacity; c.scale = scale; c.feat = feat; c.C = C;
    c.cam = *cam; c.opt = *opt;
    project_all(c);
    return c;
}

}  // namespace

extern "C" {

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

// Projection and footprint of every point. Outputs (each may be NULL):
// vis[n] (0/1), zbits[n], uvz[n*3], conic[n*3], box[n*4] (x0, x1, y0, y1),
// anchor[n*2] (i0, j0), frac[n*2] (a, b), cov[n*3] (S00, S01, S11).
void orc_project(int64_t n, const double* xyz, const double* scale, const orc_camera_t* cam,
                 const orc_opts_t* opt, int32_t* vis, uint32_t* zbits, double* uvz,
                 double* conic, int32_t* box, int32_t* anchor, double* frac, double* cov) {
    set_threads(opt);
    static const double dummy_feat = 0.0;
    std::vector<double> op((size_t)std::max<int64_t>(n, 1), 1.0);
    Ctx c = make_ctx(n, xyz, op.data(), scale, &dummy_feat, 0, cam, opt);
    for (int64_t i = 0; i < n; ++i) {
        const Splat& s = c.sp[i];
        if (vis) vis[i] = s.vis ? 1 : 0;
        if (zbits) zbits[i] = s.zbits;
        if (uvz) { uvz[3 * i] = s.u; uvz[3 * i + 1] = s.v; uvz[3 * i + 2] = s.zc; }
        if (conic) { conic[3 * i] = s.ca; conic[3 * i + 1] = s.cb; conic[3 * i + 2] = s.cc; }
        if (box) { box[4 * i] = s.bx0; box[4 * i + 1] = s.bx1; box[4 * i + 2] = s.by0; box[4 * i + 3] = s.by1; }
        if (anchor) { anchor[2 * i] = s.i0; anchor[2 * i + 1] = s.j0; }
        if (frac) { frac[2 * i] = s.a; frac[2 * i + 1] = s.b; }
        if (cov) { cov[3 * i] = s.S00; cov[3 * i + 1] = s.S01; cov[3 * i + 2] = s.S11; }
    }
}

// Per-tile copy lists ordered by (tile, depth bits, point index), for the tiles
// with want[t] != 0 (want == NULL: all tiles). Call once with tile_out == NULL
// to get the number of copies; then with buffers of that size.
// Writes tile_out[k] (tile id, row-major) and idx_out[k] (point index).
int64_t orc_tile_lists(int64_t n, const double* xyz, const double* scale, const orc_camera_t* cam,
                       const orc_opts_t* opt, const uint8_t* want, int32_t* tile_out,
                       int32_t* idx_out) {
    set_threads(opt);
    static const double dummy_feat = 0.0;
    std::vector<double> op((size_t)std::max<int64_t>(n, 1), 1.0);
    Ctx c = make_ctx(n, xyz, op.data(), scale, &dummy_feat, 0, cam, opt);
    const int Ts = opt->tile;
    const int64_t P = (int64_t)((cam->width + Ts - 1) / Ts) * ((cam->height + Ts - 1) / Ts);
    std::vector<char> w((size_t)P, 1);
    if (want) for (int64_t t = 0; t < P; ++t) w[t] = want[t] ? 1 : 0;
    TileLists tl;
    tile_lists(c, w, tl);
    const int64_t D = tl.start[P];
    if (tile_out && idx_out) {
        for (int64_t t = 0; t < P; ++t)
            for (int64_t k = tl.start[t]; k < tl.start[t + 1]; ++k) {
                tile_out[k] = (int32_t)t;
                idx_out[k] = tl.pts[k];
            }
    }
    return D;
}

// Forward render of the requested pixels (pix == NULL: every pixel, row-major).
// Outputs per requested pixel k:
//   F[k*C + c], alpha[k] = 1 - T_final, depth[k], t_final[k],
//   n_blend[k] (fragments blended), n_cover[k] (covering fragments),
//   last_pos[k] = 1 + position of the last blended fragment in its tile list
//                 (0 if none),
//   stop_pos[k] = 1 + position of the stopping fragment in the tile list if
//                 the pixel terminated early, else -1,
//   margin[k]   = smallest |T(1-a) - t_min| / t_min over the tested steps.
// Any output pointer may be NULL. Also returns, through needed_out (may be
// NULL), the records the method must read: the sum over tiles touched by the
// requested pixels of (max over in-image pixels of stop_pos if all of them
// stopped, else the tile list length). Only meaningful for full renders.
void orc_render(int64_t n, const double* xyz, const double* opacity, const double* scale,
                const double* feat, int32_t C, const orc_camera_t* cam, const orc_opts_t* opt,
                int64_t n_pix, const int64_t* pix, double* F, double* alpha, double* depth,
                double* t_final, int32_t* n_blend, int32_t* n_cover, int32_t* last_pos,
                int32_t* stop_pos, double* margin, int64_t* needed_out) {
    set_threads(opt);
    Ctx c = make_ctx(n, xyz, opacity, scale, feat, C, cam, opt);
    const int W = cam->width, H = cam->height;
    const int64_t npx = (int64_t)W * H;
    if (!pix) n_pix = npx;
    std::vector<int32_t> slot((size_t)npx, -1);
    for (int64_t k = 0; k < n_pix; ++k) slot[pix ? pix[k] : k] = (int32_t)k;
    std::vector<int64_t> st;
    std::vector<int32_t> pts;
    pixel_lists(c, slot, n_pix, st, pts);
    const int Ts = opt->tile;
    const int txn = (W + Ts - 1) / Ts, tyn = (H + Ts - 1) / Ts;
    std::vector<char> want((size_t)txn * tyn, 0);
    const bool need_tiles = last_pos || stop_pos || needed_out;
    if (need_tiles)
        for (int64_t k = 0; k < n_pix; ++k) {
            const int64_t p = pix ? pix[k] : k;
            want[(size_t)((p / W) / Ts) * txn + (p % W) / Ts] = 1;
        }
    TileLists tl;
    if (need_tiles) tile_lists(c, want, tl);
    std::vector<int64_t> stop_all((size_t)n_pix, -1);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n_pix; ++k) {
        const int64_t p = pix ? pix[k] : k;
        const int px = (int)(p % W), py = (int)(p / W);
        std::vector<double> Fk((size_t)std::max(C, 1));
        PixOut po;
        std::vector<Blended> bl;
        composite_pixel(c, px, py, pts.data() + st[k], st[k + 1] - st[k], Fk.data(), po,
                        need_tiles ? &bl : nullptr);
        if (F) for (int q = 0; q < C; ++q) F[k * C + q] = Fk[q];
        if (alpha) alpha[k] = 1.0 - po.T;
        if (depth) depth[k] = po.D;
        if (t_final) t_final[k] = po.T;
        if (n_blend) n_blend[k] = po.n_blend;
        if (n_cover) n_cover[k] = po.n_cover;
        if (margin) margin[k] = po.margin;
        if (need_tiles) {
            const int64_t t = (int64_t)(py / Ts) * txn + px / Ts;
            int32_t lp = 0;
            if (!bl.empty()) lp = 1 + (int32_t)position_in_tile(c, tl, t, bl.back().pt);
            if (last_pos) last_pos[k] = lp;
            int64_t sp = -1;
            if (po.term_idx >= 0) sp = 1 + position_in_tile(c, tl, t, pts[st[k] + po.term_idx]);
            stop_all[k] = sp;
            if (stop_pos) stop_pos[k] = (int32_t)sp;
        }
    }
    if (needed_out) {
        // Per tile: every in-image pixel that never stopped forces the whole list.
        std::vector<int64_t> need((size_t)txn * tyn, 0);
        std::vector<char> open((size_t)txn * tyn, 0);
        for (int64_t k = 0; k < n_pix; ++k) {
            const int64_t p = pix ? pix[k] : k;
            const int64_t t = (int64_t)((p / W) / Ts) * txn + (p % W) / Ts;
            if (stop_all[k] < 0) open[t] = 1;
            else need[t] = std::max(need[t], stop_all[k]);
        }
        int64_t tot = 0;
        for (int64_t t = 0; t < (int64_t)txn * tyn; ++t) {
            if (!want[t]) continue;
            const int64_t len = tl.start[t + 1] - tl.start[t];
            tot += open[t] ? len : need[t];
        }
        *needed_out = tot;
    }
    (void)H;
}

// Adjoint (appendix, corrected Eq. 2) for the points with pmask[i] != 0
// (pmask == NULL: all points). Upstream gradients: g_F [H*W*C], g_A [H*W],
// g_D [H*W] (g_A, g_D may be NULL). Outputs (FP64, zeroed here; NULL skips):
// d_feat [n*C], d_opacity [n], d_xyz [n*3] and d_scale [n] (Gaussian mode).
//
// Per pixel with blended fragments k = 1..K (T_1 = 1, T_{k+1} = T_k (1 - a_k)):
//   dL/da_k = g_F . (T_k f_k - S_k / (1 - a_k)) + g_D (T_k z_k - SD_k / (1 - a_k))
//             + g_A T_{K+1} / (1 - a_k),
//   S_k = sum_{i>k} a_i T_i f_i, SD_k = sum_{i>k} a_i T_i z_i (suffix sums, no
//   division of T), dL/df_k = T_k a_k g_F, dL/dz_k = T_k a_k g_D.
// The alpha output is 1 - T_{K+1}, which is where a background composited by
// the caller enters; the paper's "+ T_{K+1} f_bg" term is, after the chain
// rule, the -T_{K+1} f_bg / (1 - a_k) carried by g_A.
void orc_backward(int64_t n, const double* xyz, const double* opacity, const double* scale,
                  const double* feat, int32_t C, const orc_camera_t* cam, const orc_opts_t* opt,
                  const uint8_t* pmask, const double* g_F, const double* g_A, const double* g_D,
                  double* d_feat, double* d_opacity, double* d_xyz, double* d_scale) {
    set_threads(opt);
    Ctx c = make_ctx(n, xyz, opacity, scale, feat, C, cam, opt);
    const int W = cam->width;
    const int64_t npx = (int64_t)W * cam->height;
    // Pixels whose lists involve a selected point.
    std::vector<int32_t> slot((size_t)npx, -1);
    int64_t n_slots = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (pmask && !pmask[i]) continue;
        const Splat& s = c.sp[i];
        if (!s.vis) continue;
        for (int py = s.by0; py <= s.by1; ++py)
            for (int px = s.bx0; px <= s.bx1; ++px) {
                const int64_t p = (int64_t)py * W + px;
                if (slot[p] < 0) slot[p] = 0;  // mark
            }
    }
    std::vector<int64_t> pix_of_slot;
    for (int64_t p = 0; p < npx; ++p)
        if (slot[p] == 0 || (!pmask && slot[p] >= 0)) { slot[p] = (int32_t)n_slots++; pix_of_slot.push_back(p); }
    std::vector<int64_t> st;
    std::vector<int32_t> pts;
    pixel_lists(c, slot, n_slots, st, pts);

    // Per-fragment contributions, then a serial per-point sum (fixed order).
    struct Contrib { int32_t pt; double dalpha, T, alpha, g_dot_f_unused; Frag fr; };
    std::vector<std::vector<Contrib>> per_slot((size_t)n_slots);
    std::vector<std::vector<double>> dfeat_slot((size_t)n_slots);
    std::vector<std::vector<double>> dz_slot((size_t)n_slots);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n_slots; ++k) {
        const int64_t p = pix_of_slot[k];
        const int px = (int)(p % W), py = (int)(p / W);
        std::vector<double> Fk((size_t)std::max(C, 1));
        PixOut po;
        std::vector<Blended> bl;
        composite_pixel(c, px, py, pts.data() + st[k], st[k + 1] - st[k], Fk.data(), po, &bl);
        const int64_t K = (int64_t)bl.size();
        const double Tfin = po.T;
        const double* gF = g_F + p * C;
        const double gA = g_A ? g_A[p] : 0.0;
        const double gD = g_D ? g_D[p] : 0.0;
        std::vector<double> S((size_t)std::max(C, 1), 0.0);
        double SD = 0.0;
        auto& out = per_slot[k];
        out.resize((size_t)K);
        auto& dfs = dfeat_slot[k];
        dfs.assign((size_t)K * C, 0.0);
        auto& dzs = dz_slot[k];
        dzs.assign((size_t)K, 0.0);
        for (int64_t q = K - 1; q >= 0; --q) {
            const Blended& b = bl[q];
            const double a = b.fr.alpha, Tk = b.T, om = 1.0 - a;
            const double* f = c.feat + (size_t)b.pt * C;
            double da = 0.0;
            for (int j = 0; j < C; ++j) da += gF[j] * (Tk * f[j] - S[j] / om);
            da += gD * (Tk * c.sp[b.pt].zc - SD / om);
            da += gA * Tfin / om;
            out[q] = Contrib{b.pt, da, Tk, a, 0.0, b.fr};
            for (int j = 0; j < C; ++j) dfs[q * C + j] = Tk * a * gF[j];
            dzs[q] = Tk * a * gD;
            for (int j = 0; j < C; ++j) S[j] += a * Tk * f[j];
            SD += a * Tk * c.sp[b.pt].zc;
        }
    }
    if (d_feat) std::fill(d_feat, d_feat + n * C, 0.0);
    if (d_opacity) std::fill(d_opacity, d_opacity + n, 0.0);
    if (d_xyz) std::fill(d_xyz, d_xyz + 3 * n, 0.0);
    if (d_scale) std::fill(d_scale, d_scale + n, 0.0);
    // Per-point sums of the screen-space gradients.
    std::vector<double> du((size_t)n, 0.0), dv((size_t)n, 0.0), dca((size_t)n, 0.0),
        dcb((size_t)n, 0.0), dcc((size_t)n, 0.0), dz((size_t)n, 0.0);
    for (int64_t k = 0; k < n_slots; ++k) {
        const auto& out = per_slot[k];
        for (size_t q = 0; q < out.size(); ++q) {
            const Contrib& e = out[q];
            const int32_t i = e.pt;
            if (pmask && !pmask[i]) continue;
            if (d_feat) for (int j = 0; j < C; ++j) d_feat[(size_t)i * C + j] += dfeat_slot[k][q * C + j];
            dz[i] += dz_slot[k][q];
            if (!e.fr.unclamped) continue;  // alpha at the clamp: no gradient through o, w
            if (opt->mode == 0) {
                if (d_opacity) d_opacity[i] += e.fr.w_or_g * e.dalpha;  // a = o w
            } else {
                const double G = e.fr.w_or_g, o = opacity[i];
                if (d_opacity) d_opacity[i] += G * e.dalpha;         // a = o G
                const double dm = -0.5 * o * G * e.dalpha;            // G = exp(-m/2)
                const Splat& s = c.sp[i];
                // m = ca dx^2 + 2 cb dx dy + cc dy^2, dx = px + 1/2 - u, dy = py + 1/2 - v
                du[i] += dm * -(2.0 * s.ca * e.fr.dx + 2.0 * s.cb * e.fr.dy);
                dv[i] += dm * -(2.0 * s.cb * e.fr.dx + 2.0 * s.cc * e.fr.dy);
                dca[i] += dm * e.fr.dx * e.fr.dx;
                dcb[i] += dm * 2.0 * e.fr.dx * e.fr.dy;
                dcc[i] += dm * e.fr.dy * e.fr.dy;
            }
        }
    }
    if (opt->mode != 1) return;
    // Chain (u, v, conic, z) -> camera space -> world space, and -> scale.
    const double fx = cam->fx, fy = cam->fy;
    for (int64_t i = 0; i < n; ++i) {
        if (pmask && !pmask[i]) continue;
        const Splat& s = c.sp[i];
        if (!s.vis) continue;
        const double x = s.xc, y = s.yc, z = s.zc, sc = s.s;
        const double S00 = s.S00, S01 = s.S01, S11 = s.S11;
        const double det = S00 * S11 - S01 * S01, det2 = det * det;
        // conic a = S11/det, b = -S01/det, c = S00/det
        const double dS00 = dca[i] * (-S11 * S11 / det2) + dcb[i] * (S01 * S11 / det2) +
                            dcc[i] * (1.0 / det - S00 * S11 / det2);
        const double dS11 = dca[i] * (1.0 / det - S11 * S00 / det2) + dcb[i] * (S01 * S00 / det2) +
                            dcc[i] * (-S00 * S00 / det2);
        const double dS01 = dca[i] * (2.0 * S11 * S01 / det2) +
                            dcb[i] * (-1.0 / det - 2.0 * S01 * S01 / det2) +
                            dcc[i] * (2.0 * S00 * S01 / det2);
        double gx = 0, gy = 0, gz = dz[i], gs = 0;
        // u = fx x / z + cx, v = fy y / z + cy
        gx += du[i] * fx / z;
        gy += dv[i] * fy / z;
        gz += du[i] * (-fx * x / (z * z)) + dv[i] * (-fy * y / (z * z));
        const double z2 = z * z, z3 = z2 * z, z4 = z2 * z2, z5 = z4 * z, s2 = sc * sc;
        if (opt->gauss_cov == 0) {
            // S00 = s^2 (fx^2/z^2 + fx^2 x^2/z^4) + dil, S01 = s^2 fx fy x y / z^4,
            // S11 = s^2 (fy^2/z^2 + fy^2 y^2/z^4) + dil
            gx += dS00 * s2 * fx * fx * 2.0 * x / z4 + dS01 * s2 * fx * fy * y / z4;
            gy += dS11 * s2 * fy * fy * 2.0 * y / z4 + dS01 * s2 * fx * fy * x / z4;
            gz += dS00 * s2 * (-2.0 * fx * fx / z3 - 4.0 * fx * fx * x * x / z5) +
                  dS11 * s2 * (-2.0 * fy * fy / z3 - 4.0 * fy * fy * y * y / z5) +
                  dS01 * s2 * (-4.0 * fx * fy * x * y / z5);
            gs += dS00 * 2.0 * sc * (fx * fx / z2 + fx * fx * x * x / z4) +
                  dS11 * 2.0 * sc * (fy * fy / z2 + fy * fy * y * y / z4) +
                  dS01 * 2.0 * sc * (fx * fy * x * y / z4);
        } else {
            // S00 = S11 = s^2 fx fy / z^2 + dil, S01 = 0
            const double dS = dS00 + dS11;
            gz += dS * s2 * fx * fy * (-2.0 / z3);
            gs += dS * 2.0 * sc * fx * fy / z2;
        }
        if (d_xyz) {
            const float* R = cam->R;  // d world = R^T d camera
            d_xyz[3 * i + 0] = R[0] * gx + R[3] * gy + R[6] * gz;
            d_xyz[3 * i + 1] = R[1] * gx + R[4] * gy + R[7] * gz;
            d_xyz[3 * i + 2] = R[2] * gx + R[5] * gy + R[8] * gz;
        }
        if (d_scale && scale) d_scale[i] = gs;
    }
}

}  // extern "C"

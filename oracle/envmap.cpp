// CPU ORACLE for the distilled background model and the spherical
// contraction -- TEST INFRASTRUCTURE ONLY.
//
// Nothing in the product path may link, load or call this file (only the
// tests, the package's smoke check and the benchmark's CPU baseline leg). It
// shares no code with the CUDA path.
//
// What it computes (Sec. 3.2, "Faster Background Model Evaluation"): the
// background of every pixel is read from a spherical environment map, an
// H_b x W_b x C image, by bilinear interpolation along the pixel's viewing
// direction, and composited behind the blended points with the transmittance
// left after the last fragment (the T_{K+1} f_bg term of Eq. 2):
//   out = F + (1 - alpha) f_bg(d),  alpha = the blend's alpha output.
// Readings (the paper gives the map's size and the bilinear lookup, nothing
// else):
//   - viewing direction of pixel (x, y): d_c = ((x + 1/2 - c_x) / f_x,
//     (y + 1/2 - c_y) / f_y, 1), normalised, rotated to world space with R^T
//     (x_c = R x_w + t);
//   - equirectangular map: longitude lambda = atan2(d_x, d_z) in (-pi, pi],
//     polar angle theta = acos(d_y) in [0, pi]; texel centres at integer + 1/2:
//     X = (lambda / (2 pi) + 1/2) W_b - 1/2, Y = (theta / pi) H_b - 1/2;
//   - bilinear weights of the four texels around (X, Y); columns wrap around
//     (longitude is periodic), rows clamp to [0, H_b - 1] at the poles.
// Backward, for an upstream gradient g of `out`: dL/dF = g, dL/dalpha = -g . f_bg,
// dL/dmap[texel] = sum over pixels of w_texel (1 - alpha) g.
// All arithmetic is FP64, one pixel at a time.
#include <cmath>
#include <cstdint>
#include <cstring>

extern "C" {

typedef struct {
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float near_z, far_z;
    int32_t width, height;
} orc_env_camera_t;

}  // extern "C"

namespace {

struct Tap {
    int64_t idx[4];  // texel offsets (row * W_b + col)
    double w[4];
};

// Direction of pixel (x, y) in world space, then its four texels and weights.
Tap lookup(const orc_env_camera_t& c, const double* dir_cam, int x, int y, int Hb, int Wb) {
    double dc[3];
    if (dir_cam) {
        dc[0] = dir_cam[0];
        dc[1] = dir_cam[1];
        dc[2] = dir_cam[2];
    } else {
        dc[0] = (x + 0.5 - (double)c.cx) / (double)c.fx;
        dc[1] = (y + 0.5 - (double)c.cy) / (double)c.fy;
        dc[2] = 1.0;
    }
    const double len = std::sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]);
    for (double& v : dc) v /= len;
    double dw[3];
    for (int i = 0; i < 3; ++i)  // R^T d_c
        dw[i] = (double)c.R[0 * 3 + i] * dc[0] + (double)c.R[1 * 3 + i] * dc[1] + (double)c.R[2 * 3 + i] * dc[2];
    const double pi = 3.14159265358979323846;
    const double lam = std::atan2(dw[0], dw[2]);
    const double th = std::acos(std::fmax(-1.0, std::fmin(1.0, dw[1])));
    const double X = (lam / (2.0 * pi) + 0.5) * Wb - 0.5;
    const double Y = th / pi * Hb - 0.5;
    const double fx0 = std::floor(X), fy0 = std::floor(Y);
    const double a = X - fx0, b = Y - fy0;
    const int64_t x0 = (int64_t)fx0, y0 = (int64_t)fy0;
    auto wrap = [Wb](int64_t v) { v %= Wb; return v < 0 ? v + Wb : v; };
    auto clampr = [Hb](int64_t v) { return v < 0 ? 0 : (v > Hb - 1 ? Hb - 1 : v); };
    const int64_t c0 = wrap(x0), c1 = wrap(x0 + 1), r0 = clampr(y0), r1 = clampr(y0 + 1);
    Tap t;
    t.idx[0] = r0 * Wb + c0; t.w[0] = (1 - a) * (1 - b);
    t.idx[1] = r0 * Wb + c1; t.w[1] = a * (1 - b);
    t.idx[2] = r1 * Wb + c0; t.w[2] = (1 - a) * b;
    t.idx[3] = r1 * Wb + c1; t.w[3] = a * b;
    return t;
}

}  // namespace

extern "C" {

// Per-pixel camera-space unit viewing directions (H x W x 3).
void orc_env_dirs(const orc_env_camera_t* cam, double* dirs) {
    const int W = cam->width, H = cam->height;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double d[3] = {(x + 0.5 - (double)cam->cx) / (double)cam->fx,
                           (y + 0.5 - (double)cam->cy) / (double)cam->fy, 1.0};
            const double len = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double* o = dirs + ((int64_t)y * W + x) * 3;
            for (int i = 0; i < 3; ++i) o[i] = d[i] / len;
        }
}

// out = F + (1 - alpha) f_bg; also returns f_bg itself (H x W x C).
void orc_env_composite(const orc_env_camera_t* cam, const double* map, int32_t Hb, int32_t Wb, int32_t C,
                       const double* dirs, const double* F, const double* alpha, double* out, double* bg) {
    const int W = cam->width, H = cam->height;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const int64_t p = (int64_t)y * W + x;
            const Tap t = lookup(*cam, dirs ? dirs + p * 3 : nullptr, x, y, Hb, Wb);
            for (int c = 0; c < C; ++c) {
                double v = 0.0;
                for (int k = 0; k < 4; ++k) v += t.w[k] * map[t.idx[k] * C + c];
                if (bg) bg[p * C + c] = v;
                if (out) out[p * C + c] = F[p * C + c] + (1.0 - alpha[p]) * v;
            }
        }
}

// dL/dalpha (-g . f_bg, per pixel) and dL/dmap (H_b x W_b x C, overwritten).
void orc_env_backward(const orc_env_camera_t* cam, const double* map, int32_t Hb, int32_t Wb, int32_t C,
                      const double* dirs, const double* alpha, const double* g, double* d_alpha,
                      double* d_map) {
    const int W = cam->width, H = cam->height;
    std::memset(d_map, 0, sizeof(double) * (size_t)Hb * Wb * C);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const int64_t p = (int64_t)y * W + x;
            const Tap t = lookup(*cam, dirs ? dirs + p * 3 : nullptr, x, y, Hb, Wb);
            double da = 0.0;
            for (int c = 0; c < C; ++c) {
                double v = 0.0;
                for (int k = 0; k < 4; ++k) v += t.w[k] * map[t.idx[k] * C + c];
                da -= g[p * C + c] * v;
                for (int k = 0; k < 4; ++k) d_map[t.idx[k] * C + c] += t.w[k] * (1.0 - alpha[p]) * g[p * C + c];
            }
            d_alpha[p] = da;
        }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Spherical contraction of sampled positions (Sec. 3.4 "Implementation
// Improvements": applied to the points before they enter the appearance field;
// the contraction of Mip-NeRF 360): x if |x| <= 1, else (2 - 1/|x|) x / |x|.
// FP64, one point at a time.
extern "C" void orc_contract(int64_t n, const double* x, double* out) {
    for (int64_t i = 0; i < n; ++i) {
        const double a = x[3 * i], b = x[3 * i + 1], c = x[3 * i + 2];
        const double r = std::sqrt(a * a + b * b + c * c);
        const double s = r <= 1.0 ? 1.0 : (2.0 - 1.0 / r) / r;
        out[3 * i] = s * a;
        out[3 * i + 1] = s * b;
        out[3 * i + 2] = s * c;
    }
}

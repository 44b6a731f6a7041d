// FP64 CPU oracle for the tile-based Gaussian splatting hot path (projection,
// duplication + sort, alpha blending, blend gradients).
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow definition the CUDA
// library is checked against.  It shares no code, header or constant with the
// CUDA path, and only the test suite, the smoke check and the CPU-baseline leg
// of the benchmark may load it.  Every routine follows the paper's
// definitions directly (cited per function) and evaluates the splat exponent
// as the plain quadratic of Eq. 3, never via the dot-product form of Eq. 6
// (that identity has a routine of its own, oracle_power_eq6, used to pin it).
//
// Readings of passages the paper leaves open:
//  * conic: Sigma^-1 = [[A, B], [B, C]] is the inverse 2D covariance (Alg. 1);
//  * pixel (px, py) is evaluated at its centre (px + 0.5, py + 0.5);
//  * alpha = min(0.99, o * exp(min(power, 0))); a splat is skipped when
//    alpha < 1/255; compositing stops, without adding the splat, at the first
//    one whose test transmittance T * (1 - alpha) falls below 1e-4 (Eq. 1 with
//    the alpha-skip and early-termination rules of Alg. 1);
//  * n_contrib = 1 + list position of the last splat added, 0 if none;
//  * tile membership: the 3-sigma square of radius r = ceil(3 sqrt(lambda_max))
//    around the projected mean; tiles [floor((m - r)/16), floor((m + r)/16)]
//    per axis, clamped to the image (Sec. 2.1 "intersection detection");
//  * the 2D covariance gets +lowpass (0.3) on its diagonal before inversion;
//  * colour from real spherical harmonics up to degree 3, view direction from
//    the camera centre to the mean, rgb = max(0, sum + 0.5).
// Parity status per function: every exported routine is pinned by the CPU
// tests (closed forms, invariants, brute force, library special cases);
// oracle_blend_grad is pinned by central finite differences of oracle_blend.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

constexpr int kTile = 16;

// Camera layout shared with the Python wrapper: 22 doubles
// [W, H, fx, fy, cx, cy, R00..R22 (row-major), t0, t1, t2, znear, lowpass, pad]
struct Cam {
    int W, H;
    double fx, fy, cx, cy;
    double R[3][3];
    double t[3];
    double znear, lowpass;
};

Cam read_cam(const double* c) {
    Cam k;
    k.W = (int)c[0];
    k.H = (int)c[1];
    k.fx = c[2]; k.fy = c[3]; k.cx = c[4]; k.cy = c[5];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) k.R[i][j] = c[6 + 3 * i + j];
    k.t[0] = c[15]; k.t[1] = c[16]; k.t[2] = c[17];
    k.znear = c[18];
    k.lowpass = c[19];
    return k;
}

int tiles_x(int W) { return (W + kTile - 1) / kTile; }
int tiles_y(int H) { return (H + kTile - 1) / kTile; }

// Tile rectangle of a splat: tiles whose [16t, 16t+16) span meets
// [m - r, m + r] on each axis, clamped to the grid.  Returns false if empty.
bool tile_rect(double mx, double my, int r, int W, int H, int rect[4]) {
    if (r <= 0) return false;
    long x0 = (long)std::floor((mx - r) / kTile);
    long x1 = (long)std::floor((mx + r) / kTile);
    long y0 = (long)std::floor((my - r) / kTile);
    long y1 = (long)std::floor((my + r) / kTile);
    x0 = std::max(x0, 0L); y0 = std::max(y0, 0L);
    x1 = std::min(x1, (long)tiles_x(W) - 1);
    y1 = std::min(y1, (long)tiles_y(H) - 1);
    if (x0 > x1 || y0 > y1) return false;
    rect[0] = (int)x0; rect[1] = (int)x1; rect[2] = (int)y0; rect[3] = (int)y1;
    return true;
}

// Real spherical harmonics up to degree 3 at unit direction (x, y, z); the
// normalisations are written as closed forms.  Order within degree l is
// m = -l..l, and the basis is sqrt(2) Re/Im of the complex harmonics with
// the Condon-Shortley phase (the convention 3DGS uses).
void sh_basis(double x, double y, double z, double out[16]) {
    const double pi = 3.14159265358979323846;
    const double n0 = 0.5 / std::sqrt(pi);
    const double n1 = std::sqrt(3.0 / (4.0 * pi));
    const double n2a = 0.5 * std::sqrt(15.0 / pi);
    const double n2b = 0.25 * std::sqrt(5.0 / pi);
    const double n2c = 0.25 * std::sqrt(15.0 / pi);
    const double n3a = 0.25 * std::sqrt(35.0 / (2.0 * pi));
    const double n3b = 0.5 * std::sqrt(105.0 / pi);
    const double n3c = 0.25 * std::sqrt(21.0 / (2.0 * pi));
    const double n3d = 0.25 * std::sqrt(7.0 / pi);
    const double n3e = 0.25 * std::sqrt(105.0 / pi);
    out[0] = n0;
    out[1] = -n1 * y;
    out[2] = n1 * z;
    out[3] = -n1 * x;
    out[4] = n2a * x * y;
    out[5] = -n2a * y * z;
    out[6] = n2b * (2 * z * z - x * x - y * y);
    out[7] = -n2a * x * z;
    out[8] = n2c * (x * x - y * y);
    out[9] = -n3a * y * (3 * x * x - y * y);
    out[10] = n3b * x * y * z;
    out[11] = -n3c * y * (4 * z * z - x * x - y * y);
    out[12] = n3d * z * (2 * z * z - 3 * x * x - 3 * y * y);
    out[13] = -n3c * x * (4 * z * z - x * x - y * y);
    out[14] = n3e * z * (x * x - y * y);
    out[15] = -n3a * x * (x * x - 3 * y * y);
}

// Partial derivatives of the real SH basis of sh_basis with respect to the
// (unconstrained) coordinates x, y, z of its argument: grad[k] = dY_k/d(x,y,z).
void sh_basis_grad(double x, double y, double z, double grad[16][3]) {
    const double pi = 3.14159265358979323846;
    const double n1 = std::sqrt(3.0 / (4.0 * pi));
    const double n2a = 0.5 * std::sqrt(15.0 / pi);
    const double n2b = 0.25 * std::sqrt(5.0 / pi);
    const double n2c = 0.25 * std::sqrt(15.0 / pi);
    const double n3a = 0.25 * std::sqrt(35.0 / (2.0 * pi));
    const double n3b = 0.5 * std::sqrt(105.0 / pi);
    const double n3c = 0.25 * std::sqrt(21.0 / (2.0 * pi));
    const double n3d = 0.25 * std::sqrt(7.0 / pi);
    const double n3e = 0.25 * std::sqrt(105.0 / pi);
    const double g[16][3] = {
        {0, 0, 0},
        {0, -n1, 0},
        {0, 0, n1},
        {-n1, 0, 0},
        {n2a * y, n2a * x, 0},
        {0, -n2a * z, -n2a * y},
        {-2 * n2b * x, -2 * n2b * y, 4 * n2b * z},
        {-n2a * z, 0, -n2a * x},
        {2 * n2c * x, -2 * n2c * y, 0},
        {-6 * n3a * x * y, -n3a * (3 * x * x - 3 * y * y), 0},
        {n3b * y * z, n3b * x * z, n3b * x * y},
        {2 * n3c * x * y, -n3c * (4 * z * z - x * x - 3 * y * y), -8 * n3c * y * z},
        {-6 * n3d * x * z, -6 * n3d * y * z, n3d * (6 * z * z - 3 * x * x - 3 * y * y)},
        {-n3c * (4 * z * z - 3 * x * x - y * y), 2 * n3c * x * y, -8 * n3c * x * z},
        {2 * n3e * x * z, -2 * n3e * y * z, n3e * (x * x - y * y)},
        {-n3a * (3 * x * x - 3 * y * y), 6 * n3a * x * y, 0}};
    for (int k = 0; k < 16; ++k)
        for (int j = 0; j < 3; ++j) grad[k][j] = g[k][j];
}

struct Splat {
    double mx, my, A, B, C, o, c[3];
};

// Exponent of Eq. 3 for the splat at pixel centre (xp, yp):
// power = -1/2 A dx^2 - B dx dy - 1/2 C dy^2, dx = x_g - x_p, dy = y_g - y_p.
inline double power_eq3(const Splat& s, double xp, double yp) {
    double dx = s.mx - xp, dy = s.my - yp;
    return -0.5 * s.A * dx * dx - s.B * dx * dy - 0.5 * s.C * dy * dy;
}

struct PixelResult {
    double C[3];
    double T;
    int n_contrib;
    bool ambiguous;
    double err_bound;
};

// Rounding model of a lower-precision blend, for deciding which pixels are
// ambiguous (reading 12).  alpha: relative error of every alpha (= absolute
// error of the exponent) from the exponential and constants; t: relative error
// of the transmittance product from its own roundings; sum: error of the
// exponent per unit of the magnitude sum of Eq. 3's three terms (evaluating a
// sum in floating point errs by at most a small multiple of the unit roundoff
// times the sum of the terms' magnitudes, which is large against the exponent
// itself for a nearly singular conic far from the splat's centre); slack:
// offsets enlarged by this many pixels for that sum (a path that evaluates the
// exponent relative to a reference pixel within `slack` of the pixel).
struct Margins {
    double alpha, t, sum, slack;
};

// Magnitude sum of Eq. 3's terms, 1/2 |A| ax^2 + |B| ax ay + 1/2 |C| ay^2, with
// ax = |dx| + slack, ay = |dy| + slack.
inline double power_terms_magnitude(const Splat& s, double xp, double yp, double slack) {
    const double ax = std::fabs(s.mx - xp) + slack, ay = std::fabs(s.my - yp) + slack;
    return 0.5 * std::fabs(s.A) * ax * ax + std::fabs(s.B) * ax * ay + 0.5 * std::fabs(s.C) * ay * ay;
}

// Front-to-back compositing of one pixel over an ordered splat list (Eq. 1 with
// Alg. 1's alpha-skip and early termination, readings in the header).
// Decisions that lie within rounding of their threshold mark the pixel
// ambiguous: a lower-precision path may legitimately decide otherwise.  Each
// alpha carries a relative error up to eps = m.alpha + m.sum * (magnitude sum),
// and alpha decisions use that margin; the test transmittance
// T (1 - alpha) = prod (1 - alpha_k) carries a relative error up to
// m.t + sum_k eps_k alpha_k / (1 - alpha_k) (first order, Eq. 1), so its
// decision uses that bound.  err_bound: the first-order bound those errors put
// on the pixel's colour (each weight alpha_i T_i off by at most its alpha's
// and its T's relative errors), largest channel.
PixelResult composite_pixel(const std::vector<Splat>& list, double xp, double yp,
                            const double bg[3], const Margins& m) {
    PixelResult r{{0, 0, 0}, 1.0, 0, false, 0.0};
    double T = 1.0;
    double growth = 0.0;  // sum eps_k alpha_k / (1 - alpha_k) over the splats added so far
    for (size_t i = 0; i < list.size(); ++i) {
        const Splat& s = list[i];
        double power = std::min(power_eq3(s, xp, yp), 0.0);
        const double eps = m.alpha + (m.sum > 0 ? m.sum * power_terms_magnitude(s, xp, yp, m.slack) : 0.0);
        double raw = s.o * std::exp(power);
        if (std::fabs(raw - 0.99) <= eps * 0.99) r.ambiguous = true;
        double alpha = std::min(0.99, raw);
        if (std::fabs(alpha - 1.0 / 255.0) <= eps / 255.0) r.ambiguous = true;
        if (alpha < 1.0 / 255.0) continue;
        double testT = T * (1.0 - alpha);
        double tm = m.t + growth + eps * alpha / (1.0 - alpha);
        if (std::fabs(testT - 1e-4) <= tm * 1e-4) r.ambiguous = true;
        if (testT < 1e-4) break;
        const double cmax = std::max({std::fabs(s.c[0]), std::fabs(s.c[1]), std::fabs(s.c[2])});
        r.err_bound += cmax * alpha * T * (eps + growth + m.t);
        growth += eps * alpha / (1.0 - alpha);
        for (int ch = 0; ch < 3; ++ch) r.C[ch] += s.c[ch] * alpha * T;
        T = testT;
        r.n_contrib = (int)i + 1;
    }
    for (int ch = 0; ch < 3; ++ch) r.C[ch] += T * bg[ch];
    r.err_bound += T * std::max({std::fabs(bg[0]), std::fabs(bg[1]), std::fabs(bg[2])}) * (growth + m.t);
    r.T = T;
    return r;
}

Splat load_splat(uint32_t g, const double* mean2d, const double* conic,
                 const double* opac, const double* rgb) {
    Splat s;
    s.mx = mean2d[2 * (size_t)g];
    s.my = mean2d[2 * (size_t)g + 1];
    s.A = conic[3 * (size_t)g];
    s.B = conic[3 * (size_t)g + 1];
    s.C = conic[3 * (size_t)g + 2];
    s.o = opac[g];
    for (int ch = 0; ch < 3; ++ch) s.c[ch] = rgb[3 * (size_t)g + ch];
    return s;
}

template <class F>
void parallel_for(int n, int n_threads, F f) {
    if (n_threads <= 1 || n < 2) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    std::vector<std::thread> pool;
    for (int k = 0; k < n_threads; ++k)
        pool.emplace_back([=, &f]() {
            for (int i = k; i < n; i += n_threads) f(i);
        });
    for (auto& th : pool) th.join();
}

}  // namespace

extern "C" {

int oracle_abi_version() { return 1; }

// Preprocessing of Sec. 2.1 (stage 1): EWA projection of each 3D Gaussian.
// Outputs per Gaussian g: mean2d (2), cov2d (3: a, b, c with lowpass added),
// conic (3: A, B, C), depth, radius (0 = culled), rgb (3), rect (4: x0, x1, y0,
// y1 tiles inclusive, -1 if none) and tiles_touched.
void oracle_project(int n, const float* means, const float* scales, const float* quats,
                    const float* sh, int sh_degree, const double* cam_in,
                    double* mean2d, double* cov2d, double* conic, double* depth,
                    int32_t* radius, double* rgb, int32_t* rect, int64_t* tiles_touched) {
    const Cam cam = read_cam(cam_in);
    const int K = (sh_degree + 1) * (sh_degree + 1);
    // camera centre in world space: -R^T t
    double cpos[3];
    for (int j = 0; j < 3; ++j)
        cpos[j] = -(cam.R[0][j] * cam.t[0] + cam.R[1][j] * cam.t[1] + cam.R[2][j] * cam.t[2]);
    for (int g = 0; g < n; ++g) {
        radius[g] = 0;
        tiles_touched[g] = 0;
        for (int k = 0; k < 4; ++k) rect[4 * g + k] = -1;
        for (int k = 0; k < 2; ++k) mean2d[2 * g + k] = 0;
        for (int k = 0; k < 3; ++k) { cov2d[3 * g + k] = 0; conic[3 * g + k] = 0; rgb[3 * g + k] = 0; }
        depth[g] = 0;

        double mw[3] = {means[3 * g], means[3 * g + 1], means[3 * g + 2]};
        double p[3];
        for (int i = 0; i < 3; ++i)
            p[i] = cam.R[i][0] * mw[0] + cam.R[i][1] * mw[1] + cam.R[i][2] * mw[2] + cam.t[i];
        depth[g] = p[2];
        if (!(p[2] > cam.znear)) continue;

        // rotation of the unit quaternion (w, x, y, z)
        double qw = quats[4 * g], qx = quats[4 * g + 1], qy = quats[4 * g + 2], qz = quats[4 * g + 3];
        double qn = std::sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
        if (!(qn > 0)) continue;
        qw /= qn; qx /= qn; qy /= qn; qz /= qn;
        double Rq[3][3] = {
            {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
            {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
            {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
        double s[3] = {scales[3 * g], scales[3 * g + 1], scales[3 * g + 2]};
        // Sigma3 = (Rq S)(Rq S)^T
        double M[3][3], S3[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[i][j] = Rq[i][j] * s[j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += M[i][k] * M[j][k];
                S3[i][j] = acc;
            }
        // Jacobian of the perspective projection at p, times the camera rotation
        double J[2][3] = {{cam.fx / p[2], 0, -cam.fx * p[0] / (p[2] * p[2])},
                          {0, cam.fy / p[2], -cam.fy * p[1] / (p[2] * p[2])}};
        double Tm[2][3];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j)
                Tm[i][j] = J[i][0] * cam.R[0][j] + J[i][1] * cam.R[1][j] + J[i][2] * cam.R[2][j];
        double S2[2][2];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) acc += Tm[i][k] * S3[k][l] * Tm[j][l];
                S2[i][j] = acc;
            }
        double a = S2[0][0] + cam.lowpass, b = S2[0][1], c = S2[1][1] + cam.lowpass;
        cov2d[3 * g] = a; cov2d[3 * g + 1] = b; cov2d[3 * g + 2] = c;
        double det = a * c - b * b;
        if (!(det > 0)) continue;
        double mx = cam.fx * p[0] / p[2] + cam.cx;
        double my = cam.fy * p[1] / p[2] + cam.cy;
        if (!(std::fabs(mx) <= 8388608.0 && std::fabs(my) <= 8388608.0)) continue;  // 2^23
        double mid = 0.5 * (a + c);
        double lmax = mid + std::sqrt(std::max(0.0, 0.25 * (a - c) * (a - c) + b * b));
        double rr = std::ceil(3.0 * std::sqrt(lmax));
        int r = (int)std::min(rr, 16777216.0);  // 2^24
        conic[3 * g] = c / det;
        conic[3 * g + 1] = -b / det;
        conic[3 * g + 2] = a / det;
        mean2d[2 * g] = mx;
        mean2d[2 * g + 1] = my;
        int rc[4];
        if (!tile_rect(mx, my, r, cam.W, cam.H, rc)) continue;
        radius[g] = r;
        for (int k = 0; k < 4; ++k) rect[4 * g + k] = rc[k];
        tiles_touched[g] = (int64_t)(rc[1] - rc[0] + 1) * (rc[3] - rc[2] + 1);
        // colour from SH, direction camera centre -> mean
        double d[3] = {mw[0] - cpos[0], mw[1] - cpos[1], mw[2] - cpos[2]};
        double dn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double Y[16];
        sh_basis(d[0] / dn, d[1] / dn, d[2] / dn, Y);
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0;
            for (int k = 0; k < K; ++k) acc += (double)sh[((size_t)g * K + k) * 3 + ch] * Y[k];
            rgb[3 * g + ch] = std::max(0.0, acc + 0.5);
        }
    }
}

// The real SH basis alone, for pinning against a library evaluation.
void oracle_sh_basis(int n, const double* dirs, double* out) {
    for (int i = 0; i < n; ++i) sh_basis(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], out + 16 * i);
}

// Gradient of the preprocessing stage (Sec. 2.1 (a), the projection of
// oracle_project; the paper has no backward pass).  Given dL/dmean2d (n x 2),
// dL/dconic (n x 3, the entries A, B, C of [[A, B], [B, C]]) and dL/drgb
// (n x 3) of one camera, writes dL/dmeans (n x 3), dL/dscales (n x 3),
// dL/dquats (n x 4) and dL/dsh (n x K x 3).  A Gaussian with radius[g] == 0
// (culled by the forward pass) gets zeros.  The chain rule in matrix form:
//   conic = Sigma2^-1 of [[a, b], [b, c]] -> G = dL/dSigma2 (symmetric);
//   Sigma2 = T Sigma3 T^T, T = J R:  dSigma3 = T^T G T,  dT = 2 G T Sigma3,
//   dJ = dT R^T;  J and mean2d are functions of p = R mean + t;
//   Sigma3 = M M^T, M = Rq(q / |q|) diag(s):  dM = 2 dSigma3 M;
//   rgb = max(0, sum_k sh_k Y_k(u) + 0.5), u = d / |d|, d = mean - centre:
//   dsh_k = Y_k drgb (where not clamped), du = sum_k grad Y_k (sh_k . drgb),
//   dd = (I - u u^T) du / |d|.
void oracle_project_backward(int n, const float* means, const float* scales, const float* quats,
                             const float* sh, int sh_degree, const double* cam_in, const int32_t* radius,
                             const double* dmean2d, const double* dconic, const double* drgb,
                             double* dmeans, double* dscales, double* dquats, double* dsh) {
    const Cam cam = read_cam(cam_in);
    const int K = (sh_degree + 1) * (sh_degree + 1);
    double cpos[3];
    for (int j = 0; j < 3; ++j)
        cpos[j] = -(cam.R[0][j] * cam.t[0] + cam.R[1][j] * cam.t[1] + cam.R[2][j] * cam.t[2]);
    for (int g = 0; g < n; ++g) {
        for (int j = 0; j < 3; ++j) { dmeans[3 * g + j] = 0; dscales[3 * g + j] = 0; }
        for (int j = 0; j < 4; ++j) dquats[4 * g + j] = 0;
        for (int j = 0; j < 3 * K; ++j) dsh[(size_t)g * 3 * K + j] = 0;
        if (radius[g] <= 0) continue;

        // forward quantities
        const double mw[3] = {means[3 * g], means[3 * g + 1], means[3 * g + 2]};
        double p[3];
        for (int i = 0; i < 3; ++i)
            p[i] = cam.R[i][0] * mw[0] + cam.R[i][1] * mw[1] + cam.R[i][2] * mw[2] + cam.t[i];
        const double q[4] = {quats[4 * g], quats[4 * g + 1], quats[4 * g + 2], quats[4 * g + 3]};
        const double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        const double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
        const double Rq[3][3] = {
            {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
            {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
            {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
        const double s[3] = {scales[3 * g], scales[3 * g + 1], scales[3 * g + 2]};
        double M[3][3], S3[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[i][j] = Rq[i][j] * s[j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                S3[i][j] = 0;
                for (int k = 0; k < 3; ++k) S3[i][j] += M[i][k] * M[j][k];
            }
        const double iz = 1.0 / p[2];
        const double J[2][3] = {{cam.fx * iz, 0, -cam.fx * p[0] * iz * iz}, {0, cam.fy * iz, -cam.fy * p[1] * iz * iz}};
        double T[2][3];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j)
                T[i][j] = J[i][0] * cam.R[0][j] + J[i][1] * cam.R[1][j] + J[i][2] * cam.R[2][j];
        double S2[2][2];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                S2[i][j] = 0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) S2[i][j] += T[i][k] * S3[k][l] * T[j][l];
            }
        const double a = S2[0][0] + cam.lowpass, b = S2[0][1], c = S2[1][1] + cam.lowpass;
        const double det = a * c - b * b;

        // conic (A, B, C) = (c, -b, a) / det  ->  (da, db, dc), then G = [[da, db/2], [db/2, dc]]
        const double dA = dconic[3 * g], dB = dconic[3 * g + 1], dC = dconic[3 * g + 2];
        const double d2 = det * det;
        const double da = (-c * c * dA + b * c * dB - b * b * dC) / d2;
        const double db = (2 * b * c * dA - (a * c + b * b) * dB + 2 * a * b * dC) / d2;
        const double dc = (-b * b * dA + a * b * dB - a * a * dC) / d2;
        const double G[2][2] = {{da, 0.5 * db}, {0.5 * db, dc}};

        // dSigma3 = T^T G T;  dT = 2 G T Sigma3;  dJ = dT R^T
        double dS3[3][3], GT[2][3], dT[2][3], dJ[2][3];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j) GT[i][j] = G[i][0] * T[0][j] + G[i][1] * T[1][j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) dS3[i][j] = T[0][i] * GT[0][j] + T[1][i] * GT[1][j];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j) {
                dT[i][j] = 0;
                for (int k = 0; k < 3; ++k) dT[i][j] += 2 * GT[i][k] * S3[k][j];
            }
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j) dJ[i][j] = dT[i][0] * cam.R[j][0] + dT[i][1] * cam.R[j][1] + dT[i][2] * cam.R[j][2];

        // p from J and from mean2d = (fx x / z + cx, fy y / z + cy)
        const double dmx = dmean2d[2 * g], dmy = dmean2d[2 * g + 1];
        double dp[3];
        dp[0] = dJ[0][2] * (-cam.fx * iz * iz) + dmx * cam.fx * iz;
        dp[1] = dJ[1][2] * (-cam.fy * iz * iz) + dmy * cam.fy * iz;
        dp[2] = dJ[0][0] * (-cam.fx * iz * iz) + dJ[1][1] * (-cam.fy * iz * iz) +
                dJ[0][2] * (2 * cam.fx * p[0] * iz * iz * iz) + dJ[1][2] * (2 * cam.fy * p[1] * iz * iz * iz) -
                dmx * cam.fx * p[0] * iz * iz - dmy * cam.fy * p[1] * iz * iz;
        for (int j = 0; j < 3; ++j)
            dmeans[3 * g + j] = cam.R[0][j] * dp[0] + cam.R[1][j] * dp[1] + cam.R[2][j] * dp[2];

        // Sigma3 = M M^T:  dM = 2 dSigma3 M;  M = Rq diag(s)
        double dM[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                dM[i][j] = 0;
                for (int k = 0; k < 3; ++k) dM[i][j] += 2 * dS3[i][k] * M[k][j];
            }
        double dR[3][3];
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int i = 0; i < 3; ++i) {
                acc += dM[i][j] * Rq[i][j];
                dR[i][j] = dM[i][j] * s[j];
            }
            dscales[3 * g + j] = acc;
        }
        // the rotation matrix's entries as polynomials of the unit quaternion (w, x, y, z)
        double dqh[4];
        dqh[0] = 2 * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
        dqh[1] = 2 * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2 * x * dR[1][1] - w * dR[1][2] + z * dR[2][0] +
                      w * dR[2][1] - 2 * x * dR[2][2]);
        dqh[2] = 2 * (-2 * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] - w * dR[2][0] +
                      z * dR[2][1] - 2 * y * dR[2][2]);
        dqh[3] = 2 * (-2 * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2 * z * dR[1][1] +
                      y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
        // q / |q|:  dq = (I - qh qh^T) dqh / |q|
        const double qh[4] = {w, x, y, z};
        const double proj = qh[0] * dqh[0] + qh[1] * dqh[1] + qh[2] * dqh[2] + qh[3] * dqh[3];
        for (int j = 0; j < 4; ++j) dquats[4 * g + j] = (dqh[j] - qh[j] * proj) / qn;

        // colour
        const double d[3] = {mw[0] - cpos[0], mw[1] - cpos[1], mw[2] - cpos[2]};
        const double dn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const double u[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
        double Y[16], dY[16][3];
        sh_basis(u[0], u[1], u[2], Y);
        sh_basis_grad(u[0], u[1], u[2], dY);
        double dacc[3];
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0;
            for (int k = 0; k < K; ++k) acc += (double)sh[((size_t)g * K + k) * 3 + ch] * Y[k];
            dacc[ch] = acc + 0.5 > 0 ? drgb[3 * g + ch] : 0.0;
        }
        double du[3] = {0, 0, 0};
        for (int k = 0; k < K; ++k) {
            double w_k = 0;
            for (int ch = 0; ch < 3; ++ch) {
                dsh[((size_t)g * K + k) * 3 + ch] = Y[k] * dacc[ch];
                w_k += (double)sh[((size_t)g * K + k) * 3 + ch] * dacc[ch];
            }
            for (int j = 0; j < 3; ++j) du[j] += w_k * dY[k][j];
        }
        const double ud = u[0] * du[0] + u[1] * du[1] + u[2] * du[2];
        for (int j = 0; j < 3; ++j) dmeans[3 * g + j] += (du[j] - u[j] * ud) / dn;
    }
}

// Stages 2-3 of Sec. 2.1: duplicate every splat once per touched tile (in
// Gaussian order, tiles row-major within its rectangle) with key
// (tile << 32) | float_bits(depth), then stable-sort by key; tile_ranges[t]
// = [start, end) of tile t in the sorted list.  Returns the number of
// instances, or -1 if it exceeds capacity.
// Opacity-aware tile membership (the tighter tile intersection; the paper
// combines its blend with such culling, Sec. 4.2, but defines none), written
// as its definition: a splat keeps tile (tx, ty) iff the largest exponent of
// Eq. 3 over the tile's box of pixel-centre offsets d = mean - pixel,
// [mx - 16 tx - 15.5, mx - 16 tx - 0.5] x [my - 16 ty - 15.5, my - 16 ty - 0.5],
// reaches power_min, i.e. iff min over the box of
// q(d) = A dx^2 + 2 B dx dy + C dy^2 is <= tau2 = -2 power_min (so no tile if
// tau2 <= 0, which includes power_min = +inf).
// With A > 0 and C > 0, q restricted to any line dx = const or dy = const is
// a convex parabola, and q has no local minimum inside a box unless the box
// holds the origin (there q = 0 <= tau2, whatever the sign of AC - B^2).  So
// the box minimum is 0 if the box holds the origin, else the least of the
// four edge minima, each the parabola's vertex clamped to the edge.  A <= 0 or
// C <= 0 (never from a projected covariance): the whole rectangle is kept.
static double box_min_q(double A, double B, double C, double x0, double x1, double y0, double y1) {
    if (x0 > x1 || y0 > y1) return std::numeric_limits<double>::infinity();  // an empty (over-shrunk) box
    if (x0 <= 0 && 0 <= x1 && y0 <= 0 && 0 <= y1) return 0.0;
    auto q = [&](double x, double y) { return A * x * x + 2 * B * x * y + C * y * y; };
    double best = std::numeric_limits<double>::infinity();
    for (double x : {x0, x1}) best = std::min(best, q(x, std::clamp(-B * x / C, y0, y1)));
    for (double y : {y0, y1}) best = std::min(best, q(std::clamp(-B * y / A, x0, x1), y));
    return best;
}

// Decision for one (splat, tile) pair: 1 keep, 0 drop.  *ambiguous is set when
// the decision could go either way under rounding of float32 inputs and
// arithmetic: it changes somewhere within the box grown or shrunk by
// delta = 2^-20 (max(|mx|, |my|) + 16) px per side (float32 offsets of
// coordinates near |m| carry errors of about 2^-24 |m|) or tau2 scaled by
// 1 +- 1e-5.
static int tight_keep(double mx, double my, double A, double B, double C, double pmin, int tx, int ty, bool* ambiguous) {
    *ambiguous = false;
    if (!(A > 0) || !(C > 0)) return 1;
    const double tau2 = -2.0 * pmin;
    if (!(tau2 > 0)) return 0;
    const double x0 = mx - 16.0 * tx - 15.5, x1 = mx - 16.0 * tx - 0.5;
    const double y0 = my - 16.0 * ty - 15.5, y1 = my - 16.0 * ty - 0.5;
    const int keep = box_min_q(A, B, C, x0, x1, y0, y1) <= tau2;
    const double d = std::ldexp(std::max(std::fabs(mx), std::fabs(my)) + 16.0, -20);
    const bool sure_keep = box_min_q(A, B, C, x0 + d, x1 - d, y0 + d, y1 - d) <= tau2 * (1 - 1e-5);
    const bool sure_drop = box_min_q(A, B, C, x0 - d, x1 + d, y0 - d, y1 + d) > tau2 * (1 + 1e-5);
    *ambiguous = !(sure_keep || sure_drop);
    return keep;
}

// With conic_f and power_min (the CUDA path's float32 values, taken exactly
// as doubles) a tile is kept only per tight_keep; every pair of the
// rectangles whose decision is ambiguous is written to amb_out as
// (tile, Gaussian, decision) triples, up to amb_cap, and counted in *amb_count.
// tile_mask (one byte per tile, may be NULL): only the tiles marked non-zero
// get lists (the others stay empty), for sampling a large image.
int64_t oracle_bin_sort(int n, const double* mean2d, const int32_t* radius, const float* depth,
                        int W, int H, int64_t capacity, uint64_t* keys_out, uint32_t* ids_out,
                        uint32_t* tile_ranges, const float* conic_f, const float* power_min,
                        int64_t* amb_out, int64_t amb_cap, int64_t* amb_count, const uint8_t* tile_mask) {
    std::vector<uint64_t> keys;
    std::vector<uint32_t> ids;
    const bool tight = conic_f != nullptr && power_min != nullptr;
    int64_t n_amb = 0;
    for (int g = 0; g < n; ++g) {
        int rc[4];
        if (!tile_rect(mean2d[2 * g], mean2d[2 * g + 1], radius[g], W, H, rc)) continue;
        uint32_t dbits;
        std::memcpy(&dbits, &depth[g], 4);
        for (int ty = rc[2]; ty <= rc[3]; ++ty)
            for (int tx = rc[0]; tx <= rc[1]; ++tx) {
                const uint64_t tile = (uint64_t)ty * tiles_x(W) + tx;
                if (tile_mask && !tile_mask[tile]) continue;
                if (tight) {
                    bool amb = false;
                    const int keep = tight_keep(mean2d[2 * g], mean2d[2 * g + 1], conic_f[3 * g],
                                                conic_f[3 * g + 1], conic_f[3 * g + 2], power_min[g], tx, ty, &amb);
                    if (amb) {
                        if (amb_out && n_amb < amb_cap) {
                            amb_out[3 * n_amb] = (int64_t)tile;
                            amb_out[3 * n_amb + 1] = g;
                            amb_out[3 * n_amb + 2] = keep;
                        }
                        ++n_amb;
                    }
                    if (!keep) continue;
                }
                keys.push_back((tile << 32) | dbits);
                ids.push_back((uint32_t)g);
            }
    }
    if (amb_count) *amb_count = n_amb;
    int64_t I = (int64_t)keys.size();
    int ntiles = tiles_x(W) * tiles_y(H);
    for (int t = 0; t < 2 * ntiles; ++t) tile_ranges[t] = 0;
    if (I > capacity) return -1;
    std::vector<size_t> order(I);
    for (int64_t i = 0; i < I; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t b) { return keys[a] < keys[b]; });
    for (int64_t i = 0; i < I; ++i) {
        keys_out[i] = keys[order[i]];
        ids_out[i] = ids[order[i]];
    }
    for (int64_t i = 0; i < I; ++i) {
        uint32_t t = (uint32_t)(keys_out[i] >> 32);
        if (i == 0 || (uint32_t)(keys_out[i - 1] >> 32) != t) tile_ranges[2 * t] = (uint32_t)i;
        if (i == I - 1 || (uint32_t)(keys_out[i + 1] >> 32) != t) tile_ranges[2 * t + 1] = (uint32_t)(i + 1);
    }
    return I;
}

// Stage 4 (Eq. 1, Alg. 1): blend every tile over its sorted list.  Image is
// 3 x H x W (CHW).  Pixel results: T_final, n_contrib and an ambiguity flag.
// margins: {alpha, t, sum, slack} of the rounding model (Margins); err_bound
// (may be NULL) receives each pixel's first-order colour error bound.
void oracle_blend(int W, int H, const uint32_t* tile_ranges, const uint32_t* ids,
                  const double* mean2d, const double* conic, const double* opac, const double* rgb,
                  const double* bg, const double* margins, int n_threads,
                  const int32_t* tile_subset, int n_subset,
                  double* image, double* T_final, int32_t* n_contrib, uint8_t* ambiguous, double* err_bound) {
    const Margins mg{margins[0], margins[1], margins[2], margins[3]};
    const int tx = tiles_x(W);
    const int ntiles = tx * tiles_y(H);
    const int count = tile_subset ? n_subset : ntiles;
    parallel_for(count, n_threads, [&](int k) {
        int t = tile_subset ? tile_subset[k] : k;
        std::vector<Splat> list;
        for (uint32_t i = tile_ranges[2 * t]; i < tile_ranges[2 * t + 1]; ++i)
            list.push_back(load_splat(ids[i], mean2d, conic, opac, rgb));
        int x0 = (t % tx) * kTile, y0 = (t / tx) * kTile;
        for (int py = y0; py < std::min(y0 + kTile, H); ++py)
            for (int px = x0; px < std::min(x0 + kTile, W); ++px) {
                PixelResult r = composite_pixel(list, px + 0.5, py + 0.5, bg, mg);
                size_t pix = (size_t)py * W + px;
                if (err_bound) err_bound[pix] = r.err_bound;
                for (int ch = 0; ch < 3; ++ch) image[(size_t)ch * W * H + pix] = r.C[ch];
                T_final[pix] = r.T;
                n_contrib[pix] = r.n_contrib;
                ambiguous[pix] = r.ambiguous ? 1 : 0;
            }
    });
}

// Per-pixel brute force: every splat whose tile rectangle (if use_rect) covers
// the pixel's tile, ordered by (float depth, Gaussian index), composited as
// in oracle_blend.  Independent of duplication, sorting and tile ranges.
void oracle_brute_force(int n, const double* mean2d, const double* conic, const double* opac,
                        const double* rgb, const int32_t* radius, const float* depth, int W, int H,
                        const double* bg, int use_rect, double* image, double* T_final,
                        int32_t* n_contrib) {
    std::vector<int> order;
    for (int g = 0; g < n; ++g)
        if (radius[g] > 0) order.push_back(g);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return depth[a] < depth[b]; });
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            std::vector<Splat> list;
            for (int g : order) {
                if (use_rect) {
                    int rc[4];
                    if (!tile_rect(mean2d[2 * g], mean2d[2 * g + 1], radius[g], W, H, rc)) continue;
                    int tx = px / kTile, ty = py / kTile;
                    if (tx < rc[0] || tx > rc[1] || ty < rc[2] || ty > rc[3]) continue;
                }
                list.push_back(load_splat((uint32_t)g, mean2d, conic, opac, rgb));
            }
            PixelResult r = composite_pixel(list, px + 0.5, py + 0.5, bg, Margins{0.0, 0.0, 0.0, 0.0});
            size_t pix = (size_t)py * W + px;
            for (int ch = 0; ch < 3; ++ch) image[(size_t)ch * W * H + pix] = r.C[ch];
            T_final[pix] = r.T;
            n_contrib[pix] = r.n_contrib;
        }
}

// Analytic gradient of the blended image (Eq. 1) with respect to each splat's
// 2D mean, conic, opacity and colour, given dL/d(image) (3 x H x W).  For
// splat i on a pixel's list (contributors only; skipped splats carry none):
//   dC/dc_i     = alpha_i T_i
//   dC/dalpha_i = T_i (c_i - S_i),  S_i = (sum_{k>i} c_k alpha_k T_k + T_f bg) / T_{i+1}
// S_i is formed from explicit suffix sums, not from a recursion.  Then
// alpha = o e^p (unclamped branch): dalpha/do = e^p, dalpha/dp = alpha; both
// zero when the 0.99 clamp is active; dp/d* = 0 when power > 0 was clamped.
// Outputs are accumulated into the caller's zeroed arrays.
// Tiles are spread over n_threads threads, each accumulating into buffers of
// its own; the buffers are summed in thread order at the end (so the result
// is deterministic for a given thread count).  tile_subset, if given, limits
// the work to those tiles.
void oracle_blend_grad(int W, int H, const uint32_t* tile_ranges, const uint32_t* ids,
                       const double* mean2d, const double* conic, const double* opac,
                       const double* rgb, const double* bg, const double* dL_dimg, int n_gauss,
                       int n_threads, const int32_t* tile_subset, int n_subset,
                       double* dmean2d_out, double* dconic_out, double* dopac_out, double* drgb_out) {
    const int tx = tiles_x(W);
    const int ntiles = tx * tiles_y(H);
    const int count = tile_subset ? n_subset : ntiles;
    const int nt = std::max(1, std::min(n_threads, count));
    std::vector<std::vector<double>> acc(nt, std::vector<double>(9 * (size_t)n_gauss, 0.0));
    std::vector<std::thread> pool;
    for (int k = 0; k < nt; ++k)
        pool.emplace_back([&, k]() {
            double* dmean2d = acc[k].data();
            double* dconic = dmean2d + 2 * (size_t)n_gauss;
            double* dopac = dconic + 3 * (size_t)n_gauss;
            double* drgb = dopac + (size_t)n_gauss;
            for (int idx = k; idx < count; idx += nt) {
        int t = tile_subset ? tile_subset[idx] : idx;
        int x0 = (t % tx) * kTile, y0 = (t / tx) * kTile;
        for (int py = y0; py < std::min(y0 + kTile, H); ++py)
            for (int px = x0; px < std::min(x0 + kTile, W); ++px) {
                const double xp = px + 0.5, yp = py + 0.5;
                size_t pix = (size_t)py * W + px;
                double gC[3];
                for (int ch = 0; ch < 3; ++ch) gC[ch] = dL_dimg[(size_t)ch * W * H + pix];
                // forward walk, recording contributors
                struct Rec { uint32_t g; double alpha, T, e, power_raw; bool clamped; };
                std::vector<Rec> recs;
                double T = 1.0;
                for (uint32_t i = tile_ranges[2 * t]; i < tile_ranges[2 * t + 1]; ++i) {
                    Splat s = load_splat(ids[i], mean2d, conic, opac, rgb);
                    double praw = power_eq3(s, xp, yp);
                    double p = std::min(praw, 0.0);
                    double e = std::exp(p);
                    double raw = s.o * e;
                    double alpha = std::min(0.99, raw);
                    if (alpha < 1.0 / 255.0) continue;
                    double testT = T * (1.0 - alpha);
                    if (testT < 1e-4) break;
                    recs.push_back({ids[i], alpha, T, e, praw, raw > 0.99});
                    T = testT;
                }
                const double Tf = T;
                const size_t m = recs.size();
                // suffix[i] = sum_{k>i} c_k alpha_k T_k (per channel)
                std::vector<double> suffix(3 * (m + 1), 0.0);
                for (size_t i = m; i-- > 0;) {
                    Splat s = load_splat(recs[i].g, mean2d, conic, opac, rgb);
                    for (int ch = 0; ch < 3; ++ch)
                        suffix[3 * i + ch] = suffix[3 * (i + 1) + ch] + s.c[ch] * recs[i].alpha * recs[i].T;
                }
                for (size_t i = 0; i < m; ++i) {
                    const Rec& r = recs[i];
                    Splat s = load_splat(r.g, mean2d, conic, opac, rgb);
                    double Tnext = r.T * (1.0 - r.alpha);
                    double dL_dalpha = 0;
                    for (int ch = 0; ch < 3; ++ch) {
                        double S = (suffix[3 * (i + 1) + ch] + Tf * bg[ch]) / Tnext;
                        dL_dalpha += r.T * (s.c[ch] - S) * gC[ch];
                        drgb[3 * (size_t)r.g + ch] += r.alpha * r.T * gC[ch];
                    }
                    if (r.clamped) continue;
                    dopac[r.g] += dL_dalpha * r.e;
                    if (r.power_raw > 0) continue;
                    double dL_dp = dL_dalpha * r.alpha;
                    double dx = s.mx - xp, dy = s.my - yp;
                    dmean2d[2 * (size_t)r.g] += dL_dp * (-(s.A * dx + s.B * dy));
                    dmean2d[2 * (size_t)r.g + 1] += dL_dp * (-(s.B * dx + s.C * dy));
                    dconic[3 * (size_t)r.g] += dL_dp * (-0.5 * dx * dx);
                    dconic[3 * (size_t)r.g + 1] += dL_dp * (-dx * dy);
                    dconic[3 * (size_t)r.g + 2] += dL_dp * (-0.5 * dy * dy);
                }
            }
            }
        });
    for (auto& th : pool) th.join();
    for (int k = 0; k < nt; ++k) {
        const double* a = acc[k].data();
        for (size_t i = 0; i < 2 * (size_t)n_gauss; ++i) dmean2d_out[i] += a[i];
        for (size_t i = 0; i < 3 * (size_t)n_gauss; ++i) dconic_out[i] += a[2 * (size_t)n_gauss + i];
        for (size_t i = 0; i < (size_t)n_gauss; ++i) dopac_out[i] += a[5 * (size_t)n_gauss + i];
        for (size_t i = 0; i < 3 * (size_t)n_gauss; ++i) drgb_out[i] += a[6 * (size_t)n_gauss + i];
    }
}

// Eq. 6: the exponent as the dot product v_g . v_p of the Gaussian vector
// [-A/2, -C/2, -B, -A xh - B yh, -C yh - B xh, -A/2 xh^2 - C/2 yh^2 - B xh yh]
// and the pixel vector [xb^2, yb^2, xb yb, xb, yb, 1], with xh = x_g - x_c and
// xb the intra-tile offset such that x_p = x_c - xb (Eqs. 4-5).  Also returns
// the direct quadratic of Eq. 3 at dx = xh + xb for comparison.
void oracle_power_eq6(int n, const double* abc, const double* hat, const double* bar,
                      double* power_dot, double* power_direct) {
    for (int i = 0; i < n; ++i) {
        double A = abc[3 * i], B = abc[3 * i + 1], C = abc[3 * i + 2];
        double xh = hat[2 * i], yh = hat[2 * i + 1];
        double xb = bar[2 * i], yb = bar[2 * i + 1];
        double vg[6] = {-0.5 * A, -0.5 * C, -B, -A * xh - B * yh, -C * yh - B * xh,
                        -0.5 * A * xh * xh - 0.5 * C * yh * yh - B * xh * yh};
        double vp[6] = {xb * xb, yb * yb, xb * yb, xb, yb, 1.0};
        double acc = 0;
        for (int k = 0; k < 6; ++k) acc += vg[k] * vp[k];
        power_dot[i] = acc;
        double dx = xh + xb, dy = yh + yb;
        power_direct[i] = -0.5 * A * dx * dx - B * dx * dy - 0.5 * C * dy * dy;
    }
}

// Exponent matrix of one tile (what the tensor-core contraction produces,
// Eq. 8), evaluated directly with Eq. 3 in FP64: out[j * 256 + p] for list
// position j of the tile and pixel p = 16 * row + col of the tile (pixels
// outside the image are still evaluated at their centres).
void oracle_tile_power(int W, int tile, const uint32_t* tile_ranges, const uint32_t* ids,
                       const double* mean2d, const double* conic, double* out) {
    const int tx = tiles_x(W);
    int x0 = (tile % tx) * kTile, y0 = (tile / tx) * kTile;
    uint32_t a = tile_ranges[2 * tile], b = tile_ranges[2 * tile + 1];
    for (uint32_t i = a; i < b; ++i) {
        uint32_t g = ids[i];
        Splat s{mean2d[2 * (size_t)g], mean2d[2 * (size_t)g + 1], conic[3 * (size_t)g],
                conic[3 * (size_t)g + 1], conic[3 * (size_t)g + 2], 1.0, {0, 0, 0}};
        for (int p = 0; p < kTile * kTile; ++p) {
            double xp = x0 + (p % kTile) + 0.5, yp = y0 + (p / kTile) + 0.5;
            out[(size_t)(i - a) * 256 + p] = power_eq3(s, xp, yp);
        }
    }
}

}  // extern "C"

// Preprocessing stage (Sec. 2.1 (a)): EWA projection of one 3D Gaussian into
// one camera, shared by the projection kernel and the fused projection +
// binning kernel.  FP32 throughout; the 2D covariance and its inverse are
// recomputed in FP64 when the FP32 determinant is below 1e-6.
#pragma once
#include "internal.h"
#include "sh.cuh"

namespace gs {

template <typename T>
struct Cov2 {
    T a, b, c;
};

// T R Sigma3 R^T T^T with T = J (2x3) for camera-space point p; Sigma3 given
// as (Rq S): M, Sigma3 = M M^T.
template <typename T>
__device__ __forceinline__ Cov2<T> ewa_cov(const CamDev& cam, T px, T py, T pz, const T (&M)[3][3]) {
    T iz = T(1) / pz;
    T j00 = T(cam.fx) * iz, j02 = -T(cam.fx) * px * iz * iz;
    T j11 = T(cam.fy) * iz, j12 = -T(cam.fy) * py * iz * iz;
    // rows of J R
    T r0[3], r1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        r0[j] = j00 * T(cam.R[j]) + j02 * T(cam.R[6 + j]);
        r1[j] = j11 * T(cam.R[3 + j]) + j12 * T(cam.R[6 + j]);
    }
    // u = (J R) M : 2 x 3, Sigma2 = u u^T
    T u0[3], u1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        u0[k] = r0[0] * M[0][k] + r0[1] * M[1][k] + r0[2] * M[2][k];
        u1[k] = r1[0] * M[0][k] + r1[1] * M[1][k] + r1[2] * M[2][k];
    }
    Cov2<T> s;
    s.a = u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2] + T(cam.lowpass);
    s.b = u0[0] * u1[0] + u0[1] * u1[1] + u0[2] * u1[2];
    s.c = u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2] + T(cam.lowpass);
    return s;
}

template <typename T>
__device__ __forceinline__ void quat_scale_matrix(const float* q4, const float* s3, T (&M)[3][3], bool& ok) {
    T w = q4[0], x = q4[1], y = q4[2], z = q4[3];
    T nrm = w * w + x * x + y * y + z * z;
    ok = nrm > T(0);
    T inv = ok ? T(1) / sqrt(nrm) : T(0);
    w *= inv; x *= inv; y *= inv; z *= inv;
    T R[3][3] = {{T(1) - T(2) * (y * y + z * z), T(2) * (x * y - w * z), T(2) * (x * z + w * y)},
                 {T(2) * (x * y + w * z), T(1) - T(2) * (x * x + z * z), T(2) * (y * z - w * x)},
                 {T(2) * (x * z - w * y), T(2) * (y * z + w * x), T(1) - T(2) * (x * x + y * y)}};
    T s[3] = {T(s3[0]), T(s3[1]), T(s3[2])};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[i][j] = R[i][j] * s[j];
}

// Projection of Gaussian g into camera `cam`, written at index vo + g of the
// output arrays (vo = view * n for view-major outputs).  SH_DEGREE is a
// template argument so that the basis and the coefficient loop stay in
// registers; VEC16 reads the coefficients with 16-byte loads (every
// Gaussian's block of them 16-byte aligned).
template <int SH_DEGREE, bool VEC16>
__device__ __forceinline__ void project_gaussian(int g, const float* __restrict__ means,
                                                 const float* __restrict__ scales, const float* __restrict__ quats,
                                                 const float* __restrict__ sh, const CamDev& cam, size_t vo,
                                                 float2* __restrict__ mean2d_all, float* __restrict__ conic_all,
                                                 float* __restrict__ depth_all, int* __restrict__ radius_all,
                                                 float* __restrict__ rgb_all, uint32_t* __restrict__ touched_all) {
    constexpr int K = (SH_DEGREE + 1) * (SH_DEGREE + 1);
    float2* mean2d = mean2d_all + vo;
    float* conic = conic_all + 3 * vo;
    float* depth = depth_all + vo;
    int* radius = radius_all + vo;
    float* rgb = rgb_all + 3 * vo;
    uint32_t* tiles_touched = touched_all + vo;
    const float mwx = means[3 * g], mwy = means[3 * g + 1], mwz = means[3 * g + 2];
    const float px = cam.R[0] * mwx + cam.R[1] * mwy + cam.R[2] * mwz + cam.t[0];
    const float py = cam.R[3] * mwx + cam.R[4] * mwy + cam.R[5] * mwz + cam.t[1];
    const float pz = cam.R[6] * mwx + cam.R[7] * mwy + cam.R[8] * mwz + cam.t[2];

    float2 m2 = make_float2(0.f, 0.f);
    float cA = 0.f, cB = 0.f, cC = 0.f;
    int r = 0;
    uint32_t touched = 0;
    float col[3] = {0.f, 0.f, 0.f};
    bool live = pz > cam.znear;
    if (live) {
        float M[3][3];
        bool qok;
        quat_scale_matrix<float>(quats + 4 * g, scales + 3 * g, M, qok);
        live = qok;
        Cov2<float> s = ewa_cov<float>(cam, px, py, pz, M);
        float det = s.a * s.c - s.b * s.b;
        if (live && det < 1e-6f) {
            // near-singular: redo the 2D covariance and its inverse in FP64
            double Md[3][3];
            bool qd;
            quat_scale_matrix<double>(quats + 4 * g, scales + 3 * g, Md, qd);
            Cov2<double> sd = ewa_cov<double>(cam, (double)px, (double)py, (double)pz, Md);
            double dd = sd.a * sd.c - sd.b * sd.b;
            if (dd > 0.0) {
                cA = (float)(sd.c / dd);
                cB = (float)(-sd.b / dd);
                cC = (float)(sd.a / dd);
                s.a = (float)sd.a;
                s.b = (float)sd.b;
                s.c = (float)sd.c;
            } else {
                live = false;
            }
        } else if (live) {
            float id = 1.0f / det;
            cA = s.c * id;
            cB = -s.b * id;
            cC = s.a * id;
        }
        if (live) {
            const float iz = 1.0f / pz;
            m2.x = cam.fx * px * iz + cam.cx;
            m2.y = cam.fy * py * iz + cam.cy;
            live = fabsf(m2.x) <= 8388608.0f && fabsf(m2.y) <= 8388608.0f;
        }
        if (live) {
            float mid = 0.5f * (s.a + s.c);
            float hd = 0.5f * (s.a - s.c);
            float lmax = mid + sqrtf(fmaxf(0.f, hd * hd + s.b * s.b));
            float rr = ceilf(3.0f * sqrtf(lmax));
            r = rr >= 16777216.0f ? 16777216 : (int)rr;
            int x0, x1, y0, y1;
            if (tile_rect(m2.x, m2.y, r, cam.W, cam.H, x0, x1, y0, y1)) {
                touched = (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
            } else {
                live = false;
                r = 0;
            }
        } else {
            r = 0;
        }
        if (live) {
            // view direction from the camera centre c = -R^T t to the mean
            float cxw = -(cam.R[0] * cam.t[0] + cam.R[3] * cam.t[1] + cam.R[6] * cam.t[2]);
            float cyw = -(cam.R[1] * cam.t[0] + cam.R[4] * cam.t[1] + cam.R[7] * cam.t[2]);
            float czw = -(cam.R[2] * cam.t[0] + cam.R[5] * cam.t[1] + cam.R[8] * cam.t[2]);
            float dx = mwx - cxw, dy = mwy - cyw, dz = mwz - czw;
            float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
            float x = dx * inv, y = dy * inv, z = dz * inv;
            const float* c = sh + (size_t)g * K * 3;
            float basis[K];
            sh_basis<SH_DEGREE>(x, y, z, basis);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) col[ch] = 0.f;
            float cf[3 * K];
            if constexpr (VEC16) {
#pragma unroll
                for (int q = 0; q < 3 * K / 4; ++q) {
                    const float4 v = __ldg(reinterpret_cast<const float4*>(c) + q);
                    cf[4 * q] = v.x;
                    cf[4 * q + 1] = v.y;
                    cf[4 * q + 2] = v.z;
                    cf[4 * q + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 3 * K; ++q) cf[q] = __ldg(c + q);
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) col[ch] += cf[3 * k + ch] * basis[k];
            }
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) col[ch] = fmaxf(0.f, col[ch] + 0.5f);
        } else {
            cA = cB = cC = 0.f;
            m2 = make_float2(0.f, 0.f);
        }
    }
    mean2d[g] = m2;
    conic[3 * g] = cA;
    conic[3 * g + 1] = cB;
    conic[3 * g + 2] = cC;
    depth[g] = pz;
    radius[g] = live ? r : 0;
    rgb[3 * g] = col[0];
    rgb[3 * g + 1] = col[1];
    rgb[3 * g + 2] = col[2];
    tiles_touched[g] = live ? touched : 0u;
}


}  // namespace gs

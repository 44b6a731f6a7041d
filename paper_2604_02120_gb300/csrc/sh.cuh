// Real spherical harmonics up to degree 3 (the colour model of the
// preprocessing stage, Sec. 2.1 (a)): the basis at a unit direction and the
// gradient of a weighted sum of it with respect to the direction's
// coordinates.  The basis is sqrt(2) Re/Im of the complex harmonics with the
// Condon-Shortley phase, m = -l..l within degree l.
#pragma once

namespace gs {

// Normalisations of the degree 0..3 harmonics (signs folded in).
constexpr float kSH0 = 0.28209479177387814f;
constexpr float kSH1 = 0.4886025119029199f;
constexpr float kSH2_0 = 1.0925484305920792f, kSH2_1 = -1.0925484305920792f, kSH2_2 = 0.31539156525252005f,
                kSH2_3 = -1.0925484305920792f, kSH2_4 = 0.5462742152960396f;
constexpr float kSH3_0 = -0.5900435899266435f, kSH3_1 = 2.890611442640554f, kSH3_2 = -0.4570457994644658f,
                kSH3_3 = 0.3731763325901154f, kSH3_4 = -0.4570457994644658f, kSH3_5 = 1.445305721320277f,
                kSH3_6 = -0.5900435899266435f;

template <int D>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float (&Y)[(D + 1) * (D + 1)]) {
    Y[0] = kSH0;
    if constexpr (D >= 1) {
        Y[1] = -kSH1 * y;
        Y[2] = kSH1 * z;
        Y[3] = -kSH1 * x;
    }
    if constexpr (D >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kSH2_0 * x * y;
        Y[5] = kSH2_1 * y * z;
        Y[6] = kSH2_2 * (2.f * zz - xx - yy);
        Y[7] = kSH2_3 * x * z;
        Y[8] = kSH2_4 * (xx - yy);
        if constexpr (D >= 3) {
            Y[9] = kSH3_0 * y * (3.f * xx - yy);
            Y[10] = kSH3_1 * x * y * z;
            Y[11] = kSH3_2 * y * (4.f * zz - xx - yy);
            Y[12] = kSH3_3 * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = kSH3_4 * x * (4.f * zz - xx - yy);
            Y[14] = kSH3_5 * z * (xx - yy);
            Y[15] = kSH3_6 * x * (xx - 3.f * yy);
        }
    }
}

// g = sum_k w[k] * grad Y_k at (x, y, z), the basis read as polynomials of
// unconstrained x, y, z.
template <int D>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, const float (&w)[(D + 1) * (D + 1)],
                                              float& gx, float& gy, float& gz) {
    gx = gy = gz = 0.f;
    if constexpr (D >= 1) {
        gy -= kSH1 * w[1];
        gz += kSH1 * w[2];
        gx -= kSH1 * w[3];
    }
    if constexpr (D >= 2) {
        gx += kSH2_0 * y * w[4];
        gy += kSH2_0 * x * w[4];
        gy += kSH2_1 * z * w[5];
        gz += kSH2_1 * y * w[5];
        gx -= 2.f * kSH2_2 * x * w[6];
        gy -= 2.f * kSH2_2 * y * w[6];
        gz += 4.f * kSH2_2 * z * w[6];
        gx += kSH2_3 * z * w[7];
        gz += kSH2_3 * x * w[7];
        gx += 2.f * kSH2_4 * x * w[8];
        gy -= 2.f * kSH2_4 * y * w[8];
        if constexpr (D >= 3) {
            const float xx = x * x, yy = y * y, zz = z * z;
            gx += kSH3_0 * 6.f * x * y * w[9];
            gy += kSH3_0 * 3.f * (xx - yy) * w[9];
            gx += kSH3_1 * y * z * w[10];
            gy += kSH3_1 * x * z * w[10];
            gz += kSH3_1 * x * y * w[10];
            gx -= kSH3_2 * 2.f * x * y * w[11];
            gy += kSH3_2 * (4.f * zz - xx - 3.f * yy) * w[11];
            gz += kSH3_2 * 8.f * y * z * w[11];
            gx -= kSH3_3 * 6.f * x * z * w[12];
            gy -= kSH3_3 * 6.f * y * z * w[12];
            gz += kSH3_3 * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
            gx += kSH3_4 * (4.f * zz - 3.f * xx - yy) * w[13];
            gy -= kSH3_4 * 2.f * x * y * w[13];
            gz += kSH3_4 * 8.f * x * z * w[13];
            gx += kSH3_5 * 2.f * x * z * w[14];
            gy -= kSH3_5 * 2.f * y * z * w[14];
            gz += kSH3_5 * (xx - yy) * w[14];
            gx += kSH3_6 * 3.f * (xx - yy) * w[15];
            gy -= kSH3_6 * 6.f * x * y * w[15];
        }
    }
}

}  // namespace gs

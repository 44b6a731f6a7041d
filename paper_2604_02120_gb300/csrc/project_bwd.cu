// Gradient of the preprocessing stage (Sec. 2.1 (a); the paper has no backward
// pass): dL/d(means, scales, quats, sh) of the 3D Gaussians from dL/d(mean2d,
// conic, rgb) of their splats in every view, one thread per Gaussian, summed
// over the views in registers (no atomics).  FP32; the step through the 2x2
// inverse runs in FP64 where the forward did (determinant below 1e-6).
//
// With u0, u1 the rows of (J R) M, M = Rq(q/|q|) diag(s), the 2D covariance
// is [[u0.u0 + lp, u0.u1], [u0.u1, u1.u1 + lp]], so from (da, db, dc):
//   du0 = 2 da u0 + db u1,  du1 = db u0 + 2 dc u1,
//   dM += r0^T du0 + r1^T du1 and dr = du M^T for the rows r0, r1 of J R,
// and J's entries are functions of the camera-space point p = R mean + t.
// A block's SH coefficients and their gradients go through shared memory
// (coalesced loads and stores, one odd-stride row per Gaussian so the
// threads' row reads are free of bank conflicts), which keeps the registers,
// and with them the resident warps, at what the latency of HBM needs.
#include "internal.h"
#include "sh.cuh"

namespace gs {
namespace {

constexpr int kProjBwdThreads = 128;

// One view's inputs of one Gaussian.
struct ViewIn {
    int radius;
    float2 dm;
    float dA, dB, dC, dr[3];
};

__device__ __forceinline__ ViewIn load_view(size_t item, const int* radius_all, const float2* dmean2d_all,
                                            const float* dconic_all, const float* drgb_all) {
    ViewIn in;
    in.radius = radius_all[item];
    in.dm = dmean2d_all[item];
    in.dA = dconic_all[3 * item];
    in.dB = dconic_all[3 * item + 1];
    in.dC = dconic_all[3 * item + 2];
    in.dr[0] = drgb_all[3 * item];
    in.dr[1] = drgb_all[3 * item + 1];
    in.dr[2] = drgb_all[3 * item + 2];
    return in;
}

// Floats per Gaussian row of the shared coefficient arrays (odd).
template <int SH_DEGREE>
__host__ __device__ constexpr int sh_row() { return (3 * (SH_DEGREE + 1) * (SH_DEGREE + 1)) | 1; }

template <int SH_DEGREE>
__global__ void __launch_bounds__(kProjBwdThreads, 4) k_project_bwd(int n, const float* __restrict__ means,
                                                                 const float* __restrict__ scales,
                                                                 const float* __restrict__ quats,
                                                                 const float* __restrict__ sh,
                                                                 const __grid_constant__ CamViews views,
                                                                 const int* __restrict__ radius_all,
                                                                 const float2* __restrict__ dmean2d_all,
                                                                 const float* __restrict__ dconic_all,
                                                                 const float* __restrict__ drgb_all,
                                                                 float* __restrict__ dmeans, float* __restrict__ dscales,
                                                                 float* __restrict__ dquats, float* __restrict__ dsh) {
    constexpr int K = (SH_DEGREE + 1) * (SH_DEGREE + 1), KC = 3 * K, ROW = sh_row<SH_DEGREE>();
    extern __shared__ float s_sh[];  // [kProjBwdThreads][ROW] coefficients, then as many gradients
    float* s_cf = s_sh;
    float* s_dcf = s_sh + kProjBwdThreads * ROW;
    const int g0 = blockIdx.x * kProjBwdThreads;
    const int nb = min(kProjBwdThreads, n - g0);
    // every global load before the first barrier, so that a block waits for HBM once
    const int g = g0 + threadIdx.x, gc = min(g, n - 1);
    const float mw[3] = {means[3 * gc], means[3 * gc + 1], means[3 * gc + 2]};
    const float s[3] = {scales[3 * gc], scales[3 * gc + 1], scales[3 * gc + 2]};
    const float q0 = quats[4 * gc], q1 = quats[4 * gc + 1], q2 = quats[4 * gc + 2], q3 = quats[4 * gc + 3];
    const ViewIn first = load_view((size_t)gc, radius_all, dmean2d_all, dconic_all, drgb_all);
    if (nb == kProjBwdThreads) {  // a full block: a fixed trip count, many loads in flight
#pragma unroll 12
        for (int j = 0; j < KC; ++j) {
            const int i = threadIdx.x + j * kProjBwdThreads, r = i / KC, q = i - r * KC;
            s_cf[r * ROW + q] = __ldg(sh + (size_t)g0 * KC + i);
            s_dcf[r * ROW + q] = 0.f;
        }
    } else {
        for (int i = threadIdx.x; i < nb * KC; i += kProjBwdThreads) {
            const int r = i / KC, q = i - r * KC;
            s_cf[r * ROW + q] = __ldg(sh + (size_t)g0 * KC + i);
            s_dcf[r * ROW + q] = 0.f;
        }
    }
    __syncthreads();
    if (g < n) {
    const float* cf = s_cf + threadIdx.x * ROW;
    float* dcf = s_dcf + threadIdx.x * ROW;
    const float qn2 = q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3;
    const float iqn = qn2 > 0.f ? 1.0f / sqrtf(qn2) : 0.f;
    const float w = q0 * iqn, x = q1 * iqn, y = q2 * iqn, z = q3 * iqn;
    const float Rq[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                            {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                            {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
    float M[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[i][j] = Rq[i][j] * s[j];

    float dmw[3] = {0.f, 0.f, 0.f}, dM[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};

    for (int v = 0; v < views.num_views; ++v) {
        const ViewIn in =
            v == 0 ? first : load_view((size_t)v * n + g, radius_all, dmean2d_all, dconic_all, drgb_all);
        if (in.radius <= 0) continue;
        const CamDev& cam = views.cams[v];
        const float* R = cam.R;
        const float px = R[0] * mw[0] + R[1] * mw[1] + R[2] * mw[2] + cam.t[0];
        const float py = R[3] * mw[0] + R[4] * mw[1] + R[5] * mw[2] + cam.t[1];
        const float pz = R[6] * mw[0] + R[7] * mw[1] + R[8] * mw[2] + cam.t[2];
        const float iz = 1.0f / pz;
        const float j00 = cam.fx * iz, j02 = -cam.fx * px * iz * iz;
        const float j11 = cam.fy * iz, j12 = -cam.fy * py * iz * iz;
        float r0[3], r1[3], u0[3], u1[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            r0[j] = j00 * R[j] + j02 * R[6 + j];
            r1[j] = j11 * R[3 + j] + j12 * R[6 + j];
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            u0[k] = r0[0] * M[0][k] + r0[1] * M[1][k] + r0[2] * M[2][k];
            u1[k] = r1[0] * M[0][k] + r1[1] * M[1][k] + r1[2] * M[2][k];
        }
        const float a = u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2] + cam.lowpass;
        const float b = u0[0] * u1[0] + u0[1] * u1[1] + u0[2] * u1[2];
        const float cc = u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2] + cam.lowpass;
        const float dA = in.dA, dB = in.dB, dC = in.dC;
        // conic (A, B, C) = (c, -b, a) / det  ->  d(a, b, c)
        float da, db, dc;
        const float det = a * cc - b * b;
        if (det < 1e-6f) {
            double ad = 0.0, bd = 0.0, cd = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                double e0 = 0.0, e1 = 0.0;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const double mik = (double)Rq[i][k] * (double)s[k];
                    e0 += ((double)j00 * R[i] + (double)j02 * R[6 + i]) * mik;
                    e1 += ((double)j11 * R[3 + i] + (double)j12 * R[6 + i]) * mik;
                }
                ad += e0 * e0;
                bd += e0 * e1;
                cd += e1 * e1;
            }
            ad += cam.lowpass;
            cd += cam.lowpass;
            const double i2 = 1.0 / ((ad * cd - bd * bd) * (ad * cd - bd * bd));
            da = (float)((-cd * cd * dA + bd * cd * dB - bd * bd * dC) * i2);
            db = (float)((2.0 * bd * cd * dA - (ad * cd + bd * bd) * dB + 2.0 * ad * bd * dC) * i2);
            dc = (float)((-bd * bd * dA + ad * bd * dB - ad * ad * dC) * i2);
        } else {
            const float id = 1.0f / det, i2 = id * id;
            da = (-cc * cc * dA + b * cc * dB - b * b * dC) * i2;
            db = (2.f * b * cc * dA - (a * cc + b * b) * dB + 2.f * a * b * dC) * i2;
            dc = (-b * b * dA + a * b * dB - a * a * dC) * i2;
        }
        float du0[3], du1[3], dr0[3] = {0.f, 0.f, 0.f}, dr1[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            du0[k] = 2.f * da * u0[k] + db * u1[k];
            du1[k] = db * u0[k] + 2.f * dc * u1[k];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                dM[i][k] += r0[i] * du0[k] + r1[i] * du1[k];
                dr0[i] += du0[k] * M[i][k];
                dr1[i] += du1[k] * M[i][k];
            }
        const float dj00 = dr0[0] * R[0] + dr0[1] * R[1] + dr0[2] * R[2];
        const float dj02 = dr0[0] * R[6] + dr0[1] * R[7] + dr0[2] * R[8];
        const float dj11 = dr1[0] * R[3] + dr1[1] * R[4] + dr1[2] * R[5];
        const float dj12 = dr1[0] * R[6] + dr1[1] * R[7] + dr1[2] * R[8];
        const float2 dm2 = in.dm;
        const float fxz = cam.fx * iz, fyz = cam.fy * iz;
        const float dpx = (dm2.x - dj02 * iz) * fxz;
        const float dpy = (dm2.y - dj12 * iz) * fyz;
        const float dpz = -(dj00 * fxz + dj11 * fyz) * iz + 2.f * (dj02 * fxz * px + dj12 * fyz * py) * iz * iz -
                          (dm2.x * fxz * px + dm2.y * fyz * py) * iz;
#pragma unroll
        for (int j = 0; j < 3; ++j) dmw[j] += R[j] * dpx + R[3 + j] * dpy + R[6 + j] * dpz;

        // colour: rgb = max(0, sum_k cf_k Y_k(u) + 0.5), u = unit(mean - camera centre)
        const float cxw = -(R[0] * cam.t[0] + R[3] * cam.t[1] + R[6] * cam.t[2]);
        const float cyw = -(R[1] * cam.t[0] + R[4] * cam.t[1] + R[7] * cam.t[2]);
        const float czw = -(R[2] * cam.t[0] + R[5] * cam.t[1] + R[8] * cam.t[2]);
        const float ddx = mw[0] - cxw, ddy = mw[1] - cyw, ddz = mw[2] - czw;
        const float idn = rsqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
        const float ux = ddx * idn, uy = ddy * idn, uz = ddz * idn;
        float Y[K];
        sh_basis<SH_DEGREE>(ux, uy, uz, Y);
        float dacc[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc += cf[3 * k + ch] * Y[k];
            dacc[ch] = acc + 0.5f > 0.f ? in.dr[ch] : 0.f;
        }
        float wk[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            wk[k] = 0.f;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                dcf[3 * k + ch] += Y[k] * dacc[ch];
                wk[k] += cf[3 * k + ch] * dacc[ch];
            }
        }
        if constexpr (SH_DEGREE > 0) {
            float gx, gy, gz;
            sh_basis_grad<SH_DEGREE>(ux, uy, uz, wk, gx, gy, gz);
            const float ud = ux * gx + uy * gy + uz * gz;
            dmw[0] += (gx - ux * ud) * idn;
            dmw[1] += (gy - uy * ud) * idn;
            dmw[2] += (gz - uz * ud) * idn;
        }
    }

    // M = Rq diag(s):  ds_j = sum_i dM_ij Rq_ij,  dRq_ij = dM_ij s_j;  q / |q|
    float dR[3][3], ds[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        ds[j] = dM[0][j] * Rq[0][j] + dM[1][j] * Rq[1][j] + dM[2][j] * Rq[2][j];
#pragma unroll
        for (int i = 0; i < 3; ++i) dR[i][j] = dM[i][j] * s[j];
    }
    const float dw = 2.f * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
    const float dx = 2.f * (y * (dR[0][1] + dR[1][0]) + z * (dR[0][2] + dR[2][0]) + w * (dR[2][1] - dR[1][2]) -
                            2.f * x * (dR[1][1] + dR[2][2]));
    const float dy = 2.f * (x * (dR[0][1] + dR[1][0]) + w * (dR[0][2] - dR[2][0]) + z * (dR[1][2] + dR[2][1]) -
                            2.f * y * (dR[0][0] + dR[2][2]));
    const float dz = 2.f * (w * (dR[1][0] - dR[0][1]) + x * (dR[0][2] + dR[2][0]) + y * (dR[1][2] + dR[2][1]) -
                            2.f * z * (dR[0][0] + dR[1][1]));
    const float proj = w * dw + x * dx + y * dy + z * dz;
    dmeans[3 * g] = dmw[0];
    dmeans[3 * g + 1] = dmw[1];
    dmeans[3 * g + 2] = dmw[2];
    dscales[3 * g] = ds[0];
    dscales[3 * g + 1] = ds[1];
    dscales[3 * g + 2] = ds[2];
    dquats[4 * g] = (dw - w * proj) * iqn;
    dquats[4 * g + 1] = (dx - x * proj) * iqn;
    dquats[4 * g + 2] = (dy - y * proj) * iqn;
    dquats[4 * g + 3] = (dz - z * proj) * iqn;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb * KC; i += kProjBwdThreads) {
        const int r = i / KC, q = i - r * KC;
        dsh[(size_t)g0 * KC + i] = s_dcf[r * ROW + q];
    }
}

template <int D>
cudaError_t launch_deg(int n, cudaStream_t s, const float* means, const float* scales, const float* quats,
                       const float* sh, const CamViews& cams, const int* radius, const float* dmean2d,
                       const float* dconic, const float* drgb, float* dmeans, float* dscales, float* dquats,
                       float* dsh) {
    const size_t smem = 2 * sizeof(float) * kProjBwdThreads * sh_row<D>();
    static std::mutex mu;  // the attribute is set once per process, as for the blend kernels
    static bool attr = false;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!attr) {
            const cudaError_t e =
                cudaFuncSetAttribute(k_project_bwd<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
    }
    k_project_bwd<D><<<(n + kProjBwdThreads - 1) / kProjBwdThreads, kProjBwdThreads, smem, s>>>(
        n, means, scales, quats, sh, cams, radius, reinterpret_cast<const float2*>(dmean2d), dconic, drgb, dmeans,
        dscales, dquats, dsh);
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_project_bwd(int n, const float* means, const float* scales, const float* quats, const float* sh,
                               int sh_degree, const CamViews& cams, const int* radius, const float* dmean2d,
                               const float* dconic, const float* drgb, float* dmeans, float* dscales, float* dquats,
                               float* dsh, cudaStream_t s) {
    cudaError_t e;
    switch (sh_degree) {
        case 0: e = launch_deg<0>(n, s, means, scales, quats, sh, cams, radius, dmean2d, dconic, drgb, dmeans,
                                  dscales, dquats, dsh); break;
        case 1: e = launch_deg<1>(n, s, means, scales, quats, sh, cams, radius, dmean2d, dconic, drgb, dmeans,
                                  dscales, dquats, dsh); break;
        case 2: e = launch_deg<2>(n, s, means, scales, quats, sh, cams, radius, dmean2d, dconic, drgb, dmeans,
                                  dscales, dquats, dsh); break;
        default: e = launch_deg<3>(n, s, means, scales, quats, sh, cams, radius, dmean2d, dconic, drgb, dmeans,
                                   dscales, dquats, dsh); break;
    }
    if (e != cudaSuccess) return e;
    count_launches();
    return cudaGetLastError();
}

}  // namespace gs

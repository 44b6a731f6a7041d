// Opacity-aware tile membership (the tighter tile intersection; not in the
// paper), shared by the bin/sort kernels and the fused projection + binning
// kernel.
//
// A splat keeps tile (tx, ty) of its rectangle only if its exponent can reach
// power_min at some pixel centre of the tile: if the tile's box of centre
// offsets d = mean - pixel meets the region E = {d : q(d) <= tau2},
// q(d) = A dx^2 + 2 B dx dy + C dy^2, tau2 = -2 power_min.  On a line dy = y,
// E is the interval dx in [(-B y - s(y)) / A, (-B y + s(y)) / A] with
// s(y) = sqrt(A tau2 - det y^2), det = AC - B^2, so within the strip of one
// tile row E's x-extent is one interval and the row keeps one run of tiles,
// found in O(1):
//  - det > 0 (an ellipse): the right end x_r(y) is concave, largest at E's
//    rightmost point dy = -(B/C) x_max (x_max = sqrt(tau2 C / det)), or at the
//    strip edge nearest to it; the left end mirrored; |dy| <= sqrt(tau2 A / det).
//  - det <= 0 (a degenerate or indefinite form; a Gaussian with one huge
//    scale projects to a nearly singular conic): x_r(y) is convex, so it is
//    largest at one of the strip's two edges; the left end mirrored.
// det comes from Kahan's FMA evaluation of AC - B^2 (the rounding error of
// B^2 is recovered exactly by an FMA and added back), accurate to a few units
// in the last place of det itself: the plain float32 difference cancels to
// zero or below for needle-shaped splats and would keep their whole
// rectangle.  FP32 throughout in a fixed order (no contraction); square
// roots and quotients use the hardware's approximate instructions (a few
// units in the last place, far inside the margin power_min carries), so the
// rule is deterministic and every kernel that applies it decides alike.
// A <= 0 or C <= 0: whole rows; tau2 <= 0: no tile.
#pragma once

namespace gs {

__device__ __forceinline__ float tight_sqrt(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float tight_div(float a, float b) {
    float y;
    asm("div.approx.f32 %0, %1, %2;" : "=f"(y) : "f"(a), "f"(b));
    return y;
}

struct TightRows {
    int mode;  // 0: whole rows, 1: no tile, 2: ellipse (det > 0), 3: det <= 0
    float mx, my, nB, det, Atau, rA, ymax, dyr;
};

__device__ __forceinline__ TightRows tight_rows(float mx, float my, float A, float B, float C, float pmin) {
    TightRows t{0, mx, my, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (!(A > 0.f) || !(C > 0.f)) return t;
    const float bb = __fmul_rn(B, B);
    const float bb_err = __fmaf_rn(-B, B, bb);  // bb - B*B, exact
    const float det = __fadd_rn(__fmaf_rn(A, C, -bb), bb_err);
    const float tau2 = __fmul_rn(-2.0f, pmin);
    t.mode = 1;
    if (!(tau2 > 0.f)) return t;
    t.nB = -B;
    t.det = det;
    t.Atau = __fmul_rn(A, tau2);
    t.rA = tight_div(1.0f, A);
    if (det > 0.f) {
        t.mode = 2;
        t.ymax = tight_sqrt(tight_div(__fmul_rn(tau2, A), det));
        // -(B/C) x_max = -B sqrt(tau2 / (C det)); 0 for B = 0 even if the root overflows
        t.dyr = (B == 0.f) ? 0.f : __fmul_rn(-B, tight_sqrt(tight_div(tau2, __fmul_rn(C, det))));
    } else {
        t.mode = 3;
        t.ymax = __int_as_float(0x7f800000);  // +inf: the form is unbounded along its null line
    }
    return t;
}

// Right (sign +1) or left (sign -1) end of E's x-extent on the line dy = y.
__device__ __forceinline__ float tight_end(const TightRows& t, float y, float sign) {
    const float s = tight_sqrt(fmaxf(__fsub_rn(t.Atau, __fmul_rn(t.det, __fmul_rn(y, y))), 0.f));
    return __fmul_rn(__fadd_rn(__fmul_rn(t.nB, y), sign * s), t.rA);
}

// The kept tiles [first, last] of row ty within [x0, x1] (first > last: none).
__device__ __forceinline__ void tight_row(const TightRows& t, int ty, int x0, int x1, int& first, int& last) {
    first = x0;
    last = x1;
    if (t.mode == 0) return;
    last = x0 - 1;
    if (t.mode == 1) return;
    const float lo = fmaxf(__fsub_rn(t.my, __fadd_rn((float)(16 * ty), 15.5f)), -t.ymax);
    const float hi = fminf(__fsub_rn(t.my, __fadd_rn((float)(16 * ty), 0.5f)), t.ymax);
    if (!(lo <= hi)) return;
    float xr, xl;
    if (t.mode == 2) {
        xr = tight_end(t, fminf(fmaxf(t.dyr, lo), hi), 1.f);
        xl = tight_end(t, fminf(fmaxf(-t.dyr, lo), hi), -1.f);
    } else {
        xr = fmaxf(tight_end(t, lo, 1.f), tight_end(t, hi, 1.f));
        xl = fminf(tight_end(t, lo, -1.f), tight_end(t, hi, -1.f));
    }
    // tile tx has offsets [mx - 16 tx - 15.5, mx - 16 tx - 0.5]
    const float flo = __fmul_rn(__fsub_rn(__fsub_rn(t.mx, 15.5f), xr), 0.0625f);
    const float fhi = __fmul_rn(__fsub_rn(__fsub_rn(t.mx, 0.5f), xl), 0.0625f);
    first = (int)ceilf(fminf(fmaxf(flo, (float)x0), (float)(x1 + 1)));
    last = (int)floorf(fminf(fmaxf(fhi, (float)(x0 - 1)), (float)x1));
}

}  // namespace gs

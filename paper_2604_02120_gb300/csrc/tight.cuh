// Opacity-aware tile membership (the tighter tile intersection; not in the
// paper), shared by the bin/sort kernels and the fused projection + binning
// kernel.
//
// A splat keeps tile (tx, ty) of its rectangle only if its exponent can reach
// power_min at some pixel centre of the tile: if the tile's box of centre offsets d = mean - pixel meets the
// ellipse E = {d : q(d) <= tau2}, q(d) = A dx^2 + 2 B dx dy + C dy^2,
// tau2 = -2 power_min.  Within the strip of one tile row, E's x-extent is an
// interval: its right end is E's rightmost point (dy = -(B/C) x_max, x_max =
// sqrt(tau2 C / det), det = AC - B^2) with dy clamped to the strip, the left
// end the mirror image, and on a line dy = y the boundary is at
// dx = (-B y +- sqrt(A tau2 - det y^2)) / A.  So each row keeps one run of
// tiles, found in O(1).  Floating point decides an integer here, so the rule
// is FP32 with one IEEE rounding per operation in a fixed order (the oracle
// repeats it).  Not positive definite: whole rows; tau2 <= 0: no tile.
#pragma once

namespace gs {

struct TightRows {
    int mode;  // 0: whole rows, 1: no tile, 2: the ellipse rule
    float mx, my, nB, det, Atau, rA, ymax, dyr;
};

__device__ __forceinline__ TightRows tight_rows(float mx, float my, float A, float B, float C, float pmin) {
    TightRows t{0, mx, my, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const float det = __fsub_rn(__fmul_rn(A, C), __fmul_rn(B, B));
    if (!(A > 0.f) || !(det > 0.f)) return t;
    const float tau2 = __fmul_rn(-2.0f, pmin);
    t.mode = 1;
    if (!(tau2 > 0.f)) return t;
    t.mode = 2;
    t.nB = -B;
    t.det = det;
    t.Atau = __fmul_rn(A, tau2);
    t.rA = __fdiv_rn(1.0f, A);
    t.ymax = __fsqrt_rn(__fdiv_rn(__fmul_rn(tau2, A), det));
    const float xmax = __fsqrt_rn(__fdiv_rn(__fmul_rn(tau2, C), det));
    t.dyr = __fmul_rn(__fdiv_rn(-B, C), xmax);
    return t;
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
    const float yr = fminf(fmaxf(t.dyr, lo), hi), yl = fminf(fmaxf(-t.dyr, lo), hi);
    const float sr = __fsqrt_rn(fmaxf(__fsub_rn(t.Atau, __fmul_rn(t.det, __fmul_rn(yr, yr))), 0.f));
    const float sl = __fsqrt_rn(fmaxf(__fsub_rn(t.Atau, __fmul_rn(t.det, __fmul_rn(yl, yl))), 0.f));
    const float xr = __fmul_rn(__fadd_rn(__fmul_rn(t.nB, yr), sr), t.rA);
    const float xl = __fmul_rn(__fsub_rn(__fmul_rn(t.nB, yl), sl), t.rA);
    // tile tx has offsets [mx - 16 tx - 15.5, mx - 16 tx - 0.5]
    const float flo = __fmul_rn(__fsub_rn(__fsub_rn(t.mx, 15.5f), xr), 0.0625f);
    const float fhi = __fmul_rn(__fsub_rn(__fsub_rn(t.mx, 0.5f), xl), 0.0625f);
    first = (int)ceilf(fminf(fmaxf(flo, (float)x0), (float)(x1 + 1)));
    last = (int)floorf(fminf(fmaxf(fhi, (float)(x0 - 1)), (float)x1));
}

}  // namespace gs

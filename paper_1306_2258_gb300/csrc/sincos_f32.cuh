// Single-precision sine and cosine on the FP32 FMA pipe.
//
// Used for the per-pair seeds of the q recurrence, where the phase can be
// small (near pairs at low q: the value must keep full relative accuracy, so
// the hardware MUFU approximation, accurate only in absolute terms, is not
// used) or large (far pairs, a few thousand radians for elongated molecules).
//
// Method (textbook; nothing here is taken from a vendor math library):
//  1. Quadrant reduction with the Cody-Waite scheme: n = nearest integer to
//     x*2/pi, and x - n*pi/2 = y_hi + y_lo with y_hi = x - n*P1 (exact in one
//     fused multiply-add: for |x| >= 1 both operands lie on the 2^-23 grid)
//     and y_lo = -n*(P2 + P3), where P1, P2, P3 are the successive float32
//     roundings of pi/2, pi/2 - P1 and pi/2 - P1 - P2.  The polynomials take
//     y = fl(y_hi + y_lo); its rounding error d = y_lo - (y - y_hi) is kept and
//     applied as a first-order correction, sin(y + d) = sin y + d cos y,
//     cos(y + d) = cos y - d sin y.  Without it the error of y would be the
//     same for every x with the same n (a fixed offset rounded on a fixed
//     grid): a phase bias that millions of pairs would share, and that would
//     add up instead of averaging out.  The correction (below half an ulp of
//     the result) must enter before the last rounding, inside the small
//     terms: sin = y + (y^3 P(y^2) + d cos y), cos = 1 + (y^2 Q(y^2) - d y);
//     added to an already rounded result it would always round away.
//  2. Taylor polynomials on |y| <= pi/4: sin through the y^9 term (truncation
//     below 2e-9 relative), cos through the y^10 term (below 2e-10), in Horner
//     form with coefficients 1/k! rounded to float32.
//  3. The quadrant n mod 4 swaps and negates the pair.
#pragma once

namespace sas {

struct SinCos {
    float s, c;
};

__device__ __forceinline__ SinCos sincos_f32(float x)
{
    const float kTwoOverPi = 0.636619746685028076171875f;   // float32(2/pi)
    const float kP1 = 1.57079637050628662109375f;            // float32(pi/2)
    const float kP2 = -4.37113882867379300296306610107421875e-08f;
    const float kP3 = -1.71512451000588188257046e-15f;
    const float kRound = 12582912.0f;                        // 1.5 * 2^23: adds to round to integer
    float t = fmaf(x, kTwoOverPi, kRound);
    int quad = __float_as_int(t);                            // low bits of t hold n (two's complement)
    float n = t - kRound;
    const float yhi = fmaf(-n, kP1, x);
    const float ylo = fmaf(-n, kP2, -n * kP3);
    const float y = yhi + ylo;
    const float d = ylo - (y - yhi);
    float y2 = y * y;
    // sin y = y + y^3 * (-1/3! + y^2 (1/5! + y^2 (-1/7! + y^2/9!)))
    float ps = fmaf(y2, 2.75573188446287531405687332153320312e-06f, -1.98412701138295233249664306640625e-04f);
    ps = fmaf(ps, y2, 8.33333376795053482055664062500000000e-03f);
    ps = fmaf(ps, y2, -1.66666671633720397949218750000000000e-01f);
    // cos y = 1 + y^2 (-1/2 + y^2 (1/4! + y^2 (-1/6! + y^2 (1/8! - y^2/10!))))
    float pc = fmaf(y2, -2.75573199814971303567290306091308594e-07f, 2.48015876422869041562080383300781250e-05f);
    pc = fmaf(pc, y2, -1.38888892251998186111450195312500000e-03f);
    pc = fmaf(pc, y2, 4.16666679084300994873046875000000000e-02f);
    pc = fmaf(pc, y2, -0.5f);
    const float cm1 = pc * y2;                              // cos y - 1
    const float sy = y + fmaf(ps * y2, y, fmaf(d, cm1, d));  // y + (y^3 P + d cos y)
    const float cy = 1.0f + fmaf(pc, y2, -d * y);            // 1 + (y^2 Q - d sin y)
    SinCos r;
    r.s = (quad & 1) ? cy : sy;
    r.c = (quad & 1) ? sy : cy;
    if (quad & 2) r.s = -r.s;
    if ((quad + 1) & 2) r.c = -r.c;
    return r;
}

}  // namespace sas

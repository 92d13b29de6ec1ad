// Single-precision sine and cosine on the FP32 FMA pipe (one argument, or two with packed
// f32x2 arithmetic).
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

// Constants of the reduction and of the polynomials.
namespace sc {
constexpr float kTwoOverPi = 0.636619746685028076171875f;   // float32(2/pi)
constexpr float kP1 = 1.57079637050628662109375f;            // float32(pi/2)
constexpr float kP2 = -4.37113882867379300296306610107421875e-08f;
constexpr float kP3 = -1.71512451000588188257046e-15f;
constexpr float kRound = 12582912.0f;                        // 1.5 * 2^23: adds to round to integer
// sin y = y + y^3 * (S3 + y^2 (S5 + y^2 (S7 + y^2 S9))),  Sk = (-1)^((k-1)/2) / k!
constexpr float kS9 = 2.75573188446287531405687332153320312e-06f;
constexpr float kS7 = -1.98412701138295233249664306640625e-04f;
constexpr float kS5 = 8.33333376795053482055664062500000000e-03f;
constexpr float kS3 = -1.66666671633720397949218750000000000e-01f;
// cos y = 1 + y^2 (C2 + y^2 (C4 + y^2 (C6 + y^2 (C8 + y^2 C10)))),  Ck = (-1)^(k/2) / k!
constexpr float kC10 = -2.75573199814971303567290306091308594e-07f;
constexpr float kC8 = 2.48015876422869041562080383300781250e-05f;
constexpr float kC6 = -1.38888892251998186111450195312500000e-03f;
constexpr float kC4 = 4.16666679084300994873046875000000000e-02f;
constexpr float kC2 = -0.5f;
}  // namespace sc

__device__ __forceinline__ SinCos sincos_f32(float x)
{
    using namespace sc;
    float t = fmaf(x, kTwoOverPi, kRound);
    int quad = __float_as_int(t);                            // low bits of t hold n (two's complement)
    float n = t - kRound;
    const float yhi = fmaf(-n, kP1, x);
    const float ylo = fmaf(-n, kP2, -n * kP3);
    const float y = yhi + ylo;
    const float d = ylo - (y - yhi);
    float y2 = y * y;
    float ps = fmaf(y2, kS9, kS7);
    ps = fmaf(ps, y2, kS5);
    ps = fmaf(ps, y2, kS3);
    float pc = fmaf(y2, kC10, kC8);
    pc = fmaf(pc, y2, kC6);
    pc = fmaf(pc, y2, kC4);
    pc = fmaf(pc, y2, kC2);
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

// Two arguments at once with packed FP32 arithmetic (one f32x2 instruction per step for both),
// the same operations and roundings as sincos_f32 lane by lane.  Negations are folded into
// constants or into multiplications by -1, which are exact.
struct SinCos2 {
    float2 s, c;
};

__device__ __forceinline__ float2 sc_bcast(float v) { return make_float2(v, v); }

// The quadrant of lane value `quad` applied to (sy, cy): swap, then sign flips on the sign bit.
__device__ __forceinline__ void sc_quadrant(int quad, float sy, float cy, float &s, float &c)
{
    const float a = (quad & 1) ? cy : sy, b = (quad & 1) ? sy : cy;
    s = __int_as_float(__float_as_int(a) ^ ((quad & 2) << 30));
    c = __int_as_float(__float_as_int(b) ^ (((quad + 1) & 2) << 30));
}

__device__ __forceinline__ SinCos2 sincos2_f32(float2 x)
{
    using namespace sc;
    const float2 t = __ffma2_rn(x, sc_bcast(kTwoOverPi), sc_bcast(kRound));
    const float2 n = __fadd2_rn(t, sc_bcast(-kRound));
    const float2 yhi = __ffma2_rn(n, sc_bcast(-kP1), x);
    const float2 ylo = __ffma2_rn(n, sc_bcast(-kP2), __fmul2_rn(n, sc_bcast(-kP3)));
    const float2 y = __fadd2_rn(yhi, ylo);
    const float2 e = __ffma2_rn(yhi, sc_bcast(-1.f), y);     // y - yhi
    const float2 d = __ffma2_rn(e, sc_bcast(-1.f), ylo);     // ylo - (y - yhi)
    const float2 nd = __ffma2_rn(ylo, sc_bcast(-1.f), e);    // -d
    const float2 y2 = __fmul2_rn(y, y);
    float2 ps = __ffma2_rn(y2, sc_bcast(kS9), sc_bcast(kS7));
    ps = __ffma2_rn(ps, y2, sc_bcast(kS5));
    ps = __ffma2_rn(ps, y2, sc_bcast(kS3));
    float2 pc = __ffma2_rn(y2, sc_bcast(kC10), sc_bcast(kC8));
    pc = __ffma2_rn(pc, y2, sc_bcast(kC6));
    pc = __ffma2_rn(pc, y2, sc_bcast(kC4));
    pc = __ffma2_rn(pc, y2, sc_bcast(kC2));
    const float2 cm1 = __fmul2_rn(pc, y2);
    const float2 sy = __fadd2_rn(y, __ffma2_rn(__fmul2_rn(ps, y2), y, __ffma2_rn(d, cm1, d)));
    const float2 cy = __fadd2_rn(sc_bcast(1.0f), __ffma2_rn(pc, y2, __fmul2_rn(nd, y)));
    SinCos2 r;
    sc_quadrant(__float_as_int(t.x), sy.x, cy.x, r.s.x, r.c.x);
    sc_quadrant(__float_as_int(t.y), sy.y, cy.y, r.s.y, r.c.y);
    return r;
}

// Table-driven sine and cosine of the per-pair phase step t = dq r >= 0, for passes whose t is
// bounded (dq times the molecule's diameter) so that a table of (sin, cos)(k/64) covers it:
//   t = k/64 + d, k the nearest integer to 64 t, |d| <= 1/128, d exact (Sterbenz);
//   sin t = S_k cos d + C_k sin d,  cos t = C_k cos d - S_k sin d,
//   sin d = d - d^3/6 and cos d = 1 - d^2/2 (truncation below 2^-32 relative for |d| <= 1/128).
// (S_k, C_k) come from FP64 and are stored as float32 pairs hi + lo, the lo part entering the
// innermost fused multiply-add: a table entry's own rounding, shared by every t near k/64, stays
// at 2^-48 instead of becoming a coherent float32 error.  The result's errors are the roundings of
// a few products, which vary with t.  Entry k = (S_hi, C_hi, S_lo, C_lo); k is clamped to the n
// entries.  The packed form performs the same operations lane by lane.
namespace sc {
constexpr float kSixth = 0.16666667163372039794921875f;   // float32(1/6)
constexpr float kTabScale = 64.f;
constexpr float kTabStep = 0.015625f;                      // 1/64
}  // namespace sc

__device__ __forceinline__ SinCos sincos_tab(float t, const float4 *__restrict__ tab, int n)
{
    using namespace sc;
    const float kr = __fmaf_rn(t, kTabScale, kRound);   // nearest integer in the low mantissa bits
    const float kf = __fadd_rn(kr, -kRound);
    const float d = __fmaf_rn(kf, -kTabStep, t);
    const int k = min(max(__float_as_int(kr) - __float_as_int(kRound), 0), n - 1);
    const float4 e = __ldg(tab + k);
    const float d2 = __fmul_rn(d, d);
    const float d3 = __fmul_rn(d2, d);
    const float sd = __fmaf_rn(d3, -kSixth, d);
    const float nsd = __fmul_rn(sd, -1.f);
    const float cd = __fmaf_rn(d2, -0.5f, 1.f);
    SinCos r;
    r.s = __fmaf_rn(e.x, cd, __fmaf_rn(e.y, sd, e.z));
    r.c = __fmaf_rn(e.y, cd, __fmaf_rn(e.x, nsd, e.w));
    return r;
}

__device__ __forceinline__ SinCos2 sincos2_tab(float2 t, const float4 *__restrict__ tab, int n)
{
    using namespace sc;
    const float2 kr = __ffma2_rn(t, sc_bcast(kTabScale), sc_bcast(kRound));
    const float2 kf = __fadd2_rn(kr, sc_bcast(-kRound));
    const float2 d = __ffma2_rn(kf, sc_bcast(-kTabStep), t);
    const int kA = min(max(__float_as_int(kr.x) - __float_as_int(kRound), 0), n - 1);
    const int kB = min(max(__float_as_int(kr.y) - __float_as_int(kRound), 0), n - 1);
    const float4 eA = tab[kA], eB = tab[kB];   // a shared-memory copy or the global table
    const float2 d2 = __fmul2_rn(d, d);
    const float2 d3 = __fmul2_rn(d2, d);
    const float2 sd = __ffma2_rn(d3, sc_bcast(-kSixth), d);
    const float2 nsd = __fmul2_rn(sd, sc_bcast(-1.f));
    const float2 cd = __ffma2_rn(d2, sc_bcast(-0.5f), sc_bcast(1.f));
    const float2 Sh = make_float2(eA.x, eB.x), Ch = make_float2(eA.y, eB.y);
    SinCos2 r;
    r.s = __ffma2_rn(Sh, cd, __ffma2_rn(Ch, sd, make_float2(eA.z, eB.z)));
    r.c = __ffma2_rn(Ch, cd, __ffma2_rn(Sh, nsd, make_float2(eA.w, eB.w)));
    return r;
}

}  // namespace sas

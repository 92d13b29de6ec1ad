// Set-up of two pairs (i, j) and (i, j+1) for the packed FP32 recurrence of the Debye sum
// (Section I-A, Eq. 2), shared by the typed and the per-atom two-pair kernels: the distance, the
// seeds of the first two float2 blocks and the stochastically rounded coefficient 2cos(2t).
// Lane 0 of every packed value is pair A = (i, j), lane 1 pair B = (i, j+1).
#pragma once
#include "mixed_common.cuh"
#include "sincos_f32.cuh"

namespace sas {
namespace mixed {

__device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }

// Two pairs (A = lane 0, B = lane 1) after set-up: their first two float2 blocks and their
// coefficients 2cos(2t) as (+C, +C) and (-C, -C).
struct PairState2 {
    float2 w0A, w1A, w0B, w1B;
    float2 CpA, CnA, CpB, CnB;
};

// First part of the set-up of two pairs: distance (reciprocal square root and one Newton step)
// and weight.  It holds the long latencies (shared-memory loads, MUFU), so the pair loop issues it
// one step ahead, next to the previous recurrences.
struct PairHead2 {
    float2 y, r, w;   // 1/r (hardware), r, w_i w_j (0: no pair)
};

__device__ __forceinline__ void setup2_head(const float4 pxy, const float4 pzw, const float2 nX, const float2 nY,
                                            const float2 nZ, const float2 wi, bool keepA, bool keepB, PairHead2 &h)
{
    // x_j - x_i (the negated difference: its square is the same)
    const float2 dx = f2add(make_float2(pxy.x, pxy.y), nX);
    const float2 dy = f2add(make_float2(pxy.z, pxy.w), nY);
    const float2 dz = f2add(make_float2(pzw.x, pzw.y), nZ);
    float2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));
    r2.x = fmaxf(r2.x, 1e-12f);   // coincident atoms: r = 1e-6 A
    r2.y = fmaxf(r2.y, 1e-12f);
    h.y = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 r0 = f2mul(r2, h.y);
    // r = r0 + (y/2)(r2 - r0^2), as (-y/2)(r0^2 - r2) + r0
    h.r = f2fma(f2mul(h.y, bc(-0.5f)), f2fma(r0, r0, f2mul(r2, bc(-1.f))), r0);
    h.w = f2mul(wi, make_float2(pzw.z, pzw.w));
    if (!keepA) h.w.x = 0.f;
    if (!keepB) h.w.y = 0.f;
}

// Second part: sin t, cos t of t = dq r, the seeds of the first two blocks and the coefficient.
// TAB: 0 the polynomial sin/cos alone; 1 the table of (sin, cos)(k/64) of the call alone (sct, not
// null; sincos2_tab); 2 the table where sct is not null, else the polynomial (both compiled).  Which
// compiles to the faster kernel differs by form, so each kernel picks its own (measured).
// PRODUCT_SEEDS (zero start only): the seeds from the scaled sine and 4 sin^2 t, which the
// coefficient needs anyway: scale sin 2t = (2 scale sin t) cos t and scale sin 3t =
// (scale sin t)(3 - 4 sin^2 t), four packed operations fewer than by angle addition.  Used by the
// 208-q form, where it measured faster (1 %); the 104-q form measured 2-3 % slower with it.
// COEF_BOTH: the coefficient formed both ways (QChunks::coef_both; a template parameter, so that
// the kernels of calls without it are the one-form code).
// START_IS_STEP (offset start only): the chunk's first q equals its step, so the start phase is t.
template <bool ZERO_START, int TAB = 2, bool PRODUCT_SEEDS = false, bool COEF_BOTH = false, bool START_IS_STEP = false>
__device__ __forceinline__ void setup2_tail(const PairHead2 &h, float2 qs_hi, float2 qs_lo, float2 dq_hi,
                                            float2 dq_lo, unsigned hA, unsigned hB, PairState2 &o,
                                            const float4 *__restrict__ sct, int sct_n)
{
    const float2 r = h.r;
    const float2 scale = f2mul(h.w, h.y);
    const float2 t = f2fma(dq_hi, r, f2mul(dq_lo, r));
    const SinCos2 b1 = (TAB == 1 || (TAB == 2 && sct)) ? sincos2_tab(t, sct, sct_n) : sincos2_f32(t);
    const float2 s1 = b1.s, c1 = b1.c;
    const float2 s1x2 = f2add(s1, s1);
    // 2cos(2t), rounded stochastically (dither from the pair hash)
    const float2 mu = f2mul(s1x2, s1x2);
    const float2 u = f2add(make_float2(__int_as_float(0x3f800000u | (hA >> 9)),
                                       __int_as_float(0x3f800000u | (hB >> 9))),
                           bc(-1.5f));
    // the small square that keeps full relative accuracy (coef_dither): 4 sin^2 t where cos 2t >= 0,
    // 4 cos^2 t where cos 2t < 0, the coefficient then 2 - 4 sin^2 t or 4 cos^2 t - 2 (calls with
    // coef_both; the others 2 - 4 sin^2 t alone)
    float2 C, Cn;
    if (COEF_BOTH) {
        const float2 c1x2 = f2add(c1, c1);
        const float2 mc = f2mul(c1x2, c1x2);
        const bool nA = mu.x > mc.x, nB = mu.y > mc.y;
        const float2 md = f2fma(u, bc(1.1920928955078125e-7f), make_float2(nA ? mc.x : mu.x, nB ? mc.y : mu.y));
        const float2 two_minus = f2fma(md, bc(-1.f), bc(2.f)), minus_two = f2add(md, bc(-2.f));
        C = make_float2(nA ? minus_two.x : two_minus.x, nB ? minus_two.y : two_minus.y);
        Cn = make_float2(nA ? two_minus.x : minus_two.x, nB ? two_minus.y : minus_two.y);
    } else {
        const float2 md = f2fma(u, bc(1.1920928955078125e-7f), mu);
        C = f2fma(md, bc(-1.f), bc(2.f));
        Cn = f2add(md, bc(-2.f));
    }
    o.CpA = bc(C.x);
    o.CpB = bc(C.y);
    o.CnA = bc(Cn.x);
    o.CnB = bc(Cn.y);
    if (ZERO_START && PRODUCT_SEEDS) {
        const float2 a1 = f2mul(scale, s1);
        const float2 a2 = f2mul(f2add(a1, a1), c1), a3 = f2mul(a1, f2fma(mu, bc(-1.f), bc(3.f)));
        o.w0A = make_float2(0.f, a1.x);
        o.w0B = make_float2(0.f, a1.y);
        o.w1A = make_float2(a2.x, a3.x);
        o.w1B = make_float2(a2.y, a3.y);
        return;
    }
    const float2 s2 = f2mul(s1x2, c1);
    const float2 c2 = f2fma(f2mul(s1, bc(-2.f)), s1, bc(1.f));
    const float2 s3 = f2fma(s2, c1, f2mul(c2, s1));
    if (ZERO_START) {
        const float2 a1 = f2mul(scale, s1), a2 = f2mul(scale, s2), a3 = f2mul(scale, s3);
        o.w0A = make_float2(0.f, a1.x);
        o.w0B = make_float2(0.f, a1.y);
        o.w1A = make_float2(a2.x, a3.x);
        o.w1B = make_float2(a2.y, a3.y);
    } else {
        const float2 c3 = f2fma(c2, c1, f2mul(s2, f2mul(s1, bc(-1.f))));
        // the start phase q0 r (START_IS_STEP: the step phase t, at hand)
        SinCos2 ph;
        if (START_IS_STEP) {
            ph.s = s1;
            ph.c = c1;
        } else {
            ph = sincos2_f32(f2fma(qs_hi, r, f2mul(qs_lo, r)));
        }
        const float2 S = f2mul(scale, ph.s), Cc = f2mul(scale, ph.c);
        const float2 v1 = f2fma(S, c1, f2mul(Cc, s1));
        const float2 v2 = f2fma(S, c2, f2mul(Cc, s2));
        const float2 v3 = f2fma(S, c3, f2mul(Cc, s3));
        o.w0A = make_float2(S.x, v1.x);
        o.w0B = make_float2(S.y, v1.y);
        o.w1A = make_float2(v2.x, v3.x);
        o.w1B = make_float2(v2.y, v3.y);
    }
}

}  // namespace mixed
}  // namespace sas

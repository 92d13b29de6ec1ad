// Device helpers shared by the mixed-precision pair kernels (debye_mixed.cu and
// debye_mixed_pairs2.cu): packed FP32 arithmetic, the sign pattern of the
// three-term recurrence, the stochastic rounding of its coefficient, the pair
// hash, and the FP64 warp reduce-scatter of the per-thread q accumulators.
#pragma once
#include "sas_internal.h"

namespace sas {
namespace mixed {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }

// sign of block b in the (+, +, -, -) pattern, and of the coefficient of the step b -> b+1
__host__ __device__ constexpr bool block_negative(int b) { return (b & 2) != 0; }
__host__ __device__ constexpr bool step_negative(int b) { return (b & 1) != 0; }

// r = sqrt(r2) from the reciprocal square root and one Newton correction (to about 1 ulp);
// y = 1/sqrt(r2) as computed by the hardware.
__device__ __forceinline__ void dist_rsqrt(float r2, float &r, float &y)
{
    y = rsqrtf(r2);
    const float r0 = r2 * y;
    r = fmaf(0.5f * y, fmaf(-r0, r0, r2), r0);
}

// The coefficient 2cos(2x) of the recurrence from s = sin x, c = cos x, rounded stochastically.
// It is formed from whichever small square keeps full relative accuracy: 2 - 4s^2 where
// cos 2x >= 0 (the 4s^2 <= 4c^2 side, where it nears +2 as x nears a multiple of pi) and
// 4c^2 - 2 where cos 2x < 0 (where it nears -2).  Near -2 the form 2 - 4s^2 would take the
// rounding of s and of a square near 4 into the coefficient, several ulps that the recurrence
// turns into a phase drift shared by every pair of about the same distance.  A uniform offset of
// at most half an ulp of [1, 2) enters the small square before the last rounding, so the expected
// coefficient is exact (pairs at one distance, such as bonds, then do not share its rounding).
// Returns +C in Cp and -C in Cn.  both = 0 (calls whose step phase 2x stays below 0.8 pi, where the
// coefficient stays above -1.62 and 2 - 4s^2 is accurate enough): the first form alone.
__device__ __forceinline__ void coef_dither(float s, float c, unsigned hash, bool both, float &Cp, float &Cn)
{
    const float u = __int_as_float(0x3f800000u | (hash >> 9)) - 1.5f;   // uniform in [-0.5, 0.5)
    const float ms = (2.f * s) * (2.f * s);
    if (both) {
        const float mc = (2.f * c) * (2.f * c);
        const bool near_minus2 = ms > mc;
        const float md = fmaf(u, 1.1920928955078125e-7f, near_minus2 ? mc : ms);
        const float two_minus = 2.f - md, minus_two = md - 2.f;
        Cp = near_minus2 ? minus_two : two_minus;
        Cn = near_minus2 ? two_minus : minus_two;
    } else {
        const float md = fmaf(u, 1.1920928955078125e-7f, ms);
        Cp = 2.f - md;
        Cn = md - 2.f;
    }
}

// Cheap pair hash on the integer ALU (one multiply, then xorshift).
__device__ __forceinline__ unsigned pair_hash(unsigned i, unsigned j)
{
    unsigned h = i ^ (j * 0x9E3779B1u);
    h ^= h << 13;
    h ^= h >> 17;
    h ^= h << 5;
    return h;
}

// ---------------------------------------------------------------------------------------------
// FP64 warp reduce-scatter of the accumulators
// ---------------------------------------------------------------------------------------------

// Number of halving levels of the reduce-scatter for V values (at most 5, while V stays even).
__host__ __device__ constexpr int halvings(int V, int lvl = 0)
{
    return (lvl < 5 && V % 2 == 0) ? halvings(V / 2, lvl + 1) : lvl;
}

// One halving level: lanes with `up` keep the upper half of the H values, add the partner's.
template <int H, int N>
__device__ __forceinline__ void halve(double (&d)[N], bool up, int off)
{
#pragma unroll
    for (int k = 0; k < H / 2; ++k) {
        const double lo = d[k], hi = d[k + H / 2];
        const double mine = up ? hi : lo, other = up ? lo : hi;
        d[k] = mine + __shfl_xor_sync(kFull, other, off);
    }
}

// Accumulator k (q index k of the chunk) with its block sign applied.
template <int NB, int M>
__device__ __forceinline__ float acc_signed(const float2 (&acc)[2 * NB], int k)
{
    const float v = (k & 1) ? acc[k >> 1].y : acc[k >> 1].x;
    return block_negative(k / M) ? -v : v;
}

// Sum the 32 lanes' V = 4*NB accumulators (FP64 from the first cross-thread add on);
// the warp's totals land in red[0..V).
template <int NB, int M>
__device__ __forceinline__ void flush_warp(const float2 (&acc)[2 * NB], double *red, int lane)
{
    constexpr int V = 4 * NB;
    constexpr int L = halvings(V);   // reduce-scatter levels (offsets 16, 8, ...)
    constexpr int H1 = V / 2;
    constexpr int R = V >> L;        // values per lane after the reduce-scatter
    double d[H1];
    const bool up16 = lane & 16;
#pragma unroll
    for (int k = 0; k < H1; ++k) {   // the lift to FP64
        const float lo = acc_signed<NB, M>(acc, k), hi = acc_signed<NB, M>(acc, k + H1);
        const float mine = up16 ? hi : lo, other = up16 ? lo : hi;
        d[k] = (double)mine + (double)__shfl_xor_sync(kFull, other, 16);
    }
    if (L > 1) halve<(V >> 1), H1>(d, lane & 8, 8);
    if (L > 2) halve<(V >> 2), H1>(d, lane & 4, 4);
    if (L > 3) halve<(V >> 3), H1>(d, lane & 2, 2);
    if (L > 4) halve<(V >> 4), H1>(d, lane & 1, 1);
    // the lane bits not used for scattering: plain butterfly over the R remaining values
#pragma unroll
    for (int b = L; b < 5; ++b) {
        const int off = 16 >> b;
#pragma unroll
        for (int k = 0; k < R; ++k) d[k] += __shfl_xor_sync(kFull, d[k], off);
    }
    int base = 0;
#pragma unroll
    for (int b = 0; b < L; ++b)
        if (lane & (16 >> b)) base += V >> (b + 1);
    const int keep_mask = (1 << (5 - L)) - 1;   // lanes that differ only in butterfly bits hold copies
    if ((lane & keep_mask) == 0) {
#pragma unroll
        for (int k = 0; k < R; ++k) red[base + k] = d[k];
    }
}

// Resident CTAs per SM: the accumulators (4*NB floats per thread) set the register budget.
__host__ __device__ constexpr int mixed_ctas_per_sm(int NB) { return NB <= 13 ? 4 : (NB <= 26 ? 3 : 2); }

}  // namespace mixed
}  // namespace sas

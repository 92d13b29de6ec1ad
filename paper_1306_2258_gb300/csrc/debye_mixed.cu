// Mixed-precision pair kernel: the hot loop of the Debye sum (Section I-A,
// Eq. 2) over the unordered pairs i<j of one work item, for one chunk of the
// uniform q grid.
//
// The paper's kernel (Section II, Fig. 2) gives each worker one atom in
// private memory, stages a block of atoms in local memory, and walks q in the
// outermost loop, two q values per pass, because its local memory could not
// hold more.  Here q is the innermost loop instead: the distance of a pair is
// computed once and the whole q chunk is walked from it.
//
//  * One thread owns atom i of the item's I-tile (128 threads, 128 atoms) and
//    streams the item's J-range from shared memory (coalesced float4 loads,
//    broadcast reads).
//  * For each pair it computes r once, then generates w_i w_j sin(q_k r)/r for
//    every q_k of the chunk with the three-term angle-addition identity
//        sin(x + 4t) = 2 cos(4t) sin(x) - sin(x - 4t),   t = dq * r,
//    applied to four interleaved sequences (q_k, q_k+1, q_k+2, q_k+3) held as
//    two float2 values: one packed FP32 fused multiply-add per two q values,
//    and one packed FP32 add to accumulate them.  Stepping by 4t instead of t
//    keeps 2cos(4t) away from 2 for near pairs (small t), where the rounding
//    of the coefficient would otherwise make the phase drift.
//  * Seeds (the first eight q of a segment) come from an accurate FP32
//    sin/cos of the segment's start phase and of t, combined by angle
//    addition.  The sequence is re-seeded every RB blocks of four q (RB = 0:
//    only at the chunk start).
//  * The per-thread sums are FP32 over the item's J-range (one tile of the
//    precision pattern), then lifted to FP64 for a warp reduce-scatter with
//    shuffles and a fixed-order block sum; one FP64 partial per item and q.
#include "sas_internal.h"
#include "sincos_f32.cuh"

namespace sas {

namespace {

constexpr int NB = kQChunk / 4;   // blocks of four q values per chunk (52)
constexpr int NV = kQChunk;       // accumulators per thread (208 floats)
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }

// cos(j t), sin(j t) for j = 1..7 by angle addition and doubling (no 1/sin(t) amplification).
struct Multiples {
    float c[8], s[8];
};

__device__ __forceinline__ void multiples(float c1, float s1, Multiples &m)
{
    m.c[0] = 1.f;
    m.s[0] = 0.f;
    m.c[1] = c1;
    m.s[1] = s1;
    m.s[2] = 2.f * s1 * c1;
    m.c[2] = fmaf(-2.f * s1, s1, 1.f);
    m.c[3] = fmaf(m.c[2], c1, -m.s[2] * s1);
    m.s[3] = fmaf(m.s[2], c1, m.c[2] * s1);
    m.s[4] = 2.f * m.s[2] * m.c[2];
    m.c[4] = fmaf(-2.f * m.s[2], m.s[2], 1.f);
    m.c[5] = fmaf(m.c[4], c1, -m.s[4] * s1);
    m.s[5] = fmaf(m.s[4], c1, m.c[4] * s1);
    m.s[6] = 2.f * m.s[3] * m.c[3];
    m.c[6] = fmaf(-2.f * m.s[3], m.s[3], 1.f);
    m.c[7] = fmaf(m.c[6], c1, -m.s[6] * s1);
    m.s[7] = fmaf(m.s[6], c1, m.c[6] * s1);
}

// Eight consecutive terms S cos(j t) + C sin(j t), j = 0..7, as four float2.
__device__ __forceinline__ void seed8(float S, float C, const Multiples &m, float2 &p0, float2 &p1,
                                      float2 &c0, float2 &c1)
{
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = fmaf(S, m.c[j], C * m.s[j]);
    p0 = make_float2(v[0], v[1]);
    p1 = make_float2(v[2], v[3]);
    c0 = make_float2(v[4], v[5]);
    c1 = make_float2(v[6], v[7]);
}

template <int RB>
__device__ __forceinline__ void pair_terms(const float4 xi, const float4 xj, float w, float qs_hi,
                                           float qs_lo, bool zero_start, float dq_hi, float dq_lo,
                                           float2 (&acc)[2 * NB])
{
    const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
    float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    r2 = fmaxf(r2, 1e-12f);            // coincident atoms: r = 1e-6 A, sin(q r)/r -> q
    const float r = sqrtf(r2);
    const float scale = w * rsqrtf(r2); // amplitude w_i w_j / r (phase uses the rounded sqrt)
    const float t = fmaf(dq_hi, r, dq_lo * r);
    const SinCos b1 = sincos_f32(t);
    Multiples m;
    multiples(b1.c, b1.s, m);
    const float C4 = 2.f * m.c[4];      // 2 cos(4t)
    const float2 C42 = make_float2(C4, C4);
    float S, C;
    if (zero_start) {
        S = 0.f;
        C = scale;
    } else {
        const SinCos ph = sincos_f32(fmaf(qs_hi, r, qs_lo * r));
        S = scale * ph.s;
        C = scale * ph.c;
    }
    constexpr int SEGB = RB > 0 ? RB : NB;              // blocks per segment
    float cK = 1.f, sK = 0.f;
    if (SEGB < NB) {
        const SinCos k = sincos_f32(t * (float)(4 * SEGB));
        cK = k.c;
        sK = k.s;
    }
    float2 p0, p1, c0, c1;
#pragma unroll
    for (int blk = 0; blk < NB; ++blk) {
        if (blk % SEGB == 0) {        // segment start: seed blocks blk and blk+1
            if (blk > 0) {            // advance the segment phase by 4*SEGB*t
                const float S2 = fmaf(S, cK, C * sK);
                C = fmaf(C, cK, -S * sK);
                S = S2;
            }
            seed8(S, C, m, p0, p1, c0, c1);
            acc[2 * blk] = f2add(acc[2 * blk], p0);
            acc[2 * blk + 1] = f2add(acc[2 * blk + 1], p1);
        } else if (blk % SEGB == 1) {
            acc[2 * blk] = f2add(acc[2 * blk], c0);
            acc[2 * blk + 1] = f2add(acc[2 * blk + 1], c1);
        } else {
            const float2 n0 = f2fma(C42, c0, f2neg(p0));
            const float2 n1 = f2fma(C42, c1, f2neg(p1));
            acc[2 * blk] = f2add(acc[2 * blk], n0);
            acc[2 * blk + 1] = f2add(acc[2 * blk + 1], n1);
            p0 = c0;
            p1 = c1;
            c0 = n0;
            c1 = n1;
        }
    }
}

__device__ __forceinline__ float acc_elem(const float2 (&acc)[2 * NB], int k)
{
    return (k & 1) ? acc[k >> 1].y : acc[k >> 1].x;
}

// One halving level of the FP64 warp reduce-scatter: lanes with `up` keep the upper half.
template <int H>
__device__ __forceinline__ void halve(double (&d)[NV / 2], bool up, int off)
{
#pragma unroll
    for (int k = 0; k < H / 2; ++k) {
        const double lo = d[k], hi = d[k + H / 2];
        const double mine = up ? hi : lo, other = up ? lo : hi;
        d[k] = mine + __shfl_xor_sync(kFull, other, off);
    }
}

// Sum the 32 lanes' accumulators; the warp's totals land in red[0..NV).
__device__ __forceinline__ void flush_warp(const float2 (&acc)[2 * NB], double *red, int lane)
{
    constexpr int H1 = NV / 2;   // 104
    double d[H1];
    const bool up16 = lane & 16;
#pragma unroll
    for (int k = 0; k < H1; ++k) {   // lift to FP64 at the first cross-thread sum
        const float lo = acc_elem(acc, k), hi = acc_elem(acc, k + H1);
        const float mine = up16 ? hi : lo, other = up16 ? lo : hi;
        d[k] = (double)mine + (double)__shfl_xor_sync(kFull, other, 16);
    }
    halve<H1>(d, lane & 8, 8);        // 104 -> 52
    halve<H1 / 2>(d, lane & 4, 4);    // 52 -> 26
    halve<H1 / 4>(d, lane & 2, 2);    // 26 -> 13
    constexpr int R = H1 / 8;         // 13
#pragma unroll
    for (int k = 0; k < R; ++k) d[k] += __shfl_xor_sync(kFull, d[k], 1);
    const int off = ((lane & 16) ? H1 : 0) + ((lane & 8) ? H1 / 2 : 0) + ((lane & 4) ? H1 / 4 : 0) +
                    ((lane & 2) ? R : 0);
    if ((lane & 1) == 0) {
#pragma unroll
        for (int k = 0; k < R; ++k) red[off + k] = d[k];
    }
}

template <int RB>
__global__ void __launch_bounds__(kTile, 2)
    k_debye_mixed(const float4 *__restrict__ X, int64_t npad, const Item *__restrict__ items,
                  int n_items, QChunks qc, double *__restrict__ partial, int part_stride)
{
    extern __shared__ float4 sj[];
    __shared__ double red[kTile / 32][NV];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const Item item = items[it];
        const float4 *Xb = X + (int64_t)item.batch * npad;
        __syncthreads();   // the previous item is done with sj and red
        for (int j = tid; j < item.jlen; j += kTile) sj[j] = Xb[item.j0 + j];
        const float4 xi = Xb[item.i0 + tid];
        __syncthreads();
        const int ch = item.chunk;
        const float qs_hi = qc.qs_hi[ch], qs_lo = qc.qs_lo[ch];
        const bool zero_start = (qs_hi == 0.f) && (qs_lo == 0.f);
        float2 acc[2 * NB];
#pragma unroll
        for (int k = 0; k < 2 * NB; ++k) acc[k] = make_float2(0.f, 0.f);
        const int jmask = item.diag ? tid : -1;   // pairs with j <= i are not pairs of i<j
        for (int j = 0; j < item.jlen; ++j) {
            const float4 xj = sj[j];
            const float w = (j <= jmask) ? 0.f : xi.w * xj.w;
            pair_terms<RB>(xi, xj, w, qs_hi, qs_lo, zero_start, qc.dq_hi, qc.dq_lo, acc);
        }
        flush_warp(acc, red[warp], lane);
        __syncthreads();
        const int qlen = qc.q_len[ch];
        for (int k = tid; k < qlen; k += kTile) {
            double s = red[0][k];
#pragma unroll
            for (int w = 1; w < kTile / 32; ++w) s += red[w][k];
            partial[(int64_t)it * part_stride + k] = s;
        }
    }
}

template <int RB>
cudaError_t launch_rb(const float4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                      double *partial, int part_stride, int grid, int jmax, cudaStream_t s)
{
    const size_t smem = (size_t)jmax * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(k_debye_mixed<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_debye_mixed<RB><<<grid, kTile, smem, s>>>(X, npad, items, n_items, qc, partial, part_stride);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_debye_mixed(const float4 *X, int64_t npad, const Item *items, int n_items,
                               const QChunks &qc, int reseed, double *partial, int part_stride,
                               int grid, int jmax, cudaStream_t s)
{
    if (n_items == 0) return cudaSuccess;
    switch (reseed) {
    case 32:
        return launch_rb<8>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, s);
    case 64:
        return launch_rb<16>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, s);
    default:
        return launch_rb<0>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, s);
    }
}

}  // namespace sas

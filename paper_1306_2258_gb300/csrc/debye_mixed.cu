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
//        sin(x + Mt) = 2 cos(Mt) sin(x) - sin(x - Mt),   t = dq * r,
//    applied to M interleaved sequences (M = 2 or 4) held as float2 values:
//    one packed FP32 fused multiply-add per two q values, and one packed FP32
//    add to accumulate them.  A step of Mt instead of t keeps 2cos(Mt) away
//    from 2 for near pairs (small t), where the rounding of the coefficient
//    would otherwise make the phase drift.
//  * The coefficient 2cos(Mt) is rounded stochastically (unbiased, seeded by a
//    hash of the pair's slots): molecules hold thousands of pairs at the same
//    distance (bonds), whose identical rounding errors would otherwise drift
//    in phase together.
//  * The identity is ill-conditioned wherever Mt is near a multiple of pi
//    (errors grow like 1/sin(Mt) per step), so the sequences are re-seeded
//    with exact values every KQ q values: the segment's start phase advances
//    by an exact rotation through K t, and the first 2M values of a segment
//    are S cos(jt) + C sin(jt) with cos(jt), sin(jt) from an accurate FP32
//    sin/cos of t and angle addition.
//  * The per-thread sums are FP32 over the item's J-range (one tile of the
//    precision pattern), then lifted to FP64 for a warp reduce-scatter with
//    shuffles and a fixed-order block sum; one FP64 partial per item and q.
#include "sas_internal.h"
#include "sincos_f32.cuh"

namespace sas {

namespace {

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

// 2 cos(M t) = 2 - mu rounded to float32 stochastically: up or down with the probabilities that
// make its expected value exact, decided by the pair's hash.  Pairs with equal distances (bonds)
// would otherwise share one rounding error of the coefficient, and their phase drifts would add
// up coherently instead of averaging out.
__device__ __forceinline__ float coef_sr(float mu, unsigned hash)
{
    const float c = 2.f - mu;                        // nearest float32
    const float e = (2.f - c) - mu;                  // remaining error: exact value ~ c + e
    const float ulp = __int_as_float(__float_as_int(fabsf(c)) & 0x7f800000) * 1.1920928955078125e-7f;
    const float u = (float)(hash >> 8) * 5.9604644775390625e-8f;   // uniform in [0, 1)
    return (u * ulp < fabsf(e)) ? c + copysignf(ulp, e) : c;
}

__device__ __forceinline__ unsigned pair_hash(unsigned i, unsigned j)
{
    unsigned h = i * 0x9E3779B1u ^ (j * 0x85EBCA77u + 0x165667B1u);
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return h;
}

// Terms of one pair for the q values of a chunk, added into acc (float2 slot v holds q = 2v, 2v+1).
//   M  : recurrence step in q values (2 or 4): u_{k+M} = 2 cos(M t) u_k - u_{k-M}
//   KQ : re-seed interval in q values (0: only at the chunk start), a multiple of 2M
template <int NB, int M, int KQ>
__device__ __forceinline__ void pair_terms(const float4 xi, const float4 xj, float w, float qs_hi,
                                           float qs_lo, bool zero_start, float dq_hi, float dq_lo,
                                           unsigned hash, float2 (&acc)[2 * NB])
{
    static_assert(M == 2 || M == 4, "step must be 2 or 4");
    static_assert(KQ == 0 || KQ % (2 * M) == 0, "re-seed interval must be a multiple of 2M");
    constexpr int G = M / 2;                          // float2 per block of M values
    constexpr int NBM = 4 * NB / M;                   // blocks of M values per chunk
    constexpr int SEG = (KQ > 0 && KQ / M < NBM) ? KQ / M : NBM;   // blocks per segment
    const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
    float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    r2 = fmaxf(r2, 1e-12f);            // coincident atoms: r = 1e-6 A, sin(q r)/r -> q
    const float r = sqrtf(r2);
    const float scale = w * rsqrtf(r2); // amplitude w_i w_j / r (the phase uses the rounded sqrt)
    const float t = fmaf(dq_hi, r, dq_lo * r);
    const SinCos b1 = sincos_f32(t);
    Multiples m;
    multiples(b1.c, b1.s, m);
    // 2 cos(M t) = 2 - 4 sin^2(M t / 2), the small term kept with full relative accuracy
    const float sh = m.s[M / 2];
    const float CM = coef_sr(4.f * sh * sh, hash);
    const float2 CM2 = make_float2(CM, CM);
    float S, C;
    if (zero_start) {
        S = 0.f;
        C = scale;
    } else {
        const SinCos ph = sincos_f32(fmaf(qs_hi, r, qs_lo * r));
        S = scale * ph.s;
        C = scale * ph.c;
    }
    float cK = 1.f, sK = 0.f;
    if (SEG < NBM) {   // rotation of the segment start phase by (M*SEG) t
        const SinCos k = sincos_f32(t * (float)(M * SEG));
        cK = k.c;
        sK = k.s;
    }
    float2 prev[G], cur[G];
#pragma unroll
    for (int blk = 0; blk < NBM; ++blk) {
        const int v0 = blk * G;
        if (blk % SEG == 0) {        // segment start: exact values for blocks blk and blk+1
            if (blk > 0) {
                const float S2 = fmaf(S, cK, C * sK);
                C = fmaf(C, cK, -S * sK);
                S = S2;
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                prev[g] = make_float2(fmaf(S, m.c[2 * g], C * m.s[2 * g]),
                                      fmaf(S, m.c[2 * g + 1], C * m.s[2 * g + 1]));
                cur[g] = make_float2(fmaf(S, m.c[M + 2 * g], C * m.s[M + 2 * g]),
                                     fmaf(S, m.c[M + 2 * g + 1], C * m.s[M + 2 * g + 1]));
                acc[v0 + g] = f2add(acc[v0 + g], prev[g]);
            }
        } else if (blk % SEG == 1) {
#pragma unroll
            for (int g = 0; g < G; ++g) acc[v0 + g] = f2add(acc[v0 + g], cur[g]);
        } else {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const float2 n = f2fma(CM2, cur[g], f2neg(prev[g]));
                acc[v0 + g] = f2add(acc[v0 + g], n);
                prev[g] = cur[g];
                cur[g] = n;
            }
        }
    }
}

template <int NB>
__device__ __forceinline__ float acc_elem(const float2 (&acc)[2 * NB], int k)
{
    return (k & 1) ? acc[k >> 1].y : acc[k >> 1].x;
}

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

// Sum the 32 lanes' V = 4*NB accumulators (FP64 from the first cross-thread add on);
// the warp's totals land in red[0..V).
template <int NB>
__device__ __forceinline__ void flush_warp(const float2 (&acc)[2 * NB], double *red, int lane)
{
    constexpr int V = 4 * NB;
    constexpr int L = halvings(V);      // reduce-scatter levels (offsets 16, 8, ...)
    constexpr int H1 = V / 2;
    constexpr int R = V >> L;           // values per lane after the reduce-scatter
    double d[H1];
    const bool up16 = lane & 16;
#pragma unroll
    for (int k = 0; k < H1; ++k) {      // the lift to FP64
        const float lo = acc_elem<NB>(acc, k), hi = acc_elem<NB>(acc, k + H1);
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

template <int NB, int M, int KQ>
__global__ void __launch_bounds__(kTile, 2)
    k_debye_mixed(const float4 *__restrict__ X, int64_t npad, const Item *__restrict__ items,
                  int n_items, QChunks qc, double *__restrict__ partial, int part_stride)
{
    extern __shared__ float4 sj[];
    __shared__ double red[kTile / 32][4 * NB];
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
            pair_terms<NB, M, KQ>(xi, xj, w, qs_hi, qs_lo, zero_start, qc.dq_hi, qc.dq_lo,
                                  pair_hash(item.i0 + tid, item.j0 + j), acc);
        }
        flush_warp<NB>(acc, red[warp], lane);
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

template <int NB, int M, int KQ>
cudaError_t launch_v(const float4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                     double *partial, int part_stride, int grid, int jmax, cudaStream_t s)
{
    const size_t smem = (size_t)jmax * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(k_debye_mixed<NB, M, KQ>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_debye_mixed<NB, M, KQ><<<grid, kTile, smem, s>>>(X, npad, items, n_items, qc, partial, part_stride);
    return cudaGetLastError();
}

template <int NB, int M>
cudaError_t launch_k(const float4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                     int reseed, double *partial, int part_stride, int grid, int jmax, cudaStream_t s)
{
    switch (reseed) {
    case 32:
        return launch_v<NB, M, 32>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, s);
    case 64:
        return launch_v<NB, M, 64>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, s);
    default:
        return launch_v<NB, M, 0>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, s);
    }
}

template <int NB>
cudaError_t launch_nb(const float4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                      int step, int reseed, double *partial, int part_stride, int grid, int jmax,
                      cudaStream_t s)
{
    if (step == 2)
        return launch_k<NB, 2>(X, npad, items, n_items, qc, reseed, partial, part_stride, grid, jmax, s);
    return launch_k<NB, 4>(X, npad, items, n_items, qc, reseed, partial, part_stride, grid, jmax, s);
}

}  // namespace

int mixed_blocks_for(int qlen_max)
{
    const int nb = (qlen_max + 3) / 4;
    return nb <= 13 ? 13 : (nb <= 26 ? 26 : 52);
}

cudaError_t launch_debye_mixed(const float4 *X, int64_t npad, const Item *items, int n_items,
                               const QChunks &qc, int step, int reseed, double *partial, int part_stride,
                               int grid, int jmax, cudaStream_t s)
{
    if (n_items == 0) return cudaSuccess;
    int qmax = 0;
    for (int c = 0; c < qc.n_chunks; ++c) qmax = qc.q_len[c] > qmax ? qc.q_len[c] : qmax;
    switch (mixed_blocks_for(qmax)) {
    case 13:
        return launch_nb<13>(X, npad, items, n_items, qc, step, reseed, partial, part_stride, grid, jmax, s);
    case 26:
        return launch_nb<26>(X, npad, items, n_items, qc, step, reseed, partial, part_stride, grid, jmax, s);
    default:
        return launch_nb<52>(X, npad, items, n_items, qc, step, reseed, partial, part_stride, grid, jmax, s);
    }
}

}  // namespace sas

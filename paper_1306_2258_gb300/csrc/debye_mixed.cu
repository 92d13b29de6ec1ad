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
//  * The packed FMA does not negate its addend for free, so the sequences are
//    carried with the sign pattern sigma_b = (+, +, -, -) over blocks b of M
//    values: W_b = sigma_b U_b obeys W_{b+1} = (+/-) 2cos(Mt) W_b + W_{b-1},
//    the sign of the coefficient alternating with b and known at compile
//    time.  The accumulators hold sums of W; sigma is applied once, when they
//    are lifted to FP64.
//  * The coefficient 2cos(Mt), as 2 - 4 sin^2(Mt/2) or 4 cos^2(Mt/2) - 2 (whichever keeps
//    full relative accuracy: coef_dither), is rounded stochastically
//    (a dither from a hash of the pair's slots): molecules hold thousands of
//    pairs at the same distance (bonds), whose identical rounding errors would
//    otherwise drift in phase together.
//  * The identity is ill-conditioned wherever Mt is near a multiple of pi
//    (errors grow like 1/sin(Mt) per step); the sequences can be re-seeded
//    with exact values every KQ q values: the segment's start phase advances
//    by an exact rotation through KQ t, and the first 2M values of a segment
//    are S cos(jt) + C sin(jt) with cos(jt), sin(jt) from an accurate FP32
//    sin/cos of t and angle addition.
//  * The per-thread sums are FP32 over the item's J-range (one tile of the
//    precision pattern), then lifted to FP64 for a warp reduce-scatter with
//    shuffles and a fixed-order block sum; one FP64 partial per item and q.
#include "mixed_common.cuh"
#include "sas_internal.h"
#include "sincos_f32.cuh"

namespace sas {

namespace {

using namespace mixed;

// ---------------------------------------------------------------------------------------------
// 2-step recurrence from the chunk start, no re-seeding (the default path)
// ---------------------------------------------------------------------------------------------

// One pair's first two float2 blocks (q 0..3 of the chunk, block signs +, +) and its
// stochastically rounded coefficient 2cos(2t), as +C and -C.
template <bool ZERO_START, bool PRODUCT_SEEDS>
__device__ __forceinline__ void setup_m2(const float4 xi, const float4 xj, float w, float qs_hi,
                                         float qs_lo, float dq_hi, float dq_lo, unsigned hash,
                                         float2 &w0, float2 &w1, float2 &Cp, float2 &Cn,
                                         const float4 *__restrict__ sct, int sct_n, bool coef_both,
                                         int start_is_step)
{
    const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
    float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    r2 = fmaxf(r2, 1e-12f);   // coincident atoms: r = 1e-6 A, sin(q r)/r -> q
    float r, y;
    dist_rsqrt(r2, r, y);
    const float scale = w * y;   // amplitude w_i w_j / r
    const float t = fmaf(dq_hi, r, dq_lo * r);
    const SinCos b1 = sct ? sincos_tab(t, sct, sct_n) : sincos_f32(t);
    const float c1 = b1.c, s1 = b1.s;
    const float mu = (2.f * s1) * (2.f * s1);   // 4 sin^2 t
    float CM, CMn;
    coef_dither(s1, c1, hash, coef_both, CM, CMn);   // 2cos(2t)
    Cp = make_float2(CM, CM);
    Cn = make_float2(CMn, CMn);
    if (ZERO_START && PRODUCT_SEEDS) {   // the two-pair kernel's 208-q seeds (pairs2_setup.cuh)
        const float a1 = scale * s1;
        w0 = make_float2(0.f, a1);
        w1 = make_float2((a1 + a1) * c1, a1 * (3.f - mu));
        return;
    }
    const float s2 = 2.f * s1 * c1, c2 = fmaf(-2.f * s1, s1, 1.f);
    const float s3 = fmaf(s2, c1, c2 * s1);
    if (ZERO_START) {
        w0 = make_float2(0.f, scale * s1);
        w1 = make_float2(scale * s2, scale * s3);
    } else {
        const float c3 = fmaf(c2, c1, -s2 * s1);
        // the start phase q0 r (for q0 = dq the step phase t, at hand)
        SinCos ph;
        if (start_is_step) {
            ph.s = s1;
            ph.c = c1;
        } else {
            ph = sincos_f32(fmaf(qs_hi, r, qs_lo * r));
        }
        const float S = scale * ph.s, C = scale * ph.c;
        w0 = make_float2(S, fmaf(S, c1, C * s1));
        w1 = make_float2(fmaf(S, c2, C * s2), fmaf(S, c3, C * s3));
    }
}

// The recurrence over the first NV float2 blocks of the chunk (NV <= 2*NB, the chunk's q values
// rounded up to pairs): acc[v] += W_v.
template <int NB, int NV>
__device__ __forceinline__ void core_m2(float2 wp, float2 wc, const float2 Cp, const float2 Cn,
                                        float2 (&acc)[2 * NB])
{
    static_assert(NV >= 2 && NV <= 2 * NB, "slot count out of range");
    acc[0] = f2add(acc[0], wp);
    acc[1] = f2add(acc[1], wc);
#pragma unroll
    for (int v = 1; v + 1 < NV; ++v) {   // W_{v+1} = (+/-)C W_v + W_{v-1}
        const float2 n = f2fma(step_negative(v) ? Cn : Cp, wc, wp);
        acc[v + 1] = f2add(acc[v + 1], n);
        wp = wc;
        wc = n;
    }
}

// Seeds and coefficient of one pair.
struct M2Pair {
    float2 w0, w1, Cp, Cn;
};

// Set-up of pair (i, j) of the item; `valid` false gives a zero-weight stand-in (no pair).
template <bool ZERO_START, bool PRODUCT_SEEDS>
__device__ __forceinline__ void setup_at(const float4 xi, const float4 *sj, const Item &item, int tid,
                                         int jmask, int j, bool valid, float qs_hi, float qs_lo, float dq_hi,
                                         float dq_lo, M2Pair &o, const float4 *__restrict__ sct, int sct_n, bool coef_both,
                                         int start_is_step)
{
    const float4 xj = sj[j];
    const float w = (!valid || j <= jmask) ? 0.f : xi.w * xj.w;
    setup_m2<ZERO_START, PRODUCT_SEEDS>(xi, xj, w, qs_hi, qs_lo, dq_hi, dq_lo, pair_hash(item.i0 + tid, item.j0 + j), o.w0,
                         o.w1, o.Cp, o.Cn, sct, sct_n, coef_both, start_is_step);
}

// Pairs (i, j) over the item's J-range, software-pipelined: the set-up of pair j+1 does not
// depend on the recurrence of pair j, so the two interleave.  Two pair states alternate
// (unrolled by two), so no state is copied between pairs.
template <int NB, int NV, bool ZERO_START>
__device__ __forceinline__ void run_m2_pipelined(const float4 xi, const float4 *sj, const Item &item,
                                                 int tid, int jmask, float qs_hi, float qs_lo, float dq_hi,
                                                 float dq_lo, float2 (&acc)[2 * NB], const float4 *__restrict__ sct,
                                                 int sct_n, bool coef_both,
                                         int start_is_step)
{
    const int jlen = item.jlen;
    if (jlen <= 0) return;
    M2Pair a, b;
    setup_at<ZERO_START, NB == 52>(xi, sj, item, tid, jmask, 0, true, qs_hi, qs_lo, dq_hi, dq_lo, a, sct, sct_n, coef_both, start_is_step);
    int j = 0;
    for (; j + 1 < jlen; j += 2) {
        setup_at<ZERO_START, NB == 52>(xi, sj, item, tid, jmask, j + 1, true, qs_hi, qs_lo, dq_hi, dq_lo, b, sct, sct_n, coef_both, start_is_step);
        core_m2<NB, NV>(a.w0, a.w1, a.Cp, a.Cn, acc);
        const bool more = j + 2 < jlen;
        setup_at<ZERO_START, NB == 52>(xi, sj, item, tid, jmask, more ? j + 2 : j + 1, more, qs_hi, qs_lo, dq_hi, dq_lo,
                             a, sct, sct_n, coef_both, start_is_step);
        core_m2<NB, NV>(b.w0, b.w1, b.Cp, b.Cn, acc);
    }
    if (j < jlen) core_m2<NB, NV>(a.w0, a.w1, a.Cp, a.Cn, acc);   // odd J-range: its last pair
}

// The same pairs one after the other.
template <int NB, bool ZERO_START>
__device__ __forceinline__ void run_m2(const float4 xi, const float4 *sj, const Item &item, int tid,
                                       int jmask, float qs_hi, float qs_lo, float dq_hi, float dq_lo,
                                       float2 (&acc)[2 * NB], const float4 *__restrict__ sct, int sct_n, bool coef_both,
                                         int start_is_step)
{
    for (int j = 0; j < item.jlen; ++j) {
        M2Pair a;
        setup_at<ZERO_START, NB == 52>(xi, sj, item, tid, jmask, j, true, qs_hi, qs_lo, dq_hi, dq_lo, a, sct, sct_n, coef_both, start_is_step);
        core_m2<NB, 2 * NB>(a.w0, a.w1, a.Cp, a.Cn, acc);
    }
}

// The pipelined loop with the slot count fixed at compile time: the chunk's nv float2 slots,
// for nv within 3 of the capacity (beyond that the spare slots are computed and discarded).
template <int NB, bool ZERO_START>
__device__ __forceinline__ void run_m2_fitted(int nv, const float4 xi, const float4 *sj, const Item &item,
                                              int tid, int jmask, float qs_hi, float qs_lo, float dq_hi,
                                              float dq_lo, float2 (&acc)[2 * NB], const float4 *__restrict__ sct,
                                              int sct_n, bool coef_both,
                                         int start_is_step)
{
    switch (2 * NB - nv) {
    case 1:
        run_m2_pipelined<NB, 2 * NB - 1, ZERO_START>(xi, sj, item, tid, jmask, qs_hi, qs_lo, dq_hi, dq_lo, acc, sct,
                                                     sct_n, coef_both, start_is_step);
        break;
    case 2:
        run_m2_pipelined<NB, 2 * NB - 2, ZERO_START>(xi, sj, item, tid, jmask, qs_hi, qs_lo, dq_hi, dq_lo, acc, sct,
                                                     sct_n, coef_both, start_is_step);
        break;
    case 3:
        run_m2_pipelined<NB, 2 * NB - 3, ZERO_START>(xi, sj, item, tid, jmask, qs_hi, qs_lo, dq_hi, dq_lo, acc, sct,
                                                     sct_n, coef_both, start_is_step);
        break;
    default:
        run_m2_pipelined<NB, 2 * NB, ZERO_START>(xi, sj, item, tid, jmask, qs_hi, qs_lo, dq_hi, dq_lo, acc, sct,
                                                     sct_n, coef_both, start_is_step);
        break;
    }
}

// ---------------------------------------------------------------------------------------------
// General form: step M = 2 or 4, re-seeded every KQ q values
// ---------------------------------------------------------------------------------------------

// cos(j t), sin(j t) for j = 0..7 by angle addition and doubling (no 1/sin(t) amplification).
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

// Terms of one pair for the chunk, into acc (float2 slot v holds q = 2v, 2v+1; block b of M
// values holds slots b*M/2 .. b*M/2 + M/2 - 1).
template <int NB, int M, int KQ>
__device__ __forceinline__ void pair_terms(const float4 xi, const float4 xj, float w, float qs_hi,
                                           float qs_lo, bool zero_start, float dq_hi, float dq_lo,
                                           unsigned hash, bool coef_both, float2 (&acc)[2 * NB])
{
    static_assert(M == 2 || M == 4, "step must be 2 or 4");
    static_assert(KQ == 0 || KQ % (2 * M) == 0, "re-seed interval must be a multiple of 2M");
    constexpr int G = M / 2;                                       // float2 per block
    constexpr int NBM = 4 * NB / M;                                // blocks per chunk
    constexpr int SEG = (KQ > 0 && KQ / M < NBM) ? KQ / M : NBM;   // blocks per segment
    const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
    float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    r2 = fmaxf(r2, 1e-12f);
    float r, y;
    dist_rsqrt(r2, r, y);
    const float scale = w * y;
    const float t = fmaf(dq_hi, r, dq_lo * r);
    const SinCos b1 = sincos_f32(t);
    Multiples m;
    multiples(b1.c, b1.s, m);
    float CM, CMn;
    coef_dither(m.s[M / 2], m.c[M / 2], hash, coef_both, CM, CMn);   // 2cos(Mt) from (sin, cos)(Mt/2)
    const float2 Cp = make_float2(CM, CM), Cn = make_float2(CMn, CMn);
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
    float2 wp[G], wc[G];
#pragma unroll
    for (int b = 0; b < NBM; ++b) {
        const int v0 = b * G;
        if (b % SEG == 0) {   // segment start: exact (signed) values of blocks b and b+1
            if (b > 0) {
                const float S2 = fmaf(S, cK, C * sK);
                C = fmaf(C, cK, -S * sK);
                S = S2;
            }
            const float sp = block_negative(b) ? -1.f : 1.f, sc = block_negative(b + 1) ? -1.f : 1.f;
            const float Sp = sp * S, Cpp = sp * C, Sc = sc * S, Ccc = sc * C;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                wp[g] = make_float2(fmaf(Sp, m.c[2 * g], Cpp * m.s[2 * g]),
                                    fmaf(Sp, m.c[2 * g + 1], Cpp * m.s[2 * g + 1]));
                wc[g] = make_float2(fmaf(Sc, m.c[M + 2 * g], Ccc * m.s[M + 2 * g]),
                                    fmaf(Sc, m.c[M + 2 * g + 1], Ccc * m.s[M + 2 * g + 1]));
                acc[v0 + g] = f2add(acc[v0 + g], wp[g]);
            }
        } else if (b % SEG == 1) {
#pragma unroll
            for (int g = 0; g < G; ++g) acc[v0 + g] = f2add(acc[v0 + g], wc[g]);
        } else {   // W_b = (+/-)C W_{b-1} + W_{b-2}, the sign of step b-1 -> b
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const float2 n = f2fma(step_negative(b - 1) ? Cn : Cp, wc[g], wp[g]);
                acc[v0 + g] = f2add(acc[v0 + g], n);
                wp[g] = wc[g];
                wc[g] = n;
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------------------------

// Variant P: 1 = general form (any M, KQ); 3 = 2-step software-pipelined; 4 = 2-step sequential
// (variant 5, two pairs per step, is debye_mixed_pairs2.cu).
template <int NB, int M, int KQ, int P>
__global__ void __launch_bounds__(kTile, mixed_ctas_per_sm(NB))
    k_debye_mixed(const float4 *__restrict__ X, int64_t npad, const Item *__restrict__ items,
                  int n_items, QChunks qc, double *__restrict__ partial, int part_stride,
                  int *__restrict__ ticket)
{
    extern __shared__ float4 sj[];
    __shared__ double red[kTile / 32][4 * NB];
    __shared__ int next_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // Items are handed out dynamically: CTA b starts with item b, then draws tickets; the list is
    // sorted by decreasing work, so the CTAs finish close together.
    int it = blockIdx.x;
    while (it < n_items) {
        const Item item = items[it];
        const float4 *Xb = X + (int64_t)item.batch * npad;
        __syncthreads();   // the previous item is done with sj, red and next_item
        if (tid == 0) next_item = (int)gridDim.x + atomicAdd(ticket, 1);
        for (int j = tid; j < item.jlen; j += kTile) sj[j] = Xb[item.j0 + j];
        const float4 xi = Xb[item.i0 + tid];
        __syncthreads();
        const int ch = item.chunk;
        const float qs_hi = qc.qs_hi[ch], qs_lo = qc.qs_lo[ch];
        const bool zero_start = (qs_hi == 0.f) && (qs_lo == 0.f);
        const int qlen = qc.q_len[ch];
        float2 acc[2 * NB];
#pragma unroll
        for (int k = 0; k < 2 * NB; ++k) acc[k] = make_float2(0.f, 0.f);
        const int jmask = item.diag ? tid : -1;   // pairs with j <= i are not pairs of i<j
        // the step's sin/cos from the call's table where it has one, as the two-pair kernel (the same
        // operations lane by lane)
        const float4 *sct = qc.sct;
        if (P == 3) {
            const int nv = (qlen + 1) >> 1;
            if (zero_start)
                run_m2_fitted<NB, true>(nv, xi, sj, item, tid, jmask, qs_hi, qs_lo, qc.dq_hi[ch], qc.dq_lo[ch], acc, sct,
                                        qc.sct_n, qc.coef_both != 0, qc.start_is_step[ch]);
            else
                run_m2_fitted<NB, false>(nv, xi, sj, item, tid, jmask, qs_hi, qs_lo, qc.dq_hi[ch], qc.dq_lo[ch], acc, sct,
                                        qc.sct_n, qc.coef_both != 0, qc.start_is_step[ch]);
        } else if (P == 4) {
            if (zero_start)
                run_m2<NB, true>(xi, sj, item, tid, jmask, qs_hi, qs_lo, qc.dq_hi[ch], qc.dq_lo[ch], acc, sct,
                                        qc.sct_n, qc.coef_both != 0, qc.start_is_step[ch]);
            else
                run_m2<NB, false>(xi, sj, item, tid, jmask, qs_hi, qs_lo, qc.dq_hi[ch], qc.dq_lo[ch], acc, sct,
                                        qc.sct_n, qc.coef_both != 0, qc.start_is_step[ch]);
        } else {
            for (int j = 0; j < item.jlen; ++j) {
                const float4 xj = sj[j];
                const float w = (j <= jmask) ? 0.f : xi.w * xj.w;
                pair_terms<NB, M, KQ>(xi, xj, w, qs_hi, qs_lo, zero_start, qc.dq_hi[ch], qc.dq_lo[ch],
                                      pair_hash(item.i0 + tid, item.j0 + j), qc.coef_both != 0, acc);
            }
        }
        flush_warp<NB, (P == 1 ? M : 2)>(acc, red[warp], lane);
        __syncthreads();
        for (int k = tid; k < qlen; k += kTile) {
            double s = red[0][k];
#pragma unroll
            for (int w = 1; w < kTile / 32; ++w) s += red[w][k];
            partial[(int64_t)it * part_stride + k] = s;
        }
        it = next_item;
    }
}

template <int NB, int M, int KQ, int P>
cudaError_t launch_v(const float4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                     double *partial, int part_stride, int grid, int jmax, int *ticket, cudaStream_t s)
{
    const size_t smem = (size_t)jmax * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(k_debye_mixed<NB, M, KQ, P>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (grid <= 0) {   // persistent grid: every resident CTA slot of every SM
        int occ = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_debye_mixed<NB, M, KQ, P>, kTile, smem);
        if (e != cudaSuccess) return e;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        grid = (occ > 0 ? occ : 1) * sms;
    }
    if (grid > n_items) grid = n_items;
    k_debye_mixed<NB, M, KQ, P><<<grid, kTile, smem, s>>>(X, npad, items, n_items, qc, partial, part_stride,
                                                           ticket);
    return cudaGetLastError();
}

template <int NB>
cudaError_t launch_nb(const float4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                      int step, int reseed, int variant, double *partial, int part_stride, int grid, int jmax,
                      int *ticket, cudaStream_t s)
{
#define SAS_LAUNCH(M_, K_, P_) \
    launch_v<NB, M_, K_, P_>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket, s)
    if (step == 2 && reseed == 0) {
        if (variant == 5)
            return launch_debye_mixed_pairs2(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket, s);
        if (variant == 3) return SAS_LAUNCH(2, 0, 3);
        if (variant == 4) return SAS_LAUNCH(2, 0, 4);
        return SAS_LAUNCH(2, 0, 1);
    }
    if (step == 2) return reseed == 32 ? SAS_LAUNCH(2, 32, 1) : SAS_LAUNCH(2, 64, 1);
    if (reseed == 0) return SAS_LAUNCH(4, 0, 1);
    return reseed == 32 ? SAS_LAUNCH(4, 32, 1) : SAS_LAUNCH(4, 64, 1);
#undef SAS_LAUNCH
}

}  // namespace

int mixed_blocks_for(int qlen_max)
{
    const int nb = (qlen_max + 3) / 4;
    return nb <= 13 ? 13 : (nb <= 26 ? 26 : 52);
}

cudaError_t launch_debye_mixed(const float4 *X, int64_t npad, const Item *items, int n_items,
                               const QChunks &qc, int step, int reseed, int variant, double *partial,
                               int part_stride, int grid, int jmax, int *ticket, cudaStream_t s)
{
    if (n_items == 0) return cudaSuccess;
    int qmax = 0;
    for (int c = 0; c < qc.n_chunks; ++c) qmax = qc.q_len[c] > qmax ? qc.q_len[c] : qmax;
    switch (mixed_blocks_for(qmax)) {
    case 13:
        return launch_nb<13>(X, npad, items, n_items, qc, step, reseed, variant, partial, part_stride, grid,
                             jmax, ticket, s);
    case 26:
        return launch_nb<26>(X, npad, items, n_items, qc, step, reseed, variant, partial, part_stride, grid,
                             jmax, ticket, s);
    default:
        return launch_nb<52>(X, npad, items, n_items, qc, step, reseed, variant, partial, part_stride, grid,
                             jmax, ticket, s);
    }
}

}  // namespace sas

// Adjoint of the Debye sum: the gradient of a loss L(I) with respect to the
// atom positions, given g_q = dL/dI(q).  The paper computes only I(q)
// (Section I-A, Eq. 2); this is the derivative of that sum:
//
//   dI(q)/dx_i = sum_{j != i} 2 f_i f_j (cos(q r) - sinc(q r)) / r^2 (x_i - x_j)
//   G_i = sum_q g_q dI(q)/dx_i = sum_{j != i} W_ij (x_i - x_j),
//   W_ij = (2 / r^2) (A - B / r),  A = sum_q h_q cos(q r),  B = sum_q (h_q / q) sin(q r),
//   h_q = g_q f_a(q) f_b(q)   (q = 0 contributes nothing: cos 0 - sinc 0 = 0).
//
// Same work items as the forward kernel, handed out by the same ticket counter.  Each thread owns
// atom i of the I-tile and takes the J atoms two at a time: the set-up of pairs (i, j) and
// (i, j+1) runs in the two lanes of packed f32x2 instructions (the forward kernel's set-up, with
// the J atoms staged transposed into lane pairs), and then, for each pair, (cos q r, sin q r)
// runs as a float2 through the 2-step three-term recurrence in two interleaved chains (even and
// odd q), one packed FMA per q, while (A, B) accumulate with a second packed FMA against
// (h_q, h_q/q) read from shared memory as float4 broadcasts (one load serves two q values and
// both pairs).  The chains carry the sign pattern (+, +, -, -) over their blocks, so the packed
// FMA never negates its addend; the table h holds the same signs, which cancel in the products.
// W_ij is applied at once: the thread's own G_i accumulates in registers, and -W_ij (x_i - x_j)
// for atoms j and j+1 (six values) is reduce-scattered over the warp with shuffles and added to
// shared memory by six lanes.  Item totals go to a [batch][slot][3] FP64 array with FP64
// atomics, or, on a deterministic context, to per-item buffers (each warp with its own copy of the
// J-range sums) that k_adjoint_gather adds up per atom in a fixed order.
#include <algorithm>

#include "mixed_common.cuh"
#include "sas_internal.h"
#include "sincos_f32.cuh"

namespace sas {

namespace {

using namespace mixed;

__device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }

// Two pairs (A = lane 0, B = lane 1) after set-up.
struct AdjPair2 {
    float2 eA0, eA1, oA0, oA1, eB0, eB1, oB0, oB1;   // (cos, sin) at q blocks 0, 1 of the even/odd chains
    float2 CpA, CnA, CpB, CnB;                       // (C, C) and (-C, -C), C = 2cos(2t)
};

// First part of the set-up: distance (hardware reciprocal square root and a Newton step) and
// weights.  It holds the long latencies (shared-memory loads, MUFU), so the pair loop issues it
// for the next two pairs ahead of the current recurrences.
struct AdjHead2 {
    float2 y, r, w;   // 1/r (hardware), r, w_i w_j (0: no pair)
};

__device__ __forceinline__ float2 jdiff(float2 xj, float2 nxi) { return f2add(xj, nxi); }   // x_j - x_i

__device__ __forceinline__ void setup_adj2_head(const float4 pxy, const float4 pzw, const float2 nX,
                                                const float2 nY, const float2 nZ, const float2 wi, bool keepA,
                                                bool keepB, AdjHead2 &h)
{
    const float2 dx = jdiff(make_float2(pxy.x, pxy.y), nX);
    const float2 dy = jdiff(make_float2(pxy.z, pxy.w), nY);
    const float2 dz = jdiff(make_float2(pzw.x, pzw.y), nZ);
    float2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));
    r2.x = fmaxf(r2.x, 1e-12f);
    r2.y = fmaxf(r2.y, 1e-12f);
    h.y = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 r0 = f2mul(r2, h.y);
    h.r = f2fma(f2mul(h.y, bc(-0.5f)), f2fma(r0, r0, f2mul(r2, bc(-1.f))), r0);
    h.w = f2mul(wi, make_float2(pzw.z, pzw.w));
    if (!keepA) h.w.x = 0.f;
    if (!keepB) h.w.y = 0.f;
}

// Second part: sin t, cos t, the chains' first two blocks and the coefficient.
template <bool ZERO_START>
__device__ __forceinline__ void setup_adj2_tail(const AdjHead2 &h, float2 qs_hi, float2 qs_lo, float2 dq_hi,
                                                float2 dq_lo, unsigned hA, unsigned hB, AdjPair2 &o, bool coef_both)
{
    const float2 r = h.r;
    const float2 t = f2fma(dq_hi, r, f2mul(dq_lo, r));
    const SinCos2 b1 = sincos2_f32(t);
    const float2 s1 = b1.s, c1 = b1.c;
    const float2 s2 = f2mul(f2add(s1, s1), c1);
    const float2 c2 = f2fma(f2mul(s1, bc(-2.f)), s1, bc(1.f));
    const float2 s3 = f2fma(s2, c1, f2mul(c2, s1));
    const float2 c3 = f2fma(c2, c1, f2mul(s2, f2mul(s1, bc(-1.f))));
    const float2 mu = f2mul(f2mul(s1, bc(4.f)), s1);
    const float2 u = f2add(make_float2(__int_as_float(0x3f800000u | (hA >> 9)),
                                       __int_as_float(0x3f800000u | (hB >> 9))),
                           bc(-1.5f));
    // the small square that keeps full relative accuracy (coef_dither): 4 sin^2 t where cos 2t >= 0,
    // 4 cos^2 t where cos 2t < 0, the coefficient then 2 - 4 sin^2 t or 4 cos^2 t - 2 (calls with
    // coef_both; the others 2 - 4 sin^2 t alone)
    float2 C, Cn;
    if (coef_both) {
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
    if (ZERO_START) {   // phases 0, t, 2t, 3t
        o.eA0 = make_float2(1.f, 0.f);
        o.eB0 = make_float2(1.f, 0.f);
        o.oA0 = make_float2(c1.x, s1.x);
        o.oB0 = make_float2(c1.y, s1.y);
        o.eA1 = make_float2(c2.x, s2.x);
        o.eB1 = make_float2(c2.y, s2.y);
        o.oA1 = make_float2(c3.x, s3.x);
        o.oB1 = make_float2(c3.y, s3.y);
    } else {            // phi0 + (0, t, 2t, 3t): rotations of (cos phi0, sin phi0)
        const SinCos2 ph = sincos2_f32(f2fma(qs_hi, r, f2mul(qs_lo, r)));
        const float2 C0 = ph.c, S0 = ph.s, nS0 = f2mul(S0, bc(-1.f));
        const float2 c_1 = f2fma(C0, c1, f2mul(nS0, s1)), s_1 = f2fma(S0, c1, f2mul(C0, s1));
        const float2 c_2 = f2fma(C0, c2, f2mul(nS0, s2)), s_2 = f2fma(S0, c2, f2mul(C0, s2));
        const float2 c_3 = f2fma(C0, c3, f2mul(nS0, s3)), s_3 = f2fma(S0, c3, f2mul(C0, s3));
        o.eA0 = make_float2(C0.x, S0.x);
        o.eB0 = make_float2(C0.y, S0.y);
        o.oA0 = make_float2(c_1.x, s_1.x);
        o.oB0 = make_float2(c_1.y, s_1.y);
        o.eA1 = make_float2(c_2.x, s_2.x);
        o.eB1 = make_float2(c_2.y, s_2.y);
        o.oA1 = make_float2(c_3.x, s_3.x);
        o.oB1 = make_float2(c_3.y, s_3.y);
    }
}

// (A, B) of both pairs: sums over the chunk's NV float2 slots of (h, h/q) * (cos, sin); slot v holds
// q values 2v (even chain) and 2v+1 (odd chain), sh[v] = sigma_v (h_2v, h_2v/q, h_2v+1, h_2v+1/q).
template <int NV>
__device__ __forceinline__ void core_adj2(const AdjPair2 &p, const float4 *sh, float2 &abA, float2 &abB)
{
    float2 peA = p.eA0, ceA = p.eA1, poA = p.oA0, coA = p.oA1;
    float2 peB = p.eB0, ceB = p.eB1, poB = p.oB0, coB = p.oB1;
    float2 aeA, aoA, aeB, aoB;
    {
        const float4 h0 = sh[0], h1 = sh[1];
        const float2 he0 = make_float2(h0.x, h0.y), ho0 = make_float2(h0.z, h0.w);
        const float2 he1 = make_float2(h1.x, h1.y), ho1 = make_float2(h1.z, h1.w);
        aeA = f2fma(he1, ceA, f2mul(he0, peA));
        aoA = f2fma(ho1, coA, f2mul(ho0, poA));
        aeB = f2fma(he1, ceB, f2mul(he0, peB));
        aoB = f2fma(ho1, coB, f2mul(ho0, poB));
    }
#pragma unroll
    for (int v = 1; v + 1 < NV; ++v) {   // block v+1 = (+/-)C block v + block v-1
        const float4 h = sh[v + 1];
        const float2 he = make_float2(h.x, h.y), ho = make_float2(h.z, h.w);
        const float2 CA = step_negative(v) ? p.CnA : p.CpA, CB = step_negative(v) ? p.CnB : p.CpB;
        const float2 neA = f2fma(CA, ceA, peA), noA = f2fma(CA, coA, poA);
        const float2 neB = f2fma(CB, ceB, peB), noB = f2fma(CB, coB, poB);
        aeA = f2fma(he, neA, aeA);
        aoA = f2fma(ho, noA, aoA);
        aeB = f2fma(he, neB, aeB);
        aoB = f2fma(ho, noB, aoB);
        peA = ceA;
        ceA = neA;
        poA = coA;
        coA = noA;
        peB = ceB;
        ceB = neB;
        poB = coB;
        coB = noB;
    }
    abA = f2add(aeA, aoA);
    abB = f2add(aeB, aoB);
}

// Sum of 8 per-lane values over the warp, scattered: afterwards lane l holds the total of value
// (l >> 2) when (l & 3) == 0.
__device__ __forceinline__ float reduce_scatter8(const float (&v)[8], int lane)
{
    float a[4];
    {
        const bool up = lane & 16;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float mine = up ? v[k + 4] : v[k], other = up ? v[k] : v[k + 4];
            a[k] = mine + __shfl_xor_sync(kFull, other, 16);
        }
    }
    float b[2];
    {
        const bool up = lane & 8;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float mine = up ? a[k + 2] : a[k], other = up ? a[k] : a[k + 2];
            b[k] = mine + __shfl_xor_sync(kFull, other, 8);
        }
    }
    const bool up = lane & 4;
    float c = (up ? b[1] : b[0]) + __shfl_xor_sync(kFull, up ? b[0] : b[1], 4);
    c += __shfl_xor_sync(kFull, c, 2);
    c += __shfl_xor_sync(kFull, c, 1);
    return c;
}

template <int NV, bool ZERO_START, bool DET>
__device__ __forceinline__ void run_adj2(const float4 *sxy, const float4 *szw, const float4 *sh, float *gj,
                                         int jpairs, const float4 xi, const Item &item, int tid, int lane, int jmask,
                                         float2 qs_hi, float2 qs_lo, float2 dq_hi, float2 dq_lo, float2 &gx,
                                         float2 &gy, float2 &gz, bool coef_both)
{
    const float2 nX = bc(-xi.x), nY = bc(-xi.y), nZ = bc(-xi.z), wi = bc(xi.w);
    const unsigned ih = item.i0 + tid;
    const int kslot = lane >> 2;   // the value this lane adds after the reduce-scatter
    if (jpairs <= 0) return;
    AdjHead2 head;
    setup_adj2_head(sxy[0], szw[0], nX, nY, nZ, wi, 0 > jmask, 1 > jmask, head);
    for (int k = 0; k < jpairs; ++k) {
        const int j = 2 * k;
        AdjPair2 p;
        setup_adj2_tail<ZERO_START>(head, qs_hi, qs_lo, dq_hi, dq_lo, pair_hash(ih, item.j0 + j),
                                    pair_hash(ih, item.j0 + j + 1), p, coef_both);
        const float2 y = head.y, w = head.w;
        // the next two pairs' distances, issued ahead of this step's recurrences (the last step
        // reads its own slot again and discards the result)
        const bool more = k + 1 < jpairs;
        const int kn = more ? k + 1 : k;
        setup_adj2_head(sxy[kn], szw[kn], nX, nY, nZ, wi, more && j + 2 > jmask, more && j + 3 > jmask, head);
        float2 abA, abB;
        core_adj2<NV>(p, sh, abA, abB);
        // -W_ij = w (2/r^2) (B/r - A), per lane; G_i += -W_ij (x_j - x_i)
        const float2 A = make_float2(abA.x, abB.x), B = make_float2(abA.y, abB.y);
        const float2 y2 = f2mul(y, y);
        const float2 nW = f2mul(f2mul(w, f2add(y2, y2)), f2fma(B, y, f2mul(A, bc(-1.f))));
        const float4 pxy = sxy[k], pzw = szw[k];   // x_j - x_i again (cheaper than keeping it)
        const float2 dx = jdiff(make_float2(pxy.x, pxy.y), nX), dy = jdiff(make_float2(pxy.z, pxy.w), nY),
                     dz = jdiff(make_float2(pzw.x, pzw.y), nZ);
        gx = f2fma(nW, dx, gx);
        gy = f2fma(nW, dy, gy);
        gz = f2fma(nW, dz, gz);
        // atoms j, j+1 receive +W_ij (x_j - x_i) = -(-W_ij)(x_j - x_i)
        const float2 fx = f2mul(nW, dx), fy = f2mul(nW, dy), fz = f2mul(nW, dz);
        const float v[8] = {-fx.x, -fy.x, -fz.x, -fx.y, -fy.y, -fz.y, 0.f, 0.f};
        const float tot = reduce_scatter8(v, lane);
        if ((lane & 3) == 0 && kslot < 6) {
            if (DET)
                gj[3 * j + kslot] += tot;   // this warp's own copy: one writer per value
            else
                atomicAdd(&gj[3 * j + kslot], tot);
        }
    }
}

constexpr int kAdjWarps = kTile / 32;

// DET: item `it` writes its I-tile totals to PI[it][tid][3] and its J-range totals (the warps'
// copies added in warp order) to PJ[it][j][3], j < jlen; G is not touched.
template <int NV, bool DET>
__global__ void __launch_bounds__(kTile, 4)
    k_debye_adjoint(const float4 *__restrict__ X, int64_t npad, const Item *__restrict__ items, int n_items,
                    QChunks qc, const float2 *__restrict__ H, int n_pairs, int hstride, double *__restrict__ G,
                    int jcap, int *__restrict__ ticket, float *__restrict__ PI, float *__restrict__ PJ)
{
    extern __shared__ float4 smem[];
    float4 *sxy = smem;                                   // [jcap / 2]: (x_j, x_j+1, y_j, y_j+1)
    float4 *szw = smem + jcap / 2;                        // [jcap / 2]: (z_j, z_j+1, w_j, w_j+1)
    float4 *sh = smem + jcap;                             // [NV]: signed (h, h/q) for q 2v and 2v+1
    float *gj = reinterpret_cast<float *>(sh + NV);       // [DET ? kAdjWarps : 1][jcap][3]
    __shared__ int next_item;
    const int tid = threadIdx.x, lane = tid & 31;
    int it = blockIdx.x;
    while (it < n_items) {
        const Item item = items[it];
        const float4 *Xb = X + (int64_t)item.batch * npad;
        const int ch = item.chunk;
        __syncthreads();   // the previous item is done with the staging, gj and next_item
        if (tid == 0) next_item = (int)gridDim.x + atomicAdd(ticket, 1);
        const int jpairs = (item.jlen + 1) >> 1;
        for (int k = tid; k < jpairs; k += kTile) {
            const float4 a = Xb[item.j0 + 2 * k];
            const float4 b = (2 * k + 1 < item.jlen) ? Xb[item.j0 + 2 * k + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
            sxy[k] = make_float4(a.x, b.x, a.y, b.y);
            szw[k] = make_float4(a.z, b.z, a.w, b.w);
        }
        if (DET) {
            for (int k = tid; k < kAdjWarps * 3 * jcap; k += kTile) gj[k] = 0.f;
        } else {
            for (int k = tid; k < 6 * jpairs; k += kTile) gj[k] = 0.f;
        }
        const float2 *Hc = H + ((int64_t)item.batch * n_pairs + item.pair) * hstride + qc.q_begin[ch];
        const int qlen = qc.q_len[ch];
        for (int v = tid; v < NV; v += kTile) {   // zero beyond the chunk's q values
            const float2 a = (2 * v < qlen) ? Hc[2 * v] : make_float2(0.f, 0.f);
            const float2 b = (2 * v + 1 < qlen) ? Hc[2 * v + 1] : make_float2(0.f, 0.f);
            const float sg = block_negative(v) ? -1.f : 1.f;
            sh[v] = make_float4(sg * a.x, sg * a.y, sg * b.x, sg * b.y);
        }
        const float4 xi = Xb[item.i0 + tid];
        __syncthreads();
        const float2 qs_hi = bc(qc.qs_hi[ch]), qs_lo = bc(qc.qs_lo[ch]);
        const bool zero_start = (qs_hi.x == 0.f) && (qs_lo.x == 0.f);
        const int jmask = item.diag ? tid : -1;   // pairs with j <= i are not pairs of i<j
        float2 gx = make_float2(0.f, 0.f), gy = gx, gz = gx;
        float *gw = DET ? gj + (tid >> 5) * 3 * jcap : gj;
        if (zero_start)
            run_adj2<NV, true, DET>(sxy, szw, sh, gw, jpairs, xi, item, tid, lane, jmask, qs_hi, qs_lo,
                                    bc(qc.dq_hi[ch]), bc(qc.dq_lo[ch]), gx, gy, gz, qc.coef_both != 0);
        else
            run_adj2<NV, false, DET>(sxy, szw, sh, gw, jpairs, xi, item, tid, lane, jmask, qs_hi, qs_lo,
                                     bc(qc.dq_hi[ch]), bc(qc.dq_lo[ch]), gx, gy, gz, qc.coef_both != 0);
        if (DET) {
            float *pi = PI + ((int64_t)it * kTile + tid) * 3;
            pi[0] = gx.x + gx.y;
            pi[1] = gy.x + gy.y;
            pi[2] = gz.x + gz.y;
            __syncthreads();
            float *pj = PJ + (int64_t)it * 3 * jcap;
            for (int k = tid; k < 3 * item.jlen; k += kTile) {
                float t = gj[k];
                for (int w = 1; w < kAdjWarps; ++w) t += gj[w * 3 * jcap + k];
                pj[k] = t;
            }
        } else {
            double *Gb = G + (int64_t)item.batch * npad * 3;
            atomicAdd(&Gb[3 * (int64_t)(item.i0 + tid)], (double)(gx.x + gx.y));
            atomicAdd(&Gb[3 * (int64_t)(item.i0 + tid) + 1], (double)(gy.x + gy.y));
            atomicAdd(&Gb[3 * (int64_t)(item.i0 + tid) + 2], (double)(gz.x + gz.y));
            __syncthreads();
            for (int k = tid; k < 3 * item.jlen; k += kTile)
                atomicAdd(&Gb[3 * (int64_t)item.j0 + k], (double)gj[k]);
        }
        it = next_item;
    }
}

// ---- per-atom form factors ------------------------------------------------------------------------
// The vector-Jacobian product of Eq. 2 with a form factor per atom and q: the pair weight becomes
//   W_ij = (2 / r^2) (A - B / r),  A = sum_q a_i(q) f_j(q) cos(q r),  B = sum_q (a_i(q) / q) f_j(q) sin(q r),
//   a_i(q) = g_q f_i(q),
// so the per-q weight differs from pair to pair: one more packed multiply per pair and q than the
// typed form.  Thread i's weights a_i sit in shared memory (AI: per float2 slot v the signed
// (a(q_2v), a(q_2v)/q_2v, a(q_2v+1), a(q_2v+1)/q_2v+1), zero past the pass and at q = 0); the J pair's
// form factors are one float4 per slot of the forward per-atom table FJ, which every thread of the
// CTA reads at the same address (a broadcast through L1).  Passes of at most 52 q keep the weights of
// a 128-atom tile within 52 KB.
constexpr int kAtomAdjNV = 26;

template <int NV>
__device__ __forceinline__ void core_adj2_atomic(const AdjPair2 &p, const float4 *sa, const float4 *__restrict__ fj,
                                                 float2 &abA, float2 &abB)
{
    float2 peA = p.eA0, ceA = p.eA1, poA = p.oA0, coA = p.oA1;
    float2 peB = p.eB0, ceB = p.eB1, poB = p.oB0, coB = p.oB1;
    float2 aeA, aoA, aeB, aoB;
    {
        const float4 a0 = sa[0], a1 = sa[kTile];
        const float4 f0 = __ldg(fj), f1 = __ldg(fj + 1);
        const float2 ae0 = make_float2(a0.x, a0.y), ao0 = make_float2(a0.z, a0.w);
        const float2 ae1 = make_float2(a1.x, a1.y), ao1 = make_float2(a1.z, a1.w);
        aeA = f2fma(f2mul(ae1, bc(f1.x)), ceA, f2mul(f2mul(ae0, bc(f0.x)), peA));
        aoA = f2fma(f2mul(ao1, bc(f1.y)), coA, f2mul(f2mul(ao0, bc(f0.y)), poA));
        aeB = f2fma(f2mul(ae1, bc(f1.z)), ceB, f2mul(f2mul(ae0, bc(f0.z)), peB));
        aoB = f2fma(f2mul(ao1, bc(f1.w)), coB, f2mul(f2mul(ao0, bc(f0.w)), poB));
    }
#pragma unroll
    for (int v = 1; v + 1 < NV; ++v) {   // block v+1 = (+/-)C block v + block v-1
        const float4 a = sa[(v + 1) * kTile];
        const float4 f = __ldg(fj + v + 1);
        const float2 ae = make_float2(a.x, a.y), ao = make_float2(a.z, a.w);
        const float2 CA = step_negative(v) ? p.CnA : p.CpA, CB = step_negative(v) ? p.CnB : p.CpB;
        const float2 neA = f2fma(CA, ceA, peA), noA = f2fma(CA, coA, poA);
        const float2 neB = f2fma(CB, ceB, peB), noB = f2fma(CB, coB, poB);
        aeA = f2fma(f2mul(ae, bc(f.x)), neA, aeA);
        aoA = f2fma(f2mul(ao, bc(f.y)), noA, aoA);
        aeB = f2fma(f2mul(ae, bc(f.z)), neB, aeB);
        aoB = f2fma(f2mul(ao, bc(f.w)), noB, aoB);
        peA = ceA;
        ceA = neA;
        poA = coA;
        coA = noA;
        peB = ceB;
        ceB = neB;
        poB = coB;
        coB = noB;
    }
    abA = f2add(aeA, aoA);
    abB = f2add(aeB, aoB);
}

template <int NV, bool ZERO_START>
__device__ __forceinline__ void run_adj2_atomic(const float4 *sxy, const float4 *szw, const float4 *sa,
                                                const float4 *__restrict__ fjrows, float *gj, int jpairs,
                                                const float4 xi, const Item &item, int tid, int lane, int jmask,
                                                float2 qs_hi, float2 qs_lo, float2 dq_hi, float2 dq_lo, float2 &gx,
                                                float2 &gy, float2 &gz, bool coef_both)
{
    const float2 nX = bc(-xi.x), nY = bc(-xi.y), nZ = bc(-xi.z), wi = bc(xi.w);
    const unsigned ih = item.i0 + tid;
    const int kslot = lane >> 2;
    if (jpairs <= 0) return;
    AdjHead2 head;
    setup_adj2_head(sxy[0], szw[0], nX, nY, nZ, wi, 0 > jmask, 1 > jmask, head);
    for (int k = 0; k < jpairs; ++k) {
        const int j = 2 * k;
        AdjPair2 p;
        setup_adj2_tail<ZERO_START>(head, qs_hi, qs_lo, dq_hi, dq_lo, pair_hash(ih, item.j0 + j),
                                    pair_hash(ih, item.j0 + j + 1), p, coef_both);
        const float2 y = head.y, w = head.w;
        const bool more = k + 1 < jpairs;
        const int kn = more ? k + 1 : k;
        setup_adj2_head(sxy[kn], szw[kn], nX, nY, nZ, wi, more && j + 2 > jmask, more && j + 3 > jmask, head);
        float2 abA, abB;
        core_adj2_atomic<NV>(p, sa, fjrows + (int64_t)k * NV, abA, abB);
        const float2 A = make_float2(abA.x, abB.x), B = make_float2(abA.y, abB.y);
        const float2 y2 = f2mul(y, y);
        const float2 nW = f2mul(f2mul(w, f2add(y2, y2)), f2fma(B, y, f2mul(A, bc(-1.f))));
        const float4 pxy = sxy[k], pzw = szw[k];
        const float2 dx = jdiff(make_float2(pxy.x, pxy.y), nX), dy = jdiff(make_float2(pxy.z, pxy.w), nY),
                     dz = jdiff(make_float2(pzw.x, pzw.y), nZ);
        gx = f2fma(nW, dx, gx);
        gy = f2fma(nW, dy, gy);
        gz = f2fma(nW, dz, gz);
        const float2 fx = f2mul(nW, dx), fy = f2mul(nW, dy), fz = f2mul(nW, dz);
        const float v[8] = {-fx.x, -fy.x, -fz.x, -fx.y, -fy.y, -fz.y, 0.f, 0.f};
        const float tot = reduce_scatter8(v, lane);
        if ((lane & 3) == 0 && kslot < 6) atomicAdd(&gj[3 * j + kslot], tot);
    }
}

// One work item per CTA at a time (the forward per-atom schedule: one type group, items per pass);
// totals into G [batch][slot][3] with FP64 atomics as in k_debye_adjoint.
template <int NV>
__global__ void __launch_bounds__(kTile, 2)
    k_debye_adjoint_atomic(const float4 *__restrict__ X, int64_t npad, const Item *__restrict__ items, int n_items,
                           QChunks qc, const float4 *__restrict__ AI, const float4 *__restrict__ FJ,
                           double *__restrict__ G, int jcap, int *__restrict__ ticket)
{
    extern __shared__ float4 smem[];
    float4 *sxy = smem;                                          // [jcap / 2]
    float4 *szw = smem + jcap / 2;                               // [jcap / 2]
    float4 *sa = smem + jcap;                                    // [NV][kTile]
    float *gj = reinterpret_cast<float *>(sa + NV * kTile);      // [jcap][3]
    __shared__ int next_item;
    const int tid = threadIdx.x, lane = tid & 31;
    int it = blockIdx.x;
    while (it < n_items) {
        const Item item = items[it];
        const float4 *Xb = X + (int64_t)item.batch * npad;
        const int ch = item.chunk;
        __syncthreads();
        if (tid == 0) next_item = (int)gridDim.x + atomicAdd(ticket, 1);
        const int jpairs = (item.jlen + 1) >> 1;
        for (int k = tid; k < jpairs; k += kTile) {
            const float4 a = Xb[item.j0 + 2 * k];
            const float4 b = (2 * k + 1 < item.jlen) ? Xb[item.j0 + 2 * k + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
            sxy[k] = make_float4(a.x, b.x, a.y, b.y);
            szw[k] = make_float4(a.z, b.z, a.w, b.w);
        }
        for (int k = tid; k < 6 * jpairs; k += kTile) gj[k] = 0.f;
        const int64_t tab = (int64_t)item.batch * qc.n_chunks + ch;
        const float4 *ai = AI + tab * NV * npad + item.i0;
        for (int e = tid; e < NV * kTile; e += kTile) sa[e] = ai[(int64_t)(e / kTile) * npad + (e % kTile)];
        const float4 *fjrows = FJ + (tab * (npad / 2) + item.j0 / 2) * NV;
        const float4 xi = Xb[item.i0 + tid];
        __syncthreads();
        const float2 qs_hi = bc(qc.qs_hi[ch]), qs_lo = bc(qc.qs_lo[ch]);
        const bool zero_start = (qs_hi.x == 0.f) && (qs_lo.x == 0.f);
        const int jmask = item.diag ? tid : -1;
        float2 gx = make_float2(0.f, 0.f), gy = gx, gz = gx;
        if (zero_start)
            run_adj2_atomic<NV, true>(sxy, szw, sa + tid, fjrows, gj, jpairs, xi, item, tid, lane, jmask, qs_hi, qs_lo,
                                      bc(qc.dq_hi[ch]), bc(qc.dq_lo[ch]), gx, gy, gz, qc.coef_both != 0);
        else
            run_adj2_atomic<NV, false>(sxy, szw, sa + tid, fjrows, gj, jpairs, xi, item, tid, lane, jmask, qs_hi,
                                       qs_lo, bc(qc.dq_hi[ch]), bc(qc.dq_lo[ch]), gx, gy, gz, qc.coef_both != 0);
        double *Gb = G + (int64_t)item.batch * npad * 3;
        atomicAdd(&Gb[3 * (int64_t)(item.i0 + tid)], (double)(gx.x + gx.y));
        atomicAdd(&Gb[3 * (int64_t)(item.i0 + tid) + 1], (double)(gy.x + gy.y));
        atomicAdd(&Gb[3 * (int64_t)(item.i0 + tid) + 2], (double)(gz.x + gz.y));
        __syncthreads();
        for (int k = tid; k < 3 * item.jlen; k += kTile) atomicAdd(&Gb[3 * (int64_t)item.j0 + k], (double)gj[k]);
        it = next_item;
    }
}

// AI[b][c][v][slot] = sigma_v (a(q_2v), a(q_2v)/q_2v, a(q_2v+1), a(q_2v+1)/q_2v+1), a(q) = g_b(q) f_i(q), for
// the atom in `slot`; zero past the pass, at q = 0 and on padding slots (zeroed beforehand).
__global__ void k_atomic_adj_table(const double *__restrict__ ff, const double *__restrict__ gI,
                                   const int *__restrict__ slot_of, int64_t n, int64_t npad, QChunks qc, int nv,
                                   float4 *__restrict__ AI)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * nv) return;
    const int64_t atom = i % n;
    const int v = (int)(i / n);
    const int c = blockIdx.y;
    const int64_t b = blockIdx.z;
    const int len = qc.q_len[c];
    float out[4] = {0.f, 0.f, 0.f, 0.f};
    for (int h = 0; h < 2; ++h) {
        const int m = 2 * v + h;
        if (m >= len) continue;
        const int k = qc.q_begin[c] + m;
        const double q = qc.qsd[c] + m * qc.dqd[c];
        if (!(q > 0.0)) continue;
        const double a = gI[b * qc.n_q + k] * ff[(b * qc.n_q + k) * n + atom];
        out[2 * h] = (float)a;
        out[2 * h + 1] = (float)(a / q);
    }
    const float sg = block_negative(v) ? -1.f : 1.f;
    AI[((b * qc.n_chunks + c) * nv + v) * npad + slot_of[atom]] =
        make_float4(sg * out[0], sg * out[1], sg * out[2], sg * out[3]);
}

// ---- the tabulated form (default) ---------------------------------------------------------------
// Within one work item every pair has the same conformer and type pair, so the pair weight is one
// function of the distance:  W_ij = W(r_ij),  W(r) = 2 sum_q h_q (cos(q r) - sinc(q r)) / r^2,
// an entire function of r (W(0) = -(2/3) sum_q h_q q^2) whose fourth derivative is at most about
// q_max^4 times its scale.  It is tabulated per conformer and type pair on nodes r_m = m D
// (D = kAdjTabStep / q_max) in FP64 as a contraction of h with the matrix K[k][m] = 2 (cos(q_k r_m) -
// sinc(q_k r_m)) / r_m^2, and each interval [r_m, r_m+1] holds the cubic through the nodes m-1..m+2
// (W is even, so node -1 is node 1) as FP32 coefficients.  Four-point cubic interpolation errs by at
// most (9/16)/24 (q_max D)^4 = 1.5e-7 of the scale at q_max D = 0.05, below the FP32 rounding of
// the recurrence it replaces.  Per pair: the distance, one float4 load and three packed FMAs in
// place of two recurrences over the q grid; the forces are applied as in k_debye_adjoint.

// K[k][m] (row stride n_rows) = 2 (cos x - sinc x) / r^2 with x = q_k r, r = m step; for x < 1e-2 the
// series 2 q^2 (-1/3 + x^2/30 - x^4/840) (its next term is below 1e-13 relative there).
__global__ void k_adj_kmat(QChunks qc, int n_rows, double step, double *__restrict__ K)
{
    const int64_t total = (int64_t)qc.n_q * n_rows;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / n_rows), m = (int)(e % n_rows);
        const double q = q_at(qc, k), r = m * step, x = q * r;
        double v;
        if (x < 1e-2) {
            const double x2 = x * x;
            v = 2.0 * q * q * (-1.0 / 3.0 + x2 * (1.0 / 30.0 - x2 / 840.0));
        } else {
            double sn, cs;
            sincos(x, &sn, &cs);
            v = 2.0 * (cs - sn / x) / (r * r);
        }
        K[e] = v;
    }
}

// Wn[row][m] = sum_k h_row(q_k) K[k][m], h = g_b(q) f_a(q) f_c(q) for row = b P + p(a, c), FP64.
__global__ void __launch_bounds__(256)
    k_adj_wnodes(const double *__restrict__ g, const double *__restrict__ F, int n_types, int n_q,
                 const double *__restrict__ K, int n_rows, double *__restrict__ Wn)
{
    extern __shared__ double hrow[];   // [n_q]
    const int P = n_types * (n_types + 1) / 2;
    const int64_t row = blockIdx.y;
    const int64_t b = row / P;
    int a = 0, rem = (int)(row % P);
    while (rem >= n_types - a) {
        rem -= n_types - a;
        ++a;
    }
    const int c = a + rem;
    for (int k = threadIdx.x; k < n_q; k += blockDim.x)
        hrow[k] = g[b * n_q + k] * F[(int64_t)a * n_q + k] * F[(int64_t)c * n_q + k];
    __syncthreads();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_rows) return;
    double acc = 0.0;
    for (int k = 0; k < n_q; ++k) acc = fma(hrow[k], K[(int64_t)k * n_rows + m], acc);
    Wn[row * n_rows + m] = acc;
}

// tab[row][m] = (c0, c1, c2, c3) of the cubic through nodes m-1, m, m+1, m+2 at t = -1, 0, 1, 2
// (node -1 = node 1), for m < n_int = n_rows - 2.
__global__ void k_adj_wcoef(const double *__restrict__ Wn, int n_rows, int64_t rows, float4 *__restrict__ tab)
{
    const int n_int = n_rows - 2;
    const int64_t total = rows * n_int;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / n_int;
        const int m = (int)(e % n_int);
        const double *w = Wn + row * n_rows;
        const double y0 = w[m == 0 ? 1 : m - 1], y1 = w[m], y2 = w[m + 1], y3 = w[m + 2];
        tab[e] = make_float4((float)y1, (float)(-y0 / 3.0 - 0.5 * y1 + y2 - y3 / 6.0), (float)(0.5 * (y0 + y2) - y1),
                             (float)((y3 - y0) / 6.0 + 0.5 * (y1 - y2)));
    }
}

// The pair loop with W from the item's table row (tab, n_int intervals of width 1 / inv_step).
template <bool DET>
__device__ __forceinline__ void run_adj_tab(const float4 *sxy, const float4 *szw, const float4 *__restrict__ tab,
                                            int n_int, float inv_step, float *gj, int jpairs, const float4 xi,
                                            int lane, int jmask, float2 &gx, float2 &gy, float2 &gz)
{
    const float2 nX = bc(-xi.x), nY = bc(-xi.y), nZ = bc(-xi.z), wi = bc(xi.w);
    const int kslot = lane >> 2;
    const float last = (float)(n_int - 1);
    for (int k = 0; k < jpairs; ++k) {
        const int j = 2 * k;
        const float4 pxy = sxy[k], pzw = szw[k];
        AdjHead2 h;
        setup_adj2_head(pxy, pzw, nX, nY, nZ, wi, j > jmask, j + 1 > jmask, h);
        // interval and position: m = floor(r / step) (clamped to the last interval, where t <= 1 keeps
        // the cubic finite for pairs beyond it, which carry w = 0), t = r / step - m
        const float2 sv = f2mul(h.r, bc(inv_step));
        const float ma = fminf(floorf(sv.x), last), mb = fminf(floorf(sv.y), last);
        const float2 t = make_float2(fminf(sv.x - ma, 1.f), fminf(sv.y - mb, 1.f));
        const float4 ca = tab[(int)ma], cb = tab[(int)mb];
        const float2 W = f2fma(f2fma(f2fma(make_float2(ca.w, cb.w), t, make_float2(ca.z, cb.z)), t,
                                     make_float2(ca.y, cb.y)),
                               t, make_float2(ca.x, cb.x));
        const float2 nW = f2mul(f2mul(h.w, bc(-1.f)), W);   // -w_i w_j W(r); G_i += -W (x_j - x_i)
        const float2 dx = jdiff(make_float2(pxy.x, pxy.y), nX), dy = jdiff(make_float2(pxy.z, pxy.w), nY),
                     dz = jdiff(make_float2(pzw.x, pzw.y), nZ);
        gx = f2fma(nW, dx, gx);
        gy = f2fma(nW, dy, gy);
        gz = f2fma(nW, dz, gz);
        const float2 fx = f2mul(nW, dx), fy = f2mul(nW, dy), fz = f2mul(nW, dz);
        const float v[8] = {-fx.x, -fy.x, -fz.x, -fx.y, -fy.y, -fz.y, 0.f, 0.f};
        const float tot = reduce_scatter8(v, lane);
        if ((lane & 3) == 0 && kslot < 6) {
            if (DET)
                gj[3 * j + kslot] += tot;
            else
                atomicAdd(&gj[3 * j + kslot], tot);
        }
    }
}

// The tabulated form of k_debye_adjoint: same items, tickets, force accumulation and outputs.
// STAGED: the item's table row is copied to shared memory (rows of at most kAdjTabStaged intervals);
// otherwise it is read through the L1 cache.
constexpr int kAdjTabStaged = 2048;

// float4 slots of the J-range force sums gj ([copies][jcap][3] floats), rounded up so that the
// staged table after them starts on a 16-byte boundary
__host__ __device__ constexpr int adj_gj_f4(int jcap, bool det) { return ((det ? kAdjWarps : 1) * jcap * 3 + 3) / 4; }

template <bool DET, bool STAGED>
__global__ void __launch_bounds__(kTile, 4)
    k_debye_adjoint_tab(const float4 *__restrict__ X, int64_t npad, const Item *__restrict__ items, int n_items,
                        const float4 *__restrict__ tab, int n_int, float inv_step, int n_pairs, double *__restrict__ G,
                        int jcap, int *__restrict__ ticket, float *__restrict__ PI, float *__restrict__ PJ)
{
    extern __shared__ float4 smem[];
    float4 *sxy = smem;                                 // [jcap / 2]
    float4 *szw = smem + jcap / 2;                      // [jcap / 2]
    float *gj = reinterpret_cast<float *>(smem + jcap);  // [DET ? kAdjWarps : 1][jcap][3]
    float4 *stab = smem + jcap + adj_gj_f4(jcap, DET);   // [n_int] when STAGED
    __shared__ int next_item;
    const int tid = threadIdx.x, lane = tid & 31;
    int it = blockIdx.x;
    while (it < n_items) {
        const Item item = items[it];
        const float4 *Xb = X + (int64_t)item.batch * npad;
        __syncthreads();
        if (tid == 0) next_item = (int)gridDim.x + atomicAdd(ticket, 1);
        if (item.chunk != 0) {
            // the work list repeats every pair once per q pass; the table holds the sum over the
            // whole grid, so only the items of the first pass contribute (the others give zero)
            if (DET) {
                PI[((int64_t)it * kTile + tid) * 3 + 0] = 0.f;
                PI[((int64_t)it * kTile + tid) * 3 + 1] = 0.f;
                PI[((int64_t)it * kTile + tid) * 3 + 2] = 0.f;
                for (int k = tid; k < 3 * item.jlen; k += kTile) PJ[(int64_t)it * 3 * jcap + k] = 0.f;
            }
            __syncthreads();   // next_item is written
            it = next_item;
            continue;
        }
        const int jpairs = (item.jlen + 1) >> 1;
        for (int k = tid; k < jpairs; k += kTile) {
            const float4 a = Xb[item.j0 + 2 * k];
            const float4 b = (2 * k + 1 < item.jlen) ? Xb[item.j0 + 2 * k + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
            sxy[k] = make_float4(a.x, b.x, a.y, b.y);
            szw[k] = make_float4(a.z, b.z, a.w, b.w);
        }
        if (DET) {
            for (int k = tid; k < kAdjWarps * 3 * jcap; k += kTile) gj[k] = 0.f;
        } else {
            for (int k = tid; k < 6 * jpairs; k += kTile) gj[k] = 0.f;
        }
        const float4 *trow = tab + ((int64_t)item.batch * n_pairs + item.pair) * n_int;
        if (STAGED)
            for (int k = tid; k < n_int; k += kTile) stab[k] = trow[k];
        const float4 xi = Xb[item.i0 + tid];
        __syncthreads();
        const int jmask = item.diag ? tid : -1;
        float2 gx = make_float2(0.f, 0.f), gy = gx, gz = gx;
        float *gw = DET ? gj + (tid >> 5) * 3 * jcap : gj;
        run_adj_tab<DET>(sxy, szw, STAGED ? stab : trow, n_int, inv_step, gw, jpairs, xi, lane, jmask, gx, gy, gz);
        if (DET) {
            float *pi = PI + ((int64_t)it * kTile + tid) * 3;
            pi[0] = gx.x + gx.y;
            pi[1] = gy.x + gy.y;
            pi[2] = gz.x + gz.y;
            __syncthreads();
            float *pj = PJ + (int64_t)it * 3 * jcap;
            for (int k = tid; k < 3 * item.jlen; k += kTile) {
                float t = gj[k];
                for (int w = 1; w < kAdjWarps; ++w) t += gj[w * 3 * jcap + k];
                pj[k] = t;
            }
        } else {
            double *Gb = G + (int64_t)item.batch * npad * 3;
            atomicAdd(&Gb[3 * (int64_t)(item.i0 + tid)], (double)(gx.x + gx.y));
            atomicAdd(&Gb[3 * (int64_t)(item.i0 + tid) + 1], (double)(gy.x + gy.y));
            atomicAdd(&Gb[3 * (int64_t)(item.i0 + tid) + 2], (double)(gz.x + gz.y));
            __syncthreads();
            for (int k = tid; k < 3 * item.jlen; k += kTile)
                atomicAdd(&Gb[3 * (int64_t)item.j0 + k], (double)gj[k]);
        }
        it = next_item;
    }
}

template <bool DET, bool STAGED>
cudaError_t launch_tab(const float4 *X, int64_t npad, const Item *items, int n_items, const float4 *tab, int n_int,
                       float inv_step, int n_pairs, double *G, int jcap, int *ticket, float *PI, float *PJ,
                       cudaStream_t s)
{
    const size_t smem = ((size_t)jcap + adj_gj_f4(jcap, DET) + (STAGED ? (size_t)n_int : 0)) * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(k_debye_adjoint_tab<DET, STAGED>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0, dev = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_debye_adjoint_tab<DET, STAGED>, kTile, smem)) !=
        cudaSuccess)
        return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    int grid = (occ > 0 ? occ : 1) * sms;
    if (grid > n_items) grid = n_items;
    k_debye_adjoint_tab<DET, STAGED><<<grid, kTile, smem, s>>>(X, npad, items, n_items, tab, n_int, inv_step,
                                                               n_pairs, G, jcap, ticket, PI, PJ);
    return cudaGetLastError();
}

// G[b][slot][c] (every slot of every I-tile) = the item totals of the items listed for the slot's
// tile, added in list order in FP64: entry 2e is item e's I-tile, entry 2e+1 its J-range.
__global__ void k_adjoint_gather(const float *__restrict__ PI, const float *__restrict__ PJ, int jcap,
                                 const Item *__restrict__ items, const int *__restrict__ tile_off,
                                 const int *__restrict__ tile_ent, int ntiles, int64_t npad, int64_t batch,
                                 double *__restrict__ G)
{
    const int tau = blockIdx.x, tid = threadIdx.x;
    const int slot = tau * kTile + tid;
    for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
        const int64_t l = b * ntiles + tau;
        double g0 = 0.0, g1 = 0.0, g2 = 0.0;
        for (int idx = tile_off[l]; idx < tile_off[l + 1]; ++idx) {
            const int ent = tile_ent[idx], e = ent >> 1;
            const float *p;
            if (ent & 1) {
                const int k = slot - items[e].j0;
                if (k < 0 || k >= items[e].jlen) continue;
                p = PJ + ((int64_t)e * jcap + k) * 3;
            } else {
                p = PI + ((int64_t)e * kTile + tid) * 3;
            }
            g0 += (double)p[0];
            g1 += (double)p[1];
            g2 += (double)p[2];
        }
        double *g = G + (b * npad + slot) * 3;
        g[0] = g0;
        g[1] = g1;
        g[2] = g2;
    }
}

// g[b][q] = dchi2/dI = 2 w_q (I - T); chi2[b] = sum_q w_q (I - T)^2 (fixed-order block sum)
__global__ void k_chi2(const double *I, const double *T, const double *w, int n_q, double *g,
                       double *chi2)
{
    __shared__ double red[256];
    const int64_t b = blockIdx.x;
    double s = 0.0;
    for (int k = threadIdx.x; k < n_q; k += blockDim.x) {
        const double d = I[b * n_q + k] - T[k];
        s += w[k] * d * d;
        g[b * n_q + k] = 2.0 * w[k] * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && chi2) chi2[b] = red[0];
}

// H[b][p][k] = (g_bk f_a f_b, g_bk f_a f_b / q_k), zero at q = 0
__global__ void k_adjoint_coef(const double *g, const double *F, int n_types, QChunks qc, float2 *H,
                               int hstride)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b = blockIdx.y;
    if (k >= qc.n_q) return;
    const double q = q_at(qc, k);
    const int P = n_types * (n_types + 1) / 2;
    int p = 0;
    for (int a = 0; a < n_types; ++a)
        for (int c = a; c < n_types; ++c, ++p) {
            const double h = q > 0.0 ? g[b * qc.n_q + k] * F[a * qc.n_q + k] * F[c * qc.n_q + k] : 0.0;
            H[(b * P + p) * hstride + k] = make_float2((float)h, q > 0.0 ? (float)(h / q) : 0.f);
        }
}

// grad_out[b][i][c] = G[b][slot_of[i]][c] (caller's atom order)
__global__ void k_unpermute(const double *G, const int *slot_of, int64_t n, int64_t npad, int64_t batch,
                            float *grad_out)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= batch * n) return;
    const int64_t b = idx / n, i = idx % n;
    const int64_t s = slot_of[i];
    for (int c = 0; c < 3; ++c) grad_out[3 * idx + c] = (float)G[(b * npad + s) * 3 + c];
}

template <int NV, bool DET>
cudaError_t launch_nv(const float4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                      const float2 *H, int n_pairs, int hstride, double *G, int jcap, int *ticket, float *PI,
                      float *PJ, cudaStream_t s)
{
    const size_t smem = (size_t)jcap * sizeof(float4) + NV * sizeof(float4) +
                        (size_t)(DET ? kAdjWarps : 1) * jcap * 3 * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_debye_adjoint<NV, DET>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0, dev = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_debye_adjoint<NV, DET>, kTile, smem)) !=
        cudaSuccess)
        return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    int grid = (occ > 0 ? occ : 1) * sms;
    if (grid > n_items) grid = n_items;
    k_debye_adjoint<NV, DET><<<grid, kTile, smem, s>>>(X, npad, items, n_items, qc, H, n_pairs, hstride, G, jcap,
                                                       ticket, PI, PJ);
    return cudaGetLastError();
}

// NV: the slots of the longest chunk when within 3 of the capacity 2*NB, else the capacity (always
// the capacity for the deterministic form).
template <int NB>
cudaError_t launch_nb(int nv, const float4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                      const float2 *H, int n_pairs, int hstride, double *G, int jcap, int *ticket, float *PI,
                      float *PJ, cudaStream_t s)
{
    if (PI)
        return launch_nv<2 * NB, true>(X, npad, items, n_items, qc, H, n_pairs, hstride, G, jcap, ticket, PI, PJ,
                                       s);
    switch (2 * NB - nv) {
    case 1:
        return launch_nv<2 * NB - 1, false>(X, npad, items, n_items, qc, H, n_pairs, hstride, G, jcap, ticket,
                                            nullptr, nullptr, s);
    case 2:
        return launch_nv<2 * NB - 2, false>(X, npad, items, n_items, qc, H, n_pairs, hstride, G, jcap, ticket,
                                            nullptr, nullptr, s);
    case 3:
        return launch_nv<2 * NB - 3, false>(X, npad, items, n_items, qc, H, n_pairs, hstride, G, jcap, ticket,
                                            nullptr, nullptr, s);
    default:
        return launch_nv<2 * NB, false>(X, npad, items, n_items, qc, H, n_pairs, hstride, G, jcap, ticket, nullptr,
                                        nullptr, s);
    }
}

}  // namespace

cudaError_t launch_chi2(const double *I, const double *T, const double *w, int n_q, int64_t batch,
                        double *g, double *chi2, cudaStream_t s)
{
    if (batch == 0) return cudaSuccess;
    k_chi2<<<(unsigned)batch, 256, 0, s>>>(I, T, w, n_q, g, chi2);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_coef(const double *g, const double *F, int n_types, int64_t batch,
                                const QChunks &qc, float2 *H, int hstride, cudaStream_t s)
{
    if (batch == 0) return cudaSuccess;
    dim3 grid((qc.n_q + 127) / 128, (unsigned)batch);
    k_adjoint_coef<<<grid, 128, 0, s>>>(g, F, n_types, qc, H, hstride);
    return cudaGetLastError();
}

cudaError_t launch_debye_adjoint(const float4 *X, int64_t npad, const Item *items, int n_items,
                                 const QChunks &qc, const float2 *H, int n_pairs, int hstride, double *G,
                                 int jlen_max, int *ticket, float *PI, float *PJ, cudaStream_t s)
{
    if (n_items == 0) return cudaSuccess;
    const int jcap = adjoint_jcap(jlen_max);
    int qmax = 0;
    for (int c = 0; c < qc.n_chunks; ++c) qmax = qc.q_len[c] > qmax ? qc.q_len[c] : qmax;
    const int nv = (qmax + 1) / 2;
    switch (mixed_blocks_for(qmax)) {
    case 13:
        return launch_nb<13>(nv, X, npad, items, n_items, qc, H, n_pairs, hstride, G, jcap, ticket, PI, PJ, s);
    case 26:
        return launch_nb<26>(nv, X, npad, items, n_items, qc, H, n_pairs, hstride, G, jcap, ticket, PI, PJ, s);
    default:
        return launch_nb<52>(nv, X, npad, items, n_items, qc, H, n_pairs, hstride, G, jcap, ticket, PI, PJ, s);
    }
}

int adjoint_atomic_slots() { return kAtomAdjNV; }

cudaError_t launch_atomic_adj_table(const double *ff, const double *gI, const int *slot_of, int64_t n, int64_t npad,
                                    int64_t batch, const QChunks &qc, float4 *AI, cudaStream_t s)
{
    if (n == 0 || batch == 0) return cudaSuccess;
    const int threads = 256;
    const dim3 grid((unsigned)((n * kAtomAdjNV + threads - 1) / threads), (unsigned)qc.n_chunks, (unsigned)batch);
    k_atomic_adj_table<<<grid, threads, 0, s>>>(ff, gI, slot_of, n, npad, qc, kAtomAdjNV, AI);
    return cudaGetLastError();
}

cudaError_t launch_debye_adjoint_atomic(const float4 *X, int64_t npad, const Item *items, int n_items,
                                        const QChunks &qc, const float4 *AI, const float4 *FJ, double *G, int jlen_max,
                                        int *ticket, cudaStream_t s)
{
    if (n_items == 0) return cudaSuccess;
    for (int c = 0; c < qc.n_chunks; ++c)
        if (qc.q_len[c] > 2 * kAtomAdjNV) return cudaErrorInvalidValue;
    const int jcap = adjoint_jcap(jlen_max);
    const size_t smem = (size_t)jcap * sizeof(float4) + (size_t)kAtomAdjNV * kTile * sizeof(float4) +
                        (size_t)jcap * 3 * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_debye_adjoint_atomic<kAtomAdjNV>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0, dev = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_debye_adjoint_atomic<kAtomAdjNV>, kTile, smem)) !=
        cudaSuccess)
        return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    int grid = (occ > 0 ? occ : 1) * sms;
    if (grid > n_items) grid = n_items;
    k_debye_adjoint_atomic<kAtomAdjNV><<<grid, kTile, smem, s>>>(X, npad, items, n_items, qc, AI, FJ, G, jcap, ticket);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_kmat(const QChunks &qc, int n_rows, double step, double *K, cudaStream_t s)
{
    const int64_t total = (int64_t)qc.n_q * n_rows;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
    k_adj_kmat<<<blocks, 256, 0, s>>>(qc, n_rows, step, K);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_wtab(const double *g, const double *F, int n_types, int64_t batch, int n_q, const double *K,
                                int n_rows, double *Wn, float4 *tab, cudaStream_t s)
{
    const int P = n_types * (n_types + 1) / 2;
    const int64_t rows = batch * P;
    if (rows == 0) return cudaSuccess;
    if (rows > 65535) return cudaErrorInvalidValue;
    dim3 grid((n_rows + 255) / 256, (unsigned)rows);
    k_adj_wnodes<<<grid, 256, (size_t)n_q * sizeof(double), s>>>(g, F, n_types, n_q, K, n_rows, Wn);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t total = rows * (n_rows - 2);
    k_adj_wcoef<<<(int)std::min<int64_t>((total + 255) / 256, 8192), 256, 0, s>>>(Wn, n_rows, rows, tab);
    return cudaGetLastError();
}

cudaError_t launch_debye_adjoint_tab(const float4 *X, int64_t npad, const Item *items, int n_items, const float4 *tab,
                                     int n_int, float inv_step, int n_pairs, double *G, int jlen_max, int *ticket,
                                     float *PI, float *PJ, cudaStream_t s)
{
    if (n_items == 0) return cudaSuccess;
    const int jcap = adjoint_jcap(jlen_max);
    const bool staged = n_int <= kAdjTabStaged;
    if (PI)
        return staged ? launch_tab<true, true>(X, npad, items, n_items, tab, n_int, inv_step, n_pairs, G, jcap, ticket,
                                               PI, PJ, s)
                      : launch_tab<true, false>(X, npad, items, n_items, tab, n_int, inv_step, n_pairs, G, jcap,
                                                ticket, PI, PJ, s);
    return staged ? launch_tab<false, true>(X, npad, items, n_items, tab, n_int, inv_step, n_pairs, G, jcap, ticket,
                                            nullptr, nullptr, s)
                  : launch_tab<false, false>(X, npad, items, n_items, tab, n_int, inv_step, n_pairs, G, jcap, ticket,
                                             nullptr, nullptr, s);
}

cudaError_t launch_adjoint_gather(const float *PI, const float *PJ, int jcap, const Item *items,
                                  const int *tile_off, const int *tile_ent, int ntiles, int64_t npad, int64_t batch,
                                  double *G, cudaStream_t s)
{
    if (ntiles == 0 || batch == 0) return cudaSuccess;
    dim3 grid((unsigned)ntiles, (unsigned)(batch < 65535 ? batch : 65535));
    k_adjoint_gather<<<grid, kTile, 0, s>>>(PI, PJ, jcap, items, tile_off, tile_ent, ntiles, npad, batch, G);
    return cudaGetLastError();
}

cudaError_t launch_unpermute(const double *G, const int *slot_of, int64_t n, int64_t npad, int64_t batch,
                             float *grad_out, cudaStream_t s)
{
    const int64_t tot = batch * n;
    if (tot == 0) return cudaSuccess;
    k_unpermute<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(G, slot_of, n, npad, batch, grad_out);
    return cudaGetLastError();
}

}  // namespace sas

// Mixed-precision pair kernel, two pairs per step (Section I-A, Eq. 2; the recurrence, seeds,
// stochastic coefficient and FP64 reduction are those of debye_mixed.cu, step 2, seeded once
// per q chunk).
//
// Why two pairs: the recurrence itself runs on packed f32x2 instructions, and a scalar FP32
// instruction issued between packed ones holds the FP32 pipe about as long as a packed one.
// The per-pair set-up (distance, sin/cos of dq*r, seeds, coefficient: ~60 FP32 operations)
// therefore cost nearly twice its operation count when done one pair at a time.  Here each
// thread sets up pairs (i, j) and (i, j+1) together, lane 0 and lane 1 of every packed
// instruction, and then runs the two recurrences in lockstep (two independent dependency
// chains).  The J atoms are staged in shared memory already transposed into lane pairs:
// (x_j, x_j+1, y_j, y_j+1) and (z_j, z_j+1, w_j, w_j+1).
//
// The set-up is split in two: its head (shared-memory loads, distance by the hardware reciprocal
// square root and a Newton step, weights) holds the long latencies and is issued for the next two
// pairs before the current recurrences, which hide it; the tail (sin/cos, seeds, coefficient)
// stays in sequence (issuing it ahead too raised the register count and ran slower).
//
// Every operation matches the one-pair kernel lane by lane, and each accumulator receives pair
// j before pair j+1, so the partial sums are the same bit for bit.
#include "mixed_common.cuh"
#include "pairs2_setup.cuh"
#include "sas_internal.h"
#include "sincos_f32.cuh"

namespace sas {

namespace {

using namespace mixed;

// Both recurrences over the first NV float2 blocks, in lockstep; slot v receives A then B.
template <int NB, int NV>
__device__ __forceinline__ void core2(const PairState2 &p, float2 (&acc)[2 * NB])
{
    static_assert(NV >= 2 && NV <= 2 * NB, "slot count out of range");
    float2 pA = p.w0A, cA = p.w1A, pB = p.w0B, cB = p.w1B;
    acc[0] = f2add(f2add(acc[0], pA), pB);
    acc[1] = f2add(f2add(acc[1], cA), cB);
#pragma unroll
    for (int v = 1; v + 1 < NV; ++v) {   // W_{v+1} = (+/-)C W_v + W_{v-1}
        const float2 nA = f2fma(step_negative(v) ? p.CnA : p.CpA, cA, pA);
        const float2 nB = f2fma(step_negative(v) ? p.CnB : p.CpB, cB, pB);
        acc[v + 1] = f2add(f2add(acc[v + 1], nA), nB);
        pA = cA;
        cA = nA;
        pB = cB;
        cB = nB;
    }
}

template <int NB, int NV, bool ZERO_START, int TAB, bool CB, bool SS>
__device__ __forceinline__ void run_pairs2(const float4 *sxy, const float4 *szw, int jpairs, const float4 xi,
                                           const Item &item, int tid, int jmask, float2 qs_hi, float2 qs_lo,
                                           float2 dq_hi, float2 dq_lo, float2 (&acc)[2 * NB],
                                           const float4 *__restrict__ sct, int sct_n)
{
    const float2 nX = bc(-xi.x), nY = bc(-xi.y), nZ = bc(-xi.z), wi = bc(xi.w);
    const unsigned ih = item.i0 + tid;
    if (jpairs <= 0) return;
    PairHead2 head;
    setup2_head(sxy[0], szw[0], nX, nY, nZ, wi, 0 > jmask, 1 > jmask, head);
    for (int k = 0; k < jpairs; ++k) {
        const int j = 2 * k;
        PairState2 p;
        setup2_tail<ZERO_START, TAB, NB == 52, CB, SS>(head, qs_hi, qs_lo, dq_hi, dq_lo, pair_hash(ih, item.j0 + j),
                                                       pair_hash(ih, item.j0 + j + 1), p, sct, sct_n);
        // the next two pairs' distances, issued ahead of this step's recurrences (the last step
        // reads its own slot again and discards the result)
        const bool more = k + 1 < jpairs;
        const int kn = more ? k + 1 : k;
        setup2_head(sxy[kn], szw[kn], nX, nY, nZ, wi, more && j + 2 > jmask, more && j + 3 > jmask, head);
        core2<NB, NV>(p, acc);
    }
}

// TILE: the I-tile (= threads per CTA), 128, or 64 for small molecules whose type groups padded to
// 128 would waste slots.  TAB: the step's sin/cos (setup2_tail): the 208-q form is compiled with
// both the table and the polynomial and picks at run time (2), the 104-q form with one of them
// (1 where the call has a table, else 0), and so the 52-q form: each the faster build of its form
// (GB300: the 208-q form with the table alone 6 % slower, the 104-q form with both 5-8 % slower
// than with the table alone and 4-5 % slower with the polynomial alone; the 52-q form on Table 1's
// grid 8 % faster with the table than with the polynomial).
// CB: the coefficient formed both ways (calls with QChunks::coef_both, setup2_tail).  SS: every
// chunk of the call that does not start at q = 0 starts at its step (QChunks::start_is_step).
template <int NB, int NV, int TILE, int TAB, bool CB, bool SS>
__global__ void __launch_bounds__(TILE, mixed_ctas_per_sm(NB) * (kTile / TILE))
    k_debye_mixed_pairs2(const float4 *__restrict__ X, int64_t npad, const Item *__restrict__ items,
                         int n_items, QChunks qc, double *__restrict__ partial, int part_stride, int jmax,
                         int *__restrict__ ticket)
{
    extern __shared__ float4 smem[];
    float4 *sxy = smem;              // [jmax / 2]: (x_j, x_j+1, y_j, y_j+1)
    float4 *szw = smem + jmax / 2;   // [jmax / 2]: (z_j, z_j+1, w_j, w_j+1)
    float4 *stab = smem + jmax;      // [qc.sct_n]: the copy of the sine table (TAB 1, or 2 with a table)
    __shared__ double red[TILE / 32][4 * NB];
    __shared__ int next_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // the sine table, read from shared memory (1.2 % faster than through L1 on the 208-q form);
    // visible after the loop's first barrier
    const float4 *sct = nullptr;
    if (TAB == 1 || (TAB == 2 && qc.sct != nullptr)) {
        for (int k = tid; k < qc.sct_n; k += TILE) stab[k] = qc.sct[k];
        sct = stab;
    }
    int it = blockIdx.x;   // first item: the CTA's index; then tickets (items sorted by work)
    while (it < n_items) {
        const Item item = items[it];
        const float4 *Xb = X + (int64_t)item.batch * npad;
        __syncthreads();   // the previous item is done with the staging, red and next_item
        if (tid == 0) next_item = (int)gridDim.x + atomicAdd(ticket, 1);
        const int jpairs = (item.jlen + 1) >> 1;
        for (int k = tid; k < jpairs; k += TILE) {
            const float4 a = Xb[item.j0 + 2 * k];
            const float4 b = (2 * k + 1 < item.jlen) ? Xb[item.j0 + 2 * k + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
            sxy[k] = make_float4(a.x, b.x, a.y, b.y);
            szw[k] = make_float4(a.z, b.z, a.w, b.w);
        }
        const float4 xi = Xb[item.i0 + tid];
        __syncthreads();
        const int ch = item.chunk;
        const float2 qs_hi = bc(qc.qs_hi[ch]), qs_lo = bc(qc.qs_lo[ch]);
        const bool zero_start = (qs_hi.x == 0.f) && (qs_lo.x == 0.f);
        float2 acc[2 * NB];
#pragma unroll
        for (int k = 0; k < 2 * NB; ++k) acc[k] = make_float2(0.f, 0.f);
        const int jmask = item.diag ? tid : -1;   // pairs with j <= i are not pairs of i<j
        if (zero_start)
            run_pairs2<NB, NV, true, TAB, CB, SS>(sxy, szw, jpairs, xi, item, tid, jmask, qs_hi, qs_lo, bc(qc.dq_hi[ch]),
                                              bc(qc.dq_lo[ch]), acc, sct, qc.sct_n);
        else
            run_pairs2<NB, NV, false, TAB, CB, SS>(sxy, szw, jpairs, xi, item, tid, jmask, qs_hi, qs_lo, bc(qc.dq_hi[ch]),
                                               bc(qc.dq_lo[ch]), acc, sct, qc.sct_n);
        flush_warp<NB, 2>(acc, red[warp], lane);
        __syncthreads();
        const int qlen = qc.q_len[ch];
        for (int k = tid; k < qlen; k += TILE) {
            double s = red[0][k];
#pragma unroll
            for (int w = 1; w < TILE / 32; ++w) s += red[w][k];
            partial[(int64_t)it * part_stride + k] = s;
        }
        it = next_item;
    }
}

template <int NB, int NV, int TILE, int TAB, bool CB, bool SS>
cudaError_t launch_ss(const float4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                       double *partial, int part_stride, int grid, int jmax, int *ticket, cudaStream_t s)
{
    const bool staged = TAB == 1 || (TAB == 2 && qc.sct != nullptr);
    if (staged && (qc.sct == nullptr || qc.sct_n <= 0 || qc.sct_n > kStagedSincosTab))
        return cudaErrorInvalidValue;
    const size_t smem = ((size_t)jmax + (staged ? (size_t)qc.sct_n : 0)) * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(k_debye_mixed_pairs2<NB, NV, TILE, TAB, CB, SS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (grid <= 0) {   // persistent grid: every resident CTA slot of every SM
        int occ = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_debye_mixed_pairs2<NB, NV, TILE, TAB, CB, SS>, TILE, smem);
        if (e != cudaSuccess) return e;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        grid = (occ > 0 ? occ : 1) * sms;
    }
    if (grid > n_items) grid = n_items;
    k_debye_mixed_pairs2<NB, NV, TILE, TAB, CB, SS><<<grid, TILE, smem, s>>>(X, npad, items, n_items, qc, partial,
                                                                      part_stride, jmax, ticket);
    return cudaGetLastError();
}

// Every chunk of the call starts at q = 0 or at its step, and at least one at its step.
bool starts_at_step(const QChunks &qc)
{
    bool any = false;
    for (int c = 0; c < qc.n_chunks; ++c) {
        if (qc.qs_hi[c] == 0.f && qc.qs_lo[c] == 0.f) continue;
        if (!qc.start_is_step[c]) return false;
        any = true;
    }
    return any;
}

// SS instantiated for the 52- and 104-q forms only (coarse grids such as q_k = k dq, k >= 1).
template <int NB, int NV, int TILE, int TAB, bool CB>
cudaError_t launch_cb(const float4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                      double *partial, int part_stride, int grid, int jmax, int *ticket, cudaStream_t s)
{
    if constexpr (NB <= 26) {
        if (starts_at_step(qc))
            return launch_ss<NB, NV, TILE, TAB, CB, true>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax,
                                                          ticket, s);
    }
    return launch_ss<NB, NV, TILE, TAB, CB, false>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket,
                                                   s);
}

template <int NB, int NV, int TILE, int TAB>
cudaError_t launch_tab(const float4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                       double *partial, int part_stride, int grid, int jmax, int *ticket, cudaStream_t s)
{
    if (qc.coef_both)
        return launch_cb<NB, NV, TILE, TAB, true>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket,
                                                  s);
    return launch_cb<NB, NV, TILE, TAB, false>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket, s);
}

// The build of each form (TAB above).
template <int NB, int NV, int TILE>
cudaError_t launch_nv(const float4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                      double *partial, int part_stride, int grid, int jmax, int *ticket, cudaStream_t s)
{
    if constexpr (NB == 52) {
        return launch_tab<NB, NV, TILE, 2>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket, s);
    } else if constexpr (NB == 26 || NB == 13) {
        if (qc.sct != nullptr)
            return launch_tab<NB, NV, TILE, 1>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket,
                                               s);
        return launch_tab<NB, NV, TILE, 0>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket, s);
    } else {
        return launch_tab<NB, NV, TILE, 0>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket, s);
    }
}

// NV: the slots of the longest chunk when within 3 of the capacity 2*NB, else the capacity.
template <int NB, int TILE>
cudaError_t launch_nb2(int nv, const float4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                       double *partial, int part_stride, int grid, int jmax, int *ticket, cudaStream_t s)
{
    switch (2 * NB - nv) {
    case 1:
        return launch_nv<NB, 2 * NB - 1, TILE>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket,
                                               s);
    case 2:
        return launch_nv<NB, 2 * NB - 2, TILE>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket,
                                               s);
    case 3:
        return launch_nv<NB, 2 * NB - 3, TILE>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket,
                                               s);
    default:
        return launch_nv<NB, 2 * NB, TILE>(X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket, s);
    }
}

}  // namespace

cudaError_t launch_debye_mixed_pairs2(const float4 *X, int64_t npad, const Item *items, int n_items,
                                      const QChunks &qc, double *partial, int part_stride, int grid, int jmax,
                                      int *ticket, cudaStream_t s, int tile)
{
    if (n_items == 0) return cudaSuccess;
    if (jmax % 2 != 0) return cudaErrorInvalidValue;
    int qmax = 0;
    for (int c = 0; c < qc.n_chunks; ++c) qmax = qc.q_len[c] > qmax ? qc.q_len[c] : qmax;
    const int nv = (qmax + 1) / 2;
    const int nb = mixed_blocks_for(qmax);
    if (tile == 64) {   // small molecules: the 52- and 104-q forms only
        if (nb == 13) return launch_nb2<13, 64>(nv, X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket, s);
        if (nb == 26) return launch_nb2<26, 64>(nv, X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket, s);
        return cudaErrorInvalidValue;
    }
    if (tile != kTile) return cudaErrorInvalidValue;
    switch (nb) {
    case 13:
        return launch_nb2<13, kTile>(nv, X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket, s);
    case 26:
        return launch_nb2<26, kTile>(nv, X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket, s);
    default:
        return launch_nb2<52, kTile>(nv, X, npad, items, n_items, qc, partial, part_stride, grid, jmax, ticket, s);
    }
}

}  // namespace sas

// Mixed-precision pair kernel with per-atom form factors (Section I-A, Eq. 2 without type
// factoring; Section II keeps, for every q value, one form factor per atom and stages a block of
// them in local memory next to the block's positions).
//
// The term of pair (i, j) at q is f_i(q) f_j(q) sin(q r)/(q r).  The recurrence, seeds, two-pair
// lockstep and stochastic coefficient are those of the typed two-pair kernel; what changes:
//  * the item's J form factors are staged in shared memory next to the positions, one float4 per
//    J pair and float2 slot, (f_j(q_2v), f_j(q_2v+1), f_j+1(q_2v), f_j+1(q_2v+1)), and each
//    packed accumulate becomes a packed multiply-add by f_j(q) (same FP32 instruction count; one
//    broadcast 16-byte shared-memory load per slot and pair step);
//  * thread i scales its FP32 sums by f_i(q) (FP32, coalesced table loads) before the FP64 warp
//    reduce-scatter;
//  * the form factors of the item's J-range are staged in blocks of 64 atoms (208-q chunks) or
//    128 atoms (smaller chunks), so that a block fits beside the other resident CTAs while the
//    J-range itself stays long (up to 1,024 atoms: few flushes per pair).
#include "mixed_common.cuh"
#include "pairs2_setup.cuh"
#include "sas_internal.h"
#include "sincos_f32.cuh"

namespace sas {

namespace {

using namespace mixed;

// Both recurrences over NV float2 slots, each accumulate weighted by f_j(q): slot v receives A
// then B.  fj points at the pair step's NV float4 form-factor slots in shared memory.
template <int NB, int NV>
__device__ __forceinline__ void core2_atomic(const PairState2 &p, const float4 *__restrict__ fj,
                                             float2 (&acc)[2 * NB])
{
    static_assert(NV >= 2 && NV <= 2 * NB, "slot count out of range");
    float2 pA = p.w0A, cA = p.w1A, pB = p.w0B, cB = p.w1B;
    const float4 f0 = fj[0], f1 = fj[1];
    acc[0] = f2fma(make_float2(f0.z, f0.w), pB, f2fma(make_float2(f0.x, f0.y), pA, acc[0]));
    acc[1] = f2fma(make_float2(f1.z, f1.w), cB, f2fma(make_float2(f1.x, f1.y), cA, acc[1]));
#pragma unroll
    for (int v = 1; v + 1 < NV; ++v) {   // W_{v+1} = (+/-)C W_v + W_{v-1}
        const float2 nA = f2fma(step_negative(v) ? p.CnA : p.CpA, cA, pA);
        const float2 nB = f2fma(step_negative(v) ? p.CnB : p.CpB, cB, pB);
        const float4 g = fj[v + 1];
        acc[v + 1] = f2fma(make_float2(g.z, g.w), nB, f2fma(make_float2(g.x, g.y), nA, acc[v + 1]));
        pA = cA;
        cA = nA;
        pB = cB;
        cB = nB;
    }
}

// Pair steps k0 <= k < k1 of the item (pairs j = 2k, 2k+1 relative to item.j0); sf holds the form
// factors of steps k0.. (sub-block staging).
template <int NB, int NV, bool ZERO_START, bool CB>
__device__ __forceinline__ void run_atomic2(const float4 *sxy, const float4 *szw, const float4 *sf, int k0, int k1,
                                            const float4 xi, const Item &item, int tid, int jmask, float2 qs_hi,
                                            float2 qs_lo, float2 dq_hi, float2 dq_lo, float2 (&acc)[2 * NB],
                                            const float4 *__restrict__ sct, int sct_n)
{
    const float2 nX = bc(-xi.x), nY = bc(-xi.y), nZ = bc(-xi.z), wi = bc(xi.w);
    const unsigned ih = item.i0 + tid;
    if (k1 <= k0) return;
    PairHead2 head;
    setup2_head(sxy[k0], szw[k0], nX, nY, nZ, wi, 2 * k0 > jmask, 2 * k0 + 1 > jmask, head);
    for (int k = k0; k < k1; ++k) {
        const int j = 2 * k;
        PairState2 p;
        setup2_tail<ZERO_START, 0, false, CB>(head, qs_hi, qs_lo, dq_hi, dq_lo, pair_hash(ih, item.j0 + j),
                                              pair_hash(ih, item.j0 + j + 1), p, sct, sct_n);
        const bool more = k + 1 < k1;
        const int kn = more ? k + 1 : k;
        setup2_head(sxy[kn], szw[kn], nX, nY, nZ, wi, more && j + 2 > jmask, more && j + 3 > jmask, head);
        core2_atomic<NB, NV>(p, sf + (k - k0) * NV, acc);
    }
}

// J pair steps per staged form-factor block: 32 KB-54 KB of shared memory beside the positions.
__host__ __device__ constexpr int atomic_sub_pairs(int NB) { return NB >= 52 ? 32 : 64; }

// FJ: [batch][chunk][npad / 2][NV] float4, FI: [batch][chunk][NV][npad] float2 (see atomic.cu).
// CB: the coefficient formed both ways (calls with QChunks::coef_both, setup2_tail).
template <int NB, int NV, bool CB>
__global__ void __launch_bounds__(kTile, mixed_ctas_per_sm(NB))
    k_debye_atomic_pairs2(const float4 *__restrict__ X, int64_t npad, const Item *__restrict__ items, int n_items,
                          QChunks qc, const float4 *__restrict__ FJ, const float2 *__restrict__ FI,
                          double *__restrict__ partial, int part_stride, int jmax, int *__restrict__ ticket)
{
    constexpr int SUB = atomic_sub_pairs(NB);
    extern __shared__ float4 smem[];
    float4 *sxy = smem;              // [jmax / 2]: (x_j, x_j+1, y_j, y_j+1)
    float4 *szw = smem + jmax / 2;   // [jmax / 2]: (z_j, z_j+1, w_j, w_j+1)
    float4 *sf = smem + jmax;        // [SUB][NV]: form factors of one block of J pairs
    __shared__ double red[kTile / 32][4 * NB];
    __shared__ int next_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int it = blockIdx.x;
    while (it < n_items) {
        const Item item = items[it];
        const float4 *Xb = X + (int64_t)item.batch * npad;
        const int ch = item.chunk;
        const int64_t tab = (int64_t)item.batch * qc.n_chunks + ch;
        __syncthreads();   // the previous item is done with the staging, red and next_item
        if (tid == 0) next_item = (int)gridDim.x + atomicAdd(ticket, 1);
        const int jpairs = (item.jlen + 1) >> 1;
        for (int k = tid; k < jpairs; k += kTile) {
            const float4 a = Xb[item.j0 + 2 * k];
            const float4 b = (2 * k + 1 < item.jlen) ? Xb[item.j0 + 2 * k + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
            sxy[k] = make_float4(a.x, b.x, a.y, b.y);
            szw[k] = make_float4(a.z, b.z, a.w, b.w);
        }
        const float4 xi = Xb[item.i0 + tid];
        const float2 qs_hi = bc(qc.qs_hi[ch]), qs_lo = bc(qc.qs_lo[ch]);
        const bool zero_start = (qs_hi.x == 0.f) && (qs_lo.x == 0.f);
        float2 acc[2 * NB];
#pragma unroll
        for (int k = 0; k < 2 * NB; ++k) acc[k] = make_float2(0.f, 0.f);
        // pairs with j0 + j <= i0 + tid are not pairs of i < j.  Every item of this kernel lies in
        // the one type group, so the mask follows from the offset of the J-range in the group.
        const int off = item.j0 - item.i0;
        const int jmask = off < kTile ? tid - off : -1;
        const float4 *fsrc = FJ + (tab * (npad / 2) + item.j0 / 2) * NV;   // item.j0 is even
        for (int k0 = 0; k0 < jpairs; k0 += SUB) {
            const int k1 = min(k0 + SUB, jpairs);
            if (k0 > 0) __syncthreads();   // every warp is done with the previous block
            for (int k = tid; k < (k1 - k0) * NV; k += kTile) sf[k] = fsrc[k0 * NV + k];
            __syncthreads();
            if (zero_start)
                run_atomic2<NB, NV, true, CB>(sxy, szw, sf, k0, k1, xi, item, tid, jmask, qs_hi, qs_lo,
                                              bc(qc.dq_hi[ch]), bc(qc.dq_lo[ch]), acc, qc.sct, qc.sct_n);
            else
                run_atomic2<NB, NV, false, CB>(sxy, szw, sf, k0, k1, xi, item, tid, jmask, qs_hi, qs_lo,
                                               bc(qc.dq_hi[ch]), bc(qc.dq_lo[ch]), acc, qc.sct, qc.sct_n);
        }
        // f_i(q) of this thread's atom (zero on padding slots)
        const float2 *fi = FI + tab * NV * npad + item.i0 + tid;
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = f2mul(acc[v], fi[(int64_t)v * npad]);
        flush_warp<NB, 2>(acc, red[warp], lane);
        __syncthreads();
        const int qlen = qc.q_len[ch];
        for (int k = tid; k < qlen; k += kTile) {
            double s = red[0][k];
#pragma unroll
            for (int w = 1; w < kTile / 32; ++w) s += red[w][k];
            partial[(int64_t)it * part_stride + k] = s;
        }
        it = next_item;
    }
}

template <int NB, int NV, bool CB>
cudaError_t launch_atomic_cb(const float4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                             const float4 *FJ, const float2 *FI, double *partial, int part_stride, int grid, int jmax,
                             int *ticket, cudaStream_t s)
{
    const size_t smem = (size_t)jmax * sizeof(float4) + (size_t)atomic_sub_pairs(NB) * NV * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(k_debye_atomic_pairs2<NB, NV, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    if (grid <= 0) {   // every resident CTA slot of every SM
        int occ = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_debye_atomic_pairs2<NB, NV, CB>, kTile, smem);
        if (e != cudaSuccess) return e;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        grid = (occ > 0 ? occ : 1) * sms;
    }
    if (grid > n_items) grid = n_items;
    k_debye_atomic_pairs2<NB, NV, CB><<<grid, kTile, smem, s>>>(X, npad, items, n_items, qc, FJ, FI, partial, part_stride,
                                                            jmax, ticket);
    return cudaGetLastError();
}

template <int NB, int NV>
cudaError_t launch_atomic_nv(const float4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                             const float4 *FJ, const float2 *FI, double *partial, int part_stride, int grid, int jmax,
                             int *ticket, cudaStream_t s)
{
    if (qc.coef_both)
        return launch_atomic_cb<NB, NV, true>(X, npad, items, n_items, qc, FJ, FI, partial, part_stride, grid, jmax,
                                              ticket, s);
    return launch_atomic_cb<NB, NV, false>(X, npad, items, n_items, qc, FJ, FI, partial, part_stride, grid, jmax,
                                           ticket, s);
}

int qlen_max(const QChunks &qc)
{
    int qmax = 0;
    for (int c = 0; c < qc.n_chunks; ++c) qmax = qc.q_len[c] > qmax ? qc.q_len[c] : qmax;
    return qmax;
}

}  // namespace

// Slots of the per-atom tables: the kernel's NV for the longest chunk (exact where an
// instantiation fits it, else the block capacity 2*NB).
int atomic_slots(const QChunks &qc)
{
    const int qmax = qlen_max(qc), nv = (qmax + 1) / 2;
    switch (mixed_blocks_for(qmax)) {
    case 13:
        return nv <= 16 ? 16 : 26;
    case 26:
        return nv >= 51 ? nv : 52;
    default:
        return nv == 101 ? 101 : 104;
    }
}

// J-range cap: the positions of an item's J-range take jmax * 16 bytes of shared memory beside the
// form-factor block (at most 54 KB), and up to four CTAs share an SM.
int atomic_jmax(const QChunks &qc)
{
    (void)qc;
    return 1024;
}

cudaError_t launch_debye_atomic_pairs2(const float4 *X, int64_t npad, const Item *items, int n_items,
                                       const QChunks &qc, const float4 *FJ, const float2 *FI, double *partial,
                                       int part_stride, int grid, int jmax, int *ticket, cudaStream_t s)
{
    if (n_items == 0) return cudaSuccess;
    if (jmax % 2 != 0 || jmax > atomic_jmax(qc)) return cudaErrorInvalidValue;   // positions' staging
    const int nv = atomic_slots(qc);
#define SAS_ATOMIC_CASE(NB, NV)                                                                                 \
    if (mixed_blocks_for(qlen_max(qc)) == NB && nv == NV)                                                       \
        return launch_atomic_nv<NB, NV>(X, npad, items, n_items, qc, FJ, FI, partial, part_stride, grid, jmax, ticket, \
                                        s);
    SAS_ATOMIC_CASE(13, 16)
    SAS_ATOMIC_CASE(13, 26)
    SAS_ATOMIC_CASE(26, 51)
    SAS_ATOMIC_CASE(26, 52)
    SAS_ATOMIC_CASE(52, 101)
    SAS_ATOMIC_CASE(52, 104)
#undef SAS_ATOMIC_CASE
    return cudaErrorInvalidValue;
}

}  // namespace sas

// Exact pair-distance histogram by type pair: the input features of the
// learned surrogate.  Not part of the paper's method; it bins the same i<j
// pairs that the Debye sum (Section I-A, Eq. 2) runs over, using the same
// type-sorted work items.
//
// Bin rule, identical to the CPU oracle bit for bit: dx = x_i - x_j (float32,
// likewise dy, dz), r2 = fma(dz, dz, fma(dy, dy, dx*dx)), w = r_max / n_bins,
// e_k = k*w, e_k^2 = e_k*e_k (each one float32 rounding), and the pair goes to
// bin max{k : e_k^2 <= r2}, or is dropped when that is n_bins.  The square
// root only gives a first guess; the edge comparisons decide.  Counts are
// integers, so the result does not depend on the order of the atomics.
#include "sas_internal.h"

namespace sas {

namespace {

constexpr int kWarps = kTile / 32;

// The rare correction of a bin guess k that an edge comparison rejected: walk down while e_k^2 > r2,
// then up while e_{k+1}^2 <= r2 (a step or two at most).  Out of line, so that the common path
// branches around it instead of carrying it predicated.
__device__ __noinline__ float bin_fixup(float k, float r2, float w, float nb)
{
    for (int guard = 0; guard < 8 && k > 0.f; ++guard) {
        const float ek = __fmul_rn(k, w);
        if (__fmul_rn(ek, ek) <= r2) break;
        k -= 1.f;
    }
    for (int guard = 0; guard < 8 && k < nb; ++guard) {
        const float ek = __fmul_rn(k + 1.f, w);
        if (__fmul_rn(ek, ek) > r2) break;
        k += 1.f;
    }
    return k;
}

// Bin of r2 under the rule above: max{k : e_k^2 <= r2} with e_k^2 = fl(fl(k w)^2), capped at
// n_bins.  The first guess comes from the hardware reciprocal square root; the edge comparisons
// (the rule's own float32 roundings) decide: straight-line when the guess is right (almost
// always), the out-of-line walk otherwise.
__device__ __forceinline__ int bin_of(float r2, float w, float inv_w, int n_bins)
{
    const float nb = (float)n_bins;
    float k = fminf(fmaxf(floorf(r2 * rsqrtf(fmaxf(r2, 1e-30f)) * inv_w), 0.f), nb);
    const float elo = __fmul_rn(k, w), ehi = __fmul_rn(k + 1.f, w);
    const bool lo_ok = k == 0.f || __fmul_rn(elo, elo) <= r2;
    const bool hi_ok = k == nb || __fmul_rn(ehi, ehi) > r2;
    if (!(lo_ok && hi_ok)) k = bin_fixup(k, r2, w, nb);
    return __float_as_int(k + 8388608.f) - 0x4B000000;   // k < 2^23: its integer value
}

// One work item per CTA at a time.  Warp v takes the real rows i = v, v+4, ... of the I-tile (the
// padding slots at the end of a type group are skipped) and its lanes take 32 consecutive J atoms
// at a time, so every lane holds a real pair except at the end of a row.  Counts go to one shared
// histogram per warp, then to the global histogram with integer atomics.
__global__ void __launch_bounds__(kTile, 12)
    k_pair_histogram(const float4 *__restrict__ X, int64_t npad, const Item *__restrict__ items, int n_items,
                     int n_bins, float r_max, int n_pairs, int *__restrict__ hist,
                     unsigned long long *__restrict__ dropped, int jcap, int *__restrict__ ticket)
{
    extern __shared__ float4 smem[];
    float4 *sj = smem;                                            // [jcap]
    float4 *si = sj + jcap;                                       // [kTile]
    int *wh = reinterpret_cast<int *>(si + kTile);                // [kWarps][n_bins]
    __shared__ int next_item, jreal;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float w = __fdiv_rn(r_max, (float)n_bins);
    const float inv_w = __fdiv_rn(1.0f, w);
    int it = blockIdx.x;
    while (it < n_items) {
        const Item item = items[it];
        const float4 *Xb = X + (int64_t)item.batch * npad;
        __syncthreads();   // the previous item is done with the staging, histograms and next_item
        if (tid == 0) {
            next_item = (int)gridDim.x + atomicAdd(ticket, 1);
            jreal = 0;
        }
        __syncthreads();   // jreal is zero before the staging adds to it
        int real = 0;
        for (int j = tid; j < item.jlen; j += kTile) {
            const float4 x = Xb[item.j0 + j];
            sj[j] = x;
            real += x.w != 0.f;
        }
        for (int k = tid; k < kWarps * n_bins; k += kTile) wh[k] = 0;
        const float4 xt = Xb[item.i0 + tid];
        si[tid] = xt;
        if (real) atomicAdd(&jreal, real);
        // real atoms are a prefix of the tile and of the J-range (padding sits at the end of each
        // type group)
        const int ilen = __syncthreads_count(xt.w != 0.f);
        const int jlen = jreal;
        int *h = wh + warp * n_bins;
        unsigned drop = 0;
        for (int i = warp; i < ilen; i += kWarps) {
            const float4 xi = si[i];
            const int jstart = item.diag ? i + 1 : 0;   // pairs with j <= i are not pairs of i<j
#pragma unroll 2
            for (int j = jstart + lane; j < jlen; j += 32) {
                const float4 xj = sj[j];
                const float dx = __fsub_rn(xi.x, xj.x), dy = __fsub_rn(xi.y, xj.y), dz = __fsub_rn(xi.z, xj.z);
                const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                const int k = bin_of(r2, w, inv_w, n_bins);
                if (k >= n_bins)
                    ++drop;
                else
                    atomicAdd(&h[k], 1);
            }
        }
        for (int o = 16; o > 0; o >>= 1) drop += __shfl_xor_sync(0xffffffffu, drop, o);
        if (lane == 0 && drop) atomicAdd(&dropped[item.batch], (unsigned long long)drop);
        __syncthreads();
        int *hb = hist + ((int64_t)item.batch * n_pairs + item.pair) * n_bins;
        for (int k = tid; k < n_bins; k += kTile) {
            int sum = 0;
#pragma unroll
            for (int v = 0; v < kWarps; ++v) sum += wh[v * n_bins + k];
            if (sum) atomicAdd(&hb[k], sum);
        }
        it = next_item;
    }
}

}  // namespace

size_t histogram_smem(int jcap, int n_bins)
{
    return (size_t)(jcap + kTile) * sizeof(float4) + (size_t)kWarps * n_bins * sizeof(int);
}

cudaError_t launch_pair_histogram(const float4 *X, int64_t npad, const Item *items, int n_items,
                                  int n_bins, float r_max, int n_pairs, int *hist,
                                  unsigned long long *dropped, int jlen_max, int *ticket, cudaStream_t s)
{
    if (n_items == 0) return cudaSuccess;
    const size_t smem = histogram_smem(jlen_max, n_bins);
    cudaError_t e = cudaFuncSetAttribute(k_pair_histogram, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0, dev = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair_histogram, kTile, smem)) != cudaSuccess)
        return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    int grid = (occ > 0 ? occ : 1) * sms;
    if (grid > n_items) grid = n_items;
    k_pair_histogram<<<grid, kTile, smem, s>>>(X, npad, items, n_items, n_bins, r_max, n_pairs, hist, dropped,
                                               jlen_max, ticket);
    return cudaGetLastError();
}

}  // namespace sas

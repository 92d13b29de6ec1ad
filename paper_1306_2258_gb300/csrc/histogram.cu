// Exact pair-distance histogram by type pair: the input features of the
// learned surrogate.  Not part of the paper's method; it bins the same i<j
// pairs that the Debye sum (Section I-A, Eq. 2) runs over, using the same
// type-sorted work items.
//
// Bin rule, identical to the CPU oracle bit for bit: dx = x_i - x_j (float32,
// likewise dy, dz), r2 = fma(dz, dz, fma(dy, dy, dx*dx)), w = r_max / n_bins,
// e_k = k*w, e_k^2 = e_k*e_k (each one float32 rounding), and the pair goes to
// bin max{k : e_k^2 <= r2}, or is dropped when that is n_bins or more.  Counts
// are integers, so the result does not depend on the order of the atomics.
//
// The bin takes one edge comparison.  With s = sqrt(r2) / w and u = 2^-24,
// e_k^2 lies within 3u (relative) of k^2 w^2, so the rule's k satisfies
// s (1 - 2u) - 1 < k < s (1 + 2u).  The guess g = floor(r2 * rsqrt(r2) * c),
// c = (1 - 2^-16) / w, carries a relative error below 2^-21 (the approximate
// reciprocal square root within 2^-22, four float32 roundings) against the
// 2^-16 bias, so g <= k; and g > k - 2 while s (2^-16 + 2^-21 + 2u) < 1, that
// is for s below 60,000: n_bins <= 4096 leaves a wide margin.  So k = g + 1
// exactly when e_{g+1}^2 <= r2, and e_{g+1} = fma(g, w, w) is the rule's
// float32 (g + 1) * w.  The argument checks of the host keep w^2 and every
// e_k^2 normal and finite (w >= 1e-12, r_max <= 1e18).
#include <climits>

#include "sas_internal.h"

namespace sas {

namespace {

constexpr int kWarps = kTile / 32;

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Bin indices of two squared distances (packed), n_bins or more for a dropped pair.  A guess at or
// above n_bins is clamped to it (the pair is dropped either way, and the clamp keeps the guess an
// exact float32 integer).
__device__ __forceinline__ int2 bins_of(float2 r2, float w, float c, float nb)
{
    // r2 = 0 reads the reciprocal square root of 1e-30 (guess 0); r2 = inf gives a NaN guess, which
    // fminf turns into n_bins, and e^2 <= inf then makes it n_bins + 1: dropped, as the rule says
    const float2 rs = make_float2(rsqrt_approx(fmaxf(r2.x, 1e-30f)), rsqrt_approx(fmaxf(r2.y, 1e-30f)));
    const float2 sc = __fmul2_rn(__fmul2_rn(r2, rs), make_float2(c, c));
    const float2 g = make_float2(fminf(floorf(sc.x), nb), fminf(floorf(sc.y), nb));
    const float2 e = __ffma2_rn(g, make_float2(w, w), make_float2(w, w));   // (g + 1) w, one rounding
    const float2 e2 = __fmul2_rn(e, e);
    const float2 gb = __fadd2_rn(g, make_float2(8388608.f, 8388608.f));   // g <= 4096: its integer value
    return make_int2(__float_as_int(gb.x) - 0x4B000000 + (e2.x <= r2.x),
                     __float_as_int(gb.y) - 0x4B000000 + (e2.y <= r2.y));
}

// One work item per CTA at a time.  Warp v takes the real rows of the I-tile two at a time,
// i0 = v + 8m and i1 = i0 + 4 (the padding slots at the end of a type group are skipped), and its
// lanes take 32 consecutive J atoms at a time: each lane bins the pairs (i0, j) and (i1, j) with
// packed FP32 arithmetic.  Counts go to one shared histogram per warp with an overflow bin for the
// dropped pairs, then to the global histogram with integer atomics.
__global__ void __launch_bounds__(kTile, 10)
    k_pair_histogram(const float4 *__restrict__ X, int64_t npad, const Item *__restrict__ items, int n_items,
                     int n_bins, float r_max, int n_pairs, int *__restrict__ hist,
                     unsigned long long *__restrict__ dropped, int jcap, int *__restrict__ ticket)
{
    extern __shared__ float4 smem[];
    float4 *sj = smem;                                            // [jcap]
    float4 *si = sj + jcap;                                       // [kTile]
    int *wh = reinterpret_cast<int *>(si + kTile);                // [kWarps][n_bins + 1]
    __shared__ int next_item, jreal;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int stride = n_bins + 1;
    const float w = __fdiv_rn(r_max, (float)n_bins);
    const float c = __fmul_rn(__fdiv_rn(1.0f, w), 1.0f - 0x1p-16f);
    const float nb = (float)n_bins;
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
        for (int k = tid; k < kWarps * stride; k += kTile) wh[k] = 0;
        const float4 xt = Xb[item.i0 + tid];
        si[tid] = xt;
        if (real) atomicAdd(&jreal, real);
        // real atoms are a prefix of the tile and of the J-range (padding sits at the end of each
        // type group)
        const int ilen = __syncthreads_count(xt.w != 0.f);
        const int jlen = jreal;
        int *h = wh + warp * stride;
        for (int i0 = warp; i0 < ilen; i0 += 2 * kWarps) {
            const int i1 = i0 + kWarps;
            const float4 a = si[i0];
            const float4 b = si[i1 < ilen ? i1 : i0];
            // pairs with j <= i are not pairs of i<j; a missing second row takes no pair
            const int jstart = item.diag ? i0 + 1 : 0;
            const int jmin1 = i1 < ilen ? (item.diag ? i1 : -1) : INT_MAX;
#pragma unroll 2
            for (int j = jstart + lane; j < jlen; j += 32) {
                const float4 xj = sj[j];
                const float2 dx = make_float2(__fsub_rn(a.x, xj.x), __fsub_rn(b.x, xj.x));
                const float2 dy = make_float2(__fsub_rn(a.y, xj.y), __fsub_rn(b.y, xj.y));
                const float2 dz = make_float2(__fsub_rn(a.z, xj.z), __fsub_rn(b.z, xj.z));
                const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                const int2 k = bins_of(r2, w, c, nb);
                atomicAdd(&h[min(k.x, n_bins)], 1);
                if (j > jmin1) atomicAdd(&h[min(k.y, n_bins)], 1);
            }
        }
        __syncthreads();
        int *hb = hist + ((int64_t)item.batch * n_pairs + item.pair) * n_bins;
        for (int k = tid; k <= n_bins; k += kTile) {
            int sum = 0;
#pragma unroll
            for (int v = 0; v < kWarps; ++v) sum += wh[v * stride + k];
            if (sum == 0) continue;
            if (k < n_bins)
                atomicAdd(&hb[k], sum);
            else
                atomicAdd(&dropped[item.batch], (unsigned long long)sum);
        }
        it = next_item;
    }
}

}  // namespace

size_t histogram_smem(int jcap, int n_bins)
{
    return (size_t)(jcap + kTile) * sizeof(float4) + (size_t)kWarps * (n_bins + 1) * sizeof(int);
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

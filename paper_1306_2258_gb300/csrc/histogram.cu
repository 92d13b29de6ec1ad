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

__global__ void __launch_bounds__(kTile)
    k_pair_histogram(const float4 *__restrict__ X, int64_t npad, const Item *__restrict__ items,
                     int n_items, int n_bins, float r_max, int n_pairs, int *__restrict__ hist,
                     unsigned long long *__restrict__ dropped, int jmax)
{
    extern __shared__ float4 smem[];
    float4 *sj = smem;                                            // [jmax]
    float *e2 = reinterpret_cast<float *>(sj + jmax);             // [n_bins + 1]
    int *wh = reinterpret_cast<int *>(e2 + n_bins + 1);           // [kWarps][n_bins]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float w = __fdiv_rn(r_max, (float)n_bins);
    const float inv_w = __fdiv_rn(1.0f, w);
    for (int k = tid; k <= n_bins; k += kTile) {
        const float ek = __fmul_rn((float)k, w);
        e2[k] = __fmul_rn(ek, ek);
    }
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const Item item = items[it];
        const float4 *Xb = X + (int64_t)item.batch * npad;
        __syncthreads();
        for (int j = tid; j < item.jlen; j += kTile) sj[j] = Xb[item.j0 + j];
        for (int k = tid; k < kWarps * n_bins; k += kTile) wh[k] = 0;
        const float4 xi = Xb[item.i0 + tid];
        __syncthreads();
        const int jmask = item.diag ? tid : -1;
        unsigned drop = 0;
        if (xi.w != 0.f) {
            for (int j = jmask + 1; j < item.jlen; ++j) {
                const float4 xj = sj[j];
                if (xj.w == 0.f) continue;
                const float dx = __fsub_rn(xi.x, xj.x), dy = __fsub_rn(xi.y, xj.y),
                            dz = __fsub_rn(xi.z, xj.z);
                const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                int k = (int)fminf(__fmul_rn(__fsqrt_rn(r2), inv_w), (float)n_bins);
                while (k > 0 && e2[k] > r2) --k;
                while (k < n_bins && e2[k + 1] <= r2) ++k;
                if (k >= n_bins)
                    ++drop;
                else
                    atomicAdd(&wh[warp * n_bins + k], 1);
            }
        }
        for (int o = 16; o > 0; o >>= 1) drop += __shfl_xor_sync(0xffffffffu, drop, o);
        if (lane == 0 && drop) atomicAdd(&dropped[item.batch], (unsigned long long)drop);
        __syncthreads();
        int *hb = hist + ((int64_t)item.batch * n_pairs + item.pair) * n_bins;
        for (int k = tid; k < n_bins; k += kTile) {
            int s = 0;
#pragma unroll
            for (int v = 0; v < kWarps; ++v) s += wh[v * n_bins + k];
            if (s) atomicAdd(&hb[k], s);
        }
    }
}

}  // namespace

size_t histogram_smem(int jmax, int n_bins)
{
    return (size_t)jmax * sizeof(float4) + (size_t)(n_bins + 1) * sizeof(float) +
           (size_t)kWarps * n_bins * sizeof(int);
}

cudaError_t launch_pair_histogram(const float4 *X, int64_t npad, const Item *items, int n_items,
                                  int n_bins, float r_max, int n_pairs, int *hist,
                                  unsigned long long *dropped, int grid, int jmax, cudaStream_t s)
{
    if (n_items == 0) return cudaSuccess;
    const size_t smem = histogram_smem(jmax, n_bins);
    cudaError_t e = cudaFuncSetAttribute(k_pair_histogram, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_pair_histogram<<<grid, kTile, smem, s>>>(X, npad, items, n_items, n_bins, r_max, n_pairs, hist,
                                               dropped, jmax);
    return cudaGetLastError();
}

}  // namespace sas

// Screening step of the ensemble workflow: rank conformers by the surrogate's chi^2 against a
// target profile, keep the best k for exact re-scoring with the Debye kernels (Section I-A, Eq. 2;
// the paper's high-throughput setting, Section I).  Not part of the paper's method itself.
//
//   k_surrogate_chi2  one warp per conformer: chi2_c = sum_q w_q (B_cq exp(z_cq s_q + m_q) - T_q)^2, the
//                     network's standardized log-profile z mapped back by (m, s) and times a base
//                     profile B (either factor may be absent); FP64, lane-strided partial sums
//                     reduced in a fixed butterfly order (deterministic)
//   k_select_topk     one CTA: bitonic sort of (chi2, index) pairs in shared memory, ties broken by
//                     the index and NaN ordered last, so the selection is unique; writes the first k
//   k_gather_rows     dst[r] = src[idx[r]] for rows of a fixed byte size (the selected conformers'
//                     coordinates, packed for the exact kernels)
#include <algorithm>
#include <cmath>

#include <cstdio>

#include "sas_internal.h"

namespace sas {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSelectThreads = 1024;

__global__ void k_surrogate_chi2(int n_conf, int n_q, const float *__restrict__ z, int ld,
                                 const double *__restrict__ mean, const double *__restrict__ stdv,
                                 const double *__restrict__ base, int ld_base, const double *__restrict__ target,
                                 const double *__restrict__ w, double *__restrict__ chi2)
{
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (warp >= n_conf) return;
    const float *zc = z ? z + (int64_t)warp * ld : nullptr;
    const double *bc = base ? base + (int64_t)warp * ld_base : nullptr;
    double s = 0.0;
    for (int q = lane; q < n_q; q += 32) {
        double I = zc ? exp(fma((double)zc[q], stdv[q], mean[q])) : 1.0;
        if (bc) I *= bc[q];
        const double d = I - target[q];
        s = fma(w[q] * d, d, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (lane == 0) chi2[warp] = s;
}

// (chi2, index) order: smaller chi2 first, NaN after every number, equal keys by index.
__device__ __forceinline__ bool before(double a, int ia, double b, int ib)
{
    const bool na = a != a, nb = b != b;
    if (na != nb) return nb;
    if (!na && a != b) return a < b;
    return ia < ib;
}

__global__ void __launch_bounds__(kSelectThreads)
    k_select_topk(int n, int n_pow2, const double *__restrict__ chi2, int k, int32_t *__restrict__ top_idx,
                  double *__restrict__ top_chi2)
{
    extern __shared__ double key[];                         // [n_pow2]
    int *idx = reinterpret_cast<int *>(key + n_pow2);       // [n_pow2]
    for (int i = threadIdx.x; i < n_pow2; i += blockDim.x) {
        key[i] = i < n ? chi2[i] : __longlong_as_double(0x7ff8000000000000LL);   // padding: NaN, last
        idx[i] = i < n ? i : 0x7fffffff;
    }
    __syncthreads();
    for (int size = 2; size <= n_pow2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < n_pow2; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;   // ascending run
                    const bool swap = up ? before(key[j], idx[j], key[i], idx[i])
                                         : before(key[i], idx[i], key[j], idx[j]);
                    if (swap) {
                        const double tk = key[i];
                        key[i] = key[j];
                        key[j] = tk;
                        const int ti = idx[i];
                        idx[i] = idx[j];
                        idx[j] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        top_idx[i] = idx[i];
        if (top_chi2) top_chi2[i] = key[i];
    }
}

__global__ void k_gather_rows(const unsigned char *__restrict__ src, int64_t row_bytes, const int32_t *__restrict__ idx,
                              int64_t n_idx, unsigned char *__restrict__ dst, int vec16)
{
    for (int64_t r = blockIdx.y; r < n_idx; r += gridDim.y) {
        const unsigned char *s = src + (int64_t)idx[r] * row_bytes;
        unsigned char *d = dst + r * row_bytes;
        if (vec16) {
            const int64_t n16 = row_bytes / 16;
            for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n16;
                 c += (int64_t)gridDim.x * blockDim.x)
                reinterpret_cast<uint4 *>(d)[c] = reinterpret_cast<const uint4 *>(s)[c];
        } else {
            for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < row_bytes;
                 c += (int64_t)gridDim.x * blockDim.x)
                d[c] = s[c];
        }
    }
}

}  // namespace

int select_max() { return 8192; }

cudaError_t launch_surrogate_chi2(int n_conf, int n_q, const float *z, int ld, const double *mean, const double *stdv,
                                  const double *base, int ld_base, const double *target, const double *w, double *chi2,
                                  cudaStream_t s)
{
    if (n_conf <= 0) return cudaSuccess;
    const int threads = 256, per = threads / 32;
    k_surrogate_chi2<<<(n_conf + per - 1) / per, threads, 0, s>>>(n_conf, n_q, z, ld, mean, stdv, base, ld_base, target,
                                                                  w, chi2);
    return cudaGetLastError();
}

cudaError_t launch_select_topk(int n, const double *chi2, int k, int32_t *top_idx, double *top_chi2, cudaStream_t s)
{
    if (n <= 0 || k <= 0) return cudaSuccess;
    int n_pow2 = 1;
    while (n_pow2 < n) n_pow2 <<= 1;
    const size_t smem = (size_t)n_pow2 * (sizeof(double) + sizeof(int));
    cudaError_t e = cudaFuncSetAttribute(k_select_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_select_topk<<<1, kSelectThreads, smem, s>>>(n, n_pow2, chi2, k, top_idx, top_chi2);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const void *src, int64_t row_bytes, const int32_t *idx, int64_t n_idx, void *dst,
                               cudaStream_t s)
{
    if (n_idx <= 0 || row_bytes <= 0) return cudaSuccess;
    const int vec16 = (row_bytes % 16 == 0) && ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
    const int64_t units = vec16 ? row_bytes / 16 : row_bytes;
    const int threads = 256;
    const unsigned bx = (unsigned)std::min<int64_t>((units + threads - 1) / threads, 64);
    const dim3 grid(bx, (unsigned)std::min<int64_t>(n_idx, 65535));
    k_gather_rows<<<grid, threads, 0, s>>>(static_cast<const unsigned char *>(src), row_bytes, idx, n_idx,
                                           static_cast<unsigned char *>(dst), vec16);
    return cudaGetLastError();
}

}  // namespace sas

using namespace sas;

namespace {

bool dev_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

sas_status cuda_status(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return SAS_OK;
    cudaGetLastError();
    char buf[200];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return set_error(SAS_ERR_CUDA, buf);
}

}  // namespace

extern "C" {

sas_status sas_screen_select(int n_conf, int n_q, const float *z, int ld, const double *mean, const double *stdv,
                             const double *base, int ld_base, const double *target, const double *weights, int k,
                             int32_t *top_idx, double *top_chi2, double *chi2_all, void *stream)
{
    sas::NvtxRange nvtx_range("sas_screen_select");
    if (n_conf < 1 || n_conf > select_max()) return set_error(SAS_ERR_INVALID_ARG, "n_conf must be in [1, 8192]");
    if (n_q < 1) return set_error(SAS_ERR_INVALID_ARG, "need n_q >= 1");
    if (!z && !base) return set_error(SAS_ERR_INVALID_ARG, "z and base cannot both be NULL");
    if ((z && ld < n_q) || (base && ld_base < n_q)) return set_error(SAS_ERR_INVALID_ARG, "need ld, ld_base >= n_q");
    if (k < 1 || k > n_conf) return set_error(SAS_ERR_INVALID_ARG, "k must be in [1, n_conf]");
    if ((z && (!dev_ptr(z) || !dev_ptr(mean) || !dev_ptr(stdv))) || (base && !dev_ptr(base)) || !dev_ptr(target) ||
        !dev_ptr(weights) || !dev_ptr(top_idx) || !dev_ptr(chi2_all) || (top_chi2 && !dev_ptr(top_chi2)))
        return set_error(SAS_ERR_INVALID_ARG, "every buffer must be device memory (top_chi2 may be NULL)");
    cudaStream_t s = (cudaStream_t)stream;
    sas_status st = cuda_status(launch_surrogate_chi2(n_conf, n_q, z, ld, mean, stdv, base, ld_base, target, weights,
                                                      chi2_all, s),
                                "surrogate chi2");
    if (st != SAS_OK) return st;
    return cuda_status(launch_select_topk(n_conf, chi2_all, k, top_idx, top_chi2, s), "top-k selection");
}

sas_status sas_gather_rows(const void *src, int64_t row_bytes, const int32_t *idx, int64_t n_idx, void *dst,
                           void *stream)
{
    if (row_bytes < 0 || n_idx < 0) return set_error(SAS_ERR_INVALID_ARG, "negative size");
    if (row_bytes == 0 || n_idx == 0) return SAS_OK;
    if (!dev_ptr(src) || !dev_ptr(idx) || !dev_ptr(dst)) return set_error(SAS_ERR_INVALID_ARG, "device buffers required");
    return cuda_status(launch_gather_rows(src, row_bytes, idx, n_idx, dst, (cudaStream_t)stream), "gather");
}

}  // extern "C"

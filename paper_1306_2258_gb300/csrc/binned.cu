// The Debye sum over pair-distance histograms with every pair at its bin centre: the surrogate's
// baseline, the method without the network.
//   I_c(q) = sum_t n_t f_t(q)^2 + sum_{a<=b} 2 f_a(q) f_b(q) sum_k h_c[p(a,b)][k] sinc(q r_k),
//   r_k = (k + 1/2) w,  w = r_max / n_bins,
// an approximation of Eq. 2 (Section I-A) whose cost per conformer is O(T^2 n_bins Q) instead of
// O(N^2 Q), given the exact integer histograms of sas_pair_histogram.  It is a dense contraction of
// the counts [C][P n_bins] with a table [P n_bins][Q] of 2 f_a f_b sinc(q r_k).
//
// k_binned_table  the table in FP64, stored as FP32 (row (p, k), one column per q), built once per
//                 context and (n_bins, r_max)
// k_binned_diag   D(q) = sum_t n_t f_t(q)^2 in FP64
// k_binned_sum    one CTA per 8 conformers, one thread per q: the conformers' counts of 256 rows
//                 staged in shared memory as float ([row][conformer], read as float4 broadcasts),
//                 FP32 products (counts are exact in FP32 below 2^24) summed over 32 rows in FP32,
//                 then in FP64 (the pair kernels' precision split); D(q) added in FP64.
// Roofline: 1 FMA per count and q; 4,096 conformers x 3,840 rows x 101 q = 1.6e9 FMA against
// 63 MB of counts read once: FP32-pipe bound, not HBM-bound.
#include <cmath>
#include <cstring>

#include "api_internal.h"

namespace sas {
namespace {

constexpr int kBinCB = 8;      // conformers per CTA
constexpr int kBinRows = 256;  // (p, k) rows staged per step
constexpr int kBinLift = 32;   // rows summed in FP32 before the FP64 lift

struct TypeCounts {
    double n[SAS_MAX_TYPES];
};

// tab[(p n_bins + k) * n_q + i] = 2 f_a(q_i) f_b(q_i) sinc(q_i r_k) for type pair p = (a, b), a <= b
__global__ void k_binned_table(const double *__restrict__ F, int n_types, QChunks qc, int n_bins, double w,
                               float *__restrict__ tab)
{
    const int P = n_types * (n_types + 1) / 2, n_q = qc.n_q;
    const int64_t total = (int64_t)P * n_bins * n_q;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n_q);
        const int64_t row = e / n_q;
        const int k = (int)(row % n_bins), p = (int)(row / n_bins);
        int a = 0, rem = p;   // p -> (a, b), row-major over the upper triangle
        while (rem >= n_types - a) {
            rem -= n_types - a;
            ++a;
        }
        const int b = a + rem;
        const double x = q_at(qc, i) * (k + 0.5) * w;
        const double sinc = x == 0.0 ? 1.0 : sin(x) / x;
        tab[e] = (float)(2.0 * F[(int64_t)a * n_q + i] * F[(int64_t)b * n_q + i] * sinc);
    }
}

__global__ void k_binned_diag(const double *__restrict__ F, int n_types, int n_q, TypeCounts nt,
                              double *__restrict__ D)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_q) return;
    double d = 0.0;
    for (int t = 0; t < n_types; ++t) {
        const double f = F[(int64_t)t * n_q + i];
        d += nt.n[t] * f * f;
    }
    D[i] = d;
}

__global__ void __launch_bounds__(128)
    k_binned_sum(const int *__restrict__ hist, int64_t batch, int rows, const float *__restrict__ tab, int n_q,
                 const double *__restrict__ D, double *__restrict__ out)
{
    __shared__ __align__(16) float hs[kBinRows][kBinCB];
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.x * kBinCB;
    float acc[kBinCB];
    double acc64[kBinCB];
#pragma unroll
    for (int c = 0; c < kBinCB; ++c) acc[c] = 0.f, acc64[c] = 0.0;
    for (int r0 = 0; r0 < rows; r0 += kBinRows) {
        const int nr = min(kBinRows, rows - r0);
        __syncthreads();
        // element e -> (row r, conformer c) with c fastest: conflict-free shared stores; each
        // conformer's counts are read in runs of 4 consecutive rows (L1 serves the rest of a sector)
        for (int e = threadIdx.x; e < kBinRows * kBinCB; e += blockDim.x) {
            const int r = e / kBinCB, c = e % kBinCB;
            float v = 0.f;
            if (r < nr && c0 + c < batch) v = (float)__ldg(hist + (c0 + c) * rows + r0 + r);
            hs[r][c] = v;
        }
        __syncthreads();
        if (i < n_q) {
            for (int rb = 0; rb < nr; rb += kBinLift) {
                const int re = min(nr, rb + kBinLift);
                for (int r = rb; r < re; ++r) {
                    const float t = __ldg(tab + (int64_t)(r0 + r) * n_q + i);
                    const float4 *h4 = reinterpret_cast<const float4 *>(hs[r]);
#pragma unroll
                    for (int v = 0; v < kBinCB / 4; ++v) {
                        const float4 h = h4[v];
                        acc[4 * v + 0] = fmaf(h.x, t, acc[4 * v + 0]);
                        acc[4 * v + 1] = fmaf(h.y, t, acc[4 * v + 1]);
                        acc[4 * v + 2] = fmaf(h.z, t, acc[4 * v + 2]);
                        acc[4 * v + 3] = fmaf(h.w, t, acc[4 * v + 3]);
                    }
                }
#pragma unroll
                for (int c = 0; c < kBinCB; ++c) acc64[c] += (double)acc[c], acc[c] = 0.f;
            }
        }
    }
    if (i >= n_q) return;
#pragma unroll
    for (int c = 0; c < kBinCB; ++c)
        if (c0 + c < batch) out[(c0 + c) * n_q + i] = D[i] + acc64[c];
}

}  // namespace

namespace api {

// The binned table for (n_bins, r_max), cached in the context.
sas_status binned_table(sas_ctx *ctx, int n_bins, float r_max, cudaStream_t s)
{
    if (ctx->btab_bins == n_bins && ctx->btab_rmax == r_max && ctx->btab.p) return SAS_OK;
    const int T = ctx->n_types, P = T * (T + 1) / 2;
    ctx->btab_bins = 0;
    ALLOC_TRY(ctx->btab, (size_t)P * n_bins * ctx->n_q * sizeof(float));
    const double w = (double)r_max / n_bins;
    k_binned_table<<<4 * ctx->sms, 256, 0, s>>>(ctx->F.as<double>(), T, ctx->qc, n_bins, w, ctx->btab.as<float>());
    CUDA_TRY(cudaGetLastError());
    ctx->btab_bins = n_bins;
    ctx->btab_rmax = r_max;
    return SAS_OK;
}

}  // namespace api
}  // namespace sas

using namespace sas;
using namespace sas::api;

extern "C" sas_status sas_binned_profile(sas_ctx *ctx, const int32_t *hist, int64_t batch, int n_bins, float r_max,
                                         const int64_t *type_counts, double *I_out, void *stream)
{
    sas::NvtxRange nvtx_range("sas_binned_profile");
    if (!ctx) return fail(SAS_ERR_INVALID_ARG, "null context");
    if (batch < 0) return fail(SAS_ERR_INVALID_ARG, "negative batch");
    if (n_bins < 1 || n_bins > 4096) return fail(SAS_ERR_INVALID_ARG, "n_bins must be in [1, 4096]");
    if (!(r_max > 0.f) || !std::isfinite(r_max)) return fail(SAS_ERR_INVALID_ARG, "r_max must be positive");
    if (!type_counts) return fail(SAS_ERR_INVALID_ARG, "null type_counts");
    const int T = ctx->n_types, P = T * (T + 1) / 2, Q = ctx->n_q;
    TypeCounts nt;
    std::memset(&nt, 0, sizeof nt);
    for (int t = 0; t < T; ++t) {
        if (type_counts[t] < 0) return fail(SAS_ERR_INVALID_ARG, "negative type count");
        nt.n[t] = (double)type_counts[t];
    }
    if (batch > 0 && (!hist || !I_out)) return fail(SAS_ERR_INVALID_ARG, "null argument");
    if (batch == 0) return SAS_OK;
    if (batch > ((int64_t)1 << 31) / kBinCB) return fail(SAS_ERR_UNSUPPORTED, "batch too large");
    cudaStream_t s = (cudaStream_t)stream;
    const int rows = P * n_bins;
    const void *hd = nullptr;
    sas_status st = stage_in(ctx->bhist, hist, (size_t)batch * rows * sizeof(int32_t), s, hd);
    if (st != SAS_OK) return st;
    if ((st = binned_table(ctx, n_bins, r_max, s)) != SAS_OK) return st;
    ALLOC_TRY(ctx->bdiag, (size_t)Q * sizeof(double));
    k_binned_diag<<<(Q + 127) / 128, 128, 0, s>>>(ctx->F.as<double>(), T, Q, nt, ctx->bdiag.as<double>());
    CUDA_TRY(cudaGetLastError());
    const bool dev_out = on_device(I_out);
    double *I_dev = I_out;
    if (!dev_out) {
        ALLOC_TRY(ctx->bout, (size_t)batch * Q * sizeof(double));
        I_dev = ctx->bout.as<double>();
    }
    const int threads = Q >= 128 ? 128 : (Q + 31) / 32 * 32;
    dim3 grid((unsigned)((batch + kBinCB - 1) / kBinCB), (unsigned)((Q + threads - 1) / threads));
    k_binned_sum<<<grid, threads, 0, s>>>(static_cast<const int *>(hd), batch, rows, ctx->btab.as<float>(), Q,
                                          ctx->bdiag.as<double>(), I_dev);
    CUDA_TRY(cudaGetLastError());
    ctx->stats[5] = 2;
    ctx->have_partials = false;
    if (dev_out) return SAS_OK;
    HostCopies hc;
    if ((st = out_copy(hc, I_out, I_dev, (size_t)batch * Q * sizeof(double), s)) != SAS_OK) return st;
    return finish_copies(ctx, hc, s);
}

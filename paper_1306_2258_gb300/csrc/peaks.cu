// Peak microbenchmarks: the denominators of the pair kernels' rooflines, measured on the device
// they run on.  Each kernel runs independent dependency chains (8 per thread, 8 CTAs of 256
// threads per SM) of one instruction kind long enough for CUDA-event timing:
//   FFMA   scalar FP32 fused multiply-add              1 lane operation per instruction and lane
//   FFMA2  packed f32x2 fused multiply-add             2 lane operations
//   MUFU   __sinf (one multiply and one MUFU.SIN)      counted as 1 MUFU operation
//   DFMA   FP64 fused multiply-add                     1 lane operation
//   ATOMS  shared-memory integer atomic add            1 lane operation (each lane its own word,
//          a bank of its own: the conflict-free rate, the denominator of the pair histogram)
//   FFMA2 with three distinct source register pairs (each chain its own multiplier and addend, so
//          that no operand repeats between consecutive instructions): the form of the per-atom
//          kernels' cores, where every packed FMA reads three values of its own (a recurrence
//          coefficient, state and previous state; a form factor, state and accumulator)
// The chains contract toward a fixed point (x -> 0.999 x + 1e-3), so no value overflows or
// becomes subnormal.  The FFMA kernel also reads the SM clock against the global timer, which
// gives the clock the measurement ran at.
#include <cstdio>

#include "sas_internal.h"

namespace sas {

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kCtasPerSm = 8;

template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) k_peak(int iters, float m, float k, float *sink,
                                                       unsigned long long *clk)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c0 = 0, t0 = 0;
    if (KIND == 0 && tid == 0) {
        c0 = clock64();
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    }
    float r = 0.f;
    if (KIND == 0) {
        float a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = 1.f + 0.01f * (float)(c + (tid & 7));
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, k);
#pragma unroll
        for (int c = 0; c < kChains; ++c) r += a[c];
    } else if (KIND == 1) {
        float2 a[kChains];
        const float2 m2 = make_float2(m, m), k2 = make_float2(k, k);
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = make_float2(1.f + 0.01f * c, 1.f - 0.01f * (float)(tid & 7));
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = __ffma2_rn(a[c], m2, k2);
#pragma unroll
        for (int c = 0; c < kChains; ++c) r += a[c].x + a[c].y;
    } else if (KIND == 2) {
        float a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = 0.5f + 0.01f * (float)(c + (tid & 7));
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = __sinf(a[c]) + k;
#pragma unroll
        for (int c = 0; c < kChains; ++c) r += a[c];
    } else if (KIND == 5) {
        float2 a[kChains], b[kChains], d[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            a[c] = make_float2(1.f + 0.01f * c, 1.f - 0.01f * (float)(tid & 7));
            b[c] = make_float2(m - 1e-6f * c, m - 2e-6f * c - 1e-7f * (float)(tid & 3));
            d[c] = make_float2(k + 1e-6f * c, k + 2e-6f * c + 1e-7f * (float)(tid & 5));
        }
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = __ffma2_rn(b[c], a[c], d[c]);
#pragma unroll
        for (int c = 0; c < kChains; ++c) r += a[c].x + a[c].y;
    } else if (KIND == 4) {
        __shared__ int cnt[kChains][kPeakThreads];
#pragma unroll
        for (int c = 0; c < kChains; ++c) cnt[c][threadIdx.x] = 0;
        __syncthreads();
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) atomicAdd(&cnt[c][threadIdx.x], 1);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < kChains; ++c) r += (float)cnt[c][threadIdx.x];
    } else {
        double a[kChains];
        const double md = m, kd = k;
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = 1.0 + 0.01 * (double)(c + (tid & 7));
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], md, kd);
        double rd = 0.0;
#pragma unroll
        for (int c = 0; c < kChains; ++c) rd += a[c];
        r = (float)rd;
    }
    sink[tid] = r;
    if (KIND == 0 && tid == 0) {
        unsigned long long t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        clk[0] = clock64() - c0;
        clk[1] = t1 - t0;
    }
}

template <int KIND>
cudaError_t timed(int grid, int iters, float *sink, unsigned long long *clk, cudaEvent_t e0, cudaEvent_t e1,
                  cudaStream_t s, float &ms)
{
    k_peak<KIND><<<grid, kPeakThreads, 0, s>>>(iters, 0.999f, 1e-3f, sink, clk);   // warm-up
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(e0, s)) != cudaSuccess) return e;
    k_peak<KIND><<<grid, kPeakThreads, 0, s>>>(iters, 0.999f, 1e-3f, sink, clk);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(e1, s)) != cudaSuccess) return e;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
    return cudaEventElapsedTime(&ms, e0, e1);
}

}  // namespace

}  // namespace sas

using namespace sas;

extern "C" sas_status sas_measure_peaks(double *out, int n_out, void *stream)
{
    if (!out || n_out < 5) return set_error(SAS_ERR_INVALID_ARG, "need an output array of at least 5 doubles");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        return set_error(SAS_ERR_CUDA, "no CUDA device");
    }
    const int grid = sms * kCtasPerSm;
    const double threads = (double)grid * kPeakThreads;
    float *sink = nullptr;
    unsigned long long *clk = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = sas::api::dev_malloc((void **)&sink, sizeof(float) * (size_t)grid * kPeakThreads);
    if (e == cudaSuccess) e = sas::api::dev_malloc((void **)&clk, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    // iterations: about 10 ms per kernel at the expected rates
    const int it_f = 160000, it_f2 = 80000, it_m = 20000, it_d = 2500, it_a = 20000;
    if (e == cudaSuccess) e = timed<0>(grid, it_f, sink, clk, e0, e1, s, ms[0]);
    if (e == cudaSuccess) e = timed<1>(grid, it_f2, sink, clk, e0, e1, s, ms[1]);
    if (e == cudaSuccess) e = timed<2>(grid, it_m, sink, clk, e0, e1, s, ms[2]);
    if (e == cudaSuccess) e = timed<3>(grid, it_d, sink, clk, e0, e1, s, ms[3]);
    if (e == cudaSuccess && n_out >= 6) e = timed<4>(grid, it_a, sink, clk, e0, e1, s, ms[4]);
    if (e == cudaSuccess && n_out >= 7) e = timed<5>(grid, it_f2 / 2, sink, clk, e0, e1, s, ms[5]);
    unsigned long long hclk[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(hclk, clk, sizeof hclk, cudaMemcpyDeviceToHost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    sas::api::dev_free(sink);
    sas::api::dev_free(clk);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char buf[160];
        snprintf(buf, sizeof buf, "peak microbenchmarks: %s", cudaGetErrorString(e));
        return set_error(SAS_ERR_CUDA, buf);
    }
    out[0] = threads * kChains * it_f / (ms[0] * 1e-3);         // FFMA lane-ops/s
    out[1] = threads * kChains * it_f2 * 2.0 / (ms[1] * 1e-3);  // FFMA2 lane-ops/s
    out[2] = threads * kChains * it_m / (ms[2] * 1e-3);         // MUFU sin ops/s
    out[3] = threads * kChains * it_d / (ms[3] * 1e-3);         // DFMA lane-ops/s
    out[4] = hclk[1] ? (double)hclk[0] / (double)hclk[1] * 1e3 : 0.0;   // SM MHz during the FFMA run
    if (n_out >= 6) out[5] = threads * kChains * it_a / (ms[4] * 1e-3);   // shared atomic adds/s
    if (n_out >= 7) out[6] = threads * kChains * (it_f2 / 2) * 2.0 / (ms[5] * 1e-3);   // FFMA2, 3 operands
    return SAS_OK;
}

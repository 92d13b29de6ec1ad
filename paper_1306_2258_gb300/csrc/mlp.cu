// The learned surrogate: a 3-layer MLP (n_in -> h -> h -> n_out, exact-erf GELU) trained with
// MSE on a standardized log I(q), with FP32 master weights, bfloat16 GEMM operands and FP32
// accumulation on the tensor cores, and Adam.  Not part of the paper's method (which computes
// I(q) directly, Section I-A, Eq. 2); it ranks conformers before the exact kernel re-scores them.
//
// Kernels:
//   k_gemm_tn      C[M][N] = A[M][K] B[N][K]^T (+ bias), A and B bfloat16 with K contiguous (the
//                  fallback of the tcgen05 GEMM in gemm_tc.cu for operands TMA cannot describe),
//                  FP32 accumulation with mma.sync m16n8k16 (64x64 CTA tile, four 32x32 warp
//                  tiles); epilogue writes FP32 and/or bfloat16 of the value or of GELU(value).
//   k_transpose    bfloat16 [R][C] -> [C][R] (the backward GEMMs' operands)
//   k_mse_rows, k_mse_total  dY = 2 (Y - T) / (B Q) and the loss (per-row sums, then their sum; fixed order)
//   k_gelu_bwd     dZ = dA * GELU'(Z), as FP32 and bfloat16
//   k_colsum       bias gradients (8 row groups per column, then their sum; fixed order)
//   k_adam         Adam on the FP32 masters, refreshing their bfloat16 copies
// Every GEMM operand is rounded to bfloat16 exactly where the FP64 reference rounds it.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "sas_internal.h"

namespace sas {
namespace {

using bf16 = __nv_bfloat16;

constexpr int BM = 64, BN = 64, BK = 32, PADK = 8;

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad_f(float z)
{
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C = A B^T (+ bias).  Requires K % 16 == 0, lda, ldb multiples of 8 and 16-byte aligned bases.
__global__ void __launch_bounds__(128)
    k_gemm_tn(int M, int N, int K, const bf16 *__restrict__ A, int lda, const bf16 *__restrict__ B, int ldb,
              const float *__restrict__ bias, float *__restrict__ C, int ldc, bf16 *__restrict__ D, int ldd,
              int gelu)
{
    __shared__ __align__(16) bf16 As[BM][BK + PADK];
    __shared__ __align__(16) bf16 Bs[BN][BK + PADK];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;
    for (int k0 = 0; k0 < K; k0 += BK) {
        __syncthreads();
        for (int c = tid; c < BM * BK / 8; c += 128) {   // 16-byte chunks, zero outside the matrices
            const int r = c / (BK / 8), kc = (c % (BK / 8)) * 8;
            const int gk = k0 + kc;
            uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
            if (m0 + r < M && gk < K) va = *reinterpret_cast<const uint4 *>(A + (size_t)(m0 + r) * lda + gk);
            if (n0 + r < N && gk < K) vb = *reinterpret_cast<const uint4 *>(B + (size_t)(n0 + r) * ldb + gk);
            *reinterpret_cast<uint4 *>(&As[r][kc]) = va;
            *reinterpret_cast<uint4 *>(&Bs[r][kc]) = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned a[2][4], b[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r = wm + mt * 16 + g;
                a[mt][0] = *reinterpret_cast<const unsigned *>(&As[r][kk + 2 * t]);
                a[mt][1] = *reinterpret_cast<const unsigned *>(&As[r + 8][kk + 2 * t]);
                a[mt][2] = *reinterpret_cast<const unsigned *>(&As[r][kk + 2 * t + 8]);
                a[mt][3] = *reinterpret_cast<const unsigned *>(&As[r + 8][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int n = wn + nt * 8 + g;
                b[nt][0] = *reinterpret_cast<const unsigned *>(&Bs[n][kk + 2 * t]);
                b[nt][1] = *reinterpret_cast<const unsigned *>(&Bs[n][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_bf16_16816(acc[mt][nt], a[mt], b[nt]);
        }
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int r = m0 + wm + mt * 16 + g + (c >= 2 ? 8 : 0);
                const int col = n0 + wn + nt * 8 + 2 * t + (c & 1);
                if (r >= M || col >= N) continue;
                float v = acc[mt][nt][c];
                if (bias) v += bias[col];
                if (C) C[(size_t)r * ldc + col] = v;
                if (D) D[(size_t)r * ldd + col] = __float2bfloat16_rn(gelu ? gelu_f(v) : v);
            }
}

__global__ void k_to_bf16(int64_t n, const float *__restrict__ x, bf16 *__restrict__ y)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

// rows [0, R) x cols [0, C) of a [R][ldin] matrix into [C][ldout]; rows R..Rpad of the output
// columns are zeroed (batch padding)
__global__ void k_transpose(int R, int Rpad, int C, const bf16 *__restrict__ in, int ldin, bf16 *__restrict__ out,
                            int ldout)
{
    __shared__ bf16 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int r = r0 + dy, c = c0 + threadIdx.x;
        tile[dy][threadIdx.x] = (r < R && c < C) ? in[(size_t)r * ldin + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int c = c0 + dy, r = r0 + threadIdx.x;
        if (c < C && r < Rpad) out[(size_t)c * ldout + r] = tile[threadIdx.x][dy];
    }
}

// dY = 2 (Y - T) / (B Q) on the valid [B][Q] block (zero in the padding), loss = mean square
// One block per padded row b: dY, its bfloat16 copy, and the row's squared error (FP64, fixed
// tree order).
__global__ void k_mse_rows(int B, int Q, int Qpad, const float *__restrict__ Y, const float *__restrict__ T,
                           float *__restrict__ dY, bf16 *__restrict__ dYb, double *__restrict__ rows)
{
    __shared__ double red[128];
    const int b = blockIdx.x;
    const double scale = 2.0 / ((double)B * Q);
    double s = 0.0;
    for (int q = threadIdx.x; q < Qpad; q += blockDim.x) {
        const int64_t i = (int64_t)b * Qpad + q;
        float d = 0.f;
        if (b < B && q < Q) {
            const double e = (double)Y[i] - (double)T[(int64_t)b * Q + q];
            s += e * e;
            d = (float)(scale * e);
        }
        dY[i] = d;
        dYb[i] = __float2bfloat16_rn(d);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) rows[b] = red[0];
}

// loss = (sum of the row sums, fixed tree order) / (B Q)
__global__ void k_mse_total(int B, int Q, int Bpad, const double *__restrict__ rows, float *__restrict__ loss)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < Bpad; b += blockDim.x) s += rows[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(red[0] / ((double)B * Q));
}

__global__ void k_gelu_bwd(int64_t n, const float *__restrict__ dA, const float *__restrict__ Z, float *__restrict__ dZ,
                           bf16 *__restrict__ dZb)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = dA[i] * gelu_grad_f(Z[i]);
    dZ[i] = v;
    dZb[i] = __float2bfloat16_rn(v);
}

// out[c] = sum_r in[r][c] over r < R, in fixed order
// out[c] = sum over rows of in[r][c]: 32 columns per block, 8 row groups (rows r = g, g+8, ...),
// then the 8 partial sums in a fixed order.
__global__ void k_colsum(int R, int C, const float *__restrict__ in, int ld, float *__restrict__ out)
{
    __shared__ float part[8][33];
    const int c = blockIdx.x * 32 + threadIdx.x, g = threadIdx.y;
    float s = 0.f;
    if (c < C)
        for (int r = g; r < R; r += 8) s += in[(size_t)r * ld + c];
    part[g][threadIdx.x] = s;
    __syncthreads();
    if (g == 0 && c < C) {
        float t = part[0][threadIdx.x];
#pragma unroll
        for (int k = 1; k < 8; ++k) t += part[k][threadIdx.x];
        out[c] = t;
    }
}

__global__ void k_adam(int64_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                       bf16 *__restrict__ pb)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16_rn(pi);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_gemm_tn(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias,
                           float *C, int ldc, void *D, int ldd, int gelu, cudaStream_t s)
{
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    k_gemm_tn<<<grid, 128, 0, s>>>(M, N, K, static_cast<const bf16 *>(A), lda, static_cast<const bf16 *>(B), ldb, bias,
                                   C, ldc, static_cast<bf16 *>(D), ldd, gelu);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(int64_t n, const float *x, void *y, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_to_bf16<<<blocks_for(n, 256), 256, 0, s>>>(n, x, static_cast<bf16 *>(y));
    return cudaGetLastError();
}

cudaError_t launch_transpose_bf16(int R, int Rpad, int C, const void *in, int ldin, void *out, int ldout, cudaStream_t s)
{
    if (Rpad <= 0 || C <= 0) return cudaSuccess;
    dim3 grid((C + 31) / 32, (Rpad + 31) / 32);
    k_transpose<<<grid, dim3(32, 8), 0, s>>>(R, Rpad, C, static_cast<const bf16 *>(in), ldin, static_cast<bf16 *>(out),
                                             ldout);
    return cudaGetLastError();
}

cudaError_t launch_mse(int B, int Bpad, int Q, int Qpad, const float *Y, const float *T, float *dY, void *dYb,
                       double *rows, float *loss, cudaStream_t s)
{
    if (Bpad <= 0) return cudaSuccess;
    k_mse_rows<<<Bpad, 128, 0, s>>>(B, Q, Qpad, Y, T, dY, static_cast<bf16 *>(dYb), rows);
    k_mse_total<<<1, 256, 0, s>>>(B, Q, Bpad, rows, loss);
    return cudaGetLastError();
}

cudaError_t launch_gelu_bwd(int64_t n, const float *dA, const float *Z, float *dZ, void *dZb, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_gelu_bwd<<<blocks_for(n, 256), 256, 0, s>>>(n, dA, Z, dZ, static_cast<bf16 *>(dZb));
    return cudaGetLastError();
}

cudaError_t launch_colsum(int R, int C, const float *in, int ld, float *out, cudaStream_t s)
{
    if (C <= 0) return cudaSuccess;
    k_colsum<<<(C + 31) / 32, dim3(32, 8), 0, s>>>(R, C, in, ld, out);
    return cudaGetLastError();
}

cudaError_t launch_adam(int64_t n, float *p, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                        int64_t step, void *pb, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const float c1 = (float)(1.0 - std::pow((double)b1, (double)step));
    const float c2 = (float)(1.0 - std::pow((double)b2, (double)step));
    k_adam<<<blocks_for(n, 256), 256, 0, s>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2, static_cast<bf16 *>(pb));
    return cudaGetLastError();
}

}  // namespace sas

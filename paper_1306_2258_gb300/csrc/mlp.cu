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
//   k_to_bf16_t    the input to bfloat16, with its transpose (the first layer's weight-gradient operand)
//   k_transpose    bfloat16 [R][C] -> [C][R] (the backward GEMMs' operands)
//   k_splitk_gelu  the first layer's split-K slices summed in order, bias, GELU, bfloat16 and its
//                  transpose
//   k_mse_fused    dY = 2 (Y - T) / (B Q) as FP32, bfloat16 and transposed bfloat16, the output
//                  bias gradient and the loss (fixed summation orders)
//   k_act_bwd      dZ = dA * GELU'(Z) as FP32, bfloat16 and transposed bfloat16, and the bias
//                  gradient (fixed summation order)
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

// x [R][C] FP32 -> bfloat16 Xb [R][C] and its transpose Xt [C][ldt] with zero rows [R, Rpad) (batch
// padding), the operand of the first layer's weight gradient.  32 x 32 tiles, 32 x 8 threads.
__global__ void __launch_bounds__(256)
    k_to_bf16_t(int R, int Rpad, int C, const float *__restrict__ x, bf16 *__restrict__ xb, bf16 *__restrict__ xt,
                int ldt)
{
    __shared__ bf16 tile[32][34];
    const int tx = threadIdx.x, ty = threadIdx.y, c0 = blockIdx.x * 32, r0 = blockIdx.y * 32, c = c0 + tx;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = r0 + ty + 8 * k;
        bf16 h = __float2bfloat16_rn(0.f);
        if (r < R && c < C) {
            h = __float2bfloat16_rn(x[(size_t)r * C + c]);
            xb[(size_t)r * C + c] = h;
        }
        tile[ty + 8 * k][tx] = h;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {   // rows c0 + ty + 8k of xt, columns r0 + tx
        const int cc = c0 + ty + 8 * k, rr = r0 + tx;
        if (cc < C && rr < Rpad) xt[(size_t)cc * ldt + rr] = tile[tx][ty + 8 * k];
    }
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

// Split-K epilogue of the first layer: x = the slices' FP32 partials ws[z][M][N] summed in slice
// order, plus the bias; Z = x, A = bfloat16(GELU(x)), and the bfloat16 transpose At [N][ldt] of A
// with zero rows [M, Mpad) (batch padding), the operand of the weight-gradient GEMM.  32 x 32
// tiles, 32 x 8 threads.
__global__ void __launch_bounds__(256)
    k_splitk_gelu(int M, int Mpad, int N, int splits, const float *__restrict__ ws, const float *__restrict__ bias,
                  float *__restrict__ Z, bf16 *__restrict__ A, bf16 *__restrict__ At, int ldt)
{
    __shared__ bf16 tile[32][34];
    const int tx = threadIdx.x, ty = threadIdx.y, c0 = blockIdx.x * 32, r0 = blockIdx.y * 32, c = c0 + tx;
    // the four rows' sums side by side, so that their loads are in flight together
    float x[4] = {0.f, 0.f, 0.f, 0.f};
    bool in[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) in[k] = r0 + ty + 8 * k < M && c < N;
    for (int z = 0; z < splits; ++z) {
        const float *w = ws + (size_t)z * M * N + c;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (in[k]) x[k] += w[(size_t)(r0 + ty + 8 * k) * N];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = r0 + ty + 8 * k;
        bf16 a = __float2bfloat16_rn(0.f);
        if (in[k]) {
            const float v = x[k] + bias[c];
            Z[(size_t)r * N + c] = v;
            a = __float2bfloat16_rn(gelu_f(v));
            A[(size_t)r * N + c] = a;
        }
        tile[ty + 8 * k][tx] = a;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {   // rows c0 + ty + 8k of At, columns r0 + tx
        const int cc = c0 + ty + 8 * k, rr = r0 + tx;
        if (cc < N && rr < Mpad) At[(size_t)cc * ldt + rr] = tile[tx][ty + 8 * k];
    }
}

// The fused backward kernels below work on 32 x 32 tiles with 32 x 8 threads: thread (tx, ty) takes
// column c0 + tx of rows r0 + ty + 8k, k = 0..3.  Column sums (the bias gradients) run in a fixed
// order: a thread's 4 rows in order, then the 8 thread rows in order, then the row tiles in order,
// summed by the last row tile of each column strip to finish (a counter per strip, reset by that
// tile), so they repeat bit for bit.

// Column partials of one tile in order, then, in the last row tile of the strip to finish, the
// strip's column sums over the row tiles in order.  part: [row tiles][C] partials.
__device__ __forceinline__ void strip_sums(float s, int c, int C, float *__restrict__ part, float *__restrict__ out,
                                           unsigned *__restrict__ count)
{
    __shared__ float ps[8][33];
    __shared__ bool last;
    const int tx = threadIdx.x, ty = threadIdx.y;
    ps[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && c < C) {
        float t = ps[0][tx];
#pragma unroll
        for (int k = 1; k < 8; ++k) t += ps[k][tx];
        part[(size_t)blockIdx.y * C + c] = t;
        __threadfence();
    }
    __syncthreads();
    if (tx == 0 && ty == 0) last = atomicAdd(&count[blockIdx.x], 1u) == gridDim.y - 1;
    __syncthreads();
    if (!last) return;
    if (ty == 0 && c < C) {
        __threadfence();
        float t = 0.f;
        for (int y = 0; y < (int)gridDim.y; ++y) t += __ldcg(&part[(size_t)y * C + c]);
        out[c] = t;
    }
    if (tx == 0 && ty == 0) count[blockIdx.x] = 0u;
}

// Backward of z -> GELU(z) on rows [0, B) of [B][C]: dZ = dA GELU'(Z) (FP32) and bfloat16(dZ); the
// bfloat16 transpose dZt [C][ldt] with zero rows [B, Bpad) (batch padding) for the weight-gradient
// GEMM; and the bias gradient db = the column sums of dZ.
__global__ void __launch_bounds__(256)
    k_act_bwd(int B, int Bpad, int C, const float *__restrict__ dA, const float *__restrict__ Z, float *__restrict__ dZ,
              bf16 *__restrict__ dZb, bf16 *__restrict__ dZt, int ldt, float *__restrict__ part,
              float *__restrict__ db, unsigned *__restrict__ count)
{
    __shared__ bf16 tile[32][34];
    const int tx = threadIdx.x, ty = threadIdx.y, c0 = blockIdx.x * 32, r0 = blockIdx.y * 32, c = c0 + tx;
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = r0 + ty + 8 * k;
        float v = 0.f;
        if (r < B && c < C) {
            const size_t i = (size_t)r * C + c;
            v = dA[i] * gelu_grad_f(Z[i]);
            dZ[i] = v;
            dZb[i] = __float2bfloat16_rn(v);
        }
        s += v;
        tile[ty + 8 * k][tx] = __float2bfloat16_rn(v);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {   // rows c0 + ty + 8k of dZt, columns r0 + tx
        const int cc = c0 + ty + 8 * k, rr = r0 + tx;
        if (cc < C && rr < Bpad) dZt[(size_t)cc * ldt + rr] = tile[tx][ty + 8 * k];
    }
    strip_sums(s, c, C, part, db, count);
}

// The MSE loss of Y [Bpad][Qpad] against T [B][Q] and its gradient, one block per 8 padded rows
// (Bpad is a multiple of 16), thread q on column q of each row in order: dY = 2 (Y - T) / (B Q) on
// [B][Q] (zero in the rest of [Bpad][Qpad]), bfloat16(dY), and its transpose dYt [Qpad][ldt] (the
// 8 rows of a column as one 16-byte store).  Per block, FP64 squared errors (a thread's rows in
// order, then a fixed tree over the threads) into lpart and FP32 column partials into part.  The
// last block to finish then forms, in fixed orders, the loss = sum of lpart / (B Q) and the bias
// gradient db = the column partials summed over the blocks.  count: one zero-initialized counter
// (left zero).
__global__ void __launch_bounds__(128)
    k_mse_fused(int B, int Bpad, int Q, int Qpad, const float *__restrict__ Y, const float *__restrict__ T,
                float *__restrict__ dY, bf16 *__restrict__ dYb, bf16 *__restrict__ dYt, int ldt,
                double *__restrict__ lpart, float *__restrict__ part, float *__restrict__ db, float *__restrict__ loss,
                unsigned *__restrict__ count)
{
    __shared__ double red[128];
    __shared__ bool last;
    const int r0 = blockIdx.x * 8, tid = threadIdx.x;
    const double scale = 2.0 / ((double)B * Q);
    double s = 0.0;
    for (int q = tid; q < Qpad; q += blockDim.x) {
        float cs = 0.f;
        uint32_t p[4];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int r = r0 + k;
            const int64_t i = (int64_t)r * Qpad + q;
            float d = 0.f;
            if (r < B && q < Q) {
                const double e = (double)Y[i] - (double)T[(int64_t)r * Q + q];
                s += e * e;
                d = (float)(scale * e);
            }
            dY[i] = d;
            const bf16 h = __float2bfloat16_rn(d);
            dYb[i] = h;
            cs += d;
            const uint32_t u = (uint32_t)__bfloat16_as_ushort(h);
            p[k / 2] = (k & 1) ? (p[k / 2] | (u << 16)) : u;
        }
        *reinterpret_cast<uint4 *>(dYt + (int64_t)q * ldt + r0) = make_uint4(p[0], p[1], p[2], p[3]);
        part[(int64_t)blockIdx.x * Qpad + q] = cs;
    }
    red[tid] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    __threadfence();   // this block's partials before the counter
    __syncthreads();
    if (tid == 0) {
        lpart[blockIdx.x] = red[0];
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the loss: the blocks' sums, strided over the threads in order, then a fixed tree
    double t = 0.0;
    for (int y = tid; y < (int)gridDim.x; y += blockDim.x) t += __ldcg(&lpart[y]);
    red[tid] = t;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    if (tid == 0) {
        *loss = (float)(red[0] / ((double)B * Q));
        *count = 0u;
    }
    // the bias gradient: each column's block partials in block order
    for (int q = tid; q < Qpad; q += blockDim.x) {
        float c = 0.f;
#pragma unroll 8
        for (int y = 0; y < (int)gridDim.x; ++y) c += __ldcg(&part[(int64_t)y * Qpad + q]);
        db[q] = c;
    }
}

// One Adam step of element i (bias corrections c1 = 1 - b1^t, c2 = 1 - b2^t).
__device__ __forceinline__ float adam_elem(float &p, float g, float &m, float &v, float lr, float b1, float b2, float eps,
                                           float c1, float c2)
{
    m = b1 * m + (1.f - b1) * g;
    v = b2 * v + (1.f - b2) * g * g;
    p = p - lr * (m / c1) / (sqrtf(v / c2) + eps);
    return p;
}

// Four elements per thread (n is a multiple of 4: every parameter block is), 16-byte loads and
// stores; the arithmetic of each element is that of adam_elem.
__global__ void k_adam(int64_t n4, float4 *__restrict__ p, const float4 *__restrict__ g, float4 *__restrict__ m,
                       float4 *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                       uint2 *__restrict__ pb)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n4) return;
    float4 pi = p[i], mi = m[i], vi = v[i];
    const float4 gi = g[i];
    adam_elem(pi.x, gi.x, mi.x, vi.x, lr, b1, b2, eps, c1, c2);
    adam_elem(pi.y, gi.y, mi.y, vi.y, lr, b1, b2, eps, c1, c2);
    adam_elem(pi.z, gi.z, mi.z, vi.z, lr, b1, b2, eps, c1, c2);
    adam_elem(pi.w, gi.w, mi.w, vi.w, lr, b1, b2, eps, c1, c2);
    p[i] = pi;
    m[i] = mi;
    v[i] = vi;
    if (pb) {
        const __nv_bfloat162 lo = __floats2bfloat162_rn(pi.x, pi.y), hi = __floats2bfloat162_rn(pi.z, pi.w);
        pb[i] = make_uint2(*reinterpret_cast<const uint32_t *>(&lo), *reinterpret_cast<const uint32_t *>(&hi));
    }
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

cudaError_t launch_to_bf16_t(int R, int Rpad, int C, const float *x, void *xb, void *xt, int ldt, cudaStream_t s)
{
    if (Rpad <= 0 || C <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((C + 31) / 32), (unsigned)((Rpad + 31) / 32));
    k_to_bf16_t<<<grid, dim3(32, 8), 0, s>>>(R, Rpad, C, x, static_cast<bf16 *>(xb), static_cast<bf16 *>(xt), ldt);
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

cudaError_t launch_splitk_gelu(int M, int Mpad, int N, int splits, const float *ws, const float *bias, float *Z, void *A,
                               void *At, int ldt, cudaStream_t s)
{
    if (Mpad <= 0 || N <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((N + 31) / 32), (unsigned)((Mpad + 31) / 32));
    k_splitk_gelu<<<grid, dim3(32, 8), 0, s>>>(M, Mpad, N, splits, ws, bias, Z, static_cast<bf16 *>(A),
                                               static_cast<bf16 *>(At), ldt);
    return cudaGetLastError();
}

cudaError_t launch_mse_fused(int B, int Bpad, int Q, int Qpad, const float *Y, const float *T, float *dY, void *dYb,
                             void *dYt, int ldt, double *lpart, float *part, float *db, float *loss, unsigned *count,
                             cudaStream_t s)
{
    if (Bpad <= 0 || Qpad <= 0) return cudaSuccess;
    if (Bpad % 8 != 0 || ldt % 8 != 0) return cudaErrorInvalidValue;   // 16-byte column stores of dYt
    k_mse_fused<<<Bpad / 8, 128, 0, s>>>(B, Bpad, Q, Qpad, Y, T, dY, static_cast<bf16 *>(dYb), static_cast<bf16 *>(dYt),
                                         ldt, lpart, part, db, loss, count);
    return cudaGetLastError();
}

cudaError_t launch_act_bwd(int B, int Bpad, int C, const float *dA, const float *Z, float *dZ, void *dZb, void *dZt,
                           int ldt, float *part, float *db, unsigned *count, cudaStream_t s)
{
    if (Bpad <= 0 || C <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((C + 31) / 32), (unsigned)((Bpad + 31) / 32));
    k_act_bwd<<<grid, dim3(32, 8), 0, s>>>(B, Bpad, C, dA, Z, dZ, static_cast<bf16 *>(dZb), static_cast<bf16 *>(dZt),
                                           ldt, part, db, count);
    return cudaGetLastError();
}

cudaError_t launch_adam(int64_t n, float *p, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                        int64_t step, void *pb, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const float c1 = (float)(1.0 - std::pow((double)b1, (double)step));
    const float c2 = (float)(1.0 - std::pow((double)b2, (double)step));
    if (n % 4 != 0) return cudaErrorInvalidValue;
    k_adam<<<blocks_for(n / 4, 256), 256, 0, s>>>(n / 4, reinterpret_cast<float4 *>(p), reinterpret_cast<const float4 *>(g),
                                                  reinterpret_cast<float4 *>(m), reinterpret_cast<float4 *>(v), lr, b1,
                                                  b2, eps, c1, c2, static_cast<uint2 *>(pb));
    return cudaGetLastError();
}

}  // namespace sas

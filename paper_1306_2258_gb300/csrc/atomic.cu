// Per-atom form factors (Section I-A, Eq. 2 with a form factor per atom and q, as the paper's
// kernel keeps them, Section II): validation, the tables the pair kernels read, the diagonal, and
// the assembly
//
//   I(q) = sum_i f_i(q)^2 + 2 U(q)/q,   U(q) = sum_{i<j} f_i(q) f_j(q) sin(q r_ij)/r_ij,
//   I(0) = (sum_i f_i(0))^2                (sinc(0) = 1 for every pair and the diagonal).
//
// The caller's table is ff[b][k][i] = f_i(q_k) (FP64, one row of N atoms per q).  With no types the
// packed order is the caller's order (slot_of maps atom -> slot) and padding slots get f = 0.
#include <algorithm>

#include "sas_internal.h"

namespace sas {

namespace {

__global__ void k_check_finite(const double *__restrict__ v, int64_t count, int *err)
{
    int bad = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(v[k]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, kErrNonFiniteFF);
}

// One thread per (atom i, slot v) of chunk blockIdx.y, conformer blockIdx.z:
//   FI[b][c][v][slot]            = (f_i(q_2v), f_i(q_2v+1))
//   FJ[b][c][slot / 2][v] half   = the same pair, in the .xy (even slot) or .zw (odd slot) half
// with q_m the m-th value of the chunk and 0 past its end.
__global__ void k_atomic_tables(const double *__restrict__ ff, const int *__restrict__ slot_of, int64_t n,
                                int64_t npad, QChunks qc, int nv, float4 *__restrict__ FJ, float2 *__restrict__ FI)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * nv) return;
    const int64_t atom = i % n;
    const int v = (int)(i / n);
    const int c = blockIdx.y;
    const int64_t b = blockIdx.z;
    const int k0 = 2 * v, k1 = 2 * v + 1, len = qc.q_len[c];
    const double *fb = ff + b * qc.n_q * n;
    const float f0 = k0 < len ? (float)fb[(int64_t)(qc.q_begin[c] + k0) * n + atom] : 0.f;
    const float f1 = k1 < len ? (float)fb[(int64_t)(qc.q_begin[c] + k1) * n + atom] : 0.f;
    const int64_t slot = slot_of[atom];
    const int64_t tab = b * qc.n_chunks + c;
    FI[(tab * nv + v) * npad + slot] = make_float2(f0, f1);
    reinterpret_cast<float2 *>(FJ)[2 * ((tab * (npad / 2) + slot / 2) * nv + v) + (slot & 1)] = make_float2(f0, f1);
}

// F64[b][slot][k] = f_i(q_k) for the FP64 kernel (atom-major: one pair's q run is contiguous).
__global__ void k_atomic_table64(const double *__restrict__ ff, const int *__restrict__ slot_of, int64_t n,
                                 int64_t npad, int n_q, double *__restrict__ F64)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * n_q) return;
    const int64_t atom = i % n;
    const int k = (int)(i / n);
    const int64_t b = blockIdx.y;
    F64[(b * npad + slot_of[atom]) * n_q + k] = ff[(b * n_q + k) * n + atom];
}

// D[b][k] = (sum_i f_i(q_k)^2, sum_i f_i(q_k)): one CTA per (k, b), a fixed-order tree sum.
constexpr int kDiagThreads = 256;

__global__ void __launch_bounds__(kDiagThreads)
    k_atomic_diag(const double *__restrict__ ff, int64_t n, int n_q, double2 *__restrict__ D)
{
    __shared__ double s2[kDiagThreads], s1[kDiagThreads];
    const int k = blockIdx.x;
    const int64_t b = blockIdx.y;
    const double *row = ff + (b * n_q + k) * n;
    double a2 = 0.0, a1 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kDiagThreads) {
        const double f = row[i];
        a2 = fma(f, f, a2);
        a1 += f;
    }
    s2[threadIdx.x] = a2;
    s1[threadIdx.x] = a1;
    __syncthreads();
    for (int h = kDiagThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s2[threadIdx.x] += s2[threadIdx.x + h];
            s1[threadIdx.x] += s1[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) D[b * n_q + k] = make_double2(s2[0], s1[0]);
}

// S[b][k] = U(q_k)/q_k from the item reduction (one type pair per conformer).
__global__ void k_assemble_atomic(const double *__restrict__ S, const double2 *__restrict__ D, QChunks qc,
                                  double *__restrict__ I)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b = blockIdx.y;
    if (k >= qc.n_q) return;
    const double2 d = D[b * qc.n_q + k];
    I[b * qc.n_q + k] = q_at(qc, k) > 0.0 ? d.x + 2.0 * S[b * qc.n_q + k] : d.y * d.y;
}

}  // namespace

cudaError_t launch_check_finite(const double *v, int64_t count, int *err, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((count + threads - 1) / threads, 4096);
    k_check_finite<<<(unsigned)blocks, threads, 0, s>>>(v, count, err);
    return cudaGetLastError();
}

cudaError_t launch_atomic_tables(const double *ff, const int *slot_of, int64_t n, int64_t npad, int64_t batch,
                                 const QChunks &qc, int nv, float4 *FJ, float2 *FI, cudaStream_t s)
{
    if (n == 0 || batch == 0) return cudaSuccess;
    const int threads = 256;
    const dim3 grid((unsigned)((n * nv + threads - 1) / threads), (unsigned)qc.n_chunks, (unsigned)batch);
    k_atomic_tables<<<grid, threads, 0, s>>>(ff, slot_of, n, npad, qc, nv, FJ, FI);
    return cudaGetLastError();
}

cudaError_t launch_atomic_table64(const double *ff, const int *slot_of, int64_t n, int64_t npad, int64_t batch,
                                  int n_q, double *F64, cudaStream_t s)
{
    if (n == 0 || batch == 0) return cudaSuccess;
    const int threads = 256;
    const dim3 grid((unsigned)((n * n_q + threads - 1) / threads), (unsigned)batch);
    k_atomic_table64<<<grid, threads, 0, s>>>(ff, slot_of, n, npad, n_q, F64);
    return cudaGetLastError();
}

cudaError_t launch_atomic_diag(const double *ff, int64_t n, int64_t batch, int n_q, double2 *D, cudaStream_t s)
{
    if (batch == 0) return cudaSuccess;
    k_atomic_diag<<<dim3((unsigned)n_q, (unsigned)batch), kDiagThreads, 0, s>>>(ff, n, n_q, D);
    return cudaGetLastError();
}

cudaError_t launch_assemble_atomic(const double *S, const double2 *D, const QChunks &qc, int64_t batch, double *I,
                                   cudaStream_t s)
{
    if (batch == 0) return cudaSuccess;
    k_assemble_atomic<<<dim3((unsigned)((qc.n_q + 127) / 128), (unsigned)batch), 128, 0, s>>>(S, D, qc, I);
    return cudaGetLastError();
}

}  // namespace sas

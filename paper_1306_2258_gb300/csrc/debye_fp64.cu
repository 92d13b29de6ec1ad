// All-FP64 pair kernel: the plain form of the Debye sum (Section I-A, Eq. 2)
// that the mixed-precision kernel is measured against.
//
// Same work items and loop order as the mixed kernel (distance once per pair,
// q innermost), every operation in double: r by sqrt, seeds from the library
// sincos of the chunk's start phase and of t = dq*r, then the three-term
// angle-addition identity sin(x + t) = 2 cos(t) sin(x) - sin(x - t) over the
// chunk.  FP64 needs no re-seeding over 208 steps.  The same kernel serves per-atom form
// factors (each term weighted by f_i(q) f_j(q)).  The FP64 pipe is the
// bound, so the per-thread accumulators live in shared memory
// ([q][thread], conflict-free) and the J atoms are read straight from L1
// (a warp-uniform address is one broadcast transaction).
#include "sas_internal.h"

namespace sas {

namespace {

// ATOMIC: per-atom form factors F64 [batch][npad][n_q] (by packed slot): each term is weighted by
// f_j(q) and each thread's sums by f_i(q) before the block sum.
template <bool ATOMIC>
__global__ void __launch_bounds__(kTile64, 2)
    k_debye_fp64(const double4 *__restrict__ X, int64_t npad, const Item *__restrict__ items,
                 int n_items, QChunks qc, const double *__restrict__ F64, double *__restrict__ partial,
                 int part_stride)
{
    extern __shared__ double acc[];   // [kQChunk][kTile64]
    const int tid = threadIdx.x;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const Item item = items[it];
        const double4 *Xb = X + (int64_t)item.batch * npad;
        const double4 xi = Xb[item.i0 + tid];
        const int ch = item.chunk;
        const int qlen = qc.q_len[ch];
        const double qs = qc.qsd[ch], dq = qc.dqd[ch];
        const double *Fb = ATOMIC ? F64 + (int64_t)item.batch * npad * qc.n_q + qc.q_begin[ch] : nullptr;
        __syncthreads();   // the previous item's block sum is done with acc
        for (int k = 0; k < qlen; ++k) acc[k * kTile64 + tid] = 0.0;
        const int jmask = item.diag ? tid : -1;
        for (int j = 0; j < item.jlen; ++j) {
            const double4 xj = Xb[item.j0 + j];
            const double w = (j <= jmask) ? 0.0 : xi.w * xj.w;
            const double dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
            const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
            const double r = r2 > 0.0 ? sqrt(r2) : 1e-9;   // coincident atoms: sin(q r)/r -> q
            const double scale = w / r;
            double st, ct;
            sincos(dq * r, &st, &ct);
            double S = 0.0, C = scale;
            if (qs != 0.0) {
                double s0, c0;
                sincos(qs * r, &s0, &c0);
                S = scale * s0;
                C = scale * c0;
            }
            const double *fj = ATOMIC ? Fb + (int64_t)(item.j0 + j) * qc.n_q : nullptr;
            double sp = S;                    // term at q_begin
            double sc = fma(S, ct, C * st);   // term at q_begin + 1
            const double twoc = 2.0 * ct;
            if (ATOMIC) {
                acc[tid] = fma(fj[0], sp, acc[tid]);
                if (qlen > 1) acc[kTile64 + tid] = fma(fj[1], sc, acc[kTile64 + tid]);
            } else {
                acc[tid] += sp;
                if (qlen > 1) acc[kTile64 + tid] += sc;
            }
            for (int k = 2; k < qlen; ++k) {
                const double sn = fma(twoc, sc, -sp);
                if (ATOMIC)
                    acc[k * kTile64 + tid] = fma(fj[k], sn, acc[k * kTile64 + tid]);
                else
                    acc[k * kTile64 + tid] += sn;
                sp = sc;
                sc = sn;
            }
        }
        if (ATOMIC) {   // f_i(q) of this thread's atom (zero on padding slots)
            const double *fi = Fb + (int64_t)(item.i0 + tid) * qc.n_q;
            for (int k = 0; k < qlen; ++k) acc[k * kTile64 + tid] *= fi[k];
        }
        __syncthreads();
        for (int k = tid; k < qlen; k += kTile64) {   // fixed-order block sum
            double s = 0.0;
            for (int t = 0; t < kTile64; ++t) s += acc[k * kTile64 + t];
            partial[(int64_t)it * part_stride + k] = s;
        }
    }
}

template <bool ATOMIC>
cudaError_t launch_fp64(const double4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                        const double *F64, double *partial, int part_stride, int grid, cudaStream_t s)
{
    if (n_items == 0) return cudaSuccess;
    const size_t smem = (size_t)kQChunk * kTile64 * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_debye_fp64<ATOMIC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_debye_fp64<ATOMIC><<<grid, kTile64, smem, s>>>(X, npad, items, n_items, qc, F64, partial, part_stride);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_debye_fp64(const double4 *X, int64_t npad, const Item *items, int n_items,
                              const QChunks &qc, double *partial, int part_stride, int grid,
                              cudaStream_t s)
{
    return launch_fp64<false>(X, npad, items, n_items, qc, nullptr, partial, part_stride, grid, s);
}

cudaError_t launch_debye_fp64_atomic(const double4 *X, int64_t npad, const Item *items, int n_items,
                                     const QChunks &qc, const double *F64, double *partial, int part_stride,
                                     int grid, cudaStream_t s)
{
    return launch_fp64<true>(X, npad, items, n_items, qc, F64, partial, part_stride, grid, s);
}

}  // namespace sas

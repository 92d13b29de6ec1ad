// Form factors, the deterministic cross-item reduction, and the assembly of I(q).
//
// The paper reduces each workgroup's private totals in local memory, writes
// one total per workgroup to global memory and finishes the sum on the host
// (Section II).  Here every item's FP64 partial is summed on the device in a
// fixed order (the order of the item list), so repeated calls give the same
// bits; the form factors enter only now, once per type pair and q:
//
//   I(q) = sum_t n_t f_t(q)^2 + sum_{a<=b} 2 f_a(q) f_b(q) S_ab(q),
//   S_ab(q) = sum over unordered pairs of types {a,b} of sinc(q r) = U_ab(q) / q,
//
// where U_ab(q) = sum sin(q r)/r is what the pair kernels accumulate; at q = 0
// S_ab is the exact pair count (sinc(0) = 1).  A deterministic context sums the
// partials exactly instead (as 128-bit fixed-point integers), so that the shares
// of a work list split into shards add up to the unsplit sums bit for bit.
#include "sas_internal.h"

namespace sas {

namespace {

__device__ __forceinline__ double qval(const QChunks &qc, int k) { return q_at(qc, k); }

// f_t(q) = sum_{k<4} a_k exp(-b_k (q/4pi)^2) + c
__global__ void k_form_factors(const double *coef, int n_types, QChunks qc, double *F)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    if (k >= qc.n_q || t >= n_types) return;
    const double s = qval(qc, k) / (4.0 * 3.14159265358979323846);
    const double *c = coef + 9 * t;
    double f = c[8];
    for (int m = 0; m < 4; ++m) f += c[m] * exp(-c[4 + m] * s * s);
    F[t * qc.n_q + k] = f;
}

__global__ void k_reduce_items(const double *partial, int part_stride, const Item *items,
                               const int *group_items, const int *group_off, QChunks qc, double *S)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = blockIdx.y;
    if (k >= qc.n_q) return;
    double s = 0.0;
    for (int idx = group_off[g]; idx < group_off[g + 1]; ++idx) {
        const int it = group_items[idx];
        const int ch = items[it].chunk;
        const int kk = k - qc.q_begin[ch];
        if (kk >= 0 && kk < qc.q_len[ch]) s += partial[(int64_t)it * part_stride + kk];
    }
    // U(q) -> S(q) = U/q; at q = 0 the exact count of pairs is filled in by k_assemble
    const double q = qval(qc, k);
    S[(int64_t)g * qc.n_q + k] = q > 0.0 ? s / q : 0.0;
}

// Two-level form for groups of many items (one type pair over a long work list): block (seg, g)
// sums items [seg * kSegItems, ...) of group g in list order for every q (threads along q, so the
// partials are read coalesced); k_reduce_finish adds the segments in order.  A group of at most
// kSegItems items gets exactly the single-level result.
__global__ void k_reduce_segments(const double *partial, int part_stride, const Item *items, const int *group_items,
                                  const int *group_off, QChunks qc, int max_seg, double *seg_out)
{
    const int g = blockIdx.y, seg = blockIdx.x;
    const int b = group_off[g] + seg * kSegItems, e = min(group_off[g + 1], b + kSegItems);
    if (b >= e) return;
    for (int k = threadIdx.x; k < qc.n_q; k += blockDim.x) {
        double s = 0.0;
        for (int idx = b; idx < e; ++idx) {
            const int it = group_items[idx];
            const int ch = items[it].chunk;
            const int kk = k - qc.q_begin[ch];
            if (kk >= 0 && kk < qc.q_len[ch]) s += partial[(int64_t)it * part_stride + kk];
        }
        seg_out[((int64_t)g * max_seg + seg) * qc.n_q + k] = s;
    }
}

__global__ void k_reduce_finish(const double *seg_out, const int *group_off, QChunks qc, int max_seg, double *S)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = blockIdx.y;
    if (k >= qc.n_q) return;
    const int nseg = (group_off[g + 1] - group_off[g] + kSegItems - 1) / kSegItems;
    double s = 0.0;
    for (int seg = 0; seg < nseg; ++seg) s += seg_out[((int64_t)g * max_seg + seg) * qc.n_q + k];
    const double q = qval(qc, k);
    S[(int64_t)g * qc.n_q + k] = q > 0.0 ? s / q : 0.0;
}

__device__ __forceinline__ void fix_add(Fix128 &a, const Fix128 &b)
{
    const unsigned long long lo = a.lo + b.lo;
    a.hi += b.hi + (long long)(lo < a.lo);
    a.lo = lo;
}

__device__ __forceinline__ void fix_negate(Fix128 &a)
{
    a.lo = ~a.lo + 1ull;
    a.hi = ~a.hi + (long long)(a.lo == 0ull);
}

// the integer nearest v 2^kFixBits: its magnitude split at 2^64 (both parts exact in FP64, the low
// one holding fewer than 53 significant bits), then the sign
__device__ __forceinline__ Fix128 fix_from(double v)
{
    const double x = rint(ldexp(v, kFixBits));
    const double m = fabs(x);
    const double mh = floor(ldexp(m, -64));
    const double ml = m - ldexp(mh, 64);
    Fix128 r{(unsigned long long)ml, (long long)mh};
    if (x < 0.0) fix_negate(r);
    return r;
}

// a fixed function of the integer (magnitude hi 2^64 + lo, rounded), times 2^-kFixBits
__device__ __forceinline__ double fix_to(Fix128 a)
{
    const bool neg = a.hi < 0;
    if (neg) fix_negate(a);
    const double d = fma((double)(unsigned long long)a.hi, 18446744073709551616.0, (double)a.lo);
    return ldexp(neg ? -d : d, -kFixBits);
}

__global__ void k_reduce_segments_fix(const double *partial, int part_stride, const Item *items,
                                      const int *group_items, const int *group_off, QChunks qc, int max_seg,
                                      Fix128 *seg_out)
{
    const int g = blockIdx.y, seg = blockIdx.x;
    const int b = group_off[g] + seg * kSegItems, e = min(group_off[g + 1], b + kSegItems);
    if (b >= e) return;
    for (int k = threadIdx.x; k < qc.n_q; k += blockDim.x) {
        Fix128 s{0ull, 0ll};
        for (int idx = b; idx < e; ++idx) {
            const int it = group_items[idx];
            const int ch = items[it].chunk;
            const int kk = k - qc.q_begin[ch];
            if (kk >= 0 && kk < qc.q_len[ch]) fix_add(s, fix_from(partial[(int64_t)it * part_stride + kk]));
        }
        seg_out[((int64_t)g * max_seg + seg) * qc.n_q + k] = s;
    }
}

__global__ void k_reduce_finish_fix(const Fix128 *seg_out, const int *group_off, QChunks qc, int max_seg, Fix128 *U)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = blockIdx.y;
    if (k >= qc.n_q) return;
    const int nseg = (group_off[g + 1] - group_off[g] + kSegItems - 1) / kSegItems;
    Fix128 s{0ull, 0ll};
    for (int seg = 0; seg < nseg; ++seg) fix_add(s, seg_out[((int64_t)g * max_seg + seg) * qc.n_q + k]);
    U[(int64_t)g * qc.n_q + k] = s;
}

__global__ void k_fix_to_S(const Fix128 *U, int64_t n, QChunks qc, double *S)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const double q = qval(qc, (int)(idx % qc.n_q));
    S[idx] = q > 0.0 ? fix_to(U[idx]) / q : 0.0;
}

// whole = 0 (a shard other than the first of a split work list): no diagonal, and S(0) = 0, since
// the first shard carries the exact pair counts at q = 0.
__global__ void k_assemble(double *S, const double *F, const int *meta, int n_types, QChunks qc, int whole,
                           double *I)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b = blockIdx.y;
    if (k >= qc.n_q) return;
    const int P = n_types * (n_types + 1) / 2;
    const bool q0 = !(qval(qc, k) > 0.0);
    double acc = 0.0;
    for (int t = 0; whole && t < n_types; ++t) {
        const double f = F[t * qc.n_q + k];
        acc += (double)meta[t] * f * f;   // the diagonal, exactly
    }
    int p = 0;
    for (int a = 0; a < n_types; ++a)
        for (int c = a; c < n_types; ++c, ++p) {
            double *Sp = S + (b * P + p) * qc.n_q + k;
            if (q0) {   // sinc(0) = 1: the number of unordered pairs of types {a, c}
                const double na = meta[a], nc = meta[c];
                *Sp = !whole ? 0.0 : (a == c) ? na * (na - 1.0) * 0.5 : na * nc;
            }
            acc += 2.0 * F[a * qc.n_q + k] * F[c * qc.n_q + k] * (*Sp);
        }
    I[b * qc.n_q + k] = acc;
}

}  // namespace

cudaError_t launch_form_factors(const double *coef, int n_types, const QChunks &qc, double *F,
                                cudaStream_t s)
{
    dim3 grid((qc.n_q + 127) / 128, n_types);
    k_form_factors<<<grid, 128, 0, s>>>(coef, n_types, qc, F);
    return cudaGetLastError();
}

cudaError_t launch_reduce_items(const double *partial, int part_stride, const Item *items,
                                const int *group_items, const int *group_off, int n_groups,
                                const QChunks &qc, double *S, cudaStream_t s)
{
    if (n_groups == 0) return cudaSuccess;
    dim3 grid((qc.n_q + 127) / 128, n_groups);
    k_reduce_items<<<grid, 128, 0, s>>>(partial, part_stride, items, group_items, group_off, qc, S);
    return cudaGetLastError();
}

cudaError_t launch_reduce_items_seg(const double *partial, int part_stride, const Item *items,
                                    const int *group_items, const int *group_off, int n_groups, int max_group,
                                    const QChunks &qc, double *seg_out, double *S, cudaStream_t s)
{
    if (n_groups == 0) return cudaSuccess;
    if (max_group <= kSegItems)
        return launch_reduce_items(partial, part_stride, items, group_items, group_off, n_groups, qc, S, s);
    const int max_seg = (max_group + kSegItems - 1) / kSegItems;
    k_reduce_segments<<<dim3((unsigned)max_seg, (unsigned)n_groups), 256, 0, s>>>(partial, part_stride, items,
                                                                                  group_items, group_off, qc,
                                                                                  max_seg, seg_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_finish<<<dim3((unsigned)((qc.n_q + 127) / 128), (unsigned)n_groups), 128, 0, s>>>(seg_out, group_off, qc,
                                                                                               max_seg, S);
    return cudaGetLastError();
}

cudaError_t launch_fix_to_S(const Fix128 *U, int64_t n_groups, const QChunks &qc, double *S, cudaStream_t s)
{
    const int64_t n = n_groups * qc.n_q;
    if (n == 0) return cudaSuccess;
    k_fix_to_S<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(U, n, qc, S);
    return cudaGetLastError();
}

cudaError_t launch_reduce_items_fix(const double *partial, int part_stride, const Item *items,
                                    const int *group_items, const int *group_off, int n_groups, int max_group,
                                    const QChunks &qc, Fix128 *seg_out, Fix128 *U, double *S, cudaStream_t s)
{
    if (n_groups == 0) return cudaSuccess;
    const int max_seg = max_group > kSegItems ? (max_group + kSegItems - 1) / kSegItems : 1;
    k_reduce_segments_fix<<<dim3((unsigned)max_seg, (unsigned)n_groups), 256, 0, s>>>(
        partial, part_stride, items, group_items, group_off, qc, max_seg, seg_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_finish_fix<<<dim3((unsigned)((qc.n_q + 127) / 128), (unsigned)n_groups), 128, 0, s>>>(
        seg_out, group_off, qc, max_seg, U);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_fix_to_S(U, n_groups, qc, S, s);
}

cudaError_t launch_assemble(double *S, const double *F, const int *meta, int n_types, int64_t batch,
                            const QChunks &qc, int whole, double *I, cudaStream_t s)
{
    if (batch == 0) return cudaSuccess;
    dim3 grid((qc.n_q + 127) / 128, (unsigned)batch);
    k_assemble<<<grid, 128, 0, s>>>(S, F, meta, n_types, qc, whole, I);
    return cudaGetLastError();
}

}  // namespace sas

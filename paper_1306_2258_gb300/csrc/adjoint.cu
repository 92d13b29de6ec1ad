// Adjoint of the Debye sum: the gradient of a loss L(I) with respect to the
// atom positions, given g_q = dL/dI(q).  The paper computes only I(q)
// (Section I-A, Eq. 2); this is the derivative of that sum:
//
//   dI(q)/dx_i = sum_{j != i} 2 f_i f_j (cos(q r) - sinc(q r)) / r^2 (x_i - x_j)
//   G_i = sum_q g_q dI(q)/dx_i = sum_{j != i} W_ij (x_i - x_j),
//   W_ij = (2 / r^2) (A - B / r),  A = sum_q h_q cos(q r),  B = sum_q (h_q / q) sin(q r),
//   h_q = g_q f_a(q) f_b(q)   (q = 0 contributes nothing: cos 0 - sinc 0 = 0).
//
// Same work items as the forward kernel.  Each thread owns atom i of the
// I-tile and handles two J atoms per step.  For each pair, cos(q r) and
// sin(q r) run together as a float2 through the 4-step three-term recurrence
// (one packed FMA per q), and (A, B) accumulate with a second packed FMA
// against (h_q, h_q/q), which sits in shared memory and is read as float4
// broadcasts (one load serves two q values and both pairs).  W_ij is applied
// at once: the thread's own G_i accumulates in registers, and -W_ij (x_i - x_j)
// for atom j is summed over the warp with shuffles and over the block in
// shared memory.  Item totals go to a [batch][slot][3] FP64 array with FP64
// atomics.
#include "sas_internal.h"
#include "sincos_f32.cuh"

namespace sas {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }

struct PairSetup {
    float2 prev[4], cur[4];   // (cos, sin) at q_k for the 4 interleaved sequences
    float2 C4;                // (2 cos 4t, 2 cos 4t)
    float rinv;
};

__device__ __forceinline__ float coef_sr(float mu, unsigned hash)
{
    const float c = 2.f - mu;
    const float e = (2.f - c) - mu;
    const float ulp = __int_as_float(__float_as_int(fabsf(c)) & 0x7f800000) * 1.1920928955078125e-7f;
    const float u = (float)(hash >> 8) * 5.9604644775390625e-8f;
    return (u * ulp < fabsf(e)) ? c + copysignf(ulp, e) : c;
}

__device__ __forceinline__ unsigned pair_hash(unsigned i, unsigned j)
{
    unsigned h = i * 0x9E3779B1u ^ (j * 0x85EBCA77u + 0x165667B1u);
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return h;
}

// Distance, seeds and the stochastically rounded coefficient 2cos(4t) of one pair
// (the same construction as the forward kernel's).
__device__ __forceinline__ void setup_pair(const float4 xi, const float4 xj, float qs_hi, float qs_lo,
                                           bool zero_start, float dq_hi, float dq_lo, unsigned hash,
                                           PairSetup &p)
{
    const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
    float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    r2 = fmaxf(r2, 1e-12f);
    const float r = sqrtf(r2);
    p.rinv = rsqrtf(r2);
    const float t = fmaf(dq_hi, r, dq_lo * r);
    const SinCos b1 = sincos_f32(t);
    const float c1 = b1.c, s1 = b1.s;
    // cos(j t), sin(j t), j = 0..7, by angle addition and doubling
    float cj[8], sj[8];
    cj[0] = 1.f;
    sj[0] = 0.f;
    cj[1] = c1;
    sj[1] = s1;
    sj[2] = 2.f * s1 * c1;
    cj[2] = fmaf(-2.f * s1, s1, 1.f);
    cj[3] = fmaf(cj[2], c1, -sj[2] * s1);
    sj[3] = fmaf(sj[2], c1, cj[2] * s1);
    sj[4] = 2.f * sj[2] * cj[2];
    cj[4] = fmaf(-2.f * sj[2], sj[2], 1.f);
    cj[5] = fmaf(cj[4], c1, -sj[4] * s1);
    sj[5] = fmaf(sj[4], c1, cj[4] * s1);
    sj[6] = 2.f * sj[3] * cj[3];
    cj[6] = fmaf(-2.f * sj[3], sj[3], 1.f);
    cj[7] = fmaf(cj[6], c1, -sj[6] * s1);
    sj[7] = fmaf(sj[6], c1, cj[6] * s1);
    const float c4 = coef_sr(4.f * sj[2] * sj[2], hash);
    p.C4 = make_float2(c4, c4);
    float S = 0.f, C = 1.f;
    if (!zero_start) {
        const SinCos ph = sincos_f32(fmaf(qs_hi, r, qs_lo * r));
        S = ph.s;
        C = ph.c;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {   // cos/sin of (phi0 + j t) = rotation of (C, S) by j t
        p.prev[m] = make_float2(fmaf(C, cj[m], -S * sj[m]), fmaf(S, cj[m], C * sj[m]));
        p.cur[m] = make_float2(fmaf(C, cj[m + 4], -S * sj[m + 4]), fmaf(S, cj[m + 4], C * sj[m + 4]));
    }
}

template <int NB>
__global__ void __launch_bounds__(kTile, 2)
    k_debye_adjoint(const float4 *__restrict__ X, int64_t npad, const Item *__restrict__ items,
                    int n_items, QChunks qc, const float2 *__restrict__ H, int n_pairs, int hstride,
                    double *__restrict__ G, int jmax)
{
    extern __shared__ float4 smem[];
    float4 *sj = smem;                                   // [jmax]
    float4 *sh = smem + jmax;                            // [2*NB]: (h, h/q) for q 2k and 2k+1
    float *gj = reinterpret_cast<float *>(sh + 2 * NB);  // [jmax][3]
    const int tid = threadIdx.x, lane = tid & 31;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const Item item = items[it];
        const float4 *Xb = X + (int64_t)item.batch * npad;
        const int ch = item.chunk;
        __syncthreads();
        for (int j = tid; j < item.jlen; j += kTile) {
            sj[j] = Xb[item.j0 + j];
            gj[3 * j] = gj[3 * j + 1] = gj[3 * j + 2] = 0.f;
        }
        const float2 *Hc = H + ((int64_t)item.batch * n_pairs + item.pair) * hstride + qc.q_begin[ch];
        const int qlen = qc.q_len[ch];
        for (int k = tid; k < 2 * NB; k += kTile) {   // zero beyond the chunk's q values
            const float2 a = (2 * k < qlen) ? Hc[2 * k] : make_float2(0.f, 0.f);
            const float2 b = (2 * k + 1 < qlen) ? Hc[2 * k + 1] : make_float2(0.f, 0.f);
            sh[k] = make_float4(a.x, a.y, b.x, b.y);
        }
        const float4 xi = Xb[item.i0 + tid];
        __syncthreads();
        const float qs_hi = qc.qs_hi[ch], qs_lo = qc.qs_lo[ch];
        const bool zero_start = (qs_hi == 0.f) && (qs_lo == 0.f);
        const int jmask = item.diag ? tid : -1;
        float gx = 0.f, gy = 0.f, gz = 0.f;
        for (int j = 0; j < item.jlen; j += 2) {
            const float4 xa = sj[j], xb = sj[j + 1];
            PairSetup pa, pb;
            setup_pair(xi, xa, qs_hi, qs_lo, zero_start, qc.dq_hi, qc.dq_lo,
                       pair_hash(item.i0 + tid, item.j0 + j), pa);
            setup_pair(xi, xb, qs_hi, qs_lo, zero_start, qc.dq_hi, qc.dq_lo,
                       pair_hash(item.i0 + tid, item.j0 + j + 1), pb);
            float2 aa[4], ab[4];
            {
                const float4 h01 = sh[0], h23 = sh[1], h45 = sh[2], h67 = sh[3];
                const float2 h[8] = {make_float2(h01.x, h01.y), make_float2(h01.z, h01.w),
                                     make_float2(h23.x, h23.y), make_float2(h23.z, h23.w),
                                     make_float2(h45.x, h45.y), make_float2(h45.z, h45.w),
                                     make_float2(h67.x, h67.y), make_float2(h67.z, h67.w)};
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    aa[m] = f2fma(h[m], pa.prev[m], make_float2(0.f, 0.f));
                    aa[m] = f2fma(h[m + 4], pa.cur[m], aa[m]);
                    ab[m] = f2fma(h[m], pb.prev[m], make_float2(0.f, 0.f));
                    ab[m] = f2fma(h[m + 4], pb.cur[m], ab[m]);
                }
            }
#pragma unroll
            for (int blk = 2; blk < NB; ++blk) {
                const float4 hA = sh[2 * blk], hB = sh[2 * blk + 1];
                const float2 h[4] = {make_float2(hA.x, hA.y), make_float2(hA.z, hA.w),
                                     make_float2(hB.x, hB.y), make_float2(hB.z, hB.w)};
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const float2 na = f2fma(pa.C4, pa.cur[m], f2neg(pa.prev[m]));
                    const float2 nb = f2fma(pb.C4, pb.cur[m], f2neg(pb.prev[m]));
                    aa[m] = f2fma(h[m], na, aa[m]);
                    ab[m] = f2fma(h[m], nb, ab[m]);
                    pa.prev[m] = pa.cur[m];
                    pa.cur[m] = na;
                    pb.prev[m] = pb.cur[m];
                    pb.cur[m] = nb;
                }
            }
            const float Aa = (aa[0].x + aa[1].x) + (aa[2].x + aa[3].x);
            const float Ba = (aa[0].y + aa[1].y) + (aa[2].y + aa[3].y);
            const float Ab = (ab[0].x + ab[1].x) + (ab[2].x + ab[3].x);
            const float Bb = (ab[0].y + ab[1].y) + (ab[2].y + ab[3].y);
            const float wa = (j <= jmask) ? 0.f : xi.w * xa.w;
            const float wb = (j + 1 <= jmask) ? 0.f : xi.w * xb.w;
            const float Wa = wa * 2.f * pa.rinv * pa.rinv * fmaf(-Ba, pa.rinv, Aa);
            const float Wb = wb * 2.f * pb.rinv * pb.rinv * fmaf(-Bb, pb.rinv, Ab);
            const float dax = xi.x - xa.x, day = xi.y - xa.y, daz = xi.z - xa.z;
            const float dbx = xi.x - xb.x, dby = xi.y - xb.y, dbz = xi.z - xb.z;
            gx = fmaf(Wa, dax, fmaf(Wb, dbx, gx));
            gy = fmaf(Wa, day, fmaf(Wb, dby, gy));
            gz = fmaf(Wa, daz, fmaf(Wb, dbz, gz));
            // atom j receives -W (x_i - x_j): sum over the warp, then over the block
            float v[6] = {-Wa * dax, -Wa * day, -Wa * daz, -Wb * dbx, -Wb * dby, -Wb * dbz};
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                for (int c = 0; c < 6; ++c) v[c] += __shfl_xor_sync(kFull, v[c], off);
            if (lane == 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    atomicAdd(&gj[3 * j + c], v[c]);
                    atomicAdd(&gj[3 * (j + 1) + c], v[3 + c]);
                }
            }
        }
        double *Gb = G + (int64_t)item.batch * npad * 3;
        atomicAdd(&Gb[3 * (int64_t)(item.i0 + tid)], (double)gx);
        atomicAdd(&Gb[3 * (int64_t)(item.i0 + tid) + 1], (double)gy);
        atomicAdd(&Gb[3 * (int64_t)(item.i0 + tid) + 2], (double)gz);
        __syncthreads();
        for (int k = tid; k < 3 * item.jlen; k += kTile)
            atomicAdd(&Gb[3 * (int64_t)item.j0 + k], (double)gj[k]);
    }
}

// g[b][q] = dchi2/dI = 2 w_q (I - T); chi2[b] = sum_q w_q (I - T)^2 (fixed-order block sum)
__global__ void k_chi2(const double *I, const double *T, const double *w, int n_q, double *g,
                       double *chi2)
{
    __shared__ double red[256];
    const int64_t b = blockIdx.x;
    double s = 0.0;
    for (int k = threadIdx.x; k < n_q; k += blockDim.x) {
        const double d = I[b * n_q + k] - T[k];
        s += w[k] * d * d;
        g[b * n_q + k] = 2.0 * w[k] * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && chi2) chi2[b] = red[0];
}

// H[b][p][k] = (g_bk f_a f_b, g_bk f_a f_b / q_k), zero at q = 0
__global__ void k_adjoint_coef(const double *g, const double *F, int n_types, QChunks qc, float2 *H,
                               int hstride)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b = blockIdx.y;
    if (k >= qc.n_q) return;
    const double q = qc.q0 + (double)k * qc.dq;
    const int P = n_types * (n_types + 1) / 2;
    int p = 0;
    for (int a = 0; a < n_types; ++a)
        for (int c = a; c < n_types; ++c, ++p) {
            const double h = q > 0.0 ? g[b * qc.n_q + k] * F[a * qc.n_q + k] * F[c * qc.n_q + k] : 0.0;
            H[(b * P + p) * hstride + k] = make_float2((float)h, q > 0.0 ? (float)(h / q) : 0.f);
        }
}

// grad_out[b][i][c] = G[b][slot_of[i]][c] (caller's atom order)
__global__ void k_unpermute(const double *G, const int *slot_of, int64_t n, int64_t npad, int64_t batch,
                            float *grad_out)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= batch * n) return;
    const int64_t b = idx / n, i = idx % n;
    const int64_t s = slot_of[i];
    for (int c = 0; c < 3; ++c) grad_out[3 * idx + c] = (float)G[(b * npad + s) * 3 + c];
}

template <int NB>
cudaError_t launch_nb(const float4 *X, int64_t npad, const Item *items, int n_items, const QChunks &qc,
                      const float2 *H, int n_pairs, int hstride, double *G, int grid, int jmax,
                      cudaStream_t s)
{
    const size_t smem = (size_t)jmax * sizeof(float4) + 2 * NB * sizeof(float4) + (size_t)jmax * 3 * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_debye_adjoint<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_debye_adjoint<NB><<<grid, kTile, smem, s>>>(X, npad, items, n_items, qc, H, n_pairs, hstride, G, jmax);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_chi2(const double *I, const double *T, const double *w, int n_q, int64_t batch,
                        double *g, double *chi2, cudaStream_t s)
{
    if (batch == 0) return cudaSuccess;
    k_chi2<<<(unsigned)batch, 256, 0, s>>>(I, T, w, n_q, g, chi2);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_coef(const double *g, const double *F, int n_types, int64_t batch,
                                const QChunks &qc, float2 *H, int hstride, cudaStream_t s)
{
    if (batch == 0) return cudaSuccess;
    dim3 grid((qc.n_q + 127) / 128, (unsigned)batch);
    k_adjoint_coef<<<grid, 128, 0, s>>>(g, F, n_types, qc, H, hstride);
    return cudaGetLastError();
}

cudaError_t launch_debye_adjoint(const float4 *X, int64_t npad, const Item *items, int n_items,
                                 const QChunks &qc, const float2 *H, int n_pairs, int hstride, double *G,
                                 int grid, int jmax, cudaStream_t s)
{
    if (n_items == 0) return cudaSuccess;
    int qmax = 0;
    for (int c = 0; c < qc.n_chunks; ++c) qmax = qc.q_len[c] > qmax ? qc.q_len[c] : qmax;
    switch (mixed_blocks_for(qmax)) {
    case 13:
        return launch_nb<13>(X, npad, items, n_items, qc, H, n_pairs, hstride, G, grid, jmax, s);
    case 26:
        return launch_nb<26>(X, npad, items, n_items, qc, H, n_pairs, hstride, G, grid, jmax, s);
    default:
        return launch_nb<52>(X, npad, items, n_items, qc, H, n_pairs, hstride, G, grid, jmax, s);
    }
}

cudaError_t launch_unpermute(const double *G, const int *slot_of, int64_t n, int64_t npad, int64_t batch,
                             float *grad_out, cudaStream_t s)
{
    const int64_t tot = batch * n;
    if (tot == 0) return cudaSuccess;
    k_unpermute<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(G, slot_of, n, npad, batch, grad_out);
    return cudaGetLastError();
}

}  // namespace sas

// Orientation average of Eq. 1 by spherical quadrature: the approximate O(N (qD)^2) method that
// the paper weighs against the direct sum (Section I-A: orientation sampling needs a number of
// samples that grows like (qD)^2; Discussion: the choice between an approximate method at low q
// and the direct sum at high q should be made automatically from qD and N).
//
//   I(q) = < |A(q u)|^2 >_u,   A(q u) = sum_t f_t(q) B_t(q u),   B_t(q u) = sum_{j of type t} e^{i q u.(r_j - c)}
//
// averaged with a product rule on the sphere: Gauss-Legendre nodes in cos(theta) (n_theta even)
// times n_phi uniform azimuths.  With real form factors A(-u) = conj A(u), so only the nodes with
// cos(theta) > 0 are used, at twice their weight.  |A|^2 is (up to the truncation of the plane
// wave's spherical expansion) a spherical polynomial of degree 2L when every |j_l(q |r - c|)| past
// degree L is negligible; the rule integrates degree 2L exactly with n_theta >= L + 1 and
// n_phi >= 2L + 1.  L is taken from the spherical Bessel functions at x = q R (R the largest
// distance of an atom from the centroid): the smallest L with (2l+1)|j_l(x)| < 1e-10 for all l > L.
//
// Device work (per q chunk of at most 32 values and conformer): thread = one direction, two atoms
// per step in lockstep, each with (cos, sin) of q u.(r - c) on the two lanes of a packed f32x2
// value, following the three-term recurrence x_{k+1} = 2cos(dq p) x_k - x_{k-1} from seeds at the
// chunk's first two q (the sign pattern of the pair kernels keeps every step a packed
// multiply-add); per-type FP32 sums
// over at most 512 atoms are folded, weighted by f_t(q), into amplitudes kept as FP32 hi/lo pairs
// (exact two-sum) in shared memory; atoms are split into segments over CTAs, and a second kernel
// sums segments and directions in FP64 in a fixed order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "mixed_common.cuh"
#include "sas_internal.h"
#include "sincos_f32.cuh"

namespace sas {

// ---------------------------------------------------------------------------------------------
// host: degree rule and the quadrature nodes
// ---------------------------------------------------------------------------------------------

// Smallest L with (2l+1)|j_l(x)| < tol for every l > L (Miller's downward recurrence, rescaled
// against overflow and normalized by j_0 or j_1).
int quad_degree(double x, double tol)
{
    if (!(x > 0.0)) return 0;
    const int top = (int)(x + 60.0 + 8.0 * std::cbrt(x)) + 40;
    std::vector<double> j(top + 2, 0.0);
    double jp1 = 0.0, jl = 1e-300;
    for (int l = top; l >= 0; --l) {
        j[l] = jl;
        const double jm1 = (2.0 * l + 1.0) / x * jl - jp1;
        jp1 = jl;
        jl = jm1;
        if (std::fabs(jl) > 1e250) {   // rescale everything computed so far
            for (int k = l; k <= top; ++k) j[k] *= 1e-250;
            jl *= 1e-250;
            jp1 *= 1e-250;
        }
    }
    const double j0 = std::sin(x) / x, j1 = std::sin(x) / (x * x) - std::cos(x) / x;
    const double scale = std::fabs(j0) > std::fabs(j1) ? j0 / j[0] : j1 / j[1];
    int L = 0;
    for (int l = top; l >= 0; --l)
        if ((2.0 * l + 1.0) * std::fabs(j[l] * scale) >= tol) {
            L = l;
            break;
        }
    return L;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n from the Chebyshev-like guess).
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            // P_n(z) = p1, P_{n-1}(z) = p0
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        x[n - 1 - i] = -z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Directions of the hemisphere rule for degree L: (ux, uy, uz, 0) and weights summing to 1.
void quad_directions(int L, std::vector<float4> &dirs, std::vector<double> &wts)
{
    int nt = L + 1;
    nt += nt & 1;
    const int np = 2 * L + 1;
    std::vector<double> x, w;
    gauss_legendre(nt, x, w);
    const double pi = 3.14159265358979323846;
    dirs.clear();
    wts.clear();
    for (int i = 0; i < nt; ++i) {
        if (!(x[i] > 0.0)) continue;   // the upper hemisphere, twice its weight
        const double st = std::sqrt(std::max(0.0, 1.0 - x[i] * x[i]));
        for (int k = 0; k < np; ++k) {
            const double phi = 2.0 * pi * k / np;
            dirs.push_back(make_float4((float)(st * std::cos(phi)), (float)(st * std::sin(phi)), (float)x[i], 0.f));
            wts.push_back(2.0 * (w[i] / 2.0) / np);
        }
    }
}

namespace {

using namespace mixed;

// ---------------------------------------------------------------------------------------------
// centroid and radius of the packed atoms (FP64), per conformer
// ---------------------------------------------------------------------------------------------

constexpr int kGeomThreads = 256;

__global__ void __launch_bounds__(kGeomThreads) k_packed_centroid(const float4 *X, int64_t npad, double4 *cen)
{
    __shared__ double sx[kGeomThreads], sy[kGeomThreads], sz[kGeomThreads], sw[kGeomThreads];
    const float4 *Xb = X + blockIdx.x * npad;
    double ax = 0.0, ay = 0.0, az = 0.0, aw = 0.0;
    for (int64_t i = threadIdx.x; i < npad; i += kGeomThreads) {
        const float4 a = Xb[i];
        ax += (double)a.w * a.x;
        ay += (double)a.w * a.y;
        az += (double)a.w * a.z;
        aw += a.w;
    }
    sx[threadIdx.x] = ax;
    sy[threadIdx.x] = ay;
    sz[threadIdx.x] = az;
    sw[threadIdx.x] = aw;
    __syncthreads();
    for (int h = kGeomThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            sx[threadIdx.x] += sx[threadIdx.x + h];
            sy[threadIdx.x] += sy[threadIdx.x + h];
            sz[threadIdx.x] += sz[threadIdx.x + h];
            sw[threadIdx.x] += sw[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double n = sw[0] > 0.0 ? sw[0] : 1.0;
        cen[blockIdx.x] = make_double4(sx[0] / n, sy[0] / n, sz[0] / n, 0.0);
    }
}

__global__ void __launch_bounds__(kGeomThreads) k_packed_radius(const float4 *X, int64_t npad, double4 *cen)
{
    __shared__ double sr[kGeomThreads];
    const float4 *Xb = X + blockIdx.x * npad;
    const double4 c = cen[blockIdx.x];
    double r2 = 0.0;
    for (int64_t i = threadIdx.x; i < npad; i += kGeomThreads) {
        const float4 a = Xb[i];
        if (a.w == 0.f) continue;
        const double dx = a.x - c.x, dy = a.y - c.y, dz = a.z - c.z;
        r2 = fmax(r2, dx * dx + dy * dy + dz * dz);
    }
    sr[threadIdx.x] = r2;
    __syncthreads();
    for (int h = kGeomThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) sr[threadIdx.x] = fmax(sr[threadIdx.x], sr[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) cen[blockIdx.x].w = sqrt(sr[0]);
}

// ---------------------------------------------------------------------------------------------
// amplitudes
// ---------------------------------------------------------------------------------------------

constexpr int kQuadThreads = 128;   // directions per CTA
constexpr int kFoldAtoms = 512;     // FP32 sums span at most this many atoms of one type

__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }

// CTA -> chunk of the flattened launch.
__device__ __forceinline__ int find_chunk(const QuadPlan *pl, int cta)
{
    int c = 0;
    while (c + 1 < pl->n_chunks && cta >= pl->cta_off[c + 1]) ++c;
    return c;
}

// sin and cos of x (|x| up to a few hundred radians) for the chunk-start seeds: Cody-Waite
// reduction by 2pi in two parts, then the MUFU approximations on [-pi, pi] (absolute error about
// 4e-7).  A seed's error does not grow along the recurrence, and the phases of projected positions
// have no repeated values, so it is random across terms and averages out in the amplitude sums.
// (The rotation per q step, whose error would accumulate, uses the full-accuracy sincos.)
__device__ __forceinline__ void sincos_mufu(float x, float &s, float &c)
{
    constexpr float kInv2Pi = 0.15915494309189535f;
    constexpr float k2PiHi = 6.28318548202514648f;       // float32(2 pi)
    constexpr float k2PiLo = -1.7484555314695172e-07f;   // 2 pi - k2PiHi
    const float n = rintf(x * kInv2Pi);
    const float r = fmaf(-n, k2PiLo, fmaf(-n, k2PiHi, x));
    __sincosf(r, &s, &c);
}

// sin and cos of |x| <= pi/4 by the Taylor polynomials of sincos_f32 without its quadrant
// reduction (truncation below 2e-9 relative); larger |x| take the full routine.
__device__ __forceinline__ SinCos sincos_quarter(float x)
{
    using namespace sc;
    if (!(fabsf(x) <= 0.78539816f)) return sincos_f32(x);
    const float x2 = x * x;
    float ps = fmaf(x2, kS9, kS7);
    ps = fmaf(ps, x2, kS5);
    ps = fmaf(ps, x2, kS3);
    float pc = fmaf(x2, kC10, kC8);
    pc = fmaf(pc, x2, kC6);
    pc = fmaf(pc, x2, kC4);
    pc = fmaf(pc, x2, kC2);
    SinCos r;
    r.s = fmaf(ps * x2, x, x);
    r.c = fmaf(pc, x2, 1.0f);
    return r;
}

// Seeds of one atom (weight w, position d relative to the centroid) for one direction u: the
// first two (cos, sin) values of q_k u.d over the chunk and the recurrence coefficient 2cos(dq p)
// to full relative accuracy in 2 - C (the phase velocity for small steps): C = 2 - 4 sin^2(t/2).
__device__ __forceinline__ void seeds(float dx, float dy, float dz, float w, float4 u, float qs_hi, float qs_lo,
                                      float dq_hi, float dq_lo, bool zero_start, float2 &v0, float2 &v1, float &C)
{
    const float p = fmaf(u.z, dz, fmaf(u.y, dy, u.x * dx));
    const SinCos h = sincos_quarter(0.5f * fmaf(dq_hi, p, dq_lo * p));
    const float st = 2.f * h.s * h.c, ct = fmaf(-2.f * h.s, h.s, 1.f);
    float c0 = w, s0 = 0.f;
    if (!zero_start) {
        float sp, cp;
        sincos_mufu(fmaf(qs_hi, p, qs_lo * p), sp, cp);
        c0 = w * cp;
        s0 = w * sp;
    }
    v0 = make_float2(c0, s0);
    v1 = make_float2(fmaf(c0, ct, -s0 * st), fmaf(s0, ct, c0 * st));
    C = fmaf(-4.f * h.s, h.s, 2.f);
}

// Two atoms A, B in lockstep (two independent recurrence chains): add cos and sin of q_k u.d into
// acc[k] = (re, im) for the chunk's first qlen q values, with the sign pattern (+, +, -, -) over k
// carried by the accumulators (block_negative) and the coefficient (odd steps take -C).
template <int QC, bool FULL>
__device__ __forceinline__ void atoms2(const float4 A, const float4 B, float4 u, float qs_hi, float qs_lo,
                                       float dq_hi, float dq_lo, bool zero_start, int qlen, float2 (&acc)[QC])
{
    float2 a0, a1, b0, b1;
    float cA, cB;
    seeds(A.x, A.y, A.z, A.w, u, qs_hi, qs_lo, dq_hi, dq_lo, zero_start, a0, a1, cA);
    seeds(B.x, B.y, B.z, B.w, u, qs_hi, qs_lo, dq_hi, dq_lo, zero_start, b0, b1, cB);
    const float2 CA = bc2(cA), CAn = bc2(-cA), CB = bc2(cB), CBn = bc2(-cB);
    acc[0] = f2add(f2add(acc[0], a0), b0);
    acc[1] = f2add(f2add(acc[1], a1), b1);
    float2 ap = a0, ac = a1, bp = b0, bcur = b1;
#pragma unroll
    for (int k = 1; k + 1 < QC; ++k) {   // W_{k+1} = (k odd ? -C : C) W_k + W_{k-1}
        if (!FULL && k + 1 >= qlen) break;   // a pass shorter than QC (the grid's last)
        const float2 an = f2fma((k & 1) ? CAn : CA, ac, ap);
        const float2 bn = f2fma((k & 1) ? CBn : CB, bcur, bp);
        acc[k + 1] = f2add(f2add(acc[k + 1], an), bn);
        ap = ac;
        ac = an;
        bp = bcur;
        bcur = bn;
    }
}

// Fold the FP32 type sums, weighted by f_t(q_k) and the block sign, into the amplitudes kept as
// FP32 (hi, lo) pairs in shared memory ([k][re_hi, im_hi, re_lo, im_lo][thread]) by an exact
// two-sum, and clear them.
template <int QC>
__device__ __forceinline__ void fold(float2 (&acc)[QC], float *amp, const double *Ft, int qlen, int tid)
{
#pragma unroll
    for (int k = 0; k < QC; ++k) {
        if (k < qlen) {
            const float f = (float)Ft[k] * (block_negative(k) ? -1.f : 1.f);
            float *a = amp + 4 * k * kQuadThreads + tid;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float x = f * (h ? acc[k].y : acc[k].x);
                const float hi = a[h * kQuadThreads];
                const float sum = hi + x, bp = sum - hi;
                const float err = (hi - (sum - bp)) + (x - bp);
                a[h * kQuadThreads] = sum;
                a[(2 + h) * kQuadThreads] += err;
            }
        }
        acc[k] = make_float2(0.f, 0.f);
    }
}

template <int QC>
__global__ void __launch_bounds__(kQuadThreads, 3)
    k_quad_amp(const float4 *__restrict__ X, int64_t npad, const int *__restrict__ type_off, int n_types,
               const double4 *__restrict__ cen, const double *__restrict__ F, int n_q,
               const QuadPlan *__restrict__ pl, const float4 *__restrict__ dirs, double2 *__restrict__ Apart)
{
    __shared__ float4 sx[256];
    extern __shared__ float amp[];   // [QC][4][kQuadThreads]
    const int tid = threadIdx.x;
    const int b = blockIdx.y;   // conformer
    const int cta = blockIdx.x;
    const int c = find_chunk(pl, cta);
    const int n_seg = pl->n_seg[c], n_dir = pl->n_dir[c], seg_len = pl->seg_len[c], q_begin = pl->q_begin[c];
    const float qs_hi = pl->qs_hi[c], qs_lo = pl->qs_lo[c], dq_hi = pl->dq_hi[c], dq_lo = pl->dq_lo[c];
    const int local = cta - pl->cta_off[c];
    const int dblk = local / n_seg, seg = local - dblk * n_seg;
    const int m = dblk * kQuadThreads + tid;
    const bool live = m < n_dir;
    const float4 u = live ? dirs[pl->dir_off[c] + m] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int qlen = pl->q_len[c];
    const bool zero_start = qs_hi == 0.f && qs_lo == 0.f;
    const double4 cc = cen[b];
    const float cx = (float)cc.x, cy = (float)cc.y, cz = (float)cc.z;
    for (int k = 0; k < 4 * QC; ++k) amp[k * kQuadThreads + tid] = 0.f;
    float2 acc[QC];
#pragma unroll
    for (int k = 0; k < QC; ++k) acc[k] = make_float2(0.f, 0.f);
    const int64_t a0 = (int64_t)seg * seg_len, a1 = min((int64_t)npad, a0 + seg_len);
    const float4 *Xb = X + (int64_t)b * npad;
    int t = 0;
    while (t + 1 < n_types && a0 >= type_off[t + 1]) ++t;
    int since = 0;
    for (int64_t base = a0; base < a1; base += 256) {
        __syncthreads();
        const int cnt = (int)min((int64_t)256, a1 - base);
        for (int i = tid; i < 256; i += kQuadThreads) {
            float4 a = i < cnt ? Xb[base + i] : make_float4(0.f, 0.f, 0.f, 0.f);
            a.x -= cx;
            a.y -= cy;
            a.z -= cz;
            sx[i] = a;
        }
        __syncthreads();
        for (int i = 0; i < cnt; i += 2) {   // groups and segments start on even slots
            const int64_t slot = base + i;
            if (slot >= type_off[t + 1]) {   // type change (groups start on whole tiles)
                fold<QC>(acc, amp, F + (int64_t)t * n_q + q_begin, qlen, tid);
                since = 0;
                while (t + 1 < n_types && slot >= type_off[t + 1]) ++t;
            }
            if (qlen == QC)
                atoms2<QC, true>(sx[i], sx[i + 1], u, qs_hi, qs_lo, dq_hi, dq_lo, zero_start, qlen, acc);
            else
                atoms2<QC, false>(sx[i], sx[i + 1], u, qs_hi, qs_lo, dq_hi, dq_lo, zero_start, qlen, acc);
            since += 2;
            if (since >= kFoldAtoms) {
                fold<QC>(acc, amp, F + (int64_t)t * n_q + q_begin, qlen, tid);
                since = 0;
            }
        }
    }
    fold<QC>(acc, amp, F + (int64_t)t * n_q + q_begin, qlen, tid);
    if (live) {
        // Apart[b][chunk][seg][k][m]
        double2 *out = Apart + (int64_t)b * pl->amp_stride + pl->amp_off[c] + (int64_t)seg * QC * n_dir;
        for (int k = 0; k < qlen; ++k) {
            const float *a = amp + 4 * k * kQuadThreads + tid;
            out[(int64_t)k * n_dir + m] = make_double2((double)a[0] + (double)a[2 * kQuadThreads],
                                                       (double)a[kQuadThreads] + (double)a[3 * kQuadThreads]);
        }
    }
}

// I(q) = sum_m w_m |sum_seg A_seg(q, m)|^2: one CTA per (chunk, k, conformer); fixed order.
constexpr int kFinishThreads = 256;

__global__ void __launch_bounds__(kFinishThreads)
    k_quad_finish(const QuadPlan *__restrict__ pl, const double *__restrict__ wts, const double2 *__restrict__ Apart,
                  int n_q, double *__restrict__ I)
{
    __shared__ double red[kFinishThreads];
    const int c = blockIdx.x, k = blockIdx.y, b = blockIdx.z;
    if (k >= pl->q_len[c]) return;
    const int M = pl->n_dir[c], S = pl->n_seg[c], dir_off = pl->dir_off[c];
    const double2 *A = Apart + (int64_t)b * pl->amp_stride + pl->amp_off[c];
    double s = 0.0;
    for (int m = threadIdx.x; m < M; m += kFinishThreads) {
        double re = 0.0, im = 0.0;
        for (int g = 0; g < S; ++g) {
            const double2 v = A[((int64_t)g * kQuadChunk + k) * M + m];
            re += v.x;
            im += v.y;
        }
        s += wts[dir_off + m] * (re * re + im * im);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = kFinishThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) I[(int64_t)b * n_q + pl->q_begin[c] + k] = red[0];
}

}  // namespace

cudaError_t launch_packed_geometry(const float4 *X, int64_t npad, int64_t batch, double4 *cen, cudaStream_t s)
{
    if (batch == 0) return cudaSuccess;
    k_packed_centroid<<<(unsigned)batch, kGeomThreads, 0, s>>>(X, npad, cen);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_packed_radius<<<(unsigned)batch, kGeomThreads, 0, s>>>(X, npad, cen);
    return cudaGetLastError();
}

cudaError_t launch_quad(const float4 *X, int64_t npad, int64_t batch, const int *type_off, int n_types,
                        const double4 *cen, const double *F, int n_q, const QuadPlan &pl, const QuadPlan *pl_dev,
                        const float4 *dirs, const double *wts, double2 *Apart, double *I, cudaStream_t s)
{
    if (pl.n_chunks == 0 || batch == 0) return cudaSuccess;
    const dim3 grid((unsigned)pl.cta_off[pl.n_chunks], (unsigned)batch);
    const size_t smem = (size_t)4 * kQuadChunk * kQuadThreads * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_quad_amp<kQuadChunk>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_quad_amp<kQuadChunk><<<grid, kQuadThreads, smem, s>>>(X, npad, type_off, n_types, cen, F, n_q, pl_dev, dirs,
                                                             Apart);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_quad_finish<<<dim3((unsigned)pl.n_chunks, kQuadChunk, (unsigned)batch), kFinishThreads, 0, s>>>(pl_dev, wts,
                                                                                                      Apart, n_q, I);
    return cudaGetLastError();
}

int quad_threads_per_cta() { return kQuadThreads; }

}  // namespace sas

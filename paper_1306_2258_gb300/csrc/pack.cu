// Packing: validate the inputs, stable-sort atoms by type into type groups
// padded to whole tiles, and write one float4 (x, y, z, w) per slot, w = 1 for
// a real atom and 0 for padding.
//
// The paper keeps the N positions and the per-atom form factors in GPU global
// memory (Section II).  Here the form factors are not per atom at all: sorting
// by type makes every tile type-homogeneous, so each tile pair belongs to one
// type pair (a, b) and f_a(q) f_b(q) multiplies a whole partial sum instead of
// every pair term.
#include <algorithm>
#include <cmath>

#include "sas_internal.h"

namespace sas {

namespace {

__device__ __forceinline__ void load_xyz(const void *coords, int f64, int64_t idx, double &x,
                                         double &y, double &z)
{
    if (f64) {
        const double *c = static_cast<const double *>(coords) + 3 * idx;
        x = c[0];
        y = c[1];
        z = c[2];
    } else {
        const float *c = static_cast<const float *>(coords) + 3 * idx;
        x = c[0];
        y = c[1];
        z = c[2];
    }
}

// Per block of kPackThreads atoms (blockIdx.x) and slice of the conformers (blockIdx.y, every
// gridDim.y-th): validation of types (slice 0, which also counts them) and coordinates, and the
// largest squared distance from each conformer's first atom (FP32, as float bits in *extent2,
// which order like the values for non-negative floats): every conformer's diameter is at most
// twice its square root.
template <typename Real>
__global__ void k_count_types(const Real *coords, const int32_t *types, int64_t n, int64_t batch, int n_types,
                              int *blockcounts, int *errword, unsigned *extent2)
{
    __shared__ int cnt[SAS_MAX_TYPES];
    __shared__ float wmax[kPackThreads / 32];
    const bool counter = blockIdx.y == 0;
    if (counter && threadIdx.x < SAS_MAX_TYPES) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int err = 0;
    float d2max = 0.f;
    if (i < n) {
        if (counter) {
            const int t = types[i];
            if (t < 0 || t >= n_types)
                err |= kErrBadType;
            else
                atomicAdd(&cnt[t], 1);
        }
        for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
            const Real *c = coords + 3 * (b * n + i), *c0 = coords + 3 * (b * n);
            const Real x = c[0], y = c[1], z = c[2];
            if (!isfinite(x) || !isfinite(y) || !isfinite(z)) err |= kErrNonFinite;
            const float dx = (float)(x - c0[0]), dy = (float)(y - c0[1]), dz = (float)(z - c0[2]);
            const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (d2 == d2) d2max = fmaxf(d2max, d2 * 1.000001f);   // a little over: rounding
        }
    }
    if (err) atomicOr(errword, err);
    if (extent2) {
        for (int o = 16; o > 0; o >>= 1) d2max = fmaxf(d2max, __shfl_xor_sync(0xffffffffu, d2max, o));
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = d2max;
    }
    __syncthreads();
    if (counter && threadIdx.x < n_types) blockcounts[(int64_t)blockIdx.x * n_types + threadIdx.x] = cnt[threadIdx.x];
    if (extent2 && threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < kPackThreads / 32; ++w) m = fmaxf(m, wmax[w]);
        atomicMax(extent2, __float_as_uint(m));
    }
}

// One block: exclusive scan of the per-block counts for each type; totals and padded offsets.
__global__ void k_scan_counts(const int *blockcounts, int nblk, int n_types, int tile, int *blockoffs,
                              int *meta)
{
    __shared__ int tot[SAS_MAX_TYPES];
    int t = threadIdx.x;
    if (t < n_types) {
        int run = 0;
        for (int b = 0; b < nblk; ++b) {
            blockoffs[(int64_t)b * n_types + t] = run;
            run += blockcounts[(int64_t)b * n_types + t];
        }
        tot[t] = run;
        meta[t] = run;
    }
    __syncthreads();
    if (t == 0) {
        int off = 0;
        for (int k = 0; k < n_types; ++k) {
            meta[n_types + k] = off;
            off += (tot[k] + tile - 1) / tile * tile;
        }
        meta[2 * n_types] = off;
    }
}

// Centroid of each conformer in FP64, deterministic: fixed strided partial sums, fixed tree.
__global__ void k_centroid(const void *coords, int coords_f64, int64_t n, double *centroid)
{
    __shared__ double red[3][kPackThreads];
    int64_t b = blockIdx.x;
    double sx = 0, sy = 0, sz = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double x, y, z;
        load_xyz(coords, coords_f64, b * n + i, x, y, z);
        sx += x;
        sy += y;
        sz += z;
    }
    red[0][threadIdx.x] = sx;
    red[1][threadIdx.x] = sy;
    red[2][threadIdx.x] = sz;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) centroid[3 * b + threadIdx.x] = n > 0 ? red[threadIdx.x][0] / (double)n : 0.0;
}

// Stable scatter: slot = group offset + (atoms of the same type before this one).
// Slot of every atom (stable by type) and its packed coordinates for the conformers of slice
// blockIdx.y (every gridDim.y-th): FP32 inputs are copied as they are, FP64 inputs centred on the
// conformer's FP64 centroid (when given) before the FP32 or FP64 store.
template <typename Real>
__global__ void k_scatter(const Real *coords, const int32_t *types, int64_t n, int64_t batch, int n_types,
                          const int *blockoffs, const int *meta, const double *centroid, int out_f64, void *X,
                          int64_t npad, int *slot_of)
{
    __shared__ int wcnt[kPackThreads / 32][SAS_MAX_TYPES];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < (kPackThreads / 32) * SAS_MAX_TYPES; k += blockDim.x)
        (&wcnt[0][0])[k] = 0;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int t = (i < n) ? types[i] : -1;
    if (t >= n_types) t = -1;
    unsigned peers = __match_any_sync(0xffffffffu, t);
    int rank_in_warp = __popc(peers & ((1u << lane) - 1u));
    if (t >= 0 && rank_in_warp == 0) wcnt[warp][t] = __popc(peers);
    __syncthreads();
    if (t < 0) return;
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wcnt[w][t];
    int rank = blockoffs[(int64_t)blockIdx.x * n_types + t] + before + rank_in_warp;
    int slot = meta[n_types + t] + rank;
    if (blockIdx.y == 0) slot_of[i] = slot;
    for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
        const Real *c = coords + 3 * (b * n + i);
        if (out_f64) {
            static_cast<double4 *>(X)[b * npad + slot] = make_double4(c[0], c[1], c[2], 1.0);
        } else if (centroid) {
            static_cast<float4 *>(X)[b * npad + slot] =
                make_float4((float)((double)c[0] - centroid[3 * b]), (float)((double)c[1] - centroid[3 * b + 1]),
                            (float)((double)c[2] - centroid[3 * b + 2]), 1.0f);
        } else {
            static_cast<float4 *>(X)[b * npad + slot] = make_float4((float)c[0], (float)c[1], (float)c[2], 1.0f);
        }
    }
}

}  // namespace

cudaError_t launch_count_types(const void *coords, int coords_f64, const int32_t *types, int64_t n,
                               int64_t batch, int n_types, int *blockcounts, int *errword,
                               unsigned *extent2, cudaStream_t s)
{
    int nblk = (int)((n + kPackThreads - 1) / kPackThreads);
    if (nblk == 0) return cudaSuccess;
    // conformer slices: enough CTAs to fill the device for large batches of small molecules
    const unsigned ys = (unsigned)std::max<int64_t>(1, std::min<int64_t>(batch, (1216 + nblk - 1) / nblk));
    const dim3 grid((unsigned)nblk, ys);
    if (coords_f64)
        k_count_types<double><<<grid, kPackThreads, 0, s>>>(static_cast<const double *>(coords), types, n, batch,
                                                          n_types, blockcounts, errword, extent2);
    else
        k_count_types<float><<<grid, kPackThreads, 0, s>>>(static_cast<const float *>(coords), types, n, batch,
                                                         n_types, blockcounts, errword, extent2);
    return cudaGetLastError();
}

cudaError_t launch_scan_counts(const int *blockcounts, int nblk, int n_types, int tile,
                               int *blockoffs, int *meta, cudaStream_t s)
{
    k_scan_counts<<<1, 32, 0, s>>>(blockcounts, nblk, n_types, tile, blockoffs, meta);
    return cudaGetLastError();
}

cudaError_t launch_centroid(const void *coords, int coords_f64, int64_t n, int64_t batch,
                            double *centroid, cudaStream_t s)
{
    if (batch == 0) return cudaSuccess;
    k_centroid<<<(unsigned)batch, kPackThreads, 0, s>>>(coords, coords_f64, n, centroid);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const void *coords, int coords_f64, const int32_t *types, int64_t n,
                           int64_t batch, int n_types, const int *blockoffs, const int *meta,
                           const double *centroid, int out_f64, void *X, int64_t npad,
                           int *slot_of, cudaStream_t s)
{
    int nblk = (int)((n + kPackThreads - 1) / kPackThreads);
    if (nblk == 0) return cudaSuccess;
    const unsigned ys = (unsigned)std::max<int64_t>(1, std::min<int64_t>(batch, (1216 + nblk - 1) / nblk));
    const dim3 grid((unsigned)nblk, ys);
    if (coords_f64)
        k_scatter<double><<<grid, kPackThreads, 0, s>>>(static_cast<const double *>(coords), types, n, batch, n_types,
                                                        blockoffs, meta, centroid, out_f64, X, npad, slot_of);
    else
        k_scatter<float><<<grid, kPackThreads, 0, s>>>(static_cast<const float *>(coords), types, n, batch, n_types,
                                                       blockoffs, meta, centroid, out_f64, X, npad, slot_of);
    return cudaGetLastError();
}

}  // namespace sas

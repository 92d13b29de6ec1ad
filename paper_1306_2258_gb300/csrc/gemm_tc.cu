// Dense GEMM of the surrogate network on the 5th-generation tensor cores:
//   C[M][N] = A[M][K] B[N][K]^T (+ bias[N]), bfloat16 A and B with K contiguous, FP32 accumulation,
//   epilogue writing FP32 and/or bfloat16 of the value or of GELU(value).
// Not part of the paper's method (the surrogate ranks conformers before the exact Debye kernel,
// Section I-A Eq. 2, re-scores them).
//
// One CTA computes a 128 x BN tile (BN = 64 or 128) with four warps:
//  * thread 0 streams K in slices of 64 (one 128-byte row of bfloat16 per tile row) with 2-D TMA
//    loads (cp.async.bulk.tensor, 128-byte swizzle, zero fill outside the matrices) into a ring
//    of shared-memory stages, each guarded by a "full" mbarrier (transaction bytes);
//  * thread 32 issues tcgen05.mma (kind::f16, M = 128, N = BN, K = 16) from shared-memory matrix
//    descriptors into an FP32 accumulator in tensor memory, and frees a stage by committing the
//    stage's MMAs to its "empty" mbarrier; a last commit signals "done";
//  * then every warp reads its 32 accumulator lanes (rows) with tcgen05.ld and applies the
//    epilogue (eight independent columns at a time, 16-byte stores where aligned).
// Split-K (launch_gemm_splitk): the grid's z dimension cuts K into slices of whole stages, each
// CTA writing its slice's FP32 product to its own output plane; the caller sums the planes.
// Problems of at least two 128 x 256 tiles per SM take the persistent form k_gemm_tcp instead: one
// CTA per SM walks its tiles with warp-specialized roles (producer, MMA issuer, four epilogue warps)
// and two accumulators in tensor memory, so a tile's epilogue runs under the next tile's main loop.
// Every mbarrier wait gives up after 2 s (or an iteration limit); a wait that gives up sets the
// error word, the other roles stop at their next wait, and the kernel still frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "sas_internal.h"

namespace sas {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kTcM = 128;                 // tile rows: the M of one tcgen05.mma
constexpr int kTcK = 64;                  // K per stage: 64 bfloat16 = one 128-byte swizzle row
constexpr uint32_t kSpinLimit = 1u << 26;
constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s: far beyond any wait of a correct run
constexpr uint32_t kABytes = kTcM * kTcK * 2;

__device__ int g_tc_error;   // set when a wait ran out of iterations (never reset by the kernels)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until the phase of parity `parity` has completed; false after kWaitNs of waiting (or the
// iteration limit), or, with `fail` given, as soon as another role has set *fail.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, const volatile int *fail = nullptr)
{
    const uint32_t a = smem_u32(b);
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n"
            ".reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n"
            "}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((i & 255u) == 255u) {
            if (fail && *fail) return false;
            if (global_ns() - t0 > kWaitNs) return false;
        }
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the 128-byte swizzle:
// rows of 128 bytes, groups of 8 rows 1024 bytes apart (stride byte offset), start address in
// 16-byte units; the leading byte offset is not used by this layout.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                      // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;   // stride byte offset: 8 rows x 128 bytes
    d |= (uint64_t)1 << 46;                      // descriptor version of this architecture
    d |= (uint64_t)2 << 61;                      // layout: 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, bfloat16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 8 consecutive FP32 accumulator columns of this thread's lane (row).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

// Optional transposed copy of the bfloat16 output: Dt[col][row] (leading dimension ld), with zero
// columns for the rows [M, mpad) (batch padding of the operand that multiplies along the batch).
struct TOut {
    bf16 *p;
    int ld, mpad;
};

// Epilogue of 8 consecutive columns col0.. of one row (col0 < N): x = accumulator (+ bias) to C in
// FP32 and bfloat16(x or GELU(x)) to D (and its transpose to t.p).  The eight values are
// independent (their GELUs overlap), and whole aligned groups go out as 16-byte stores; the
// transposed stores of a warp's 32 rows are contiguous.
__device__ __forceinline__ void store8(const float (&v)[8], bool have_acc, int row, int col0, int N,
                                       const float *__restrict__ bias, float *__restrict__ C, int ldc,
                                       bf16 *__restrict__ D, int ldd, int gelu, TOut t = TOut{nullptr, 0, 0})
{
    const bool whole = col0 + 8 <= N;
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        x[k] = have_acc ? v[k] : 0.f;
        if (bias && (whole || col0 + k < N)) x[k] += bias[col0 + k];
    }
    if (C) {
        float *cp = C + (size_t)row * ldc + col0;
        if (whole && (reinterpret_cast<uintptr_t>(cp) & 15) == 0) {
            reinterpret_cast<float4 *>(cp)[0] = make_float4(x[0], x[1], x[2], x[3]);
            reinterpret_cast<float4 *>(cp)[1] = make_float4(x[4], x[5], x[6], x[7]);
        } else {
            for (int k = 0; k < 8 && col0 + k < N; ++k) cp[k] = x[k];
        }
    }
    if (D) {
        uint32_t p[4];
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
            const float a = gelu ? gelu_f(x[k]) : x[k], b = gelu ? gelu_f(x[k + 1]) : x[k + 1];
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(a, b);   // .x = a (lower address), .y = b
            p[k / 2] = *reinterpret_cast<const uint32_t *>(&h2);
        }
        bf16 *dp = D + (size_t)row * ldd + col0;
        const bf16 *h = reinterpret_cast<const bf16 *>(p);
        if (whole && (reinterpret_cast<uintptr_t>(dp) & 15) == 0) {
            *reinterpret_cast<uint4 *>(dp) = make_uint4(p[0], p[1], p[2], p[3]);
        } else {
            for (int k = 0; k < 8 && col0 + k < N; ++k) dp[k] = h[k];
        }
        if (t.p)
            for (int k = 0; k < 8 && col0 + k < N; ++k) t.p[(size_t)(col0 + k) * t.ld + row] = h[k];
    }
}

// S shared-memory stages (launch_bn chooses: a deep ring for grids that leave SMs idle, else about
// 97 KB so that two CTAs share an SM and one's epilogue overlaps the other's main loop).
template <int BN, int S>
__global__ void __launch_bounds__(128, 2)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
              const float *__restrict__ bias, float *__restrict__ C, int ldc, bf16 *__restrict__ D, int ldd, int gelu,
              int kper, int64_t c_split, TOut tout)
{
    constexpr uint32_t kBBytes = BN * kTcK * 2;
    extern __shared__ uint8_t smem_raw[];
    // stage tiles on 1024-byte boundaries (the 128-byte swizzle pattern repeats every 8 rows)
    uint8_t *smem = smem_raw + (((smem_u32(smem_raw) + 1023u) & ~1023u) - smem_u32(smem_raw));
    uint8_t *sA = smem;                       // [S][128 rows][128 B]
    uint8_t *sB = smem + S * kABytes;   // [S][BN rows][128 B]
    __shared__ __align__(8) uint64_t full[S], empty[S], done;
    __shared__ uint32_t tmem_base;
    __shared__ int fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kTcM, n0 = blockIdx.x * BN;
    // split-K: slice z of the K range (kper stages of 64) into its own FP32 output C + z c_split
    const int kbeg = blockIdx.z * kper;
    const int ksteps = max(0, min(kper, (K + kTcK - 1) / kTcK - kbeg));
    if (C) C += blockIdx.z * c_split;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (warp == 0) {   // BN accumulator columns of 128 lanes (a power of two >= 32)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"((uint32_t)BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (threadIdx.x == 0) {   // TMA producer
        int issued = 0;
        for (int ks = 0; ks < ksteps; ++ks) {
            const int s = ks % S;
            if (ks >= S && !mbar_wait(&empty[s], (uint32_t)((ks / S) - 1) & 1u)) {
                fail = 1;
                break;
            }
            mbar_expect_tx(&full[s], kABytes + kBBytes);
            tma_load_2d(sA + s * kABytes, &tmA, &full[s], (kbeg + ks) * kTcK, m0);
            tma_load_2d(sB + s * kBBytes, &tmB, &full[s], (kbeg + ks) * kTcK, n0);
            issued = ks + 1;
        }
        // the copies still in flight (normally all were consumed already): wait for the last phase
        // of every stage that received one
        for (int ks = issued > S ? issued - S : 0; ks < issued; ++ks)
            if (!mbar_wait(&full[ks % S], (uint32_t)(ks / S) & 1u)) fail = 1;
    } else if (threadIdx.x == 32) {   // MMA issuer
        const uint32_t idesc = idesc_bf16(kTcM, BN);
        for (int ks = 0; ks < ksteps; ++ks) {
            const int s = ks % S;
            if (!mbar_wait(&full[s], (uint32_t)(ks / S) & 1u)) {
                fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sA + s * kABytes), b0 = smem_u32(sB + s * kBBytes);
#pragma unroll
            for (int kk = 0; kk < kTcK / 16; ++kk)   // K = 16 per MMA: 32 bytes along the swizzled row
                umma_bf16(tmem, sw128_desc(a0 + 32u * kk), sw128_desc(b0 + 32u * kk), idesc,
                          (ks > 0 || kk > 0) ? 1u : 0u);
            umma_commit(&empty[s]);   // the stage is free once these MMAs have read it
        }
        umma_commit(&done);           // arrives when every MMA issued above has completed
    }
    __syncwarp();
    if (!mbar_wait(&done, 0)) fail = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncwarp();   // the tensor-memory loads below are warp-collective

    const int row = m0 + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 8) {
        float v[8];
        tmem_ld8(trow + (uint32_t)c0, v);   // warp-collective: every lane of the warp takes part
        if (row < M && n0 + c0 < N) {
            store8(v, ksteps > 0, row, n0 + c0, N, bias, C, ldc, D, ldd, gelu, tout);
        } else if (tout.p && row < tout.mpad) {   // zero padding of the transposed copy
            for (int k = 0; k < 8 && n0 + c0 + k < N; ++k)
                tout.p[(size_t)(n0 + c0 + k) * tout.ld + row] = __float2bfloat16_rn(0.f);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && fail) atomicExch(&g_tc_error, 1);
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

// Persistent form for grids of at least one tile per SM: one CTA per SM walks tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... (M fastest, so neighbouring CTAs share B tiles in L2).  Warp 0 lane 0
// streams A and B slices with TMA into S stages; warp 1 lane 0 issues the MMAs into one of two
// accumulators in tensor memory (tile i uses accumulator i & 1) and commits "full" when a tile is
// done; warps 2-5 (tensor-memory lane quarters 2, 3, 0, 1) read the finished accumulator, apply the
// epilogue and release it, so the epilogue of one tile runs under the main loop of the next.
// Tile t of the persistent walk: groups of `group` row tiles, each group covering every column tile
// before the next starts (rows fastest inside a group), so the CTAs in flight share both A and B
// tiles in L2.
__device__ __forceinline__ void tile_of(int t, int mt, int nt, int group, int &m0, int &n0, int bn)
{
    const int per = group * nt, g = t / per, local = t - g * per;
    const int gm = min(group, mt - g * group);
    m0 = (g * group + local % gm) * kTcM;
    n0 = (local / gm) * bn;
}

template <int BN, int S>
__global__ void __launch_bounds__(192, 1)
    k_gemm_tcp(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
               const float *__restrict__ bias, float *__restrict__ C, int ldc, bf16 *__restrict__ D, int ldd, int gelu,
               int group)
{
    constexpr uint32_t kBBytes = BN * kTcK * 2;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_raw + (((smem_u32(smem_raw) + 1023u) & ~1023u) - smem_u32(smem_raw));
    uint8_t *sA = smem;                 // [S][128 rows][128 B]
    uint8_t *sB = smem + S * kABytes;   // [S][BN rows][128 B]
    __shared__ __align__(8) uint64_t full[S], empty[S], tfull[2], tempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = (M + kTcM - 1) / kTcM, nt = (N + BN - 1) / BN, tiles = mt * nt;
    const int ksteps = (K + kTcK - 1) / kTcK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);   // one arrival per epilogue warp
        }
        fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (warp == 0) {   // two accumulators of BN columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"((uint32_t)(2 * BN))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {   // TMA producer
            int it = 0, issued = 0;
            for (int t = blockIdx.x; t < tiles && !fail; t += gridDim.x) {
                int m0, n0;
                tile_of(t, mt, nt, group, m0, n0, BN);
                for (int ks = 0; ks < ksteps; ++ks, ++it) {
                    const int s = it % S;
                    if (it >= S && !mbar_wait(&empty[s], (uint32_t)((it / S) - 1) & 1u, &fail)) {
                        fail = 1;
                        break;
                    }
                    mbar_expect_tx(&full[s], kABytes + kBBytes);
                    tma_load_2d(sA + s * kABytes, &tmA, &full[s], ks * kTcK, m0);
                    tma_load_2d(sB + s * kBBytes, &tmB, &full[s], ks * kTcK, n0);
                    issued = it + 1;
                }
            }
            // copies still in flight (normally all were consumed): the last phase of each used stage
            for (int k = issued > S ? issued - S : 0; k < issued; ++k)
                if (!mbar_wait(&full[k % S], (uint32_t)(k / S) & 1u)) fail = 1;
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            const uint32_t idesc = idesc_bf16(kTcM, BN);
            int it = 0, i = 0;
            for (int t = blockIdx.x; t < tiles && !fail; t += gridDim.x, ++i) {
                const int acc = i & 1;
                if (i >= 2 && !mbar_wait(&tempty[acc], (uint32_t)((i / 2) - 1) & 1u, &fail)) {
                    fail = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t td = tmem + (uint32_t)(acc * BN);
                for (int ks = 0; ks < ksteps; ++ks, ++it) {
                    const int s = it % S;
                    if (!mbar_wait(&full[s], (uint32_t)(it / S) & 1u, &fail)) {
                        fail = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem_u32(sA + s * kABytes), b0 = smem_u32(sB + s * kBBytes);
#pragma unroll
                    for (int kk = 0; kk < kTcK / 16; ++kk)
                        umma_bf16(td, sw128_desc(a0 + 32u * kk), sw128_desc(b0 + 32u * kk), idesc,
                                  (ks > 0 || kk > 0) ? 1u : 0u);
                    umma_commit(&empty[s]);
                }
                umma_commit(&tfull[acc]);   // arrives when this tile's MMAs have completed
            }
        }
    } else {   // epilogue warps
        const int quarter = warp & 3;   // the tensor-memory lanes this warp may read
        int i = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
            const int acc = i & 1;
            int ok = 1;
            if (lane == 0) ok = mbar_wait(&tfull[acc], (uint32_t)(i / 2) & 1u, &fail) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int m0, n0;
            tile_of(t, mt, nt, group, m0, n0, BN);
            const int row = m0 + quarter * 32 + lane;
            const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * BN);
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 8) {
                float v[8];
                tmem_ld8(trow + (uint32_t)c0, v);
                if (row < M) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int col = n0 + c0 + k;
                        if (col >= N) break;
                        float x = ksteps > 0 ? v[k] : 0.f;
                        if (bias) x += bias[col];
                        if (C) C[(size_t)row * ldc + col] = x;
                        if (D) D[(size_t)row * ldd + col] = __float2bfloat16_rn(gelu ? gelu_f(x) : x);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && fail) atomicExch(&g_tc_error, 1);
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * BN))
                     : "memory");
    }
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Row-major [rows][K] bfloat16 with row stride ld elements, boxes of box_rows x 64.
bool make_map(CUtensorMap &map, const void *base, int rows, int K, int ld, int box_rows)
{
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int S>
cudaError_t launch_bs(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias, float *C,
                      int ldc, void *D, int ldd, int gelu, cudaStream_t s,
                      int splits = 1, TOut tout = TOut{nullptr, 0, 0})
{
    CUtensorMap ta, tb;
    if (!make_map(ta, A, M, K, lda, kTcM) || !make_map(tb, B, N, K, ldb, BN)) return cudaErrorInvalidValue;
    const size_t smem = (size_t)S * (kABytes + BN * kTcK * 2) + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<BN, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int kt = (K + kTcK - 1) / kTcK;
    const int kper = splits > 1 ? (kt + splits - 1) / splits : kt;
    const dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + kTcM - 1) / kTcM), (unsigned)(splits > 1 ? splits : 1));
    k_gemm_tc<BN, S><<<grid, 128, smem, s>>>(ta, tb, M, N, K, bias, C, ldc, static_cast<bf16 *>(D), ldd, gelu, kper,
                                             (int64_t)M * ldc, tout);
    return cudaGetLastError();
}

template <int BN, int S>
cudaError_t launch_persistent(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias,
                              float *C, int ldc, void *D, int ldd, int gelu, int sms, cudaStream_t s)
{
    CUtensorMap ta, tb;
    if (!make_map(ta, A, M, K, lda, kTcM) || !make_map(tb, B, N, K, ldb, BN)) return cudaErrorInvalidValue;
    const size_t smem = (size_t)S * (kABytes + BN * kTcK * 2) + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tcp<BN, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int tiles = ((M + kTcM - 1) / kTcM) * ((N + BN - 1) / BN);
    const int group = 16;   // 8192^3: 1234 TFLOP/s with rows fastest over all of M, 1336 with groups of 16
    k_gemm_tcp<BN, S><<<std::min(tiles, sms), 192, smem, s>>>(ta, tb, M, N, K, bias, C, ldc, static_cast<bf16 *>(D),
                                                               ldd, gelu, group);
    return cudaGetLastError();
}

// Stages: with a grid that leaves SMs idle, one CTA per SM with a deep ring (8 stages of 24 KB for
// 64-column tiles, 5 of 32 KB for 128-column ones) keeps more TMA loads in flight; otherwise about
// 97 KB per CTA so that two CTAs share an SM.
template <int BN>
cudaError_t launch_bn(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias, float *C,
                      int ldc, void *D, int ldd, int gelu, cudaStream_t s, TOut tout = TOut{nullptr, 0, 0})
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return cudaErrorInvalidDevice;
    const int64_t ctas = (int64_t)((N + BN - 1) / BN) * ((M + kTcM - 1) / kTcM);
    const bool deep = ctas <= sms;
    if (BN == 64)
        return deep ? launch_bs<64, 8>(M, N, K, A, lda, B, ldb, bias, C, ldc, D, ldd, gelu, s, 1, tout)
                    : launch_bs<64, 4>(M, N, K, A, lda, B, ldb, bias, C, ldc, D, ldd, gelu, s, 1, tout);
    return deep ? launch_bs<128, 5>(M, N, K, A, lda, B, ldb, bias, C, ldc, D, ldd, gelu, s, 1, tout)
                : launch_bs<128, 3>(M, N, K, A, lda, B, ldb, bias, C, ldc, D, ldd, gelu, s, 1, tout);
}

}  // namespace

bool gemm_tc_supported(int K, const void *A, int lda, const void *B, int ldb)
{
    return K >= 0 && lda % 8 == 0 && ldb % 8 == 0 && lda >= K && ldb >= K &&
           ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) == 0 && encoder() != nullptr;
}

cudaError_t launch_gemm_tc(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias,
                           float *C, int ldc, void *D, int ldd, int gelu, cudaStream_t s)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cudaErrorInvalidDevice;
    // large problems: the persistent kernel with 128 x 256 tiles when every SM gets several
    const int mt = (M + kTcM - 1) / kTcM;
    if (N >= 256 && mt * ((N + 255) / 256) >= 2 * sms)
        return launch_persistent<256, 4>(M, N, K, A, lda, B, ldb, bias, C, ldc, D, ldd, gelu, sms, s);
    // 64-column tiles when 128-column ones would leave most SMs idle
    const int tiles128 = mt * ((N + 127) / 128);
    if (N <= 64 || tiles128 < 64) return launch_bn<64>(M, N, K, A, lda, B, ldb, bias, C, ldc, D, ldd, gelu, s);
    return launch_bn<128>(M, N, K, A, lda, B, ldb, bias, C, ldc, D, ldd, gelu, s);
}

cudaError_t launch_gemm_splitk(int M, int N, int K, const void *A, int lda, const void *B, int ldb, float *ws, int splits,
                               cudaStream_t s)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    const int kt = (K + kTcK - 1) / kTcK;
    if (splits < 1 || (kt + splits - 1) / splits * (splits - 1) >= kt || !gemm_tc_supported(K, A, lda, B, ldb))
        return cudaErrorInvalidValue;   // every slice must hold at least one stage
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cudaErrorInvalidDevice;
    const int64_t ctas = (int64_t)((N + 63) / 64) * ((M + kTcM - 1) / kTcM) * splits;
    return ctas <= sms ? launch_bs<64, 8>(M, N, K, A, lda, B, ldb, nullptr, ws, N, nullptr, 0, 0, s, splits)
                       : launch_bs<64, 4>(M, N, K, A, lda, B, ldb, nullptr, ws, N, nullptr, 0, 0, s, splits);
}

cudaError_t launch_gemm(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias,
                        float *C, int ldc, void *D, int ldd, int gelu, cudaStream_t s)
{
    if (gemm_tc_supported(K, A, lda, B, ldb))
        return launch_gemm_tc(M, N, K, A, lda, B, ldb, bias, C, ldc, D, ldd, gelu, s);
    return launch_gemm_tn(M, N, K, A, lda, B, ldb, bias, C, ldc, D, ldd, gelu, s);
}

cudaError_t launch_gemm_t(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias,
                          float *C, int ldc, void *D, int ldd, int gelu, void *Dt, int ldt, int Mpad, cudaStream_t s)
{
    if (!D || !Dt || Mpad < M || ldt < Mpad) return cudaErrorInvalidValue;
    if (M <= 0 || N <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cudaErrorInvalidDevice;
    const int mt = (M + kTcM - 1) / kTcM;
    const bool persistent = N >= 256 && mt * ((N + 255) / 256) >= 2 * sms;
    if (gemm_tc_supported(K, A, lda, B, ldb) && !persistent) {   // the transposed copy from the epilogue
        const TOut t{static_cast<bf16 *>(Dt), ldt, Mpad};
        const int tiles128 = mt * ((N + 127) / 128);
        if (N <= 64 || tiles128 < 64) return launch_bn<64>(M, N, K, A, lda, B, ldb, bias, C, ldc, D, ldd, gelu, s, t);
        return launch_bn<128>(M, N, K, A, lda, B, ldb, bias, C, ldc, D, ldd, gelu, s, t);
    }
    cudaError_t e = launch_gemm(M, N, K, A, lda, B, ldb, bias, C, ldc, D, ldd, gelu, s);
    if (e != cudaSuccess) return e;
    return launch_transpose_bf16(M, Mpad, N, D, ldd, Dt, ldt, s);
}

cudaError_t gemm_tc_error(int *err)
{
    return cudaMemcpyFromSymbol(err, g_tc_error, sizeof(int));
}

}  // namespace sas

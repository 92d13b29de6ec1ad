// Internal declarations shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sas.h"

namespace sas {

constexpr int kTile = 128;      // atoms per I-tile of the mixed kernel (= its threads per CTA); group padding
constexpr int kTile64 = 64;     // atoms per I-tile of the FP64 kernel
constexpr int kQChunk = 208;    // q values one pass of a pair kernel covers (52 blocks of 4)
constexpr int kMaxChunks = 64;    // passes of one q grid (runs of uniform spacing, split)
constexpr int kPackThreads = 256;

// One unit of pair work: an I-tile of one type against a contiguous J-range of
// one type (both inside one conformer), for one chunk of the q grid.  All
// pairs of an item share the type pair, so the item's sums belong to one S_ab.
struct Item {
    int batch;   // conformer
    int pair;    // type-pair index p(a,b), a <= b
    int i0;      // first slot of the I-tile
    int j0;      // first slot of the J-range
    int jlen;    // J-range length in slots (a multiple of the I-tile)
    int chunk;   // q chunk
    int diag;    // 1 when the J-range starts at the I-tile (same type): pairs with j <= i are masked
    int work;    // jlen * tile (for scheduling)
};

// The q grid as runs of uniform spacing (one run for a uniform grid), each run split into passes
// of at most kQChunk values: chunk c holds q_k = qsd[c] + (k - q_begin[c]) dqd[c] for
// q_begin[c] <= k < q_begin[c] + q_len[c].
// Largest (sin, cos)(k/64) table a call uses (entries): the 208-q two-pair kernel stages it in
// shared memory.
constexpr int kStagedSincosTab = 2048;

struct QChunks {
    int n_q;
    int n_chunks;
    int q_begin[kMaxChunks];
    int q_len[kMaxChunks];
    float qs_hi[kMaxChunks];   // first q of the chunk as a float32 pair (hi + lo)
    float qs_lo[kMaxChunks];
    float dq_hi[kMaxChunks];   // step of the chunk as a float32 pair
    float dq_lo[kMaxChunks];
    double qsd[kMaxChunks];    // the same in FP64
    double dqd[kMaxChunks];
    // 1 when the chunk's first q equals its step (a grid q_k = k dq, k >= 1): the start phase of a
    // pair is then its step phase dq r, whose sin and cos the mixed kernels form anyway
    int start_is_step[kMaxChunks];
    // (sin, cos)(k/64) for k < sct_n <= kStagedSincosTab as float32 hi/lo (sincos_tab), covering every
    // pair's step phase dq r of the call; null: the polynomial sincos
    const float4 *sct = nullptr;
    int sct_n = 0;
    // 1: the mixed kernels form each pair's coefficient 2cos(2t) from 4 sin^2 t or 4 cos^2 t,
    // whichever is smaller (set where the call's step phase can come near pi); 0: from 4 sin^2 t
    int coef_both = 0;
};

// Largest step phase M dq D from which the mixed kernels form their coefficients both ways.
constexpr double kCoefBothPhase = 0.8 * 3.14159265358979323846;

// q_k of the grid (a short scan over the chunks).
__host__ __device__ inline double q_at(const QChunks &qc, int k)
{
    int c = 0;
    while (c + 1 < qc.n_chunks && qc.q_begin[c + 1] <= k) ++c;
    return qc.qsd[c] + (double)(k - qc.q_begin[c]) * qc.dqd[c];
}

// Fill qc for q[0..n_q): maximal runs of uniform spacing (deviation <= tol * max|q|), split into
// passes of at most max_len (<= kQChunk) values.  False if the grid needs more than kMaxChunks passes.
bool make_chunks(const double *q, int n_q, QChunks &qc, int max_len = kQChunk);

// ---- packing (pack.cu) -------------------------------------------------------
// meta layout (int32): [0,T) real counts, [T, 2T+1) padded group offsets, [2T+1] error bits
enum { kErrBadType = 1, kErrNonFinite = 2, kErrNonFiniteFF = 4 };

// extent2 (may be NULL): max over conformers and atoms of the squared distance from the
// conformer's first atom, as float bits (atomicMax; zero it first)
cudaError_t launch_count_types(const void *coords, int coords_f64, const int32_t *types, int64_t n,
                               int64_t batch, int n_types, int *blockcounts, int *errword,
                               unsigned *extent2, cudaStream_t s);
cudaError_t launch_scan_counts(const int *blockcounts, int nblk, int n_types, int tile,
                               int *blockoffs, int *meta, cudaStream_t s);
cudaError_t launch_centroid(const void *coords, int coords_f64, int64_t n, int64_t batch,
                            double *centroid, cudaStream_t s);
// X: float4 [batch][npad] (mixed) or double4 (fp64); padding slots must be zero beforehand.
cudaError_t launch_scatter(const void *coords, int coords_f64, const int32_t *types, int64_t n,
                           int64_t batch, int n_types, const int *blockoffs, const int *meta,
                           const double *centroid, int out_f64, void *X, int64_t npad,
                           int *slot_of, cudaStream_t s);

// ---- form factors and assembly (reduce.cu) -----------------------------------
// F [T][n_q] f64 from coefficients [T][9]
cudaError_t launch_form_factors(const double *coef, int n_types, const QChunks &qc, double *F,
                                cudaStream_t s);
// S[b][p][k] = sum over the items of group (b,p) of partial[item][k - q_begin(chunk)] (fixed order)
cudaError_t launch_reduce_items(const double *partial, int part_stride, const Item *items,
                                const int *group_items, const int *group_off, int n_groups,
                                const QChunks &qc, double *S, cudaStream_t s);
// The same sums for groups of any size: groups of more than kSegItems items are summed as
// segments of kSegItems (in list order) and then the segments in order; seg_out holds
// n_groups * ceil(max_group / kSegItems) * n_q doubles.
constexpr int kSegItems = 256;
cudaError_t launch_reduce_items_seg(const double *partial, int part_stride, const Item *items,
                                    const int *group_items, const int *group_off, int n_groups, int max_group,
                                    const QChunks &qc, double *seg_out, double *S, cudaStream_t s);
// Exact cross-item sums (deterministic contexts): a partial sum v enters as the integer nearest
// v * 2^kFixBits (ties to even; v itself when |v| >= 2^-7, whose 53 significant bits then lie above
// 2^-60), held in 128-bit two's complement, so that a sum of partials does not depend on the order
// or grouping of its terms.  |v| and every sum stay below 2^67.
constexpr int kFixBits = 60;
struct Fix128 {
    unsigned long long lo;
    long long hi;
};
// U[g][k] = the exact sum of group g's item partials at q_k (segment sums in seg_out
// [n_groups][max(1, ceil(max_group / kSegItems))][n_q]), then S as launch_fix_to_S.
cudaError_t launch_reduce_items_fix(const double *partial, int part_stride, const Item *items,
                                    const int *group_items, const int *group_off, int n_groups, int max_group,
                                    const QChunks &qc, Fix128 *seg_out, Fix128 *U, double *S, cudaStream_t s);
// S[g][k] = (q_k > 0 ? double(U[g][k]) 2^-kFixBits / q_k : 0) for n_groups groups.
cudaError_t launch_fix_to_S(const Fix128 *U, int64_t n_groups, const QChunks &qc, double *S, cudaStream_t s);
// I[b][k] = sum_t n_t F_t^2 + sum_p 2 F_a F_b (q_k > 0 ? S/q_k : count_p)
cudaError_t launch_assemble(double *S, const double *F, const int *meta, int n_types, int64_t batch,
                            const QChunks &qc, int whole, double *I, cudaStream_t s);

// ---- pair kernels -------------------------------------------------------------
// partial [n_items][part_stride] f64: sum over the item's pairs of w_i w_j sin(q r)/r.
// ticket: one device int, zero when the kernel starts (the CTAs draw items from it).
cudaError_t launch_debye_mixed(const float4 *X, int64_t npad, const Item *items, int n_items,
                               const QChunks &qc, int step, int reseed, int variant, double *partial,
                               int part_stride, int grid, int jmax, int *ticket, cudaStream_t s);
// The two-pairs-per-step form of the 2-step kernel without re-seeding (same arguments and result).
cudaError_t launch_debye_mixed_pairs2(const float4 *X, int64_t npad, const Item *items, int n_items,
                                      const QChunks &qc, double *partial, int part_stride, int grid, int jmax,
                                      int *ticket, cudaStream_t s, int tile = kTile);
cudaError_t launch_debye_fp64(const double4 *X, int64_t npad, const Item *items, int n_items,
                              const QChunks &qc, double *partial, int part_stride, int grid,
                              cudaStream_t s);
// q capacity (in blocks of four q) of the mixed-precision kernels for a chunk of qlen_max values
int mixed_blocks_for(int qlen_max);
// Automatic re-seed interval of the mixed recurrence (0: none) for a molecule of n_atoms, passes
// of up to n_q_chunk q values and a largest phase step M dq D (radians).
int reseed_auto(int64_t n_atoms, int n_q_chunk, double step_phase_max);

// ---- adjoint (adjoint.cu) -------------------------------------------------------
// g[b][k] = 2 w_k (I_bk - T_k), chi2[b] = sum_k w_k (I_bk - T_k)^2 (chi2 may be null)
cudaError_t launch_chi2(const double *I, const double *T, const double *w, int n_q, int64_t batch,
                        double *g, double *chi2, cudaStream_t s);
// H[b][p][k] = (g f_a f_b, g f_a f_b / q) as float2, row stride hstride
cudaError_t launch_adjoint_coef(const double *g, const double *F, int n_types, int64_t batch,
                                const QChunks &qc, float2 *H, int hstride, cudaStream_t s);
// G[b][slot][3] += d(sum_q g_q I(q)) / dx (G must be zeroed); jlen_max: the longest J-range of
// the items (sets the shared memory); ticket: one device int, zero when the kernel starts.
// PI == nullptr: item totals added to G (zeroed by the caller) with FP64 atomics.  Otherwise the
// deterministic form: item e's totals go to PI [n_items][kTile][3] and PJ [n_items][adjoint_jcap][3]
// (G untouched), and launch_adjoint_gather adds them up per atom over the tile lists
// (tile_off [batch * ntiles + 1], tile_ent: 2e for item e's I-tile, 2e + 1 for its J-range, in a
// fixed order), writing every slot of G.
inline int adjoint_jcap(int jlen_max) { return (jlen_max + 1) / 2 * 2; }
cudaError_t launch_debye_adjoint(const float4 *X, int64_t npad, const Item *items, int n_items,
                                 const QChunks &qc, const float2 *H, int n_pairs, int hstride, double *G,
                                 int jlen_max, int *ticket, float *PI, float *PJ, cudaStream_t s);
// The tabulated form: K [n_q][n_rows] FP64 (r_m = m step), then per conformer and type pair the FP64
// nodes Wn [batch P][n_rows] and the cubic coefficients tab [batch P][n_rows - 2] float4 of
// W(r) = 2 sum_q h_q (cos(q r) - sinc(q r)) / r^2, h_q = g_q f_a(q) f_b(q) (batch P <= 65535), and
// the pair kernel over the table (same arguments and outputs as launch_debye_adjoint otherwise).
constexpr double kAdjTabStep = 0.05;   // q_max times the node spacing
cudaError_t launch_adjoint_kmat(const QChunks &qc, int n_rows, double step, double *K, cudaStream_t s);
cudaError_t launch_adjoint_wtab(const double *g, const double *F, int n_types, int64_t batch, int n_q, const double *K,
                                int n_rows, double *Wn, float4 *tab, cudaStream_t s);
cudaError_t launch_debye_adjoint_tab(const float4 *X, int64_t npad, const Item *items, int n_items, const float4 *tab,
                                     int n_int, float inv_step, int n_pairs, double *G, int jlen_max, int *ticket,
                                     float *PI, float *PJ, cudaStream_t s);
// Per-atom form factors: the weights AI [b][pass][slots][npad] float4 from the caller's ff [b][k][i] and
// g [b][k], and the pair kernel over them and the forward table FJ [b][pass][npad/2][slots] (passes of
// at most 2 * adjoint_atomic_slots() q; G as launch_debye_adjoint without PI).
int adjoint_atomic_slots();
cudaError_t launch_atomic_adj_table(const double *ff, const double *gI, const int *slot_of, int64_t n, int64_t npad,
                                    int64_t batch, const QChunks &qc, float4 *AI, cudaStream_t s);
cudaError_t launch_debye_adjoint_atomic(const float4 *X, int64_t npad, const Item *items, int n_items,
                                        const QChunks &qc, const float4 *AI, const float4 *FJ, double *G, int jlen_max,
                                        int *ticket, cudaStream_t s);
cudaError_t launch_adjoint_gather(const float *PI, const float *PJ, int jcap, const Item *items,
                                  const int *tile_off, const int *tile_ent, int ntiles, int64_t npad, int64_t batch,
                                  double *G, cudaStream_t s);
cudaError_t launch_unpermute(const double *G, const int *slot_of, int64_t n, int64_t npad, int64_t batch,
                             float *grad_out, cudaStream_t s);

// ---- histogram (histogram.cu) -----------------------------------------------------
size_t histogram_smem(int jcap, int n_bins);
// jlen_max: the longest J-range of the items; ticket: one device int, zero when the kernel starts.
cudaError_t launch_pair_histogram(const float4 *X, int64_t npad, const Item *items, int n_items,
                                  int n_bins, float r_max, int n_pairs, int *hist,
                                  unsigned long long *dropped, int jlen_max, int *ticket, cudaStream_t s);

// ---- MLP (mlp.cu) -------------------------------------------------------------------
// C[M][N] = A[M][K] B[N][K]^T (+ bias); bfloat16 A, B (K % 16 == 0, ld % 8 == 0, 16-byte
// aligned), FP32 C (may be null); D (bfloat16, may be null) gets the value or GELU(value).
cudaError_t launch_gemm_tn(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias,
                           float *C, int ldc, void *D, int ldd, int gelu, cudaStream_t s);
// The same product on the tcgen05 tensor cores (TMA-fed, TMEM accumulator); usable when
// gemm_tc_supported(K, A, lda, B, ldb).  gemm_tc_error reads the device error word (nonzero after
// a wait inside the kernel ran out of iterations).
bool gemm_tc_supported(int K, const void *A, int lda, const void *B, int ldb);
cudaError_t launch_gemm_tc(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias,
                           float *C, int ldc, void *D, int ldd, int gelu, cudaStream_t s);
cudaError_t gemm_tc_error(int *err);
// Screening: surrogate chi^2 per conformer, top-k selection (n <= select_max()), row gather.
int select_max();
cudaError_t launch_surrogate_chi2(int n_conf, int n_q, const float *z, int ld, const double *mean, const double *stdv,
                                  const double *base, int ld_base, const double *target, const double *w, double *chi2,
                                  cudaStream_t s);
cudaError_t launch_select_topk(int n, const double *chi2, int k, int32_t *top_idx, double *top_chi2, cudaStream_t s);
cudaError_t launch_gather_rows(const void *src, int64_t row_bytes, const int32_t *idx, int64_t n_idx, void *dst,
                               cudaStream_t s);
// Split-K on the tcgen05 GEMM: K cut into `splits` slices of whole 64-wide stages (none empty), slice
// z's FP32 product of A [M][K] and B [N][K] into ws + z M N ([M][N], no bias).  cudaErrorInvalidValue
// where the operands do not suit TMA or a slice would be empty.
cudaError_t launch_gemm_splitk(int M, int N, int K, const void *A, int lda, const void *B, int ldb, float *ws, int splits,
                               cudaStream_t s);
cudaError_t launch_splitk_gelu(int M, int Mpad, int N, int splits, const float *ws, const float *bias, float *Z, void *A,
                               void *At, int ldt, cudaStream_t s);
// launch_gemm with D (required) also written transposed: Dt[col][row] (leading dimension ldt >= Mpad),
// zero for rows [M, Mpad); from the tcgen05 epilogue where it runs that form, else by a transpose.
cudaError_t launch_gemm_t(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias,
                          float *C, int ldc, void *D, int ldd, int gelu, void *Dt, int ldt, int Mpad, cudaStream_t s);
// launch_gemm_tc where supported, else launch_gemm_tn.
cudaError_t launch_gemm(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias,
                        float *C, int ldc, void *D, int ldd, int gelu, cudaStream_t s);
cudaError_t launch_to_bf16(int64_t n, const float *x, void *y, cudaStream_t s);
cudaError_t launch_to_bf16_t(int R, int Rpad, int C, const float *x, void *xb, void *xt, int ldt, cudaStream_t s);
cudaError_t launch_transpose_bf16(int R, int Rpad, int C, const void *in, int ldin, void *out, int ldout,
                                  cudaStream_t s);
// Fused backward steps of the surrogate (mlp.cu).  lpart: [Bpad / 8] FP64; part: FP32 partials,
// [Bpad / 8][Qpad] for the MSE and [ceil(Bpad / 32)][C] for the activation; count: zero-initialized
// counters, at least ceil(C / 32) (each launch leaves them zero).
cudaError_t launch_mse_fused(int B, int Bpad, int Q, int Qpad, const float *Y, const float *T, float *dY, void *dYb,
                             void *dYt, int ldt, double *lpart, float *part, float *db, float *loss, unsigned *count,
                             cudaStream_t s);
cudaError_t launch_act_bwd(int B, int Bpad, int C, const float *dA, const float *Z, float *dZ, void *dZb, void *dZt,
                           int ldt, float *part, float *db, unsigned *count, cudaStream_t s);
cudaError_t launch_adam(int64_t n, float *p, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                        int64_t step, void *pb, cudaStream_t s);

// the calling thread's error message (sas_last_error)
sas_status set_error(sas_status st, const char *msg);

// A named NVTX range over one entry point, so that a profiler can select a call's kernels by name
// (ncu --nvtx --nvtx-include NAME/); without a tool attached the header-only NVTX calls do nothing.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ---- per-atom form factors (atomic.cu, atomic_pairs2.cu) -------------------------------------
int atomic_slots(const QChunks &qc);
int atomic_jmax(const QChunks &qc);
cudaError_t launch_check_finite(const double *v, int64_t count, int *err, cudaStream_t s);
cudaError_t launch_atomic_tables(const double *ff, const int *slot_of, int64_t n, int64_t npad, int64_t batch,
                                 const QChunks &qc, int nv, float4 *FJ, float2 *FI, cudaStream_t s);
cudaError_t launch_atomic_table64(const double *ff, const int *slot_of, int64_t n, int64_t npad, int64_t batch,
                                  int n_q, double *F64, cudaStream_t s);
cudaError_t launch_atomic_diag(const double *ff, int64_t n, int64_t batch, int n_q, double2 *D, cudaStream_t s);
cudaError_t launch_assemble_atomic(const double *S, const double2 *D, const QChunks &qc, int64_t batch, double *I,
                                   cudaStream_t s);
cudaError_t launch_debye_atomic_pairs2(const float4 *X, int64_t npad, const Item *items, int n_items,
                                       const QChunks &qc, const float4 *FJ, const float2 *FI, double *partial,
                                       int part_stride, int grid, int jmax, int *ticket, cudaStream_t s);
cudaError_t launch_debye_fp64_atomic(const double4 *X, int64_t npad, const Item *items, int n_items,
                                     const QChunks &qc, const double *F64, double *partial, int part_stride,
                                     int grid, cudaStream_t s);

// ---- orientation average by quadrature (quadrature.cu) --------------------------------------
constexpr int kQuadChunk = 32;   // q values of one quadrature pass
// The launch plan of the quadrature method: per q chunk its q run, its direction set (an offset
// into the direction array), its split of the packed atoms into segments over CTAs, and the
// offset of its partial amplitudes ([segment][kQuadChunk][direction] double2 per conformer).
struct QuadPlan {
    int n_chunks;
    int q_begin[kMaxChunks], q_len[kMaxChunks];
    float qs_hi[kMaxChunks], qs_lo[kMaxChunks], dq_hi[kMaxChunks], dq_lo[kMaxChunks];
    int dir_off[kMaxChunks], n_dir[kMaxChunks], n_seg[kMaxChunks], seg_len[kMaxChunks];
    int64_t amp_off[kMaxChunks];
    int cta_off[kMaxChunks + 1];
    int64_t amp_stride;   // double2 per conformer
};
int quad_degree(double x, double tol);
void quad_directions(int L, std::vector<float4> &dirs, std::vector<double> &wts);
int quad_threads_per_cta();
// cen[b] = (FP64 centroid of the real atoms of conformer b, largest distance from it)
cudaError_t launch_packed_geometry(const float4 *X, int64_t npad, int64_t batch, double4 *cen, cudaStream_t s);
// I[b][q_begin[c] + k] for every chunk of the plan (F: [n_types][n_q] form factors of the full grid)
// (pl on the host for the launch shape, pl_dev its device copy for the kernels)
cudaError_t launch_quad(const float4 *X, int64_t npad, int64_t batch, const int *type_off, int n_types,
                        const double4 *cen, const double *F, int n_q, const QuadPlan &pl, const QuadPlan *pl_dev,
                        const float4 *dirs, const double *wts, double2 *Apart, double *I, cudaStream_t s);

namespace api {
// Every device allocation of the library (guard.cu): cudaMalloc / cudaFree, with guard bands
// around the buffer while they are switched on (sas_guard_bands).
cudaError_t dev_malloc(void **p, size_t bytes);
void dev_free(void *p);
}  // namespace api

}  // namespace sas

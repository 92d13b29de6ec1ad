/*
 * sas.h — C ABI of the GB300 (sm_103a) direct Debye summation library (libsas.so).
 *
 * The operation is the Debye sum of Berlin, Gumerov, Duraiswami and Fushman,
 * "Performance of a GPU-based Direct Summation Algorithm for Computation of
 * Small Angle Scattering Profile" (Section I-A, Eq. 2):
 *
 *     I(q) = sum_k sum_j f_k(q) f_j(q) sin(q r_jk) / (q r_jk),   sinc(0) = 1,
 *
 * over all N atoms of a molecule, on a grid of q values made of uniform runs, with the
 * per-atom form factors f_j(q) taken from a small set of atom types:
 *
 *     f_t(q) = sum_{k=1..4} a_k exp(-b_k (q / 4 pi)^2) + c      (coefficients per type t),
 *
 * or given per atom and q (sas_profile_atomic).
 *
 * Conventions for every entry point
 *  - Every function returns a sas_status; nothing throws across the ABI.
 *    sas_last_error() gives a message for the calling thread's last failure.
 *  - The caller owns every input and output buffer.  Pointers may be host or
 *    device memory (told apart with cudaPointerGetAttributes).  Device
 *    buffers are used in place on the caller's stream; host buffers are
 *    staged through context-owned device memory, and a call with a host
 *    output returns only after the result has been copied back.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *  - Validation (n < 0, null pointers, type out of range, non-finite
 *    coordinate or form factor) happens before any output is written: on an
 *    error the outputs are untouched.  Device-resident inputs are validated by
 *    a kernel whose verdict (with the type counts) the host reads back, so
 *    these calls synchronize on the stream once, before packing (the
 *    quadrature method of SAS_OPT_METHOD reads back the molecule's radius
 *    once more, after packing).
 *  - A context is not thread-safe: use one context per host thread.
 *  - Layouts are C order (row-major): coords [batch][n][3], outputs [batch][...].
 *  - Atom pairs are counted as unordered distinct pairs i<j (Section II: only
 *    j <= k is computed); the diagonal sum_i f_i^2 is added exactly in FP64.
 */
#ifndef SAS_H
#define SAS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sas_ctx sas_ctx; /* opaque; owns the form-factor table and device workspace */

typedef enum {
    SAS_OK = 0,
    SAS_ERR_INVALID_ARG = 1, /* bad size, null pointer, type out of range, NaN/Inf coordinate */
    SAS_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed */
    SAS_ERR_ALLOC = 3,       /* device or host allocation failed (nothing leaked) */
    SAS_ERR_UNSUPPORTED = 4, /* q grid of too many uniform runs, too many q values or types */
    SAS_ERR_TIMEOUT = 5,     /* a wait on the device exceeded its limit */
    SAS_ERR_CORRUPT = 6      /* a guard band around a device buffer was overwritten (sas_guard_check) */
} sas_status;

/* precision (sas_create flags) */
enum {
    SAS_MIXED = 0, /* FP32 pair terms and per-thread sums, FP64 from the first cross-thread sum on */
    SAS_FP64 = 1   /* every step in FP64 (the plain form) */
};

/*
 * SAS_DETERMINISTIC (sas_create flag, ORed with the precision): every output of the context is the
 * same bit for bit on every call with the same inputs, options and device, and a profile split
 * into shards (SAS_OPT_SHARD) can be put back together bit for bit (sas_exact_sums,
 * sas_assemble_exact).  The profiles, partials, histograms and quadrature sums repeat on every
 * context (each work item writes its own partial sums, which are added in a fixed order).  The flag
 * (1) makes the direct profile add the items' partial sums exactly (sas_exact_sums) and keeps its
 * I-tiles at 128 atoms, and (2) changes the adjoint (sas_profile_grad, sas_profile_vjp), whose
 * per-atom gradient sums otherwise use FP64 atomics in whatever order the items finish: every work
 * item writes its gradient totals to a buffer of its own (12 * (128 + J) bytes per item, J the
 * longest J-range of the call, at most 512 atoms) and a further kernel adds them per atom in a
 * fixed order.  Results differ from a context without the flag by the rounding of the regrouped
 * sums.
 */
#define SAS_DETERMINISTIC 16

/* coordinate element type (per call) */
enum { SAS_COORDS_F32 = 0, SAS_COORDS_F64 = 1 };

/* limits */
#define SAS_MAX_TYPES 16
#define SAS_MAX_Q 1664

/*
 * Create a context for n_types atom types and a q grid.
 *   ff_coef  [n_types][9] host, (a1..a4, b1..b4, c) per type; copied.
 *   q        [n_q] host, strictly ascending, q[0] >= 0; copied.  The grid is taken as maximal runs
 *            of uniform spacing (every point within 1e-9 max|q| of its run's line; a uniform grid
 *            is one run, an irregular one runs of two points), each run computed from its own
 *            start and step; at most 64 runs after cutting each into pieces of <= 208 values.
 *   flags    SAS_MIXED or SAS_FP64, optionally | SAS_DETERMINISTIC.
 * Errors: INVALID_ARG (n_types outside 1..SAS_MAX_TYPES, n_q outside 1..SAS_MAX_Q,
 * null pointer, negative or non-finite q or coefficient), UNSUPPORTED (q not strictly ascending,
 * more than 64 runs), ALLOC, CUDA.  *out is set only on success.
 */
sas_status sas_create(int n_types, const double *ff_coef, const double *q, int n_q, unsigned flags,
                      sas_ctx **out);

/* Free the context and all of its device memory.  NULL is accepted. */
sas_status sas_destroy(sas_ctx *ctx);

/*
 * I(q) of one molecule (Eq. 2).
 *   coords  [n_atoms][3] float (coords_type SAS_COORDS_F32) or double (SAS_COORDS_F64), Å.
 *   types   [n_atoms] int32 in [0, n_types).
 *   I_out   [n_q] double.
 * n_atoms = 0 gives I = 0; n_atoms = 1 gives f^2.
 */
sas_status sas_profile(sas_ctx *ctx, const void *coords, int coords_type, const int32_t *types,
                       int64_t n_atoms, double *I_out, void *stream);

/*
 * I(q) of `batch` conformers of one molecule (shared types), one launch per step.
 *   coords [batch][n_atoms][3], I_out [batch][n_q].
 */
sas_status sas_profile_batch(sas_ctx *ctx, const void *coords, int coords_type, const int32_t *types,
                             int64_t n_atoms, int64_t batch, double *I_out, void *stream);

/*
 * Refinement objective and its gradient (derivative of Eq. 2 with respect to the positions):
 *   chi2_b   = sum_q w_q (I_b(q) - T(q))^2
 *   grad_b,i = d chi2_b / d x_i = sum_{j != i} w_ij (x_i - x_j),
 *   w_ij     = (2 / r^2) sum_q g_q f_i f_j (cos(q r) - sinc(q r)),  g_q = 2 w_q (I(q) - T(q)).
 *   coords [batch][n_atoms][3] float, target [n_q] double, weights [n_q] double,
 *   chi2_out [batch] double, grad_out [batch][n_atoms][3] float (caller's atom order),
 *   I_out [batch][n_q] double or NULL.
 * Mixed precision only (SAS_MIXED context): FP32 pair terms, FP64 accumulation of gradients.
 */
sas_status sas_profile_grad(sas_ctx *ctx, const float *coords, const int32_t *types, int64_t n_atoms,
                            int64_t batch, const double *target, const double *weights,
                            double *chi2_out, float *grad_out, double *I_out, void *stream);

/*
 * Vector-Jacobian product of Eq. 2 (the backward of I(q) for autograd):
 *   grad_out[b][i] = sum_q grad_I[b][q] dI_b(q)/dx_i.
 *   coords [batch][n_atoms][3] float, grad_I [batch][n_q] double, grad_out [batch][n_atoms][3] float.
 */
sas_status sas_profile_vjp(sas_ctx *ctx, const float *coords, const int32_t *types, int64_t n_atoms,
                           int64_t batch, const double *grad_I, float *grad_out, void *stream);

/*
 * The last profile call's type-pair sinc sums (the factoring of Eq. 2 over atom types):
 *   S_out[b][p][k] = sum over unordered pairs i<j with types {a,b} of sinc(q_k r_ij),
 *   p = a*T - a(a-1)/2 + (b - a) for a <= b, T = n_types.  S_out has batch*T(T+1)/2*n_q doubles.
 * Then I(q) = sum_t n_t f_t(q)^2 + sum_p 2 f_a(q) f_b(q) S_p(q).
 */
sas_status sas_partials(sas_ctx *ctx, double *S_out, int64_t capacity, void *stream);

/*
 * Exact sums for splitting one molecule over shards (SAS_OPT_SHARD) on SAS_DETERMINISTIC contexts,
 * whose direct profile calls add the work items' partial sums U_p(q) = sum sin(q r)/r exactly: each
 * partial v enters as the integer nearest v * 2^60 (v itself for |v| >= 2^-7), held in 128-bit two's
 * complement, so the sum does not depend on the order or grouping of its terms.
 *
 * sas_exact_sums: the last sas_profile / sas_profile_batch call's (direct sum, SAS_OPT_METHOD 0) exact
 *   sums, U_out[b][p][k][0..1] = (low 64 bits as unsigned, high 64 bits as signed) of U_p(q_k) * 2^60
 *   (0 at q = 0), batch * T(T+1)/2 * n_q * 2 int64, pair index p as in sas_partials.  On a shard
 *   these are the shard's own; the 128-bit sums over all shards equal the unsplit call's.
 * sas_assemble_exact: I(q) of the whole molecule from such sums U (e.g. added over all shards; same
 *   layout, device or host), with the type counts of the context's last profile call (same molecule,
 *   batch as then): the arithmetic of an unsplit call after its sums, so the result equals that
 *   call's bit for bit.
 * Errors: INVALID_ARG (null pointer, capacity too small, no direct profile since the last other
 * call, batch differing from the last call's), UNSUPPORTED (context without SAS_DETERMINISTIC), CUDA.
 */
sas_status sas_exact_sums(sas_ctx *ctx, int64_t *U_out, int64_t capacity, void *stream);
sas_status sas_assemble_exact(sas_ctx *ctx, const int64_t *U, int64_t batch, double *I_out, void *stream);

/*
 * I(q) with a form factor per atom and q, no types (Section I-A, Eq. 2 as written: with a hydration
 * layer the products f_k f_j do not reduce to a few types; Section II keeps, for every q value, one
 * form factor per atom).  The context supplies the q grid, precision and options; its type
 * coefficients are not used.
 *   coords [batch][n_atoms][3] float or double (coords_type), device or host.
 *   ff     [batch][n_q][n_atoms] double, f_i(q_k) at ff[(b * n_q + k) * n_atoms + i], device or host.
 *   I_out  [batch][n_q] double: sum_i f_i(q)^2 + 2 sum_{i<j} f_i(q) f_j(q) sinc(q r_ij), and at
 *          q = 0 exactly (sum_i f_i(0))^2.
 * The mixed path weights each FP32 recurrence term by f_j(q) in FP32 and each atom's sums by
 * f_i(q) in FP32 before the FP64 reduction; the diagonal and q = 0 are FP64.  Small molecules
 * (the automatic re-seed rule of SAS_OPT_RESEED) run the q grid in passes of the re-seed interval.
 * Errors: INVALID_ARG (null pointer, bad coords_type, non-finite coordinate or form factor),
 * UNSUPPORTED (sharded context, batch > 65535, q grid needing more than 64 passes), ALLOC, CUDA,
 * TIMEOUT.  sas_partials is not available after this call.
 */
sas_status sas_profile_atomic(sas_ctx *ctx, const void *coords, int coords_type, int64_t n_atoms, int64_t batch,
                              const double *ff, double *I_out, void *stream);

/*
 * Vector-Jacobian product of the per-atom profile (the derivative of Eq. 2 with a form factor per
 * atom and q, for refinement against data with a hydration layer or excluded volume, Section I-A
 * after Eq. 2): grad_out[b][i] = sum_q grad_I[b][q] dI_b(q)/dx_i
 *   = sum_{j != i} W_ij (x_i - x_j),  W_ij = 2 sum_q grad_I[q] f_i(q) f_j(q) (cos(q r) - sinc(q r)) / r^2,
 * with the form factors held fixed.  coords [batch][n_atoms][3] float, ff [batch][n_q][n_atoms] as in
 * sas_profile_atomic, grad_I [batch][n_q] double, grad_out [batch][n_atoms][3] float (host or device).
 * The sums over q run in passes of at most 52 q by the FP32 recurrence with FP64 accumulation of the
 * atom totals.  A SAS_MIXED, non-deterministic, unsharded context is needed (else UNSUPPORTED).
 * Errors: INVALID_ARG (sizes, null pointers, non-finite coordinates or form factors), UNSUPPORTED,
 * ALLOC, CUDA, TIMEOUT.
 */
sas_status sas_profile_vjp_atomic(sas_ctx *ctx, const float *coords, int64_t n_atoms, int64_t batch, const double *ff,
                                  const double *grad_I, float *grad_out, void *stream);

/*
 * Peak microbenchmarks of the current device (the denominators of the pair kernels' rooflines):
 * out[0] FP32 FMA lane operations/s (scalar FFMA), out[1] the same with packed f32x2 FMA (2 per
 * instruction and lane), out[2] MUFU sine operations/s (__sinf), out[3] FP64 FMA lane
 * operations/s, out[4] the SM clock (MHz) seen during the FFMA run (clock64 against the global
 * timer), and with n_out >= 6 out[5] shared-memory integer atomic adds/s without bank conflicts
 * (each lane adding to a word of its own bank), with n_out >= 7 out[6] packed FMA lane operations/s
 * when every instruction reads three distinct register pairs (no operand shared with the previous
 * instruction).  Each kernel runs about 10 ms on `stream`; the
 * call waits for them.  out is host memory of n_out >= 5 doubles.  Errors: INVALID_ARG, CUDA.
 */
sas_status sas_measure_peaks(double *out, int n_out, void *stream);

/*
 * Exact integer histogram of unordered pair distances by type pair.
 *   coords [batch][n_atoms][3] float; types [n_atoms]; hist_out [batch][T(T+1)/2][n_bins] int32;
 *   dropped_out [batch] int64 (pairs beyond the last edge) or NULL.
 * Distance rule (identical on every platform): dx = x_i - x_j (likewise dy, dz) in float32,
 *   r2 = fmaf(dz, dz, fmaf(dy, dy, dx*dx)); w = r_max / n_bins; e_k = (float)k * w; e_k2 = e_k*e_k;
 *   bin = max{k : e_k2 <= r2}, dropped if bin >= n_bins.
 * n_bins in [1, 4096]; r_max <= 1e18 and r_max / n_bins >= 1e-12 (so that every e_k2 is a normal
 * float), else SAS_ERR_INVALID_ARG.
 * The caller's float32 coordinates are used unchanged (no centering).
 */
sas_status sas_pair_histogram(sas_ctx *ctx, const float *coords, const int32_t *types, int64_t n_atoms,
                              int64_t batch, int n_bins, float r_max, int32_t *hist_out,
                              int64_t *dropped_out, void *stream);

/*
 * The Debye sum over pair-distance histograms with every pair at its bin centre: Eq. 2 (Section
 * I-A) with each pair distance replaced by the centre r_k = (k + 1/2) r_max / n_bins of its
 * histogram bin, which costs O(T^2 n_bins) per q instead of O(N^2).  Not the paper's method (which
 * sums every pair exactly); the baseline a learned surrogate must beat.
 *   I_c(q) = sum_t n_t f_t(q)^2 + sum_{a<=b} 2 f_a(q) f_b(q) sum_k hist_c[p(a,b)][k] sinc(q r_k)
 * hist [batch][T(T+1)/2][n_bins] int32 (sas_pair_histogram's layout; host or device, counts below
 * 2^24), type_counts [T] host int64 (atoms of each type, the same for every conformer), I_out
 * [batch][n_q] double (host or device), with the context's form factors and q grid.  The table of
 * 2 f_a f_b sinc(q r_k) is built on the first call for an (n_bins, r_max) and kept in the context.
 * FP32 products summed over 32 bins in FP32, then in FP64.  Asynchronous for device outputs.
 * Errors: INVALID_ARG (sizes, null pointers, negative counts), UNSUPPORTED (batch > 2^28), ALLOC,
 * CUDA, TIMEOUT.
 */
sas_status sas_binned_profile(sas_ctx *ctx, const int32_t *hist, int64_t batch, int n_bins, float r_max,
                              const int64_t *type_counts, double *I_out, void *stream);

/* Tuning and diagnostics (values are validated; unknown options give INVALID_ARG). */
enum {
    SAS_OPT_JMAX = 1,        /* longest J-range of one work item, atoms (multiple of 128 up to 8192; 0 = automatic) */
    SAS_OPT_RESEED = 2,      /* re-seed interval of the q recurrence in q steps: -1 automatic (default:
                                none from 8,192 atoms, or from 2,000 atoms when a q chunk holds at most
                                104 values, except every 64 when a chunk holds more than 128 values and
                                the phase step M dq D reaches 0.9 pi, M the q steps per recurrence step
                                (SAS_OPT_STEP) and D twice the largest distance from the first atom of a
                                conformer; otherwise 32), 0, 32 or 64 */
    SAS_OPT_VALIDATE = 3,    /* must stay 1: the device-side validation verdict is always read back */
    SAS_OPT_GRID = 4,        /* persistent CTAs per SM for the pair kernels (0 = automatic) */
    SAS_OPT_TIMEOUT_MS = 5,  /* limit of every host-side wait for device work (default 600000) */
    SAS_OPT_STEP = 6,        /* q steps per recurrence step of the mixed kernel: 2 (default) or 4 */
    SAS_OPT_VARIANT = 7,     /* mixed kernel form for step 2 without re-seed: 0 auto, 1 general,
                                2 set-up of the next pair overlapped, 3 pairs in sequence,
                                4 two pairs per step on packed FP32 (same result bit for bit as 2 and 3) */
    SAS_OPT_SHARD = 8,       /* world * 65536 + rank (default 1 * 65536 + 0): later calls compute shard
                                `rank` of a work list split into `world` contiguous parts of equal pair
                                work.  sas_profile / sas_profile_batch then return that shard's share
                                of I(q) (the diagonal and the exact q = 0 pair counts go to rank 0),
                                so the shards of all ranks sum to the whole profile; sas_partials,
                                sas_profile_vjp and sas_pair_histogram likewise return additive
                                shares; sas_profile_grad needs the whole profile and returns
                                UNSUPPORTED while world > 1. */
    SAS_OPT_METHOD = 9,      /* sas_profile / sas_profile_batch on a SAS_MIXED context: 0 the direct sum
                                (default); 1 hybrid: the orientation average of Eq. 1 by spherical
                                quadrature (Gauss-Legendre x uniform azimuth, degree from the spherical
                                Bessel tail at q R, R the largest distance from the centroid) on the low-q
                                prefix of the grid where it is cheaper than the pair count, the direct sum
                                on the rest; 2 quadrature on every q.  The quadrature error is kept below
                                1e-10 of the amplitude terms; sas_partials is not available after 1 or 2;
                                sas_last_stats entry 6 gives the q values computed by quadrature and
                                entry 7 its directions */
    SAS_OPT_ADJOINT = 10,    /* gradient kernels (sas_profile_grad, sas_profile_vjp): 0 (default) the pair weight
                                W(r) = 2 sum_q h_q (cos(q r) - sinc(q r)) / r^2, a function of the distance alone
                                within one conformer and type pair, tabulated on nodes 0.05 / q_max apart up to
                                the diameter bound and interpolated by cubics (error below 2e-7 of its scale),
                                falling back to 1 when the tables would exceed 2 GB or 65535 conformer type
                                pairs; 1 the sums over q by the three-term recurrence for every pair */
    SAS_OPT_COEF = 11        /* how the mixed kernels form the recurrence coefficient 2cos(2t), t = dq r, of each
                                pair: 0 (default) automatic, both ways once the call's step phase 2 dq D (D as for
                                SAS_OPT_RESEED) reaches 0.8 pi, else as 2 - 4 sin^2 t; 1 always as 2 - 4 sin^2 t;
                                2 always both ways: 2 - 4 sin^2 t where cos 2t >= 0 and 4 cos^2 t - 2 where
                                cos 2t < 0, each from the square that keeps full relative accuracy.  Near
                                2t = pi the first form carries the rounding of sin t and of a square near 4 into
                                the coefficient, which the recurrence turns into a phase drift shared by pairs of
                                similar distance (coarse q grids on large molecules) */
};
sas_status sas_set_option(sas_ctx *ctx, int option, int64_t value);

/*
 * Statistics of the last call: [0] work items, [1] pair slots (incl. padding),
 * [2] unordered real pairs, [3] q values, [4] pair-kernel time in nanoseconds
 * (CUDA events on the call's stream; this call waits for them), [5] kernels launched,
 * [6] q values computed by quadrature (SAS_OPT_METHOD), [7] quadrature directions, [8] atoms per
 * I-tile of the last packing (128, or 64 for small molecules on the two-pair kernel).  n <= 9.
 */
sas_status sas_last_stats(sas_ctx *ctx, int64_t *stats_out, int n);

/*
 * Allocation-free variant of sas_profile for callers that must not allocate GPU memory at the
 * point of use (a memory budget reserved up front, an allocator that must not be re-entered, or
 * a loop where cudaMalloc/cudaFree, which synchronize the device, are not allowed).  The paper
 * has no counterpart; the arithmetic is that of sas_profile on a SAS_MIXED context.
 *   coords [n_atoms][3] float, types [n_atoms] int32, I_out [n_q] double: device memory only.
 *   ff_coef [n_types][9] host memory, as in sas_create.  q_k = q0 + k*dq, k < n_q.
 * No context, no cudaMalloc/cudaFree, no host heap: all scratch lives in one fixed __device__
 * array of SAS_STATIC_SCRATCH_BYTES that every GPU loading the library holds until exit.
 * Limits: n_atoms <= SAS_STATIC_MAX_ATOMS, n_q <= 208, n_types <= SAS_MAX_TYPES; larger sizes
 * give SAS_ERR_UNSUPPORTED; device inputs on the host give SAS_ERR_INVALID_ARG.  The call
 * returns when I_out is written: it waits for `stream` twice, once to read the type counts back
 * (the work list is built from them on the host) and once at the end.  Errors are reported by
 * the status code only (sas_last_error is not updated).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  All calls on a device share the array and
 * it keeps the last call's contents (each call clears what must start at zero); calls that
 * overlap on the GPU race on it.  The library serializes its own calls from several host
 * threads with a lock held until the call's stream has finished; the host-side work list
 * (about 130 KB) is static storage under that lock, not the caller's stack.
 */
#define SAS_STATIC_MAX_ATOMS 16384
#define SAS_STATIC_SCRATCH_BYTES (7 << 20)
sas_status sas_profile_static(const float *coords, const int32_t *types, int64_t n_atoms, int n_types,
                              const double *ff_coef, double q0, double dq, int n_q, double *I_out,
                              void *stream);

/* ---- learned surrogate -------------------------------------------------------------------
 * Not part of the paper's method: a multilayer perceptron that maps per-type-pair distance
 * histograms (sas_pair_histogram) to a standardized log I(q), used to rank conformers before the
 * exact Debye kernel re-scores the best ones.
 *   y = W3 GELU(W2 GELU(W1 x + b1) + b2) + b3,  GELU(z) = z (1 + erf(z / sqrt 2)) / 2,
 *   loss = mean over batch and outputs of (y - t)^2, Adam (beta = 0.9, 0.999, eps = 1e-8).
 * FP32 master weights; every GEMM operand is rounded to bfloat16 and accumulated in FP32 on the
 * tensor cores.  Parameters travel in the packed order W1 [h][n_in], b1 [h], W2 [h][h], b2 [h],
 * W3 [n_out][h], b3 [n_out] (float32, sas_mlp_param_count values).  Inputs x [batch][n_in] and
 * targets t [batch][n_out] are float32, host or device; outputs likewise.
 */
typedef struct sas_mlp sas_mlp;

/* n_in and n_hidden: positive multiples of 16; max_batch <= 65536.  Parameters start at zero. */
sas_status sas_mlp_create(int n_in, int n_hidden, int n_out, int max_batch, sas_mlp **out);
sas_status sas_mlp_destroy(sas_mlp *mlp);
int64_t sas_mlp_param_count(const sas_mlp *mlp);

/* Load / read the full training state (host buffers of sas_mlp_param_count floats each; adam_m and
 * adam_v may be NULL: zero on load, skipped on read).  For checkpoints and deterministic resume. */
sas_status sas_mlp_set_state(sas_mlp *mlp, const float *params, const float *adam_m, const float *adam_v,
                             int64_t step);
sas_status sas_mlp_get_state(sas_mlp *mlp, float *params, float *adam_m, float *adam_v, int64_t *step);

/* y [batch][n_out] = network(x). */
sas_status sas_mlp_forward(sas_mlp *mlp, const float *x, int batch, float *y, void *stream);

/* One Adam step on the MSE loss of (x, t); the batch loss (before the step) goes to loss_out if given. */
sas_status sas_mlp_train_step(sas_mlp *mlp, const float *x, const float *t, int batch, float lr, float *loss_out,
                              void *stream);

/* Loss and gradients (packed order, host) of (x, t) without updating anything. */
sas_status sas_mlp_grads(sas_mlp *mlp, const float *x, const float *t, int batch, float *grads, float *loss_out,
                         void *stream);

/* Intermediate tensors of the network's last passes, for tests and inspection: the forward pass
 * of the last sas_mlp_forward, sas_mlp_grads or sas_mlp_train_step call (X .. Y) and the backward
 * pass of the last sas_mlp_grads or sas_mlp_train_step call (DY .. DZ1B).  Rows [0, batch) of
 * tensor `which` go to out [batch][width] (float32; bfloat16 tensors are widened exactly; host or
 * device memory); width is n_in for X, n_out for Y, DY and DYB, n_hidden otherwise, and is stored
 * to *width_out if that is not NULL.  batch must be in [1, max_batch]; rows beyond the batch of the
 * pass that wrote the tensor hold stale values.  Synchronizes the device.
 *   XB   bfloat16(x)                           Z1   XB W1b^T + b1 (FP32)   A1B  bfloat16(GELU(Z1))
 *   Z2   A1B W2b^T + b2                        A2B  bfloat16(GELU(Z2))     Y    A2B W3b^T + b3
 *   DY   2 (Y - t) / (batch n_out)             DYB  bfloat16(DY)           DA2  DYB W3b
 *   DZ2  DA2 GELU'(Z2)    DZ2B bfloat16(DZ2)   DA1  DZ2B W2b               DZ1  DA1 GELU'(Z1)
 *   DZ1B bfloat16(DZ1)
 * (W1b, W2b, W3b: the bfloat16 copies of the master weights.) */
enum {
    SAS_MLP_BUF_XB = 0, SAS_MLP_BUF_Z1 = 1, SAS_MLP_BUF_A1B = 2, SAS_MLP_BUF_Z2 = 3, SAS_MLP_BUF_A2B = 4,
    SAS_MLP_BUF_Y = 5, SAS_MLP_BUF_DY = 6, SAS_MLP_BUF_DYB = 7, SAS_MLP_BUF_DA2 = 8, SAS_MLP_BUF_DZ2 = 9,
    SAS_MLP_BUF_DZ2B = 10, SAS_MLP_BUF_DA1 = 11, SAS_MLP_BUF_DZ1 = 12, SAS_MLP_BUF_DZ1B = 13,
    SAS_MLP_BUF_COUNT = 14
};
sas_status sas_mlp_read_buffer(sas_mlp *mlp, int which, int batch, float *out, int *width_out);

/* C[M][N] = A[M][K] B[N][K]^T (+ bias[N]): bfloat16 A and B (device, K contiguous, 16-byte aligned,
 * K % 16 == 0, lda and ldb multiples of 8), float32 C (device), FP32 accumulation on the tcgen05
 * tensor cores (TMA-fed shared-memory stages, accumulator in tensor memory).  Asynchronous on the
 * stream; a failed internal wait is reported by the next synchronizing sas_mlp_* call. */
sas_status sas_gemm_bf16(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias,
                         float *C, int ldc, void *stream);

/*
 * Screening of a conformer ensemble (the high-throughput setting of Section I; not part of the
 * paper's method): chi2_c = sum_q w_q (P_cq - target_q)^2 for n_conf predicted profiles
 *   P_cq = base_cq * exp(z_cq stdv_q + mean_q),
 * z a standardized log-profile (float32, row stride ld) and base a profile (double, row stride
 * ld_base) that it multiplies; either may be NULL (factor 1), not both; mean and stdv are needed
 * with z.  chi2 goes to chi2_all [n_conf]; then the indices of the k smallest chi2 in increasing
 * order (equal values by index, NaN last) to top_idx [k] and their chi2 to top_chi2 [k] (may be
 * NULL).  Every buffer is device memory; chi2_all is required.  Limits: 1 <= n_conf <= 8192 (one
 * CTA sorts them in shared memory), 1 <= k <= n_conf, ld and ld_base >= n_q.  Asynchronous on the
 * stream.
 */
sas_status sas_screen_select(int n_conf, int n_q, const float *z, int ld, const double *mean, const double *stdv,
                             const double *base, int ld_base, const double *target, const double *weights, int k,
                             int32_t *top_idx, double *top_chi2, double *chi2_all, void *stream);

/* dst[r] = src[idx[r]] for r < n_idx, rows of row_bytes bytes (device src, idx, dst; idx values
 * must address rows of src).  Packs selected conformers for the exact kernels. */
sas_status sas_gather_rows(const void *src, int64_t row_bytes, const int32_t *idx, int64_t n_idx, void *dst,
                           void *stream);

/* ---- guard bands (a debugging aid; the paper has no counterpart) --------------------------
 * With guard bands on, every device buffer the library allocates from then on (context and network
 * workspace, microbenchmark scratch) lies between two 256-byte bands of a fixed byte pattern, the
 * second starting at the buffer's exact end, so that a kernel writing past either end of a buffer
 * leaves a trace that sas_guard_check finds.  They stand in for a device memory checker in tests and
 * debugging.  Buffers allocated while the bands are off stay plain; a guarded buffer keeps its bands
 * until freed.  Setting up the bands waits for the device: do not allocate (first calls, larger
 * sizes) under stream capture while they are on.  The environment variable SAS_GUARD_BANDS=1 turns
 * them on when the library is loaded.  The fixed array of sas_profile_static has none.
 *
 * sas_guard_bands: enable 1 (on) or 0 (off) for later allocations.  Errors: INVALID_ARG.
 * sas_guard_check: waits for every device holding a guarded buffer, then compares every band of
 *   every live guarded buffer with the pattern; *n_checked_out (may be NULL) gets the number of
 *   buffers checked.  Errors: CORRUPT (a band changed; the message names the first buffer and side),
 *   CUDA.  Thread-safe.
 * sas_guard_list: the live guarded buffers' device addresses and sizes, up to cap of them, into
 *   ptr_out [cap] and bytes_out [cap] (host); *n_out gets their total count.  Errors: INVALID_ARG.
 */
sas_status sas_guard_bands(int enable);
sas_status sas_guard_check(int64_t *n_checked_out);
sas_status sas_guard_list(int64_t cap, void **ptr_out, int64_t *bytes_out, int64_t *n_out);

/* Thread-local message of the calling thread's last failure ("" if none). */
const char *sas_last_error(void);

/* Library version string. */
const char *sas_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SAS_H */

// Internal interface of the C-ABI implementation (sas_api.cu and the entry points split from it:
// api_hybrid.cu, api_atomic.cu): the context, device buffers, status helpers and the shared steps
// of a profile call.  Not installed.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "sas_internal.h"

namespace sas {
namespace api {

// Set the calling thread's error message (printf format) and return st.
sas_status fail(sas_status st, const char *fmt, ...);

#define CUDA_TRY(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            cudaGetLastError();                                                              \
            return fail(SAS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));              \
        }                                                                                    \
    } while (0)

// Test hook: SAS_TEST_FAIL_ALLOC=k makes the k-th device allocation (1-based) fail.
extern long g_alloc_count;
long alloc_fail_at();

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release()
    {
        if (p) dev_free(p);
        p = nullptr;
        cap = 0;
    }
    // Grow to at least `bytes`.  Returns false (and leaves the buffer empty) on failure.
    bool ensure(size_t bytes)
    {
        if (bytes <= cap && p) return true;
        release();
        ++g_alloc_count;
        if (alloc_fail_at() > 0 && g_alloc_count == alloc_fail_at()) return false;
        if (dev_malloc(&p, bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return false;
        }
        cap = bytes;
        return true;
    }
    template <class T>
    T *as() const
    {
        return static_cast<T *>(p);
    }
};

#define ALLOC_TRY(buf, bytes)                                                                \
    do {                                                                                     \
        if (!(buf).ensure(bytes))                                                            \
            return fail(SAS_ERR_ALLOC, "device allocation of %zu bytes failed", (size_t)(bytes)); \
    } while (0)

}  // namespace api
}  // namespace sas

// The opaque context of sas.h (global scope, as declared there).
struct sas_ctx {
    int n_types = 0, n_q = 0;
    unsigned flags = 0;
    std::vector<double> coef, q;
    sas::QChunks qc{};
    int sms = 1;
    int64_t opt_jmax = 0;
    int opt_reseed = -1;   // -1: automatic (see reseed_for)
    int opt_step = 2;
    int opt_variant = 0;
    int opt_grid = 0;
    int opt_shard_rank = 0, opt_shard_world = 1;   // this call computes shard rank of world
    int opt_method = 0;                             // 0 direct sum, 1 hybrid by qD and N, 2 quadrature
    int opt_adjoint = 0;
    int opt_coef = 0;                               // 0 automatic, 1 one form, 2 both forms (SAS_OPT_COEF)                            // 0 tabulated radial weight (if it fits), 1 q recurrence
    double diam = 0.0;                              // bound on the diameter of the last call's conformers
    int pad = sas::kTile, tile_used = sas::kTile;             // type-group padding and I-tile of the last packing
    int64_t opt_timeout_ms = 600000;
    sas::api::DevBuf coef_d, F, meta, blockcounts, blockoffs, centroid, X, slot_of, items, group_items,
        group_off, partial, ticket, S, in_coords, in_types, out_buf, Ibuf, gbuf, chi2buf, H, G, gout, tgt, wts,
        hist, dropped, in_ff, zero_types, FJ, FI, F64t, D2, segbuf, cen, qdirs, qwts, type_off, Apart, Fsub, Itmp, qplan,
        tile_off, tile_ent, adj_pi, adj_pj, Ufix, segfix, Ustage, Sx, Ix, btab, bdiag, bhist, bout, adj_k, adj_wn, adj_tab, adj_ai, sct;
    int sct_n = 0;            // entries of the (sin, cos)(k/64) table in sct
    int btab_bins = 0;        // (n_bins, r_max) of the binned-sum table in btab (0: none)
    float btab_rmax = 0.f;
    int det_ntiles = -1;   // I-tiles per conformer of the current schedule's tile lists (-1: none built)
    int *h_meta = nullptr;   // pinned
    // schedule cache
    std::vector<int64_t> sched_key;
    int n_items = 0, n_groups = 0, jmax_used = 0, jlen_max = 0, max_group = 0;
    int64_t pair_slots = 0;
    int64_t last_batch = 0;
    bool have_partials = false;
    int64_t stats[9] = {0, 0, 0, 0, 0, 0, 0, 0, 128};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // around the last pair-kernel launch
    bool ev_pending = false;
    double4 *h_cen = nullptr;   // pinned: centroid and radius per conformer (quadrature method)
    int64_t h_cen_cap = 0;
    void *h_stage = nullptr;   // pinned staging of host outputs
    size_t h_stage_cap = 0;
};

namespace sas {
namespace api {

struct HostCopies {
    void *dst[4];
    const void *src[4];
    size_t bytes[4];
    int n = 0;
};

bool on_device(const void *p);
sas_status with_sincos_table(sas_ctx *ctx, QChunks &qc, cudaStream_t s);
int reseed_for(int opt, int64_t n_atoms, int n_q_chunk, double step_phase_max);
int mixed_variant(int opt);
double step_phase(const sas_ctx *ctx, const QChunks &qc);
// Sets qc.coef_both from the call's step phase (the validation read-back's diameter bound).
void with_coef_form(const sas_ctx *ctx, QChunks &qc);
sas_status wait_stream(sas_ctx *ctx, cudaStream_t s);
sas_status schedule_for(sas_ctx *ctx, int T, int64_t batch, int tile, int n_chunks, int64_t jmax_cap, cudaStream_t s);
sas_status prepare(sas_ctx *ctx, const void *coords, int coords_f64, const int32_t *types, int64_t n,
                   int64_t batch, bool out_f64, bool center, int tile, int n_chunks, int64_t jmax_cap,
                   cudaStream_t s, int &launches, int T, const double *ff_check = nullptr, int64_t ff_count = 0);
sas_status zero_out(void *out, size_t bytes, cudaStream_t s);
sas_status reduce_items(sas_ctx *ctx, const QChunks &qc, cudaStream_t s);
sas_status out_copy(HostCopies &hc, void *dst, const void *src, size_t bytes, cudaStream_t s);
sas_status finish_copies(sas_ctx *ctx, HostCopies &hc, cudaStream_t s);
sas_status stage_in(DevBuf &buf, const void *src, size_t bytes, cudaStream_t s, const void *&dev);
// I(q) on a prefix of the grid by the orientation average and on the rest by the direct sum
// (SAS_OPT_METHOD 1 or 2; api_hybrid.cu).
sas_status forward_hybrid(sas_ctx *ctx, const void *coords, int coords_type, const int32_t *types, int64_t n,
                          int64_t batch, double *I_dev, int64_t jmax_cap, cudaStream_t s, int &launches);

}  // namespace api
}  // namespace sas

// sas_profile_atomic: the Debye sum with a form factor per atom and q (Section I-A, Eq. 2 without
// types): validation of the table, the tables the pair kernels read, the pair kernel (mixed or
// FP64), the item reduction and the assembly with the FP64 diagonal (atomic.cu, atomic_pairs2.cu).
// sas_profile_vjp_atomic: its vector-Jacobian product (adjoint.cu, k_debye_adjoint_atomic).
#include <algorithm>

#include "api_internal.h"
#include "sas_internal.h"

using namespace sas;
using namespace sas::api;

extern "C" {

sas_status sas_profile_atomic(sas_ctx *ctx, const void *coords, int coords_type, int64_t n_atoms, int64_t batch,
                              const double *ff, double *I_out, void *stream)
{
    sas::NvtxRange nvtx_range("sas_profile_atomic");
    if (!ctx) return fail(SAS_ERR_INVALID_ARG, "null context");
    const int64_t n = n_atoms;
    if (n < 0 || batch < 0) return fail(SAS_ERR_INVALID_ARG, "negative size");
    if (coords_type != SAS_COORDS_F32 && coords_type != SAS_COORDS_F64)
        return fail(SAS_ERR_INVALID_ARG, "coords_type must be SAS_COORDS_F32 or SAS_COORDS_F64");
    if (n > (int64_t)1 << 28) return fail(SAS_ERR_UNSUPPORTED, "more than 2^28 atoms");
    if (batch > 65535) return fail(SAS_ERR_UNSUPPORTED, "more than 65535 conformers");
    if (batch * (n + kTile) > ((int64_t)1 << 31)) return fail(SAS_ERR_UNSUPPORTED, "batch * atoms too large");
    if (batch > 0 && !I_out) return fail(SAS_ERR_INVALID_ARG, "null output");
    if (batch > 0 && n > 0 && (!coords || !ff)) return fail(SAS_ERR_INVALID_ARG, "null input");
    if (ctx->opt_shard_world > 1) return fail(SAS_ERR_UNSUPPORTED, "per-atom form factors run as a single shard");
    ctx->have_partials = false;
    if (batch == 0) return SAS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int Q = ctx->n_q;
    if (n == 0) {
        ctx->stats[0] = ctx->stats[1] = ctx->stats[2] = 0;
        return zero_out(I_out, (size_t)batch * Q * sizeof(double), s);
    }
    const bool fp64 = (ctx->flags & SAS_FP64) != 0;
    // q passes: the context's, or passes of the re-seed interval (a pass restarts the recurrence
    // from exact seeds, so this is the re-seeding of the typed kernels)
    // (re-seeded from the diameter bound below, once the validation read-back has it)
    QChunks qf = ctx->qc;
    int reseed = fp64 ? 0 : reseed_for(ctx->opt_reseed, n, std::min(Q, kQChunk), 0.0);
    if (reseed > 0 && !make_chunks(ctx->q.data(), Q, qf, std::max(2, std::min(reseed, kQChunk))))
        return fail(SAS_ERR_UNSUPPORTED, "the q grid needs more than %d passes at a re-seed interval of %d",
                    kMaxChunks, reseed);
    int launches = 0;
    const void *ffd = nullptr;
    const size_t ffbytes = (size_t)batch * Q * n * sizeof(double);
    sas_status st = stage_in(ctx->in_ff, ff, ffbytes, s, ffd);
    if (st != SAS_OK) return st;
    const double *F = static_cast<const double *>(ffd);
    ALLOC_TRY(ctx->zero_types, (size_t)n * sizeof(int32_t));
    CUDA_TRY(cudaMemsetAsync(ctx->zero_types.p, 0, (size_t)n * sizeof(int32_t), s));
    const int tile = fp64 ? kTile64 : kTile;
    const int64_t jcap = fp64 ? 8192 : atomic_jmax(qf);
    st = prepare(ctx, coords, coords_type == SAS_COORDS_F64, ctx->zero_types.as<int32_t>(), n, batch, fp64,
                 !fp64 && coords_type == SAS_COORDS_F64, tile, qf.n_chunks, jcap, s, launches, 1, F,
                 (int64_t)batch * Q * n);
    if (st != SAS_OK) return st;
    const int64_t npad = ctx->h_meta[2];
    if (!fp64 && reseed == 0 && reseed_for(ctx->opt_reseed, n, std::min(Q, kQChunk), step_phase(ctx, qf)) > 0) {
        // an ill-conditioned phase step: passes of 32 q (exact slots of the 52-q form), rescheduled
        reseed = 32;
        if (!make_chunks(ctx->q.data(), Q, qf, reseed))
            return fail(SAS_ERR_UNSUPPORTED, "the q grid needs more than %d passes at a re-seed interval of %d",
                        kMaxChunks, reseed);
        st = schedule_for(ctx, 1, batch, kTile, qf.n_chunks, atomic_jmax(qf), s);
        if (st != SAS_OK) return st;
    }
    const int nv = atomic_slots(qf);
    if (!fp64) with_coef_form(ctx, qf);
    if (fp64) {
        ALLOC_TRY(ctx->F64t, (size_t)batch * npad * Q * sizeof(double));
        CUDA_TRY(cudaMemsetAsync(ctx->F64t.p, 0, (size_t)batch * npad * Q * sizeof(double), s));
        CUDA_TRY(launch_atomic_table64(F, ctx->slot_of.as<int>(), n, npad, batch, Q, ctx->F64t.as<double>(), s));
    } else {
        const size_t fj = (size_t)batch * qf.n_chunks * (npad / 2) * nv * sizeof(float4);
        const size_t fi = (size_t)batch * qf.n_chunks * nv * npad * sizeof(float2);
        ALLOC_TRY(ctx->FJ, fj);
        ALLOC_TRY(ctx->FI, fi);
        CUDA_TRY(cudaMemsetAsync(ctx->FJ.p, 0, fj, s));
        CUDA_TRY(cudaMemsetAsync(ctx->FI.p, 0, fi, s));
        CUDA_TRY(launch_atomic_tables(F, ctx->slot_of.as<int>(), n, npad, batch, qf, nv, ctx->FJ.as<float4>(),
                                      ctx->FI.as<float2>(), s));
    }
    ALLOC_TRY(ctx->D2, (size_t)batch * Q * sizeof(double2));
    CUDA_TRY(launch_atomic_diag(F, n, batch, Q, ctx->D2.as<double2>(), s));
    ALLOC_TRY(ctx->partial, (size_t)std::max(ctx->n_items, 1) * kQChunk * sizeof(double));
    const int grid_per_sm = ctx->opt_grid > 0 ? ctx->opt_grid : 2;
    CUDA_TRY(cudaEventRecord(ctx->ev0, s));
    if (fp64) {
        const int grid = std::max(1, std::min(ctx->n_items, grid_per_sm * ctx->sms));
        CUDA_TRY(launch_debye_fp64_atomic(ctx->X.as<double4>(), npad, ctx->items.as<Item>(), ctx->n_items, qf,
                                          ctx->F64t.as<double>(), ctx->partial.as<double>(), kQChunk, grid, s));
    } else {
        ALLOC_TRY(ctx->ticket, sizeof(int));
        CUDA_TRY(cudaMemsetAsync(ctx->ticket.p, 0, sizeof(int), s));
        CUDA_TRY(launch_debye_atomic_pairs2(ctx->X.as<float4>(), npad, ctx->items.as<Item>(), ctx->n_items, qf,
                                            ctx->FJ.as<float4>(), ctx->FI.as<float2>(), ctx->partial.as<double>(),
                                            kQChunk, ctx->opt_grid > 0 ? ctx->opt_grid * ctx->sms : 0,
                                            ctx->jmax_used, ctx->ticket.as<int>(), s));
    }
    CUDA_TRY(cudaEventRecord(ctx->ev1, s));
    ctx->ev_pending = true;
    ALLOC_TRY(ctx->S, (size_t)batch * Q * sizeof(double));
    st = reduce_items(ctx, qf, s);
    if (st != SAS_OK) return st;
    const bool host_out = !on_device(I_out);
    double *Id = I_out;
    if (host_out) {
        ALLOC_TRY(ctx->out_buf, (size_t)batch * Q * sizeof(double));
        Id = ctx->out_buf.as<double>();
    }
    CUDA_TRY(launch_assemble_atomic(ctx->S.as<double>(), ctx->D2.as<double2>(), qf, batch, Id, s));
    launches += 5;
    if (host_out) {
        HostCopies hc;
        st = out_copy(hc, I_out, Id, (size_t)batch * Q * sizeof(double), s);
        if (st == SAS_OK) st = finish_copies(ctx, hc, s);
        if (st != SAS_OK) return st;
    }
    ctx->stats[5] = launches;
    return SAS_OK;
}

sas_status sas_profile_vjp_atomic(sas_ctx *ctx, const float *coords, int64_t n_atoms, int64_t batch, const double *ff,
                                  const double *grad_I, float *grad_out, void *stream)
{
    sas::NvtxRange nvtx_range("sas_profile_vjp_atomic");
    if (!ctx) return fail(SAS_ERR_INVALID_ARG, "null context");
    const int64_t n = n_atoms;
    if (n < 0 || batch < 0) return fail(SAS_ERR_INVALID_ARG, "negative size");
    if (n > (int64_t)1 << 28) return fail(SAS_ERR_UNSUPPORTED, "more than 2^28 atoms");
    if (batch > 65535) return fail(SAS_ERR_UNSUPPORTED, "more than 65535 conformers");
    if (batch * (n + kTile) > ((int64_t)1 << 31)) return fail(SAS_ERR_UNSUPPORTED, "batch * atoms too large");
    if (batch > 0 && n > 0 && (!coords || !ff || !grad_I || !grad_out)) return fail(SAS_ERR_INVALID_ARG, "null argument");
    if (ctx->flags & SAS_FP64) return fail(SAS_ERR_UNSUPPORTED, "the adjoint needs a SAS_MIXED context");
    if (ctx->flags & SAS_DETERMINISTIC)
        return fail(SAS_ERR_UNSUPPORTED, "the per-atom adjoint has no deterministic form");
    if (ctx->opt_shard_world > 1) return fail(SAS_ERR_UNSUPPORTED, "per-atom form factors run as a single shard");
    ctx->have_partials = false;
    if (batch == 0 || n == 0) return SAS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int Q = ctx->n_q;
    // passes of at most 2 * slots q values (their weights of a 128-atom tile fit shared memory)
    QChunks qf{};
    if (!make_chunks(ctx->q.data(), Q, qf, 2 * adjoint_atomic_slots()))
        return fail(SAS_ERR_UNSUPPORTED, "the q grid needs more than %d passes of %d values", kMaxChunks,
                    2 * adjoint_atomic_slots());
    int launches = 0;
    const void *ffd = nullptr, *gId = nullptr;
    sas_status st = stage_in(ctx->in_ff, ff, (size_t)batch * Q * n * sizeof(double), s, ffd);
    if (st != SAS_OK) return st;
    st = stage_in(ctx->gbuf, grad_I, (size_t)batch * Q * sizeof(double), s, gId);
    if (st != SAS_OK) return st;
    const double *F = static_cast<const double *>(ffd);
    ALLOC_TRY(ctx->zero_types, (size_t)n * sizeof(int32_t));
    CUDA_TRY(cudaMemsetAsync(ctx->zero_types.p, 0, (size_t)n * sizeof(int32_t), s));
    st = prepare(ctx, coords, 0, ctx->zero_types.as<int32_t>(), n, batch, false, false, kTile, qf.n_chunks, 1024, s,
                 launches, 1, F, (int64_t)batch * Q * n);
    if (st != SAS_OK) return st;
    const int64_t npad = ctx->h_meta[2];
    with_coef_form(ctx, qf);
    const int nv = adjoint_atomic_slots();
    const size_t fj = (size_t)batch * qf.n_chunks * (npad / 2) * nv * sizeof(float4);
    const size_t fi = (size_t)batch * qf.n_chunks * nv * npad * sizeof(float2);
    const size_t ai = (size_t)batch * qf.n_chunks * nv * npad * sizeof(float4);
    ALLOC_TRY(ctx->FJ, fj);
    ALLOC_TRY(ctx->FI, fi);
    ALLOC_TRY(ctx->adj_ai, ai);
    CUDA_TRY(cudaMemsetAsync(ctx->FJ.p, 0, fj, s));
    CUDA_TRY(cudaMemsetAsync(ctx->FI.p, 0, fi, s));
    CUDA_TRY(cudaMemsetAsync(ctx->adj_ai.p, 0, ai, s));
    CUDA_TRY(launch_atomic_tables(F, ctx->slot_of.as<int>(), n, npad, batch, qf, nv, ctx->FJ.as<float4>(),
                                  ctx->FI.as<float2>(), s));
    CUDA_TRY(launch_atomic_adj_table(F, static_cast<const double *>(gId), ctx->slot_of.as<int>(), n, npad, batch, qf,
                                     ctx->adj_ai.as<float4>(), s));
    ALLOC_TRY(ctx->G, (size_t)batch * npad * 3 * sizeof(double));
    CUDA_TRY(cudaMemsetAsync(ctx->G.p, 0, (size_t)batch * npad * 3 * sizeof(double), s));
    ALLOC_TRY(ctx->ticket, sizeof(int));
    CUDA_TRY(cudaMemsetAsync(ctx->ticket.p, 0, sizeof(int), s));
    CUDA_TRY(launch_debye_adjoint_atomic(ctx->X.as<float4>(), npad, ctx->items.as<Item>(), ctx->n_items, qf,
                                         ctx->adj_ai.as<float4>(), ctx->FJ.as<float4>(), ctx->G.as<double>(),
                                         ctx->jlen_max, ctx->ticket.as<int>(), s));
    float *gd = grad_out;
    const bool h = !on_device(grad_out);
    if (h) {
        ALLOC_TRY(ctx->gout, (size_t)batch * n * 3 * sizeof(float));
        gd = ctx->gout.as<float>();
    }
    CUDA_TRY(launch_unpermute(ctx->G.as<double>(), ctx->slot_of.as<int>(), n, npad, batch, gd, s));
    launches += 4;
    ctx->stats[5] = launches;
    HostCopies hc;
    if (h && (st = out_copy(hc, grad_out, gd, (size_t)batch * n * 3 * sizeof(float), s)) != SAS_OK) return st;
    return finish_copies(ctx, hc, s);
}

}  // extern "C"

// The hybrid of the direct sum and the orientation average of Eq. 1 (SAS_OPT_METHOD 1 and 2):
// the split of the q grid by a cost model, the quadrature plan, and the launch of both methods.
// (The paper's Discussion: the choice between an approximate method at low q and the direct sum at
// high q is to be made automatically from qD and N; quadrature.cu has the kernels.)
#include <algorithm>
#include <cmath>
#include <vector>

#include "api_internal.h"
#include "sas_internal.h"

namespace sas {
namespace api {

namespace {

// Cost model of the hybrid split: a pair costs 2 NV + kDirectSetup units per pass of the direct
// kernel (NV the float2 slots it computes, fitted to the pass or its block capacity; the set-up
// from the 30,000-atom rod at 101 q against the 50,000-atom globule at 201 q: 9.0 and 13.0 ps per
// pair), a (direction, atom) pair of the quadrature kQuadStepCost units per q of its 32-value
// pass (2.5e13 direct units/s against 5.6e12 quadrature steps/s, both measured on GB300).
constexpr double kDirectSetup = 120.0;
constexpr double kQuadStepCost = 4.5;
constexpr double kQuadTol = 1e-10;                  // (2l+1)|j_l(qR)| below this past the degree L
constexpr size_t kQuadAmpBytes = (size_t)4 << 30;   // partial amplitudes held at once

// Directions of the hemisphere rule of degree L (quad_directions).
int quad_dirs_for(int L)
{
    int nt = L + 1;
    nt += nt & 1;
    return (nt / 2) * (2 * L + 1);
}

}  // namespace

// I(q) by the orientation average of Eq. 1 on a prefix of whole 32-q passes of the grid and by the
// direct sum on the rest.  Method 1 (hybrid) takes the prefix of least modelled total cost; method
// 2 takes every q.
sas_status forward_hybrid(sas_ctx *ctx, const void *coords, int coords_type, const int32_t *types, int64_t n,
                          int64_t batch, double *I_dev, int64_t jmax_cap, cudaStream_t s, int &launches)
{
    const int T = ctx->n_types, Q = ctx->n_q, Pn = T * (T + 1) / 2;
    if (ctx->opt_shard_world > 1) return fail(SAS_ERR_UNSUPPORTED, "the quadrature method runs as a single shard");
    sas_status st = prepare(ctx, coords, coords_type, types, n, batch, false, coords_type == SAS_COORDS_F64, kTile,
                            ctx->qc.n_chunks, jmax_cap, s, launches, T);
    if (st != SAS_OK) return st;
    const int64_t npad = ctx->h_meta[2 * T];
    ctx->have_partials = false;
    // centroid and radius of every conformer
    ALLOC_TRY(ctx->cen, (size_t)batch * sizeof(double4));
    CUDA_TRY(launch_packed_geometry(ctx->X.as<float4>(), npad, batch, ctx->cen.as<double4>(), s));
    launches += 2;
    if (ctx->h_cen_cap < batch) {
        if (ctx->h_cen) cudaFreeHost(ctx->h_cen);
        ctx->h_cen = nullptr;
        ctx->h_cen_cap = 0;
        if (cudaMallocHost((void **)&ctx->h_cen, (size_t)batch * sizeof(double4)) != cudaSuccess) {
            cudaGetLastError();
            ctx->h_cen = nullptr;
            return fail(SAS_ERR_ALLOC, "pinned host allocation failed");
        }
        ctx->h_cen_cap = batch;
    }
    CUDA_TRY(cudaMemcpyAsync(ctx->h_cen, ctx->cen.p, (size_t)batch * sizeof(double4), cudaMemcpyDeviceToHost, s));
    st = wait_stream(ctx, s);
    if (st != SAS_OK) return st;
    double R = 0.0;
    for (int64_t b = 0; b < batch; ++b) R = std::max(R, ctx->h_cen[b].w);
    // the split: the quadrature on whole 32-value passes from q[0], the direct sum on the rest,
    // at the least modelled cost
    int k_split = 0;
    if (ctx->opt_method == 2) {
        k_split = Q;
    } else {
        const double pairs = 0.5 * (double)n * (double)(n - 1);
        auto direct_cost = [&](int Qd) {
            double c = 0.0;
            for (int b = 0; b < Qd; b += kQChunk) {
                const int len = std::min(kQChunk, Qd - b), nb = mixed_blocks_for(len), nv = (len + 1) / 2;
                c += pairs * (2.0 * ((2 * nb - nv <= 3) ? nv : 2 * nb) + kDirectSetup);
            }
            return c;
        };
        double best = direct_cost(Q), quad = 0.0;
        for (int s0 = 0; s0 < Q; s0 += kQuadChunk) {
            const int e = std::min(Q, s0 + kQuadChunk);
            quad += kQuadStepCost * (double)n * kQuadChunk * quad_dirs_for(quad_degree(ctx->q[e - 1] * R, kQuadTol));
            if (quad > best) break;
            const double total = quad + direct_cost(Q - e);
            if (total < best) {
                best = total;
                k_split = e;
            }
        }
    }
    int64_t n_dirs = 0;
    CUDA_TRY(cudaEventRecord(ctx->ev0, s));
    if (k_split > 0) {   // quadrature on q[0, k_split)
        QChunks qq{};
        if (!make_chunks(ctx->q.data(), k_split, qq, kQuadChunk))
            return fail(SAS_ERR_UNSUPPORTED, "the quadrature range needs more than %d passes", kMaxChunks);
        QuadPlan pl{};
        std::vector<float4> dirs, d;
        std::vector<double> wts, w;
        int ctas = 0;
        int64_t amp = 0;
        for (int c = 0; c < qq.n_chunks; ++c) {
            const double qmax = ctx->q[qq.q_begin[c] + qq.q_len[c] - 1];
            quad_directions(quad_degree(qmax * R, kQuadTol), d, w);
            const int M = (int)d.size();
            const int dblk = (M + quad_threads_per_cta() - 1) / quad_threads_per_cta();
            const int64_t tiles = npad / 256 + 1;
            int nseg = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (3 * ctx->sms + dblk * batch - 1) / (dblk * batch)));
            const int64_t seg_len = ((npad + nseg - 1) / nseg + 255) / 256 * 256;
            nseg = (int)((npad + seg_len - 1) / seg_len);
            pl.q_begin[c] = qq.q_begin[c];
            pl.q_len[c] = qq.q_len[c];
            pl.qs_hi[c] = qq.qs_hi[c];
            pl.qs_lo[c] = qq.qs_lo[c];
            pl.dq_hi[c] = qq.dq_hi[c];
            pl.dq_lo[c] = qq.dq_lo[c];
            pl.dir_off[c] = (int)dirs.size();
            pl.n_dir[c] = M;
            pl.n_seg[c] = nseg;
            pl.seg_len[c] = (int)seg_len;
            pl.cta_off[c] = ctas;
            pl.amp_off[c] = amp;
            ctas += dblk * nseg;
            amp += (int64_t)nseg * kQuadChunk * M;
            dirs.insert(dirs.end(), d.begin(), d.end());
            wts.insert(wts.end(), w.begin(), w.end());
        }
        pl.n_chunks = qq.n_chunks;
        pl.cta_off[qq.n_chunks] = ctas;
        pl.amp_stride = amp;
        n_dirs = (int64_t)dirs.size();
        std::vector<int> toff(T + 1, 0);
        for (int t = 0; t < T; ++t) toff[t + 1] = toff[t] + (ctx->h_meta[t] + kTile - 1) / kTile * kTile;
        ALLOC_TRY(ctx->qdirs, dirs.size() * sizeof(float4));
        ALLOC_TRY(ctx->qwts, wts.size() * sizeof(double));
        ALLOC_TRY(ctx->type_off, (T + 1) * sizeof(int));
        ALLOC_TRY(ctx->qplan, sizeof(QuadPlan));
        CUDA_TRY(cudaMemcpyAsync(ctx->qplan.p, &pl, sizeof(QuadPlan), cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(ctx->qdirs.p, dirs.data(), dirs.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(ctx->qwts.p, wts.data(), wts.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(ctx->type_off.p, toff.data(), (T + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
        const int64_t group = std::max<int64_t>(1, std::min<int64_t>(batch, (int64_t)(kQuadAmpBytes / (amp * sizeof(double2)))));
        ALLOC_TRY(ctx->Apart, (size_t)group * amp * sizeof(double2));
        for (int64_t b0 = 0; b0 < batch; b0 += group) {
            const int64_t nb = std::min(group, batch - b0);
            CUDA_TRY(launch_quad(ctx->X.as<float4>() + b0 * npad, npad, nb, ctx->type_off.as<int>(), T,
                                 ctx->cen.as<double4>() + b0, ctx->F.as<double>(), Q, pl, ctx->qplan.as<QuadPlan>(),
                                 ctx->qdirs.as<float4>(),
                                 ctx->qwts.as<double>(), ctx->Apart.as<double2>(), I_dev + b0 * Q, s));
            launches += 2;
        }
        // (copies from pageable host memory have read their source when cudaMemcpyAsync returns)
    }
    if (k_split < Q) {   // the direct sum on q[k_split, Q)
        const int Qd = Q - k_split;
        QChunks qd{};
        if (!make_chunks(ctx->q.data() + k_split, Qd, qd))
            return fail(SAS_ERR_UNSUPPORTED, "the direct range needs more than %d passes", kMaxChunks);
        st = schedule_for(ctx, T, batch, kTile, qd.n_chunks, jmax_cap, s);
        if (st != SAS_OK) return st;
        ALLOC_TRY(ctx->Fsub, (size_t)T * Qd * sizeof(double));
        CUDA_TRY(launch_form_factors(ctx->coef_d.as<double>(), T, qd, ctx->Fsub.as<double>(), s));
        ALLOC_TRY(ctx->partial, (size_t)std::max(ctx->n_items, 1) * kQChunk * sizeof(double));
        ALLOC_TRY(ctx->ticket, sizeof(int));
        CUDA_TRY(cudaMemsetAsync(ctx->ticket.p, 0, sizeof(int), s));
        st = with_sincos_table(ctx, qd, s);
        if (st != SAS_OK) return st;
        CUDA_TRY(launch_debye_mixed(ctx->X.as<float4>(), npad, ctx->items.as<Item>(), ctx->n_items, qd, ctx->opt_step,
                                    reseed_for(ctx->opt_reseed, n, std::min(Qd, kQChunk), step_phase(ctx, qd)),
                                    mixed_variant(ctx->opt_variant), ctx->partial.as<double>(),
                                    kQChunk, ctx->opt_grid > 0 ? ctx->opt_grid * ctx->sms : 0, ctx->jmax_used,
                                    ctx->ticket.as<int>(), s));
        ALLOC_TRY(ctx->S, (size_t)batch * Pn * Qd * sizeof(double));
        st = reduce_items(ctx, qd, s);
        if (st != SAS_OK) return st;
        ALLOC_TRY(ctx->Itmp, (size_t)batch * Qd * sizeof(double));
        CUDA_TRY(launch_assemble(ctx->S.as<double>(), ctx->Fsub.as<double>(), ctx->meta.as<int>(), T, batch, qd, 1,
                                 ctx->Itmp.as<double>(), s));
        CUDA_TRY(cudaMemcpy2DAsync(I_dev + k_split, (size_t)Q * sizeof(double), ctx->Itmp.p, (size_t)Qd * sizeof(double),
                                   (size_t)Qd * sizeof(double), (size_t)batch, cudaMemcpyDeviceToDevice, s));
        launches += 4;
    }
    CUDA_TRY(cudaEventRecord(ctx->ev1, s));
    ctx->ev_pending = true;
    ctx->stats[6] = k_split;
    ctx->stats[7] = n_dirs;
    ctx->last_batch = batch;
    return SAS_OK;
}

}  // namespace api
}  // namespace sas

// The C ABI (include/sas.h): argument checks, host/device staging, the work
// schedule, and the launch sequence of one profile call:
//
//   count types + validate -> scan -> (read back counts) -> schedule ->
//   pack -> pair kernel (mixed or FP64) -> fixed-order item reduction ->
//   assembly of I(q) with the form factors.
//
// The schedule follows the paper's block scheme (Section II, Fig. 2): atoms
// are split into blocks (tiles) and every block is paired with the blocks
// after it, so only j > i is computed.  When there are fewer tiles than the
// GPU has workers, the paper splits the inner loop of a worker among p
// workers; here the J-range of a tile is cut into pieces of at most JMAX
// atoms, JMAX chosen so that every SM gets several items.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "api_internal.h"
#include "sas_internal.h"

using namespace sas;
using namespace sas::api;

namespace sas {
namespace api {

thread_local std::string g_err;

sas_status fail(sas_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

}  // namespace api
}  // namespace sas

namespace sas {
sas_status set_error(sas_status st, const char *msg)
{
    g_err = msg;
    return st;
}

// Runs of uniform spacing: a run starting at s extends while every q_k stays within tol of the
// line through its end points; each run is then cut into passes of at most kQChunk values.
bool make_chunks(const double *q, int n_q, QChunks &qc, int max_len)
{
    double qmax = 0.0;
    for (int k = 0; k < n_q; ++k) qmax = std::max(qmax, std::fabs(q[k]));
    const double tol = 1e-9 * std::max(qmax, 1e-300);
    qc = QChunks{};
    qc.n_q = n_q;
    int nc = 0;
    int s = 0;
    while (s < n_q) {
        int e = std::min(s + 2, n_q);   // run [s, e): one or two points always form a run
        while (e < n_q) {
            const double step = (q[e] - q[s]) / (double)(e - s);
            bool ok = true;
            for (int k = s + 1; k < e && ok; ++k) ok = std::fabs(q[k] - (q[s] + (k - s) * step)) <= tol;
            if (!ok) break;
            ++e;
        }
        const double step = e - s > 1 ? (q[e - 1] - q[s]) / (double)(e - s - 1) : 0.0;
        for (int b = s; b < e; b += max_len) {
            if (nc == kMaxChunks) return false;
            const double qs = q[s] + (b - s) * step;
            qc.q_begin[nc] = b;
            qc.q_len[nc] = std::min(max_len, e - b);
            qc.qsd[nc] = qs;
            qc.dqd[nc] = step;
            qc.qs_hi[nc] = (float)qs;
            qc.qs_lo[nc] = (float)(qs - (double)qc.qs_hi[nc]);
            qc.dq_hi[nc] = (float)step;
            qc.dq_lo[nc] = (float)(step - (double)qc.dq_hi[nc]);
            qc.start_is_step[nc] = (step > 0.0 && std::fabs(qs - step) <= 1e-12 * qs) ? 1 : 0;
            ++nc;
        }
        s = e;
    }
    qc.n_chunks = nc;
    return true;
}
// Re-seed interval of the mixed kernel.  The drift of the FP32 recurrence for near pairs is
// random across pairs, so its effect on I(q) shrinks as the molecule grows, and it grows with the
// number of recurrence steps, i.e. with the q values of a chunk.  Measured with the 2-step
// recurrence and no re-seeding (max over q and six seeded globules each): 201 q (0..1/A):
// 2.5e-5 at 600 atoms, 1.0e-5 at 3,000, 6.4e-6 at 8,000, 2.7e-6 at 50,000; 101 q (0..0.5/A):
// 8.1e-6 at 600, 4.1e-6 at 1,000, 2.8e-6 at 2,000, 1.2e-6 at 5,000 atoms.  Automatic: no
// re-seeding from 8,192 atoms, or from 2,000 atoms when a chunk holds at most 104 q values;
// otherwise every 32 q values (at most 3.5e-6 in the same study).
// The recurrence with coefficient 2cos(M t), t = dq r, is ill-conditioned where M t nears pi
// (its error grows like 1/sin(M t) per step, and with the number of steps): the 200,000-atom
// globule (diameter 350 A, 201 q on 0..1/A, M t up to 3.5) reached 6.2e-5 at q = 0.975 without
// re-seeding and 1.3e-6 with a re-seed every 64 q; with passes of at most 101 q the same globule
// (0..0.5/A), the 30,000-atom rod and the 200,000-bead chain (M t far beyond pi) stayed at
// <= 2.1e-6 without, and so did the 150,000-atom globule at 201 q (318 A).  So once M dq D can
// reach 0.9 pi (D bounded by twice the largest distance from the first atom), passes longer
// than 128 q are re-seeded every 64 q.
int reseed_auto(int64_t n_atoms, int n_q_chunk, double step_phase_max)
{
    const bool ill = step_phase_max >= 0.9 * 3.14159265358979323846 && n_q_chunk > 128;
    if (n_atoms >= 8192) return ill ? 64 : 0;
    if (n_q_chunk <= 104 && n_atoms >= 2000) return ill ? 64 : 0;
    return 32;
}

}  // namespace sas

namespace sas {
namespace api {


// Test hook: SAS_TEST_FAIL_ALLOC=k makes the k-th device allocation (1-based) fail.
long g_alloc_count = 0;
long alloc_fail_at()
{
    static long v = [] {
        const char *e = std::getenv("SAS_TEST_FAIL_ALLOC");
        return e ? std::atol(e) : 0L;
    }();
    return v;
}


bool on_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The table of (sin, cos)(k/64) (sincos_tab) covering every pair's step phase dq r of a call: r is
// at most the diameter bound of the call's conformers (ctx->diam, set by prepare), so 64 dq diam + 3
// entries suffice (the 3 cover the float32 rounding of r and t).  Built in FP64 on the host once per
// context and rebuilt larger when a call needs more.  Beyond kSincosTabMax = 2,048 entries (t above
// 32 rad, a molecule thousands of Å long) the kernels keep the polynomial sincos: the two-pair
// kernel copies the table into shared memory beside its J-range, 32 KB at most.
constexpr int kSincosTabMax = kStagedSincosTab;

sas_status with_sincos_table(sas_ctx *ctx, QChunks &qc, cudaStream_t s)
{
    qc.sct = nullptr;
    qc.sct_n = 0;
    with_coef_form(ctx, qc);
    double dq = 0.0;
    for (int c = 0; c < qc.n_chunks; ++c) dq = std::max(dq, qc.dqd[c]);
    const double tmax = dq * ctx->diam;
    if (!(tmax >= 0.0) || tmax * 64.0 > kSincosTabMax - 3) return SAS_OK;
    const int n = (int)std::floor(tmax * 64.0 * (1.0 + 1e-6)) + 3;
    if (ctx->sct_n < n) {
        const int m = std::max(n, 1024);
        std::vector<float4> h((size_t)m);
        for (int k = 0; k < m; ++k) {
            const double x = k / 64.0, sv = std::sin(x), cv = std::cos(x);
            const float sh = (float)sv, ch = (float)cv;
            h[(size_t)k] = make_float4(sh, ch, (float)(sv - (double)sh), (float)(cv - (double)ch));
        }
        ctx->sct_n = 0;
        ALLOC_TRY(ctx->sct, (size_t)m * sizeof(float4));
        // pageable source: the call returns once the data are staged, so h may go out of scope
        CUDA_TRY(cudaMemcpyAsync(ctx->sct.p, h.data(), (size_t)m * sizeof(float4), cudaMemcpyHostToDevice, s));
        ctx->sct_n = m;
    }
    qc.sct = ctx->sct.as<float4>();
    qc.sct_n = n;   // the entries this call can index (the allocation may hold more)
    return SAS_OK;
}

int reseed_for(int opt, int64_t n_atoms, int n_q_chunk, double step_phase_max)
{
    if (opt >= 0) return opt;
    return reseed_auto(n_atoms, n_q_chunk, step_phase_max);
}

// SAS_OPT_VARIANT (0 auto, 1 general, 2 pipelined, 3 sequential, 4 two pairs per step) -> kernel
// variant code.  Auto: two pairs per step, the fastest form for every q capacity (measured on the
// 50,000- and 10,000-atom globules, 201 q, and the 30,000-atom rod, 101 q).
int mixed_variant(int opt)
{
    if (opt == 1) return 1;
    if (opt == 2) return 3;
    if (opt == 3) return 4;
    return 5;
}

int pair_index(int a, int b, int T)
{
    if (a > b) std::swap(a, b);
    return a * T - a * (a - 1) / 2 + (b - a);
}

}  // namespace api
}  // namespace sas


namespace sas {
namespace api {

// Largest phase step M dq D of the mixed recurrence over the passes of qc (D from the last
// validation read-back).
double step_phase(const sas_ctx *ctx, const QChunks &qc)
{
    double dq = 0.0;
    for (int c = 0; c < qc.n_chunks; ++c) dq = std::max(dq, std::fabs(qc.dqd[c]));
    return ctx->opt_step * dq * ctx->diam;
}

// The mixed kernels form the recurrence coefficient both ways (QChunks::coef_both) where the
// call's step phase can come near pi.  Measured (GB300, 50 q at spacing 0.02 A^-1 and 100 q at
// 0.01, random-walk globules): 2 - 4 sin^2 t alone reached 5.3e-5 and 2.5e-4 at 100,000 atoms
// (3.9e-5 and 7.1e-5 at 40,000), both forms 3.8e-6 and 8.5e-6; below the threshold (the 201-q
// grids up to 50,000 atoms, step phase <= 2.2) the one form stays within the bound.
void with_coef_form(const sas_ctx *ctx, QChunks &qc)
{
    if (ctx->opt_coef != 0)
        qc.coef_both = ctx->opt_coef == 2 ? 1 : 0;
    else
        qc.coef_both = step_phase(ctx, qc) >= kCoefBothPhase ? 1 : 0;
}

// Wait for the work queued on `s` so far, giving up after the context's time limit.
sas_status wait_stream(sas_ctx *ctx, cudaStream_t s)
{
    cudaEvent_t ev;
    CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, s);
    if (e != cudaSuccess) {
        cudaEventDestroy(ev);
        return fail(SAS_ERR_CUDA, "cudaEventRecord: %s", cudaGetErrorString(e));
    }
    const auto t0 = std::chrono::steady_clock::now();
    for (long spin = 0;; ++spin) {
        e = cudaEventQuery(ev);
        if (e != cudaErrorNotReady) break;
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                            std::chrono::steady_clock::now() - t0)
                            .count();
        if (ms > ctx->opt_timeout_ms) {
            cudaEventDestroy(ev);
            return fail(SAS_ERR_TIMEOUT, "device work did not finish within %lld ms",
                        (long long)ctx->opt_timeout_ms);
        }
        if (spin > 64) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    cudaEventDestroy(ev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SAS_ERR_CUDA, "device work failed: %s", cudaGetErrorString(e));
    }
    return SAS_OK;
}

struct Schedule {
    std::vector<Item> items;        // execution order
    std::vector<int> group_items;   // per group, execution positions in canonical order
    std::vector<int> group_off;     // [n_groups + 1]
    int jmax = 0;
    int jlen_max = 0;   // longest J-range of the items
    int64_t pair_slots = 0;
    // For the deterministic adjoint: per conformer and I-tile of the packed array, the items whose
    // I-tile (entry 2e) or J-range (entry 2e + 1) touches it, in execution order.
    int ntiles = -1;   // -1: not built
    std::vector<int> tile_off, tile_ent;
};

// Items of one conformer-independent layout; `counts` are the real atoms per type.
void build_schedule(const int *counts, int T, int64_t batch, int tile, int pad, int n_chunks, int grid,
                    int64_t jmax_opt, int64_t jmax_cap, int shard_rank, int shard_world, bool tile_lists,
                    Schedule &out)
{
    // Type group t occupies slots [O[t], O[t] + P[t]) of the packed array (its count padded to a
    // multiple of `pad`), its atoms the first counts[t]; an I-tile spans `tile` slots, a J-range
    // ends at E[t], the count rounded up to 4 (the slots past the count hold zero-weight padding).
    std::vector<int64_t> P(T), O(T), E(T);
    int64_t off = 0;
    for (int t = 0; t < T; ++t) {
        P[t] = (counts[t] + pad - 1) / pad * pad;
        O[t] = off;
        E[t] = off + std::min<int64_t>(P[t], (counts[t] + 3) / 4 * 4);
        off += P[t];
    }
    auto n_items_for = [&](int64_t jmax) {
        int64_t c = 0;
        for (int a = 0; a < T; ++a)
            for (int b = a; b < T; ++b) {
                if (P[a] == 0 || P[b] == 0) continue;
                for (int64_t i0 = O[a]; i0 < O[a] + counts[a]; i0 += tile) {
                    const int64_t js = (a == b) ? i0 : O[b], je = E[b];
                    if (je > js) c += (je - js + jmax - 1) / jmax;
                }
            }
        return c * batch * n_chunks;
    };
    int64_t jmax = jmax_opt;
    if (jmax <= 0) {
        const int64_t cands[] = {4096, 2048, 1024, 512, 256, 128};
        jmax = std::min<int64_t>(128, jmax_cap);
        for (int64_t c : cands)
            if (c <= jmax_cap && n_items_for(c) >= 4 * (int64_t)grid) {
                jmax = c;
                break;
            }
    }
    out.jmax = (int)jmax;
    const int Pn = T * (T + 1) / 2;
    std::vector<Item> canon;
    std::vector<int> canon_group;
    out.pair_slots = 0;
    for (int64_t bb = 0; bb < batch; ++bb)
        for (int a = 0; a < T; ++a)
            for (int b = a; b < T; ++b) {
                if (P[a] == 0 || P[b] == 0) continue;
                const int g = (int)(bb * Pn + pair_index(a, b, T));
                for (int64_t i0 = O[a]; i0 < O[a] + counts[a]; i0 += tile) {
                    const int64_t js = (a == b) ? i0 : O[b], je = E[b];
                    for (int64_t j0 = js; j0 < je; j0 += jmax) {
                        const int64_t jl = std::min(jmax, je - j0);
                        for (int ch = 0; ch < n_chunks; ++ch) {
                            Item it;
                            it.batch = (int)bb;
                            it.pair = pair_index(a, b, T);
                            it.i0 = (int)i0;
                            it.j0 = (int)j0;
                            it.jlen = (int)jl;
                            it.chunk = ch;
                            it.diag = (a == b && j0 == i0) ? 1 : 0;
                            it.work = (int)(jl * tile);
                            out.jlen_max = std::max(out.jlen_max, it.jlen);
                            canon.push_back(it);
                            canon_group.push_back(g);
                            out.pair_slots += jl * tile;
                        }
                    }
                }
            }
    if (shard_world > 1) {   // keep this shard's items: contiguous runs of the canonical order, balanced by work
        int64_t total = 0;
        for (const Item &it : canon) total += it.work;
        std::vector<Item> keep;
        std::vector<int> keep_group;
        int64_t before = 0;
        out.pair_slots = 0;
        out.jlen_max = 0;
        for (size_t k = 0; k < canon.size(); ++k) {
            const int64_t mid2 = 2 * before + canon[k].work;   // twice the item's midpoint
            const int owner = (int)std::min<int64_t>(mid2 * shard_world / (2 * std::max<int64_t>(total, 1)),
                                                     shard_world - 1);
            before += canon[k].work;
            if (owner != shard_rank) continue;
            keep.push_back(canon[k]);
            keep_group.push_back(canon_group[k]);
            out.pair_slots += canon[k].work;
            out.jlen_max = std::max(out.jlen_max, canon[k].jlen);
        }
        canon.swap(keep);
        canon_group.swap(keep_group);
    }
    const int n = (int)canon.size();
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return canon[x].work > canon[y].work; });
    std::vector<int> pos(n);
    out.items.resize(n);
    for (int e = 0; e < n; ++e) {
        out.items[e] = canon[order[e]];
        pos[order[e]] = e;
    }
    const int n_groups = (int)(batch * Pn);
    out.group_off.assign(n_groups + 1, 0);
    for (int i = 0; i < n; ++i) out.group_off[canon_group[i] + 1]++;
    for (int g = 0; g < n_groups; ++g) out.group_off[g + 1] += out.group_off[g];
    out.group_items.resize(n);
    std::vector<int> fill(out.group_off.begin(), out.group_off.end() - 1);
    for (int i = 0; i < n; ++i) out.group_items[fill[canon_group[i]]++] = pos[i];
    if (tile_lists && off % tile == 0) {
        const int64_t ntiles = off / tile;
        std::vector<int64_t> cnt(batch * ntiles + 1, 0);
        auto visit = [&](auto &&f) {
            for (int e = 0; e < n; ++e) {
                const Item &it = out.items[e];
                const int64_t base = (int64_t)it.batch * ntiles;
                f(base + it.i0 / tile, 2 * e);
                for (int64_t t = it.j0 / tile; t <= (it.j0 + (int64_t)it.jlen - 1) / tile; ++t) f(base + t, 2 * e + 1);
            }
        };
        visit([&](int64_t l, int) { cnt[l + 1]++; });
        for (size_t l = 1; l < cnt.size(); ++l) cnt[l] += cnt[l - 1];
        if (cnt.back() < (int64_t)INT32_MAX) {
            out.ntiles = (int)ntiles;
            out.tile_off.assign(cnt.begin(), cnt.end());
            out.tile_ent.resize((size_t)cnt.back());
            std::vector<int64_t> at(cnt.begin(), cnt.end() - 1);
            visit([&](int64_t l, int ent) { out.tile_ent[(size_t)at[l]++] = ent; });
        }
    }
}

bool finite_all(const double *v, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// The work list of the packed layout in ctx->h_meta (counts of T types) for `n_chunks` q passes
// (cached while counts, batch, tile and options are unchanged).
sas_status schedule_for(sas_ctx *ctx, int T, int64_t batch, int tile, int n_chunks, int64_t jmax_cap, cudaStream_t s)
{
    const int grid_per_sm = ctx->opt_grid > 0 ? ctx->opt_grid : 2;
    const int grid_cap = grid_per_sm * ctx->sms;
    std::vector<int64_t> key(ctx->h_meta, ctx->h_meta + T);
    key.push_back(batch);
    key.push_back(tile);
    key.push_back(ctx->opt_jmax);
    key.push_back(grid_cap);
    key.push_back(n_chunks);
    key.push_back(jmax_cap);
    key.push_back(ctx->opt_shard_rank);
    key.push_back(ctx->opt_shard_world);
    key.push_back(ctx->pad);
    if (key != ctx->sched_key) {
        Schedule sc;
        const int64_t jm = ctx->opt_jmax > 0 ? std::min(ctx->opt_jmax, jmax_cap) : 0;
        const bool lists = (ctx->flags & SAS_DETERMINISTIC) && tile == kTile;
        build_schedule(ctx->h_meta, T, batch, tile, ctx->pad, n_chunks, grid_cap, jm, jmax_cap, ctx->opt_shard_rank,
                       ctx->opt_shard_world, lists, sc);
        const int ni = (int)sc.items.size();
        const int ng = (int)sc.group_off.size() - 1;
        ctx->sched_key.clear();   // invalid until the upload succeeded
        ALLOC_TRY(ctx->items, (size_t)std::max(ni, 1) * sizeof(Item));
        ALLOC_TRY(ctx->group_items, (size_t)std::max(ni, 1) * sizeof(int));
        ALLOC_TRY(ctx->group_off, (size_t)(ng + 1) * sizeof(int));
        if (ni) {
            CUDA_TRY(cudaMemcpyAsync(ctx->items.p, sc.items.data(), ni * sizeof(Item),
                                     cudaMemcpyHostToDevice, s));
            CUDA_TRY(cudaMemcpyAsync(ctx->group_items.p, sc.group_items.data(), ni * sizeof(int),
                                     cudaMemcpyHostToDevice, s));
        }
        CUDA_TRY(cudaMemcpyAsync(ctx->group_off.p, sc.group_off.data(), (ng + 1) * sizeof(int),
                                 cudaMemcpyHostToDevice, s));
        ctx->det_ntiles = -1;
        if (sc.ntiles >= 0) {
            ALLOC_TRY(ctx->tile_off, sc.tile_off.size() * sizeof(int));
            ALLOC_TRY(ctx->tile_ent, std::max<size_t>(sc.tile_ent.size(), 1) * sizeof(int));
            CUDA_TRY(cudaMemcpyAsync(ctx->tile_off.p, sc.tile_off.data(), sc.tile_off.size() * sizeof(int),
                                     cudaMemcpyHostToDevice, s));
            if (!sc.tile_ent.empty())
                CUDA_TRY(cudaMemcpyAsync(ctx->tile_ent.p, sc.tile_ent.data(), sc.tile_ent.size() * sizeof(int),
                                         cudaMemcpyHostToDevice, s));
            ctx->det_ntiles = sc.ntiles;
        }
        ctx->n_items = ni;
        ctx->n_groups = ng;
        ctx->max_group = 0;
        for (int g = 0; g < ng; ++g) ctx->max_group = std::max(ctx->max_group, sc.group_off[g + 1] - sc.group_off[g]);
        ctx->jmax_used = sc.jmax;
        ctx->jlen_max = sc.jlen_max;
        ctx->pair_slots = sc.pair_slots;
        ctx->sched_key = key;
    }
    ctx->stats[0] = ctx->n_items;
    ctx->stats[1] = ctx->pair_slots;
    return SAS_OK;
}

// Shared front half of every pair computation: stage, validate, count, schedule, pack.
// On success the context holds X (packed), slot_of, meta (counts/offsets) and the item list.
// T: the types of this call (1 for per-atom form factors, whose table ff_check [ff_count] is
// validated with the coordinates).  tile 0: the mixed typed path chooses its I-tile after the
// read-back (see the choice below); otherwise the given tile and groups padded to 128 slots.
sas_status prepare(sas_ctx *ctx, const void *coords, int coords_f64, const int32_t *types, int64_t n,
                   int64_t batch, bool out_f64, bool center, int tile, int n_chunks, int64_t jmax_cap,
                   cudaStream_t s, int &launches, int T, const double *ff_check, int64_t ff_count)
{
    const size_t esz = coords_f64 ? sizeof(double) : sizeof(float);
    const void *cd = coords;
    const int32_t *td = types;
    if (!on_device(coords)) {
        ALLOC_TRY(ctx->in_coords, (size_t)batch * n * 3 * esz);
        CUDA_TRY(cudaMemcpyAsync(ctx->in_coords.p, coords, (size_t)batch * n * 3 * esz,
                                 cudaMemcpyHostToDevice, s));
        cd = ctx->in_coords.p;
    }
    if (!on_device(types)) {
        ALLOC_TRY(ctx->in_types, (size_t)n * sizeof(int32_t));
        CUDA_TRY(cudaMemcpyAsync(ctx->in_types.p, types, (size_t)n * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, s));
        td = ctx->in_types.as<int32_t>();
    }
    const int nblk = (int)((n + kPackThreads - 1) / kPackThreads);
    ALLOC_TRY(ctx->blockcounts, (size_t)nblk * T * sizeof(int));
    ALLOC_TRY(ctx->blockoffs, (size_t)nblk * T * sizeof(int));
    ALLOC_TRY(ctx->meta, (size_t)(2 * T + 3) * sizeof(int));
    CUDA_TRY(cudaMemsetAsync(ctx->meta.p, 0, (size_t)(2 * T + 3) * sizeof(int), s));
    CUDA_TRY(launch_count_types(cd, coords_f64, td, n, batch, T, ctx->blockcounts.as<int>(),
                                ctx->meta.as<int>() + 2 * T + 1,
                                reinterpret_cast<unsigned *>(ctx->meta.as<int>() + 2 * T + 2), s));
    CUDA_TRY(launch_scan_counts(ctx->blockcounts.as<int>(), nblk, T, kTile, ctx->blockoffs.as<int>(),
                                ctx->meta.as<int>(), s));
    launches += 2;
    if (ff_check) {
        CUDA_TRY(launch_check_finite(ff_check, ff_count, ctx->meta.as<int>() + 2 * T + 1, s));
        launches += 1;
    }
    CUDA_TRY(cudaMemcpyAsync(ctx->h_meta, ctx->meta.p, (size_t)(2 * T + 3) * sizeof(int),
                             cudaMemcpyDeviceToHost, s));
    sas_status st = wait_stream(ctx, s);
    if (st != SAS_OK) return st;
    const int err = ctx->h_meta[2 * T + 1];
    if (err & kErrBadType) return fail(SAS_ERR_INVALID_ARG, "atom type outside [0, %d)", T);
    if (err & kErrNonFinite) return fail(SAS_ERR_INVALID_ARG, "non-finite coordinate");
    if (err & kErrNonFiniteFF) return fail(SAS_ERR_INVALID_ARG, "non-finite form factor");
    {
        float r2;
        const unsigned bits = (unsigned)ctx->h_meta[2 * T + 2];
        std::memcpy(&r2, &bits, sizeof r2);
        ctx->diam = 2.0 * std::sqrt((double)r2);
    }
    ctx->pad = kTile;
    if (tile == 0) {
        // Tiles of 64 atoms where the automatic kernel form is the two-pair kernel (no re-seeding,
        // passes of at most 104 q; an explicit SAS_OPT_VARIANT keeps the 128-slot layout, whose
        // variants agree bit for bit; so do sharded and deterministic contexts, whose work items
        // must be those of every shard count) and type groups padded to 128 slots would waste more than 5 %
        // of them (small molecules:
        // 2,000 atoms of 5 types pad to 2,560 slots, against 2,240 in groups of 64).  The scan ran
        // with 128; the group offsets are redone here and written back before the packing.
        tile = kTile;
        int qmax = 0;
        for (int c = 0; c < ctx->qc.n_chunks; ++c) qmax = std::max(qmax, ctx->qc.q_len[c]);
        int64_t p128 = 0, p64 = 0;
        for (int t = 0; t < T; ++t) {
            p128 += ((int64_t)ctx->h_meta[t] + 127) / 128 * 128;
            p64 += ((int64_t)ctx->h_meta[t] + 63) / 64 * 64;
        }
        if (ctx->opt_variant == 0 && ctx->opt_step == 2 && mixed_blocks_for(qmax) <= 26 &&
            reseed_for(ctx->opt_reseed, n, qmax, step_phase(ctx, ctx->qc)) == 0 && ctx->opt_shard_world == 1 &&
            !(ctx->flags & SAS_DETERMINISTIC) && (double)p128 > 1.05 * (double)p64) {
            tile = 64;
            ctx->pad = 64;
            int off = 0;
            for (int t = 0; t < T; ++t) {
                ctx->h_meta[T + t] = off;
                off += (ctx->h_meta[t] + 63) / 64 * 64;
            }
            ctx->h_meta[2 * T] = off;
            CUDA_TRY(cudaMemcpyAsync(ctx->meta.as<int>() + T, ctx->h_meta + T, (size_t)(T + 1) * sizeof(int),
                                     cudaMemcpyHostToDevice, s));
        }
    }
    ctx->tile_used = tile;
    ctx->stats[8] = tile;
    const int64_t npad = ctx->h_meta[2 * T];
    st = schedule_for(ctx, T, batch, tile, n_chunks, jmax_cap, s);
    if (st != SAS_OK) return st;
    // pack
    const size_t xsz = out_f64 ? sizeof(double4) : sizeof(float4);
    ALLOC_TRY(ctx->X, (size_t)batch * npad * xsz);
    ALLOC_TRY(ctx->slot_of, (size_t)n * sizeof(int));
    CUDA_TRY(cudaMemsetAsync(ctx->X.p, 0, (size_t)batch * npad * xsz, s));
    const double *cen = nullptr;
    if (center) {
        ALLOC_TRY(ctx->centroid, (size_t)batch * 3 * sizeof(double));
        CUDA_TRY(launch_centroid(cd, coords_f64, n, batch, ctx->centroid.as<double>(), s));
        cen = ctx->centroid.as<double>();
        launches += 1;
    }
    CUDA_TRY(launch_scatter(cd, coords_f64, td, n, batch, T, ctx->blockoffs.as<int>(),
                            ctx->meta.as<int>(), cen, out_f64 ? 1 : 0, ctx->X.p, npad,
                            ctx->slot_of.as<int>(), s));
    launches += 1;
    ctx->stats[0] = ctx->n_items;
    ctx->stats[1] = ctx->pair_slots;
    ctx->stats[2] = batch * (n * (n - 1) / 2);
    ctx->stats[3] = ctx->n_q;
    return SAS_OK;
}

sas_status check_common(sas_ctx *ctx, const void *coords, const int32_t *types, int64_t n,
                        int64_t batch)
{
    if (!ctx) return fail(SAS_ERR_INVALID_ARG, "null context");
    if (n < 0 || batch < 0) return fail(SAS_ERR_INVALID_ARG, "negative size");
    if (n > (int64_t)1 << 28) return fail(SAS_ERR_UNSUPPORTED, "more than 2^28 atoms");
    if (n > 0 && batch > 0 && (!coords || !types)) return fail(SAS_ERR_INVALID_ARG, "null input");
    if (batch * (n + (int64_t)ctx->n_types * kTile) > ((int64_t)1 << 31))
        return fail(SAS_ERR_UNSUPPORTED, "batch * atoms too large");
    return SAS_OK;
}

sas_status zero_out(void *out, size_t bytes, cudaStream_t s)
{
    if (!bytes) return SAS_OK;
    if (on_device(out)) {
        CUDA_TRY(cudaMemsetAsync(out, 0, bytes, s));
    } else {
        std::memset(out, 0, bytes);
    }
    return SAS_OK;
}

// The items' partials -> S (fixed order; segmented for long groups).
sas_status reduce_items(sas_ctx *ctx, const QChunks &qc, cudaStream_t s)
{
    if (ctx->flags & SAS_DETERMINISTIC) {   // exact sums, kept in Ufix for sas_exact_sums
        const int max_seg = ctx->max_group > kSegItems ? (ctx->max_group + kSegItems - 1) / kSegItems : 1;
        ALLOC_TRY(ctx->segfix, (size_t)ctx->n_groups * max_seg * qc.n_q * sizeof(Fix128));
        ALLOC_TRY(ctx->Ufix, (size_t)ctx->n_groups * qc.n_q * sizeof(Fix128));
        CUDA_TRY(launch_reduce_items_fix(ctx->partial.as<double>(), kQChunk, ctx->items.as<Item>(),
                                         ctx->group_items.as<int>(), ctx->group_off.as<int>(), ctx->n_groups,
                                         ctx->max_group, qc, ctx->segfix.as<Fix128>(), ctx->Ufix.as<Fix128>(),
                                         ctx->S.as<double>(), s));
        return SAS_OK;
    }
    if (ctx->max_group > kSegItems)
        ALLOC_TRY(ctx->segbuf,
                  (size_t)ctx->n_groups * ((ctx->max_group + kSegItems - 1) / kSegItems) * qc.n_q * sizeof(double));
    CUDA_TRY(launch_reduce_items_seg(ctx->partial.as<double>(), kQChunk, ctx->items.as<Item>(),
                                     ctx->group_items.as<int>(), ctx->group_off.as<int>(), ctx->n_groups,
                                     ctx->max_group, qc, ctx->segbuf.as<double>(), ctx->S.as<double>(), s));
    return SAS_OK;
}

// I(q) of `batch` conformers into the device buffer I_dev (all steps on stream s).
sas_status forward(sas_ctx *ctx, const void *coords, int coords_type, const int32_t *types, int64_t n,
                   int64_t batch, double *I_dev, int64_t jmax_cap, cudaStream_t s, int &launches,
                   bool hybrid_ok = false)
{
    const int T = ctx->n_types, Q = ctx->n_q, Pn = T * (T + 1) / 2;
    const bool fp64 = (ctx->flags & SAS_FP64) != 0;
    ctx->stats[6] = ctx->stats[7] = 0;
    if (hybrid_ok && !fp64 && ctx->opt_method != 0)
        return forward_hybrid(ctx, coords, coords_type, types, n, batch, I_dev, jmax_cap, s, launches);
    // plain profile calls may take 64-atom tiles (chosen in prepare); the gradient's adjoint kernel
    // reuses the forward's packing with 128-atom tiles
    const int tile = fp64 ? kTile64 : (hybrid_ok ? 0 : kTile);
    sas_status st = prepare(ctx, coords, coords_type, types, n, batch, fp64,
                            !fp64 && coords_type == SAS_COORDS_F64, tile, ctx->qc.n_chunks, jmax_cap, s,
                            launches, T);
    if (st != SAS_OK) return st;
    const int64_t npad = ctx->h_meta[2 * T];
    ALLOC_TRY(ctx->partial, (size_t)std::max(ctx->n_items, 1) * kQChunk * sizeof(double));
    const int grid_per_sm = ctx->opt_grid > 0 ? ctx->opt_grid : 2;
    const int grid = std::max(1, std::min(ctx->n_items, grid_per_sm * ctx->sms));
    if (!fp64) {
        ALLOC_TRY(ctx->ticket, sizeof(int));
        CUDA_TRY(cudaMemsetAsync(ctx->ticket.p, 0, sizeof(int), s));
    }
    QChunks qk = ctx->qc;   // with the call's sine table for the mixed kernels
    if (!fp64) {
        st = with_sincos_table(ctx, qk, s);
        if (st != SAS_OK) return st;
    }
    CUDA_TRY(cudaEventRecord(ctx->ev0, s));
    if (fp64) {
        CUDA_TRY(launch_debye_fp64(ctx->X.as<double4>(), npad, ctx->items.as<Item>(), ctx->n_items,
                                   ctx->qc, ctx->partial.as<double>(), kQChunk, grid, s));
    } else if (ctx->tile_used != kTile) {   // the two-pair kernel on 64-atom tiles (chosen in prepare)
        CUDA_TRY(launch_debye_mixed_pairs2(ctx->X.as<float4>(), npad, ctx->items.as<Item>(), ctx->n_items, qk,
                                           ctx->partial.as<double>(), kQChunk,
                                           ctx->opt_grid > 0 ? ctx->opt_grid * ctx->sms : 0,
                                           std::min(ctx->jmax_used, ctx->jlen_max + (ctx->jlen_max & 1)),
                                           ctx->ticket.as<int>(), s, ctx->tile_used));
    } else {
        CUDA_TRY(launch_debye_mixed(ctx->X.as<float4>(), npad, ctx->items.as<Item>(), ctx->n_items,
                                    qk, ctx->opt_step,
                                    reseed_for(ctx->opt_reseed, n, std::min(ctx->n_q, kQChunk), step_phase(ctx, ctx->qc)),
                                    mixed_variant(ctx->opt_variant), ctx->partial.as<double>(),
                                    kQChunk, ctx->opt_grid > 0 ? ctx->opt_grid * ctx->sms : 0, ctx->jmax_used,
                                    ctx->ticket.as<int>(), s));
    }
    CUDA_TRY(cudaEventRecord(ctx->ev1, s));
    ctx->ev_pending = true;
    ALLOC_TRY(ctx->S, (size_t)batch * Pn * Q * sizeof(double));
    st = reduce_items(ctx, ctx->qc, s);
    if (st != SAS_OK) return st;
    CUDA_TRY(launch_assemble(ctx->S.as<double>(), ctx->F.as<double>(), ctx->meta.as<int>(), T, batch,
                             ctx->qc, ctx->opt_shard_rank == 0, I_dev, s));
    launches += 3;
    ctx->last_batch = batch;
    ctx->have_partials = true;
    return SAS_OK;
}


// Outputs of one call: device destinations are copied at once on the stream; host destinations
// are staged through pinned memory, so that the wait for them obeys the context's time limit
// (a copy into pageable memory would block inside cudaMemcpyAsync instead).

sas_status out_copy(HostCopies &hc, void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    if (!dst || !bytes || dst == src) return SAS_OK;
    if (on_device(dst)) {
        CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
        return SAS_OK;
    }
    hc.dst[hc.n] = dst;
    hc.src[hc.n] = src;
    hc.bytes[hc.n] = bytes;
    ++hc.n;
    return SAS_OK;
}

sas_status finish_copies(sas_ctx *ctx, HostCopies &hc, cudaStream_t s)
{
    if (hc.n == 0) return SAS_OK;
    size_t total = 0;
    for (int k = 0; k < hc.n; ++k) total += (hc.bytes[k] + 255) / 256 * 256;
    if (ctx->h_stage_cap < total) {
        if (ctx->h_stage) {
            cudaDeviceSynchronize();
            cudaFreeHost(ctx->h_stage);
            ctx->h_stage = nullptr;
            ctx->h_stage_cap = 0;
        }
        if (cudaMallocHost(&ctx->h_stage, total) != cudaSuccess) {
            cudaGetLastError();
            ctx->h_stage = nullptr;
            return fail(SAS_ERR_ALLOC, "pinned allocation of %zu bytes failed", total);
        }
        ctx->h_stage_cap = total;
    }
    size_t off = 0;
    for (int k = 0; k < hc.n; ++k) {
        CUDA_TRY(cudaMemcpyAsync(static_cast<char *>(ctx->h_stage) + off, hc.src[k], hc.bytes[k],
                                 cudaMemcpyDeviceToHost, s));
        off += (hc.bytes[k] + 255) / 256 * 256;
    }
    sas_status st = wait_stream(ctx, s);
    if (st != SAS_OK) return st;
    off = 0;
    for (int k = 0; k < hc.n; ++k) {
        std::memcpy(hc.dst[k], static_cast<const char *>(ctx->h_stage) + off, hc.bytes[k]);
        off += (hc.bytes[k] + 255) / 256 * 256;
    }
    hc.n = 0;
    return SAS_OK;
}

// A device copy of a small caller array (host or device) of `bytes`.
sas_status stage_in(DevBuf &buf, const void *src, size_t bytes, cudaStream_t s, const void *&dev)
{
    if (on_device(src)) {
        dev = src;
        return SAS_OK;
    }
    ALLOC_TRY(buf, bytes);
    CUDA_TRY(cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, s));
    dev = buf.p;
    return SAS_OK;
}

sas_status run_profile(sas_ctx *ctx, const void *coords, int coords_type, const int32_t *types,
                       int64_t n, int64_t batch, double *I_out, cudaStream_t s)
{
    sas_status st = check_common(ctx, coords, types, n, batch);
    if (st != SAS_OK) return st;
    if (coords_type != SAS_COORDS_F32 && coords_type != SAS_COORDS_F64)
        return fail(SAS_ERR_INVALID_ARG, "coords_type must be SAS_COORDS_F32 or SAS_COORDS_F64");
    if (batch > 0 && !I_out) return fail(SAS_ERR_INVALID_ARG, "null output");
    ctx->have_partials = false;
    if (batch == 0) return SAS_OK;
    const int Q = ctx->n_q;
    if (n == 0) {
        ctx->stats[0] = ctx->stats[1] = ctx->stats[2] = 0;
        return zero_out(I_out, (size_t)batch * Q * sizeof(double), s);
    }
    int launches = 0;
    const bool host_out = !on_device(I_out);
    double *Id = I_out;
    if (host_out) {
        ALLOC_TRY(ctx->out_buf, (size_t)batch * Q * sizeof(double));
        Id = ctx->out_buf.as<double>();
    }
    st = forward(ctx, coords, coords_type, types, n, batch, Id, 8192, s, launches, true);
    if (st != SAS_OK) return st;
    if (host_out) {
        HostCopies hc;
        st = out_copy(hc, I_out, Id, (size_t)batch * Q * sizeof(double), s);
        if (st == SAS_OK) st = finish_copies(ctx, hc, s);
        if (st != SAS_OK) return st;
    }
    ctx->stats[5] = launches;
    return SAS_OK;
}

// Shared back half of sas_profile_grad / sas_profile_vjp: g [batch][Q] (device) -> gradient.
// Longest J-range of the adjoint's work items: shorter on a deterministic context, whose kernel keeps
// one copy of the J-range sums per warp in shared memory.
int64_t adjoint_jmax_cap(const sas_ctx *ctx) { return (ctx->flags & SAS_DETERMINISTIC) ? 512 : 2048; }

sas_status adjoint(sas_ctx *ctx, int64_t n, int64_t batch, const double *g_dev, float *grad_out,
                   cudaStream_t s, int &launches, HostCopies &hc)
{
    const int T = ctx->n_types, Q = ctx->n_q, Pn = T * (T + 1) / 2;
    const int64_t npad = ctx->h_meta[2 * T];
    ALLOC_TRY(ctx->H, (size_t)batch * Pn * Q * sizeof(float2));
    CUDA_TRY(launch_adjoint_coef(g_dev, ctx->F.as<double>(), T, batch, ctx->qc, ctx->H.as<float2>(), Q, s));
    ALLOC_TRY(ctx->G, (size_t)batch * npad * 3 * sizeof(double));
    const bool det = (ctx->flags & SAS_DETERMINISTIC) != 0;
    float *PI = nullptr, *PJ = nullptr;
    const int jcap = adjoint_jcap(ctx->jlen_max);
    if (det) {   // per-item totals, then a fixed-order sum per atom
        if (ctx->det_ntiles < 0 || (int64_t)ctx->det_ntiles * kTile != npad)
            return fail(SAS_ERR_UNSUPPORTED, "deterministic adjoint: work list too long for its tile lists");
        ALLOC_TRY(ctx->adj_pi, (size_t)std::max(ctx->n_items, 1) * kTile * 3 * sizeof(float));
        ALLOC_TRY(ctx->adj_pj, (size_t)std::max(ctx->n_items, 1) * jcap * 3 * sizeof(float));
        PI = ctx->adj_pi.as<float>();
        PJ = ctx->adj_pj.as<float>();
    } else {
        CUDA_TRY(cudaMemsetAsync(ctx->G.p, 0, (size_t)batch * npad * 3 * sizeof(double), s));
    }
    ALLOC_TRY(ctx->ticket, sizeof(int));
    CUDA_TRY(cudaMemsetAsync(ctx->ticket.p, 0, sizeof(int), s));
    // The tabulated radial weight W(r) per conformer and type pair (default), on nodes spaced
    // kAdjTabStep / q_max apart up to the validated diameter bound; the q recurrence when the tables
    // would be too large or SAS_OPT_ADJOINT asks for it.
    const double qmax = std::max(ctx->q.back(), 1e-6), step = kAdjTabStep / qmax;
    const double n_int_d = std::ceil(ctx->diam * (1.0 + 1e-5) / step) + 2.0;
    const int64_t rows = batch * Pn;
    const double tab_bytes = (double)Q * (n_int_d + 2) * 8 + (double)rows * (n_int_d + 2) * 8 + (double)rows * n_int_d * 16;
    if (ctx->opt_adjoint == 0 && rows <= 65535 && n_int_d < 1e8 && tab_bytes <= 2e9) {
        const int n_int = (int)n_int_d, n_rows = n_int + 2;
        ALLOC_TRY(ctx->adj_k, (size_t)Q * n_rows * sizeof(double));
        ALLOC_TRY(ctx->adj_wn, (size_t)rows * n_rows * sizeof(double));
        ALLOC_TRY(ctx->adj_tab, (size_t)rows * n_int * sizeof(float4));
        CUDA_TRY(launch_adjoint_kmat(ctx->qc, n_rows, step, ctx->adj_k.as<double>(), s));
        CUDA_TRY(launch_adjoint_wtab(g_dev, ctx->F.as<double>(), T, batch, Q, ctx->adj_k.as<double>(), n_rows,
                                     ctx->adj_wn.as<double>(), ctx->adj_tab.as<float4>(), s));
        CUDA_TRY(launch_debye_adjoint_tab(ctx->X.as<float4>(), npad, ctx->items.as<Item>(), ctx->n_items,
                                          ctx->adj_tab.as<float4>(), n_int, (float)(1.0 / step), Pn,
                                          ctx->G.as<double>(), ctx->jlen_max, ctx->ticket.as<int>(), PI, PJ, s));
        launches += 3;
    } else {
        QChunks qa = ctx->qc;
        with_coef_form(ctx, qa);
        CUDA_TRY(launch_debye_adjoint(ctx->X.as<float4>(), npad, ctx->items.as<Item>(), ctx->n_items, qa,
                                      ctx->H.as<float2>(), Pn, Q, ctx->G.as<double>(), ctx->jlen_max,
                                      ctx->ticket.as<int>(), PI, PJ, s));
    }
    if (det) {
        CUDA_TRY(launch_adjoint_gather(PI, PJ, jcap, ctx->items.as<Item>(), ctx->tile_off.as<int>(),
                                       ctx->tile_ent.as<int>(), ctx->det_ntiles, npad, batch, ctx->G.as<double>(),
                                       s));
        launches += 1;
    }
    float *gd = grad_out;
    const bool h = !on_device(grad_out);
    if (h) {
        ALLOC_TRY(ctx->gout, (size_t)batch * n * 3 * sizeof(float));
        gd = ctx->gout.as<float>();
    }
    CUDA_TRY(launch_unpermute(ctx->G.as<double>(), ctx->slot_of.as<int>(), n, npad, batch, gd, s));
    launches += 3;
    if (h) return out_copy(hc, grad_out, gd, (size_t)batch * n * 3 * sizeof(float), s);
    return SAS_OK;
}

}  // namespace api
}  // namespace sas

extern "C" {

const char *sas_last_error(void) { return g_err.c_str(); }

const char *sas_version(void) { return "sas 0.1 (sm_103a)"; }

sas_status sas_create(int n_types, const double *ff_coef, const double *q, int n_q, unsigned flags,
                      sas_ctx **out)
{
    if (!out) return fail(SAS_ERR_INVALID_ARG, "null output handle");
    if (n_types < 1 || n_types > SAS_MAX_TYPES)
        return fail(SAS_ERR_INVALID_ARG, "n_types must be in [1, %d]", SAS_MAX_TYPES);
    if (n_q < 1 || n_q > SAS_MAX_Q) return fail(SAS_ERR_INVALID_ARG, "n_q must be in [1, %d]", SAS_MAX_Q);
    if (!ff_coef || !q) return fail(SAS_ERR_INVALID_ARG, "null coefficients or q grid");
    if (flags & ~(unsigned)(SAS_FP64 | SAS_DETERMINISTIC)) return fail(SAS_ERR_INVALID_ARG, "unknown flags");
    if (!finite_all(ff_coef, (size_t)9 * n_types)) return fail(SAS_ERR_INVALID_ARG, "non-finite coefficient");
    if (!finite_all(q, (size_t)n_q)) return fail(SAS_ERR_INVALID_ARG, "non-finite q");
    if (q[0] < 0) return fail(SAS_ERR_INVALID_ARG, "negative q");
    for (int k = 1; k < n_q; ++k)
        if (!(q[k] > q[k - 1])) return fail(SAS_ERR_UNSUPPORTED, "q grid must be strictly ascending");
    QChunks qcand{};
    if (!make_chunks(q, n_q, qcand))
        return fail(SAS_ERR_UNSUPPORTED, "q grid needs more than %d uniform runs of at most %d values", kMaxChunks,
                    kQChunk);
    sas_ctx *c = new (std::nothrow) sas_ctx;
    if (!c) return fail(SAS_ERR_ALLOC, "host allocation failed");
    c->n_types = n_types;
    c->n_q = n_q;
    c->flags = flags;
    c->coef.assign(ff_coef, ff_coef + 9 * n_types);
    c->q.assign(q, q + n_q);
    c->qc = qcand;
    int dev = 0;
    auto bail = [&](sas_status st) {
        delete c;
        return st;
    };
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(SAS_ERR_CUDA, "no usable CUDA device"));
    }
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(SAS_ERR_CUDA, "event creation failed"));
    }
    if (cudaMallocHost((void **)&c->h_meta, (2 * SAS_MAX_TYPES + 3) * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        c->h_meta = nullptr;
        return bail(fail(SAS_ERR_ALLOC, "pinned allocation failed"));
    }
    if (!c->coef_d.ensure(9 * n_types * sizeof(double)) ||
        !c->F.ensure((size_t)n_types * n_q * sizeof(double)))
        return bail(fail(SAS_ERR_ALLOC, "device allocation failed"));
    if (cudaMemcpy(c->coef_d.p, ff_coef, 9 * n_types * sizeof(double), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        launch_form_factors(c->coef_d.as<double>(), n_types, c->qc, c->F.as<double>(), 0) != cudaSuccess ||
        cudaStreamSynchronize(0) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(SAS_ERR_CUDA, "form-factor table failed"));
    }
    *out = c;
    return SAS_OK;
}

sas_status sas_destroy(sas_ctx *ctx)
{
    if (!ctx) return SAS_OK;
    if (ctx->h_meta) cudaFreeHost(ctx->h_meta);
    if (ctx->h_cen) cudaFreeHost(ctx->h_cen);
    if (ctx->h_stage) {
        cudaDeviceSynchronize();   // copies of a call that timed out may still target it
        cudaFreeHost(ctx->h_stage);
    }
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    delete ctx;
    return SAS_OK;
}

sas_status sas_profile(sas_ctx *ctx, const void *coords, int coords_type, const int32_t *types,
                       int64_t n_atoms, double *I_out, void *stream)
{
    sas::NvtxRange nvtx_range("sas_profile");
    return run_profile(ctx, coords, coords_type, types, n_atoms, 1, I_out, (cudaStream_t)stream);
}

sas_status sas_profile_batch(sas_ctx *ctx, const void *coords, int coords_type, const int32_t *types,
                             int64_t n_atoms, int64_t batch, double *I_out, void *stream)
{
    sas::NvtxRange nvtx_range("sas_profile_batch");
    return run_profile(ctx, coords, coords_type, types, n_atoms, batch, I_out, (cudaStream_t)stream);
}


sas_status sas_partials(sas_ctx *ctx, double *S_out, int64_t capacity, void *stream)
{
    if (!ctx || !S_out) return fail(SAS_ERR_INVALID_ARG, "null argument");
    if (!ctx->have_partials) return fail(SAS_ERR_INVALID_ARG, "no profile computed since the last change");
    const int Pn = ctx->n_types * (ctx->n_types + 1) / 2;
    const int64_t need = ctx->last_batch * Pn * ctx->n_q;
    if (capacity < need) return fail(SAS_ERR_INVALID_ARG, "capacity %lld < %lld", (long long)capacity, (long long)need);
    cudaStream_t s = (cudaStream_t)stream;
    HostCopies hc;
    sas_status st = out_copy(hc, S_out, ctx->S.p, (size_t)need * sizeof(double), s);
    if (st != SAS_OK) return st;
    return finish_copies(ctx, hc, s);
}

sas_status sas_exact_sums(sas_ctx *ctx, int64_t *U_out, int64_t capacity, void *stream)
{
    if (!ctx || !U_out) return fail(SAS_ERR_INVALID_ARG, "null argument");
    if (!(ctx->flags & SAS_DETERMINISTIC)) return fail(SAS_ERR_UNSUPPORTED, "exact sums need a SAS_DETERMINISTIC context");
    if (!ctx->have_partials) return fail(SAS_ERR_INVALID_ARG, "no profile computed since the last change");
    const int Pn = ctx->n_types * (ctx->n_types + 1) / 2;
    const int64_t need = ctx->last_batch * Pn * ctx->n_q * 2;
    if (capacity < need) return fail(SAS_ERR_INVALID_ARG, "capacity %lld < %lld", (long long)capacity, (long long)need);
    cudaStream_t s = (cudaStream_t)stream;
    HostCopies hc;
    sas_status st = out_copy(hc, U_out, ctx->Ufix.p, (size_t)need * sizeof(int64_t), s);
    if (st != SAS_OK) return st;
    return finish_copies(ctx, hc, s);
}

sas_status sas_assemble_exact(sas_ctx *ctx, const int64_t *U, int64_t batch, double *I_out, void *stream)
{
    if (!ctx || !U || !I_out) return fail(SAS_ERR_INVALID_ARG, "null argument");
    if (!(ctx->flags & SAS_DETERMINISTIC)) return fail(SAS_ERR_UNSUPPORTED, "exact sums need a SAS_DETERMINISTIC context");
    if (!ctx->have_partials) return fail(SAS_ERR_INVALID_ARG, "no profile computed since the last change");
    if (batch != ctx->last_batch)
        return fail(SAS_ERR_INVALID_ARG, "batch %lld differs from the last call's %lld", (long long)batch,
                    (long long)ctx->last_batch);
    const int T = ctx->n_types, Pn = T * (T + 1) / 2, Q = ctx->n_q;
    const int64_t groups = batch * Pn;
    cudaStream_t s = (cudaStream_t)stream;
    const void *Ud = nullptr;
    sas_status st = stage_in(ctx->Ustage, U, (size_t)groups * Q * sizeof(Fix128), s, Ud);
    if (st != SAS_OK) return st;
    ALLOC_TRY(ctx->Sx, (size_t)groups * Q * sizeof(double));
    CUDA_TRY(launch_fix_to_S(static_cast<const Fix128 *>(Ud), groups, ctx->qc, ctx->Sx.as<double>(), s));
    const bool host_out = !on_device(I_out);
    double *Id = I_out;
    if (host_out) {
        ALLOC_TRY(ctx->Ix, (size_t)batch * Q * sizeof(double));
        Id = ctx->Ix.as<double>();
    }
    CUDA_TRY(launch_assemble(ctx->Sx.as<double>(), ctx->F.as<double>(), ctx->meta.as<int>(), T, batch, ctx->qc, 1,
                             Id, s));
    HostCopies hc;
    st = out_copy(hc, I_out, Id, (size_t)batch * Q * sizeof(double), s);
    if (st != SAS_OK) return st;
    return finish_copies(ctx, hc, s);
}

sas_status sas_set_option(sas_ctx *ctx, int option, int64_t value)
{
    if (!ctx) return fail(SAS_ERR_INVALID_ARG, "null context");
    switch (option) {
    case SAS_OPT_JMAX:
        if (value < 0 || value % kTile || value > 8192)
            return fail(SAS_ERR_INVALID_ARG, "JMAX must be 0 or a multiple of %d up to 8192", kTile);
        ctx->opt_jmax = value;
        return SAS_OK;
    case SAS_OPT_RESEED:
        if (value != -1 && value != 0 && value != 32 && value != 64)
            return fail(SAS_ERR_INVALID_ARG, "RESEED must be -1 (automatic), 0, 32 or 64");
        ctx->opt_reseed = (int)value;
        return SAS_OK;
    case SAS_OPT_STEP:
        if (value != 2 && value != 4) return fail(SAS_ERR_INVALID_ARG, "STEP must be 2 or 4");
        ctx->opt_step = (int)value;
        return SAS_OK;
    case SAS_OPT_VARIANT:
        if (value < 0 || value > 4) return fail(SAS_ERR_INVALID_ARG, "VARIANT must be in [0, 4]");
        ctx->opt_variant = (int)value;
        return SAS_OK;
    case SAS_OPT_VALIDATE:
        if (value != 1) return fail(SAS_ERR_UNSUPPORTED, "validation cannot be switched off");
        return SAS_OK;
    case SAS_OPT_GRID:
        if (value < 0 || value > 8) return fail(SAS_ERR_INVALID_ARG, "GRID must be in [0, 8]");
        ctx->opt_grid = (int)value;
        return SAS_OK;
    case SAS_OPT_TIMEOUT_MS:
        if (value <= 0) return fail(SAS_ERR_INVALID_ARG, "timeout must be positive");
        ctx->opt_timeout_ms = value;
        return SAS_OK;
    case SAS_OPT_METHOD:
        if (value < 0 || value > 2) return fail(SAS_ERR_INVALID_ARG, "METHOD must be 0, 1 or 2");
        ctx->opt_method = (int)value;
        return SAS_OK;
    case SAS_OPT_ADJOINT:
        if (value < 0 || value > 1) return fail(SAS_ERR_INVALID_ARG, "ADJOINT must be 0 or 1");
        ctx->opt_adjoint = (int)value;
        return SAS_OK;
    case SAS_OPT_COEF:
        if (value < 0 || value > 2) return fail(SAS_ERR_INVALID_ARG, "COEF must be 0, 1 or 2");
        ctx->opt_coef = (int)value;
        return SAS_OK;
    case SAS_OPT_SHARD: {
        const int64_t world = value >> 16, rank = value & 0xFFFF;
        if (world < 1 || world > 65535 || rank >= world)
            return fail(SAS_ERR_INVALID_ARG, "SHARD must be world * 65536 + rank with 1 <= world and rank < world");
        ctx->opt_shard_world = (int)world;
        ctx->opt_shard_rank = (int)rank;
        return SAS_OK;
    }
    default:
        return fail(SAS_ERR_INVALID_ARG, "unknown option %d", option);
    }
}

sas_status sas_last_stats(sas_ctx *ctx, int64_t *stats_out, int n)
{
    if (!ctx || !stats_out || n < 0) return fail(SAS_ERR_INVALID_ARG, "bad argument");
    if (ctx->ev_pending) {   // pair-kernel time of the last call, in nanoseconds
        CUDA_TRY(cudaEventSynchronize(ctx->ev1));
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        ctx->stats[4] = (int64_t)((double)ms * 1.0e6);
        ctx->ev_pending = false;
    }
    for (int i = 0; i < n && i < 9; ++i) stats_out[i] = ctx->stats[i];
    return SAS_OK;
}

sas_status sas_profile_grad(sas_ctx *ctx, const float *coords, const int32_t *types, int64_t n,
                            int64_t batch, const double *target, const double *weights,
                            double *chi2_out, float *grad_out, double *I_out, void *stream)
{
    sas::NvtxRange nvtx_range("sas_profile_grad");
    sas_status st = check_common(ctx, coords, types, n, batch);
    if (st != SAS_OK) return st;
    if (ctx->flags & SAS_FP64) return fail(SAS_ERR_UNSUPPORTED, "the adjoint needs a SAS_MIXED context");
    if (ctx->opt_shard_world > 1)
        return fail(SAS_ERR_UNSUPPORTED, "chi^2 needs the whole profile: use a single shard (or sas_profile_vjp per "
                                         "shard with the gathered dchi^2/dI)");
    if (batch > 0 && (!target || !weights || !chi2_out || (n > 0 && !grad_out)))
        return fail(SAS_ERR_INVALID_ARG, "null argument");
    if (batch == 0) return SAS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int Q = ctx->n_q;
    int launches = 0;
    HostCopies hc;
    const void *tg = nullptr, *wt = nullptr;
    st = stage_in(ctx->tgt, target, Q * sizeof(double), s, tg);
    if (st != SAS_OK) return st;
    st = stage_in(ctx->wts, weights, Q * sizeof(double), s, wt);
    if (st != SAS_OK) return st;
    ALLOC_TRY(ctx->Ibuf, (size_t)batch * Q * sizeof(double));
    if (n == 0) {
        CUDA_TRY(cudaMemsetAsync(ctx->Ibuf.p, 0, (size_t)batch * Q * sizeof(double), s));
    } else {
        st = forward(ctx, coords, SAS_COORDS_F32, types, n, batch, ctx->Ibuf.as<double>(), adjoint_jmax_cap(ctx), s,
                     launches);
        if (st != SAS_OK) return st;
    }
    ALLOC_TRY(ctx->gbuf, (size_t)batch * Q * sizeof(double));
    ALLOC_TRY(ctx->chi2buf, (size_t)batch * sizeof(double));
    CUDA_TRY(launch_chi2(ctx->Ibuf.as<double>(), (const double *)tg, (const double *)wt, Q, batch,
                         ctx->gbuf.as<double>(), ctx->chi2buf.as<double>(), s));
    launches += 1;
    if (n > 0) {
        st = adjoint(ctx, n, batch, ctx->gbuf.as<double>(), grad_out, s, launches, hc);
        if (st != SAS_OK) return st;
    }
    st = out_copy(hc, chi2_out, ctx->chi2buf.p, (size_t)batch * sizeof(double), s);
    if (st != SAS_OK) return st;
    st = out_copy(hc, I_out, ctx->Ibuf.p, (size_t)batch * Q * sizeof(double), s);
    if (st != SAS_OK) return st;
    ctx->stats[5] = launches;
    return finish_copies(ctx, hc, s);
}

sas_status sas_profile_vjp(sas_ctx *ctx, const float *coords, const int32_t *types, int64_t n,
                           int64_t batch, const double *grad_I, float *grad_out, void *stream)
{
    sas::NvtxRange nvtx_range("sas_profile_vjp");
    sas_status st = check_common(ctx, coords, types, n, batch);
    if (st != SAS_OK) return st;
    if (ctx->flags & SAS_FP64) return fail(SAS_ERR_UNSUPPORTED, "the adjoint needs a SAS_MIXED context");
    if (batch > 0 && n > 0 && (!grad_I || !grad_out)) return fail(SAS_ERR_INVALID_ARG, "null argument");
    if (batch == 0 || n == 0) return SAS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int Q = ctx->n_q;
    int launches = 0;
    HostCopies hc;
    const void *gI = nullptr;
    st = stage_in(ctx->gbuf, grad_I, (size_t)batch * Q * sizeof(double), s, gI);
    if (st != SAS_OK) return st;
    // the adjoint needs the packed coordinates and items: pack without the pair kernel
    st = prepare(ctx, coords, SAS_COORDS_F32, types, n, batch, false, false, kTile, ctx->qc.n_chunks,
                 adjoint_jmax_cap(ctx), s, launches, ctx->n_types);
    if (st != SAS_OK) return st;
    st = adjoint(ctx, n, batch, (const double *)gI, grad_out, s, launches, hc);
    if (st != SAS_OK) return st;
    ctx->stats[5] = launches;
    return finish_copies(ctx, hc, s);
}

sas_status sas_pair_histogram(sas_ctx *ctx, const float *coords, const int32_t *types, int64_t n,
                              int64_t batch, int n_bins, float r_max, int32_t *hist_out,
                              int64_t *dropped_out, void *stream)
{
    sas::NvtxRange nvtx_range("sas_pair_histogram");
    sas_status st = check_common(ctx, coords, types, n, batch);
    if (st != SAS_OK) return st;
    if (n_bins < 1 || n_bins > 4096) return fail(SAS_ERR_INVALID_ARG, "n_bins must be in [1, 4096]");
    if (!(r_max > 0.f) || !std::isfinite(r_max)) return fail(SAS_ERR_INVALID_ARG, "r_max must be positive");
    if (!(r_max <= 1e18f) || !(r_max / (float)n_bins >= 1e-12f))
        return fail(SAS_ERR_INVALID_ARG, "r_max must be at most 1e18 and r_max / n_bins at least 1e-12");
    if (batch > 0 && !hist_out) return fail(SAS_ERR_INVALID_ARG, "null output");
    if (batch == 0) return SAS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int T = ctx->n_types, Pn = T * (T + 1) / 2;
    const size_t hbytes = (size_t)batch * Pn * n_bins * sizeof(int32_t);
    if (n == 0) {
        st = zero_out(hist_out, hbytes, s);
        if (st == SAS_OK && dropped_out) st = zero_out(dropped_out, (size_t)batch * sizeof(int64_t), s);
        return st;
    }
    int launches = 0;
    const int64_t jcap = 4096;
    st = prepare(ctx, coords, SAS_COORDS_F32, types, n, batch, false, false, kTile, 1, jcap, s, launches,
                 ctx->n_types);
    if (st != SAS_OK) return st;
    const int64_t npad = ctx->h_meta[2 * T];
    ALLOC_TRY(ctx->hist, hbytes);
    ALLOC_TRY(ctx->dropped, (size_t)batch * sizeof(int64_t));
    CUDA_TRY(cudaMemsetAsync(ctx->hist.p, 0, hbytes, s));
    CUDA_TRY(cudaMemsetAsync(ctx->dropped.p, 0, (size_t)batch * sizeof(int64_t), s));
    ALLOC_TRY(ctx->ticket, sizeof(int));
    CUDA_TRY(cudaMemsetAsync(ctx->ticket.p, 0, sizeof(int), s));
    CUDA_TRY(launch_pair_histogram(ctx->X.as<float4>(), npad, ctx->items.as<Item>(), ctx->n_items, n_bins,
                                   r_max, Pn, ctx->hist.as<int>(), ctx->dropped.as<unsigned long long>(),
                                   ctx->jlen_max, ctx->ticket.as<int>(), s));
    launches += 1;
    HostCopies hc;
    st = out_copy(hc, hist_out, ctx->hist.p, hbytes, s);
    if (st != SAS_OK) return st;
    st = out_copy(hc, dropped_out, ctx->dropped.p, (size_t)batch * sizeof(int64_t), s);
    if (st != SAS_OK) return st;
    ctx->stats[5] = launches;
    ctx->have_partials = false;
    return finish_copies(ctx, hc, s);
}

}  // extern "C"

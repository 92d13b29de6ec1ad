// sas_profile_static: the mixed-precision profile of one molecule without any allocation.
//
// Some callers cannot allocate GPU memory at the point where they need a profile: code running
// under a memory budget that was reserved up front, allocators that must not be re-entered, or
// hosts that forbid cudaMalloc/cudaFree (which synchronize the device) inside a latency-critical
// loop.  This entry point serves them: every intermediate buffer (packed coordinates, the
// type-pair table, the work list, the per-item partial sums, the form-factor table) lives in one
// file-scope __device__ array of fixed size, and the host side uses fixed static arrays (no heap,
// a few hundred bytes of stack).  The arithmetic is that of sas_profile on a SAS_MIXED context:
// the same pack, pair, reduction and assembly kernels, given pointers into the fixed array.
//
// Set-up: the address of the array on the current device is taken with cudaGetSymbolAddress by
// the first call on that device (the host-side name of the array is not a device address) and
// kept for later calls.  Do that first call outside any stream capture.
// Synchronization: a call waits for its stream twice, once to read the type counts back (the
// work list is built from them on the host) and once at the end.
// Sharing: every call on a device uses the same array, and it keeps the previous call's
// contents; the calls clear what has to start at zero.  Two calls whose work overlaps on the
// GPU race on the array.  Calls from several host threads are serialized by a lock that is held
// until the call's stream has finished, which also guards the static host-side work list.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "sas_internal.h"

namespace sas {
namespace {

constexpr int kStaticJmax = 2048;
constexpr int kStaticTypes = SAS_MAX_TYPES;
constexpr int kStaticPairs = kStaticTypes * (kStaticTypes + 1) / 2;
constexpr int64_t kStaticNpad = SAS_STATIC_MAX_ATOMS + (int64_t)kStaticTypes * kTile;
constexpr int kStaticTiles = (int)(kStaticNpad / kTile);
// per I-tile and type pair at most ceil(P_b / JMAX) <= P_b / JMAX + 1 items
constexpr int kStaticItems = kStaticTiles * (int)(kStaticNpad / kStaticJmax + kStaticTypes);
constexpr int kStaticBlocks = (SAS_STATIC_MAX_ATOMS + kPackThreads - 1) / kPackThreads;

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Byte offsets of the regions inside the array.
constexpr size_t kOffX = 0;
constexpr size_t kOffSlot = kOffX + align256(sizeof(float4) * kStaticNpad);
constexpr size_t kOffMeta = kOffSlot + align256(sizeof(int) * SAS_STATIC_MAX_ATOMS);
constexpr size_t kOffCounts = kOffMeta + align256(sizeof(int) * (2 * kStaticTypes + 3));
constexpr size_t kOffOffs = kOffCounts + align256(sizeof(int) * kStaticBlocks * kStaticTypes);
constexpr size_t kOffItems = kOffOffs + align256(sizeof(int) * kStaticBlocks * kStaticTypes);
constexpr size_t kOffGroupItems = kOffItems + align256(sizeof(Item) * kStaticItems);
constexpr size_t kOffGroupOff = kOffGroupItems + align256(sizeof(int) * kStaticItems);
constexpr size_t kOffPartial = kOffGroupOff + align256(sizeof(int) * (kStaticPairs + 1));
constexpr size_t kOffS = kOffPartial + align256(sizeof(double) * kStaticItems * kQChunk);
constexpr size_t kOffF = kOffS + align256(sizeof(double) * kStaticPairs * kQChunk);
constexpr size_t kOffCoef = kOffF + align256(sizeof(double) * kStaticTypes * kQChunk);
constexpr size_t kOffTicket = kOffCoef + align256(sizeof(double) * 9 * kStaticTypes);
constexpr size_t kStaticBytes = kOffTicket + align256(sizeof(int));

// The scratch array.  Device code could name it directly; host code must not pass its name to a
// kernel (there it is a host-side stand-in), only the address cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
// Held for a whole call: it guards the per-device addresses and the host-side work list below,
// and keeps calls from different host threads from overlapping on the shared array.
std::mutex g_static_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};
// Host-side work list of the current call (static storage, about 130 KB, rather than the
// caller's stack, which may be small on worker threads).
Item g_h_items[kStaticItems];
int g_h_group_items[kStaticItems];
int g_h_group_off[kStaticPairs + 1];

// The entry point reports through its status code only (the messages below document the cases).
sas_status static_fail(sas_status st, const char *msg, const char *detail = "")
{
    (void)msg;
    (void)detail;
    return st;
}

int pair_index_static(int a, int b, int T)
{
    if (a > b) std::swap(a, b);
    return a * T - a * (a - 1) / 2 + (b - a);
}

bool is_device_pointer(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace sas

using namespace sas;

static_assert(kStaticBytes <= (size_t)SAS_STATIC_SCRATCH_BYTES, "scratch larger than documented");

extern "C" sas_status sas_profile_static(const float *coords, const int32_t *types, int64_t n, int n_types,
                                         const double *ff_coef, double q0, double dq, int n_q, double *I_out,
                                         void *stream)
{
    sas::NvtxRange nvtx_range("sas_profile_static");
    if (n < 0 || n > SAS_STATIC_MAX_ATOMS)
        return static_fail(SAS_ERR_UNSUPPORTED, "n_atoms must be in [0, SAS_STATIC_MAX_ATOMS]");
    if (n_types < 1 || n_types > kStaticTypes) return static_fail(SAS_ERR_INVALID_ARG, "n_types must be in [1, 16]");
    if (n_q < 1 || n_q > kQChunk) return static_fail(SAS_ERR_UNSUPPORTED, "n_q must be in [1, 208]");
    if (!ff_coef || !I_out || (n > 0 && (!coords || !types))) return static_fail(SAS_ERR_INVALID_ARG, "null pointer");
    if (!std::isfinite(q0) || !std::isfinite(dq) || q0 < 0 || dq < 0 || (n_q > 1 && !(dq > 0)))
        return static_fail(SAS_ERR_INVALID_ARG, "q grid must be q0 >= 0 with a positive step");
    for (int k = 0; k < 9 * n_types; ++k)
        if (!std::isfinite(ff_coef[k])) return static_fail(SAS_ERR_INVALID_ARG, "non-finite coefficient");
    if (!is_device_pointer(I_out) || (n > 0 && (!is_device_pointer(coords) || !is_device_pointer(types))))
        return static_fail(SAS_ERR_INVALID_ARG, "coords, types and I_out must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
#define STATIC_TRY(call)                                                                       \
    do {                                                                                       \
        if ((e = (call)) != cudaSuccess) {                                                     \
            cudaGetLastError();                                                                \
            return static_fail(SAS_ERR_CUDA, #call ": ", cudaGetErrorString(e));               \
        }                                                                                      \
    } while (0)

    // set-up, once per device: the device address of the scratch array
    int dev = 0;
    STATIC_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return static_fail(SAS_ERR_UNSUPPORTED, "device ordinal too large");
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        STATIC_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
        g_scratch_ptr[dev] = p;
    }
    unsigned char *base = static_cast<unsigned char *>(g_scratch_ptr[dev]);
    if (n == 0) {
        STATIC_TRY(cudaMemsetAsync(I_out, 0, sizeof(double) * n_q, s));
        return SAS_OK;
    }
    float4 *X = reinterpret_cast<float4 *>(base + kOffX);
    int *slot_of = reinterpret_cast<int *>(base + kOffSlot);
    int *meta = reinterpret_cast<int *>(base + kOffMeta);
    int *blockcounts = reinterpret_cast<int *>(base + kOffCounts);
    int *blockoffs = reinterpret_cast<int *>(base + kOffOffs);
    Item *items = reinterpret_cast<Item *>(base + kOffItems);
    int *group_items = reinterpret_cast<int *>(base + kOffGroupItems);
    int *group_off = reinterpret_cast<int *>(base + kOffGroupOff);
    double *partial = reinterpret_cast<double *>(base + kOffPartial);
    double *S = reinterpret_cast<double *>(base + kOffS);
    double *F = reinterpret_cast<double *>(base + kOffF);
    double *coef = reinterpret_cast<double *>(base + kOffCoef);
    int *ticket = reinterpret_cast<int *>(base + kOffTicket);

    // the q grid as one chunk
    QChunks qc{};
    qc.n_q = n_q;
    qc.n_chunks = 1;
    qc.qsd[0] = q0;
    qc.dqd[0] = dq;
    qc.dq_hi[0] = (float)dq;
    qc.dq_lo[0] = (float)(dq - (double)qc.dq_hi[0]);
    qc.q_begin[0] = 0;
    qc.q_len[0] = n_q;
    qc.qs_hi[0] = (float)q0;
    qc.qs_lo[0] = (float)(q0 - (double)qc.qs_hi[0]);

    // form factors, validation and type counts (the previous contents of meta are cleared)
    const int T = n_types, Pn = T * (T + 1) / 2;
    const int nblk = (int)((n + kPackThreads - 1) / kPackThreads);
    STATIC_TRY(cudaMemcpyAsync(coef, ff_coef, sizeof(double) * 9 * T, cudaMemcpyHostToDevice, s));
    STATIC_TRY(launch_form_factors(coef, T, qc, F, s));
    STATIC_TRY(cudaMemsetAsync(meta, 0, sizeof(int) * (2 * T + 3), s));
    STATIC_TRY(launch_count_types(coords, 0, types, n, 1, T, blockcounts, meta + 2 * T + 1,
                                  reinterpret_cast<unsigned *>(meta + 2 * T + 2), s));
    STATIC_TRY(launch_scan_counts(blockcounts, nblk, T, kTile, blockoffs, meta, s));
    int h_meta[2 * kStaticTypes + 3];
    STATIC_TRY(cudaMemcpyAsync(h_meta, meta, sizeof(int) * (2 * T + 3), cudaMemcpyDeviceToHost, s));
    STATIC_TRY(cudaStreamSynchronize(s));
    if (h_meta[2 * T + 1] & kErrBadType) return static_fail(SAS_ERR_INVALID_ARG, "atom type outside [0, n_types)");
    if (h_meta[2 * T + 1] & kErrNonFinite) return static_fail(SAS_ERR_INVALID_ARG, "non-finite coordinate");
    const int64_t npad = h_meta[2 * T];

    // work list in canonical order (groups (a, b) in row-major order), in the static host arrays
    Item *h_items = g_h_items;
    int *h_group_items = g_h_group_items;
    int *h_group_off = g_h_group_off;
    int ni = 0;
    {
        int64_t P[kStaticTypes], O[kStaticTypes], off = 0;
        for (int t = 0; t < T; ++t) {
            P[t] = (h_meta[t] + kTile - 1) / kTile * kTile;
            O[t] = off;
            off += P[t];
        }
        int g = 0;
        for (int a = 0; a < T; ++a)
            for (int b = a; b < T; ++b, ++g) {
                h_group_off[g] = ni;
                if (P[a] == 0 || P[b] == 0) continue;
                for (int64_t i0 = O[a]; i0 < O[a] + P[a]; i0 += kTile) {
                    const int64_t js = (a == b) ? i0 : O[b], je = O[b] + P[b];
                    for (int64_t j0 = js; j0 < je; j0 += kStaticJmax) {
                        if (ni >= kStaticItems) return static_fail(SAS_ERR_UNSUPPORTED, "work list too long");
                        Item &it = h_items[ni];
                        it.batch = 0;
                        it.pair = pair_index_static(a, b, T);
                        it.i0 = (int)i0;
                        it.j0 = (int)j0;
                        it.jlen = (int)std::min<int64_t>(kStaticJmax, je - j0);
                        it.chunk = 0;
                        it.diag = (a == b && j0 == i0) ? 1 : 0;
                        it.work = it.jlen * kTile;
                        h_group_items[ni] = ni;
                        ++ni;
                    }
                }
            }
        h_group_off[Pn] = ni;
    }
    STATIC_TRY(cudaMemcpyAsync(items, h_items, sizeof(Item) * ni, cudaMemcpyHostToDevice, s));
    STATIC_TRY(cudaMemcpyAsync(group_items, h_group_items, sizeof(int) * ni, cudaMemcpyHostToDevice, s));
    STATIC_TRY(cudaMemcpyAsync(group_off, h_group_off, sizeof(int) * (Pn + 1), cudaMemcpyHostToDevice, s));

    // pack (padding slots cleared first), pair kernel, item reduction, assembly
    STATIC_TRY(cudaMemsetAsync(X, 0, sizeof(float4) * npad, s));
    STATIC_TRY(launch_scatter(coords, 0, types, n, 1, T, blockoffs, meta, nullptr, 0, X, npad, slot_of, s));
    // the automatic re-seed rule of sas_profile (no re-seeding from 8,192 atoms, or from 2,000 atoms
    // when the chunk holds at most 104 q values)
    float r2;
    const unsigned bits = (unsigned)h_meta[2 * T + 2];
    std::memcpy(&r2, &bits, sizeof r2);
    const double phase = 2.0 * std::fabs(dq) * 2.0 * std::sqrt((double)r2);   // step phase 2 dq D
    const int reseed = reseed_auto(n, std::min(n_q, kQChunk), phase);
    qc.coef_both = phase >= kCoefBothPhase ? 1 : 0;
    STATIC_TRY(cudaMemsetAsync(ticket, 0, sizeof(int), s));
    STATIC_TRY(launch_debye_mixed(X, npad, items, ni, qc, 2, reseed, reseed == 0 ? 5 : 1, partial, kQChunk, 0,
                                  kStaticJmax, ticket, s));
    STATIC_TRY(launch_reduce_items(partial, kQChunk, items, group_items, group_off, Pn, qc, S, s));
    STATIC_TRY(launch_assemble(S, F, meta, T, 1, qc, 1, I_out, s));
    // the next call reuses the host-side arrays: wait until the copies from them are done
    STATIC_TRY(cudaStreamSynchronize(s));
#undef STATIC_TRY
    return SAS_OK;
}

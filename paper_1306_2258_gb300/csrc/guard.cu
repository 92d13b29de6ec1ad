// Guard bands around the library's device buffers: a debugging aid that stands in for a memory
// checker where none can run (not part of the paper's method).
//
// While guard bands are on (sas_guard_bands, or SAS_GUARD_BANDS=1 in the environment when the
// library is loaded), every device buffer the library allocates is placed between two bands of
// kGuardBytes filled with kGuardByte: the allocation is kGuardBytes + bytes + kGuardBytes, the
// buffer starts after the first band (so its 256-byte alignment is kept) and the second band starts
// at the buffer's exact end.  A kernel that writes past either end of a buffer changes a band;
// sas_guard_check waits for the devices and compares every band of every live guarded buffer with
// the pattern.  Buffers allocated while guard bands are off stay plain, and a guarded buffer keeps
// its bands until it is freed, whatever the switch says by then.
//
// Every allocation site of the library goes through dev_malloc / dev_free: the context buffers
// (DevBuf), the surrogate network's buffers and the peak microbenchmarks' scratch.  The fixed array
// of the allocation-free entry point is not an allocation and has no bands.  Setting up the bands
// waits for the device, so a guarded allocation must not happen during stream capture.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "api_internal.h"
#include "sas.h"

namespace sas {
namespace api {

namespace {

constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;

struct Guarded {
    unsigned char *raw;   // start of the allocation (the front band)
    size_t bytes;         // the buffer's size; the back band starts at user + bytes
    int device;
};

std::mutex g_mu;
std::unordered_map<void *, Guarded> g_live;   // user pointer -> allocation
bool g_on = [] {
    const char *e = std::getenv("SAS_GUARD_BANDS");
    return e && e[0] == '1';
}();

}  // namespace

cudaError_t dev_malloc(void **p, size_t bytes)
{
    bool on;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        on = g_on;
    }
    if (!on) return cudaMalloc(p, bytes);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    void *raw = nullptr;
    if ((e = cudaMalloc(&raw, bytes + 2 * kGuardBytes)) != cudaSuccess) return e;
    unsigned char *r = static_cast<unsigned char *>(raw);
    e = cudaMemset(r, kGuardByte, kGuardBytes);
    if (e == cudaSuccess) e = cudaMemset(r + kGuardBytes + bytes, kGuardByte, kGuardBytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();   // the bands are set before any kernel can use the buffer
    if (e != cudaSuccess) {
        cudaFree(raw);
        return e;
    }
    *p = r + kGuardBytes;
    std::lock_guard<std::mutex> lk(g_mu);
    g_live[*p] = Guarded{r, bytes, dev};
    return cudaSuccess;
}

void dev_free(void *p)
{
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_live.find(p);
        if (it != g_live.end()) {
            void *raw = it->second.raw;
            g_live.erase(it);
            cudaFree(raw);
            return;
        }
    }
    cudaFree(p);
}

}  // namespace api
}  // namespace sas

using namespace sas::api;

extern "C" sas_status sas_guard_bands(int enable)
{
    if (enable != 0 && enable != 1) return fail(SAS_ERR_INVALID_ARG, "enable must be 0 or 1");
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = enable == 1;
    return SAS_OK;
}

extern "C" sas_status sas_guard_check(int64_t *n_checked_out)
{
    std::vector<std::pair<void *, Guarded>> live;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        live.assign(g_live.begin(), g_live.end());
    }
    if (n_checked_out) *n_checked_out = 0;
    if (live.empty()) return SAS_OK;
    int dev0 = 0;
    if (cudaGetDevice(&dev0) != cudaSuccess) {
        cudaGetLastError();
        return fail(SAS_ERR_CUDA, "cudaGetDevice failed");
    }
    std::vector<unsigned char> band(kGuardBytes);
    int64_t checked = 0, bad = 0;
    void *first_bad = nullptr;
    size_t first_bytes = 0;
    const char *first_side = "";
    sas_status st = SAS_OK;
    int synced = -1;
    for (const auto &kv : live) {
        const Guarded &g = kv.second;
        if (cudaSetDevice(g.device) != cudaSuccess) {
            st = SAS_ERR_CUDA;
            break;
        }
        if (synced != g.device && cudaDeviceSynchronize() != cudaSuccess) {   // kernels may still write
            st = SAS_ERR_CUDA;
            break;
        }
        synced = g.device;
        const unsigned char *bands[2] = {g.raw, g.raw + kGuardBytes + g.bytes};
        for (int side = 0; side < 2 && st == SAS_OK; ++side) {
            if (cudaMemcpy(band.data(), bands[side], kGuardBytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
                st = SAS_ERR_CUDA;
                break;
            }
            bool ok = true;
            for (unsigned char b : band) ok = ok && b == kGuardByte;
            if (!ok) {
                if (bad == 0) {
                    first_bad = kv.first;
                    first_bytes = g.bytes;
                    first_side = side == 0 ? "before" : "after";
                }
                ++bad;
            }
        }
        if (st != SAS_OK) break;
        ++checked;
    }
    cudaSetDevice(dev0);
    if (st != SAS_OK) {
        cudaGetLastError();
        return fail(SAS_ERR_CUDA, "reading the guard bands failed");
    }
    if (n_checked_out) *n_checked_out = checked;
    if (bad > 0)
        return fail(SAS_ERR_CORRUPT, "%lld guard band(s) overwritten; first: the band %s the %zu-byte buffer at %p",
                    (long long)bad, first_side, first_bytes, first_bad);
    return SAS_OK;
}

extern "C" sas_status sas_guard_list(int64_t cap, void **ptr_out, int64_t *bytes_out, int64_t *n_out)
{
    if (cap < 0 || !n_out || (cap > 0 && (!ptr_out || !bytes_out)))
        return fail(SAS_ERR_INVALID_ARG, "cap < 0 or a null output");
    std::lock_guard<std::mutex> lk(g_mu);
    int64_t k = 0;
    for (const auto &kv : g_live) {
        if (k < cap) {
            ptr_out[k] = kv.first;
            bytes_out[k] = (int64_t)kv.second.bytes;
        }
        ++k;
    }
    *n_out = k;
    return SAS_OK;
}

// C ABI of the surrogate MLP (include/sas.h): the network object, its training step and
// inference, state transfer for checkpoints, and a plain bfloat16 GEMM for tests.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "sas_internal.h"

using namespace sas;

namespace {

using bf16 = __nv_bfloat16;

sas_status mlp_fail(sas_status st, const char *what, cudaError_t e = cudaSuccess)
{
    char buf[256];
    if (e != cudaSuccess) {
        cudaGetLastError();
        snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    } else {
        snprintf(buf, sizeof buf, "%s", what);
    }
    return set_error(st, buf);
}

#define MLP_TRY(call)                                                          \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) return mlp_fail(SAS_ERR_CUDA, #call, e_);       \
    } while (0)

// After a synchronization: the tensor-core GEMM's error word (a wait that ran out of iterations).
sas_status gemm_check()
{
    int err = 0;
    MLP_TRY(gemm_tc_error(&err));
    return err ? mlp_fail(SAS_ERR_TIMEOUT, "a tensor-core GEMM wait ran out of iterations") : SAS_OK;
}

bool on_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline int round16(int x) { return (x + 15) / 16 * 16; }

}  // namespace

struct sas_mlp {
    int n_in = 0, h = 0, n_out = 0, n_outp = 0, max_b = 0;
    // packed parameter block in device layout: W1 [h][n_in], b1 [h], W2 [h][h], b2 [h],
    // W3 [n_outp][h] (rows >= n_out stay zero), b3 [n_outp]
    int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0, np = 0;
    float *P = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr;
    bf16 *Pb = nullptr;             // bfloat16 mirror of P
    bf16 *W2t = nullptr, *W3t = nullptr;
    float *Xf = nullptr, *Tf = nullptr, *Z1 = nullptr, *Z2 = nullptr, *Y = nullptr, *dY = nullptr, *dA2 = nullptr,
          *dZ2 = nullptr, *dA1 = nullptr, *dZ1 = nullptr, *loss = nullptr;
    // scratch of the fused backward kernels: column partials, row losses, counters (left zero)
    float *part = nullptr;
    double *lpart = nullptr;
    unsigned *count = nullptr;
    // split-K slices of the first layer for small batches (few output tiles, K = n_in long)
    float *ws = nullptr;
    int ws_rows = 0, ws_splits = 0;
    bf16 *Xb = nullptr, *Xt = nullptr, *A1b = nullptr, *A1t = nullptr, *A2b = nullptr, *A2t = nullptr, *dYb = nullptr,
         *dYt = nullptr, *dZ2b = nullptr, *dZ2t = nullptr, *dZ1b = nullptr, *dZ1t = nullptr;
    std::vector<void *> owned;
    int64_t step = 0;
    // the forward and backward launches of a training step, captured once per batch size on an
    // internal stream and replayed on the caller's stream (they read the inputs from Xf and Tf)
    cudaStream_t capture_stream = nullptr;
    std::vector<std::pair<int, cudaGraphExec_t>> step_graphs;
};

namespace {

template <class T>
bool mlp_alloc(sas_mlp *m, T *&p, int64_t n)
{
    void *q = nullptr;
    if (sas::api::dev_malloc(&q, sizeof(T) * (size_t)(n > 0 ? n : 1)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    m->owned.push_back(q);
    p = static_cast<T *>(q);
    return true;
}

void mlp_free(sas_mlp *m)
{
    for (void *p : m->owned) sas::api::dev_free(p);
    m->owned.clear();
}

// Slices of the first layer's K range for batch B: 0 (one pass) unless its output tiles (128 x 64)
// would leave three quarters of the SMs idle and K holds at least 8 stages of 64; then enough
// slices of at least 4 stages to bring the CTAs near the SM count.
int splitk_slices(const sas_mlp *m, int B)
{
    if (!m->ws || B > m->ws_rows) return 0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int tiles = ((B + 127) / 128) * ((m->h + 63) / 64), kt = (m->n_in + 63) / 64;
    if (kt < 8 || 4 * tiles > sms) return 0;
    int z = std::min({m->ws_splits, sms / tiles, kt / 4});
    while (z > 1 && (kt + z - 1) / z * (z - 1) >= kt) --z;   // no empty slice
    return z >= 2 ? z : 0;
}

// The forward launches from device input xd [B][n_in] f32 to Y.  The bfloat16 operands X, A1 and A2
// are also written transposed (batch padding zero), as the weight-gradient GEMMs take them.
sas_status mlp_forward_dev(sas_mlp *m, const float *xd, int B, cudaStream_t s)
{
    const int Bp = round16(B);
    MLP_TRY(launch_to_bf16_t(B, Bp, m->n_in, xd, m->Xb, m->Xt, Bp, s));
    const bf16 *W1b = m->Pb + m->oW1, *W2b = m->Pb + m->oW2, *W3b = m->Pb + m->oW3;
    if (const int z = splitk_slices(m, B)) {
        // first layer in K slices, then their sum, the bias, GELU and A1's transpose in one pass
        MLP_TRY(launch_gemm_splitk(B, m->h, m->n_in, m->Xb, m->n_in, W1b, m->n_in, m->ws, z, s));
        MLP_TRY(launch_splitk_gelu(B, Bp, m->h, z, m->ws, m->P + m->ob1, m->Z1, m->A1b, m->A1t, Bp, s));
    } else {
        MLP_TRY(launch_gemm_t(B, m->h, m->n_in, m->Xb, m->n_in, W1b, m->n_in, m->P + m->ob1, m->Z1, m->h, m->A1b, m->h,
                              1, m->A1t, Bp, Bp, s));
    }
    MLP_TRY(launch_gemm_t(B, m->h, m->h, m->A1b, m->h, W2b, m->h, m->P + m->ob2, m->Z2, m->h, m->A2b, m->h, 1, m->A2t,
                          Bp, Bp, s));
    MLP_TRY(launch_gemm(B, m->n_outp, m->h, m->A2b, m->h, W3b, m->h, m->P + m->ob3, m->Y, m->n_outp, nullptr, 0, 0,
                           s));
    return SAS_OK;
}

// x (host or device, [B][n_in] f32) and optionally t ([B][n_out]) to device; forward to Y.  With
// `stage_x` the input is always copied into Xf (the captured graph reads it there).
sas_status mlp_forward(sas_mlp *m, const float *x, const float *t, int B, cudaStream_t s, bool stage_x = false)
{
    if (B < 1 || B > m->max_b) return mlp_fail(SAS_ERR_INVALID_ARG, "batch outside [1, max_batch]");
    const float *xd = x;
    if (stage_x || !on_device_ptr(x)) {
        MLP_TRY(cudaMemcpyAsync(m->Xf, x, sizeof(float) * (size_t)B * m->n_in, cudaMemcpyDefault, s));
        xd = m->Xf;
    }
    if (t) {
        MLP_TRY(cudaMemcpyAsync(m->Tf, t, sizeof(float) * (size_t)B * m->n_out,
                                on_device_ptr(t) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    }
    if (stage_x) return SAS_OK;   // the launches are the captured graph's
    return mlp_forward_dev(m, xd, B, s);
}

// Gradients of the MSE loss for the batch already in Xb/Tf (after mlp_forward) into G.
sas_status mlp_backward(sas_mlp *m, int B, cudaStream_t s)
{
    const int Bp = round16(B), h = m->h, Qp = m->n_outp;
    // layer 3: dY (with its transpose, the bias gradient and the loss)
    MLP_TRY(launch_mse_fused(B, Bp, m->n_out, Qp, m->Y, m->Tf, m->dY, m->dYb, m->dYt, Bp, m->lpart, m->part,
                             m->G + m->ob3, m->loss, m->count, s));
    MLP_TRY(launch_gemm(Qp, h, Bp, m->dYt, Bp, m->A2t, Bp, nullptr, m->G + m->oW3, h, nullptr, 0, 0, s));
    MLP_TRY(launch_gemm(B, h, Qp, m->dYb, Qp, m->W3t, Qp, nullptr, m->dA2, h, nullptr, 0, 0, s));
    // layer 2
    MLP_TRY(launch_act_bwd(B, Bp, h, m->dA2, m->Z2, m->dZ2, m->dZ2b, m->dZ2t, Bp, m->part, m->G + m->ob2, m->count,
                           s));
    MLP_TRY(launch_gemm(h, h, Bp, m->dZ2t, Bp, m->A1t, Bp, nullptr, m->G + m->oW2, h, nullptr, 0, 0, s));
    MLP_TRY(launch_gemm(B, h, h, m->dZ2b, h, m->W2t, h, nullptr, m->dA1, h, nullptr, 0, 0, s));
    // layer 1
    MLP_TRY(launch_act_bwd(B, Bp, h, m->dA1, m->Z1, m->dZ1, m->dZ1b, m->dZ1t, Bp, m->part, m->G + m->ob1, m->count,
                           s));
    MLP_TRY(launch_gemm(h, m->n_in, Bp, m->dZ1t, Bp, m->Xt, Bp, nullptr, m->G + m->oW1, m->n_in, nullptr, 0, 0, s));
    return SAS_OK;
}

// bfloat16 mirror of the masters (unless the Adam step has just written it) and the transposed
// weights the backward pass uses
sas_status mlp_refresh(sas_mlp *m, cudaStream_t s, bool convert = true)
{
    if (convert) MLP_TRY(launch_to_bf16(m->np, m->P, m->Pb, s));
    MLP_TRY(launch_transpose_bf16(m->h, m->h, m->h, m->Pb + m->oW2, m->h, m->W2t, m->h, s));
    MLP_TRY(launch_transpose_bf16(m->n_outp, m->n_outp, m->h, m->Pb + m->oW3, m->h, m->W3t, m->n_outp, s));
    return SAS_OK;
}

// The training step's forward and backward launches for batch B as a graph (captured on first use).
sas_status step_graph(sas_mlp *m, int B, cudaGraphExec_t &ex)
{
    for (auto &g : m->step_graphs)
        if (g.first == B) {
            ex = g.second;
            return SAS_OK;
        }
    if (!m->capture_stream) MLP_TRY(cudaStreamCreateWithFlags(&m->capture_stream, cudaStreamNonBlocking));
    cudaStream_t cs = m->capture_stream;
    MLP_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    sas_status st = mlp_forward_dev(m, m->Xf, B, cs);
    if (st == SAS_OK) st = mlp_backward(m, B, cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (st != SAS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return mlp_fail(SAS_ERR_CUDA, "capture of the training step", e);
    const cudaError_t ei = cudaGraphInstantiate(&ex, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return mlp_fail(SAS_ERR_CUDA, "instantiation of the training step", ei);
    if (m->step_graphs.size() >= 8) {   // a small cache: the oldest batch size goes
        cudaGraphExecDestroy(m->step_graphs.front().second);
        m->step_graphs.erase(m->step_graphs.begin());
    }
    m->step_graphs.emplace_back(B, ex);
    return SAS_OK;
}

// Device layout <-> packed layout (W3 and b3 with n_out rows) for one float block.
void pack_layout(const sas_mlp *m, const float *dev_layout, float *packed)
{
    const int64_t nW3 = (int64_t)m->n_out * m->h;
    std::memcpy(packed, dev_layout, sizeof(float) * (size_t)m->oW3);
    std::memcpy(packed + m->oW3, dev_layout + m->oW3, sizeof(float) * (size_t)nW3);
    std::memcpy(packed + m->oW3 + nW3, dev_layout + m->ob3, sizeof(float) * (size_t)m->n_out);
}

void unpack_layout(const sas_mlp *m, const float *packed, float *dev_layout)
{
    const int64_t nW3 = (int64_t)m->n_out * m->h;
    std::memset(dev_layout, 0, sizeof(float) * (size_t)m->np);
    std::memcpy(dev_layout, packed, sizeof(float) * (size_t)m->oW3);
    std::memcpy(dev_layout + m->oW3, packed + m->oW3, sizeof(float) * (size_t)nW3);
    std::memcpy(dev_layout + m->ob3, packed + m->oW3 + nW3, sizeof(float) * (size_t)m->n_out);
}

int64_t packed_count(const sas_mlp *m) { return m->oW3 + (int64_t)m->n_out * m->h + m->n_out; }

sas_status copy_block(const sas_mlp *m, const float *dev, float *host_packed)
{
    std::vector<float> tmp((size_t)m->np);
    MLP_TRY(cudaMemcpy(tmp.data(), dev, sizeof(float) * (size_t)m->np, cudaMemcpyDeviceToHost));
    pack_layout(m, tmp.data(), host_packed);
    return SAS_OK;
}

}  // namespace

extern "C" {

sas_status sas_mlp_create(int n_in, int n_hidden, int n_out, int max_batch, sas_mlp **out)
{
    if (!out) return mlp_fail(SAS_ERR_INVALID_ARG, "null output handle");
    if (n_in < 16 || n_in % 16 || n_hidden < 16 || n_hidden % 16 || n_out < 1 || max_batch < 1 || max_batch > 65536)
        return mlp_fail(SAS_ERR_INVALID_ARG, "n_in and n_hidden must be positive multiples of 16, n_out >= 1, "
                                             "max_batch in [1, 65536]");
    sas_mlp *m = new (std::nothrow) sas_mlp;
    if (!m) return mlp_fail(SAS_ERR_ALLOC, "host allocation failed");
    m->n_in = n_in;
    m->h = n_hidden;
    m->n_out = n_out;
    m->n_outp = round16(n_out);
    m->max_b = max_batch;
    const int64_t h = n_hidden, Qp = m->n_outp, Bp = round16(max_batch);
    m->oW1 = 0;
    m->ob1 = h * n_in;
    m->oW2 = m->ob1 + h;
    m->ob2 = m->oW2 + h * h;
    m->oW3 = m->ob2 + h;
    m->ob3 = m->oW3 + Qp * h;
    m->np = m->ob3 + Qp;
    // split-K slices of the first layer: batches up to 512 rows, at most 16 slices and 32 MB
    m->ws_rows = (int)std::min<int64_t>(Bp, 512);
    m->ws_splits = (int)std::max<int64_t>(2, std::min<int64_t>(16, ((int64_t)32 << 20) / ((int64_t)m->ws_rows * h * 4)));
    bool ok = mlp_alloc(m, m->P, m->np) && mlp_alloc(m, m->G, m->np) && mlp_alloc(m, m->Mo, m->np) &&
              mlp_alloc(m, m->Vo, m->np) && mlp_alloc(m, m->Pb, m->np) && mlp_alloc(m, m->W2t, h * h) &&
              mlp_alloc(m, m->W3t, h * Qp) && mlp_alloc(m, m->Xf, Bp * n_in) && mlp_alloc(m, m->Tf, Bp * n_out) &&
              mlp_alloc(m, m->Z1, Bp * h) && mlp_alloc(m, m->Z2, Bp * h) && mlp_alloc(m, m->Y, Bp * Qp) &&
              mlp_alloc(m, m->dY, Bp * Qp) && mlp_alloc(m, m->dA2, Bp * h) && mlp_alloc(m, m->dZ2, Bp * h) &&
              mlp_alloc(m, m->dA1, Bp * h) && mlp_alloc(m, m->dZ1, Bp * h) && mlp_alloc(m, m->loss, 1) &&
              mlp_alloc(m, m->part, std::max((Bp + 31) / 32 * h, Bp / 8 * Qp)) &&
              mlp_alloc(m, m->lpart, Bp / 8) &&
              mlp_alloc(m, m->count, std::max(h, Qp) / 32 + 2) &&
              mlp_alloc(m, m->ws, (int64_t)m->ws_rows * h * m->ws_splits) &&
              mlp_alloc(m, m->Xb, Bp * n_in) && mlp_alloc(m, m->Xt, Bp * n_in) && mlp_alloc(m, m->A1b, Bp * h) &&
              mlp_alloc(m, m->A1t, Bp * h) && mlp_alloc(m, m->A2b, Bp * h) && mlp_alloc(m, m->A2t, Bp * h) &&
              mlp_alloc(m, m->dYb, Bp * Qp) && mlp_alloc(m, m->dYt, Bp * Qp) && mlp_alloc(m, m->dZ2b, Bp * h) &&
              mlp_alloc(m, m->dZ2t, Bp * h) && mlp_alloc(m, m->dZ1b, Bp * h) && mlp_alloc(m, m->dZ1t, Bp * h);
    if (!ok) {
        mlp_free(m);
        delete m;
        return mlp_fail(SAS_ERR_ALLOC, "device allocation failed");
    }
    if (cudaMemset(m->P, 0, sizeof(float) * m->np) != cudaSuccess ||
        cudaMemset(m->Mo, 0, sizeof(float) * m->np) != cudaSuccess ||
        cudaMemset(m->Vo, 0, sizeof(float) * m->np) != cudaSuccess ||
        cudaMemset(m->G, 0, sizeof(float) * m->np) != cudaSuccess ||
        cudaMemset(m->count, 0, sizeof(unsigned) * (size_t)(std::max(h, Qp) / 32 + 2)) != cudaSuccess ||
        mlp_refresh(m, 0) != SAS_OK ||
        cudaStreamSynchronize(0) != cudaSuccess) {
        cudaGetLastError();
        mlp_free(m);
        delete m;
        return mlp_fail(SAS_ERR_CUDA, "initialisation failed");
    }
    *out = m;
    return SAS_OK;
}

sas_status sas_mlp_destroy(sas_mlp *m)
{
    if (!m) return SAS_OK;
    cudaDeviceSynchronize();
    for (auto &g : m->step_graphs) cudaGraphExecDestroy(g.second);
    m->step_graphs.clear();
    if (m->capture_stream) cudaStreamDestroy(m->capture_stream);
    m->capture_stream = nullptr;
    mlp_free(m);
    delete m;
    return SAS_OK;
}

int64_t sas_mlp_param_count(const sas_mlp *m) { return m ? packed_count(m) : 0; }

sas_status sas_mlp_set_state(sas_mlp *m, const float *params, const float *adam_m, const float *adam_v,
                             int64_t step)
{
    if (!m || !params || step < 0) return mlp_fail(SAS_ERR_INVALID_ARG, "bad argument");
    std::vector<float> tmp((size_t)m->np);
    const float *src[3] = {params, adam_m, adam_v};
    float *dst[3] = {m->P, m->Mo, m->Vo};
    for (int k = 0; k < 3; ++k) {
        if (src[k])
            unpack_layout(m, src[k], tmp.data());
        else
            std::fill(tmp.begin(), tmp.end(), 0.f);
        MLP_TRY(cudaMemcpy(dst[k], tmp.data(), sizeof(float) * (size_t)m->np, cudaMemcpyHostToDevice));
    }
    m->step = step;
    sas_status st = mlp_refresh(m, 0);
    if (st != SAS_OK) return st;
    MLP_TRY(cudaStreamSynchronize(0));
    return SAS_OK;
}

sas_status sas_mlp_get_state(sas_mlp *m, float *params, float *adam_m, float *adam_v, int64_t *step)
{
    if (!m) return mlp_fail(SAS_ERR_INVALID_ARG, "null network");
    MLP_TRY(cudaDeviceSynchronize());
    sas_status st;
    if (params && (st = copy_block(m, m->P, params)) != SAS_OK) return st;
    if (adam_m && (st = copy_block(m, m->Mo, adam_m)) != SAS_OK) return st;
    if (adam_v && (st = copy_block(m, m->Vo, adam_v)) != SAS_OK) return st;
    if (step) *step = m->step;
    return SAS_OK;
}

sas_status sas_mlp_forward(sas_mlp *m, const float *x, int batch, float *y, void *stream)
{
    sas::NvtxRange nvtx_range("sas_mlp_forward");
    if (!m || !x || !y) return mlp_fail(SAS_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    sas_status st = mlp_forward(m, x, nullptr, batch, s);
    if (st != SAS_OK) return st;
    const bool host = !on_device_ptr(y);
    MLP_TRY(cudaMemcpy2DAsync(y, sizeof(float) * m->n_out, m->Y, sizeof(float) * m->n_outp, sizeof(float) * m->n_out,
                              batch, host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    if (host) {
        MLP_TRY(cudaStreamSynchronize(s));
        return gemm_check();
    }
    return SAS_OK;
}

sas_status sas_mlp_grads(sas_mlp *m, const float *x, const float *t, int batch, float *grads, float *loss_out,
                         void *stream)
{
    sas::NvtxRange nvtx_range("sas_mlp_grads");
    if (!m || !x || !t) return mlp_fail(SAS_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    sas_status st = mlp_forward(m, x, t, batch, s);
    if (st == SAS_OK) st = mlp_backward(m, batch, s);
    if (st != SAS_OK) return st;
    MLP_TRY(cudaStreamSynchronize(s));
    if ((st = gemm_check()) != SAS_OK) return st;
    if (grads && (st = copy_block(m, m->G, grads)) != SAS_OK) return st;
    if (loss_out) MLP_TRY(cudaMemcpy(loss_out, m->loss, sizeof(float), cudaMemcpyDefault));
    return SAS_OK;
}

sas_status sas_mlp_train_step(sas_mlp *m, const float *x, const float *t, int batch, float lr, float *loss_out,
                              void *stream)
{
    sas::NvtxRange nvtx_range("sas_mlp_train_step");
    if (!m || !x || !t) return mlp_fail(SAS_ERR_INVALID_ARG, "null argument");
    if (!(lr > 0.f) || !std::isfinite(lr)) return mlp_fail(SAS_ERR_INVALID_ARG, "learning rate must be positive");
    cudaStream_t s = (cudaStream_t)stream;
    // inputs into Xf and Tf, then the captured forward and backward launches (the same kernels in the
    // same order as sas_mlp_grads), then Adam, which writes the bfloat16 copy of the masters itself
    sas_status st = mlp_forward(m, x, t, batch, s, true);
    if (st != SAS_OK) return st;
    cudaGraphExec_t ex = nullptr;
    if ((st = step_graph(m, batch, ex)) != SAS_OK) return st;
    MLP_TRY(cudaGraphLaunch(ex, s));
    m->step += 1;
    MLP_TRY(launch_adam(m->np, m->P, m->G, m->Mo, m->Vo, lr, 0.9f, 0.999f, 1e-8f, m->step, m->Pb, s));
    st = mlp_refresh(m, s, false);
    if (st != SAS_OK) return st;
    if (loss_out) {
        const bool host = !on_device_ptr(loss_out);
        MLP_TRY(cudaMemcpyAsync(loss_out, m->loss, sizeof(float), host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                s));
        if (host) {
            MLP_TRY(cudaStreamSynchronize(s));
            return gemm_check();
        }
    }
    return SAS_OK;
}

sas_status sas_mlp_read_buffer(sas_mlp *m, int which, int batch, float *out, int *width_out)
{
    if (!m || !out) return mlp_fail(SAS_ERR_INVALID_ARG, "null argument");
    if (batch < 1 || batch > m->max_b) return mlp_fail(SAS_ERR_INVALID_ARG, "batch outside [1, max_batch]");
    const int h = m->h, Qp = m->n_outp;
    // (buffer, row stride, width, bfloat16?) per SAS_MLP_BUF_* value
    const void *src = nullptr;
    int ld = 0, width = 0;
    bool is_bf16 = false;
    switch (which) {
    case SAS_MLP_BUF_XB: src = m->Xb, ld = m->n_in, width = m->n_in, is_bf16 = true; break;
    case SAS_MLP_BUF_Z1: src = m->Z1, ld = h, width = h; break;
    case SAS_MLP_BUF_A1B: src = m->A1b, ld = h, width = h, is_bf16 = true; break;
    case SAS_MLP_BUF_Z2: src = m->Z2, ld = h, width = h; break;
    case SAS_MLP_BUF_A2B: src = m->A2b, ld = h, width = h, is_bf16 = true; break;
    case SAS_MLP_BUF_Y: src = m->Y, ld = Qp, width = m->n_out; break;
    case SAS_MLP_BUF_DY: src = m->dY, ld = Qp, width = m->n_out; break;
    case SAS_MLP_BUF_DYB: src = m->dYb, ld = Qp, width = m->n_out, is_bf16 = true; break;
    case SAS_MLP_BUF_DA2: src = m->dA2, ld = h, width = h; break;
    case SAS_MLP_BUF_DZ2: src = m->dZ2, ld = h, width = h; break;
    case SAS_MLP_BUF_DZ2B: src = m->dZ2b, ld = h, width = h, is_bf16 = true; break;
    case SAS_MLP_BUF_DA1: src = m->dA1, ld = h, width = h; break;
    case SAS_MLP_BUF_DZ1: src = m->dZ1, ld = h, width = h; break;
    case SAS_MLP_BUF_DZ1B: src = m->dZ1b, ld = h, width = h, is_bf16 = true; break;
    default: return mlp_fail(SAS_ERR_INVALID_ARG, "unknown buffer");
    }
    MLP_TRY(cudaDeviceSynchronize());
    sas_status st = gemm_check();
    if (st != SAS_OK) return st;
    const size_t n = (size_t)batch * width, esz = is_bf16 ? sizeof(bf16) : sizeof(float);
    std::vector<float> host(n);
    if (is_bf16) {
        std::vector<bf16> tmp(n);
        MLP_TRY(cudaMemcpy2D(tmp.data(), esz * width, src, esz * ld, esz * width, batch, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) host[i] = __bfloat162float(tmp[i]);
    } else {
        MLP_TRY(cudaMemcpy2D(host.data(), esz * width, src, esz * ld, esz * width, batch, cudaMemcpyDeviceToHost));
    }
    MLP_TRY(cudaMemcpy(out, host.data(), sizeof(float) * n, cudaMemcpyDefault));
    if (width_out) *width_out = width;
    return SAS_OK;
}

sas_status sas_gemm_bf16(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias, float *C,
                         int ldc, void *stream)
{
    if (M < 0 || N < 0 || K < 0 || K % 16 || lda % 8 || ldb % 8 || lda < K || ldb < K || ldc < N)
        return mlp_fail(SAS_ERR_INVALID_ARG, "sizes: K % 16 == 0, lda and ldb multiples of 8 and >= K, ldc >= N");
    if ((M && N && K) && (!A || !B || !C)) return mlp_fail(SAS_ERR_INVALID_ARG, "null argument");
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15)
        return mlp_fail(SAS_ERR_INVALID_ARG, "A and B must be 16-byte aligned");
    MLP_TRY(launch_gemm(M, N, K, A, lda, B, ldb, bias, C, ldc, nullptr, 0, 0, (cudaStream_t)stream));
    return SAS_OK;
}

}  // extern "C"

// C ABI of the proposal network: create, weights in/out, forward, loss and
// gradient, Adam training over logged bond-formation events.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <random>
#include <vector>

#include "../../include/snap.h"
#include "snap_mlp.h"

using snap::kMlpParams;

namespace {

snap_status grow_rows(snap_mlp *m, long long rows)
{
    if (rows <= m->cap_rows) return SNAP_OK;
    cudaFree(m->y);
    cudaFree(m->dy);
    m->y = m->dy = nullptr;
    const long long cap = std::max<long long>(rows, 1024);
    if (cudaMalloc(&m->y, sizeof(float) * cap) != cudaSuccess || cudaMalloc(&m->dy, sizeof(float) * cap) != cudaSuccess) {
        cudaGetLastError();
        m->cap_rows = 0;
        return SNAP_ERR_OOM;
    }
    m->cap_rows = cap;
    return SNAP_OK;
}

}  // namespace

extern "C" snap_status snap_mlp_create(snap_mlp **out, void *stream)
{
    if (!out) return SNAP_ERR_ARG;
    *out = nullptr;
    snap_mlp *m = new snap_mlp();
    m->stream = static_cast<cudaStream_t>(stream);
    bool ok = cudaMalloc(&m->dev.w, sizeof(float) * kMlpParams) == cudaSuccess &&
              cudaMalloc(&m->dev.grad, sizeof(float) * kMlpParams) == cudaSuccess &&
              cudaMalloc(&m->dev.m, sizeof(float) * kMlpParams) == cudaSuccess &&
              cudaMalloc(&m->dev.v, sizeof(float) * kMlpParams) == cudaSuccess &&
              cudaMalloc(&m->loss, sizeof(double)) == cudaSuccess;
    if (ok) {
        ok = cudaMemsetAsync(m->dev.w, 0, sizeof(float) * kMlpParams, m->stream) == cudaSuccess &&
             cudaMemsetAsync(m->dev.grad, 0, sizeof(float) * kMlpParams, m->stream) == cudaSuccess &&
             cudaMemsetAsync(m->dev.m, 0, sizeof(float) * kMlpParams, m->stream) == cudaSuccess &&
             cudaMemsetAsync(m->dev.v, 0, sizeof(float) * kMlpParams, m->stream) == cudaSuccess &&
             snap::mlp_configure() == cudaSuccess && cudaStreamSynchronize(m->stream) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        snap_mlp_destroy(m);
        return SNAP_ERR_CUDA;
    }
    *out = m;
    return SNAP_OK;
}

extern "C" snap_status snap_mlp_set_weights(snap_mlp *m, const float *w)
{
    if (!m || !w) return SNAP_ERR_ARG;
    if (cudaMemcpyAsync(m->dev.w, w, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->dev.m, 0, sizeof(float) * kMlpParams, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->dev.v, 0, sizeof(float) * kMlpParams, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->dev.grad, 0, sizeof(float) * kMlpParams, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        return SNAP_ERR_CUDA;
    }
    m->adam_t = 0;
    return SNAP_OK;
}

extern "C" snap_status snap_mlp_get_weights(snap_mlp *m, float *w)
{
    if (!m || !w) return SNAP_ERR_ARG;
    if (cudaMemcpyAsync(w, m->dev.w, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        return SNAP_ERR_CUDA;
    }
    return SNAP_OK;
}

extern "C" snap_status snap_mlp_forward(snap_mlp *m, const float *d_feat, int64_t rows, float *d_logits)
{
    if (!m || rows < 0 || (rows > 0 && (!d_feat || !d_logits))) return SNAP_ERR_ARG;
    if (snap::mlp_forward(m->dev, d_feat, rows, d_logits, m->stream) != cudaSuccess) return SNAP_ERR_CUDA;
    return SNAP_OK;
}

extern "C" snap_status snap_mlp_loss_grad(snap_mlp *m, const float *d_feat, int64_t rows, const int32_t *d_offsets,
                                          const int32_t *d_labels, int64_t events, double *loss, float *grad)
{
    if (!m || rows < 0 || events < 0 || (events > 0 && (!d_feat || !d_offsets || !d_labels))) return SNAP_ERR_ARG;
    snap_status st = grow_rows(m, rows);
    if (st != SNAP_OK) return st;
    if (cudaMemsetAsync(m->dev.grad, 0, sizeof(float) * kMlpParams, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->loss, 0, sizeof(double), m->stream) != cudaSuccess ||
        snap::mlp_loss_grad(m->dev, d_feat, rows, d_offsets, 0, d_labels, events, m->y, m->dy, m->loss,
                            m->stream) != cudaSuccess) {
        cudaGetLastError();
        return SNAP_ERR_CUDA;
    }
    double l = 0.0;
    if (cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        (grad && cudaMemcpyAsync(grad, m->dev.grad, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost,
                                 m->stream) != cudaSuccess) ||
        cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        return SNAP_ERR_CUDA;
    }
    if (loss) *loss = events > 0 ? l / (double)events : 0.0;
    return SNAP_OK;
}

extern "C" snap_status snap_mlp_train(snap_mlp *m, const float *d_feat, int64_t rows, const int32_t *d_offsets,
                                      const int32_t *d_labels, int64_t events, int32_t epochs, int64_t batch_events,
                                      float lr, uint64_t seed, double *losses)
{
    if (!m || rows < 0 || events <= 0 || epochs < 1 || batch_events < 1 || !(lr > 0.f) || !d_feat ||
        !d_offsets || !d_labels)
        return SNAP_ERR_ARG;
    std::vector<int32_t> off(events + 1);
    if (cudaMemcpyAsync(off.data(), d_offsets, sizeof(int32_t) * (events + 1), cudaMemcpyDeviceToHost, m->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        return SNAP_ERR_CUDA;
    }
    if (off[0] != 0 || off[events] != rows) return SNAP_ERR_ARG;
    const long long nb = (events + batch_events - 1) / batch_events;
    long long max_rows = 0;
    for (long long b = 0; b < nb; ++b) {
        const long long e0 = b * batch_events, e1 = std::min<long long>(events, e0 + batch_events);
        max_rows = std::max<long long>(max_rows, off[e1] - off[e0]);
    }
    snap_status st = grow_rows(m, max_rows);
    if (st != SNAP_OK) return st;
    std::vector<long long> order(nb);
    std::iota(order.begin(), order.end(), 0);
    std::mt19937_64 rng(seed);
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(order.begin(), order.end(), rng);
        if (cudaMemsetAsync(m->loss, 0, sizeof(double), m->stream) != cudaSuccess) return SNAP_ERR_CUDA;
        for (long long bi : order) {
            const long long e0 = bi * batch_events, e1 = std::min<long long>(events, e0 + batch_events);
            const long long r0 = off[e0], nr = off[e1] - off[e0];
            if (snap::mlp_loss_grad(m->dev, d_feat + r0 * snap::kMlpFeatures, nr, d_offsets + e0, (int32_t)r0,
                                    d_labels + e0, e1 - e0, m->y, m->dy, m->loss, m->stream) != cudaSuccess ||
                snap::mlp_adam(m->dev, lr, ++m->adam_t, m->stream) != cudaSuccess) {
                cudaGetLastError();
                return SNAP_ERR_CUDA;
            }
        }
        double l = 0.0;
        if (cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
            cudaStreamSynchronize(m->stream) != cudaSuccess) {
            cudaGetLastError();
            return SNAP_ERR_CUDA;
        }
        // the loss kernel accumulates per-event cross-entropies: mean over the epoch
        if (losses) losses[ep] = l / (double)events;
    }
    return SNAP_OK;
}

extern "C" void snap_mlp_destroy(snap_mlp *m)
{
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    cudaFree(m->dev.w);
    cudaFree(m->dev.grad);
    cudaFree(m->dev.m);
    cudaFree(m->dev.v);
    cudaFree(m->y);
    cudaFree(m->dy);
    cudaFree(m->loss);
    delete m;
}

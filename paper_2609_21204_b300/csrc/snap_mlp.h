// Proposal network (12 -> 64 -> 64 -> 1, ReLU) shared by the MLP kernels,
// its C ABI and the Metropolis–Hastings sweep.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace snap {

constexpr int kMlpFeatures = 12;
constexpr int kMlpParams = 16 * 64 + 64 + 64 * 64 + 64 + 64 + 1;   // 5313

struct MlpDev {
    float *w;      // FP32 master parameters (packed, see mlp.cu)
    float *grad;   // gradient accumulator (zeroed by each Adam step)
    float *m, *v;  // Adam moments
};

size_t mlp_forward_smem();
size_t mlp_backward_smem();
cudaError_t mlp_configure();
cudaError_t mlp_forward(const MlpDev &M, const float *X, long long rows, float *y, cudaStream_t s);
// the same with the row count read on the device (at most max_rows rows)
cudaError_t mlp_forward_counted(const MlpDev &M, const float *X, const int32_t *rows_dev, long long max_rows,
                                float *y, cudaStream_t s);
cudaError_t mlp_loss_grad(const MlpDev &M, const float *X, long long rows, const int32_t *off, int32_t row_base,
                          const int32_t *label, long long events, float *y, float *dy, double *loss_sum,
                          cudaStream_t s);
cudaError_t mlp_adam(const MlpDev &M, float lr, int t, cudaStream_t s);

}  // namespace snap

// the network object behind the C ABI (also read by the MH sweep)
struct snap_mlp {
    snap::MlpDev dev{};
    cudaStream_t stream = nullptr;
    float *y = nullptr, *dy = nullptr;   // per-row scratch
    long long cap_rows = 0;
    double *loss = nullptr;
    int adam_t = 0;
};

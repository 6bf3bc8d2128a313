// gc_neural.h -- the neural field's state on the device and its host entry points
// (gc_neural.cu): parameters, evaluation, training targets, loss and gradient, Adam.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gc_siren.h"

namespace gcn {

// Grid the training targets are interpolated from (the loaded field, node-centred,
// [phi][theta][r][8], FP32 or FP64).
struct GridRef {
    const void *nodes;
    int is_f64;
    int n_r, n_th, n_ph;
    double r_min, dr;
};

struct Neural {
    bool ready = false;
    float *P = nullptr;   // FP32 master parameters
    float *G = nullptr;   // gradient, same layout
    float *Mo = nullptr;  // Adam first moment
    float *Vo = nullptr;  // Adam second moment
    __nv_bfloat16 *Wh = nullptr;  // W2..W4 in BF16, [3][256][256]
    __nv_bfloat16 *W5p = nullptr; // W5 in BF16 padded to 16 rows
    gcs::SirenNet net{};
    double omega0 = 30.0, r_max = 0.0, B_scale = 1.0, E_scale = 1.0;
    int64_t adam_t = 0;

    // per-batch work buffers of the training (rows = samples)
    int64_t wcap = 0;
    float *Z = nullptr;          // 4 x wcap x 256 pre-activations z_1..z_4
    __nv_bfloat16 *H = nullptr;  // 4 x wcap x 256 activations h_1..h_4
    __nv_bfloat16 *dZ = nullptr; // wcap x 256
    float *dH = nullptr;         // wcap x 256
    double *d_loss = nullptr;    // [1]
    int *d_err = nullptr;        // error word of the fused evaluation

    // fit: samples and targets
    float *Xs = nullptr, *Ts = nullptr;
    int64_t scap = 0;
};

cudaError_t neural_free(Neural &nn);
// load parameters (host or device, kSirenNParams floats) and the scaling; resets Adam
cudaError_t neural_set(Neural &nn, const float *params, bool on_device, double omega0, double r_max,
                       double B_scale, double E_scale, cudaStream_t s);
// raw outputs y (n x 8) and optionally J (n x 8 x 3), or the physical field (n x 24)
cudaError_t neural_eval(Neural &nn, const float *x, int64_t n, float *y, float *J, cudaStream_t s);
cudaError_t neural_field(Neural &nn, const float *x, int64_t n, float *field, cudaStream_t s);
// field samples for the push: R (cap x 3, metres), point count on the device (n_dev, or cap
// when null), samples with `stride` floats per point
cudaError_t neural_field_at(Neural &nn, const float *R, int64_t cap, const int32_t *n_dev, float *samples,
                            int stride, cudaStream_t s);
// scaled 8-channel targets of the grid interpolant at x (n x 3, scaled by r_max)
cudaError_t neural_targets(const Neural &nn, const GridRef &g, const float *x, int64_t n, float *t,
                           cudaStream_t s);
// mean-squared error over n samples (n a multiple of 128) and its gradient into grad (or nn.G)
cudaError_t neural_loss_grad(Neural &nn, const float *x, const float *t, int64_t n, float *grad, double *loss,
                             cudaStream_t s);
// error word of the fused evaluation (0 = none); reading clears it (synchronises s)
int neural_read_error(Neural &nn, cudaStream_t s);
// one Adam step on nn.G
cudaError_t neural_adam(Neural &nn, double lr, double beta1, double beta2, double eps, cudaStream_t s);
// training: targets from the grid, then n_epochs passes of batches (the last partial batch
// is dropped); loss_out[e] = mean batch loss of epoch e before each update
cudaError_t neural_fit(Neural &nn, const GridRef &g, const float *samples, bool on_device, int64_t n_samples,
                       int64_t batch, int n_epochs, double lr, double beta1, double beta2, double eps,
                       float *loss_out, cudaStream_t s);

} // namespace gcn

// Tile-planner network on the GPU (kernels_mlp.cu): host pointers in and out; device
// workspace is allocated per call.
#pragma once

#include <cuda_runtime.h>

namespace oc {

int mlp_nparams();
cudaError_t mlp_forward(const float* params, const float* X, int n, float* Y);
cudaError_t mlp_loss_grad(const float* params, const float* X, const float* T, int n, float* grad,
                          double* loss);
// Full-batch Adam for `epochs` steps, updating params in place; loss_hist (optional) gets
// the loss before each step.
cudaError_t mlp_train(float* params, const float* X, const float* T, int n, int epochs, float lr,
                      float* loss_hist);

}  // namespace oc

// fr_mlp.cuh -- launch interface of the learned adaptation indicator (fr_mlp.cu).
#pragma once
#include "fr_internal.cuh"

namespace frg {

constexpr int MLP_HIDDEN = 64;

int mlp_param_count(int in);
// input width: 2 * 3^dim + 1
int mlp_in_dim(int dim);
// features [M][mlp_in_dim] (BF16) of the FP64 state
int mlp_features(int dim, int p, const double* u, const uint64_t* keys, int64_t M, const KG& g,
                 int Dbase, double gamma, const DevOps& ops, void* d_X, cudaStream_t s, Err* err);
// logits [n][3] and/or flags (argmax - 1) of n feature rows (1 <= in <= 64), on the tensor
// cores; *d_status becomes nonzero if a tensor-core completion wait gave up
// bound (clock cycles) of the inference kernel's completion waits; <= 0 restores the default
void mlp_set_wait_cycles(long long cycles);
int mlp_forward(const float* d_params, int in, const void* d_X, int64_t n, float* d_logits,
                int8_t* d_flags, int* d_status, cudaStream_t s, Err* err);
// cw[0..2] class weights (coarsen, keep, refine), cw[3] = 1 / (sum over the batch of w_label)
int mlp_grad(const float* d_params, int in, const void* d_X, const int8_t* d_y, int64_t B,
             const float* cw, float* d_grad, float* d_loss, Alloc& A, cudaStream_t s, Err* err);
int mlp_train_step(float* d_params, float* d_m, float* d_v, int64_t step, int in, const void* d_X,
                   const int8_t* d_y, int64_t B, const float* cw, float lr, float* d_loss,
                   Alloc& A, cudaStream_t s, Err* err);

}  // namespace frg

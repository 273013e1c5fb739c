// Learned smoother (mlp.cu): parameter layout and host-side helpers.
#pragma once

#include <cuda_bf16.h>

#include "ops.cuh"

namespace cpm {

// FP32 parameter vector: W1 (32 x 64, row 31 = zero feature), b1 (64),
// W2 (64 x 64), b2 (64), w3 (64), b3 (1); W[k][n] at k * 64 + n.
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + 32 * 64;
constexpr int kOffW2 = kOffB1 + 64;
constexpr int kOffB2 = kOffW2 + 64 * 64;
constexpr int kOffW3 = kOffB2 + 64;
constexpr int kOffB3 = kOffW3 + 64;
constexpr int kNParams = kOffB3 + 1;

// Per-level static inputs of the network: 27-neighbourhood indices and the
// geometric features (cp offset, dx^2 M_ii).
struct MlpLevelData {
  int32_t nB = 0;
  DBuf<int32_t> nbr27;
  DBuf<float> stat;
  void build(const Level& lev, const double* diagM, cudaStream_t st);
};

struct MlpTrainBuffers {
  int32_t n = -1;
  int64_t np = -1;
  int nparts = 0;
  DBuf<__nv_bfloat16> Xs, H1, H2;
  DBuf<float> S, du, Mdu, z, w, t, et, dy, part, grad;
  DBuf<double> lpart, loss;
  void ensure(int32_t nB, int64_t nplus);
};

// du = network correction of residual r (u_add != null: u_add += du instead);
// tb != null also stores the activations for the backward pass.
void mlp_forward(const float* params, const MlpLevelData& D, const float* r, float dx2, float* du,
                 float* u_add, const MlpTrainBuffers* tb, cudaStream_t st);
// Loss ||r - A du||^2 / ||r||^2 (tb.loss: [||z||^2, ||r||^2]) and gradient (tb.grad).
void mlp_loss_grad(const float* params, const MlpLevelData& D, const LevelView<float>& L,
                   const float* cvec, float cval, const float* r, MlpTrainBuffers& tb,
                   cudaStream_t st);
void mlp_adam(float* params, const float* grad, float* m, float* v, int64_t step, float lr,
              cudaStream_t st);

}  // namespace cpm

struct cpm_mlp_s {
  cpm::DBuf<float> params, m, v;
  int64_t step = 0;
  cpm::MlpTrainBuffers tb;
};

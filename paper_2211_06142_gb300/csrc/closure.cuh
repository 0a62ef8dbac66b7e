// closure.cuh -- layout of the learned-closure network's parameter vector.
//
// Network: 5 inputs -> 3 hidden layers of 64 SiLU units -> 2 outputs.
// Parameter vector (FP32): mu[5], inv_sigma[5] (input standardisation
// x_hat = (x - mu) * inv_sigma), then per layer the weights W[out][in] row
// by row followed by the biases b[out].
#pragma once

namespace closure {

constexpr int N_IN = 5, N_H = 64, N_OUT = 2;
constexpr int OFF_MU = 0;
constexpr int OFF_ISG = OFF_MU + N_IN;
constexpr int OFF_W1 = OFF_ISG + N_IN;
constexpr int OFF_B1 = OFF_W1 + N_H * N_IN;
constexpr int OFF_W2 = OFF_B1 + N_H;
constexpr int OFF_B2 = OFF_W2 + N_H * N_H;
constexpr int OFF_W3 = OFF_B2 + N_H;
constexpr int OFF_B3 = OFF_W3 + N_H * N_H;
constexpr int OFF_W4 = OFF_B3 + N_H;
constexpr int OFF_B4 = OFF_W4 + N_OUT * N_H;
constexpr int N_PARAMS = OFF_B4 + N_OUT;
static_assert(N_PARAMS == 8844, "parameter vector length");

}  // namespace closure

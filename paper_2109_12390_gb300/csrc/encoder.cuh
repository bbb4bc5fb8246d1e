// Encoder network of Section 4.1 / Table 1 (trained with the decoder in place of the latent
// table): shape bookkeeping and the launches train.cu uses.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace mpmrom {

constexpr int kEncKernel = 6;        // convolution kernel size (Table 1)
constexpr int kEncStride = 2;        // convolution stride (Table 1)
constexpr int kEncFC = 32;           // width of the first fully connected layer (Table 1)
constexpr int kEncMinLen = 32;       // convolutions stop before the length drops below this
constexpr int kEncMaxConv = 12;
constexpr int kEncMaxL0 = 8192;      // d x subset size
constexpr int kEncThreads = 256;

// Parameter vector: per convolution l, w_l[0..5] then b_l (7 floats); W1 (32 x d_conv, row-major);
// b1 (32); W2 (r x 32, row-major); b2 (r).
struct EncDesc {
  int d, r, n_sub, n_conv, act;
  int L[kEncMaxConv + 1];   // L[0] = d n_sub, L[l + 1] = (L[l] - 6) / 2 + 1
  int oW1, ob1, oW2, ob2;
  int n_params;
};

// Fills the shape of an encoder over n_sub particles; false if the shape is not supported.
bool enc_describe(int d, int r, int n_sub, int act, EncDesc* e);

// Shared-memory limits of the encoder kernels for this shape (outside stream capture).
mpm_status enc_prepare(const EncDesc& e);
// Standardised, particle-major encoder inputs U (n, L0) of snapshots whose particle rows are
// row_base[s] .. row_base[s + 1] - 1 of x (d floats each): subset particle j of snapshot s is row
// row_base[s] + floor(j P_s / n_sub); shift_scale = [shift (d), scale (d)] on the device.
mpm_status enc_gather(const EncDesc& e, const float* x, const int64_t* row_base, int64_t n, const float* shift_scale,
                      float* U, cudaStream_t s);
// Per-coordinate mean and standard deviation of the subset positions (FP64 sums; work holds 2 d
// doubles), written as shift_scale on the device.
mpm_status enc_moments(const EncDesc& e, const float* x, const int64_t* row_base, int64_t n, double* work,
                       float* shift_scale, cudaStream_t s);
// latents (n, r) = enc(U)
mpm_status enc_forward(const EncDesc& e, const float* params, const float* U, int64_t n, float* latents, int n_sm,
                       cudaStream_t s);
// grads (n_params) += d/dparams sum_s g_lat[s] . enc(U[s])
mpm_status enc_backward(const EncDesc& e, const float* params, const float* U, int64_t n, const float* g_lat,
                        float* grads, int n_sm, cudaStream_t s);

}  // namespace mpmrom

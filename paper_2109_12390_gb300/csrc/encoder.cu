// Encoder network (Section 4.1, Table 1) on the CUDA cores, FP32: the standardised, particle-major
// positions of a fixed particle subset of one snapshot pass through single-channel convolutions
// (kernel 6, stride 2, ELU) down to the last length >= 32, a 32-wide fully connected ELU layer and
// a linear layer to the r generalized coordinates.  Trained with the decoder: the decoder's
// per-snapshot latent gradients are pulled back through the encoder (enc_backward) and Adam moves
// its parameters instead of a latent table.
//
// One CTA works on one snapshot at a time (grid-stride over snapshots), all layer vectors in shared
// memory.  The backward kernel recomputes the forward pass of its snapshot, so no activations are
// stored between the launches; weight gradients are summed per CTA (fully connected entries in
// registers of the thread that owns them, convolution taps by warp reductions into shared memory)
// and added to the global gradient once per CTA.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "encoder.cuh"

namespace mpmrom {

namespace {

__device__ __forceinline__ float enc_act(int act, float z) { return act == 0 ? (z > 0.f ? z : expm1f(z)) : z; }
// derivative from the activation value h = act(z): ELU'(z) = 1 for z > 0, exp(z) = h + 1 otherwise
__device__ __forceinline__ float enc_act_d1_of_h(int act, float h) { return act == 0 ? (h > 0.f ? 1.f : h + 1.f) : 1.f; }

__global__ void enc_gather_kernel(EncDesc e, const float* __restrict__ x, const int64_t* __restrict__ row_base,
                                  int64_t n, const float* __restrict__ shift_scale, float* __restrict__ U) {
  const int L0 = e.L[0];
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * L0; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = q / L0;
    const int c = (int)(q - s * L0);
    const int j = c / e.d, a = c - j * e.d;
    const int64_t P = row_base[s + 1] - row_base[s];
    const int64_t row = row_base[s] + ((int64_t)j * P) / e.n_sub;
    U[q] = (x[row * e.d + a] - shift_scale[a]) / shift_scale[e.d + a];
  }
}

__global__ void enc_moments_kernel(EncDesc e, const float* __restrict__ x, const int64_t* __restrict__ row_base,
                                   int64_t n, double* work) {
  __shared__ double s_acc[6];
  if (threadIdx.x < 2 * e.d) s_acc[threadIdx.x] = 0.0;
  __syncthreads();
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * e.n_sub; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = q / e.n_sub;
    const int j = (int)(q - s * e.n_sub);
    const int64_t P = row_base[s + 1] - row_base[s];
    const int64_t row = row_base[s] + ((int64_t)j * P) / e.n_sub;
    for (int a = 0; a < e.d; ++a) {
      const double v = x[row * e.d + a];
      acc[a] += v;
      acc[3 + a] += v * v;
    }
  }
  for (int a = 0; a < e.d; ++a) {
    atomicAdd(&s_acc[a], acc[a]);
    atomicAdd(&s_acc[e.d + a], acc[3 + a]);
  }
  __syncthreads();
  if (threadIdx.x < 2 * e.d) atomicAdd(&work[threadIdx.x], s_acc[threadIdx.x]);
}

__global__ void enc_moments_finish(EncDesc e, int64_t count, const double* work, float* shift_scale) {
  const int a = threadIdx.x;
  if (a < e.d) {
    const double mean = work[a] / (double)count;
    const double var = fmax(work[e.d + a] / (double)count - mean * mean, 0.0);
    shift_scale[a] = (float)mean;
    shift_scale[e.d + a] = var > 0.0 ? (float)sqrt(var) : 1.f;
  }
}

// Forward pass of one snapshot held in h0 (L0 floats of shared memory).  With `keep`, layer l's
// output is written at h0 + off[l + 1] (off[0] = 0) and the fully connected activation at a;
// otherwise two buffers alternate.  Returns the buffer holding the last convolution's output.
__device__ float* enc_forward_one(const EncDesc& e, const float* __restrict__ P, float* h0, float* h1, bool keep,
                                  float* a) {
  float* cur = h0;
  float* nxt = keep ? h0 + e.L[0] : h1;
  for (int l = 0; l < e.n_conv; ++l) {
    const float* w = P + 7 * l;
    const float w0 = w[0], w1 = w[1], w2 = w[2], w3 = w[3], w4 = w[4], w5 = w[5], b = w[6];
    const int Lo = e.L[l + 1];
    for (int i = threadIdx.x; i < Lo; i += blockDim.x) {
      const float* hc = cur + kEncStride * i;
      float z = b;
      z = fmaf(w0, hc[0], z);
      z = fmaf(w1, hc[1], z);
      z = fmaf(w2, hc[2], z);
      z = fmaf(w3, hc[3], z);
      z = fmaf(w4, hc[4], z);
      z = fmaf(w5, hc[5], z);
      nxt[i] = enc_act(e.act, z);
    }
    __syncthreads();
    if (keep) {
      cur = nxt;
      nxt = cur + Lo;
    } else {
      float* t = cur;
      cur = nxt;
      nxt = t;
    }
  }
  // fully connected layer 1: warp w computes outputs w, w + 8, ...
  const int dc = e.L[e.n_conv];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int o = warp; o < kEncFC; o += nw) {
    const float* W = P + e.oW1 + o * dc;
    float acc = 0.f;
    for (int i = lane; i < dc; i += 32) acc = fmaf(W[i], cur[i], acc);
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
    if (lane == 0) a[o] = enc_act(e.act, acc + P[e.ob1 + o]);
  }
  __syncthreads();
  return cur;
}

__global__ void __launch_bounds__(kEncThreads) enc_forward_kernel(EncDesc e, const float* __restrict__ P,
                                                                   const float* __restrict__ U, int64_t n,
                                                                   float* __restrict__ latents) {
  extern __shared__ __align__(16) float esm[];
  const int L0 = e.L[0];
  float* h0 = esm;
  float* h1 = esm + L0;
  float* a = h1 + L0;
  for (int64_t s = blockIdx.x; s < n; s += gridDim.x) {
    for (int i = threadIdx.x; i < L0; i += blockDim.x) h0[i] = U[s * L0 + i];
    __syncthreads();
    enc_forward_one(e, P, h0, h1, false, a);
    // linear output layer: thread o < r
    if (threadIdx.x < e.r) {
      const float* W = P + e.oW2 + threadIdx.x * kEncFC;
      float acc = P[e.ob2 + threadIdx.x];
#pragma unroll 8
      for (int i = 0; i < kEncFC; ++i) acc = fmaf(W[i], a[i], acc);
      latents[s * e.r + threadIdx.x] = acc;
    }
    __syncthreads();
  }
}

constexpr int kEncFCPerThread = 16;   // fully connected parameters owned per thread (<= 16 x 256)

__global__ void __launch_bounds__(kEncThreads) enc_backward_kernel(EncDesc e, const float* __restrict__ P,
                                                                    const float* __restrict__ U, int64_t n,
                                                                    const float* __restrict__ g_lat,
                                                                    float* __restrict__ grads) {
  extern __shared__ __align__(16) float esm[];
  const int L0 = e.L[0];
  int off[kEncMaxConv + 2];
  off[0] = 0;
  for (int l = 0; l <= e.n_conv; ++l) off[l + 1] = off[l] + e.L[l];
  float* H = esm;                      // layer vectors h_0 .. h_{n_conv} back to back (off[])
  float* a = H + off[e.n_conv + 1];    // fully connected activation (32)
  float* g = a + kEncFC;               // latent gradient (r <= 32)
  float* dz1 = g + 32;                 // (32)
  float* D0 = dz1 + kEncFC;            // two gradient buffers (L0 floats each)
  float* D1 = D0 + L0;
  float* cacc = D1 + L0;               // convolution tap gradients (7 n_conv)
  const int t = threadIdx.x, lane = t & 31;
  for (int e7 = t; e7 < 7 * e.n_conv; e7 += blockDim.x) cacc[e7] = 0.f;
  const int dc = e.L[e.n_conv];
  const int nfc = e.n_params - e.oW1;
  // owned fully connected entries: index into P, and the two factors' shared-memory positions
  float facc[kEncFCPerThread];
  int fa_idx[kEncFCPerThread], fb_idx[kEncFCPerThread];   // factor 1 (dz1 or g), factor 2 (h_last or a; -1: 1)
#pragma unroll
  for (int q = 0; q < kEncFCPerThread; ++q) {
    facc[q] = 0.f;
    const int k = t + q * kEncThreads;
    fa_idx[q] = -1;
    fb_idx[q] = -1;
    if (k < nfc) {
      const int pidx = e.oW1 + k;
      if (pidx < e.ob1) {
        const int o = (pidx - e.oW1) / dc, i = (pidx - e.oW1) - o * dc;
        fa_idx[q] = 0 * 64 + o;              // dz1[o]
        fb_idx[q] = off[e.n_conv] + i;       // h_last[i]
      } else if (pidx < e.oW2) {
        fa_idx[q] = pidx - e.ob1;            // dz1[o]
      } else if (pidx < e.ob2) {
        const int o = (pidx - e.oW2) / kEncFC, i = (pidx - e.oW2) - o * kEncFC;
        fa_idx[q] = 64 + o;                  // g[o]
        fb_idx[q] = -2 - i;                  // a[i]
      } else {
        fa_idx[q] = 64 + (pidx - e.ob2);     // g[o]
      }
    }
  }
  __syncthreads();
  for (int64_t s = blockIdx.x; s < n; s += gridDim.x) {
    for (int i = t; i < L0; i += blockDim.x) H[i] = U[s * L0 + i];
    if (t < e.r) g[t] = g_lat[s * e.r + t];
    __syncthreads();
    enc_forward_one(e, P, H, nullptr, true, a);
    // d(xhat)/da and the first fully connected layer's pre-activation gradient
    if (t < kEncFC) {
      float da = 0.f;
      for (int o = 0; o < e.r; ++o) da = fmaf(P[e.oW2 + o * kEncFC + t], g[o], da);
      dz1[t] = da * enc_act_d1_of_h(e.act, a[t]);
    }
    __syncthreads();
    // owned fully connected entries
#pragma unroll
    for (int q = 0; q < kEncFCPerThread; ++q) {
      if (fa_idx[q] < 0) continue;
      const float f1 = fa_idx[q] < 64 ? dz1[fa_idx[q]] : g[fa_idx[q] - 64];
      const float f2 = fb_idx[q] == -1 ? 1.f : (fb_idx[q] <= -2 ? a[-2 - fb_idx[q]] : H[fb_idx[q]]);
      facc[q] = fmaf(f1, f2, facc[q]);
    }
    // gradient of the last convolution output
    float* dh = D0;
    float* dh_prev = D1;
    for (int i = t; i < dc; i += blockDim.x) {
      float acc = 0.f;
      for (int o = 0; o < kEncFC; ++o) acc = fmaf(P[e.oW1 + o * dc + i], dz1[o], acc);
      dh[i] = acc;
    }
    __syncthreads();
    for (int l = e.n_conv - 1; l >= 0; --l) {
      const int Lo = e.L[l + 1], Li = e.L[l];
      const float* hin = H + off[l];
      const float* hout = H + off[l + 1];
      // dz = dh * act'(z) in place
      for (int i = t; i < Lo; i += blockDim.x) dh[i] *= enc_act_d1_of_h(e.act, hout[i]);
      __syncthreads();
      // tap and bias gradients: thread partials, warp sums, one shared atomic per warp and tap
      float p[7] = {0, 0, 0, 0, 0, 0, 0};
      for (int i = t; i < Lo; i += blockDim.x) {
        const float dzi = dh[i];
        const float* hc = hin + kEncStride * i;
#pragma unroll
        for (int k = 0; k < kEncKernel; ++k) p[k] = fmaf(dzi, hc[k], p[k]);
        p[6] += dzi;
      }
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        float v = p[k];
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
        if (lane == 0) atomicAdd(&cacc[7 * l + k], v);
      }
      if (l > 0) {
        // gradient of the layer input: dh_prev[j] = sum over taps k with (j - k) even and
        // 0 <= (j - k) / 2 < Lo of w[k] dz[(j - k) / 2]
        const float* w = P + 7 * l;
        for (int j = t; j < Li; j += blockDim.x) {
          float acc = 0.f;
#pragma unroll
          for (int k = 0; k < kEncKernel; ++k) {
            const int m = j - k;
            if (m >= 0 && (m & 1) == 0 && (m >> 1) < Lo) acc = fmaf(w[k], dh[m >> 1], acc);
          }
          dh_prev[j] = acc;
        }
        __syncthreads();
        float* tmp = dh;
        dh = dh_prev;
        dh_prev = tmp;
      }
    }
    __syncthreads();
  }
  // per-CTA sums into the global gradient
#pragma unroll
  for (int q = 0; q < kEncFCPerThread; ++q)
    if (fa_idx[q] >= 0) atomicAdd(&grads[e.oW1 + t + q * kEncThreads], facc[q]);
  __syncthreads();
  for (int e7 = t; e7 < 7 * e.n_conv; e7 += blockDim.x) atomicAdd(&grads[e7], cacc[e7]);
}

size_t enc_fwd_smem(const EncDesc& e) { return (size_t)(2 * e.L[0] + kEncFC) * sizeof(float); }

size_t enc_bwd_smem(const EncDesc& e) {
  int tot = 0;
  for (int l = 0; l <= e.n_conv; ++l) tot += e.L[l];
  return (size_t)(tot + kEncFC + 32 + kEncFC + 2 * e.L[0] + 7 * e.n_conv) * sizeof(float);
}

}  // namespace

bool enc_describe(int d, int r, int n_sub, int act, EncDesc* e) {
  if (d < 2 || d > 3 || r < 1 || r > 32 || n_sub < 1) return false;
  EncDesc x{};
  x.d = d;
  x.r = r;
  x.n_sub = n_sub;
  x.act = act;
  x.L[0] = d * n_sub;
  if (x.L[0] > kEncMaxL0 || x.L[0] < kEncMinLen) return false;
  int nc = 0;
  while ((x.L[nc] - kEncKernel) / kEncStride + 1 >= kEncMinLen) {
    if (nc == kEncMaxConv) return false;
    x.L[nc + 1] = (x.L[nc] - kEncKernel) / kEncStride + 1;
    ++nc;
  }
  x.n_conv = nc;
  const int dc = x.L[nc];
  x.oW1 = 7 * nc;
  x.ob1 = x.oW1 + kEncFC * dc;
  x.oW2 = x.ob1 + kEncFC;
  x.ob2 = x.oW2 + r * kEncFC;
  x.n_params = x.ob2 + r;
  if (x.n_params - x.oW1 > kEncFCPerThread * kEncThreads) return false;
  *e = x;
  return true;
}

mpm_status enc_prepare(const EncDesc& e) {
  MPM_CUDA_TRY(
      cudaFuncSetAttribute(enc_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)enc_fwd_smem(e)));
  MPM_CUDA_TRY(
      cudaFuncSetAttribute(enc_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)enc_bwd_smem(e)));
  return MPM_OK;
}

mpm_status enc_gather(const EncDesc& e, const float* x, const int64_t* row_base, int64_t n, const float* shift_scale,
                      float* U, cudaStream_t s) {
  if (n <= 0) return MPM_OK;
  const int64_t tot = n * e.L[0];
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 65536);
  enc_gather_kernel<<<blocks, 256, 0, s>>>(e, x, row_base, n, shift_scale, U);
  MPM_CUDA_TRY(cudaGetLastError());
  return MPM_OK;
}

mpm_status enc_moments(const EncDesc& e, const float* x, const int64_t* row_base, int64_t n, double* work,
                       float* shift_scale, cudaStream_t s) {
  MPM_CUDA_TRY(cudaMemsetAsync(work, 0, sizeof(double) * 2 * e.d, s));
  const int64_t tot = n * e.n_sub;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 1024));
  enc_moments_kernel<<<blocks, 256, 0, s>>>(e, x, row_base, n, work);
  MPM_CUDA_TRY(cudaGetLastError());
  enc_moments_finish<<<1, 32, 0, s>>>(e, tot, work, shift_scale);
  MPM_CUDA_TRY(cudaGetLastError());
  return MPM_OK;
}

mpm_status enc_forward(const EncDesc& e, const float* params, const float* U, int64_t n, float* latents, int n_sm,
                       cudaStream_t s) {
  if (n <= 0) return MPM_OK;
  const size_t smem = enc_fwd_smem(e);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)n_sm * 4));
  enc_forward_kernel<<<blocks, kEncThreads, smem, s>>>(e, params, U, n, latents);
  MPM_CUDA_TRY(cudaGetLastError());
  return MPM_OK;
}

mpm_status enc_backward(const EncDesc& e, const float* params, const float* U, int64_t n, const float* g_lat,
                        float* grads, int n_sm, cudaStream_t s) {
  if (n <= 0) return MPM_OK;
  const size_t smem = enc_bwd_smem(e);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)n_sm * 2));
  enc_backward_kernel<<<blocks, kEncThreads, smem, s>>>(e, params, U, n, g_lat, grads);
  MPM_CUDA_TRY(cudaGetLastError());
  return MPM_OK;
}

}  // namespace mpmrom

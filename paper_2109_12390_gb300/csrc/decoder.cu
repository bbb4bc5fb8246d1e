// Implicit neural decoder g(X; xhat) (Section 3.1, Eq. kinematicRestriction;
// Section 4, Table 1) with its Jacobians (Eq. defGrad: dg/dX; Eq. timederOne:
// dg/dxhat) on sm_103a tensor cores.
//
// Network: h0 = act(W0 [Xn, xhat] + b0), h_l = act(W_l h_{l-1} + b_l) for the
// square hidden layers, y = Wout h + bout, g = out_scale * y + out_shift,
// Xn = (X - X_min) / X_range (min-max input scaling and output
// standardisation of Appendix B), act = ELU.
//
// Derivatives are propagated forward as extra rows of the same GEMMs: every
// point contributes R rows to a 128-row tile (kind-major: rows kind*Pt + q),
//   kind 0          primal              h = act(z)
//   tangent kinds   dg along an input direction   t = act'(z) . (W t_prev)
//   secant kind     g(xhat + delta) - g(xhat)     s = act(z + W s_prev) - act(z)
//   mixed kinds     d/d(input b) of the JVP row   m = act''(z) (W u)(W t) + act'(z) (W m_prev)
// where z is the primal pre-activation of the same point and, for a mixed row,
// W u and W t are the pre-activations of the JVP row and of the input-b tangent
// row of the same point; the pre-activations of a 32-column chunk are
// exchanged between the rows of a tile through shared memory.  The secant rows give differences of decoder outputs without
// the BF16 rounding of the two absolute evaluations (the Gauss-Newton
// residual needs differences far below BF16 resolution).
//
// Per tile: layer 0 (K = d + r <= 35) and the output layer (N = d) run in
// FP32 on the CUDA cores; each square 128 x 128 layer is one M=128, N=128,
// K=128 tcgen05.mma chain (BF16 operands from shared memory in the 128-byte
// swizzled K-major layout, FP32 accumulator in tensor memory), read back with
// tcgen05.ld for the bias/activation/tangent epilogue, which writes the next
// layer's BF16 operand tile in place.  All square-layer weights stay resident
// in shared memory (loaded once per CTA with bulk async copies); the kernel
// is persistent over tiles.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "tc.cuh"

#include "decoder_common.cuh"

namespace mpmrom {

// --------------------------------------------------------------------------
// Decoders without square layers (linear, or a single hidden layer): SIMT.
// --------------------------------------------------------------------------
__global__ void decoder_simt(DecArgs a) {
  const int64_t n = dec_count(a);
  const int64_t rows = n * a.R;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < rows; g += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(g / n);
    RowInfo ri;
    ri.p = g % n;
    ri.q = 0;
    ri.kind = a.kinds[k];
    ri.cls = kind_class(ri.kind);
    float in[40], dir[40];
    row_inputs(a, ri, in, dir);
    const int K = a.d + a.r;
    float y[3] = {0.f, 0.f, 0.f};
    if (a.linear) {
      // an affine map has no mixed second derivative
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (i >= a.d) break;
        float z = 0.f;
        if (ri.cls != 3)
          for (int c = 0; c < K; ++c) z = fmaf(a.W0[i * K + c], ri.cls == 0 ? in[c] : dir[c], z);
        y[i] = z + (ri.cls == 0 ? a.b0[i] : 0.f);
      }
    } else {
      for (int c = 0; c < kW; ++c) {
        float z = a.b0[c], zd = 0.f;
        for (int i = 0; i < K; ++i) {
          z = fmaf(a.W0[c * K + i], in[i], z);
          zd = fmaf(a.W0[c * K + i], dir[i], zd);
        }
        float h;
        if (ri.cls == 0) h = act_f(a.act, z);
        else if (ri.cls == 1) h = act_d1(a.act, z) * zd;
        else if (ri.cls == 2) h = act_sec(a.act, z, zd);
        else h = act_d2(a.act, z) * zd * mixed_t0(a, a.W0 + c * K, ri.kind);
#pragma unroll
        for (int i = 0; i < 3; ++i)
          if (i < a.d) y[i] = fmaf(a.Wout[i * kW + c], h, y[i]);
      }
      if (ri.cls == 0)
#pragma unroll
        for (int i = 0; i < 3; ++i)
          if (i < a.d) y[i] += a.bout[i];
    }
    float* o = a.out + ((int64_t)k * a.n + ri.p) * a.d;   // kind stride = capacity a.n
#pragma unroll
    for (int i = 0; i < 3; ++i)
      if (i < a.d) o[i] = y[i] * a.norm[3 * a.d + i] + (ri.cls == 0 ? a.norm[2 * a.d + i] : 0.f);
  }
}

// --------------------------------------------------------------------------
// Tensor-core decoder kernel: 256 threads.  Warps w and w + 4 read the same
// tensor-memory lane group (lanes 32 (w % 4) ..): thread t owns tile row
// rw = 32 (w % 4) + lane and the column half h = w / 4 (columns 64 h .. 64 h + 63)
// of every layer, so each row's epilogue is split over two warps.
// --------------------------------------------------------------------------
constexpr int kDecThreads = 256;
constexpr int kXbStride = 33;                            // padded row stride of the exchange
constexpr int kW0Stride = 40;                            // first-layer row stride (d + r <= 40)

__device__ __forceinline__ float elu_bf16_input(float z) {
  // ELU whose result feeds a BF16 operand (or the FP32 output layer): exp(z) - 1
  // with the fast exponential; its absolute error (~1e-7) is far below BF16
  // resolution of the activations
  return z > 0.f ? z : __expf(z) - 1.0f;
}

// The operand tile of the next square layer: BF16, or (split) the BF16 pair hi = bf16(v),
// lo = bf16(v - hi) in two tiles kLayerBytes apart.
template <bool SPLIT>
__device__ __forceinline__ void store_operand(uint8_t* tile, int row, int col, const float* v) {
  if (!SPLIT) {
    store_bf16x8(tile, row, col, v);
  } else {
    float hi[8], lo[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      hi[i] = __bfloat162float(__float2bfloat16_rn(v[i]));
      lo[i] = v[i] - hi[i];   // exact in FP32
    }
    store_bf16x8(tile, row, col, hi);
    store_bf16x8(tile + kLayerBytes, row, col, lo);
  }
}

// SPLIT = false: BF16 operands, all square layers resident in shared memory.
// SPLIT = true: FP32-accurate square layers from split BF16 operands (hi + lo for the
// activations and the weights), three MMAs per K step into the same FP32 accumulator,
//   A W ~ A_hi W_hi + A_hi W_lo + A_lo W_hi,
// the dropped A_lo W_lo term and the residuals of the splits being about 2^-16 of each product;
// the two weight images of one layer at a time are streamed into shared memory while the
// previous layer's epilogue runs, and the activations take the accurate exponential.
template <bool SPLIT>
__global__ void __launch_bounds__(kDecThreads, 1) decoder_tc(DecArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte alignment for the swizzled operand tiles
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* wsm = smem;                                   // n_tc x 32 KB (split: the current layer, hi and lo)
  uint8_t* atile = smem + (SPLIT ? 2 : kMaxTC) * kLayerBytes;  // 32 KB (split: hi and lo, 64 KB)
  // first layer: FP32 [128][kW0Stride], zero-padded (CUDA cores), or its 16 KB split BF16 image
  uint8_t* w0s = atile + (SPLIT ? 2 : 1) * kLayerBytes;
  float* sW0 = (float*)w0s;
  float* xb = sW0 + kW * kW0Stride;                      // [2 halves][128 rows][33]: one chunk per half
  float* ypart = xb + 2 * 128 * kXbStride;               // [128 rows][3]: output partial of half 1
  float* sb0 = ypart + 128 * 3;                          // [128]
  float* sbh = sb0 + kW;                                 // [kMaxTC][128] square-layer biases
  float* sWout = sbh + kMaxTC * kW;                      // [3][128] output layer
  DecSmemTail* tail = (DecSmemTail*)(sWout + 3 * kW);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int rw = (warp & 3) * 32 + lane;                 // tile row / tensor-memory lane
  const int h = warp >> 2;                               // column half

  if (t == 0) {
    tc::mbar_init(&tail->bar_w, 1);
    tc::mbar_init(&tail->bar_mma, 1);
    tail->abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc<kW>(&tail->tmem);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tail->tmem;

  // The first layer runs on the tensor cores when its inputs fit 32 entries of the padded layout:
  // z = W0 [in] from split BF16 pairs, in_hi W0_hi + in_hi W0_lo + in_lo W0_hi (FP32 accumulate),
  // the dropped products and the residuals of the splits about 2^-16 of each product.
  const int K0 = kTcLat + a.r;                           // first-layer inputs in the padded layout
  const bool l0_tc = !SPLIT && a.w0img != nullptr && K0 <= 32;

  // FP32 first layer (CUDA-core form), biases and output layer staged in shared memory (read by
  // every row of every tile)
  {
    const int K0s = a.d + a.r;
    // the tensor-core input layout (row_inputs_tc): coordinates at 0 .. 3, latents from kTcLat
    for (int e = t; e < (l0_tc ? 0 : kW * kW0Stride); e += kDecThreads) {
      const int c = e / kW0Stride, ii = e % kW0Stride;
      const int i = ii < kTcLat ? (ii < a.d ? ii : -1) : (ii - kTcLat < a.r ? a.d + ii - kTcLat : -1);
      sW0[e] = i >= 0 ? a.W0[c * K0s + i] : 0.f;
    }
    for (int e = t; e < kW; e += kDecThreads) sb0[e] = a.b0[e];
    for (int e = t; e < a.n_tc * kW; e += kDecThreads) sbh[e] = a.bh[e];
    for (int e = t; e < a.d * kW; e += kDecThreads) sWout[e] = a.Wout[e];
  }
  // resident weights of the square layers; split: the first layer's two images (thread 0 waits
  // for them before its first MMA)
  uint32_t w_phase = 0;
  bool w_pending = false;   // thread 0: a weight copy is in flight
  if (!SPLIT) {
    if (t == 0) {
      tc::mbar_expect_tx(&tail->bar_w, (uint32_t)(a.n_tc * kLayerBytes + (l0_tc ? kLayerBytes / 2 : 0)));
      for (int l = 0; l < a.n_tc; ++l)
        tc::bulk_g2s(wsm + l * kLayerBytes, a.wimg + (size_t)l * kLayerBytes, kLayerBytes, &tail->bar_w);
      if (l0_tc) tc::bulk_g2s(w0s, a.w0img, kLayerBytes / 2, &tail->bar_w);
    }
    if (!tc::mbar_wait(&tail->bar_w, 0)) {
      raise_status(a.status, STATUS_TIMEOUT);
      atomicExch(&tail->abort, 1);
    }
  } else if (t == 0) {
    tc::mbar_expect_tx(&tail->bar_w, (uint32_t)(2 * kLayerBytes));
    tc::bulk_g2s(wsm, a.wimg, kLayerBytes, &tail->bar_w);
    tc::bulk_g2s(wsm + kLayerBytes, a.wimg_lo, kLayerBytes, &tail->bar_w);
    w_pending = true;
  }
  __syncthreads();

  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, kW);
  uint32_t mma_phase = 0;
  const int64_t n_pts = dec_count(a);
  const int64_t n_tiles = (n_pts + a.Pt - 1) / a.Pt;
  float* xh = xb + h * 128 * kXbStride;                  // this half's exchange buffer

  for (int64_t tile = blockIdx.x; tile < n_tiles && !tail->abort; tile += gridDim.x) {
    const int64_t first = tile * a.Pt;
    const RowInfo ri = row_info(a, rw, first, n_pts);
    float in[40], dir[40];
    if (ri.cls >= 0) row_inputs_tc(a, ri, in, dir);

    if (l0_tc) {
      // ---- the first layer's operand row: the primal rows' input, the tangent and secant rows'
      // direction (their pre-activation tangent or increment), zero for the mixed rows (the first
      // layer is linear: their second-order part starts at zero) and the unused rows; half 0
      // stores the high parts at columns 0 .. 31, half 1 the low parts at 32 .. 63
#pragma unroll
      for (int c0 = 0; c0 < 32; c0 += 8) {
        float p[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float v = ri.cls == 0 ? in[c0 + j] : (ri.cls == 1 || ri.cls == 2) ? dir[c0 + j] : 0.f;
          const float hi = __bfloat162float(__float2bfloat16_rn(v));
          p[j] = h == 0 ? hi : v - hi;
        }
        store_bf16x8(atile, rw, 32 * h + c0, p);
      }
    } else
    // ---- layer 0 on the CUDA cores (FP32), this thread's 64 columns, 8 at a time
    for (int c0 = 64 * h; c0 < 64 * h + 64; c0 += 8) {
      // the 8 columns' sums advance together over the inputs (16 independent chains), so that
      // their FMAs and the broadcast weight loads overlap instead of running column by column
      float z[8], zd[8], hv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        z[j] = sb0[c0 + j];
        zd[j] = 0.f;
      }
      if (ri.cls == 0) {   // primal rows: no directional part
#pragma unroll
        for (int i4 = 0; i4 < kW0Stride / 4; ++i4) {
          if (4 * i4 < K0) {   // padded weights are zero, as are in[] and dir[] beyond K0
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const float4 w = *reinterpret_cast<const float4*>(sW0 + (c0 + j) * kW0Stride + 4 * i4);
              z[j] = fmaf(w.x, in[4 * i4 + 0], z[j]);
              z[j] = fmaf(w.y, in[4 * i4 + 1], z[j]);
              z[j] = fmaf(w.z, in[4 * i4 + 2], z[j]);
              z[j] = fmaf(w.w, in[4 * i4 + 3], z[j]);
            }
          }
        }
      } else if (ri.cls > 0) {
#pragma unroll
        for (int i4 = 0; i4 < kW0Stride / 4; ++i4) {
          if (4 * i4 < K0) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const float4 w = *reinterpret_cast<const float4*>(sW0 + (c0 + j) * kW0Stride + 4 * i4);
              z[j] = fmaf(w.x, in[4 * i4 + 0], z[j]);
              z[j] = fmaf(w.y, in[4 * i4 + 1], z[j]);
              z[j] = fmaf(w.z, in[4 * i4 + 2], z[j]);
              z[j] = fmaf(w.w, in[4 * i4 + 3], z[j]);
              zd[j] = fmaf(w.x, dir[4 * i4 + 0], zd[j]);
              zd[j] = fmaf(w.y, dir[4 * i4 + 1], zd[j]);
              zd[j] = fmaf(w.z, dir[4 * i4 + 2], zd[j]);
              zd[j] = fmaf(w.w, dir[4 * i4 + 3], zd[j]);
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = c0 + j;
        if (ri.cls < 0) hv[j] = 0.f;
        else if (ri.cls == 0) hv[j] = a.act == 0 ? (SPLIT ? elu(z[j]) : elu_bf16_input(z[j])) : z[j];
        else if (ri.cls == 1) hv[j] = act_d1(a.act, z[j]) * zd[j];
        else if (ri.cls == 2) hv[j] = act_sec(a.act, z[j], zd[j]);
        else {
          const int b = ri.kind - KIND_MIXED - 1;   // input of the mixed derivative, padded layout below
          const float t0 = b < a.d ? sW0[c * kW0Stride + b] / a.norm[a.d + b] : sW0[c * kW0Stride + kTcLat + b - a.d];
          hv[j] = act_d2(a.act, z[j]) * zd[j] * t0;
        }
        if (a.dstore && ri.cls == 0)
          a.dstore[(int64_t)c * a.rows_total + tile * 128 + rw] = __float2bfloat16_rn(act_slope_record(a.act, z[j]));
      }
      store_operand<SPLIT>(atile, rw, c0, hv);
    }

    float y[3] = {0.f, 0.f, 0.f};
    // layer -1 is the first layer when it runs on the tensor cores
    for (int l = l0_tc ? -1 : 0; l < a.n_tc; ++l) {
      // make the generic-proxy writes of the operand tile visible to the tensor core
      tc::fence_async_smem();
      tc::tc_fence_before();
      __syncthreads();
      if (t == 0) {
        tc::tc_fence_after();
        bool w_ok = true;
        if (SPLIT && w_pending) {
          w_ok = tc::mbar_wait(&tail->bar_w, w_phase);
          w_phase ^= 1u;
          w_pending = false;
          if (!w_ok) {
            raise_status(a.status, STATUS_TIMEOUT);
            atomicExch(&tail->abort, 1);
          }
        }
        if (w_ok && l < 0) {
          // two K steps of 16 over the 32 padded inputs; hi at byte 0 of a row, lo at byte 64
          const uint32_t a_base = tc::smem_addr(atile), b_base = tc::smem_addr(w0s);
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const uint32_t hi = (uint32_t)(k * 32), lo = (uint32_t)(64 + k * 32);
            tc::mma_bf16(tmem, tc::smem_desc_sw128(a_base + hi), tc::smem_desc_sw128(b_base + hi), idesc,
                         k > 0 ? 1u : 0u);
            tc::mma_bf16(tmem, tc::smem_desc_sw128(a_base + hi), tc::smem_desc_sw128(b_base + lo), idesc, 1u);
            tc::mma_bf16(tmem, tc::smem_desc_sw128(a_base + lo), tc::smem_desc_sw128(b_base + hi), idesc, 1u);
          }
        } else if (w_ok) {
          const uint32_t a_base = tc::smem_addr(atile);
          const uint32_t b_base = tc::smem_addr(wsm + (SPLIT ? 0 : l * kLayerBytes));
#pragma unroll
          for (int k = 0; k < kW / 16; ++k) {
            const uint32_t koff = (uint32_t)((k >> 2) * (kW * 128) + (k & 3) * 32);
            tc::mma_bf16(tmem, tc::smem_desc_sw128(a_base + koff), tc::smem_desc_sw128(b_base + koff), idesc,
                         k > 0 ? 1u : 0u);
            if (SPLIT) {
              tc::mma_bf16(tmem, tc::smem_desc_sw128(a_base + koff),
                           tc::smem_desc_sw128(b_base + kLayerBytes + koff), idesc, 1u);
              tc::mma_bf16(tmem, tc::smem_desc_sw128(a_base + kLayerBytes + koff),
                           tc::smem_desc_sw128(b_base + koff), idesc, 1u);
            }
          }
        }
        tc::mma_commit(&tail->bar_mma);
      }
      // training: the previous layer's activations leave the operand tile while the tensor core
      // reads it (both are reads; the barrier after the wait orders them before the next writes)
      if (!SPLIT && a.astore && l > (l0_tc ? -1 : 0))
        copy_out_tile(a.astore + (int64_t)l * kW * a.rows_total, a.rows_total, atile, tile, t);
      if (!tc::mbar_wait(&tail->bar_mma, mma_phase)) {
        raise_status(a.status, STATUS_TIMEOUT);
        atomicExch(&tail->abort, 1);
      }
      mma_phase ^= 1u;
      if (SPLIT && t == 0 && a.n_tc > 1 && !tail->abort) {
        // the MMAs have read the buffer: stream the next layer's images (this tile's next layer, or
        // the first layer of the CTA's next tile) while the epilogue runs
        const int nl = (l + 1) % a.n_tc;
        if (l + 1 < a.n_tc || tile + gridDim.x < n_tiles) {
          tc::mbar_expect_tx(&tail->bar_w, (uint32_t)(2 * kLayerBytes));
          tc::bulk_g2s(wsm, a.wimg + (size_t)nl * kLayerBytes, kLayerBytes, &tail->bar_w);
          tc::bulk_g2s(wsm + kLayerBytes, a.wimg_lo + (size_t)nl * kLayerBytes, kLayerBytes, &tail->bar_w);
          w_pending = true;
        }
      }
      tc::tc_fence_after();
      __syncthreads();
      if (tail->abort) break;
      const bool last = (l == a.n_tc - 1);
      const float* bl = l < 0 ? sb0 : sbh + l * kW;
      for (int i2 = 0; i2 < 2; ++i2) {
        const int ch = 2 * h + i2;
        float acc[32];
        tc::tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + ch * 32, acc);
        if (ri.cls == 0) {
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[i] += bl[ch * 32 + i];
        }
        if (a.R > 1) {
          // publish this row's pre-activations of the chunk (stride 33: conflict-free)
#pragma unroll
          for (int i = 0; i < 32; ++i) xh[rw * kXbStride + i] = acc[i];
          __syncthreads();
          // training: the primal rows' activation slopes (the backward's act' and act'' terms), from
          // the published pre-activations, spread over the half's four warps: feature = lane, 8 rows
          // per thread, one 16-byte store of 8 rows of one feature (the training calls have R > 1)
          if (a.dstore) {
            for (int k = warp & 3; 8 * k < a.Pt; k += 4) {
              float v[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                // in place: the primal rows' slopes replace their pre-activations in the exchange
                float* e = xh + (8 * k + j) * kXbStride + lane;
                v[j] = act_slope_record(a.act, *e);
                *e = v[j];
              }
              __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]), p1 = __floats2bfloat162_rn(v[2], v[3]);
              __nv_bfloat162 p2 = __floats2bfloat162_rn(v[4], v[5]), p3 = __floats2bfloat162_rn(v[6], v[7]);
              uint4 u;
              u.x = *reinterpret_cast<uint32_t*>(&p0);
              u.y = *reinterpret_cast<uint32_t*>(&p1);
              u.z = *reinterpret_cast<uint32_t*>(&p2);
              u.w = *reinterpret_cast<uint32_t*>(&p3);
              *reinterpret_cast<uint4*>(a.dstore + ((int64_t)(l + 1) * kW + ch * 32 + lane) * a.rows_total +
                                        tile * 128 + 8 * k) = u;
            }
            __syncthreads();
          }
        }
        // the primal row of point q is tile row q (kind index 0)
        const float* zq = xh + ri.q * kXbStride;
        if (a.dstore) {
          // training (primal and tangent rows only): the slope s of the primal row, e^z where z < 0
          // and -1 elsewhere, gives both activations without another exponential: ELU(z) = s - 1
          // (z where s < 0), act'(z) = s (1 where s < 0); the same values as below
          if (ri.cls == 0) {
#pragma unroll
            for (int i = 0; i < 32; ++i) acc[i] = zq[i] < 0.f ? acc[i] : zq[i] - 1.0f;
          } else if (ri.cls == 1) {
#pragma unroll
            for (int i = 0; i < 32; ++i) acc[i] *= zq[i] < 0.f ? 1.0f : zq[i];
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) acc[i] = 0.f;
          }
        } else if (ri.cls == 0) {
          if (a.act == 0) {
#pragma unroll
            for (int i = 0; i < 32; ++i) acc[i] = SPLIT ? elu(acc[i]) : elu_bf16_input(acc[i]);
          }
        } else if (ri.cls == 1) {
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[i] *= act_d1(a.act, zq[i]);
        } else if (ri.cls == 2) {
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[i] = act_sec(a.act, zq[i], acc[i]);
        } else if (ri.cls == 3) {
          const float* uq = xh + (ri.ja * a.Pt + ri.q) * kXbStride;
          const float* tq = xh + (ri.jb * a.Pt + ri.q) * kXbStride;
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[i] = act_d2(a.act, zq[i]) * uq[i] * tq[i] + act_d1(a.act, zq[i]) * acc[i];
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[i] = 0.f;
        }
        if (last) {
          // output layer fused into the last epilogue (FP32), partial over this half's columns
#pragma unroll
          for (int o = 0; o < 3; ++o) {   // compile-time bound: y stays in registers
            if (o >= a.d) break;
            float sacc = 0.f;
#pragma unroll
            for (int i = 0; i < 32; ++i) sacc = fmaf(sWout[o * kW + ch * 32 + i], acc[i], sacc);
            y[o] += sacc;
          }
        }
        // the next layer's operand tile; in training also the last layer's, for the copy-out
        if (!last || (!SPLIT && a.astore)) {
#pragma unroll
          for (int j = 0; j < 32; j += 8) store_operand<SPLIT>(atile, rw, ch * 32 + j, acc + j);
        }
        if (a.R > 1) __syncthreads();
      }
      tc::tc_fence_before();
    }
    if (tail->abort) break;
    // combine the two column halves of the output layer
    if (h == 1) {
#pragma unroll
      for (int o = 0; o < 3; ++o)
        if (o < a.d) ypart[rw * 3 + o] = y[o];
    }
    __syncthreads();
    // training: the last layer's activations (the barrier at the end of the tile orders these
    // reads before the next tile's first operand writes)
    if (!SPLIT && a.astore) copy_out_tile(a.astore + (int64_t)a.n_tc * kW * a.rows_total, a.rows_total, atile, tile, t);
    if (h == 0 && ri.cls >= 0) {
      const int kidx = rw / a.Pt;  // position of this row's kind in `kinds`
      float* o = a.out + ((int64_t)kidx * a.n + ri.p) * a.d;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (i >= a.d) break;
        float v = y[i] + ypart[rw * 3 + i] + (ri.cls == 0 ? __ldg(&a.bout[i]) : 0.f);
        o[i] = v * a.norm[3 * a.d + i] + (ri.cls == 0 ? a.norm[2 * a.d + i] : 0.f);
      }
    }
    __syncthreads();
  }
  // a weight copy still in flight (an aborted tile loop) lands before the CTA exits
  if (SPLIT && t == 0 && w_pending) (void)tc::mbar_wait(&tail->bar_w, w_phase);
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_free<kW>(tmem);
}

// --------------------------------------------------------------------------
// Tensor-core decoder for calls of primal rows only (one row kind), inputs of at most 32
// entries in the padded layout, BF16 operands: two 128-row tiles in flight per CTA.  512
// threads in two groups of eight warps; each group runs decoder_tc's tile loop (split-BF16 first
// layer, square layers, fused output layer) on its own operand tile, tensor-memory columns, MMA
// barrier and named barrier, so that one group's epilogue overlaps the other group's MMAs.  The
// weights and the first layer's split image are resident once per CTA.  Same arithmetic, in the
// same order, as decoder_tc<false>.
// --------------------------------------------------------------------------
constexpr int kPrimThreads = 512;

struct __align__(8) PrimSmemTail {
  uint64_t bar_w;
  uint64_t bar_mma[2];
  uint32_t tmem;
  int abort[2];   // per group: set before a group barrier, read after it
};

__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, 256;" ::"r"(1 + g) : "memory"); }

__global__ void __launch_bounds__(kPrimThreads, 1) decoder_tc_primal(DecArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* wsm = smem;                                   // kMaxTC x 32 KB square layers
  uint8_t* w0s = smem + kMaxTC * kLayerBytes;            // 16 KB first-layer split image
  uint8_t* atiles = w0s + kLayerBytes / 2;               // 2 x 32 KB operand tiles, one per group
  float* ypart = (float*)(atiles + 2 * kLayerBytes);     // [2 groups][128 rows][3]
  float* sb0 = ypart + 2 * 128 * 3;                      // [128]
  float* sbh = sb0 + kW;                                 // [kMaxTC][128]
  float* sWout = sbh + kMaxTC * kW;                      // [3][128]
  PrimSmemTail* tail = (PrimSmemTail*)(sWout + 3 * kW);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int g = warp >> 3, tg = t & 255;                 // group, thread within the group
  const int rw = (warp & 3) * 32 + lane;                 // tile row / tensor-memory lane
  const int h = (warp >> 2) & 1;                         // column half
  uint8_t* atile = atiles + g * kLayerBytes;
  float* yp = ypart + g * 128 * 3;

  if (t == 0) {
    tc::mbar_init(&tail->bar_w, 1);
    tc::mbar_init(&tail->bar_mma[0], 1);
    tc::mbar_init(&tail->bar_mma[1], 1);
    tail->abort[0] = 0;
    tail->abort[1] = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc<2 * kW>(&tail->tmem);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tail->tmem + (uint32_t)(g * kW);   // this group's 128 columns

  for (int e = t; e < kW; e += kPrimThreads) sb0[e] = a.b0[e];
  for (int e = t; e < a.n_tc * kW; e += kPrimThreads) sbh[e] = a.bh[e];
  for (int e = t; e < a.d * kW; e += kPrimThreads) sWout[e] = a.Wout[e];
  if (t == 0) {
    tc::mbar_expect_tx(&tail->bar_w, (uint32_t)(a.n_tc * kLayerBytes + kLayerBytes / 2));
    for (int l = 0; l < a.n_tc; ++l)
      tc::bulk_g2s(wsm + l * kLayerBytes, a.wimg + (size_t)l * kLayerBytes, kLayerBytes, &tail->bar_w);
    tc::bulk_g2s(w0s, a.w0img, kLayerBytes / 2, &tail->bar_w);
  }
  if (!tc::mbar_wait(&tail->bar_w, 0)) {
    raise_status(a.status, STATUS_TIMEOUT);
    tail->abort[0] = 1;
    tail->abort[1] = 1;
  }
  __syncthreads();

  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, kW);
  uint32_t mma_phase = 0;
  const int64_t n_pts = dec_count(a);
  const int64_t n_tiles = (n_pts + 127) / 128;
  for (int64_t tile = 2 * (int64_t)blockIdx.x + g; tile < n_tiles && !tail->abort[g]; tile += 2 * (int64_t)gridDim.x) {
    const int64_t first = tile * 128;
    const RowInfo ri = row_info(a, rw, first, n_pts);
    {
      float in[40], dir[40];
      if (ri.cls >= 0) row_inputs_tc(a, ri, in, dir);
      // the first layer's operand row: half 0 stores the high parts at columns 0 .. 31, half 1
      // the low parts at 32 .. 63; zero for rows past the end
#pragma unroll
      for (int c0 = 0; c0 < 32; c0 += 8) {
        float p[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float v = ri.cls == 0 ? in[c0 + j] : 0.f;
          const float hi = __bfloat162float(__float2bfloat16_rn(v));
          p[j] = h == 0 ? hi : v - hi;
        }
        store_bf16x8(atile, rw, 32 * h + c0, p);
      }
    }
    float y[3] = {0.f, 0.f, 0.f};
    for (int l = -1; l < a.n_tc; ++l) {
      tc::fence_async_smem();
      tc::tc_fence_before();
      group_sync(g);
      if (tg == 0) {
        tc::tc_fence_after();
        const uint32_t a_base = tc::smem_addr(atile);
        if (l < 0) {
          const uint32_t b_base = tc::smem_addr(w0s);
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const uint32_t hi = (uint32_t)(k * 32), lo = (uint32_t)(64 + k * 32);
            tc::mma_bf16(tmem, tc::smem_desc_sw128(a_base + hi), tc::smem_desc_sw128(b_base + hi), idesc,
                         k > 0 ? 1u : 0u);
            tc::mma_bf16(tmem, tc::smem_desc_sw128(a_base + hi), tc::smem_desc_sw128(b_base + lo), idesc, 1u);
            tc::mma_bf16(tmem, tc::smem_desc_sw128(a_base + lo), tc::smem_desc_sw128(b_base + hi), idesc, 1u);
          }
        } else {
          const uint32_t b_base = tc::smem_addr(wsm + l * kLayerBytes);
#pragma unroll
          for (int k = 0; k < kW / 16; ++k) {
            const uint32_t koff = (uint32_t)((k >> 2) * (kW * 128) + (k & 3) * 32);
            tc::mma_bf16(tmem, tc::smem_desc_sw128(a_base + koff), tc::smem_desc_sw128(b_base + koff), idesc,
                         k > 0 ? 1u : 0u);
          }
        }
        tc::mma_commit(&tail->bar_mma[g]);
      }
      if (!tc::mbar_wait(&tail->bar_mma[g], mma_phase)) {
        raise_status(a.status, STATUS_TIMEOUT);
        tail->abort[g] = 1;
      }
      mma_phase ^= 1u;
      tc::tc_fence_after();
      group_sync(g);
      if (tail->abort[g]) break;
      const bool last = (l == a.n_tc - 1);
      const float* bl = l < 0 ? sb0 : sbh + l * kW;
      for (int i2 = 0; i2 < 2; ++i2) {
        const int ch = 2 * h + i2;
        float acc[32];
        tc::tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + ch * 32, acc);
        if (ri.cls == 0) {
#pragma unroll
          for (int i = 0; i < 32; i += 4) {
            const float4 b4 = *reinterpret_cast<const float4*>(bl + ch * 32 + i);
            acc[i] += b4.x;
            acc[i + 1] += b4.y;
            acc[i + 2] += b4.z;
            acc[i + 3] += b4.w;
          }
          if (a.act == 0) {
#pragma unroll
            for (int i = 0; i < 32; ++i) acc[i] = elu_bf16_input(acc[i]);
          }
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[i] = 0.f;
        }
        if (last) {
#pragma unroll
          for (int o = 0; o < 3; ++o) {   // compile-time bound: y stays in registers
            if (o >= a.d) break;
            float sacc = 0.f;
#pragma unroll
            for (int i = 0; i < 32; ++i) sacc = fmaf(sWout[o * kW + ch * 32 + i], acc[i], sacc);
            y[o] += sacc;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; j += 8) store_bf16x8(atile, rw, ch * 32 + j, acc + j);
        }
      }
      tc::tc_fence_before();
    }
    if (tail->abort[g]) break;
    // combine the two column halves of the output layer
    if (h == 1) {
#pragma unroll
      for (int o = 0; o < 3; ++o)
        if (o < a.d) yp[rw * 3 + o] = y[o];
    }
    group_sync(g);
    if (h == 0 && ri.cls >= 0) {
      float* o = a.out + ri.p * a.d;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (i >= a.d) break;
        const float v = y[i] + yp[rw * 3 + i] + __ldg(&a.bout[i]);
        o[i] = v * a.norm[3 * a.d + i] + a.norm[2 * a.d + i];
      }
    }
    group_sync(g);
  }
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_free<2 * kW>(tail->tmem);
}

// --------------------------------------------------------------------------
// FP32 decoder on the CUDA cores, for calls whose rows are too few to keep the
// tensor cores busy and whose results need FP32 accuracy (the reduced step's
// positions and gradients).  Same row kinds as decoder_tc; one persistent CTA
// of 512 threads (16 warps) per SM; tiles of TR = 32 or 64 row slots.
// Rows reach the tiles in one of two ways:
//   aligned  (mixed rows present) slot k Pt + q = kind k of point q, Pt = TR / R
//            points per tile, as in decoder_tc;
//   packed   the call's rows in (point, kind) order, U <= TR - 1 per tile,
//            chosen so that the tiles spread over all SMs; slot 0 recomputes
//            the primal row of the tile's first point (its derivative rows may
//            start mid-point) and is not written out.
// Per tile:
//   layer 0       512 / TR threads per row, each 128 TR / 512 columns; inputs
//                 staged in shared memory first
//   square layer  128 x TR x 128 FP32 GEMM from shared memory: TR / 4 warps,
//                 warp w features (512 / TR) w .. + 512 / TR - 1 of every slot,
//                 lane = (slot group of 4, feature group of 4): per k one float4
//                 of activations and one of weights (two or three shared-memory
//                 wavefronts per warp for 16 FMAs per lane); weights
//                 double-buffered from a transposed copy by asynchronous copies;
//                 activations by warps w < TR / 4, slots 4 w .. 4 w + 3
//   exchange      pre-activations to a second buffer (row-major, float4 quads
//                 permuted per row group); derivative rows read the primal
//                 (and, for mixed rows, JVP and tangent) rows' values as float4
//                 of the thread's own 4 features
//   output layer  512 / TR threads per row, interleaved k, shuffle reduction
// Activations (the GEMM's input) are stored feature-major, [f][TR slots], the
// slots in float4 groups permuted per feature (group g of feature f at
// g ^ (f mod TR / 4)) so that the feature-strided stores of a warp spread over
// the banks.  Two barriers per square layer.
// --------------------------------------------------------------------------
constexpr int kF32Threads = 512;
constexpr int kF32Rows = 64;              // largest tile (row slots)
constexpr int kF32In = 41;                // staged input row stride (d + r <= 40)

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gmem_src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// ELU for the FP32 path: exp(z) - 1 with the fast exponential (absolute error at the FP32 ulp of
// values near 1, far below the parity tolerance)
__device__ __forceinline__ float act_f32path(int act, float z) {
  return act == 0 ? (z > 0.f ? z : __expf(z) - 1.0f) : z;
}

// Offset of (feature f, slot) in an activation buffer of TR slots.
template <int TR>
__device__ __forceinline__ int f32_slot(int f, int slot) {
  return f * TR + 4 * ((slot >> 2) ^ (f & (TR / 4 - 1))) + (slot & 3);
}

// Offset of the float4 of features f .. f + 3 (f a multiple of 4) of a slot in the row-major
// pre-activation buffer.
__device__ __forceinline__ int f32_zslot(int slot, int f) { return slot * kW + 4 * ((f >> 2) ^ ((slot >> 2) & 7)); }

// Activation of a derivative row from its own pre-activation zo, the primal row's zq and, for a
// mixed row, the JVP row's za and the tangent row's zb (same point, same feature).
__device__ __forceinline__ float f32_deriv_act(int act, int cls, float zo, float zq, float za, float zb) {
  if (cls == 1) return act_d1(act, zq) * zo;
  if (cls == 2) return act_sec(act, zq, zo);
  return act_d2(act, zq) * za * zb + act_d1(act, zq) * zo;
}

// One slot of an FP32-path tile: the row (kind, class, point), the slots of its partner rows and
// the output block it is written to (-1: not written).
struct F32Row {
  RowInfo ri;
  int qs, as, bs;
  int kidx;
};

__device__ __forceinline__ F32Row f32_row(const DecArgs& a, int slot, int64_t tile, int64_t n_pts) {
  F32Row fr;
  if (a.f32_U == 0) {
    fr.ri = row_info(a, slot, tile * a.Pt, n_pts);
    fr.qs = fr.ri.q;
    fr.as = fr.ri.ja * a.Pt + fr.ri.q;
    fr.bs = fr.ri.jb * a.Pt + fr.ri.q;
    fr.kidx = fr.ri.cls >= 0 ? slot / a.Pt : -1;
    return fr;
  }
  const int U = a.f32_U;
  const int64_t g0 = tile * U;
  const int64_t g = slot == 0 ? (g0 / a.R) * a.R : g0 + slot - 1;
  fr.ri.q = fr.ri.ja = fr.ri.jb = 0;
  fr.qs = fr.as = fr.bs = 0;
  if (slot > U || g >= n_pts * a.R) {
    fr.ri.cls = -1;
    fr.ri.kind = -1;
    fr.ri.p = 0;
    fr.kidx = -1;
    return fr;
  }
  const int64_t p = g / a.R;
  const int k = (int)(g - p * a.R);
  fr.ri.p = p;
  fr.ri.kind = a.kinds[k];
  fr.ri.cls = kind_class(fr.ri.kind);
  const int64_t gp = p * a.R;   // the point's primal row: in this tile, or recomputed in slot 0
  fr.qs = gp >= g0 ? (int)(gp - g0 + 1) : 0;
  fr.kidx = slot == 0 ? -1 : k;
  return fr;
}

template <int TR>
__global__ void __launch_bounds__(kF32Threads, 1) decoder_f32(DecArgs a) {
  constexpr int G = TR / 4;                   // 4-slot groups = GEMM warps = activation warps
  constexpr int TPR = kF32Threads / TR;       // threads per row in layer 0 and the output layer
  constexpr int CPT = kW / TPR;               // layer-0 columns per thread
  extern __shared__ __align__(16) float fsm[];
  float* A0 = fsm;                            // [128 f][TR slots] activations (GEMM input)
  float* A1 = A0 + kW * kF32Rows;             // [TR slots][128 f] pre-activations; staged inputs at layer 0
  float* Wt0 = A1 + kW * kF32Rows;            // two [128 in][128 out] weight buffers, transposed
  float* W0T = Wt0 + 2 * kW * kW;             // [40 in][128 out] first layer, transposed
  float* sb0 = W0T + kW0Stride * kW;          // [128]
  float* sbh = sb0 + kW;                      // [kMaxTC][128]
  float* sWout = sbh + kMaxTC * kW;           // [3][128]
  F32Row* srow = reinterpret_cast<F32Row*>(sWout + 3 * kW);        // [TR] the tile's rows
  int64_t* sxrow = reinterpret_cast<int64_t*>(srow + kF32Rows);    // [TR] their X rows
  int* sli = reinterpret_cast<int*>(sxrow + kF32Rows);             // [TR] their latent rows
  float* IN = A1;                             // [TR][kF32In] normalised inputs (layer 0 only)
  float* DIR = A1 + kF32Rows * kF32In;        // [TR][kF32In] input directions
  const int t = threadIdx.x;
  const int K0 = a.d + a.r;
  // constant operands: all loads issued before any is used
#pragma unroll
  for (int j = 0; j < (kW0Stride * kW) / kF32Threads; ++j) {
    const int e = t + j * kF32Threads;   // e = i * 128 + c
    const int i = e >> 7, c = e & (kW - 1);
    if (i < K0) W0T[e] = a.W0[c * K0 + i];
  }
  if (t < kW) sb0[t] = a.b0[t];
  if (t < a.n_tc * kW) sbh[t] = a.bh[t];
  if (t < a.d * kW) sWout[t] = a.Wout[t];
  // weights of square layer l into buffer l % 2 (asynchronous copy, waited before its GEMM)
  auto prefetch = [&](int l) {
    const float* src = a.wsqT + (size_t)l * kW * kW;
    float* dst = Wt0 + (l & 1) * kW * kW;
#pragma unroll
    for (int j = 0; j < kW * kW / 4 / kF32Threads; ++j) {
      const int e = t + j * kF32Threads;
      cp_async16(dst + 4 * e, src + 4 * e);
    }
    cp_async_commit();
  };

  const int64_t n_pts = dec_count(a);
  const int64_t n_tiles = a.f32_U ? (n_pts * a.R + a.f32_U - 1) / a.f32_U : (n_pts + a.Pt - 1) / a.Pt;
  const int warp = t >> 5, lane = t & 31;
  const int f0 = 4 * lane;                    // activations: features f0 .. f0 + 3 of slots 4 warp .. 4 warp + 3
  const int rw = t % TR, cg = t / TR;         // layer 0: slot rw, columns CPT cg .. CPT cg + CPT - 1
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    if (a.n_tc > 0) prefetch(0);
    // ---- the tile's rows (integer divisions once per slot) and their inputs
    if (t < TR) {
      const F32Row fr = f32_row(a, t, tile, n_pts);
      srow[t] = fr;
      int64_t xrow = 0;
      int li = 0;
      if (fr.ri.cls >= 0) row_source(a, fr.ri, xrow, li);
      sxrow[t] = xrow;
      sli[t] = li;
    }
    __syncthreads();
    for (int e = t; e < TR * K0; e += kF32Threads) {
      const int slot = e / K0, i = e - slot * K0;
      const F32Row& fr = srow[slot];
      float vin = 0.f, vdir = 0.f;
      if (fr.ri.cls >= 0) row_input_from(a, fr.ri, sxrow[slot], sli[slot], i, vin, vdir);
      IN[slot * kF32In + i] = vin;
      DIR[slot * kF32In + i] = vdir;
    }
    __syncthreads();
    // ---- layer 0 (FP32)
    {
      const RowInfo ri = srow[rw].ri;
      float z[CPT], zd[CPT];
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        z[c] = sb0[CPT * cg + c];
        zd[c] = 0.f;
      }
      for (int i = 0; i < K0; ++i) {
        const float vin = IN[rw * kF32In + i], vdir = DIR[rw * kF32In + i];
        const float4* w4 = reinterpret_cast<const float4*>(W0T + i * kW + CPT * cg);
#pragma unroll
        for (int q = 0; q < CPT / 4; ++q) {
          const float4 w = w4[q];
          z[4 * q + 0] = fmaf(w.x, vin, z[4 * q + 0]);
          z[4 * q + 1] = fmaf(w.y, vin, z[4 * q + 1]);
          z[4 * q + 2] = fmaf(w.z, vin, z[4 * q + 2]);
          z[4 * q + 3] = fmaf(w.w, vin, z[4 * q + 3]);
          zd[4 * q + 0] = fmaf(w.x, vdir, zd[4 * q + 0]);
          zd[4 * q + 1] = fmaf(w.y, vdir, zd[4 * q + 1]);
          zd[4 * q + 2] = fmaf(w.z, vdir, zd[4 * q + 2]);
          zd[4 * q + 3] = fmaf(w.w, vdir, zd[4 * q + 3]);
        }
      }
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int col = CPT * cg + c;
        float hv = 0.f;
        if (ri.cls == 0) hv = act_f32path(a.act, z[c]);
        else if (ri.cls == 1) hv = act_d1(a.act, z[c]) * zd[c];
        else if (ri.cls == 2) hv = act_sec(a.act, z[c], zd[c]);
        else if (ri.cls == 3) {
          const int b = ri.kind - KIND_MIXED - 1;
          const float t0 = b < a.d ? W0T[b * kW + col] / a.norm[a.d + b] : W0T[b * kW + col];
          hv = act_d2(a.act, z[c]) * zd[c] * t0;
        }
        A0[f32_slot<TR>(col, rw)] = hv;
      }
    }
    for (int l = 0; l < a.n_tc; ++l) {
      cp_async_wait_all();
      __syncthreads();                                  // A0 complete, weights of layer l landed, A1 free
      if (l + 1 < a.n_tc) prefetch(l + 1);              // overlaps the GEMM below
      if (warp < G) {
        // GEMM: lane (sg, fg) of warp w computes slots 4 sg .. 4 sg + 3 and features
        // fbase .. fbase + 3 (fbase = (512 / TR) w + 4 fg): per k one float4 of activations (eight
        // or sixteen distinct in the warp) and one of weights (four or two distinct)
        constexpr int FG = 128 / TR;                  // feature groups per warp
        const int sg = lane / FG, fg = lane % FG;
        const int fbase = (512 / TR) * warp + 4 * fg;
        const float* Wt = Wt0 + (l & 1) * kW * kW;
        float acc[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[j][i] = 0.f;
#pragma unroll 8
        for (int k = 0; k < kW; ++k) {
          const float4 av = *reinterpret_cast<const float4*>(A0 + k * TR + 4 * (sg ^ (k & (G - 1))));
          const float4 wv = *reinterpret_cast<const float4*>(Wt + k * kW + fbase);
          const float ar[4] = {av.x, av.y, av.z, av.w};
          const float wr[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[j][i] = fmaf(ar[j], wr[i], acc[j][i]);
        }
        // pre-activations (bias on primal rows) to A1
        const float4 b4 = *reinterpret_cast<const float4*>(sbh + l * kW + fbase);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (srow[4 * sg + j].ri.cls == 0) {
            acc[j][0] += b4.x;
            acc[j][1] += b4.y;
            acc[j][2] += b4.z;
            acc[j][3] += b4.w;
          }
          *reinterpret_cast<float4*>(A1 + f32_zslot(4 * sg + j, fbase)) =
              make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
        }
      }
      __syncthreads();                                  // A1 complete, every GEMM has read A0
      {
        // activations of the next layer into A0: every warp takes SPW = TR / 16 slots (warp w:
        // slots SPW w ..), so that the short dependent chains of the activations run on all
        // sixteen warps; derivative rows read their partners' pre-activations
        constexpr int SPW = TR / 16;
        float h[SPW][4];
#pragma unroll
        for (int j = 0; j < SPW; ++j) {
          const F32Row& fr = srow[SPW * warp + j];
          const float4 z4 = *reinterpret_cast<const float4*>(A1 + f32_zslot(SPW * warp + j, f0));
          const float zr[4] = {z4.x, z4.y, z4.z, z4.w};
          if (fr.ri.cls == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) h[j][i] = act_f32path(a.act, zr[i]);
          } else if (fr.ri.cls < 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) h[j][i] = 0.f;
          } else {
            const float4 q4 = *reinterpret_cast<const float4*>(A1 + f32_zslot(fr.qs, f0));
            float4 a4 = q4, c4 = q4;
            if (fr.ri.cls == 3) {
              a4 = *reinterpret_cast<const float4*>(A1 + f32_zslot(fr.as, f0));
              c4 = *reinterpret_cast<const float4*>(A1 + f32_zslot(fr.bs, f0));
            }
            h[j][0] = f32_deriv_act(a.act, fr.ri.cls, zr[0], q4.x, a4.x, c4.x);
            h[j][1] = f32_deriv_act(a.act, fr.ri.cls, zr[1], q4.y, a4.y, c4.y);
            h[j][2] = f32_deriv_act(a.act, fr.ri.cls, zr[2], q4.z, a4.z, c4.z);
            h[j][3] = f32_deriv_act(a.act, fr.ri.cls, zr[3], q4.w, a4.w, c4.w);
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (SPW == 4) {
            *reinterpret_cast<float4*>(A0 + f32_slot<TR>(f0 + i, 4 * warp)) =
                make_float4(h[0][i], h[1][i], h[2 % SPW][i], h[3 % SPW][i]);
          } else {
            *reinterpret_cast<float2*>(A0 + f32_slot<TR>(f0 + i, SPW * warp)) = make_float2(h[0][i], h[1 % SPW][i]);
          }
        }
      }
    }
    __syncthreads();                                    // A0 complete
    // ---- output layer (FP32): TPR threads per row, k interleaved, combined by shuffles
    {
      const int slot = t / TPR, part = t % TPR;
      const F32Row fr = srow[slot];
      float y[3] = {0.f, 0.f, 0.f};
#pragma unroll 4
      for (int kk = 0; kk < kW / TPR; ++kk) {
        const int k = part + TPR * kk;
        const float h = A0[f32_slot<TR>(k, slot)];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          if (i < a.d) y[i] = fmaf(sWout[i * kW + k], h, y[i]);
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int o = 1; o < TPR; o <<= 1) y[i] += __shfl_xor_sync(0xffffffffu, y[i], o);
      if (part == 0 && fr.kidx >= 0) {
        const RowInfo& ri = fr.ri;
        float* o = a.out + ((int64_t)fr.kidx * a.n + ri.p) * a.d;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          if (i >= a.d) break;
          const float v = y[i] + (ri.cls == 0 ? a.bout[i] : 0.f);
          o[i] = v * a.norm[3 * a.d + i] + (ri.cls == 0 ? a.norm[2 * a.d + i] : 0.f);
        }
      }
    }
    __syncthreads();                                    // A0 / A1 / weight buffer 0 free for the next tile
  }
  cp_async_wait_all();
}

// Transposed FP32 copies of the square layers for the CUDA-core path:
// WT[l][k][f] = W[l][f][k].
__global__ void decoder_transpose(const float* W, int n_layers, float* WT) {
  __shared__ float tileT[32][33];
  for (int l = 0; l < n_layers; ++l) {
    for (int b = blockIdx.x; b < 16; b += gridDim.x) {
      const int f0 = (b / 4) * 32, k0 = (b % 4) * 32;
      const int tx = threadIdx.x & 31, tyy = threadIdx.x >> 5;
      for (int y = tyy; y < 32; y += blockDim.x / 32) tileT[y][tx] = W[(size_t)l * kW * kW + (f0 + y) * kW + k0 + tx];
      __syncthreads();
      for (int y = tyy; y < 32; y += blockDim.x / 32) WT[(size_t)l * kW * kW + (k0 + y) * kW + f0 + tx] = tileT[tx][y];
      __syncthreads();
    }
  }
}

// Packs the square-layer weights (FP32, (out, in) row-major) into BF16 images
// in the 128-byte swizzled K-major layout the MMA reads: img = bf16(w) and, when
// img_lo is set, img_lo = bf16(w - bf16(w)) (the split operands).
__global__ void decoder_pack(const float* W, int n_layers, int64_t stride, uint8_t* img, uint8_t* img_lo) {
  const int64_t total = (int64_t)n_layers * kW * kW;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int l = (int)(i / (kW * kW));
    int rem = (int)(i % (kW * kW));
    int row = rem / kW, k = rem % kW;
    const float w = W[l * stride + rem];
    const __nv_bfloat16 v = __float2bfloat16_rn(w);
    const size_t o = (size_t)l * kLayerBytes + tc::sw128_offset(row, k, kW);
    *reinterpret_cast<__nv_bfloat16*>(img + o) = v;
    if (img_lo) *reinterpret_cast<__nv_bfloat16*>(img_lo + o) = __float2bfloat16_rn(w - __bfloat162float(v));
  }
}

// Packs the first layer (FP32, (W, d + r) row-major) for the tensor cores: row c of the image
// holds bf16(w) of the padded inputs (coordinates at 0 .. 3, latents from kTcLat) at K 0 .. 31
// and bf16(w - bf16(w)) at K 32 .. 63, zero where no input sits, in the 128-byte swizzled
// K-major layout (one 16 KB atom column).
__global__ void decoder_pack_w0(const float* W0, int d, int r, uint8_t* img) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kW * 32; e += gridDim.x * blockDim.x) {
    const int c = e / 32, ii = e % 32;
    const int i = ii < kTcLat ? (ii < d ? ii : -1) : (ii - kTcLat < r ? d + ii - kTcLat : -1);
    const float w = i >= 0 ? W0[c * (d + r) + i] : 0.f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(w);
    *reinterpret_cast<__nv_bfloat16*>(img + tc::sw128_offset(c, ii, kW)) = hi;
    *reinterpret_cast<__nv_bfloat16*>(img + tc::sw128_offset(c, 32 + ii, kW)) =
        __float2bfloat16_rn(w - __bfloat162float(hi));
  }
}

}  // namespace mpmrom

using namespace mpmrom;



namespace {

size_t dec_smem_bytes(bool split) {
  return 1024 + (split ? 2 : kMaxTC) * kLayerBytes + (split ? 2 : 1) * kLayerBytes +
         (2 * 128 * kXbStride + 128 * 3 + kW * kW0Stride + kW + kMaxTC * kW + 3 * kW) * sizeof(float) +
         sizeof(DecSmemTail);
}

size_t dec_primal_smem_bytes() {
  return 1024 + kMaxTC * kLayerBytes + kLayerBytes / 2 + 2 * kLayerBytes +
         (2 * 128 * 3 + kW + kMaxTC * kW + 3 * kW) * sizeof(float) + sizeof(PrimSmemTail);
}

size_t dec_f32_smem_bytes() {
  return (size_t)(2 * kW * kF32Rows + 2 * kW * kW + kW0Stride * kW + kW + kMaxTC * kW + 3 * kW) * sizeof(float) +
         kF32Rows * (sizeof(F32Row) + sizeof(int64_t) + sizeof(int));
}

mpm_status refresh_derived_impl(mpm_decoder* dec, cudaStream_t s) {
  if (dec->n_tc == 0) return MPM_OK;
  for (int l = 0; l < dec->n_tc; ++l) {
    MPM_CUDA_TRY(cudaMemcpyAsync(dec->wsq + (size_t)l * kW * kW, dec->params + dec->w_off[1 + l],
                                 sizeof(float) * kW * kW, cudaMemcpyDeviceToDevice, s));
    MPM_CUDA_TRY(cudaMemcpyAsync(dec->bsq + (size_t)l * kW, dec->params + dec->b_off[1 + l], sizeof(float) * kW,
                                 cudaMemcpyDeviceToDevice, s));
  }
  decoder_pack<<<std::max(1, std::min(dec->n_sm * 4, dec->n_tc * 64)), 256, 0, s>>>(dec->wsq, dec->n_tc,
                                                                                    (int64_t)kW * kW, dec->wimg,
                                                                                    dec->wimg_lo);
  MPM_CUDA_TRY(cudaGetLastError());
  decoder_transpose<<<16, 256, 0, s>>>(dec->wsq, dec->n_tc, dec->wsqT);
  MPM_CUDA_TRY(cudaGetLastError());
  if (dec->w0img) {
    decoder_pack_w0<<<16, 256, 0, s>>>(dec->params + dec->w_off[0], dec->d, dec->r, dec->w0img);
    MPM_CUDA_TRY(cudaGetLastError());
  }
  return MPM_OK;
}

}  // namespace

namespace mpmrom {
mpm_status decoder_refresh(mpm_decoder* dec, cudaStream_t s) { return refresh_derived_impl(dec, s); }
// Coordinate and latent widths of a decoder, for code that holds it as an opaque handle.
void decoder_shape(const mpm_decoder* dec, int* d, int* r) {
  *d = dec->d;
  *r = dec->r;
}
// Internal launcher for on-device point sets (used by the reduced-order step).
mpm_status decoder_launch_dev(const mpm_decoder* dec, const float* X, const int32_t* idx, const int32_t* n_dev,
                              int n_rep, int64_t capacity, const float* latents, const float* dirs,
                              const int* kinds, int R, float* out, cudaStream_t s);
}

extern "C" {

mpm_status decoder_create(const decoder_desc* desc, mpm_decoder** out) {
  MPM_CHECK_ARG(desc && out, "null argument");
  *out = nullptr;
  MPM_CHECK_ARG(desc->d == 2 || desc->d == 3, "d must be 2 or 3");
  MPM_CHECK_ARG(desc->r >= 0 && desc->d + desc->r <= 40, "d + r must be <= 40");
  MPM_CHECK_ARG(desc->n_hidden >= 0, "n_hidden >= 0");
  MPM_CHECK_ARG(desc->activation == 0 || desc->activation == 1, "activation: 0 ELU, 1 identity");
  MPM_CHECK_ARG(desc->n_hidden == 0 || desc->width == kW, "hidden width must be 128");
  MPM_CHECK_ARG(desc->n_hidden <= kMaxTC + 1, "at most 5 hidden layers");
  auto* dec = new mpm_decoder();
  dec->d = desc->d;
  dec->r = desc->r;
  dec->width = desc->width;
  dec->n_hidden = desc->n_hidden;
  dec->act = desc->activation;
  dec->n_tc = std::max(0, desc->n_hidden - 1);
  std::vector<int> dims;
  dims.push_back(dec->d + dec->r);
  for (int l = 0; l < dec->n_hidden; ++l) dims.push_back(kW);
  dims.push_back(dec->d);
  int64_t off = 0;
  for (size_t l = 0; l + 1 < dims.size(); ++l) {
    dec->w_off.push_back(off);
    off += (int64_t)dims[l] * dims[l + 1];
    dec->b_off.push_back(off);
    off += dims[l + 1];
  }
  dec->n_params = off;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&dec->n_sm, cudaDevAttrMultiProcessorCount, dev);
  dec->smem = dec_smem_bytes(false);
  dec->smem_split = dec_smem_bytes(true);
  cudaError_t e = cudaMalloc((void**)&dec->params, sizeof(float) * dec->n_params);
  if (e == cudaSuccess) e = cudaMalloc((void**)&dec->norm, sizeof(float) * 4 * dec->d);
  if (e == cudaSuccess) e = cudaMalloc((void**)&dec->status, sizeof(uint32_t));
  if (e == cudaSuccess && dec->n_tc > 0) {
    e = cudaMalloc((void**)&dec->wsq, sizeof(float) * dec->n_tc * kW * kW);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dec->bsq, sizeof(float) * dec->n_tc * kW);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dec->wimg, (size_t)dec->n_tc * kLayerBytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dec->wimg_lo, (size_t)dec->n_tc * kLayerBytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dec->wsqT, sizeof(float) * dec->n_tc * kW * kW);
    if (e == cudaSuccess && kTcLat + dec->r <= 32) e = cudaMalloc((void**)&dec->w0img, (size_t)kLayerBytes / 2);
  }
  if (e == cudaSuccess) e = cudaMemset(dec->params, 0, sizeof(float) * dec->n_params);
  if (e == cudaSuccess) e = cudaMemset(dec->status, 0, sizeof(uint32_t));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(decoder_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dec->smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(decoder_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dec->smem_split);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(decoder_tc_primal, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dec_primal_smem_bytes());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(decoder_f32<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dec_f32_smem_bytes());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(decoder_f32<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dec_f32_smem_bytes());
  if (e != cudaSuccess) {
    decoder_destroy(dec);
    return set_error(MPM_ENOMEM, std::string("decoder_create: ") + cudaGetErrorString(e));
  }
  *out = dec;
  return MPM_OK;
}

void decoder_destroy(mpm_decoder* dec) {
  if (!dec) return;
  cudaFree(dec->params);
  cudaFree(dec->norm);
  cudaFree(dec->wsq);
  cudaFree(dec->bsq);
  cudaFree(dec->wimg);
  cudaFree(dec->wimg_lo);
  cudaFree(dec->wsqT);
  cudaFree(dec->w0img);
  cudaFree(dec->status);
  delete dec;
}

int64_t decoder_num_params(const mpm_decoder* dec) { return dec ? dec->n_params : 0; }

mpm_status decoder_set_concurrency(mpm_decoder* dec, int k) {
  MPM_CHECK_ARG(dec, "null decoder");
  MPM_CHECK_ARG(k >= 1, "k >= 1");
  dec->concurrency = k;
  return MPM_OK;
}

mpm_status decoder_set_precision(mpm_decoder* dec, int fp32) {
  MPM_CHECK_ARG(dec, "null decoder");
  MPM_CHECK_ARG(fp32 >= 0 && fp32 <= 2, "precision: 0 BF16, 1 FP32 CUDA cores, 2 split BF16 tensor cores");
  dec->fp32 = fp32;
  return MPM_OK;
}

mpm_status decoder_set_params(mpm_decoder* dec, const float* params, const float* norm, void* stream) {
  MPM_CHECK_ARG(dec && params && norm, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  MPM_CUDA_TRY(cudaMemcpyAsync(dec->params, params, sizeof(float) * dec->n_params, cudaMemcpyDefault, s));
  MPM_CUDA_TRY(cudaMemcpyAsync(dec->norm, norm, sizeof(float) * 4 * dec->d, cudaMemcpyDefault, s));
  return refresh_derived_impl(dec, s);
}

mpm_status decoder_get_params(const mpm_decoder* dec, float* params, float* norm, void* stream) {
  MPM_CHECK_ARG(dec, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (params) MPM_CUDA_TRY(cudaMemcpyAsync(params, dec->params, sizeof(float) * dec->n_params, cudaMemcpyDefault, s));
  if (norm) MPM_CUDA_TRY(cudaMemcpyAsync(norm, dec->norm, sizeof(float) * 4 * dec->d, cudaMemcpyDefault, s));
  return MPM_OK;
}

static mpm_status decoder_launch(const mpm_decoder* dec, const float* X, const int32_t* lat_idx,
                                 const float* latents, const float* dirs, const int32_t* kinds, int R, int64_t n,
                                 float* out, const int32_t* idx, const int32_t* n_dev, int n_rep, cudaStream_t s,
                                 const DecArgs* extra = nullptr);

mpm_status decoder_eval(const mpm_decoder* dec, const float* X, const int32_t* lat_idx, const float* latents,
                        const float* dirs, const int32_t* kinds, int R, int64_t n, float* out, void* stream) {
  MPM_CHECK_ARG(dec && kinds, "null argument");
  MPM_CHECK_ARG(n >= 0, "n >= 0");
  if (n == 0) return MPM_OK;
  return decoder_launch(dec, X, lat_idx, latents, dirs, kinds, R, n, out, nullptr, nullptr, 1,
                        (cudaStream_t)stream);
}

static mpm_status decoder_launch(const mpm_decoder* dec, const float* X, const int32_t* lat_idx,
                                 const float* latents, const float* dirs, const int32_t* kinds, int R, int64_t n,
                                 float* out, const int32_t* idx, const int32_t* n_dev, int n_rep, cudaStream_t s,
                                 const DecArgs* extra) {
  MPM_CHECK_ARG(R >= 1 && R <= kMaxR && R <= 128, "R must be in [1, 64]");
  MPM_CHECK_ARG(X && latents && out, "null argument");
  DecArgs a{};
  a.d = dec->d;
  a.r = dec->r;
  a.n_tc = dec->n_tc;
  a.act = dec->act;
  a.linear = dec->n_hidden == 0;
  a.W0 = dec->params + dec->w_off[0];
  a.b0 = dec->params + dec->b_off[0];
  a.bh = dec->bsq;
  const int L = (int)dec->w_off.size();
  a.Wout = dec->params + dec->w_off[L - 1];
  a.bout = dec->params + dec->b_off[L - 1];
  a.norm = dec->norm;
  a.wimg = dec->wimg;
  a.wimg_lo = dec->wimg_lo;
  a.w0img = dec->w0img;
  a.wsq = dec->wsq;
  a.wsqT = dec->wsqT;
  a.X = X;
  a.lat = lat_idx;
  a.latents = latents;
  a.dirs = dirs;
  a.n = n;
  a.R = R;
  a.Pt = 128 / R;
  a.n_dirs = 1;
  bool need_dirs = false, has_mixed = false;
  for (int k = 0; k < R; ++k) {
    const int c = kinds[k];
    const bool mixed = c > KIND_MIXED && c <= KIND_MIXED + dec->d + dec->r;
    const bool secant_dir = c >= KIND_SECANT_DIR && c < KIND_SECANT_DIR + kMaxR;
    MPM_CHECK_ARG(c == KIND_PRIMAL || (c >= 1 && c <= dec->d + dec->r) || c == KIND_JVP || c == KIND_SECANT ||
                      mixed || secant_dir,
                  "unknown row kind");
    need_dirs |= (c == KIND_JVP || c == KIND_SECANT || mixed || secant_dir);
    if (secant_dir) a.n_dirs = std::max(a.n_dirs, c - KIND_SECANT_DIR + 1);
    has_mixed |= mixed;
    a.kinds[k] = c;
    a.mix_jvp[k] = 0;
    a.mix_tan[k] = 0;
    if (mixed) {
      int kj = -1, kt = -1;
      for (int q = 0; q < R; ++q) {
        if (kinds[q] == KIND_JVP && kj < 0) kj = q;
        if (kinds[q] == c - KIND_MIXED && kt < 0) kt = q;
      }
      MPM_CHECK_ARG(kj >= 0 && kt >= 0, "a mixed row needs the JVP row and the tangent row of its input in the call");
      a.mix_jvp[k] = (int8_t)kj;
      a.mix_tan[k] = (int8_t)kt;
    }
  }
  MPM_CHECK_ARG(!need_dirs || dirs, "JVP / secant rows need dirs");
  MPM_CHECK_ARG(kinds[0] == KIND_PRIMAL || dec->n_tc == 0, "the first row kind must be the primal (0)");
  a.out = out;
  a.status = dec->status;
  a.idx = idx;
  a.n_dev = n_dev;
  a.n_rep = n_rep;
  if (extra) {
    a.lat_per_point = extra->lat_per_point;
    a.dstore = extra->dstore;
    a.astore = extra->astore;
    a.rows_total = extra->rows_total;
    MPM_CHECK_ARG(!a.dstore || dec->n_tc > 0, "training stores need square hidden layers");
    MPM_CHECK_ARG(!a.dstore || !has_mixed, "training stores take no mixed rows");
    MPM_CHECK_ARG(!a.dstore || R > 1, "training stores need the tangent rows (R > 1)");
    for (int k = 0; k < R && a.dstore; ++k)
      MPM_CHECK_ARG(a.kinds[k] == KIND_PRIMAL || (a.kinds[k] >= 1 && a.kinds[k] <= dec->d + dec->r) ||
                        a.kinds[k] == KIND_JVP,
                    "training stores take primal, tangent and JVP rows only");
  }
  // the tensor-core kernel's input layout holds r <= 36 latents (decoder_create allows d + r <= 40):
  // larger latents take the FP32 kernel
  const bool f32_path = (dec->fp32 == 1 || dec->r > 40 - kTcLat) && !a.dstore;
  if (dec->n_tc == 0) {
    int64_t rows = n * R;
    int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((rows + 127) / 128, dec->n_sm * 8));
    decoder_simt<<<blocks, 128, 0, s>>>(a);
  } else if (f32_path) {
    MPM_CHECK_ARG(R <= kF32Rows, "the FP32 path takes at most 64 row kinds");
    int64_t tiles;
    bool small = false;
    if (has_mixed) {
      // mixed rows read their JVP and tangent partners: point-aligned tiles
      a.f32_U = 0;
      a.Pt = kF32Rows / R;
      tiles = (n + a.Pt - 1) / a.Pt;
    } else {
      // packed tiles: about one per SM (per SM share of the concurrent callers), 32 or 64 slots
      const int64_t rows = n * R;
      const int64_t target = std::max(1, dec->n_sm / std::max(1, dec->concurrency));
      const int64_t U = std::max<int64_t>(1, std::min<int64_t>((rows + target - 1) / target, kF32Rows - 1));
      a.f32_U = (int)U;
      a.Pt = 1;
      small = U + 1 <= 32;
      tiles = (rows + U - 1) / U;
    }
    int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, dec->n_sm));
    if (small)
      decoder_f32<32><<<blocks, kF32Threads, dec_f32_smem_bytes(), s>>>(a);
    else
      decoder_f32<64><<<blocks, kF32Threads, dec_f32_smem_bytes(), s>>>(a);
  } else if (dec->fp32 == 0 && R == 1 && a.kinds[0] == KIND_PRIMAL && !a.dstore && !a.astore && dec->w0img &&
             kTcLat + dec->r <= 32) {
    // primal rows only: two tiles in flight per CTA
    const int64_t tiles = (n + 127) / 128;
    int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((tiles + 1) / 2, dec->n_sm));
    decoder_tc_primal<<<blocks, kPrimThreads, dec_primal_smem_bytes(), s>>>(a);
  } else {
    const int64_t tiles = (n + a.Pt - 1) / a.Pt;
    int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, dec->n_sm));
    if (dec->fp32 == 2 && !a.dstore)
      decoder_tc<true><<<blocks, kDecThreads, dec->smem_split, s>>>(a);
    else
      decoder_tc<false><<<blocks, kDecThreads, dec->smem, s>>>(a);
  }
  MPM_CUDA_TRY(cudaGetLastError());
  return MPM_OK;
}

}  // extern "C"

namespace mpmrom {
// Training forward: one latent and one JVP direction per point; stores the
// per-layer activations of every tile row and the primal rows' activation slopes.
mpm_status decoder_launch_train(const mpm_decoder* dec, const float* X, const float* latents, const float* dirs,
                                const int* kinds, int R, int64_t n, float* out, __nv_bfloat16* dstore,
                                __nv_bfloat16* astore, int64_t rows_total, cudaStream_t s) {
  DecArgs extra{};
  extra.lat_per_point = 1;
  extra.dstore = dstore;
  extra.astore = astore;
  extra.rows_total = rows_total;
  return decoder_launch(dec, X, nullptr, latents, dirs, kinds, R, n, out, nullptr, nullptr, 1, s, &extra);
}

mpm_status decoder_launch_dev(const mpm_decoder* dec, const float* X, const int32_t* idx, const int32_t* n_dev,
                              int n_rep, int64_t capacity, const float* latents, const float* dirs,
                              const int* kinds, int R, float* out, cudaStream_t s) {
  if (capacity <= 0) return MPM_OK;
  return decoder_launch(dec, X, nullptr, latents, dirs, kinds, R, capacity, out, idx, n_dev, n_rep, s);
}
}  // namespace mpmrom

extern "C" {

mpm_status decoder_status_word(mpm_decoder* dec, uint32_t* out, int clear, void* stream) {
  MPM_CHECK_ARG(dec && out, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t h = 0;
  MPM_CUDA_TRY(cudaMemcpyAsync(&h, dec->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  if (clear) MPM_CUDA_TRY(cudaMemsetAsync(dec->status, 0, sizeof(uint32_t), s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  *out = h;
  return MPM_OK;
}

}  // extern "C"

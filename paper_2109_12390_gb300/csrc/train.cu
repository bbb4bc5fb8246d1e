// Decoder training (Section 4.2 loss, Appendix B optimiser) on sm_103a.
//
// Per minibatch of B (snapshot, particle) pairs, rows per point
// [primal, dg/dX_0 .. dg/dX_{d-1}, JVP along (xhat_{n+1} - xhat_n) / dt_snap]:
//   train_sample     counter-based draw of the pairs (SplitMix64 of
//                    (seed, step, i), uniform over all pairs), gather of X,
//                    latents, JVP directions and targets
//   decoder_tc       forward (tensor cores), storing every hidden layer's
//                    activations and the primal rows' activation slopes (BF16,
//                    feature-major)
//   train_bwd_tc     loss residuals and output-layer gradients (FP32), then the
//                    reverse sweep: z_bar = act'(z) h_bar + act''(z) sum_j zdot_j t_bar_j
//                    for primal rows, zdot_bar = act'(z) t_bar for tangent rows; for
//                    ELU act''(z) zdot_j = [z < 0] a_j, the tangent row's stored
//                    activation, so the slope record and the activations suffice
//                    (exchanged through shared memory), next adjoint rows by a
//                    tcgen05 GEMM with the transposed weights resident in shared
//                    memory; layer 0 and the latent adjoints in FP32
//   train_dw_gemm    weight gradients of the square layers, dW = Zbar^T A, as
//                    split-K tcgen05 GEMMs over all rows (both operands stored
//                    row-contiguous, i.e. K-major), FP32 atomics across splits
//   train_dw0        first-layer weight gradient (K = d + r, FP32)
//   train_lat_scatter latent-table gradient (snapshot n gets d/dxhat_n of its
//                    own rows and -u_bar / dt; its successor gets +u_bar / dt)
//   train_adam       Adam on the FP32 master parameters and the latent table,
//                    learning rate decaying geometrically lr0 -> lr1
//   + re-pack of the BF16 weight images (forward and transposed)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "decoder_common.cuh"
#include "encoder.cuh"

namespace mpmrom {
mpm_status decoder_launch_train(const mpm_decoder* dec, const float* X, const float* latents, const float* dirs,
                                const int* kinds, int R, int64_t n, float* out, __nv_bfloat16* dstore,
                                __nv_bfloat16* astore, int64_t rows_total, cudaStream_t s);

__device__ __forceinline__ uint64_t tr_splitmix(uint64_t state, uint64_t k) {
  uint64_t z = state + 0x9E3779B97F4A7C15ull * (k + 1ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}


struct Store {
  int d, r;
  int n_snap;
  const int64_t* snap_base;   // (n_snap + 1) offsets of each snapshot's particle rows
  const int32_t* snap_inst;
  const int32_t* snap_next;
  const int64_t* inst_off;    // particle offsets into X
  const float* X;
  const float* x;
  const float* v;
  const float* F;
};

struct Batch {
  int64_t B;
  float* X;        // (B, d)
  float* xh;       // (B, r)
  float* u;        // (B, r)
  float* tx;       // (B, d)
  float* tv;       // (B, d)
  float* tF;       // (B, d, d)
  float* mask;     // (B)
  int32_t* snap;   // (B)
  int32_t* next;   // (B)
  int32_t* part;   // (B) particle index within its instance
};

// ------------------------------------------------------------- sampler
__global__ void train_sample(Store st, Batch b, const float* latents, float dt_snap, uint64_t seed,
                             const int64_t* step, double* loss, int64_t i_offset) {
  const int d = st.d, r = st.r;
  const int64_t total = st.snap_base[st.n_snap];
  const uint64_t s0 = tr_splitmix(seed, (uint64_t)*step);
  if (blockIdx.x == 0 && threadIdx.x == 0) *loss = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b.B; i += (int64_t)gridDim.x * blockDim.x) {
    // draw i_offset + i of the step's minibatch (a data-parallel shard holds a contiguous range)
    const uint64_t h = tr_splitmix(s0, (uint64_t)(i + i_offset));
    const int64_t g = (int64_t)(h % (uint64_t)total);
    // snapshot containing pair g: largest s with snap_base[s] <= g
    int lo = 0, hi = st.n_snap - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (st.snap_base[mid] <= g) lo = mid;
      else hi = mid - 1;
    }
    const int s = lo;
    const int64_t local = g - st.snap_base[s];
    const int inst = st.snap_inst[s];
    const int64_t pidx = st.inst_off[inst] + local;
    const int nx = st.snap_next[s];
    b.snap[i] = s;
    b.next[i] = nx;
    b.part[i] = (int32_t)local;
    for (int a = 0; a < d; ++a) {
      b.X[i * d + a] = st.X[pidx * d + a];
      b.tx[i * d + a] = st.x[g * d + a];
      b.tv[i * d + a] = st.v[g * d + a];
      for (int c = 0; c < d; ++c) b.tF[(i * d + a) * d + c] = st.F[(g * d + a) * d + c];
    }
    b.mask[i] = nx >= 0 ? 1.f : 0.f;
    for (int j = 0; j < r; ++j) {
      const float xs = latents[(int64_t)s * r + j];
      b.xh[i * r + j] = xs;
      b.u[i * r + j] = nx >= 0 ? (latents[(int64_t)nx * r + j] - xs) / dt_snap : 0.f;
    }
  }
}

// ------------------------------------------------------------- backward
struct BwdArgs {
  float n_norm;   // points of the whole minibatch (over all data-parallel shards)
  int d, r, n_hidden, n_tc, act, R, Pt;
  int64_t n, rows_total;
  const float* W0;      // (W, d + r)
  const float* Wout;    // (d, W)
  const float* norm;
  const __nv_bfloat16* dstore;   // primal rows' activation slopes (act_slope_record), feature-major
  const __nv_bfloat16* astore;
  const uint8_t* wtimg;
  const float* fwd;     // (R, n, d)
  Batch b;
  float lamF, lamv;
  __nv_bfloat16* zbstore;   // (n_tc, W, rows)
  float* zb0;               // (W, rows)
  float* gparams;
  int64_t gW0_off, gb0_off, gWout_off, gbout_off;
  int64_t gb_off[kMaxTC + 1];   // bias-gradient offsets of hidden layers 0..n_hidden-1
  float* g_lat_pt;          // (n, r)
  float* g_u_pt;            // (n, r)
  double* loss;
  uint32_t* status;
};

constexpr int kExchRows = 104;
constexpr int kBwdMaxR = 5;           // rows per point in training: primal, d <= 3 tangents, JVP
constexpr int kChunkStride = 33;      // padded row stride of one 32-feature chunk: distinct banks

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gmem_src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_groups() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// 256 threads: warps w and w + 4 read the same tensor-memory lane group; thread
// t owns tile row rw = 32 (w % 4) + lane and the feature half h = w / 4
// (features 64 h .. 64 h + 63) of every layer.
constexpr int kBwdThreads = 256;

__global__ void __launch_bounds__(kBwdThreads, 1) train_bwd_tc(BwdArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* wt = smem;                                 // n_tc x 32 KB (transposed square weights)
  uint8_t* atile = smem + kMaxTC * kLayerBytes;       // 32 KB
  float* exch = (float*)(atile + kLayerBytes);        // [2 halves][kExchRows][33]: tangent-row terms of the chunk
  __nv_bfloat16* sD = (__nv_bfloat16*)(exch + 2 * kExchRows * kChunkStride);  // [64 f][128 rows] slopes
  __nv_bfloat16* sA = sD + 64 * 128;                  // [64 f][128 rows] activations (f: 32 h + feature of chunk)
  float* sy = (float*)(sA + 64 * 128);                // 128 x 3
  float* sbias = sy + 128 * 3;                        // 128
  DecSmemTail* tail = (DecSmemTail*)(sbias + kW);
  __shared__ double s_loss[8];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int rw = (warp & 3) * 32 + lane;              // tile row / tensor-memory lane
  const int h = warp >> 2;                            // feature half
  const int d = a.d, R = a.R, Pt = a.Pt;

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
  if (t == 0 && a.n_tc > 0) {
    tc::mbar_expect_tx(&tail->bar_w, (uint32_t)(a.n_tc * kLayerBytes));
    for (int l = 0; l < a.n_tc; ++l)
      tc::bulk_g2s(wt + l * kLayerBytes, a.wtimg + (size_t)l * kLayerBytes, kLayerBytes, &tail->bar_w);
  }
  if (a.n_tc > 0 && !tc::mbar_wait(&tail->bar_w, 0)) {
    raise_status(a.status, STATUS_TIMEOUT);
    atomicExch(&tail->abort, 1);
  }
  if (t < kW) sbias[t] = 0.f;
  __syncthreads();
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, kW);
  uint32_t mma_phase = 0;
  const int64_t n_tiles = (a.n + Pt - 1) / Pt;
  const float* scale = a.norm + 3 * d;
  double my_loss = 0.0;

  for (int64_t tile = blockIdx.x; tile < n_tiles && !tail->abort; tile += gridDim.x) {
    const int64_t row0 = tile * 128;
    const int k = rw / Pt, q = rw % Pt;
    const int64_t p = tile * Pt + q;
    const bool valid = (k < R) && (p < a.n);
    const int cls = !valid ? -1 : (k == 0 ? 0 : 1);
    const int64_t gr = row0 + rw;
    // the slopes and activations of step i2z of layer lz (chunk 2 hh + i2z of each half hh),
    // copied asynchronously into the staging buffers in 16-byte pieces (8 rows of one feature) one
    // step ahead of their use, so that the loads overlap the current step: the activations of the
    // tile's 128 rows, the slope records of its first 32 rows only (the primal rows, Pt <= 32)
    auto prefetch_z = [&](int lz, int i2z) {
#pragma unroll
      for (int k2 = 0; k2 < 5; ++k2) {
        const int w = t + kBwdThreads * k2;                    // 64 features x (16 + 4) pieces
        const bool act = w < 64 * 16;
        const int fl = act ? w >> 4 : (w - 64 * 16) >> 2, c8 = act ? w & 15 : w & 3;
        const int fg = (2 * (fl >> 5) + i2z) * 32 + (fl & 31);   // global feature
        const __nv_bfloat16* src = (act ? a.astore : a.dstore) + ((int64_t)lz * kW + fg) * a.rows_total + row0 + 8 * c8;
        cp_async16((act ? sA : sD) + fl * 128 + 8 * c8, src);
      }
      cp_async_commit_group();
    };
    prefetch_z(a.n_hidden - 1, 0);
    // ---- output layer: residual adjoints ybar (FP32)
    float ybar[3] = {0.f, 0.f, 0.f};
    if (valid) {
      const float* o = a.fwd + ((int64_t)k * a.n + p) * d;
      // loops over the d <= 3 output components have compile-time bounds: with the runtime bound
      // the small register arrays they index (ybar, acc) are placed in local memory
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (i >= d) break;
        float e, w;
        if (k == 0) {
          e = o[i] - a.b.tx[p * d + i];
          w = 1.f;
        } else if (k <= d) {
          e = o[i] - a.b.tF[(p * d + i) * d + (k - 1)];
          w = a.lamF;
        } else {
          e = a.b.mask[p] * (o[i] - a.b.tv[p * d + i]);
          w = a.lamv;
        }
        if (h == 0) my_loss += (double)w * e * e;
        ybar[i] = 2.f * w * e * scale[i] / a.n_norm;
      }
    }
    if (h == 0)
      for (int i = 0; i < 3; ++i) sy[rw * 3 + i] = ybar[i];
    __syncthreads();
    {
      // dWout[i][f] = sum_rows ybar_i a_last[f]: thread = feature f = t % 128, rows 64 (t / 128) ..
      const int f = t & 127, rh = t >> 7;
      const __nv_bfloat16* al = a.astore + (int64_t)(a.n_hidden - 1) * kW * a.rows_total + (int64_t)f * a.rows_total +
                                row0 + 64 * rh;
      float acc[3] = {0.f, 0.f, 0.f};
      // unrolled: the eight 16-byte loads of the stored activations are in flight together
#pragma unroll
      for (int c = 0; c < 64; c += 8) {
        const uint4 u = *reinterpret_cast<const uint4*>(al + c);
        const __nv_bfloat16* hv = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float av = __bfloat162float(hv[j]);
#pragma unroll
          for (int i = 0; i < 3; ++i)
            if (i < d) acc[i] = fmaf(sy[(64 * rh + c + j) * 3 + i], av, acc[i]);
        }
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (i < d) atomicAdd(&a.gparams[a.gWout_off + i * kW + f], acc[i]);
      if (t < d) {
        float sb = 0.f;
        for (int q2 = 0; q2 < Pt; ++q2) sb += sy[q2 * 3 + t];
        atomicAdd(&a.gparams[a.gbout_off + t], sb);
      }
    }
    // ---- reverse sweep over the hidden layers
    for (int l = a.n_hidden - 1; l >= 0; --l) {
      const bool from_tmem = (l < a.n_hidden - 1);
      if (from_tmem) {
        if (!tc::mbar_wait(&tail->bar_mma, mma_phase)) {
          raise_status(a.status, STATUS_TIMEOUT);
          atomicExch(&tail->abort, 1);
        }
        mma_phase ^= 1u;
        tc::tc_fence_after();
      }
      cp_async_wait_groups();   // this thread's staging copies of the step have landed
      __syncthreads();
      if (tail->abort) break;
      for (int i2 = 0; i2 < 2; ++i2) {
        const int ch = 2 * h + i2;
        float hb[32];
        if (from_tmem) {
          tc::tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + ch * 32, hb);
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            float sacc = 0.f;
#pragma unroll
            for (int o = 0; o < 3; ++o)
              if (o < d) sacc = fmaf(__ldg(&a.Wout[o * kW + ch * 32 + i]), ybar[o], sacc);
            hb[i] = sacc;
          }
        }
        float zb[32];
        // the point's primal slope record s (row q): act'(z) = s, or 1 where s < 0; for tangent
        // rows the curvature term act''(z) zdot is the row's own activation where s >= 0 (z < 0)
        float sown[32];
        const __nv_bfloat16* hD = sD + (h * 32) * 128;
        const __nv_bfloat16* hA = sA + (h * 32) * 128;
        if (cls == 0) {   // before the barrier: the staging buffer is refilled after it
#pragma unroll
          for (int i = 0; i < 32; ++i) sown[i] = __bfloat162float(hD[i * 128 + rw]);
        }
        float* hexch = exch + h * kExchRows * kChunkStride;
        if (cls == 1) {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float sp = __bfloat162float(hD[i * 128 + q]);
            const float at = __bfloat162float(hA[i * 128 + rw]);
            zb[i] = (sp < 0.f ? 1.f : sp) * hb[i];
            hexch[(rw - Pt) * kChunkStride + i] = (sp >= 0.f ? at : 0.f) * hb[i];
          }
        }
        __syncthreads();
        // every row has read the staged step: stage the next one (this layer's other chunk of
        // each half, or the next layer's first)
        if (i2 == 0) prefetch_z(l, 1);
        else if (l > 0) prefetch_z(l - 1, 0);
        if (cls == 0) {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            float sacc = (sown[i] < 0.f ? 1.f : sown[i]) * hb[i];
            // compile-time bound (R <= kBwdMaxR): with the runtime bound this loop, inside the
            // unrolled feature loop, ran about 1,000 cycles per feature
#pragma unroll
            for (int kk = 1; kk < kBwdMaxR; ++kk)
              if (kk < R) sacc += hexch[((kk - 1) * Pt + q) * kChunkStride + i];
            zb[i] = sacc;
          }
        } else if (cls < 0) {
#pragma unroll
          for (int i = 0; i < 32; ++i) zb[i] = 0.f;
        }
        // bias gradient: sum of the primal rows' z_bar (primal rows all sit in lane group 0);
        // transpose-reduce the 32 columns across the warp so lane i ends with column i
        if ((warp & 3) == 0) {
          float v[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = (cls == 0) ? zb[i] : 0.f;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < o; ++i) {
              // lanes with bit o set keep the upper half of the columns, the others the lower half
              const float send = up ? v[i] : v[i + o];
              const float keep = up ? v[i + o] : v[i];
              v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
          }
          sbias[ch * 32 + lane] += v[0];
        }
        if (l >= 1) {
#pragma unroll
          for (int j = 0; j < 32; j += 8) store_bf16x8(atile, rw, ch * 32 + j, zb + j);
        } else {
          // first-layer adjoints (FP32); the first-layer weight gradient and the latent
          // adjoints are formed from them by train_dw0_lat
          float* zs = a.zb0 + gr;
#pragma unroll
          for (int i = 0; i < 32; ++i) zs[(int64_t)(ch * 32 + i) * a.rows_total] = zb[i];
        }
        if (i2 == 0) cp_async_wait_groups();   // the next chunk's staging has landed
        __syncthreads();
      }
      // bias gradient of layer l (sbias was filled before the last barrier)
      if (t < kW) {
        atomicAdd(&a.gparams[a.gb_off[l] + t], sbias[t]);
        sbias[t] = 0.f;
      }
      if (l >= 1) {
        // next adjoint rows: h_bar_{l-1} = z_bar_l W_l  (B operand = W_l^T image)
        tc::fence_async_smem();
        tc::tc_fence_before();
        __syncthreads();
        if (t == 0) {
          tc::tc_fence_after();
          const uint32_t a_base = tc::smem_addr(atile), b_base = tc::smem_addr(wt + (l - 1) * kLayerBytes);
#pragma unroll
          for (int kk = 0; kk < kW / 16; ++kk) {
            const uint32_t koff = (uint32_t)((kk >> 2) * (kW * 128) + (kk & 3) * 32);
            tc::mma_bf16(tmem, tc::smem_desc_sw128(a_base + koff), tc::smem_desc_sw128(b_base + koff), idesc,
                         kk > 0 ? 1u : 0u);
          }
          tc::mma_commit(&tail->bar_mma);
        }
        // the adjoints of layer l (BF16, for the weight-gradient GEMMs) leave the operand tile while
        // the tensor core reads it; the barrier after the next wait orders these reads before the
        // next writes of the tile
        copy_out_tile(a.zbstore + (int64_t)(l - 1) * kW * a.rows_total, a.rows_total, atile, tile, t);
      }
    }
    if (tail->abort) break;
    tc::tc_fence_before();
    __syncthreads();
  }
  // loss (sum over rows of w e^2; the caller divides by n)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_loss += __shfl_down_sync(0xffffffffu, my_loss, o);
  if ((t & 31) == 0) s_loss[warp] = my_loss;
  __syncthreads();
  if (t == 0) {
    double tot = 0.0;
    for (int w = 0; w < kBwdThreads / 32; ++w) tot += s_loss[w];
    atomicAdd(a.loss, tot);
  }
  cp_async_wait_groups();   // no staging copy outlives the CTA (an aborted sweep)
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_free<kW>(tmem);
}

// ------------------------------------------- weight gradients (split-K GEMM)
// dW_l[out][in] = sum_rows Zbar[out][row] A[in][row]; Zbar = zbstore[l], A = astore[l]
// (the activations entering square layer l + 1).  Grid (n_tc, splits), 128 threads.
__global__ void __launch_bounds__(128, 1) train_dw_gemm(const __nv_bfloat16* zbstore, const __nv_bfloat16* astore,
                                                        int64_t rows_total, int64_t k_per_split, float* gparams,
                                                        const int64_t* w_off, uint32_t* status) {
  __shared__ __align__(1024) uint8_t sA[kW * 128];
  __shared__ __align__(1024) uint8_t sB[kW * 128];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  const int t = threadIdx.x, warp = t >> 5;
  const int l = blockIdx.x;
  const __nv_bfloat16* Z = zbstore + (int64_t)l * kW * rows_total;
  const __nv_bfloat16* A = astore + (int64_t)l * kW * rows_total;
  const int64_t k0 = (int64_t)blockIdx.y * k_per_split;
  const int64_t k1 = min(rows_total, k0 + k_per_split);
  if (t == 0) {
    tc::mbar_init(&bar, 1);
    abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc<kW>(&tslot);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tslot;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, kW);
  uint32_t phase = 0;
  bool any = false;
  for (int64_t kb = k0; kb < k1; kb += 64) {
    // stage 128 x 64 blocks of both operands (K-major, 128-byte swizzle)
    for (int e = t; e < kW * 8; e += blockDim.x) {
      const int row = e >> 3, c = e & 7;
      uint4 za = make_uint4(0, 0, 0, 0), zb = make_uint4(0, 0, 0, 0);
      if (kb + c * 8 < k1) {
        za = *reinterpret_cast<const uint4*>(Z + (int64_t)row * rows_total + kb + c * 8);
        zb = *reinterpret_cast<const uint4*>(A + (int64_t)row * rows_total + kb + c * 8);
      }
      *reinterpret_cast<uint4*>(sA + tc::sw128_offset(row, c * 8, kW)) = za;
      *reinterpret_cast<uint4*>(sB + tc::sw128_offset(row, c * 8, kW)) = zb;
    }
    tc::fence_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc::tc_fence_after();
      const uint32_t a_base = tc::smem_addr(sA), b_base = tc::smem_addr(sB);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        tc::mma_bf16(tmem, tc::smem_desc_sw128(a_base + kk * 32), tc::smem_desc_sw128(b_base + kk * 32), idesc,
                     (any || kk > 0) ? 1u : 0u);
      tc::mma_commit(&bar);
    }
    any = true;
    if (!tc::mbar_wait(&bar, phase)) {
      raise_status(status, STATUS_TIMEOUT);
      atomicExch(&abort_flag, 1);
    }
    phase ^= 1u;
    tc::tc_fence_after();
    __syncthreads();
    if (abort_flag) break;
  }
  if (any && !abort_flag) {
    float* g = gparams + w_off[l + 1];
    for (int ch = 0; ch < kW / 32; ++ch) {
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + ch * 32, v);
      float4* g4 = reinterpret_cast<float4*>(g + t * kW + ch * 32);
#pragma unroll
      for (int i = 0; i < 8; ++i) atomicAdd(g4 + i, make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]));
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_free<kW>(tmem);
}

// First-layer weight gradient dW0[f][j] = sum_rows zbar0[f][row] in[row][j] and the latent
// adjoints of the primal rows (d loss / d xhat) and of the JVP rows (d loss / d u),
// sum_f zbar0[f][row] W0[f][d + j], from one pass over zbar0.  in[row] is the layer-0 input of
// the row: [Xn, xhat] (primal), e_k / X_range_k (X tangent k), [0, u] (JVP).
// One 128-row training tile at a time (rows k Pt + q: kind k of point q): its 128 x 128 block of
// zbar0 is staged in shared memory by float4 loads (512 contiguous bytes per feature), the
// points' inputs beside it.  Thread (f, half) sums the weight gradient of feature f over half
// of the tile's points in registers for every tile the CTA takes, and adds it to dW0 once;
// the latent adjoints take (row, 4 latents) per thread.
constexpr int kMaxIn = 40;
constexpr int kDw0Stride = 132;       // floats per staged feature row (128 rows + pad; float4 aligned)
constexpr int kDw0MaxPt = 64;         // points per tile (R >= 2)
template <int D>
__global__ void __launch_bounds__(256) train_dw0_lat(const float* zb0, int64_t rows_total, Batch b, int r, int Pt,
                                                     const float* norm, const float* W0, float* gW0, float* g_lat_pt,
                                                     float* g_u_pt) {
  constexpr int d = D;
  extern __shared__ __align__(16) float dsm[];
  float* sz = dsm;                                   // [128 f][kDw0Stride]: zbar0 of the tile's rows
  float* sin0 = sz + kW * kDw0Stride;                // [kDw0MaxPt][kMaxIn]: primal inputs of the points
  float* su = sin0 + kDw0MaxPt * kMaxIn;             // [kDw0MaxPt][32]: JVP directions
  float* sWl = su + kDw0MaxPt * 32;                  // [128][36]: latent columns of W0 (float4 rows)
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int K = d + r;
  for (int e = t; e < kW * 36; e += blockDim.x) {
    const int ff = e / 36, j = e % 36;
    sWl[e] = j < r ? W0[ff * K + d + j] : 0.f;
  }
  const int f = t & (kW - 1), half = t >> 7;
  const int q_lo = half ? (Pt + 1) / 2 : 0, q_hi = half ? Pt : (Pt + 1) / 2;
  float inv_range[D];
#pragma unroll
  for (int a2 = 0; a2 < D; ++a2) inv_range[a2] = 1.f / norm[D + a2];
  float acc[kMaxIn];
#pragma unroll
  for (int j = 0; j < kMaxIn; ++j) acc[j] = 0.f;
  const int64_t n_tiles = rows_total / 128;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t row0 = tile * 128;
    __syncthreads();   // the previous tile's staged values are consumed
    // zbar0 rows of the tile: warp w stages features w, w + 8, ..., one float4 per lane
    for (int ff = warp; ff < kW; ff += 8) {
      const float4 v = *reinterpret_cast<const float4*>(zb0 + (int64_t)ff * rows_total + row0 + 4 * lane);
      *reinterpret_cast<float4*>(sz + ff * kDw0Stride + 4 * lane) = v;
    }
    // the points' primal inputs [Xn, xhat] and JVP directions
    for (int e = t; e < Pt * kMaxIn; e += blockDim.x) {
      const int q = e / kMaxIn, j = e % kMaxIn;
      const int64_t pnt = tile * Pt + q;
      float in = 0.f;
      if (pnt < b.B && j < K) in = j < d ? (b.X[pnt * d + j] - norm[j]) / norm[d + j] : b.xh[pnt * r + (j - d)];
      sin0[q * kMaxIn + j] = in;
    }
    for (int e = t; e < Pt * 32; e += blockDim.x) {
      const int q = e >> 5, j = e & 31;
      const int64_t pnt = tile * Pt + q;
      su[e] = (pnt < b.B && j < r) ? b.u[pnt * r + j] : 0.f;
    }
    __syncthreads();
    // (a) weight gradient of feature f over this thread's points (rows of invalid points are zero)
    const float* zf = sz + f * kDw0Stride;
    // four points at a time with float4 reads of the staged adjoints where the rows allow it (a
    // quarter warp's 16-byte reads then fall in distinct banks; the scalar reads of lanes 132
    // floats apart conflict 4 ways)
    const bool vec4 = (Pt & 3) == 0 && (q_lo & 3) == 0 && (q_hi & 3) == 0;
    for (int q4 = q_lo; vec4 && q4 < q_hi; q4 += 4) {
      const float4 zp4 = *reinterpret_cast<const float4*>(zf + q4);
      float4 zt4[D];
#pragma unroll
      for (int a2 = 0; a2 < D; ++a2) zt4[a2] = *reinterpret_cast<const float4*>(zf + (1 + a2) * Pt + q4);
      const float4 zj4 = *reinterpret_cast<const float4*>(zf + (D + 1) * Pt + q4);
#pragma unroll
      for (int u4 = 0; u4 < 4; ++u4) {
        const int q = q4 + u4;
        const float zp = u4 == 0 ? zp4.x : u4 == 1 ? zp4.y : u4 == 2 ? zp4.z : zp4.w;
        const float zj = u4 == 0 ? zj4.x : u4 == 1 ? zj4.y : u4 == 2 ? zj4.z : zj4.w;
        const float* in = sin0 + q * kMaxIn;
#pragma unroll
        for (int j = 0; j < kMaxIn; j += 4) {
          if (j < K) {
            const float4 v = *reinterpret_cast<const float4*>(in + j);
            acc[j] = fmaf(zp, v.x, acc[j]);
            acc[j + 1] = fmaf(zp, v.y, acc[j + 1]);
            acc[j + 2] = fmaf(zp, v.z, acc[j + 2]);
            acc[j + 3] = fmaf(zp, v.w, acc[j + 3]);
          }
        }
#pragma unroll
        for (int a2 = 0; a2 < D; ++a2) {
          const float zt = u4 == 0 ? zt4[a2].x : u4 == 1 ? zt4[a2].y : u4 == 2 ? zt4[a2].z : zt4[a2].w;
          acc[a2] = fmaf(zt, inv_range[a2], acc[a2]);
        }
        const float* uq = su + q * 32;
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          if (j < r) {
            const float4 v = *reinterpret_cast<const float4*>(uq + j);
            acc[D + j] = fmaf(zj, v.x, acc[D + j]);
            acc[D + j + 1] = fmaf(zj, v.y, acc[D + j + 1]);
            acc[D + j + 2] = fmaf(zj, v.z, acc[D + j + 2]);
            acc[D + j + 3] = fmaf(zj, v.w, acc[D + j + 3]);
          }
        }
      }
    }
    for (int q = q_lo; !vec4 && q < q_hi; ++q) {
      const float zp = zf[q];                        // primal row
      const float* in = sin0 + q * kMaxIn;
#pragma unroll
      for (int j = 0; j < kMaxIn; j += 4) {
        if (j < K) {
          const float4 v = *reinterpret_cast<const float4*>(in + j);
          acc[j] = fmaf(zp, v.x, acc[j]);
          acc[j + 1] = fmaf(zp, v.y, acc[j + 1]);
          acc[j + 2] = fmaf(zp, v.z, acc[j + 2]);
          acc[j + 3] = fmaf(zp, v.w, acc[j + 3]);
        }
      }
#pragma unroll
      for (int a2 = 0; a2 < D; ++a2)                 // X-tangent rows: one input each
        acc[a2] = fmaf(zf[(1 + a2) * Pt + q], inv_range[a2], acc[a2]);
      const float zj = zf[(D + 1) * Pt + q];         // JVP row: [0, u] (u zero-padded to 32)
      const float* uq = su + q * 32;
#pragma unroll
      for (int j = 0; j < 32; j += 4) {
        if (j < r) {
          const float4 v = *reinterpret_cast<const float4*>(uq + j);
          acc[D + j] = fmaf(zj, v.x, acc[D + j]);
          acc[D + j + 1] = fmaf(zj, v.y, acc[D + j + 1]);
          acc[D + j + 2] = fmaf(zj, v.z, acc[D + j + 2]);
          acc[D + j + 3] = fmaf(zj, v.w, acc[D + j + 3]);
        }
      }
    }
    // (b) latent adjoints of the primal (k = 0) and JVP (k = d + 1) rows: (row, 4 latents) per thread
    const int n_groups = (r + 3) / 4;
    for (int o = t; o < 2 * Pt * n_groups; o += blockDim.x) {
      const int g = o % n_groups, rr = o / n_groups;
      const int q = rr % Pt, jvp = rr / Pt;
      const int64_t pnt = tile * Pt + q;
      const int row = (jvp ? d + 1 : 0) * Pt + q;
      float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
#pragma unroll 8
      for (int ff = 0; ff < kW; ++ff) {
        const float z = sz[ff * kDw0Stride + row];
        const float4 w = *reinterpret_cast<const float4*>(sWl + ff * 36 + 4 * g);
        v0 = fmaf(z, w.x, v0);
        v1 = fmaf(z, w.y, v1);
        v2 = fmaf(z, w.z, v2);
        v3 = fmaf(z, w.w, v3);
      }
      if (pnt < b.B) {
        float* dst = (jvp ? g_u_pt : g_lat_pt) + pnt * r + 4 * g;
        const int nj = min(4, r - 4 * g);
        if (nj > 0) dst[0] = v0;
        if (nj > 1) dst[1] = v1;
        if (nj > 2) dst[2] = v2;
        if (nj > 3) dst[3] = v3;
      }
    }
  }
  // combine the two halves of each feature, then one atomic per weight
  __syncthreads();
  float* red = sz;   // reused as [128][kMaxIn + 1]
  if (half == 1) {
#pragma unroll
    for (int j = 0; j < kMaxIn; ++j) red[f * (kMaxIn + 1) + j] = acc[j];
  }
  __syncthreads();
  if (half == 0) {
#pragma unroll
    for (int j = 0; j < kMaxIn; ++j)
      if (j < K) atomicAdd(&gW0[f * K + j], acc[j] + red[f * (kMaxIn + 1) + j]);
  }
}

size_t dw0_smem_bytes() {
  return (size_t)(kW * kDw0Stride + kDw0MaxPt * kMaxIn + kDw0MaxPt * 32 + kW * 36) * sizeof(float);
}

__global__ void train_lat_scatter(Batch b, int r, const float* g_lat_pt, const float* g_u_pt, float dt_snap,
                                  float* g_lat) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < b.B; p += (int64_t)gridDim.x * blockDim.x) {
    const int s = b.snap[p], nx = b.next[p];
    for (int j = 0; j < r; ++j) {
      const float gu = g_u_pt[p * r + j] / dt_snap;
      atomicAdd(&g_lat[(int64_t)s * r + j], g_lat_pt[p * r + j] - (nx >= 0 ? gu : 0.f));
      if (nx >= 0) atomicAdd(&g_lat[(int64_t)nx * r + j], gu);
    }
  }
}

// Adam (Kingma and Ba 2015) on two parameter ranges; zeroes the gradients.
__global__ void train_adam(float* p0, float* g0, float* m0, float* v0, int64_t n0, float* p1, float* g1, float* m1,
                           float* v1, int64_t n1, const int64_t* step, int64_t total_steps, float lr0, float lr1,
                           float beta1, float beta2, float eps, int update) {
  const int64_t t = *step;
  const float frac = total_steps > 1 ? (float)min(t, total_steps - 1) / (float)(total_steps - 1) : 0.f;
  const float lr = lr0 * powf(lr1 / lr0, frac);
  const float bc1 = 1.f - powf(beta1, (float)(t + 1)), bc2 = 1.f - powf(beta2, (float)(t + 1));
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n0 + n1; i += (int64_t)gridDim.x * blockDim.x) {
    float *p, *g, *m, *v;
    int64_t j = i;
    if (i < n0) {
      p = p0; g = g0; m = m0; v = v0;
    } else {
      j = i - n0;
      p = p1; g = g1; m = m1; v = v1;
    }
    const float gr = g[j];
    g[j] = 0.f;
    if (!update) continue;
    const float mm = beta1 * m[j] + (1.f - beta1) * gr;
    const float vv = beta2 * v[j] + (1.f - beta2) * gr * gr;
    m[j] = mm;
    v[j] = vv;
    p[j] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
  }
}

__global__ void train_step_inc(int64_t* step) { *step += 1; }

// Transposed BF16 images of the square layers: image row = input feature, K = output feature.
__global__ void train_pack_transposed(const float* params, const int64_t* w_off, int n_tc, uint8_t* img) {
  const int64_t total = (int64_t)n_tc * kW * kW;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(i / (kW * kW));
    const int rem = (int)(i % (kW * kW));
    const int out = rem / kW, in = rem % kW;
    const float w = params[w_off[l + 1] + rem];  // W[out][in]
    *reinterpret_cast<__nv_bfloat16*>(img + (size_t)l * kLayerBytes + tc::sw128_offset(in, out, kW)) =
        __float2bfloat16_rn(w);
  }
}

}  // namespace mpmrom

using namespace mpmrom;

struct trainer_ctx {
  mpm_decoder* dec = nullptr;
  train_config cfg{};
  int d = 0, r = 0, R = 0, Pt = 0, n_sm = 0;
  int64_t B = 0, n_tiles = 0, rows_total = 0, n_snap = 0;
  int64_t i_offset = 0;   // first draw of this shard in the step's minibatch
  float n_norm = 0.f;     // points of the whole minibatch (batch x shards)
  Store st{};
  Batch b{};
  // device buffers
  int64_t* snap_base = nullptr;
  int32_t* snap_inst = nullptr;
  int32_t* snap_next = nullptr;
  int64_t* inst_off = nullptr;
  float* X = nullptr;
  float* sx = nullptr;
  float* sv = nullptr;
  float* sF = nullptr;
  float* latents = nullptr;
  float* g_lat = nullptr;
  float* m_lat = nullptr;
  float* v_lat = nullptr;
  float* gparams = nullptr;
  float* m_par = nullptr;
  float* v_par = nullptr;
  float* batch_mem = nullptr;
  int32_t* batch_idx = nullptr;
  float* fwd = nullptr;
  __nv_bfloat16* dstore = nullptr;   // primal rows' activation slopes (n_hidden, W, rows)
  __nv_bfloat16* astore = nullptr;
  __nv_bfloat16* zbstore = nullptr;
  float* zb0 = nullptr;
  float* g_lat_pt = nullptr;
  float* g_u_pt = nullptr;
  uint8_t* wtimg = nullptr;
  int64_t* d_w_off = nullptr;
  int64_t* step = nullptr;
  double* loss = nullptr;
  uint32_t* status = nullptr;
  size_t bwd_smem = 0;
  // encoder (Section 4.1) in place of the latent table
  bool enc = false;
  EncDesc E{};
  float* U = nullptr;           // (n_snap, L0) standardised subset positions
  float* enc_p = nullptr;       // parameters, gradients, Adam moments
  float* enc_g = nullptr;
  float* enc_m = nullptr;
  float* enc_v = nullptr;
  float* enc_ss = nullptr;      // shift (d), scale (d)
  double* enc_work = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  cudaGraphExec_t graph_noupdate = nullptr;
};


// ---------------------------------------------------------------------------------------------
// Input and output scaling of Appendix B: per coordinate, min-max of the reference positions X
// and mean / standard deviation of every snapshot position x.  Pass 1: per-block minimum and
// maximum of X and FP64 sum of x; pass 2: FP64 sum of (x - mean)^2 with the pass-1 mean.  One
// block reduces the partials after each pass.
// ---------------------------------------------------------------------------------------------
constexpr int kScaleThreads = 256;

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;   // valid in thread 0
}

__device__ __forceinline__ float block_minmax(float v, bool is_max, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float u = __shfl_down_sync(0xffffffffu, v, o);
    v = is_max ? fmaxf(v, u) : fminf(v, u);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  float t = v;
  if (threadIdx.x == 0)
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = is_max ? fmaxf(t, sh[w]) : fminf(t, sh[w]);
  return t;   // valid in thread 0
}

// pass 0: part[b] = {min X_a, max X_a, sum x_a}, pass 1: part[b] = {sum (x_a - mean_a)^2}
__global__ void __launch_bounds__(kScaleThreads) scale_partials(int pass, int d, const float* __restrict__ X,
                                                                int64_t nX, const float* __restrict__ x, int64_t nx,
                                                                const double* __restrict__ mean, double* part) {
  __shared__ double shd[kScaleThreads / 32];
  __shared__ float shf[kScaleThreads / 32];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int a = 0; a < d; ++a) {
    if (pass == 0) {
      float lo = INFINITY, hi = -INFINITY;
      for (int64_t i = i0; i < nX; i += stride) {
        const float u = X[i * d + a];
        lo = fminf(lo, u);
        hi = fmaxf(hi, u);
      }
      double s = 0.0;
      for (int64_t i = i0; i < nx; i += stride) s += (double)x[i * d + a];
      lo = block_minmax(lo, false, shf);
      hi = block_minmax(hi, true, shf);
      s = block_sum_d(s, shd);
      if (threadIdx.x == 0) {
        part[(size_t)blockIdx.x * 3 * d + 3 * a + 0] = lo;
        part[(size_t)blockIdx.x * 3 * d + 3 * a + 1] = hi;
        part[(size_t)blockIdx.x * 3 * d + 3 * a + 2] = s;
      }
    } else {
      const double m = mean[a];
      double s = 0.0;
      for (int64_t i = i0; i < nx; i += stride) {
        const double e = (double)x[i * d + a] - m;
        s = fma(e, e, s);
      }
      s = block_sum_d(s, shd);
      if (threadIdx.x == 0) part[(size_t)blockIdx.x * d + a] = s;
    }
  }
}

// one thread per coordinate: reduce the partials; pass 0 leaves the mean in stats[0..d), pass 1
// writes the decoder's scaling {X_min, X_range, mean, std} (as floats) into norm
__global__ void scale_finish(int pass, int d, int n_part, int64_t nx, const double* part, double* stats,
                             float* norm) {
  const int a = threadIdx.x;
  if (a >= d) return;
  if (pass == 0) {
    double lo = INFINITY, hi = -INFINITY, s = 0.0;
    for (int b = 0; b < n_part; ++b) {
      lo = fmin(lo, part[(size_t)b * 3 * d + 3 * a + 0]);
      hi = fmax(hi, part[(size_t)b * 3 * d + 3 * a + 1]);
      s += part[(size_t)b * 3 * d + 3 * a + 2];
    }
    stats[a] = s / (double)nx;
    stats[d + a] = lo;
    stats[2 * d + a] = hi;
  } else {
    double ss = 0.0;
    for (int b = 0; b < n_part; ++b) ss += part[(size_t)b * d + a];
    norm[a] = (float)stats[d + a];
    norm[d + a] = (float)(stats[2 * d + a] - stats[d + a]);
    norm[2 * d + a] = (float)stats[a];
    norm[3 * d + a] = (float)sqrt(ss / (double)nx);
  }
}

namespace {

mpm_status train_launch_update(trainer_ctx* c, cudaStream_t s);

mpm_status train_launch_step(trainer_ctx* c, cudaStream_t s, int update) {
  mpm_decoder* dec = c->dec;
  const int d = c->d, r = c->r;
  int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((c->B + 255) / 256, (int64_t)c->n_sm * 8));
  if (c->enc) {
    // latents of every snapshot from the encoder
    mpm_status se = enc_forward(c->E, c->enc_p, c->U, c->n_snap, c->latents, c->n_sm, s);
    if (se != MPM_OK) return se;
  }
  train_sample<<<blocks, 256, 0, s>>>(c->st, c->b, c->latents, c->cfg.dt_snap, c->cfg.seed, c->step, c->loss,
                                      c->i_offset);
  MPM_CUDA_TRY(cudaGetLastError());
  int kinds[8];
  kinds[0] = 0;
  for (int a = 0; a < d; ++a) kinds[1 + a] = 1 + a;
  kinds[1 + d] = 1000;
  mpm_status st = decoder_launch_train(dec, c->b.X, c->b.xh, c->b.u, kinds, c->R, c->B, c->fwd, c->dstore, c->astore,
                                       c->rows_total, s);
  if (st != MPM_OK) return st;
  BwdArgs a{};
  a.d = d;
  a.r = r;
  a.n_hidden = dec->n_hidden;
  a.n_tc = dec->n_tc;
  a.act = dec->act;
  a.R = c->R;
  a.Pt = c->Pt;
  a.n = c->B;
  a.n_norm = c->n_norm;
  a.rows_total = c->rows_total;
  const int L = (int)dec->w_off.size();
  a.W0 = dec->params + dec->w_off[0];
  a.Wout = dec->params + dec->w_off[L - 1];
  a.norm = dec->norm;
  a.dstore = c->dstore;
  a.astore = c->astore;
  a.wtimg = c->wtimg;
  a.fwd = c->fwd;
  a.b = c->b;
  a.lamF = c->cfg.lambda_F;
  a.lamv = c->cfg.lambda_v;
  a.zbstore = c->zbstore;
  a.zb0 = c->zb0;
  a.gparams = c->gparams;
  a.gW0_off = dec->w_off[0];
  a.gb0_off = dec->b_off[0];
  a.gWout_off = dec->w_off[L - 1];
  a.gbout_off = dec->b_off[L - 1];
  for (int l = 0; l < dec->n_hidden; ++l) a.gb_off[l] = dec->b_off[l];
  a.g_lat_pt = c->g_lat_pt;
  a.g_u_pt = c->g_u_pt;
  a.loss = c->loss;
  a.status = c->status;
  const int bw = (int)std::max<int64_t>(1, std::min<int64_t>(c->n_tiles, c->n_sm));
  train_bwd_tc<<<bw, kBwdThreads, c->bwd_smem, s>>>(a);
  MPM_CUDA_TRY(cudaGetLastError());
  if (dec->n_tc > 0) {
    // four CTAs per SM (32 KB of shared memory and 128 TMEM columns each), so that four K blocks'
    // loads are in flight per SM; the splits' partial sums meet in vector reductions
    const int splits = std::max(1, 4 * c->n_sm / dec->n_tc);
    int64_t kps = (c->rows_total + splits - 1) / splits;
    kps = (kps + 63) / 64 * 64;
    dim3 g(dec->n_tc, (unsigned)((c->rows_total + kps - 1) / kps));
    train_dw_gemm<<<g, 128, 0, s>>>(c->zbstore, c->astore, c->rows_total, kps, c->gparams, c->d_w_off, c->status);
    MPM_CUDA_TRY(cudaGetLastError());
  }
  if (d == 2)
    train_dw0_lat<2><<<c->n_sm * 2, 256, dw0_smem_bytes(), s>>>(c->zb0, c->rows_total, c->b, r, c->Pt, dec->norm,
                                                               dec->params + dec->w_off[0], c->gparams + dec->w_off[0],
                                                               c->g_lat_pt, c->g_u_pt);
  else
    train_dw0_lat<3><<<c->n_sm * 2, 256, dw0_smem_bytes(), s>>>(c->zb0, c->rows_total, c->b, r, c->Pt, dec->norm,
                                                               dec->params + dec->w_off[0], c->gparams + dec->w_off[0],
                                                               c->g_lat_pt, c->g_u_pt);
  MPM_CUDA_TRY(cudaGetLastError());
  train_lat_scatter<<<blocks, 256, 0, s>>>(c->b, r, c->g_lat_pt, c->g_u_pt, c->cfg.dt_snap, c->g_lat);
  MPM_CUDA_TRY(cudaGetLastError());
  if (c->enc) {
    // pull the per-snapshot latent gradients back through the encoder
    st = enc_backward(c->E, c->enc_p, c->U, c->n_snap, c->g_lat, c->enc_g, c->n_sm, s);
    if (st != MPM_OK) return st;
  }
  if (update) return train_launch_update(c, s);
  return MPM_OK;
}

// Adam on the decoder and on the latent table or the encoder (the gradients are consumed and
// zeroed), re-pack of the weight images, step count.
mpm_status train_launch_update(trainer_ctx* c, cudaStream_t s) {
  mpm_decoder* dec = c->dec;
  const int r = c->r;
  mpm_status st = MPM_OK;
  {
    const int64_t n0 = dec->n_params, n1 = c->enc ? (int64_t)c->E.n_params : c->n_snap * r;
    float* p1 = c->enc ? c->enc_p : c->latents;
    float* g1 = c->enc ? c->enc_g : c->g_lat;
    float* m1 = c->enc ? c->enc_m : c->m_lat;
    float* v1 = c->enc ? c->enc_v : c->v_lat;
    if (c->enc) MPM_CUDA_TRY(cudaMemsetAsync(c->g_lat, 0, sizeof(float) * c->n_snap * r, s));
    int ba = (int)std::max<int64_t>(1, std::min<int64_t>((n0 + n1 + 255) / 256, (int64_t)c->n_sm * 8));
    train_adam<<<ba, 256, 0, s>>>(dec->params, c->gparams, c->m_par, c->v_par, n0, p1, g1, m1, v1, n1, c->step,
                                  c->cfg.total_steps, c->cfg.lr0, c->cfg.lr1, 0.9f, 0.999f, 1e-8f, 1);
    MPM_CUDA_TRY(cudaGetLastError());
    st = decoder_refresh(dec, s);
    if (st != MPM_OK) return st;
    if (dec->n_tc > 0) {
      train_pack_transposed<<<std::max(1, dec->n_tc * 64), 256, 0, s>>>(dec->params, c->d_w_off, dec->n_tc, c->wtimg);
      MPM_CUDA_TRY(cudaGetLastError());
    }
    train_step_inc<<<1, 1, 0, s>>>(c->step);
    MPM_CUDA_TRY(cudaGetLastError());
  }
  return MPM_OK;
}

template <typename T>
mpm_status talloc(T** p, size_t count, bool zero = true) {
  cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return set_error(MPM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  if (zero) {
    e = cudaMemset(*p, 0, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return set_error(MPM_ECUDA, std::string("cudaMemset: ") + cudaGetErrorString(e));
  }
  return MPM_OK;
}

mpm_status capture(trainer_ctx* c, int update, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  MPM_CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  mpm_status st = train_launch_step(c, c->cap_stream, update);
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (st != MPM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return set_error(MPM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return set_error(MPM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return MPM_OK;
}

}  // namespace

extern "C" {

mpm_status decoder_fit_scaling(mpm_decoder* dec, const snapshot_desc* sd, void* stream) {
  MPM_CHECK_ARG(dec && sd && sd->X && sd->x && sd->inst_offsets && sd->snap_inst, "null argument");
  MPM_CHECK_ARG(sd->dim == dec->d, "snapshot dim differs from the decoder's");
  MPM_CHECK_ARG(sd->n_inst >= 1 && sd->n_snap >= 1, "empty snapshot store");
  for (const void* ptr : {(const void*)sd->X, (const void*)sd->x}) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
      cudaGetLastError();
      return set_error(MPM_EINVAL, "decoder_fit_scaling: X and x must be device pointers");
    }
    MPM_CHECK_ARG(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged,
                  "decoder_fit_scaling: X and x must be device (or managed) pointers");
  }
  int64_t nx = 0;
  for (int s = 0; s < sd->n_snap; ++s) {
    const int inst = sd->snap_inst[s];
    MPM_CHECK_ARG(inst >= 0 && inst < sd->n_inst, "snap_inst out of range");
    nx += sd->inst_offsets[inst + 1] - sd->inst_offsets[inst];
  }
  const int64_t nX = sd->inst_offsets[sd->n_inst];
  MPM_CHECK_ARG(nX >= 1 && nx >= 1, "no particles");
  const int d = dec->d;
  cudaStream_t s = (cudaStream_t)stream;
  int devn = 0, n_sm = 0;
  MPM_CUDA_TRY(cudaGetDevice(&devn));
  MPM_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, devn));
  const int blocks = std::max(1, std::min<int>(n_sm * 4, (int)((std::max(nX, nx) + kScaleThreads - 1) / kScaleThreads)));
  double* mem = nullptr;
  MPM_CUDA_TRY(cudaMallocAsync((void**)&mem, sizeof(double) * ((size_t)blocks * 3 * d + 3 * d), s));
  double* part = mem;
  double* stats = mem + (size_t)blocks * 3 * d;
  scale_partials<<<blocks, kScaleThreads, 0, s>>>(0, d, sd->X, nX, sd->x, nx, nullptr, part);
  scale_finish<<<1, 32, 0, s>>>(0, d, blocks, nx, part, stats, nullptr);
  scale_partials<<<blocks, kScaleThreads, 0, s>>>(1, d, sd->X, nX, sd->x, nx, stats, part);
  scale_finish<<<1, 32, 0, s>>>(1, d, blocks, nx, part, stats, dec->norm);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(mem, s);
  if (e != cudaSuccess) return set_error(MPM_ECUDA, std::string("decoder_fit_scaling: ") + cudaGetErrorString(e));
  return decoder_refresh(dec, s);
}

mpm_status trainer_create(mpm_decoder* dec, const train_config* cfg, const snapshot_desc* sd, const float* latents0,
                          trainer_ctx** out) {
  MPM_CHECK_ARG(dec && cfg && sd && out, "null argument");
  *out = nullptr;
  MPM_CHECK_ARG(dec->n_tc >= 1, "training needs at least two hidden layers (square tensor-core layers)");
  MPM_CHECK_ARG(sd->dim == dec->d, "snapshot dimension must match the decoder");
  MPM_CHECK_ARG(sd->n_inst >= 1 && sd->inst_offsets && sd->X, "instances");
  MPM_CHECK_ARG(sd->n_snap >= 1 && sd->snap_inst && sd->snap_next && sd->x && sd->v && sd->F, "snapshots");
  MPM_CHECK_ARG(cfg->batch >= 1 && cfg->dt_snap > 0 && cfg->lr0 > 0 && cfg->lr1 > 0, "batch, dt_snap, lr");
  MPM_CHECK_ARG(dec->r <= 32, "latent dimension <= 32");
  MPM_CHECK_ARG(cfg->shard_count >= 0 && cfg->shard_index >= 0 && cfg->shard_index < std::max(1, cfg->shard_count),
                "shard_index must be in [0, shard_count)");
  auto* c = new trainer_ctx();
  c->dec = dec;
  c->cfg = *cfg;
  c->d = dec->d;
  c->r = dec->r;
  c->R = c->d + 2;
  c->Pt = 128 / c->R;
  c->B = cfg->batch;
  c->i_offset = (int64_t)cfg->shard_index * cfg->batch;
  c->n_norm = (float)((double)cfg->batch * std::max(1, cfg->shard_count));
  c->n_tiles = (c->B + c->Pt - 1) / c->Pt;
  c->rows_total = c->n_tiles * 128;
  c->n_snap = sd->n_snap;
  int devn = 0;
  cudaGetDevice(&devn);
  cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, devn);
  const int d = c->d, r = c->r;
  mpm_status st;
  struct Owner {  // destroys the partly built context on every early return
    trainer_ctx* c;
    ~Owner() { trainer_destroy(c); }
  } owner{c};
  // snapshot bookkeeping (host)
  std::vector<int64_t> base(sd->n_snap + 1, 0);
  for (int s = 0; s < sd->n_snap; ++s) {
    const int inst = sd->snap_inst[s];
    if (inst < 0 || inst >= sd->n_inst) return set_error(MPM_EINVAL, "snap_inst out of range");
    if (sd->snap_next[s] >= sd->n_snap) return set_error(MPM_EINVAL, "snap_next out of range");
    base[s + 1] = base[s] + (sd->inst_offsets[inst + 1] - sd->inst_offsets[inst]);
  }
  const int64_t total = base[sd->n_snap];
  const int64_t Ptot = sd->inst_offsets[sd->n_inst];
  if ((st = talloc(&c->snap_base, sd->n_snap + 1)) != MPM_OK) return st;
  if ((st = talloc(&c->snap_inst, sd->n_snap)) != MPM_OK) return st;
  if ((st = talloc(&c->snap_next, sd->n_snap)) != MPM_OK) return st;
  if ((st = talloc(&c->inst_off, sd->n_inst + 1)) != MPM_OK) return st;
  if ((st = talloc(&c->X, (size_t)Ptot * d, false)) != MPM_OK) return st;
  if ((st = talloc(&c->sx, (size_t)total * d, false)) != MPM_OK) return st;
  if ((st = talloc(&c->sv, (size_t)total * d, false)) != MPM_OK) return st;
  if ((st = talloc(&c->sF, (size_t)total * d * d, false)) != MPM_OK) return st;
  MPM_CUDA_TRY(cudaMemcpy(c->snap_base, base.data(), sizeof(int64_t) * (sd->n_snap + 1), cudaMemcpyHostToDevice));
  MPM_CUDA_TRY(cudaMemcpy(c->snap_inst, sd->snap_inst, sizeof(int32_t) * sd->n_snap, cudaMemcpyDefault));
  MPM_CUDA_TRY(cudaMemcpy(c->snap_next, sd->snap_next, sizeof(int32_t) * sd->n_snap, cudaMemcpyDefault));
  MPM_CUDA_TRY(cudaMemcpy(c->inst_off, sd->inst_offsets, sizeof(int64_t) * (sd->n_inst + 1), cudaMemcpyDefault));
  MPM_CUDA_TRY(cudaMemcpy(c->X, sd->X, sizeof(float) * Ptot * d, cudaMemcpyDefault));
  MPM_CUDA_TRY(cudaMemcpy(c->sx, sd->x, sizeof(float) * total * d, cudaMemcpyDefault));
  MPM_CUDA_TRY(cudaMemcpy(c->sv, sd->v, sizeof(float) * total * d, cudaMemcpyDefault));
  MPM_CUDA_TRY(cudaMemcpy(c->sF, sd->F, sizeof(float) * total * d * d, cudaMemcpyDefault));
  // latent table + optimiser state
  const size_t nl = (size_t)sd->n_snap * r;
  if ((st = talloc(&c->latents, nl)) != MPM_OK) return st;
  if (latents0) MPM_CUDA_TRY(cudaMemcpy(c->latents, latents0, sizeof(float) * nl, cudaMemcpyDefault));
  if ((st = talloc(&c->g_lat, nl)) != MPM_OK) return st;
  if ((st = talloc(&c->m_lat, nl)) != MPM_OK) return st;
  if ((st = talloc(&c->v_lat, nl)) != MPM_OK) return st;
  if (cfg->encoder_subset > 0) {
    c->enc = true;
    if (!enc_describe(d, r, cfg->encoder_subset, 0, &c->E))
      return set_error(MPM_EINVAL, "encoder_subset: d x subset must be in [32, 8192]");
    for (int i = 0; i < sd->n_inst; ++i)
      if (sd->inst_offsets[i + 1] - sd->inst_offsets[i] < cfg->encoder_subset)
        return set_error(MPM_EINVAL, "encoder_subset larger than an instance");
    const int np = c->E.n_params;
    if ((st = talloc(&c->U, (size_t)sd->n_snap * c->E.L[0], false)) != MPM_OK) return st;
    if ((st = talloc(&c->enc_p, np)) != MPM_OK) return st;
    if ((st = talloc(&c->enc_g, np)) != MPM_OK) return st;
    if ((st = talloc(&c->enc_m, np)) != MPM_OK) return st;
    if ((st = talloc(&c->enc_v, np)) != MPM_OK) return st;
    if ((st = talloc(&c->enc_ss, 2 * d)) != MPM_OK) return st;
    if ((st = talloc(&c->enc_work, 2 * d)) != MPM_OK) return st;
    if ((st = enc_prepare(c->E)) != MPM_OK) return st;
    if ((st = enc_moments(c->E, c->sx, c->snap_base, sd->n_snap, c->enc_work, c->enc_ss, 0)) != MPM_OK) return st;
    if ((st = enc_gather(c->E, c->sx, c->snap_base, sd->n_snap, c->enc_ss, c->U, 0)) != MPM_OK) return st;
    // Xavier-uniform initial weights (fan-in / fan-out of each layer's linear map), zero biases,
    // uniform numbers from SplitMix64 seeded with the training seed
    std::vector<float> h(np, 0.f);
    uint64_t state = cfg->seed ^ 0x656e636f646572ull;
    auto uni = [&](float lim) {
      state += 0x9E3779B97F4A7C15ull;
      uint64_t z = state;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      return lim * (2.f * (float)((z >> 40) * (1.0 / 16777216.0)) - 1.f);
    };
    const float lc = std::sqrt(6.f / (kEncKernel + 1));
    for (int l = 0; l < c->E.n_conv; ++l)
      for (int k = 0; k < kEncKernel; ++k) h[7 * l + k] = uni(lc);
    const int dc = c->E.L[c->E.n_conv];
    const float l1 = std::sqrt(6.f / (dc + kEncFC)), l2 = std::sqrt(6.f / (kEncFC + r));
    for (int i = 0; i < kEncFC * dc; ++i) h[c->E.oW1 + i] = uni(l1);
    for (int i = 0; i < r * kEncFC; ++i) h[c->E.oW2 + i] = uni(l2);
    MPM_CUDA_TRY(cudaMemcpy(c->enc_p, h.data(), sizeof(float) * np, cudaMemcpyHostToDevice));
  }
  if ((st = talloc(&c->gparams, dec->n_params)) != MPM_OK) return st;
  if ((st = talloc(&c->m_par, dec->n_params)) != MPM_OK) return st;
  if ((st = talloc(&c->v_par, dec->n_params)) != MPM_OK) return st;
  // batch
  const int64_t B = c->B;
  const size_t per_pt = (size_t)(d + 2 * r + d + d + d * d + 1);
  if ((st = talloc(&c->batch_mem, per_pt * B)) != MPM_OK) return st;
  if ((st = talloc(&c->batch_idx, (size_t)3 * B)) != MPM_OK) return st;
  float* m = c->batch_mem;
  c->b.B = B;
  c->b.X = m;
  m += B * d;
  c->b.xh = m;
  m += B * r;
  c->b.u = m;
  m += B * r;
  c->b.tx = m;
  m += B * d;
  c->b.tv = m;
  m += B * d;
  c->b.tF = m;
  m += B * d * d;
  c->b.mask = m;
  c->b.snap = c->batch_idx;
  c->b.next = c->batch_idx + B;
  c->b.part = c->batch_idx + 2 * B;
  // activation stores
  const size_t rows = (size_t)c->rows_total;
  if ((st = talloc(&c->fwd, (size_t)c->R * B * d)) != MPM_OK) return st;
  if ((st = talloc(&c->dstore, (size_t)dec->n_hidden * kW * rows)) != MPM_OK) return st;
  if ((st = talloc(&c->astore, (size_t)dec->n_hidden * kW * rows)) != MPM_OK) return st;
  if ((st = talloc(&c->zbstore, (size_t)dec->n_tc * kW * rows)) != MPM_OK) return st;
  if ((st = talloc(&c->zb0, (size_t)kW * rows)) != MPM_OK) return st;
  if ((st = talloc(&c->g_lat_pt, (size_t)B * r)) != MPM_OK) return st;
  if ((st = talloc(&c->g_u_pt, (size_t)B * r)) != MPM_OK) return st;
  if ((st = talloc(&c->wtimg, (size_t)dec->n_tc * kLayerBytes)) != MPM_OK) return st;
  if ((st = talloc(&c->d_w_off, dec->w_off.size())) != MPM_OK) return st;
  MPM_CUDA_TRY(cudaMemcpy(c->d_w_off, dec->w_off.data(), sizeof(int64_t) * dec->w_off.size(), cudaMemcpyHostToDevice));
  if ((st = talloc(&c->step, 1)) != MPM_OK) return st;
  if ((st = talloc(&c->loss, 1)) != MPM_OK) return st;
  if ((st = talloc(&c->status, 1)) != MPM_OK) return st;
  c->st.d = d;
  c->st.r = r;
  c->st.n_snap = sd->n_snap;
  c->st.snap_base = c->snap_base;
  c->st.snap_inst = c->snap_inst;
  c->st.snap_next = c->snap_next;
  c->st.inst_off = c->inst_off;
  c->st.X = c->X;
  c->st.x = c->sx;
  c->st.v = c->sv;
  c->st.F = c->sF;
  c->bwd_smem = 1024 + kMaxTC * kLayerBytes + kLayerBytes + (size_t)2 * kExchRows * kChunkStride * 4 +
                2 * 64 * 128 * 2 + 128 * 3 * 4 + kW * 4 + sizeof(DecSmemTail);
  MPM_CUDA_TRY(cudaFuncSetAttribute(train_bwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->bwd_smem));
  MPM_CUDA_TRY(cudaFuncSetAttribute(train_dw0_lat<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dw0_smem_bytes()));
  MPM_CUDA_TRY(cudaFuncSetAttribute(train_dw0_lat<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dw0_smem_bytes()));
  train_pack_transposed<<<std::max(1, dec->n_tc * 64), 256>>>(dec->params, c->d_w_off, dec->n_tc, c->wtimg);
  MPM_CUDA_TRY(cudaGetLastError());
  MPM_CUDA_TRY(cudaDeviceSynchronize());
  MPM_CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  owner.c = nullptr;
  *out = c;
  return MPM_OK;
}

void trainer_destroy(trainer_ctx* c) {
  if (!c) return;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->graph_noupdate) cudaGraphExecDestroy(c->graph_noupdate);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  void* bufs[] = {c->snap_base, c->snap_inst, c->snap_next, c->inst_off, c->X, c->sx, c->sv, c->sF, c->latents,
                  c->g_lat, c->m_lat, c->v_lat, c->gparams, c->m_par, c->v_par, c->batch_mem, c->batch_idx, c->fwd,
                  c->dstore, c->astore, c->zbstore, c->zb0, c->g_lat_pt, c->g_u_pt, c->wtimg, c->d_w_off, c->step,
                  c->loss, c->status, c->U, c->enc_p, c->enc_g, c->enc_m, c->enc_v, c->enc_ss, c->enc_work};
  for (void* p : bufs) cudaFree(p);
  delete c;
}

mpm_status decoder_train(trainer_ctx* c, int n_steps, void* stream) {
  MPM_CHECK_ARG(c, "null context");
  MPM_CHECK_ARG(n_steps >= 0, "n_steps >= 0");
  if (!c->graph) {
    mpm_status st = capture(c, 1, &c->graph);
    if (st != MPM_OK) return st;
  }
  for (int i = 0; i < n_steps; ++i) MPM_CUDA_TRY(cudaGraphLaunch(c->graph, (cudaStream_t)stream));
  return MPM_OK;
}

mpm_status trainer_loss(trainer_ctx* c, double* loss, int64_t* step, void* stream) {
  MPM_CHECK_ARG(c, "null context");
  cudaStream_t s = (cudaStream_t)stream;
  double h = 0.0;
  MPM_CUDA_TRY(cudaMemcpyAsync(&h, c->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (step) MPM_CUDA_TRY(cudaMemcpyAsync(step, c->step, sizeof(int64_t), cudaMemcpyDefault, s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  if (loss) *loss = h / (double)c->n_norm;
  return MPM_OK;
}

mpm_status trainer_gradient_sizes(const trainer_ctx* c, int64_t* n_params, int64_t* n_second) {
  MPM_CHECK_ARG(c, "null context");
  if (n_params) *n_params = c->dec->n_params;
  if (n_second) *n_second = c->enc ? (int64_t)c->E.n_params : c->n_snap * c->r;
  return MPM_OK;
}

mpm_status trainer_compute_gradients(trainer_ctx* c, float* g_params, float* g_second, void* stream) {
  MPM_CHECK_ARG(c && g_params && g_second, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  mpm_status st = train_launch_step(c, s, 0);
  if (st != MPM_OK) return st;
  const size_t n1 = c->enc ? (size_t)c->E.n_params : (size_t)c->n_snap * c->r;
  float* g1 = c->enc ? c->enc_g : c->g_lat;
  MPM_CUDA_TRY(cudaMemcpyAsync(g_params, c->gparams, sizeof(float) * c->dec->n_params, cudaMemcpyDeviceToDevice, s));
  MPM_CUDA_TRY(cudaMemcpyAsync(g_second, g1, sizeof(float) * n1, cudaMemcpyDeviceToDevice, s));
  MPM_CUDA_TRY(cudaMemsetAsync(c->gparams, 0, sizeof(float) * c->dec->n_params, s));
  MPM_CUDA_TRY(cudaMemsetAsync(c->g_lat, 0, sizeof(float) * c->n_snap * c->r, s));
  if (c->enc) MPM_CUDA_TRY(cudaMemsetAsync(c->enc_g, 0, sizeof(float) * c->E.n_params, s));
  return MPM_OK;
}

mpm_status trainer_apply_gradients(trainer_ctx* c, const float* g_params, const float* g_second, void* stream) {
  MPM_CHECK_ARG(c && g_params && g_second, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n1 = c->enc ? (size_t)c->E.n_params : (size_t)c->n_snap * c->r;
  float* g1 = c->enc ? c->enc_g : c->g_lat;
  MPM_CUDA_TRY(cudaMemcpyAsync(c->gparams, g_params, sizeof(float) * c->dec->n_params, cudaMemcpyDeviceToDevice, s));
  MPM_CUDA_TRY(cudaMemcpyAsync(g1, g_second, sizeof(float) * n1, cudaMemcpyDeviceToDevice, s));
  return train_launch_update(c, s);
}

mpm_status trainer_get_latents(trainer_ctx* c, float* latents, void* stream) {
  MPM_CHECK_ARG(c && latents, "null argument");
  MPM_CUDA_TRY(cudaMemcpyAsync(latents, c->latents, sizeof(float) * c->n_snap * c->r, cudaMemcpyDefault,
                               (cudaStream_t)stream));
  return MPM_OK;
}

mpm_status trainer_status_word(trainer_ctx* c, uint32_t* out, int clear, void* stream) {
  MPM_CHECK_ARG(c && out, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t h = 0;
  MPM_CUDA_TRY(cudaMemcpyAsync(&h, c->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  if (clear) MPM_CUDA_TRY(cudaMemsetAsync(c->status, 0, sizeof(uint32_t), s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  *out = h;
  return MPM_OK;
}

mpm_status trainer_gradients(trainer_ctx* c, float* g_params, float* g_latents, float* g_encoder, int32_t* batch_snap,
                             int32_t* batch_part, double* loss, void* stream) {
  MPM_CHECK_ARG(c, "null context");
  cudaStream_t s = (cudaStream_t)stream;
  // one forward + backward on the batch of the current step, no update
  mpm_status st = train_launch_step(c, s, 0);
  if (st != MPM_OK) return st;
  if (g_params) MPM_CUDA_TRY(cudaMemcpyAsync(g_params, c->gparams, sizeof(float) * c->dec->n_params, cudaMemcpyDefault, s));
  if (g_latents) MPM_CUDA_TRY(cudaMemcpyAsync(g_latents, c->g_lat, sizeof(float) * c->n_snap * c->r, cudaMemcpyDefault, s));
  if (g_encoder && c->enc)
    MPM_CUDA_TRY(cudaMemcpyAsync(g_encoder, c->enc_g, sizeof(float) * c->E.n_params, cudaMemcpyDefault, s));
  if (batch_snap) MPM_CUDA_TRY(cudaMemcpyAsync(batch_snap, c->b.snap, sizeof(int32_t) * c->B, cudaMemcpyDefault, s));
  if (batch_part) MPM_CUDA_TRY(cudaMemcpyAsync(batch_part, c->b.part, sizeof(int32_t) * c->B, cudaMemcpyDefault, s));
  double h = 0.0;
  MPM_CUDA_TRY(cudaMemcpyAsync(&h, c->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  MPM_CUDA_TRY(cudaMemsetAsync(c->gparams, 0, sizeof(float) * c->dec->n_params, s));
  MPM_CUDA_TRY(cudaMemsetAsync(c->g_lat, 0, sizeof(float) * c->n_snap * c->r, s));
  if (c->enc) MPM_CUDA_TRY(cudaMemsetAsync(c->enc_g, 0, sizeof(float) * c->E.n_params, s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  if (loss) *loss = h / (double)c->n_norm;
  return MPM_OK;
}

mpm_status trainer_encoder_params(trainer_ctx* c, float* params, float* shift_scale, int64_t* n_params, void* stream) {
  MPM_CHECK_ARG(c, "null context");
  MPM_CHECK_ARG(c->enc, "the trainer has no encoder (train_config.encoder_subset = 0)");
  cudaStream_t s = (cudaStream_t)stream;
  if (n_params) *n_params = c->E.n_params;
  if (params) MPM_CUDA_TRY(cudaMemcpyAsync(params, c->enc_p, sizeof(float) * c->E.n_params, cudaMemcpyDefault, s));
  if (shift_scale) MPM_CUDA_TRY(cudaMemcpyAsync(shift_scale, c->enc_ss, sizeof(float) * 2 * c->d, cudaMemcpyDefault, s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  return MPM_OK;
}

mpm_status trainer_set_encoder_params(trainer_ctx* c, const float* params, const float* shift_scale, void* stream) {
  MPM_CHECK_ARG(c, "null context");
  MPM_CHECK_ARG(c->enc, "the trainer has no encoder (train_config.encoder_subset = 0)");
  cudaStream_t s = (cudaStream_t)stream;
  if (params) MPM_CUDA_TRY(cudaMemcpyAsync(c->enc_p, params, sizeof(float) * c->E.n_params, cudaMemcpyDefault, s));
  if (shift_scale) {
    MPM_CUDA_TRY(cudaMemcpyAsync(c->enc_ss, shift_scale, sizeof(float) * 2 * c->d, cudaMemcpyDefault, s));
    mpm_status st = enc_gather(c->E, c->sx, c->snap_base, c->n_snap, c->enc_ss, c->U, s);
    if (st != MPM_OK) return st;
  }
  MPM_CUDA_TRY(cudaMemsetAsync(c->enc_m, 0, sizeof(float) * c->E.n_params, s));
  MPM_CUDA_TRY(cudaMemsetAsync(c->enc_v, 0, sizeof(float) * c->E.n_params, s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  return MPM_OK;
}

mpm_status trainer_encode(trainer_ctx* c, const float* x, int64_t n, int64_t n_particles, float* latents,
                          void* stream) {
  MPM_CHECK_ARG(c, "null context");
  MPM_CHECK_ARG(c->enc, "the trainer has no encoder (train_config.encoder_subset = 0)");
  MPM_CHECK_ARG(n >= 0 && n_particles >= c->E.n_sub, "n >= 0 and n_particles >= the encoder subset");
  if (n == 0) return MPM_OK;
  MPM_CHECK_ARG(x && latents, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int d = c->d;
  float *xd = nullptr, *Ud = nullptr, *ld = nullptr;
  int64_t* base = nullptr;
  std::vector<int64_t> hb(n + 1);
  for (int64_t i = 0; i <= n; ++i) hb[i] = i * n_particles;
  mpm_status st = MPM_OK;
  cudaError_t e = cudaMalloc((void**)&xd, sizeof(float) * n * n_particles * d);
  if (e == cudaSuccess) e = cudaMalloc((void**)&Ud, sizeof(float) * n * c->E.L[0]);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ld, sizeof(float) * n * c->r);
  if (e == cudaSuccess) e = cudaMalloc((void**)&base, sizeof(int64_t) * (n + 1));
  if (e == cudaSuccess) e = cudaMemcpyAsync(xd, x, sizeof(float) * n * n_particles * d, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base, hb.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    st = enc_gather(c->E, xd, base, n, c->enc_ss, Ud, s);
    if (st == MPM_OK) st = enc_forward(c->E, c->enc_p, Ud, n, ld, c->n_sm, s);
    if (st == MPM_OK) e = cudaMemcpyAsync(latents, ld, sizeof(float) * n * c->r, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  cudaFree(xd);
  cudaFree(Ud);
  cudaFree(ld);
  cudaFree(base);
  if (e != cudaSuccess) return set_error(MPM_ECUDA, std::string("trainer_encode: ") + cudaGetErrorString(e));
  return st;
}

}  // extern "C"

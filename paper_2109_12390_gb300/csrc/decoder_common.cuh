// Device pieces shared by the decoder evaluation kernels (decoder.cu) and the
// decoder training kernels (train.cu): argument block, activation functions,
// row bookkeeping of the 128-row tiles, BF16 tile stores.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "tc.cuh"

namespace mpmrom {

constexpr int kW = 128;          // hidden width of the tensor-core layers
constexpr int kMaxTC = 4;        // square layers resident in shared memory
constexpr int kMaxR = 64;        // row kinds per point
constexpr int kLayerBytes = kW * kW * 2;

struct DecArgs {
  int d, r, n_tc, act;
  const float* W0;    // (W, d + r)
  const float* b0;    // (W)
  const float* bh;    // (n_tc, W)
  const float* Wout;  // (d, W)
  const float* bout;  // (d)
  const float* norm;  // X_min[d], X_range[d], out_shift[d], out_scale[d]
  const uint8_t* wimg;
  const uint8_t* wimg_lo;   // bf16(w - bf16(w)) images (split operands)
  // first layer as split BF16 pairs for the tensor cores (inputs of at most 32 entries in the
  // padded layout): rows = output features, hi at K 0 .. 31 and lo at K 32 .. 63 of one
  // 128-byte swizzled row; null when the first layer runs on the CUDA cores
  const uint8_t* w0img;
  const float* wsq;   // (n_tc, W, W) FP32 square-layer weights, (out, in) row-major
  const float* wsqT;  // (n_tc, W, W) the same transposed, (in, out) row-major
  const float* X;
  const int32_t* lat;
  const float* latents;
  const float* dirs;
  int64_t n;          // points (upper bound when n_dev is set)
  int R, Pt;
  int kinds[kMaxR];
  // mixed rows: kind indices of the JVP row and of the tangent row they pair
  int8_t mix_jvp[kMaxR];
  int8_t mix_tan[kMaxR];
  float* out;         // (R, n, d)
  // on-device point sets (reduced-order step): when n_dev is set, the point
  // count is (*n_dev) * n_rep, point p reads X row idx[p % *n_dev] (or
  // p % *n_dev when idx is null) and latent row p / *n_dev.
  const int32_t* idx;
  const int32_t* n_dev;
  int n_rep;
  uint32_t* status;
  // linear decoder (no hidden layer): y = W0 [Xn, xhat] + b0 with W0 (d, d + r)
  int linear;
  // latent row = point index (training batches carry one latent per point)
  int lat_per_point;
  // FP32 path: useful rows per packed tile (0: point-aligned tiles of Pt points)
  int f32_U;
  // direction blocks per latent row in `dirs` (KIND_SECANT_DIR rows; 1 otherwise)
  int n_dirs;
  // training: per hidden layer l, stored feature-major [l][feature][row] (row =
  // tile * 128 + t, rows_total = n_tiles * 128), BF16: dstore the primal rows'
  // activation slope act'(z), or -1 where z >= 0 (slope 1, no curvature term;
  // other rows not written), astore every row's activation a
  __nv_bfloat16* dstore;
  __nv_bfloat16* astore;
  int64_t rows_total;
};

__device__ __forceinline__ float elu(float z) { return z > 0.f ? z : expm1f(z); }
__device__ __forceinline__ float elu_d1(float z) { return z > 0.f ? 1.f : __expf(z); }
__device__ __forceinline__ float elu_d2(float z) { return z > 0.f ? 0.f : __expf(z); }
// exp(x) - 1 for the small increments of secant rows: below |x| = 1/32 the Taylor polynomial
// x + x^2/2 + ... + x^6/720 in Horner form (truncation below 1e-12 relative there), else expm1f
__device__ __forceinline__ float expm1_small(float x) {
  if (fabsf(x) < 0.03125f)
    return x * fmaf(0.5f * x,
                    fmaf(x * (1.f / 3.f), fmaf(0.25f * x, fmaf(0.2f * x, fmaf(x, 1.f / 6.f, 1.f), 1.f), 1.f), 1.f),
                    1.f);
  return expm1f(x);
}

// act(z + dz) - act(z) without cancellation on the negative branch.  The common cases (both ends
// positive: dz; both negative with a small increment: e^z times the Taylor polynomial of
// expm1(dz)) are evaluated without branches, so that the lanes of a warp, whose features take
// different cases, do not run them one after another; the rest (ends of opposite sign, or an
// increment of 1/32 or more) takes the branch, with the same arithmetic as the case split.
__device__ __forceinline__ float elu_secant(float z, float dz) {
  const float z1 = z + dz;
  const bool pos = (z > 0.f) & (z1 > 0.f);
  const bool neg = (z <= 0.f) & (z1 <= 0.f);
  const bool small = fabsf(dz) < 0.03125f;
  const float poly =
      dz * fmaf(0.5f * dz, fmaf(dz * (1.f / 3.f), fmaf(0.25f * dz, fmaf(0.2f * dz, fmaf(dz, 1.f / 6.f, 1.f), 1.f), 1.f), 1.f),
                1.f);
  float res = pos ? dz : __expf(fminf(z, 0.f)) * poly;
  if (!pos && !(neg && small)) res = neg ? __expf(z) * expm1f(dz) : elu(z1) - elu(z);
  return res;
}

__device__ __forceinline__ float act_f(int act, float z) { return act == 0 ? elu(z) : z; }
// The training record of a primal pre-activation: ELU's slope exp(z) where z < 0 (the
// curvature there equals it), -1 elsewhere (slope 1, no curvature)
__device__ __forceinline__ float act_slope_record(int act, float z) { return (act == 0 && z < 0.f) ? __expf(z) : -1.f; }
__device__ __forceinline__ float act_d1(int act, float z) { return act == 0 ? elu_d1(z) : 1.f; }
__device__ __forceinline__ float act_d2(int act, float z) { return act == 0 ? elu_d2(z) : 0.f; }
__device__ __forceinline__ float act_sec(int act, float z, float dz) { return act == 0 ? elu_secant(z, dz) : dz; }

// row-kind codes (see decoder_eval in include/mpmrom.h)
constexpr int KIND_PRIMAL = 0;
constexpr int KIND_JVP = 1000;
constexpr int KIND_SECANT = 1001;
// KIND_MIXED + b (b = 1 .. d + r): derivative along input b of the JVP row
constexpr int KIND_MIXED = 2000;
// KIND_SECANT_DIR + m (m < 64): secant along the m-th direction block of the point's latent row
constexpr int KIND_SECANT_DIR = 3000;

struct RowInfo {
  int kind;      // code
  int cls;       // 0 primal, 1 tangent, 2 secant, 3 mixed, -1 padding
  int q;         // point within tile
  int64_t p;     // global point index
  int ja, jb;    // mixed rows: kind indices of the paired JVP and tangent rows
};

__device__ __forceinline__ int kind_class(int kind) {
  if (kind == KIND_PRIMAL) return 0;
  if (kind == KIND_SECANT || kind >= KIND_SECANT_DIR) return 2;
  return kind > KIND_MIXED ? 3 : 1;
}

// Offset of the direction of a row (JVP, secant, mixed: block 0; KIND_SECANT_DIR + m: block m) of
// latent row li in `dirs`, laid out (n_lat, n_dirs, r).
__device__ __forceinline__ int64_t dir_offset(const DecArgs& a, int kind, int li) {
  const int m = kind >= KIND_SECANT_DIR ? kind - KIND_SECANT_DIR : 0;
  return ((int64_t)li * a.n_dirs + m) * a.r;
}

__device__ __forceinline__ int64_t dec_count(const DecArgs& a) {
  return a.n_dev ? (int64_t)(*a.n_dev) * a.n_rep : a.n;
}

__device__ __forceinline__ RowInfo row_info(const DecArgs& a, int t, int64_t tile_first, int64_t n) {
  RowInfo ri;
  ri.q = t % a.Pt;
  int k = t / a.Pt;
  ri.p = tile_first + ri.q;
  if (k >= a.R || ri.p >= n) {
    ri.cls = -1;
    ri.kind = -1;
    return ri;
  }
  ri.kind = a.kinds[k];
  ri.cls = kind_class(ri.kind);
  ri.ja = a.mix_jvp[k];
  ri.jb = a.mix_tan[k];
  return ri;
}

// Input vector (normalised) and direction of one row.
__device__ __forceinline__ void row_inputs(const DecArgs& a, const RowInfo& ri, float* in, float* dir) {
  const int d = a.d, r = a.r;
  int64_t xrow = ri.p;
  int li = a.lat ? a.lat[ri.p] : (a.lat_per_point ? (int)ri.p : 0);
  if (a.n_dev) {
    const int cnt = max(*a.n_dev, 1);
    xrow = ri.p % cnt;
    li = (int)(ri.p / cnt);
    if (a.idx) xrow = a.idx[xrow];
  }
  // unrolled to the 40-entry bound so that in[] and dir[] stay in registers
#pragma unroll
  for (int i = 0; i < 40; ++i) {
    const int K = d + r;
    float vin = 0.f, vdir = 0.f;
    if (i < K) {
      if (i < d) {
        vin = (a.X[xrow * d + i] - a.norm[i]) / a.norm[d + i];
      } else {
        vin = a.latents[(int64_t)li * r + (i - d)];
      }
      if (ri.cls == 1) {
        if (ri.kind >= 1 && ri.kind <= d + r) vdir = (i == ri.kind - 1) ? (i < d ? 1.f / a.norm[d + i] : 1.f) : 0.f;
        else if (ri.kind == KIND_JVP && i >= d) vdir = a.dirs[dir_offset(a, ri.kind, li) + (i - d)];
      } else if ((ri.cls == 2 || ri.cls == 3) && i >= d) {
        // secant increment, or the JVP direction that a mixed row differentiates
        vdir = a.dirs[dir_offset(a, ri.kind, li) + (i - d)];
      }
    }
    in[i] = vin;
    dir[i] = vdir;
  }
}

// Row of X and latent row of the point of `ri`.
__device__ __forceinline__ void row_source(const DecArgs& a, const RowInfo& ri, int64_t& xrow, int& li);

// Input vector and direction of one row in the tensor-core kernel's layout: the d normalised
// coordinates at entries 0 .. 3 (zero-padded), the r <= 36 latents from entry 4, so that the
// latent part sits at a fixed offset and is loaded as float4 when r is a multiple of 4.
constexpr int kTcLat = 4;   // offset of the latent part
__device__ __forceinline__ void row_inputs_tc(const DecArgs& a, const RowInfo& ri, float* in, float* dir) {
  const int d = a.d, r = a.r;
  int64_t xrow;
  int li;
  row_source(a, ri, xrow, li);
#pragma unroll
  for (int i = 0; i < kTcLat; ++i) {
    in[i] = i < d ? (a.X[xrow * d + i] - a.norm[i]) / a.norm[d + i] : 0.f;
    dir[i] = (i < d && ri.cls == 1 && ri.kind == i + 1) ? 1.f / a.norm[d + i] : 0.f;
  }
  const float* lat = a.latents + (int64_t)li * r;
  const bool has_dir = (ri.cls == 1 && ri.kind == KIND_JVP) || ri.cls == 2 || ri.cls == 3;
  const float* dv = has_dir ? a.dirs + dir_offset(a, ri.kind, li) : lat;
  const bool vec = (r & 3) == 0 && (((uintptr_t)lat | (uintptr_t)dv) & 15u) == 0;
  const int lat_tangent = (ri.cls == 1 && ri.kind > d && ri.kind <= d + r) ? ri.kind - 1 - d : -1;
#pragma unroll
  for (int q = 0; q < (40 - kTcLat) / 4; ++q) {
    float lv[4] = {0.f, 0.f, 0.f, 0.f}, dvv[4] = {0.f, 0.f, 0.f, 0.f};
    if (4 * q < r) {
      if (vec) {
        const float4 l4 = *reinterpret_cast<const float4*>(lat + 4 * q);
        lv[0] = l4.x; lv[1] = l4.y; lv[2] = l4.z; lv[3] = l4.w;
        if (has_dir) {
          const float4 d4 = *reinterpret_cast<const float4*>(dv + 4 * q);
          dvv[0] = d4.x; dvv[1] = d4.y; dvv[2] = d4.z; dvv[3] = d4.w;
        }
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (4 * q + c < r) {
            lv[c] = lat[4 * q + c];
            if (has_dir) dvv[c] = dv[4 * q + c];
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      in[kTcLat + 4 * q + c] = lv[c];
      dir[kTcLat + 4 * q + c] = (4 * q + c == lat_tangent) ? 1.f : dvv[c];
    }
  }
}
__device__ __forceinline__ void row_source(const DecArgs& a, const RowInfo& ri, int64_t& xrow, int& li) {
  xrow = ri.p;
  li = a.lat ? a.lat[ri.p] : (a.lat_per_point ? (int)ri.p : 0);
  if (a.n_dev) {
    const int cnt = max(*a.n_dev, 1);
    xrow = ri.p % cnt;
    li = (int)(ri.p / cnt);
    if (a.idx) xrow = a.idx[xrow];
  }
}

// Input i of the row's layer-0 input and direction, from its point's sources (row_source).
__device__ __forceinline__ void row_input_from(const DecArgs& a, const RowInfo& ri, int64_t xrow, int li, int i,
                                               float& vin, float& vdir) {
  const int d = a.d, r = a.r;
  vin = i < d ? (a.X[xrow * d + i] - a.norm[i]) / a.norm[d + i] : a.latents[(int64_t)li * r + (i - d)];
  vdir = 0.f;
  if (ri.cls == 1) {
    if (ri.kind >= 1 && ri.kind <= d + r) vdir = (i == ri.kind - 1) ? (i < d ? 1.f / a.norm[d + i] : 1.f) : 0.f;
    else if (ri.kind == KIND_JVP && i >= d) vdir = a.dirs[dir_offset(a, ri.kind, li) + (i - d)];
  } else if ((ri.cls == 2 || ri.cls == 3) && i >= d) {
    vdir = a.dirs[dir_offset(a, ri.kind, li) + (i - d)];
  }
}

// Entry i (< d + r) of row_inputs: normalised input and direction of one row.
__device__ __forceinline__ void row_input_elem(const DecArgs& a, const RowInfo& ri, int i, float& vin, float& vdir) {
  int64_t xrow;
  int li;
  row_source(a, ri, xrow, li);
  row_input_from(a, ri, xrow, li, i, vin, vdir);
}

// Layer-0 tangent of a mixed row along input b (the normalised X axes scale by
// 1 / X_range): the weight column itself.
__device__ __forceinline__ float mixed_t0(const DecArgs& a, const float* W0row, int kind) {
  const int b = kind - KIND_MIXED - 1;
  return b < a.d ? W0row[b] / a.norm[a.d + b] : W0row[b];
}

struct __align__(8) DecSmemTail {
  uint64_t bar_w;
  uint64_t bar_mma;
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ void store_bf16x8(uint8_t* tile, int row, int col, const float* v) {
  __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]);
  __nv_bfloat162 p1 = __floats2bfloat162_rn(v[2], v[3]);
  __nv_bfloat162 p2 = __floats2bfloat162_rn(v[4], v[5]);
  __nv_bfloat162 p3 = __floats2bfloat162_rn(v[6], v[7]);
  uint4 u;
  u.x = *reinterpret_cast<uint32_t*>(&p0);
  u.y = *reinterpret_cast<uint32_t*>(&p1);
  u.z = *reinterpret_cast<uint32_t*>(&p2);
  u.w = *reinterpret_cast<uint32_t*>(&p3);
  *reinterpret_cast<uint4*>(tile + tc::sw128_offset(row, col, kW)) = u;
}


__device__ __forceinline__ uint32_t u4_word(const uint4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// Copies a 128 x 128 BF16 operand tile (row-major, 128-byte swizzled, as the MMA reads it) to a
// feature-major store, dst[feature * rows_total + tile * 128 + row], with the CTA's 256 threads:
// each moves an 8 x 8 block (8 rows x 8 features) by eight 16-byte shared loads (the 8 threads
// of a quarter warp read 8 different 16-byte columns: no bank conflict), a register transpose
// and eight 16-byte stores of 8 rows of one feature.
__device__ __forceinline__ void copy_out_tile(__nv_bfloat16* dst, int64_t rows_total, const uint8_t* tile_smem,
                                              int64_t tile, int t) {
  const int fg = (t & 7) + 8 * (t >> 7), rg = (t >> 3) & 15;   // feature group 0 .. 15, row group 0 .. 15
  uint4 u[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) u[j] = *reinterpret_cast<const uint4*>(tile_smem + tc::sw128_offset(8 * rg + j, 8 * fg, kW));
  __nv_bfloat16* base = dst + (int64_t)(8 * fg) * rows_total + tile * 128 + 8 * rg;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    // feature e of the group sits in word e / 2 of each row's 16 bytes, low half for even e
    const uint32_t sel = (e & 1) ? 0x7632u : 0x5410u;
    uint4 o;
    o.x = __byte_perm(u4_word(u[0], e >> 1), u4_word(u[1], e >> 1), sel);
    o.y = __byte_perm(u4_word(u[2], e >> 1), u4_word(u[3], e >> 1), sel);
    o.z = __byte_perm(u4_word(u[4], e >> 1), u4_word(u[5], e >> 1), sel);
    o.w = __byte_perm(u4_word(u[6], e >> 1), u4_word(u[7], e >> 1), sel);
    *reinterpret_cast<uint4*>(base + (int64_t)e * rows_total) = o;
  }
}

}  // namespace mpmrom

#include <vector>

// Host-side decoder object (shared by decoder.cu and train.cu).
struct mpm_decoder {
  int d = 0, r = 0, width = 0, n_hidden = 0, act = 0;
  int n_tc = 0;
  int64_t n_params = 0;
  std::vector<int64_t> w_off, b_off;  // per linear layer offsets into params
  float* params = nullptr;            // FP32 master copy
  float* norm = nullptr;
  float* wsq = nullptr;               // square-layer weights gathered contiguously (n_tc, W, W)
  float* bsq = nullptr;               // their biases (n_tc, W)
  float* wsqT = nullptr;              // transposed FP32 copies (n_tc, W, W) for the CUDA-core path
  uint8_t* wimg = nullptr;            // BF16 swizzled images
  uint8_t* wimg_lo = nullptr;         // residual images bf16(w - bf16(w)) for the split-BF16 path
  uint8_t* w0img = nullptr;           // first-layer split image (16 KB) when kTcLat + r <= 32
  uint32_t* status = nullptr;
  int n_sm = 0;
  size_t smem = 0;
  size_t smem_split = 0;
  int fp32 = 0;                       // square layers: 0 BF16 tensor cores, 1 FP32 CUDA cores, 2 split BF16 tensor cores
  int concurrency = 1;                // expected concurrent calls (FP32 tiling)
};

namespace mpmrom {
// Re-packs the BF16 shared-memory images of the square layers from the FP32 master copy.
mpm_status decoder_refresh(mpm_decoder* dec, cudaStream_t s);
}  // namespace mpmrom

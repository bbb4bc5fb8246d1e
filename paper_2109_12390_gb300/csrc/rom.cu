// Reduced-order step (Algorithm 2) on sm_103a.
//
// One step, all on the device (no host round trip; replayable as a graph), with the Lagrangian
// quadrature of Algorithm 3 (default):
//   decoder        x_n^p = g(X^p; xhat_n) for all particles (Alg. 3, tracking); when the
//                  neighbourhood covers most of the body this one decode also produces the
//                  quadrature rows below for every particle
//   rom_select     one CTA: clears the previous basis set on the grid, draws the
//                  sample set P as the bottom-k of a SplitMix64 hash per
//                  particle (8-pass radix select over the 64-bit hashes, ties
//                  by particle id) plus, with kinematic boundaries, each
//                  group's smallest-hash particles, marks the basis set I
//                  (stencil nodes of the samples) with a per-step stamp, finds
//                  the neighbour set N (particles outside P with a stencil
//                  node in I) and writes the quadrature list Q = [P, N] (Alg. 3)
//   decoder        dg/dX (deformation gradient, Eq. defGrad) and the JVP along
//                  vhat_n (velocity, Eq. timederOne) at Q
//   rom_p2g        particle-to-grid from Q onto the nodes of I only (Alg. 5,
//                  no affine term unless asked), stress from the same device
//                  functions as the full-order step
//   rom_g2p        grid update + grid-to-particle to the samples: v_trial (the
//                  prescribed velocity for kinematic samples), x_trial = x_n +
//                  dt v_trial (Alg. 5)
//   decoder        dg/dxhat at (X^P, xhat_n)
//   rom_normal     normal equations J^T J, J^T b (multi-CTA, compensated FP32
//                  sums added in FP64); the last CTA to finish solves them (FP32
//                  Cholesky with FP64 refinement, FP64 Cholesky fallback):
//                  vhat_{n+1} (Eq. nonlinear_projection:vel), or a Gauss-Newton
//                  step delta for xhat (Eq. ...:pos)
//   per Gauss-Newton iteration (initial guess 2 xhat_n - xhat_{n-1}):
//     decoder      dg/dxhat and the secant g(xhat_n) - g(xhat_k) at the samples
//     rom_normal   residual r = g(xhat_k) - x_trial = -(secant) - dt v_trial;
//                  solve J^T J delta = -J^T r; prepare 11 trial steps 2^-m delta
//     decoder      secants g(xhat_k + 2^-m delta) - g(xhat_n), m = 0..10, in one launch
//                  (one primal row and 11 secant rows along direction blocks per sample)
//     rom_linesearch  objective of every trial (FP64); the last CTA takes the
//                  first trial that meets the Armijo condition (the same
//                  choice as sequential backtracking) and updates xhat.
// With the Eulerian quadrature of Algorithm 4 the samples are decoded alone and
// the quadrature points are cell points whose reference positions come from a
// Newton inversion of the decoder (rom_eul_* kernels).
// The Gauss-Newton residual is formed from secant rows (exact differences of
// decoder outputs) so that BF16 GEMMs resolve latent increments of ~1e-5.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "mpm_math.cuh"

struct mpm_decoder;
namespace mpmrom {
mpm_status decoder_launch_dev(const mpm_decoder* dec, const float* X, const int32_t* idx, const int32_t* n_dev,
                              int n_rep, int64_t capacity, const float* latents, const float* dirs,
                              const int* kinds, int R, float* out, cudaStream_t s);
void decoder_shape(const mpm_decoder* dec, int* d, int* r);
}

namespace mpmrom {

constexpr int kLS = 11;          // line-search trials 2^0 .. 2^-10
constexpr int kMaxGnIters = 16;   // cfg.gn_iters <= 16
constexpr int kMaxRl = 32;       // latent dimension bound of the solver
constexpr int kNormBlock = 256;

// ----------------------------------------------------------------- hashing
__device__ __forceinline__ uint64_t splitmix_out(uint64_t state, uint64_t k) {
  uint64_t z = state + 0x9E3779B97F4A7C15ull * (k + 1ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct RomDev {
  int d, r, P, n, k;         // dims, particles, grid nodes per axis, samples
  float dx, inv_dx, dt;
  float g[3];
  int bc, bc_width;
  float mass, vol, mu, lam;
  uint64_t seed;
  int inst;
  // buffers
  const float* X;
  float* x_all;              // (P, d)
  int32_t* qlist;            // (P) samples then neighbours
  int32_t* counts;           // [0] nP, [1] nQ, [2] nI (basis-node list length)
  int32_t* nodes;            // (k * 3^d) basis nodes of the last step (for clearing)
  uint32_t* stamp;           // (n^d) node stamps
  float4* grid;              // (n^d)
  float* v_trial;            // (k, d)
  float* x_trial;            // (k, d)
  int64_t* step;             // device step counter
  uint32_t* status;
  const float* Fref_inv;     // (P, d, d) inverse reference gradients, or null (f_reference = 0)
  int q_by_pid;              // quadrature decoder rows indexed by particle id (one decode of all particles)
  // Eulerian quadrature (Algorithm 4)
  int eulerian;              // 1: samples only in rom_select; quadrature points on cells
  int ell;                   // points per cell per dimension
  const float* x_samp;       // (k, d) decoded sample positions (Eulerian mode), or null
  uint32_t* cstamp;          // (n^d) cell stamps
  int32_t* clist;            // (cap_cells) cells of the quadrature set
  int cap_cells;
  float* qX;                 // (cap_cells ell^d, d) reference positions of the quadrature points
  float* qm;                 // (cap_cells ell^d) mass (0 outside the body)
  float* qV0;                // (cap_cells ell^d) reference volume V_q / J
  const uint8_t* occ;        // reference-domain occupancy of boxes of side occ_h
  float occ_origin[3];
  float occ_h;
  int occ_shape[3];
  // kinematic (Dirichlet) boundaries
  const int32_t* kin_group;  // group per particle (-1 free), or null
  const float* kin_vel;      // prescribed velocity per group (3 floats each)
  const int32_t* kg_off;     // (n_groups + 1) offsets into kg_ids
  const int32_t* kg_ids;     // particles of each group, ascending
  int n_groups, m_kin;
  uint32_t* sel_bits;        // ((P + 31) / 32) sample membership of the current step
  // neighbour test on every SM for P > kSelMaxBits (rom_nb_flags, rom_nb_list)
  int nb_multi;
  uint32_t* smp_bits;        // ((P + 31) / 32) samples of the step
  uint32_t* nb_bits;         // ((P + 31) / 32) neighbours of the step
  int32_t* nb_cnt;           // (grid of rom_nb_flags) neighbours per CTA
};

// Inverse of a small matrix by its adjugate (F of a quadrature point, det F > 0).
template <int D>
__device__ __forceinline__ void inverse(const float* F, float* Fi);
template <>
__device__ __forceinline__ void inverse<2>(const float* F, float* Fi) {
  const float id = 1.0f / (F[0] * F[3] - F[1] * F[2]);
  Fi[0] = F[3] * id;
  Fi[1] = -F[1] * id;
  Fi[2] = -F[2] * id;
  Fi[3] = F[0] * id;
}
template <>
__device__ __forceinline__ void inverse<3>(const float* F, float* Fi) {
  const float c00 = F[4] * F[8] - F[5] * F[7], c01 = F[5] * F[6] - F[3] * F[8], c02 = F[3] * F[7] - F[4] * F[6];
  const float id = 1.0f / (F[0] * c00 + F[1] * c01 + F[2] * c02);
  Fi[0] = c00 * id;
  Fi[3] = c01 * id;
  Fi[6] = c02 * id;
  Fi[1] = (F[2] * F[7] - F[1] * F[8]) * id;
  Fi[4] = (F[0] * F[8] - F[2] * F[6]) * id;
  Fi[7] = (F[1] * F[6] - F[0] * F[7]) * id;
  Fi[2] = (F[1] * F[5] - F[2] * F[4]) * id;
  Fi[5] = (F[2] * F[3] - F[0] * F[5]) * id;
  Fi[8] = (F[0] * F[4] - F[1] * F[3]) * id;
}

// Block-wide exclusive scan of one int per thread (blockDim.x <= 1024).
__device__ __forceinline__ int block_exclusive_scan(int v, int* total, int* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < nwarps ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  int excl = x - v + (warp > 0 ? s_warp[warp - 1] : 0);
  *total = s_warp[nwarps - 1];
  __syncthreads();
  return excl;
}

template <int D>
__device__ __forceinline__ int node_linear(const int node[D], int n) {
  int l = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) l = l * n + node[a];
  return l;
}

// ------------------------------------------------------------ rom_select
constexpr int kMaxKin = 32;          // samples forced from one kinematic group, at most
constexpr int kSelMaxBits = 65536;   // particles whose neighbour decisions rom_select keeps in shared memory

// Algorithm 3's neighbour test of particle p: a node of its stencil carries the step's stamp (is
// in the basis set I).  The stencil's stamps are loaded together (independent loads).
template <int D>
__device__ __forceinline__ bool nb_hit(const RomDev& R, int p, uint32_t stamp, bool flag_out_of_grid) {
  constexpr int NS = (D == 2) ? 9 : 27;
  int base[D];
  bool ok = true;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int b = stencil_base(R.x_all[(size_t)p * D + a], R.inv_dx);
    ok &= (b >= 0) & (b + 2 <= R.n - 1);
    base[a] = min(max(b, 0), R.n - 3);
  }
  if (!ok && flag_out_of_grid) raise_status(R.status, STATUS_OUT_OF_GRID);
  uint32_t st[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    int node[D];
    node[0] = base[0] + (D == 2 ? s / 3 : s / 9);
    node[D - 1] = base[D - 1] + s % 3;
    if (D == 3) node[1] = base[1] + (s / 3) % 3;
    st[s] = R.stamp[node_linear<D>(node, R.n)];
  }
  bool hit = false;
#pragma unroll
  for (int s = 0; s < NS; ++s) hit |= st[s] == stamp;
  return hit;
}

template <int D>
__global__ void __launch_bounds__(1024) rom_select(RomDev R) {
  __shared__ uint32_t s_nbits[kSelMaxBits / 32];
  __shared__ int s_hist[256];
  __shared__ int s_warp[32];
  __shared__ unsigned long long s_prefix;
  __shared__ int s_remaining;
  __shared__ int s_nP;
  const int t = threadIdx.x, T = blockDim.x;
  const int P = R.P, k = min(R.k, P);
  const int per = (P + T - 1) / T;
  const int p0 = min(t * per, P), p1 = min(p0 + per, P);
  const int64_t step = *R.step;
  const uint32_t stamp = (uint32_t)(step + 1);
  const uint64_t s1 = splitmix_out(splitmix_out(R.seed, (uint64_t)R.inst), (uint64_t)step);

  // clear the grid nodes of the previous basis set
  const int n_prev = R.counts[2];
  for (int i = t; i < n_prev; i += T) R.grid[R.nodes[i]] = make_float4(0.f, 0.f, 0.f, 0.f);

  // radix select of the k-th smallest hash
  if (t == 0) {
    s_prefix = 0ull;
    s_remaining = k;
  }
  unsigned long long mask = 0ull;
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 56 - 8 * pass;
    for (int i = t; i < 256; i += T) s_hist[i] = 0;
    __syncthreads();
    const unsigned long long prefix = s_prefix;
    for (int p = p0; p < p1; ++p) {
      const uint64_t h = splitmix_out(s1, (uint64_t)p);
      if ((h & mask) == prefix) atomicAdd(&s_hist[(h >> shift) & 255], 1);
    }
    __syncthreads();
    if (t < 32) {
      // first bin b whose cumulative count reaches the remaining rank (warp 0:
      // lane l holds bins 8 l .. 8 l + 7)
      const int lane = t;
      const int rem = s_remaining;
      int c[8], tot = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        c[j] = s_hist[lane * 8 + j];
        tot += c[j];
      }
      int incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned cross = __ballot_sync(0xffffffffu, incl >= rem);
      const int owner = cross ? __ffs(cross) - 1 : 31;
      if (lane == owner) {
        int acc = incl - tot, b = lane * 8 + 7;
        bool found = false;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (!found && acc + c[j] >= rem) {
            b = lane * 8 + j;
            found = true;
          } else if (!found) {
            acc += c[j];
          }
        }
        s_remaining = rem - acc;
        s_prefix = prefix | ((unsigned long long)b << shift);
      }
    }
    mask |= 255ull << shift;
    __syncthreads();
  }
  const uint64_t thr = s_prefix;
  const int need_eq = s_remaining;  // hashes equal to thr to take, lowest ids first
  // select: h < thr, or h == thr among the first need_eq by id
  int n_less = 0, n_eq = 0;
  for (int p = p0; p < p1; ++p) {
    const uint64_t h = splitmix_out(s1, (uint64_t)p);
    n_less += h < thr;
    n_eq += h == thr;
  }
  int eq_total;
  const int eq_before = block_exclusive_scan(n_eq, &eq_total, s_warp);
  int sel = 0;
  {
    int e = eq_before;
    for (int p = p0; p < p1; ++p) {
      const uint64_t h = splitmix_out(s1, (uint64_t)p);
      if (h < thr) ++sel;
      else if (h == thr) {
        if (e < need_eq) ++sel;
        ++e;
      }
    }
  }
  int n_sel;
  int pos = block_exclusive_scan(sel, &n_sel, s_warp);
  {
    int e = eq_before;
    for (int p = p0; p < p1; ++p) {
      const uint64_t h = splitmix_out(s1, (uint64_t)p);
      bool take = h < thr;
      if (h == thr) {
        take = e < need_eq;
        ++e;
      }
      if (take) R.qlist[pos++] = p;
    }
  }
  __syncthreads();
  int nP = k;
  if (R.n_groups > 0) {
    // kinematic boundaries: each group's min(m_kin, |g|) particles of smallest (hash, id) join
    // the draw; those not already drawn are appended, group by group, in ascending id
    for (int w = t; w < (P + 31) / 32; w += T) R.sel_bits[w] = 0u;
    __syncthreads();
    for (int i = t; i < k; i += T) {
      const int q = R.qlist[i];
      atomicOr(&R.sel_bits[q >> 5], 1u << (q & 31));
    }
    __syncthreads();
    if (t < 32) {
      const unsigned full = 0xffffffffu;
      int cnt = k;
      for (int g = 0; g < R.n_groups; ++g) {
        const int a0 = R.kg_off[g], a1 = R.kg_off[g + 1];
        const int rounds = min(R.m_kin, a1 - a0);
        unsigned long long ph = 0ull;
        int pid_prev = -1;
        int picked[kMaxKin];
        int np = 0;
        for (int round = 0; round < rounds; ++round) {
          unsigned long long bh = ~0ull;
          int bid = 0x7fffffff;
          for (int e = a0 + t; e < a1; e += 32) {
            const int q = R.kg_ids[e];
            const unsigned long long h = splitmix_out(s1, (uint64_t)q);
            const bool after = round == 0 || h > ph || (h == ph && q > pid_prev);
            if (after && (h < bh || (h == bh && q < bid))) {
              bh = h;
              bid = q;
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long oh = __shfl_xor_sync(full, bh, o);
            const int oid = __shfl_xor_sync(full, bid, o);
            if (oh < bh || (oh == bh && oid < bid)) {
              bh = oh;
              bid = oid;
            }
          }
          ph = bh;
          pid_prev = bid;
          if (t == 0 && !((R.sel_bits[bid >> 5] >> (bid & 31)) & 1u)) picked[np++] = bid;
        }
        if (t == 0) {
          for (int i = 1; i < np; ++i) {   // ascending ids
            const int v = picked[i];
            int j = i - 1;
            while (j >= 0 && picked[j] > v) {
              picked[j + 1] = picked[j];
              --j;
            }
            picked[j + 1] = v;
          }
          for (int i = 0; i < np; ++i) {
            R.qlist[cnt++] = picked[i];
            R.sel_bits[picked[i] >> 5] |= 1u << (picked[i] & 31);
          }
        }
        cnt = __shfl_sync(full, cnt, 0);
        __syncwarp();
      }
      if (t == 0) s_nP = cnt;
    }
    __syncthreads();
    nP = s_nP;
  }
  if (R.eulerian) {
    // Algorithm 4: only the samples; their basis set and the quadrature cells come after the
    // samples are decoded (rom_eul_cells)
    if (t == 0) R.counts[0] = nP;
    return;
  }
  // basis set I: stamp the stencil nodes of the samples (and keep them for clearing)
  constexpr int NS = (D == 2) ? 9 : 27;
  for (int i = t; i < nP; i += T) {
    const int p = R.qlist[i];
    int base[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      int b = stencil_base(R.x_all[(size_t)p * D + a], R.inv_dx);
      if (b < 0 || b + 2 > R.n - 1) raise_status(R.status, STATUS_OUT_OF_GRID);
      base[a] = min(max(b, 0), R.n - 3);
    }
    for (int s = 0; s < NS; ++s) {
      int node[D];
      node[0] = base[0] + (D == 2 ? s / 3 : s / 9);
      node[D - 1] = base[D - 1] + s % 3;
      if (D == 3) node[1] = base[1] + (s / 3) % 3;
      const int l = node_linear<D>(node, R.n);
      R.stamp[l] = stamp;
      R.nodes[i * NS + s] = l;
    }
  }
  __threadfence_block();
  __syncthreads();
  // neighbour set N: other particles with a stencil node in I (ascending ids).  The stencil's
  // stamps are loaded together (independent loads), and for P <= kSelMaxBits the first pass
  // keeps its decisions in a shared bit mask for the second.
  auto is_sample_of = [&](int p, uint64_t h) {
    if (R.n_groups > 0) return ((R.sel_bits[p >> 5] >> (p & 31)) & 1u) != 0u;
    bool smp = h < thr;
    if (h == thr) {
      // rank of p among equal hashes (only within this thread's range matters, plus eq_before)
      int e = eq_before;
      for (int q = p0; q < p; ++q) e += (splitmix_out(s1, (uint64_t)q) == thr);
      smp = e < need_eq;
    }
    return smp;
  };
  auto neighbour_hit = [&](int p, bool flag_out_of_grid) { return nb_hit<D>(R, p, stamp, flag_out_of_grid); };
  if (R.nb_multi) {
    // large P: the neighbour test runs on every SM (rom_nb_flags, rom_nb_list); here only the
    // samples' membership bits for it
    const int nw = (P + 31) / 32;
    if (R.n_groups > 0) {
      for (int w = t; w < nw; w += T) R.smp_bits[w] = R.sel_bits[w];
    } else {
      for (int w = t; w < nw; w += T) R.smp_bits[w] = 0u;
      __syncthreads();
      for (int i = t; i < nP; i += T) {
        const int q = R.qlist[i];
        atomicOr(&R.smp_bits[q >> 5], 1u << (q & 31));
      }
    }
    if (t == 0) {
      R.counts[0] = nP;
      R.counts[2] = nP * NS;
    }
    return;
  }
  const bool keep_bits = P <= kSelMaxBits;
  for (int w = t; w < (P + 31) / 32 && keep_bits; w += T) s_nbits[w] = 0u;
  __syncthreads();
  int nb = 0;
  for (int p = p0; p < p1; ++p) {
    if (is_sample_of(p, splitmix_out(s1, (uint64_t)p))) continue;
    const bool hit = neighbour_hit(p, true);
    nb += hit;
    if (hit && keep_bits) atomicOr(&s_nbits[p >> 5], 1u << (p & 31));
  }
  int n_nb;
  int npos = block_exclusive_scan(nb, &n_nb, s_warp);
  for (int p = p0; p < p1; ++p) {
    bool hit;
    if (keep_bits) {
      hit = (s_nbits[p >> 5] >> (p & 31)) & 1u;
    } else {
      if (is_sample_of(p, splitmix_out(s1, (uint64_t)p))) continue;
      hit = neighbour_hit(p, false);
    }
    if (hit) R.qlist[nP + npos++] = p;
  }
  if (t == 0) {
    R.counts[0] = nP;
    R.counts[1] = nP + n_nb;
    R.counts[2] = nP * NS;
  }
}

// Neighbour set N for large P, on every SM: warp w tests the 32 particles of bit word w (samples
// excluded) and writes the word of their decisions; per-CTA counts for rom_nb_list.
template <int D>
__global__ void __launch_bounds__(256) rom_nb_flags(RomDev R) {
  __shared__ int s_warp[32];
  const int P = R.P, nw = (P + 31) / 32;
  const uint32_t stamp = (uint32_t)(*R.step + 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wpc = (nw + gridDim.x - 1) / gridDim.x;
  const int w0 = min((int)blockIdx.x * wpc, nw), w1 = min(w0 + wpc, nw);
  int cnt = 0;
  for (int w = w0 + warp; w < w1; w += blockDim.x / 32) {
    const int p = 32 * w + lane;
    bool hit = false;
    if (p < P && !((R.smp_bits[w] >> lane) & 1u)) hit = nb_hit<D>(R, p, stamp, true);
    const uint32_t bits = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) {
      R.nb_bits[w] = bits;
      cnt += __popc(bits);
    }
  }
  int total;
  (void)block_exclusive_scan(cnt, &total, s_warp);
  if (threadIdx.x == 0) R.nb_cnt[blockIdx.x] = total;
}

// The neighbour ids in ascending order after the samples: each CTA's words (the same split as
// rom_nb_flags) from the offset of the CTAs before it, 256 words at a time.
template <int D>
__global__ void __launch_bounds__(256) rom_nb_list(RomDev R) {
  __shared__ int s_warp[32];
  const int P = R.P, nw = (P + 31) / 32;
  const int wpc = (nw + gridDim.x - 1) / gridDim.x;
  const int w0 = min((int)blockIdx.x * wpc, nw), w1 = min(w0 + wpc, nw);
  int before = 0, all = 0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const int c = R.nb_cnt[b];
    all += c;
    if (b < (int)blockIdx.x) before += c;
  }
  int n_before, n_all;
  (void)block_exclusive_scan(before, &n_before, s_warp);
  (void)block_exclusive_scan(all, &n_all, s_warp);
  const int nP = R.counts[0];
  if (blockIdx.x == 0 && threadIdx.x == 0) R.counts[1] = nP + n_all;
  int base = nP + n_before;
  for (int w = w0; w < w1; w += blockDim.x) {
    const int my = w + threadIdx.x;
    uint32_t bits = my < w1 ? R.nb_bits[my] : 0u;
    int chunk;
    int pos = base + block_exclusive_scan(__popc(bits), &chunk, s_warp);
    while (bits) {
      const int j = __ffs(bits) - 1;
      bits &= bits - 1;
      R.qlist[pos++] = 32 * my + j;
    }
    base += chunk;
  }
}

// ----------------------------------------------------- local P2G (Alg. 5)
// dec_out: (R, capQ, d) decoder output at Q with kinds [primal, dX_0..dX_{d-1}, JVP]
// and, with AFFINE, the mixed rows d/dX_b of the JVP (dv/dX).
template <int D, int MATERIAL, int TRANSFER, bool AFFINE>
__global__ void rom_p2g(RomDev R, const float* __restrict__ dec_out, int64_t capQ) {
  const int nQ = R.counts[1];
  const uint32_t stamp = (uint32_t)(*R.step + 1);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nQ; i += gridDim.x * blockDim.x) {
    const int pid = R.qlist[i];
    const int qi = R.q_by_pid ? pid : i;   // row of this point in dec_out
    float x[D], v[D], F[D * D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      x[a] = R.x_all[(size_t)pid * D + a];
      v[a] = dec_out[((size_t)(1 + D) * capQ + qi) * D + a];
#pragma unroll
      for (int b = 0; b < D; ++b) F[a * D + b] = dec_out[((size_t)(1 + b) * capQ + qi) * D + a];
    }
    // deformation gradient for the stress: measured from the decoded reference
    // configuration (F G_p) when the f_reference option holds G_p
    float Fs[D * D];
    if (R.Fref_inv) {
      const float* G = R.Fref_inv + (size_t)pid * D * D;
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
          float acc = 0.f;
#pragma unroll
          for (int e = 0; e < D; ++e) acc = fmaf(F[a * D + e], G[e * D + b], acc);
          Fs[a * D + b] = acc;
        }
    } else {
#pragma unroll
      for (int e = 0; e < D * D; ++e) Fs[e] = F[e];
    }
    float tau[D * D];
    kirchhoff<D, MATERIAL, POLAR_FP64>(Fs, R.mu, R.lam, tau);
    // MLS: A = m C - dt V0 (4/dx^2) tau, C = (dv/dX) F^-1 with AFFINE, else 0
    // (C is the same with or without the reference: both factors carry G_p)
    float A[D * D];
    const float kml = R.dt * R.vol * 4.0f * R.inv_dx * R.inv_dx;
#pragma unroll
    for (int e = 0; e < D * D; ++e) A[e] = -kml * tau[e];
    if (AFFINE && TRANSFER == MPM_TRANSFER_MLS) {
      float G[D * D], Fi[D * D];
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) G[a * D + b] = dec_out[((size_t)(2 + D + b) * capQ + qi) * D + a];
      inverse<D>(F, Fi);
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
          float c = 0.f;
#pragma unroll
          for (int e = 0; e < D; ++e) c = fmaf(G[a * D + e], Fi[e * D + b], c);
          A[a * D + b] = fmaf(R.mass, c, A[a * D + b]);
        }
    }
    int base[D];
    float w[D][3], dw[D][3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      base[a] = stencil_base(x[a], R.inv_dx);
      ok &= (base[a] >= 0) & (base[a] + 2 <= R.n - 1);
      const float fx = x[a] * R.inv_dx - (float)base[a];
      bspline_w(fx, w[a]);
      bspline_dw(fx, dw[a]);
    }
    if (!ok) continue;  // flagged by rom_select
    constexpr int NS = (D == 2) ? 9 : 27;
#pragma unroll 1
    for (int s = 0; s < NS; ++s) {
      int off[D];
      off[0] = (D == 2 ? s / 3 : s / 9);
      off[D - 1] = s % 3;
      if (D == 3) off[1] = (s / 3) % 3;
      int node[D];
      float wt = 1.f;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        node[a] = base[a] + off[a];
        wt *= w[a][off[a]];
      }
      const int l = node_linear<D>(node, R.n);
      if (R.stamp[l] != stamp) continue;   // only the basis set I is assembled
      float mom[D];
      if (TRANSFER == MPM_TRANSFER_MLS) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float q = R.mass * v[a];
#pragma unroll
          for (int b = 0; b < D; ++b) q = fmaf(A[a * D + b], (float)node[b] * R.dx - x[b], q);
          mom[a] = wt * q;
        }
      } else {
        float grad[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float gg = dw[a][off[a]] * R.inv_dx;
#pragma unroll
          for (int b = 0; b < D; ++b)
            if (b != a) gg *= w[b][off[b]];
          grad[a] = gg;
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float f = 0.f;
#pragma unroll
          for (int b = 0; b < D; ++b) f = fmaf(tau[a * D + b], grad[b], f);
          mom[a] = wt * R.mass * v[a] - R.dt * R.vol * f;
        }
      }
      atomicAdd(&R.grid[l], make_float4(wt * R.mass, mom[0], D > 1 ? mom[1] : 0.f, D > 2 ? mom[D - 1] : 0.f));
    }
  }
}

// Inverse reference gradients G_p = [(dg/dX)(X_p; xhat_ref)]^-1 from decoder rows
// [primal, dX_0 .. dX_{d-1}] over all particles.
template <int D>
__global__ void rom_reference(const float* __restrict__ dec_out, int64_t cap, int P, float* Fref_inv,
                              uint32_t* status) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    float F[D * D], G[D * D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) F[a * D + b] = dec_out[((size_t)(1 + b) * cap + p) * D + a];
    inverse<D>(F, G);
    bool ok = true;
#pragma unroll
    for (int e = 0; e < D * D; ++e) ok &= isfinite(G[e]);
    if (!ok) raise_status(status, STATUS_NONFINITE);
#pragma unroll
    for (int e = 0; e < D * D; ++e) Fref_inv[(size_t)p * D * D + e] = ok ? G[e] : (e % (D + 1) == 0 ? 1.f : 0.f);
  }
}

// ------------------------------------------- Eulerian quadrature (Alg. 4)
// Basis set I from the decoded sample positions (stamps, node list for the next
// clear) and the quadrature cells: every cell whose points reach a node of I,
// cells i - 2 .. i + 1 per axis around node i, kept when their stencils stay in
// the grid.  A cell is appended once per step (atomic exchange of its stamp).
// One CTA.  counts[1] = number of quadrature points (cells x ell^d).
template <int D>
__global__ void __launch_bounds__(1024) rom_eul_cells(RomDev R) {
  __shared__ int s_nc;
  const int t = threadIdx.x, T = blockDim.x;
  const int k = R.counts[0];
  const uint32_t stamp = (uint32_t)(*R.step + 1);
  constexpr int NS = (D == 2) ? 9 : 27;
  constexpr int NC = (D == 2) ? 16 : 64;     // cells -2 .. 1 around a node, per axis 4
  if (t == 0) s_nc = 0;
  __syncthreads();
  for (int i = t; i < k; i += T) {
    int base[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int b = stencil_base(R.x_samp[(size_t)i * D + a], R.inv_dx);
      if (b < 0 || b + 2 > R.n - 1) raise_status(R.status, STATUS_OUT_OF_GRID);
      base[a] = min(max(b, 0), R.n - 3);
    }
    for (int s = 0; s < NS; ++s) {
      int node[D];
      node[0] = base[0] + (D == 2 ? s / 3 : s / 9);
      node[D - 1] = base[D - 1] + s % 3;
      if (D == 3) node[1] = base[1] + (s / 3) % 3;
      const int l = node_linear<D>(node, R.n);
      R.stamp[l] = stamp;
      R.nodes[i * NS + s] = l;
    }
  }
  __syncthreads();
  for (int e = t; e < k * NS * NC; e += T) {
    const int l = R.nodes[e / NC];
    const int o = e % NC;
    int c[D];
    int rem = l;
#pragma unroll
    for (int a = D - 1; a >= 0; --a) {
      c[a] = rem % R.n;
      rem /= R.n;
    }
    bool ok = true;
    int oo = o;
#pragma unroll
    for (int a = D - 1; a >= 0; --a) {
      c[a] += (oo % 4) - 2;
      oo /= 4;
      ok &= (c[a] >= 1) & (c[a] <= R.n - 3);
    }
    if (!ok) continue;
    const int cl = node_linear<D>(c, R.n);
    if (atomicExch(&R.cstamp[cl], stamp) != stamp) {
      const int slot = atomicAdd(&s_nc, 1);
      if (slot < R.cap_cells) R.clist[slot] = cl;
      else raise_status(R.status, STATUS_CAPACITY);
    }
  }
  __syncthreads();
  if (t == 0) {
    int pts = 1;
    for (int a = 0; a < D; ++a) pts *= R.ell;
    R.counts[1] = min(s_nc, R.cap_cells) * pts;
    R.counts[2] = k * NS;
  }
}

// Position of quadrature point q: cell clist[q / ell^d], sub-point q % ell^d
// (lexicographic, last axis fastest), at (c + (j + 1/2) / ell) dx.
template <int D>
__device__ __forceinline__ void eul_point(const RomDev& R, int q, float x[D]) {
  int pts = 1;
#pragma unroll
  for (int a = 0; a < D; ++a) pts *= R.ell;
  int rem = R.clist[q / pts];
  int sub = q % pts;
  int c[D], j[D];
#pragma unroll
  for (int a = D - 1; a >= 0; --a) {
    c[a] = rem % R.n;
    rem /= R.n;
    j[a] = sub % R.ell;
    sub /= R.ell;
  }
#pragma unroll
  for (int a = 0; a < D; ++a) x[a] = ((float)c[a] + ((float)j[a] + 0.5f) / (float)R.ell) * R.dx;
}

// Initial reference positions: the point minus the samples' mean displacement.
template <int D>
__global__ void __launch_bounds__(1024) rom_eul_guess(RomDev R) {
  __shared__ float s_sum[32][3];
  __shared__ float s_mean[3];
  const int t = threadIdx.x, T = blockDim.x, lane = t & 31, warp = t >> 5;
  const int k = R.counts[0];
  float acc[3] = {0.f, 0.f, 0.f};
  for (int i = t; i < k; i += T) {
    const int pid = R.qlist[i];
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] += R.x_samp[(size_t)i * D + a] - R.X[(size_t)pid * D + a];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
    if (lane == 0) s_sum[warp][a] = acc[a];
  }
  __syncthreads();
  if (t < D) {
    float sm = 0.f;
    for (int w = 0; w < T / 32; ++w) sm += s_sum[w][t];
    s_mean[t] = sm / (float)max(k, 1);
  }
  __syncthreads();
  const int nq = R.counts[1];
  for (int q = t; q < nq; q += T) {
    float x[D];
    eul_point<D>(R, q, x);
#pragma unroll
    for (int a = 0; a < D; ++a) R.qX[(size_t)q * D + a] = x[a] - s_mean[a];
  }
}

// One Newton step of the decoder inversion, X <- X - (dg/dX)^-1 (g(X) - x_q), from
// decoder rows [primal, dX_0 .. dX_{d-1}] at X.
template <int D>
__global__ void rom_eul_newton(RomDev R, const float* __restrict__ dec, int64_t cap) {
  const int nq = R.counts[1];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    float x[D], F[D * D], Fi[D * D], r[D];
    eul_point<D>(R, q, x);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      r[a] = dec[(size_t)q * D + a] - x[a];
#pragma unroll
      for (int b = 0; b < D; ++b) F[a * D + b] = dec[((size_t)(1 + b) * cap + q) * D + a];
    }
    inverse<D>(F, Fi);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      float dX = 0.f;
#pragma unroll
      for (int b = 0; b < D; ++b) dX = fmaf(Fi[a * D + b], r[b], dX);
      if (isfinite(dX)) R.qX[(size_t)q * D + a] -= dX;
    }
  }
}

// Mass, reference volume and local P2G of the Eulerian quadrature points (Algorithms 4 and 5).
// dec rows [primal, dX_0 .. dX_{d-1}, JVP] at the points' final reference positions X.  A point
// carries mass rho0 V_q / J and reference volume V_q / J when X lies in the reference domain (the
// occupancy boxes) and the inversion converged (|g(X) - x_q| < tol); otherwise none.  Stress from
// F = dg/dX, C = 0, assembled onto the nodes of the basis set only.
template <int D, int MATERIAL, int TRANSFER>
__global__ void rom_eul_p2g(RomDev R, const float* __restrict__ dec, int64_t cap, float tol) {
  const int nq = R.counts[1];
  const uint32_t stamp = (uint32_t)(*R.step + 1);
  float Vq = 1.f;
#pragma unroll
  for (int a = 0; a < D; ++a) Vq *= R.dx / (float)R.ell;
  const float rho0 = R.mass / R.vol;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    float x[D], v[D], F[D * D];
    eul_point<D>(R, q, x);
    float res2 = 0.f;
    bool inside = true;
    int lin = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const float r = dec[(size_t)q * D + a] - x[a];
      res2 = fmaf(r, r, res2);
      v[a] = dec[((size_t)(1 + D) * cap + q) * D + a];
#pragma unroll
      for (int b = 0; b < D; ++b) F[a * D + b] = dec[((size_t)(1 + b) * cap + q) * D + a];
      const float ib = floorf((R.qX[(size_t)q * D + a] - R.occ_origin[a]) / R.occ_h);
      inside &= (ib >= 0.f) & (ib < (float)R.occ_shape[a]);
      lin = lin * R.occ_shape[a] + (inside ? (int)ib : 0);
    }
    inside = inside && R.occ[lin] != 0;
    const float J = det_minus_one<D>(F) + 1.0f;
    const bool ok = inside && (res2 < tol * tol) && (J > 0.f) && isfinite(J);
    const float V0 = ok ? Vq / J : 0.f;
    const float mq = ok ? rho0 * V0 : 0.f;
    R.qV0[q] = V0;
    R.qm[q] = mq;
    if (!ok) continue;
    float tau[D * D];
    kirchhoff<D, MATERIAL, POLAR_FP64>(F, R.mu, R.lam, tau);
    int base[D];
    float w[D][3], dw[D][3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      base[a] = stencil_base(x[a], R.inv_dx);
      const float fx = x[a] * R.inv_dx - (float)base[a];
      bspline_w(fx, w[a]);
      bspline_dw(fx, dw[a]);
    }
    constexpr int NS = (D == 2) ? 9 : 27;
    const float kml = R.dt * V0 * 4.0f * R.inv_dx * R.inv_dx;
#pragma unroll 1
    for (int s = 0; s < NS; ++s) {
      int off[D];
      off[0] = (D == 2 ? s / 3 : s / 9);
      off[D - 1] = s % 3;
      if (D == 3) off[1] = (s / 3) % 3;
      int node[D];
      float wt = 1.f;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        node[a] = base[a] + off[a];
        wt *= w[a][off[a]];
      }
      const int l = node_linear<D>(node, R.n);
      if (R.stamp[l] != stamp) continue;   // only the basis set I is assembled
      float mom[D];
      if (TRANSFER == MPM_TRANSFER_MLS) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float qq = mq * v[a];
#pragma unroll
          for (int b = 0; b < D; ++b) qq = fmaf(-kml * tau[a * D + b], (float)node[b] * R.dx - x[b], qq);
          mom[a] = wt * qq;
        }
      } else {
        float grad[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float gg = dw[a][off[a]] * R.inv_dx;
#pragma unroll
          for (int b = 0; b < D; ++b)
            if (b != a) gg *= w[b][off[b]];
          grad[a] = gg;
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float f = 0.f;
#pragma unroll
          for (int b = 0; b < D; ++b) f = fmaf(tau[a * D + b], grad[b], f);
          mom[a] = wt * mq * v[a] - R.dt * V0 * f;
        }
      }
      atomicAdd(&R.grid[l], make_float4(wt * mq, mom[0], D > 1 ? mom[1] : 0.f, D > 2 ? mom[D - 1] : 0.f));
    }
  }
}

// ---------------------------------------- grid update + G2P to the samples
template <int D>
__global__ void rom_g2p(RomDev R) {
  const int nP = R.counts[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nP; i += gridDim.x * blockDim.x) {
    const int pid = R.qlist[i];
    float x[D], w[D][3];
    int base[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      x[a] = R.x_samp ? R.x_samp[(size_t)i * D + a] : R.x_all[(size_t)pid * D + a];
      base[a] = min(max(stencil_base(x[a], R.inv_dx), 0), R.n - 3);
      bspline_w(x[a] * R.inv_dx - (float)base[a], w[a]);
    }
    float v[D];
#pragma unroll
    for (int a = 0; a < D; ++a) v[a] = 0.f;
    constexpr int NS = (D == 2) ? 9 : 27;
    for (int s = 0; s < NS; ++s) {
      int off[D], node[D];
      off[0] = (D == 2 ? s / 3 : s / 9);
      off[D - 1] = s % 3;
      if (D == 3) off[1] = (s / 3) % 3;
      float wt = 1.f;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        node[a] = base[a] + off[a];
        wt *= w[a][off[a]];
      }
      float vi[D];
      grid_node_velocity<D>(R.grid[node_linear<D>(node, R.n)], node, R.n, R.bc, R.bc_width, R.dt, R.g, vi);
#pragma unroll
      for (int a = 0; a < D; ++a) v[a] = fmaf(wt, vi[a], v[a]);
    }
    if (R.kin_group) {
      // kinematic sample: its prescribed velocity (the Dirichlet condition of the full-space update)
      const int kg = R.kin_group[pid];
      if (kg >= 0) {
#pragma unroll
        for (int a = 0; a < D; ++a) v[a] = R.kin_vel[3 * kg + a];
      }
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      R.v_trial[(size_t)i * D + a] = v[a];
      R.x_trial[(size_t)i * D + a] = fmaf(R.dt, v[a], x[a]);
    }
  }
}

// ----------------------------------------------------------- least squares
// Solver state in FP64 (per reduced-order instance).
struct RomSolve {
  double* xh;        // xhat_n
  double* xh_prev;   // xhat_{n-1}
  double* vh;        // vhat_n
  double* vh_new;    // vhat_{n+1}
  double* xk;        // Gauss-Newton iterate
  double* delta;     // Gauss-Newton step
  double* scal;      // [0] f0, [1] slope, [2] |delta|
  double* acc;       // normal-equation accumulators: r(r+1)/2 + r + 1
  double* fls;       // line-search objectives (kLS)
  uint32_t* counter; // last-CTA counters [0] normal, [1] line search
  int32_t* picks;    // per Gauss-Newton iteration of the last step: accepted trial m (step 2^-m), -1 none
  // FP32 copies fed to the decoder
  float* xh32;       // xhat_n
  float* vh32;       // vhat_n
  float* xk32;       // iterate
  float* dk32;       // xhat_n - iterate
  float* ls_base32;  // kLS x r, rows = xhat_n
  float* ls_dir32;   // kLS x r, rows = (xk - xhat_n) + 2^-m delta
};

enum { NE_VEL = 0, NE_GN = 1, NE_FIT = 2 };
constexpr int kNERows = 32;      // normal-equation rows per CTA tile

// One term of a compensated dot product (Ogita, Rump and Oishi, "Accurate sum and dot product",
// 2005, Dot2): the product x y is split exactly into p + pe by an FMA, p is added to the running
// sum sh by an error-free two-sum, and both rounding errors are collected in sc.  sh + sc carries
// the dot product to about twice the working precision.
// The _rn intrinsics keep the compiler from contracting the product into the sums.
__device__ __forceinline__ void dot2_term(float x, float y, float& sh, float& sc) {
  const float p = __fmul_rn(x, y);
  const float pe = fmaf(x, y, -p);
  const float t = __fadd_rn(sh, p);
  const float z = __fsub_rn(t, sh);
  sc += __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z)) + pe;
  sh = t;
}

// Cholesky solve of the SPD system A x = b held in shared memory (A: r x r,
// row-major, r <= 32) by the block's first warp, synchronised with __syncwarp
// only; the other warps wait at the final barrier.  Column j: every lane reads
// the pivot and forms its reciprocal square root itself (Newton-Raphson in FP64
// from an FP32 seed: no broadcast, no FP64 division or square root, which are
// long-latency sequences on this GPU); lane q owns row j + 1 + q of the
// column and of the trailing update.  The substitutions multiply by the stored
// reciprocal pivots.  Returns false, for the whole block, if a pivot is not
// positive.
__device__ bool chol_solve(double* A, double* b, int r) {
  __shared__ int s_bad;
  __shared__ double s_rdiag[kMaxRl];
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int bad = 0;
    for (int j = 0; j < r; ++j) {
      const double piv = A[j * r + j];
      if (!(piv > 0.0)) {
        bad = 1;
        break;
      }
      // 1 / sqrt(piv) by Newton-Raphson on f(y) = 1/y^2 - piv: y <- y (3 - piv y^2) / 2,
      // quadratic convergence, two steps from the FP32 seed reach FP64 precision
      double y = (double)rsqrtf((float)piv);
      y = y * (1.5 - 0.5 * piv * y * y);
      y = y * (1.5 - 0.5 * piv * y * y);
      const int i = j + 1 + lane;
      double l = 0.0;
      if (i < r) {
        l = A[i * r + j] * y;
        A[i * r + j] = l;
      }
      if (lane == 0) {
        A[j * r + j] = piv * y;
        s_rdiag[j] = y;
      }
      __syncwarp();
      if (i < r)
        for (int k = j + 1; k <= i; ++k) A[i * r + k] -= l * A[k * r + j];
      __syncwarp();
    }
    if (!bad) {
      // L y = b, by columns
      for (int k = 0; k < r; ++k) {
        const double yk = b[k] * s_rdiag[k];
        __syncwarp();
        if (lane == 0) b[k] = yk;
        const int i = k + 1 + lane;
        if (i < r) b[i] -= A[i * r + k] * yk;
        __syncwarp();
      }
      // L^T x = y, by rows of L
      for (int i = r - 1; i >= 0; --i) {
        const double xi = b[i] * s_rdiag[i];
        __syncwarp();
        if (lane == 0) b[i] = xi;
        if (lane < i) b[lane] -= A[i * r + lane] * xi;
        __syncwarp();
      }
    }
    if (lane == 0) s_bad = bad;
  }
  __syncthreads();
  return !s_bad;
}

// Solve of the same SPD system by an FP32 Cholesky factor with iterative refinement in FP64
// (the first warp; FP64 arithmetic has a ~65-cycle dependent latency on this GPU, FP32 ~5): the
// correction of each sweep solves L L^T d = b - A x with the FP32 factor, the residual is formed in
// FP64 from the unmodified A, and the sweeps stop once the correction is below 2^-40 of x (the
// entries of A and b, assembled by compensated FP32 sums, carry about that relative accuracy).
// Converges when cond(A) is well below 1 / FP32 epsilon; returns false (A and b untouched) if the
// FP32 factorisation breaks down or 8 sweeps do not converge, and the caller falls back to
// chol_solve.  On success b holds the solution.
// The factor lives in registers: lane i holds row i of L (KR >= r entries, unrolled loops with
// compile-time bounds), the columns pass between lanes by shuffles, and a copy of L in shared
// memory gives each lane its column for the back substitution.
template <int KR>
__device__ bool chol_solve_refined_reg(const double* A, double* b, int r) {
  __shared__ float Lsm[kMaxRl * (kMaxRl + 1)];
  __shared__ double s_x[kMaxRl];
  __shared__ int s_ok;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    float Lr[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k) Lr[k] = (lane < r && k < r) ? (float)A[lane * r + k] : 0.f;
    float rd = 0.f;   // 1 / L[lane][lane]
    bool ok = true;
#pragma unroll
    for (int j = 0; j < KR; ++j) {
      if (j < r && ok) {
        const float piv = __shfl_sync(0xffffffffu, Lr[j], j);
        if (!(piv > 0.f) || !(piv < 3.0e38f)) {
          ok = false;   // uniform: every lane sees the same pivot
        } else {
          const float y = rsqrtf(piv);
          const float l = lane > j ? Lr[j] * y : 0.f;
          if (lane == j) {
            Lr[j] = piv * y;
            rd = y;
          } else if (lane > j) {
            Lr[j] = l;
          }
#pragma unroll
          for (int k = j + 1; k < KR; ++k) {
            if (k < r) {
              const float lk = __shfl_sync(0xffffffffu, l, k);
              if (lane >= k) Lr[k] = fmaf(-l, lk, Lr[k]);
            }
          }
        }
      }
    }
    int conv = 0;
    if (ok) {
#pragma unroll
      for (int k = 0; k < KR; ++k) Lsm[lane * (kMaxRl + 1) + k] = Lr[k];
      __syncwarp();
      float Lc[KR];   // column `lane` of L: Lc[i] = L[i][lane]
#pragma unroll
      for (int i = 0; i < KR; ++i) Lc[i] = Lsm[i * (kMaxRl + 1) + lane];
      if (lane < r) s_x[lane] = 0.0;
      float v = lane < r ? (float)b[lane] : 0.f;
      __syncwarp();
      for (int sweep = 0; sweep < 8 && !conv; ++sweep) {
        // L L^T d = v (FP32), d in v: forward by columns, backward by rows of L
#pragma unroll
        for (int k = 0; k < KR; ++k) {
          if (k < r) {
            const float yk = __shfl_sync(0xffffffffu, v * rd, k);
            if (lane == k) v = yk;
            else if (lane > k) v = fmaf(-Lr[k], yk, v);
          }
        }
#pragma unroll
        for (int i = KR - 1; i >= 0; --i) {
          if (i < r) {
            const float xi = __shfl_sync(0xffffffffu, v * rd, i);
            if (lane == i) v = xi;
            else if (lane < i) v = fmaf(-Lc[i], xi, v);
          }
        }
        // x += d; residual b - A x in FP64 (four independent partial sums per row)
        float dmax = 0.f, xmax = 0.f;
        if (lane < r) {
          const double xn = s_x[lane] + (double)v;
          s_x[lane] = xn;
          dmax = fabsf(v);
          xmax = fabsf((float)xn);
        }
        __syncwarp();
        if (lane < r) {
          double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
          int jj = 0;
          for (; jj + 3 < r; jj += 4) {
            p0 = fma(A[lane * r + jj], s_x[jj], p0);
            p1 = fma(A[lane * r + jj + 1], s_x[jj + 1], p1);
            p2 = fma(A[lane * r + jj + 2], s_x[jj + 2], p2);
            p3 = fma(A[lane * r + jj + 3], s_x[jj + 3], p3);
          }
          for (; jj < r; ++jj) p0 = fma(A[lane * r + jj], s_x[jj], p0);
          v = (float)(b[lane] - ((p0 + p1) + (p2 + p3)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
          xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
        }
        conv = dmax <= 9.1e-13f * xmax;   // 2^-40 of x: below the accuracy of the assembled system
        __syncwarp();
      }
    }
    if (conv && lane < r) b[lane] = s_x[lane];
    if (lane == 0) s_ok = conv;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ bool chol_solve_refined(const double* A, double* b, int r) {
  if (r <= 8) return chol_solve_refined_reg<8>(A, b, r);
  if (r <= 16) return chol_solve_refined_reg<16>(A, b, r);
  return chol_solve_refined_reg<kMaxRl>(A, b, r);
}

__global__ void __launch_bounds__(kNormBlock) rom_normal(RomDev R, RomSolve S, const float* __restrict__ dec,
                                                         int64_t cap, int mode, const float* __restrict__ target,
                                                         int projection, int n_rows_override, float ridge) {
  const int d = R.d, r = R.r;
  const int nP = n_rows_override > 0 ? n_rows_override : R.counts[0];
  const int rows = nP * d;
  const int n_mat = r * (r + 1) / 2;
  const int n_acc = n_mat + r + 1;
  __shared__ float sJ[kNERows][kMaxRl + 1];
  __shared__ float sb[kNERows];
  __shared__ bool s_last;
  // hi / lo FP32 split of vhat_n (FP64) for the velocity right-hand side
  __shared__ float s_vh_hi[kMaxRl], s_vh_lo[kMaxRl];
  if (mode == NE_VEL && threadIdx.x < r) {
    const double v = S.vh[threadIdx.x];
    const float hi = (float)v;
    s_vh_hi[threadIdx.x] = hi;
    s_vh_lo[threadIdx.x] = (float)(v - (double)hi);
  }
  __syncthreads();
  for (int row0 = blockIdx.x * kNERows; row0 < rows; row0 += gridDim.x * kNERows) {
    const int nr = min(kNERows, rows - row0);
    for (int e = threadIdx.x; e < nr * r; e += blockDim.x) {
      const int rr = e / r, c = e % r;
      const int row = row0 + rr, p = row / d, a = row % d;
      sJ[rr][c] = dec[((size_t)(1 + c) * cap + p) * d + a];
    }
    if (threadIdx.x < nr) {
      const int rr = threadIdx.x;
      const int row = row0 + rr, p = row / d, a = row % d;
      float b;
      if (mode == NE_VEL) {
        // right-hand side of the velocity increment: v_trial - J vhat_n, J vhat_n by a compensated
        // dot product of the FP32 row with the hi / lo parts of vhat_n
        float sh = 0.f, sc = 0.f;
        for (int c = 0; c < r; ++c) {
          const float x = dec[((size_t)(1 + c) * cap + p) * d + a];
          dot2_term(x, s_vh_hi[c], sh, sc);
          dot2_term(x, s_vh_lo[c], sh, sc);
        }
        b = (R.v_trial[(size_t)p * d + a] - sh) - sc;
      } else if (mode == NE_GN) {
        b = dec[((size_t)(1 + r) * cap + p) * d + a] + R.dt * R.v_trial[(size_t)p * d + a];
      } else {
        b = target[(size_t)p * d + a] - dec[(size_t)p * d + a];
      }
      sb[rr] = b;
    }
    __syncthreads();
    // entries of J^T J (upper triangle), J^T b and b^T b over this tile's rows: compensated FP32
    // dot products (Dot2: exact products by FMA, error-free sums), added in FP64
    for (int e = threadIdx.x; e < n_acc; e += blockDim.x) {
      float sh = 0.f, sc = 0.f;
      if (e < n_mat) {
        // upper-triangle index e -> (i, j), i <= j
        int i = 0, rem = e;
        while (rem >= r - i) {
          rem -= r - i;
          ++i;
        }
        const int j = i + rem;
        for (int q = 0; q < nr; ++q) dot2_term(sJ[q][i], sJ[q][j], sh, sc);
      } else if (e < n_mat + r) {
        const int i = e - n_mat;
        for (int q = 0; q < nr; ++q) dot2_term(sJ[q][i], sb[q], sh, sc);
      } else {
        for (int q = 0; q < nr; ++q) dot2_term(sb[q], sb[q], sh, sc);
      }
      atomicAdd(&S.acc[e], (double)sh + (double)sc);
    }
    __syncthreads();
  }
  // last CTA: factor and solve
  __threadfence();
  if (threadIdx.x == 0) s_last = atomicAdd(&S.counter[0], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ double A[kMaxRl * kMaxRl];
  __shared__ double A_keep[kMaxRl * kMaxRl];
  __shared__ double bvec[kMaxRl];
  __shared__ double s_rhs[kMaxRl];
  __shared__ double s_bb, s_shift;
  for (int e = threadIdx.x; e < n_mat; e += blockDim.x) {
    int i = 0, rem = e;
    while (rem >= r - i) {
      rem -= r - i;
      ++i;
    }
    const int j = i + rem;
    const double v = atomicAdd(&S.acc[e], 0.0);
    A[i * r + j] = v;
    A[j * r + i] = v;
    A_keep[i * r + j] = v;
    A_keep[j * r + i] = v;
  }
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    bvec[i] = atomicAdd(&S.acc[n_mat + i], 0.0);
    s_rhs[i] = bvec[i];
  }
  if (threadIdx.x == 0) s_bb = atomicAdd(&S.acc[n_mat + r], 0.0);
  __syncthreads();
  for (int e = threadIdx.x; e < n_acc; e += blockDim.x) S.acc[e] = 0.0;
  if (threadIdx.x == 0) S.counter[0] = 0u;
  __syncthreads();
  // Ridge rho tr(A) / r (rho = max(ridge, 1e-10)): the regularised least
  // squares of the ridge option, and with the 1e-10 floor it keeps the
  // factorisation defined when latent directions do not move the samples
  // (rank-deficient J^T J; the solution then tends to the minimum-norm one).
  // One retry with a larger ridge; after that the step is skipped and
  // CHOLESKY raised.
  if (threadIdx.x < 32) {
    // trace by a warp reduction (serial FP64 sums are long dependency chains on this GPU)
    double tr = threadIdx.x < r ? A_keep[threadIdx.x * r + threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if (threadIdx.x == 0) s_shift = (tr > 0 ? tr : 1.0) / r;
  }
  __syncthreads();
  bool ok = false;
  for (int attempt = 0; attempt < 2 && !ok; ++attempt) {
    const double rr = attempt == 0 ? fmax(1e-10, (double)ridge) : fmax(1e-6, 100.0 * (double)ridge);
    const double ridge_abs = rr * s_shift;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) A[e] = A_keep[e] + ((e / r) == (e % r) ? ridge_abs : 0.0);
    for (int i = threadIdx.x; i < r; i += blockDim.x) bvec[i] = s_rhs[i];
    __syncthreads();
    ok = chol_solve_refined(A, bvec, r) || chol_solve(A, bvec, r);
  }
  if (!ok) {
    if (threadIdx.x == 0) raise_status(R.status, STATUS_CHOLESKY);
    for (int i = threadIdx.x; i < r; i += blockDim.x) bvec[i] = 0.0;  // no step
    __syncthreads();
  }
  if (mode == NE_VEL) {
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
      // the solve gave the increment from vhat_n (zero if the factorisation failed)
      const double v = S.vh[i] + bvec[i];
      S.vh_new[i] = v;
      if (projection == 1) {
        // velocity-only projection (Alg. 7): xhat_{n+1} = xhat_n + dt vhat_{n+1}
        S.xk[i] = S.xh[i] + (double)R.dt * v;
      } else {
        // Gauss-Newton initial guess 2 xhat_n - xhat_{n-1}
        const double g = 2.0 * S.xh[i] - S.xh_prev[i];
        S.xk[i] = g;
        S.xk32[i] = (float)g;
        S.dk32[i] = (float)(S.xh[i] - g);
      }
    }
  } else {
    // GN step: J^T J delta = J^T b with b = -residual
    __shared__ double s_slope, s_dn;
    if (threadIdx.x < 32) {
      double sl = threadIdx.x < r ? s_rhs[threadIdx.x] * bvec[threadIdx.x] : 0.0;
      double dn = threadIdx.x < r ? bvec[threadIdx.x] * bvec[threadIdx.x] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sl += __shfl_xor_sync(0xffffffffu, sl, o);
        dn += __shfl_xor_sync(0xffffffffu, dn, o);
      }
      if (threadIdx.x == 0) {
        s_slope = -2.0 * sl;   // d/dalpha |res + alpha J delta|^2 at 0 = 2 res^T J delta = -2 b^T J delta
        s_dn = sqrt(dn);
        S.scal[0] = s_bb;      // f0 = |res|^2
        S.scal[1] = s_slope;
        S.scal[2] = s_dn;
      }
    }
    for (int i = threadIdx.x; i < r; i += blockDim.x) S.delta[i] = bvec[i];
    __syncthreads();
    const float* base32 = (mode == NE_FIT) ? S.xk32 : S.xh32;
    for (int e = threadIdx.x; e < kLS * r; e += blockDim.x) {
      const int m = e / r, i = e % r;
      const double alpha = ldexp(1.0, -m);
      const double basev = (mode == NE_FIT) ? S.xk[i] : S.xh[i];
      S.ls_base32[e] = base32[i];
      S.ls_dir32[e] = (float)((S.xk[i] - basev) + alpha * bvec[i]);
    }
  }
}

// Line-search objectives f(alpha_m) = |g(xhat_k + alpha_m delta) - x_trial|^2 for all
// trials at once; dec = decoder output (1 + kLS, cap, d) at the nP samples with kinds
// [primal, secant along trial direction 0, ..., kLS - 1] (one primal row per sample).  The last CTA picks the
// first trial meeting Armijo and updates the iterate; on the final iteration it
// also commits the step.
__global__ void __launch_bounds__(kNormBlock) rom_linesearch(RomDev R, RomSolve S, const float* __restrict__ dec,
                                                             int64_t cap, int mode, const float* __restrict__ target,
                                                             int final_iter, double armijo_c, int n_rows_override,
                                                             int iter) {
  const int d = R.d, r = R.r;
  const int nP = n_rows_override > 0 ? n_rows_override : R.counts[0];
  const int per = nP * d;
  __shared__ double s_red[kNormBlock / 32];
  __shared__ bool s_last;
  for (int m = blockIdx.x; m < kLS; m += gridDim.x) {
    double s = 0.0;
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int p = e / d, a = e % d;
      // rows: kind 0 the primal at the base latent, kind 1 + m the secant of trial m
      const double sec = (double)dec[((size_t)(1 + m) * cap + p) * d + a];
      double res;
      if (mode == NE_FIT) {
        // secant from the iterate: g(xk + alpha delta) = g(xk) + secant; residual vs target
        res = sec + (double)dec[(size_t)p * d + a] - (double)target[(size_t)p * d + a];
      } else {
        // g(xhat_k + alpha delta) - x_trial = secant_from_xhat_n - dt v_trial
        res = sec - (double)R.dt * R.v_trial[(size_t)p * d + a];
      }
      s = fma(res, res, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0;
      for (int w = 0; w < kNormBlock / 32; ++w) tot += s_red[w];
      S.fls[m] = tot;
    }
    __syncthreads();
  }
  __threadfence();
  if (threadIdx.x == 0) s_last = atomicAdd(&S.counter[1], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ int s_pick;
  if (threadIdx.x == 0) {
    S.counter[1] = 0u;
    const double f0 = S.scal[0], slope = S.scal[1], dn = S.scal[2];
    int pick = -1;
    for (int m = 0; m < kLS; ++m) {
      const double f = *((volatile double*)&S.fls[m]);
      if (f <= f0 + armijo_c * ldexp(1.0, -m) * slope) {
        pick = m;
        break;
      }
    }
    // no trial decreased the objective: a failure only if the step is not
    // negligible and the linear model promised a decrease well above the FP32
    // resolution of the objective (-slope / 2 = |J delta|^2 > 1e-3 f0);
    // otherwise the iterate has converged
    double xn = 0;
    for (int i = 0; i < r; ++i) xn += S.xk[i] * S.xk[i];
    if (pick < 0 && dn > 1e-8 * (1.0 + sqrt(xn)) && -0.5 * slope > 1e-3 * f0)
      raise_status(R.status, STATUS_GN_NO_DECREASE);
    if (iter >= 0 && iter < kMaxGnIters) S.picks[iter] = pick;
    s_pick = pick;
  }
  __syncthreads();
  const int pick = s_pick;
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    double xk = S.xk[i];
    if (pick >= 0) xk += ldexp(1.0, -pick) * S.delta[i];
    S.xk[i] = xk;
    S.xk32[i] = (float)xk;
    const double basev = (mode == NE_FIT) ? xk : S.xh[i];
    S.dk32[i] = (float)(basev - xk);
  }
  if (final_iter && mode != NE_FIT) {
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
      S.xh_prev[i] = S.xh[i];
      S.xh[i] = S.xk[i];
      S.vh[i] = S.vh_new[i];
      S.xh32[i] = (float)S.xk[i];
      S.vh32[i] = (float)S.vh_new[i];
    }
    if (threadIdx.x == 0) *R.step += 1;
  }
}

// Commit of the velocity-only projection (Alg. 7).
__global__ void rom_commit_velocity_only(RomDev R, RomSolve S) {
  for (int i = threadIdx.x; i < R.r; i += blockDim.x) {
    S.xh_prev[i] = S.xh[i];
    S.xh[i] = S.xk[i];
    S.vh[i] = S.vh_new[i];
    S.xh32[i] = (float)S.xk[i];
    S.vh32[i] = (float)S.vh_new[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) *R.step += 1;
}

// Accumulated position error of Section 5: acc[0] += sum |a - b|^2, acc[1] += sum |b|^2 (FP64).
__global__ void metric_accumulate_kernel(const float* __restrict__ a, const float* __restrict__ b, int64_t n,
                                         double* acc) {
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = a[i], y = b[i];
    s0 = fma(x - y, x - y, s0);
    s1 = fma(y, y, s1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], s0);
    atomicAdd(&acc[1], s1);
  }
}

}  // namespace mpmrom

// ============================================================================
// Host runtime and C ABI
// ============================================================================
using namespace mpmrom;

struct rom_ctx {
  rom_config cfg{};
  const mpm_decoder* dec = nullptr;
  int d = 0, r = 0, P = 0, k = 0, n = 0;
  int n_sm = 0;
  RomDev dv{};
  RomSolve sv{};
  // device buffers
  float* X = nullptr;
  float* x_all = nullptr;       // decoded positions (the primal block of outQ when merged)
  float* x_all_buf = nullptr;
  bool merged = false;          // one decode of all particles serves positions and quadrature rows
  int32_t* qlist = nullptr;
  uint32_t* smp_bits = nullptr;  // large P: neighbour test on every SM
  uint32_t* nb_bits = nullptr;
  int32_t* nb_cnt = nullptr;
  int nb_ctas = 0;
  int32_t* counts = nullptr;
  int32_t* nodes = nullptr;
  uint32_t* stamp = nullptr;
  float4* grid = nullptr;
  float* v_trial = nullptr;
  float* x_trial = nullptr;
  int64_t* step = nullptr;
  uint32_t* status = nullptr;
  int32_t* nP_all = nullptr;    // device constant P (decode-all point count)
  float* outQ = nullptr;        // (2 d + 2, P, d)
  float* Fref_inv = nullptr;    // (P, d, d) with f_reference
  float* xref32 = nullptr;      // (r) reference latent
  float* outS = nullptr;        // (r + 2, k, d)
  float* outLS = nullptr;       // (1 + kLS, k, d) (capacity P for the fit)
  double* solve_mem = nullptr;
  float* solve32 = nullptr;
  uint32_t* counters = nullptr;
  int32_t* picks = nullptr;        // line-search choices of the last step (kMaxGnIters)
  // kinematic boundaries: sample capacity k_cap = k + m_kin x n_groups
  int k_cap = 0;
  int32_t* kin_group = nullptr;
  float* kin_vel = nullptr;
  int32_t* kg_off = nullptr;
  int32_t* kg_ids = nullptr;
  uint32_t* sel_bits = nullptr;
  // Eulerian quadrature (Algorithm 4)
  bool eulerian = false;
  int ell = 0, newton_iters = 0;
  float newton_tol = 0.f;
  int64_t cap_q = 0;            // quadrature-point capacity (cells x ell^d)
  uint32_t* cstamp = nullptr;
  int32_t* clist = nullptr;
  float* qX = nullptr;
  float* qm = nullptr;
  float* qV0 = nullptr;
  uint8_t* occ = nullptr;
  float* outE = nullptr;        // (d + 2, cap_q, d) decoder rows at the quadrature points
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  // set while rom_set_kinematic replaces buffers; still set if it failed half way, after which
  // rom_step refuses to run (the step would read buffers that are gone)
  bool reconfig_failed = false;
  // incremented whenever the step's kernel arguments change (its captured graph is dropped); a
  // batch built from this context refuses to run once it differs from the value it recorded
  uint64_t generation = 0;
};

// Many reduced-order contexts stepped by one graph launch: each context's step graph is a child
// graph of one parent graph, all children independent (parallel branches).
struct rom_batch {
  std::vector<rom_ctx*> ctx;
  std::vector<uint64_t> gen;
  cudaGraphExec_t exec = nullptr;
};

namespace {

// Lagrangian quadrature (Algorithm 3): decoded positions, samples, basis and neighbour sets, F
// and v at the quadrature points, local P2G onto the basis set.
mpm_status rom_launch_lagrangian(rom_ctx* c, const int* kq, int Rq, bool affine, cudaStream_t s) {
  const int d = c->d;
  const int M = c->cfg.material, T = c->cfg.transfer;
  mpm_status st = MPM_OK;
  if (c->merged) {
    // 1 + 3. one decode of every particle with the quadrature rows: positions (x_all is its
    // primal block) and F, v for whichever particles the neighbourhood selects
    st = decoder_launch_dev(c->dec, c->X, nullptr, c->nP_all, 1, c->P, c->sv.xh32, c->sv.vh32, kq, Rq, c->outQ, s);
    if (st != MPM_OK) return st;
  } else {
    // 1. decode all particles at xhat_n
    int k_primal[1] = {0};
    st = decoder_launch_dev(c->dec, c->X, nullptr, c->nP_all, 1, c->P, c->sv.xh32, nullptr, k_primal, 1, c->x_all, s);
    if (st != MPM_OK) return st;
  }
  // 2. samples, basis set, neighbours (for large P the neighbour test on every SM)
  if (d == 2)
    rom_select<2><<<1, 1024, 0, s>>>(c->dv);
  else
    rom_select<3><<<1, 1024, 0, s>>>(c->dv);
  MPM_CUDA_TRY(cudaGetLastError());
  if (c->dv.nb_multi) {
    if (d == 2) {
      rom_nb_flags<2><<<c->nb_ctas, 256, 0, s>>>(c->dv);
      rom_nb_list<2><<<c->nb_ctas, 256, 0, s>>>(c->dv);
    } else {
      rom_nb_flags<3><<<c->nb_ctas, 256, 0, s>>>(c->dv);
      rom_nb_list<3><<<c->nb_ctas, 256, 0, s>>>(c->dv);
    }
    MPM_CUDA_TRY(cudaGetLastError());
  }
  if (!c->merged) {
    // 3. F and v at the quadrature points Q
    st = decoder_launch_dev(c->dec, c->X, c->qlist, c->counts + 1, 1, c->P, c->sv.xh32, c->sv.vh32, kq, Rq, c->outQ,
                            s);
    if (st != MPM_OK) return st;
  }
  // 4. local P2G onto I
  const int b_q = std::max(1, std::min(ceil_div(c->P, 256), c->n_sm * 4));
#define P2G_CASE(dd, mm, tt)                                                                     \
  if (d == dd && M == mm && T == tt) {                                                           \
    if (affine)                                                                                  \
      rom_p2g<dd, mm, tt, true><<<b_q, 256, 0, s>>>(c->dv, c->outQ, c->P);                       \
    else                                                                                         \
      rom_p2g<dd, mm, tt, false><<<b_q, 256, 0, s>>>(c->dv, c->outQ, c->P);                      \
  }
  P2G_CASE(2, 0, 0) P2G_CASE(2, 0, 1) P2G_CASE(2, 1, 0) P2G_CASE(2, 1, 1)
  P2G_CASE(3, 0, 0) P2G_CASE(3, 0, 1) P2G_CASE(3, 1, 0) P2G_CASE(3, 1, 1)
#undef P2G_CASE
  MPM_CUDA_TRY(cudaGetLastError());
  return MPM_OK;
}

mpm_status rom_launch_step(rom_ctx* c, cudaStream_t s) {
  const int d = c->d, r = c->r;
  const bool affine = c->cfg.affine && c->cfg.transfer == MPM_TRANSFER_MLS;
  int kq[8];
  kq[0] = 0;
  for (int a = 0; a < d; ++a) kq[1 + a] = 1 + a;
  kq[1 + d] = 1000;  // JVP along vhat_n
  for (int a = 0; a < d; ++a) kq[2 + d + a] = 2000 + 1 + a;  // d/dX_a of the JVP
  const int Rq = affine ? 2 * d + 2 : d + 2;
  mpm_status st = MPM_OK;
  int ks[kMaxRl + 2];
  ks[0] = 0;
  for (int j = 0; j < r; ++j) ks[1 + j] = 1 + d + j;
  const int b_s = std::max(1, ceil_div(c->k_cap, 128));
  const int b_ne = std::max(1, std::min(ceil_div((int64_t)c->k_cap * d, kNERows), 64));
  const int M = c->cfg.material, T = c->cfg.transfer;
  if (c->eulerian) {
    // Algorithm 4.  1. samples
    if (d == 2)
      rom_select<2><<<1, 1024, 0, s>>>(c->dv);
    else
      rom_select<3><<<1, 1024, 0, s>>>(c->dv);
    MPM_CUDA_TRY(cudaGetLastError());
    // 2. positions and latent Jacobian at the samples (the rows of the velocity projection)
    st = decoder_launch_dev(c->dec, c->X, c->qlist, c->counts + 0, 1, c->k_cap, c->sv.xh32, nullptr, ks, r + 1, c->outS,
                            s);
    if (st != MPM_OK) return st;
    // 3. basis set, quadrature cells and points, initial reference positions
    if (d == 2) {
      rom_eul_cells<2><<<1, 1024, 0, s>>>(c->dv);
      rom_eul_guess<2><<<1, 1024, 0, s>>>(c->dv);
    } else {
      rom_eul_cells<3><<<1, 1024, 0, s>>>(c->dv);
      rom_eul_guess<3><<<1, 1024, 0, s>>>(c->dv);
    }
    MPM_CUDA_TRY(cudaGetLastError());
    // 4. Newton inversion of the decoder at the points
    const int b_e = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(c->cap_q, (int64_t)256), c->n_sm * 4));
    int kn[4] = {0, 1, 2, 3};
    for (int it = 0; it < c->newton_iters; ++it) {
      st = decoder_launch_dev(c->dec, c->qX, nullptr, c->counts + 1, 1, c->cap_q, c->sv.xh32, nullptr, kn, 1 + d,
                              c->outE, s);
      if (st != MPM_OK) return st;
      if (d == 2)
        rom_eul_newton<2><<<b_e, 256, 0, s>>>(c->dv, c->outE, c->cap_q);
      else
        rom_eul_newton<3><<<b_e, 256, 0, s>>>(c->dv, c->outE, c->cap_q);
      MPM_CUDA_TRY(cudaGetLastError());
    }
    // 5. F, v at the final reference positions; mass; local P2G onto I
    st = decoder_launch_dev(c->dec, c->qX, nullptr, c->counts + 1, 1, c->cap_q, c->sv.xh32, c->sv.vh32, kq, d + 2,
                            c->outE, s);
    if (st != MPM_OK) return st;
    const float tol = c->newton_tol * c->cfg.dx;
#define EUL_CASE(dd, mm, tt) \
    if (d == dd && M == mm && T == tt) rom_eul_p2g<dd, mm, tt><<<b_e, 256, 0, s>>>(c->dv, c->outE, c->cap_q, tol);
    EUL_CASE(2, 0, 0) EUL_CASE(2, 0, 1) EUL_CASE(2, 1, 0) EUL_CASE(2, 1, 1)
    EUL_CASE(3, 0, 0) EUL_CASE(3, 0, 1) EUL_CASE(3, 1, 0) EUL_CASE(3, 1, 1)
#undef EUL_CASE
    MPM_CUDA_TRY(cudaGetLastError());
  } else {
    st = rom_launch_lagrangian(c, kq, Rq, affine, s);
    if (st != MPM_OK) return st;
  }
  if (d == 2)
    rom_g2p<2><<<b_s, 128, 0, s>>>(c->dv);
  else
    rom_g2p<3><<<b_s, 128, 0, s>>>(c->dv);
  MPM_CUDA_TRY(cudaGetLastError());
  // 6. velocity projection: J = dg/dxhat at (X^P, xhat_n) (decoded in step 2 with the Eulerian quadrature)
  if (!c->eulerian) {
    st = decoder_launch_dev(c->dec, c->X, c->qlist, c->counts + 0, 1, c->k_cap, c->sv.xh32, nullptr, ks, r + 1, c->outS,
                            s);
    if (st != MPM_OK) return st;
  }
  rom_normal<<<b_ne, kNormBlock, 0, s>>>(c->dv, c->sv, c->outS, c->k_cap, NE_VEL, nullptr, c->cfg.projection, 0,
                                         c->cfg.ridge);
  MPM_CUDA_TRY(cudaGetLastError());
  if (c->cfg.projection == 1) {
    rom_commit_velocity_only<<<1, 64, 0, s>>>(c->dv, c->sv);
    MPM_CUDA_TRY(cudaGetLastError());
    return MPM_OK;
  }
  // 7. Gauss-Newton on the positions
  ks[1 + r] = 1001;  // secant g(xhat_n) - g(xhat_k)
  int kls[1 + kLS];
  kls[0] = 0;
  for (int m = 0; m < kLS; ++m) kls[1 + m] = 3000 + m;   // secant along trial direction m
  for (int it = 0; it < c->cfg.gn_iters; ++it) {
    st = decoder_launch_dev(c->dec, c->X, c->qlist, c->counts + 0, 1, c->k_cap, c->sv.xk32, c->sv.dk32, ks, r + 2,
                            c->outS, s);
    if (st != MPM_OK) return st;
    rom_normal<<<b_ne, kNormBlock, 0, s>>>(c->dv, c->sv, c->outS, c->k_cap, NE_GN, nullptr, 0, 0, c->cfg.ridge);
    MPM_CUDA_TRY(cudaGetLastError());
    st = decoder_launch_dev(c->dec, c->X, c->qlist, c->counts + 0, 1, c->k_cap, c->sv.ls_base32, c->sv.ls_dir32, kls,
                            1 + kLS, c->outLS, s);
    if (st != MPM_OK) return st;
    rom_linesearch<<<kLS, kNormBlock, 0, s>>>(c->dv, c->sv, c->outLS, c->k_cap, NE_GN, nullptr,
                                              it == c->cfg.gn_iters - 1, 1e-4, 0, it);
    MPM_CUDA_TRY(cudaGetLastError());
  }
  return MPM_OK;
}

template <typename T>
mpm_status ralloc(T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return set_error(MPM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  e = cudaMemset(*p, 0, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return set_error(MPM_ECUDA, std::string("cudaMemset: ") + cudaGetErrorString(e));
  return MPM_OK;
}

// Cell and point buffers of the Eulerian quadrature for up to n_samp samples: the union over the
// samples of the 6^d cells around their 3^d stencil nodes (clipped to the grid), ell^d points per
// cell.  While the buffers are replaced the capacity reads 0, so a failed allocation leaves a
// context whose step has no quadrature points and raises STATUS_CAPACITY instead of touching freed
// memory.
mpm_status rom_alloc_quadrature(rom_ctx* c, int n_samp) {
  const int d = c->d;
  int64_t cells_grid = 1, cells_samp = n_samp, pts = 1;
  for (int a = 0; a < d; ++a) {
    cells_grid *= c->n - 3;
    cells_samp *= 6;
    pts *= c->ell;
  }
  const int64_t cap_cells = std::min(cells_grid, cells_samp);
  MPM_CHECK_ARG(cap_cells * pts < (int64_t)1 << 30, "quadrature-point capacity");
  c->cap_q = 0;
  c->dv.cap_cells = 0;
  cudaFree(c->clist);
  cudaFree(c->qX);
  cudaFree(c->qm);
  cudaFree(c->qV0);
  cudaFree(c->outE);
  c->clist = nullptr;
  c->qX = c->qm = c->qV0 = c->outE = nullptr;
  c->dv.clist = nullptr;
  c->dv.qX = c->dv.qm = c->dv.qV0 = nullptr;
  const int64_t cap_q = cap_cells * pts;
  mpm_status st;
  if ((st = ralloc(&c->clist, (size_t)cap_cells)) != MPM_OK) return st;
  if ((st = ralloc(&c->qX, (size_t)cap_q * d)) != MPM_OK) return st;
  if ((st = ralloc(&c->qm, (size_t)cap_q)) != MPM_OK) return st;
  if ((st = ralloc(&c->qV0, (size_t)cap_q)) != MPM_OK) return st;
  if ((st = ralloc(&c->outE, (size_t)(d + 2) * cap_q * d)) != MPM_OK) return st;
  c->dv.clist = c->clist;
  c->dv.qX = c->qX;
  c->dv.qm = c->qm;
  c->dv.qV0 = c->qV0;
  c->dv.cap_cells = (int)cap_cells;
  c->cap_q = cap_q;
  return MPM_OK;
}

}  // namespace

extern "C" {

mpm_status rom_create(const rom_config* cfg, const mpm_decoder* dec, const float* X, int64_t n_particles,
                      rom_ctx** out) {
  MPM_CHECK_ARG(cfg && dec && X && out, "null argument");
  *out = nullptr;
  MPM_CHECK_ARG(cfg->dim == 2 || cfg->dim == 3, "dim must be 2 or 3");
  MPM_CHECK_ARG(n_particles >= 1 && n_particles < (1 << 30), "particle count");
  MPM_CHECK_ARG(cfg->n_samples >= 1, "n_samples >= 1");
  MPM_CHECK_ARG(cfg->gn_iters >= 1 && cfg->gn_iters <= kMaxGnIters, "gn_iters in [1, 16]");
  MPM_CHECK_ARG(cfg->projection == 0 || cfg->projection == 1, "projection: 0 position-velocity, 1 velocity-only");
  MPM_CHECK_ARG(cfg->latent_dim >= 1 && cfg->latent_dim <= kMaxRl, "latent dimension in [1, 32]");
  int dec_d = 0, dec_r = 0;
  decoder_shape(dec, &dec_d, &dec_r);
  MPM_CHECK_ARG(dec_d == cfg->dim && dec_r == cfg->latent_dim, "the decoder's d and r must equal dim and latent_dim");
  MPM_CHECK_ARG(cfg->n_grid >= 8, "n_grid");
  MPM_CHECK_ARG(cfg->dx > 0 && cfg->dt > 0 && cfg->rho > 0 && cfg->p_vol > 0, "dx, dt, rho, p_vol must be > 0");
  MPM_CHECK_ARG(cfg->E > 0 && cfg->nu > -1 && cfg->nu < 0.5f, "E must be > 0 and -1 < nu < 0.5");
  MPM_CHECK_ARG(cfg->bc == MPM_BC_STICKY || cfg->bc == MPM_BC_SLIP_FLOOR, "bc");
  MPM_CHECK_ARG(cfg->bc_width >= 0, "bc_width");
  MPM_CHECK_ARG(cfg->material == MPM_NEO_HOOKEAN || cfg->material == MPM_FIXED_COROTATED, "material");
  MPM_CHECK_ARG(cfg->transfer == MPM_TRANSFER_MLS || cfg->transfer == MPM_TRANSFER_PIC, "transfer");
  MPM_CHECK_ARG(cfg->ridge >= 0.f, "ridge >= 0");
  MPM_CHECK_ARG(cfg->affine == 0 || cfg->affine == 1, "affine: 0 or 1");
  MPM_CHECK_ARG(cfg->f_reference == 0 || cfg->f_reference == 1, "f_reference: 0 or 1");
  MPM_CHECK_ARG(cfg->quadrature == 0 || cfg->quadrature == 1, "quadrature: 0 Lagrangian, 1 Eulerian");
  MPM_CHECK_ARG(cfg->ell >= 0 && cfg->ell <= 4, "ell in [1, 4] (0: default 2)");
  MPM_CHECK_ARG(cfg->newton_iters >= 0 && cfg->newton_iters <= 16, "newton_iters in [1, 16] (0: default 4)");
  MPM_CHECK_ARG(cfg->newton_tol >= 0.f, "newton_tol >= 0 (0: default 1e-3)");
  MPM_CHECK_ARG(!(cfg->quadrature == 1 && cfg->f_reference == 1), "f_reference needs the Lagrangian quadrature");
  MPM_CHECK_ARG(!(cfg->quadrature == 1 && cfg->affine == 1), "affine needs the Lagrangian quadrature");
  auto* c = new rom_ctx();
  c->cfg = *cfg;
  c->dec = dec;
  c->d = cfg->dim;
  c->r = cfg->latent_dim;
  c->P = (int)n_particles;
  c->k = std::min<int>(cfg->n_samples, c->P);
  c->k_cap = c->k;
  c->n = cfg->n_grid;
  int devn = 0;
  cudaGetDevice(&devn);
  cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, devn);
  const int d = c->d, r = c->r, P = c->P, k = c->k;
  const int NS = d == 2 ? 9 : 27;
  const size_t gn = d == 2 ? (size_t)c->n * c->n : (size_t)c->n * c->n * c->n;
  mpm_status st;
  struct Owner {  // destroys the partly built context on every early return
    rom_ctx* c;
    ~Owner() { rom_destroy(c); }
  } owner{c};
  if ((st = ralloc(&c->X, (size_t)P * d)) != MPM_OK) return st;
  if ((st = ralloc(&c->x_all_buf, (size_t)P * d)) != MPM_OK) return st;
  if ((st = ralloc(&c->qlist, P)) != MPM_OK) return st;
  if (P > kSelMaxBits) {
    c->nb_ctas = std::max(1, c->n_sm * 4);
    if ((st = ralloc(&c->smp_bits, (size_t)(P + 31) / 32)) != MPM_OK) return st;
    if ((st = ralloc(&c->nb_bits, (size_t)(P + 31) / 32)) != MPM_OK) return st;
    if ((st = ralloc(&c->nb_cnt, (size_t)c->nb_ctas)) != MPM_OK) return st;
  }
  if ((st = ralloc(&c->counts, 4)) != MPM_OK) return st;
  if ((st = ralloc(&c->nodes, (size_t)k * NS)) != MPM_OK) return st;
  if ((st = ralloc(&c->stamp, gn)) != MPM_OK) return st;
  if ((st = ralloc(&c->grid, gn)) != MPM_OK) return st;
  if ((st = ralloc(&c->v_trial, (size_t)P * d)) != MPM_OK) return st;
  if ((st = ralloc(&c->x_trial, (size_t)P * d)) != MPM_OK) return st;
  if ((st = ralloc(&c->step, 1)) != MPM_OK) return st;
  if ((st = ralloc(&c->status, 1)) != MPM_OK) return st;
  if ((st = ralloc(&c->nP_all, 1)) != MPM_OK) return st;
  if ((st = ralloc(&c->outQ, (size_t)(2 * d + 2) * P * d)) != MPM_OK) return st;
  if (cfg->f_reference) {
    if ((st = ralloc(&c->Fref_inv, (size_t)P * d * d)) != MPM_OK) return st;
    if ((st = ralloc(&c->xref32, (size_t)r)) != MPM_OK) return st;
  }
  // one decode of all particles per step when the neighbourhood of the samples covers most of
  // the body anyway (2D: a sample's neighbourhood spans 5 x 5 cells, ~100 particles at 4 per cell)
  c->eulerian = cfg->quadrature == 1;
  c->merged = !c->eulerian && (int64_t)P <= 32 * (int64_t)c->k;
  c->x_all = c->merged ? c->outQ : c->x_all_buf;
  if ((st = ralloc(&c->outS, (size_t)(r + 2) * P * d)) != MPM_OK) return st;
  if ((st = ralloc(&c->outLS, (size_t)(1 + kLS) * P * d)) != MPM_OK) return st;
  const int n_acc = r * (r + 1) / 2 + r + 1;
  const size_t n64 = 6 * (size_t)r + 3 + n_acc + kLS;
  if ((st = ralloc(&c->solve_mem, n64)) != MPM_OK) return st;
  if ((st = ralloc(&c->solve32, (size_t)4 * r + 2 * kLS * r)) != MPM_OK) return st;
  if ((st = ralloc(&c->counters, 2)) != MPM_OK) return st;
  if ((st = ralloc(&c->picks, kMaxGnIters)) != MPM_OK) return st;
  MPM_CUDA_TRY(cudaMemcpy(c->X, X, sizeof(float) * P * d, cudaMemcpyDefault));
  MPM_CUDA_TRY(cudaMemcpy(c->nP_all, &c->P, sizeof(int32_t), cudaMemcpyHostToDevice));
  RomDev& v = c->dv;
  if (c->eulerian) {
    c->ell = cfg->ell ? cfg->ell : 2;
    c->newton_iters = cfg->newton_iters ? cfg->newton_iters : 4;
    c->newton_tol = cfg->newton_tol > 0.f ? cfg->newton_tol : 1e-3f;
    if ((st = ralloc(&c->cstamp, gn)) != MPM_OK) return st;
    if ((st = rom_alloc_quadrature(c, k)) != MPM_OK) return st;
    // reference domain: union of the particles' volume boxes of side h = V0^(1/d) centred on X,
    // as occupancy flags of a box grid of spacing h from origin = min X - h / 2
    std::vector<float> hX((size_t)P * d);
    MPM_CUDA_TRY(cudaMemcpy(hX.data(), c->X, sizeof(float) * P * d, cudaMemcpyDeviceToHost));
    const double h = std::pow((double)cfg->p_vol, 1.0 / d);
    double lo[3] = {0, 0, 0};
    int64_t shape[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) {
      lo[a] = hX[a];
      for (int p = 0; p < P; ++p) lo[a] = std::min(lo[a], (double)hX[(size_t)p * d + a]);
      lo[a] -= 0.5 * h;
      int64_t mx = 0;
      for (int p = 0; p < P; ++p) mx = std::max<int64_t>(mx, (int64_t)std::floor(((double)hX[(size_t)p * d + a] - lo[a]) / h));
      shape[a] = mx + 1;
    }
    const int64_t n_occ = shape[0] * shape[1] * shape[2];
    MPM_CHECK_ARG(n_occ <= ((int64_t)1 << 28), "reference occupancy grid too large (particle volume vs extent)");
    std::vector<uint8_t> occ((size_t)n_occ, 0);
    for (int p = 0; p < P; ++p) {
      int64_t lin = 0;
      for (int a = 0; a < d; ++a)
        lin = lin * shape[a] + (int64_t)std::floor(((double)hX[(size_t)p * d + a] - lo[a]) / h);
      occ[(size_t)lin] = 1;
    }
    if ((st = ralloc(&c->occ, (size_t)n_occ)) != MPM_OK) return st;
    MPM_CUDA_TRY(cudaMemcpy(c->occ, occ.data(), (size_t)n_occ, cudaMemcpyHostToDevice));
    v.eulerian = 1;
    v.ell = c->ell;
    v.x_samp = c->outS;   // primal block of the sample decode
    v.cstamp = c->cstamp;
    v.occ = c->occ;
    for (int a = 0; a < 3; ++a) {
      v.occ_origin[a] = (float)lo[a];
      v.occ_shape[a] = (int)shape[a];
    }
    v.occ_h = (float)h;
  }
  v.d = d;
  v.r = r;
  v.P = P;
  v.n = c->n;
  v.k = k;
  v.dx = cfg->dx;
  v.inv_dx = (float)(1.0 / cfg->dx);
  v.dt = cfg->dt;
  for (int a = 0; a < 3; ++a) v.g[a] = cfg->gravity[a];
  v.bc = cfg->bc;
  v.bc_width = cfg->bc_width;
  v.mass = cfg->rho * cfg->p_vol;
  v.vol = cfg->p_vol;
  const double E = cfg->E, nu = cfg->nu;
  v.mu = (float)(E / (2 * (1 + nu)));
  v.lam = (float)(E * nu / ((1 + nu) * (1 - 2 * nu)));
  v.seed = cfg->seed;
  v.inst = cfg->instance;
  v.X = c->X;
  v.x_all = c->x_all;
  v.q_by_pid = c->merged ? 1 : 0;
  v.qlist = c->qlist;
  v.nb_multi = c->nb_bits ? 1 : 0;
  v.smp_bits = c->smp_bits;
  v.nb_bits = c->nb_bits;
  v.nb_cnt = c->nb_cnt;
  v.counts = c->counts;
  v.nodes = c->nodes;
  v.stamp = c->stamp;
  v.grid = c->grid;
  v.v_trial = c->v_trial;
  v.x_trial = c->x_trial;
  v.step = c->step;
  v.status = c->status;
  RomSolve& S = c->sv;
  double* m = c->solve_mem;
  S.xh = m;
  S.xh_prev = m + r;
  S.vh = m + 2 * r;
  S.vh_new = m + 3 * r;
  S.xk = m + 4 * r;
  S.delta = m + 5 * r;
  S.scal = m + 6 * r;
  S.acc = m + 6 * r + 3;
  S.fls = S.acc + n_acc;
  S.counter = c->counters;
  S.picks = c->picks;
  float* f = c->solve32;
  S.xh32 = f;
  S.vh32 = f + r;
  S.xk32 = f + 2 * r;
  S.dk32 = f + 3 * r;
  S.ls_base32 = f + 4 * r;
  S.ls_dir32 = f + 4 * r + kLS * r;
  MPM_CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  owner.c = nullptr;
  *out = c;
  return MPM_OK;
}

void rom_destroy(rom_ctx* c) {
  if (!c) return;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  cudaFree(c->X);
  cudaFree(c->x_all_buf);
  cudaFree(c->kin_group);
  cudaFree(c->kin_vel);
  cudaFree(c->kg_off);
  cudaFree(c->kg_ids);
  cudaFree(c->sel_bits);
  cudaFree(c->cstamp);
  cudaFree(c->clist);
  cudaFree(c->qX);
  cudaFree(c->qm);
  cudaFree(c->qV0);
  cudaFree(c->occ);
  cudaFree(c->outE);
  cudaFree(c->qlist);
  cudaFree(c->smp_bits);
  cudaFree(c->nb_bits);
  cudaFree(c->nb_cnt);
  cudaFree(c->counts);
  cudaFree(c->nodes);
  cudaFree(c->stamp);
  cudaFree(c->grid);
  cudaFree(c->v_trial);
  cudaFree(c->x_trial);
  cudaFree(c->step);
  cudaFree(c->status);
  cudaFree(c->nP_all);
  cudaFree(c->outQ);
  cudaFree(c->Fref_inv);
  cudaFree(c->xref32);
  cudaFree(c->outS);
  cudaFree(c->outLS);
  cudaFree(c->solve_mem);
  cudaFree(c->solve32);
  cudaFree(c->counters);
  cudaFree(c->picks);
  delete c;
}

mpm_status rom_set_state(rom_ctx* c, const double* xhat, const double* vhat, const double* xhat_prev, int64_t step,
                         void* stream) {
  MPM_CHECK_ARG(c && xhat && vhat && xhat_prev, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int r = c->r;
  std::vector<double> h(3 * r);
  MPM_CUDA_TRY(cudaMemcpyAsync(h.data(), xhat, sizeof(double) * r, cudaMemcpyDefault, s));
  MPM_CUDA_TRY(cudaMemcpyAsync(h.data() + r, vhat, sizeof(double) * r, cudaMemcpyDefault, s));
  MPM_CUDA_TRY(cudaMemcpyAsync(h.data() + 2 * r, xhat_prev, sizeof(double) * r, cudaMemcpyDefault, s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<float> h32(2 * r);
  for (int i = 0; i < r; ++i) {
    h32[i] = (float)h[i];
    h32[r + i] = (float)h[r + i];
  }
  MPM_CUDA_TRY(cudaMemcpyAsync(c->sv.xh, h.data(), sizeof(double) * r, cudaMemcpyHostToDevice, s));
  MPM_CUDA_TRY(cudaMemcpyAsync(c->sv.vh, h.data() + r, sizeof(double) * r, cudaMemcpyHostToDevice, s));
  MPM_CUDA_TRY(cudaMemcpyAsync(c->sv.xh_prev, h.data() + 2 * r, sizeof(double) * r, cudaMemcpyHostToDevice, s));
  MPM_CUDA_TRY(cudaMemcpyAsync(c->sv.xh32, h32.data(), sizeof(float) * r, cudaMemcpyHostToDevice, s));
  MPM_CUDA_TRY(cudaMemcpyAsync(c->sv.vh32, h32.data() + r, sizeof(float) * r, cudaMemcpyHostToDevice, s));
  MPM_CUDA_TRY(cudaMemcpyAsync(c->step, &step, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  // a new step index may repeat stamps of an earlier run: start from an empty grid
  const size_t gn = c->d == 2 ? (size_t)c->n * c->n : (size_t)c->n * c->n * c->n;
  MPM_CUDA_TRY(cudaMemsetAsync(c->stamp, 0, sizeof(uint32_t) * gn, s));
  MPM_CUDA_TRY(cudaMemsetAsync(c->grid, 0, sizeof(float4) * gn, s));
  MPM_CUDA_TRY(cudaMemsetAsync(c->counts, 0, sizeof(int32_t) * 4, s));
  if (c->cstamp) MPM_CUDA_TRY(cudaMemsetAsync(c->cstamp, 0, sizeof(uint32_t) * gn, s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  return MPM_OK;
}

mpm_status rom_get_state(rom_ctx* c, double* xhat, double* vhat, double* xhat_prev, int64_t* step, void* stream) {
  MPM_CHECK_ARG(c, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int r = c->r;
  if (xhat) MPM_CUDA_TRY(cudaMemcpyAsync(xhat, c->sv.xh, sizeof(double) * r, cudaMemcpyDefault, s));
  if (vhat) MPM_CUDA_TRY(cudaMemcpyAsync(vhat, c->sv.vh, sizeof(double) * r, cudaMemcpyDefault, s));
  if (xhat_prev) MPM_CUDA_TRY(cudaMemcpyAsync(xhat_prev, c->sv.xh_prev, sizeof(double) * r, cudaMemcpyDefault, s));
  if (step) MPM_CUDA_TRY(cudaMemcpyAsync(step, c->step, sizeof(int64_t), cudaMemcpyDefault, s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  return MPM_OK;
}

// Captures one step of context c (on its private stream) into a graph.
static mpm_status rom_capture_step(rom_ctx* c, cudaGraph_t* out) {
  cudaGraph_t g = nullptr;
  MPM_CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  mpm_status st = rom_launch_step(c, c->cap_stream);
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (st != MPM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return set_error(MPM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  *out = g;
  return MPM_OK;
}

mpm_status rom_batch_create(rom_ctx* const* ctxs, int32_t n, rom_batch** out) {
  MPM_CHECK_ARG(ctxs && out && n >= 1, "null argument or n < 1");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    MPM_CHECK_ARG(ctxs[i], "null context in the batch");
    MPM_CHECK_ARG(!ctxs[i]->reconfig_failed, "a failed rom_set_kinematic left a context without its buffers");
    for (int j = 0; j < i; ++j)
      MPM_CHECK_ARG(ctxs[j] != ctxs[i], "a context appears twice in the batch (its steps would race)");
  }
  cudaGraph_t parent = nullptr;
  MPM_CUDA_TRY(cudaGraphCreate(&parent, 0));
  mpm_status st = MPM_OK;
  for (int i = 0; i < n && st == MPM_OK; ++i) {
    cudaGraph_t g = nullptr;
    st = rom_capture_step(ctxs[i], &g);
    if (st != MPM_OK) break;
    cudaGraphNode_t node;
    const cudaError_t e = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, g);   // clones g
    cudaGraphDestroy(g);
    if (e != cudaSuccess) st = set_error(MPM_ECUDA, std::string("child graph: ") + cudaGetErrorString(e));
  }
  cudaGraphExec_t exec = nullptr;
  if (st == MPM_OK) {
    const cudaError_t e = cudaGraphInstantiate(&exec, parent, 0);
    if (e != cudaSuccess) st = set_error(MPM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  cudaGraphDestroy(parent);
  if (st != MPM_OK) return st;
  auto* b = new rom_batch();
  b->ctx.assign(ctxs, ctxs + n);
  for (int i = 0; i < n; ++i) b->gen.push_back(ctxs[i]->generation);
  b->exec = exec;
  *out = b;
  return MPM_OK;
}

mpm_status rom_batch_step(rom_batch* b, int n_steps, void* stream) {
  MPM_CHECK_ARG(b, "null batch");
  MPM_CHECK_ARG(n_steps >= 0, "n_steps >= 0");
  for (size_t i = 0; i < b->ctx.size(); ++i)
    MPM_CHECK_ARG(b->ctx[i]->generation == b->gen[i] && !b->ctx[i]->reconfig_failed,
                  "a context of the batch was reconfigured after the batch was built: rebuild the batch");
  for (int k = 0; k < n_steps; ++k) MPM_CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  return MPM_OK;
}

void rom_batch_destroy(rom_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  delete b;
}

mpm_status rom_step(rom_ctx* c, int n_steps, void* stream) {
  MPM_CHECK_ARG(c, "null context");
  MPM_CHECK_ARG(n_steps >= 0, "n_steps >= 0");
  MPM_CHECK_ARG(!c->reconfig_failed, "a failed rom_set_kinematic left the context without its buffers");
  cudaStream_t s = (cudaStream_t)stream;
  if (!c->graph) {
    // capture one step on a private stream; every launch reads its dynamic
    // values (step counter, set sizes, latent state) from device memory
    cudaGraph_t g = nullptr;
    MPM_CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    mpm_status st = rom_launch_step(c, c->cap_stream);
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (st != MPM_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return set_error(MPM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return set_error(MPM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  for (int i = 0; i < n_steps; ++i) MPM_CUDA_TRY(cudaGraphLaunch(c->graph, s));
  return MPM_OK;
}

mpm_status rom_status_word(rom_ctx* c, uint32_t* out, int clear, void* stream) {
  MPM_CHECK_ARG(c && out, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t h = 0;
  MPM_CUDA_TRY(cudaMemcpyAsync(&h, c->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  if (clear) MPM_CUDA_TRY(cudaMemsetAsync(c->status, 0, sizeof(uint32_t), s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  *out = h;
  return MPM_OK;
}

mpm_status rom_debug(rom_ctx* c, int32_t* qlist, int32_t* counts, float* x_all, float* v_trial, float* x_trial,
                     void* stream) {
  MPM_CHECK_ARG(c, "null context");
  cudaStream_t s = (cudaStream_t)stream;
  if (counts) MPM_CUDA_TRY(cudaMemcpyAsync(counts, c->counts, sizeof(int32_t) * 3, cudaMemcpyDefault, s));
  if (qlist) MPM_CUDA_TRY(cudaMemcpyAsync(qlist, c->qlist, sizeof(int32_t) * c->P, cudaMemcpyDefault, s));
  if (x_all) MPM_CUDA_TRY(cudaMemcpyAsync(x_all, c->x_all, sizeof(float) * c->P * c->d, cudaMemcpyDefault, s));
  if (v_trial) MPM_CUDA_TRY(cudaMemcpyAsync(v_trial, c->v_trial, sizeof(float) * c->k_cap * c->d, cudaMemcpyDefault, s));
  if (x_trial) MPM_CUDA_TRY(cudaMemcpyAsync(x_trial, c->x_trial, sizeof(float) * c->k_cap * c->d, cudaMemcpyDefault, s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  return MPM_OK;
}

mpm_status rom_debug_line_search(rom_ctx* c, int32_t* picks, int32_t* n_iters, void* stream) {
  MPM_CHECK_ARG(c && picks && n_iters, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  MPM_CUDA_TRY(cudaMemcpyAsync(picks, c->picks, sizeof(int32_t) * kMaxGnIters, cudaMemcpyDefault, s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  *n_iters = c->cfg.projection == 1 ? 0 : c->cfg.gn_iters;
  return MPM_OK;
}

mpm_status rom_debug_quadrature(rom_ctx* c, int32_t* n_points, float* x_points, float* X_points, float* mass,
                                float* V0, void* stream) {
  MPM_CHECK_ARG(c, "null context");
  MPM_CHECK_ARG(c->eulerian, "rom_debug_quadrature needs the Eulerian quadrature");
  cudaStream_t s = (cudaStream_t)stream;
  int32_t cnt[2] = {0, 0};
  MPM_CUDA_TRY(cudaMemcpyAsync(cnt, c->counts, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  const int64_t nq = cnt[1];
  if (n_points) *n_points = (int32_t)nq;
  if (X_points) MPM_CUDA_TRY(cudaMemcpyAsync(X_points, c->qX, sizeof(float) * nq * c->d, cudaMemcpyDefault, s));
  if (mass) MPM_CUDA_TRY(cudaMemcpyAsync(mass, c->qm, sizeof(float) * nq, cudaMemcpyDefault, s));
  if (V0) MPM_CUDA_TRY(cudaMemcpyAsync(V0, c->qV0, sizeof(float) * nq, cudaMemcpyDefault, s));
  if (x_points) {
    // cell ids, expanded on the host into the points' positions (c + (j + 1/2) / ell) dx
    const int d = c->d, ell = c->ell;
    int pts = 1;
    for (int a = 0; a < d; ++a) pts *= ell;
    std::vector<int32_t> cells((size_t)(nq / pts));
    MPM_CUDA_TRY(cudaMemcpyAsync(cells.data(), c->clist, sizeof(int32_t) * cells.size(), cudaMemcpyDeviceToHost, s));
    MPM_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<float> xp((size_t)nq * d);
    for (int64_t q = 0; q < nq; ++q) {
      int rem = cells[(size_t)(q / pts)], sub = (int)(q % pts);
      int cc[3], jj[3];
      for (int a = d - 1; a >= 0; --a) {
        cc[a] = rem % c->n;
        rem /= c->n;
        jj[a] = sub % ell;
        sub /= ell;
      }
      for (int a = 0; a < d; ++a)
        xp[(size_t)q * d + a] = ((float)cc[a] + ((float)jj[a] + 0.5f) / (float)ell) * c->cfg.dx;
    }
    MPM_CUDA_TRY(cudaMemcpyAsync(x_points, xp.data(), sizeof(float) * nq * d, cudaMemcpyDefault, s));
  }
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  return MPM_OK;
}

mpm_status rom_decode_all(rom_ctx* c, float* x_out, void* stream) {
  MPM_CHECK_ARG(c && x_out, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  int k_primal[1] = {0};
  mpm_status st = decoder_launch_dev(c->dec, c->X, nullptr, c->nP_all, 1, c->P, c->sv.xh32, nullptr, k_primal, 1,
                                     x_out, s);
  return st;
}

mpm_status rom_set_kinematic(rom_ctx* c, const int32_t* group, int32_t n_groups, const float* velocities,
                             int32_t min_samples, void* stream) {
  MPM_CHECK_ARG(c, "null context");
  MPM_CHECK_ARG(n_groups >= 0, "n_groups >= 0");
  const bool on = n_groups > 0 && group;
  if (on) {
    MPM_CHECK_ARG(velocities, "velocities of the kinematic groups");
    MPM_CHECK_ARG(min_samples >= 1 && min_samples <= kMaxKin, "min_samples in [1, 32]");
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int P = c->P, NS = c->d == 2 ? 9 : 27;
  // read and check everything before the context changes: a rejected call leaves it as it was
  std::vector<int32_t> h, off, ids;
  std::vector<float> v3;
  if (on) {
    h.resize(P);
    std::vector<float> hv((size_t)n_groups * c->d);
    MPM_CUDA_TRY(cudaMemcpyAsync(h.data(), group, sizeof(int32_t) * P, cudaMemcpyDefault, s));
    MPM_CUDA_TRY(cudaMemcpyAsync(hv.data(), velocities, sizeof(float) * hv.size(), cudaMemcpyDefault, s));
    MPM_CUDA_TRY(cudaStreamSynchronize(s));
    off.assign(n_groups + 1, 0);
    for (int p = 0; p < P; ++p) {
      MPM_CHECK_ARG(h[p] >= -1 && h[p] < n_groups, "group ids in [-1, n_groups)");
      if (h[p] >= 0) ++off[h[p] + 1];
    }
    for (float vv : hv) MPM_CHECK_ARG(std::isfinite(vv), "finite group velocities");
    for (int g = 0; g < n_groups; ++g) off[g + 1] += off[g];
    ids.resize(off[n_groups]);
    std::vector<int32_t> fill(off.begin(), off.end() - 1);
    for (int p = 0; p < P; ++p)
      if (h[p] >= 0) ids[fill[h[p]]++] = p;   // ascending within each group
    v3.assign((size_t)n_groups * 3, 0.f);
    for (int g = 0; g < n_groups; ++g)
      for (int a = 0; a < c->d; ++a) v3[(size_t)3 * g + a] = hv[(size_t)c->d * g + a];
  }
  // from here on the buffers the captured step reads are replaced: drop the graph first, and
  // mark the context unusable until every buffer is in place again
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  ++c->generation;
  c->reconfig_failed = true;
  cudaFree(c->kin_group);
  cudaFree(c->kin_vel);
  cudaFree(c->kg_off);
  cudaFree(c->kg_ids);
  cudaFree(c->sel_bits);
  c->kin_group = nullptr;
  c->kin_vel = nullptr;
  c->kg_off = nullptr;
  c->kg_ids = nullptr;
  c->sel_bits = nullptr;
  c->dv.kin_group = nullptr;
  c->dv.kin_vel = nullptr;
  c->dv.kg_off = nullptr;
  c->dv.kg_ids = nullptr;
  c->dv.sel_bits = nullptr;
  c->dv.n_groups = 0;
  c->dv.m_kin = 0;
  int k_cap = c->k;
  if (on) {
    mpm_status st;
    if ((st = ralloc(&c->kin_group, P)) != MPM_OK) return st;
    if ((st = ralloc(&c->kin_vel, v3.size())) != MPM_OK) return st;
    if ((st = ralloc(&c->kg_off, off.size())) != MPM_OK) return st;
    if ((st = ralloc(&c->kg_ids, ids.size())) != MPM_OK) return st;
    if ((st = ralloc(&c->sel_bits, (size_t)(P + 31) / 32)) != MPM_OK) return st;
    MPM_CUDA_TRY(cudaMemcpy(c->kin_group, h.data(), sizeof(int32_t) * P, cudaMemcpyHostToDevice));
    MPM_CUDA_TRY(cudaMemcpy(c->kin_vel, v3.data(), sizeof(float) * v3.size(), cudaMemcpyHostToDevice));
    MPM_CUDA_TRY(cudaMemcpy(c->kg_off, off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice));
    if (!ids.empty())
      MPM_CUDA_TRY(cudaMemcpy(c->kg_ids, ids.data(), sizeof(int32_t) * ids.size(), cudaMemcpyHostToDevice));
    c->dv.kin_group = c->kin_group;
    c->dv.kin_vel = c->kin_vel;
    c->dv.kg_off = c->kg_off;
    c->dv.kg_ids = c->kg_ids;
    c->dv.sel_bits = c->sel_bits;
    c->dv.n_groups = n_groups;
    c->dv.m_kin = min_samples;
    k_cap = std::min(P, c->k + min_samples * n_groups);
  }
  // the basis-node list depends on the sample capacity
  if (k_cap != c->k_cap) {
    cudaFree(c->nodes);
    c->nodes = nullptr;
    c->dv.nodes = nullptr;
    mpm_status st = ralloc(&c->nodes, (size_t)k_cap * NS);
    if (st != MPM_OK) return st;
    c->dv.nodes = c->nodes;
    // the old node list is gone: start from an empty grid, as rom_set_state does
    const size_t gn = c->d == 2 ? (size_t)c->n * c->n : (size_t)c->n * c->n * c->n;
    MPM_CUDA_TRY(cudaMemset(c->counts, 0, sizeof(int32_t) * 4));
    MPM_CUDA_TRY(cudaMemset(c->grid, 0, sizeof(float4) * gn));
    MPM_CUDA_TRY(cudaMemset(c->stamp, 0, sizeof(uint32_t) * gn));
    c->k_cap = k_cap;
    // the Eulerian quadrature cells around the larger sample set
    if (c->eulerian && (st = rom_alloc_quadrature(c, k_cap)) != MPM_OK) return st;
  }
  c->reconfig_failed = false;
  return MPM_OK;
}

mpm_status rom_decode_points(rom_ctx* c, const float* X, int64_t n, float* x_out, void* stream) {
  MPM_CHECK_ARG(c && (X || n == 0) && (x_out || n == 0), "null argument");
  MPM_CHECK_ARG(n >= 0, "n >= 0");
  if (n == 0) return MPM_OK;
  int k_primal[1] = {0};
  return decoder_launch_dev(c->dec, X, nullptr, nullptr, 1, n, c->sv.xh32, nullptr, k_primal, 1, x_out,
                            (cudaStream_t)stream);
}

mpm_status rom_set_reference(rom_ctx* c, const double* xhat_ref, void* stream) {
  MPM_CHECK_ARG(c && xhat_ref, "null argument");
  MPM_CHECK_ARG(c->cfg.f_reference == 1, "rom_set_reference needs cfg.f_reference = 1");
  cudaStream_t s = (cudaStream_t)stream;
  const int d = c->d, r = c->r, P = c->P;
  std::vector<double> h(r);
  MPM_CUDA_TRY(cudaMemcpyAsync(h.data(), xhat_ref, sizeof(double) * r, cudaMemcpyDefault, s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<float> h32(h.begin(), h.end());
  MPM_CUDA_TRY(cudaMemcpyAsync(c->xref32, h32.data(), sizeof(float) * r, cudaMemcpyHostToDevice, s));
  int kr[4] = {0, 1, 2, 3};
  mpm_status st = decoder_launch_dev(c->dec, c->X, nullptr, c->nP_all, 1, P, c->xref32, nullptr, kr, d + 1, c->outQ, s);
  if (st != MPM_OK) return st;
  const int b = std::max(1, std::min(ceil_div(P, 256), c->n_sm * 4));
  if (d == 2)
    rom_reference<2><<<b, 256, 0, s>>>(c->outQ, P, P, c->Fref_inv, c->status);
  else
    rom_reference<3><<<b, 256, 0, s>>>(c->outQ, P, P, c->Fref_inv, c->status);
  MPM_CUDA_TRY(cudaGetLastError());
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  // the captured step graph holds the kernel arguments: recapture on the next step
  c->dv.Fref_inv = c->Fref_inv;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  ++c->generation;
  return MPM_OK;
}

mpm_status rom_fit_initial(rom_ctx* c, const float* target, const float* V0, int iters, void* stream) {
  MPM_CHECK_ARG(c && target && V0, "null argument");
  MPM_CHECK_ARG(iters >= 1 && iters <= 100, "iters in [1, 100]");
  cudaStream_t s = (cudaStream_t)stream;
  const int d = c->d, r = c->r, P = c->P;
  // Gauss-Newton over all particles (Eq. essentialSpecInt, first line), from xhat = 0
  float* tgt = nullptr;
  float* vel = nullptr;
  MPM_CUDA_TRY(cudaMalloc((void**)&tgt, sizeof(float) * P * d));
  MPM_CUDA_TRY(cudaMalloc((void**)&vel, sizeof(float) * P * d));
  MPM_CUDA_TRY(cudaMemcpyAsync(tgt, target, sizeof(float) * P * d, cudaMemcpyDefault, s));
  MPM_CUDA_TRY(cudaMemcpyAsync(vel, V0, sizeof(float) * P * d, cudaMemcpyDefault, s));
  MPM_CUDA_TRY(cudaMemsetAsync(c->sv.xk, 0, sizeof(double) * r, s));
  MPM_CUDA_TRY(cudaMemsetAsync(c->sv.xk32, 0, sizeof(float) * r, s));
  MPM_CUDA_TRY(cudaMemsetAsync(c->sv.dk32, 0, sizeof(float) * r, s));
  int ks[kMaxRl + 2];
  ks[0] = 0;
  for (int j = 0; j < r; ++j) ks[1 + j] = 1 + d + j;
  int kls[1 + kLS];
  kls[0] = 0;
  for (int m = 0; m < kLS; ++m) kls[1 + m] = 3000 + m;
  const int b_ne = std::max(1, std::min(ceil_div((int64_t)P * d, kNERows), c->n_sm));
  mpm_status st = MPM_OK;
  for (int it = 0; it < iters && st == MPM_OK; ++it) {
    st = decoder_launch_dev(c->dec, c->X, nullptr, c->nP_all, 1, P, c->sv.xk32, nullptr, ks, r + 1, c->outS, s);
    if (st != MPM_OK) break;
    rom_normal<<<b_ne, kNormBlock, 0, s>>>(c->dv, c->sv, c->outS, P, NE_FIT, tgt, 0, P, 0.f);
    // trials: secant from the iterate; base rows hold the iterate
    st = decoder_launch_dev(c->dec, c->X, nullptr, c->nP_all, 1, P, c->sv.ls_base32, c->sv.ls_dir32, kls, 1 + kLS,
                            c->outLS, s);
    if (st != MPM_OK) break;
    rom_linesearch<<<kLS, kNormBlock, 0, s>>>(c->dv, c->sv, c->outLS, P, NE_FIT, tgt, 0, 1e-4, P, -1);
  }
  // velocity fit at the fitted xhat_0 (Eq. essentialSpecInt, second line)
  if (st == MPM_OK) {
    st = decoder_launch_dev(c->dec, c->X, nullptr, c->nP_all, 1, P, c->sv.xk32, nullptr, ks, r + 1, c->outS, s);
  }
  if (st == MPM_OK) {
    // NE_VEL reads v_trial: stage V0 there; rows = all particles; the prior vhat is zero
    MPM_CUDA_TRY(cudaMemcpyAsync(c->v_trial, vel, sizeof(float) * P * d, cudaMemcpyDeviceToDevice, s));
    MPM_CUDA_TRY(cudaMemsetAsync(c->sv.vh, 0, sizeof(double) * r, s));
    // solve J^T J vhat = J^T V0 (projection flag 1 keeps xk: the commit below sets the state)
    MPM_CUDA_TRY(cudaMemcpyAsync(c->sv.xh, c->sv.xk, sizeof(double) * r, cudaMemcpyDeviceToDevice, s));
    rom_normal<<<b_ne, kNormBlock, 0, s>>>(c->dv, c->sv, c->outS, P, NE_VEL, nullptr, 1, P, 0.f);
  }
  cudaFree(tgt);
  cudaFree(vel);
  MPM_CUDA_TRY(cudaGetLastError());
  if (st != MPM_OK) return st;
  // xhat_0 = fitted, vhat_0 = velocity fit, xhat_{-1} = xhat_0 - dt vhat_0
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<double> xh(r), vh(r), xp(r);
  MPM_CUDA_TRY(cudaMemcpy(xh.data(), c->sv.xh, sizeof(double) * r, cudaMemcpyDeviceToHost));
  MPM_CUDA_TRY(cudaMemcpy(vh.data(), c->sv.vh_new, sizeof(double) * r, cudaMemcpyDeviceToHost));
  for (int i = 0; i < r; ++i) xp[i] = xh[i] - (double)c->cfg.dt * vh[i];
  if (c->cfg.f_reference) {
    const mpm_status sr = rom_set_reference(c, xh.data(), stream);
    if (sr != MPM_OK) return sr;
  }
  return rom_set_state(c, xh.data(), vh.data(), xp.data(), 0, stream);
}

mpm_status metric_accumulate(const float* a, const float* b, int64_t n, double* acc, void* stream) {
  MPM_CHECK_ARG(a && b && acc, "null argument");
  MPM_CHECK_ARG(n >= 0, "n >= 0");
  if (n == 0) return MPM_OK;
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)n_sm * 4));
  metric_accumulate_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(a, b, n, acc);
  MPM_CUDA_TRY(cudaGetLastError());
  return MPM_OK;
}

}  // extern "C"

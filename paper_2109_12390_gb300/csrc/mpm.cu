// Full-order explicit MPM step (Algorithm 1, Section 2.2) on sm_103a.
//
// Data layout in HBM (all owned by mpm_ctx):
//   state[2]   particle state, structure of arrays, one float stream per
//              component: x[D], v[D], F[D*D], C[D*D]  (stream c at base + c*P),
//              plus id[P] (the caller's particle index).  Two buffers: a step
//              gathers from one and writes the other in block order.
//   key[P]     grid-block key of every particle of the current buffer:
//              inst * nblk + block of floor(x/dx - 0.5).
//   perm[P]    binned order: perm[j] = index in the current buffer of the
//              j-th particle when sorted by key.
//   grid[2]    per instance a dense n^D array of float4 {m, p_x, p_y, p_z}
//              (p = m v + dt f, the momentum after the internal-force impulse).
//              grid[g] holds the particle-to-grid transfer of the current
//              state; grid[1-g] is zero except for blocks flagged in touched.
//
// One step = three kernels, captured in a CUDA graph by the caller if wanted:
//   mpm_g2p2g      per work item (<= 256 particles of one grid block): load
//                  the block's node tile of grid[g], apply the grid update of
//                  Algorithm 1 (v = p/m + dt g, walls) while loading, gather to
//                  the particles (grid-to-particle + advection), write the new
//                  state contiguously, then scatter the new state's
//                  particle-to-grid contributions into a shared-memory node
//                  tile and flush it with vector atomics into grid[1-g]
//                  (= the first half of the next step).  New keys are counted
//                  with warp-aggregated atomics.
//   mpm_scan       single-pass exclusive scan of the key counts (decoupled
//                  look-back over tiles of 1024 keys), work list.
//   mpm_permute    binned order of the new keys (warp-aggregated slot
//                  claims) and clearing of the grid that was just consumed.
// Particle state therefore moves through HBM once per step (gather-read of
// x, F; write of x, v, F, C), and the grid update costs no pass of its own.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "mpm_math.cuh"

namespace mpmrom {

constexpr int kChunk = 256;           // threads per CTA of the fused kernel
constexpr int kSlots = 2;             // particles per thread
constexpr int kItem = kSlots * kChunk; // particles per work item at most

// Dynamic shared memory of the fused kernel: per slot its P2G record (2 D + D^2 floats), its
// position in cell order, its cell and its rank within the cell.
template <int D>
constexpr int fused_dyn_smem() { return kItem * ((2 * D + D * D) * 4 + 3 * 2); }
static_assert(fused_dyn_smem<3>() <= 48 * 1024, "the fused kernel launches without raising its shared-memory limit");

template <int D> struct Blk;
template <> struct Blk<2> { static constexpr int B = 8; };
template <> struct Blk<3> { static constexpr int B = 4; };

struct DevParams {
  int P;
  int n;            // grid nodes per axis
  int nb;           // blocks per axis
  int nblk;         // blocks per instance
  int n_keys;       // n_inst * nblk
  int64_t gnodes;   // nodes per instance
  float dx, inv_dx, dt;
  float g[3];
  int bc, bc_width;
  float mass, vol;
  const float2* mu_lam;  // per instance
  float sv_lo, sv_hi;    // plastic material: bounds of the singular values of F
  const int32_t* kin_group;  // kinematic group per particle id (-1 free), or null
  const float* kin_vel;      // prescribed velocity per group (3 floats each)
};

struct StateView {
  float* base;  // component c at base + c * P
  int32_t* id;
};

template <int D>
__device__ __forceinline__ int key_of_base(const int b[D], int inst, const DevParams& p) {
  constexpr int B = Blk<D>::B;
  int k = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) k = k * p.nb + b[a] / B;
  return inst * p.nblk + k;
}

// Grid update of Algorithm 1 for one node (shared with the reduced-order step).
template <int D>
__device__ __forceinline__ void node_velocity(float4 mp, const int node[D], const DevParams& p, float v[D]) {
  grid_node_velocity<D>(mp, node, p.n, p.bc, p.bc_width, p.dt, p.g, v);
}

template <int D>
__device__ __forceinline__ int64_t grid_index(const int node[D], int inst, const DevParams& p) {
  int64_t g = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) g = g * p.n + node[a];
  return (int64_t)inst * p.gnodes + g;
}

__device__ __forceinline__ void atomic_add_node(float4* addr, float4 val) {
  atomicAdd(addr, val);  // vector red.global (sm_90+)
}

// Particle-to-grid contribution of one particle straight into the global grid (a
// particle that moved more than one cell out of its work item's block: rare).
//   MLS:  m_i += w m;  p_i += w (m v + A (x_i - x_p)),  A = m C - dt V0 (4/dx^2) tau
//   PIC:  m_i += w m;  p_i += w m v - dt V0 tau grad N_i
template <int D, int TRANSFER>
__device__ __forceinline__ void scatter_particle(const float x[D], const float v[D], const float C[D * D],
                                                 const float tau[D * D], int inst, float4* grid, uint8_t* touched,
                                                 const DevParams& p, uint32_t* status) {
  int base[D];
  float w[D][3], dw[D][3], fx[D];
  bool out_of_grid = false;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    base[a] = stencil_base(x[a], p.inv_dx);
    fx[a] = x[a] * p.inv_dx - (float)base[a];
    bspline_w(fx[a], w[a]);
    if (TRANSFER == MPM_TRANSFER_PIC) bspline_dw(fx[a], dw[a]);
    out_of_grid |= (base[a] < 0) | (base[a] + 2 > p.n - 1);
  }
  if (out_of_grid) {
    raise_status(status, STATUS_OUT_OF_GRID);
    return;
  }
  float A[D * D];
  if (TRANSFER == MPM_TRANSFER_MLS) {
    const float k = p.dt * p.vol * 4.0f * p.inv_dx * p.inv_dx;
#pragma unroll
    for (int i = 0; i < D * D; ++i) A[i] = p.mass * C[i] - k * tau[i];
  }
  const int NS = (D == 2) ? 9 : 27;
  // Stencil nodes are visited in a lane-rotated order: lanes whose particles
  // share a cell then hit different nodes in the same iteration, which keeps
  // the shared-memory atomics of a warp from serialising on one address.
  const int lane = threadIdx.x & 31;
#pragma unroll 1
  for (int s = 0; s < NS; ++s) {
    const int q = (s + lane) % NS;
    int off[D];
    if (D == 2) {
      off[0] = q / 3;
      off[1] = q - 3 * off[0];
    } else {
      off[0] = q / 9;
      off[1] = (q / 3) % 3;
      off[2] = q % 3;
    }
    float wt = 1.f;
    float wsel[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      wsel[a] = off[a] == 0 ? w[a][0] : (off[a] == 1 ? w[a][1] : w[a][2]);
      wt *= wsel[a];
    }
    float mom[D];
    if (TRANSFER == MPM_TRANSFER_MLS) {
      float dpos[D];
#pragma unroll
      for (int a = 0; a < D; ++a) dpos[a] = (float)(base[a] + off[a]) * p.dx - x[a];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        float q = p.mass * v[a];
#pragma unroll
        for (int b = 0; b < D; ++b) q = fmaf(A[a * D + b], dpos[b], q);
        mom[a] = wt * q;
      }
    } else {
      float grad[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        float gg = (off[a] == 0 ? dw[a][0] : (off[a] == 1 ? dw[a][1] : dw[a][2])) * p.inv_dx;
#pragma unroll
        for (int b = 0; b < D; ++b)
          if (b != a) gg *= wsel[b];
        grad[a] = gg;
      }
      const float k = p.dt * p.vol;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        float f = 0.f;
#pragma unroll
        for (int b = 0; b < D; ++b) f = fmaf(tau[a * D + b], grad[b], f);
        mom[a] = wt * p.mass * v[a] - k * f;
      }
    }
    int node[D];
#pragma unroll
    for (int a = 0; a < D; ++a) node[a] = base[a] + off[a];
    float4 val = make_float4(wt * p.mass, mom[0], D > 1 ? mom[1] : 0.f, D > 2 ? mom[D - 1] : 0.f);
    atomic_add_node(&grid[grid_index<D>(node, inst, p)], val);
    uint8_t* f = &touched[key_of_base<D>(node, inst, p)];
    if (*f == 0) *f = 1;
  }
}

// Flags the grid blocks named by a mask of written blocks: bit (d_0 + 1) 3^(D-1) + ... +
// (d_{D-1} + 1) for the block at offset d in {-1, 0, 1}^D from the item's block (the nodes a work
// item's particles reach lie in those), one plain store per written block.
template <int D>
__device__ __forceinline__ void flag_blocks(unsigned bits, const int b0[D], int inst, uint8_t* touched,
                                            const DevParams& p) {
  constexpr int B = Blk<D>::B;
  const int t = threadIdx.x;
  if (t < (D == 2 ? 9 : 27) && ((bits >> t) & 1u)) {
    int bb[D];
    int r = t;
#pragma unroll
    for (int a = D - 1; a >= 0; --a) {
      bb[a] = b0[a] / B + (r % 3) - 1;
      r /= 3;
    }
    int k = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) k = k * p.nb + bb[a];
    touched[(size_t)inst * p.nblk + k] = 1;
  }
}

__device__ __forceinline__ void prefetch_l2(const void* ptr) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
}

// L2 prefetch of the lines of particle s that the fused kernel's gather reads (x, F, id).
template <int D>
__device__ __forceinline__ void prefetch_state(const StateView& src, int s, int P) {
#pragma unroll
  for (int a = 0; a < D; ++a) prefetch_l2(&src.base[(size_t)a * P + s]);
#pragma unroll
  for (int i = 0; i < D * D; ++i) prefetch_l2(&src.base[(size_t)(2 * D + i) * P + s]);
  prefetch_l2(&src.id[s]);
}

// Programmatic dependent launch: the step's kernels are launched so that the next one may be
// scheduled while this one drains.  Every step kernel first waits until the previous grid has
// completed and its writes are visible (a no-op when launched without the attribute), then lets
// its own dependents be scheduled.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void count_key_aggregated(int key, int32_t* counts) {
  unsigned active = __activemask();
  unsigned peers = __match_any_sync(active, key);
  int leader = __ffs(peers) - 1;
  if ((int)(threadIdx.x & 31) == leader && key >= 0) atomicAdd(&counts[key], __popc(peers));
}

// --------------------------------------------------------------------------
// The fused step kernel.  FIRST = true runs only the particle-to-grid half
// (the transfer of a freshly loaded state).
// --------------------------------------------------------------------------
template <int D, int MATERIAL, int TRANSFER, bool FIRST, int POLAR>
__global__ void __launch_bounds__(kChunk, 3) mpm_g2p2g(DevParams p, StateView src, StateView dst,
                                                        const int32_t* __restrict__ perm,
                                                        const int4* __restrict__ work, const int32_t* n_work,
                                                        const float4* __restrict__ grid_cur, float4* grid_nxt,
                                                        uint8_t* touched_nxt, int32_t* key_out,
                                                        int32_t* counts, uint32_t* status) {
  constexpr int B = Blk<D>::B;
  constexpr int TG = B + 2;  // grid-to-particle tile: nodes [b0, b0 + B + 2)
  constexpr int TC = B + 2;  // particle-to-grid cells (stencil bases) [b0 - 1, b0 + B + 1)
  constexpr int NG = (D == 2) ? TG * TG : TG * TG * TG;
  constexpr int NC = (D == 2) ? TC * TC : TC * TC * TC;
  constexpr int DD = D * D;
  constexpr int PD = 2 * D + DD;                 // per-particle P2G record
  constexpr int NSLAB = 3;                       // tasks per cell (leading stencil offset)
  __shared__ float4 s_v4[NG];
  __shared__ int s_cnt[NC];
  __shared__ int s_off[NC + 1];
  __shared__ int s_cells[NC];
  __shared__ int s_nne;
  __shared__ unsigned s_tmask;   // grid blocks written by the item's flush
  extern __shared__ __align__(16) float s_dyn[];
  float* s_rec = s_dyn;                      // P2G records by slot
  short* s_idx = (short*)(s_rec + kItem * PD); // slots in cell order
  short* s_lc = s_idx + kItem;                 // cell of each slot (-1: none)
  short* s_rank = s_lc + kItem;                // rank of the slot within its cell

  pdl_enter();
  const int nw = *n_work;
  const int P = p.P;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tmask = 0u;
  for (int w = blockIdx.x; w < nw; w += gridDim.x) {
    const int4 item = work[w];  // {key, start, count, -}
    const int key = item.x;
    const int inst = key / p.nblk;
    int bk = key - inst * p.nblk;
    int b0[D];
#pragma unroll
    for (int a = D - 1; a >= 0; --a) {
      b0[a] = (bk % p.nb) * B;
      bk /= p.nb;
    }
    const float2 ml = p.mu_lam[inst];
    int tile_lo[D];
#pragma unroll
    for (int a = 0; a < D; ++a) tile_lo[a] = b0[a] - 1;
    // kSlots particles per thread: slots threadIdx.x + sl kChunk of the item.  The first slot's
    // gather (binned order -> state) is issued before the node tile, so that its two dependent HBM
    // latencies overlap the tile's; the other slots' lines are fetched into L2.
    int s_src = 0, pid = 0;
    float x[D], F[DD];
    if (threadIdx.x < item.z) {
      s_src = perm[item.y + threadIdx.x];
#pragma unroll
      for (int a = 0; a < D; ++a) x[a] = src.base[(size_t)a * P + s_src];
#pragma unroll
      for (int i = 0; i < DD; ++i) F[i] = src.base[(size_t)(2 * D + i) * P + s_src];
      pid = src.id[s_src];
    }
#pragma unroll
    for (int sl = 1; sl < kSlots; ++sl) {
      if (threadIdx.x + sl * kChunk < item.z)
        prefetch_state<D>(src, perm[item.y + threadIdx.x + sl * kChunk], P);
    }
    // grid-to-particle tile with the grid update of Algorithm 1 applied on load
    if (!FIRST) {
      for (int t = threadIdx.x; t < NG; t += blockDim.x) {
        int node[D];
        int r = t;
        bool inside = true;
#pragma unroll
        for (int a = D - 1; a >= 0; --a) {
          node[a] = b0[a] + r % TG;
          r /= TG;
          inside &= node[a] < p.n;
        }
        float v[3] = {0.f, 0.f, 0.f};
        if (inside) node_velocity<D>(grid_cur[grid_index<D>(node, inst, p)], node, p, v);
        s_v4[t] = make_float4(v[0], v[1], D > 2 ? v[2] : 0.f, 0.f);
      }
    }
    for (int t = threadIdx.x; t < NC; t += blockDim.x) s_cnt[t] = 0;
    __syncthreads();

    if (threadIdx.x == 0) s_tmask = 0u;   // every thread read the previous item's mask before the barrier
#pragma unroll 1
    for (int sl = 0; sl < kSlots; ++sl) {
    const int slot = threadIdx.x + sl * kChunk;
    const int j = item.y + slot;
    const bool active = slot < item.z;
    if (sl > 0 && active) {
      s_src = perm[j];
#pragma unroll
      for (int a = 0; a < D; ++a) x[a] = src.base[(size_t)a * P + s_src];
#pragma unroll
      for (int i = 0; i < DD; ++i) F[i] = src.base[(size_t)(2 * D + i) * P + s_src];
      pid = src.id[s_src];
    }
    int new_key = -1;
    int lc = -1, rank = 0;
    float rec[PD];
    if (active) {
      const int s = s_src;
      float v[D], C[DD];
      if (FIRST) {
#pragma unroll
        for (int a = 0; a < D; ++a) v[a] = src.base[(size_t)(D + a) * P + s];
#pragma unroll
        for (int i = 0; i < DD; ++i) C[i] = src.base[(size_t)(2 * D + DD + i) * P + s];
      } else {
        // grid-to-particle (Algorithm 1 step 3), separable over the stencil axes
        int rel[D];
        float w[D][3], g[D][3];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const int bse = stencil_base(x[a], p.inv_dx);
          // in range for every particle binned to this block; the clamp only
          // keeps clamped out-of-grid particles (already flagged) in bounds
          rel[a] = min(max(bse - b0[a], 0), B - 1);
          const float fx = x[a] * p.inv_dx - (float)bse;
          bspline_w(fx, w[a]);
          if (TRANSFER == MPM_TRANSFER_MLS) {
#pragma unroll
            for (int k = 0; k < 3; ++k) g[a][k] = w[a][k] * ((float)k - fx) * p.dx;  // w (x_i - x_p)
          } else {
            float dw[3];
            bspline_dw(fx, dw);
#pragma unroll
            for (int k = 0; k < 3; ++k) g[a][k] = dw[k] * p.inv_dx;  // dN/dx
          }
        }
        float Bm[DD];
#pragma unroll
        for (int a = 0; a < D; ++a) v[a] = 0.f;
#pragma unroll
        for (int i = 0; i < DD; ++i) Bm[i] = 0.f;
        if (D == 2) {
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            float S0[2] = {0.f, 0.f}, S1[2] = {0.f, 0.f};
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) {
              const float4 nv = s_v4[(rel[0] + i) * TG + rel[D - 1] + jj];
              const float wy = w[D - 1][jj], gy = g[D - 1][jj];
              S0[0] = fmaf(wy, nv.x, S0[0]);
              S0[1] = fmaf(wy, nv.y, S0[1]);
              S1[0] = fmaf(gy, nv.x, S1[0]);
              S1[1] = fmaf(gy, nv.y, S1[1]);
            }
            // value weights: x-axis w (or dw for the x-gradient), y handled above
            const float wx = w[0][i];
            const float gx = (TRANSFER == MPM_TRANSFER_MLS) ? g[0][i] : g[0][i];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
              v[a] = fmaf(wx, S0[a], v[a]);
              Bm[a * D + 0] = fmaf(gx, S0[a], Bm[a * D + 0]);
              Bm[a * D + 1] = fmaf(wx, S1[a], Bm[a * D + 1]);
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            float T0[3] = {0.f, 0.f, 0.f}, Ty[3] = {0.f, 0.f, 0.f}, Tz[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) {
              float S0[3] = {0.f, 0.f, 0.f}, S1[3] = {0.f, 0.f, 0.f};
#pragma unroll
              for (int kk = 0; kk < 3; ++kk) {
                const float4 nv = s_v4[((rel[0] + i) * TG + rel[1] + jj) * TG + rel[D - 1] + kk];
                const float wz = w[D - 1][kk], gz = g[D - 1][kk];
                S0[0] = fmaf(wz, nv.x, S0[0]);
                S0[1] = fmaf(wz, nv.y, S0[1]);
                S0[2] = fmaf(wz, nv.z, S0[2]);
                S1[0] = fmaf(gz, nv.x, S1[0]);
                S1[1] = fmaf(gz, nv.y, S1[1]);
                S1[2] = fmaf(gz, nv.z, S1[2]);
              }
              const float wy = w[1][jj], gy = g[1][jj];
#pragma unroll
              for (int a = 0; a < 3; ++a) {
                T0[a] = fmaf(wy, S0[a], T0[a]);
                Ty[a] = fmaf(gy, S0[a], Ty[a]);
                Tz[a] = fmaf(wy, S1[a], Tz[a]);
              }
            }
            const float wx = w[0][i], gx = g[0][i];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              v[a] = fmaf(wx, T0[a], v[a]);
              Bm[a * D + 0] = fmaf(gx, T0[a], Bm[a * D + 0]);
              Bm[a * D + 1] = fmaf(wx, Ty[a], Bm[a * D + 1]);
              Bm[a * D + 2] = fmaf(wx, Tz[a], Bm[a * D + 2]);
            }
          }
        }
        float G[DD];  // velocity gradient used for F
        if (TRANSFER == MPM_TRANSFER_MLS) {
          const float k = 4.0f * p.inv_dx * p.inv_dx;
#pragma unroll
          for (int i = 0; i < DD; ++i) {
            C[i] = k * Bm[i];
            G[i] = C[i];
          }
        } else {
#pragma unroll
          for (int i = 0; i < DD; ++i) {
            C[i] = 0.f;
            G[i] = Bm[i];
          }
        }
        // F <- (I + dt G) F
        float Fn[DD];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int b = 0; b < D; ++b) {
            float acc = F[a * D + b];
#pragma unroll
            for (int c = 0; c < D; ++c) acc = fmaf(p.dt * G[a * D + c], F[c * D + b], acc);
            Fn[a * D + b] = acc;
          }
#pragma unroll
        for (int i = 0; i < DD; ++i) F[i] = Fn[i];
        if (MATERIAL == MPM_FIXED_COROTATED_PLASTIC) plastic_return<D>(F, p.sv_lo, p.sv_hi);
        if (p.kin_group) {
          // kinematic (Dirichlet) particle: prescribed velocity, no affine velocity; F follows the grid
          const int kg = p.kin_group[pid];
          if (kg >= 0) {
#pragma unroll
            for (int a = 0; a < D; ++a) v[a] = p.kin_vel[3 * kg + a];
#pragma unroll
            for (int i = 0; i < DD; ++i) C[i] = 0.f;
          }
        }
#pragma unroll
        for (int a = 0; a < D; ++a) x[a] = fmaf(p.dt, v[a], x[a]);
        // write the new state contiguously (block order of the old keys)
#pragma unroll
        for (int a = 0; a < D; ++a) dst.base[(size_t)a * P + j] = x[a];
#pragma unroll
        for (int a = 0; a < D; ++a) dst.base[(size_t)(D + a) * P + j] = v[a];
#pragma unroll
        for (int i = 0; i < DD; ++i) dst.base[(size_t)(2 * D + i) * P + j] = F[i];
#pragma unroll
        for (int i = 0; i < DD; ++i) dst.base[(size_t)(2 * D + DD + i) * P + j] = C[i];
        dst.id[j] = pid;
        // health checks
        bool finite = true;
#pragma unroll
        for (int a = 0; a < D; ++a) finite &= isfinite(x[a]) && isfinite(v[a]);
#pragma unroll
        for (int i = 0; i < DD; ++i) finite &= isfinite(F[i]);
        if (!finite) raise_status(status, STATUS_NONFINITE);
        else if (det_minus_one<D>(F) <= -1.0f) raise_status(status, STATUS_INVERTED);
        // new key (clamped into the grid so that binning stays in range)
        int nbse[D];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          float xs = finite ? x[a] : 0.f;
          int b = stencil_base(xs, p.inv_dx);
          nbse[a] = min(max(b, 0), p.n - 1);
        }
        new_key = key_of_base<D>(nbse, inst, p);
        key_out[j] = new_key;
      }
      // particle-to-grid record of the (new) state
      float tau[DD];
      kirchhoff<D, MATERIAL, POLAR>(F, ml.x, ml.y, tau);
      int nb[D];
      bool out_of_grid = false, in_cells = true;
      float fx[D];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        nb[a] = stencil_base(x[a], p.inv_dx);
        fx[a] = x[a] * p.inv_dx - (float)nb[a];
        out_of_grid |= (nb[a] < 0) | (nb[a] + 2 > p.n - 1);
        const int r = nb[a] - tile_lo[a];
        in_cells &= (r >= 0) & (r < TC);
      }
      if (out_of_grid) {
        raise_status(status, STATUS_OUT_OF_GRID);
      } else if (!in_cells) {
        // moved more than one cell out of the block: scatter straight to the global grid
        scatter_particle<D, TRANSFER>(x, v, C, tau, inst, grid_nxt, touched_nxt, p, status);
      } else {
        int cidx = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) cidx = cidx * TC + (nb[a] - tile_lo[a]);
        lc = cidx;
        rank = atomicAdd(&s_cnt[lc], 1);
        // record: fractional position in cells, then (MLS) c = m v - A (x_p - x_base)
        // and A = m C - dt V0 (4/dx^2) tau, or (PIC) m v and dt V0 tau
#pragma unroll
        for (int a = 0; a < D; ++a) rec[a] = fx[a];
        if (TRANSFER == MPM_TRANSFER_MLS) {
          const float k = p.dt * p.vol * 4.0f * p.inv_dx * p.inv_dx;
          float A[DD];
#pragma unroll
          for (int i = 0; i < DD; ++i) A[i] = p.mass * C[i] - k * tau[i];
#pragma unroll
          for (int a = 0; a < D; ++a) {
            float c = p.mass * v[a];
#pragma unroll
            for (int b = 0; b < D; ++b) c = fmaf(-A[a * D + b], fx[b] * p.dx, c);
            rec[D + a] = c;
          }
#pragma unroll
          for (int i = 0; i < DD; ++i) rec[2 * D + i] = A[i];
        } else {
          const float k = p.dt * p.vol;
#pragma unroll
          for (int a = 0; a < D; ++a) rec[D + a] = p.mass * v[a];
#pragma unroll
          for (int i = 0; i < DD; ++i) rec[2 * D + i] = k * tau[i];
        }
      }
    }
    if (lc >= 0) {
      float* dstr = s_rec + (size_t)slot * PD;
#pragma unroll
      for (int i = 0; i < PD; ++i) dstr[i] = rec[i];
    }
    if (active) {
      s_lc[slot] = (short)lc;
      s_rank[slot] = (short)rank;
    }
    if (!FIRST) count_key_aggregated(new_key, counts);
    }  // slots
    __syncthreads();
    // exclusive scan of the cell counts and list of non-empty cells (warp 0)
    if (warp == 0) {
      constexpr int PER = (NC + 31) / 32;
      int cnt[PER], nz = 0, tot = 0;
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int c = lane * PER + q;
        cnt[q] = c < NC ? s_cnt[c] : 0;
        tot += cnt[q];
        nz += cnt[q] > 0;
      }
      int x0 = tot, z0 = nz;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y0 = __shfl_up_sync(0xffffffffu, x0, o), y1 = __shfl_up_sync(0xffffffffu, z0, o);
        if (lane >= o) {
          x0 += y0;
          z0 += y1;
        }
      }
      int off = x0 - tot, zoff = z0 - nz;
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int c = lane * PER + q;
        if (c < NC) {
          s_off[c] = off;
          if (cnt[q] > 0) s_cells[zoff++] = c;
        }
        off += cnt[q];
      }
      if (lane == 31) {
        s_off[NC] = off;
        s_nne = zoff;
      }
    }
    __syncthreads();
    // counting sort of the slots by cell
#pragma unroll
    for (int sl = 0; sl < kSlots; ++sl) {
      const int slot = threadIdx.x + sl * kChunk;
      if (slot < item.z) {
        const int lc = s_lc[slot];
        if (lc >= 0) s_idx[s_off[lc] + s_rank[slot]] = (short)slot;
      }
    }
    __syncthreads();
    // cell-owner accumulation: one task per (non-empty cell, leading stencil
    // offset o0) sums its cell's particles in registers over the 3 (2D) or
    // 3 x 3 (3D) stencil nodes with that offset, then adds each node's sums to
    // the global grid with one vector reduction (native in L2; shared-memory
    // float atomics are compare-and-swap loops on this GPU)
    unsigned tbits = 0u;
    const int n_tasks = s_nne * NSLAB;
    for (int task = threadIdx.x; task < n_tasks; task += blockDim.x) {
      const int cell = s_cells[task / NSLAB];
      const int o0 = task % NSLAB;
      int crel[D];
      {
        int r = cell;
#pragma unroll
        for (int a = D - 1; a >= 0; --a) {
          crel[a] = r % TC;
          r /= TC;
        }
      }
      constexpr int NROW = (D == 2) ? 1 : 3;   // rows of 3 nodes (middle-axis offset o1)
      float am[NROW][3], ap[NROW][3][D];
#pragma unroll
      for (int o1 = 0; o1 < NROW; ++o1)
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
          am[o1][kk] = 0.f;
#pragma unroll
          for (int a = 0; a < D; ++a) ap[o1][kk][a] = 0.f;
        }
      const int q1 = s_off[cell + 1];
      for (int q = s_off[cell]; q < q1; ++q) {
        const float* rr = s_rec + (size_t)s_idx[q] * PD;
        float wl[3], wlast[3], wmid[3];
        bspline_w(rr[0], wl);
        bspline_w(rr[D - 1], wlast);
        if (D == 3) bspline_w(rr[1], wmid);
        const float w0 = (o0 == 0 ? wl[0] : (o0 == 1 ? wl[1] : wl[2]));
        if (TRANSFER == MPM_TRANSFER_MLS) {
          // mom = w (c + A (o dx)) with o the node offset from the cell base
          const float* c = rr + D;
          const float* A = rr + 2 * D;
          float c0[D];
#pragma unroll
          for (int a = 0; a < D; ++a) c0[a] = fmaf(A[a * D + 0], (float)o0 * p.dx, c[a]);
#pragma unroll
          for (int o1 = 0; o1 < NROW; ++o1) {
            const float w01 = (D == 3) ? w0 * wmid[o1] : w0;
            float c1[D];
#pragma unroll
            for (int a = 0; a < D; ++a) c1[a] = (D == 3) ? fmaf(A[a * D + 1], (float)o1 * p.dx, c0[a]) : c0[a];
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
              const float wt = w01 * wlast[kk];
              am[o1][kk] = fmaf(wt, p.mass, am[o1][kk]);
#pragma unroll
              for (int a = 0; a < D; ++a)
                ap[o1][kk][a] = fmaf(wt, fmaf(A[a * D + D - 1], (float)kk * p.dx, c1[a]), ap[o1][kk][a]);
            }
          }
        } else {
          float dwl[3], dwlast[3], dwmid[3];
          bspline_dw(rr[0], dwl);
          bspline_dw(rr[D - 1], dwlast);
          if (D == 3) bspline_dw(rr[1], dwmid);
          const float* mv = rr + D;
          const float* kt = rr + 2 * D;
          const float dw0 = (o0 == 0 ? dwl[0] : (o0 == 1 ? dwl[1] : dwl[2]));
#pragma unroll
          for (int o1 = 0; o1 < NROW; ++o1) {
            const float wm1 = (D == 3) ? wmid[o1] : 1.f;
            const float dwm1 = (D == 3) ? dwmid[o1] : 0.f;
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
              const float wt = w0 * wm1 * wlast[kk];
              float grad[3];
              grad[0] = dw0 * p.inv_dx * wm1 * wlast[kk];
              if (D == 3) grad[1] = w0 * dwm1 * p.inv_dx * wlast[kk];
              grad[D - 1] = w0 * wm1 * dwlast[kk] * p.inv_dx;
              am[o1][kk] = fmaf(wt, p.mass, am[o1][kk]);
#pragma unroll
              for (int a = 0; a < D; ++a) {
                float f = 0.f;
#pragma unroll
                for (int b = 0; b < D; ++b) f = fmaf(kt[a * D + b], grad[b], f);
                ap[o1][kk][a] += wt * mv[a] - f;
              }
            }
          }
        }
      }
      // add the task's nodes to the grid: node = cell + offset (cells start at b0 - 1)
#pragma unroll
      for (int o1 = 0; o1 < NROW; ++o1)
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
          if (am[o1][kk] == 0.f) continue;
          int node[D];
          node[0] = tile_lo[0] + crel[0] + o0;
          if (D == 3) node[1] = tile_lo[1] + crel[1] + o1;
          node[D - 1] = tile_lo[D - 1] + crel[D - 1] + kk;
          atomic_add_node(&grid_nxt[grid_index<D>(node, inst, p)],
                          make_float4(am[o1][kk], ap[o1][kk][0], D > 1 ? ap[o1][kk][1] : 0.f,
                                      D > 2 ? ap[o1][kk][D - 1] : 0.f));
          int bit = 0;
#pragma unroll
          for (int a = 0; a < D; ++a) bit = bit * 3 + (node[a] / B - b0[a] / B + 1);
          tbits |= 1u << bit;
        }
    }
    tbits = __reduce_or_sync(0xffffffffu, tbits);
    if (lane == 0 && tbits) atomicOr(&s_tmask, tbits);
    __syncthreads();
    flag_blocks<D>(s_tmask, b0, inst, touched_nxt, p);
  }
}

// Exclusive scan of the key counts and work list: single pass over tiles of
// 1024 keys with decoupled look-back (Merrill and Garland 2016).  Each CTA
// publishes its tile aggregate, then its inclusive prefix, in one 64-bit word
// per tile: bits 0-31 particle count, bits 32-61 work items, bits 62-63 flag
// (1 = aggregate, 2 = inclusive prefix).  Predecessor polls are bounded; on
// timeout the CTA raises TIMEOUT and treats the missing prefix as zero.
// Work item = {key, start, count, 0}.  Counts and cursors are zeroed.
constexpr int kScanTile = 1024;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__global__ void __launch_bounds__(kScanTile) mpm_scan(int n_keys, int P, int32_t* counts, int32_t* offsets,
                                                       int32_t* cursor, int4* work, int32_t* n_work, int max_work,
                                                       unsigned long long* tile_state, uint32_t* status) {
  __shared__ int s_a[32], s_b[32];
  __shared__ long long s_prefix[2];
  pdl_enter();
  const int tile = blockIdx.x;
  const int k = tile * kScanTile + threadIdx.x;
  const int c = k < n_keys ? counts[k] : 0;
  const int nw = (c + kItem - 1) / kItem;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int a = c, b = nw;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int ya = __shfl_up_sync(0xffffffffu, a, o), yb = __shfl_up_sync(0xffffffffu, b, o);
    if (lane >= o) {
      a += ya;
      b += yb;
    }
  }
  if (lane == 31) {
    s_a[warp] = a;
    s_b[warp] = b;
  }
  __syncthreads();
  if (warp == 0) {
    int sa = s_a[lane], sb = s_b[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int ya = __shfl_up_sync(0xffffffffu, sa, o), yb = __shfl_up_sync(0xffffffffu, sb, o);
      if (lane >= o) {
        sa += ya;
        sb += yb;
      }
    }
    s_a[lane] = sa;
    s_b[lane] = sb;
    // publish this tile's aggregate, then look back 32 predecessors at a time
    const unsigned long long agg = (unsigned long long)(uint32_t)__shfl_sync(0xffffffffu, sa, 31) |
                                   ((unsigned long long)(uint32_t)__shfl_sync(0xffffffffu, sb, 31) << 32);
    const int tot_a = __shfl_sync(0xffffffffu, sa, 31), tot_b = __shfl_sync(0xffffffffu, sb, 31);
    if (lane == 0) st_release_u64(&tile_state[tile], agg | (1ull << 62));
    long long pa = 0, pb = 0;
    int q_hi = tile - 1;  // window [q_hi - 31, q_hi], lane i reads q_hi - i
    bool done = q_hi < 0;
    while (!done) {
      const int q = q_hi - lane;
      unsigned long long v = 0;
      if (q >= 0) {
        uint32_t tries = 0;
        do {
          v = ld_acquire_u64(&tile_state[q]);
        } while ((v >> 62) == 0 && ++tries < (1u << 24));
        if ((v >> 62) == 0) raise_status(status, STATUS_TIMEOUT);
      }
      // the nearest inclusive prefix in the window ends the look-back
      const unsigned incl = __ballot_sync(0xffffffffu, q >= 0 && (v >> 62) == 2);
      const int stop = incl ? (__ffs(incl) - 1) : 31;
      long long ca = (q >= 0 && lane <= stop) ? (long long)(v & 0xffffffffull) : 0;
      long long cb = (q >= 0 && lane <= stop) ? (long long)((v >> 32) & 0x3fffffffull) : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ca += __shfl_down_sync(0xffffffffu, ca, o);
        cb += __shfl_down_sync(0xffffffffu, cb, o);
      }
      pa += __shfl_sync(0xffffffffu, ca, 0);
      pb += __shfl_sync(0xffffffffu, cb, 0);
      done = incl != 0 || q_hi - 31 < 0;
      q_hi -= 32;
    }
    if (lane == 0) {
      const unsigned long long inc = (unsigned long long)(uint32_t)(pa + tot_a) |
                                     ((unsigned long long)(uint32_t)(pb + tot_b) << 32);
      st_release_u64(&tile_state[tile], inc | (2ull << 62));
      s_prefix[0] = pa;
      s_prefix[1] = pb;
    }
  }
  __syncthreads();
  const int off = (int)s_prefix[0] + a - c + (warp > 0 ? s_a[warp - 1] : 0);
  int woff = (int)s_prefix[1] + b - nw + (warp > 0 ? s_b[warp - 1] : 0);
  if (k < n_keys) {
    offsets[k] = off;
    for (int q = 0; q < nw; ++q) {
      // nw items of near-equal size (at most kItem particles each)
      const int lo = (int)((long long)q * c / nw), hi = (int)((long long)(q + 1) * c / nw);
      if (woff < max_work) work[woff] = make_int4(k, off + lo, hi - lo, 0);
      ++woff;
    }
    counts[k] = 0;
    cursor[k] = 0;
  }
  if (tile == gridDim.x - 1 && threadIdx.x == kScanTile - 1) {
    const int total = (int)s_prefix[0] + s_a[31];
    const int wtotal = (int)s_prefix[1] + s_b[31];
    offsets[n_keys] = total;
    *n_work = min(wtotal, max_work);
    if (wtotal > max_work || total != P) raise_status(status, STATUS_CAPACITY);
  }
}

// Binned order of the keys (warp-aggregated slot claims; the order inside a
// block is not specified) and clearing of the consumed grid.
template <int D>
__global__ void mpm_permute(DevParams p, const int32_t* __restrict__ key, const int32_t* __restrict__ offsets,
                            int32_t* cursor, int32_t* perm, float4* grid_clear, uint8_t* touched_clear,
                            unsigned long long* tile_state, int n_tiles) {
  constexpr int B = Blk<D>::B;
  constexpr int BN = (D == 2) ? B * B : B * B * B;
  const int stride = gridDim.x * blockDim.x;
  pdl_enter();
  // the scan that produced `offsets` has finished: reset its look-back words
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_tiles; q += stride) tile_state[q] = 0ull;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i - (int)threadIdx.x < p.P; i += stride) {
    int k = i < p.P ? key[i] : -1;
    unsigned peers = __match_any_sync(0xffffffffu, k);
    int leader = __ffs(peers) - 1;
    int lane = threadIdx.x & 31;
    int basev = 0;
    if (lane == leader && k >= 0) basev = atomicAdd(&cursor[k], __popc(peers));
    basev = __shfl_sync(0xffffffffu, basev, leader);
    if (k >= 0) {
      int rank = __popc(peers & ((1u << lane) - 1u));
      perm[offsets[k] + basev + rank] = i;
    }
  }
  // clear flagged blocks of the consumed grid
  if (grid_clear == nullptr) return;
  const int warps_total = stride / 32;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  for (int k = gw; k < p.n_keys; k += warps_total) {
    if (!touched_clear[k]) continue;
    const int inst = k / p.nblk;
    int bk = k - inst * p.nblk;
    int b0[D];
#pragma unroll
    for (int a = D - 1; a >= 0; --a) {
      b0[a] = (bk % p.nb) * B;
      bk /= p.nb;
    }
    for (int t = lane; t < BN; t += 32) {
      int node[D];
      int r = t;
#pragma unroll
      for (int a = D - 1; a >= 0; --a) {
        node[a] = b0[a] + r % B;
        r /= B;
      }
      grid_clear[grid_index<D>(node, inst, p)] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
    if (lane == 0) touched_clear[k] = 0;
  }
}

// Caller layout (AoS rows) -> internal SoA, keys and counts.
template <int D>
__global__ void mpm_load(DevParams p, const float* __restrict__ x, const float* __restrict__ v,
                         const float* __restrict__ F, const float* __restrict__ C, StateView dst,
                         const int64_t* __restrict__ inst_offsets, int n_inst, int32_t* key, int32_t* counts,
                         int zero_C, uint32_t* status) {
  constexpr int DD = D * D;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i - (int)threadIdx.x < p.P; i += gridDim.x * blockDim.x) {
    int k = -1;
    if (i < p.P) {
      // instance of particle i (n_inst is small; linear search over offsets)
      int inst = 0;
      while (inst + 1 < n_inst && inst_offsets[inst + 1] <= i) ++inst;
      int b[D];
      bool ok = true;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        float xa = x[(size_t)i * D + a];
        dst.base[(size_t)a * p.P + i] = xa;
        dst.base[(size_t)(D + a) * p.P + i] = v[(size_t)i * D + a];
        ok &= isfinite(xa);
        int bb = stencil_base(ok ? xa : 0.f, p.inv_dx);
        if (bb < 0 || bb + 2 > p.n - 1) raise_status(status, STATUS_OUT_OF_GRID);
        b[a] = min(max(bb, 0), p.n - 1);
      }
      if (!ok) raise_status(status, STATUS_NONFINITE);
#pragma unroll
      for (int q = 0; q < DD; ++q) {
        dst.base[(size_t)(2 * D + q) * p.P + i] = F[(size_t)i * DD + q];
        dst.base[(size_t)(2 * D + DD + q) * p.P + i] = (zero_C || C == nullptr) ? 0.f : C[(size_t)i * DD + q];
      }
      dst.id[i] = i;
      k = key_of_base<D>(b, inst, p);
      key[i] = k;
    }
    count_key_aggregated(k, counts);
  }
}

// Internal SoA -> caller layout in the caller's particle order.
template <int D>
__global__ void mpm_store(DevParams p, StateView src, float* x, float* v, float* F, float* C) {
  constexpr int DD = D * D;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.P; i += gridDim.x * blockDim.x) {
    int q = src.id[i];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      if (x) x[(size_t)q * D + a] = src.base[(size_t)a * p.P + i];
      if (v) v[(size_t)q * D + a] = src.base[(size_t)(D + a) * p.P + i];
    }
#pragma unroll
    for (int r = 0; r < DD; ++r) {
      if (F) F[(size_t)q * DD + r] = src.base[(size_t)(2 * D + r) * p.P + i];
      if (C) C[(size_t)q * DD + r] = src.base[(size_t)(2 * D + DD + r) * p.P + i];
    }
  }
}

// Binned position of every particle id (the inverse of src.id), for writes in the caller's order.
__global__ void mpm_inverse_ids(int P, const int32_t* __restrict__ id, int32_t* inv) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) inv[id[i]] = i;
}

// Internal SoA -> one caller array of rows (P, ncomp) holding components comp0 .. comp0 + ncomp - 1,
// in the caller's particle order: each thread writes four consecutive floats of the flattened
// array (one 16-byte store when `out` is 16-byte aligned), so that a warp's stores are 512
// contiguous bytes: the form in which writes to host memory over the chip-to-chip link are whole
// lines.
__global__ void mpm_store_rows(int P, StateView src, const int32_t* __restrict__ inv, float* out, int comp0,
                               int ncomp) {
  const int64_t total = (int64_t)P * ncomp;
  const bool vec = ((uintptr_t)out & 15u) == 0;
  for (int64_t e0 = 4 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); e0 < total;
       e0 += 4 * (int64_t)gridDim.x * blockDim.x) {
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t e = e0 + k;
      v[k] = 0.f;
      if (e < total) {
        const int q = (int)(e / ncomp), c = (int)(e % ncomp);
        v[k] = src.base[(size_t)(comp0 + c) * P + inv[q]];
      }
    }
    if (vec && e0 + 3 < total) {
      *reinterpret_cast<float4*>(out + e0) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (e0 + k < total) out[e0 + k] = v[k];
    }
  }
}

template <int D>
__global__ void mpm_bins(DevParams p, StateView src, const int32_t* key, int32_t* cell_keys, int32_t* block_keys) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.P; i += gridDim.x * blockDim.x) {
    int q = src.id[i];
    int c = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) c = c * p.n + stencil_base(src.base[(size_t)a * p.P + i], p.inv_dx);
    cell_keys[q] = c;
    block_keys[q] = key[i];
  }
}

template <int D>
__global__ void mpm_grid_dump(DevParams p, int n_inst, const float4* grid, float* mass, float* mom, float* vel) {
  const int64_t total = (int64_t)n_inst * p.gnodes;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    float4 mp = grid[g];
    int64_t r = g % p.gnodes;
    int node[D];
#pragma unroll
    for (int a = D - 1; a >= 0; --a) {
      node[a] = (int)(r % p.n);
      r /= p.n;
    }
    if (mass) mass[g] = mp.x;
    float comp[3] = {mp.y, mp.z, mp.w};
    if (mom)
#pragma unroll
      for (int a = 0; a < D; ++a) mom[g * D + a] = comp[a];
    if (vel) {
      float v[D];
      node_velocity<D>(mp, node, p, v);
#pragma unroll
      for (int a = 0; a < D; ++a) vel[g * D + a] = v[a];
    }
  }
}

}  // namespace mpmrom

// ============================================================================
// Host runtime and C ABI
// ============================================================================
using namespace mpmrom;

struct mpm_ctx {
  int D = 0, n = 0, B = 0, nb = 0, nblk = 0, n_keys = 0, P = 0, n_inst = 0;
  int material = 0, transfer = 0, polar_eft = 0;
  int64_t gnodes = 0;
  mpm_config cfg{};
  std::vector<float> E, nu;
  std::vector<int64_t> offs;
  int n_sm = 0, fused_grid = 0, max_work = 0;
  // device
  float* state[2] = {nullptr, nullptr};
  int32_t* id[2] = {nullptr, nullptr};
  int32_t *key = nullptr, *perm = nullptr, *counts = nullptr, *offsets = nullptr, *cursor = nullptr;
  int4* work = nullptr;
  int32_t* n_work = nullptr;
  unsigned long long* tile_state = nullptr;
  int n_scan_tiles = 0;
  float4* grid[2] = {nullptr, nullptr};
  uint8_t* touched[2] = {nullptr, nullptr};
  float2* mu_lam = nullptr;
  int64_t* d_offs = nullptr;
  uint32_t* status = nullptr;
  float* staging = nullptr;  // AoS x, v, F, C
  int32_t* inv_id = nullptr; // binned position of every particle id (get_state)
  int32_t* kin_group = nullptr;  // kinematic group per particle (caller's order = particle id)
  float* kin_vel = nullptr;      // prescribed velocity per group (3 floats each)
  int cur = 0, g = 0;
  bool loaded = false;
  DevParams dp{};
};

namespace {

template <typename T>
mpm_status dalloc(T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return set_error(MPM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  return MPM_OK;
}

#define MPM_TRY(expr)            \
  do {                           \
    mpm_status _s = (expr);      \
    if (_s != MPM_OK) return _s; \
  } while (0)

// Launches a step kernel with programmatic stream serialization (see pdl_enter).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, (KArgs)args...);
}

template <int D, int MAT, int TR, bool FIRST, int POLAR>
mpm_status launch_fused_t(mpm_ctx* c, cudaStream_t s) {
  StateView src{c->state[c->cur], c->id[c->cur]};
  StateView dst{c->state[1 - c->cur], c->id[1 - c->cur]};
  float4* gcur = c->grid[c->g];
  float4* gnxt = FIRST ? c->grid[c->g] : c->grid[1 - c->g];
  uint8_t* tn = FIRST ? c->touched[c->g] : c->touched[1 - c->g];
  MPM_CUDA_TRY(launch_pdl(mpm_g2p2g<D, MAT, TR, FIRST, POLAR>, c->fused_grid, kChunk, fused_dyn_smem<D>(), s, c->dp,
                          src, dst,
                          (const int32_t*)c->perm, (const int4*)c->work, (const int32_t*)c->n_work,
                          (const float4*)gcur, gnxt, tn, c->key, c->counts, c->status));
  return MPM_OK;
}

template <bool FIRST>
mpm_status launch_fused(mpm_ctx* c, cudaStream_t s) {
  const int D = c->D, M = c->material, T = c->transfer;
  // the polar variant matters for the 3D fixed-corotated material only
#define CASE(d, m, t)                                                                       \
  if (D == d && M == m && T == t) return launch_fused_t<d, m, t, FIRST, POLAR_EFT>(c, s);
  CASE(2, 0, 0) CASE(2, 0, 1) CASE(2, 1, 0) CASE(2, 1, 1) CASE(2, 2, 0) CASE(2, 2, 1)
  CASE(3, 0, 0) CASE(3, 0, 1)
#undef CASE
#define CASE3(m, t)                                                                                              \
  if (D == 3 && M == m && T == t)                                                                               \
    return c->polar_eft ? launch_fused_t<3, m, t, FIRST, POLAR_EFT>(c, s) : launch_fused_t<3, m, t, FIRST, POLAR_FP64>(c, s);
  CASE3(1, 0) CASE3(1, 1) CASE3(2, 0) CASE3(2, 1)
#undef CASE3
  return set_error(MPM_EINVAL, "unsupported (dim, material, transfer)");
}

mpm_status launch_scan_permute(mpm_ctx* c, cudaStream_t s, bool clear_consumed) {
  MPM_CUDA_TRY(launch_pdl(mpm_scan, c->n_scan_tiles, kScanTile, 0, s, c->n_keys, c->P, c->counts, c->offsets, c->cursor,
                          c->work, c->n_work, c->max_work, c->tile_state, c->status));
  int blocks = std::max(1, std::min(ceil_div(c->P, 256), c->n_sm * 8));
  float4* gclr = clear_consumed ? c->grid[c->g] : nullptr;
  uint8_t* tclr = clear_consumed ? c->touched[c->g] : nullptr;
  if (c->D == 2)
    MPM_CUDA_TRY(launch_pdl(mpm_permute<2>, blocks, 256, 0, s, c->dp, (const int32_t*)c->key,
                            (const int32_t*)c->offsets, c->cursor, c->perm, gclr, tclr, c->tile_state,
                            c->n_scan_tiles));
  else
    MPM_CUDA_TRY(launch_pdl(mpm_permute<3>, blocks, 256, 0, s, c->dp, (const int32_t*)c->key,
                            (const int32_t*)c->offsets, c->cursor, c->perm, gclr, tclr, c->tile_state,
                            c->n_scan_tiles));
  return MPM_OK;
}

}  // namespace

// ----------------------------------------------------------------------------
// Fixed scratch of mpm_step_noalloc.  Every GPU that loads the library holds
// this array until the process exits; the entry point carves its work
// buffers out of it instead of calling cudaMalloc.
// ----------------------------------------------------------------------------
constexpr size_t kNoAllocBytes = size_t(8) << 20;  // 8 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

constexpr int kNoAllocMaxDevices = 64;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// Device address of the scratch array for the current device.  The host-side
// symbol is only a stand-in, so the address comes from cudaGetSymbolAddress,
// looked up once per device with that device current.
mpm_status noalloc_scratch(void** out) {
  int dev = 0;
  MPM_CUDA_TRY(cudaGetDevice(&dev));
  MPM_CHECK_ARG(dev >= 0 && dev < kNoAllocMaxDevices, "device index out of range for the fixed scratch table");
  if (g_noalloc_ptr[dev] == nullptr) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr)
      return set_error(MPM_ECUDA, std::string("cudaGetSymbolAddress(fixed scratch): ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return MPM_OK;
}

struct Carve {
  char* base;
  size_t used, cap;
  template <typename T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + std::max<size_t>(count, 1) * sizeof(T);
    return used <= cap ? reinterpret_cast<T*>(base + off) : nullptr;
  }
};

}  // namespace

extern "C" {

mpm_status mpm_init(const mpm_config* cfg, mpm_ctx** out) {
  MPM_CHECK_ARG(cfg && out, "null argument");
  *out = nullptr;
  MPM_CHECK_ARG(cfg->dim == 2 || cfg->dim == 3, "dim must be 2 or 3");
  const int B = cfg->dim == 2 ? Blk<2>::B : Blk<3>::B;
  MPM_CHECK_ARG(cfg->n_grid >= 8 && cfg->n_grid % B == 0, "n_grid must be a multiple of 8 (2D) / 4 (3D)");
  MPM_CHECK_ARG(cfg->n_inst >= 1 && cfg->E && cfg->nu && cfg->inst_offsets, "instances");
  MPM_CHECK_ARG(cfg->dx > 0 && cfg->dt > 0 && cfg->rho > 0 && cfg->p_vol > 0, "dx, dt, rho, p_vol must be > 0");
  MPM_CHECK_ARG(cfg->material == MPM_NEO_HOOKEAN || cfg->material == MPM_FIXED_COROTATED ||
                    cfg->material == MPM_FIXED_COROTATED_PLASTIC,
                "material");
  MPM_CHECK_ARG(cfg->material != MPM_FIXED_COROTATED_PLASTIC ||
                    (cfg->plastic_compression >= 0.f && cfg->plastic_compression < 1.f && cfg->plastic_stretch >= 0.f),
                "plastic bounds: 0 <= plastic_compression < 1, plastic_stretch >= 0");
  MPM_CHECK_ARG(cfg->transfer == MPM_TRANSFER_MLS || cfg->transfer == MPM_TRANSFER_PIC, "transfer");
  MPM_CHECK_ARG(cfg->bc == MPM_BC_STICKY || cfg->bc == MPM_BC_SLIP_FLOOR, "bc");
  MPM_CHECK_ARG(cfg->polar_eft == 0 || cfg->polar_eft == 1, "polar_eft: 0 or 1");
  MPM_CHECK_ARG(cfg->bc_width >= 0, "bc_width");
  MPM_CHECK_ARG(cfg->inst_offsets[0] == 0, "inst_offsets[0] must be 0");
  for (int k = 0; k < cfg->n_inst; ++k)
    MPM_CHECK_ARG(cfg->inst_offsets[k + 1] >= cfg->inst_offsets[k], "inst_offsets must be non-decreasing");
  const int64_t P64 = cfg->inst_offsets[cfg->n_inst];
  MPM_CHECK_ARG(P64 >= 1 && P64 < (1ll << 30), "particle count out of range");
  for (int k = 0; k < cfg->n_inst; ++k)
    MPM_CHECK_ARG(cfg->E[k] > 0 && cfg->nu[k] > -1 && cfg->nu[k] < 0.5f, "E must be > 0 and -1 < nu < 0.5");
  auto* c = new mpm_ctx();
  c->cfg = *cfg;
  c->D = cfg->dim;
  c->n = cfg->n_grid;
  c->B = B;
  c->nb = c->n / B;
  c->nblk = c->D == 2 ? c->nb * c->nb : c->nb * c->nb * c->nb;
  c->n_inst = cfg->n_inst;
  const int64_t nk = (int64_t)c->n_inst * c->nblk;
  if (nk >= (1ll << 30)) {
    delete c;
    return set_error(MPM_EINVAL, "too many grid blocks");
  }
  c->n_keys = (int)nk;
  c->P = (int)P64;
  c->material = cfg->material;
  c->transfer = cfg->transfer;
  c->polar_eft = cfg->polar_eft;
  c->gnodes = c->D == 2 ? (int64_t)c->n * c->n : (int64_t)c->n * c->n * c->n;
  c->E.assign(cfg->E, cfg->E + c->n_inst);
  c->nu.assign(cfg->nu, cfg->nu + c->n_inst);
  c->offs.assign(cfg->inst_offsets, cfg->inst_offsets + c->n_inst + 1);
  c->cfg.E = nullptr;
  c->cfg.nu = nullptr;
  c->cfg.inst_offsets = nullptr;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, dev);
  c->max_work = ceil_div(c->P, kItem) + std::min(c->n_keys, c->P) + 1;

  const int D = c->D, DD = D * D;
  const size_t comps = 2 * D + 2 * DD;
  mpm_status st = MPM_OK;
  auto fail = [&](mpm_status s) {
    mpm_destroy(c);
    return s;
  };
  for (int b = 0; b < 2; ++b) {
    if ((st = dalloc(&c->state[b], comps * c->P)) != MPM_OK) return fail(st);
    if ((st = dalloc(&c->id[b], c->P)) != MPM_OK) return fail(st);
    if ((st = dalloc(&c->grid[b], (size_t)c->n_inst * c->gnodes)) != MPM_OK) return fail(st);
    if ((st = dalloc(&c->touched[b], c->n_keys)) != MPM_OK) return fail(st);
  }
  if ((st = dalloc(&c->key, c->P)) != MPM_OK) return fail(st);
  if ((st = dalloc(&c->perm, c->P)) != MPM_OK) return fail(st);
  if ((st = dalloc(&c->counts, c->n_keys)) != MPM_OK) return fail(st);
  if ((st = dalloc(&c->cursor, c->n_keys)) != MPM_OK) return fail(st);
  if ((st = dalloc(&c->offsets, c->n_keys + 1)) != MPM_OK) return fail(st);
  if ((st = dalloc(&c->work, c->max_work)) != MPM_OK) return fail(st);
  if ((st = dalloc(&c->n_work, 1)) != MPM_OK) return fail(st);
  c->n_scan_tiles = ceil_div(c->n_keys, kScanTile);
  if ((st = dalloc(&c->tile_state, c->n_scan_tiles)) != MPM_OK) return fail(st);
  if ((st = dalloc(&c->mu_lam, c->n_inst)) != MPM_OK) return fail(st);
  if ((st = dalloc(&c->d_offs, c->n_inst + 1)) != MPM_OK) return fail(st);
  if ((st = dalloc(&c->status, 1)) != MPM_OK) return fail(st);
  if ((st = dalloc(&c->staging, comps * c->P)) != MPM_OK) return fail(st);
  if ((st = dalloc(&c->inv_id, c->P)) != MPM_OK) return fail(st);
  std::vector<float2> ml(c->n_inst);
  for (int k = 0; k < c->n_inst; ++k) {
    double E = c->E[k], nu = c->nu[k];
    ml[k] = make_float2((float)(E / (2 * (1 + nu))), (float)(E * nu / ((1 + nu) * (1 - 2 * nu))));
  }
  cudaError_t e = cudaSuccess;
  e = cudaMemcpy(c->mu_lam, ml.data(), sizeof(float2) * c->n_inst, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_offs, c->offs.data(), sizeof(int64_t) * (c->n_inst + 1), cudaMemcpyHostToDevice);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMemset(c->grid[b], 0, sizeof(float4) * (size_t)c->n_inst * c->gnodes);
    if (e == cudaSuccess) e = cudaMemset(c->touched[b], 0, c->n_keys);
  }
  if (e == cudaSuccess) e = cudaMemset(c->counts, 0, sizeof(int32_t) * c->n_keys);
  if (e == cudaSuccess) e = cudaMemset(c->cursor, 0, sizeof(int32_t) * c->n_keys);
  if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(c->n_work, 0, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(c->tile_state, 0, sizeof(unsigned long long) * c->n_scan_tiles);
  if (e != cudaSuccess) return fail(set_error(MPM_ECUDA, std::string("init: ") + cudaGetErrorString(e)));

  DevParams& p = c->dp;
  p.P = c->P;
  p.n = c->n;
  p.nb = c->nb;
  p.nblk = c->nblk;
  p.n_keys = c->n_keys;
  p.gnodes = c->gnodes;
  p.dx = cfg->dx;
  p.inv_dx = (float)(1.0 / cfg->dx);
  p.dt = cfg->dt;
  for (int a = 0; a < 3; ++a) p.g[a] = cfg->gravity[a];
  p.bc = cfg->bc;
  p.bc_width = cfg->bc_width;
  p.mass = cfg->rho * cfg->p_vol;
  p.vol = cfg->p_vol;
  p.mu_lam = c->mu_lam;
  p.sv_lo = 1.f - cfg->plastic_compression;
  p.sv_hi = 1.f + cfg->plastic_stretch;
  c->fused_grid = std::max(1, std::min(c->max_work, c->n_sm * 8));
  *out = c;
  return MPM_OK;
}

void mpm_destroy(mpm_ctx* c) {
  if (!c) return;
  for (int b = 0; b < 2; ++b) {
    cudaFree(c->state[b]);
    cudaFree(c->id[b]);
    cudaFree(c->grid[b]);
    cudaFree(c->touched[b]);
  }
  cudaFree(c->key);
  cudaFree(c->perm);
  cudaFree(c->counts);
  cudaFree(c->cursor);
  cudaFree(c->offsets);
  cudaFree(c->work);
  cudaFree(c->n_work);
  cudaFree(c->tile_state);
  cudaFree(c->mu_lam);
  cudaFree(c->d_offs);
  cudaFree(c->status);
  cudaFree(c->staging);
  cudaFree(c->inv_id);
  cudaFree(c->kin_group);
  cudaFree(c->kin_vel);
  delete c;
}

mpm_status mpm_set_kinematic(mpm_ctx* c, const int32_t* group, int32_t n_groups, const float* velocities,
                             void* stream) {
  MPM_CHECK_ARG(c, "null context");
  MPM_CHECK_ARG(n_groups >= 0, "n_groups >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  if (n_groups == 0 || !group) {
    c->dp.kin_group = nullptr;
    c->dp.kin_vel = nullptr;
    return MPM_OK;
  }
  MPM_CHECK_ARG(velocities, "velocities of the kinematic groups");
  std::vector<int32_t> h((size_t)c->P);
  std::vector<float> hv((size_t)n_groups * c->D);
  MPM_CUDA_TRY(cudaMemcpyAsync(h.data(), group, sizeof(int32_t) * c->P, cudaMemcpyDefault, s));
  MPM_CUDA_TRY(cudaMemcpyAsync(hv.data(), velocities, sizeof(float) * hv.size(), cudaMemcpyDefault, s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  for (int i = 0; i < c->P; ++i) MPM_CHECK_ARG(h[i] >= -1 && h[i] < n_groups, "group ids in [-1, n_groups)");
  std::vector<float> v3((size_t)n_groups * 3, 0.f);
  for (int g = 0; g < n_groups; ++g)
    for (int a = 0; a < c->D; ++a) v3[(size_t)3 * g + a] = hv[(size_t)c->D * g + a];
  cudaFree(c->kin_group);
  cudaFree(c->kin_vel);
  c->kin_group = nullptr;
  c->kin_vel = nullptr;
  c->dp.kin_group = nullptr;
  c->dp.kin_vel = nullptr;
  MPM_CUDA_TRY(cudaMalloc((void**)&c->kin_group, sizeof(int32_t) * c->P));
  MPM_CUDA_TRY(cudaMalloc((void**)&c->kin_vel, sizeof(float) * v3.size()));
  MPM_CUDA_TRY(cudaMemcpy(c->kin_group, h.data(), sizeof(int32_t) * c->P, cudaMemcpyHostToDevice));
  MPM_CUDA_TRY(cudaMemcpy(c->kin_vel, v3.data(), sizeof(float) * v3.size(), cudaMemcpyHostToDevice));
  c->dp.kin_group = c->kin_group;
  c->dp.kin_vel = c->kin_vel;
  return MPM_OK;
}

// A pointer through which kernels may access `p` directly: device or managed memory, or page-locked
// host memory mapped into the device's address space (read over the host link by the kernel
// itself); nullptr for pageable host memory, which is staged by a copy.
static const void* device_view(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return p;
  if (at.type == cudaMemoryTypeHost && at.devicePointer) {
    // the mapping covers the allocation: offset of p within it
    return (const uint8_t*)at.devicePointer + ((const uint8_t*)p - (const uint8_t*)at.hostPointer);
  }
  return nullptr;
}

mpm_status mpm_set_state(mpm_ctx* c, const float* x, const float* v, const float* F, const float* C, void* stream) {
  MPM_CHECK_ARG(c && x && v && F, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int D = c->D, DD = D * D;
  const size_t P = c->P;
  // device-accessible inputs are read by the load kernel directly; the others are staged
  const float* sx = (const float*)device_view(x);
  const float* sv = (const float*)device_view(v);
  const float* sF = (const float*)device_view(F);
  const float* sC = (const float*)device_view(C);
  float* stage = c->staging;
  if (!sx) {
    MPM_CUDA_TRY(cudaMemcpyAsync(stage, x, sizeof(float) * P * D, cudaMemcpyDefault, s));
    sx = stage;
  }
  if (!sv) {
    MPM_CUDA_TRY(cudaMemcpyAsync(stage + P * D, v, sizeof(float) * P * D, cudaMemcpyDefault, s));
    sv = stage + P * D;
  }
  if (!sF) {
    MPM_CUDA_TRY(cudaMemcpyAsync(stage + 2 * P * D, F, sizeof(float) * P * DD, cudaMemcpyDefault, s));
    sF = stage + 2 * P * D;
  }
  const bool zeroC = (C == nullptr) || c->transfer == MPM_TRANSFER_PIC;
  if (!zeroC && !sC) {
    MPM_CUDA_TRY(cudaMemcpyAsync(stage + 2 * P * D + P * DD, C, sizeof(float) * P * DD, cudaMemcpyDefault, s));
    sC = stage + 2 * P * D + P * DD;
  }
  // a fresh start: both grids zero, no pending clears
  for (int b = 0; b < 2; ++b) {
    MPM_CUDA_TRY(cudaMemsetAsync(c->grid[b], 0, sizeof(float4) * (size_t)c->n_inst * c->gnodes, s));
    MPM_CUDA_TRY(cudaMemsetAsync(c->touched[b], 0, c->n_keys, s));
  }
  MPM_CUDA_TRY(cudaMemsetAsync(c->counts, 0, sizeof(int32_t) * c->n_keys, s));
  c->cur = 0;
  c->g = 0;
  StateView dst{c->state[0], c->id[0]};
  int blocks = std::max(1, std::min(ceil_div(c->P, 256), c->n_sm * 8));
  if (D == 2)
    mpm_load<2><<<blocks, 256, 0, s>>>(c->dp, sx, sv, sF, sC, dst, c->d_offs, c->n_inst, c->key, c->counts,
                                       zeroC ? 1 : 0, c->status);
  else
    mpm_load<3><<<blocks, 256, 0, s>>>(c->dp, sx, sv, sF, sC, dst, c->d_offs, c->n_inst, c->key, c->counts,
                                       zeroC ? 1 : 0, c->status);
  MPM_CUDA_TRY(cudaGetLastError());
  MPM_TRY(launch_scan_permute(c, s, /*clear_consumed=*/false));
  MPM_TRY(launch_fused<true>(c, s));
  c->loaded = true;
  return MPM_OK;
}

mpm_status mpm_step(mpm_ctx* c, int n_steps, void* stream) {
  MPM_CHECK_ARG(c, "null context");
  MPM_CHECK_ARG(c->loaded, "mpm_set_state must be called first");
  MPM_CHECK_ARG(n_steps >= 0, "n_steps must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  for (int k = 0; k < n_steps; ++k) {
    MPM_TRY(launch_fused<false>(c, s));
    // the new state lives in the other buffer; the consumed grid is cleared
    c->cur = 1 - c->cur;
    MPM_TRY(launch_scan_permute(c, s, /*clear_consumed=*/true));
    c->g = 1 - c->g;
  }
  return MPM_OK;
}

mpm_status mpm_step_profiled(mpm_ctx* c, int n_steps, void* flush_buf, size_t flush_bytes, float* kernel_ms,
                             void* stream) {
  MPM_CHECK_ARG(c && kernel_ms, "null argument");
  MPM_CHECK_ARG(c->loaded, "mpm_set_state must be called first");
  MPM_CHECK_ARG(n_steps >= 0, "n_steps must be >= 0");
  MPM_CHECK_ARG(flush_bytes == 0 || flush_buf, "flush_buf is null");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<cudaEvent_t> ev((size_t)4 * n_steps, nullptr);
  mpm_status st = MPM_OK;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) st = set_error(MPM_ECUDA, "cudaEventCreate");
  for (int k = 0; k < n_steps && st == MPM_OK; ++k) {
    cudaEvent_t* e = ev.data() + 4 * k;
    if (k > 0 && flush_bytes > 0 && cudaMemsetAsync(flush_buf, k & 0xff, flush_bytes, s) != cudaSuccess) {
      st = set_error(MPM_ECUDA, "flush memset");
      break;
    }
    cudaEventRecord(e[0], s);
    st = launch_fused<false>(c, s);
    if (st != MPM_OK) break;
    c->cur = 1 - c->cur;
    cudaEventRecord(e[1], s);
    mpm_scan<<<c->n_scan_tiles, kScanTile, 0, s>>>(c->n_keys, c->P, c->counts, c->offsets, c->cursor, c->work,
                                                   c->n_work, c->max_work, c->tile_state, c->status);
    cudaEventRecord(e[2], s);
    int blocks = std::max(1, std::min(ceil_div(c->P, 256), c->n_sm * 8));
    if (c->D == 2)
      mpm_permute<2><<<blocks, 256, 0, s>>>(c->dp, c->key, c->offsets, c->cursor, c->perm, c->grid[c->g],
                                            c->touched[c->g], c->tile_state, c->n_scan_tiles);
    else
      mpm_permute<3><<<blocks, 256, 0, s>>>(c->dp, c->key, c->offsets, c->cursor, c->perm, c->grid[c->g],
                                            c->touched[c->g], c->tile_state, c->n_scan_tiles);
    cudaEventRecord(e[3], s);
    c->g = 1 - c->g;
  }
  if (st == MPM_OK && n_steps > 0) {
    if (cudaEventSynchronize(ev.back()) != cudaSuccess) st = set_error(MPM_ECUDA, "event sync");
    for (int k = 0; k < n_steps && st == MPM_OK; ++k) {
      const cudaEvent_t* e = ev.data() + 4 * k;
      for (int q = 0; q < 3; ++q) cudaEventElapsedTime(&kernel_ms[4 * k + q], e[q], e[q + 1]);
      cudaEventElapsedTime(&kernel_ms[4 * k + 3], e[0], e[3]);
    }
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (st != MPM_OK) return st;
  MPM_CUDA_TRY(cudaGetLastError());
  return MPM_OK;
}

mpm_status mpm_step_timed(mpm_ctx* c, int n_steps, void* flush_buf, size_t flush_bytes, float* step_ms,
                          void* stream) {
  MPM_CHECK_ARG(c && step_ms, "null argument");
  MPM_CHECK_ARG(c->loaded, "mpm_set_state must be called first");
  MPM_CHECK_ARG(n_steps >= 0, "n_steps must be >= 0");
  MPM_CHECK_ARG(flush_bytes == 0 || flush_buf, "flush_buf is null");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<cudaEvent_t> ev((size_t)2 * n_steps, nullptr);
  mpm_status st = MPM_OK;
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) st = set_error(MPM_ECUDA, "cudaEventCreate");
  for (int k = 0; k < n_steps && st == MPM_OK; ++k) {
    if (k > 0 && flush_bytes > 0 && cudaMemsetAsync(flush_buf, k & 0xff, flush_bytes, s) != cudaSuccess) {
      st = set_error(MPM_ECUDA, "flush memset");
      break;
    }
    cudaEventRecord(ev[2 * k], s);
    st = launch_fused<false>(c, s);
    if (st != MPM_OK) break;
    c->cur = 1 - c->cur;
    st = launch_scan_permute(c, s, /*clear_consumed=*/true);
    c->g = 1 - c->g;
    cudaEventRecord(ev[2 * k + 1], s);
  }
  if (st == MPM_OK && n_steps > 0) {
    if (cudaEventSynchronize(ev.back()) != cudaSuccess) st = set_error(MPM_ECUDA, "event sync");
    for (int k = 0; k < n_steps && st == MPM_OK; ++k) cudaEventElapsedTime(&step_ms[k], ev[2 * k], ev[2 * k + 1]);
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (st != MPM_OK) return st;
  MPM_CUDA_TRY(cudaGetLastError());
  return MPM_OK;
}

mpm_status mpm_get_state(mpm_ctx* c, float* x, float* v, float* F, float* C, void* stream) {
  MPM_CHECK_ARG(c && c->loaded, "no state loaded");
  cudaStream_t s = (cudaStream_t)stream;
  const int D = c->D, DD = D * D;
  const size_t P = c->P;
  StateView src{c->state[c->cur], c->id[c->cur]};
  int blocks = std::max(1, std::min(ceil_div(c->P, 256), c->n_sm * 8));
  // device-accessible outputs are written by the kernels directly, in the caller's order
  float* const outs[4] = {x, v, F, C};
  float* views[4];
  bool any_view = false, any_staged = false;
  for (int k = 0; k < 4; ++k) {
    views[k] = (float*)device_view(outs[k]);
    any_view |= views[k] != nullptr;
    any_staged |= outs[k] != nullptr && views[k] == nullptr;
  }
  if (any_view) {
    mpm_inverse_ids<<<blocks, 256, 0, s>>>(c->P, src.id, c->inv_id);
    MPM_CUDA_TRY(cudaGetLastError());
    const int comp0[4] = {0, D, 2 * D, 2 * D + DD}, ncomp[4] = {D, D, DD, DD};
    for (int k = 0; k < 4; ++k) {
      if (!views[k]) continue;
      const int64_t n4 = ((int64_t)P * ncomp[k] + 3) / 4;
      const int b = (int)std::max<int64_t>(1, std::min<int64_t>((n4 + 255) / 256, (int64_t)c->n_sm * 8));
      mpm_store_rows<<<b, 256, 0, s>>>(c->P, src, c->inv_id, views[k], comp0[k], ncomp[k]);
      MPM_CUDA_TRY(cudaGetLastError());
    }
  }
  if (any_staged) {
    float* sx = c->staging;
    float* sv = sx + P * D;
    float* sF = sv + P * D;
    float* sC = sF + P * DD;
    float* st[4] = {sx, sv, sF, sC};
    for (int k = 0; k < 4; ++k)
      if (!outs[k] || views[k]) st[k] = nullptr;
    if (D == 2)
      mpm_store<2><<<blocks, 256, 0, s>>>(c->dp, src, st[0], st[1], st[2], st[3]);
    else
      mpm_store<3><<<blocks, 256, 0, s>>>(c->dp, src, st[0], st[1], st[2], st[3]);
    MPM_CUDA_TRY(cudaGetLastError());
    const size_t bytes[4] = {sizeof(float) * P * D, sizeof(float) * P * D, sizeof(float) * P * DD,
                             sizeof(float) * P * DD};
    for (int k = 0; k < 4; ++k)
      if (st[k]) MPM_CUDA_TRY(cudaMemcpyAsync(outs[k], st[k], bytes[k], cudaMemcpyDefault, s));
  }
  return MPM_OK;
}

mpm_status mpm_status_word(mpm_ctx* c, uint32_t* out, int clear, void* stream) {
  MPM_CHECK_ARG(c && out, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t h = 0;
  MPM_CUDA_TRY(cudaMemcpyAsync(&h, c->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  if (clear) MPM_CUDA_TRY(cudaMemsetAsync(c->status, 0, sizeof(uint32_t), s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  *out = h;
  return MPM_OK;
}

int64_t mpm_num_block_keys(const mpm_ctx* c) { return c ? c->n_keys : 0; }

mpm_status mpm_step_noalloc(const mpm_config* cfg, float* x, float* v, float* F, float* C, int n_steps,
                            uint32_t* status_out, void* stream) {
  MPM_CHECK_ARG(cfg && x && v && F, "null argument");
  MPM_CHECK_ARG(n_steps >= 0, "n_steps must be >= 0");
  MPM_CHECK_ARG(cfg->dim == 2 || cfg->dim == 3, "dim must be 2 or 3");
  const int B = cfg->dim == 2 ? Blk<2>::B : Blk<3>::B;
  MPM_CHECK_ARG(cfg->n_grid >= 8 && cfg->n_grid % B == 0, "n_grid must be a multiple of 8 (2D) / 4 (3D)");
  MPM_CHECK_ARG(cfg->n_inst >= 1 && cfg->n_inst <= 64 && cfg->E && cfg->nu && cfg->inst_offsets,
                "instances (1..64 for the fixed-scratch step)");
  MPM_CHECK_ARG(cfg->dx > 0 && cfg->dt > 0 && cfg->rho > 0 && cfg->p_vol > 0, "dx, dt, rho, p_vol must be > 0");
  MPM_CHECK_ARG(cfg->material == MPM_NEO_HOOKEAN || cfg->material == MPM_FIXED_COROTATED ||
                    cfg->material == MPM_FIXED_COROTATED_PLASTIC,
                "material");
  MPM_CHECK_ARG(cfg->material != MPM_FIXED_COROTATED_PLASTIC ||
                    (cfg->plastic_compression >= 0.f && cfg->plastic_compression < 1.f && cfg->plastic_stretch >= 0.f),
                "plastic bounds: 0 <= plastic_compression < 1, plastic_stretch >= 0");
  MPM_CHECK_ARG(cfg->transfer == MPM_TRANSFER_MLS || cfg->transfer == MPM_TRANSFER_PIC, "transfer");
  MPM_CHECK_ARG(cfg->bc == MPM_BC_STICKY || cfg->bc == MPM_BC_SLIP_FLOOR, "bc");
  MPM_CHECK_ARG(cfg->polar_eft == 0 || cfg->polar_eft == 1, "polar_eft: 0 or 1");
  MPM_CHECK_ARG(cfg->bc_width >= 0 && cfg->inst_offsets[0] == 0, "bc_width, inst_offsets[0]");
  for (int k = 0; k < cfg->n_inst; ++k)
    MPM_CHECK_ARG(cfg->inst_offsets[k + 1] >= cfg->inst_offsets[k], "inst_offsets must be non-decreasing");
  const int64_t P64 = cfg->inst_offsets[cfg->n_inst];
  MPM_CHECK_ARG(P64 >= 1 && P64 < (1ll << 30), "particle count out of range");
  // per-instance Lame parameters and offsets, checked before anything is enqueued: a rejected
  // call touches nothing on the device (the scratch is shared with every other call)
  float2 ml[64];
  int64_t offs[65];
  for (int k = 0; k < cfg->n_inst; ++k) {
    const double E = cfg->E[k], nu = cfg->nu[k];
    MPM_CHECK_ARG(E > 0 && nu > -1 && nu < 0.5, "E must be > 0 and -1 < nu < 0.5");
    ml[k] = make_float2((float)(E / (2 * (1 + nu))), (float)(E * nu / ((1 + nu) * (1 - 2 * nu))));
  }
  for (int k = 0; k <= cfg->n_inst; ++k) offs[k] = cfg->inst_offsets[k];
  // the state arrays are read and written by kernels: they must be device (or managed) memory
  {
    const void* arrs[4] = {x, v, F, C};
    const char* names[4] = {"x", "v", "F", "C"};
    for (int a = 0; a < 4; ++a) {
      if (!arrs[a]) continue;
      cudaPointerAttributes at{};
      if (cudaPointerGetAttributes(&at, arrs[a]) != cudaSuccess) {
        cudaGetLastError();
        return set_error(MPM_EINVAL, std::string("mpm_step_noalloc: ") + names[a] + " is not a CUDA pointer");
      }
      MPM_CHECK_ARG(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged,
                    std::string("mpm_step_noalloc: ") + names[a] + " must be device or managed memory");
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  void* scratch = nullptr;
  MPM_TRY(noalloc_scratch(&scratch));

  // a context whose device pointers all point into the fixed scratch
  mpm_ctx c;
  c.cfg = *cfg;
  c.D = cfg->dim;
  c.n = cfg->n_grid;
  c.B = B;
  c.nb = c.n / B;
  c.nblk = c.D == 2 ? c.nb * c.nb : c.nb * c.nb * c.nb;
  c.n_inst = cfg->n_inst;
  const int64_t nk = (int64_t)c.n_inst * c.nblk;
  MPM_CHECK_ARG(nk < (1ll << 30), "too many grid blocks");
  c.n_keys = (int)nk;
  c.P = (int)P64;
  c.material = cfg->material;
  c.transfer = cfg->transfer;
  c.polar_eft = cfg->polar_eft;
  c.gnodes = c.D == 2 ? (int64_t)c.n * c.n : (int64_t)c.n * c.n * c.n;
  int dev = 0;
  MPM_CUDA_TRY(cudaGetDevice(&dev));
  MPM_CUDA_TRY(cudaDeviceGetAttribute(&c.n_sm, cudaDevAttrMultiProcessorCount, dev));
  c.max_work = ceil_div(c.P, kItem) + std::min(c.n_keys, c.P) + 1;
  c.n_scan_tiles = ceil_div(c.n_keys, kScanTile);
  const int D = c.D, DD = D * D;
  const size_t comps = 2 * D + 2 * DD;
  Carve cv{(char*)scratch, 0, kNoAllocBytes};
  for (int b = 0; b < 2; ++b) {
    c.state[b] = cv.take<float>(comps * c.P);
    c.id[b] = cv.take<int32_t>(c.P);
    c.grid[b] = cv.take<float4>((size_t)c.n_inst * c.gnodes);
    c.touched[b] = cv.take<uint8_t>(c.n_keys);
  }
  c.key = cv.take<int32_t>(c.P);
  c.perm = cv.take<int32_t>(c.P);
  c.counts = cv.take<int32_t>(c.n_keys);
  c.cursor = cv.take<int32_t>(c.n_keys);
  c.offsets = cv.take<int32_t>(c.n_keys + 1);
  c.work = cv.take<int4>(c.max_work);
  c.n_work = cv.take<int32_t>(1);
  c.tile_state = cv.take<unsigned long long>(c.n_scan_tiles);
  c.mu_lam = cv.take<float2>(c.n_inst);
  c.d_offs = cv.take<int64_t>(c.n_inst + 1);
  c.status = cv.take<uint32_t>(1);
  if (cv.used > cv.cap)
    return set_error(MPM_EINVAL, "mpm_step_noalloc: this configuration needs " + std::to_string(cv.used) +
                                     " bytes of work memory; the fixed scratch holds " +
                                     std::to_string(kNoAllocBytes) + " bytes (8 MiB)");
  // the scratch keeps the previous call's contents: clear what must start at zero
  for (int b = 0; b < 2; ++b) {
    MPM_CUDA_TRY(cudaMemsetAsync(c.grid[b], 0, sizeof(float4) * (size_t)c.n_inst * c.gnodes, s));
    MPM_CUDA_TRY(cudaMemsetAsync(c.touched[b], 0, c.n_keys, s));
  }
  MPM_CUDA_TRY(cudaMemsetAsync(c.counts, 0, sizeof(int32_t) * c.n_keys, s));
  MPM_CUDA_TRY(cudaMemsetAsync(c.cursor, 0, sizeof(int32_t) * c.n_keys, s));
  MPM_CUDA_TRY(cudaMemsetAsync(c.tile_state, 0, sizeof(unsigned long long) * c.n_scan_tiles, s));
  MPM_CUDA_TRY(cudaMemsetAsync(c.n_work, 0, sizeof(int32_t), s));
  MPM_CUDA_TRY(cudaMemsetAsync(c.status, 0, sizeof(uint32_t), s));
  MPM_CUDA_TRY(cudaMemcpyAsync(c.mu_lam, ml, sizeof(float2) * c.n_inst, cudaMemcpyHostToDevice, s));
  MPM_CUDA_TRY(cudaMemcpyAsync(c.d_offs, offs, sizeof(int64_t) * (c.n_inst + 1), cudaMemcpyHostToDevice, s));
  DevParams& p = c.dp;
  p.P = c.P;
  p.n = c.n;
  p.nb = c.nb;
  p.nblk = c.nblk;
  p.n_keys = c.n_keys;
  p.gnodes = c.gnodes;
  p.dx = cfg->dx;
  p.inv_dx = (float)(1.0 / cfg->dx);
  p.dt = cfg->dt;
  for (int a = 0; a < 3; ++a) p.g[a] = cfg->gravity[a];
  p.bc = cfg->bc;
  p.bc_width = cfg->bc_width;
  p.mass = cfg->rho * cfg->p_vol;
  p.vol = cfg->p_vol;
  p.mu_lam = c.mu_lam;
  p.sv_lo = 1.f - cfg->plastic_compression;
  p.sv_hi = 1.f + cfg->plastic_stretch;
  c.fused_grid = std::max(1, std::min(c.max_work, c.n_sm * 8));
  // load the caller's state, bin it and transfer it to the grid, then step
  c.cur = 0;
  c.g = 0;
  const bool zeroC = (C == nullptr) || c.transfer == MPM_TRANSFER_PIC;
  StateView dst{c.state[0], c.id[0]};
  const int blocks = std::max(1, std::min(ceil_div(c.P, 256), c.n_sm * 8));
  if (D == 2)
    mpm_load<2><<<blocks, 256, 0, s>>>(c.dp, x, v, F, C, dst, c.d_offs, c.n_inst, c.key, c.counts, zeroC ? 1 : 0,
                                       c.status);
  else
    mpm_load<3><<<blocks, 256, 0, s>>>(c.dp, x, v, F, C, dst, c.d_offs, c.n_inst, c.key, c.counts, zeroC ? 1 : 0,
                                       c.status);
  MPM_CUDA_TRY(cudaGetLastError());
  MPM_TRY(launch_scan_permute(&c, s, /*clear_consumed=*/false));
  MPM_TRY(launch_fused<true>(&c, s));
  for (int k = 0; k < n_steps; ++k) {
    MPM_TRY(launch_fused<false>(&c, s));
    c.cur = 1 - c.cur;
    MPM_TRY(launch_scan_permute(&c, s, /*clear_consumed=*/true));
    c.g = 1 - c.g;
  }
  // write the new state back into the caller's arrays (caller's particle order)
  StateView src{c.state[c.cur], c.id[c.cur]};
  if (D == 2)
    mpm_store<2><<<blocks, 256, 0, s>>>(c.dp, src, x, v, F, C);
  else
    mpm_store<3><<<blocks, 256, 0, s>>>(c.dp, src, x, v, F, C);
  MPM_CUDA_TRY(cudaGetLastError());
  if (status_out) {
    uint32_t h = 0;
    MPM_CUDA_TRY(cudaMemcpyAsync(&h, c.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    MPM_CUDA_TRY(cudaStreamSynchronize(s));
    *status_out = h;
  }
  return MPM_OK;
}


mpm_status mpm_debug_bins(mpm_ctx* c, int32_t* cell_keys, int32_t* block_keys, int32_t* block_offsets, void* stream) {
  MPM_CHECK_ARG(c && c->loaded && cell_keys && block_keys, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  int32_t *dc = nullptr, *db = nullptr;
  MPM_CUDA_TRY(cudaMallocAsync((void**)&dc, sizeof(int32_t) * c->P, s));
  MPM_CUDA_TRY(cudaMallocAsync((void**)&db, sizeof(int32_t) * c->P, s));
  StateView src{c->state[c->cur], c->id[c->cur]};
  int blocks = std::max(1, std::min(ceil_div(c->P, 256), c->n_sm * 8));
  if (c->D == 2)
    mpm_bins<2><<<blocks, 256, 0, s>>>(c->dp, src, c->key, dc, db);
  else
    mpm_bins<3><<<blocks, 256, 0, s>>>(c->dp, src, c->key, dc, db);
  MPM_CUDA_TRY(cudaGetLastError());
  MPM_CUDA_TRY(cudaMemcpyAsync(cell_keys, dc, sizeof(int32_t) * c->P, cudaMemcpyDefault, s));
  MPM_CUDA_TRY(cudaMemcpyAsync(block_keys, db, sizeof(int32_t) * c->P, cudaMemcpyDefault, s));
  if (block_offsets)
    MPM_CUDA_TRY(cudaMemcpyAsync(block_offsets, c->offsets, sizeof(int32_t) * (c->n_keys + 1), cudaMemcpyDefault, s));
  MPM_CUDA_TRY(cudaFreeAsync(dc, s));
  MPM_CUDA_TRY(cudaFreeAsync(db, s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  return MPM_OK;
}

mpm_status mpm_debug_grid(mpm_ctx* c, float* mass, float* momentum, float* velocity, void* stream) {
  MPM_CHECK_ARG(c && c->loaded, "no state loaded");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = (size_t)c->n_inst * c->gnodes;
  float *dm = nullptr, *dp = nullptr, *dv = nullptr;
  if (mass) MPM_CUDA_TRY(cudaMallocAsync((void**)&dm, sizeof(float) * N, s));
  if (momentum) MPM_CUDA_TRY(cudaMallocAsync((void**)&dp, sizeof(float) * N * c->D, s));
  if (velocity) MPM_CUDA_TRY(cudaMallocAsync((void**)&dv, sizeof(float) * N * c->D, s));
  int blocks = std::max(1, std::min(ceil_div((long long)N, 256), c->n_sm * 16));
  if (c->D == 2)
    mpm_grid_dump<2><<<blocks, 256, 0, s>>>(c->dp, c->n_inst, c->grid[c->g], dm, dp, dv);
  else
    mpm_grid_dump<3><<<blocks, 256, 0, s>>>(c->dp, c->n_inst, c->grid[c->g], dm, dp, dv);
  MPM_CUDA_TRY(cudaGetLastError());
  if (mass) MPM_CUDA_TRY(cudaMemcpyAsync(mass, dm, sizeof(float) * N, cudaMemcpyDefault, s));
  if (momentum) MPM_CUDA_TRY(cudaMemcpyAsync(momentum, dp, sizeof(float) * N * c->D, cudaMemcpyDefault, s));
  if (velocity) MPM_CUDA_TRY(cudaMemcpyAsync(velocity, dv, sizeof(float) * N * c->D, cudaMemcpyDefault, s));
  if (dm) MPM_CUDA_TRY(cudaFreeAsync(dm, s));
  if (dp) MPM_CUDA_TRY(cudaFreeAsync(dp, s));
  if (dv) MPM_CUDA_TRY(cudaFreeAsync(dv, s));
  MPM_CUDA_TRY(cudaStreamSynchronize(s));
  return MPM_OK;
}

}  // extern "C"

/*
 * mpmrom: C ABI of a GB300 (sm_103a) implementation of the data-parallel hot
 * path of "Model reduction for the material point method via an implicit
 * neural representation of the deformation map" (Chen, Chiaramonte,
 * Grinspun, Carlberg).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every call returns an mpm_status; MPM_OK is 0.  On failure a message is
 *   available from mpm_last_error() (thread-local, valid until the next call
 *   on the same thread).  No C++ exception crosses this boundary.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Calls are asynchronous on that stream unless stated otherwise.
 * - Pointers marked "host or device" are copied with cudaMemcpyAsync(...,
 *   cudaMemcpyDefault): they may be device memory or (pinned or pageable)
 *   host memory.  The caller keeps ownership and must keep them alive until
 *   the stream reaches the copy.
 * - Contexts own every work buffer they need; they allocate only in *_init
 *   and free in *_destroy.  Step calls allocate nothing.
 * - Failures detected on the device (non-finite values, inverted elements,
 *   particles leaving the grid, solver breakdown) are OR-ed into a device
 *   status word; read it with the *_status call of the object.
 * - All floating-point arrays are float32, row-major, C order.
 */
#ifndef MPMROM_H
#define MPMROM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int mpm_status;
enum {
  MPM_OK = 0,
  MPM_EINVAL = 1,      /* invalid argument or configuration */
  MPM_ENOMEM = 2,      /* device allocation failed */
  MPM_ECUDA = 3,       /* CUDA runtime error (message has the details) */
  MPM_EUNSTABLE = 4,   /* simulation produced non-finite or inverted state */
  MPM_ENOCONV = 5,     /* Gauss-Newton made no progress */
  MPM_ETIMEOUT = 6,    /* a bounded device wait ran out */
  MPM_ENOTIMPL = 7     /* option not available in this build */
};

/* Device status bits reported by mpm_status_word / rom_status_word. */
enum {
  MPM_STATUS_NONFINITE = 1 << 0,
  MPM_STATUS_INVERTED = 1 << 1,
  MPM_STATUS_OUT_OF_GRID = 1 << 2,
  MPM_STATUS_GN_NO_DECREASE = 1 << 3,
  MPM_STATUS_CHOLESKY = 1 << 4,
  MPM_STATUS_TIMEOUT = 1 << 5,
  MPM_STATUS_CAPACITY = 1 << 6
};

enum { MPM_TRANSFER_MLS = 0, MPM_TRANSFER_PIC = 1 };
enum { MPM_NEO_HOOKEAN = 0, MPM_FIXED_COROTATED = 1, MPM_FIXED_COROTATED_PLASTIC = 2 };
enum { MPM_BC_STICKY = 0, MPM_BC_SLIP_FLOOR = 1 };

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* mpm_last_error(void);

/* ======================================================================
 * Full-order model: explicit MPM step (Algorithm 1, Section 2.2)
 * ====================================================================== */

/*
 * Configuration of a batch of independent MPM instances that share the grid
 * geometry, the time step and the material law, each on its own grid.
 *   dim           2 or 3.
 *   n_grid        grid nodes per axis; node i sits at i*dx (i = 0..n_grid-1).
 *                 Must be a multiple of 8 (2D) or 4 (3D).
 *   dx, dt        grid spacing and time step.
 *   gravity[3]    body acceleration g (the external force of Algorithm 1 is
 *                 f^e_i = m_i g); only the first dim entries are used.
 *   bc            MPM_BC_STICKY: nodes with any index < bc_width or
 *                 > n_grid-1-bc_width get zero velocity.  MPM_BC_SLIP_FLOOR:
 *                 the low-y band clamps v_y >= 0; the other walls are sticky.
 *   material      MPM_NEO_HOOKEAN or MPM_FIXED_COROTATED (Stomakhin et al.
 *                 2012, the material of Section 5); Lame parameters from
 *                 (E, nu) per instance.  MPM_FIXED_COROTATED_PLASTIC: the
 *                 fixed-corotated law on an elastic F whose singular values
 *                 are clamped, after every F update, to
 *                 [1 - plastic_compression, 1 + plastic_stretch] (a
 *                 snow-like plastic body, Stomakhin et al. 2013 without
 *                 hardening; the reduced-order model does not cover it).
 *   transfer      MPM_TRANSFER_MLS (MLS-MPM with APIC affine velocity, the
 *                 default) or MPM_TRANSFER_PIC (the literal transfers of
 *                 Algorithm 1 with exact basis gradients).
 *   rho, p_vol    density and particle reference volume V0; the particle
 *                 mass is rho * p_vol.
 *   n_inst        number of instances (>= 1).
 *   E, nu         host arrays of n_inst Young's moduli and Poisson ratios.
 *   inst_offsets  host array of n_inst+1 int64: particles of instance k are
 *                 rows inst_offsets[k] .. inst_offsets[k+1]-1 of the state
 *                 arrays.
 *   polar_eft     3D fixed-corotated only: the polar factor R of F is an FP32
 *                 scaled Newton iteration plus one rotation correction whose
 *                 cancelling sums need more than FP32.  0 (default): those
 *                 sums in FP64.  1: as compensated sums of FP32 error-free
 *                 transformations (as accurate as twice FP32 precision, at
 *                 FP32 throughput; GB300's FP64 rate is a small fraction of
 *                 its FP32 rate).
 *   plastic_compression, plastic_stretch   theta_c, theta_s of the plastic
 *                 material (e.g. 2.5e-2, 7.5e-3); ignored otherwise.
 */
typedef struct mpm_config {
  int32_t dim;
  int32_t n_grid;
  float dx;
  float dt;
  float gravity[3];
  int32_t bc;
  int32_t bc_width;
  int32_t material;
  int32_t transfer;
  float rho;
  float p_vol;
  int32_t n_inst;
  const float* E;
  const float* nu;
  const int64_t* inst_offsets;
  int32_t polar_eft;
  float plastic_compression;
  float plastic_stretch;
} mpm_config;

typedef struct mpm_ctx mpm_ctx;

/*
 * Creates a context (allocates all device buffers: two particle-state
 * buffers, two grids per instance, binning tables).  The configuration is
 * copied; the host arrays in it may be freed after the call.  Synchronous.
 * Errors: MPM_EINVAL (bad sizes or parameters), MPM_ENOMEM, MPM_ECUDA.
 */
mpm_status mpm_init(const mpm_config* cfg, mpm_ctx** out);

/* Frees the context and everything it owns.  NULL is allowed. */
void mpm_destroy(mpm_ctx* ctx);

/*
 * Loads the particle state {x, v, F, C} (Algorithm 1, Data) in the caller's
 * particle order: x and v are (P, dim), F and C are (P, dim, dim) with
 * F[p][i][j] = F_ij.  C is the APIC affine velocity (ignored and zeroed in PIC
 * mode; may be NULL, meaning zero).  Host or device pointers.  The context
 * then bins the particles by grid block and performs the particle-to-grid
 * transfer of the loaded state, so that the next mpm_step starts from it.
 */
mpm_status mpm_set_state(mpm_ctx* ctx, const float* x, const float* v, const float* F,
                         const float* C, void* stream);

/*
 * Copies the current particle state back in the caller's original particle
 * order (same layouts as mpm_set_state).  Any pointer may be NULL to skip
 * that quantity.  Host or device pointers.
 */
mpm_status mpm_get_state(mpm_ctx* ctx, float* x, float* v, float* F, float* C, void* stream);

/*
 * Advances every instance by n_steps symplectic-Euler steps of Algorithm 1:
 * particle-to-grid, grid update with gravity and walls, grid-to-particle with
 * the velocity / affine / deformation-gradient update, advection.  Each step
 * is one fused kernel that finishes step n (grid update + grid-to-particle)
 * and starts step n+1 (particle-to-grid of the new state into the other
 * grid), followed by the re-binning of the particles.
 */
mpm_status mpm_step(mpm_ctx* ctx, int n_steps, void* stream);

/*
 * mpm_step with CUDA events recorded around each kernel of every step on
 * `stream`, for measurement.  All n_steps steps are enqueued before the one
 * synchronisation at the end, so the host adds no gaps between them.  If
 * flush_bytes > 0, flush_buf (caller-owned device buffer of flush_bytes
 * bytes) is overwritten between steps, outside the timed intervals (to evict
 * the working set from L2).  Writes the device durations in milliseconds of
 * [fused step kernel, scan, re-binning] for step k to kernel_ms[4k .. 4k+2]
 * and the whole step (first to last event) to kernel_ms[4k+3] (host array of
 * 4 * n_steps floats).
 */
mpm_status mpm_step_profiled(mpm_ctx* ctx, int n_steps, void* flush_buf, size_t flush_bytes, float* kernel_ms,
                             void* stream);

/*
 * mpm_step with CUDA events only at step boundaries (none between a step's
 * kernels), for measuring whole steps: as mpm_step_profiled, with the device
 * duration in milliseconds of step k written to step_ms[k] (host array of
 * n_steps floats).
 */
mpm_status mpm_step_timed(mpm_ctx* ctx, int n_steps, void* flush_buf, size_t flush_bytes, float* step_ms,
                          void* stream);

/*
 * Kinematic (essential, Dirichlet) boundaries: group[p] (n_particles int32, host or device, the
 * caller's particle order; -1 = free) assigns particles to n_groups groups with prescribed
 * velocities (n_groups, dim floats).  After every grid-to-particle transfer a particle of group g
 * takes velocity[g], moves with it and carries no affine velocity (its F follows the grid like
 * every particle's).  n_groups = 0 or group = NULL removes them.  Synchronous.  Errors:
 * MPM_EINVAL for group ids outside [-1, n_groups).
 */
mpm_status mpm_set_kinematic(mpm_ctx* ctx, const int32_t* group, int32_t n_groups, const float* velocities,
                             void* stream);

/*
 * Synchronises `stream`, then returns the OR of MPM_STATUS_* bits raised by
 * the device since the last clear in *out (clears it when `clear` != 0).
 */
mpm_status mpm_status_word(mpm_ctx* ctx, uint32_t* out, int clear, void* stream);

/*
 * Diagnostics of the binning step (the cell sort).  For the current state,
 * in the caller's particle order: cell_keys[p] = linear index of the lowest
 * stencil node floor(x/dx - 0.5) (first axis slowest) and block_keys[p] =
 * instance * n_blocks + grid block of that node.  block_offsets (n_keys+1
 * entries, may be NULL) gets the start of every block's run in the binned
 * order.  Device or host pointers.  Synchronous.
 */
mpm_status mpm_debug_bins(mpm_ctx* ctx, int32_t* cell_keys, int32_t* block_keys,
                          int32_t* block_offsets, void* stream);

/*
 * mpm_step_noalloc: the MPM step for callers that may not allocate device
 * memory.  (This entry point has no counterpart in the paper; it is a
 * deployment convenience.)  Some callers cannot call cudaMalloc at the point
 * where they step a simulation: a host application that owns the whole
 * device-memory budget and forbids allocations inside its frame loop, or
 * code that must never risk an allocation failure or the implicit device
 * synchronisation that cudaMalloc / cudaFree can cause.  This variant
 * allocates nothing: all of its work memory (two particle-state buffers,
 * the binning tables, two grids per instance) is carved out of one fixed,
 * file-scope device array of 8 MiB inside the library, which every GPU that
 * loads the library holds until the process exits.  It makes no
 * cudaMalloc, cudaFree or other allocating call.
 *
 *   cfg          as for mpm_init (1..64 instances); copied per call.
 *   x, v, F, C   device (or managed) arrays in the layout of mpm_set_state,
 *                read as the starting state and overwritten with the state
 *                after n_steps steps (caller's particle order).  C may be
 *                NULL (zero).  Host pointers are rejected (MPM_EINVAL); the
 *                lengths cannot be checked here: each array must hold
 *                P x dim (x, v) or P x dim x dim (F, C) floats, P =
 *                inst_offsets[n_inst].
 *   status_out   if not NULL, the call synchronises `stream` and stores the
 *                MPM_STATUS_* bits raised during the call.
 *
 * Each call loads the state, bins it, performs the particle-to-grid transfer
 * and n_steps steps of mpm_step, and stores the state back; nothing carries
 * over between calls.  The configuration must fit in the fixed array (for
 * example a 2D block of 4096 particles on a 128^2 grid needs about 1 MiB, a
 * 3D scene on a 32^3 grid with 16384 particles about 5 MiB); larger
 * configurations are rejected with MPM_EINVAL and a message giving the bytes
 * needed.  Every argument is checked before anything is enqueued, so a
 * rejected call leaves the shared array untouched.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) once for
 * that device; with lazy module loading that lookup may be the moment the
 * driver loads the library's device code and commits the 8 MiB array, so
 * make the first call at set-up time, before any stream capture.  Each call
 * copies its per-instance constants from host memory and, with status_out,
 * synchronises the stream.  All calls share the one array and every call
 * clears the parts that must start at zero, so calls whose work overlaps on
 * the GPU (other streams, other host threads) race: serialise them.
 */
mpm_status mpm_step_noalloc(const mpm_config* cfg, float* x, float* v, float* F, float* C, int n_steps,
                            uint32_t* status_out, void* stream);

/* Number of block keys (instances x blocks per grid); for sizing block_offsets. */
int64_t mpm_num_block_keys(const mpm_ctx* ctx);

/*
 * Diagnostics of the grid: for the current state, the particle-to-grid
 * result of Algorithm 1 step 1 and the grid update of step 2, dense per
 * instance: mass (n_inst, n_grid^dim), momentum (n_inst, n_grid^dim, dim)
 * = m_i v_i + dt f_i, velocity (n_inst, n_grid^dim, dim) after gravity and
 * walls.  Any pointer may be NULL.  Synchronous.
 */
mpm_status mpm_debug_grid(mpm_ctx* ctx, float* mass, float* momentum, float* velocity,
                          void* stream);

/* ======================================================================
 * Implicit neural decoder g(X; xhat) and its Jacobians
 * (Section 3.1, Eqs. kinematicRestriction, defGrad, timederOne; Section 4,
 * Table 1; input/output scaling of Appendix B)
 * ====================================================================== */

/*
 *   d           spatial dimension (2 or 3).
 *   r           latent dimension (d + r <= 40; with r > 36 every evaluation runs in FP32 on
 *               the CUDA cores, as the tensor-core kernel holds 36 latents).
 *   width       hidden width; must be 128 when n_hidden >= 1.
 *   n_hidden    number of hidden (activated) layers, 0..5.  0 is the linear
 *               manifold of Section 5 (one linear map, no activation).
 *   activation  0 = ELU (the paper's choice), 1 = identity.
 * Layers: [d + r] -> width (n_hidden times, activated) -> d (linear).
 */
typedef struct decoder_desc {
  int32_t d;
  int32_t r;
  int32_t width;
  int32_t n_hidden;
  int32_t activation;
} decoder_desc;

typedef struct mpm_decoder mpm_decoder;

/* Allocates a decoder (parameters zero).  Synchronous. */
mpm_status decoder_create(const decoder_desc* desc, mpm_decoder** out);
void decoder_destroy(mpm_decoder* dec);

/* Number of FP32 parameters: sum over layers of out*in + out. */
int64_t decoder_num_params(const mpm_decoder* dec);

/*
 * Sets the FP32 master parameters and the scaling.  `params` holds, layer by
 * layer, W (out x in, row-major) then b (out); `norm` holds 4*d floats:
 * X_min[d], X_range[d], out_shift[d], out_scale[d]; the network evaluates
 * g = out_scale * MLP((X - X_min) / X_range, xhat) + out_shift.  Host or
 * device pointers.  Also refreshes the BF16 copies used by the tensor cores.
 */
mpm_status decoder_set_params(mpm_decoder* dec, const float* params, const float* norm, void* stream);
mpm_status decoder_get_params(const mpm_decoder* dec, float* params, float* norm, void* stream);

/* Row kinds of decoder_eval. */
enum {
  DECODER_PRIMAL = 0,     /* g(X; xhat) */
  /* 1 .. d:          dg/dX_k, k = kind - 1                             */
  /* d+1 .. d+r:      dg/dxhat_j, j = kind - d - 1                      */
  DECODER_JVP = 1000,     /* (dg/dxhat) u with u = dirs[lat_idx[p]]       */
  DECODER_SECANT = 1001,  /* g(X; xhat + u) - g(X; xhat), u = dirs[lat_idx[p]] */
  /* DECODER_MIXED + b, b = 1 .. d + r: d/d(input b) of the DECODER_JVP row,
   * i.e. d/dX_k ((dg/dxhat) u) for b = k + 1 <= d: the material gradient of the
   * decoded velocity (Eq. timederOne) that the reduced step's affine
   * quadrature velocity needs.  The call must also request DECODER_JVP and
   * tangent kind b. */
  DECODER_MIXED = 2000,
  /* DECODER_SECANT_DIR + m, m = 0 .. 63: g(X; xhat + u_m) - g(X; xhat) with u_m the
   * m-th direction of the point's latent row: dirs then holds (n_lat, n_dirs, r),
   * n_dirs = 1 + the largest m requested (the JVP, secant and mixed rows use
   * direction 0).  Several secants of one point share its primal row. */
  DECODER_SECANT_DIR = 3000
};

/*
 * Evaluates the decoder and derivatives at n points.  Device pointers:
 *   X        (n, d) reference positions.
 *   lat_idx  (n) int32 row of `latents` (and `dirs`) per point, or NULL (row 0).
 *   latents  (n_lat, r) latent coordinates xhat.
 *   dirs     (n_lat, r) directions for DECODER_JVP / DECODER_SECANT /
 *            DECODER_MIXED rows (NULL if none is requested).
 *   kinds    host array of R row kinds (R in 1..64); kinds[0] must be
 *            DECODER_PRIMAL.
 *   out      (R, n, d): out[k][p] = the quantity of kinds[k] at point p.
 * The square hidden layers run as BF16 x BF16 -> FP32 tcgen05 GEMMs; the
 * output layer (N = d) in FP32; the first layer (K = d + r) on the tensor
 * cores in split BF16 when r <= 28 (inputs and weights each hi + lo, three
 * products per K step, about 2^-16 relative error per product, so the input
 * coordinates keep far more than BF16 resolution), otherwise in FP32.
 * Derivative rows propagate with the primal pre-activations of the same
 * point (forward-mode chain rule); secant rows propagate the exact
 * difference act(z + dz) - act(z), so they resolve latent increments far
 * below BF16 resolution; mixed rows propagate act''(z) (W u)(W t) +
 * act'(z) (W m) (forward over forward).  Errors: MPM_EINVAL for an unknown
 * kind, a mixed row without its JVP / tangent partner rows, or missing dirs.
 */
mpm_status decoder_eval(const mpm_decoder* dec, const float* X, const int32_t* lat_idx, const float* latents,
                        const float* dirs, const int32_t* kinds, int R, int64_t n, float* out, void* stream);

/* Synchronises `stream`; OR of MPM_STATUS_* bits raised by decoder kernels. */
mpm_status decoder_status_word(mpm_decoder* dec, uint32_t* out, int clear, void* stream);

/*
 * Arithmetic of the square hidden layers in decoder_eval and in the reduced
 * step's decoder calls (training always uses the tensor cores).  fp32 = 0
 * (default): BF16 x BF16 -> FP32 tcgen05 GEMMs.  fp32 = 1: FP32 GEMMs on the
 * CUDA cores from the FP32 master weights; for the reduced step's small calls,
 * whose time is set by per-tile latency rather than throughput, this costs
 * little and removes the BF16 rounding of positions and gradients.  fp32 = 2:
 * split BF16 on the tensor cores: activations and weights are each the sum of
 * two BF16 numbers (hi = bf16(v), lo = bf16(v - hi)) and every product is
 * A_hi W_hi + A_hi W_lo + A_lo W_hi accumulated in FP32, so each product keeps
 * about 16 bits (relative error near 2^-16 against 2^-24 for FP32, against
 * 2^-8 for BF16) at tensor-core throughput: for many concurrent reduced-order
 * instances.  The output layer is FP32 in every mode, the first layer FP32 in
 * modes 1 and 2 and split BF16 in mode 0 (FP32 there when r > 28).  Takes effect
 * for reduced-order contexts created afterwards.  Errors: MPM_EINVAL.
 */
mpm_status decoder_set_precision(mpm_decoder* dec, int fp32);

/*
 * Expected number of decoder calls running at the same time on different
 * streams (k >= 1, default 1).  The FP32 path spreads a call's rows over about
 * (SM count / k) tiles: one tile per SM gives the lowest latency to a single
 * caller, fewer and fuller tiles leave SMs to concurrent callers (many
 * reduced-order instances served at once).  Affects launches made, and step
 * graphs captured, afterwards.  Errors: MPM_EINVAL.
 */
mpm_status decoder_set_concurrency(mpm_decoder* dec, int k);

/* ======================================================================
 * Reduced-order step (Algorithm 2 with Lagrangian quadrature: Algorithms 3,
 * 5 and 6 or 7) and the accumulated position error (Section 5)
 * ====================================================================== */

/*
 * Configuration of one reduced-order instance.  Grid, time step, walls,
 * material and transfer as in mpm_config (single instance: E, nu scalars).
 *   latent_dim   r, 1..32.
 *   n_samples    |P|, sample material points re-drawn every step (Sec. 3.2.1)
 *                as the n_samples particles with the smallest 64-bit hash
 *                h = out(out(out(seed, instance), step), particle), out(s, k)
 *                the (k+1)-th output of SplitMix64 seeded with s; ties by id.
 *   gn_iters     Gauss-Newton iterations of the position projection (Alg. 6);
 *                Armijo c = 1e-4 with up to 10 step halvings, evaluated as 11
 *                trial steps at once (the same choice as sequential
 *                backtracking).
 *   projection   0 = position-velocity projection (Alg. 6),
 *                1 = velocity-only projection (Alg. 7).
 *   ridge        rho >= 0: the projections solve the regularised least-squares
 *                problems min |J a - b|^2 + rho (tr(J^T J) / r) |a|^2 (J the
 *                latent Jacobian at the samples) for the increment a of the
 *                unknown from its prior: the Gauss-Newton step from the current
 *                iterate, and vhat_{n+1} - vhat_n for the velocity (so that
 *                latent directions the samples do not resolve keep their
 *                velocity).  rho = 0 is the plain least squares of Algorithms 6
 *                and 7 (a 1e-10 relative ridge is always kept so that
 *                rank-deficient J^T J stays factorisable).
 *   affine       MLS transfer only.  0: the quadrature points enter the local
 *                particle-to-grid transfer with C = 0, as Algorithm 5 writes
 *                it.  1: they carry the affine velocity of the decoded motion,
 *                C = (dv/dX) (dg/dX)^-1 with v = (dg/dxhat) vhat_n (the state an
 *                APIC particle of that motion carries; the full-order MLS model
 *                transfers it too).  Ignored with the PIC transfer.
 *   f_reference  0: the quadrature points' deformation gradient is the decoder's
 *                dg/dX (Eq. defGrad).  1: it is measured from the decoded initial
 *                configuration, F = (dg/dX)(X; xhat_n) [(dg/dX)(X; xhat_ref)]^-1
 *                with xhat_ref the fitted initial latent state (rom_fit_initial)
 *                or the one given to rom_set_reference: the decoder's
 *                approximation error of the undeformed configuration then
 *                produces no stress.  For initial states with F = I.
 *   quadrature   0: Lagrangian quadrature (Alg. 3): the samples and the
 *                particles whose stencils reach their basis set.  1: Eulerian
 *                quadrature (Alg. 4): ell^d points per grid cell at
 *                (c + (j + 1/2) / ell) dx on every cell whose points reach a
 *                node of the basis set (cells i - 2 .. i + 1 around node i,
 *                restricted to cells 1 .. n_grid - 3); each point's reference
 *                position X_q solves g(X_q; xhat_n) = x_q by newton_iters Newton
 *                steps from x_q minus the samples' mean displacement; the point
 *                carries mass rho V_q / J and reference volume V_q / J
 *                (V_q = (dx / ell)^d, J = det dg/dX) when X_q lies in the
 *                reference domain (the union of the particles' boxes of side
 *                p_vol^(1/d) centred on X) and |g(X_q) - x_q| < newton_tol dx,
 *                none otherwise.  Excludes affine and f_reference.
 *   ell          points per cell per axis, 1..4 (0: 2).
 *   newton_iters decoder inversion steps, 1..16 (0: 4).
 *   newton_tol   convergence threshold in units of dx (0: 1e-3).
 */
typedef struct rom_config {
  int32_t dim;
  int32_t n_grid;
  float dx;
  float dt;
  float gravity[3];
  int32_t bc;
  int32_t bc_width;
  int32_t material;
  int32_t transfer;
  float rho;
  float p_vol;
  float E;
  float nu;
  int32_t latent_dim;
  int32_t n_samples;
  uint64_t seed;
  int32_t instance;
  int32_t gn_iters;
  int32_t projection;
  float ridge;
  int32_t affine;
  int32_t f_reference;
  int32_t quadrature;
  int32_t ell;
  int32_t newton_iters;
  float newton_tol;
} rom_config;

typedef struct rom_ctx rom_ctx;

/*
 * Creates a reduced-order context over n_particles material points with
 * reference positions X (n_particles, dim) (host or device; copied).  The
 * decoder must outlive the context and its latent dimension must equal
 * cfg->latent_dim.  Synchronous.
 */
mpm_status rom_create(const rom_config* cfg, const mpm_decoder* dec, const float* X, int64_t n_particles,
                      rom_ctx** out);
void rom_destroy(rom_ctx* ctx);

/* Sets xhat_n, vhat_n, xhat_{n-1} (r doubles each, host or device) and the step index. Synchronous. */
mpm_status rom_set_state(rom_ctx* ctx, const double* xhat, const double* vhat, const double* xhat_prev,
                         int64_t step, void* stream);
/* Reads them back (any pointer may be NULL).  Synchronous. */
mpm_status rom_get_state(rom_ctx* ctx, double* xhat, double* vhat, double* xhat_prev, int64_t* step, void* stream);

/*
 * Initial condition by least squares (Eq. essentialSpecInt): xhat_0 by
 * `iters` Gauss-Newton iterations of min sum_p |g(X^p; xhat) - target_p|^2
 * from xhat = 0 over all particles, vhat_0 = argmin sum_p |(dg/dxhat) vhat - V0_p|^2;
 * sets the state (xhat_{-1} = xhat_0 - dt vhat_0, step 0).  target and V0
 * are (n_particles, dim), host or device.  Synchronous.
 */
mpm_status rom_fit_initial(rom_ctx* ctx, const float* target, const float* V0, int iters, void* stream);

/*
 * Reference configuration of the f_reference option: decodes dg/dX at every
 * particle at xhat_ref (r doubles, host or device) and keeps its inverse
 * (P x d x d floats, owned by the context).  rom_fit_initial calls it with the
 * fitted xhat_0 when cfg.f_reference = 1.  Errors: MPM_EINVAL if f_reference
 * is 0.
 */
mpm_status rom_set_reference(rom_ctx* ctx, const double* xhat_ref, void* stream);

/*
 * Advances the reduced state by n_steps steps of Algorithm 2: decoder at all
 * particles, sample / basis / neighbour sets (Alg. 3), dg/dX and the velocity
 * at the quadrature points, local particle-to-grid / grid update /
 * grid-to-particle to the samples (Alg. 5), velocity least squares and the
 * Gauss-Newton position projection (Alg. 6) or the velocity-only projection
 * (Alg. 7).  With the Eulerian quadrature (cfg.quadrature = 1) the samples are
 * decoded alone and the quadrature points come from Algorithm 4 instead of the
 * neighbour set.  All on the device: one captured CUDA graph per step,
 * launched on `stream`.  Solver failures raise MPM_STATUS_* bits
 * (rom_status_word; MPM_STATUS_CAPACITY if the cells exceed the capacity).
 */
mpm_status rom_step(rom_ctx* ctx, int n_steps, void* stream);

mpm_status rom_status_word(rom_ctx* ctx, uint32_t* out, int clear, void* stream);

/*
 * Diagnostics of the last step (any pointer may be NULL; synchronous):
 * qlist (n_particles int32): samples ascending then neighbours ascending;
 * counts (3 int32): |P| (with kinematic groups up to n_samples + min_samples x
 * n_groups; v_trial, x_trial then hold that many rows), |P| + |N| (the number of Eulerian quadrature points
 * with cfg.quadrature = 1), basis-node list length; x_all
 * (n_particles, dim): decoded positions g(X; xhat_n) the step used;
 * v_trial, x_trial (|P|, dim): Algorithm 5 outputs of the samples.
 */
mpm_status rom_debug(rom_ctx* ctx, int32_t* qlist, int32_t* counts, float* x_all, float* v_trial,
                     float* x_trial, void* stream);

/*
 * Line-search choices of the last step's Gauss-Newton iterations (Algorithm 6, backtracking):
 * picks (16 int32, host or device) receives for iteration i < *n_iters the m of the accepted step
 * length 2^-m (the first of the trials 2^0 .. 2^-10 meeting the sufficient-decrease condition), or
 * -1 when none did and the iterate stayed; entries from *n_iters on are unspecified.  *n_iters
 * (host) is cfg.gn_iters, or 0 with the velocity-only projection (no line search).  Where the
 * condition's margin is at the rounding level of the FP32 residual rows, either choice is a
 * correct outcome; tests compare the oracle run with these choices.  Synchronous.  Errors:
 * MPM_EINVAL for a NULL argument.
 */
mpm_status rom_debug_line_search(rom_ctx* ctx, int32_t* picks, int32_t* n_iters, void* stream);

/*
 * Eulerian quadrature of the last step (cfg.quadrature = 1; synchronous; any
 * output pointer may be NULL): the number of points n_points, their positions
 * x_points and reference positions X_points (n_points, dim), mass and
 * reference volume (n_points; zero for points outside the body).  Points are
 * ordered by cell in the order the cells were collected, then by sub-point
 * (last axis fastest).  Output buffers (host or device) must hold the point
 * capacity: min((n_grid - 3)^dim, 6^dim n_samples) ell^dim points.  Errors:
 * MPM_EINVAL with the Lagrangian quadrature.
 */
mpm_status rom_debug_quadrature(rom_ctx* ctx, int32_t* n_points, float* x_points, float* X_points, float* mass,
                                float* V0, void* stream);

/*
 * Kinematic (Dirichlet) boundaries of the reduced model (either quadrature): group[p]
 * (n_particles int32, host or device; -1 = free), n_groups prescribed velocities (n_groups, dim
 * floats).  Every step's sample set is the n_samples-particle draw plus, for each group, those of
 * its min(min_samples, |group|) particles of smallest hash (the same SplitMix64 hash, ties by id)
 * that the draw missed, appended group by group in ascending id (min_samples in [1, 32]; the
 * paper finds 5 enough); kinematic samples take their prescribed velocity as trial velocity.
 * n_groups = 0 removes them.  Resets the grid and the step graph (call before stepping, then
 * set the state).  Synchronous.  Errors: MPM_EINVAL (bad arguments, group ids outside
 * [-1, n_groups), non-finite velocities) is detected before the context changes and leaves it as
 * it was; MPM_ENOMEM / MPM_ECUDA after that point leave the context without its kinematic
 * buffers, and rom_step then returns MPM_EINVAL until a later rom_set_kinematic succeeds.
 */
mpm_status rom_set_kinematic(rom_ctx* ctx, const int32_t* group, int32_t n_groups, const float* velocities,
                             int32_t min_samples, void* stream);

/* g(X^p; xhat_n) for every particle into device array x_out (n_particles, dim). */
mpm_status rom_decode_all(rom_ctx* ctx, float* x_out, void* stream);

/*
 * Batched serving: n reduced-order contexts (each with its own scene, sample
 * count, latent dimension and decoder) stepped by one CUDA graph launch.
 * rom_batch_create captures one step of every context and makes the captures
 * independent child graphs of one graph; rom_batch_step launches it n_steps
 * times on `stream`, each launch advancing every context by one step exactly
 * as rom_step would (the branches run concurrently on the GPU).  The contexts
 * stay owned by the caller and must outlive the batch; each may appear once.
 * State calls (rom_set_state, rom_get_state, rom_decode_*) act on the members
 * as usual between launches.  Calls that change a member's step
 * (rom_set_kinematic, rom_set_reference, rom_fit_initial with the reference
 * gradient) make rom_batch_step return MPM_EINVAL until the batch is rebuilt.
 * A member stepped on its own while a batch launch runs races with it.  Errors:
 * MPM_EINVAL, MPM_ECUDA.
 */
typedef struct rom_batch rom_batch;
mpm_status rom_batch_create(rom_ctx* const* ctxs, int32_t n, rom_batch** out);
mpm_status rom_batch_step(rom_batch* batch, int n_steps, void* stream);
void rom_batch_destroy(rom_batch* batch);

/*
 * g(X; xhat_n) at n reference positions X (n, dim) that need not be particles of
 * the context: the decoder is defined on the whole reference domain, so the
 * reduced state can be rendered at any resolution (the zero-shot
 * super-resolution of Section 5).  X and x_out are device arrays.  Asynchronous
 * on `stream`.
 */
mpm_status rom_decode_points(rom_ctx* ctx, const float* X, int64_t n, float* x_out, void* stream);

/*
 * Accumulated position error of Section 5: acc[0] += sum_i (a_i - b_i)^2,
 * acc[1] += sum_i b_i^2 over n floats (device pointers; acc is 2 doubles on
 * the device).  The error in percent is 100 sqrt(acc[0] / acc[1]).
 */
mpm_status metric_accumulate(const float* a, const float* b, int64_t n, double* acc, void* stream);

/* ======================================================================
 * Decoder training (loss of Section 4.2, optimiser and scaling of
 * Appendix B) on snapshots of the full-order model, with the latent table
 * the remark of Section 4.1 allows in place of the encoder
 * ====================================================================== */

/*
 * Snapshot store.  Instance k has particles inst_offsets[k] .. inst_offsets[k+1]-1
 * of X (reference positions).  Snapshot s belongs to instance snap_inst[s];
 * its successor in time is snap_next[s] (-1 if none); its particle rows are
 * stored consecutively in x, v (dim floats each) and F (dim*dim floats,
 * row-major), snapshots back to back in index order.  Host or device pointers
 * (copied by trainer_create).
 */
typedef struct snapshot_desc {
  int32_t dim;
  int32_t n_inst;
  const int64_t* inst_offsets;  /* host, n_inst + 1 */
  const float* X;
  int32_t n_snap;
  const int32_t* snap_inst;     /* host, n_snap */
  const int32_t* snap_next;     /* host, n_snap */
  const float* x;
  const float* v;
  const float* F;
} snapshot_desc;

/*
 * Input and output scaling of Appendix B, computed on the device from a
 * snapshot store: per coordinate a, X_min[a] and X_range[a] = max - min of
 * the reference positions X (all inst_offsets[n_inst] particles), and the
 * mean and standard deviation (population, 1/N) of the positions x of every
 * snapshot row.  Sets the decoder's scaling to {X_min, X_range, mean, std}
 * (the layout of decoder_set_params' norm) and re-packs its derived weight
 * images; the network parameters are unchanged.  sd->X and sd->x must be
 * device (or managed) pointers; inst_offsets and snap_inst are host arrays.
 * Asynchronous on `stream` (its work memory is allocated and freed in
 * stream order).  Errors: MPM_EINVAL (dim mismatch, empty store, host pointers,
 * snap_inst out of range).
 */
mpm_status decoder_fit_scaling(mpm_decoder* dec, const snapshot_desc* snaps, void* stream);

/*
 *   lambda_F, lambda_v  penalty weights of the deformation-gradient and
 *                       velocity terms of the loss.
 *   dt_snap             time between a snapshot and its successor (the
 *                       latent finite difference (xhat_{n+1} - xhat_n) / dt_snap).
 *   lr0, lr1            Adam learning rate, decaying geometrically from lr0
 *                       to lr1 over total_steps (Appendix B: 1e-3 -> 1e-6).
 *   batch               (snapshot, particle) pairs per step, drawn uniformly
 *                       over all pairs by a counter-based SplitMix64 hash of
 *                       (seed, step, i).
 *   encoder_subset      0: one trainable latent per snapshot (the latent
 *                       table the Remark of Section 4.1 allows).  n > 0: the
 *                       latents come from the encoder network of Section 4.1
 *                       / Table 1, trained with the decoder, whose input is the
 *                       positions of n particles of each snapshot (ids
 *                       floor(j P / n), j < n, P the instance's particle
 *                       count), standardised per coordinate (mean and standard
 *                       deviation over all snapshots) and concatenated
 *                       particle-major; single-channel convolutions of kernel
 *                       6 and stride 2 (ELU) down to the last length >= 32, a
 *                       32-wide ELU layer and a linear layer to r.  dim x n in
 *                       [32, 8192].  Weights Xavier-uniform from `seed`.
 *   shard_index,        data-parallel training (shard_count > 1): this context
 *   shard_count         draws draws shard_index * batch .. (shard_index + 1) *
 *                       batch - 1 of the step's minibatch of shard_count * batch
 *                       points, and normalises its loss and gradients by the
 *                       whole minibatch, so that the sum of the shards'
 *                       gradients is the gradient of the whole minibatch; the
 *                       shards then add their gradients (an all-reduce) between
 *                       trainer_compute_gradients and trainer_apply_gradients.
 *                       shard_count 0 or 1: one process owns the minibatch.
 */
typedef struct train_config {
  float lambda_F;
  float lambda_v;
  float dt_snap;
  float lr0;
  float lr1;
  int32_t batch;
  int64_t total_steps;
  uint64_t seed;
  int32_t encoder_subset;
  int32_t shard_index;
  int32_t shard_count;
} train_config;

typedef struct trainer_ctx trainer_ctx;

/*
 * Creates a trainer for `dec` (which must have >= 2 hidden layers; its
 * parameters are updated in place by decoder_train).  latents0: (n_snap, r)
 * initial latent table or NULL (zeros); ignored with an encoder.  Synchronous.
 */
mpm_status trainer_create(mpm_decoder* dec, const train_config* cfg, const snapshot_desc* snaps,
                          const float* latents0, trainer_ctx** out);
void trainer_destroy(trainer_ctx* ctx);

/*
 * n_steps optimisation steps: minibatch draw, forward with the tangent rows
 * (dg/dX for the lambda_F term, the latent JVP for the lambda_v term) on the
 * tensor cores, hand-written backward through the tangents (including the
 * second-derivative terms of the activation), tensor-core weight-gradient
 * GEMMs, latent-table gradients and Adam.  One captured graph per step.
 */
mpm_status decoder_train(trainer_ctx* ctx, int n_steps, void* stream);

/*
 * Data-parallel training, one optimisation step in two calls.
 * trainer_compute_gradients: this shard's minibatch draw, forward and backward
 * (as decoder_train without the update); copies the gradients of the decoder
 * parameters (decoder_num_params floats) and of the latent table (n_snap x r)
 * or, with the encoder, of the encoder parameters, into g_params and g_second
 * (device buffers of the sizes trainer_gradient_sizes gives), and zeroes the
 * context's own accumulators.  The caller adds the shards' gradients (an
 * all-reduce over the shards) and passes the sums to
 * trainer_apply_gradients, which takes the Adam step of decoder_train with
 * them (same learning-rate schedule and step count).  Asynchronous on
 * `stream`.  With one shard, compute + apply is one decoder_train step.
 */
mpm_status trainer_gradient_sizes(const trainer_ctx* ctx, int64_t* n_params, int64_t* n_second);
mpm_status trainer_compute_gradients(trainer_ctx* ctx, float* g_params, float* g_second, void* stream);
mpm_status trainer_apply_gradients(trainer_ctx* ctx, const float* g_params, const float* g_second, void* stream);

/* Loss of the last step (mean over the whole minibatch; with shards, this shard's part of that
 * mean) and the step count.  Synchronous. */
mpm_status trainer_loss(trainer_ctx* ctx, double* loss, int64_t* step, void* stream);

/* Copies the latents (n_snap, r) out (host or device pointer): the table, or the
 * encoder's output at the start of the last step. */
mpm_status trainer_get_latents(trainer_ctx* ctx, float* latents, void* stream);

mpm_status trainer_status_word(trainer_ctx* ctx, uint32_t* out, int clear, void* stream);

/*
 * Gradient check: one forward/backward on the minibatch of the current step
 * without updating.  Returns the parameter gradients (decoder_num_params
 * floats, same layout as decoder_set_params), the per-snapshot latent
 * gradients (n_snap, r), with an encoder its parameter gradients
 * (trainer_encoder_params layout), the batch (snapshot index and particle
 * index within its instance, batch int32 each) and the loss.  Any output may
 * be NULL.  Synchronous.
 */
mpm_status trainer_gradients(trainer_ctx* ctx, float* g_params, float* g_latents, float* g_encoder,
                             int32_t* batch_snap, int32_t* batch_part, double* loss, void* stream);

/*
 * Encoder parameters (trainer created with encoder_subset > 0): *n_params
 * floats, per convolution l its taps w_l[0..5] then its bias, then W1 (32 x
 * d_conv, row-major), b1 (32), W2 (r x 32, row-major), b2 (r); and the input
 * standardisation shift_scale = [shift (dim), scale (dim)].  Any output may be
 * NULL.  Errors: MPM_EINVAL without an encoder.  Synchronous.
 */
mpm_status trainer_encoder_params(trainer_ctx* ctx, float* params, float* shift_scale, int64_t* n_params,
                                  void* stream);
/* Replaces the encoder parameters and/or the standardisation (NULL keeps it) and
 * resets the encoder's Adam moments.  Synchronous. */
mpm_status trainer_set_encoder_params(trainer_ctx* ctx, const float* params, const float* shift_scale,
                                      void* stream);
/*
 * Generalized coordinates of n full-order states: x (n, n_particles, dim), host
 * or device, particle order of the training instances; latents (n, r), host or
 * device.  Uses the trainer's subset rule and standardisation.  Synchronous.
 */
mpm_status trainer_encode(trainer_ctx* ctx, const float* x, int64_t n, int64_t n_particles, float* latents,
                          void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MPMROM_H */

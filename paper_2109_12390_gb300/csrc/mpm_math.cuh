// Device math of the explicit MPM step: quadratic B-spline stencil, Lame
// parameters, Kirchhoff stress of the neo-Hookean and fixed-corotated laws,
// polar factor of F.  Used by the full-order kernels and by the local step of
// the reduced model.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace mpmrom {

// Quadratic B-spline (the basis reading of Section 2.2): node k of the
// stencil sits at t = fx - k cells, fx = x/dx - base in [0.5, 1.5).
__device__ __forceinline__ void bspline_w(float fx, float w[3]) {
  float a = 1.5f - fx, b = fx - 1.0f, c = fx - 0.5f;
  w[0] = 0.5f * a * a;
  w[1] = 0.75f - b * b;
  w[2] = 0.5f * c * c;
}
// Derivative dN/dfx of the three stencil weights (per cell).
__device__ __forceinline__ void bspline_dw(float fx, float dw[3]) {
  dw[0] = fx - 1.5f;
  dw[1] = -2.0f * (fx - 1.0f);
  dw[2] = fx - 0.5f;
}

// floor(x * inv_dx - 0.5); exact for power-of-two dx (x * inv_dx is a scaling
// by a power of two and the subtraction of 0.5 is exact), the same integer the
// FP64 definition gives.
// The floor is clamped before the conversion: a NaN or a huge coordinate then
// gives an index that every range check rejects and for which base + 2 cannot
// overflow.
__device__ __forceinline__ int stencil_base(float x, float inv_dx) {
  const float b = floorf(x * inv_dx - 0.5f);
  return (int)fminf(fmaxf(b, -16.0f), 16777216.0f);
}

// det(F) - 1 without cancellation (fma keeps the product exact before the -1).
template <int D>
__device__ __forceinline__ float det_minus_one(const float F[D * D]);

template <>
__device__ __forceinline__ float det_minus_one<2>(const float F[4]) {
  return fmaf(F[0], F[3], -1.0f) - F[1] * F[2];
}

template <>
__device__ __forceinline__ float det_minus_one<3>(const float F[9]) {
  // det = F00 (F11 F22 - F12 F21) - F01 (F10 F22 - F12 F20) + F02 (F10 F21 - F11 F20)
  float c0 = fmaf(F[4], F[8], -F[5] * F[7]);
  float c1 = fmaf(F[3], F[8], -F[5] * F[6]);
  float c2 = fmaf(F[3], F[7], -F[4] * F[6]);
  return fmaf(F[0], c0, -1.0f) - F[1] * c1 + F[2] * c2;
}

// --------------------------------------------------------------------------
// Polar factor R of F = R S (det R = +1 for det F > 0).
//
// 2D: closed form, R = [[c, -s], [s, c]] with (c, s) along
// (F00 + F11, F10 - F01).
//
// 3D: scaled Newton iteration X <- (z X + (z X)^-T) / 2, z = |det X|^(-1/3)
// (Higham 1986) in FP32, followed by a correction of the rotation: with R0 the
// FP32 iterate, M = R0^T F = e^W S up to the FP32 error W (antisymmetric), and
// the axial vector w of W solves (tr(S) I - S) w = axial(M - M^T).  The axial
// vector of M - M^T is a difference of O(1) products that cancels to O(1e-7);
// it is accumulated either in FP64 (POLAR_FP64) or, at FP32 throughput, as an
// exact sum of FP32 error-free transformations (POLAR_EFT: every product a b
// split into p + e with e = fma(a, b, -p) exactly (Dekker 1971), the p summed
// with Knuth's TwoSum and all rounding errors added at the end, the
// compensated summation of Ogita, Rump and Oishi 2005: as accurate as
// summing in twice the working precision).  R = R0 (I + W + W^2/2).
// Returns F - R directly (the fixed-corotated stress needs only that), with
// F - R0 formed in FP32 where its entries cancel exactly (Sterbenz) and the
// small rotation correction subtracted afterwards.
// --------------------------------------------------------------------------
__device__ __forceinline__ void f_minus_polar_2d(const float F[4], float out[4]) {
  float c = F[0] + F[3], s = F[2] - F[1];
  float inv = rsqrtf(c * c + s * s);
  c *= inv;
  s *= inv;
  out[0] = F[0] - c;
  out[1] = F[1] + s;
  out[2] = F[2] - s;
  out[3] = F[3] - c;
}

__device__ __forceinline__ void cofactor3(const float X[9], float C[9]) {
  C[0] = fmaf(X[4], X[8], -X[5] * X[7]);
  C[1] = fmaf(X[5], X[6], -X[3] * X[8]);
  C[2] = fmaf(X[3], X[7], -X[4] * X[6]);
  C[3] = fmaf(X[2], X[7], -X[1] * X[8]);
  C[4] = fmaf(X[0], X[8], -X[2] * X[6]);
  C[5] = fmaf(X[1], X[6], -X[0] * X[7]);
  C[6] = fmaf(X[1], X[5], -X[2] * X[4]);
  C[7] = fmaf(X[2], X[3], -X[0] * X[5]);
  C[8] = fmaf(X[0], X[4], -X[1] * X[3]);
}

constexpr int POLAR_FP32 = 0;  // scaled Newton only
constexpr int POLAR_FP64 = 1;  // + FP64 rotation correction
constexpr int POLAR_EFT = 2;   // + rotation correction from compensated FP32 sums

// s + err = a + b exactly (Knuth's TwoSum; no reassociation under nvcc's
// default floating-point rules)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = a + b;
  const float bb = s - a;
  err = (a - (s - bb)) + (b - bb);
}

// sum_k x_k y_k (6 terms) by Dot2 of Ogita, Rump and Oishi 2005: each product
// split exactly into p + e, the p summed with TwoSum, every rounding error
// collected in c and added once at the end.
__device__ __forceinline__ float dot6_compensated(const float x[6], const float y[6]) {
  float s = 0.f, c = 0.f;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float p = x[k] * y[k];
    const float e = fmaf(x[k], y[k], -p);
    float err;
    two_sum(s, p, s, err);
    c += err + e;
  }
  return s + c;
}

template <int REFINE>
__device__ __forceinline__ void f_minus_polar_3d(const float F[9], float out[9]) {
  float X[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) X[i] = F[i];
  // scaled Newton in FP32; converges quadratically, 10 iterations bound it
  for (int it = 0; it < 10; ++it) {
    float C[9];
    cofactor3(X, C);
    float det = X[0] * C[0] + X[1] * C[1] + X[2] * C[2];
    float z = rcbrtf(fabsf(det));
    float zi = __frcp_rn(z * det);   // correctly rounded 1 / x, the value 1.0f / x gives
    float diff = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      float nx = 0.5f * (z * X[i] + zi * C[i]);
      diff = fmaxf(diff, fabsf(nx - X[i]));
      X[i] = nx;
    }
    if (diff < 2e-7f) break;
  }
  // F - R0 (row-major); entries that cancel are exact in FP32
#pragma unroll
  for (int i = 0; i < 9; ++i) out[i] = F[i] - X[i];
  if (REFINE != POLAR_FP32) {
    // axial vector of M - M^T with M = R0^T F:
    //   a0 = sum_k r2k f1k - r1k f2k, a1 = sum_k r0k f2k - r2k f0k, a2 = sum_k r1k f0k - r0k f1k
    float av0, av1, av2;
    if (REFINE == POLAR_FP64) {
      double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double r0 = X[3 * k + 0], r1 = X[3 * k + 1], r2 = X[3 * k + 2];
        double f0 = F[3 * k + 0], f1 = F[3 * k + 1], f2 = F[3 * k + 2];
        a0 = fma(r2, f1, fma(-r1, f2, a0));
        a1 = fma(r0, f2, fma(-r2, f0, a1));
        a2 = fma(r1, f0, fma(-r0, f1, a2));
      }
      av0 = (float)a0;
      av1 = (float)a1;
      av2 = (float)a2;
    } else {
      float x0[6], y0[6], x1[6], y1[6], x2[6], y2[6];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float r0 = X[3 * k + 0], r1 = X[3 * k + 1], r2 = X[3 * k + 2];
        const float f0 = F[3 * k + 0], f1 = F[3 * k + 1], f2 = F[3 * k + 2];
        x0[2 * k] = r2;  y0[2 * k] = f1;  x0[2 * k + 1] = -r1; y0[2 * k + 1] = f2;
        x1[2 * k] = r0;  y1[2 * k] = f2;  x1[2 * k + 1] = -r2; y1[2 * k + 1] = f0;
        x2[2 * k] = r1;  y2[2 * k] = f0;  x2[2 * k + 1] = -r0; y2[2 * k + 1] = f1;
      }
      av0 = dot6_compensated(x0, y0);
      av1 = dot6_compensated(x1, y1);
      av2 = dot6_compensated(x2, y2);
    }
    // S ~ sym(R0^T F) is needed only to first order: S = R0^T F in FP32
    float S[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        S[3 * i + j] = X[i] * F[j] + X[3 + i] * F[3 + j] + X[6 + i] * F[6 + j];
    float s01 = 0.5f * (S[1] + S[3]), s02 = 0.5f * (S[2] + S[6]), s12 = 0.5f * (S[5] + S[7]);
    float tr = S[0] + S[4] + S[8];
    // A = tr(S) I - S (symmetric); w = A^-1 a
    float A[9] = {tr - S[0], -s01, -s02, -s01, tr - S[4], -s12, -s02, -s12, tr - S[8]};
    float Ac[9];
    cofactor3(A, Ac);
    float detA = A[0] * Ac[0] + A[1] * Ac[1] + A[2] * Ac[2];
    float ia = __frcp_rn(detA);
    float w0 = (Ac[0] * av0 + Ac[3] * av1 + Ac[6] * av2) * ia;  // A symmetric: A^-1 = cof^T / det
    float w1 = (Ac[1] * av0 + Ac[4] * av1 + Ac[7] * av2) * ia;
    float w2 = (Ac[2] * av0 + Ac[5] * av1 + Ac[8] * av2) * ia;
    // W = hat(w); E = W + W^2 / 2
    float W[9] = {0.f, -w2, w1, w2, 0.f, -w0, -w1, w0, 0.f};
    float E[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        E[3 * i + j] = W[3 * i + j] + 0.5f * (W[3 * i] * W[j] + W[3 * i + 1] * W[3 + j] + W[3 * i + 2] * W[6 + j]);
    // F - R = (F - R0) - R0 E
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        out[3 * i + j] -= X[3 * i] * E[j] + X[3 * i + 1] * E[3 + j] + X[3 * i + 2] * E[6 + j];
  }
}

// ------------------------------------------------------------- plasticity
// Rotation of the polar decomposition F = R S: 2D in closed form (as in f_minus_polar_2d), 3D by
// the FP32 scaled Newton iteration of f_minus_polar_3d.
template <int D>
__device__ __forceinline__ void polar_rotation(const float F[D * D], float R[D * D]);
template <>
__device__ __forceinline__ void polar_rotation<2>(const float F[4], float R[4]) {
  float c = F[0] + F[3], s = F[2] - F[1];
  const float inv = rsqrtf(c * c + s * s);
  c *= inv;
  s *= inv;
  R[0] = c;
  R[1] = -s;
  R[2] = s;
  R[3] = c;
}
template <>
__device__ __forceinline__ void polar_rotation<3>(const float F[9], float R[9]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = F[i];
  for (int it = 0; it < 10; ++it) {
    float C[9];
    cofactor3(R, C);
    const float det = R[0] * C[0] + R[1] * C[1] + R[2] * C[2];
    const float z = rcbrtf(fabsf(det));
    const float zi = __frcp_rn(z * det);
    float diff = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const float nx = 0.5f * (z * R[i] + zi * C[i]);
      diff = fmaxf(diff, fabsf(nx - R[i]));
      R[i] = nx;
    }
    if (diff < 2e-7f) break;
  }
}

// Eigen-decomposition A = Q diag(l) Q^T of a symmetric D x D matrix by cyclic Jacobi rotations
// (Golub and Van Loan, Matrix Computations, Sec. 8.5): each rotation zeroes one off-diagonal
// entry, with t = sign(th) / (|th| + sqrt(th^2 + 1)), th = (a_qq - a_pp) / (2 a_pq); one rotation
// is exact in 2D, five sweeps converge to FP32 precision in 3D.
template <int D>
__device__ __forceinline__ void jacobi_eig_sym(float A[D * D], float Q[D * D], float l[D]) {
#pragma unroll
  for (int i = 0; i < D * D; ++i) Q[i] = (i % (D + 1) == 0) ? 1.f : 0.f;
  constexpr int SWEEPS = D == 2 ? 1 : 5;
  for (int sw = 0; sw < SWEEPS; ++sw) {
#pragma unroll
    for (int pq = 0; pq < (D == 2 ? 1 : 3); ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      const float apq = A[p * D + q];
      if (apq == 0.f) continue;
      const float th = (A[q * D + q] - A[p * D + p]) / (2.f * apq);
      const float t = copysignf(1.f, th) / (fabsf(th) + sqrtf(fmaf(th, th, 1.f)));
      const float c = rsqrtf(fmaf(t, t, 1.f)), sn = t * c;
      // A <- J^T A J, Q <- Q J with J the rotation in the (p, q) plane
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float akp = A[k * D + p], akq = A[k * D + q];
        A[k * D + p] = c * akp - sn * akq;
        A[k * D + q] = sn * akp + c * akq;
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float apk = A[p * D + k], aqk = A[q * D + k];
        A[p * D + k] = c * apk - sn * aqk;
        A[q * D + k] = sn * apk + c * aqk;
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float qkp = Q[k * D + p], qkq = Q[k * D + q];
        Q[k * D + p] = c * qkp - sn * qkq;
        Q[k * D + q] = sn * qkp + c * qkq;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < D; ++i) l[i] = A[i * D + i];
}

// Return mapping of the plastic fixed-corotated material: with F = R S and S = Q diag(l) Q^T
// (so F = (R Q) diag(l) Q^T is its singular value decomposition), the singular values are clamped
// to [lo, hi] and F rebuilt as R Q diag(clamped) Q^T; F is left untouched when no value moves.
template <int D>
__device__ __forceinline__ void plastic_return(float F[D * D], float lo, float hi) {
  float R[D * D], S[D * D], Q[D * D], l[D];
  polar_rotation<D>(F, R);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) acc = fmaf(R[k * D + i], F[k * D + j], acc);
      S[i * D + j] = acc;
    }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i + 1; j < D; ++j) {
      const float m = 0.5f * (S[i * D + j] + S[j * D + i]);
      S[i * D + j] = m;
      S[j * D + i] = m;
    }
  jacobi_eig_sym<D>(S, Q, l);
  bool moved = false;
  float lc[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    lc[i] = fminf(fmaxf(l[i], lo), hi);
    moved |= lc[i] != l[i];
  }
  if (!moved) return;
  // U = R Q; F = U diag(lc) Q^T
  float U[D * D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) acc = fmaf(R[i * D + k], Q[k * D + j], acc);
      U[i * D + j] = acc;
    }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) acc = fmaf(U[i * D + k] * lc[k], Q[j * D + k], acc);
      F[i * D + j] = acc;
    }
}

// Kirchhoff stress tau = P F^T.
//   neo-Hookean:      tau = mu (F F^T - I) + lam ln(J) I
//   fixed-corotated:  tau = 2 mu (F - R) F^T + lam (J - 1) J I
// ln J and J - 1 come from det(F) - 1 computed without cancellation.
template <int D, int MATERIAL, int POLAR>
__device__ __forceinline__ void kirchhoff(const float F[D * D], float mu, float lam, float tau[D * D]) {
  float jm1 = det_minus_one<D>(F);
  if (MATERIAL == 0) {
    float l = lam * log1pf(jm1);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) s = fmaf(F[i * D + k], F[j * D + k], s);
        tau[i * D + j] = mu * (s - (i == j ? 1.f : 0.f)) + (i == j ? l : 0.f);
      }
  } else {
    float FR[D * D];
    if (D == 2)
      f_minus_polar_2d(F, FR);
    else
      f_minus_polar_3d<POLAR>(F, FR);
    float l = lam * jm1 * (jm1 + 1.0f);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) s = fmaf(FR[i * D + k], F[j * D + k], s);
        tau[i * D + j] = 2.f * mu * s + (i == j ? l : 0.f);
      }
  }
}

// Grid update of Algorithm 1 for one node (step 2): v = p / m + dt g when
// m > 0 (p already holds m v + dt f), then the walls: nodes with any index
// < bc_width or > n - 1 - bc_width are sticky (zero velocity); with the slip
// floor (bc == 1) the low-y band instead clamps v_y >= 0.
template <int D>
__device__ __forceinline__ void grid_node_velocity(float4 mp, const int node[D], int n, int bc, int bc_width,
                                                   float dt, const float g[3], float v[D]) {
  float comp[3] = {mp.y, mp.z, mp.w};
  if (mp.x > 0.f) {
    float im = __frcp_rn(mp.x);
#pragma unroll
    for (int a = 0; a < D; ++a) v[a] = comp[a] * im + dt * g[a];
  } else {
#pragma unroll
    for (int a = 0; a < D; ++a) v[a] = 0.f;
  }
  const int lo = bc_width, hi = n - 1 - bc_width;
  bool sticky = false;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    bool l = node[a] < lo, h = node[a] > hi;
    if (bc == 1 && a == 1) {
      sticky |= h;
      if (l) v[1] = fmaxf(v[1], 0.f);
    } else {
      sticky |= (l | h);
    }
  }
  if (sticky) {
#pragma unroll
    for (int a = 0; a < D; ++a) v[a] = 0.f;
  }
}

}  // namespace mpmrom

// Elastic term of the incremental potential: compressible Neo-Hookean tetrahedra (IPC's variant,
// Li et al. 2020, which the GIPC solver embedded by TacEx builds on):
//   Psi(F) = mu/2 (tr F^T F - 3) - mu ln J + lambda/2 (ln J)^2,   F = Ds Dm^-1,  J = det F.
//
// Per tet (one thread each): energy V Psi, gradient V P D_a (P = dPsi/dF = mu F + (lambda ln J -
// mu) F^-T) and the 12x12 Hessian PSD-projected in deformation-gradient space with the analytic
// eigensystem of isotropic energies (Smith, de Goes & Kim 2019, "Analytic Eigensystems for
// Isotropic Distortion Energies"): in the frame of the SVD F = U S V^T the tangent is block
// diagonal -- a 3x3 "scaling" block d2Psi/dsigma2 on the diagonal entries and, for every pair
// i < j, a 2x2 block on (F_ij, F_ji) whose eigenvalues are
//   twist  (antisymmetric mode):  mu - (mu - lambda ln J) / (s_i s_j)
//   flip   (symmetric mode):      mu + (mu - lambda ln J) / (s_i s_j)
// Negative eigenvalues are clamped to zero and the clamped tangent is mapped to the vertex
// blocks  H_ab = V U Hhat_ab U^T  with  Hhat_ab[i][l] = sum_{jm} Dhat_a[j] Dhat_b[m] Chat[(ij),(lm)],
// Dhat_a = V^T D_a.  Only the 10 blocks a <= b are written.
//
// The energy used by the line search is evaluated in the displacement-gradient form
// (H = F - I from u = x - X, j = J - 1 = tr H + c2 + c3) to avoid the O(1) cancellation of the
// literal formula near rest; it is the same function.
#pragma once
#include "txgel_common.cuh"

namespace txg {

// ---------------------------------------------------------------- small dense linear algebra
template <typename R>
__device__ __forceinline__ void jacobi3(R a[3][3], R w[3], R V[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? R(1) : R(0);
  const R tiny = sizeof(R) == 8 ? R(1e-26) : R(1e-12);
  for (int sweep = 0; sweep < 10; ++sweep) {
    R off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    R dg = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (!(off > tiny * dg)) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0;
      const int q = pq == 0 ? 1 : 2;
      const int r = 3 - p - q;
      R apq = a[p][q];
      if (apq == R(0)) continue;
      R theta = (a[q][q] - a[p][p]) / (R(2) * apq);
      R t = (theta >= R(0) ? R(1) : R(-1)) / (fabs(theta) + sqrt(theta * theta + R(1)));
      R c = R(1) / sqrt(t * t + R(1));
      R s = t * c;
      a[p][p] -= t * apq;
      a[q][q] += t * apq;
      a[p][q] = a[q][p] = R(0);
      R arp = a[r][p], arq = a[r][q];
      a[r][p] = a[p][r] = c * arp - s * arq;
      a[r][q] = a[q][r] = s * arp + c * arq;
      for (int k = 0; k < 3; ++k) {
        R vkp = V[k][p], vkq = V[k][q];
        V[k][p] = c * vkp - s * vkq;
        V[k][q] = s * vkp + c * vkq;
      }
    }
  }
  w[0] = a[0][0];
  w[1] = a[1][1];
  w[2] = a[2][2];
}

// Symmetric 3x3 eigen-decomposition to FP64 accuracy at a fraction of an FP64 Jacobi's cost
// (GB300 issues FP64 at 1/64 of the FP32 rate): the basis from FP32 cyclic Jacobi, one
// Newton-Schulz step X <- X (3 I - X^T X) / 2 to make it orthonormal in FP64, then FP64 Jacobi
// sweeps on the nearly diagonal B = X^T C X with the rotation angle taken from the FP32 quotient
// (the rotation itself, c = 1 / sqrt(1 + t^2), s = t c, and all updates in FP64); entries below
// 1e-15 max|C| are left alone, a sweep without rotations ends the refinement.
__device__ __forceinline__ void eig3_refined(const double C[3][3], double w[3], double V[3][3]) {
  float Cf[3][3], wf[3], Vf[3][3];
  double mx = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Cf[i][j] = (float)C[i][j];
      mx = fmax(mx, fabs(C[i][j]));
    }
  jacobi3<float>(Cf, wf, Vf);
  double X[3][3], S[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) X[i][j] = (double)Vf[i][j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) S[i][j] = fma(X[0][i], X[0][j], fma(X[1][i], X[1][j], X[2][i] * X[2][j]));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = 1.5 * X[i][j] - 0.5 * fma(X[i][0], S[0][j], fma(X[i][1], S[1][j], X[i][2] * S[2][j]));
  double T[3][3], B[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) T[i][j] = fma(C[i][0], V[0][j], fma(C[i][1], V[1][j], C[i][2] * V[2][j]));
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) B[i][j] = B[j][i] = fma(V[0][i], T[0][j], fma(V[1][i], T[1][j], V[2][i] * T[2][j]));
  const double tau = 1e-15 * mx;
  for (int sweep = 0; sweep < 4; ++sweep) {
    bool rot = false;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0;
      const int q = pq == 0 ? 1 : 2;
      const int r = 3 - p - q;
      const double bpq = B[p][q];
      if (!(fabs(bpq) > tau)) continue;
      rot = true;
      const float th = (float)(B[q][q] - B[p][p]) / (2.f * (float)bpq);
      const double t = (double)((th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(fmaf(th, th, 1.f))));
      const double c = rsqrt(fma(t, t, 1.0)), sn = t * c;
      const double bpp = B[p][p], bqq = B[q][q];
      B[p][p] = c * c * bpp - 2.0 * c * sn * bpq + sn * sn * bqq;
      B[q][q] = sn * sn * bpp + 2.0 * c * sn * bpq + c * c * bqq;
      B[p][q] = B[q][p] = c * sn * (bpp - bqq) + (c * c - sn * sn) * bpq;
      const double brp = B[r][p], brq = B[r][q];
      B[r][p] = B[p][r] = c * brp - sn * brq;
      B[r][q] = B[q][r] = sn * brp + c * brq;
      for (int k = 0; k < 3; ++k) {
        const double vkp = V[k][p], vkq = V[k][q];
        V[k][p] = c * vkp - sn * vkq;
        V[k][q] = sn * vkp + c * vkq;
      }
    }
    if (!rot) break;
  }
  w[0] = B[0][0];
  w[1] = B[1][1];
  w[2] = B[2][2];
}

template <typename R>
__device__ __forceinline__ R det3(const R F[3][3]) {
  return F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) -
         F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
         F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
}

// j - ln(1 + j): alternating series for |j| < 0.1 (22 terms, error < 1e-23 j^2), else direct
__device__ __forceinline__ double j_minus_log1p(double j) {
  if (fabs(j) < 0.1) {
    double s = 0.0;
    for (int k = 22; k >= 2; --k) s = s * j + ((k & 1) ? -1.0 : 1.0) / k;
    return s * j * j;
  }
  return j - log1p(j);
}

// V Psi from the displacement gradient H = F - I; +inf when J <= 0
__device__ __forceinline__ double psi_disp(const double H[3][3], double mu, double lam) {
  double tr = H[0][0] + H[1][1] + H[2][2];
  double n2 = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) n2 += H[i][k] * H[i][k];
  double c2 = H[0][0] * H[1][1] - H[0][1] * H[1][0] + H[0][0] * H[2][2] - H[0][2] * H[2][0] +
              H[1][1] * H[2][2] - H[1][2] * H[2][1];
  double c3 = det3(H);
  double j = tr + c2 + c3;
  if (!(j > -1.0)) return CUDART_INF;
  double L = log1p(j);
  return 0.5 * mu * n2 - mu * (c2 + c3) + mu * j_minus_log1p(j) + 0.5 * lam * L * L;
}

// dF/dx_a = D[a] (outer structure): D[a] = row a-1 of Dm^-1, D[0] = -sum
__device__ __forceinline__ void tet_D(const double* Dmi, double D[4][3]) {
  for (int j = 0; j < 3; ++j) {
    D[1][j] = Dmi[j];
    D[2][j] = Dmi[3 + j];
    D[3][j] = Dmi[6 + j];
    D[0][j] = -(D[1][j] + D[2][j] + D[3][j]);
  }
}

// Displacement gradient H = sum_a (x_a - X_a) D_a^T of one tet and F = I + H
// (sum_a X_a D_a^T = I by the definition of Dm^-1)
__device__ __forceinline__ void tet_F(const double xs[4][3], const double Xs[4][3], const double D[4][3],
                                      double F[3][3], double Hd[3][3]) {
  double u[4][3];
  for (int a = 0; a < 4; ++a)
    for (int i = 0; i < 3; ++i) u[a][i] = xs[a][i] - Xs[a][i];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double h = u[0][i] * D[0][j] + u[1][i] * D[1][j] + u[2][i] * D[2][j] + u[3][i] * D[3][j];
      Hd[i][j] = h;
      F[i][j] = i == j ? 1.0 + h : h;
    }
}

__host__ __device__ __forceinline__ int ublk(int a, int b) { return a * 4 - (a * (a - 1)) / 2 + (b - a); }

// Projected Hessian blocks (10 blocks of 9 values, block (a<=b) at ublk(a,b)*BS, row-major 3x3)
// in precision R.  F, J and ln J come in FP64 (the gradient needs them there anyway).
template <typename R>
__device__ __forceinline__ R rsqrt_r(R v) {
  if constexpr (sizeof(R) == 8)
    return rsqrt(v);
  else
    return rsqrtf(v);
}

// One vertex block H_ab = U Hhat_ab U^T (Ap, P2, Q2 already scaled by the rest volume); x =
// Dhat_a, y = Dhat_b.  A diagonal block (x == y) is symmetric: its lower half is mirrored.
template <typename R, bool DIAG>
__device__ __forceinline__ void nh_vertex_block(const R U[3][3], const R Ap[3][3], const R P2[3][3],
                                                const R Q2[3][3], const R x[3], const R y[3], R H[3][3]) {
  R Hh[3][3];
  const R w0 = x[0] * y[0], w1 = x[1] * y[1], w2 = x[2] * y[2];
  Hh[0][0] = w0 * Ap[0][0] + w1 * P2[0][1] + w2 * P2[0][2];
  Hh[1][1] = w1 * Ap[1][1] + w0 * P2[1][0] + w2 * P2[1][2];
  Hh[2][2] = w2 * Ap[2][2] + w0 * P2[2][0] + w1 * P2[2][1];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int l = 0; l < 3; ++l)
      if (i != l) Hh[i][l] = (x[i] * y[l]) * Ap[i][l] + (x[l] * y[i]) * Q2[i][l];
  R T[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int l = 0; l < 3; ++l) T[i][l] = Hh[i][0] * U[l][0] + Hh[i][1] * U[l][1] + Hh[i][2] * U[l][2];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      if (DIAG && l < i) continue;
      H[i][l] = U[i][0] * T[0][l] + U[i][1] * T[1][l] + U[i][2] * T[2][l];
    }
  if (DIAG) {
    H[1][0] = H[0][1];
    H[2][0] = H[0][2];
    H[2][1] = H[1][2];
  }
}

template <typename OutT, int BS, typename R>
__device__ __forceinline__ void nh_store_block(OutT* o, const R H[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int l = 0; l < 3; ++l) o[3 * i + l] = (OutT)H[i][l];
}

// Projected Hessian blocks (10 blocks of 9 values, block (a<=b) at ublk(a,b)*BS, row-major 3x3)
// in precision R.  F, J and ln J come in FP64 (the gradient needs them there anyway).  D[0] is
// minus the sum of D[1..3] (translation invariance), so H is bilinear in the D's and the blocks
// of vertex 0 follow from the other six: H_0b = -sum_{a>=1} H_ab, H_00 = -sum_{b>=1} H_0b.
template <typename R, typename OutT, int BS = 9>
__device__ __forceinline__ void nh_blocks(const double Fd[3][3], double Jd, double lnJd, double mu_d, double lam_d,
                          double vol_d, const double Dd[4][3], bool project, OutT* out) {
  R F[3][3], D[4][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) F[i][j] = (R)Fd[i][j];
  for (int a = 1; a < 4; ++a)
    for (int j = 0; j < 3; ++j) D[a][j] = (R)Dd[a][j];
  const R mu = (R)mu_d, lam = (R)lam_d, vol = (R)vol_d;
  // SVD of F through the eigen-decomposition of F^T F
  R C[3][3], s2[3], V[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) C[i][j] = C[j][i] = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
  if constexpr (sizeof(R) == 8)
    eig3_refined(C, s2, V);
  else
    jacobi3<R>(C, s2, V);
  int o0 = 0, o1 = 1, o2 = 2;  // descending order of s2
  if (s2[o0] < s2[o1]) { int t = o0; o0 = o1; o1 = t; }
  if (s2[o1] < s2[o2]) { int t = o1; o1 = o2; o2 = t; }
  if (s2[o0] < s2[o1]) { int t = o0; o0 = o1; o1 = t; }
  R sg[3], is[3];  // singular values and their reciprocals
  sg[o0] = sqrt(fmax(s2[o0], R(0)));
  sg[o1] = sqrt(fmax(s2[o1], R(0)));
  R U[3][3];
  {
    R u0[3], u1[3];
    for (int i = 0; i < 3; ++i) {
      u0[i] = F[i][0] * V[0][o0] + F[i][1] * V[1][o0] + F[i][2] * V[2][o0];
      u1[i] = F[i][0] * V[0][o1] + F[i][1] * V[1][o1] + F[i][2] * V[2][o1];
    }
    const R r0 = rsqrt_r(u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2]);
    for (int i = 0; i < 3; ++i) u0[i] *= r0;
    R d = u0[0] * u1[0] + u0[1] * u1[1] + u0[2] * u1[2];
    for (int i = 0; i < 3; ++i) u1[i] -= d * u0[i];
    const R r1 = rsqrt_r(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
    for (int i = 0; i < 3; ++i) u1[i] *= r1;
    R u2[3] = {u0[1] * u1[2] - u0[2] * u1[1], u0[2] * u1[0] - u0[0] * u1[2],
               u0[0] * u1[1] - u0[1] * u1[0]};
    for (int i = 0; i < 3; ++i) {
      U[i][o0] = u0[i];
      U[i][o1] = u1[i];
      U[i][o2] = u2[i];
    }
    // det U must equal det V (J > 0)
    if ((det3(U) > R(0)) != (det3(V) > R(0)))
      for (int i = 0; i < 3; ++i) U[i][o2] = -U[i][o2];
  }
  {
    const R p01 = sg[o0] * sg[o1], iJ = R(1) / (R)Jd, ip01 = R(1) / p01;
    sg[o2] = (R)Jd * ip01;
    is[o0] = sg[o1] * ip01;
    is[o1] = sg[o0] * ip01;
    is[o2] = p01 * iJ;
  }
  const R m = mu - lam * (R)lnJd;  // mu - lambda ln J
  // scaling block A = diag(mu + m / s_i^2) + lambda s s^T with s_i = 1 / sigma_i: PSD as it
  // stands when the diagonal part is (lambda >= 0), which holds unless the volume grows by ~25 %
  // or more
  R A[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) A[i][j] = (i == j) ? mu + (m + lam) * (is[i] * is[i]) : lam * (is[i] * is[j]);
  R Ap[3][3];
  const bool psd = (mu + m * (is[0] * is[0]) >= R(0)) && (mu + m * (is[1] * is[1]) >= R(0)) &&
                   (mu + m * (is[2] * is[2]) >= R(0)) && lam >= R(0);
  if (project && !psd) {
    R w[3], Q[3][3];
    if constexpr (sizeof(R) == 8)
      eig3_refined(A, w, Q);
    else
      jacobi3<R>(A, w, Q);
    for (int i = 0; i < 3; ++i) w[i] = fmax(w[i], R(0)) * vol;
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j)
        Ap[i][j] = Ap[j][i] = Q[i][0] * w[0] * Q[j][0] + Q[i][1] * w[1] * Q[j][1] + Q[i][2] * w[2] * Q[j][2];
  } else {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Ap[i][j] = A[i][j] * vol;
  }
  // pair blocks: diagonal p and off-diagonal q of the 2x2 block of every pair i != j (symmetric
  // in i, j), scaled by the volume
  R P2[3][3], Q2[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j) {
      const R k = m * (is[i] * is[j]);
      R lt = mu - k, lf = mu + k;  // twist (antisymmetric), flip (symmetric)
      if (project) { lt = fmax(lt, R(0)); lf = fmax(lf, R(0)); }
      P2[i][j] = P2[j][i] = R(0.5) * vol * (lf + lt);
      Q2[i][j] = Q2[j][i] = R(0.5) * vol * (lf - lt);
    }
  // Dhat_a = V^T D_a (a = 1..3)
  R Dh[4][3];
  for (int a = 1; a < 4; ++a)
    for (int i = 0; i < 3; ++i) Dh[a][i] = V[0][i] * D[a][0] + V[1][i] * D[a][1] + V[2][i] * D[a][2];
  // blocks of vertices 1..3, accumulating minus the column sums into the vertex-0 blocks
  R H0[3][3][3];  // H0[b-1] = H_0b
  for (int b = 0; b < 3; ++b)
    for (int i = 0; i < 3; ++i)
      for (int l = 0; l < 3; ++l) H0[b][i][l] = R(0);
#pragma unroll
  for (int a = 1; a < 4; ++a) {
    {
      R H[3][3];
      nh_vertex_block<R, true>(U, Ap, P2, Q2, Dh[a], Dh[a], H);
      nh_store_block<OutT, BS>(out + ublk(a, a) * BS, H);
      for (int i = 0; i < 3; ++i)
        for (int l = 0; l < 3; ++l) H0[a - 1][i][l] -= H[i][l];
    }
#pragma unroll
    for (int b = a + 1; b < 4; ++b) {
      R H[3][3];
      nh_vertex_block<R, false>(U, Ap, P2, Q2, Dh[a], Dh[b], H);
      nh_store_block<OutT, BS>(out + ublk(a, b) * BS, H);
      for (int i = 0; i < 3; ++i)
        for (int l = 0; l < 3; ++l) {
          H0[b - 1][i][l] -= H[i][l];  // H_ab contributes to H_0b
          H0[a - 1][i][l] -= H[l][i];  // H_ba = H_ab^T contributes to H_0a
        }
    }
  }
  R H00[3][3];
  for (int i = 0; i < 3; ++i)
    for (int l = 0; l < 3; ++l) H00[i][l] = -(H0[0][i][l] + H0[1][i][l] + H0[2][i][l]);
  for (int i = 0; i < 3; ++i)
    for (int l = i + 1; l < 3; ++l) H00[l][i] = H00[i][l] = R(0.5) * (H00[i][l] + H00[l][i]);
  nh_store_block<OutT, BS>(out + ublk(0, 0) * BS, H00);
  for (int b = 1; b < 4; ++b) nh_store_block<OutT, BS>(out + ublk(0, b) * BS, H0[b - 1]);
}

// Gradient of V Psi (12) and energy; returns false if J <= 0
__device__ __forceinline__ bool nh_grad(const double F[3][3], const double Hd[3][3], double mu,
                                        double lam, double vol, const double D[4][3], double g[12],
                                        double* e, double* Jo, double* lnJo) {
  double tr = Hd[0][0] + Hd[1][1] + Hd[2][2];
  double c2 = Hd[0][0] * Hd[1][1] - Hd[0][1] * Hd[1][0] + Hd[0][0] * Hd[2][2] - Hd[0][2] * Hd[2][0] +
              Hd[1][1] * Hd[2][2] - Hd[1][2] * Hd[2][1];
  double j = tr + c2 + det3(Hd);
  if (!(j > -1.0)) return false;
  double J = 1.0 + j, lnJ = log1p(j);
  // F^-T = cof(F) / J
  double cof[3][3];
  cof[0][0] = F[1][1] * F[2][2] - F[1][2] * F[2][1];
  cof[0][1] = F[1][2] * F[2][0] - F[1][0] * F[2][2];
  cof[0][2] = F[1][0] * F[2][1] - F[1][1] * F[2][0];
  cof[1][0] = F[0][2] * F[2][1] - F[0][1] * F[2][2];
  cof[1][1] = F[0][0] * F[2][2] - F[0][2] * F[2][0];
  cof[1][2] = F[0][1] * F[2][0] - F[0][0] * F[2][1];
  cof[2][0] = F[0][1] * F[1][2] - F[0][2] * F[1][1];
  cof[2][1] = F[0][2] * F[1][0] - F[0][0] * F[1][2];
  cof[2][2] = F[0][0] * F[1][1] - F[0][1] * F[1][0];
  const double k = vol * (lam * lnJ - mu) / J, vmu = vol * mu;
  double P[3][3];  // V dPsi/dF
  for (int i = 0; i < 3; ++i)
    for (int l = 0; l < 3; ++l) P[i][l] = vmu * F[i][l] + k * cof[i][l];
  for (int a = 1; a < 4; ++a)
    for (int i = 0; i < 3; ++i) g[3 * a + i] = P[i][0] * D[a][0] + P[i][1] * D[a][1] + P[i][2] * D[a][2];
  for (int i = 0; i < 3; ++i) g[i] = -(g[3 + i] + g[6 + i] + g[9 + i]);  // D_0 = -(D_1 + D_2 + D_3)
  if (e) *e = vol * psi_disp(Hd, mu, lam);
  *Jo = J;
  *lnJo = lnJ;
  return true;
}

// Energy of one tet at x + alpha p (the line-search trial point); used by the energy kernel.
__device__ __forceinline__ double tet_energy_at(const Dev& d, int t, double alpha, double mu, double lam) {
  const int4 tv = d.tets[t];
  const int ids[4] = {tv.x, tv.y, tv.z, tv.w};
  double D[4][3], Hd[3][3];
  tet_D(d.Dminv + 9 * t, D);
  double u[4][3];
  for (int a = 0; a < 4; ++a) {
    const double4_32a x = d.x[ids[a]], X = d.X[ids[a]];
    u[a][0] = x.x - X.x;
    u[a][1] = x.y - X.y;
    u[a][2] = x.z - X.z;
    if (alpha != 0.0) {
      const double4_32a p = d.p[ids[a]];
      u[a][0] += alpha * p.x;
      u[a][1] += alpha * p.y;
      u[a][2] += alpha * p.z;
    }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Hd[i][j] = u[0][i] * D[0][j] + u[1][i] * D[1][j] + u[2][i] * D[2][j] + u[3][i] * D[3][j];
  return d.vol[t] * psi_disp(Hd, mu, lam);
}

}  // namespace txg

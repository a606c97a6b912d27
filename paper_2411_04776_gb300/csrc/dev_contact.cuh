// Contact term of the incremental potential (IPC, Li et al. 2020): unsigned distances between
// the gel surface and the kinematic indenter, the log barrier b(d) = -(d - dhat)^2 ln(d/dhat),
// its gradient and Hessian, the edge-edge mollifier, and additive CCD (Li, Kaufman & Jiang 2021,
// "Codimensional IPC").
//
// Distances are evaluated on the closest-feature pair: for a point vs a triangle the face
// interior when the projection falls strictly inside, otherwise the nearest edge (interior) or
// vertex; for two segments the line-line distance when both closest points are strictly
// interior, otherwise the nearest endpoint-vs-segment case.  Each case has a smooth squared
// distance D written on at most three difference vectors of the four points:
//   PP  D = |u|^2                          u = P_i - P_j
//   PE  D = c(w, e) / |e|^2                w = P_i - P_j, e = P_k - P_j
//   PT  D = s^2 / c(e1, e2)                s = w . (e1 x e2), w = P_i - P_j, e1 = P_k - P_j, e2 = P_l - P_j
//   LL  D = s^2 / c(ea, eb)                w = P_k - P_i, ea = P_j - P_i, eb = P_l - P_k
// with the cross norm c(a, b) = |a x b|^2 = |a|^2 |b|^2 - (a.b)^2.  Derivatives are hand-derived
// in difference-vector space (triple product, cross norm, quotient rule) and mapped to the points.
#pragma once
#include "txgel_common.cuh"

namespace txg {

enum DForm : int { DF_PP = 0, DF_PE = 1, DF_PT = 2, DF_LL = 3 };

struct DType {
  int f;
  int i[4];
};

__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__device__ __forceinline__ void sub3(const double* a, const double* b, double* r) {
  r[0] = a[0] - b[0];
  r[1] = a[1] - b[1];
  r[2] = a[2] - b[2];
}
__device__ __forceinline__ void cross3(const double* a, const double* b, double* r) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

// squared distance of point p to segment [a, b]; type PE (interior) or PP (endpoint)
__device__ __forceinline__ double seg_d2(const double P[4][3], int ip, int ia, int ib, DType* ty) {
  double e[3], w[3];
  sub3(P[ib], P[ia], e);
  sub3(P[ip], P[ia], w);
  const double ee = dot3(e, e);
  const double t = dot3(w, e) / ee;
  if (t <= 0.0) {
    *ty = DType{DF_PP, {ip, ia, -1, -1}};
    return dot3(w, w);
  }
  if (t >= 1.0) {
    double v[3];
    sub3(P[ip], P[ib], v);
    *ty = DType{DF_PP, {ip, ib, -1, -1}};
    return dot3(v, v);
  }
  double c[3];
  cross3(w, e, c);
  *ty = DType{DF_PE, {ip, ia, ib, -1}};
  return dot3(c, c) / ee;
}

// point P[0] vs triangle P[1..3]
__device__ __forceinline__ double pt_classify(const double P[4][3], DType* ty) {
  double e1[3], e2[3], w[3];
  sub3(P[2], P[1], e1);
  sub3(P[3], P[1], e2);
  sub3(P[0], P[1], w);
  const double a = dot3(e1, e1), b = dot3(e1, e2), c = dot3(e2, e2);
  const double d = dot3(e1, w), f = dot3(e2, w);
  const double den = a * c - b * b;
  const double b1 = (c * d - b * f) / den, b2 = (a * f - b * d) / den;
  if (b1 > 0.0 && b2 > 0.0 && b1 + b2 < 1.0) {
    double n[3];
    cross3(e1, e2, n);
    const double s = dot3(w, n);
    *ty = DType{DF_PT, {0, 1, 2, 3}};
    return s * s / dot3(n, n);
  }
  DType t0, t1, t2;
  double d0 = seg_d2(P, 0, 1, 2, &t0);
  double d1 = seg_d2(P, 0, 2, 3, &t1);
  double d2 = seg_d2(P, 0, 3, 1, &t2);
  if (d0 <= d1 && d0 <= d2) { *ty = t0; return d0; }
  if (d1 <= d2) { *ty = t1; return d1; }
  *ty = t2;
  return d2;
}

// segment P[0]P[1] vs segment P[2]P[3]
__device__ __forceinline__ double ee_classify(const double P[4][3], DType* ty) {
  double u[3], v[3], w[3];
  sub3(P[1], P[0], u);
  sub3(P[3], P[2], v);
  sub3(P[0], P[2], w);
  const double a = dot3(u, u), b = dot3(u, v), c = dot3(v, v), d = dot3(u, w), e = dot3(v, w);
  const double den = a * c - b * b;
  if (den > 1e-14 * a * c) {
    const double s = (b * e - c * d) / den, t = (a * e - b * d) / den;
    if (s > 0.0 && s < 1.0 && t > 0.0 && t < 1.0) {
      double n[3], ww[3];
      cross3(u, v, n);
      sub3(P[2], P[0], ww);
      const double q = dot3(ww, n);
      *ty = DType{DF_LL, {0, 1, 2, 3}};
      return q * q / dot3(n, n);
    }
  }
  DType t[4];
  double dd[4];
  dd[0] = seg_d2(P, 0, 2, 3, &t[0]);
  dd[1] = seg_d2(P, 1, 2, 3, &t[1]);
  dd[2] = seg_d2(P, 2, 0, 1, &t[2]);
  dd[3] = seg_d2(P, 3, 0, 1, &t[3]);
  int k = 0;
  for (int m = 1; m < 4; ++m)
    if (dd[m] < dd[k]) k = m;
  *ty = t[k];
  return dd[k];
}

__device__ __forceinline__ double pair_d2(int kind, const double P[4][3], DType* ty) {
  return kind == 0 ? pt_classify(P, ty) : ee_classify(P, ty);
}

// ---------------------------------------------------------------- derivatives of D
// [v]x
__device__ __forceinline__ void skew(const double* v, double S[3][3]) {
  S[0][0] = 0.0;   S[0][1] = -v[2]; S[0][2] = v[1];
  S[1][0] = v[2];  S[1][1] = 0.0;   S[1][2] = -v[0];
  S[2][0] = -v[1]; S[2][1] = v[0];  S[2][2] = 0.0;
}

// cross norm c(a,b) and its gradient/Hessian over (a,b) written into a space of dimension n at
// offsets oa, ob (g: n, H: n x n, accumulated)
__device__ __forceinline__ double crossnorm_acc(const double* a, const double* b, int n, int oa, int ob,
                                                double* g, double* H) {
  const double aa = dot3(a, a), bb = dot3(b, b), ab = dot3(a, b);
  for (int i = 0; i < 3; ++i) {
    g[oa + i] += 2.0 * bb * a[i] - 2.0 * ab * b[i];
    g[ob + i] += 2.0 * aa * b[i] - 2.0 * ab * a[i];
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double I = i == j ? 1.0 : 0.0;
      H[(oa + i) * n + oa + j] += 2.0 * bb * I - 2.0 * b[i] * b[j];
      H[(ob + i) * n + ob + j] += 2.0 * aa * I - 2.0 * a[i] * a[j];
      const double x = 4.0 * a[i] * b[j] - 2.0 * b[i] * a[j] - 2.0 * ab * I;
      H[(oa + i) * n + ob + j] += x;
      H[(ob + j) * n + oa + i] += x;
    }
  return aa * bb - ab * ab;
}

// triple product s = w.(e1 x e2) with gradient / Hessian over (w, e1, e2) = offsets 0, 3, 6 of a
// 9-dimensional space (written, not accumulated)
__device__ __forceinline__ double triple9(const double* w, const double* e1, const double* e2,
                                          double g[9], double H[81]) {
  double n[3], a[3], b[3];
  cross3(e1, e2, n);
  cross3(e2, w, a);
  cross3(w, e1, b);
  for (int i = 0; i < 3; ++i) {
    g[i] = n[i];
    g[3 + i] = a[i];
    g[6 + i] = b[i];
  }
  for (int k = 0; k < 81; ++k) H[k] = 0.0;
  double S1[3][3], S2[3][3], Sw[3][3];
  skew(e1, S1);
  skew(e2, S2);
  skew(w, Sw);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      H[i * 9 + 3 + j] = -S2[i][j];      // d2s / dw de1
      H[(3 + j) * 9 + i] = -S2[i][j];
      H[i * 9 + 6 + j] = S1[i][j];       // d2s / dw de2
      H[(6 + j) * 9 + i] = S1[i][j];
      H[(3 + i) * 9 + 6 + j] = -Sw[i][j];  // d2s / de1 de2
      H[(6 + j) * 9 + 3 + i] = -Sw[i][j];
    }
  return dot3(w, n);
}

// difference vector: plus point, minus point (slots 0..3)
struct DVec {
  int pl, mi;
};

// add (gradient, Hessian) over nd difference vectors to the 12-dimensional point space
__device__ __forceinline__ void dv_scatter(int nd, const DVec* dv, const double* gdv, const double* Hdv,
                                           double g[12], double H[144]) {
  const int n = 3 * nd;
  for (int a = 0; a < nd; ++a)
    for (int c = 0; c < 3; ++c) {
      g[3 * dv[a].pl + c] += gdv[3 * a + c];
      g[3 * dv[a].mi + c] -= gdv[3 * a + c];
    }
  for (int a = 0; a < nd; ++a)
    for (int b = 0; b < nd; ++b)
      for (int c = 0; c < 3; ++c)
        for (int e = 0; e < 3; ++e) {
          const double v = Hdv[(3 * a + c) * n + 3 * b + e];
          H[(3 * dv[a].pl + c) * 12 + 3 * dv[b].pl + e] += v;
          H[(3 * dv[a].pl + c) * 12 + 3 * dv[b].mi + e] -= v;
          H[(3 * dv[a].mi + c) * 12 + 3 * dv[b].pl + e] -= v;
          H[(3 * dv[a].mi + c) * 12 + 3 * dv[b].mi + e] += v;
        }
}

// D, grad D (12), Hess D (144) of the given closest-feature type
static __device__ __noinline__ double dist_derivs(const DType& t, const double P[4][3], double g[12], double H[144]) {
  for (int k = 0; k < 12; ++k) g[k] = 0.0;
  for (int k = 0; k < 144; ++k) H[k] = 0.0;
  if (t.f == DF_PP) {
    const int i = t.i[0], j = t.i[1];
    double u[3];
    sub3(P[i], P[j], u);
    DVec dv[1] = {{i, j}};
    double gd[3] = {2 * u[0], 2 * u[1], 2 * u[2]};
    double Hd[9] = {2, 0, 0, 0, 2, 0, 0, 0, 2};
    dv_scatter(1, dv, gd, Hd, g, H);
    return dot3(u, u);
  }
  if (t.f == DF_PE) {
    const int i = t.i[0], j = t.i[1], k = t.i[2];
    double w[3], e[3];
    sub3(P[i], P[j], w);
    sub3(P[k], P[j], e);
    double gN[6] = {0}, HN[36] = {0};
    const double N = crossnorm_acc(w, e, 6, 0, 3, gN, HN);
    const double L = dot3(e, e);
    const double D = N / L;
    // W = L(e): grad 2e on e, Hess 2I on e
    double gD[6], HD[36];
    for (int a = 0; a < 6; ++a) gD[a] = (gN[a] - (a >= 3 ? D * 2.0 * e[a - 3] : 0.0)) / L;
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b) {
        const double gLa = a >= 3 ? 2.0 * e[a - 3] : 0.0, gLb = b >= 3 ? 2.0 * e[b - 3] : 0.0;
        const double HL = (a >= 3 && a == b) ? 2.0 : 0.0;
        HD[a * 6 + b] = (HN[a * 6 + b] - D * HL - gD[a] * gLb - gLa * gD[b]) / L;
      }
    DVec dv[2] = {{i, j}, {k, j}};
    dv_scatter(2, dv, gD, HD, g, H);
    return D;
  }
  // PT or LL: D = s^2 / c(e1, e2)
  double w[3], e1[3], e2[3];
  DVec dv[3];
  if (t.f == DF_PT) {
    const int i = t.i[0], j = t.i[1], k = t.i[2], l = t.i[3];
    sub3(P[i], P[j], w);
    sub3(P[k], P[j], e1);
    sub3(P[l], P[j], e2);
    dv[0] = {i, j};
    dv[1] = {k, j};
    dv[2] = {l, j};
  } else {
    const int i = t.i[0], j = t.i[1], k = t.i[2], l = t.i[3];
    sub3(P[k], P[i], w);
    sub3(P[j], P[i], e1);
    sub3(P[l], P[k], e2);
    dv[0] = {k, i};
    dv[1] = {j, i};
    dv[2] = {l, k};
  }
  double gs[9], Hs[81];
  const double s = triple9(w, e1, e2, gs, Hs);
  double gW[9] = {0}, HW[81] = {0};
  const double W = crossnorm_acc(e1, e2, 9, 3, 6, gW, HW);
  const double D = s * s / W;
  double gD[9], HD[81];
  for (int a = 0; a < 9; ++a) gD[a] = (2.0 * s * gs[a] - D * gW[a]) / W;
  for (int a = 0; a < 9; ++a)
    for (int b = 0; b < 9; ++b)
      HD[a * 9 + b] = (2.0 * gs[a] * gs[b] + 2.0 * s * Hs[a * 9 + b] - D * HW[a * 9 + b] -
                       gD[a] * gW[b] - gW[a] * gD[b]) / W;
  dv_scatter(3, dv, gD, HD, g, H);
  return D;
}

// b(d) on D = d^2: value, dB/dD, d2B/dD2
__device__ __forceinline__ void barrier_D(double D, double dhat, double* b, double* bD, double* bDD) {
  const double d = sqrt(D);
  const double r = d - dhat;
  const double L = log(d / dhat);
  *b = -r * r * L;
  const double b1 = -2.0 * r * L - r * r / d;
  const double b2 = -2.0 * L - 4.0 * r / d + r * r / (d * d);
  *bD = b1 / (2.0 * d);
  *bDD = (b2 - b1 / d) / (4.0 * D);
}

// PSD projection of a symmetric n x n block (n <= 9): A <- V max(w, 0) V^T.
// GB300 issues FP64 at 1/64 of the FP32 rate, so the eigenbasis is found in two precisions:
//   1. cyclic Jacobi in FP32 gives an approximate eigenbasis Q (orthonormal to ~1e-7);
//   2. in FP64, Q is re-orthonormalised (modified Gram-Schmidt, two passes), so B = Q^T A Q is a
//      similarity, diagonal up to ~1e-7; one FP64 Jacobi sweep (plus a second if needed)
//      diagonalises it to FP64 accuracy, W;
//   3. V = Q W, w = diag(B), and the clamp is assembled in FP64.
// The result equals the FP64 eigen-clamp of A to FP64 round-off of the refinement.
static __device__ __noinline__ void psd_clamp(int n, double* A) {
  float a32[81], q32[81];
  for (int i = 0; i < n * n; ++i) a32[i] = (float)A[i];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) q32[i * n + j] = (i == j) ? 1.f : 0.f;
  for (int sweep = 0; sweep < 12; ++sweep) {
    float off = 0.f, dg = 0.f;
    for (int i = 0; i < n; ++i) {
      dg += a32[i * n + i] * a32[i * n + i];
      for (int j = i + 1; j < n; ++j) off += a32[i * n + j] * a32[i * n + j];
    }
    if (!(off > 1e-13f * dg)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const float apq = a32[p * n + q];
        if (fabsf(apq) <= 1e-9f * (fabsf(a32[p * n + p]) + fabsf(a32[q * n + q]))) continue;
        const float th = (a32[q * n + q] - a32[p * n + p]) / (2.f * apq);
        const float t = (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(th * th + 1.f));
        const float c = rsqrtf(t * t + 1.f), s = t * c;
        a32[p * n + p] -= t * apq;
        a32[q * n + q] += t * apq;
        a32[p * n + q] = a32[q * n + p] = 0.f;
        for (int r = 0; r < n; ++r) {
          if (r == p || r == q) continue;
          const float arp = a32[r * n + p], arq = a32[r * n + q];
          a32[r * n + p] = a32[p * n + r] = c * arp - s * arq;
          a32[r * n + q] = a32[q * n + r] = s * arp + c * arq;
        }
        for (int k = 0; k < n; ++k) {
          const float vkp = q32[k * n + p], vkq = q32[k * n + q];
          q32[k * n + p] = c * vkp - s * vkq;
          q32[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  // FP64: orthonormal Q (columns), then B = Q^T A Q
  double Q[81], T[81], B[81];
  for (int i = 0; i < n * n; ++i) Q[i] = (double)q32[i];
  for (int pass = 0; pass < 2; ++pass)
    for (int j = 0; j < n; ++j) {
      for (int k = 0; k < j; ++k) {
        double dp = 0.0;
        for (int i = 0; i < n; ++i) dp = fma(Q[i * n + k], Q[i * n + j], dp);
        for (int i = 0; i < n; ++i) Q[i * n + j] = fma(-dp, Q[i * n + k], Q[i * n + j]);
      }
      double nn = 0.0;
      for (int i = 0; i < n; ++i) nn = fma(Q[i * n + j], Q[i * n + j], nn);
      const double inv = rsqrt(nn);
      for (int i = 0; i < n; ++i) Q[i * n + j] *= inv;
    }
  for (int i = 0; i < n; ++i)  // T = A Q
    for (int j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc = fma(A[i * n + k], Q[k * n + j], acc);
      T[i * n + j] = acc;
    }
  for (int i = 0; i < n; ++i)  // B = Q^T T (upper triangle, mirrored)
    for (int j = i; j < n; ++j) {
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc = fma(Q[k * n + i], T[k * n + j], acc);
      B[i * n + j] = B[j * n + i] = acc;
    }
  // FP64 refinement sweeps on the nearly diagonal B, accumulating into Q
  for (int sweep = 0; sweep < 4; ++sweep) {
    double off = 0.0, dg = 0.0;
    for (int i = 0; i < n; ++i) {
      dg += B[i * n + i] * B[i * n + i];
      for (int j = i + 1; j < n; ++j) off += B[i * n + j] * B[i * n + j];
    }
    if (!(off > 1e-28 * dg)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double bpq = B[p * n + q];
        if (fabs(bpq) <= 1e-18 * (fabs(B[p * n + p]) + fabs(B[q * n + q]))) continue;
        const double th = (B[q * n + q] - B[p * n + p]) / (2.0 * bpq);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double c = rsqrt(t * t + 1.0), s = t * c;
        B[p * n + p] -= t * bpq;
        B[q * n + q] += t * bpq;
        B[p * n + q] = B[q * n + p] = 0.0;
        for (int r = 0; r < n; ++r) {
          if (r == p || r == q) continue;
          const double brp = B[r * n + p], brq = B[r * n + q];
          B[r * n + p] = B[p * n + r] = c * brp - s * brq;
          B[r * n + q] = B[q * n + r] = s * brp + c * brq;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = Q[k * n + p], vkq = Q[k * n + q];
          Q[k * n + p] = c * vkp - s * vkq;
          Q[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  double w[9];
  for (int i = 0; i < n; ++i) w[i] = fmax(B[i * n + i], 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) {
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc = fma(Q[i * n + k] * w[k], Q[j * n + k], acc);
      A[i * n + j] = A[j * n + i] = acc;
    }
}

// Projected barrier block of a pair with a single free point: the barrier depends on that point
// only through d, so its Hessian is b''(d) u u^T + b'(d) grad^2 d with u = grad d; grad^2 d is
// PSD-orthogonal to u and b' < 0, so the PSD projection keeps b''(d) u u^T (b'' > 0 inside
// dhat).  H3 = kappa-free 3x3 block, from gD = grad of D = d^2 restricted to the point.
__device__ __forceinline__ void single_point_block(double bpp, const double gD[3], double H3[9]) {
  const double n2 = gD[0] * gD[0] + gD[1] * gD[1] + gD[2] * gD[2];
  const double k = n2 > 0.0 ? fmax(bpp, 0.0) / n2 : 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) H3[3 * i + j] = k * gD[i] * gD[j];
}

// Barrier of one pair (kind 0: point-triangle, 1: edge-edge with mollifier threshold eps_x):
// value, gradient (12) and Hessian (144) in point space.  Returns false when d >= dhat.
// Optional outputs: the points the value depends on (bit mask), b''(d) and grad D (12).
static __device__ __noinline__ bool pair_barrier_derivs(int kind, const double P[4][3], double dhat, double eps_x,
                                                        double* bv, double g[12], double H[144], DType* tyo,
                                                        int* involved = nullptr, double* bpp = nullptr,
                                                        double* gDo = nullptr) {
  DType ty;
  const double D0 = pair_d2(kind, P, &ty);
  if (tyo) *tyo = ty;
  if (!(D0 < dhat * dhat)) return false;
  double gD[12], HD[144];
  const double D = dist_derivs(ty, P, gD, HD);
  double b, bD, bDD;
  barrier_D(D, dhat, &b, &bD, &bDD);
  if (involved) {
    const int np = ty.f == DF_PP ? 2 : (ty.f == DF_PE ? 3 : 4);
    int m = 0;
    for (int k = 0; k < np; ++k) m |= 1 << ty.i[k];
    *involved = m;
  }
  if (bpp) {
    const double d = sqrt(D), r = d - dhat;
    *bpp = -2.0 * log(d / dhat) - 4.0 * r / d + r * r / (d * d);
  }
  if (gDo)
    for (int k = 0; k < 12; ++k) gDo[k] = gD[k];
  for (int a = 0; a < 12; ++a) g[a] = bD * gD[a];
  for (int a = 0; a < 12; ++a)
    for (int c = 0; c < 12; ++c) H[a * 12 + c] = bDD * gD[a] * gD[c] + bD * HD[a * 12 + c];
  if (kind == 1) {
    double ea[3], eb[3];
    sub3(P[1], P[0], ea);
    sub3(P[3], P[2], eb);
    double gc6[6] = {0}, Hc6[36] = {0};
    const double c = crossnorm_acc(ea, eb, 6, 0, 3, gc6, Hc6);
    if (c < eps_x) {
      if (involved) *involved = 0xF;  // the mollifier couples all four points
      const double q = c / eps_x;
      const double m = (2.0 - q) * q;
      const double m1 = 2.0 * (1.0 - q) / eps_x;
      const double m2 = -2.0 / (eps_x * eps_x);
      double gc[12] = {0}, Hc[144];
      for (int k = 0; k < 144; ++k) Hc[k] = 0.0;
      DVec dv[2] = {{1, 0}, {3, 2}};
      dv_scatter(2, dv, gc6, Hc6, gc, Hc);
      // B = m b
      for (int a = 0; a < 12; ++a)
        for (int k = 0; k < 12; ++k) {
          const double gma = m1 * gc[a], gmk = m1 * gc[k];
          const double Hm = m2 * gc[a] * gc[k] + m1 * Hc[a * 12 + k];
          H[a * 12 + k] = m * H[a * 12 + k] + gma * g[k] + g[a] * gmk + b * Hm;
        }
      for (int a = 0; a < 12; ++a) g[a] = m * g[a] + b * m1 * gc[a];
      b *= m;
    }
  }
  *bv = b;
  return true;
}

// Additive CCD along P + t dP: 0 no hit in [0, tc], 1 hit (toi), 2 iteration cap.
static __device__ __noinline__ int accd_pair(int kind, const double P0[4][3], const double dP0[4][3], double s,
                                      double tc, int maxit, double* toi) {
  double P[4][3], dP[4][3], mean[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < 4; ++k)
    for (int c = 0; c < 3; ++c) mean[c] += 0.25 * dP0[k][c];
  double nrm[4];
  for (int k = 0; k < 4; ++k) {
    for (int c = 0; c < 3; ++c) {
      dP[k][c] = dP0[k][c] - mean[c];
      P[k][c] = P0[k][c];
    }
    nrm[k] = sqrt(dot3(dP[k], dP[k]));
  }
  const double lp = kind == 0 ? nrm[0] + fmax(nrm[1], fmax(nrm[2], nrm[3]))
                              : fmax(nrm[0], nrm[1]) + fmax(nrm[2], nrm[3]);
  if (lp == 0.0) return 0;
  DType ty;
  double d = sqrt(pair_d2(kind, P, &ty));
  if (!(d > 0.0)) {
    *toi = 0.0;
    return 1;
  }
  const double gap = s * d;
  double t = 0.0, tl = (1.0 - s) * d / lp;
  for (int it = 0; it < maxit; ++it) {
    for (int k = 0; k < 4; ++k)
      for (int c = 0; c < 3; ++c) P[k][c] += tl * dP[k][c];
    d = sqrt(pair_d2(kind, P, &ty));
    if (t > 0.0 && d < gap) {
      *toi = t;
      return 1;
    }
    t += tl;
    if (t > tc) return 0;
    tl = 0.9 * d / lp;
  }
  return 2;
}

// ---------------------------------------------------------------- pairs of the batch
// points of a candidate pair (slots: PT [gel v, ind tri], TP [ind v, gel tri], EE [gel edge,
// ind edge]); gel positions at x + alpha p, indenter at iv_cur (or iv_prev); `rows` gets the
// gel row of each slot or -1 for indenter slots.
__device__ __forceinline__ void pair_points(const Dev& d, const int4& pr, double alpha, bool prev_ind,
                                            double P[4][3], int rows[4]) {
  const double4_32a* ind = prev_ind ? d.iv_prev : d.iv_cur;
  auto gel = [&](int slot, int row) {
    const double4_32a x = d.x[row];
    if (alpha != 0.0) {
      const double4_32a p = d.p[row];
      P[slot][0] = x.x + alpha * p.x;
      P[slot][1] = x.y + alpha * p.y;
      P[slot][2] = x.z + alpha * p.z;
    } else {
      P[slot][0] = x.x;
      P[slot][1] = x.y;
      P[slot][2] = x.z;
    }
    rows[slot] = row;
  };
  auto indv = [&](int slot, int id) {
    const double4_32a q = ind[id];
    P[slot][0] = q.x;
    P[slot][1] = q.y;
    P[slot][2] = q.z;
    rows[slot] = -1;
  };
  if (pr.x == PAIR_PT) {
    gel(0, d.sv[pr.y]);
    const int4 t = d.it[pr.z];
    indv(1, t.x);
    indv(2, t.y);
    indv(3, t.z);
  } else if (pr.x == PAIR_TP) {
    indv(0, pr.z);
    const int4 t = d.st[pr.y];
    gel(1, t.x);
    gel(2, t.y);
    gel(3, t.z);
  } else {
    const int2 e = d.se[pr.y];
    gel(0, e.x);
    gel(1, e.y);
    const int2 f = d.ie[pr.z];
    indv(2, f.x);
    indv(3, f.y);
  }
}

__device__ __forceinline__ double pair_eps_x(const Dev& d, const int4& pr) {
  return pr.x == PAIR_EE ? 1e-3 * d.se_len2[pr.y] * d.ie_len2[pr.z] : 0.0;
}

// barrier energy (without kappa) of a pair at its current points; +inf when d <= 0
__device__ __forceinline__ double pair_energy(int kind, const double P[4][3], double dhat, double eps_x,
                                              double* dist) {
  DType ty;
  const double D = pair_d2(kind, P, &ty);
  *dist = sqrt(D);
  if (!(D > 0.0)) return CUDART_INF;
  if (!(D < dhat * dhat)) return 0.0;
  const double dd = sqrt(D);
  const double r = dd - dhat;
  double b = -r * r * log(dd / dhat);
  if (kind == 1) {
    double ea[3], eb[3], n[3];
    sub3(P[1], P[0], ea);
    sub3(P[3], P[2], eb);
    cross3(ea, eb, n);
    const double c = dot3(n, n);
    if (c < eps_x) {
      const double q = c / eps_x;
      b *= (2.0 - q) * q;
    }
  }
  return b;
}

}  // namespace txg

// FP64 CPU ORACLE of one implicit time step of a gelpad pressed by a kinematic rigid indenter,
// solved as an incremental-potential-contact (IPC) minimisation.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference the CUDA library is checked
// against.  Only the tests, the smoke check and the benchmark's CPU-baseline leg load it; the
// product path never does.  It shares no code with the CUDA library (no headers, no helpers, no
// generated tables).  Every derivative here comes from a forward-mode second-order automatic
// differentiation type applied to the plain energy formulas, never from hand-derived gradient or
// Hessian expressions, so a mistake in the CUDA library's hand-derived formulas cannot be
// reproduced here.
//
// What is computed (TacEx, Sec. "General GIPC Simulation Pipeline": the GIPC solver moves the
// free gel vertices for one step while attachment/kinematic targets are prescribed; the solver
// is IPC [Li et al. 2020, cited by TacEx], inversion- and intersection-free per TacEx App. A
// "Choice of the Simulation Methods"):
//
//   E(x) = sum_i m_i |x_i - xt_i|^2 / (2 h^2)                       inertia, xt = x_n + h v_n
//        + sum_t V_t Psi(F_t)                                      compressible Neo-Hookean
//        + kappa sum_k m_k b(d_k)                                  log barrier, 0 < d_k < dhat
//
//   Psi(F) = mu/2 (tr F^T F - 3) - mu ln J + lambda/2 (ln J)^2,    J = det F
//   b(d)   = -(d - dhat)^2 ln(d / dhat)
//   m_k    = IPC edge-edge mollifier (1 for point-triangle pairs)
//
// plus, when a friction coefficient mu_f > 0 is set, IPC's lagged dissipative friction (Li et
// al. 2020, Sec. 5): for every pair in contact at the start of the (sub)step (gel at x_n,
// indenter at its previous pose)
//   D_k(x) = mu_f lambda_k f0(|u_k(x)|),  u_k = T_k^T (relative displacement of the closest points
//   over the step), lambda_k = kappa m_k |b'(d_k)| (the pair's normal force), T_k an orthonormal
//   basis of the tangent plane, all taken at the start and held fixed (lagged) during the solve;
//   f0(y) = -y^3 / (3 e^2) + y^2 / e + e / 3 below e = eps_v h and f0(y) = y above (f0' = f1 is 1
//   when sliding faster than eps_v, so the force is mu_f lambda_k: Coulomb; below it a stiff
//   spring: static friction).
//
// minimised by projected Newton: per-element PSD-projected Hessians, direction from the linear
// system on the free degrees of freedom, step capped by additive CCD (ACCD, Li et al. 2021 "C-IPC")
// and by det F > 0, backtracking on E.  Readings of points the paper leaves open are marked
// READING and listed in the design notes:
//   * mass lumping m_i = rho * sum_{t ni i} V_t / 4;
//   * kappa = 0 means kappa = E * (mean rest length of the gel surface edges);
//   * contact primitives: gel surface vertices vs indenter triangles, indenter vertices vs gel
//     surface triangles, gel surface edges vs indenter edges (no self-contact within a body);
//     a tet mesh of several connected components (bodies) also pairs the surfaces of different
//     bodies (surface vertex vs surface triangle, surface edge vs surface edge: GIPC's
//     soft-to-soft contact), without friction and outside the indenter force; body 0 (the body
//     of the first vertex in a tet) is the gelpad of the readouts;
//   * distance classification: the closest feature pair (vertex/edge/face) of the primitive pair;
//   * EE mollifier threshold eps_x = 1e-3 |a1-a0|^2 |b1-b0|^2 at rest;
//   * ACCD: C-IPC's additive CCD with s = 0.1 (the gap may shrink to 10%), t_c = 1, thickness 0,
//     over the pairs whose swept bounding boxes come within dhat of each other;
//   * line search: alpha_0 = min(1, ACCD time of impact), halving until E(x + alpha p) <= E(x)
//     with every tet keeping det F > 0 (a tet with det F <= 0 has E = +inf); if halving reaches
//     alpha < 1e-12 alpha_0 and the model decrease -g.p is below 1e-10 |E| the iterate counts as
//     converged (stationary to FP64 energy resolution), otherwise the step fails;
//   * convergence: ||p||_inf / h < newton_tol * (rest bounding-box diagonal);
//   * kinematic indenter: it is placed at the step's target pose before the solve; if its linear
//     sweep from the previous pose against the gel at x_n has an ACCD hit (or any distance <= 0
//     after placement), the step is split into two half steps (pose midpoint, dt/2 each),
//     recursively up to a maximum depth.
//
// The linear system is solved with a Jacobi-preconditioned conjugate gradient to a tight relative
// residual (default 1e-10); any accurate solver gives the same minimiser.
//
// The elastic energy is evaluated in the displacement-gradient form H = F - I,
//   Psi = mu/2 |H|^2 - mu (c2 + c3) + mu (j - ln(1+j)) + lambda/2 ln(1+j)^2,
//   j = J - 1 = tr H + c2 + c3, c2 = sum of principal 2x2 minors of H, c3 = det H,
// which is the same function as the definition above (det(I+H) = 1 + tr H + c2 + c3) but free of
// the O(1) cancellation the literal form has near the rest state; the line search needs E to
// resolve energy decreases far below E itself.
//
// Threads: when built with OpenMP, the loops over tets, contact pairs, broad-phase primitives and
// matrix rows run in parallel, but every such loop only writes per-element results; all sums and
// minima over elements are then taken serially in index order.  The results are therefore
// bitwise identical for any thread count (or_set_threads), and equal to a one-thread run.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <map>
#include <utility>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double INF = std::numeric_limits<double>::infinity();

// ------------------------------------------------------------------------------------------
// Forward-mode second-order AD: value, gradient and full Hessian w.r.t. N seeded inputs.
// ------------------------------------------------------------------------------------------
template <int N>
struct AD {
  double v;
  double g[N];
  double h[N][N];
  AD() {}
  AD(double c) : v(c) {  // NOLINT: implicit on purpose (constants mix with variables)
    std::memset(g, 0, sizeof(g));
    std::memset(h, 0, sizeof(h));
  }
};

template <int N>
AD<N> ad_var(double c, int i) {
  AD<N> r(c);
  r.g[i] = 1.0;
  return r;
}

// r = f(a) with f(a.v) = f0, f'(a.v) = f1, f''(a.v) = f2
template <int N>
AD<N> ad_chain(const AD<N>& a, double f0, double f1, double f2) {
  AD<N> r;
  r.v = f0;
  for (int i = 0; i < N; ++i) r.g[i] = f1 * a.g[i];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) r.h[i][j] = f1 * a.h[i][j] + f2 * a.g[i] * a.g[j];
  return r;
}

template <int N>
AD<N> operator+(const AD<N>& a, const AD<N>& b) {
  AD<N> r;
  r.v = a.v + b.v;
  for (int i = 0; i < N; ++i) r.g[i] = a.g[i] + b.g[i];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) r.h[i][j] = a.h[i][j] + b.h[i][j];
  return r;
}
template <int N>
AD<N> operator-(const AD<N>& a, const AD<N>& b) {
  AD<N> r;
  r.v = a.v - b.v;
  for (int i = 0; i < N; ++i) r.g[i] = a.g[i] - b.g[i];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) r.h[i][j] = a.h[i][j] - b.h[i][j];
  return r;
}
template <int N>
AD<N> operator-(const AD<N>& a) {
  return AD<N>(0.0) - a;
}
template <int N>
AD<N> operator*(const AD<N>& a, const AD<N>& b) {
  AD<N> r;
  r.v = a.v * b.v;
  for (int i = 0; i < N; ++i) r.g[i] = a.v * b.g[i] + b.v * a.g[i];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      r.h[i][j] = a.v * b.h[i][j] + b.v * a.h[i][j] + a.g[i] * b.g[j] + b.g[i] * a.g[j];
  return r;
}
template <int N>
AD<N> operator*(double c, const AD<N>& a) {
  AD<N> r;
  r.v = c * a.v;
  for (int i = 0; i < N; ++i) r.g[i] = c * a.g[i];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) r.h[i][j] = c * a.h[i][j];
  return r;
}
template <int N>
AD<N> operator*(const AD<N>& a, double c) {
  return c * a;
}
template <int N>
AD<N> operator-(double c, const AD<N>& a) {
  return AD<N>(c) - a;
}
template <int N>
AD<N> operator+(const AD<N>& a, double c) {
  AD<N> r = a;
  r.v += c;
  return r;
}
template <int N>
AD<N> operator-(const AD<N>& a, double c) {
  AD<N> r = a;
  r.v -= c;
  return r;
}
template <int N>
AD<N> ad_inv(const AD<N>& a) {
  double iv = 1.0 / a.v;
  return ad_chain(a, iv, -iv * iv, 2.0 * iv * iv * iv);
}
template <int N>
AD<N> operator/(const AD<N>& a, const AD<N>& b) {
  return a * ad_inv(b);
}
template <int N>
AD<N> operator/(const AD<N>& a, double c) {
  return (1.0 / c) * a;
}

// plain-double versions of the elementary functions, overloaded for AD below
double vsqrt(double a) { return std::sqrt(a); }
double vlog(double a) { return std::log(a); }
double vlog1p(double a) { return std::log1p(a); }
double value(double a) { return a; }

// j - ln(1 + j), accurately for small |j| (alternating Taylor series), directly otherwise
double jml_value(double j) {
  if (std::fabs(j) < 0.1) {
    double s = 0.0, p = j * j;
    for (int k = 2; k <= 22; ++k) {
      s += ((k & 1) ? -p : p) / k;
      p *= j;
    }
    return s;
  }
  return j - std::log1p(j);
}
double vjml(double j) { return jml_value(j); }

template <int N>
AD<N> vsqrt(const AD<N>& a) {
  double s = std::sqrt(a.v);
  return ad_chain(a, s, 0.5 / s, -0.25 / (s * a.v));
}
template <int N>
AD<N> vlog(const AD<N>& a) {
  return ad_chain(a, std::log(a.v), 1.0 / a.v, -1.0 / (a.v * a.v));
}
template <int N>
AD<N> vlog1p(const AD<N>& a) {
  double q = 1.0 + a.v;
  return ad_chain(a, std::log1p(a.v), 1.0 / q, -1.0 / (q * q));
}
template <int N>
AD<N> vjml(const AD<N>& a) {  // d/dj (j - ln(1+j)) = j/(1+j), second derivative 1/(1+j)^2
  double q = 1.0 + a.v;
  return ad_chain(a, jml_value(a.v), a.v / q, 1.0 / (q * q));
}
template <int N>
double value(const AD<N>& a) {
  return a.v;
}

// ------------------------------------------------------------------------------------------
// small vector helpers (templated so the same formula serves values and AD numbers)
// ------------------------------------------------------------------------------------------
template <class T>
void sub3(const T a[3], const T b[3], T r[3]) {
  for (int i = 0; i < 3; ++i) r[i] = a[i] - b[i];
}
template <class T>
T dot3(const T a[3], const T b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
template <class T>
void cross3(const T a[3], const T b[3], T r[3]) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

// ------------------------------------------------------------------------------------------
// Neo-Hookean energy density (IPC's compressible variant) in terms of H = F - I (row-major).
// Returns false when J <= 0 (energy undefined / +inf).
// ------------------------------------------------------------------------------------------
template <class T>
bool psi_of_H(const T H[9], double mu, double lam, T* out) {
  T tr = H[0] + H[4] + H[8];
  T nrm2 = H[0] * H[0];
  for (int k = 1; k < 9; ++k) nrm2 = nrm2 + H[k] * H[k];
  T c2 = H[0] * H[4] - H[1] * H[3] + H[0] * H[8] - H[2] * H[6] + H[4] * H[8] - H[5] * H[7];
  T c3 = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
         H[2] * (H[3] * H[7] - H[4] * H[6]);
  T j = tr + c2 + c3;  // J - 1
  if (!(value(j) > -1.0)) return false;
  T L = vlog1p(j);
  *out = 0.5 * mu * nrm2 - mu * (c2 + c3) + mu * vjml(j) + 0.5 * lam * (L * L);
  return true;
}

// 3x3 inverse (row-major), returns determinant
double inv3(const double A[9], double R[9]) {
  double c00 = A[4] * A[8] - A[5] * A[7];
  double c01 = A[5] * A[6] - A[3] * A[8];
  double c02 = A[3] * A[7] - A[4] * A[6];
  double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  double id = 1.0 / det;
  R[0] = c00 * id;
  R[1] = (A[2] * A[7] - A[1] * A[8]) * id;
  R[2] = (A[1] * A[5] - A[2] * A[4]) * id;
  R[3] = c01 * id;
  R[4] = (A[0] * A[8] - A[2] * A[6]) * id;
  R[5] = (A[2] * A[3] - A[0] * A[5]) * id;
  R[6] = c02 * id;
  R[7] = (A[1] * A[6] - A[0] * A[7]) * id;
  R[8] = (A[0] * A[4] - A[1] * A[3]) * id;
  return det;
}

// ------------------------------------------------------------------------------------------
// Symmetric eigen-decomposition by cyclic Jacobi rotations; PSD projection clamps eigenvalues < 0.
// ------------------------------------------------------------------------------------------
void jacobi_eig(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& V) {
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += A[i * n + i] * A[i * n + i];
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    }
    if (off <= 1e-32 * diag || off == 0.0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        double app = A[p * n + p], aqq = A[q * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
}

void psd_project(int n, double* M) {
  std::vector<double> A(M, M + n * n), w, V;
  for (int i = 0; i < n; ++i)  // symmetrise
    for (int j = i + 1; j < n; ++j) A[i * n + j] = A[j * n + i] = 0.5 * (A[i * n + j] + A[j * n + i]);
  jacobi_eig(n, A, w, V);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k)
        if (w[k] > 0.0) s += V[i * n + k] * w[k] * V[j * n + k];
      M[i * n + j] = s;
    }
}

// ------------------------------------------------------------------------------------------
// Tetrahedron: rest shape data, energy, gradient and (PSD-projected) Hessian.
// ------------------------------------------------------------------------------------------
struct TetRest {
  double Dminv[9];  // inverse of Dm = [X1-X0 | X2-X0 | X3-X0] (row-major)
  double vol;       // rest volume det(Dm)/6
};

bool tet_rest(const double X[4][3], TetRest* r) {
  double Dm[9];
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 3; ++a) Dm[i * 3 + a] = X[a + 1][i] - X[0][i];
  double det = inv3(Dm, r->Dminv);
  r->vol = det / 6.0;
  return det > 0.0;
}

// displacement gradient H = Du Dm^{-1}, Du = [u1-u0 | u2-u0 | u3-u0], u = x - X
void tet_H(const TetRest& tr, const double X[4][3], const double x[4][3], double H[9]) {
  double Du[9];
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 3; ++a) Du[i * 3 + a] = (x[a + 1][i] - X[a + 1][i]) - (x[0][i] - X[0][i]);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += Du[i * 3 + k] * tr.Dminv[k * 3 + j];
      H[i * 3 + j] = s;
    }
}

double tet_energy(const TetRest& tr, const double X[4][3], const double x[4][3], double mu, double lam) {
  double H[9], psi;
  tet_H(tr, X, x, H);
  if (!psi_of_H(H, mu, lam, &psi)) return INF;
  return tr.vol * psi;
}

// dF_ij / dx_{a,l} = delta_il * D[a][j]
void tet_D(const TetRest& tr, double D[4][3]) {
  for (int j = 0; j < 3; ++j) {
    D[0][j] = 0.0;
    for (int a = 1; a < 4; ++a) {
      D[a][j] = tr.Dminv[(a - 1) * 3 + j];
      D[0][j] -= D[a][j];
    }
  }
}

// energy, gradient (12) and Hessian (12x12) of V*Psi; projection of d2Psi/dF2 (9x9) if asked
bool tet_derivs(const TetRest& tr, const double X[4][3], const double x[4][3], double mu, double lam,
                bool project, double* e, double g[12], double Hs[144]) {
  double H[9];
  tet_H(tr, X, x, H);
  AD<9> Hv[9];
  for (int k = 0; k < 9; ++k) Hv[k] = ad_var<9>(H[k], k);
  AD<9> psi;
  if (!psi_of_H(Hv, mu, lam, &psi)) return false;
  double C[81];
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 9; ++j) C[i * 9 + j] = psi.h[i][j];
  if (project) psd_project(9, C);
  double D[4][3];
  tet_D(tr, D);
  // B: 9 x 12, B[(i,j)][(a,l)] = delta_il D[a][j]
  double B[9][12];
  std::memset(B, 0, sizeof(B));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int a = 0; a < 4; ++a) B[i * 3 + j][a * 3 + i] = D[a][j];
  *e = tr.vol * psi.v;
  for (int c = 0; c < 12; ++c) {
    double s = 0.0;
    for (int r = 0; r < 9; ++r) s += B[r][c] * psi.g[r];
    g[c] = tr.vol * s;
  }
  double CB[9][12];
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 12; ++c) {
      double s = 0.0;
      for (int k = 0; k < 9; ++k) s += C[r * 9 + k] * B[k][c];
      CB[r][c] = s;
    }
  for (int a = 0; a < 12; ++a)
    for (int b = 0; b < 12; ++b) {
      double s = 0.0;
      for (int r = 0; r < 9; ++r) s += B[r][a] * CB[r][b];
      Hs[a * 12 + b] = tr.vol * s;
    }
  return true;
}

// ------------------------------------------------------------------------------------------
// Distances between primitives.  Four point-index slots P[0..3].  A distance "type" names the
// closest-feature pair and which smooth squared-distance formula applies.
// ------------------------------------------------------------------------------------------
enum Formula { F_PP = 0, F_PE = 1, F_PT = 2, F_LL = 3 };
struct DType {
  int f;
  int i[4];
};

template <class T>
T d2_pp(const T a[3], const T b[3]) {
  T u[3];
  sub3(a, b, u);
  return dot3(u, u);
}
// point p to the line through e0, e1
template <class T>
T d2_pe(const T p[3], const T e0[3], const T e1[3]) {
  T a[3], b[3], c[3], e[3];
  sub3(e0, p, a);
  sub3(e1, p, b);
  cross3(a, b, c);
  sub3(e1, e0, e);
  return dot3(c, c) / dot3(e, e);
}
// point p to the plane through t0, t1, t2
template <class T>
T d2_pt(const T p[3], const T t0[3], const T t1[3], const T t2[3]) {
  T e1[3], e2[3], n[3], w[3];
  sub3(t1, t0, e1);
  sub3(t2, t0, e2);
  cross3(e1, e2, n);
  sub3(p, t0, w);
  T s = dot3(w, n);
  return s * s / dot3(n, n);
}
// line through a0, a1 to line through b0, b1
template <class T>
T d2_ll(const T a0[3], const T a1[3], const T b0[3], const T b1[3]) {
  T ea[3], eb[3], n[3], w[3];
  sub3(a1, a0, ea);
  sub3(b1, b0, eb);
  cross3(ea, eb, n);
  sub3(b0, a0, w);
  T s = dot3(w, n);
  return s * s / dot3(n, n);
}

template <class T>
T d2_of_type(const DType& t, const T P[4][3]) {
  switch (t.f) {
    case F_PP: return d2_pp(P[t.i[0]], P[t.i[1]]);
    case F_PE: return d2_pe(P[t.i[0]], P[t.i[1]], P[t.i[2]]);
    case F_PT: return d2_pt(P[t.i[0]], P[t.i[1]], P[t.i[2]], P[t.i[3]]);
    default: return d2_ll(P[t.i[0]], P[t.i[1]], P[t.i[2]], P[t.i[3]]);
  }
}

// closest feature of segment (a, b) to point p: interior -> PE, else the nearer endpoint -> PP
DType seg_type(const double P[4][3], int ip, int ia, int ib) {
  double e[3], w[3];
  sub3(P[ib], P[ia], e);
  sub3(P[ip], P[ia], w);
  double t = dot3(w, e) / dot3(e, e);
  if (t <= 0.0) return DType{F_PP, {ip, ia, -1, -1}};
  if (t >= 1.0) return DType{F_PP, {ip, ib, -1, -1}};
  return DType{F_PE, {ip, ia, ib, -1}};
}

// point P[0] vs triangle P[1..3]: the face interior if the projection lands strictly inside,
// otherwise the nearest of the three edges (each classified as above)
DType pt_type(const double P[4][3]) {
  double e1[3], e2[3], w[3];
  sub3(P[2], P[1], e1);
  sub3(P[3], P[1], e2);
  sub3(P[0], P[1], w);
  double a = dot3(e1, e1), b = dot3(e1, e2), c = dot3(e2, e2), d = dot3(e1, w), f = dot3(e2, w);
  double det = a * c - b * b;
  double l1 = (c * d - b * f) / det, l2 = (a * f - b * d) / det;
  if (l1 > 0.0 && l2 > 0.0 && l1 + l2 < 1.0) return DType{F_PT, {0, 1, 2, 3}};
  DType best{};
  double bd = INF;
  const int E[3][2] = {{1, 2}, {2, 3}, {3, 1}};
  for (auto& ed : E) {
    DType t = seg_type(P, 0, ed[0], ed[1]);
    double v = d2_of_type(t, P);
    if (v < bd) {
      bd = v;
      best = t;
    }
  }
  return best;
}

// segment P[0]P[1] vs segment P[2]P[3]: both closest points interior -> LL, otherwise the
// nearest of the four endpoint-vs-segment problems
DType ee_type(const double P[4][3]) {
  double u[3], v[3], w[3];
  sub3(P[1], P[0], u);
  sub3(P[3], P[2], v);
  sub3(P[0], P[2], w);
  double a = dot3(u, u), b = dot3(u, v), c = dot3(v, v), d = dot3(u, w), e = dot3(v, w);
  double den = a * c - b * b;
  if (den > 1e-14 * a * c) {
    double s = (b * e - c * d) / den, t = (a * e - b * d) / den;
    if (s > 0.0 && s < 1.0 && t > 0.0 && t < 1.0) return DType{F_LL, {0, 1, 2, 3}};
  }
  DType cands[4] = {seg_type(P, 0, 2, 3), seg_type(P, 1, 2, 3), seg_type(P, 2, 0, 1),
                    seg_type(P, 3, 0, 1)};
  DType best{};
  double bd = INF;
  for (auto& t : cands) {
    double vv = d2_of_type(t, P);
    if (vv < bd) {
      bd = vv;
      best = t;
    }
  }
  return best;
}

enum PairKind { K_PT = 0, K_EE = 1 };

DType classify(int kind, const double P[4][3]) { return kind == K_PT ? pt_type(P) : ee_type(P); }

double pair_d2(int kind, const double P[4][3]) { return d2_of_type(classify(kind, P), P); }

// barrier b(d) = -(d - dhat)^2 ln(d/dhat) on d^2, times the EE mollifier
template <class T>
T pair_barrier(int kind, const DType& ty, const T P[4][3], double dhat, double eps_x) {
  T D = d2_of_type(ty, P);
  T d = vsqrt(D);
  T dd = d - dhat;
  T b = -(dd * dd) * vlog(d / dhat);
  if (kind == K_EE) {
    T ea[3], eb[3], n[3];
    sub3(P[1], P[0], ea);
    sub3(P[3], P[2], eb);
    cross3(ea, eb, n);
    T c = dot3(n, n);
    if (value(c) < eps_x) {
      T q = c / eps_x;
      b = b * ((2.0 - q) * q);  // mollifier -c^2/eps^2 + 2c/eps
    }
  }
  return b;
}

// ------------------------------------------------------------------------------------------
// Additive CCD (C-IPC, Li, Kaufman & Jiang 2021): conservative time of impact along linear
// trajectories P + t dP, t in [0, tc].  Returns 0 = no hit in [0, tc], 1 = hit (toi set),
// 2 = iteration cap.  Thickness 0.
// ------------------------------------------------------------------------------------------
int accd(int kind, const double P0[4][3], const double dP0[4][3], double s, double tc, int maxit,
         double* toi) {
  double P[4][3], dP[4][3], mean[3] = {0, 0, 0};
  for (int k = 0; k < 4; ++k)
    for (int i = 0; i < 3; ++i) mean[i] += 0.25 * dP0[k][i];
  for (int k = 0; k < 4; ++k)
    for (int i = 0; i < 3; ++i) {
      dP[k][i] = dP0[k][i] - mean[i];
      P[k][i] = P0[k][i];
    }
  double n[4];
  for (int k = 0; k < 4; ++k) n[k] = std::sqrt(dot3(dP[k], dP[k]));
  double lp = kind == K_PT ? n[0] + std::max(n[1], std::max(n[2], n[3]))
                           : std::max(n[0], n[1]) + std::max(n[2], n[3]);
  if (lp == 0.0) return 0;
  double d = std::sqrt(pair_d2(kind, P));
  if (!(d > 0.0)) {
    *toi = 0.0;
    return 1;
  }
  double g = s * d;
  double t = 0.0;
  double tl = (1.0 - s) * d / lp;
  for (int it = 0; it < maxit; ++it) {
    for (int k = 0; k < 4; ++k)
      for (int i = 0; i < 3; ++i) P[k][i] += tl * dP[k][i];
    d = std::sqrt(pair_d2(kind, P));
    if (t > 0.0 && d < g) {
      *toi = t;
      return 1;
    }
    t += tl;
    if (t > tc) return 0;
    tl = 0.9 * d / lp;
  }
  return 2;
}

// ------------------------------------------------------------------------------------------
// The gel.
// ------------------------------------------------------------------------------------------
enum Status {
  OK = 0, ERR_ARG = 1, ERR_OOM = 2, ERR_MESH_INVERTED = 3, ERR_INFEASIBLE = 4,
  ERR_NEWTON_MAXIT = 5, ERR_PCG_MAXIT = 6, ERR_LINESEARCH = 7, ERR_CCD_MAXIT = 8
};

struct Box {
  double lo[3], hi[3];
};
Box box_of(const double* const* pts, int n) {
  Box b;
  for (int i = 0; i < 3; ++i) {
    b.lo[i] = INF;
    b.hi[i] = -INF;
  }
  for (int k = 0; k < n; ++k)
    for (int i = 0; i < 3; ++i) {
      b.lo[i] = std::min(b.lo[i], pts[k][i]);
      b.hi[i] = std::max(b.hi[i], pts[k][i]);
    }
  return b;
}
// the candidate rule: boxes within `pad` of each other along every axis
bool near_boxes(const Box& a, const Box& b, double pad) {
  for (int i = 0; i < 3; ++i)
    if (a.lo[i] - pad > b.hi[i] || b.lo[i] - pad > a.hi[i]) return false;
  return true;
}

struct Gel {
  int N = 0, T = 0, M = 0, K = 0;
  std::vector<double> X;     // rest positions 3N
  std::vector<int> tets;     // 4T
  std::vector<uint8_t> dir;  // N
  std::vector<TetRest> rest;
  std::vector<double> mass;  // N
  std::vector<int> sverts, stris, sedges;
  std::vector<double> sedge_len2;
  // connected components of the tet mesh (READING R25: a second deformable body, f4): vertex
  // component, and the component of each surface vertex / triangle / edge
  int ncomp = 1;
  std::vector<int> comp, sv_comp, st_comp, se_comp;
  std::vector<double> IV;  // indenter verts in its own frame, 3M
  std::vector<int> itris, iedges;
  std::vector<double> iedge_len2;
  double mu = 0, lam = 0, rho = 0, young = 0;
  double dhat = 1e-4, kappa = 0, newton_tol = 1e-5, pcg_tol = 1e-10, bbox_diag = 0;
  double grav[3] = {0, 0, 0};
  int newton_max = 200, pcg_max = 100000, ls_max = 60, accd_max = 100000, split_depth = 4;
  double fric_mu = 0.0, fric_epsv = 1e-3;  // friction coefficient (0: none), velocity threshold [m/s]
  std::vector<struct FricPair> fric;        // lagged friction pairs of the running (sub)step
  double fric_eh = 0.0;                     // eps_v h of the running (sub)step
  // adaptive barrier stiffness (READING R5b): kappa is part of the state; after a step whose final
  // closest pair is nearer than kappa_dmin and nearer than at the end of the step before, kappa
  // doubles (up to kappa_cap) for the steps that follow; reset and set_state return to kappa0
  // (kappa_cap = 0: kappa stays kappa0)
  double kappa0 = 0.0, kappa_cap = 0.0, kappa_dmin = 0.0, dmin_last = INF;
  // state
  std::vector<double> x, v;
  double pose[7] = {1, 0, 0, 0, 0, 0, 0};
  double case_pose[7] = {1, 0, 0, 0, 0, 0, 0};  // pose of the Dirichlet (attached) vertices' frame
  double fc[3] = {0, 0, 0};
  // stats of the last step
  int st_newton = 0, st_pcg = 0, st_ls = 0, st_substeps = 0, st_pairs = 0;
  int st_stationary = 0;  // solves of the last step ended by the stationarity rule (READING R8b)
  int st_kappa_doublings = 0;  // doublings of kappa after the last step (READING R5b)
  double st_energy = 0, st_min_d = INF;
};

void pose_apply(const double pose[7], const double* local, int M, double* world) {
  double w = pose[0], qx = pose[1], qy = pose[2], qz = pose[3];
  double nn = std::sqrt(w * w + qx * qx + qy * qy + qz * qz);
  w /= nn;
  qx /= nn;
  qy /= nn;
  qz /= nn;
  double R[9] = {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - w * qz),     2 * (qx * qz + w * qy),
                 2 * (qx * qy + w * qz),     1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - w * qx),
                 2 * (qx * qz - w * qy),     2 * (qy * qz + w * qx),     1 - 2 * (qx * qx + qy * qy)};
  for (int k = 0; k < M; ++k)
    for (int i = 0; i < 3; ++i)
      world[3 * k + i] = R[3 * i] * local[3 * k] + R[3 * i + 1] * local[3 * k + 1] +
                         R[3 * i + 2] * local[3 * k + 2] + pose[4 + i];
}

// midpoint pose: translation average, normalised quaternion average on the short arc
void pose_mid(const double a[7], const double b[7], double m[7]) {
  double dq = a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3];
  double sgn = dq < 0 ? -1.0 : 1.0, nn = 0.0;
  for (int i = 0; i < 4; ++i) {
    m[i] = a[i] + sgn * b[i];
    nn += m[i] * m[i];
  }
  nn = std::sqrt(nn);
  for (int i = 0; i < 4; ++i) m[i] /= nn;
  for (int i = 4; i < 7; ++i) m[i] = 0.5 * (a[i] + b[i]);
}

// One contact pair instance: kind, gel-side primitive and indenter-side primitive.
//   PT  (type 0): gel surface vertex  vs indenter triangle   P = [gv, it0, it1, it2], gel slot 0
//   TP  (type 1): indenter vertex     vs gel surface triangle P = [iv, gt0, gt1, gt2], gel 1..3
//   EE  (type 2): gel surface edge    vs indenter edge        P = [ga0, ga1, ib0, ib1], gel 0..1
// and, between two deformable bodies (surface primitives of different mesh components):
//   SPT (type 3): surface vertex      vs surface triangle     P = [sv, st0, st1, st2], all mesh
//   SEE (type 4): surface edge        vs surface edge         P = [sa0, sa1, sb0, sb1], all mesh
struct PairRef {
  int type, g, k;
};

struct Scene {
  const Gel* G;
  const double* x;   // gel positions 3N
  const double* IW;  // indenter world verts 3M
};

void pair_points(const Gel& G, const double* x, const double* IW, const PairRef& pr, double P[4][3],
                 int gidx[4]) {
  auto put = [&](int slot, const double* src, int id, bool gel) {
    for (int i = 0; i < 3; ++i) P[slot][i] = src[3 * id + i];
    gidx[slot] = gel ? id : -1;
  };
  if (pr.type == 0) {
    put(0, x, G.sverts[pr.g], true);
    for (int c = 0; c < 3; ++c) put(1 + c, IW, G.itris[3 * pr.k + c], false);
  } else if (pr.type == 1) {
    put(0, IW, pr.k, false);
    for (int c = 0; c < 3; ++c) put(1 + c, x, G.stris[3 * pr.g + c], true);
  } else if (pr.type == 2) {
    put(0, x, G.sedges[2 * pr.g], true);
    put(1, x, G.sedges[2 * pr.g + 1], true);
    put(2, IW, G.iedges[2 * pr.k], false);
    put(3, IW, G.iedges[2 * pr.k + 1], false);
  } else if (pr.type == 3) {
    put(0, x, G.sverts[pr.g], true);
    for (int c = 0; c < 3; ++c) put(1 + c, x, G.stris[3 * pr.k + c], true);
  } else {
    put(0, x, G.sedges[2 * pr.g], true);
    put(1, x, G.sedges[2 * pr.g + 1], true);
    put(2, x, G.sedges[2 * pr.k], true);
    put(3, x, G.sedges[2 * pr.k + 1], true);
  }
}

double pair_eps_x(const Gel& G, const PairRef& pr) {
  if (pr.type == 4) return 1e-3 * G.sedge_len2[pr.g] * G.sedge_len2[pr.k];
  return pr.type == 2 ? 1e-3 * G.sedge_len2[pr.g] * G.iedge_len2[pr.k] : 0.0;
}

// All primitive pairs whose boxes (gel side swept from x0 to x1, indenter side swept from I0 to
// I1) come within `pad` along every axis.  Brute force over every pair.
std::vector<PairRef> candidate_pairs(const Gel& G, const double* x0, const double* x1,
                                     const double* I0, const double* I1, double pad) {
  std::vector<PairRef> out;
  auto gbox = [&](const int* ids, int n) {
    const double* pts[6];
    for (int k = 0; k < n; ++k) {
      pts[2 * k] = x0 + 3 * ids[k];
      pts[2 * k + 1] = x1 + 3 * ids[k];
    }
    return box_of(pts, 2 * n);
  };
  auto ibox = [&](const int* ids, int n) {
    const double* pts[6];
    for (int k = 0; k < n; ++k) {
      pts[2 * k] = I0 + 3 * ids[k];
      pts[2 * k + 1] = I1 + 3 * ids[k];
    }
    return box_of(pts, 2 * n);
  };
  std::vector<Box> itb(G.K), iedb(G.iedges.size() / 2), ivb(G.M);
  for (int k = 0; k < G.K; ++k) itb[k] = ibox(&G.itris[3 * k], 3);
  for (size_t k = 0; k < iedb.size(); ++k) iedb[k] = ibox(&G.iedges[2 * k], 2);
  for (int k = 0; k < G.M; ++k) ivb[k] = ibox(&k, 1);
  // every (gel primitive, indenter primitive) combination of each type, listed gel primitive by
  // gel primitive (the scan of one gel primitive may run on any thread; the lists are joined in
  // gel-primitive order)
  auto scan = [&](int type, int ng, int nvert, const int* ids, const std::vector<Box>& ib) {
    std::vector<std::vector<int>> hits(ng);
#pragma omp parallel for schedule(dynamic, 64)
    for (int g = 0; g < ng; ++g) {
      Box b = gbox(ids + (size_t)nvert * g, nvert);
      for (int k = 0; k < (int)ib.size(); ++k)
        if (near_boxes(b, ib[k], pad)) hits[g].push_back(k);
    }
    for (int g = 0; g < ng; ++g)
      for (int k : hits[g]) out.push_back({type, g, k});
  };
  scan(0, (int)G.sverts.size(), 1, G.sverts.data(), itb);
  scan(1, (int)(G.stris.size() / 3), 3, G.stris.data(), ivb);
  scan(2, (int)(G.sedges.size() / 2), 2, G.sedges.data(), iedb);
  if (G.ncomp > 1) {  // READING R25: the surfaces of different components against each other
    const int nsv = (int)G.sverts.size(), nst = (int)(G.stris.size() / 3), nse = (int)(G.sedges.size() / 2);
    std::vector<Box> stb(nst), seb(nse);
    for (int k = 0; k < nst; ++k) stb[k] = gbox(&G.stris[3 * k], 3);
    for (int k = 0; k < nse; ++k) seb[k] = gbox(&G.sedges[2 * k], 2);
    std::vector<std::vector<int>> hv(nsv), he(nse);
#pragma omp parallel for schedule(dynamic, 64)
    for (int g = 0; g < nsv; ++g) {  // every vertex against the triangles of the other bodies
      const Box b = gbox(&G.sverts[g], 1);
      for (int k = 0; k < nst; ++k)
        if (G.st_comp[k] != G.sv_comp[g] && near_boxes(b, stb[k], pad)) hv[g].push_back(k);
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int g = 0; g < nse; ++g)  // each pair of edges of different bodies once (g < k)
      for (int k = g + 1; k < nse; ++k)
        if (G.se_comp[k] != G.se_comp[g] && near_boxes(seb[g], seb[k], pad)) he[g].push_back(k);
    for (int g = 0; g < nsv; ++g)
      for (int k : hv[g]) out.push_back({3, g, k});
    for (int g = 0; g < nse; ++g)
      for (int k : he[g]) out.push_back({4, g, k});
  }
  return out;
}

int kind_of(const PairRef& pr) { return (pr.type == 2 || pr.type == 4) ? K_EE : K_PT; }
bool soft_soft(const PairRef& pr) { return pr.type >= 3; }

// ---------------- lagged friction ----------------
struct FricPair {
  PairRef pr;
  double w[4];        // closest-point weights: relative displacement = sum_k w[k] (P_k - Plag_k)
  double T[3][2];     // orthonormal tangent basis (columns) at the lagged state
  double lam;         // lagged normal force magnitude kappa m |b'(d)|
  double Plag[4][3];  // the pair's points at the lagged state
};

// lagged data of one pair from its points at the start of the step; false if not in contact
bool fric_setup(int kind, const double P[4][3], double dhat, double kappa, double eps_x, FricPair* f) {
  const DType ty = classify(kind, P);
  const double D = d2_of_type(ty, P);
  if (!(D > 0.0) || !(D < dhat * dhat)) return false;
  const double d = std::sqrt(D);
  double m = 1.0;
  if (kind == K_EE) {  // the mollifier at the lagged state scales the normal force
    double ea[3], eb[3], n[3];
    sub3(P[1], P[0], ea);
    sub3(P[3], P[2], eb);
    cross3(ea, eb, n);
    const double c = dot3(n, n);
    if (c < eps_x) m = (2.0 - c / eps_x) * (c / eps_x);
  }
  const double bp = -2.0 * (d - dhat) * std::log(d / dhat) - (d - dhat) * (d - dhat) / d;  // b'(d) < 0
  f->lam = kappa * m * std::fabs(bp);
  for (int k = 0; k < 4; ++k) {
    f->w[k] = 0.0;
    for (int c = 0; c < 3; ++c) f->Plag[k][c] = P[k][c];
  }
  double nrm[3];  // a normal of the tangent plane
  const int* i = ty.i;
  if (ty.f == F_PP) {
    f->w[i[0]] = 1.0;
    f->w[i[1]] = -1.0;
    sub3(P[i[0]], P[i[1]], nrm);
  } else if (ty.f == F_PE) {
    double e[3], w[3];
    sub3(P[i[2]], P[i[1]], e);
    sub3(P[i[0]], P[i[1]], w);
    const double t = dot3(w, e) / dot3(e, e);
    f->w[i[0]] = 1.0;
    f->w[i[1]] = -(1.0 - t);
    f->w[i[2]] = -t;
    for (int c = 0; c < 3; ++c) nrm[c] = P[i[0]][c] - ((1.0 - t) * P[i[1]][c] + t * P[i[2]][c]);
  } else if (ty.f == F_PT) {
    double e1[3], e2[3], w[3];
    sub3(P[i[2]], P[i[1]], e1);
    sub3(P[i[3]], P[i[1]], e2);
    sub3(P[i[0]], P[i[1]], w);
    const double a = dot3(e1, e1), b = dot3(e1, e2), c = dot3(e2, e2), dd = dot3(e1, w), ff = dot3(e2, w);
    const double det = a * c - b * b;
    const double l1 = (c * dd - b * ff) / det, l2 = (a * ff - b * dd) / det;
    f->w[i[0]] = 1.0;
    f->w[i[1]] = -(1.0 - l1 - l2);
    f->w[i[2]] = -l1;
    f->w[i[3]] = -l2;
    cross3(e1, e2, nrm);
  } else {
    double u[3], v[3], w[3];
    sub3(P[i[1]], P[i[0]], u);
    sub3(P[i[3]], P[i[2]], v);
    sub3(P[i[0]], P[i[2]], w);
    const double a = dot3(u, u), b = dot3(u, v), c = dot3(v, v), dd = dot3(u, w), e = dot3(v, w);
    const double den = a * c - b * b;
    const double s = (b * e - c * dd) / den, t = (a * e - b * dd) / den;
    f->w[i[0]] = 1.0 - s;
    f->w[i[1]] = s;
    f->w[i[2]] = -(1.0 - t);
    f->w[i[3]] = -t;
    cross3(u, v, nrm);
  }
  const double nn = std::sqrt(dot3(nrm, nrm));
  for (int c = 0; c < 3; ++c) nrm[c] /= nn;
  // first tangent: the coordinate axis least aligned with the normal, made orthogonal to it
  int ax = 0;
  for (int c = 1; c < 3; ++c)
    if (std::fabs(nrm[c]) < std::fabs(nrm[ax])) ax = c;
  double t1[3] = {0.0, 0.0, 0.0}, t2[3];
  t1[ax] = 1.0;
  const double pn = dot3(t1, nrm);
  for (int c = 0; c < 3; ++c) t1[c] -= pn * nrm[c];
  const double n1 = std::sqrt(dot3(t1, t1));
  for (int c = 0; c < 3; ++c) t1[c] /= n1;
  cross3(nrm, t1, t2);
  for (int c = 0; c < 3; ++c) {
    f->T[c][0] = t1[c];
    f->T[c][1] = t2[c];
  }
  return true;
}

// f0 as a function of s = |u|^2 (smooth at s = 0): value, d/ds, d2/ds2
void fric_f0_s(double s, double eh, double* g0, double* g1, double* g2) {
  const double y = std::sqrt(s);
  if (y >= eh) {
    *g0 = y;
    *g1 = 0.5 / y;
    *g2 = -0.25 / (y * s);
    return;
  }
  *g0 = -s * y / (3.0 * eh * eh) + s / eh + eh / 3.0;
  *g1 = -0.5 * y / (eh * eh) + 1.0 / eh;
  *g2 = s > 0.0 ? -0.25 / (y * eh * eh) : 0.0;  // times (ds)^2 = 4 (u.du)^2, which is 0 at s = 0
}

double fric_value(double s, double eh) {
  double a, b, c;
  fric_f0_s(s, eh, &a, &b, &c);
  return a;
}
template <int N>
AD<N> fric_value(const AD<N>& s, double eh) {
  double a, b, c;
  fric_f0_s(s.v, eh, &a, &b, &c);
  return ad_chain(s, a, b, c);
}

// D = mu lambda f0(|T^T sum_k w_k (P_k - Plag_k)|) for the pair's current points P
template <class T>
T fric_energy(const FricPair& f, const T P[4][3], double mu, double eh) {
  T dl[3];
  for (int c = 0; c < 3; ++c) {
    dl[c] = f.w[0] * (P[0][c] - f.Plag[0][c]);
    for (int k = 1; k < 4; ++k) dl[c] = dl[c] + f.w[k] * (P[k][c] - f.Plag[k][c]);
  }
  T u0 = dl[0] * f.T[0][0] + dl[1] * f.T[1][0] + dl[2] * f.T[2][0];
  T u1 = dl[0] * f.T[0][1] + dl[1] * f.T[1][1] + dl[2] * f.T[2][1];
  T s = u0 * u0 + u1 * u1;
  return (mu * f.lam) * fric_value(s, eh);
}

// ---------------- energy ----------------
struct EnergyParts {
  double inertia, elastic, barrier, min_d;
  int active;
  double friction;
};

EnergyParts energy(const Gel& G, const double* x, const double* xt, double h, const double* IW) {
  EnergyParts e{0, 0, 0, INF, 0, 0};
  for (int i = 0; i < G.N; ++i) {
    double s = 0.0;
    for (int c = 0; c < 3; ++c) s += (x[3 * i + c] - xt[3 * i + c]) * (x[3 * i + c] - xt[3 * i + c]);
    e.inertia += G.mass[i] * s / (2.0 * h * h);
  }
  std::vector<double> te(G.T);
#pragma omp parallel for schedule(static)
  for (int t = 0; t < G.T; ++t) {
    double Xl[4][3], xl[4][3];
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 3; ++c) {
        Xl[a][c] = G.X[3 * G.tets[4 * t + a] + c];
        xl[a][c] = x[3 * G.tets[4 * t + a] + c];
      }
    te[t] = tet_energy(G.rest[t], Xl, xl, G.mu, G.lam);
  }
  for (int t = 0; t < G.T; ++t) e.elastic += te[t];
  std::vector<PairRef> pairs = candidate_pairs(G, x, x, IW, IW, G.dhat);
  const int np = (int)pairs.size();
  std::vector<double> pd2(np), pb(np, 0.0);
#pragma omp parallel for schedule(dynamic, 64)
  for (int k = 0; k < np; ++k) {
    double P[4][3];
    int gi[4];
    pair_points(G, x, IW, pairs[k], P, gi);
    int kind = kind_of(pairs[k]);
    DType ty = classify(kind, P);
    double D = d2_of_type(ty, P);
    pd2[k] = D;
    if (D > 0.0 && D < G.dhat * G.dhat) pb[k] = pair_barrier<double>(kind, ty, P, G.dhat, pair_eps_x(G, pairs[k]));
  }
  for (int k = 0; k < np; ++k) {
    const double D = pd2[k];
    e.min_d = std::min(e.min_d, std::sqrt(D));
    if (!(D > 0.0)) {
      e.barrier = INF;
      continue;
    }
    if (D >= G.dhat * G.dhat) continue;
    e.active++;
    e.barrier += G.kappa * pb[k];
  }
  const int nfr = (int)G.fric.size();
  std::vector<double> fe(nfr);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nfr; ++k) {  // lagged friction (empty unless mu_f > 0)
    double P[4][3];
    int gi[4];
    pair_points(G, x, IW, G.fric[k].pr, P, gi);
    fe[k] = fric_energy<double>(G.fric[k], P, G.fric_mu, G.fric_eh);
  }
  for (int k = 0; k < nfr; ++k) e.friction += fe[k];
  return e;
}

double total(const EnergyParts& e) {
  const double s = e.inertia + e.elastic + e.barrier;
  return e.friction != 0.0 ? s + e.friction : s;
}

// ---------------- gradient and projected Hessian ----------------
struct Triplet {
  int r, c;
  double v;
};

// free DOF numbering: dof[3*i + c] = index or -1 for Dirichlet vertices
void assemble(const Gel& G, const double* x, const double* xt, double h, const double* IW,
              const std::vector<int>& dof, std::vector<double>& grad, std::vector<Triplet>& trip,
              double fc[3], bool project) {
  grad.assign(3 * G.N, 0.0);
  trip.clear();
  fc[0] = fc[1] = fc[2] = 0.0;
  auto add = [&](int gi, int gj, double v) {
    if (dof[gi] >= 0 && dof[gj] >= 0 && v != 0.0) trip.push_back({dof[gi], dof[gj], v});
  };
  for (int i = 0; i < G.N; ++i)
    for (int c = 0; c < 3; ++c) {
      grad[3 * i + c] += G.mass[i] * (x[3 * i + c] - xt[3 * i + c]) / (h * h);
      add(3 * i + c, 3 * i + c, G.mass[i] / (h * h));
    }
  {
    // per-tet derivatives (parallel), then added in tet order
    std::vector<double> tg(12 * (size_t)G.T), tH(144 * (size_t)G.T);
#pragma omp parallel for schedule(static)
    for (int t = 0; t < G.T; ++t) {
      double Xl[4][3], xl[4][3], e;
      for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 3; ++c) {
          Xl[a][c] = G.X[3 * G.tets[4 * t + a] + c];
          xl[a][c] = x[3 * G.tets[4 * t + a] + c];
        }
      tet_derivs(G.rest[t], Xl, xl, G.mu, G.lam, project, &e, &tg[12 * (size_t)t], &tH[144 * (size_t)t]);
    }
    for (int t = 0; t < G.T; ++t) {
      const double* g = &tg[12 * (size_t)t];
      const double* H = &tH[144 * (size_t)t];
      for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 3; ++c) {
          int gi = 3 * G.tets[4 * t + a] + c;
          grad[gi] += g[3 * a + c];
          for (int b = 0; b < 4; ++b)
            for (int d = 0; d < 3; ++d) add(gi, 3 * G.tets[4 * t + b] + d, H[(3 * a + c) * 12 + 3 * b + d]);
        }
    }
  }
  // per-pair contributions on the gel's points (computed in parallel, added in pair order)
  struct PairTerm {
    bool on = false, ss = false;  // ss: between two deformable bodies (not in the indenter force)
    int nf = 0, fidx[12], gi[4];
    double g[12], H[144];
  };
  auto add_terms = [&](const std::vector<PairTerm>& terms) {
    for (const PairTerm& q : terms) {
      if (!q.on) continue;
      for (int r = 0; r < q.nf; ++r) {
        int kr = q.fidx[r] / 3, cr = q.fidx[r] % 3;
        int gr = 3 * q.gi[kr] + cr;
        grad[gr] += q.g[r];
        if (!q.ss) fc[cr] -= q.g[r];
        for (int c = 0; c < q.nf; ++c) {
          int kc = q.fidx[c] / 3, cc = q.fidx[c] % 3;
          add(gr, 3 * q.gi[kc] + cc, q.H[r * q.nf + c]);
        }
      }
    }
  };
  std::vector<PairRef> pairs = candidate_pairs(G, x, x, IW, IW, G.dhat);
  {
    const int np = (int)pairs.size();
    std::vector<PairTerm> terms(np);
#pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < np; ++k) {
      const PairRef& pr = pairs[k];
      PairTerm& q = terms[k];
      double P[4][3];
      pair_points(G, x, IW, pr, P, q.gi);
      int kind = kind_of(pr);
      DType ty = classify(kind, P);
      double D = d2_of_type(ty, P);
      if (!(D < G.dhat * G.dhat) || !(D > 0.0)) continue;
      q.on = true;
      q.ss = soft_soft(pr);
      AD<12> Pv[4][3];
      for (int j = 0; j < 4; ++j)
        for (int c = 0; c < 3; ++c) Pv[j][c] = ad_var<12>(P[j][c], 3 * j + c);
      AD<12> b = pair_barrier<AD<12>>(kind, ty, Pv, G.dhat, pair_eps_x(G, pr));
      // free sub-block: the gel's points only
      for (int j = 0; j < 4; ++j)
        if (q.gi[j] >= 0)
          for (int c = 0; c < 3; ++c) q.fidx[q.nf++] = 3 * j + c;
      for (int r = 0; r < q.nf; ++r)
        for (int c = 0; c < q.nf; ++c) q.H[r * q.nf + c] = G.kappa * b.h[q.fidx[r]][q.fidx[c]];
      if (project) psd_project(q.nf, q.H);
      for (int r = 0; r < q.nf; ++r) q.g[r] = G.kappa * b.g[q.fidx[r]];
    }
    add_terms(terms);
  }
  // lagged friction: convex in u, so its Hessian is PSD as it stands (projected all the same)
  {
    const int nfr = (int)G.fric.size();
    std::vector<PairTerm> terms(nfr);
#pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < nfr; ++k) {
      const FricPair& f = G.fric[k];
      PairTerm& q = terms[k];
      double P[4][3];
      pair_points(G, x, IW, f.pr, P, q.gi);
      q.on = true;
      AD<12> Pv[4][3];
      for (int j = 0; j < 4; ++j)
        for (int c = 0; c < 3; ++c) Pv[j][c] = ad_var<12>(P[j][c], 3 * j + c);
      AD<12> D = fric_energy<AD<12>>(f, Pv, G.fric_mu, G.fric_eh);
      for (int j = 0; j < 4; ++j)
        if (q.gi[j] >= 0)
          for (int c = 0; c < 3; ++c) q.fidx[q.nf++] = 3 * j + c;
      for (int r = 0; r < q.nf; ++r)
        for (int c = 0; c < q.nf; ++c) q.H[r * q.nf + c] = D.h[q.fidx[r]][q.fidx[c]];
      if (project) psd_project(q.nf, q.H);
      for (int r = 0; r < q.nf; ++r) q.g[r] = D.g[q.fidx[r]];
    }
    add_terms(terms);
  }
}

struct CSR {
  int n = 0;
  std::vector<int> rp, ci;
  std::vector<double> va;
};

// CSR of the summed triplets.  The triplets of each row are gathered in the order they were
// generated, ordered by column with a stable sort, and the entries of one (row, column) position
// are summed in generation order.
CSR to_csr(int n, std::vector<Triplet>& t) {
  CSR A;
  A.n = n;
  std::vector<size_t> start(n + 1, 0);
  for (const Triplet& e : t) start[e.r + 1]++;
  for (int i = 0; i < n; ++i) start[i + 1] += start[i];
  std::vector<size_t> fill(start.begin(), start.end() - 1);
  std::vector<std::pair<int, double>> byrow(t.size());
  for (const Triplet& e : t) byrow[fill[e.r]++] = {e.c, e.v};
  std::vector<int> nnz(n, 0);
#pragma omp parallel for schedule(dynamic, 256)
  for (int i = 0; i < n; ++i) {
    auto b = byrow.begin() + start[i], e = byrow.begin() + start[i + 1];
    std::stable_sort(b, e, [](const std::pair<int, double>& u, const std::pair<int, double>& w) {
      return u.first < w.first;
    });
    for (auto k = b; k != e; ++k)
      if (k == b || k->first != (k - 1)->first) nnz[i]++;
  }
  A.rp.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) A.rp[i + 1] = A.rp[i] + nnz[i];
  A.ci.resize(A.rp[n]);
  A.va.resize(A.rp[n]);
#pragma omp parallel for schedule(dynamic, 256)
  for (int i = 0; i < n; ++i) {
    int o = A.rp[i];
    for (size_t k = start[i]; k < start[i + 1];) {
      size_t m = k;
      double s = 0.0;
      while (m < start[i + 1] && byrow[m].first == byrow[k].first) s += byrow[m++].second;
      A.ci[o] = byrow[k].first;
      A.va[o] = s;
      ++o;
      k = m;
    }
  }
  return A;
}

void spmv(const CSR& A, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < A.n; ++i) {
    double s = 0.0;
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) s += A.va[k] * x[A.ci[k]];
    y[i] = s;
  }
}

// sum_i a_i b_i in index order
double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

// Jacobi-preconditioned CG for A x = b, x0 = 0, stop at |r| <= tol |b|.  Returns iterations or -1.
int pcg(const CSR& A, const std::vector<double>& b, std::vector<double>& x, double tol, int maxit) {
  int n = A.n;
  x.assign(n, 0.0);
  std::vector<double> r = b, z(n), p(n), q(n), dinv(n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k)
      if (A.ci[k] == i) dinv[i] = 1.0 / A.va[k];
  double bb = dot(b, b);
  if (bb == 0.0) return 0;
  for (int i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
  p = z;
  double rz = dot(r, z);
  for (int it = 1; it <= maxit; ++it) {
    spmv(A, p.data(), q.data());
    double pq = dot(p, q);
    double alpha = rz / pq;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    double rr = dot(r, r);
    if (rr <= tol * tol * bb) return it;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
    double rz2 = dot(r, z);
    double beta = rz2 / rz;
    rz = rz2;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
  }
  return -1;
}

// smallest ACCD time of impact over the candidate pairs (1 if none), or an error status
int min_toi(const Gel& G, const double* x0, const double* dx, const double* I0, const double* dI,
            double* out) {
  std::vector<double> x1(3 * G.N), I1(3 * G.M);
  for (int i = 0; i < 3 * G.N; ++i) x1[i] = x0[i] + dx[i];
  for (int i = 0; i < 3 * G.M; ++i) I1[i] = I0[i] + dI[i];
  std::vector<PairRef> pairs = candidate_pairs(G, x0, x1.data(), I0, I1.data(), G.dhat);
  const int np = (int)pairs.size();
  std::vector<int> res(np);
  std::vector<double> toi(np);
#pragma omp parallel for schedule(dynamic, 16)
  for (int q = 0; q < np; ++q) {
    double P[4][3], dP[4][3];
    int gi[4];
    pair_points(G, x0, I0, pairs[q], P, gi);
    double Pd[4][3];
    int gd[4];
    pair_points(G, dx, dI, pairs[q], Pd, gd);
    for (int k = 0; k < 4; ++k)
      for (int c = 0; c < 3; ++c) dP[k][c] = Pd[k][c];
    res[q] = accd(kind_of(pairs[q]), P, dP, 0.1, 1.0, G.accd_max, &toi[q]);
  }
  double best = 1.0;
  for (int q = 0; q < np; ++q) {
    if (res[q] == 2) return ERR_CCD_MAXIT;
    if (res[q] == 1) best = std::min(best, toi[q]);
  }
  *out = best;
  return OK;
}

// ---------------- Newton solve of one (sub)step ----------------
// READING R8b: after a line search that found no decrease down to 1e-12 alpha_0, the iterate counts
// as converged when the model decrease -g.p of the direction is at most 1e-10 |E| (below what FP64
// evaluations of E can resolve), otherwise the step fails.
bool stationary_to_resolution(double gp, double E) { return -gp <= 1e-10 * std::fabs(E); }

int newton_iterate(Gel& G, double h, const double* IW) {
  int n3 = 3 * G.N;
  std::vector<double> xn = G.x, xt(n3);
  for (int i = 0; i < G.N; ++i)
    for (int c = 0; c < 3; ++c)
      xt[3 * i + c] = G.dir[i] ? G.x[3 * i + c] : G.x[3 * i + c] + h * G.v[3 * i + c] + h * h * G.grav[c];
  std::vector<int> dof(n3, -1);
  int nf = 0;
  for (int i = 0; i < G.N; ++i)
    if (!G.dir[i])
      for (int c = 0; c < 3; ++c) dof[3 * i + c] = nf++;
  std::vector<double>& x = G.x;
  EnergyParts ep = energy(G, x.data(), xt.data(), h, IW);
  double E = total(ep);
  if (!std::isfinite(E)) return ERR_INFEASIBLE;
  std::vector<double> grad, rhs(nf), sol, p(n3, 0.0), xtrial(n3), zeroI(3 * G.M, 0.0);
  std::vector<Triplet> trip;
  double tol = G.newton_tol * G.bbox_diag * h;
  for (int it = 0; it <= G.newton_max; ++it) {
    assemble(G, x.data(), xt.data(), h, IW, dof, grad, trip, G.fc, true);
    CSR A = to_csr(nf, trip);
    for (int i = 0; i < n3; ++i)
      if (dof[i] >= 0) rhs[dof[i]] = -grad[i];
    int pit = pcg(A, rhs, sol, G.pcg_tol, G.pcg_max);
    if (pit < 0) return ERR_PCG_MAXIT;
    G.st_pcg += pit;
    double pinf = 0.0;
    for (int i = 0; i < n3; ++i) {
      p[i] = dof[i] >= 0 ? sol[dof[i]] : 0.0;
      pinf = std::max(pinf, std::fabs(p[i]));
    }
    if (pinf < tol) {
      G.st_energy = E;
      G.st_pairs = ep.active;
      G.st_min_d = ep.min_d;
      return OK;
    }
    if (it == G.newton_max) break;
    double a0;
    int s = min_toi(G, x.data(), p.data(), IW, zeroI.data(), &a0);
    if (s != OK) return s;
    double alpha = a0;
    bool accepted = false;
    EnergyParts et{};
    for (int ls = 0; ls <= G.ls_max; ++ls) {
      for (int i = 0; i < n3; ++i) xtrial[i] = x[i] + alpha * p[i];
      et = energy(G, xtrial.data(), xt.data(), h, IW);
      if (total(et) <= E) {
        accepted = true;
        break;
      }
      alpha *= 0.5;
      G.st_ls++;
      if (alpha < 1e-12 * a0) break;
    }
    if (!accepted) {
      // READING: a direction whose model decrease -g.p is below 1e-10 |E| cannot be resolved by
      // FP64 energy evaluations (barrier energies carry absolute noise from coordinate round-off);
      // such an iterate is stationary to energy resolution and is taken as converged.
      double gp = 0.0;
      for (int i = 0; i < n3; ++i)
        if (dof[i] >= 0) gp += grad[i] * p[i];
      if (stationary_to_resolution(gp, E)) {
        G.st_energy = E;
        G.st_pairs = ep.active;
        G.st_min_d = ep.min_d;
        G.st_stationary++;
        return OK;
      }
      return ERR_LINESEARCH;
    }
    x = xtrial;
    E = total(et);
    ep = et;
    G.st_newton++;
  }
  return ERR_NEWTON_MAXIT;
}

// Newton solve of one (sub)step with the indenter at IW; with friction, the lagged pairs are
// taken first at the step's start (gel at x_n, indenter at I0) and dropped afterwards
int newton_solve(Gel& G, double h, const double* I0, const double* IW) {
  G.fric.clear();
  if (G.fric_mu > 0.0) {
    G.fric_eh = G.fric_epsv * h;
    for (const PairRef& pr : candidate_pairs(G, G.x.data(), G.x.data(), I0, I0, G.dhat)) {
      if (soft_soft(pr)) continue;  // READING R25: friction against the rigid indenter only
      double P[4][3];
      int gi[4];
      pair_points(G, G.x.data(), I0, pr, P, gi);
      FricPair f;
      f.pr = pr;
      if (fric_setup(kind_of(pr), P, G.dhat, G.kappa, pair_eps_x(G, pr), &f)) G.fric.push_back(f);
    }
  }
  const int s = newton_iterate(G, h, IW);
  G.fric.clear();
  return s;
}

// feasibility of moving the indenter from I0 to I1 with the gel fixed at its current x
bool placement_ok(const Gel& G, const double* I0, const double* I1, int* err) {
  std::vector<double> dI(3 * G.M), zx(3 * G.N, 0.0);
  for (int i = 0; i < 3 * G.M; ++i) dI[i] = I1[i] - I0[i];
  double t;
  int s = min_toi(G, G.x.data(), zx.data(), I0, dI.data(), &t);
  *err = s;
  if (s != OK) return false;
  std::vector<PairRef> pairs = candidate_pairs(G, G.x.data(), G.x.data(), I0, I1, G.dhat);
  const int np = (int)pairs.size();
  std::vector<int> res(np);
#pragma omp parallel for schedule(dynamic, 16)
  for (int q = 0; q < np; ++q) {  // same pairs the sweep examined: any hit means t < 1
    double P[4][3], dP[4][3], Pd[4][3];
    int gi[4], gd[4];
    pair_points(G, G.x.data(), I0, pairs[q], P, gi);
    pair_points(G, zx.data(), dI.data(), pairs[q], Pd, gd);
    for (int k = 0; k < 4; ++k)
      for (int c = 0; c < 3; ++c) dP[k][c] = Pd[k][c];
    double tt;
    res[q] = accd(kind_of(pairs[q]), P, dP, 0.1, 1.0, G.accd_max, &tt);
  }
  for (int q = 0; q < np; ++q)
    if (res[q] == 1) return false;
  // after placement every pair must be strictly separated
  std::vector<PairRef> after = candidate_pairs(G, G.x.data(), G.x.data(), I1, I1, G.dhat);
  const int na = (int)after.size();
  std::vector<char> sep(na);
#pragma omp parallel for schedule(static)
  for (int q = 0; q < na; ++q) {
    double P[4][3];
    int gi[4];
    pair_points(G, G.x.data(), I1, after[q], P, gi);
    sep[q] = pair_d2(kind_of(after[q]), P) > 0.0;
  }
  for (int q = 0; q < na; ++q)
    if (!sep[q]) return false;
  return true;
}

// Dirichlet (attached) vertices at the case pose: their rest positions carried by it
void place_attached(Gel& G, const double cpose[7]) {
  std::vector<double> Xd, xd;
  for (int i = 0; i < G.N; ++i)
    if (G.dir[i])
      for (int c = 0; c < 3; ++c) Xd.push_back(G.X[3 * i + c]);
  xd.resize(Xd.size());
  pose_apply(cpose, Xd.data(), (int)(Xd.size() / 3), xd.data());
  for (int i = 0, k = 0; i < G.N; ++i)
    if (G.dir[i]) {
      for (int c = 0; c < 3; ++c) G.x[3 * i + c] = xd[3 * k + c];
      ++k;
    }
}

// One (sub)step moving the indenter from pose pa to pb; with case poses (ca, cb) the attached
// vertices are also moved to their targets at cb first (kinematic attachments: the paper's GIPC
// step sets the attachment points' targets, then solves), and a split halves both motions.
int substep(Gel& G, const double pa[7], const double pb[7], double dt, int depth, const double* ca = nullptr,
            const double* cb = nullptr) {
  std::vector<double> I0(3 * G.M), I1(3 * G.M);
  pose_apply(pa, G.IV.data(), G.M, I0.data());
  pose_apply(pb, G.IV.data(), G.M, I1.data());
  std::vector<double> xn = G.x;
  if (cb) place_attached(G, cb);
  int err = OK;
  if (!placement_ok(G, I0.data(), I1.data(), &err)) {
    G.x = xn;
    if (err != OK) return err;
    if (depth >= G.split_depth) return ERR_INFEASIBLE;
    double pm[7], cm[7];
    pose_mid(pa, pb, pm);
    if (cb) pose_mid(ca, cb, cm);
    int s = substep(G, pa, pm, 0.5 * dt, depth + 1, ca, cb ? cm : nullptr);
    if (s != OK) return s;
    return substep(G, pm, pb, 0.5 * dt, depth + 1, cb ? cm : nullptr, cb);
  }
  int s = newton_solve(G, dt, I0.data(), I1.data());
  if (s != OK) {
    G.x = xn;
    return s;
  }
  for (int i = 0; i < 3 * G.N; ++i) G.v[i] = (G.x[i] - xn[i]) / dt;
  for (int i = 0; i < 7; ++i) G.pose[i] = pb[i];
  G.st_substeps++;
  return OK;
}

}  // namespace

// ==========================================================================================
// C interface (ctypes)
// ==========================================================================================
extern "C" {

// fparams: [dhat, kappa, newton_tol, pcg_tol, gx, gy, gz]
// iparams: [newton_max, pcg_max, ls_max, accd_max, split_depth]
void* or_create(int N, const double* X, int T, const int* tets, const uint8_t* dir, double E,
                double nu, double rho, int M, const double* IV, int K, const int* itris,
                const double* pose0, const double* fparams, const int* iparams, int* status) {
  *status = OK;
  if (N <= 0 || T < 0 || M < 0 || K < 0) {
    *status = ERR_ARG;
    return nullptr;
  }
  for (int k = 0; k < 4 * T; ++k)
    if (tets[k] < 0 || tets[k] >= N) {
      *status = ERR_ARG;
      return nullptr;
    }
  for (int k = 0; k < 3 * K; ++k)
    if (itris[k] < 0 || itris[k] >= M) {
      *status = ERR_ARG;
      return nullptr;
    }
  Gel* G = new Gel();
  G->N = N;
  G->T = T;
  G->M = M;
  G->K = K;
  G->X.assign(X, X + 3 * N);
  G->tets.assign(tets, tets + 4 * T);
  G->dir.assign(dir, dir + N);
  G->young = E;
  G->mu = E / (2.0 * (1.0 + nu));
  G->lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  G->rho = rho;
  G->rest.resize(T);
  G->mass.assign(N, 0.0);
  for (int t = 0; t < T; ++t) {
    double Xl[4][3];
    for (int a = 0; a < 4; ++a)
      for (int c = 0; c < 3; ++c) Xl[a][c] = X[3 * tets[4 * t + a] + c];
    if (!tet_rest(Xl, &G->rest[t])) {
      *status = ERR_MESH_INVERTED;
      delete G;
      return nullptr;
    }
    for (int a = 0; a < 4; ++a) G->mass[tets[4 * t + a]] += rho * G->rest[t].vol / 4.0;
  }
  // boundary faces: faces of exactly one tet
  std::map<std::vector<int>, std::vector<int>> faces;
  const int FI[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
  for (int t = 0; t < T; ++t)
    for (auto& f : FI) {
      std::vector<int> tri = {tets[4 * t + f[0]], tets[4 * t + f[1]], tets[4 * t + f[2]]};
      std::vector<int> key = tri;
      std::sort(key.begin(), key.end());
      auto it = faces.find(key);
      if (it == faces.end())
        faces[key] = tri;
      else
        it->second.clear();
    }
  std::vector<char> isv(N, 0);
  std::map<std::pair<int, int>, int> edges;
  for (auto& kv : faces) {
    if (kv.second.empty()) continue;
    for (int c = 0; c < 3; ++c) {
      G->stris.push_back(kv.second[c]);
      isv[kv.second[c]] = 1;
      int a = kv.second[c], b = kv.second[(c + 1) % 3];
      edges[{std::min(a, b), std::max(a, b)}] = 1;
    }
  }
  for (int i = 0; i < N; ++i)
    if (isv[i]) G->sverts.push_back(i);
  double lsum = 0.0;
  for (auto& kv : edges) {
    G->sedges.push_back(kv.first.first);
    G->sedges.push_back(kv.first.second);
    double l2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      double d = X[3 * kv.first.first + c] - X[3 * kv.first.second + c];
      l2 += d * d;
    }
    G->sedge_len2.push_back(l2);
    lsum += std::sqrt(l2);
  }
  // connected components: vertices joined by a tet (union-find, each root the smallest index);
  // numbered in the order of their smallest vertex, so the body of the first vertex in a tet is
  // component 0 (the gelpad)
  {
    std::vector<int> up(N);
    for (int i = 0; i < N; ++i) up[i] = i;
    auto root = [&](int i) {
      while (up[i] != i) i = up[i] = up[up[i]];
      return i;
    };
    for (int t = 0; t < T; ++t)
      for (int a = 1; a < 4; ++a) {
        const int r0 = root(tets[4 * t]), r1 = root(tets[4 * t + a]);
        if (r0 != r1) up[std::max(r0, r1)] = std::min(r0, r1);
      }
    std::vector<int> id(N, -1);
    std::vector<char> used(N, 0);
    for (int k = 0; k < 4 * T; ++k) used[tets[k]] = 1;
    G->comp.assign(N, 0);
    G->ncomp = 0;
    for (int i = 0; i < N; ++i) {
      if (!used[i]) continue;  // in no tet: on no surface, never in a pair (left in component 0)
      const int r = root(i);
      if (id[r] < 0) id[r] = G->ncomp++;
      G->comp[i] = id[r];
    }
    G->ncomp = std::max(G->ncomp, 1);
    for (int v : G->sverts) G->sv_comp.push_back(G->comp[v]);
    for (size_t k = 0; k < G->stris.size() / 3; ++k) G->st_comp.push_back(G->comp[G->stris[3 * k]]);
    for (size_t k = 0; k < G->sedges.size() / 2; ++k) G->se_comp.push_back(G->comp[G->sedges[2 * k]]);
  }
  G->IV.assign(IV, IV + 3 * M);
  G->itris.assign(itris, itris + 3 * K);
  std::map<std::pair<int, int>, int> iedges;
  for (int k = 0; k < K; ++k)
    for (int c = 0; c < 3; ++c) {
      int a = itris[3 * k + c], b = itris[3 * k + (c + 1) % 3];
      iedges[{std::min(a, b), std::max(a, b)}] = 1;
    }
  for (auto& kv : iedges) {
    G->iedges.push_back(kv.first.first);
    G->iedges.push_back(kv.first.second);
    double l2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      double d = IV[3 * kv.first.first + c] - IV[3 * kv.first.second + c];
      l2 += d * d;
    }
    G->iedge_len2.push_back(l2);
  }
  G->dhat = fparams[0];
  G->kappa = fparams[1] > 0 ? fparams[1] : E * (edges.empty() ? 0.0 : lsum / edges.size());
  G->kappa0 = G->kappa;
  G->newton_tol = fparams[2];
  G->pcg_tol = fparams[3];
  for (int c = 0; c < 3; ++c) G->grav[c] = fparams[4 + c];
  G->newton_max = iparams[0];
  G->pcg_max = iparams[1];
  G->ls_max = iparams[2];
  G->accd_max = iparams[3];
  G->split_depth = iparams[4];
  double lo[3] = {INF, INF, INF}, hi[3] = {-INF, -INF, -INF};
  for (int i = 0; i < N; ++i)
    for (int c = 0; c < 3; ++c) {
      lo[c] = std::min(lo[c], X[3 * i + c]);
      hi[c] = std::max(hi[c], X[3 * i + c]);
    }
  G->bbox_diag = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                           (hi[2] - lo[2]) * (hi[2] - lo[2]));
  G->x = G->X;
  G->v.assign(3 * N, 0.0);
  for (int i = 0; i < 7; ++i) G->pose[i] = pose0[i];
  return G;
}

void or_destroy(void* g) { delete static_cast<Gel*>(g); }

// stats: [newton_iters, pcg_iters, ls_halvings, substeps, active_pairs]; fstats: [E, min_d]
int or_step_attached(void* g, const double* pose, const double* case_pose, double dt, int* stats, double* fstats);

int or_step(void* g, const double* pose, double dt, int* stats, double* fstats) {
  return or_step_attached(g, pose, nullptr, dt, stats, fstats);
}

// One step with the indenter driven to `pose` and, if case_pose is given, the attached (Dirichlet)
// vertices driven with their frame to case_pose (their rest positions carried by it)
int or_step_attached(void* g, const double* pose, const double* case_pose, double dt, int* stats, double* fstats) {
  Gel& G = *static_cast<Gel*>(g);
  G.st_newton = G.st_pcg = G.st_ls = G.st_substeps = G.st_pairs = G.st_stationary = 0;
  G.st_kappa_doublings = 0;
  G.st_energy = 0;
  G.st_min_d = INF;
  std::vector<double> x0 = G.x, v0 = G.v;
  double p0[7], c0[7];
  std::memcpy(p0, G.pose, sizeof(p0));
  std::memcpy(c0, G.case_pose, sizeof(c0));
  int s = substep(G, G.pose, pose, dt, 0, case_pose ? c0 : nullptr, case_pose);
  if (s != OK) {  // transactional: leave the state at x_n
    G.x = x0;
    G.v = v0;
    std::memcpy(G.pose, p0, sizeof(p0));
  } else if (case_pose) {
    std::memcpy(G.case_pose, case_pose, sizeof(G.case_pose));
  }
  if (s == OK) {
    // READING R5b (IPC's adaptive barrier stiffness at step granularity: the kinematic indenter is
    // placed before the solve, so pairs close in between steps, not across Newton iterates): a
    // final closest pair nearer than kappa_dmin that came nearer than at the end of the step before
    // doubles kappa for the next steps
    if (G.kappa_cap > 0.0 && G.st_min_d < G.kappa_dmin && G.st_min_d < G.dmin_last && G.kappa < G.kappa_cap) {
      G.kappa = std::min(2.0 * G.kappa, G.kappa_cap);
      G.st_kappa_doublings = 1;
    }
    G.dmin_last = G.st_min_d;
  }
  if (stats) {
    stats[0] = G.st_newton;
    stats[1] = G.st_pcg;
    stats[2] = G.st_ls;
    stats[3] = G.st_substeps;
    stats[4] = G.st_pairs;
  }
  if (fstats) {
    fstats[0] = G.st_energy;
    fstats[1] = G.st_min_d;
  }
  return s;
}

void or_get_state(void* g, double* x, double* v, double* fc, double* pose) {
  Gel& G = *static_cast<Gel*>(g);
  if (x) std::memcpy(x, G.x.data(), sizeof(double) * 3 * G.N);
  if (v) std::memcpy(v, G.v.data(), sizeof(double) * 3 * G.N);
  if (fc) std::memcpy(fc, G.fc, sizeof(G.fc));
  if (pose) std::memcpy(pose, G.pose, sizeof(G.pose));
}

void or_set_state(void* g, const double* x, const double* v, const double* pose) {
  Gel& G = *static_cast<Gel*>(g);
  G.kappa = G.kappa0;  // READING R5b
  G.dmin_last = INF;
  if (x) G.x.assign(x, x + 3 * G.N);
  if (v) G.v.assign(v, v + 3 * G.N);
  if (pose) std::memcpy(G.pose, pose, sizeof(G.pose));
}

void or_reset(void* g) {
  Gel& G = *static_cast<Gel*>(g);
  G.kappa = G.kappa0;  // READING R5b
  G.dmin_last = INF;
  G.x = G.X;
  G.v.assign(3 * G.N, 0.0);
  const double id[7] = {1, 0, 0, 0, 0, 0, 0};
  std::memcpy(G.case_pose, id, sizeof(id));
}

// pose of the attached vertices' frame (their positions are not moved until the next step)
void or_set_case_pose(void* g, const double* pose) {
  Gel& G = *static_cast<Gel*>(g);
  std::memcpy(G.case_pose, pose, sizeof(G.case_pose));
}

// scalar properties: [mu, lambda, kappa, bbox_diag, total mass]; counts: [surf verts, surf tris,
// surf edges, indenter edges]
void or_info(void* g, double* f, int* c) {
  Gel& G = *static_cast<Gel*>(g);
  double m = 0.0;
  for (double q : G.mass) m += q;
  f[0] = G.mu;
  f[1] = G.lam;
  f[2] = G.kappa;
  f[3] = G.bbox_diag;
  f[4] = m;
  c[0] = (int)G.sverts.size();
  c[1] = (int)G.stris.size() / 3;
  c[2] = (int)G.sedges.size() / 2;
  c[3] = (int)G.iedges.size() / 2;
}

void or_mass(void* g, double* m) {
  Gel& G = *static_cast<Gel*>(g);
  std::memcpy(m, G.mass.data(), sizeof(double) * G.N);
}

// E(x) with predictor xt and the indenter at `pose`; parts = [inertia, elastic, barrier, min_d,
// active pairs]
double or_energy(void* g, const double* x, const double* xt, double h, const double* pose,
                 double* parts) {
  Gel& G = *static_cast<Gel*>(g);
  std::vector<double> IW(3 * G.M);
  pose_apply(pose, G.IV.data(), G.M, IW.data());
  EnergyParts e = energy(G, x, xt, h, IW.data());
  if (parts) {
    parts[0] = e.inertia;
    parts[1] = e.elastic;
    parts[2] = e.barrier;
    parts[3] = e.min_d;
    parts[4] = e.active;
  }
  return total(e);
}

// full gradient (3N; Dirichlet rows included) and, optionally, the projected Hessian on the
// free DOFs as COO triplets (capacity cap; returns the number of triplets, -1 if over capacity)
int or_gradient(void* g, const double* x, const double* xt, double h, const double* pose,
                double* grad, double* fc, int project, int cap, int* rows, int* cols, double* vals) {
  Gel& G = *static_cast<Gel*>(g);
  std::vector<double> IW(3 * G.M);
  pose_apply(pose, G.IV.data(), G.M, IW.data());
  std::vector<int> dof(3 * G.N, -1);
  for (int i = 0; i < 3 * G.N; ++i) dof[i] = G.dir[i / 3] ? -1 : i;  // global DOF ids
  std::vector<double> gr;
  std::vector<Triplet> trip;
  double f[3];
  assemble(G, x, xt, h, IW.data(), dof, gr, trip, f, project != 0);
  std::memcpy(grad, gr.data(), sizeof(double) * 3 * G.N);
  if (fc) std::memcpy(fc, f, sizeof(f));
  if (!rows) return 0;
  CSR A = to_csr(3 * G.N, trip);
  int nnz = (int)A.va.size();
  if (nnz > cap) return -1;
  for (int i = 0; i < A.n; ++i)
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      rows[k] = i;
      cols[k] = A.ci[k];
      vals[k] = A.va[k];
    }
  return nnz;
}

// ---- unit-level entry points (for derivative checks and kernel parity) ----
// One tet: rest corners X (4x3), current x (4x3).  Returns 0, or 3 if the rest tet is inverted,
// or 1 if det F <= 0.
int or_tet(const double* X, const double* x, double mu, double lam, int project, double* e,
           double* g, double* H) {
  double Xl[4][3], xl[4][3];
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 3; ++c) {
      Xl[a][c] = X[3 * a + c];
      xl[a][c] = x[3 * a + c];
    }
  TetRest tr;
  if (!tet_rest(Xl, &tr)) return 3;
  if (!g) {
    *e = tet_energy(tr, Xl, xl, mu, lam);
    return std::isfinite(*e) ? 0 : 1;
  }
  return tet_derivs(tr, Xl, xl, mu, lam, project != 0, e, g, H) ? 0 : 1;
}

// Neo-Hookean density Psi and its derivatives w.r.t. F (row-major 9), via H = F - I.
int or_psi(const double* F, double mu, double lam, double* psi, double* P, double* C) {
  AD<9> Hv[9];
  for (int k = 0; k < 9; ++k) Hv[k] = ad_var<9>(F[k] - ((k % 4) == 0 ? 1.0 : 0.0), k);
  AD<9> r;
  if (!psi_of_H(Hv, mu, lam, &r)) return 1;
  *psi = r.v;
  if (P)
    for (int k = 0; k < 9; ++k) P[k] = r.g[k];
  if (C)
    for (int i = 0; i < 9; ++i)
      for (int j = 0; j < 9; ++j) C[9 * i + j] = r.h[i][j];
  return 0;
}

// squared distance and type of a primitive pair: kind 0 = point P0 vs triangle P1..3,
// kind 1 = segment P0P1 vs segment P2P3.  type_out = [formula, i0, i1, i2, i3].
double or_distance2(int kind, const double* Pf, int* type_out) {
  double P[4][3];
  for (int k = 0; k < 4; ++k)
    for (int c = 0; c < 3; ++c) P[k][c] = Pf[3 * k + c];
  DType t = classify(kind, P);
  if (type_out) {
    type_out[0] = t.f;
    for (int i = 0; i < 4; ++i) type_out[1 + i] = t.i[i];
  }
  return d2_of_type(t, P);
}

// barrier of one pair (without kappa): b, gradient (12) and Hessian (12x12) w.r.t. all 4 points.
// If free_mask != 0, the Hessian's block on the points whose bit is set is PSD-projected in
// place (the other entries are left unprojected).  Returns 1 if d >= dhat (all zero), 2 if d <= 0.
int or_pair_barrier(int kind, const double* Pf, double dhat, double eps_x, int free_mask, double* b,
                    double* g, double* H) {
  double P[4][3];
  for (int k = 0; k < 4; ++k)
    for (int c = 0; c < 3; ++c) P[k][c] = Pf[3 * k + c];
  DType ty = classify(kind, P);
  double D = d2_of_type(ty, P);
  std::memset(g, 0, sizeof(double) * 12);
  std::memset(H, 0, sizeof(double) * 144);
  *b = 0.0;
  if (!(D > 0.0)) return 2;
  if (D >= dhat * dhat) return 1;
  AD<12> Pv[4][3];
  for (int k = 0; k < 4; ++k)
    for (int c = 0; c < 3; ++c) Pv[k][c] = ad_var<12>(P[k][c], 3 * k + c);
  AD<12> r = pair_barrier<AD<12>>(kind, ty, Pv, dhat, eps_x);
  *b = r.v;
  for (int i = 0; i < 12; ++i) g[i] = r.g[i];
  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < 12; ++j) H[12 * i + j] = r.h[i][j];
  if (free_mask) {
    int idx[12], nf = 0;
    for (int k = 0; k < 4; ++k)
      if (free_mask & (1 << k))
        for (int c = 0; c < 3; ++c) idx[nf++] = 3 * k + c;
    std::vector<double> S(nf * nf);
    for (int i = 0; i < nf; ++i)
      for (int j = 0; j < nf; ++j) S[i * nf + j] = H[12 * idx[i] + idx[j]];
    psd_project(nf, S.data());
    for (int i = 0; i < nf; ++i)
      for (int j = 0; j < nf; ++j) H[12 * idx[i] + idx[j]] = S[i * nf + j];
  }
  return 0;
}

// ACCD on one pair: returns 0 no hit, 1 hit (toi), 2 cap
int or_accd(int kind, const double* Pf, const double* dPf, double s, double tc, int maxit,
            double* toi) {
  double P[4][3], dP[4][3];
  for (int k = 0; k < 4; ++k)
    for (int c = 0; c < 3; ++c) {
      P[k][c] = Pf[3 * k + c];
      dP[k][c] = dPf[3 * k + c];
    }
  *toi = 1.0;
  return accd(kind, P, dP, s, tc, maxit, toi);
}

void or_psd_project(int n, double* A) { psd_project(n, A); }

// ---------------- gel-surface readout (markers, height map) ----------------
// The top surface: the boundary triangles whose rest outward normal points up (+z), the side the
// indenter comes from.  Barycentric coordinates of the point (px, py) in the xy projection of
// triangle (a, b, c) of positions P; false if outside (or degenerate).
static bool xy_bary(const double* P, int a, int b, int c, double px, double py, double l[3]) {
  const double ax = P[3 * a], ay = P[3 * a + 1], bx = P[3 * b], by = P[3 * b + 1], cx = P[3 * c], cy = P[3 * c + 1];
  const double det = (bx - ax) * (cy - ay) - (cx - ax) * (by - ay);
  if (det == 0.0) return false;
  l[1] = ((px - ax) * (cy - ay) - (cx - ax) * (py - ay)) / det;
  l[2] = ((bx - ax) * (py - ay) - (px - ax) * (by - ay)) / det;
  l[0] = 1.0 - l[1] - l[2];
  const double eps = -1e-12;
  return l[0] >= eps && l[1] >= eps && l[2] >= eps;
}

static std::vector<int> top_tris(const Gel& G) {
  std::vector<int> out;
  for (size_t k = 0; k < G.stris.size() / 3; ++k) {
    if (G.st_comp[k] != 0) continue;  // the gelpad: component 0
    const int a = G.stris[3 * k], b = G.stris[3 * k + 1], c = G.stris[3 * k + 2];
    double e1[3], e2[3], n[3];
    sub3(&G.X[3 * b], &G.X[3 * a], e1);
    sub3(&G.X[3 * c], &G.X[3 * a], e2);
    cross3(e1, e2, n);
    if (n[2] > 0.0) out.push_back((int)k);
  }
  return out;
}

// Markers at rest points (mx, my) of the top surface, carried by the gel at positions x: the
// barycentric combination of the containing top triangle's vertices.  found[i] = 0 off the top.
void or_markers(void* g, const double* x, int n, const double* rest_xy, double* out, int* found) {
  const Gel& G = *static_cast<Gel*>(g);
  const std::vector<int> top = top_tris(G);
  for (int i = 0; i < n; ++i) {
    found[i] = 0;
    for (int c = 0; c < 3; ++c) out[3 * i + c] = 0.0;
    for (int k : top) {
      const int a = G.stris[3 * k], b = G.stris[3 * k + 1], c = G.stris[3 * k + 2];
      double l[3];
      if (!xy_bary(G.X.data(), a, b, c, rest_xy[2 * i], rest_xy[2 * i + 1], l)) continue;
      for (int q = 0; q < 3; ++q) out[3 * i + q] = l[0] * x[3 * a + q] + l[1] * x[3 * b + q] + l[2] * x[3 * c + q];
      found[i] = 1;
      break;
    }
  }
}

// Height map of the gel's top surface at positions x: pixel (i, j) at (x0 + (i + 1/2) dx,
// y0 + (j + 1/2) dy) gets the largest z of the top triangles covering it in the xy projection
// (the surface seen from above), NaN where none does.  out is ny x nx, row j = y.
void or_height_map(void* g, const double* x, int nx, int ny, double x0, double y0, double dx, double dy,
                   double* out) {
  const Gel& G = *static_cast<Gel*>(g);
  const std::vector<int> top = top_tris(G);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const double px = x0 + (i + 0.5) * dx, py = y0 + (j + 0.5) * dy;
      double best = std::numeric_limits<double>::quiet_NaN();
      for (int k : top) {
        const int a = G.stris[3 * k], b = G.stris[3 * k + 1], c = G.stris[3 * k + 2];
        double l[3];
        if (!xy_bary(x, a, b, c, px, py, l)) continue;
        const double z = l[0] * x[3 * a + 2] + l[1] * x[3 * b + 2] + l[2] * x[3 * c + 2];
        if (!(z <= best)) best = z;  // also replaces the initial NaN
      }
      out[j * nx + i] = best;
    }
}

// friction coefficient (0: no friction, the default) and velocity threshold eps_v [m/s]
void or_set_friction(void* g, double mu, double eps_v) {
  Gel& G = *static_cast<Gel*>(g);
  G.fric_mu = mu;
  G.fric_epsv = eps_v;
}

// Lagged friction of one pair: setup from the points Plag at the start of the step (normal
// force from kappa, dhat, eps_x), then D, dD/dP (12) and d2D/dP2 (144) at the points Pnow;
// eh = eps_v h.  Returns 1 if the pair is in contact at the start (else 0 and zeros), and the
// lagged normal force in *lam.
int or_friction_pair(int kind, const double* Plag, const double* Pnow, double dhat, double kappa,
                     double eps_x, double mu, double eh, double* e, double* g, double* H, double* lam) {
  double P0[4][3];
  AD<12> Pv[4][3];
  for (int k = 0; k < 4; ++k)
    for (int c = 0; c < 3; ++c) {
      P0[k][c] = Plag[3 * k + c];
      Pv[k][c] = ad_var<12>(Pnow[3 * k + c], 3 * k + c);
    }
  FricPair f;
  *e = 0.0;
  *lam = 0.0;
  for (int i = 0; i < 12; ++i) g[i] = 0.0;
  for (int i = 0; i < 144; ++i) H[i] = 0.0;
  if (!fric_setup(kind, P0, dhat, kappa, eps_x, &f)) return 0;
  const AD<12> D = fric_energy<AD<12>>(f, Pv, mu, eh);
  *e = D.v;
  *lam = f.lam;
  for (int i = 0; i < 12; ++i) g[i] = D.g[i];
  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < 12; ++j) H[12 * i + j] = D.h[i][j];
  return 1;
}

// The stationarity rule on its own: 1 if a failed line search with model decrease -gp at energy E
// ends the solve as converged, 0 if the step fails (READING R8b).
int or_stationary_rule(double gp, double E) { return stationary_to_resolution(gp, E) ? 1 : 0; }

// Solves of the last step that ended by the stationarity rule (READING R8b: the line search
// found no resolvable decrease and -g.p <= 1e-10 |E|).
int or_last_stationary(void* g) { return static_cast<Gel*>(g)->st_stationary; }
int or_last_kappa_doublings(void* g) { return static_cast<Gel*>(g)->st_kappa_doublings; }
double or_kappa(void* g) { return static_cast<Gel*>(g)->kappa; }
// READING R5b: adaptive kappa with cap = scale * kappa0 (scale <= 0: off) and threshold dmin [m]
void or_set_kappa_adapt(void* g, double scale, double dmin) {
  Gel& G = *static_cast<Gel*>(g);
  G.kappa_cap = scale > 0.0 ? scale * G.kappa0 : 0.0;
  G.kappa_dmin = dmin;
}

// Threads of the parallel loops (n <= 0: all available); results do not depend on it.
void or_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
  (void)n;
#endif
}
int or_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_eigh(int n, const double* A, double* w, double* V) {
  std::vector<double> M(A, A + n * n), ww, VV;
  jacobi_eig(n, M, ww, VV);
  std::memcpy(w, ww.data(), sizeof(double) * n);
  std::memcpy(V, VV.data(), sizeof(double) * n * n);
}

// Jacobi-PCG on a CSR system (test hook); returns iterations or -1
int or_pcg_csr(int n, const int* rp, const int* ci, const double* va, const double* b, double* x,
               double tol, int maxit) {
  CSR A;
  A.n = n;
  A.rp.assign(rp, rp + n + 1);
  A.ci.assign(ci, ci + rp[n]);
  A.va.assign(va, va + rp[n]);
  std::vector<double> bb(b, b + n), xx;
  int it = pcg(A, bb, xx, tol, maxit);
  std::memcpy(x, xx.data(), sizeof(double) * n);
  return it;
}

// Number of candidate pairs of each type (PT, TP, EE, SPT, SEE) for the gel at x and the
// indenter at `pose`, then the number of those within dhat (active): counts[0..4], counts[5..9].
void or_pair_counts(void* g, const double* x, const double* pose, int* counts) {
  Gel& G = *static_cast<Gel*>(g);
  std::vector<double> IW(3 * G.M);
  pose_apply(pose, G.IV.data(), G.M, IW.data());
  std::vector<PairRef> pairs = candidate_pairs(G, x, x, IW.data(), IW.data(), G.dhat);
  for (int i = 0; i < 10; ++i) counts[i] = 0;
  for (const PairRef& pr : pairs) {
    counts[pr.type]++;
    double P[4][3];
    int gi[4];
    pair_points(G, x, IW.data(), pr, P, gi);
    if (pair_d2(kind_of(pr), P) < G.dhat * G.dhat) counts[5 + pr.type]++;
  }
}

// Number of connected components of the tet mesh, and the component of each vertex (comp[N]).
int or_components(void* g, int* comp) {
  const Gel& G = *static_cast<Gel*>(g);
  if (comp) std::copy(G.comp.begin(), G.comp.end(), comp);
  return G.ncomp;
}

}  // extern "C"

// Barrier derivatives of one contact pair on the threads of a team (a warp or a CTA), and the
// PSD projection of its Hessian block by a team-parallel Jacobi eigen-solve.  The contact
// kernels use a warp per pair; the code also runs on a whole CTA (every thread calls it).
//
// The squared distance D of every closest-feature form is a function of nd <= 3 difference
// vectors v_a = P[pl_a] - P[mi_a] (see dev_contact.cuh).  Its gradient over the v_a is cheap and
// is formed once per pair (struct DV); every entry of its Hessian over the v_a has a closed form
// (cross norm c(x, y) = |x|^2 |y|^2 - (x.y)^2, triple product s = w.(e1 x e2), quotient rule), so
// the threads of a team compute the entries of the point-space block they own independently:
//   d2D/dP_I dP_J = sum_{a,b} sigma(I, a) sigma(J, b) d2D/dv_a dv_b,  sigma = +1 (plus point),
//   -1 (minus point), 0.
// The barrier on D and the IPC edge-edge mollifier are then applied entry by entry.
//
// Projection (Li et al. 2020: per-pair Hessians are projected to PSD before assembly).  Cyclic
// Jacobi with the round-robin ("parallel") ordering of Brent & Luk: each round applies m/2
// disjoint rotations at once; thread k owns the 2x2 block (pair a, pair b) of the matrix it
// transforms, so no two threads write the same entry.  GB300 issues FP64 at 1/64 of the FP32
// rate, so the eigenbasis is found in FP32 first; FP64 then re-orthonormalises it and refines
// only what FP32 could not resolve; the clamp X max(lam, 0) X^T is assembled in FP64.
#pragma once
#include "dev_contact.cuh"

namespace txg {

// The threads that work on one pair: a warp (NT = 32) or a whole CTA (NT = 64, 128, ...; every
// thread of the CTA calls the team functions).  id is the thread's index in the team; red is
// NT / 32 doubles of shared scratch for the CTA-wide reductions (unused by a warp).
template <int NT>
struct Team {
  int id;
  double* red;
  __device__ __forceinline__ void sync() const {
    if constexpr (NT == 32)
      __syncwarp();
    else
      __syncthreads();
  }
  __device__ __forceinline__ bool any(bool p) const {
    if constexpr (NT == 32)
      return __any_sync(0xffffffffu, p);
    else
      return __syncthreads_or(p) != 0;
  }
  template <typename T>
  __device__ __forceinline__ T sum(T v) const {
    v = warp_sum(v);
    if constexpr (NT == 32) {
      return v;
    } else {
      __syncthreads();  // the previous reduction's readers are done with red
      if ((id & 31) == 0) red[id >> 5] = (double)v;
      __syncthreads();
      T t = T(0);
#pragma unroll
      for (int w = 0; w < NT / 32; ++w) t += (T)red[w];
      return t;
    }
  }
  template <typename T>
  __device__ __forceinline__ T max(T v) const {
    v = warp_max(v);
    if constexpr (NT == 32) {
      return v;
    } else {
      __syncthreads();
      if ((id & 31) == 0) red[id >> 5] = (double)v;
      __syncthreads();
      T t = (T)red[0];
#pragma unroll
      for (int w = 1; w < NT / 32; ++w) t = t > (T)red[w] ? t : (T)red[w];
      return t;
    }
  }
};

// closest-feature data of a pair in difference-vector space
struct DV {
  int form, nd;
  int pl[3], mi[3];
  double v[3][3];
  double D;
  double s, W;     // PT / LL: s = w.(e1 x e2), W = c(e1, e2);  PE: s = c(w, e), W = |e|^2
  double iW;       // 1 / W
  double gD[9];    // dD/dv
  double gs[9];    // PT / LL: ds/dv;  PE: d c(w, e)/dv
  double gW[9];    // dW/dv
};

__device__ __forceinline__ void cn_grad(const double* x, const double* y, double* gx, double* gy) {
  const double xx = dot3(x, x), yy = dot3(y, y), xy = dot3(x, y);
  for (int c = 0; c < 3; ++c) {
    gx[c] = 2.0 * yy * x[c] - 2.0 * xy * y[c];
    gy[c] = 2.0 * xx * y[c] - 2.0 * xy * x[c];
  }
}

__device__ __forceinline__ void dv_setup(const DType& t, const double P[4][3], DV& o) {
  o.form = t.f;
  for (int k = 0; k < 9; ++k) o.gD[k] = o.gs[k] = o.gW[k] = 0.0;
  for (int a = 0; a < 3; ++a) {
    o.pl[a] = o.mi[a] = -1;
    o.v[a][0] = o.v[a][1] = o.v[a][2] = 0.0;
  }
  o.s = 0.0;
  o.W = 1.0;
  o.iW = 1.0;
  if (t.f == DF_PP) {
    o.nd = 1;
    o.pl[0] = t.i[0];
    o.mi[0] = t.i[1];
    sub3(P[t.i[0]], P[t.i[1]], o.v[0]);
    o.D = dot3(o.v[0], o.v[0]);
    for (int c = 0; c < 3; ++c) o.gD[c] = 2.0 * o.v[0][c];
    return;
  }
  if (t.f == DF_PE) {
    o.nd = 2;
    o.pl[0] = t.i[0]; o.mi[0] = t.i[1];
    o.pl[1] = t.i[2]; o.mi[1] = t.i[1];
    sub3(P[t.i[0]], P[t.i[1]], o.v[0]);
    sub3(P[t.i[2]], P[t.i[1]], o.v[1]);
    const double* w = o.v[0];
    const double* e = o.v[1];
    const double we = dot3(w, e);
    o.s = dot3(w, w) * dot3(e, e) - we * we;
    o.W = dot3(e, e);
    cn_grad(w, e, o.gs, o.gs + 3);
    for (int c = 0; c < 3; ++c) o.gW[3 + c] = 2.0 * e[c];
    o.D = o.s / o.W;
    o.iW = 1.0 / o.W;
    for (int k = 0; k < 6; ++k) o.gD[k] = (o.gs[k] - o.D * o.gW[k]) / o.W;
    return;
  }
  o.nd = 3;
  if (t.f == DF_PT) {
    o.pl[0] = t.i[0]; o.mi[0] = t.i[1];
    o.pl[1] = t.i[2]; o.mi[1] = t.i[1];
    o.pl[2] = t.i[3]; o.mi[2] = t.i[1];
  } else {  // LL
    o.pl[0] = t.i[2]; o.mi[0] = t.i[0];
    o.pl[1] = t.i[1]; o.mi[1] = t.i[0];
    o.pl[2] = t.i[3]; o.mi[2] = t.i[2];
  }
  for (int a = 0; a < 3; ++a) sub3(P[o.pl[a]], P[o.mi[a]], o.v[a]);
  const double* w = o.v[0];
  const double* e1 = o.v[1];
  const double* e2 = o.v[2];
  double n[3];
  cross3(e1, e2, n);
  cross3(e2, w, o.gs + 3);
  cross3(w, e1, o.gs + 6);
  for (int c = 0; c < 3; ++c) o.gs[c] = n[c];
  o.s = dot3(w, n);
  const double ee = dot3(e1, e2);
  o.W = dot3(e1, e1) * dot3(e2, e2) - ee * ee;
  cn_grad(e1, e2, o.gW + 3, o.gW + 6);
  o.D = o.s * o.s / o.W;
  o.iW = 1.0 / o.W;
  for (int k = 0; k < 9; ++k) o.gD[k] = (2.0 * o.s * o.gs[k] - o.D * o.gW[k]) / o.W;
}

// sign of point p in difference vector a
__device__ __forceinline__ double dv_sigma(const DV& o, int p, int a) {
  return (o.pl[a] == p ? 1.0 : 0.0) - (o.mi[a] == p ? 1.0 : 0.0);
}

// Hessian entry of the cross norm c(x, y): variables a, b in {0: x, 1: y}, components c, e
__device__ __forceinline__ double cn_entry(const double* x, const double* y, int a, int c, int b, int e) {
  const double dl = c == e ? 1.0 : 0.0;
  if (a == 0 && b == 0) return 2.0 * dot3(y, y) * dl - 2.0 * y[c] * y[e];
  if (a == 1 && b == 1) return 2.0 * dot3(x, x) * dl - 2.0 * x[c] * x[e];
  if (a == 0) return 4.0 * x[c] * y[e] - 2.0 * y[c] * x[e] - 2.0 * dot3(x, y) * dl;
  return 4.0 * x[e] * y[c] - 2.0 * y[e] * x[c] - 2.0 * dot3(x, y) * dl;
}

// entry (i, j) of the cross-product matrix [v]x
__device__ __forceinline__ double skew_entry(const double* v, int i, int j) {
  if (i == j) return 0.0;
  const int k = 3 - i - j;
  return j == (i + 1) % 3 ? -v[k] : v[k];
}

// d2D / dv_a,c dv_b,e
__device__ __forceinline__ double hD_dv(const DV& o, int a, int c, int b, int e) {
  if (o.form == DF_PP) return c == e ? 2.0 : 0.0;
  const int ia = 3 * a + c, ib = 3 * b + e;
  if (o.form == DF_PE) {
    const double HN = cn_entry(o.v[0], o.v[1], a, c, b, e);
    const double HL = (a == 1 && b == 1 && c == e) ? 2.0 : 0.0;
    return (HN - o.D * HL - o.gD[ia] * o.gW[ib] - o.gW[ia] * o.gD[ib]) * o.iW;
  }
  // second derivatives of the triple product w.(e1 x e2) (zero within one vector)
  double Hs = 0.0;
  if (a != b) {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    const int r = a < b ? c : e, q = a < b ? e : c;  // component of the lower / higher vector
    if (lo == 0 && hi == 1) Hs = -skew_entry(o.v[2], r, q);
    else if (lo == 0 && hi == 2) Hs = skew_entry(o.v[1], r, q);
    else Hs = -skew_entry(o.v[0], r, q);
  }
  const double HW = (a >= 1 && b >= 1) ? cn_entry(o.v[1], o.v[2], a - 1, c, b - 1, e) : 0.0;
  return (2.0 * o.gs[ia] * o.gs[ib] + 2.0 * o.s * Hs - o.D * HW - o.gD[ia] * o.gW[ib] - o.gW[ia] * o.gD[ib]) * o.iW;
}

// d2D / dP_I dP_J (point-space dofs I, J in [0, 12))
__device__ __forceinline__ double hD_point(const DV& o, int I, int J) {
  const int p = I / 3, c = I % 3, q = J / 3, e = J % 3;
  double h = 0.0;
  for (int a = 0; a < o.nd; ++a) {
    const double sa = dv_sigma(o, p, a);
    if (sa == 0.0) continue;
    for (int b = 0; b < o.nd; ++b) {
      const double sb = dv_sigma(o, q, b);
      if (sb == 0.0) continue;
      h += sa * sb * hD_dv(o, a, c, b, e);
    }
  }
  return h;
}

// point-space gradient of D
__device__ __forceinline__ void gD_point(const DV& o, double g[12]) {
  for (int k = 0; k < 12; ++k) g[k] = 0.0;
  for (int a = 0; a < o.nd; ++a)
    for (int c = 0; c < 3; ++c) {
      g[3 * o.pl[a] + c] += o.gD[3 * a + c];
      g[3 * o.mi[a] + c] -= o.gD[3 * a + c];
    }
}

// Barrier of a pair in point space (without kappa).  kind 1 (edge-edge) carries the IPC mollifier
// m(c) = (2 - c/eps) c/eps of the edges' cross norm c below eps_x.
struct PairBarrier {
  DV dv;
  double b0, bD, bDD;     // b(D), db/dD, d2b/dD2 (unmollified)
  double gDp[12];         // dD/dP
  int moll;               // mollifier active
  double m, m1, m2;       // m(c), m'(c), m''(c)
  double ea[3], eb[3];    // edge vectors (kind 1)
  double gcp[12];         // dc/dP (kind 1, mollified)
  double b;               // mollified barrier value
  int involved;           // bit mask of the points the value depends on
};

// Returns false when d >= dhat.
__device__ __forceinline__ bool pair_barrier_setup(int kind, const double P[4][3], double dhat, double eps_x,
                                                   PairBarrier& pb, DType* tyo = nullptr) {
  DType ty;
  const double D0 = pair_d2(kind, P, &ty);
  if (tyo) *tyo = ty;
  if (!(D0 < dhat * dhat)) return false;
  dv_setup(ty, P, pb.dv);
  barrier_D(pb.dv.D, dhat, &pb.b0, &pb.bD, &pb.bDD);
  gD_point(pb.dv, pb.gDp);
  const int np = ty.f == DF_PP ? 2 : (ty.f == DF_PE ? 3 : 4);
  int msk = 0;
  for (int k = 0; k < np; ++k) msk |= 1 << ty.i[k];
  pb.involved = msk;
  pb.moll = 0;
  pb.m = 1.0;
  pb.m1 = pb.m2 = 0.0;
  pb.b = pb.b0;
  for (int k = 0; k < 12; ++k) pb.gcp[k] = 0.0;
  if (kind == 1) {
    sub3(P[1], P[0], pb.ea);
    sub3(P[3], P[2], pb.eb);
    const double ab = dot3(pb.ea, pb.eb);
    const double c = dot3(pb.ea, pb.ea) * dot3(pb.eb, pb.eb) - ab * ab;
    if (c < eps_x) {
      pb.moll = 1;
      pb.involved = 0xF;
      const double q = c / eps_x;
      pb.m = (2.0 - q) * q;
      pb.m1 = 2.0 * (1.0 - q) / eps_x;
      pb.m2 = -2.0 / (eps_x * eps_x);
      double ga[3], gb[3];
      cn_grad(pb.ea, pb.eb, ga, gb);
      for (int c3 = 0; c3 < 3; ++c3) {
        pb.gcp[c3] = -ga[c3];
        pb.gcp[3 + c3] = ga[c3];
        pb.gcp[6 + c3] = -gb[c3];
        pb.gcp[9 + c3] = gb[c3];
      }
      pb.b = pb.m * pb.b0;
    }
  }
  return true;
}

__device__ __forceinline__ double pair_grad_entry(const PairBarrier& pb, int I) {
  const double gb = pb.bD * pb.gDp[I];
  return pb.moll ? pb.m * gb + pb.b0 * pb.m1 * pb.gcp[I] : gb;
}

// d2b/dP_I dP_J of the (mollified) barrier, given hDp = d2D/dP_I dP_J
__device__ __forceinline__ double pair_hess_compose(const PairBarrier& pb, int I, int J, double hDp) {
  double h = pb.bDD * pb.gDp[I] * pb.gDp[J] + pb.bD * hDp;
  if (pb.moll) {
    const int p = I / 3, c = I % 3, q = J / 3, e = J % 3;
    // cross-norm Hessian over the points: edge a = (P0 -> P1), edge b = (P2 -> P3)
    const int ap = p < 2 ? 0 : 1, aq = q < 2 ? 0 : 1;
    const double sp = (p == 1 || p == 3) ? 1.0 : -1.0, sq = (q == 1 || q == 3) ? 1.0 : -1.0;
    const double Hc = sp * sq * cn_entry(pb.ea, pb.eb, ap, c, aq, e);
    const double gbI = pb.bD * pb.gDp[I], gbJ = pb.bD * pb.gDp[J];
    h = pb.m * h + pb.m1 * (pb.gcp[I] * gbJ + gbI * pb.gcp[J]) +
        pb.b0 * (pb.m2 * pb.gcp[I] * pb.gcp[J] + pb.m1 * Hc);
  }
  return h;
}

__device__ __forceinline__ double pair_hess_entry(const PairBarrier& pb, int I, int J) {
  return pair_hess_compose(pb, I, J, hD_point(pb.dv, I, J));
}

// position of round-robin slot pa (1..m-1) in round r: slots 1..m-1 rotate by r
__device__ __forceinline__ int rr_pos(int pa, int r, int m) {
  int x = pa - 1 + r;  // < 2 (m - 1)
  if (x >= m - 1) x -= m - 1;
  return x + 1;
}
// v / h for v < 2^16 / h, with ih = ceil(2^16 / h) (h <= 12 here, v < 200)
__device__ __forceinline__ int div_small(int v, unsigned ih) { return (int)(((unsigned)v * ih) >> 16); }

// The block of the barrier Hessian on the point dofs fd[0, nf) into H (row stride m, rows and
// columns nf..m-1 zero), by the threads of a team: the difference-vector Hessian of D is formed
// once (Hdv: (3 nd)^2 scratch), every point entry is then a signed sum of its entries.  Entries
// (i, j) and (j, i) are computed in the same order, so H is exactly symmetric.
template <int NT>
__device__ __forceinline__ void team_pair_block(const PairBarrier& pb, const int* fd, int nf, int m, double* Hdv,
                                                double* H, const Team<NT>& tm) {
  const DV& o = pb.dv;
  const int n3 = 3 * o.nd;
  const unsigned in3 = (65536u + n3 - 1) / n3, im = (65536u + m - 1) / m;
  for (int e = tm.id; e < n3 * n3; e += NT) {
    const int r = div_small(e, in3), c = e - r * n3;
    const int a = r < c ? r : c, b = r < c ? c : r;
    Hdv[e] = hD_dv(o, a / 3, a % 3, b / 3, b % 3);
  }
  tm.sync();
  for (int e = tm.id; e < m * m; e += NT) {
    const int r = div_small(e, im), c = e - r * m;
    const int i = r < c ? r : c, j = r < c ? c : r;
    double v = 0.0;
    if (j < nf) {
      const int I = fd[i], J = fd[j];
      const int p = I / 3, ci = I - 3 * p, q = J / 3, cj = J - 3 * q;
      double h = 0.0;
      for (int a = 0; a < o.nd; ++a) {
        const double sa = dv_sigma(o, p, a);
        if (sa == 0.0) continue;
        for (int b = 0; b < o.nd; ++b) {
          const double sb = dv_sigma(o, q, b);
          if (sb == 0.0) continue;
          const double x = Hdv[(3 * a + ci) * n3 + 3 * b + cj];
          h += sa * sb > 0.0 ? x : -x;
        }
      }
      v = pair_hess_compose(pb, I, J, h);
    }
    H[e] = v;
  }
  tm.sync();
}

// ---------------------------------------------------------------- team-parallel Jacobi
constexpr int PW_MAXN = 12;  // largest block: all four points of a pair

template <typename T>
struct RotWS {
  T c[PW_MAXN / 2], s[PW_MAXN / 2], t[PW_MAXN / 2];
  int p[PW_MAXN / 2], q[PW_MAXN / 2];
};

__device__ __forceinline__ float jabs(float v) { return fabsf(v); }
__device__ __forceinline__ double jabs(double v) { return fabs(v); }
__device__ __forceinline__ float jsqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double jsqrt(double v) { return sqrt(v); }

// Cyclic Jacobi on the symmetric m x m matrix A (m even, row stride m) in shared memory,
// accumulating the rotations into V (A <- J^T A J, V <- V J).  Stops when the squared
// off-diagonal norm is at most rel_tol times the squared diagonal norm.  Rotations whose
// off-diagonal entry is below skip_rel (|a_pp| + |a_qq|) are skipped (exact identity).
// Called by every thread of the team.
template <typename T, int NT>
__device__ void team_jacobi(T* A, T* V, int m, int max_sweeps, T rel_tol, T skip_rel, RotWS<T>& rw,
                            const Team<NT>& tm) {
  const int h = m >> 1;
  const unsigned ih = (65536u + h - 1) / h, im = (65536u + m - 1) / m;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    T off = 0, dg = 0;
    for (int e = tm.id; e < m * m; e += NT) {
      const int i = div_small(e, im), j = e - i * m;
      const T v = A[e];
      if (i == j) dg += v * v;
      else if (i < j) off += v * v;
    }
    off = tm.sum(off);
    dg = tm.sum(dg);
    if (!(off > rel_tol * dg)) break;
    for (int r = 0; r < m - 1; ++r) {
      if (tm.id < h) {
        // round-robin: position 0 fixed, positions 1..m-1 rotate by r
        const int pa = tm.id == 0 ? 0 : tm.id + 1, pb = tm.id == 0 ? 1 : m - tm.id;
        int p = pa == 0 ? 0 : rr_pos(pa, r, m);
        int q = rr_pos(pb, r, m);
        if (p > q) {
          const int x = p;
          p = q;
          q = x;
        }
        const T apq = A[p * m + q], app = A[p * m + p], aqq = A[q * m + q];
        T c = 1, s = 0, t = 0;
        if (apq != T(0) && jabs(apq) > skip_rel * (jabs(app) + jabs(aqq))) {
          if constexpr (sizeof(T) == 4) {  // approximate quotients: the FP64 refinement follows
            const float th = __fdividef(aqq - app, 2.f * apq);
            t = copysignf(__fdividef(1.f, fabsf(th) + sqrtf(fmaf(th, th, 1.f))), th);
            c = rsqrtf(fmaf(t, t, 1.f));
          } else {
            const T th = (aqq - app) / (T(2) * apq);
            t = (th >= T(0) ? T(1) : T(-1)) / (jabs(th) + jsqrt(th * th + T(1)));
            c = T(1) / jsqrt(t * t + T(1));
          }
          s = t * c;
        }
        rw.p[tm.id] = p;
        rw.q[tm.id] = q;
        rw.c[tm.id] = c;
        rw.s[tm.id] = s;
        rw.t[tm.id] = t;
      }
      tm.sync();
      for (int blk = tm.id; blk < h * h; blk += NT) {
        const int a = div_small(blk, ih), b = blk - a * h;
        const int pa = rw.p[a], qa = rw.q[a], pb = rw.p[b], qb = rw.q[b];
        if (a == b) {
          const T t = rw.t[a];
          if (t != T(0)) {
            const T apq = A[pa * m + qa];
            A[pa * m + pa] -= t * apq;
            A[qa * m + qa] += t * apq;
            A[pa * m + qa] = A[qa * m + pa] = T(0);
          }
        } else {
          const T ca = rw.c[a], sa = rw.s[a], cb = rw.c[b], sb = rw.s[b];
          const T x00 = A[pa * m + pb], x01 = A[pa * m + qb], x10 = A[qa * m + pb], x11 = A[qa * m + qb];
          const T y00 = ca * x00 - sa * x10, y01 = ca * x01 - sa * x11;
          const T y10 = sa * x00 + ca * x10, y11 = sa * x01 + ca * x11;
          A[pa * m + pb] = cb * y00 - sb * y01;
          A[pa * m + qb] = sb * y00 + cb * y01;
          A[qa * m + pb] = cb * y10 - sb * y11;
          A[qa * m + qb] = sb * y10 + cb * y11;
        }
      }
      for (int task = tm.id; task < m * h; task += NT) {
        const int k = div_small(task, ih), a = task - k * h;
        const int p = rw.p[a], q = rw.q[a];
        const T c = rw.c[a], s = rw.s[a];
        const T vp = V[k * m + p], vq = V[k * m + q];
        V[k * m + p] = c * vp - s * vq;
        V[k * m + q] = s * vp + c * vq;
      }
      tm.sync();
    }
  }
}

// FP64 refinement sweeps of cyclic Jacobi (round-robin order) on a symmetric A that an
// orthonormal basis already nearly diagonalises.  Rotation angles come from the FP32 quotient
// (a_qq - a_pp) / (2 a_pq); the rotation itself (c = 1 / sqrt(1 + t^2), s = t c) and every update
// are FP64, so each sweep multiplies the off-diagonal entries by ~1e-7 and keeps V orthonormal to
// FP64 round-off.  Entries below tau (absolute) are left alone, and a round none of whose pairs
// needs a rotation is skipped by the whole team; a sweep without rotations ends the refinement.
template <int NT>
__device__ void team_jacobi_refine(double* A, double* V, int m, int max_sweeps, double tau, RotWS<double>& rw,
                                   const Team<NT>& tm) {
  const int h = m >> 1;
  const unsigned ih = (65536u + h - 1) / h;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    bool rotated = false;
    for (int r = 0; r < m - 1; ++r) {
      bool rot = false;
      if (tm.id < h) {
        const int pa = tm.id == 0 ? 0 : tm.id + 1, pb = tm.id == 0 ? 1 : m - tm.id;
        int p = pa == 0 ? 0 : rr_pos(pa, r, m);
        int q = rr_pos(pb, r, m);
        if (p > q) {
          const int x = p;
          p = q;
          q = x;
        }
        const double apq = A[p * m + q];
        double c = 1.0, s = 0.0;
        if (fabs(apq) > tau) {
          const float th = (float)(A[q * m + q] - A[p * m + p]) / (2.f * (float)apq);
          const float t32 = (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(fmaf(th, th, 1.f)));
          const double t = (double)t32;
          c = rsqrt(fma(t, t, 1.0));
          s = t * c;
          rot = true;
        }
        rw.p[tm.id] = p;
        rw.q[tm.id] = q;
        rw.c[tm.id] = c;
        rw.s[tm.id] = s;
      }
      if (!tm.any(rot)) continue;
      rotated = true;
      tm.sync();
      for (int blk = tm.id; blk < h * h; blk += NT) {
        const int a = div_small(blk, ih), b = blk - a * h;
        const int pa = rw.p[a], qa = rw.q[a], pb = rw.p[b], qb = rw.q[b];
        const double ca = rw.c[a], sa = rw.s[a], cb = rw.c[b], sb = rw.s[b];
        const double x00 = A[pa * m + pb], x01 = A[pa * m + qb], x10 = A[qa * m + pb], x11 = A[qa * m + qb];
        const double y00 = ca * x00 - sa * x10, y01 = ca * x01 - sa * x11;
        const double y10 = sa * x00 + ca * x10, y11 = sa * x01 + ca * x11;
        A[pa * m + pb] = cb * y00 - sb * y01;
        A[pa * m + qb] = sb * y00 + cb * y01;
        A[qa * m + pb] = cb * y10 - sb * y11;
        A[qa * m + qb] = sb * y10 + cb * y11;
      }
      for (int task = tm.id; task < m * h; task += NT) {
        const int k = div_small(task, ih), a = task - k * h;
        const int p = rw.p[a], q = rw.q[a];
        const double c = rw.c[a], s = rw.s[a];
        const double vp = V[k * m + p], vq = V[k * m + q];
        V[k * m + p] = c * vp - s * vq;
        V[k * m + q] = s * vp + c * vq;
      }
      tm.sync();
    }
    if (!rotated) break;
  }
}

// per-team workspace of the projection
struct ProjWS {
  double H[PW_MAXN * PW_MAXN];  // in: symmetric block (stride m); out: its PSD projection
  double X[PW_MAXN * PW_MAXN], T[PW_MAXN * PW_MAXN], B[PW_MAXN * PW_MAXN];
  float a32[PW_MAXN * PW_MAXN];
  float v32[PW_MAXN * PW_MAXN];
  RotWS<float> r32;
  RotWS<double> r64;
};

// (i, j), i <= j, of the t-th entry of the upper triangle of an m x m matrix, row by row
__device__ __forceinline__ void upper_ij(int t, int m, int& i, int& j) {
  i = 0;
  while (t >= m - i) {
    t -= m - i;
    ++i;
  }
  j = i + t;
}

// PSD projection of w.H (n x n symmetric, stored with stride m = n rounded up to even, padding
// rows / columns zero); every thread of the team calls it.
//   1. scale by a power of two (exact): max |A| in [1, 2);
//   2. FP32 round-robin Jacobi: eigenvector estimate X (orthonormal to ~1e-7);
//   3. one Newton-Schulz step X <- X (3 I - X^T X) / 2 in FP64 (orthonormal to ~1e-14);
//   4. B = X^T A X (FP64), refined by FP64 Jacobi sweeps until its off-diagonal entries are
//      below 1e-13 max|A| -- the well-separated part needs one sweep, close or tiny eigenvalues
//      (the barrier's Hessian spans many orders of magnitude) as many as they take;
//   5. H = X max(diag B, 0) X^T (FP64), scaled back.
template <int NT>
__device__ void team_psd_project(ProjWS& w, int n, const Team<NT>& tm) {
  const int m = n + (n & 1), mm = m * m, nu = m * (m + 1) / 2;
  const unsigned im = (65536u + m - 1) / m;
  double mx = 0.0;
  for (int e = tm.id; e < mm; e += NT) mx = fmax(mx, fabs(w.H[e]));
  mx = tm.max(mx);
  if (!(mx > 0.0)) return;  // zero block: already its own projection
  const int ex = ilogb(mx);
  const double sc = ldexp(1.0, -ex);
  for (int e = tm.id; e < mm; e += NT) {
    const int i = div_small(e, im), j = e - i * m;
    const double v = w.H[e] * sc;
    w.H[e] = v;
    w.a32[e] = (float)v;
    w.v32[e] = i == j ? 1.f : 0.f;
  }
  tm.sync();
  team_jacobi<float, NT>(w.a32, w.v32, m, 10, 1e-12f, 1e-9f, w.r32, tm);
  for (int e = tm.id; e < mm; e += NT) w.X[e] = (double)w.v32[e];
  tm.sync();
  for (int t = tm.id; t < nu; t += NT) {  // T = X^T X (upper, mirrored)
    int i, j;
    upper_ij(t, m, i, j);
    double acc = 0.0;
    for (int k = 0; k < m; ++k) acc = fma(w.X[k * m + i], w.X[k * m + j], acc);
    w.T[i * m + j] = w.T[j * m + i] = acc;
  }
  tm.sync();
  for (int e = tm.id; e < mm; e += NT) {  // B = X (3 I - T) / 2
    const int i = div_small(e, im), j = e - i * m;
    double acc = 0.0;
    for (int k = 0; k < m; ++k) acc = fma(w.X[i * m + k], w.T[k * m + j], acc);
    w.B[e] = 1.5 * w.X[e] - 0.5 * acc;
  }
  tm.sync();
  for (int e = tm.id; e < mm; e += NT) {  // T = A X
    const int i = div_small(e, im), j = e - i * m;
    double acc = 0.0;
    for (int k = 0; k < m; ++k) acc = fma(w.H[i * m + k], w.B[k * m + j], acc);
    w.T[e] = acc;
  }
  tm.sync();
  for (int e = tm.id; e < mm; e += NT) w.X[e] = w.B[e];
  tm.sync();
  for (int t = tm.id; t < nu; t += NT) {  // B = X^T T (upper, mirrored)
    int i, j;
    upper_ij(t, m, i, j);
    double acc = 0.0;
    for (int k = 0; k < m; ++k) acc = fma(w.X[k * m + i], w.T[k * m + j], acc);
    w.B[i * m + j] = w.B[j * m + i] = acc;
  }
  tm.sync();
  team_jacobi_refine<NT>(w.B, w.X, m, 6, 1e-13, w.r64, tm);
  const double isc = ldexp(1.0, ex);
  for (int t = tm.id; t < nu; t += NT) {  // H = X max(diag B, 0) X^T
    int i, j;
    upper_ij(t, m, i, j);
    double acc = 0.0;
    for (int k = 0; k < m; ++k) {
      const double lk = w.B[k * m + k];
      if (lk > 0.0) acc = fma(w.X[i * m + k] * lk, w.X[j * m + k], acc);
    }
    w.H[i * m + j] = w.H[j * m + i] = acc * isc;
  }
  tm.sync();
}

}  // namespace txg

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
// in difference-vector space (triple product, cross norm, quotient rule; dev_pairwarp.cuh).
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
  } else if (pr.x == PAIR_EE) {
    const int2 e = d.se[pr.y];
    gel(0, e.x);
    gel(1, e.y);
    const int2 f = d.ie[pr.z];
    indv(2, f.x);
    indv(3, f.y);
  } else if (pr.x == PAIR_SPT) {  // both primitives on the gel's mesh
    gel(0, d.sv[pr.y]);
    const int4 t = d.st[pr.z];
    gel(1, t.x);
    gel(2, t.y);
    gel(3, t.z);
  } else {
    const int2 e = d.se[pr.y], f = d.se[pr.z];
    gel(0, e.x);
    gel(1, e.y);
    gel(2, f.x);
    gel(3, f.y);
  }
}

// gel row of each slot of a candidate pair (-1 for indenter slots), as in pair_points
__device__ __forceinline__ void pair_rows(const Dev& d, const int4& pr, int rows[4]) {
  if (pr.x == PAIR_PT) {
    rows[0] = d.sv[pr.y];
    rows[1] = rows[2] = rows[3] = -1;
  } else if (pr.x == PAIR_TP) {
    const int4 t = d.st[pr.y];
    rows[0] = -1;
    rows[1] = t.x;
    rows[2] = t.y;
    rows[3] = t.z;
  } else if (pr.x == PAIR_EE) {
    const int2 e = d.se[pr.y];
    rows[0] = e.x;
    rows[1] = e.y;
    rows[2] = rows[3] = -1;
  } else if (pr.x == PAIR_SPT) {
    const int4 t = d.st[pr.z];
    rows[0] = d.sv[pr.y];
    rows[1] = t.x;
    rows[2] = t.y;
    rows[3] = t.z;
  } else {
    const int2 e = d.se[pr.y], f = d.se[pr.z];
    rows[0] = e.x;
    rows[1] = e.y;
    rows[2] = f.x;
    rows[3] = f.y;
  }
}

// IPC's edge-edge mollifier threshold eps_x = 1e-3 |e_a|^2 |e_b|^2 from the rest lengths
__device__ __forceinline__ double pair_eps_x(const Dev& d, const int4& pr) {
  if (pr.x == PAIR_SEE) return 1e-3 * d.se_len2[pr.y] * d.se_len2[pr.z];
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

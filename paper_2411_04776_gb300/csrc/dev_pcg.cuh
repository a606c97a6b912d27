// Device pieces shared by the persistent PCG kernels (k_solve.cu: matrix and vectors in global
// memory; k_pcg_res.cu: one slice per warp with the matrix in shared memory and the row vectors
// in registers): group barrier, deterministic group sums, the solve epilogue.
#pragma once
#include "txgel_common.cuh"

namespace txg {

// ---------------------------------------------------------------- persistent PCG
constexpr int PCG_T = 256;  // threads per CTA (8 warps)
constexpr int PCG_MAXG = 64; // gels one CTA may touch

__device__ __forceinline__ double4_32a mul3(const double* M, const double4_32a v) {
  return make_double4_32a(fma(M[2], v.z, fma(M[1], v.y, M[0] * v.x)), fma(M[5], v.z, fma(M[4], v.y, M[3] * v.x)),
                          fma(M[8], v.z, fma(M[7], v.y, M[6] * v.x)), 0.0);
}
__device__ __forceinline__ double dot4(const double4_32a a, const double4_32a b) {
  return fma(a.z, b.z, fma(a.y, b.y, a.x * b.x));
}

// SpMV of one slice (row = lane of the warp): y = A u, FP64.  Unrolled so that several block
// loads (column index, 9 values, gathered vector) are in flight at once.
__device__ __forceinline__ double4_32a spmv_row64(const Dev& d, int s, int lane, const double4_32a* u) {
  const int o = d.slice_off[s], w = (d.slice_off[s + 1] - o) >> 5;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll 4
  for (int k = 0; k < w; ++k) {
    const int bp = o + 32 * k + lane;
    const int c = __ldg(d.colidx + bp);
    const double4_32a uc = u[c];
    double v[9];
    load_block64(d.vals + (size_t)9 * (o + 32 * k), lane, v);
    a0 = fma(v[0], uc.x, a0);
    a1 = fma(v[3], uc.x, a1);
    a2 = fma(v[6], uc.x, a2);
    a0 = fma(v[1], uc.y, a0);
    a1 = fma(v[4], uc.y, a1);
    a2 = fma(v[7], uc.y, a2);
    a0 = fma(v[2], uc.z, a0);
    a1 = fma(v[5], uc.z, a1);
    a2 = fma(v[8], uc.z, a2);
  }
  return make_double4_32a(a0, a1, a2, 0.0);
}

// Per-CTA view of its group (gels [g0, g0 + ng), CTAs [c0, c0 + nc)).  A group of several CTAs
// holds a single gel; a group of one CTA may hold several small gels.
struct PcgCta {
  int s0, s1;  // slices of this CTA
  int c0, nc, g0, ng;
  unsigned* bar;
  unsigned epoch;
};

__device__ __forceinline__ PcgCta pcg_cta(const Dev& d, const PcgPlan& plan) {
  PcgCta c;
  const int2 r = plan.cta_rng[blockIdx.x];
  c.s0 = r.x;
  c.s1 = r.y;
  const int gr = plan.cta_grp[blockIdx.x];
  const int4 G = plan.grp[gr];
  c.c0 = G.x;
  c.nc = G.y;
  c.g0 = G.z;
  c.ng = G.w;
  c.bar = d.bar + gr;
  c.epoch = 0;
  return c;
}

// Barrier of the nc CTAs of one group (all co-resident: cooperative launch).  Arrival is a
// release add on the group's counter, the wait an acquire poll bounded by d.wait_limit polls; a
// wait that gives up sets *err and the CTA returns false (the host reports a device timeout).
// d.wait_extra (0 in normal operation; set only by the library's fault-injection test hook) adds
// arrivals that never come, so that every wait runs into its limit.
__device__ __forceinline__ bool group_barrier(PcgCta& c, const Dev& d, int* s_fail) {
  __syncthreads();
  c.epoch += 1;
  if ((c.nc > 1 || d.wait_extra) && threadIdx.x == 0) {
    const unsigned target = c.epoch * (unsigned)c.nc + d.wait_extra;
    __threadfence();
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(c.bar) : "memory");
    unsigned spins = 0, cur;
    while (true) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(c.bar) : "memory");
      if (cur >= target) break;
      if (++spins > d.wait_limit) {
        atomicExch(d.err, 1);
        *s_fail = 1;
        break;
      }
      __nanosleep(20);
    }
  }
  __syncthreads();
  return *s_fail == 0;
}

// Group totals of quantities [k0, k1) from the per-slice partials dsm[(s - s0) * 4 + k]: every
// CTA sums its slices of each gel (one warp per (gel, quantity), fixed lane order); a group of
// several CTAs (one gel) exchanges the CTA sums through d.part and every CTA adds them up in CTA
// order.  Bitwise identical in every CTA of the group and in every run.  Includes the group
// barrier between the two levels.
// (A = float: the CTA-level sum of an FP32 inner iteration's partials is taken in FP32.)
template <typename A = double>
__device__ __forceinline__ bool group_sum(const Dev& d, PcgCta& c, const double* dsm, int k0, int k1,
                                          double (*tot)[4], int* s_fail) {
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nk = k1 - k0;
  for (int t = wid; t < c.ng * nk; t += (int)(blockDim.x >> 5)) {
    const int j = t / nk, k = k0 + t % nk;
    const GelInfo& G = d.gi[c.g0 + j];
    const int a = max(c.s0, G.s0), b = min(c.s1, G.s0 + G.ns);
    A v = A(0);
    for (int s = a + lane; s < b; s += 32) v += (A)dsm[(s - c.s0) * 4 + k];
    v = warp_sum(v);
    if (lane == 0) {
      if (c.nc == 1)
        tot[j][k] = v;
      else
        d.part[(size_t)k * gridDim.x + blockIdx.x] = v;
    }
  }
  if (c.nc > 1) {
    if (!group_barrier(c, d, s_fail)) return false;
    for (int t = wid; t < nk; t += (int)(blockDim.x >> 5)) {
      const int k = k0 + t;
      double v = 0.0;
      for (int q = c.c0 + lane; q < c.c0 + c.nc; q += 32) v += d.part[(size_t)k * gridDim.x + q];
      v = warp_sum(v);
      if (lane == 0) tot[0][k] = v;
    }
  }
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------- coarse space of a free body
// A body held by no vertex (a soft ball between the gelpad and the indenter) has six rigid motions
// that only its mass resists (M / h^2, some 1e4 below the elastic diagonal): block-Jacobi leaves
// them as the smallest eigenvalues of the preconditioned matrix and CG needs hundreds of
// iterations.  The two-level additive preconditioner M^-1 + Z E^-1 Z^T adds an exact solve on
// those motions (Z: per body row i, the 3 x 6 block [I | -[d_i]x] with d_i = x_i - c, E = Z^T A Z,
// the rigid-body coarse space of additive Schwarz methods); it is SPD, so CG stays CG.  Z^T v of a
// row vector v is (v, d x v); Z c is c_t + c_r x d.
__device__ __forceinline__ void cz_zt(const double4_32a v, const double dd[3], double* o) {
  o[0] += v.x;
  o[1] += v.y;
  o[2] += v.z;
  o[3] += dd[1] * v.z - dd[2] * v.y;
  o[4] += dd[2] * v.x - dd[0] * v.z;
  o[5] += dd[0] * v.y - dd[1] * v.x;
}

// 6 x 6 SPD solve from the packed upper triangle E (row-major, i <= j) by Cholesky; false if E is
// not numerically positive definite
__device__ __forceinline__ bool cz_chol(const double* E, double* L) {
  double A[6][6];
  for (int i = 0, q = 0; i < 6; ++i)
    for (int j = i; j < 6; ++j, ++q) A[i][j] = A[j][i] = E[q];
  for (int j = 0; j < 6; ++j) {
    double s = A[j][j];
    for (int k = 0; k < j; ++k) s -= L[6 * j + k] * L[6 * j + k];
    if (!(s > 1e-14 * fabs(A[j][j])) || !(s > 0.0)) return false;
    L[6 * j + j] = sqrt(s);
    for (int i = j + 1; i < 6; ++i) {
      double t = A[i][j];
      for (int k = 0; k < j; ++k) t -= L[6 * i + k] * L[6 * j + k];
      L[6 * i + j] = t / L[6 * j + j];
    }
  }
  return true;
}
__device__ __forceinline__ void cz_solve(const double* L, const double* b, double* x) {
  double y[6];
  for (int i = 0; i < 6; ++i) {
    double t = b[i];
    for (int k = 0; k < i; ++k) t -= L[6 * i + k] * y[k];
    y[i] = t / L[6 * i + i];
  }
  for (int i = 5; i >= 0; --i) {
    double t = y[i];
    for (int k = i + 1; k < 6; ++k) t -= L[6 * k + i] * x[k];
    x[i] = t / L[6 * i + i];
  }
}

// row q of the 6 x 6 product M v (M row-major)
__device__ __forceinline__ double cz_mv(const double* M, const double* v, int q) {
  double t = 0.0;
  for (int k = 0; k < 6; ++k) t = fma(M[6 * q + k], v[k], t);
  return t;
}

// (A Z)_r of a body row, and its contribution Z_r^T (A Z)_r to the packed upper triangle of E
__device__ __forceinline__ void cz_row_e(const Dev& d, int s, int lane, int cb, const double* ctr, const double dr[3],
                                         double* e21) {
  const int o = d.slice_off[s], w = (d.slice_off[s + 1] - o) >> 5;
  double y[3][6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int m = 0; m < 6; ++m) y[i][m] = 0.0;
  for (int k = 0; k < w; ++k) {
    const int c = __ldg(d.colidx + o + 32 * k + lane);
    if (d.vcomp[c] != cb || d.fixed[c]) continue;
    double v[9];
    load_block64(d.vals + (size_t)9 * (o + 32 * k), lane, v);
    const double4_32a xc = d.x[c];
    const double dc[3] = {xc.x - ctr[0], xc.y - ctr[1], xc.z - ctr[2]};
    // Z_c columns: e_0, e_1, e_2, e_0 x dc, e_1 x dc, e_2 x dc
    const double z[3][3] = {{0.0, -dc[2], dc[1]}, {dc[2], 0.0, -dc[0]}, {-dc[1], dc[0], 0.0}};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int m = 0; m < 3; ++m) y[i][m] += v[3 * i + m];
#pragma unroll
      for (int q = 0; q < 3; ++q) y[i][3 + q] += v[3 * i] * z[q][0] + v[3 * i + 1] * z[q][1] + v[3 * i + 2] * z[q][2];
    }
  }
  double col[6][6];  // Z_r^T y: column m = (y_m, dr x y_m)
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    col[0][m] = y[0][m];
    col[1][m] = y[1][m];
    col[2][m] = y[2][m];
    col[3][m] = dr[1] * y[2][m] - dr[2] * y[1][m];
    col[4][m] = dr[2] * y[0][m] - dr[0] * y[2][m];
    col[5][m] = dr[0] * y[1][m] - dr[1] * y[0][m];
  }
  for (int i = 0, q = 0; i < 6; ++i)
    for (int m = i; m < 6; ++m, ++q) e21[q] += col[i][m];
}

// g . p (stationarity test of the line search) and ||p||_inf per gel after a solve
__device__ __forceinline__ void pcg_epilogue(const Dev& d, const PcgPlan& plan, PcgCta& c, double* dsm,
                                             double (*tot)[4], const int* gact, int* s_fail) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (!group_barrier(c, d, s_fail)) return;  // p complete, exchange slots free
  for (int s = c.s0 + wid; s < c.s1; s += (int)(blockDim.x >> 5)) {
    const int j = plan.slice_gel[s] - c.g0;
    double gp = 0.0, m = 0.0;
    if (gact[j]) {
      const double4_32a x = d.p[32 * s + lane];
      gp = dot4(d.grad[32 * s + lane], x);
      m = fmax(fabs(x.x), fmax(fabs(x.y), fabs(x.z)));
    }
    gp = warp_sum(gp);
    m = warp_max(m);
    if (lane == 0) {
      dsm[(s - c.s0) * 4 + 3] = gp;
      if (gact[j]) atomic_max_pos(&d.gv[c.g0 + j].pnorm_bits, m);
    }
  }
  if (!group_sum(d, c, dsm, 3, 4, tot, s_fail)) return;
  if (blockIdx.x == c.c0)
    for (int j = threadIdx.x; j < c.ng; j += blockDim.x)
      if (gact[j]) d.gv[c.g0 + j].gtp = tot[j][3];
}


__device__ __forceinline__ float4 mul3f(const float* M, const float4 v) {
  return make_float4(fmaf(M[2], v.z, fmaf(M[1], v.y, M[0] * v.x)), fmaf(M[5], v.z, fmaf(M[4], v.y, M[3] * v.x)),
                     fmaf(M[8], v.z, fmaf(M[7], v.y, M[6] * v.x)), 0.f);
}
__device__ __forceinline__ float dot4f(const float4 a, const float4 b) { return fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)); }


}  // namespace txg

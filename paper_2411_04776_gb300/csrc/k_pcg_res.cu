// Persistent PCG for groups whose CTAs own at most one 32-row slice per warp (a single gel, or
// a few gels, spread over many SMs).  Every warp keeps its slice for the whole solve: the CTA
// copies its slices of the sliced BSR (values and column indices) into shared memory once, the
// row vectors of the solve (r, pp, s, the direction, the preconditioner block) stay in the
// owning lane's registers, and only u -- the vector the SpMV gathers from neighbouring rows --
// goes through global memory (L2).  Per iteration this leaves the gathers of u, the group sum and
// the group barrier as the only global traffic.  Arithmetic, stopping rules and the fixed-order
// reductions are those of the kernels in k_solve.cu.
#include "dev_pcg.cuh"

namespace txg {

constexpr int RES_MAXW = 8;  // warps (slices) per CTA

// warp-owned image of slice s in shared memory: values [k][9][32], column indices [k][32]
template <typename V>
__device__ __forceinline__ int res_load(const Dev& d, int s, const V* gval, V* sv, int* sc, int lane) {
  const int o = d.slice_off[s], w = (d.slice_off[s + 1] - o) >> 5;
  for (int k = 0; k < w; ++k) {
    sc[32 * k + lane] = d.colidx[o + 32 * k + lane];
    const V* src = gval + (size_t)9 * (o + 32 * k) + lane;
#pragma unroll
    for (int e = 0; e < 9; ++e) sv[288 * k + 32 * e + lane] = src[32 * e];
  }
  return w;
}

// y = A u for the lane's row, values from shared memory, u gathered from global memory
template <typename V, typename U, typename A>
__device__ __forceinline__ void res_spmv(const V* sv, const int* sc, int w, int lane, const U* u, A& a0, A& a1,
                                         A& a2) {
  a0 = a1 = a2 = A(0);
#pragma unroll 8
  for (int k = 0; k < w; ++k) {
    const int c = sc[32 * k + lane];
    const U uc = u[c];
    const V* v = sv + 288 * k + lane;
    a0 = fma((A)v[0], (A)uc.x, a0);
    a1 = fma((A)v[96], (A)uc.x, a1);
    a2 = fma((A)v[192], (A)uc.x, a2);
    a0 = fma((A)v[32], (A)uc.y, a0);
    a1 = fma((A)v[128], (A)uc.y, a1);
    a2 = fma((A)v[224], (A)uc.y, a2);
    a0 = fma((A)v[64], (A)uc.z, a0);
    a1 = fma((A)v[160], (A)uc.z, a1);
    a2 = fma((A)v[256], (A)uc.z, a2);
  }
}

// CG scalars with two levels of division: beta = ga / ga_prev and t = ga / al_prev are independent
__device__ __forceinline__ void cg_scalars(int k, double ga, double de, double gprev, double aprev, double& al,
                                           double& be) {
  if (k == 1) {
    be = 0.0;
    al = ga / de;
  } else {
    be = ga / gprev;
    const double t = ga / aprev;
    al = ga / (de - be * t);
  }
}

// shared memory: [dsm: 4 per slice][values: warps x wmax x 288][columns: warps x wmax x 32]
template <typename V>
__device__ __forceinline__ void res_smem(double* dyn, int max_slices, int wmax, double*& dsm, V*& sv, int*& sc) {
  const int nw = blockDim.x >> 5, wid = threadIdx.x >> 5;
  dsm = dyn;
  V* vbase = reinterpret_cast<V*>(dyn + 4 * max_slices);
  sv = vbase + (size_t)wid * wmax * 288;
  sc = reinterpret_cast<int*>(vbase + (size_t)nw * wmax * 288) + (size_t)wid * wmax * 32;
}

__global__ void __launch_bounds__(32 * RES_MAXW) k_pcg64_res(Dev d, int phase, PcgPlan plan, double eta2, int maxit,
                                                             int wmax) {
  extern __shared__ double dyn[];
  __shared__ double tot[PCG_MAXG][4];
  __shared__ double bbj[PCG_MAXG], gprev[PCG_MAXG], aprev[PCG_MAXG], alj[PCG_MAXG], bej[PCG_MAXG];
  __shared__ int gact[PCG_MAXG], run[PCG_MAXG];
  __shared__ int s_fail, s_any;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  PcgCta c = pcg_cta(d, plan);
  double* dsm;
  double* sv;
  int* sc;
  res_smem<double>(dyn, plan.max_slices, wmax, dsm, sv, sc);
  if (threadIdx.x == 0) s_fail = 0;
  for (int j = threadIdx.x; j < c.ng; j += blockDim.x) {
    gact[j] = d.gc[c.g0 + j].phase == phase ? 1 : 0;
    run[j] = gact[j];
  }
  __syncthreads();
  const int s = c.s0 + wid, row = 32 * s + lane;
  const bool has = s < c.s1;
  const int j = has ? plan.slice_gel[s] - c.g0 : 0;
  const bool mine = has && gact[j];
  int w = 0;
  double r0 = 0, r1 = 0, r2 = 0, u0 = 0, u1 = 0, u2 = 0, p0 = 0, p1 = 0, p2 = 0;
  double q0 = 0, q1 = 0, q2 = 0, x0 = 0, x1 = 0, x2 = 0, w0 = 0, w1 = 0, w2 = 0;
  double M[9];
  for (int e = 0; e < 9; ++e) M[e] = 0.0;
  const bool fixed = mine && d.fixed[row];
  // ---- init: r = -grad, x = 0, u = M^-1 r; partial |b|^2
  if (mine) {
    w = res_load<double>(d, s, d.vals, sv, sc, lane);
    for (int e = 0; e < 9; ++e) M[e] = d.Minv[9 * row + e];
    const double4_32a gr = d.grad[row];
    r0 = -gr.x; r1 = -gr.y; r2 = -gr.z;
    u0 = fma(M[2], r2, fma(M[1], r1, M[0] * r0));
    u1 = fma(M[5], r2, fma(M[4], r1, M[3] * r0));
    u2 = fma(M[8], r2, fma(M[7], r1, M[6] * r0));
    d.u[row] = make_double4_32a(u0, u1, u2, 0.0);
  }
  if (has) {
    const double bb = warp_sum(fma(r2, r2, fma(r1, r1, r0 * r0)));
    if (lane == 0) dsm[4 * wid + 3] = bb;
  }
  if (!group_sum(d, c, dsm, 3, 4, tot, &s_fail)) return;
  for (int q = threadIdx.x; q < c.ng; q += blockDim.x) bbj[q] = tot[q][3];
  if (!group_barrier(c.bar, c.nc, c.epoch, d.err, &s_fail)) return;  // u complete before the SpMV
  for (int k = 1;; ++k) {
    // ---- w = A u; partials gamma = (r, u), delta = (w, u), rr = (r, r)
    if (has) {
      double ga = 0.0, de = 0.0, rr = 0.0;
      if (run[j]) {
        res_spmv<double, double4_32a, double>(sv, sc, w, lane, d.u, w0, w1, w2);
        if (fixed) w0 = w1 = w2 = 0.0;
        ga = fma(r2, u2, fma(r1, u1, r0 * u0));
        de = fma(w2, u2, fma(w1, u1, w0 * u0));
        rr = fma(r2, r2, fma(r1, r1, r0 * r0));
      }
      ga = warp_sum(ga);
      de = warp_sum(de);
      rr = warp_sum(rr);
      if (lane == 0) {
        dsm[4 * wid + 0] = ga;
        dsm[4 * wid + 1] = de;
        dsm[4 * wid + 2] = rr;
      }
    }
    if (!group_sum(d, c, dsm, 0, 3, tot, &s_fail)) return;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    for (int q = threadIdx.x; q < c.ng; q += blockDim.x) {
      if (!run[q]) continue;
      const double ga = tot[q][0], de = tot[q][1], rr = tot[q][2];
      if (!(rr > eta2 * bbj[q]) || k > maxit) {
        run[q] = 0;
        if (blockIdx.x == c.c0) {
          d.gv[c.g0 + q].pcg_it = k - 1;
          d.gv[c.g0 + q].bb = bbj[q];
          d.gv[c.g0 + q].pcg_done = 1;
        }
        continue;
      }
      s_any = 1;
      double al, be;
      cg_scalars(k, ga, de, gprev[q], aprev[q], al, be);
      gprev[q] = ga;
      aprev[q] = al;
      alj[q] = al;
      bej[q] = be;
    }
    __syncthreads();
    if (!s_any) break;
    // ---- vector updates (registers); u to global memory for the neighbours' SpMV
    if (has && run[j]) {
      const double be = bej[j], al = alj[j];
      p0 = fma(be, p0, u0); p1 = fma(be, p1, u1); p2 = fma(be, p2, u2);
      q0 = fma(be, q0, w0); q1 = fma(be, q1, w1); q2 = fma(be, q2, w2);
      x0 = fma(al, p0, x0); x1 = fma(al, p1, x1); x2 = fma(al, p2, x2);
      r0 = fma(-al, q0, r0); r1 = fma(-al, q1, r1); r2 = fma(-al, q2, r2);
      u0 = fma(M[2], r2, fma(M[1], r1, M[0] * r0));
      u1 = fma(M[5], r2, fma(M[4], r1, M[3] * r0));
      u2 = fma(M[8], r2, fma(M[7], r1, M[6] * r0));
      d.u[row] = make_double4_32a(u0, u1, u2, 0.0);
    }
    if (!group_barrier(c.bar, c.nc, c.epoch, d.err, &s_fail)) return;
  }
  if (mine) d.p[row] = make_double4_32a(x0, x1, x2, 0.0);
  pcg_epilogue(d, plan, c, dsm, tot, gact, &s_fail);
}

__global__ void __launch_bounds__(32 * RES_MAXW) k_pcg_mixed_res(Dev d, int phase, PcgPlan plan, double eta2,
                                                                 int maxit, int refine_max, int wmax) {
  extern __shared__ double dyn[];
  __shared__ double tot[PCG_MAXG][4];
  __shared__ double bbj[PCG_MAXG], tolj[PCG_MAXG], rr0j[PCG_MAXG], gprev[PCG_MAXG], aprev[PCG_MAXG];
  __shared__ float alj[PCG_MAXG], bej[PCG_MAXG];
  __shared__ int gact[PCG_MAXG], run[PCG_MAXG], inner[PCG_MAXG], itj[PCG_MAXG];
  __shared__ int s_fail, s_any;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  PcgCta c = pcg_cta(d, plan);
  double* dsm;
  float* sv;
  int* sc;
  res_smem<float>(dyn, plan.max_slices, wmax, dsm, sv, sc);
  if (threadIdx.x == 0) s_fail = 0;
  for (int q = threadIdx.x; q < c.ng; q += blockDim.x) {
    gact[q] = d.gc[c.g0 + q].phase == phase ? 1 : 0;
    run[q] = gact[q];
    itj[q] = 0;
  }
  __syncthreads();
  const int s = c.s0 + wid, row = 32 * s + lane;
  const bool has = s < c.s1;
  const int j = has ? plan.slice_gel[s] - c.g0 : 0;
  const bool mine = has && gact[j];
  const bool fixed = mine && d.fixed[row];
  int w = 0;
  double g0 = 0, g1 = 0, g2 = 0, R0 = 0, R1 = 0, R2 = 0, P0 = 0, P1 = 0, P2 = 0;  // FP64: grad, r, p
  float M[9];
  for (int e = 0; e < 9; ++e) M[e] = 0.f;
  if (mine) {
    w = res_load<float>(d, s, d.vals32, sv, sc, lane);
    for (int e = 0; e < 9; ++e) M[e] = d.Minv32[9 * row + e];
    const double4_32a gr = d.grad[row];
    g0 = gr.x; g1 = gr.y; g2 = gr.z;
    R0 = -g0; R1 = -g1; R2 = -g2;
  }
  if (has) {
    const double bb = warp_sum(fma(R2, R2, fma(R1, R1, R0 * R0)));
    if (lane == 0) {
      dsm[4 * wid + 3] = bb;
      dsm[4 * wid + 2] = bb;
    }
  }
  if (!group_sum(d, c, dsm, 2, 4, tot, &s_fail)) return;
  for (int q = threadIdx.x; q < c.ng; q += blockDim.x) bbj[q] = tot[q][3];
  __syncthreads();
  for (int round = 0;; ++round) {
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    for (int q = threadIdx.x; q < c.ng; q += blockDim.x) {
      inner[q] = 0;
      if (!run[q]) continue;
      const double rr = tot[q][2], bb = bbj[q];
      if (!(rr > eta2 * bb) || round >= refine_max) {
        run[q] = 0;
        if (blockIdx.x == c.c0) {
          d.gv[c.g0 + q].pcg_done = 1;
          d.gv[c.g0 + q].rounds = round;
          d.gv[c.g0 + q].bb = bb;
          d.gv[c.g0 + q].pcg_it = itj[q];
        }
        continue;
      }
      s_any = 1;
      inner[q] = 1;
      tolj[q] = fmax(eta2 * bb / rr, 1e-11);
    }
    __syncthreads();
    if (!s_any) break;
    // ---- inner init: r32 = r64, x32 = 0, u32 = M^-1 r32
    float r0 = 0.f, r1 = 0.f, r2 = 0.f, u0 = 0.f, u1 = 0.f, u2 = 0.f, p0 = 0.f, p1 = 0.f, p2 = 0.f;
    float q0 = 0.f, q1 = 0.f, q2 = 0.f, x0 = 0.f, x1 = 0.f, x2 = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f;
    const bool in = has && inner[j];
    if (in) {
      r0 = (float)R0; r1 = (float)R1; r2 = (float)R2;
      u0 = fmaf(M[2], r2, fmaf(M[1], r1, M[0] * r0));
      u1 = fmaf(M[5], r2, fmaf(M[4], r1, M[3] * r0));
      u2 = fmaf(M[8], r2, fmaf(M[7], r1, M[6] * r0));
      d.u32[row] = make_float4(u0, u1, u2, 0.f);
    }
    if (!group_barrier(c.bar, c.nc, c.epoch, d.err, &s_fail)) return;
    for (int k = 1;; ++k) {
      if (has) {
        double ga = 0.0, de = 0.0, rr = 0.0;
        if (inner[j]) {
          res_spmv<float, float4, float>(sv, sc, w, lane, d.u32, w0, w1, w2);
          if (fixed) w0 = w1 = w2 = 0.f;
          ga = fmaf(r2, u2, fmaf(r1, u1, r0 * u0));
          de = fmaf(w2, u2, fmaf(w1, u1, w0 * u0));
          rr = fmaf(r2, r2, fmaf(r1, r1, r0 * r0));
        }
        ga = warp_sum(ga);
        de = warp_sum(de);
        rr = warp_sum(rr);
        if (lane == 0) {
          dsm[4 * wid + 0] = ga;
          dsm[4 * wid + 1] = de;
          dsm[4 * wid + 2] = rr;
        }
      }
      if (!group_sum(d, c, dsm, 0, 3, tot, &s_fail)) return;
      if (threadIdx.x == 0) s_any = 0;
      __syncthreads();
      for (int q = threadIdx.x; q < c.ng; q += blockDim.x) {
        if (!inner[q]) continue;
        const double ga = tot[q][0], de = tot[q][1], rr = tot[q][2];
        if (k == 1) rr0j[q] = rr;
        if (!(rr > tolj[q] * rr0j[q]) || k > maxit) {
          inner[q] = 0;
          itj[q] += k - 1;
          continue;
        }
        s_any = 1;
        double al, be;
        cg_scalars(k, ga, de, gprev[q], aprev[q], al, be);
        gprev[q] = ga;
        aprev[q] = al;
        alj[q] = (float)al;
        bej[q] = (float)be;
      }
      __syncthreads();
      if (!s_any) break;
      if (has && inner[j]) {
        const float fb = bej[j], fa = alj[j];
        p0 = fmaf(fb, p0, u0); p1 = fmaf(fb, p1, u1); p2 = fmaf(fb, p2, u2);
        q0 = fmaf(fb, q0, w0); q1 = fmaf(fb, q1, w1); q2 = fmaf(fb, q2, w2);
        x0 = fmaf(fa, p0, x0); x1 = fmaf(fa, p1, x1); x2 = fmaf(fa, p2, x2);
        r0 = fmaf(-fa, q0, r0); r1 = fmaf(-fa, q1, r1); r2 = fmaf(-fa, q2, r2);
        u0 = fmaf(M[2], r2, fmaf(M[1], r1, M[0] * r0));
        u1 = fmaf(M[5], r2, fmaf(M[4], r1, M[3] * r0));
        u2 = fmaf(M[8], r2, fmaf(M[7], r1, M[6] * r0));
        d.u32[row] = make_float4(u0, u1, u2, 0.f);
      }
      if (!group_barrier(c.bar, c.nc, c.epoch, d.err, &s_fail)) return;
    }
    // ---- p += x32 (FP64), then the FP64 residual r64 = b - A p (FP32 values, FP64 arithmetic)
    const bool rn = has && run[j];
    if (rn) {
      P0 += (double)x0;
      P1 += (double)x1;
      P2 += (double)x2;
      d.p[row] = make_double4_32a(P0, P1, P2, 0.0);
    }
    if (!group_barrier(c.bar, c.nc, c.epoch, d.err, &s_fail)) return;
    if (has) {
      double rr = 0.0;
      if (rn) {
        double a0, a1, a2;
        res_spmv<float, double4_32a, double>(sv, sc, w, lane, d.p, a0, a1, a2);
        R0 = -g0 - a0;
        R1 = -g1 - a1;
        R2 = -g2 - a2;
        if (fixed) R0 = R1 = R2 = 0.0;
        rr = fma(R2, R2, fma(R1, R1, R0 * R0));
      }
      rr = warp_sum(rr);
      if (lane == 0) dsm[4 * wid + 2] = rr;
    }
    if (!group_sum(d, c, dsm, 2, 3, tot, &s_fail)) return;
  }
  if (mine) d.p[row] = make_double4_32a(P0, P1, P2, 0.0);
  pcg_epilogue(d, plan, c, dsm, tot, gact, &s_fail);
}

// dynamic shared memory of the resident kernels
size_t pcg_res_smem(bool mixed, int max_slices, int wmax) {
  const size_t nw = (size_t)max_slices;
  return sizeof(double) * 4 * max_slices + nw * wmax * 288 * (mixed ? sizeof(float) : sizeof(double)) +
         nw * wmax * 32 * sizeof(int);
}

// co-resident CTAs per SM of the resident kernel (0 if it cannot be launched so)
int pcg_res_ctas_per_sm(bool mixed, int max_slices, int wmax) {
  if (max_slices > RES_MAXW) return 0;
  const size_t smem = pcg_res_smem(mixed, max_slices, wmax);
  const void* fn = mixed ? (const void*)k_pcg_mixed_res : (const void*)k_pcg64_res;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, 32 * max_slices, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_pcg_res(const Dev& d, int phase, const PcgPlan& plan, int nctas, bool mixed, double eta,
                           int maxit, int refine_max, int wmax, cudaStream_t st) {
  double eta2 = eta * eta;
  Dev dd = d;
  PcgPlan pp = plan;
  const size_t smem = pcg_res_smem(mixed, plan.max_slices, wmax);
  count_launch(1);
  if (mixed) {
    void* args[] = {(void*)&dd, (void*)&phase, (void*)&pp, (void*)&eta2, (void*)&maxit, (void*)&refine_max,
                    (void*)&wmax};
    return cudaLaunchCooperativeKernel((const void*)k_pcg_mixed_res, dim3(nctas), dim3(32 * plan.max_slices), args,
                                       smem, st);
  }
  void* args[] = {(void*)&dd, (void*)&phase, (void*)&pp, (void*)&eta2, (void*)&maxit, (void*)&wmax};
  return cudaLaunchCooperativeKernel((const void*)k_pcg64_res, dim3(nctas), dim3(32 * plan.max_slices), args, smem,
                                     st);
}

}  // namespace txg

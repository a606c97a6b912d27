// Persistent PCG for groups whose CTAs own at most one 32-row slice per warp (a single gel, or a
// few gels, spread over many SMs), as pipelined CG with one group barrier per iteration.  Every
// warp keeps its slice for the whole solve: the CTA copies its slices of the sliced BSR (values
// and column indices) into shared memory once, the row vectors of the solve stay in the owning
// lane's registers, and only the vector the SpMV gathers from neighbouring rows goes through
// global memory (L2).  Per iteration this leaves those gathers, the group sum and the group
// barrier as the only global traffic.  Stopping rules and the fixed-order reductions are those
// of the kernels in k_solve.cu.
#include "dev_pcg.cuh"

namespace txg {

constexpr int RES_MAXW = 8;    // warps (slices) per CTA
// FP64: two warps per slice (an owner and a helper splitting its SpMV blocks) while a CTA holds at
// most RES_SPLIT_MAXS slices.  A warp issues an FP64 FMA only about every 67 cycles, and with one
// warp per sub-partition every bubble in its stream (operand loads, dependencies) idles the
// sub-partition's FP64 pipe; a second warp fills them.
constexpr int RES_SPLIT_MAXS = 4;
constexpr int RES_SPLIT_W = 2 * RES_SPLIT_MAXS + 1;  // warps per CTA: owners, helpers, control
constexpr int RES_MAXNC = 256; // CTAs of one group (exchange slots a lane prefetches: 8)

// warp-owned image of slice s in shared memory: values [k][9][32], column indices [k][32].  Both
// are contiguous in the sliced BSR (a slice starts at a multiple of 32 positions, so at a 16-byte
// boundary of the 256-byte aligned arrays) with the same layout, so the warp copies them as
// 16-byte pieces with cp.async: every piece in flight at once, none through registers.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gsrc) : "memory");
}

// tid / nthr: this thread's index among the nthr threads that copy the image together; each
// waits for its own pieces, and a barrier over those threads must follow before the image is read
template <typename V>
__device__ __forceinline__ int res_load(const Dev& d, int s, const V* gval, V* sv, int* sc, int tid, int nthr) {
  const int o = d.slice_off[s], w = (d.slice_off[s + 1] - o) >> 5;
  const char* vsrc = reinterpret_cast<const char*>(gval + (size_t)9 * o);
  char* vdst = reinterpret_cast<char*>(sv);
  const int nv = w * 288 * (int)sizeof(V) / 16;
  for (int i = tid; i < nv; i += nthr) cp_async16(vdst + 16 * i, vsrc + 16 * i);
  const char* csrc = reinterpret_cast<const char*>(d.colidx + o);
  char* cdst = reinterpret_cast<char*>(sc);
  for (int i = tid; i < 8 * w; i += nthr) cp_async16(cdst + 16 * i, csrc + 16 * i);
  asm volatile("cp.async.wait_all;" ::: "memory");
  return w;
}

// one block of the lane's row: a += A_k uc (values from the slice image in shared memory, in the
// sliced BSR's value layout: pairs of FP64 or quads of FP32 per 16-byte load)
template <typename V, typename U, typename A>
__device__ __forceinline__ void res_block(const V* sv, int k, int lane, const U uc, A& a0, A& a1, A& a2) {
  V v[9];
  if constexpr (sizeof(V) == 8)
    load_block64(reinterpret_cast<const double*>(sv) + 288 * k, lane, reinterpret_cast<double*>(v));
  else
    load_block32(reinterpret_cast<const float*>(sv) + 288 * k, lane, reinterpret_cast<float*>(v));
  a0 = fma((A)v[0], (A)uc.x, a0);
  a1 = fma((A)v[3], (A)uc.x, a1);
  a2 = fma((A)v[6], (A)uc.x, a2);
  a0 = fma((A)v[1], (A)uc.y, a0);
  a1 = fma((A)v[4], (A)uc.y, a1);
  a2 = fma((A)v[7], (A)uc.y, a2);
  a0 = fma((A)v[2], (A)uc.z, a0);
  a1 = fma((A)v[5], (A)uc.z, a1);
  a2 = fma((A)v[8], (A)uc.z, a2);
}

// y = A u for the lane's row: values from shared memory, u gathered from global memory (L2)
// RES_PF blocks ahead of the block being multiplied (a register ring), so that the gathers'
// latency hides behind the FP64 work of the blocks before them; even and odd blocks accumulate
// separately (six independent FMA chains), then add
constexpr int RES_PF = 4;  // even: a ring slot keeps the parity of its blocks
template <typename V, typename U, typename A>
__device__ __forceinline__ void res_spmv(const V* sv, const int* sc, int w, int lane, const U* u, A& y0, A& y1,
                                         A& y2) {
  A a0 = A(0), a1 = A(0), a2 = A(0), b0 = A(0), b1 = A(0), b2 = A(0);
  U ring[RES_PF];
#pragma unroll
  for (int t = 0; t < RES_PF; ++t)
    if (t < w) ring[t] = u[sc[32 * t + lane]];
  for (int k0 = 0; k0 < w; k0 += RES_PF) {
#pragma unroll
    for (int t = 0; t < RES_PF; ++t) {
      const int k = k0 + t;
      if (k < w) {
        const U uc = ring[t];
        if (k + RES_PF < w) ring[t] = u[sc[32 * (k + RES_PF) + lane]];
        if (t & 1)
          res_block(sv, k, lane, uc, b0, b1, b2);
        else
          res_block(sv, k, lane, uc, a0, a1, a2);
      }
    }
  }
  y0 = a0 + b0;
  y1 = a1 + b1;
  y2 = a2 + b2;
}

// The blocks k = k0, k0 + 2, ... of the lane's row: the share of one of the two warps of a slice
// (split FP64 kernel); its even and odd blocks accumulate separately (six FMA chains), then add.
__device__ __forceinline__ void res_spmv_half(const double* sv, const int* sc, int w, int k0, int lane,
                                              const double4_32a* u, double& y0, double& y1, double& y2) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, b0 = 0.0, b1 = 0.0, b2 = 0.0;
  int k = k0;
#pragma unroll 2
  for (; k + 2 < w; k += 4) {
    res_block(sv, k, lane, u[sc[32 * k + lane]], a0, a1, a2);
    res_block(sv, k + 2, lane, u[sc[32 * (k + 2) + lane]], b0, b1, b2);
  }
  if (k < w) res_block(sv, k, lane, u[sc[32 * k + lane]], a0, a1, a2);
  y0 = a0 + b0;
  y1 = a1 + b1;
  y2 = a2 + b2;
}

// Warp sums of three per-lane FP64 values with 6 adds per lane instead of three butterflies'
// 15 (the FP64 pipe is the scarce unit): at the first level lanes 0-15 carry (a, b) and lanes
// 16-31 (c, -), at the second each lane keeps one of its two, and three butterfly levels finish
// it.  Afterwards lanes 0-7 hold the sum of a, lanes 8-15 that of b, lanes 16-23 that of c.
// Fixed order: bitwise the same in every warp and run.
__device__ __forceinline__ double warp_sum3(double a, double b, double c, int lane) {
  const bool h16 = lane & 16, h8 = lane & 8;
  double k0 = h16 ? c : a, k1 = h16 ? 0.0 : b;
  const double g0 = h16 ? a : c, g1 = h16 ? b : 0.0;
  k0 += __shfl_xor_sync(0xffffffffu, g0, 16);
  k1 += __shfl_xor_sync(0xffffffffu, g1, 16);
  double v = h8 ? k1 : k0;
  v += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// the three sums of warp_sum3 into dsm[base + 0..2]
__device__ __forceinline__ void put_sum3(double* dsm, int base, double v, int lane) {
  if ((lane & 7) == 0 && lane < 24) dsm[base + (lane >> 3)] = v;
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

// shared memory: [dsm: 4 per slice][split kernel: helper partials, 96 per slice]
// [values: slices x wmax x 288][columns: slices x wmax x 32]; sw: the warp's slice in the CTA
// (the control warp's points past the images and is never used)
template <typename V>
__device__ __forceinline__ void res_smem(double* dyn, int max_slices, int wmax, int sw, bool split, double*& dsm,
                                         double*& hs, V*& sv, int*& sc) {
  const int nw = max_slices;
  dsm = dyn;
  hs = dyn + 4 * nw;
  V* vbase = reinterpret_cast<V*>(dyn + 4 * nw + (split ? 96 * nw : 0));
  sv = vbase + (size_t)sw * wmax * 288;
  sc = reinterpret_cast<int*>(vbase + (size_t)nw * wmax * 288) + (size_t)sw * wmax * 32;
}

// Split group sums of the pipelined kernels (one group barrier between post and collect).
// post: every CTA adds the per-warp partials dsm[4 w + k] of each of its gels in warp order; a
// CTA alone in its group keeps the totals, a CTA of a multi-CTA group (one gel) publishes its sum
// in exchange set `set` of d.part.  The prefetch / finish pair of collect adds a multi-CTA group's
// published sums in CTA order; the prefetch loads them into registers before the SpMV so that
// their latency overlaps it.  Bitwise identical in every CTA of the group.
__device__ __forceinline__ void res_post(const Dev& d, const PcgCta& c, const double* dsm, int k0, int k1, int set,
                                         double (*tot)[4]) {
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nk = k1 - k0;
  for (int t = wid; t < c.ng * nk; t += (int)(blockDim.x >> 5)) {
    const int j = t / nk, k = k0 + t % nk;
    const GelInfo& G = d.gi[c.g0 + j];
    const int a = max(c.s0, G.s0), b = min(c.s1, G.s0 + G.ns);
    // a CTA owns at most RES_MAXW - 1 slices: lane 0 adds their partials in slice order
    double v = 0.0;
    if (lane == 0 && a < b) {
      v = dsm[(a - c.s0) * 4 + k];
      for (int s = a + 1; s < b; ++s) v += dsm[(s - c.s0) * 4 + k];
    }
    if (lane == 0) {
      if (c.nc == 1)
        tot[j][k] = v;
      else
        d.part[(size_t)(4 * set + k) * gridDim.x + blockIdx.x] = v;
    }
  }
}

// res_post for the FP32 inner iteration: the per-gel CTA sums of FP32 partials in FP32
__device__ __forceinline__ void res_post_f(const Dev& d, const PcgCta& c, const double* dsm, int k0, int k1, int set,
                                           double (*tot)[4]) {
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nk = k1 - k0;
  for (int t = wid; t < c.ng * nk; t += (int)(blockDim.x >> 5)) {
    const int j = t / nk, k = k0 + t % nk;
    const GelInfo& G = d.gi[c.g0 + j];
    const int a = max(c.s0, G.s0), b = min(c.s1, G.s0 + G.ns);
    float v = 0.f;
    for (int s = a + lane; s < b; s += 32) v += (float)dsm[(s - c.s0) * 4 + k];
    v = warp_sum(v);
    if (lane == 0) {
      if (c.nc == 1)
        tot[j][k] = v;
      else
        d.part[(size_t)(4 * set + k) * gridDim.x + blockIdx.x] = v;
    }
  }
}

struct ResPrefetch {
  double v[RES_MAXNC / 32];
};

__device__ __forceinline__ void res_prefetch(const Dev& d, const PcgCta& c, int k0, int k1, int set, ResPrefetch& pf) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < RES_MAXNC / 32; ++t) {
    const int q = c.c0 + lane + 32 * t;
    pf.v[t] = (c.nc > 1 && wid < k1 - k0 && q < c.c0 + c.nc) ? d.part[(size_t)(4 * set + k0 + wid) * gridDim.x + q] : 0.0;
  }
}

__device__ __forceinline__ void res_finish(const PcgCta& c, int k0, int k1, const ResPrefetch& pf, double (*tot)[4]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (c.nc > 1 && wid < k1 - k0) {
    double v = 0.0;
#pragma unroll
    for (int t = 0; t < RES_MAXNC / 32; ++t) v += pf.v[t];
    v = warp_sum(v);
    if (lane == 0) tot[0][k0 + wid] = v;
  }
  __syncthreads();
}

// The control warp's collect of quantities [k0, k1) from exchange set `set` (no block barrier): a
// multi-CTA group's published CTA sums are added in CTA order; a one-CTA group already has them.
__device__ __forceinline__ void ctl_collect(const Dev& d, const PcgCta& c, int k0, int k1, int set, double (*tot)[4]) {
  if (c.nc == 1) return;
  const int lane = threadIdx.x & 31;
  double v[3][RES_MAXNC / 32];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int t = 0; t < RES_MAXNC / 32; ++t) {
      const int q = c.c0 + lane + 32 * t;
      v[k][t] = (k < k1 - k0 && q < c.c0 + c.nc) ? d.part[(size_t)(4 * set + k0 + k) * gridDim.x + q] : 0.0;
    }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double a = 0.0;
#pragma unroll
    for (int t = 0; t < RES_MAXNC / 32; ++t) a += v[k][t];
    a = warp_sum(a);
    if (lane == 0 && k < k1 - k0) tot[0][k0 + k] = a;
  }
  __syncwarp();
}

// Pipelined CG (Ghysels & Vanroose 2014, preconditioned): with m = M^-1 w and n = A m the
// recurrences z = n + beta z, q = m + beta q, s = w + beta s, p = u + beta p, x += alpha p,
// r -= alpha s, u -= alpha q, w -= alpha z keep u = M^-1 r and w = A u, so the dot products
// (r, u), (w, u), (r, r) of the next iteration are formed with the vector updates and their group
// reduction overlaps the next SpMV: one group barrier per iteration.  m is exchanged through two
// alternating global buffers (its SpMV reads the neighbours' m of this iteration while they may
// already write the next one).  Same scalars (alpha, beta) and stopping rule as the CG of
// k_solve.cu: |r| <= eta |b| or maxit iterations.  One extra (control) warp per CTA collects the
// group totals and takes the per-gel decisions while the slice warps run the SpMV, so neither is
// on the critical path; run flags are double-buffered (the slice warps read this iteration's,
// the control warp writes the next one's).  SPLIT = 2: each slice has an owner warp (its rows'
// vectors, the update) and a helper warp; the two take alternate blocks of every SpMV and the
// helper hands its partial products over in shared memory.
template <int SPLIT>
__global__ void __launch_bounds__(SPLIT == 2 ? 32 * RES_SPLIT_W : 32 * RES_MAXW, 1)
    k_pcg64_res(Dev d, int phase, PcgPlan plan, int maxit, int wmax) {
  extern __shared__ __align__(16) double dyn[];
  __shared__ double tot[PCG_MAXG][4];
  __shared__ double bbj[PCG_MAXG], thj[PCG_MAXG], gprev[PCG_MAXG], aprev[PCG_MAXG], alj[PCG_MAXG], bej[PCG_MAXG];
  __shared__ double rhoj[PCG_MAXG];
  __shared__ int gact[PCG_MAXG], run[2][PCG_MAXG];
  __shared__ int s_fail, s_any;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nsw = plan.max_slices, ctl = SPLIT * nsw;
  const bool helper = SPLIT == 2 && wid >= nsw && wid < ctl;
  const int sw = helper ? wid - nsw : wid;  // the warp's slice in the CTA
  PcgCta c = pcg_cta(d, plan);
  double* dsm;
  double* hs;
  double* sv;
  int* sc;
  res_smem<double>(dyn, nsw, wmax, sw, SPLIT == 2, dsm, hs, sv, sc);
  if (threadIdx.x == 0) s_fail = 0;
  for (int q = threadIdx.x; q < c.ng; q += blockDim.x) {
    gact[q] = d.gc[c.g0 + q].phase == phase ? 1 : 0;
    run[0][q] = gact[q];
  }
  __syncthreads();
  const int s = c.s0 + sw, row = 32 * s + lane;
  const bool has = s < c.s1;  // owners and helpers of the CTA's slices
  double* hsw = hs + 96 * sw + lane;  // split: the helper's partial products of the lane's row
  const int j = has ? plan.slice_gel[s] - c.g0 : 0;
  const bool mine = has && gact[j];
  const bool fixed = mine && d.fixed[row];
  double4_32a* mbuf[2] = {d.pp, d.s};
  int w = 0;
  double M[9];
  for (int e = 0; e < 9; ++e) M[e] = 0.0;
  double x0 = 0, x1 = 0, x2 = 0, r0 = 0, r1 = 0, r2 = 0, u0 = 0, u1 = 0, u2 = 0, w0 = 0, w1 = 0, w2 = 0;
  double z0 = 0, z1 = 0, z2 = 0, q0 = 0, q1 = 0, q2 = 0, t0 = 0, t1 = 0, t2 = 0, p0 = 0, p1 = 0, p2 = 0;
  double m0 = 0, m1 = 0, m2 = 0;
  // ---- init: r = b = -grad; start from x0 = rho p_prev, the minimiser of the quadratic model
  // along the gel's previous Newton direction (one Galerkin step: rho = b.p / p.A p, 0 without
  // one); the linear Newton contraction makes it a good start, and the A-norm error cannot grow
  double xp0 = 0.0, xp1 = 0.0, xp2 = 0.0, a0 = 0.0, a1 = 0.0, a2 = 0.0;
  if (mine) {
    w = res_load<double>(d, s, d.vals, sv, sc, lane + (helper ? 32 : 0), 32 * SPLIT);
    if (!helper) {
      for (int e = 0; e < 9; ++e) M[e] = d.Minv[9 * row + e];
      const double4_32a gr = d.grad[row];
      r0 = -gr.x; r1 = -gr.y; r2 = -gr.z;
      if (!fixed) {
        const double4_32a pv = d.p[row];
        xp0 = pv.x; xp1 = pv.y; xp2 = pv.z;
      }
    }
  }
  __syncthreads();  // slice images complete
  if (mine && !fixed) {
    if (SPLIT == 2)
      res_spmv_half(sv, sc, w, helper ? 1 : 0, lane, d.p, a0, a1, a2);
    else
      res_spmv<double, double4_32a, double>(sv, sc, w, lane, d.p, a0, a1, a2);
  }
  if (SPLIT == 2) {
    if (helper && mine && !fixed) {
      hsw[0] = a0; hsw[32] = a1; hsw[64] = a2;
    }
    __syncthreads();
    if (!helper && mine && !fixed) {
      a0 += hsw[0]; a1 += hsw[32]; a2 += hsw[64];
    }
  }
  if (has && !helper) {
    const double v = warp_sum3(fma(r2, xp2, fma(r1, xp1, r0 * xp0)), fma(a2, xp2, fma(a1, xp1, a0 * xp0)),
                               fma(r2, r2, fma(r1, r1, r0 * r0)), lane);
    put_sum3(dsm, 4 * sw, v, lane);
  }
  res_post(d, c, dsm, 0, 3, 0, tot);
  if (!group_barrier(c, d, &s_fail)) return;
  {
    ResPrefetch pf;
    res_prefetch(d, c, 0, 3, 0, pf);
    res_finish(c, 0, 3, pf, tot);
  }
  for (int q = threadIdx.x; q < c.ng; q += blockDim.x) {
    bbj[q] = tot[q][2];
    thj[q] = d.gv[c.g0 + q].eta2 * bbj[q];  // stop at |r|^2 <= eta^2 |b|^2 (the gel's forcing term)
    const double pw = tot[q][1], rho = tot[q][0] / pw;
    rhoj[q] = (pw > 0.0 && isfinite(rho)) ? rho : 0.0;
  }
  __syncthreads();
  // a non-finite entry of the previous direction anywhere in the gel makes its sums non-finite
  // and rho = 0: the solve then starts from zero without touching that direction
  if (mine && !helper) {
    const double rho = rhoj[j];
    if (rho != 0.0) {
      x0 = rho * xp0; x1 = rho * xp1; x2 = rho * xp2;
      r0 = fma(-rho, a0, r0); r1 = fma(-rho, a1, r1); r2 = fma(-rho, a2, r2);
    }
    u0 = fma(M[2], r2, fma(M[1], r1, M[0] * r0));
    u1 = fma(M[5], r2, fma(M[4], r1, M[3] * r0));
    u2 = fma(M[8], r2, fma(M[7], r1, M[6] * r0));
    d.u[row] = make_double4_32a(u0, u1, u2, 0.0);
  }
  // u complete before the SpMV; every CTA has read the start's sums before any reuses their slots
  if (!group_barrier(c, d, &s_fail)) return;
  // ---- w = A u, m = M^-1 w; dot products of iteration 0
  if (mine) {
    if (SPLIT == 2)
      res_spmv_half(sv, sc, w, helper ? 1 : 0, lane, d.u, w0, w1, w2);
    else
      res_spmv<double, double4_32a, double>(sv, sc, w, lane, d.u, w0, w1, w2);
  }
  if (SPLIT == 2) {
    if (helper && mine) {
      hsw[0] = w0; hsw[32] = w1; hsw[64] = w2;
    }
    __syncthreads();
    if (!helper && mine) {
      w0 += hsw[0]; w1 += hsw[32]; w2 += hsw[64];
    }
  }
  if (has && !helper) {
    double ga = 0.0, de = 0.0, rr = 0.0;
    if (mine) {
      if (fixed) w0 = w1 = w2 = 0.0;
      m0 = fma(M[2], w2, fma(M[1], w1, M[0] * w0));
      m1 = fma(M[5], w2, fma(M[4], w1, M[3] * w0));
      m2 = fma(M[8], w2, fma(M[7], w1, M[6] * w0));
      mbuf[0][row] = make_double4_32a(m0, m1, m2, 0.0);
      ga = fma(r2, u2, fma(r1, u1, r0 * u0));
      de = fma(w2, u2, fma(w1, u1, w0 * u0));
      rr = fma(r2, r2, fma(r1, r1, r0 * r0));
    }
    put_sum3(dsm, 4 * sw, warp_sum3(ga, de, rr, lane), lane);
  }
  res_post(d, c, dsm, 0, 3, 0, tot);
  if (!group_barrier(c, d, &s_fail)) return;
  for (int i = 0;; ++i) {
    const int par = i & 1;
    double n0 = 0, n1 = 0, n2 = 0;
    if (wid == ctl) {
      ctl_collect(d, c, 0, 3, par, tot);
      int any = 0;
      for (int q = lane; q < c.ng; q += 32) {
        run[par ^ 1][q] = 0;
        if (!run[par][q]) continue;
        const double ga = tot[q][0], de = tot[q][1], rr = tot[q][2];
        if (!(rr > thj[q]) || i >= maxit) {
          if (blockIdx.x == c.c0) {
            d.gv[c.g0 + q].pcg_it = i;
            d.gv[c.g0 + q].bb = bbj[q];
            d.gv[c.g0 + q].res2 = bbj[q] > 0.0 ? rr / bbj[q] : 0.0;
            d.gv[c.g0 + q].pcg_done = 1;
          }
          continue;
        }
        any = 1;
        run[par ^ 1][q] = 1;
        double al, be;
        cg_scalars(i + 1, ga, de, gprev[q], aprev[q], al, be);
        gprev[q] = ga;
        aprev[q] = al;
        alj[q] = al;
        bej[q] = be;
      }
      any = __any_sync(0xffffffffu, any);
      if (lane == 0) s_any = any;
    } else if (has && run[par][j]) {
      if (SPLIT == 2) {
        res_spmv_half(sv, sc, w, helper ? 1 : 0, lane, mbuf[par], n0, n1, n2);
        if (helper) {
          hsw[0] = n0; hsw[32] = n1; hsw[64] = n2;
        }
      } else {
        res_spmv<double, double4_32a, double>(sv, sc, w, lane, mbuf[par], n0, n1, n2);
      }
    }
    __syncthreads();
    if (!s_any) break;
    if (has && !helper) {
      double ga = 0.0, de = 0.0, rr = 0.0;
      if (run[par ^ 1][j]) {  // implies run[par][j]: this iteration's SpMV ran
        if (SPLIT == 2) {
          n0 += hsw[0]; n1 += hsw[32]; n2 += hsw[64];
        }
        if (fixed) n0 = n1 = n2 = 0.0;
        const double be = bej[j], al = alj[j];
        z0 = fma(be, z0, n0); z1 = fma(be, z1, n1); z2 = fma(be, z2, n2);
        q0 = fma(be, q0, m0); q1 = fma(be, q1, m1); q2 = fma(be, q2, m2);
        t0 = fma(be, t0, w0); t1 = fma(be, t1, w1); t2 = fma(be, t2, w2);
        p0 = fma(be, p0, u0); p1 = fma(be, p1, u1); p2 = fma(be, p2, u2);
        x0 = fma(al, p0, x0); x1 = fma(al, p1, x1); x2 = fma(al, p2, x2);
        r0 = fma(-al, t0, r0); r1 = fma(-al, t1, r1); r2 = fma(-al, t2, r2);
        u0 = fma(-al, q0, u0); u1 = fma(-al, q1, u1); u2 = fma(-al, q2, u2);
        w0 = fma(-al, z0, w0); w1 = fma(-al, z1, w1); w2 = fma(-al, z2, w2);
        m0 = fma(M[2], w2, fma(M[1], w1, M[0] * w0));
        m1 = fma(M[5], w2, fma(M[4], w1, M[3] * w0));
        m2 = fma(M[8], w2, fma(M[7], w1, M[6] * w0));
        mbuf[par ^ 1][row] = make_double4_32a(m0, m1, m2, 0.0);
        ga = fma(r2, u2, fma(r1, u1, r0 * u0));
        de = fma(w2, u2, fma(w1, u1, w0 * u0));
        rr = fma(r2, r2, fma(r1, r1, r0 * r0));
      }
      put_sum3(dsm, 4 * sw, warp_sum3(ga, de, rr, lane), lane);
    }
    res_post(d, c, dsm, 0, 3, par ^ 1, tot);
    if (!group_barrier(c, d, &s_fail)) return;
  }
  if (mine && !helper) d.p[row] = make_double4_32a(x0, x1, x2, 0.0);
  pcg_epilogue(d, plan, c, dsm, tot, gact, &s_fail);
}

__global__ void __launch_bounds__(32 * RES_MAXW, 1) k_pcg_mixed_res(Dev d, int phase, PcgPlan plan,
                                                                 int maxit, int refine_max, int wmax) {
  extern __shared__ __align__(16) double dyn[];
  __shared__ double tot[PCG_MAXG][4];
  __shared__ double bbj[PCG_MAXG], thj[PCG_MAXG], tolj[PCG_MAXG], rr0j[PCG_MAXG], rhoj[PCG_MAXG];
  __shared__ float alj[PCG_MAXG], bej[PCG_MAXG], gprf[PCG_MAXG], aprf[PCG_MAXG];
  __shared__ int gact[PCG_MAXG], run[PCG_MAXG], inner[2][PCG_MAXG], itj[PCG_MAXG];
  __shared__ int s_fail, s_any;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, ctl = plan.max_slices;
  PcgCta c = pcg_cta(d, plan);
  double* dsm;
  double* hs;
  float* sv;
  int* sc;
  res_smem<float>(dyn, plan.max_slices, wmax, wid, false, dsm, hs, sv, sc);
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
  float4* mbuf[2] = {d.pp32, d.s32};
  int w = 0;
  double g0 = 0, g1 = 0, g2 = 0, R0 = 0, R1 = 0, R2 = 0, P0 = 0, P1 = 0, P2 = 0;  // FP64: grad, r, p
  float M[9];
  for (int e = 0; e < 9; ++e) M[e] = 0.f;
  // start from p = rho p_prev, the minimiser of the quadratic model along the gel's previous
  // Newton direction (FP64 arithmetic on the FP32 matrix, as the residual refinement)
  double xp0 = 0.0, xp1 = 0.0, xp2 = 0.0, a0 = 0.0, a1 = 0.0, a2 = 0.0;
  if (mine) {
    w = res_load<float>(d, s, d.vals32, sv, sc, lane, 32);
    __syncwarp();
    for (int e = 0; e < 9; ++e) M[e] = d.Minv32[9 * row + e];
    const double4_32a gr = d.grad[row];
    g0 = gr.x; g1 = gr.y; g2 = gr.z;
    R0 = -g0; R1 = -g1; R2 = -g2;
    if (!fixed) {
      const double4_32a pv = d.p[row];
      xp0 = pv.x; xp1 = pv.y; xp2 = pv.z;
      res_spmv<float, double4_32a, double>(sv, sc, w, lane, d.p, a0, a1, a2);
    }
  }
  if (has) {
    const double bp = warp_sum(fma(R2, xp2, fma(R1, xp1, R0 * xp0)));
    const double pw = warp_sum(fma(a2, xp2, fma(a1, xp1, a0 * xp0)));
    const double bb = warp_sum(fma(R2, R2, fma(R1, R1, R0 * R0)));
    if (lane == 0) {
      dsm[4 * wid + 0] = bp;
      dsm[4 * wid + 1] = pw;
      dsm[4 * wid + 2] = bb;
    }
  }
  res_post(d, c, dsm, 0, 3, 0, tot);
  if (!group_barrier(c, d, &s_fail)) return;
  {
    ResPrefetch pf;
    res_prefetch(d, c, 0, 3, 0, pf);
    res_finish(c, 0, 3, pf, tot);
  }
  for (int q = threadIdx.x; q < c.ng; q += blockDim.x) {
    bbj[q] = tot[q][2];
    thj[q] = d.gv[c.g0 + q].eta2 * bbj[q];  // stop at |r|^2 <= eta^2 |b|^2 (the gel's forcing term)
    const double pw = tot[q][1], rho = tot[q][0] / pw;
    rhoj[q] = (pw > 0.0 && isfinite(rho)) ? rho : 0.0;
  }
  __syncthreads();
  if (mine && rhoj[j] != 0.0) {  // rho = 0 (no usable previous direction): start from zero
    const double rho = rhoj[j];
    P0 = rho * xp0; P1 = rho * xp1; P2 = rho * xp2;
    R0 = fma(-rho, a0, R0); R1 = fma(-rho, a1, R1); R2 = fma(-rho, a2, R2);
  }
  if (has) {  // |r|^2 at the start, through the other exchange set (the first one may still be read)
    const double rr = warp_sum(fma(R2, R2, fma(R1, R1, R0 * R0)));
    if (lane == 0) dsm[4 * wid + 2] = rr;
  }
  res_post(d, c, dsm, 2, 3, 1, tot);
  if (!group_barrier(c, d, &s_fail)) return;
  {
    ResPrefetch pf;
    res_prefetch(d, c, 2, 3, 1, pf);
    res_finish(c, 2, 3, pf, tot);
  }
  for (int round = 0;; ++round) {
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    for (int q = threadIdx.x; q < c.ng; q += blockDim.x) {
      inner[0][q] = 0;
      if (!run[q]) continue;
      const double rr = tot[q][2], bb = bbj[q];
      if (!(rr > thj[q]) || round >= refine_max) {
        run[q] = 0;
        if (blockIdx.x == c.c0) {
          d.gv[c.g0 + q].res2 = bb > 0.0 ? rr / bb : 0.0;
          d.gv[c.g0 + q].pcg_done = 1;
          d.gv[c.g0 + q].rounds = round;
          d.gv[c.g0 + q].bb = bb;
          d.gv[c.g0 + q].pcg_it = itj[q];
        }
        continue;
      }
      s_any = 1;
      inner[0][q] = 1;
      tolj[q] = fmax(thj[q] / rr, 1e-11);
    }
    __syncthreads();
    if (!s_any) break;
    // ---- inner init: r = r64, x = 0, u = M^-1 r (to global), then w = A u, m = M^-1 w
    float x0 = 0.f, x1 = 0.f, x2 = 0.f, r0 = 0.f, r1 = 0.f, r2 = 0.f, u0 = 0.f, u1 = 0.f, u2 = 0.f;
    float w0 = 0.f, w1 = 0.f, w2 = 0.f, z0 = 0.f, z1 = 0.f, z2 = 0.f, q0 = 0.f, q1 = 0.f, q2 = 0.f;
    float t0 = 0.f, t1 = 0.f, t2 = 0.f, p0 = 0.f, p1 = 0.f, p2 = 0.f, m0 = 0.f, m1 = 0.f, m2 = 0.f;
    const bool in = has && inner[0][j];
    if (in) {
      r0 = (float)R0; r1 = (float)R1; r2 = (float)R2;
      u0 = fmaf(M[2], r2, fmaf(M[1], r1, M[0] * r0));
      u1 = fmaf(M[5], r2, fmaf(M[4], r1, M[3] * r0));
      u2 = fmaf(M[8], r2, fmaf(M[7], r1, M[6] * r0));
      d.u32[row] = make_float4(u0, u1, u2, 0.f);
    }
    if (!group_barrier(c, d, &s_fail)) return;
    if (has) {
      double ga = 0.0, de = 0.0, rr = 0.0;
      if (in) {
        res_spmv<float, float4, float>(sv, sc, w, lane, d.u32, w0, w1, w2);
        if (fixed) w0 = w1 = w2 = 0.f;
        m0 = fmaf(M[2], w2, fmaf(M[1], w1, M[0] * w0));
        m1 = fmaf(M[5], w2, fmaf(M[4], w1, M[3] * w0));
        m2 = fmaf(M[8], w2, fmaf(M[7], w1, M[6] * w0));
        mbuf[0][row] = make_float4(m0, m1, m2, 0.f);
        ga = warp_sum(fmaf(r2, u2, fmaf(r1, u1, r0 * u0)));
        de = warp_sum(fmaf(w2, u2, fmaf(w1, u1, w0 * u0)));
        rr = warp_sum(fmaf(r2, r2, fmaf(r1, r1, r0 * r0)));
      }
      if (lane == 0) {
        dsm[4 * wid + 0] = ga;
        dsm[4 * wid + 1] = de;
        dsm[4 * wid + 2] = rr;
      }
    }
    res_post_f(d, c, dsm, 0, 3, 0, tot);
    if (!group_barrier(c, d, &s_fail)) return;
    // ---- inner pipelined CG in FP32
    for (int i = 0;; ++i) {
      const int par = i & 1;
      float n0 = 0.f, n1 = 0.f, n2 = 0.f;
      if (wid == ctl) {
        ctl_collect(d, c, 0, 3, par, tot);
        int any = 0;
        for (int q = lane; q < c.ng; q += 32) {
          inner[par ^ 1][q] = 0;
          if (!inner[par][q]) continue;
          const double ga = tot[q][0], de = tot[q][1], rr = tot[q][2];
          if (i == 0) rr0j[q] = rr;
          if (!(rr > tolj[q] * rr0j[q]) || i >= maxit) {
            itj[q] += i;
            continue;
          }
          any = 1;
          inner[par ^ 1][q] = 1;
          // FP32 scalars for the FP32 iteration: beta = ga / ga_prev, alpha = ga / (de - beta ga / al_prev)
          const float gf = (float)ga, df = (float)de;
          float al, be;
          if (i == 0) {
            be = 0.f;
            al = gf / df;
          } else {
            be = gf / gprf[q];
            al = gf / (df - be * (gf / aprf[q]));
          }
          gprf[q] = gf;
          aprf[q] = al;
          alj[q] = al;
          bej[q] = be;
        }
        any = __any_sync(0xffffffffu, any);
        if (lane == 0) s_any = any;
      } else if (has && inner[par][j]) {
        res_spmv<float, float4, float>(sv, sc, w, lane, mbuf[par], n0, n1, n2);
        if (fixed) n0 = n1 = n2 = 0.f;
      }
      __syncthreads();
      if (!s_any) break;
      if (has) {
        double ga = 0.0, de = 0.0, rr = 0.0;
        if (inner[par ^ 1][j]) {
          const float be = bej[j], al = alj[j];
          z0 = fmaf(be, z0, n0); z1 = fmaf(be, z1, n1); z2 = fmaf(be, z2, n2);
          q0 = fmaf(be, q0, m0); q1 = fmaf(be, q1, m1); q2 = fmaf(be, q2, m2);
          t0 = fmaf(be, t0, w0); t1 = fmaf(be, t1, w1); t2 = fmaf(be, t2, w2);
          p0 = fmaf(be, p0, u0); p1 = fmaf(be, p1, u1); p2 = fmaf(be, p2, u2);
          x0 = fmaf(al, p0, x0); x1 = fmaf(al, p1, x1); x2 = fmaf(al, p2, x2);
          r0 = fmaf(-al, t0, r0); r1 = fmaf(-al, t1, r1); r2 = fmaf(-al, t2, r2);
          u0 = fmaf(-al, q0, u0); u1 = fmaf(-al, q1, u1); u2 = fmaf(-al, q2, u2);
          w0 = fmaf(-al, z0, w0); w1 = fmaf(-al, z1, w1); w2 = fmaf(-al, z2, w2);
          m0 = fmaf(M[2], w2, fmaf(M[1], w1, M[0] * w0));
          m1 = fmaf(M[5], w2, fmaf(M[4], w1, M[3] * w0));
          m2 = fmaf(M[8], w2, fmaf(M[7], w1, M[6] * w0));
          mbuf[par ^ 1][row] = make_float4(m0, m1, m2, 0.f);
          ga = warp_sum(fmaf(r2, u2, fmaf(r1, u1, r0 * u0)));
          de = warp_sum(fmaf(w2, u2, fmaf(w1, u1, w0 * u0)));
          rr = warp_sum(fmaf(r2, r2, fmaf(r1, r1, r0 * r0)));
        }
        if (lane == 0) {
          dsm[4 * wid + 0] = ga;
          dsm[4 * wid + 1] = de;
          dsm[4 * wid + 2] = rr;
        }
      }
      res_post_f(d, c, dsm, 0, 3, par ^ 1, tot);
      if (!group_barrier(c, d, &s_fail)) return;
    }
    // ---- p += x32 (FP64), then the FP64 residual r64 = b - A p (FP32 values, FP64 arithmetic)
    const bool rn = has && run[j];
    if (rn) {
      P0 += (double)x0;
      P1 += (double)x1;
      P2 += (double)x2;
      d.p[row] = make_double4_32a(P0, P1, P2, 0.0);
    }
    if (!group_barrier(c, d, &s_fail)) return;
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
    res_post(d, c, dsm, 2, 3, 0, tot);
    if (!group_barrier(c, d, &s_fail)) return;
    {
      ResPrefetch pf;
      res_prefetch(d, c, 2, 3, 0, pf);
      res_finish(c, 2, 3, pf, tot);
    }
  }
  if (mine) d.p[row] = make_double4_32a(P0, P1, P2, 0.0);
  pcg_epilogue(d, plan, c, dsm, tot, gact, &s_fail);
}

// the FP64 kernel takes two warps per slice while a CTA holds at most RES_SPLIT_MAXS slices
static bool res_split(bool mixed, int max_slices) { return !mixed && max_slices <= RES_SPLIT_MAXS; }

static const void* res_kernel(bool mixed, int max_slices) {
  if (mixed) return (const void*)k_pcg_mixed_res;
  return res_split(false, max_slices) ? (const void*)k_pcg64_res<2> : (const void*)k_pcg64_res<1>;
}

static int res_threads(bool mixed, int max_slices) {
  return 32 * ((res_split(mixed, max_slices) ? 2 : 1) * max_slices + 1);
}

// dynamic shared memory of the resident kernels
size_t pcg_res_smem(bool mixed, int max_slices, int wmax) {
  const size_t nw = (size_t)max_slices;
  return sizeof(double) * (4 + (res_split(mixed, max_slices) ? 96 : 0)) * nw +
         nw * wmax * 288 * (mixed ? sizeof(float) : sizeof(double)) + nw * wmax * 32 * sizeof(int);
}

// co-resident CTAs per SM of the resident kernel (0 if it cannot be launched so)
int pcg_res_ctas_per_sm(bool mixed, int max_slices, int wmax) {
  if (max_slices + 1 > RES_MAXW) return 0;
  const size_t smem = pcg_res_smem(mixed, max_slices, wmax);
  const void* fn = res_kernel(mixed, max_slices);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, res_threads(mixed, max_slices), smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_pcg_res(const Dev& d, int phase, const PcgPlan& plan, int nctas, bool mixed, int maxit,
                           int refine_max, int wmax, cudaStream_t st) {
  Dev dd = d;
  PcgPlan pp = plan;
  const size_t smem = pcg_res_smem(mixed, plan.max_slices, wmax);
  count_launch(1);
  if (mixed) {
    void* args[] = {(void*)&dd, (void*)&phase, (void*)&pp, (void*)&maxit, (void*)&refine_max, (void*)&wmax};
    return cudaLaunchCooperativeKernel((const void*)k_pcg_mixed_res, dim3(nctas), dim3(32 * (plan.max_slices + 1)), args,
                                       smem, st);
  }
  void* args[] = {(void*)&dd, (void*)&phase, (void*)&pp, (void*)&maxit, (void*)&wmax};
  return cudaLaunchCooperativeKernel(res_kernel(false, plan.max_slices), dim3(nctas),
                                     dim3(res_threads(false, plan.max_slices)), args, smem, st);
}

}  // namespace txg

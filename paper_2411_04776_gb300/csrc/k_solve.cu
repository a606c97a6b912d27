// Newton-system assembly, block-Jacobi PCG, incremental-potential energy and the per-gel
// Newton / line-search bookkeeping.
//
//   * gather: every 3x3 block of the sliced BSR sums its per-tet contributions in a fixed order
//     (plus M/h^2 on the diagonal); diagonal blocks also gather the gradient
//     g = M (x - xt) / h^2 + sum_t V_t P_t D_a.  Dirichlet rows get g = 0.
//   * PCG (batches too large for the resident kernels of k_pcg_res.cu): one persistent cooperative
//     kernel per Newton iteration runs every PCG iteration of every gel of the batch
//     (Chronopoulos-Gear single-reduction CG), in one of two forms.  Per-gel CTA groups: each gel
//     (or run of small gels) has its own CTAs and group barrier; best for a few gels.  Pooled:
//     one CTA per SM splits the slices of the gels still iterating evenly at every phase, so no SM
//     idles while the slowest gel finishes; best for many gels.  Dot products are per-slice (or
//     per-CTA) partials added in a fixed order: results are reproducible.
//   * energy: E(x + alpha p) per gel = inertia + elastic + barrier, as per-piece partial sums
//     (pieces never straddle gels) reduced per gel in a fixed order; the reduction kernel also
//     takes the line-search decision (accept on E <= E_cur, else halve alpha).
#include <type_traits>

#include "dev_contact.cuh"
#include "dev_elastic.cuh"
#include "dev_pcg.cuh"

namespace txg {

static inline int nblk(int n, int t) { return (n + t - 1) / t; }

// ---------------------------------------------------------------- exclusive scan (int)
constexpr int SCAN_T = 1024;

__global__ void k_scan_blocks(const int* in, int* out, int* bsum, int n) {
  __shared__ int s[SCAN_T];
  const int i = blockIdx.x * SCAN_T + threadIdx.x;
  const int v = i < n ? in[i] : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < SCAN_T; off <<= 1) {
    int t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = s[threadIdx.x] - v;
  if (threadIdx.x == SCAN_T - 1) bsum[blockIdx.x] = s[SCAN_T - 1];
}

__global__ void k_scan_sums(int* bsum, int nb, int* total_out) {
  __shared__ int s[SCAN_T];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += SCAN_T) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? bsum[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < SCAN_T; off <<= 1) {
      int t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nb) bsum[i] = carry + s[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == SCAN_T - 1) carry += s[SCAN_T - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_add(int* out, const int* bsum, int n, const int* total, int* out_end) {
  const int i = blockIdx.x * SCAN_T + threadIdx.x;
  if (i < n) out[i] += bsum[blockIdx.x];
  if (i == 0) *out_end = *total;
}

// out[0..n] = exclusive scan of in[0..n), out[n] = total.  tmp: >= nblk(n)+1 ints.
void launch_scan(const int* in, int* out, int n, int* tmp, cudaStream_t st) {
  const int nb = nblk(n, SCAN_T);
  if (n == 0) {
    cudaMemsetAsync(out, 0, sizeof(int), st);
    return;
  }
  k_scan_blocks<<<nb, SCAN_T, 0, st>>>(in, out, tmp, n);
  count_launch(1);
  k_scan_sums<<<1, SCAN_T, 0, st>>>(tmp, nb, tmp + nb);
  count_launch(1);
  k_scan_add<<<nb, SCAN_T, 0, st>>>(out, tmp, n, tmp + nb, out + n);
  count_launch(1);
}

// ---------------------------------------------------------------- gather (assembly)

template <bool MIXED>
__global__ void __launch_bounds__(256) k_gather(Dev d, int phase, int nbp) {
  const int bp = blockIdx.x * blockDim.x + threadIdx.x;
  if (bp >= nbp) return;
  const int r = d.bp_row[bp];
  const int g = d.vgel[r];
  if (d.gc[g].phase != phase) return;
  const int c = d.colidx[bp];
  const bool diag = d.diag_pos[r] == bp;
  // the block sum in the precision of the stored block (FP64 adds run at 1/64 of the FP32 rate);
  // the gradient stays FP64
  using HT = typename std::conditional<MIXED, float, double>::type;
  HT h[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) h[e] = HT(0);
  double gr[3] = {0.0, 0.0, 0.0};
  const int c0 = d.ctr_ptr[bp], c1 = d.ctr_ptr[bp + 1];
#pragma unroll 2
  for (int k = c0; k < c1; ++k) {
    const int code = d.ctr[k];
    const int t = code >> 4, a = (code >> 2) & 3, b = code & 3;
    const bool tr = a > b;
    const int blk = tr ? ublk(b, a) : ublk(a, b);
    HT v[12];  // the block as stored (row-major 3x3, padded), read with 16-byte loads
    if (MIXED) {
      const float4* s = reinterpret_cast<const float4*>(d.tscr32 + (size_t)t * TS32 + BLK32 * blk);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float4 f = s[q];
        v[4 * q] = f.x;
        v[4 * q + 1] = f.y;
        v[4 * q + 2] = f.z;
        v[4 * q + 3] = f.w;
      }
    } else {
      const double2* s = reinterpret_cast<const double2*>(d.tscr + (size_t)t * TS + BLK64 * blk);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const double2 f = s[q];
        v[2 * q] = (HT)f.x;
        v[2 * q + 1] = (HT)f.y;
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) h[3 * i + j] += tr ? v[3 * j + i] : v[3 * i + j];
    if (diag) {
      const double* s = d.tscr + (size_t)t * TS + GOFF + 3 * a;
      gr[0] += s[0];
      gr[1] += s[1];
      gr[2] += s[2];
    }
  }
  if (diag) {
    const double h2 = d.gc[g].h * d.gc[g].h;
    const double m = d.mass[r] / h2;
    h[0] += (HT)m;
    h[4] += (HT)m;
    h[8] += (HT)m;
    const double4_32a x = d.x[r], xt = d.xt[r];
    double4_32a go;
    if (d.fixed[r]) {
      go = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    } else {
      const double4_32a cg = d.cgrad[r];  // the contact kernels' part
      go.x = gr[0] + m * (x.x - xt.x) + cg.x;
      go.y = gr[1] + m * (x.y - xt.y) + cg.y;
      go.z = gr[2] + m * (x.z - xt.z) + cg.z;
      go.w = 0.0;
    }
    d.grad[r] = go;
  }
  (void)c;
  // the block in the slice's value layout (val_addr64 / val_addr32): 16-byte stores of its pairs
  // (FP64) or quads (FP32), then the ninth element
  const int l = bp & 31;
  if (MIXED) {
    float* b = d.vals32 + (size_t)9 * (bp & ~31);
    *reinterpret_cast<float4*>(b + 4 * l) = make_float4((float)h[0], (float)h[1], (float)h[2], (float)h[3]);
    *reinterpret_cast<float4*>(b + 128 + 4 * l) = make_float4((float)h[4], (float)h[5], (float)h[6], (float)h[7]);
    b[256 + l] = (float)h[8];
  } else {
    double* b = d.vals + (size_t)9 * (bp & ~31);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      *reinterpret_cast<double2*>(b + 64 * q + 2 * l) = make_double2((double)h[2 * q], (double)h[2 * q + 1]);
    b[256 + l] = (double)h[8];
  }
}

void launch_gather(const Dev& d, int phase, int nbp, bool mixed, cudaStream_t st) {
  if (mixed)
    k_gather<true><<<nblk(nbp, 256), 256, 0, st>>>(d, phase, nbp);
  else
    k_gather<false><<<nblk(nbp, 256), 256, 0, st>>>(d, phase, nbp);
  count_launch(1);
}

// block-Jacobi preconditioner: inverse of every free row's 3x3 diagonal block
template <bool MIXED>
__global__ void k_precond(Dev d, int phase) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.nrows) return;
  const int g = d.vgel[r];
  if (d.gc[g].phase != phase) return;
  double A[9], R[9];
  const int bp = d.diag_pos[r];
  for (int e = 0; e < 9; ++e) A[e] = MIXED ? (double)d.vals32[val_addr32(bp, e)] : d.vals[val_addr64(bp, e)];
  if (d.fixed[r]) {
    for (int e = 0; e < 9; ++e) R[e] = 0.0;
  } else {
    const double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    const double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    const double id = 1.0 / det;
    R[0] = c00 * id;
    R[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    R[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    R[3] = c01 * id;
    R[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    R[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    R[6] = c02 * id;
    R[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    R[8] = (A[0] * A[4] - A[1] * A[3]) * id;
  }
  for (int e = 0; e < 9; ++e) {
    if (MIXED)
      d.Minv32[9 * r + e] = (float)R[e];
    else
      d.Minv[9 * r + e] = R[e];
  }
}

void launch_precond(const Dev& d, int phase, bool mixed, cudaStream_t st) {
  if (mixed)
    k_precond<true><<<nblk(d.nrows, 128), 128, 0, st>>>(d, phase);
  else
    k_precond<false><<<nblk(d.nrows, 128), 128, 0, st>>>(d, phase);
  count_launch(1);
}

// One projected-Newton direction per gel of the gels in `phase`: block-Jacobi preconditioned CG
// on H p = -g (Chronopoulos-Gear: one reduction phase per iteration), FP64, stops per gel when
// |r| <= eta |g| or after maxit iterations.
__global__ void __launch_bounds__(PCG_T, 4) k_pcg64(Dev d, int phase, PcgPlan plan, int maxit) {
  extern __shared__ double dsm[];  // [slices of this CTA][4]
  __shared__ double tot[PCG_MAXG][4];
  __shared__ double bbj[PCG_MAXG], thj[PCG_MAXG], gprev[PCG_MAXG], aprev[PCG_MAXG], alj[PCG_MAXG], bej[PCG_MAXG];
  __shared__ double rhoj[PCG_MAXG];
  __shared__ int gact[PCG_MAXG], run[PCG_MAXG];
  __shared__ int s_fail, s_any;
  // coarse space (a group of one gel that has a free body): per-warp partials, E^-1, the
  // recurrences Z^T r and Z^T s, the coarse correction c = E^-1 Z^T r, the group totals
  __shared__ double czw[PCG_T / 32][CZ_N];
  __shared__ double czEi[36], czr[6], czs[6], czc[6], czt[CZ_N];
  __shared__ int cz_on;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  PcgCta c = pcg_cta(d, plan);
  if (threadIdx.x == 0) {
    s_fail = 0;
    cz_on = 0;
  }
  for (int j = threadIdx.x; j < c.ng; j += PCG_T) {
    gact[j] = d.gc[c.g0 + j].phase == phase ? 1 : 0;
    run[j] = gact[j];
  }
  __syncthreads();
  const GelInfo& G0 = d.gi[c.g0];
  const bool coarse = c.ng == 1 && G0.cbody >= 0 && gact[0];  // uniform over the group
  const int cb = G0.cbody;
  // body row r: d = x_r - c (false for every other row)
  auto cz_row = [&](int r, double dd[3]) {
    if (!coarse || d.vcomp[r] != cb || d.fixed[r]) return false;
    const double4_32a xr = d.x[r];
    dd[0] = xr.x - G0.cctr[0];
    dd[1] = xr.y - G0.cctr[1];
    dd[2] = xr.z - G0.cctr[2];
    return true;
  };
  // the CTA's sum of the per-warp partials [0, n) to its exchange slots (the group sum's barrier
  // that follows makes them visible; they are read before the next group barrier)
  auto cz_publish = [&](int n) {
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += PCG_T) {
      double v = 0.0;
      for (int q = 0; q < PCG_T / 32; ++q) v += czw[q][k];
      d.czpart[(size_t)k * gridDim.x + blockIdx.x] = v;
    }
  };
  // the group's totals [0, n) in CTA order (identical in every CTA), into czt
  auto cz_collect = [&](int n) {
    for (int k = threadIdx.x; k < n; k += PCG_T) {
      double v = 0.0;
      for (int q = c.c0; q < c.c0 + c.nc; ++q) v += d.czpart[(size_t)k * gridDim.x + q];
      czt[k] = v;
    }
    __syncthreads();
  };
  // ---- Galerkin start: x0 = rho p_prev, the minimiser of the quadratic model along the gel's
  // previous Newton direction (in d.p; rho = b.p_prev / p_prev.A p_prev, 0 without a usable one);
  // a = A p_prev goes to d.w.  Partials b.p_prev (k = 0), p_prev.a (1), |b|^2 (3).  (With a
  // coarse space, k_pcg_cz_setup left this CTA's partials of E = Z^T A Z, Z^T b and Z^T a.)
  for (int s = c.s0 + wid; s < c.s1; s += PCG_T / 32) {
    double bp = 0.0, pw = 0.0, bb = 0.0;
    if (gact[plan.slice_gel[s] - c.g0]) {
      const int r = 32 * s + lane;
      const double4_32a gr = d.grad[r];
      const double4_32a b = make_double4_32a(-gr.x, -gr.y, -gr.z, 0.0);
      const bool fx = d.fixed[r] != 0;
      const double4_32a pv = fx ? make_double4_32a(0.0, 0.0, 0.0, 0.0) : d.p[r];
      const double4_32a a = fx ? make_double4_32a(0.0, 0.0, 0.0, 0.0) : spmv_row64(d, s, lane, d.p);
      d.w[r] = a;
      bp = dot4(b, pv);
      pw = dot4(pv, a);
      bb = dot4(b, b);
    }
    bp = warp_sum(bp);
    pw = warp_sum(pw);
    bb = warp_sum(bb);
    if (lane == 0) {
      dsm[(s - c.s0) * 4 + 0] = bp;
      dsm[(s - c.s0) * 4 + 1] = pw;
      dsm[(s - c.s0) * 4 + 2] = 0.0;
      dsm[(s - c.s0) * 4 + 3] = bb;
    }
  }
  // (the group sum's barrier also ends every CTA's SpMV on d.p before d.p is overwritten below)
  if (!group_sum(d, c, dsm, 0, 4, tot, &s_fail)) return;
  for (int j = threadIdx.x; j < c.ng; j += PCG_T) {
    bbj[j] = tot[j][3];
    thj[j] = d.gv[c.g0 + j].eta2 * bbj[j];  // stop at |r|^2 <= eta^2 |b|^2 (the gel's forcing term)
    const double pw = tot[j][1], rho = tot[j][0] / pw;
    rhoj[j] = (pw > 0.0 && isfinite(rho)) ? rho : 0.0;  // a non-finite p_prev anywhere gives 0
  }
  __syncthreads();
  if (coarse) {  // E^-1, Z^T b and Z^T a of the group (k_pcg_cz_factor)
    const double* f = d.czfac + (size_t)CZ_F * c.c0;
    for (int q = threadIdx.x; q < 48; q += PCG_T) {
      if (q < 36) czEi[q] = f[q];
      else czt[q - 36] = f[q];
    }
    if (threadIdx.x == 0) cz_on = f[48] != 0.0;  // off for this solve if E was not numerically SPD
    __syncthreads();
    if (threadIdx.x < 6) {
      czr[threadIdx.x] = czt[threadIdx.x] - rhoj[0] * czt[6 + threadIdx.x];  // Z^T r0, r0 = b - rho a
      czs[threadIdx.x] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x < 6) czc[threadIdx.x] = cz_on ? cz_mv(czEi, czr, threadIdx.x) : 0.0;
    __syncthreads();
  }
  // ---- x = rho p_prev, r = b - rho a, u = M^-1 r, pp = s = 0
  for (int s = c.s0 + wid; s < c.s1; s += PCG_T / 32) {
    const int j = plan.slice_gel[s] - c.g0;
    if (!gact[j]) continue;
    const int r = 32 * s + lane;
    const double4_32a gr = d.grad[r];
    double4_32a b = make_double4_32a(-gr.x, -gr.y, -gr.z, 0.0);
    double4_32a x = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    const double rho = rhoj[j];
    if (rho != 0.0 && !d.fixed[r]) {
      const double4_32a pv = d.p[r], a = d.w[r];
      x = make_double4_32a(rho * pv.x, rho * pv.y, rho * pv.z, 0.0);
      b.x = fma(-rho, a.x, b.x);
      b.y = fma(-rho, a.y, b.y);
      b.z = fma(-rho, a.z, b.z);
    }
    const double4_32a z = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    d.r[r] = b;
    d.p[r] = x;
    d.pp[r] = z;
    d.s[r] = z;
    double4_32a u0 = mul3(d.Minv + 9 * r, b);
    double dd[3];
    if (cz_on && cz_row(r, dd)) {  // + Z c
      u0.x += czc[0] + czc[4] * dd[2] - czc[5] * dd[1];
      u0.y += czc[1] + czc[5] * dd[0] - czc[3] * dd[2];
      u0.z += czc[2] + czc[3] * dd[1] - czc[4] * dd[0];
    }
    d.u[r] = u0;
  }
  if (!group_barrier(c, d, &s_fail)) return;  // u complete before the SpMV
  const bool czi = coarse && cz_on;  // the coarse correction runs in this solve (uniform)
  for (int k = 1;; ++k) {
    // ---- w = A u; partials gamma = (r, u), delta = (w, u), rr = (r, r); with a coarse space Z^T w
    // (added per slice into the warp's slots)
    if (czi && lane == 0)
      for (int q = 0; q < 6; ++q) czw[wid][q] = 0.0;
    for (int s = c.s0 + wid; s < c.s1; s += PCG_T / 32) {
      double ga = 0.0, de = 0.0, rr = 0.0;
      if (run[plan.slice_gel[s] - c.g0]) {
        const int r = 32 * s + lane;
        double4_32a w = spmv_row64(d, s, lane, d.u);
        if (d.fixed[r]) w = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        d.w[r] = w;
        const double4_32a rv = d.r[r], uv = d.u[r];
        ga = dot4(rv, uv);
        de = dot4(w, uv);
        rr = dot4(rv, rv);
        if (czi) {
          double czq[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, dd[3];
          if (cz_row(r, dd)) cz_zt(w, dd, czq);
          for (int q = 0; q < 6; ++q) {
            const double v = warp_sum(czq[q]);
            if (lane == 0) czw[wid][q] += v;
          }
        }
      }
      ga = warp_sum(ga);
      de = warp_sum(de);
      rr = warp_sum(rr);
      if (lane == 0) {
        dsm[(s - c.s0) * 4 + 0] = ga;
        dsm[(s - c.s0) * 4 + 1] = de;
        dsm[(s - c.s0) * 4 + 2] = rr;
      }
    }
    if (czi) cz_publish(6);
    if (!group_sum(d, c, dsm, 0, 3, tot, &s_fail)) return;
    if (czi) cz_collect(6);
    // ---- per-gel scalars and convergence (identical in every CTA of the group)
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < c.ng; j += PCG_T) {
      if (!run[j]) continue;
      const double ga = tot[j][0], de = tot[j][1], rr = tot[j][2];
      if (!(rr > thj[j]) || k > maxit) {
        run[j] = 0;
        if (blockIdx.x == c.c0) {
          d.gv[c.g0 + j].pcg_it = k - 1;
          d.gv[c.g0 + j].bb = bbj[j];
          d.gv[c.g0 + j].res2 = bbj[j] > 0.0 ? rr / bbj[j] : 0.0;
          d.gv[c.g0 + j].pcg_done = 1;
        }
        continue;
      }
      s_any = 1;
      const double beta = k == 1 ? 0.0 : ga / gprev[j];
      const double alpha = k == 1 ? ga / de : ga / (de - beta * ga / aprev[j]);
      gprev[j] = ga;
      aprev[j] = alpha;
      alj[j] = alpha;
      bej[j] = beta;
      if (czi) {  // (one gel: j = 0) Z^T s = beta Z^T s + Z^T w, Z^T r -= alpha Z^T s
        for (int q = 0; q < 6; ++q) {
          czs[q] = fma(beta, czs[q], czt[q]);
          czr[q] = fma(-alpha, czs[q], czr[q]);
        }
      }
    }
    __syncthreads();
    if (!s_any) break;
    if (czi) {  // c = E^-1 Z^T r
      if (threadIdx.x < 6) czc[threadIdx.x] = cz_mv(czEi, czr, threadIdx.x);
      __syncthreads();
    }
    // ---- vector updates
    for (int s = c.s0 + wid; s < c.s1; s += PCG_T / 32) {
      const int j = plan.slice_gel[s] - c.g0;
      if (!run[j]) continue;
      const double beta = bej[j], alpha = alj[j];
      const int r = 32 * s + lane;
      const double4_32a u = d.u[r], w = d.w[r];
      double4_32a pp = d.pp[r], sv = d.s[r], x = d.p[r], rv = d.r[r];
      pp.x = fma(beta, pp.x, u.x); pp.y = fma(beta, pp.y, u.y); pp.z = fma(beta, pp.z, u.z);
      sv.x = fma(beta, sv.x, w.x); sv.y = fma(beta, sv.y, w.y); sv.z = fma(beta, sv.z, w.z);
      x.x = fma(alpha, pp.x, x.x); x.y = fma(alpha, pp.y, x.y); x.z = fma(alpha, pp.z, x.z);
      rv.x = fma(-alpha, sv.x, rv.x); rv.y = fma(-alpha, sv.y, rv.y); rv.z = fma(-alpha, sv.z, rv.z);
      d.pp[r] = pp;
      d.s[r] = sv;
      d.p[r] = x;
      d.r[r] = rv;
      double4_32a un = mul3(d.Minv + 9 * r, rv);
      double dd[3];
      if (czi && cz_row(r, dd)) {  // + Z c
        un.x += czc[0] + czc[4] * dd[2] - czc[5] * dd[1];
        un.y += czc[1] + czc[5] * dd[0] - czc[3] * dd[2];
        un.z += czc[2] + czc[3] * dd[1] - czc[4] * dd[0];
      }
      d.u[r] = un;
    }
    if (!group_barrier(c, d, &s_fail)) return;
  }
  pcg_epilogue(d, plan, c, dsm, tot, gact, &s_fail);
}

// Coarse-space set-up of the streaming FP64 PCG, launched just before it over the same CTA
// partition: per CTA (a group of one gel with a free body) the partial sums over its slices of
// E = Z^T A Z (packed upper triangle, 21), Z^T b (6, b = -grad) and Z^T A p_prev (6), to d.czpart
// (k_pcg64 adds them up in CTA order).  Its own kernel keeps the set-up's registers out of the
// iteration kernel.
__global__ void __launch_bounds__(PCG_T) k_pcg_cz_setup(Dev d, int phase, PcgPlan plan) {
  __shared__ double czw[PCG_T / 32][CZ_N];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const PcgCta c = pcg_cta(d, plan);
  const GelInfo& G0 = d.gi[c.g0];
  if (!(c.ng == 1 && G0.cbody >= 0 && d.gc[c.g0].phase == phase)) return;
  const int cb = G0.cbody;
  double acc[CZ_N];
  for (int q = 0; q < CZ_N; ++q) acc[q] = 0.0;
  for (int s = c.s0 + wid; s < c.s1; s += PCG_T / 32) {
    const int r = 32 * s + lane;
    if (d.vcomp[r] != cb || d.fixed[r]) continue;
    const double4_32a xr = d.x[r], gr = d.grad[r];
    const double dd[3] = {xr.x - G0.cctr[0], xr.y - G0.cctr[1], xr.z - G0.cctr[2]};
    cz_row_e(d, s, lane, cb, G0.cctr, dd, acc);
    cz_zt(make_double4_32a(-gr.x, -gr.y, -gr.z, 0.0), dd, acc + 21);
    cz_zt(spmv_row64(d, s, lane, d.p), dd, acc + 27);
  }
  for (int q = 0; q < CZ_N; ++q) {
    const double v = warp_sum(acc[q]);
    if (lane == 0) czw[wid][q] = v;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < CZ_N; k += PCG_T) {
    double v = 0.0;
    for (int q = 0; q < PCG_T / 32; ++q) v += czw[q][k];
    d.czpart[(size_t)k * gridDim.x + blockIdx.x] = v;
  }
}

// ... and the inverse: the first CTA of each such group adds the group's partials in CTA order,
// inverts E by Cholesky and leaves [E^-1 (36, row-major) | Z^T b (6) | Z^T A p_prev (6) | ok] in
// d.czfac at the group's first CTA
__global__ void __launch_bounds__(64) k_pcg_cz_factor(Dev d, int phase, PcgPlan plan, int nctas) {
  __shared__ double t[CZ_N];
  const PcgCta c = pcg_cta(d, plan);
  const GelInfo& G0 = d.gi[c.g0];
  if (blockIdx.x != c.c0 || !(c.ng == 1 && G0.cbody >= 0 && d.gc[c.g0].phase == phase)) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = wid; k < CZ_N; k += blockDim.x >> 5) {  // a warp per quantity, lanes over the CTAs
    double v = 0.0;
    for (int q = c.c0 + lane; q < c.c0 + c.nc; q += 32) v += d.czpart[(size_t)k * nctas + q];
    v = warp_sum(v);
    if (lane == 0) t[k] = v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double* f = d.czfac + (size_t)CZ_F * c.c0;
  double L[36];
  for (int q = 0; q < 36; ++q) L[q] = 0.0;
  const bool ok = cz_chol(t, L);
  for (int k = 0; k < 6; ++k) {  // E^-1, column k
    double e[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, x[6];
    e[k] = 1.0;
    cz_solve(L, e, x);
    for (int i = 0; i < 6; ++i) f[6 * i + k] = ok ? x[i] : 0.0;
  }
  for (int q = 0; q < 12; ++q) f[36 + q] = t[21 + q];
  f[48] = ok ? 1.0 : 0.0;
}

void launch_pcg_cz_setup(const Dev& d, int phase, const PcgPlan& plan, int nctas, cudaStream_t st) {
  k_pcg_cz_setup<<<nctas, PCG_T, 0, st>>>(d, phase, plan);
  k_pcg_cz_factor<<<nctas, 64, 0, st>>>(d, phase, plan, nctas);
  count_launch(2);
}

cudaError_t launch_pcg64(const Dev& d, int phase, const PcgPlan& plan, int nctas, int maxit, cudaStream_t st) {
  Dev dd = d;
  PcgPlan pp = plan;
  void* args[] = {(void*)&dd, (void*)&phase, (void*)&pp, (void*)&maxit};
  count_launch(1);
  const size_t smem = (size_t)plan.max_slices * 4 * sizeof(double);
  return cudaLaunchCooperativeKernel((const void*)k_pcg64, dim3(nctas), dim3(PCG_T), args, smem, st);
}

// ---------------------------------------------------------------- pooled streaming PCG
// Every CTA of the launch belongs to one group (the pool).  At each phase the slices of the gels
// still taking part are split evenly over the CTAs: a prefix sum over the gels' slice counts, the
// same in every CTA.  So a gel that converges early leaves no SM idle while the others iterate
// (with a fixed group of CTAs per gel, the whole launch waits for the slowest gel).  Per-slice
// partial sums go to d.pslice; after a pool barrier the owner warp of each gel (in CTA j mod the
// grid, so that the owners' work spreads over the SMs) adds its gel's partials in slice order, takes the gel's decisions and
// publishes them in d.pool, and a second barrier makes them visible to every CTA.  Same
// arithmetic, scalars and stopping rules as the per-group kernels; the sums are deterministic.

constexpr int POOL_T = 1024;  // one CTA per SM: the pool barrier has one arrival per SM
constexpr int POOL_W = POOL_T / 32;

__device__ __forceinline__ bool pool_flag(const Dev& d, int g, int mode, int phase) {
  if (mode == 0) return d.gc[g].phase == phase;
  return mode == 1 ? d.pool[g].run != 0 : d.pool[g].inner != 0;
}

// pre[j] (j = 0..ng): slices of the gels g0 .. g0 + j - 1 whose flag `mode` is set (0: in the
// solve's phase, 1: run, 2: inner); returns pre[ng].  Block-wide, identical in every CTA.
__device__ int pool_prefix(const Dev& d, const PoolPlan& pl, int mode, int phase, int* pre) {
  __shared__ int wtot[POOL_W];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int per = (pl.ng + POOL_T - 1) / POOL_T, j0 = min((int)threadIdx.x * per, pl.ng), j1 = min(j0 + per, pl.ng);
  int loc = 0;
  for (int j = j0; j < j1; ++j) {
    pre[j] = pool_flag(d, pl.g0 + j, mode, phase) ? d.gi[pl.g0 + j].ns : 0;
    loc += pre[j];
  }
  int inc = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) wtot[wid] = inc;
  __syncthreads();
  int base = 0, total = 0;
#pragma unroll
  for (int w = 0; w < POOL_W; ++w) {
    if (w < wid) base += wtot[w];
    total += wtot[w];
  }
  int ex = base + inc - loc;
  for (int j = j0; j < j1; ++j) {
    const int n = pre[j];
    pre[j] = ex;
    ex += n;
  }
  if (threadIdx.x == 0) pre[pl.ng] = total;
  __syncthreads();
  return total;
}

// the CTA's share [a0, a1) of the S active slices
__device__ __forceinline__ void pool_share(int S, int& a0, int& a1) {
  a0 = (int)((long long)blockIdx.x * S / gridDim.x);
  a1 = (int)((long long)(blockIdx.x + 1) * S / gridDim.x);
}

// gel index j (relative to g0) of active slice a: pre[j] <= a < pre[j + 1]
__device__ __forceinline__ int pool_gel_at(const int* pre, int ng, int a) {
  int lo = 0, hi = ng;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= a)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// The CTA's share of the S active slices as a list in shared memory: lst[i] = (slice, gel) for
// the i-th of them (all threads, one entry each); returns its length.  cap: the list's room.
__device__ int pool_list(const Dev& d, const PoolPlan& pl, const int* pre, int S, int2* lst, int cap) {
  int a0, a1;
  pool_share(S, a0, a1);
  const int n = min(a1 - a0, cap);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int a = a0 + i, j = pool_gel_at(pre, pl.ng, a), g = pl.g0 + j;
    lst[i] = make_int2(d.gi[g].s0 + (a - pre[j]), g);
  }
  __syncthreads();
  return n;
}

// the owner warp's sums of partials k in [k0, k1) over gel g's slices, in slice order per lane
// and a fixed warp tree (every lane gets them)
__device__ __forceinline__ void pool_total(const Dev& d, int g, int k0, int k1, double* t) {
  const int lane = threadIdx.x & 31;
  const GelInfo& G = d.gi[g];
  for (int k = k0; k < k1; ++k) {
    double v = 0.0;
    for (int s = G.s0 + lane; s < G.s0 + G.ns; s += 32) v += d.pslice[4 * (size_t)s + k];
    t[k] = warp_sum(v);
  }
}

__device__ __forceinline__ PcgCta pool_cta(const Dev& d, const PoolPlan& pl) {
  PcgCta c;
  c.s0 = c.s1 = 0;
  c.c0 = 0;
  c.nc = gridDim.x;
  c.g0 = pl.g0;
  c.ng = pl.ng;
  c.bar = d.bar;
  c.epoch = 0;
  return c;
}

// g . p and ||p||_inf of the new direction per gel of the solve (the line search's model slope)
__device__ bool pool_epilogue(const Dev& d, const PoolPlan& pl, PcgCta& c, int phase, int* pre, int2* lst,
                              int* s_fail) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gw = wid * gridDim.x + blockIdx.x, nw = gridDim.x * POOL_W;  // owners spread over the CTAs first
  const int nl = pool_list(d, pl, pre, pool_prefix(d, pl, 0, phase, pre), lst, pl.cap);
  for (int i = wid; i < nl; i += POOL_W) {
    const int s = lst[i].x, g = lst[i].y;
    const double4_32a x = d.p[32 * s + lane];
    double gp = dot4(d.grad[32 * s + lane], x);
    double m = fmax(fabs(x.x), fmax(fabs(x.y), fabs(x.z)));
    gp = warp_sum(gp);
    m = warp_max(m);
    if (lane == 0) {
      d.pslice[4 * (size_t)s + 3] = gp;
      atomic_max_pos(&d.gv[g].pnorm_bits, m);
    }
  }
  if (!group_barrier(c, d, s_fail)) return false;
  for (int j = gw; j < pl.ng; j += nw) {  // owner: CTA j mod grid, then warp
    const int g = pl.g0 + j;
    if (d.gc[g].phase != phase) continue;
    double t[4];
    pool_total(d, g, 3, 4, t);
    if (lane == 0) d.gv[g].gtp = t[3];
  }
  return true;
}

// FP64 pooled PCG: block-Jacobi preconditioned CG on H p = -g (Chronopoulos-Gear: one reduction
// phase per iteration), started from x0 = rho p_prev, the minimiser of the quadratic model along
// the gel's previous Newton direction; stops per gel when |r| <= eta |g| or after maxit iterations
__global__ void __launch_bounds__(POOL_T, 1) k_pcg64_pool(Dev d, int phase, PoolPlan pl, int maxit) {
  extern __shared__ int pre[];  // ng + 1, then the CTA's slice list
  int2* lst = reinterpret_cast<int2*>(pre + ((pl.ng + 2) & ~1));
  __shared__ int s_fail;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gw = wid * gridDim.x + blockIdx.x, nw = gridDim.x * POOL_W;  // owners spread over the CTAs first
  PcgCta c = pool_cta(d, pl);
  if (threadIdx.x == 0) s_fail = 0;
  // ---- Galerkin start: a = A p_prev into d.w; partials b.p_prev (0), p_prev.a (1),
  // |b|^2 (3)
  int S = pool_prefix(d, pl, 0, phase, pre);
  int nl = pool_list(d, pl, pre, S, lst, pl.cap);
  for (int i = wid; i < nl; i += POOL_W) {
    const int s = lst[i].x, r = 32 * s + lane;
    const double4_32a gr = d.grad[r];
    const double4_32a b = make_double4_32a(-gr.x, -gr.y, -gr.z, 0.0);
    const bool fx = d.fixed[r] != 0;
    const double4_32a pv = fx ? make_double4_32a(0.0, 0.0, 0.0, 0.0) : d.p[r];
    const double4_32a av = fx ? make_double4_32a(0.0, 0.0, 0.0, 0.0) : spmv_row64(d, s, lane, d.p);
    d.w[r] = av;
    const double bp = warp_sum(dot4(b, pv)), pw = warp_sum(dot4(pv, av)), bb = warp_sum(dot4(b, b));
    if (lane == 0) {
      d.pslice[4 * (size_t)s + 0] = bp;
      d.pslice[4 * (size_t)s + 1] = pw;
      d.pslice[4 * (size_t)s + 3] = bb;
    }
  }
  if (!group_barrier(c, d, &s_fail)) return;  // also ends every SpMV on d.p before it is overwritten
  for (int j = gw; j < pl.ng; j += nw) {  // owner: CTA j mod grid, then warp
    const int g = pl.g0 + j;
    PoolGel& P = d.pool[g];
    if (d.gc[g].phase != phase) {
      if (lane == 0) P.act = P.run = P.inner = 0;
      continue;
    }
    double t[4];
    pool_total(d, g, 0, 2, t);
    pool_total(d, g, 3, 4, t);
    if (lane == 0) {
      P.act = P.run = 1;
      P.inner = 0;
      P.it = 0;
      P.bb = t[3];
      P.th = d.gv[g].eta2 * t[3];  // stop at |r|^2 <= eta^2 |b|^2 (the gel's forcing term)
      const double rho = t[0] / t[1];
      P.rho = (t[1] > 0.0 && isfinite(rho)) ? rho : 0.0;  // a non-finite p_prev anywhere gives 0
    }
  }
  if (!group_barrier(c, d, &s_fail)) return;
  // ---- x = rho p_prev, r = b - rho a, u = M^-1 r, pp = s = 0 (same share as above)
  for (int i = wid; i < nl; i += POOL_W) {
    const int s = lst[i].x, g = lst[i].y, r = 32 * s + lane;
    const double4_32a gr = d.grad[r];
    double4_32a b = make_double4_32a(-gr.x, -gr.y, -gr.z, 0.0);
    double4_32a x = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    const double rho = d.pool[g].rho;
    if (rho != 0.0 && !d.fixed[r]) {
      const double4_32a pv = d.p[r], av = d.w[r];
      x = make_double4_32a(rho * pv.x, rho * pv.y, rho * pv.z, 0.0);
      b.x = fma(-rho, av.x, b.x);
      b.y = fma(-rho, av.y, b.y);
      b.z = fma(-rho, av.z, b.z);
    }
    const double4_32a z = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    d.r[r] = b;
    d.p[r] = x;
    d.pp[r] = z;
    d.s[r] = z;
    d.u[r] = mul3(d.Minv + 9 * r, b);
  }
  if (!group_barrier(c, d, &s_fail)) return;  // u complete before the SpMV
  S = pool_prefix(d, pl, 1, phase, pre);
  nl = pool_list(d, pl, pre, S, lst, pl.cap);
  for (int k = 1;; ++k) {
    // ---- w = A u; partials gamma = (r, u), delta = (w, u), rr = (r, r)
    for (int i = wid; i < nl; i += POOL_W) {
      const int s = lst[i].x, r = 32 * s + lane;
      double4_32a w = spmv_row64(d, s, lane, d.u);
      if (d.fixed[r]) w = make_double4_32a(0.0, 0.0, 0.0, 0.0);
      d.w[r] = w;
      const double4_32a rv = d.r[r], uv = d.u[r];
      const double ga = warp_sum(dot4(rv, uv)), de = warp_sum(dot4(w, uv)), rr = warp_sum(dot4(rv, rv));
      if (lane == 0) {
        d.pslice[4 * (size_t)s + 0] = ga;
        d.pslice[4 * (size_t)s + 1] = de;
        d.pslice[4 * (size_t)s + 2] = rr;
      }
    }
    if (!group_barrier(c, d, &s_fail)) return;
    // ---- per-gel scalars and convergence, by the gel's owner warp
    for (int j = gw; j < pl.ng; j += nw) {  // owner: CTA j mod grid, then warp
      const int g = pl.g0 + j;
      PoolGel& P = d.pool[g];
      if (!P.run) continue;
      double t[4];
      pool_total(d, g, 0, 3, t);
      if (lane == 0) {
        const double ga = t[0], de = t[1], rr = t[2];
        if (!(rr > P.th) || k > maxit) {
          P.run = 0;
          d.gv[g].pcg_it = k - 1;
          d.gv[g].bb = P.bb;
          d.gv[g].res2 = P.bb > 0.0 ? rr / P.bb : 0.0;
          d.gv[g].pcg_done = 1;
        } else {
          const double beta = k == 1 ? 0.0 : ga / P.gprev;
          const double alpha = k == 1 ? ga / de : ga / (de - beta * ga / P.aprev);
          P.gprev = ga;
          P.aprev = alpha;
          P.al = alpha;
          P.be = beta;
        }
      }
    }
    if (!group_barrier(c, d, &s_fail)) return;
    S = pool_prefix(d, pl, 1, phase, pre);
    nl = pool_list(d, pl, pre, S, lst, pl.cap);
    if (S == 0) break;
    // ---- vector updates
    for (int i = wid; i < nl; i += POOL_W) {
      const int s = lst[i].x, g = lst[i].y, r = 32 * s + lane;
      const double beta = d.pool[g].be, alpha = d.pool[g].al;
      const double4_32a u = d.u[r], w = d.w[r];
      double4_32a pp = d.pp[r], sv = d.s[r], x = d.p[r], rv = d.r[r];
      pp.x = fma(beta, pp.x, u.x); pp.y = fma(beta, pp.y, u.y); pp.z = fma(beta, pp.z, u.z);
      sv.x = fma(beta, sv.x, w.x); sv.y = fma(beta, sv.y, w.y); sv.z = fma(beta, sv.z, w.z);
      x.x = fma(alpha, pp.x, x.x); x.y = fma(alpha, pp.y, x.y); x.z = fma(alpha, pp.z, x.z);
      rv.x = fma(-alpha, sv.x, rv.x); rv.y = fma(-alpha, sv.y, rv.y); rv.z = fma(-alpha, sv.z, rv.z);
      d.pp[r] = pp;
      d.s[r] = sv;
      d.p[r] = x;
      d.r[r] = rv;
      d.u[r] = mul3(d.Minv + 9 * r, rv);
    }
    if (!group_barrier(c, d, &s_fail)) return;
  }
  pool_epilogue(d, pl, c, phase, pre, lst, &s_fail);
}

// ---------------------------------------------------------------- mixed-precision PCG
// Mixed precision Newton direction: the Hessian is stored in FP32 (elastic blocks computed in
// FP32, barrier blocks rounded from FP64); the direction p solves H p = -g by iterative
// refinement: in every round the FP64 residual r = -g - H p (FP32 values, FP64 vectors and
// accumulation) is formed, then H d = r is solved by the same block-Jacobi CG in FP32 to the
// FP32 accuracy limit, and p += d in FP64.  Rounds stop once |r| <= eta |g| (FP64 residual).

// y = A32 u32 (FP32)
__device__ __forceinline__ float4 spmv_row32(const Dev& d, int s, int lane, const float4* u) {
  const int o = d.slice_off[s], w = (d.slice_off[s + 1] - o) >> 5;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll 4
  for (int k = 0; k < w; ++k) {
    const int bp = o + 32 * k + lane;
    const int c = __ldg(d.colidx + bp);
    const float4 uc = u[c];
    float v[9];
    load_block32(d.vals32 + (size_t)9 * (o + 32 * k), lane, v);
    a0 = fmaf(v[0], uc.x, a0);
    a1 = fmaf(v[3], uc.x, a1);
    a2 = fmaf(v[6], uc.x, a2);
    a0 = fmaf(v[1], uc.y, a0);
    a1 = fmaf(v[4], uc.y, a1);
    a2 = fmaf(v[7], uc.y, a2);
    a0 = fmaf(v[2], uc.z, a0);
    a1 = fmaf(v[5], uc.z, a1);
    a2 = fmaf(v[8], uc.z, a2);
  }
  return make_float4(a0, a1, a2, 0.f);
}

// y = A32 x64 with FP64 products and accumulation
__device__ __forceinline__ double4_32a spmv_row_res(const Dev& d, int s, int lane, const double4_32a* x) {
  const int o = d.slice_off[s], w = (d.slice_off[s + 1] - o) >> 5;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll 4
  for (int k = 0; k < w; ++k) {
    const int bp = o + 32 * k + lane;
    const int c = __ldg(d.colidx + bp);
    const double4_32a xc = x[c];
    float v[9];
    load_block32(d.vals32 + (size_t)9 * (o + 32 * k), lane, v);
    a0 = fma((double)v[0], xc.x, a0);
    a1 = fma((double)v[3], xc.x, a1);
    a2 = fma((double)v[6], xc.x, a2);
    a0 = fma((double)v[1], xc.y, a0);
    a1 = fma((double)v[4], xc.y, a1);
    a2 = fma((double)v[7], xc.y, a2);
    a0 = fma((double)v[2], xc.z, a0);
    a1 = fma((double)v[5], xc.z, a1);
    a2 = fma((double)v[8], xc.z, a2);
  }
  return make_double4_32a(a0, a1, a2, 0.0);
}

__global__ void __launch_bounds__(PCG_T, 3) k_pcg_mixed(Dev d, int phase, PcgPlan plan, int maxit,
                                                     int refine_max) {
  extern __shared__ double dsm[];
  __shared__ double tot[PCG_MAXG][4];
  __shared__ double bbj[PCG_MAXG], thj[PCG_MAXG], tolj[PCG_MAXG], rr0j[PCG_MAXG], gprev[PCG_MAXG], aprev[PCG_MAXG];
  __shared__ double rhoj[PCG_MAXG];
  __shared__ float alj[PCG_MAXG], bej[PCG_MAXG];
  __shared__ int gact[PCG_MAXG], run[PCG_MAXG], inner[PCG_MAXG], itj[PCG_MAXG];
  __shared__ int s_fail, s_any;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  PcgCta c = pcg_cta(d, plan);
  if (threadIdx.x == 0) s_fail = 0;
  for (int j = threadIdx.x; j < c.ng; j += PCG_T) {
    gact[j] = d.gc[c.g0 + j].phase == phase ? 1 : 0;
    run[j] = gact[j];
    itj[j] = 0;
  }
  __syncthreads();
  // ---- Galerkin start along the previous Newton direction (as in k_pcg64; a = A32 p_prev with
  // FP64 arithmetic, into d.w): partials b.p_prev (k = 0), p_prev.a (1), |b|^2 (3)
  for (int s = c.s0 + wid; s < c.s1; s += PCG_T / 32) {
    double bp = 0.0, pw = 0.0, bb = 0.0;
    if (gact[plan.slice_gel[s] - c.g0]) {
      const int r = 32 * s + lane;
      const double4_32a gr = d.grad[r];
      const double4_32a b = make_double4_32a(-gr.x, -gr.y, -gr.z, 0.0);
      const bool fx = d.fixed[r] != 0;
      const double4_32a pv = fx ? make_double4_32a(0.0, 0.0, 0.0, 0.0) : d.p[r];
      const double4_32a a = fx ? make_double4_32a(0.0, 0.0, 0.0, 0.0) : spmv_row_res(d, s, lane, d.p);
      d.w[r] = a;
      bp = dot4(b, pv);
      pw = dot4(pv, a);
      bb = dot4(b, b);
    }
    bp = warp_sum(bp);
    pw = warp_sum(pw);
    bb = warp_sum(bb);
    if (lane == 0) {
      dsm[(s - c.s0) * 4 + 0] = bp;
      dsm[(s - c.s0) * 4 + 1] = pw;
      dsm[(s - c.s0) * 4 + 2] = 0.0;
      dsm[(s - c.s0) * 4 + 3] = bb;
    }
  }
  if (!group_sum(d, c, dsm, 0, 4, tot, &s_fail)) return;  // its barrier ends every SpMV on d.p
  for (int j = threadIdx.x; j < c.ng; j += PCG_T) {
    bbj[j] = tot[j][3];
    thj[j] = d.gv[c.g0 + j].eta2 * bbj[j];  // stop at |r|^2 <= eta^2 |b|^2 (the gel's forcing term)
    const double pw = tot[j][1], rho = tot[j][0] / pw;
    rhoj[j] = (pw > 0.0 && isfinite(rho)) ? rho : 0.0;
  }
  __syncthreads();
  // ---- p = rho p_prev, r64 = b - rho a; partial |r|^2 (k = 2)
  for (int s = c.s0 + wid; s < c.s1; s += PCG_T / 32) {
    double rr = 0.0;
    const int j = plan.slice_gel[s] - c.g0;
    if (gact[j]) {
      const int r = 32 * s + lane;
      const double4_32a gr = d.grad[r];
      double4_32a b = make_double4_32a(-gr.x, -gr.y, -gr.z, 0.0);
      double4_32a x = make_double4_32a(0.0, 0.0, 0.0, 0.0);
      const double rho = rhoj[j];
      if (rho != 0.0 && !d.fixed[r]) {
        const double4_32a pv = d.p[r], a = d.w[r];
        x = make_double4_32a(rho * pv.x, rho * pv.y, rho * pv.z, 0.0);
        b.x = fma(-rho, a.x, b.x);
        b.y = fma(-rho, a.y, b.y);
        b.z = fma(-rho, a.z, b.z);
      }
      d.r[r] = b;
      d.p[r] = x;
      rr = dot4(b, b);
    }
    rr = warp_sum(rr);
    if (lane == 0) dsm[(s - c.s0) * 4 + 2] = rr;
  }
  if (!group_sum(d, c, dsm, 2, 3, tot, &s_fail)) return;
  for (int round = 0;; ++round) {
    // ---- round start: outer convergence on the FP64 residual; inner init r32 = r64, x32 = 0
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < c.ng; j += PCG_T) {
      inner[j] = 0;
      if (!run[j]) continue;
      const double rr = tot[j][2], bb = bbj[j];
      if (!(rr > thj[j]) || round >= refine_max) {
        run[j] = 0;
        if (blockIdx.x == c.c0) {
          d.gv[c.g0 + j].res2 = bb > 0.0 ? rr / bb : 0.0;
          d.gv[c.g0 + j].pcg_done = 1;
          d.gv[c.g0 + j].rounds = round;
          d.gv[c.g0 + j].bb = bb;
          d.gv[c.g0 + j].pcg_it = itj[j];
        }
        continue;
      }
      s_any = 1;
      inner[j] = 1;
      // inner target: reach eta |b| in one round if FP32 allows, else the FP32 floor
      tolj[j] = fmax(thj[j] / rr, 1e-11);
    }
    __syncthreads();
    if (!s_any) break;
    for (int s = c.s0 + wid; s < c.s1; s += PCG_T / 32) {
      if (!inner[plan.slice_gel[s] - c.g0]) continue;
      const int r = 32 * s + lane;
      const double4_32a rv = d.r[r];
      const float4 r32 = make_float4((float)rv.x, (float)rv.y, (float)rv.z, 0.f);
      d.r32[r] = r32;
      d.x32[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      d.pp32[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      d.s32[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      d.u32[r] = mul3f(d.Minv32 + 9 * r, r32);
    }
    if (!group_barrier(c, d, &s_fail)) return;
    // ---- inner FP32 CG (Chronopoulos-Gear), same structure as the FP64 kernel
    for (int k = 1;; ++k) {
      for (int s = c.s0 + wid; s < c.s1; s += PCG_T / 32) {
        double ga = 0.0, de = 0.0, rr = 0.0;
        if (inner[plan.slice_gel[s] - c.g0]) {
          const int r = 32 * s + lane;
          float4 w = spmv_row32(d, s, lane, d.u32);
          if (d.fixed[r]) w = make_float4(0.f, 0.f, 0.f, 0.f);
          d.w32[r] = w;
          const float4 rv = d.r32[r], uv = d.u32[r];
          // FP32 warp sums: the inner solve's dot products are FP32 quantities (GB300 runs FP64
          // adds at 1/64 of the FP32 rate); slices and CTAs are then added in FP64
          ga = warp_sum(dot4f(rv, uv));
          de = warp_sum(dot4f(w, uv));
          rr = warp_sum(dot4f(rv, rv));
        }
        if (lane == 0) {
          dsm[(s - c.s0) * 4 + 0] = ga;
          dsm[(s - c.s0) * 4 + 1] = de;
          dsm[(s - c.s0) * 4 + 2] = rr;
        }
      }
      if (!group_sum<float>(d, c, dsm, 0, 3, tot, &s_fail)) return;
      if (threadIdx.x == 0) s_any = 0;
      __syncthreads();
      for (int j = threadIdx.x; j < c.ng; j += PCG_T) {
        if (!inner[j]) continue;
        const double ga = tot[j][0], de = tot[j][1], rr = tot[j][2];
        // converged once |r32|^2 <= tol |r32 at the round start|^2 (FP32 accuracy floor 1e-11)
        if (k == 1) rr0j[j] = rr;
        if (!(rr > tolj[j] * rr0j[j]) || k > maxit) {
          inner[j] = 0;
          itj[j] += k - 1;
          continue;
        }
        s_any = 1;
        const double beta = k == 1 ? 0.0 : ga / gprev[j];
        const double alpha = k == 1 ? ga / de : ga / (de - beta * ga / aprev[j]);
        gprev[j] = ga;
        aprev[j] = alpha;
        alj[j] = (float)alpha;
        bej[j] = (float)beta;
      }
      __syncthreads();
      if (!s_any) break;
      for (int s = c.s0 + wid; s < c.s1; s += PCG_T / 32) {
        const int j = plan.slice_gel[s] - c.g0;
        if (!inner[j]) continue;
        const float fb = bej[j], fa = alj[j];
        const int r = 32 * s + lane;
        const float4 u = d.u32[r], w = d.w32[r];
        float4 pp = d.pp32[r], sv = d.s32[r], x = d.x32[r], rv = d.r32[r];
        pp.x = fmaf(fb, pp.x, u.x); pp.y = fmaf(fb, pp.y, u.y); pp.z = fmaf(fb, pp.z, u.z);
        sv.x = fmaf(fb, sv.x, w.x); sv.y = fmaf(fb, sv.y, w.y); sv.z = fmaf(fb, sv.z, w.z);
        x.x = fmaf(fa, pp.x, x.x); x.y = fmaf(fa, pp.y, x.y); x.z = fmaf(fa, pp.z, x.z);
        rv.x = fmaf(-fa, sv.x, rv.x); rv.y = fmaf(-fa, sv.y, rv.y); rv.z = fmaf(-fa, sv.z, rv.z);
        d.pp32[r] = pp;
        d.s32[r] = sv;
        d.x32[r] = x;
        d.r32[r] = rv;
        d.u32[r] = mul3f(d.Minv32 + 9 * r, rv);
      }
      if (!group_barrier(c, d, &s_fail)) return;
    }
    // ---- p += x32 (FP64), then the FP64 residual r64 = b - A p
    for (int s = c.s0 + wid; s < c.s1; s += PCG_T / 32) {
      if (!run[plan.slice_gel[s] - c.g0]) continue;
      const int r = 32 * s + lane;
      const float4 x = d.x32[r];
      double4_32a p = d.p[r];
      p.x += (double)x.x;
      p.y += (double)x.y;
      p.z += (double)x.z;
      d.p[r] = p;
    }
    if (!group_barrier(c, d, &s_fail)) return;
    for (int s = c.s0 + wid; s < c.s1; s += PCG_T / 32) {
      double rr = 0.0;
      if (run[plan.slice_gel[s] - c.g0]) {
        const int r = 32 * s + lane;
        double4_32a ap = spmv_row_res(d, s, lane, d.p);
        const double4_32a gr = d.grad[r];
        double4_32a rv = make_double4_32a(-gr.x - ap.x, -gr.y - ap.y, -gr.z - ap.z, 0.0);
        if (d.fixed[r]) rv = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        d.r[r] = rv;
        rr = dot4(rv, rv);
      }
      rr = warp_sum(rr);
      if (lane == 0) dsm[(s - c.s0) * 4 + 2] = rr;
    }
    if (!group_sum(d, c, dsm, 2, 3, tot, &s_fail)) return;
  }
  pcg_epilogue(d, plan, c, dsm, tot, gact, &s_fail);
}

cudaError_t launch_pcg_mixed(const Dev& d, int phase, const PcgPlan& plan, int nctas, int maxit, int refine_max,
                             cudaStream_t st) {
  Dev dd = d;
  PcgPlan pp = plan;
  void* args[] = {(void*)&dd, (void*)&phase, (void*)&pp, (void*)&maxit, (void*)&refine_max};
  count_launch(1);
  const size_t smem = (size_t)plan.max_slices * 4 * sizeof(double);
  return cudaLaunchCooperativeKernel((const void*)k_pcg_mixed, dim3(nctas), dim3(PCG_T), args, smem, st);
}

// co-resident CTAs per SM of the persistent solvers (both must fit a cooperative launch)
int pcg_max_ctas_per_sm(int max_slices) {
  int a = 0, b = 0;
  const size_t smem = (size_t)max_slices * 4 * sizeof(double);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pcg64, PCG_T, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pcg_mixed, PCG_T, smem);
  return a < b ? a : b;
}

// the owner's decision at the start of a refinement round from the gel's FP64 residual rr: the
// solve ends (rounds done = round) or the round's FP32 inner solve starts with its target
__device__ __forceinline__ void pool_round_start(const Dev& d, int g, double rr, int round, int refine_max) {
  PoolGel& P = d.pool[g];
  P.rr = rr;
  if (!(rr > P.th) || round >= refine_max) {
    P.run = 0;
    P.inner = 0;
    d.gv[g].res2 = P.bb > 0.0 ? rr / P.bb : 0.0;
    d.gv[g].pcg_done = 1;
    d.gv[g].rounds = round;
    d.gv[g].bb = P.bb;
    d.gv[g].pcg_it = P.it;
  } else {
    P.inner = 1;
    P.tol = fmax(P.th / rr, 1e-11);  // reach eta |b| in one round if FP32 allows, else the FP32 floor
  }
}

// mixed-precision pooled PCG: FP64 residual refinement rounds around an FP32 inner CG (above)
__global__ void __launch_bounds__(POOL_T, 1) k_pcg_mixed_pool(Dev d, int phase, PoolPlan pl, int maxit,
                                                         int refine_max) {
  extern __shared__ int pre[];  // ng + 1, then the CTA's slice list
  int2* lst = reinterpret_cast<int2*>(pre + ((pl.ng + 2) & ~1));
  __shared__ int s_fail;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gw = wid * gridDim.x + blockIdx.x, nw = gridDim.x * POOL_W;  // owners spread over the CTAs first
  PcgCta c = pool_cta(d, pl);
  if (threadIdx.x == 0) s_fail = 0;
  // ---- Galerkin start (FP64 arithmetic on the FP32 matrix): a = A32 p_prev into d.w
  int S = pool_prefix(d, pl, 0, phase, pre);
  int nl = pool_list(d, pl, pre, S, lst, pl.cap);
  for (int i = wid; i < nl; i += POOL_W) {
    const int s = lst[i].x, r = 32 * s + lane;
    const double4_32a gr = d.grad[r];
    const double4_32a b = make_double4_32a(-gr.x, -gr.y, -gr.z, 0.0);
    const bool fx = d.fixed[r] != 0;
    const double4_32a pv = fx ? make_double4_32a(0.0, 0.0, 0.0, 0.0) : d.p[r];
    const double4_32a av = fx ? make_double4_32a(0.0, 0.0, 0.0, 0.0) : spmv_row_res(d, s, lane, d.p);
    d.w[r] = av;
    const double bp = warp_sum(dot4(b, pv)), pw = warp_sum(dot4(pv, av)), bb = warp_sum(dot4(b, b));
    if (lane == 0) {
      d.pslice[4 * (size_t)s + 0] = bp;
      d.pslice[4 * (size_t)s + 1] = pw;
      d.pslice[4 * (size_t)s + 3] = bb;
    }
  }
  if (!group_barrier(c, d, &s_fail)) return;
  for (int j = gw; j < pl.ng; j += nw) {  // owner: CTA j mod grid, then warp
    const int g = pl.g0 + j;
    PoolGel& P = d.pool[g];
    if (d.gc[g].phase != phase) {
      if (lane == 0) P.act = P.run = P.inner = 0;
      continue;
    }
    double t[4];
    pool_total(d, g, 0, 2, t);
    pool_total(d, g, 3, 4, t);
    if (lane == 0) {
      P.act = P.run = 1;
      P.inner = 0;
      P.it = 0;
      P.bb = t[3];
      P.th = d.gv[g].eta2 * t[3];  // stop at |r|^2 <= eta^2 |b|^2 (the gel's forcing term)
      const double rho = t[0] / t[1];
      P.rho = (t[1] > 0.0 && isfinite(rho)) ? rho : 0.0;
    }
  }
  if (!group_barrier(c, d, &s_fail)) return;
  // ---- p = rho p_prev, r64 = b - rho a; partial |r|^2 (2)
  for (int i = wid; i < nl; i += POOL_W) {
    const int s = lst[i].x, g = lst[i].y, r = 32 * s + lane;
    const double4_32a gr = d.grad[r];
    double4_32a b = make_double4_32a(-gr.x, -gr.y, -gr.z, 0.0);
    double4_32a x = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    const double rho = d.pool[g].rho;
    if (rho != 0.0 && !d.fixed[r]) {
      const double4_32a pv = d.p[r], av = d.w[r];
      x = make_double4_32a(rho * pv.x, rho * pv.y, rho * pv.z, 0.0);
      b.x = fma(-rho, av.x, b.x);
      b.y = fma(-rho, av.y, b.y);
      b.z = fma(-rho, av.z, b.z);
    }
    d.r[r] = b;
    d.p[r] = x;
    const double rr = warp_sum(dot4(b, b));
    if (lane == 0) d.pslice[4 * (size_t)s + 2] = rr;
  }
  if (!group_barrier(c, d, &s_fail)) return;
  for (int j = gw; j < pl.ng; j += nw) {  // owner: CTA j mod grid, then warp
    const int g = pl.g0 + j;
    if (!d.pool[g].run) continue;
    double t[4];
    pool_total(d, g, 2, 3, t);
    if (lane == 0) pool_round_start(d, g, t[2], 0, refine_max);
  }
  if (!group_barrier(c, d, &s_fail)) return;
  for (int round = 0;; ++round) {
    S = pool_prefix(d, pl, 2, phase, pre);
    nl = pool_list(d, pl, pre, S, lst, pl.cap);
    if (S == 0) break;  // no gel starts a round: every solve has ended
    // ---- inner init: r32 = r64, x32 = pp32 = s32 = 0, u32 = M^-1 r32
    for (int i = wid; i < nl; i += POOL_W) {
      const int s = lst[i].x, r = 32 * s + lane;
      const double4_32a rv = d.r[r];
      const float4 r32 = make_float4((float)rv.x, (float)rv.y, (float)rv.z, 0.f);
      d.r32[r] = r32;
      d.x32[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      d.pp32[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      d.s32[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      d.u32[r] = mul3f(d.Minv32 + 9 * r, r32);
    }
    if (!group_barrier(c, d, &s_fail)) return;
    // ---- inner FP32 CG (Chronopoulos-Gear)
    for (int k = 1;; ++k) {
      for (int i = wid; i < nl; i += POOL_W) {
        const int s = lst[i].x, r = 32 * s + lane;
        float4 w = spmv_row32(d, s, lane, d.u32);
        if (d.fixed[r]) w = make_float4(0.f, 0.f, 0.f, 0.f);
        d.w32[r] = w;
        const float4 rv = d.r32[r], uv = d.u32[r];
        // FP32 warp sums (FP32 quantities of the inner solve); the owner adds the slices in FP64
        const float ga = warp_sum(dot4f(rv, uv)), de = warp_sum(dot4f(w, uv)), rr = warp_sum(dot4f(rv, rv));
        if (lane == 0) {
          d.pslice[4 * (size_t)s + 0] = ga;
          d.pslice[4 * (size_t)s + 1] = de;
          d.pslice[4 * (size_t)s + 2] = rr;
        }
      }
      if (!group_barrier(c, d, &s_fail)) return;
      for (int j = gw; j < pl.ng; j += nw) {  // owner: CTA j mod grid, then warp
        const int g = pl.g0 + j;
        PoolGel& P = d.pool[g];
        if (!P.inner) continue;
        double t[4];
        pool_total(d, g, 0, 3, t);
        if (lane == 0) {
          const double ga = t[0], de = t[1], rr = t[2];
          // converged once |r32|^2 <= tol |r32 at the round start|^2 (FP32 accuracy floor 1e-11)
          if (k == 1) P.rr0 = rr;
          if (!(rr > P.tol * P.rr0) || k > maxit) {
            P.inner = 0;
            P.it += k - 1;
          } else {
            const double beta = k == 1 ? 0.0 : ga / P.gprev;
            const double alpha = k == 1 ? ga / de : ga / (de - beta * ga / P.aprev);
            P.gprev = ga;
            P.aprev = alpha;
            P.al = alpha;
            P.be = beta;
          }
        }
      }
      if (!group_barrier(c, d, &s_fail)) return;
      S = pool_prefix(d, pl, 2, phase, pre);
      nl = pool_list(d, pl, pre, S, lst, pl.cap);
      if (S == 0) break;
      for (int i = wid; i < nl; i += POOL_W) {
        const int s = lst[i].x, g = lst[i].y, r = 32 * s + lane;
        const float fb = (float)d.pool[g].be, fa = (float)d.pool[g].al;
        const float4 u = d.u32[r], w = d.w32[r];
        float4 pp = d.pp32[r], sv = d.s32[r], x = d.x32[r], rv = d.r32[r];
        pp.x = fmaf(fb, pp.x, u.x); pp.y = fmaf(fb, pp.y, u.y); pp.z = fmaf(fb, pp.z, u.z);
        sv.x = fmaf(fb, sv.x, w.x); sv.y = fmaf(fb, sv.y, w.y); sv.z = fmaf(fb, sv.z, w.z);
        x.x = fmaf(fa, pp.x, x.x); x.y = fmaf(fa, pp.y, x.y); x.z = fmaf(fa, pp.z, x.z);
        rv.x = fmaf(-fa, sv.x, rv.x); rv.y = fmaf(-fa, sv.y, rv.y); rv.z = fmaf(-fa, sv.z, rv.z);
        d.pp32[r] = pp;
        d.s32[r] = sv;
        d.x32[r] = x;
        d.r32[r] = rv;
        d.u32[r] = mul3f(d.Minv32 + 9 * r, rv);
      }
      if (!group_barrier(c, d, &s_fail)) return;
    }
    // ---- p += x32 (FP64) for the gels still in their rounds
    S = pool_prefix(d, pl, 1, phase, pre);
    nl = pool_list(d, pl, pre, S, lst, pl.cap);
    for (int i = wid; i < nl; i += POOL_W) {
      const int s = lst[i].x, r = 32 * s + lane;
      const float4 x = d.x32[r];
      double4_32a p = d.p[r];
      p.x += (double)x.x;
      p.y += (double)x.y;
      p.z += (double)x.z;
      d.p[r] = p;
    }
    if (!group_barrier(c, d, &s_fail)) return;
    // ---- the FP64 residual r64 = b - A p; partial |r|^2 (2)
    for (int i = wid; i < nl; i += POOL_W) {
      const int s = lst[i].x, r = 32 * s + lane;
      const double4_32a ap = spmv_row_res(d, s, lane, d.p);
      const double4_32a gr = d.grad[r];
      double4_32a rv = make_double4_32a(-gr.x - ap.x, -gr.y - ap.y, -gr.z - ap.z, 0.0);
      if (d.fixed[r]) rv = make_double4_32a(0.0, 0.0, 0.0, 0.0);
      d.r[r] = rv;
      const double rr = warp_sum(dot4(rv, rv));
      if (lane == 0) d.pslice[4 * (size_t)s + 2] = rr;
    }
    if (!group_barrier(c, d, &s_fail)) return;
    for (int j = gw; j < pl.ng; j += nw) {  // owner: CTA j mod grid, then warp
      const int g = pl.g0 + j;
      if (!d.pool[g].run) continue;
      double t[4];
      pool_total(d, g, 2, 3, t);
      if (lane == 0) pool_round_start(d, g, t[2], round + 1, refine_max);
    }
    if (!group_barrier(c, d, &s_fail)) return;
  }
  pool_epilogue(d, pl, c, phase, pre, lst, &s_fail);
}

// dynamic shared memory of the pooled kernels: the gel prefix (ng + 1 ints, padded to 8 bytes),
// then the CTA's slice list (cap entries)
size_t pcg_pool_smem(const PoolPlan& pl) {
  return sizeof(int) * (size_t)((pl.ng + 2) & ~1) + sizeof(int2) * (size_t)pl.cap;
}

cudaError_t launch_pcg_pool(const Dev& d, int phase, const PoolPlan& pl, int nctas, bool mixed, int maxit,
                            int refine_max, cudaStream_t st) {
  Dev dd = d;
  PoolPlan pp = pl;
  const size_t smem = pcg_pool_smem(pl);
  count_launch(1);
  if (mixed) {
    void* args[] = {(void*)&dd, (void*)&phase, (void*)&pp, (void*)&maxit, (void*)&refine_max};
    return cudaLaunchCooperativeKernel((const void*)k_pcg_mixed_pool, dim3(nctas), dim3(POOL_T), args, smem, st);
  }
  void* args[] = {(void*)&dd, (void*)&phase, (void*)&pp, (void*)&maxit};
  return cudaLaunchCooperativeKernel((const void*)k_pcg64_pool, dim3(nctas), dim3(POOL_T), args, smem, st);
}

// co-resident CTAs per SM of the pooled solvers for the plan (both must fit a cooperative launch)
int pcg_pool_ctas_per_sm(const PoolPlan& pl) {
  int a = 0, b = 0;
  const size_t smem = pcg_pool_smem(pl);
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute((const void*)k_pcg64_pool, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute((const void*)k_pcg_mixed_pool, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pcg64_pool, POOL_T, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pcg_mixed_pool, POOL_T, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return a < b ? a : b;
}

// ---------------------------------------------------------------- per-row / per-gel steps
// rest position X carried by the pose (R, t)
__device__ __forceinline__ double4_32a carry(const double* R, const double* t, const double4_32a X) {
  return make_double4_32a(fma(R[2], X.z, fma(R[1], X.y, R[0] * X.x)) + t[0],
                          fma(R[5], X.z, fma(R[4], X.y, R[3] * X.x)) + t[1],
                          fma(R[8], X.z, fma(R[7], X.y, R[6] * X.x)) + t[2], 0.0);
}

// attachment-driven (sub)step: the attached (Dirichlet) vertices of the gel move to their rest
// positions carried by the case pose at the end of the (sub)step (TacEx, Sec. "General GIPC
// Simulation Pipeline": the attachment targets are set from the sensor-case pose, then the solver
// runs); done before the indenter placement check, which sees the moved gel
__global__ void k_place_attached(Dev d, int phase) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.nrows) return;
  const int g = d.vgel[r];
  const GelCtl& c = d.gc[g];
  if (c.phase != phase || !c.attached || !d.fixed[r] || r - d.gi[g].v0 >= d.gi[g].nv) return;
  d.x[r] = carry(c.Rc, c.tc, d.X[r]);
}

// step begin: x_n = x, xt = x + h v + h^2 g on free rows (xt = x on fixed rows; an attached vertex
// moved by its case has x_n = its position at the case pose of the step's start)
__global__ void k_predictor(Dev d, int phase) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.nrows) return;
  const int g = d.vgel[r];
  if (d.gc[g].phase != phase) return;
  const GelCtl& c = d.gc[g];
  const double4_32a x = d.x[r], v = d.v[r];
  const bool moved = c.attached && d.fixed[r] && r - d.gi[g].v0 < d.gi[g].nv;
  d.xn[r] = moved ? carry(c.Rcp, c.tcp, d.X[r]) : x;
  double4_32a xt = x;
  if (!d.fixed[r]) {
    const double h = c.h;
    xt.x = x.x + h * v.x + h * h * c.grav[0];
    xt.y = x.y + h * v.y + h * h * c.grav[1];
    xt.z = x.z + h * v.z + h * h * c.grav[2];
  }
  d.xt[r] = xt;
}

// x += alpha p for gels whose line search accepted
__global__ void k_update(Dev d, int phase) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.nrows) return;
  const int g = d.vgel[r];
  if (d.gc[g].phase != phase || d.gv[g].ls_state != 1) return;
  const double a = d.gv[g].alpha;
  double4_32a x = d.x[r];
  const double4_32a p = d.p[r];
  x.x += a * p.x;
  x.y += a * p.y;
  x.z += a * p.z;
  d.x[r] = x;
}

// v = (x - x_n) / h
__global__ void k_finalize(Dev d, int phase) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.nrows) return;
  const int g = d.vgel[r];
  if (d.gc[g].phase != phase) return;
  const double ih = 1.0 / d.gc[g].h;
  const double4_32a x = d.x[r], xn = d.xn[r];
  d.v[r] = make_double4_32a((x.x - xn.x) * ih, (x.y - xn.y) * ih, (x.z - xn.z) * ih, 0.0);
}

// restore x_n (failed step)
__global__ void k_restore(Dev d, int phase) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.nrows) return;
  const int g = d.vgel[r];
  if (d.gc[g].phase != phase) return;
  d.x[r] = d.xn[r];
}

constexpr double NEAR_FACTOR = 2.0;

// per gel bookkeeping: op 0 = reset the assembly / PCG accumulators; 1 = after the PCG:
// converged = ||p||_inf < tol on a direction solved to the near forcing term, next forcing term,
// prepare the ACCD minimum; 2 = after the ACCD: alpha0 = min(1, toi), start the line search;
// 3 = reset the per-step feasibility state and start with the far forcing term.
//
// Forcing terms (inexact Newton): the projected Newton iteration converges linearly (the PSD
// projection drops curvature), so solving the linear system much more accurately than the
// contraction of the Newton steps buys nothing while ||p|| is large.  The next solve runs to
// eta_near when the next ||p||_inf, predicted from the last one and the last contraction
// ratio, falls below NEAR_FACTOR tol (the direction that may end the solve), to eta_far
// otherwise.  Convergence is only declared on a direction whose solve reached eta_near (a zero
// right-hand side counts), so the stopping test sees the same direction quality as with a
// fixed eta_near; a far solve that lands below tol costs one more iteration.
__global__ void k_gel_op(Dev d, int phase, int op) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= d.n_gels) return;
  if (d.gc[g].phase != phase) return;
  GelVar& v = d.gv[g];
  if (op == 0) {
    v.fc[0] = v.fc[1] = v.fc[2] = 0.0;
    v.active_pairs = 0;
    v.pnorm_bits = 0ull;
    v.pcg_done = 0;
    v.pcg_it = 0;
    v.inner_done = 0;
    v.rounds = 0;
    v.flags &= ~(4 | 16);
  } else if (op == 1) {
    const GelCtl& c = d.gc[g];
    const double pn = bitsd(v.pnorm_bits);
    const bool near = v.eta2 <= c.eta2_near || v.res2 <= c.eta2_near;  // solved to eta_near (or capped there)
    v.converged = (pn < c.tol_p && near) ? 1 : 0;
    const double rho = v.pn_prev > 0.0 ? fmin(pn / v.pn_prev, 1.0) : 1.0;
    v.eta2 = pn * rho < NEAR_FACTOR * c.tol_p ? c.eta2_near : c.eta2_far;
    v.pn_prev = pn;
    v.toi_bits = dbits(1.0);
    v.flags &= ~8;
  } else if (op == 2) {
    if (v.converged) {
      v.ls_state = 3;
    } else if (v.flags & 32) {
      v.ls_state = 4;  // candidate segment overflowed: the host grows it and redoes this part
    } else {
      v.alpha0 = fmin(1.0, bitsd(v.toi_bits));
      v.alpha = v.alpha0;
      v.ls_state = 0;
    }
  } else if (op == 3) {
    v.eta2 = d.gc[g].eta2_far;
    v.pn_prev = 0.0;
    v.toi_bits = dbits(1.0);
    v.dmin_bits = dbits(CUDART_INF);
    v.flags = 0;
    v.ls_total = 0;
    v.ss_cut = 0;
    v.active_pairs = 0;
  } else if (op == 4) {  // the final state's distance minimum and active-pair count follow
    v.dmin_bits = dbits(CUDART_INF);
    v.active_pairs = 0;
  } else if (op == 5) {
    if (v.ls_state == 1) v.ls_state = 3;  // the accepted step has been applied
  } else if (op == 6) {
    v.flags &= ~32;
    v.toi_bits = dbits(1.0);
  }
}

void launch_rows(int which, const Dev& d, int phase, cudaStream_t st) {
  const int nb = nblk(d.nrows, 256);
  if (which == 0) {
    k_predictor<<<nb, 256, 0, st>>>(d, phase);
    count_launch(1);
  }
  if (which == 1) {
    k_update<<<nb, 256, 0, st>>>(d, phase);
    count_launch(1);
  }
  if (which == 2) {
    k_finalize<<<nb, 256, 0, st>>>(d, phase);
    count_launch(1);
  }
  if (which == 3) {
    k_restore<<<nb, 256, 0, st>>>(d, phase);
    count_launch(1);
  }
  if (which == 4) {
    k_place_attached<<<nb, 256, 0, st>>>(d, phase);
    count_launch(1);
  }
}
void launch_gel_op(const Dev& d, int phase, int op, cudaStream_t st) {
  k_gel_op<<<nblk(d.n_gels, 128), 128, 0, st>>>(d, phase, op);
  count_launch(1);
}

}  // namespace txg

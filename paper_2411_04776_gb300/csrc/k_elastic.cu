// Elastic kernels: per-tet assembly into the scratch and the unit-level evaluation entry.
#include "dev_elastic.cuh"

namespace txg {

// ---------------------------------------------------------------- kernels on the batch
// Assembly: per tet gradient + projected Hessian into the per-tet scratch.
template <bool MIXED>
__global__ void __launch_bounds__(128) k_tet_assemble(Dev d, int phase) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.ntets) return;
  const int g = d.tgel[t];
  if (d.gc[g].phase != phase) return;
  const GelInfo& G = d.gi[g];
  const int4 tv = d.tets[t];
  const int ids[4] = {tv.x, tv.y, tv.z, tv.w};
  double xs[4][3], Xs[4][3], D[4][3];
  for (int a = 0; a < 4; ++a) {
    ld3(d.x[ids[a]], xs[a]);
    ld3(d.X[ids[a]], Xs[a]);
  }
  tet_D(d.Dminv + 9 * t, D);
  double F[3][3], Hd[3][3];
  tet_F(xs, Xs, D, F, Hd);
  double gr[12], J, lnJ;
  double* out = d.tscr + (size_t)t * TS;
  if (!nh_grad(F, Hd, G.mu, G.lam, d.vol[t], D, gr, nullptr, &J, &lnJ)) {
    // inverted element (cannot happen after a successful line search): flag and zero it
    atomicOr(&d.gv[g].flags, 4);
    for (int k = 0; k < TS; ++k) out[k] = 0.0;
    return;
  }
  for (int k = 0; k < 12; ++k) out[GOFF + k] = gr[k];
  if (MIXED)
    nh_blocks<float, float, BLK32>(F, J, lnJ, G.mu, G.lam, d.vol[t], D, true, d.tscr32 + (size_t)t * TS32);
  else
    nh_blocks<double, double, BLK64>(F, J, lnJ, G.mu, G.lam, d.vol[t], D, true, out);
}

void launch_tet_assemble(const Dev& d, int phase, bool mixed, cudaStream_t st) {
  if (d.ntets == 0) return;
  const int nb = (d.ntets + 127) / 128;
  if (mixed)
    k_tet_assemble<true><<<nb, 128, 0, st>>>(d, phase);
  else
    k_tet_assemble<false><<<nb, 128, 0, st>>>(d, phase);
  count_launch(1);
}

// ---------------------------------------------------------------- unit-level entry
__global__ void k_eval_tets(int n, const double* X, const double* x, double mu, double lam,
                            int project, double* e, double* g, double* H) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double Xs[4][3], xs[4][3];
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 3; ++c) {
      Xs[a][c] = X[12 * t + 3 * a + c];
      xs[a][c] = x[12 * t + 3 * a + c];
    }
  // rest data
  double Dm[3][3], Dmi[9];
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 3; ++a) Dm[i][a] = Xs[a + 1][i] - Xs[0][i];
  double det = det3(Dm);
  double vol = det / 6.0;
  {
    const double id = 1.0 / det;
    Dmi[0] = (Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1]) * id;
    Dmi[1] = (Dm[0][2] * Dm[2][1] - Dm[0][1] * Dm[2][2]) * id;
    Dmi[2] = (Dm[0][1] * Dm[1][2] - Dm[0][2] * Dm[1][1]) * id;
    Dmi[3] = (Dm[1][2] * Dm[2][0] - Dm[1][0] * Dm[2][2]) * id;
    Dmi[4] = (Dm[0][0] * Dm[2][2] - Dm[0][2] * Dm[2][0]) * id;
    Dmi[5] = (Dm[0][2] * Dm[1][0] - Dm[0][0] * Dm[1][2]) * id;
    Dmi[6] = (Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0]) * id;
    Dmi[7] = (Dm[0][1] * Dm[2][0] - Dm[0][0] * Dm[2][1]) * id;
    Dmi[8] = (Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0]) * id;
  }
  double D[4][3], F[3][3], Hd[3][3];
  tet_D(Dmi, D);
  tet_F(xs, Xs, D, F, Hd);
  double gr[12], en, J, lnJ;
  if (!nh_grad(F, Hd, mu, lam, vol, D, gr, &en, &J, &lnJ)) {
    e[t] = CUDART_INF;
    return;
  }
  e[t] = en;
  if (g)
    for (int k = 0; k < 12; ++k) g[12 * t + k] = gr[k];
  if (H) {
    double blk[90];
    nh_blocks<double, double>(F, J, lnJ, mu, lam, vol, D, project != 0, blk);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        for (int i = 0; i < 3; ++i)
          for (int l = 0; l < 3; ++l) {
            double v = a <= b ? blk[ublk(a, b) * 9 + 3 * i + l] : blk[ublk(b, a) * 9 + 3 * l + i];
            H[144 * t + (3 * a + i) * 12 + 3 * b + l] = v;
          }
  }
}

void launch_eval_tets(int n, const double* X, const double* x, double mu, double lam, int project,
                      double* e, double* g, double* H, cudaStream_t st) {
  if (n <= 0) return;
  k_eval_tets<<<(n + 127) / 128, 128, 0, st>>>(n, X, x, mu, lam, project, e, g, H);
  count_launch(1);
}

}  // namespace txg

// Host side of the gelpad IPC step library: rest-state preprocessing, device layout, the
// per-gel Newton state machine (continuous batching at Newton-iteration granularity) and the C ABI.
//
// One time step of a gel (TacEx, Sec. "General GIPC Simulation Pipeline"): the indenter is moved
// to the requested pose (kinematic target), then the free gel vertices are found by minimising the
// incremental potential with projected Newton.  Per gel and step:
//   begin   : indenter placed at the target pose; spatial hash of its primitives swept from the
//             previous pose; candidates against the gel at x_n; ACCD sweep of the indenter motion
//             and distances after placement.  Any hit (or distance <= 0) splits the step into two
//             half steps (midpoint pose, dt/2), recursively, up to max_split_depth; otherwise
//             x_n = x, xt = x_n + h v_n (+ h^2 g), E(x_n) and the static hash at the target pose.
//   newton  : assemble (elastic scratch + gather + barrier + inertia), block-Jacobi PCG, test
//             ||p||_inf / h < tol * bbox diagonal; else candidates swept along p, ACCD cap
//             alpha_0 = min(1, toi), backtracking E(x + alpha p) <= E(x) (det F <= 0 or d <= 0
//             give E = +inf), x += alpha p.
//   finish  : v = (x - x_n) / h.
// Every gel of a handle runs this machine independently; each host round admits new requests
// (begin) and advances every running gel by one Newton iteration, with one device->host read of
// the per-gel state per round.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "tx_gel.h"
#include "txgel_common.cuh"

namespace txg {
void launch_tet_assemble(const Dev& d, int phase, bool mixed, cudaStream_t st);
void launch_eval_tets(int n, const double* X, const double* x, double mu, double lam, int project,
                      double* e, double* g, double* H, cudaStream_t st);
void launch_indenter_pose(const Dev& d, int phase, int n_ind_verts, cudaStream_t st);
void launch_hash_build(const Dev& d, int phase, int swept, cudaStream_t st);
void launch_query(const Dev& d, int phase, int mode, cudaStream_t st);
void launch_pair_ranges(const Dev& d, int phase, int skip_conv, cudaStream_t st);
int launch_ss_pairs(const Dev& d, int phase, int mode, cudaStream_t st);
void launch_pcg_cz_setup(const Dev& d, int phase, const PcgPlan& plan, int nctas, cudaStream_t st);
void launch_ss_reset(const Dev& d, cudaStream_t st);
void launch_contact_compute(const Dev& d, int phase, bool mixed, cudaStream_t st);
void launch_contact_merge(const Dev& d, bool mixed, cudaStream_t st);
void launch_accd(const Dev& d, int phase, int mode, int maxit, cudaStream_t st);
void launch_min_dist(const Dev& d, int phase, cudaStream_t st);
void launch_fric_setup(const Dev& d, int phase, cudaStream_t st);
void launch_markers(const Dev& d, int g, int n, int ntop, const double* rest_xy, int* tri, double* out, int* found,
                    cudaStream_t st);
void launch_height_map(const Dev& d, int g, int ntop, int nx, int ny, double x0, double y0, double dx, double dy,
                       unsigned long long* img, double* out, cudaStream_t st);
void launch_fric(const Dev& d, int phase, int mode, bool mixed, cudaStream_t st);
void launch_eval_pairs(int n, const int* kind, const double* P, double dhat, const double* eps_x,
                       const int* free_mask, double* b, double* g, double* H, int* dtype, cudaStream_t st);
void launch_eval_accd(int n, const int* kind, const double* P, const double* dP, double s, double tc,
                      int maxit, double* toi, int* hit, cudaStream_t st);
void launch_scan(const int* in, int* out, int n, int* tmp, cudaStream_t st);
void launch_gather(const Dev& d, int phase, int nbp, bool mixed, cudaStream_t st);
void launch_precond(const Dev& d, int phase, bool mixed, cudaStream_t st);
cudaError_t launch_pcg_pool(const Dev& d, int phase, const PoolPlan& pl, int nctas, bool mixed, int maxit,
                            int refine_max, cudaStream_t st);
cudaError_t launch_pcg64(const Dev& d, int phase, const PcgPlan& plan, int nctas, int maxit, cudaStream_t st);
cudaError_t launch_pcg_mixed(const Dev& d, int phase, const PcgPlan& plan, int nctas, int maxit, int refine_max,
                             cudaStream_t st);
int pcg_max_ctas_per_sm(int max_slices);
int pcg_pool_ctas_per_sm(const PoolPlan& pl);
size_t pair_record_doubles();
int pcg_res_ctas_per_sm(bool mixed, int max_slices, int wmax);
cudaError_t launch_pcg_res(const Dev& d, int phase, const PcgPlan& plan, int nctas, bool mixed, int maxit,
                           int refine_max, int wmax, cudaStream_t st);
void launch_energy(const Dev& d, int phase, const int4* pieces, int npieces, const int* gel_piece,
                   double* part_e, unsigned* ticket, int mode, cudaStream_t st);
void launch_rows(int which, const Dev& d, int phase, cudaStream_t st);
void launch_gel_op(const Dev& d, int phase, int op, cudaStream_t st);
}  // namespace txg

#include <atomic>

namespace txg {
static std::atomic<long long> g_launch_count{0};
void count_launch(int k) { g_launch_count.fetch_add(k, std::memory_order_relaxed); }
void set_last_error(const char* msg);
}  // namespace txg

using namespace txg;

namespace {

thread_local std::string g_err;
long long g_launch_mark = 0;
}  // namespace

void txg::set_last_error(const char* msg) { g_err = msg; }

namespace {

constexpr int PCG_MAXG_HOST = 64;  // must match PCG_MAXG in the PCG kernel
// default slices (32 rows) per PCG CTA: FP64 spreads a gel over many SMs (the FP64 pipe bounds
// the SpMV); FP32 keeps groups small so that their barriers are cheap
constexpr int PCG_SLICES_FP64 = 4;
constexpr int PCG_SLICES_FP64_LARGE = 6;  // one FP64 gel on the streaming kernels
constexpr int PCG_SLICES_MIXED = 4;
constexpr int TUNE_N = 5;
constexpr int TUNE_SPC[TUNE_N] = {4, 2, 3, 6, 8};  // candidate slices per CTA (first: the default)
// contact pairs whose barrier setup is kept for the warp Hessian kernel (others recompute it)
constexpr int CREC_PER_GEL = 512;
constexpr int CREC_BASE = 8192;
constexpr int PCG_RES_MAXNC = 256;  // CTAs of one group the resident PCG kernels handle
constexpr int PCG_POOL_MIN_GELS = 32;  // automatic plan: pooled streaming kernels from this many gels
// soft-soft contact: spare block positions of a surface row near another body, and "near": within
// this fraction of that body's rest bounding-box diagonal (plus d_hat) of its rest box
constexpr int SS_SLOTS = 12;
constexpr double SS_NEAR = 0.25;
                                      // being solved on (per-gel CTA groups below: measured faster
                                      // up to 16 gels, slower from 64)
constexpr int PCG_CTAS_PER_SM_CAP = 8;  // plan arrays are sized for this many CTAs per SM
constexpr int PIECE_HOST = 512;
constexpr int PAIR_PIECES = 16;  // energy pieces over a gel's candidate pairs (a few thousand: one each per thread)
constexpr int FRIC_PIECES = 4;   // energy pieces over a gel's friction records

#define CK(call)                                                          \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) {                                              \
      g_err = std::string(#call) + ": " + cudaGetErrorString(e_);         \
      return TX_ERR_CUDA;                                                 \
    }                                                                     \
  } while (0)

double bitsd_host(unsigned long long u) {
  double v;
  std::memcpy(&v, &u, sizeof(v));
  return v;
}

int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

void quat_R(const double q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double n = std::sqrt(w * w + x * x + y * y + z * z);
  w /= n; x /= n; y /= n; z /= n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

void pose_mid(const double a[7], const double b[7], double m[7]) {
  double dq = a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3];
  double sg = dq < 0 ? -1.0 : 1.0, nn = 0.0;
  for (int i = 0; i < 4; ++i) {
    m[i] = a[i] + sg * b[i];
    nn += m[i] * m[i];
  }
  nn = std::sqrt(nn);
  for (int i = 0; i < 4; ++i) m[i] /= nn;
  for (int i = 4; i < 7; ++i) m[i] = 0.5 * (a[i] + b[i]);
}

// ---------------------------------------------------------------- rest-state preprocessing
struct Mesh {
  int nv = 0, nt = 0, niv = 0, nit = 0;
  std::vector<double> X;
  std::vector<int> tets;
  std::vector<uint8_t> fixed;
  std::vector<double> Dminv, vol, mass;
  std::vector<int> sv;
  std::vector<std::array<int, 3>> st;
  std::vector<std::array<int, 2>> se;
  std::vector<double> se_len2;
  std::vector<double> IV;
  std::vector<std::array<int, 3>> it;
  std::vector<std::array<int, 2>> ie;
  std::vector<double> ie_len2;
  std::vector<std::vector<int>> adj;  // sorted neighbour lists (incl. self)
  std::vector<int8_t> comp;           // connected component of each vertex (vertex 0: component 0)
  int ncomp = 1;
  double mu = 0, lam = 0, kappa = 0, bbox = 0, cell = 0, org[3] = {0, 0, 0};
  double mean_se = 0, lo[3] = {0, 0, 0};
  tx_params prm{};
  double pose0[7];
};

// common argument validation of a description
tx_status check_desc(const tx_gel_desc* d) {
  if (!d || d->n_verts <= 0 || d->n_tets < 0 || !d->verts || (d->n_tets > 0 && !d->tets) ||
      d->n_ind_verts < 0 || d->n_ind_tris < 0 || (d->n_ind_verts > 0 && !d->ind_verts) ||
      (d->n_ind_tris > 0 && !d->ind_tris))
    return TX_ERR_ARG;
  if (!(d->young > 0) || !(d->poisson > -1.0 && d->poisson < 0.5) || !(d->density > 0)) return TX_ERR_ARG;
  const tx_params& p = d->params;
  if (!(p.dhat > 0) || !(p.newton_tol > 0) || !(p.pcg_rel_tol > 0) || !(p.pcg_rel_tol_far >= 0) || p.newton_max_iter < 1 ||
      p.pcg_max_iter < 1 || p.ls_max_halvings < 1 || p.accd_max_iter < 1 || p.max_split_depth < 0 ||
      p.pcg_cta_slices < -1 || p.pcg_plan < 0 || p.pcg_plan > 2 || (p.pcg_coarse_off != 0 && p.pcg_coarse_off != 1) || !(p.friction >= 0.0) ||
      !(p.friction_eps_v > 0.0) || !(p.kappa_adapt_max == 0.0 || (p.kappa_adapt_max >= 1.0 && std::isfinite(p.kappa_adapt_max))) ||
      (p.kappa_adapt_max > 0.0 && !(p.kappa_adapt_dmin > 0.0 && std::isfinite(p.kappa_adapt_dmin))))
    return TX_ERR_ARG;
  for (int k = 0; k < 4 * d->n_tets; ++k)
    if (d->tets[k] < 0 || d->tets[k] >= d->n_verts) return TX_ERR_ARG;
  for (int k = 0; k < 3 * d->n_ind_tris; ++k)
    if (d->ind_tris[k] < 0 || d->ind_tris[k] >= d->n_ind_verts) return TX_ERR_ARG;
  return TX_OK;
}

// Rest data of the gel itself (depends on its vertices, tets, Dirichlet mask and density):
// Dm^-1, volumes, lumped masses, boundary triangles / vertices / edges, vertex adjacency.
tx_status build_gel_part(const tx_gel_desc* d, Mesh& m) {
  m.nv = d->n_verts;
  m.nt = d->n_tets;
  m.X.assign(d->verts, d->verts + 3 * m.nv);
  m.tets.assign(d->tets, d->tets + 4 * m.nt);
  m.fixed.assign(m.nv, 0);
  if (d->dirichlet)
    for (int i = 0; i < m.nv; ++i) m.fixed[i] = d->dirichlet[i] ? 1 : 0;
  m.Dminv.resize(9 * (size_t)m.nt);
  m.vol.resize(m.nt);
  m.mass.assign(m.nv, 0.0);
  for (int t = 0; t < m.nt; ++t) {
    const int* v = &m.tets[4 * t];
    double A[9];
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 3; ++a) A[3 * i + a] = m.X[3 * v[a + 1] + i] - m.X[3 * v[0] + i];
    const double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    const double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (!(det > 0.0)) return TX_ERR_MESH_INVERTED;
    const double id = 1.0 / det;
    double* R = &m.Dminv[9 * (size_t)t];
    R[0] = c00 * id;
    R[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    R[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    R[3] = c01 * id;
    R[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    R[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    R[6] = c02 * id;
    R[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    R[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    m.vol[t] = det / 6.0;
    for (int a = 0; a < 4; ++a) m.mass[v[a]] += d->density * m.vol[t] / 4.0;
  }
  // boundary faces (faces of exactly one tet): sort the 4T faces by their vertex set
  const int FI[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
  std::vector<std::pair<std::array<int, 3>, std::array<int, 3>>> faces;
  faces.reserve(4 * (size_t)m.nt);
  for (int t = 0; t < m.nt; ++t)
    for (auto& f : FI) {
      std::array<int, 3> tri = {m.tets[4 * t + f[0]], m.tets[4 * t + f[1]], m.tets[4 * t + f[2]]};
      std::array<int, 3> key = tri;
      std::sort(key.begin(), key.end());
      faces.push_back({key, tri});
    }
  std::sort(faces.begin(), faces.end());
  std::vector<char> on(m.nv, 0);
  std::vector<std::pair<int, int>> edges;
  for (size_t k = 0; k < faces.size();) {
    size_t e = k;
    while (e < faces.size() && faces[e].first == faces[k].first) ++e;
    if (e - k == 1) {
      const auto& tri = faces[k].second;
      m.st.push_back(tri);
      for (int c = 0; c < 3; ++c) {
        const int a = tri[c], b = tri[(c + 1) % 3];
        on[a] = 1;
        edges.push_back({std::min(a, b), std::max(a, b)});
      }
    }
    k = e;
  }
  std::sort(edges.begin(), edges.end());
  edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
  for (int i = 0; i < m.nv; ++i)
    if (on[i]) m.sv.push_back(i);
  double lsum = 0.0;
  for (auto& ed : edges) {
    m.se.push_back({ed.first, ed.second});
    double l2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double dd = m.X[3 * ed.first + c] - m.X[3 * ed.second + c];
      l2 += dd * dd;
    }
    m.se_len2.push_back(l2);
    lsum += std::sqrt(l2);
  }
  m.mean_se = edges.empty() ? 0.0 : lsum / edges.size();
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = 0; i < m.nv; ++i)
    for (int c = 0; c < 3; ++c) {
      lo[c] = std::min(lo[c], m.X[3 * i + c]);
      hi[c] = std::max(hi[c], m.X[3 * i + c]);
    }
  for (int c = 0; c < 3; ++c) m.lo[c] = lo[c];
  m.bbox = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                     (hi[2] - lo[2]) * (hi[2] - lo[2]));
  // vertex adjacency through tets
  m.adj.assign(m.nv, {});
  for (int i = 0; i < m.nv; ++i) m.adj[i].push_back(i);
  for (int t = 0; t < m.nt; ++t)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) m.adj[m.tets[4 * t + a]].push_back(m.tets[4 * t + b]);
  for (auto& l : m.adj) {
    std::sort(l.begin(), l.end());
    l.erase(std::unique(l.begin(), l.end()), l.end());
  }
  // connected components through the tets, numbered in the order of their first vertex; a mesh of
  // several bodies takes part in soft-soft contact, up to SS_MAXC of them
  m.comp.assign(m.nv, -1);
  m.ncomp = 0;
  std::vector<int> stack;
  for (int i = 0; i < m.nv; ++i)
    if (m.adj[i].size() == 1) m.comp[i] = 0;  // in no tet: on no surface, never in a pair
  for (int i = 0; i < m.nv; ++i) {
    if (m.comp[i] >= 0) continue;
    if (m.ncomp == SS_MAXC) return TX_ERR_ARG;
    m.comp[i] = (int8_t)m.ncomp;
    stack.assign(1, i);
    while (!stack.empty()) {
      const int v = stack.back();
      stack.pop_back();
      for (int u : m.adj[v])
        if (m.comp[u] < 0) {
          m.comp[u] = (int8_t)m.ncomp;
          stack.push_back(u);
        }
    }
    ++m.ncomp;
  }
  return TX_OK;
}

// Material constants, the indenter (edges, lengths) and the per-gel solver constants.
void build_rest_part(const tx_gel_desc* d, Mesh& m) {
  const tx_params& p = d->params;
  m.niv = d->n_ind_verts;
  m.nit = d->n_ind_tris;
  m.prm = p;
  std::memcpy(m.pose0, d->ind_pose, sizeof(m.pose0));
  m.mu = d->young / (2.0 * (1.0 + d->poisson));
  m.lam = d->young * d->poisson / ((1.0 + d->poisson) * (1.0 - 2.0 * d->poisson));
  m.IV.assign(d->ind_verts, d->ind_verts + 3 * m.niv);
  std::vector<std::pair<int, int>> iedges;
  for (int k = 0; k < m.nit; ++k) {
    m.it.push_back({d->ind_tris[3 * k], d->ind_tris[3 * k + 1], d->ind_tris[3 * k + 2]});
    for (int c = 0; c < 3; ++c) {
      const int a = d->ind_tris[3 * k + c], b = d->ind_tris[3 * k + (c + 1) % 3];
      iedges.push_back({std::min(a, b), std::max(a, b)});
    }
  }
  std::sort(iedges.begin(), iedges.end());
  iedges.erase(std::unique(iedges.begin(), iedges.end()), iedges.end());
  double isum = 0.0;
  for (auto& ed : iedges) {
    m.ie.push_back({ed.first, ed.second});
    double l2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double dd = m.IV[3 * ed.first + c] - m.IV[3 * ed.second + c];
      l2 += dd * dd;
    }
    m.ie_len2.push_back(l2);
    isum += std::sqrt(l2);
  }
  const double mean_ie = iedges.empty() ? 0.0 : isum / iedges.size();
  m.kappa = p.kappa > 0 ? p.kappa : d->young * m.mean_se;
  m.cell = std::max(std::max(m.mean_se, mean_ie), 4.0 * p.dhat);
  for (int c = 0; c < 3; ++c) m.org[c] = m.lo[c] - 64.0 * m.cell;
}

tx_status build_mesh(const tx_gel_desc* d, Mesh& m) {
  tx_status s = check_desc(d);
  if (s != TX_OK) return s;
  s = build_gel_part(d, m);
  if (s != TX_OK) return s;
  build_rest_part(d, m);
  return TX_OK;
}

// 64-bit FNV-1a over a byte range
uint64_t fnv(const void* p, size_t n, uint64_t h) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t k = 0; k < n; ++k) h = (h ^ c[k]) * 1099511628211ull;
  return h;
}

// ---------------------------------------------------------------- fault injection (test hook)
// Host-side only: an allocation made to fail before it reaches the CUDA runtime, and bounded
// device waits told to wait for an arrival that never comes.  Nothing faults the device.
std::atomic<int> g_inject_alloc{0};  // > 0: the allocation this many allocations from now fails
std::atomic<int> g_inject_wait{0};   // Newton iterations whose PCG barriers wait for a missing arrival
constexpr unsigned WAIT_LIMIT = 1u << 22;        // polls of a bounded device wait (~0.1-1 s)
constexpr unsigned WAIT_LIMIT_INJECTED = 1u << 12;  // the same when a timeout is being injected

bool injected_alloc_failure() {
  int k = g_inject_alloc.load();
  while (k > 0) {
    if (g_inject_alloc.compare_exchange_weak(k, k - 1)) return k == 1;
  }
  return false;
}

// ---------------------------------------------------------------- device allocation
struct DevMem {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  bool failed = false;  // some get() returned nullptr
  template <class T>
  T* get(size_t n) {
    if (n == 0) n = 1;
    void* p = nullptr;
    if (injected_alloc_failure() || cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      failed = true;
      return nullptr;
    }
    ptrs.push_back(p);
    bytes += n * sizeof(T);
    return static_cast<T*>(p);
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
    bytes = 0;
    failed = false;
  }
};

cudaError_t host_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaHostAlloc(p, bytes, cudaHostAllocDefault);
}

struct Task {
  double pa[7], pb[7];
  double ca[7], cb[7];  // case pose at the start / end (attachment-driven steps only)
  double dt;
  int depth;
  bool first;
  bool attached;
};

struct Run {
  std::vector<Task> stack;  // back = next substep
  bool in_request = false;
  int phase = PH_IDLE;
  tx_status status = TX_OK;
  int newton_sub = 0;       // Newton updates in the current substep
  tx_step_stats acc{};      // accumulating stats of the request
  tx_step_stats last{};     // last finished request
  double pose[7];           // indenter pose at the end of the last finished substep
  double pose_req[7];       // pose at the start of the request (for rollback)
  double case_pose[7] = {1, 0, 0, 0, 0, 0, 0};  // pose of the attached vertices' frame (the sensor case)
  double case_req[7] = {1, 0, 0, 0, 0, 0, 0};   // ... at the start of the request (for rollback)
  // barrier stiffness of the next step and the final smallest pair distance of the last step
  // (tx_params.kappa_adapt_max: doubled after a step that ended nearer than kappa_adapt_dmin and
  // nearer than the step before)
  double kappa = 0.0, dmin_last = 1e300;
};

}  // namespace

namespace {
enum Phase2 : int { PR_BEGIN = 0, PR_TET, PR_GATHER, PR_CONTACT, PR_PRECOND, PR_PCG, PR_QUERY, PR_ACCD,
                    PR_LS, PR_FINAL, PR_N };
const char* const kPhaseNames[PR_N] = {"begin", "tet_assemble", "gather", "contact_assemble", "precond",
                                       "pcg", "query", "accd", "line_search", "finalize"};
struct Prof {
  bool on = false;
  double ms[PR_N] = {};
  long long launches[PR_N] = {};
  double flops[PR_N] = {};
  double bytes[PR_N] = {};
  long long pcg_iters = 0, newton_iters = 0;
  long long pcg_res = 0, pcg_stream = 0, pcg_pool = 0;  // PCG launches per kernel family
  struct Pending {
    cudaEvent_t a, b;
    int phase;
    bool graph;  // events owned by a captured Newton-iteration graph (not returned to the pool)
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pending;
  int open_phase = -1;
  cudaEvent_t open_ev = nullptr;
};
}  // namespace

struct tx_batch {
  int n = 0;
  Prof prof;
  std::vector<double> nnzb_real;  // per gel: real 3x3 blocks of its Hessian
  std::vector<double> nfree;      // per gel: free rows
  cudaStream_t st = nullptr;
  bool mixed = false;
  std::vector<Mesh> mesh;
  std::vector<GelInfo> gi;
  std::vector<Run> run;
  std::vector<int> ss_gel_h;  // the gels whose mesh holds several bodies (soft-soft contact)
  bool has_cbody = false;     // some gel has a body held by no vertex (coarse space of k_pcg64)
  GelCtl* gc_h = nullptr;   // pinned
  GelVar* gv_h = nullptr;   // pinned
  Dev d{};
  DevMem mem;
  DevMem pair_mem;          // pairs + slot map (regrown on overflow)
  DevMem readout_mem;       // scratch of the surface readout (grown on demand)
  size_t readout_bytes = 0;
  DevMem hash_mem;          // hash entries (regrown on overflow)
  int nbp = 0;
  // PCG
  PcgPlan plan{};
  int nctas = 0;
  bool pcg_res = false;  // resident kernels: one slice per warp, matrix in shared memory
  int pcg_wmax = 0;      // widest slice (blocks per row)
  int pcg_spc_min = 4;   // slices per CTA at least
  int pcg_cta_cap = 0;   // capacity of the device plan arrays (CTAs)
  int nsm = 0;
  std::vector<int> plan_key;  // active gels of the plan on the device
  int plan_spc = 0;           // slices per CTA it was built with
  long long plan_version = 0; // bumped whenever the device plan changes
  // A round's solve may run as several consecutive PCG launches ("parts"), each over a subset
  // of the gels whose FP32 matrices fit in L2 together, so that its iterations after the first
  // read the matrix from L2 instead of HBM.  Each part has its own plan arrays.
  struct PlanPart {
    PcgPlan plan{};
    int nctas = 0;
    bool res = false;
    bool pool_on = false;  // streaming in the pooled form
    PoolPlan pool{};       // its gel range and CTAs
    int pool_nctas = 0;
  };
  std::vector<PlanPart> parts;
  int nparts = 0;
  std::vector<double> nbp_gel;  // per gel: block positions of its sliced BSR
  DevMem plan_mem;
  int plan_parts_cap = 0;
  double l2_budget = 0.0;     // bytes of FP32 matrices and vectors one part may hold
  // captured Newton iteration (launch part), replayed while its inputs stay the same
  struct NewtonGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<int> key;
    Dev dev{};
    long long plan_version = -1;
    int nctas = 0;
    bool res = false, prof = false, tune = false;
    int pcg_max = 0, refine = 0, accd_max = 0;
    long long launches = 0;
    long long phase_launches[PR_N] = {};
    std::vector<Prof::Pending> prof_pairs;
  } graph;
  // PCG work-split autotuner (opt-in: a negative pcg_cta_slices): per class of active sets
  // (number of gels, total slices in powers of 2^(1/2)) the candidate splits are tried on
  // successive Newton rounds, timed per PCG iteration, and the fastest is kept
  struct Tune {
    int idx = 0;
    double us[8] = {};
    int best = -1;
  };
  int plan_mode = 0;  // the largest tx_params.pcg_plan of the gels: 0 automatic, 1 per-gel-group
                      // streaming, 2 pooled streaming
  bool friction = false;      // some gel has lagged friction (tx_params.friction > 0)
  bool tune_on = false;
  std::map<long long, Tune> tune;
  long long tune_key = -1;  // class of the current round (-1: not timing)
  cudaEvent_t tev0 = nullptr, tev1 = nullptr;
  int graphs = -1;  // -1 undecided, 0 off (unsupported or disabled), 1 on
  bool capturing = false;  // profile events become event-record nodes of the graph
  cudaStream_t gst = nullptr;          // stream the graph is captured on and replayed on
  cudaStream_t st2 = nullptr;          // side stream of the contact assembly (fork / join events)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool side_ok = false;
  cudaEvent_t gev_in = nullptr, gev_out = nullptr;  // order it after / before the caller's stream
  std::vector<int2> plan_rng_h;
  std::vector<int> plan_grp_of_h;
  std::vector<int4> plan_grp_h;
  // energy pieces
  int4* pieces = nullptr;
  int npieces = 0;
  int* gel_piece = nullptr;
  std::vector<int4> pieces_h;
  std::vector<int> gel_piece_h;
  double* part_e = nullptr;
  unsigned* en_ticket = nullptr;  // per gel: pieces of the running energy launch done
  int* scan_tmp = nullptr;
  double4_32a *x0 = nullptr, *v0 = nullptr;  // request start state (rollback)
  double4_32a *ex = nullptr, *ext = nullptr; // evaluation save area
  int total_rows = 0;
  std::vector<int> done_queue;
};

struct tx_gel {
  tx_batch* b;
};

namespace {

cudaEvent_t prof_event(tx_batch* b) {
  if (!b->prof.pool.empty()) {
    cudaEvent_t e = b->prof.pool.back();
    b->prof.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
// inside a stream capture a plain record would only order the graph's nodes; the external
// flag makes it a record node that fires on every replay, so the phase times stay measurable
void prof_record(tx_batch* b, cudaEvent_t e, cudaStream_t s = nullptr) {
  if (!s) s = b->st;
  if (b->capturing)
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else
    cudaEventRecord(e, s);
}

// phase timing on the stream its launches go to (the library stream unless given)
void prof_open(tx_batch* b, int phase, cudaStream_t s = nullptr) {
  if (!b->prof.on) return;
  b->prof.open_phase = phase;
  b->prof.open_ev = prof_event(b);
  prof_record(b, b->prof.open_ev, s);
}
void prof_close(tx_batch* b, int nlaunch, cudaStream_t s = nullptr) {
  if (!b->prof.on || b->prof.open_phase < 0) return;
  cudaEvent_t e = prof_event(b);
  prof_record(b, e, s);
  b->prof.pending.push_back({b->prof.open_ev, e, b->prof.open_phase, false});
  b->prof.launches[b->prof.open_phase] += nlaunch;
  b->prof.open_phase = -1;
}
// after a stream synchronisation: fold the finished event pairs into the counters
void prof_resolve(tx_batch* b) {
  for (auto& p : b->prof.pending) {
    float ms = 0.f;
    const cudaError_t e = cudaEventElapsedTime(&ms, p.a, p.b);
    if (e == cudaSuccess)
      b->prof.ms[p.phase] += ms;
    else
      g_err = std::string("profile event: ") + cudaGetErrorString(e);
    cudaGetLastError();
    if (p.graph) continue;
    b->prof.pool.push_back(p.a);
    b->prof.pool.push_back(p.b);
  }
  b->prof.pending.clear();
}

// per-gel pair capacity and hash sizes (initial guesses; grown on overflow)
int initial_pcap(const Mesh& m) {
  return std::max(4096, 2 * (int)(m.sv.size() + m.st.size() + m.se.size()));
}

tx_status upload_ctl(tx_batch* b) {
  CK(cudaMemcpyAsync((void*)b->d.gc, b->gc_h, sizeof(GelCtl) * b->n, cudaMemcpyHostToDevice, b->st));
  return TX_OK;
}
tx_status download_var(tx_batch* b) {
  CK(cudaMemcpyAsync(b->gv_h, b->d.gv, sizeof(GelVar) * b->n, cudaMemcpyDeviceToHost, b->st));
  CK(cudaStreamSynchronize(b->st));
  prof_resolve(b);
  return TX_OK;
}
tx_status upload_info(tx_batch* b) {
  CK(cudaMemcpyAsync((void*)b->d.gi, b->gi.data(), sizeof(GelInfo) * b->n, cudaMemcpyHostToDevice, b->st));
  return TX_OK;
}

// (Re)allocate the candidate-pair segments with the capacities in gi[].pcap.
// The new segments are allocated before the old ones are freed: if the device is out of memory the
// handle keeps its previous segments and capacities (TX_ERR_OOM), never a null segment.
tx_status alloc_pairs(tx_batch* b) {
  CK(cudaStreamSynchronize(b->st));
  std::vector<GelInfo> old = b->gi;
  int total = 0;
  for (int g = 0; g < b->n; ++g) {
    b->gi[g].pbase = total;
    total += b->gi[g].pcap;
  }
  DevMem nm;
  Dev nd = b->d;
  nd.pairs = nm.get<int4>(total);
  nd.pslot_gel = nm.get<int>(total);
  nd.cwork = nm.get<int>(total);
  nd.crec_cap = std::min(total, CREC_PER_GEL * b->n + CREC_BASE);
  nd.crec = reinterpret_cast<PairBarrier*>(nm.get<double>((size_t)nd.crec_cap * pair_record_doubles()));
  nd.chv = nm.get<double>((size_t)nd.crec_cap * CH_STRIDE);
  nd.chbp = nm.get<int>((size_t)nd.crec_cap * CH_BP);
  nd.c1rec = nm.get<C1Rec>(total);
  nd.fric = b->friction ? nm.get<FricRec>(total) : nullptr;
  if (nm.failed) {
    nm.release();
    b->gi = old;
    return TX_ERR_OOM;
  }
  if (b->friction && b->d.fric) {  // the lagged friction records of running substeps move along
    for (int g = 0; g < b->n; ++g)
      if (old[g].pcap > 0)
        CK(cudaMemcpyAsync(nd.fric + b->gi[g].pbase, b->d.fric + old[g].pbase,
                           sizeof(FricRec) * std::min(old[g].pcap, b->gi[g].pcap), cudaMemcpyDeviceToDevice, b->st));
    CK(cudaStreamSynchronize(b->st));
  }
  b->pair_mem.release();
  b->pair_mem = nm;
  b->d = nd;
  b->d.npslots = total;
  std::vector<int> slot(total);
  for (int g = 0; g < b->n; ++g)
    for (int k = 0; k < b->gi[g].pcap; ++k) slot[b->gi[g].pbase + k] = g;
  CK(cudaMemcpy(b->d.pslot_gel, slot.data(), sizeof(int) * total, cudaMemcpyHostToDevice));
  return upload_info(b);
}

tx_status alloc_hash(tx_batch* b) {
  CK(cudaStreamSynchronize(b->st));
  std::vector<GelInfo> old = b->gi;
  int total = 0;
  for (int g = 0; g < b->n; ++g)
    for (int t = 0; t < NTAB; ++t) {
      b->gi[g].he0[t] = total;
      total += b->gi[g].hcap[t];
    }
  DevMem nm;
  int2* hent = nm.get<int2>(total);
  if (nm.failed) {
    nm.release();
    b->gi = old;
    return TX_ERR_OOM;
  }
  b->hash_mem.release();
  b->hash_mem = nm;
  b->d.hent = hent;
  return upload_info(b);
}

// Block positions each row of a gel needs in its slice: its mesh neighbours (incl. itself), and
// in a mesh of several bodies SS_SLOTS more for every free surface row that lies, at rest, near
// the box of another body (room for the blocks of soft-soft pairs, claimed during the assembly)
std::vector<int> row_block_needs(const Mesh& m) {
  std::vector<int> need(m.nv);
  for (int i = 0; i < m.nv; ++i) need[i] = (int)m.adj[i].size();
  if (m.ncomp <= 1) return need;
  double lo[SS_MAXC][3], hi[SS_MAXC][3];
  for (int c = 0; c < SS_MAXC; ++c)
    for (int a = 0; a < 3; ++a) {
      lo[c][a] = INFINITY;
      hi[c][a] = -INFINITY;
    }
  for (int i = 0; i < m.nv; ++i)
    for (int a = 0; a < 3; ++a) {
      lo[m.comp[i]][a] = std::min(lo[m.comp[i]][a], m.X[3 * i + a]);
      hi[m.comp[i]][a] = std::max(hi[m.comp[i]][a], m.X[3 * i + a]);
    }
  for (int i : m.sv) {
    if (m.fixed[i]) continue;
    bool near = false;
    for (int c = 0; c < m.ncomp && !near; ++c) {
      if (c == m.comp[i]) continue;
      double diag2 = 0.0;
      for (int a = 0; a < 3; ++a) diag2 += (hi[c][a] - lo[c][a]) * (hi[c][a] - lo[c][a]);
      const double pad = SS_NEAR * std::sqrt(diag2) + m.prm.dhat;
      near = true;
      for (int a = 0; a < 3; ++a)
        if (m.X[3 * i + a] < lo[c][a] - pad || m.X[3 * i + a] > hi[c][a] + pad) near = false;
    }
    if (near) need[i] += SS_SLOTS;
  }
  return need;
}

// ---------------------------------------------------------------- creation
tx_status create_batch(const tx_gel_desc* descs, int n, void* stream, tx_batch** out) {
  if (!descs || n <= 0 || !out) return TX_ERR_ARG;
  tx_batch* b = new tx_batch();
  b->n = n;
  b->st = (cudaStream_t)stream;
  b->mesh.resize(n);
  // gels with identical rest meshes (vertices, tets, Dirichlet mask, density) share one
  // preprocessing pass; only the indenter part is per gel
  std::map<uint64_t, int> seen;
  for (int g = 0; g < n; ++g) {
    const tx_gel_desc* d = &descs[g];
    tx_status s = check_desc(d);
    if (s != TX_OK) {
      delete b;
      return s;
    }
    uint64_t h = 1469598103934665603ull;
    h = fnv(&d->n_verts, sizeof(d->n_verts), h);
    h = fnv(&d->n_tets, sizeof(d->n_tets), h);
    h = fnv(&d->density, sizeof(d->density), h);
    h = fnv(d->verts, sizeof(double) * 3 * d->n_verts, h);
    h = fnv(d->tets, sizeof(int32_t) * 4 * d->n_tets, h);
    if (d->dirichlet) h = fnv(d->dirichlet, d->n_verts, h);
    auto it = seen.find(h);
    bool reused = false;
    if (it != seen.end()) {
      const tx_gel_desc* o = &descs[it->second];
      const bool same = o->n_verts == d->n_verts && o->n_tets == d->n_tets && o->density == d->density &&
                        std::memcmp(o->verts, d->verts, sizeof(double) * 3 * d->n_verts) == 0 &&
                        std::memcmp(o->tets, d->tets, sizeof(int32_t) * 4 * d->n_tets) == 0 &&
                        ((!o->dirichlet && !d->dirichlet) ||
                         (o->dirichlet && d->dirichlet && std::memcmp(o->dirichlet, d->dirichlet, d->n_verts) == 0));
      if (same) {
        b->mesh[g] = b->mesh[it->second];  // copies the gel part (and a stale indenter part)
        Mesh& m = b->mesh[g];
        m.IV.clear();
        m.it.clear();
        m.ie.clear();
        m.ie_len2.clear();
        reused = true;
      }
    }
    if (!reused) {
      s = build_gel_part(d, b->mesh[g]);
      if (s != TX_OK) {
        delete b;
        return s;
      }
      seen[h] = g;
    }
    build_rest_part(d, b->mesh[g]);
  }
  b->mixed = descs[0].params.precision == TX_PREC_MIXED;
  for (int g = 1; g < n; ++g)
    if ((descs[g].params.precision == TX_PREC_MIXED) != b->mixed) {
      delete b;
      return TX_ERR_ARG;
    }
  // mixed precision needs every body held by a vertex: a free body's rigid motions, resisted by
  // its mass alone, are beyond the FP32 inner solves (its solves stop at a wrong state)
  for (int g = 0; g < n && b->mixed; ++g) {
    const Mesh& m = b->mesh[g];
    std::vector<char> used(m.ncomp, 0), held(m.ncomp, 0);
    for (int i = 0; i < m.nv; ++i)
      if (m.adj[i].size() > 1) {
        used[m.comp[i]] = 1;
        held[m.comp[i]] |= m.fixed[i];
      }
    for (int q = 0; q < m.ncomp; ++q)
      if (used[q] && !held[q]) {
        set_last_error("mixed precision needs every body of the mesh held by a vertex (a free body: use FP64)");
        delete b;
        return TX_ERR_ARG;
      }
  }
  // ---- offsets
  b->gi.resize(n);
  int rows = 0, tets = 0, nsv = 0, nst = 0, nse = 0, nq = 0, niv = 0, nit = 0, nie = 0, hb = 0, max_hnb = 1;
  for (int g = 0; g < n; ++g) {
    const Mesh& m = b->mesh[g];
    GelInfo& G = b->gi[g];
    std::memset(&G, 0, sizeof(G));
    G.v0 = rows;
    G.nv = m.nv;
    G.s0 = rows / SLICE;
    G.ns = (m.nv + SLICE - 1) / SLICE;
    rows += G.ns * SLICE;
    G.t0 = tets;
    G.nt = m.nt;
    tets += m.nt;
    G.q0 = nq;
    G.nsv = (int)m.sv.size();
    G.nst = (int)m.st.size();
    G.nse = (int)m.se.size();
    G.nq = G.nsv + G.nst + G.nse;
    nq += G.nq;
    G.sv0 = nsv;
    G.st0 = nst;
    G.se0 = nse;
    nsv += G.nsv;
    nst += G.nst;
    nse += G.nse;
    G.iv0 = niv;
    G.niv = m.niv;
    G.it0 = nit;
    G.nit = m.nit;
    G.ie0 = nie;
    G.nie = (int)m.ie.size();
    niv += G.niv;
    nit += G.nit;
    nie += G.nie;
    const int np[NTAB] = {G.nit, G.niv, G.nie};
    for (int t = 0; t < NTAB; ++t) {
      G.hnb[t] = next_pow2(std::max(16, 2 * np[t]));
      max_hnb = std::max(max_hnb, G.hnb[t]);
      G.hb0[t] = hb;
      hb += G.hnb[t] + 1;
      G.hcap[t] = std::max(256, 8 * np[t]);
    }
    G.pcap = initial_pcap(m);
    G.mu = m.mu;
    G.lam = m.lam;
    G.kappa = m.kappa;
    G.dhat = m.prm.dhat;
    G.cell = m.cell;
    G.bbox_diag = m.bbox;
    G.newton_tol = m.prm.newton_tol;
    G.mu_f = m.prm.friction;
    G.eps_v = m.prm.friction_eps_v;
    if (G.mu_f > 0.0) b->friction = true;
    for (int c = 0; c < 3; ++c) G.org[c] = m.org[c];
    int fc = 0;
    for (auto f : m.fixed) fc += f;
    G.fixed_count = fc;
    G.ncomp = m.ncomp;
    G.ss = -1;
    {  // the largest body with no held vertex: the coarse space of the streaming FP64 PCG
      std::vector<int> nv(m.ncomp, 0), nfix(m.ncomp, 0);
      std::vector<double> cs(3 * (size_t)m.ncomp, 0.0);
      for (int i = 0; i < m.nv; ++i) {
        if (m.adj[i].size() == 1) continue;  // in no tet
        nv[m.comp[i]] += 1;
        nfix[m.comp[i]] += m.fixed[i];
        for (int a = 0; a < 3; ++a) cs[3 * m.comp[i] + a] += m.X[3 * i + a];
      }
      G.cbody = -1;
      for (int q = 0; q < m.ncomp && !m.prm.pcg_coarse_off; ++q)
        if (nfix[q] == 0 && nv[q] > 0 && (G.cbody < 0 || nv[q] > nv[G.cbody])) G.cbody = q;
      for (int a = 0; a < 3; ++a) G.cctr[a] = G.cbody >= 0 ? cs[3 * G.cbody + a] / nv[G.cbody] : 0.0;
      if (G.cbody >= 0) b->has_cbody = true;
    }
    if (m.ncomp > 1) {
      G.ss = (int)b->ss_gel_h.size();
      b->ss_gel_h.push_back(g);
    }
  }
  b->total_rows = rows;
  const int nslices = rows / SLICE;
  // ---- sliced BSR pattern.  A mesh of several bodies gives the free surface rows that lie, at
  // rest, near the box of another body SS_SLOTS spare positions for the blocks of soft-soft
  // pairs (claimed during the assembly); other rows keep only the padding of their slice.
  std::vector<int> slice_off(nslices + 1, 0);
  for (int g = 0; g < n; ++g) {
    const Mesh& m = b->mesh[g];
    const GelInfo& G = b->gi[g];
    const std::vector<int> need = row_block_needs(m);
    for (int s = 0; s < G.ns; ++s) {
      int w = 1;
      for (int l = 0; l < SLICE; ++l) {
        const int i = s * SLICE + l;
        if (i < m.nv) w = std::max(w, need[i]);
      }
      slice_off[G.s0 + s + 1] = w * SLICE;
    }
  }
  for (int s = 0; s < nslices; ++s) slice_off[s + 1] += slice_off[s];
  const int nbp = slice_off[nslices];
  b->nbp = nbp;
  std::vector<int> colidx(nbp), bp_row(nbp), diag_pos(rows), ctr_cnt(nbp + 1, 0);
  std::vector<int> vgel(rows), slice_gel(nslices);
  std::vector<uint8_t> fixed(rows, 1);
  std::vector<double> mass(rows, 0.0);
  for (int g = 0; g < n; ++g) {
    const Mesh& m = b->mesh[g];
    const GelInfo& G = b->gi[g];
    for (int s = 0; s < G.ns; ++s) slice_gel[G.s0 + s] = g;
    for (int l = 0; l < G.ns * SLICE; ++l) {
      const int r = G.v0 + l;
      vgel[r] = g;
      const int s = r / SLICE, lane = r % SLICE;
      const int w = (slice_off[s + 1] - slice_off[s]) / SLICE;
      for (int k = 0; k < w; ++k) {
        const int bp = slice_off[s] + SLICE * k + lane;
        bp_row[bp] = r;
        if (l < m.nv && k < (int)m.adj[l].size()) {
          colidx[bp] = G.v0 + m.adj[l][k];
          if (m.adj[l][k] == l) diag_pos[r] = bp;
        } else {
          colidx[bp] = r;
          if (l >= m.nv && k == 0) diag_pos[r] = bp;
        }
      }
      if (l < m.nv) {
        fixed[r] = m.fixed[l];
        mass[r] = m.mass[l];
      }
    }
  }
  // soft-soft gels: every padding position of their rows may be claimed once per assembly
  std::vector<int8_t> vcomp(rows, 0);
  long long claim_cap = 0;
  for (int g = 0; g < n; ++g) {
    const Mesh& m = b->mesh[g];
    const GelInfo& G = b->gi[g];
    for (int l = 0; l < m.nv; ++l) vcomp[G.v0 + l] = m.comp[l];
    if (m.ncomp > 1)
      for (int l = 0; l < m.nv; ++l) {
        const int r = G.v0 + l, s = r / SLICE;
        claim_cap += (slice_off[s + 1] - slice_off[s]) / SLICE - (long long)m.adj[l].size();
      }
  }
  auto bp_of = [&](int g, int li, int lj) {
    const Mesh& m = b->mesh[g];
    const auto& a = m.adj[li];
    const int k = (int)(std::lower_bound(a.begin(), a.end(), lj) - a.begin());
    const int r = b->gi[g].v0 + li;
    return slice_off[r / SLICE] + SLICE * k + r % SLICE;
  };
  for (int g = 0; g < n; ++g) {
    const Mesh& m = b->mesh[g];
    for (int t = 0; t < m.nt; ++t)
      for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 4; ++c) ctr_cnt[bp_of(g, m.tets[4 * t + a], m.tets[4 * t + c]) + 1]++;
  }
  for (int k = 0; k < nbp; ++k) ctr_cnt[k + 1] += ctr_cnt[k];
  std::vector<int> ctr(ctr_cnt[nbp]), fillp(ctr_cnt.begin(), ctr_cnt.end() - 1);
  for (int g = 0; g < n; ++g) {
    const Mesh& m = b->mesh[g];
    for (int t = 0; t < m.nt; ++t)
      for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 4; ++c) {
          const int bp = bp_of(g, m.tets[4 * t + a], m.tets[4 * t + c]);
          ctr[fillp[bp]++] = ((b->gi[g].t0 + t) << 4) | (a << 2) | c;
        }
  }
  // ---- top surface (readout): boundary triangles whose rest outward normal points up
  std::vector<int4> top4;
  for (int g = 0; g < n; ++g) {
    const Mesh& m = b->mesh[g];
    GelInfo& G = b->gi[g];
    G.top0 = (int)top4.size();
    for (const auto& t : m.st) {
      if (m.comp[t[0]] != 0) continue;  // the gelpad: component 0 (a mesh may hold other bodies)
      const double* A = &m.X[3 * t[0]];
      const double* Bv = &m.X[3 * t[1]];
      const double* C = &m.X[3 * t[2]];
      const double nz = (Bv[0] - A[0]) * (C[1] - A[1]) - (Bv[1] - A[1]) * (C[0] - A[0]);
      if (nz > 0.0) top4.push_back(make_int4(G.v0 + t[0], G.v0 + t[1], G.v0 + t[2], g));
    }
    G.ntop = (int)top4.size() - G.top0;
  }
  // ---- host arrays of the concatenated gels
  std::vector<double4_32a> X(rows);
  std::vector<int4> tet4(std::max(tets, 1));
  std::vector<int> tgel(std::max(tets, 1));
  std::vector<double> Dminv(9 * (size_t)std::max(tets, 1)), vol(std::max(tets, 1));
  std::vector<int> sv(std::max(nsv, 1)), q_gel(std::max(nq, 1)), q_tp(std::max(nq, 1));
  std::vector<int4> st4(std::max(nst, 1));
  std::vector<int2> se2(std::max(nse, 1));
  std::vector<double> se_len2(std::max(nse, 1));
  std::vector<double4_32a> ivl(std::max(niv, 1));
  std::vector<int4> it4(std::max(nit, 1));
  std::vector<int2> ie2(std::max(nie, 1));
  std::vector<double> ie_len2(std::max(nie, 1));
  std::vector<int> iv_gel(std::max(niv, 1)), it_gel(std::max(nit, 1)), ie_gel(std::max(nie, 1));
  for (int g = 0; g < n; ++g) {
    const Mesh& m = b->mesh[g];
    const GelInfo& G = b->gi[g];
    for (int r = 0; r < G.ns * SLICE; ++r)
      X[G.v0 + r] = r < m.nv ? make_double4_32a(m.X[3 * r], m.X[3 * r + 1], m.X[3 * r + 2], 0.0)
                             : make_double4_32a(0.0, 0.0, 0.0, 0.0);
    for (int t = 0; t < m.nt; ++t) {
      tet4[G.t0 + t] = make_int4(G.v0 + m.tets[4 * t], G.v0 + m.tets[4 * t + 1], G.v0 + m.tets[4 * t + 2],
                                 G.v0 + m.tets[4 * t + 3]);
      tgel[G.t0 + t] = g;
      for (int k = 0; k < 9; ++k) Dminv[9 * (size_t)(G.t0 + t) + k] = m.Dminv[9 * (size_t)t + k];
      vol[G.t0 + t] = m.vol[t];
    }
    for (int k = 0; k < G.nsv; ++k) sv[G.sv0 + k] = G.v0 + m.sv[k];
    for (int k = 0; k < G.nst; ++k) st4[G.st0 + k] = make_int4(G.v0 + m.st[k][0], G.v0 + m.st[k][1], G.v0 + m.st[k][2], 0);
    for (int k = 0; k < G.nse; ++k) {
      se2[G.se0 + k] = make_int2(G.v0 + m.se[k][0], G.v0 + m.se[k][1]);
      se_len2[G.se0 + k] = m.se_len2[k];
    }
    for (int k = 0; k < G.nq; ++k) {
      q_gel[G.q0 + k] = g;
      if (k < G.nsv)
        q_tp[G.q0 + k] = (PAIR_PT << 28) | k;
      else if (k < G.nsv + G.nst)
        q_tp[G.q0 + k] = (PAIR_TP << 28) | (k - G.nsv);
      else
        q_tp[G.q0 + k] = (PAIR_EE << 28) | (k - G.nsv - G.nst);
    }
    for (int k = 0; k < G.niv; ++k) {
      ivl[G.iv0 + k] = make_double4_32a(m.IV[3 * k], m.IV[3 * k + 1], m.IV[3 * k + 2], 0.0);
      iv_gel[G.iv0 + k] = g;
    }
    for (int k = 0; k < G.nit; ++k) {
      it4[G.it0 + k] = make_int4(G.iv0 + m.it[k][0], G.iv0 + m.it[k][1], G.iv0 + m.it[k][2], 0);
      it_gel[G.it0 + k] = g;
    }
    for (int k = 0; k < G.nie; ++k) {
      ie2[G.ie0 + k] = make_int2(G.iv0 + m.ie[k][0], G.iv0 + m.ie[k][1]);
      ie_len2[G.ie0 + k] = m.ie_len2[k];
      ie_gel[G.ie0 + k] = g;
    }
  }
  // ---- PCG plan: independent groups (a large gel over several CTAs, small gels packed into one)
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    g_err = "no CUDA device";
    delete b;
    return TX_ERR_CUDA;
  }
  int spc_min = 0;  // slices (32 rows) per CTA at least
  for (int g = 0; g < n; ++g) {
    spc_min = std::max(spc_min, b->mesh[g].prm.pcg_cta_slices);
    if (b->mesh[g].prm.pcg_cta_slices < 0) b->tune_on = true;
    b->plan_mode = std::max(b->plan_mode, (int)b->mesh[g].prm.pcg_plan);
  }
  if (spc_min <= 0) spc_min = b->mixed ? PCG_SLICES_MIXED : PCG_SLICES_FP64;
  b->pcg_spc_min = spc_min;
  b->nsm = nsm;
  for (int q = 0; q < nslices; ++q) b->pcg_wmax = std::max(b->pcg_wmax, (slice_off[q + 1] - slice_off[q]) / SLICE);
  b->nbp_gel.resize(n);
  for (int g = 0; g < n; ++g)
    b->nbp_gel[g] = (double)(slice_off[b->gi[g].s0 + b->gi[g].ns] - slice_off[b->gi[g].s0]);
  const int cta_cap = PCG_CTAS_PER_SM_CAP * nsm;  // largest co-resident grid of any plan
  b->pcg_cta_cap = cta_cap;
  // ---- energy pieces
  for (int g = 0; g < n; ++g) {
    const GelInfo& G = b->gi[g];
    b->gel_piece_h.push_back((int)b->pieces_h.size());
    for (int t = G.t0; t < G.t0 + G.nt; t += PIECE_HOST)
      b->pieces_h.push_back(make_int4(g, 0, t, std::min(t + PIECE_HOST, G.t0 + G.nt)));
    for (int r = G.v0; r < G.v0 + G.nv; r += PIECE_HOST)
      b->pieces_h.push_back(make_int4(g, 1, r, std::min(r + PIECE_HOST, G.v0 + G.nv)));
    for (int k = 0; k < PAIR_PIECES; ++k) b->pieces_h.push_back(make_int4(g, 2, k, PAIR_PIECES));
    if (G.mu_f > 0.0)  // lagged friction records
      for (int k = 0; k < FRIC_PIECES; ++k) b->pieces_h.push_back(make_int4(g, 3, k, FRIC_PIECES));
  }
  b->gel_piece_h.push_back((int)b->pieces_h.size());
  b->npieces = (int)b->pieces_h.size();
  // ---- device allocation
  DevMem& M = b->mem;
  Dev& d = b->d;
  d.n_gels = n;
  d.nrows = rows;
  d.ntets = tets;
  d.nslices = nslices;
  d.nq = nq;
  d.niv_total = niv;
  d.gi = M.get<GelInfo>(n);
  d.gc = M.get<GelCtl>(n);
  d.gv = M.get<GelVar>(n);
  d.X = M.get<double4_32a>(rows);
  d.x = M.get<double4_32a>(rows);
  d.xn = M.get<double4_32a>(rows);
  d.v = M.get<double4_32a>(rows);
  d.xt = M.get<double4_32a>(rows);
  d.p = M.get<double4_32a>(rows);
  d.grad = M.get<double4_32a>(rows);
  d.cgrad = M.get<double4_32a>(rows);
  b->x0 = M.get<double4_32a>(rows);
  b->v0 = M.get<double4_32a>(rows);
  b->ex = M.get<double4_32a>(rows);
  b->ext = M.get<double4_32a>(rows);
  d.mass = M.get<double>(rows);
  d.fixed = M.get<uint8_t>(rows);
  d.vgel = M.get<int>(rows);
  d.tets = M.get<int4>(tets);
  d.Dminv = M.get<double>(9 * (size_t)tets);
  d.vol = M.get<double>(tets);
  d.tgel = M.get<int>(tets);
  d.tscr = M.get<double>((size_t)TS * tets);
  d.tscr32 = b->mixed ? M.get<float>((size_t)TS32 * tets) : nullptr;
  d.slice_off = M.get<int>(nslices + 1);
  d.colidx = M.get<int>(nbp);
  d.bp_row = M.get<int>(nbp);
  d.vals = b->mixed ? nullptr : M.get<double>(9 * (size_t)nbp);
  d.vals32 = b->mixed ? M.get<float>(9 * (size_t)nbp) : nullptr;
  d.ctr_ptr = M.get<int>(nbp + 1);
  d.ctr = M.get<int>(ctr.size());
  d.diag_pos = M.get<int>(rows);
  d.Minv = b->mixed ? nullptr : M.get<double>(9 * (size_t)rows);
  d.Minv32 = b->mixed ? M.get<float>(9 * (size_t)rows) : nullptr;
  d.r = M.get<double4_32a>(rows);
  d.u = M.get<double4_32a>(rows);
  d.w = M.get<double4_32a>(rows);
  d.pp = M.get<double4_32a>(rows);
  d.s = M.get<double4_32a>(rows);
  d.part = M.get<double>(8 * (size_t)cta_cap);
  d.czpart = M.get<double>(CZ_N * (size_t)cta_cap);
  d.czfac = M.get<double>(CZ_F * (size_t)cta_cap);
  d.pslice = M.get<double>(4 * (size_t)nslices);
  d.pool = M.get<PoolGel>(n);
  d.bar = M.get<unsigned>(n);
  d.sv = M.get<int>(nsv);
  d.st = M.get<int4>(nst);
  d.se = M.get<int2>(nse);
  d.se_len2 = M.get<double>(nse);
  d.q_gel = M.get<int>(nq);
  d.q_tp = M.get<int>(nq);
  d.iv_loc = M.get<double4_32a>(niv);
  d.iv_cur = M.get<double4_32a>(niv);
  d.iv_prev = M.get<double4_32a>(niv);
  d.it = M.get<int4>(nit);
  d.ie = M.get<int2>(nie);
  d.ie_len2 = M.get<double>(nie);
  d.iv_gel = M.get<int>(niv);
  d.it_gel = M.get<int>(nit);
  d.ie_gel = M.get<int>(nie);
  d.nit_total = nit;
  d.nie_total = nie;
  d.pbox = M.get<double4_32a>(2 * ((size_t)nit + niv + nie));
  d.hstart = M.get<int>(hb);
  d.hcount = M.get<int>(hb);
  d.max_hnb = max_hnb;
  d.qcount = M.get<int>(nq + 1);
  d.qoff = M.get<int>(nq + 1);
  d.qnear = M.get<int>(nq + 1);
  d.qnear_n = M.get<int>(4);
  d.err = M.get<int>(4);
  d.top = M.get<int4>(std::max<size_t>(top4.size(), 1));
  d.cwork_n = M.get<int>(4);
  d.c1_n = M.get<int>(4);
  d.vcomp = M.get<int8_t>(rows);
  d.n_ss = (int)b->ss_gel_h.size();
  d.ss_maxq = 0;
  for (int g : b->ss_gel_h) d.ss_maxq = std::max(d.ss_maxq, b->gi[g].nq);
  d.ss_gel = M.get<int>(std::max(d.n_ss, 1));
  d.ss_box = M.get<double>((size_t)std::max(d.n_ss, 1) * SS_MAXC * 6);
  d.ss_cnt = M.get<int>(3 * (size_t)std::max(d.n_ss, 1));
  d.ss_list = M.get<int>(std::max(nq, 1));
  d.ss_claim_cap = (int)std::min<long long>(std::max<long long>(claim_cap, 1), 1LL << 30);
  d.ss_claim = M.get<int>(d.ss_claim_cap);
  d.ss_nclaim = M.get<int>(4);
  b->pieces = M.get<int4>(b->npieces);
  b->gel_piece = M.get<int>(n + 1);
  b->part_e = M.get<double>(b->npieces);
  b->en_ticket = M.get<unsigned>(n);
  b->scan_tmp = M.get<int>((nq + 1023) / 1024 + 2);
  int* sg_buf = M.get<int>(nslices);
  if (M.failed) {
    M.release();
    delete b;
    return TX_ERR_OOM;
  }
  d.wait_limit = WAIT_LIMIT;
  d.wait_extra = 0;
  b->plan.slice_gel = sg_buf;
  b->plan.max_slices = 1;
  b->plan.ngroups = 0;
  // L2-sized parts measured slower than one launch over all gels on the 64-gel batch (the parts'
  // stragglers add up and every part re-reads its matrix once): off (0 = no split)
  b->l2_budget = 0.0;
  if (b->mixed) {  // FP32 PCG vectors live in the upper half of dedicated buffers
    d.u32 = (float4*)M.get<float4>(rows);
    d.w32 = (float4*)M.get<float4>(rows);
    d.pp32 = (float4*)M.get<float4>(rows);
    d.s32 = (float4*)M.get<float4>(rows);
    d.r32 = (float4*)M.get<float4>(rows);
    d.x32 = (float4*)M.get<float4>(rows);
  }
  host_alloc((void**)&b->gc_h, sizeof(GelCtl) * n);
  host_alloc((void**)&b->gv_h, sizeof(GelVar) * n);
  auto fail_create = [&](tx_status st) {
    b->pair_mem.release();
    b->hash_mem.release();
    M.release();
    if (b->gc_h) cudaFreeHost(b->gc_h);
    if (b->gv_h) cudaFreeHost(b->gv_h);
    cudaGetLastError();
    delete b;
    return st;
  };
  if (M.failed || !b->gc_h || !b->gv_h) return fail_create(TX_ERR_OOM);
  std::memset(b->gc_h, 0, sizeof(GelCtl) * n);
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  cudaError_t e = cudaSuccess;
  auto U = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = up(dst, src, bytes);
  };
  U((void*)d.gi, b->gi.data(), sizeof(GelInfo) * n);
  U((void*)d.gc, b->gc_h, sizeof(GelCtl) * n);
  U(d.X, X.data(), sizeof(double4_32a) * rows);
  U(d.x, X.data(), sizeof(double4_32a) * rows);
  U(d.xn, X.data(), sizeof(double4_32a) * rows);
  U(d.xt, X.data(), sizeof(double4_32a) * rows);
  U(d.mass, mass.data(), sizeof(double) * rows);
  U(d.fixed, fixed.data(), rows);
  U(d.vgel, vgel.data(), sizeof(int) * rows);
  U(d.tets, tet4.data(), sizeof(int4) * tets);
  U(d.Dminv, Dminv.data(), sizeof(double) * 9 * (size_t)tets);
  U(d.vol, vol.data(), sizeof(double) * tets);
  U(d.tgel, tgel.data(), sizeof(int) * tets);
  U(d.slice_off, slice_off.data(), sizeof(int) * (nslices + 1));
  U(d.colidx, colidx.data(), sizeof(int) * nbp);
  U(d.bp_row, bp_row.data(), sizeof(int) * nbp);
  U(d.ctr_ptr, ctr_cnt.data(), sizeof(int) * (nbp + 1));
  U(d.ctr, ctr.data(), sizeof(int) * ctr.size());
  U(d.diag_pos, diag_pos.data(), sizeof(int) * rows);
  U(d.sv, sv.data(), sizeof(int) * nsv);
  U(d.st, st4.data(), sizeof(int4) * nst);
  U(d.se, se2.data(), sizeof(int2) * nse);
  U(d.se_len2, se_len2.data(), sizeof(double) * nse);
  U(d.q_gel, q_gel.data(), sizeof(int) * nq);
  U(d.q_tp, q_tp.data(), sizeof(int) * nq);
  U(d.iv_loc, ivl.data(), sizeof(double4_32a) * niv);
  U(d.it, it4.data(), sizeof(int4) * nit);
  U(d.ie, ie2.data(), sizeof(int2) * nie);
  U(d.ie_len2, ie_len2.data(), sizeof(double) * nie);
  U(d.iv_gel, iv_gel.data(), sizeof(int) * niv);
  U(d.it_gel, it_gel.data(), sizeof(int) * nit);
  U(d.ie_gel, ie_gel.data(), sizeof(int) * nie);
  U(d.top, top4.data(), sizeof(int4) * top4.size());
  U(d.vcomp, vcomp.data(), rows);
  U(d.ss_gel, b->ss_gel_h.data(), sizeof(int) * b->ss_gel_h.size());
  U(b->pieces, b->pieces_h.data(), sizeof(int4) * b->npieces);
  U(b->gel_piece, b->gel_piece_h.data(), sizeof(int) * (n + 1));
  U((void*)b->plan.slice_gel, slice_gel.data(), sizeof(int) * nslices);
  if (e == cudaSuccess) e = cudaMemset(b->en_ticket, 0, sizeof(unsigned) * n);
  if (e == cudaSuccess) e = cudaMemset(d.v, 0, sizeof(double4_32a) * rows);
  if (e == cudaSuccess) e = cudaMemset(d.p, 0, sizeof(double4_32a) * rows);
  if (e == cudaSuccess) e = cudaMemset(d.gv, 0, sizeof(GelVar) * n);
  if (e == cudaSuccess) e = cudaMemset(d.err, 0, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMemset(d.ss_nclaim, 0, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMemset(d.qcount, 0, sizeof(int) * (nq + 1));
  if (e == cudaSuccess) e = cudaMemset(d.tscr, 0, sizeof(double) * TS * (size_t)std::max(tets, 1));
  if (e != cudaSuccess) {
    g_err = cudaGetErrorString(e);
    return fail_create(TX_ERR_CUDA);
  }
  tx_status s = alloc_pairs(b);
  if (s == TX_OK) s = alloc_hash(b);
  if (s == TX_OK && cudaDeviceSynchronize() != cudaSuccess) s = TX_ERR_CUDA;
  if (s != TX_OK) return fail_create(s);
  b->run.resize(n);
  for (int g = 0; g < n; ++g) b->run[g].kappa = b->gc_h[g].kappa = b->mesh[g].kappa;
  b->nnzb_real.assign(n, 0.0);
  b->nfree.assign(n, 0.0);
  for (int g = 0; g < n; ++g) {
    for (int i = 0; i < b->mesh[g].nv; ++i) {
      b->nnzb_real[g] += (double)b->mesh[g].adj[i].size();
      b->nfree[g] += b->mesh[g].fixed[i] ? 0.0 : 1.0;
    }
  }
  for (int g = 0; g < n; ++g) {
    std::memcpy(b->run[g].pose, b->mesh[g].pose0, sizeof(double) * 7);
    b->run[g].last.status = TX_OK;
  }
  *out = b;
  return TX_OK;
}

void fill_ctl(tx_batch* b, int g, int phase, const Task& t) {
  GelCtl& c = b->gc_h[g];
  const Mesh& m = b->mesh[g];
  c.phase = phase;
  c.kappa = b->run[g].kappa;
  c.h = t.dt;
  c.tol_p = m.prm.newton_tol * m.bbox * t.dt;
  const double far = std::max(m.prm.pcg_rel_tol_far, m.prm.pcg_rel_tol);
  c.eta2_near = m.prm.pcg_rel_tol * m.prm.pcg_rel_tol;
  c.eta2_far = far * far;
  for (int k = 0; k < 3; ++k) c.grav[k] = m.prm.gravity[k];
  quat_R(t.pb, c.R);
  quat_R(t.pa, c.Rp);
  for (int k = 0; k < 3; ++k) {
    c.t[k] = t.pb[4 + k];
    c.tp[k] = t.pa[4 + k];
  }
  c.attached = t.attached ? 1 : 0;
  if (t.attached) {
    quat_R(t.cb, c.Rc);
    quat_R(t.ca, c.Rcp);
    for (int k = 0; k < 3; ++k) {
      c.tc[k] = t.cb[4 + k];
      c.tcp[k] = t.ca[4 + k];
    }
  }
}

void finish_request(tx_batch* b, int g, tx_status s) {
  Run& R = b->run[g];
  R.acc.status = s;
  R.acc.kappa = R.kappa;
  R.last = R.acc;
  R.in_request = false;
  R.stack.clear();
  R.phase = PH_IDLE;
  b->gc_h[g].phase = PH_IDLE;
  b->done_queue.push_back(g);
}

// a failed request leaves the gel at the state it had when the request started
tx_status rollback(tx_batch* b, const std::vector<int>& gels) {
  for (int g : gels) {
    const GelInfo& G = b->gi[g];
    CK(cudaMemcpyAsync(b->d.x + G.v0, b->x0 + G.v0, sizeof(double4_32a) * G.ns * SLICE, cudaMemcpyDeviceToDevice, b->st));
    CK(cudaMemcpyAsync(b->d.v + G.v0, b->v0 + G.v0, sizeof(double4_32a) * G.ns * SLICE, cudaMemcpyDeviceToDevice, b->st));
    // the failed solve's direction must not seed the next solve's Galerkin start
    CK(cudaMemsetAsync(b->d.p + G.v0, 0, sizeof(double4_32a) * G.ns * SLICE, b->st));
    std::memcpy(b->run[g].pose, b->run[g].pose_req, sizeof(double) * 7);
    std::memcpy(b->run[g].case_pose, b->run[g].case_req, sizeof(double) * 7);
  }
  return TX_OK;
}

// ---------------------------------------------------------------- begin (admission of substeps)
tx_status do_begin(tx_batch* b, std::vector<int> set, int retries = 0) {
  if (set.empty()) return TX_OK;
  Dev& d = b->d;
  cudaStream_t st = b->st;
  // save the request start state of gels starting a new request
  for (int g = 0; g < b->n; ++g) b->gc_h[g].phase = (b->run[g].phase == PH_NEWTON) ? PH_PARK : b->gc_h[g].phase;
  for (int g : set) {
    const Task& t = b->run[g].stack.back();
    if (t.first) {
      const GelInfo& G = b->gi[g];
      CK(cudaMemcpyAsync(b->x0 + G.v0, d.x + G.v0, sizeof(double4_32a) * G.ns * SLICE, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(b->v0 + G.v0, d.v + G.v0, sizeof(double4_32a) * G.ns * SLICE, cudaMemcpyDeviceToDevice, st));
    }
    fill_ctl(b, g, PH_BEGIN, t);
  }
  tx_status s = upload_ctl(b);
  if (s != TX_OK) return s;
  prof_open(b, PR_BEGIN);
  launch_gel_op(d, PH_BEGIN, 3, st);
  launch_rows(4, d, PH_BEGIN, st);  // attached vertices to the case pose of the substep's end
  launch_indenter_pose(d, PH_BEGIN, d.niv_total, st);
  launch_hash_build(d, PH_BEGIN, 1, st);
  launch_query(d, PH_BEGIN, 4, st);
  launch_scan(d.qcount, d.qoff, d.nq, b->scan_tmp, st);
  launch_query(d, PH_BEGIN, 1 | 4, st);
  launch_pair_ranges(d, PH_BEGIN, 0, st);
  const int nss = launch_ss_pairs(d, PH_BEGIN, 0, st);
  const int accd_max = b->mesh[set[0]].prm.accd_max_iter;
  launch_accd(d, PH_BEGIN, 1, accd_max, st);
  launch_min_dist(d, PH_BEGIN, st);
  prof_close(b, 13 + nss);
  CK(cudaGetLastError());
  s = download_var(b);
  if (s != TX_OK) return s;
  std::vector<int> retry, start;
  bool regrow_pairs = false, regrow_hash = false;
  for (int g : set) {
    const GelVar& v = b->gv_h[g];
    Run& R = b->run[g];
    if (v.flags & 1) {
      for (int t = 0; t < NTAB; ++t) b->gi[g].hcap[t] = std::max(b->gi[g].hcap[t], 2 * v.hent[t] + 64);
      regrow_hash = true;
      retry.push_back(g);
      continue;
    }
    if (v.flags & 32) {
      b->gi[g].pcap = std::max(2 * b->gi[g].pcap, v.npair + v.npair / 2 + 64);
      regrow_pairs = true;
      retry.push_back(g);
      continue;
    }
    if (v.flags & 2) {
      std::vector<int> one{g};
      finish_request(b, g, TX_ERR_CCD_MAXIT);
      s = rollback(b, one);
      if (s != TX_OK) return s;
      continue;
    }
    const bool hit = (v.flags & 8) != 0;
    const double dmin = bitsd_host(v.dmin_bits);
    if (hit || !(dmin > 0.0)) {
      Task t = R.stack.back();
      if (t.depth >= b->mesh[g].prm.max_split_depth) {
        std::vector<int> one{g};
        finish_request(b, g, TX_ERR_INFEASIBLE);
        s = rollback(b, one);
        if (s != TX_OK) return s;
        continue;
      }
      R.stack.pop_back();
      Task a = t, c = t;
      double mid[7];
      pose_mid(t.pa, t.pb, mid);
      std::memcpy(a.pb, mid, sizeof(mid));
      std::memcpy(c.pa, mid, sizeof(mid));
      if (t.attached) {  // the case motion is halved with the indenter's
        pose_mid(t.ca, t.cb, mid);
        std::memcpy(a.cb, mid, sizeof(mid));
        std::memcpy(c.ca, mid, sizeof(mid));
      }
      a.dt = c.dt = 0.5 * t.dt;
      a.depth = c.depth = t.depth + 1;
      c.first = false;
      R.stack.push_back(c);
      R.stack.push_back(a);
      R.phase = PH_IDLE;
      b->gc_h[g].phase = PH_IDLE;
      continue;
    }
    start.push_back(g);
  }
  for (int g = 0; g < b->n; ++g)
    if (b->gc_h[g].phase == PH_BEGIN) b->gc_h[g].phase = PH_PARK;
  if (!start.empty()) {
    for (int g : start) b->gc_h[g].phase = PH_START;
    s = upload_ctl(b);
    if (s != TX_OK) return s;
    prof_open(b, PR_BEGIN);
    launch_rows(0, d, PH_START, st);         // x_n, predictor
    if (b->friction) launch_fric_setup(d, PH_START, st);  // lagged friction at the substep start
    launch_hash_build(d, PH_START, 0, st);   // static tables at the target pose
    launch_energy(d, PH_START, b->pieces, b->npieces, b->gel_piece, b->part_e, b->en_ticket, 0, st);
    prof_close(b, b->friction ? 5 : 4);
    CK(cudaGetLastError());
    for (int g : start) {
      Run& R = b->run[g];
      R.phase = PH_NEWTON;
      R.newton_sub = 0;
      R.acc.substeps += 1;
    }
  }
  for (int g = 0; g < b->n; ++g) {
    if (b->run[g].phase == PH_NEWTON) b->gc_h[g].phase = PH_NEWTON;
    else if (b->gc_h[g].phase == PH_PARK || b->gc_h[g].phase == PH_START) b->gc_h[g].phase = PH_IDLE;
  }
  s = upload_ctl(b);
  if (s != TX_OK) return s;
  if (!retry.empty()) {
    if (retries > 4) {
      for (int g : retry) finish_request(b, g, TX_ERR_OOM);
      return TX_OK;
    }
    if (regrow_pairs) s = alloc_pairs(b);
    if (s == TX_OK && regrow_hash) s = alloc_hash(b);
    if (s == TX_ERR_OOM) {  // the gels that needed more room fail their request; the rest go on
      for (int g : retry) finish_request(b, g, TX_ERR_OOM);
      return rollback(b, retry);
    }
    if (s != TX_OK) return s;
    return do_begin(b, retry, retries + 1);
  }
  return TX_OK;
}

}  // namespace

namespace {

// ---------------------------------------------------------------- one Newton iteration
// The part after the PCG: candidates along p, ACCD, line search.  Runs for the gels whose
// control phase is PH_NEWTON.
// The part after the PCG, launch side: candidates along p, ACCD, the first line-search trial.
void post_pcg_launch(tx_batch* b, int accd_max) {
  Dev& d = b->d;
  cudaStream_t st = b->st;
  prof_open(b, PR_QUERY);
  launch_query(d, PH_NEWTON, 2 | 8, st);
  launch_scan(d.qcount, d.qoff, d.nq, b->scan_tmp, st);
  launch_query(d, PH_NEWTON, 1 | 2 | 8, st);
  launch_pair_ranges(d, PH_NEWTON, 1, st);
  const int nss = launch_ss_pairs(d, PH_NEWTON, 2 | 8, st);
  prof_close(b, 7 + nss);
  prof_open(b, PR_ACCD);
  launch_accd(d, PH_NEWTON, 0, accd_max, st);
  launch_gel_op(d, PH_NEWTON, 2, st);
  prof_close(b, 2);
  // first trial; usually accepted
  prof_open(b, PR_LS);
  launch_energy(d, PH_NEWTON, b->pieces, b->npieces, b->gel_piece, b->part_e, b->en_ticket, 1, st);
  launch_rows(1, d, PH_NEWTON, st);
  launch_gel_op(d, PH_NEWTON, 5, st);
  prof_close(b, 4);
}

// ... and the host side: read the per-gel state, run further halvings while gels search.
tx_status post_pcg_finish(tx_batch* b) {
  Dev& d = b->d;
  cudaStream_t st = b->st;
  int ls_max = 1;
  for (int g = 0; g < b->n; ++g)
    if (b->gc_h[g].phase == PH_NEWTON) ls_max = std::max(ls_max, b->mesh[g].prm.ls_max_halvings);
  CK(cudaGetLastError());
  tx_status s = download_var(b);
  if (s != TX_OK) return s;
  for (int trial = 1; trial <= ls_max + 1; ++trial) {
    bool searching = false;
    for (int g = 0; g < b->n; ++g)
      if (b->gc_h[g].phase == PH_NEWTON && !b->gv_h[g].converged && b->gv_h[g].ls_state == 0) searching = true;
    if (!searching) break;
    prof_open(b, PR_LS);
    for (int k = 0; k < 4; ++k) {  // a few halvings per host round trip
      launch_energy(d, PH_NEWTON, b->pieces, b->npieces, b->gel_piece, b->part_e, b->en_ticket, 1, st);
      launch_rows(1, d, PH_NEWTON, st);
      launch_gel_op(d, PH_NEWTON, 5, st);
    }
    prof_close(b, 16);
    CK(cudaGetLastError());
    s = download_var(b);
    if (s != TX_OK) return s;
  }
  return TX_OK;
}

int newton_accd_max(tx_batch* b) {
  int accd_max = 1;
  for (int g = 0; g < b->n; ++g)
    if (b->gc_h[g].phase == PH_NEWTON) accd_max = std::max(accd_max, b->mesh[g].prm.accd_max_iter);
  return accd_max;
}

tx_status post_pcg(tx_batch* b) {
  post_pcg_launch(b, newton_accd_max(b));
  return post_pcg_finish(b);
}

tx_status finalize_substeps(tx_batch* b, const std::vector<int>& fin) {
  if (fin.empty()) return TX_OK;
  Dev& d = b->d;
  for (int g = 0; g < b->n; ++g) b->gc_h[g].phase = PH_PARK;
  for (int g : fin) b->gc_h[g].phase = PH_FINAL;
  tx_status s = upload_ctl(b);
  if (s != TX_OK) return s;
  prof_open(b, PR_FINAL);
  launch_rows(2, d, PH_FINAL, b->st);      // v = (x - x_n) / h
  launch_gel_op(d, PH_FINAL, 4, b->st);    // distance minimum at the final state
  launch_min_dist(d, PH_FINAL, b->st);
  prof_close(b, 3);
  CK(cudaGetLastError());
  s = download_var(b);
  if (s != TX_OK) return s;
  for (int g : fin) {
    Run& R = b->run[g];
    const GelVar& v = b->gv_h[g];
    Task t = R.stack.back();
    R.stack.pop_back();
    R.acc.newton_iters += R.newton_sub;
    R.acc.ls_halvings += v.ls_total;
    R.acc.soft_pairs_cut += v.ss_cut;
    R.acc.energy = v.E_cur;
    R.acc.active_pairs = v.active_pairs;
    R.acc.candidate_pairs = v.npair;
    R.acc.min_distance = bitsd_host(v.dmin_bits);
    for (int c = 0; c < 3; ++c) R.acc.contact_force[c] = v.fc[c];
    std::memcpy(R.pose, t.pb, sizeof(double) * 7);
    if (t.attached) std::memcpy(R.case_pose, t.cb, sizeof(double) * 7);
    R.phase = PH_IDLE;
    if (R.stack.empty()) {
      // adaptive barrier stiffness (IPC's kappa update at step granularity: the indenter is placed
      // before each solve, so pairs close in between steps): a step that ended nearer than
      // kappa_adapt_dmin, and nearer than the step before, doubles kappa for the next steps
      const tx_params& P = b->mesh[g].prm;
      if (P.kappa_adapt_max > 0.0) {
        const double dfin = R.acc.min_distance, cap = P.kappa_adapt_max * b->mesh[g].kappa;
        if (dfin < P.kappa_adapt_dmin && dfin < R.dmin_last && R.kappa < cap) R.kappa = std::min(2.0 * R.kappa, cap);
        R.dmin_last = dfin;
      }
      finish_request(b, g, TX_OK);
    }
  }
  for (int g = 0; g < b->n; ++g) b->gc_h[g].phase = b->run[g].phase == PH_NEWTON ? PH_NEWTON : PH_IDLE;
  return upload_ctl(b);
}

// PCG partition for the gels of `set` (in index order), rebuilt only when the set changes.
// Groups: a gel with more than spc slices is spread over ceil(ns / spc) CTAs; runs of small gels
// (index span <= 64, slice span <= spc) share one CTA.  spc grows from its minimum until the CTAs
// fit co-resident on the device; the resident kernels are used when every CTA has at most a
// slice per warp and they fit, else the streaming kernels.
// device arrays for `np` plan parts (each: CTA ranges, CTA groups, groups)
tx_status ensure_plan_parts(tx_batch* b, int np) {
  if (np <= b->plan_parts_cap) return TX_OK;
  CK(cudaStreamSynchronize(b->st));
  b->plan_mem.release();
  const int cap = std::max(np, 2 * b->plan_parts_cap);
  const size_t C = (size_t)b->pcg_cta_cap, G = (size_t)b->n;
  int2* rng = b->plan_mem.get<int2>(C * cap);
  int* cg = b->plan_mem.get<int>(C * cap);
  int4* gr = b->plan_mem.get<int4>(G * cap);
  if (b->plan_mem.failed) return TX_ERR_OOM;
  b->parts.resize(cap);
  for (int k = 0; k < cap; ++k) {
    PcgPlan& P = b->parts[k].plan;
    P = b->plan;
    P.cta_rng = rng + C * k;
    P.cta_grp = cg + C * k;
    P.grp = gr + G * k;
  }
  b->plan_parts_cap = cap;
  return TX_OK;
}

// PCG partition of one subset of the gels (in index order) into the given part.
// Groups: a gel with more than spc slices is spread over ceil(ns / spc) CTAs; runs of small gels
// (index span <= 64, slice span <= spc) share one CTA.  spc grows from its minimum until the CTAs
// fit co-resident on the device; the resident kernels are used when every CTA has at most a
// slice per warp and they fit, else the streaming kernels.
tx_status plan_part(tx_batch* b, const std::vector<int>& set, int spc0, tx_batch::PlanPart& part) {
  const int nsm = b->nsm;
  int spc = std::max(spc0, 1), max_slices = 1;
  std::vector<int2>& rng = b->plan_rng_h;
  std::vector<int>& cgrp = b->plan_grp_of_h;
  std::vector<int4>& grp = b->plan_grp_h;
  bool res = false;
  for (int attempt = 0;; ++attempt) {
    rng.clear();
    cgrp.clear();
    grp.clear();
    size_t k = 0;
    while (k < set.size()) {
      const int g = set[k];
      const GelInfo& G = b->gi[g];
      if (G.ns > spc) {
        const int nc = (G.ns + spc - 1) / spc;
        grp.push_back(make_int4((int)rng.size(), nc, g, 1));
        for (int q = 0; q < nc; ++q) {
          rng.push_back(make_int2(G.s0 + (int)((long long)q * G.ns / nc), G.s0 + (int)((long long)(q + 1) * G.ns / nc)));
          cgrp.push_back((int)grp.size() - 1);
        }
        ++k;
        continue;
      }
      size_t e = k + 1;  // pack the following small gels while the spans allow
      while (e < set.size()) {
        const GelInfo& H = b->gi[set[e]];
        if (H.ns > spc || set[e] - g >= PCG_MAXG_HOST || H.s0 + H.ns - G.s0 > spc) break;
        ++e;
      }
      const GelInfo& L = b->gi[set[e - 1]];
      grp.push_back(make_int4((int)rng.size(), 1, g, set[e - 1] - g + 1));
      rng.push_back(make_int2(G.s0, L.s0 + L.ns));
      cgrp.push_back((int)grp.size() - 1);
      k = e;
    }
    const int nctas = (int)rng.size();
    max_slices = 1;
    int max_nc = 0;
    for (const int2& r : rng) max_slices = std::max(max_slices, r.y - r.x);
    for (const int4& q : grp) max_nc = std::max(max_nc, q.y);
    const int occ_res = pcg_res_ctas_per_sm(b->mixed, max_slices, b->pcg_wmax);
    // a multi-CTA group reduces three quantities at once, one warp each: two slice warps and the
    // control warp at least
    res = b->plan_mode == 0 && occ_res > 0 && nctas <= nsm * occ_res && max_nc <= PCG_RES_MAXNC &&
          (max_nc == 1 || max_slices >= 2);
    const int occ = std::max(1, pcg_max_ctas_per_sm(max_slices));
    if (res || (nctas <= nsm * occ && nctas <= b->pcg_cta_cap)) {
      // one FP64 gel too large for the resident kernels, at the default split: fewer, fuller CTAs
      // (measured on the 41x51x9 gel + 20^3 soft ball, 26,819 rows: 93.4 / 73.6 / 74.2 / 109.1 ms
      // per step at 4 / 6 / 8 / 12 slices per CTA)
      if (!res && !b->mixed && set.size() == 1 && spc0 == PCG_SLICES_FP64 && spc < PCG_SLICES_FP64_LARGE &&
          b->plan_mode != 2) {
        spc = PCG_SLICES_FP64_LARGE;
        continue;
      }
      break;
    }
    if (attempt > 400) {
      set_last_error("PCG partition does not fit the device");
      return TX_ERR_ARG;
    }
    spc = spc + spc / 4 + 1;
  }
  const int nctas = (int)rng.size();
  cudaStream_t st = b->st;
  // pageable sources: the copies take the data when enqueued, the vectors can be reused at once.
  // (the pooled kernels need no CTA plan)
  // the pooled form (streaming, many gels or asked for) needs no CTA plan
  part.pool_on = !res && (b->plan_mode == 2 || (b->plan_mode == 0 && (int)set.size() >= PCG_POOL_MIN_GELS));
  if (!part.pool_on) {
    if (nctas > b->pcg_cta_cap) {
      set_last_error("PCG partition does not fit the device");
      return TX_ERR_ARG;
    }
    CK(cudaMemcpyAsync((void*)part.plan.cta_rng, rng.data(), sizeof(int2) * nctas, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync((void*)part.plan.cta_grp, cgrp.data(), sizeof(int) * nctas, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync((void*)part.plan.grp, grp.data(), sizeof(int4) * grp.size(), cudaMemcpyHostToDevice, st));
  }
  part.plan.max_slices = max_slices;
  part.plan.ngroups = (int)grp.size();
  part.nctas = nctas;
  part.res = res;
  if (part.pool_on) {  // the pooled kernels over the set's gel range, one CTA per SM
    part.pool.g0 = set.front();
    part.pool.ng = set.back() - set.front() + 1;
    long long tot = 0;  // slices of the gel range: bounds every CTA's share
    for (int g = part.pool.g0; g < part.pool.g0 + part.pool.ng; ++g) tot += b->gi[g].ns;
    part.pool.cap = (int)(tot / nsm) + 2;  // one CTA per SM (checked below)
    const int occp = pcg_pool_ctas_per_sm(part.pool);
    if (occp < 1) {
      set_last_error("pooled PCG does not fit the device");
      return TX_ERR_ARG;
    }
    part.pool_nctas = nsm;
  }
  return TX_OK;
}

// The round's PCG plan for the gels of `set`, rebuilt only when the set changes.  With a nonzero
// l2_budget, mixed precision splits the set into consecutive subsets whose FP32 blocks and Krylov
// vectors fit in that budget (one PCG launch each); by default one launch covers the whole set.
tx_status prepare_pcg_plan(tx_batch* b, const std::vector<int>& set) {
  int total = 0;
  for (int g : set) total += b->gi[g].ns;
  int spc0 = b->pcg_spc_min;
  b->tune_key = -1;
  if (b->tune_on) {
    const long long key = (long long)std::min<size_t>(set.size(), 64) * 1000 +
                          (long long)std::lround(2.0 * std::log2(std::max(total, 1)));
    tx_batch::Tune& T = b->tune[key];
    if (T.best < 0) {
      spc0 = TUNE_SPC[T.idx];
      b->tune_key = key;
    } else {
      spc0 = TUNE_SPC[T.best];
    }
  }
  if (set == b->plan_key && b->nctas > 0 && spc0 == b->plan_spc) return TX_OK;
  std::vector<std::vector<int>> subsets(1);
  double acc = 0.0;
  for (int g : set) {
    const double bytes = b->mixed ? 40.0 * b->nbp_gel[g] + 160.0 * b->gi[g].nv : 0.0;
    if (b->mixed && b->l2_budget > 0.0 && !subsets.back().empty() && acc + bytes > b->l2_budget) {
      subsets.emplace_back();
      acc = 0.0;
    }
    subsets.back().push_back(g);
    acc += bytes;
  }
  tx_status s = ensure_plan_parts(b, (int)subsets.size());
  if (s != TX_OK) return s;
  for (size_t k = 0; k < subsets.size(); ++k) {
    s = plan_part(b, subsets[k], spc0, b->parts[k]);
    if (s != TX_OK) return s;
  }
  b->nparts = (int)subsets.size();
  b->nctas = b->parts[0].nctas;
  b->plan_key = set;
  b->plan_spc = spc0;
  b->plan_version += 1;
  return TX_OK;
}

// after the round's synchronisation: the PCG time per iteration of the candidate being tried
void tune_record(tx_batch* b, const std::vector<int>& set) {
  if (b->tune_key < 0) return;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, b->tev0, b->tev1) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  int it = 1;
  for (int g : set) it = std::max(it, b->gv_h[g].pcg_it);
  tx_batch::Tune& T = b->tune[b->tune_key];
  T.us[T.idx] = 1e3 * ms / it;
  if (++T.idx == TUNE_N) {
    T.best = 0;
    for (int k = 1; k < TUNE_N; ++k)
      if (T.us[k] < T.us[T.best]) T.best = k;
  }
  b->tune_key = -1;
}

void tune_event(tx_batch* b, cudaEvent_t& e) {
  if (!e) cudaEventCreate(&e);
  if (b->capturing)
    cudaEventRecordWithFlags(e, b->st, cudaEventRecordExternal);
  else
    cudaEventRecord(e, b->st);
}

// Launches of one Newton iteration for the gels in PH_NEWTON, up to the first line-search trial.
tx_status newton_launches(tx_batch* b, int pcg_max, int refine, int accd_max) {
  Dev& d = b->d;
  cudaStream_t st = b->st;
  launch_gel_op(d, PH_NEWTON, 0, st);
  // the contact terms (latency-bound: a thread per candidate pair, a warp per pair Hessian) on the
  // side stream, beside the elastic assembly; the gather waits for them.  Only for a single gel
  // in mixed precision: the FP64 elastic assembly, or a batch's, leaves no FP64 issue slots to the
  // contact kernels and the overlap measured no gain (FP64) or a loss (64-gel batches).
  cudaStream_t cs = st;
  if (b->side_ok && b->mixed && b->n == 1) {
    CK(cudaEventRecord(b->ev_fork, st));
    CK(cudaStreamWaitEvent(b->st2, b->ev_fork, 0));
    cs = b->st2;
  }
  prof_open(b, PR_CONTACT, cs);
  if (d.n_ss > 0) launch_ss_reset(d, cs);  // the cross-body blocks of the last assembly give their slots back
  launch_contact_compute(d, PH_NEWTON, b->mixed, cs);
  if (b->friction) launch_fric(d, PH_NEWTON, 0, b->mixed, cs);  // friction gradient and force
  prof_close(b, (b->friction ? 3 : 2) + (d.n_ss > 0 ? 1 : 0), cs);
  if (cs != st) CK(cudaEventRecord(b->ev_join, cs));
  prof_open(b, PR_TET);
  launch_tet_assemble(d, PH_NEWTON, b->mixed, st);
  prof_close(b, 1);
  if (cs != st) CK(cudaStreamWaitEvent(st, b->ev_join, 0));
  prof_open(b, PR_GATHER);
  launch_gather(d, PH_NEWTON, b->nbp, b->mixed, st);
  launch_contact_merge(d, b->mixed, st);
  if (b->friction) launch_fric(d, PH_NEWTON, 1, b->mixed, st);  // friction blocks into the matrix
  prof_close(b, b->friction ? 3 : 2);
  prof_open(b, PR_PRECOND);
  launch_precond(d, PH_NEWTON, b->mixed, st);
  prof_close(b, 1);
  if (b->tune_key >= 0) tune_event(b, b->tev0);
  prof_open(b, PR_PCG);
  int npcg = b->nparts;
  for (int k = 0; k < b->nparts; ++k) {
    const tx_batch::PlanPart& P = b->parts[k];
    CK(cudaMemsetAsync(d.bar, 0, sizeof(unsigned) * P.plan.ngroups, st));
    if (b->mixed) {
      if (P.res)
        CK(launch_pcg_res(d, PH_NEWTON, P.plan, P.nctas, true, pcg_max, refine, b->pcg_wmax, st));
      else
        CK(P.pool_on ? launch_pcg_pool(d, PH_NEWTON, P.pool, P.pool_nctas, true, pcg_max, refine, st)
                     : launch_pcg_mixed(d, PH_NEWTON, P.plan, P.nctas, pcg_max, refine, st));
    } else {
      if (P.res) {
        CK(launch_pcg_res(d, PH_NEWTON, P.plan, P.nctas, false, pcg_max, 0, b->pcg_wmax, st));
      } else {
        if (!P.pool_on && b->has_cbody) {  // the coarse space of a free body (k_pcg64)
          launch_pcg_cz_setup(d, PH_NEWTON, P.plan, P.nctas, st);
          npcg += 2;
        }
        CK(P.pool_on ? launch_pcg_pool(d, PH_NEWTON, P.pool, P.pool_nctas, false, pcg_max, 0, st)
                     : launch_pcg64(d, PH_NEWTON, P.plan, P.nctas, pcg_max, st));
      }
    }
  }
  prof_close(b, npcg);
  if (b->tune_key >= 0) tune_event(b, b->tev1);
  launch_gel_op(d, PH_NEWTON, 1, st);
  post_pcg_launch(b, accd_max);
  return TX_OK;
}

void drop_newton_graph(tx_batch* b) {
  auto& G = b->graph;
  if (G.exec) cudaGraphExecDestroy(G.exec);
  G.exec = nullptr;
  for (auto& p : G.prof_pairs) {
    b->prof.pool.push_back(p.a);
    b->prof.pool.push_back(p.b);
  }
  G.prof_pairs.clear();
  G.key.clear();
}

// The iteration's launches as a CUDA graph: captured on the first iteration of a given set of
// gels (and whenever anything its kernels were captured with changes: the PCG partition, device
// buffers, solver parameters, profiling), then replayed with one launch.  Falls back to plain
// launches for good if capture is refused (TXG_NO_GRAPHS=1 also disables it).
tx_status run_newton_launches(tx_batch* b, const std::vector<int>& set, int pcg_max, int refine,
                              int accd_max) {
  if (!b->side_ok && !b->st2) {  // side stream of the contact assembly (plain sequence if refused)
    b->side_ok = cudaStreamCreateWithFlags(&b->st2, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) == cudaSuccess;
    if (!b->side_ok) cudaGetLastError();
  }
  if (b->graphs < 0) {
    const char* e = std::getenv("TXG_NO_GRAPHS");
    b->graphs = (e && e[0] == '1') ? 0 : 1;
    // capture needs a stream of its own (the caller's may be the legacy default stream)
    if (b->graphs && (cudaStreamCreateWithFlags(&b->gst, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaEventCreateWithFlags(&b->gev_in, cudaEventDisableTiming) != cudaSuccess ||
                      cudaEventCreateWithFlags(&b->gev_out, cudaEventDisableTiming) != cudaSuccess)) {
      cudaGetLastError();
      b->graphs = 0;
    }
  }
  if (b->graphs == 0) return newton_launches(b, pcg_max, refine, accd_max);
  auto& G = b->graph;
  const bool same = G.exec && G.key == set && G.nctas == b->nctas && !G.tune &&
                    b->tune_key < 0 &&
                    G.prof == b->prof.on && G.pcg_max == pcg_max && G.refine == refine &&
                    G.accd_max == accd_max && std::memcmp(&G.dev, &b->d, sizeof(Dev)) == 0 &&
                    G.plan_version == b->plan_version;
  if (!same) {
    drop_newton_graph(b);
    const long long l0 = g_launch_count.load();
    long long pl0[PR_N];
    std::memcpy(pl0, b->prof.launches, sizeof(pl0));
    const size_t pend0 = b->prof.pending.size();
    cudaGraph_t graph = nullptr;
    cudaStream_t user = b->st;
    b->st = b->gst;  // every launch of the iteration goes to the capture stream
    bool ok = cudaStreamBeginCapture(b->gst, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    std::string why;
    if (ok) {
      b->capturing = true;
      const tx_status s = newton_launches(b, pcg_max, refine, accd_max);
      b->capturing = false;
      if (s != TX_OK) why = g_err;
      const cudaError_t e = cudaStreamEndCapture(b->gst, &graph);
      if (e != cudaSuccess && why.empty()) why = std::string("end capture: ") + cudaGetErrorString(e);
      ok = e == cudaSuccess && s == TX_OK && graph;
    } else {
      why = "begin capture refused";
    }
    b->st = user;
    if (ok) {
      const cudaError_t e = cudaGraphInstantiate(&G.exec, graph, 0);
      if (e != cudaSuccess) why = std::string("instantiate: ") + cudaGetErrorString(e);
      ok = e == cudaSuccess;
    }
    if (!ok) g_err = "Newton-iteration graph not used (" + why + "); plain launches";
    if (graph) cudaGraphDestroy(graph);
    // nothing ran during the capture: undo its launch and profile bookkeeping
    const long long nl = g_launch_count.load() - l0;
    count_launch((int)-nl);
    long long dl[PR_N];
    for (int k = 0; k < PR_N; ++k) {
      dl[k] = b->prof.launches[k] - pl0[k];
      b->prof.launches[k] = pl0[k];
    }
    std::vector<Prof::Pending> pairs(b->prof.pending.begin() + pend0, b->prof.pending.end());
    b->prof.pending.resize(pend0);
    cudaGetLastError();
    if (!ok) {
      if (G.exec) cudaGraphExecDestroy(G.exec);
      G.exec = nullptr;
      for (auto& p : pairs) {
        b->prof.pool.push_back(p.a);
        b->prof.pool.push_back(p.b);
      }
      b->graphs = 0;
      return newton_launches(b, pcg_max, refine, accd_max);
    }
    for (auto& p : pairs) p.graph = true;
    G.prof_pairs = pairs;
    G.key = set;
    G.dev = b->d;
    G.plan_version = b->plan_version;
    G.nctas = b->nctas;
    G.prof = b->prof.on;
    G.tune = b->tune_key >= 0;
    G.pcg_max = pcg_max;
    G.refine = refine;
    G.accd_max = accd_max;
    G.launches = nl;
    std::memcpy(G.phase_launches, dl, sizeof(dl));
  }
  CK(cudaEventRecord(b->gev_in, b->st));
  CK(cudaStreamWaitEvent(b->gst, b->gev_in, 0));
  CK(cudaGraphLaunch(G.exec, b->gst));
  CK(cudaEventRecord(b->gev_out, b->gst));
  CK(cudaStreamWaitEvent(b->st, b->gev_out, 0));
  count_launch((int)G.launches);
  for (int k = 0; k < PR_N; ++k) b->prof.launches[k] += G.phase_launches[k];
  for (const auto& p : G.prof_pairs) b->prof.pending.push_back(p);
  return TX_OK;
}

tx_status do_newton(tx_batch* b) {
  std::vector<int> set;
  for (int g = 0; g < b->n; ++g) {
    b->gc_h[g].phase = b->run[g].phase == PH_NEWTON ? PH_NEWTON : PH_IDLE;
    if (b->run[g].phase == PH_NEWTON) set.push_back(g);
  }
  if (set.empty()) return TX_OK;
  Dev& d = b->d;
  cudaStream_t st = b->st;
  tx_status s = upload_ctl(b);
  if (s != TX_OK) return s;
  int pcg_max = 1;
  for (int g : set) pcg_max = std::max(pcg_max, b->mesh[g].prm.pcg_max_iter);
  int refine = 1;
  for (int g : set) refine = std::max(refine, b->mesh[g].prm.refine_max);
  s = prepare_pcg_plan(b, set);
  if (s != TX_OK) return s;
  const int accd_max = newton_accd_max(b);
  // fault-injection test hook: this iteration's PCG barriers wait for an arrival that never comes
  // (with a short limit), so every wait gives up and the step reports a device timeout
  struct WaitGuard {
    Dev& d;
    ~WaitGuard() {
      d.wait_extra = 0;
      d.wait_limit = WAIT_LIMIT;
    }
  } wait_guard{d};
  for (int k = g_inject_wait.load(); k > 0; k = g_inject_wait.load())
    if (g_inject_wait.compare_exchange_weak(k, k - 1)) {
      d.wait_extra = 1;
      d.wait_limit = WAIT_LIMIT_INJECTED;
      break;
    }
  s = run_newton_launches(b, set, pcg_max, refine, accd_max);
  if (s != TX_OK) return s;
  for (int k = 0; k < b->nparts; ++k) {
    (b->parts[k].res ? b->prof.pcg_res : b->prof.pcg_stream) += 1;
    if (b->parts[k].pool_on) b->prof.pcg_pool += 1;
  }
  s = post_pcg_finish(b);
  if (s != TX_OK) return s;
  tune_record(b, set);
  int derr = 0;
  CK(cudaMemcpy(&derr, d.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (derr) {
    CK(cudaMemset(d.err, 0, sizeof(int)));
    std::vector<int> fail;
    for (int g : set) {
      finish_request(b, g, TX_ERR_DEVICE_TIMEOUT);
      fail.push_back(g);
    }
    return rollback(b, fail);
  }
  // pair-segment overflow: grow and redo the line-search part for those gels
  for (int attempt = 0; attempt < 4; ++attempt) {
    std::vector<int> over;
    for (int g : set)
      if (b->gv_h[g].ls_state == 4) over.push_back(g);
    if (over.empty()) break;
    for (int g : over) b->gi[g].pcap = std::max(2 * b->gi[g].pcap, b->gv_h[g].npair + b->gv_h[g].npair / 2 + 64);
    s = alloc_pairs(b);
    if (s == TX_ERR_OOM) {
      for (int g : over) finish_request(b, g, TX_ERR_OOM);
      s = rollback(b, over);
      if (s != TX_OK) return s;
      break;
    }
    if (s != TX_OK) return s;
    for (int g = 0; g < b->n; ++g) b->gc_h[g].phase = PH_PARK;
    for (int g : over) b->gc_h[g].phase = PH_NEWTON;
    s = upload_ctl(b);
    if (s != TX_OK) return s;
    launch_gel_op(d, PH_NEWTON, 6, st);  // clear the overflow flag
    s = post_pcg(b);
    if (s != TX_OK) return s;
  }
  std::vector<int> fin, fail;
  if (b->prof.on) {
    // the solvers' Galerkin start: one SpMV (FP64 arithmetic), three dot products and two updates
    // per solve
    for (int g : set) {
      const double it = b->gv_h[g].pcg_it;
      const GelInfo& G = b->gi[g];
      b->prof.flops[PR_PCG] += 18.0 * b->nnzb_real[g] + 30.0 * b->nfree[g];
      b->prof.bytes[PR_PCG] += (b->mixed ? 40.0 : 76.0) * b->nnzb_real[g] + 96.0 * G.nv;
      // per PCG iteration and row: SpMV 18 flops per 3x3 block, preconditioner 18, four
      // axpys 24, three dot products 18; mixed precision adds one FP64 residual SpMV per round
      const double rounds = b->mixed ? b->gv_h[g].rounds : 0.0;
      b->prof.flops[PR_PCG] += it * (18.0 * b->nnzb_real[g] + 60.0 * b->nfree[g]) + rounds * 18.0 * b->nnzb_real[g];
      // algorithmic bytes of a streaming iteration: block values + column index per block, and
      // per row the preconditioner block, six vectors read and five written (FP64: 72 + 4 B per
      // block, 72 + 11 x 32 B per row; mixed: 36 + 4 B per block, 36 + 11 x 16 B per row); a
      // refinement round adds the FP64 residual SpMV (FP32 blocks, three FP64 row vectors)
      if (b->mixed)
        b->prof.bytes[PR_PCG] += it * (40.0 * b->nnzb_real[g] + 212.0 * G.nv) +
                                 rounds * (40.0 * b->nnzb_real[g] + 96.0 * G.nv);
      else
        b->prof.bytes[PR_PCG] += it * (76.0 * b->nnzb_real[g] + 424.0 * G.nv);
      b->prof.pcg_iters += b->gv_h[g].pcg_it;
      b->prof.newton_iters += 1;
      b->prof.flops[PR_TET] += 0.0;
    }
  }
  for (int g : set) {
    Run& R = b->run[g];
    if (!R.in_request) continue;  // already finished (out of memory while growing its pair segment)
    const GelVar& v = b->gv_h[g];
    R.acc.pcg_iters += v.pcg_it;
    R.acc.refine_rounds += v.rounds;
    if (v.converged || v.ls_state == 6) {
      fin.push_back(g);
    } else if (v.ls_state == 2) {
      finish_request(b, g, TX_ERR_LINESEARCH);
      fail.push_back(g);
    } else if (v.ls_state == 3) {
      R.newton_sub += 1;
      if (R.newton_sub >= b->mesh[g].prm.newton_max_iter) {
        finish_request(b, g, TX_ERR_NEWTON_MAXIT);
        fail.push_back(g);
      }
    } else {
      finish_request(b, g, TX_ERR_OOM);
      fail.push_back(g);
    }
  }
  s = rollback(b, fail);
  if (s != TX_OK) return s;
  return finalize_substeps(b, fin);
}

tx_status advance(tx_batch* b) {
  std::vector<int> begin;
  for (int g = 0; g < b->n; ++g) {
    Run& R = b->run[g];
    if (R.in_request && R.phase == PH_IDLE && !R.stack.empty()) begin.push_back(g);
  }
  tx_status s = do_begin(b, begin);
  if (s != TX_OK) return s;
  return do_newton(b);
}

bool valid_pose(const double p[7]) {
  double qn = 0.0;
  for (int k = 0; k < 7; ++k)
    if (!std::isfinite(p[k])) return false;
  for (int k = 0; k < 4; ++k) qn += p[k] * p[k];
  return qn > 0.0;
}

tx_status submit_one(tx_batch* b, int g, const double pose[7], double dt, const double* case_pose = nullptr) {
  if (g < 0 || g >= b->n || !pose || !(dt > 0.0) || !std::isfinite(dt)) return TX_ERR_ARG;
  if (!valid_pose(pose) || (case_pose && !valid_pose(case_pose))) return TX_ERR_ARG;
  Run& R = b->run[g];
  if (R.in_request) return TX_ERR_ARG;
  R.in_request = true;
  R.acc = tx_step_stats{};
  R.newton_sub = 0;
  std::memcpy(R.pose_req, R.pose, sizeof(double) * 7);
  std::memcpy(R.case_req, R.case_pose, sizeof(double) * 7);
  Task t;
  std::memcpy(t.pa, R.pose, sizeof(double) * 7);
  std::memcpy(t.pb, pose, sizeof(double) * 7);
  t.attached = case_pose != nullptr;
  std::memcpy(t.ca, R.case_pose, sizeof(double) * 7);
  std::memcpy(t.cb, case_pose ? case_pose : R.case_pose, sizeof(double) * 7);
  t.dt = dt;
  t.depth = 0;
  t.first = true;
  R.stack.clear();
  R.stack.push_back(t);
  return TX_OK;
}

tx_status copy_rows_out(tx_batch* b, int g, const double4_32a* src, double* dst, bool device_ptrs) {
  const GelInfo& G = b->gi[g];
  CK(cudaMemcpy2DAsync(dst, 3 * sizeof(double), src + G.v0, sizeof(double4_32a), 3 * sizeof(double), G.nv,
                       device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->st));
  if (!device_ptrs) CK(cudaStreamSynchronize(b->st));
  return TX_OK;
}

tx_status copy_rows_in(tx_batch* b, int g, double4_32a* dst, const double* src) {
  const GelInfo& G = b->gi[g];
  CK(cudaMemcpy2DAsync(dst + G.v0, sizeof(double4_32a), src, 3 * sizeof(double), 3 * sizeof(double), G.nv,
                       cudaMemcpyHostToDevice, b->st));
  CK(cudaStreamSynchronize(b->st));
  return TX_OK;
}

// positions at which to evaluate: x, xt (host), indenter at pose; leaves the state untouched
tx_status eval_setup(tx_batch* b, int g, const double* x, const double* xt, double h, const double pose[7]) {
  if (!x || !xt || !pose || !(h > 0.0)) return TX_ERR_ARG;
  for (int k = 0; k < b->n; ++k)
    if (b->run[k].in_request) return TX_ERR_ARG;
  const GelInfo& G = b->gi[g];
  Dev& d = b->d;
  CK(cudaMemcpyAsync(b->ex + G.v0, d.x + G.v0, sizeof(double4_32a) * G.ns * SLICE, cudaMemcpyDeviceToDevice, b->st));
  CK(cudaMemcpyAsync(b->ext + G.v0, d.xt + G.v0, sizeof(double4_32a) * G.ns * SLICE, cudaMemcpyDeviceToDevice, b->st));
  tx_status s = copy_rows_in(b, g, d.x, x);
  if (s == TX_OK) s = copy_rows_in(b, g, d.xt, xt);
  if (s != TX_OK) return s;
  for (int k = 0; k < b->n; ++k) b->gc_h[k].phase = PH_IDLE;
  Task t{};
  std::memcpy(t.pa, pose, sizeof(double) * 7);
  std::memcpy(t.pb, pose, sizeof(double) * 7);
  t.dt = h;
  t.attached = false;
  fill_ctl(b, g, PH_EVAL, t);
  s = upload_ctl(b);
  if (s != TX_OK) return s;
  launch_gel_op(d, PH_EVAL, 3, b->st);
  launch_indenter_pose(d, PH_EVAL, d.niv_total, b->st);
  launch_hash_build(d, PH_EVAL, 0, b->st);
  launch_query(d, PH_EVAL, 0, b->st);
  launch_scan(d.qcount, d.qoff, d.nq, b->scan_tmp, b->st);
  launch_query(d, PH_EVAL, 1, b->st);
  launch_pair_ranges(d, PH_EVAL, 0, b->st);
  launch_ss_pairs(d, PH_EVAL, 0, b->st);
  CK(cudaGetLastError());
  s = download_var(b);
  if (s != TX_OK) return s;
  if (b->gv_h[g].flags & (1 | 32)) {  // grow and redo
    const GelVar& v = b->gv_h[g];
    for (int tb = 0; tb < NTAB; ++tb) b->gi[g].hcap[tb] = std::max(b->gi[g].hcap[tb], 2 * v.hent[tb] + 64);
    b->gi[g].pcap = std::max(b->gi[g].pcap, v.npair + v.npair / 2 + 64);
    s = alloc_hash(b);
    if (s == TX_OK) s = alloc_pairs(b);
    if (s != TX_OK) return s;
    launch_gel_op(d, PH_EVAL, 3, b->st);
    launch_hash_build(d, PH_EVAL, 0, b->st);
    launch_query(d, PH_EVAL, 0, b->st);
    launch_scan(d.qcount, d.qoff, d.nq, b->scan_tmp, b->st);
    launch_query(d, PH_EVAL, 1, b->st);
    launch_pair_ranges(d, PH_EVAL, 0, b->st);
    launch_ss_pairs(d, PH_EVAL, 0, b->st);
  }
  return TX_OK;
}

tx_status eval_restore(tx_batch* b, int g) {
  const GelInfo& G = b->gi[g];
  Dev& d = b->d;
  CK(cudaMemcpyAsync(d.x + G.v0, b->ex + G.v0, sizeof(double4_32a) * G.ns * SLICE, cudaMemcpyDeviceToDevice, b->st));
  CK(cudaMemcpyAsync(d.xt + G.v0, b->ext + G.v0, sizeof(double4_32a) * G.ns * SLICE, cudaMemcpyDeviceToDevice, b->st));
  b->gc_h[g].phase = PH_IDLE;
  tx_status s = upload_ctl(b);
  if (s != TX_OK) return s;
  CK(cudaStreamSynchronize(b->st));
  return TX_OK;
}

void destroy_batch(tx_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->st);
  prof_resolve(b);
  drop_newton_graph(b);
  if (b->st2) {
    cudaStreamSynchronize(b->st2);
    cudaStreamDestroy(b->st2);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->gst) {
    cudaStreamSynchronize(b->gst);
    cudaStreamDestroy(b->gst);
  }
  if (b->gev_in) cudaEventDestroy(b->gev_in);
  if (b->tev0) cudaEventDestroy(b->tev0);
  if (b->tev1) cudaEventDestroy(b->tev1);
  if (b->gev_out) cudaEventDestroy(b->gev_out);
  for (cudaEvent_t e : b->prof.pool) cudaEventDestroy(e);
  b->mem.release();
  b->pair_mem.release();
  b->hash_mem.release();
  b->plan_mem.release();
  b->readout_mem.release();
  if (b->gc_h) cudaFreeHost(b->gc_h);
  if (b->gv_h) cudaFreeHost(b->gv_h);
  delete b;
}

}  // namespace

// ======================================================================================= C ABI
extern "C" {

void tx_params_default(tx_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->dhat = 1e-4;
  p->kappa = 0.0;
  p->newton_tol = 1e-5;
  p->pcg_rel_tol = 1e-3;
  p->pcg_rel_tol_far = 0.1;
  p->newton_max_iter = 200;
  p->pcg_max_iter = 2000;
  p->ls_max_halvings = 60;
  p->accd_max_iter = 1000000;
  p->max_split_depth = 4;
  p->precision = TX_PREC_FP64;
  p->refine_max = 3;
  p->pcg_cta_slices = 0;
  p->friction = 0.0;
  p->friction_eps_v = 1e-3;
  p->kappa_adapt_max = 0.0;
  p->kappa_adapt_dmin = 0.0;
}

const char* tx_status_str(tx_status s) {
  switch (s) {
    case TX_OK: return "TX_OK";
    case TX_ERR_ARG: return "TX_ERR_ARG";
    case TX_ERR_OOM: return "TX_ERR_OOM";
    case TX_ERR_MESH_INVERTED: return "TX_ERR_MESH_INVERTED";
    case TX_ERR_INFEASIBLE: return "TX_ERR_INFEASIBLE";
    case TX_ERR_NEWTON_MAXIT: return "TX_ERR_NEWTON_MAXIT";
    case TX_ERR_PCG_MAXIT: return "TX_ERR_PCG_MAXIT";
    case TX_ERR_LINESEARCH: return "TX_ERR_LINESEARCH";
    case TX_ERR_CCD_MAXIT: return "TX_ERR_CCD_MAXIT";
    case TX_ERR_CUDA: return "TX_ERR_CUDA";
    case TX_ERR_DEVICE_TIMEOUT: return "TX_ERR_DEVICE_TIMEOUT";
  }
  return "TX_ERR_UNKNOWN";
}

const char* tx_last_error(void) { return g_err.c_str(); }

tx_status tx_debug_inject(int32_t kind, int32_t count) {
  if (count < 0) return TX_ERR_ARG;
  if (kind == TX_INJECT_ALLOC_FAIL) {
    g_inject_alloc.store(count);
    return TX_OK;
  }
  if (kind == TX_INJECT_WAIT_TIMEOUT) {
    g_inject_wait.store(count);
    return TX_OK;
  }
  return TX_ERR_ARG;
}

tx_status tx_batch_create(const tx_gel_desc* descs, int32_t n, void* stream, tx_batch** out) {
  if (!out) return TX_ERR_ARG;
  *out = nullptr;
  return create_batch(descs, n, stream, out);
}

void tx_batch_destroy(tx_batch* b) { destroy_batch(b); }

int32_t tx_batch_size(const tx_batch* b) { return b ? b->n : 0; }

tx_status tx_batch_submit(tx_batch* b, int32_t count, const int32_t* ids, const double* poses,
                          const double* dts) {
  if (!b || count < 0 || (count > 0 && (!ids || !poses || !dts))) return TX_ERR_ARG;
  for (int k = 0; k < count; ++k) {
    const int g = ids[k];
    if (g < 0 || g >= b->n || b->run[g].in_request) return TX_ERR_ARG;
  }
  for (int k = 0; k < count; ++k) {
    tx_status s = submit_one(b, ids[k], poses + 7 * k, dts[k]);
    if (s != TX_OK) return s;
  }
  return TX_OK;
}

tx_status tx_batch_advance(tx_batch* b, int32_t* n_done, int32_t* done_ids, tx_status* done_status) {
  if (!b || !n_done) return TX_ERR_ARG;
  b->done_queue.clear();
  tx_status s = advance(b);
  *n_done = (int32_t)b->done_queue.size();
  for (size_t k = 0; k < b->done_queue.size(); ++k) {
    if (done_ids) done_ids[k] = b->done_queue[k];
    if (done_status) done_status[k] = (tx_status)b->run[b->done_queue[k]].last.status;
  }
  return s;
}

int32_t tx_batch_pending(const tx_batch* b) {
  if (!b) return 0;
  int c = 0;
  for (const Run& R : b->run) c += R.in_request ? 1 : 0;
  return c;
}

tx_status tx_batch_step_attached(tx_batch* b, const double* poses, const double* case_poses, const double* dts,
                                 tx_status* statuses) {
  if (!b || !poses || !dts) return TX_ERR_ARG;
  for (int g = 0; g < b->n; ++g)
    if (b->run[g].in_request) return TX_ERR_ARG;
  for (int g = 0; g < b->n; ++g) {
    tx_status s = submit_one(b, g, poses + 7 * g, dts[g], case_poses ? case_poses + 7 * g : nullptr);
    if (s != TX_OK) {
      for (int k = 0; k < g; ++k) {
        b->run[k].in_request = false;
        b->run[k].stack.clear();
      }
      return s;
    }
  }
  while (tx_batch_pending(b) > 0) {
    b->done_queue.clear();
    tx_status s = advance(b);
    if (s != TX_OK) return s;
  }
  tx_status worst = TX_OK;
  for (int g = 0; g < b->n; ++g) {
    const tx_status s = (tx_status)b->run[g].last.status;
    if (statuses) statuses[g] = s;
    if (s != TX_OK && worst == TX_OK) worst = s;
  }
  return worst;
}

tx_status tx_batch_step(tx_batch* b, const double* poses, const double* dts, tx_status* statuses) {
  return tx_batch_step_attached(b, poses, nullptr, dts, statuses);
}

tx_status tx_batch_state(const tx_batch* bc, int32_t g, double* x, double* v, double f_contact[3],
                         tx_step_stats* stats) {
  tx_batch* b = const_cast<tx_batch*>(bc);
  if (!b || g < 0 || g >= b->n) return TX_ERR_ARG;
  tx_status s = TX_OK;
  if (x) s = copy_rows_out(b, g, b->d.x, x, false);
  if (s == TX_OK && v) s = copy_rows_out(b, g, b->d.v, v, false);
  if (s != TX_OK) return s;
  const tx_step_stats& L = b->run[g].last;
  if (f_contact)
    for (int c = 0; c < 3; ++c) f_contact[c] = L.contact_force[c];
  if (stats) {
    *stats = L;
    std::vector<double> xs(3 * (size_t)b->gi[g].nv);
    s = copy_rows_out(b, g, b->d.x, xs.data(), false);
    if (s != TX_OK) return s;
    for (int c = 0; c < 3; ++c) {
      double m = 0.0;
      for (int i = 0; i < b->gi[g].nv; ++i) m += xs[3 * i + c];
      stats->mean_position[c] = m / b->gi[g].nv;
    }
  }
  return TX_OK;
}

tx_status tx_batch_set_state(tx_batch* b, int32_t g, const double* x, const double* v, const double pose[7]) {
  if (!b || g < 0 || g >= b->n || b->run[g].in_request) return TX_ERR_ARG;
  tx_status s = TX_OK;
  if (x) s = copy_rows_in(b, g, b->d.x, x);
  if (s == TX_OK && v) s = copy_rows_in(b, g, b->d.v, v);
  if (s != TX_OK) return s;
  // a new state: no previous Newton direction (the next solve starts from zero)
  const GelInfo& G = b->gi[g];
  CK(cudaMemsetAsync(b->d.p + G.v0, 0, sizeof(double4_32a) * G.ns * SLICE, b->st));
  CK(cudaStreamSynchronize(b->st));
  if (pose) std::memcpy(b->run[g].pose, pose, sizeof(double) * 7);
  b->run[g].kappa = b->mesh[g].kappa;  // a new state: the initial barrier stiffness
  b->run[g].dmin_last = 1e300;
  return TX_OK;
}

tx_status tx_batch_reset(tx_batch* b, int32_t g) {
  if (!b || g < 0 || g >= b->n || b->run[g].in_request) return TX_ERR_ARG;
  const GelInfo& G = b->gi[g];
  CK(cudaMemcpyAsync(b->d.x + G.v0, b->d.X + G.v0, sizeof(double4_32a) * G.ns * SLICE, cudaMemcpyDeviceToDevice, b->st));
  CK(cudaMemsetAsync(b->d.v + G.v0, 0, sizeof(double4_32a) * G.ns * SLICE, b->st));
  CK(cudaMemsetAsync(b->d.p + G.v0, 0, sizeof(double4_32a) * G.ns * SLICE, b->st));  // no previous direction
  CK(cudaStreamSynchronize(b->st));
  std::memcpy(b->run[g].pose, b->mesh[g].pose0, sizeof(double) * 7);
  const double ident[7] = {1, 0, 0, 0, 0, 0, 0};
  std::memcpy(b->run[g].case_pose, ident, sizeof(ident));  // the attached vertices are back at rest
  b->run[g].last = tx_step_stats{};
  b->run[g].kappa = b->mesh[g].kappa;
  b->run[g].dmin_last = 1e300;
  return TX_OK;
}

// ---- single gel = batch of one
tx_status tx_gel_create(const tx_gel_desc* desc, void* stream, tx_gel** out) {
  if (!out) return TX_ERR_ARG;
  *out = nullptr;
  tx_batch* b = nullptr;
  tx_status s = create_batch(desc, 1, stream, &b);
  if (s != TX_OK) return s;
  *out = new tx_gel{b};
  return TX_OK;
}

void tx_gel_destroy(tx_gel* g) {
  if (!g) return;
  destroy_batch(g->b);
  delete g;
}

tx_status tx_gel_step(tx_gel* g, const double pose[7], double dt) {
  if (!g || !pose) return TX_ERR_ARG;
  tx_status st = TX_OK;
  tx_status s = tx_batch_step(g->b, pose, &dt, &st);
  return s != TX_OK ? s : st;
}

tx_status tx_gel_step_attached(tx_gel* g, const double pose[7], const double case_pose[7], double dt) {
  if (!g || !pose || !case_pose) return TX_ERR_ARG;
  tx_status st = TX_OK;
  tx_status s = tx_batch_step_attached(g->b, pose, case_pose, &dt, &st);
  return s != TX_OK ? s : st;
}

// device scratch of the readout calls, grown on demand (the handle keeps it)
void* readout_scratch(tx_batch* b, size_t bytes) {
  if (bytes <= b->readout_bytes) return b->readout_mem.ptrs.empty() ? nullptr : b->readout_mem.ptrs[0];
  cudaStreamSynchronize(b->st);
  b->readout_mem.release();
  const size_t want = std::max(bytes, 2 * b->readout_bytes);
  unsigned char* p = b->readout_mem.get<unsigned char>(want);
  b->readout_bytes = p ? want : 0;
  return p;
}

tx_status tx_batch_markers(tx_batch* b, int32_t gel, int32_t n, const double* rest_xy, double* out, int32_t* found) {
  if (!b || gel < 0 || gel >= b->n || n < 0 || (n > 0 && (!rest_xy || !out || !found))) return TX_ERR_ARG;
  if (b->run[gel].in_request) return TX_ERR_ARG;
  if (n == 0) return TX_OK;
  const size_t nb = (size_t)n;
  if (nb * (size_t)b->gi[gel].ntop > ((size_t)1 << 38)) return TX_ERR_ARG;  // (marker, triangle) pairs of the search
  unsigned char* p = static_cast<unsigned char*>(readout_scratch(b, nb * (2 + 3) * sizeof(double) + 2 * nb * sizeof(int)));
  if (!p) return TX_ERR_OOM;
  double* dxy = reinterpret_cast<double*>(p);
  double* dout = dxy + 2 * nb;
  int* dfound = reinterpret_cast<int*>(dout + 3 * nb);
  int* dtri = dfound + nb;
  CK(cudaMemcpyAsync(dxy, rest_xy, sizeof(double) * 2 * nb, cudaMemcpyHostToDevice, b->st));
  launch_markers(b->d, gel, n, b->gi[gel].ntop, dxy, dtri, dout, dfound, b->st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, dout, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, b->st));
  CK(cudaMemcpyAsync(found, dfound, sizeof(int) * nb, cudaMemcpyDeviceToHost, b->st));
  CK(cudaStreamSynchronize(b->st));
  return TX_OK;
}

tx_status tx_batch_height_map(tx_batch* b, int32_t gel, int32_t nx, int32_t ny, double x0, double y0, double dx,
                              double dy, double* out) {
  if (!b || gel < 0 || gel >= b->n || nx < 1 || ny < 1 || (size_t)nx * (size_t)ny > ((size_t)1 << 26) || !out ||
      !std::isfinite(x0) || !std::isfinite(y0) || !(dx > 0.0) || !(dy > 0.0) || !std::isfinite(dx) ||
      !std::isfinite(dy))
    return TX_ERR_ARG;
  if (b->run[gel].in_request) return TX_ERR_ARG;
  const size_t np = (size_t)nx * (size_t)ny;
  unsigned char* p = static_cast<unsigned char*>(readout_scratch(b, np * (sizeof(unsigned long long) + sizeof(double))));
  if (!p) return TX_ERR_OOM;
  unsigned long long* img = reinterpret_cast<unsigned long long*>(p);
  double* dout = reinterpret_cast<double*>(img + np);
  CK(cudaMemsetAsync(img, 0, sizeof(unsigned long long) * np, b->st));
  launch_height_map(b->d, gel, b->gi[gel].ntop, nx, ny, x0, y0, dx, dy, img, dout, b->st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, dout, sizeof(double) * np, cudaMemcpyDeviceToHost, b->st));
  CK(cudaStreamSynchronize(b->st));
  return TX_OK;
}

tx_status tx_gel_markers(tx_gel* g, int32_t n, const double* rest_xy, double* out, int32_t* found) {
  if (!g) return TX_ERR_ARG;
  return tx_batch_markers(g->b, 0, n, rest_xy, out, found);
}

tx_status tx_gel_height_map(tx_gel* g, int32_t nx, int32_t ny, double x0, double y0, double dx, double dy,
                            double* out) {
  if (!g) return TX_ERR_ARG;
  return tx_batch_height_map(g->b, 0, nx, ny, x0, y0, dx, dy, out);
}

tx_status tx_gel_case_pose(const tx_gel* g, double case_pose[7]) {
  if (!g || !case_pose) return TX_ERR_ARG;
  std::memcpy(case_pose, g->b->run[0].case_pose, sizeof(double) * 7);
  return TX_OK;
}

tx_status tx_gel_state(const tx_gel* g, double* x, double* v, double f_contact[3], tx_step_stats* stats,
                       int32_t device_ptrs) {
  if (!g) return TX_ERR_ARG;
  tx_batch* b = g->b;
  if (device_ptrs) {
    tx_status s = TX_OK;
    if (x) s = copy_rows_out(b, 0, b->d.x, x, true);
    if (s == TX_OK && v) s = copy_rows_out(b, 0, b->d.v, v, true);
    if (s != TX_OK) return s;
    return tx_batch_state(b, 0, nullptr, nullptr, f_contact, stats);
  }
  return tx_batch_state(b, 0, x, v, f_contact, stats);
}

tx_status tx_gel_get_state(const tx_gel* g, double* x, double* v, double pose[7]) {
  if (!g) return TX_ERR_ARG;
  tx_status s = tx_batch_state(g->b, 0, x, v, nullptr, nullptr);
  if (s == TX_OK && pose) std::memcpy(pose, g->b->run[0].pose, sizeof(double) * 7);
  return s;
}

tx_status tx_gel_set_state(tx_gel* g, const double* x, const double* v, const double pose[7]) {
  if (!g) return TX_ERR_ARG;
  return tx_batch_set_state(g->b, 0, x, v, pose);
}

tx_status tx_gel_reset(tx_gel* g) {
  if (!g) return TX_ERR_ARG;
  return tx_batch_reset(g->b, 0);
}

size_t tx_gel_footprint_bytes(const tx_gel_desc* desc) {
  Mesh m;
  if (build_mesh(desc, m) != TX_OK) return 0;
  const bool mixed = desc->params.precision == TX_PREC_MIXED;
  const size_t rows = (size_t)((m.nv + SLICE - 1) / SLICE) * SLICE;
  const std::vector<int> need = row_block_needs(m);
  size_t nbp = 0;
  for (size_t s = 0; s < rows / SLICE; ++s) {
    size_t w = 1;
    for (int l = 0; l < SLICE; ++l) {
      const size_t i = s * SLICE + l;
      if (i < (size_t)m.nv) w = std::max(w, (size_t)need[i]);
    }
    nbp += w * SLICE;
  }
  const size_t nt = m.nt, nq = m.sv.size() + m.st.size() + m.se.size();
  size_t bytes = rows * (17 * sizeof(double4_32a) + 8 + 1 + 4 + 4 + 72 + 1);  // (+ body id)
  if (mixed) bytes += rows * (6 * sizeof(float4) + 36);
  bytes += nt * (16 + 72 + 8 + 4 + 64 + TS * 8 + (mixed ? TS32 * 4 : 0));
  bytes += nbp * (4 + 4 + 4 + (mixed ? 36 : 72));
  bytes += nq * (5 * 4) + (size_t)m.niv * 96 + (size_t)m.nit * 20 + m.ie.size() * 20;  // (+ soft-soft list)
  if (m.ncomp > 1) bytes += nbp * 4;  // soft-soft claim list (at most every padding position)
  bytes += ((size_t)m.niv + m.nit + m.ie.size()) * 2 * sizeof(double4_32a);  // primitive boxes
  bytes += (size_t)initial_pcap(m) * (32 + sizeof(C1Rec)) +
           (size_t)CREC_PER_GEL * (pair_record_doubles() * 8 + CH_STRIDE * 8 + CH_BP * 4);
  return bytes;
}

tx_status tx_gel_energy(tx_gel* gl, const double* x, const double* xt, double h, const double pose[7],
                        double* energy, double parts[5]) {
  if (!gl) return TX_ERR_ARG;
  tx_batch* b = gl->b;
  tx_status s = eval_setup(b, 0, x, xt, h, pose);
  if (s != TX_OK) return s;
  Dev& d = b->d;
  launch_energy(d, PH_EVAL, b->pieces, b->npieces, b->gel_piece, b->part_e, b->en_ticket, 2, b->st);
  launch_min_dist(d, PH_EVAL, b->st);
  CK(cudaGetLastError());
  std::vector<double> pe(b->npieces);
  CK(cudaMemcpyAsync(pe.data(), b->part_e, sizeof(double) * b->npieces, cudaMemcpyDeviceToHost, b->st));
  s = download_var(b);
  if (s != TX_OK) return s;
  if (energy) *energy = b->gv_h[0].E_try;
  if (parts) {
    double p3[3] = {0.0, 0.0, 0.0};
    for (int k = b->gel_piece_h[0]; k < b->gel_piece_h[1]; ++k) {
      const int kind = b->pieces_h[k].y;
      p3[kind == 0 ? 1 : (kind == 1 ? 0 : 2)] += pe[k];
    }
    parts[0] = p3[0];
    parts[1] = p3[1];
    parts[2] = p3[2];
    parts[3] = bitsd_host(b->gv_h[0].dmin_bits);
    parts[4] = b->gv_h[0].active_pairs;
  }
  return eval_restore(b, 0);
}

tx_status tx_gel_gradient(tx_gel* gl, const double* x, const double* xt, double h, const double pose[7],
                          double* grad, double f_contact[3]) {
  if (!gl || !grad) return TX_ERR_ARG;
  tx_batch* b = gl->b;
  tx_status s = eval_setup(b, 0, x, xt, h, pose);
  if (s != TX_OK) return s;
  Dev& d = b->d;
  launch_gel_op(d, PH_EVAL, 0, b->st);
  if (d.n_ss > 0) launch_ss_reset(d, b->st);
  launch_contact_compute(d, PH_EVAL, b->mixed, b->st);
  launch_tet_assemble(d, PH_EVAL, b->mixed, b->st);
  launch_gather(d, PH_EVAL, b->nbp, b->mixed, b->st);
  launch_contact_merge(d, b->mixed, b->st);
  CK(cudaGetLastError());
  s = copy_rows_out(b, 0, d.grad, grad, false);
  if (s != TX_OK) return s;
  s = download_var(b);
  if (s != TX_OK) return s;
  if (f_contact)
    for (int c = 0; c < 3; ++c) f_contact[c] = b->gv_h[0].fc[c];
  return eval_restore(b, 0);
}

tx_status tx_batch_profile(tx_batch* b, int32_t enable, tx_profile* out) {
  if (!b) return TX_ERR_ARG;
  CK(cudaStreamSynchronize(b->st));
  prof_resolve(b);
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->n_phases = PR_N;
    for (int k = 0; k < PR_N; ++k) {
      out->names[k] = kPhaseNames[k];
      out->ms[k] = b->prof.ms[k];
      out->launches[k] = b->prof.launches[k];
      out->flops[k] = b->prof.flops[k];
      out->bytes[k] = b->prof.bytes[k];
    }
    out->pcg_iters = b->prof.pcg_iters;
    out->newton_iters = b->prof.newton_iters;
    out->pcg_resident_launches = b->prof.pcg_res;
    out->pcg_streaming_launches = b->prof.pcg_stream;
    out->pcg_pool_launches = b->prof.pcg_pool;
    out->kernel_launches = g_launch_count.load() - g_launch_mark;
  }
  g_launch_mark = g_launch_count.load();
  std::vector<cudaEvent_t> pool = std::move(b->prof.pool);
  b->prof = Prof{};
  b->prof.pool = std::move(pool);
  b->prof.on = enable != 0;
  return TX_OK;
}

tx_status tx_gel_profile(tx_gel* g, int32_t enable, tx_profile* out) {
  if (!g) return TX_ERR_ARG;
  return tx_batch_profile(g->b, enable, out);
}

tx_status tx_eval_tets(int32_t n, const double* X, const double* x, double mu, double lambda, int32_t project,
                       double* e, double* g, double* H, void* stream) {
  if (n < 0 || (n > 0 && (!X || !x || !e))) return TX_ERR_ARG;
  launch_eval_tets(n, X, x, mu, lambda, project, e, g, H, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return TX_OK;
}

tx_status tx_eval_pairs(int32_t n, const int32_t* kind, const double* P, double dhat, const double* eps_x,
                        const int32_t* free_mask, double* bo, double* g, double* H, int32_t* dtype, void* stream) {
  if (n < 0 || (n > 0 && (!kind || !P || !bo)) || !(dhat > 0)) return TX_ERR_ARG;
  launch_eval_pairs(n, kind, P, dhat, eps_x, free_mask, bo, g, H, dtype, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return TX_OK;
}

tx_status tx_eval_accd(int32_t n, const int32_t* kind, const double* P, const double* dP, double s, double tc,
                       int32_t max_iter, double* toi, int32_t* hit, void* stream) {
  if (n < 0 || (n > 0 && (!kind || !P || !dP || !toi || !hit)) || !(s > 0 && s < 1) || max_iter < 1)
    return TX_ERR_ARG;
  launch_eval_accd(n, kind, P, dP, s, tc, max_iter, toi, hit, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return TX_OK;
}

}  // extern "C"

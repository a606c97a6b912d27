// Standalone block-Jacobi preconditioned conjugate gradient on a caller-provided symmetric
// positive definite matrix with 3x3 blocks (block CSR) -- the linear solve of the projected
// Newton step, exposed on its own.
//
// One persistent cooperative kernel runs every iteration; grid-wide dot products are per-CTA
// partials that every CTA sums in the same order after a bounded grid barrier, so all CTAs take
// identical decisions and the result does not depend on timing.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "tx_gel.h"
#include "txgel_common.cuh"

namespace txg {

constexpr int BP_T = 256;

struct BsrPcgArgs {
  int n;
  const int* rp;
  const int* ci;
  const double* va;
  const double* b;
  double* x;
  double tol2;
  int maxit;
  // scratch
  double* r;
  double* z;
  double* p;
  double* q;
  double* minv;   // 9 per row
  double* part;   // 2 per CTA
  unsigned* bar;  // grid barrier counter (zero at launch)
  int* err;       // barrier timeout flag (zero at launch)
  double* out;    // [iterations, relative residual]
};

__device__ __forceinline__ double grid_total(const BsrPcgArgs& a, int k, double* sm) {
  double v = 0.0;
  for (int c = threadIdx.x; c < (int)gridDim.x; c += BP_T) v += a.part[2 * c + k];
  return block_sum<BP_T>(v, sm);
}

__global__ void __launch_bounds__(BP_T) k_bsr_pcg(BsrPcgArgs a) {
  __shared__ double sm[BP_T / 32];
  unsigned epoch = 0;
  const int n = a.n, stride = gridDim.x * BP_T;
  double rz = 0.0, bb = 0.0;
  // init: M^-1 = inverse diagonal blocks, x = 0, r = b, z = M^-1 r, p = z
  for (int i = blockIdx.x * BP_T + threadIdx.x; i < n; i += stride) {
    double A[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = a.rp[i]; k < a.rp[i + 1]; ++k)
      if (a.ci[k] == i)
        for (int e = 0; e < 9; ++e) A[e] = a.va[9 * (size_t)k + e];
    const double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    const double id = 1.0 / (A[0] * c00 + A[1] * c01 + A[2] * c02);
    double* M = a.minv + 9 * (size_t)i;
    M[0] = c00 * id;
    M[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    M[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    M[3] = c01 * id;
    M[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    M[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    M[6] = c02 * id;
    M[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    M[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    for (int c = 0; c < 3; ++c) {
      const double bv = a.b[3 * i + c];
      a.x[3 * i + c] = 0.0;
      a.r[3 * i + c] = bv;
      bb += bv * bv;
    }
    for (int c = 0; c < 3; ++c) {
      const double zv = M[3 * c] * a.r[3 * i] + M[3 * c + 1] * a.r[3 * i + 1] + M[3 * c + 2] * a.r[3 * i + 2];
      a.z[3 * i + c] = zv;
      a.p[3 * i + c] = zv;
      rz += a.r[3 * i + c] * zv;
    }
  }
  rz = block_sum<BP_T>(rz, sm);
  bb = block_sum<BP_T>(bb, sm);
  if (threadIdx.x == 0) {
    a.part[2 * blockIdx.x] = rz;
    a.part[2 * blockIdx.x + 1] = bb;
  }
  if (!grid_barrier(a.bar, epoch, a.err)) return;
  rz = grid_total(a, 0, sm);
  bb = grid_total(a, 1, sm);
  double rr = bb;
  int it = 0;
  while (rr > a.tol2 * bb && it < a.maxit) {
    if (!grid_barrier(a.bar, epoch, a.err)) return;  // everyone has read the partials
    // q = A p, partial p.q
    double pq = 0.0;
    for (int i = blockIdx.x * BP_T + threadIdx.x; i < n; i += stride) {
      double q0 = 0.0, q1 = 0.0, q2 = 0.0;
      for (int k = a.rp[i]; k < a.rp[i + 1]; ++k) {
        const int j = a.ci[k];
        const double* v = a.va + 9 * (size_t)k;
        const double p0 = a.p[3 * j], p1 = a.p[3 * j + 1], p2 = a.p[3 * j + 2];
        q0 += v[0] * p0 + v[1] * p1 + v[2] * p2;
        q1 += v[3] * p0 + v[4] * p1 + v[5] * p2;
        q2 += v[6] * p0 + v[7] * p1 + v[8] * p2;
      }
      a.q[3 * i] = q0;
      a.q[3 * i + 1] = q1;
      a.q[3 * i + 2] = q2;
      pq += a.p[3 * i] * q0 + a.p[3 * i + 1] * q1 + a.p[3 * i + 2] * q2;
    }
    pq = block_sum<BP_T>(pq, sm);
    if (threadIdx.x == 0) a.part[2 * blockIdx.x] = pq;
    if (!grid_barrier(a.bar, epoch, a.err)) return;
    pq = grid_total(a, 0, sm);
    const double alpha = rz / pq;
    if (!grid_barrier(a.bar, epoch, a.err)) return;  // partial slot 0 is reused below
    // x += alpha p, r -= alpha q, z = M^-1 r; partials r.z, r.r
    double rz2 = 0.0, rr2 = 0.0;
    for (int i = blockIdx.x * BP_T + threadIdx.x; i < n; i += stride) {
      for (int c = 0; c < 3; ++c) {
        a.x[3 * i + c] += alpha * a.p[3 * i + c];
        a.r[3 * i + c] -= alpha * a.q[3 * i + c];
      }
      const double* M = a.minv + 9 * (size_t)i;
      for (int c = 0; c < 3; ++c) {
        const double zv = M[3 * c] * a.r[3 * i] + M[3 * c + 1] * a.r[3 * i + 1] + M[3 * c + 2] * a.r[3 * i + 2];
        a.z[3 * i + c] = zv;
        rz2 += a.r[3 * i + c] * zv;
        rr2 += a.r[3 * i + c] * a.r[3 * i + c];
      }
    }
    rz2 = block_sum<BP_T>(rz2, sm);
    rr2 = block_sum<BP_T>(rr2, sm);
    if (threadIdx.x == 0) {
      a.part[2 * blockIdx.x] = rz2;
      a.part[2 * blockIdx.x + 1] = rr2;
    }
    if (!grid_barrier(a.bar, epoch, a.err)) return;
    rz2 = grid_total(a, 0, sm);
    rr = grid_total(a, 1, sm);
    const double beta = rz2 / rz;
    rz = rz2;
    ++it;
    for (int i = blockIdx.x * BP_T + threadIdx.x; i < n; i += stride)
      for (int c = 0; c < 3; ++c) a.p[3 * i + c] = a.z[3 * i + c] + beta * a.p[3 * i + c];
    if (!grid_barrier(a.bar, epoch, a.err)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.out[0] = it;
    a.out[1] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  }
}

// cooperative launch over at most one CTA per SM (at least one row per thread)
static cudaError_t launch_bsr_pcg(BsrPcgArgs a, cudaStream_t st, int* nctas_out) {
  int dev = 0, nsm = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bsr_pcg, BP_T, 0);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorCooperativeLaunchTooLarge;
  int nctas = (a.n + BP_T - 1) / BP_T;
  if (nctas > nsm) nctas = nsm;
  if (nctas < 1) nctas = 1;
  *nctas_out = nctas;
  void* args[] = {(void*)&a};
  count_launch(1);
  return cudaLaunchCooperativeKernel((const void*)k_bsr_pcg, dim3(nctas), dim3(BP_T), args, 0, st);
}

static tx_status check_bsr_args(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* vals,
                                const double* b, double* x, double rel_tol, int32_t max_iter) {
  if (n < 0 || (n > 0 && (!row_ptr || !col_idx || !vals || !b || !x)) || !(rel_tol >= 0.0) || max_iter < 0)
    return TX_ERR_ARG;
  return TX_OK;
}

// ------------------------------------------------------------------ no-allocation variant
// Scratch of tx_bsr_pcg_noalloc: a fixed array in the module's global memory, so that a call
// needs no cudaMalloc.  Every GPU that loads the library holds it until the process exits.
constexpr int NOALLOC_MAX_ROWS = 65536;
constexpr int NOALLOC_MAX_CTAS = 1024;
// r, z, p, q (3 n each) + inverse diagonal blocks (9 n) + 2 partials per CTA + out/barrier/error
constexpr size_t NOALLOC_DOUBLES = (size_t)21 * NOALLOC_MAX_ROWS + 2 * NOALLOC_MAX_CTAS + 4;
static __device__ __align__(256) double g_pcg_scratch[NOALLOC_DOUBLES];

// Device addresses of the scratch array, one per CUDA context that used it.  The symbol's
// host-side name is only a stand-in, so its address is looked up (cudaGetSymbolAddress, with the
// context current) the first time a context calls; the cache is keyed by the context's unique
// id, so a context created after a device reset (where the module, and the array, may have moved)
// looks the address up again instead of using a stale one.
constexpr int NOALLOC_MAX_CONTEXTS = 64;
struct ScratchEntry {
  unsigned long long ctx_id;
  double* ptr;
};
static ScratchEntry g_scratch_ctx[NOALLOC_MAX_CONTEXTS];
static int g_scratch_n = 0;
static std::mutex g_scratch_mu;

// unique id of the current context (driver entry points taken through the runtime); false if
// there is none yet or the driver does not offer it
static bool current_context_id(unsigned long long* id) {
  typedef CUresult (*GetCurrentFn)(CUcontext*);
  typedef CUresult (*GetIdFn)(CUcontext, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f0 = nullptr;
    void* f1 = nullptr;
    cudaDriverEntryPointQueryResult q0, q1;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        q0 == cudaDriverEntryPointSuccess && q1 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<GetCurrentFn>(f0);
      get_id = reinterpret_cast<GetIdFn>(f1);
    }
    cudaGetLastError();
  }
  if (!get_current || !get_id) return false;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the scratch array in the current context.
static cudaError_t scratch_in_current_context(double** out) {
  unsigned long long id = 0;
  const bool have_id = current_context_id(&id);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (have_id)
    for (int k = 0; k < g_scratch_n; ++k)
      if (g_scratch_ctx[k].ctx_id == id) {
        *out = g_scratch_ctx[k].ptr;
        return cudaSuccess;
      }
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_pcg_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(ptr);
  if (have_id) {  // remember it (the oldest entry makes room when the table is full)
    if (g_scratch_n == NOALLOC_MAX_CONTEXTS) {
      for (int k = 1; k < NOALLOC_MAX_CONTEXTS; ++k) g_scratch_ctx[k - 1] = g_scratch_ctx[k];
      g_scratch_n -= 1;
    }
    g_scratch_ctx[g_scratch_n++] = {id, *out};
  }
  return cudaSuccess;
}

void set_last_error(const char* msg);

}  // namespace txg

using namespace txg;

extern "C" tx_status tx_bsr_pcg(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* vals,
                                const double* b, double* x, double rel_tol, int32_t max_iter, int32_t* iters,
                                double* rel_res, void* stream) {
  tx_status s = check_bsr_args(n, row_ptr, col_idx, vals, b, x, rel_tol, max_iter);
  if (s != TX_OK) return s;
  if (n == 0) {
    if (iters) *iters = 0;
    if (rel_res) *rel_res = 0.0;
    return TX_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TX_ERR_CUDA;
  const size_t vec = (size_t)3 * n;
  const size_t total = 4 * vec + 9 * (size_t)n + 2 * (size_t)nsm + 2 + 4;
  double* buf = nullptr;
  if (cudaMalloc(&buf, total * sizeof(double)) != cudaSuccess) return TX_ERR_OOM;
  BsrPcgArgs a;
  a.n = n;
  a.rp = row_ptr;
  a.ci = col_idx;
  a.va = vals;
  a.b = b;
  a.x = x;
  a.tol2 = rel_tol * rel_tol;
  a.maxit = max_iter;
  a.r = buf;
  a.z = a.r + vec;
  a.p = a.z + vec;
  a.q = a.p + vec;
  a.minv = a.q + vec;
  a.part = a.minv + 9 * (size_t)n;
  a.out = a.part + 2 * (size_t)nsm;
  a.bar = reinterpret_cast<unsigned*>(a.out + 2);
  a.err = reinterpret_cast<int*>(a.out + 3);
  tx_status res = TX_OK;
  int nctas = 0;
  double out[2] = {0.0, 0.0};
  int derr = 0;
  if (cudaMemsetAsync(a.out, 0, 4 * sizeof(double), st) != cudaSuccess || launch_bsr_pcg(a, st, &nctas) != cudaSuccess ||
      cudaMemcpyAsync(out, a.out, sizeof(out), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&derr, a.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    res = TX_ERR_CUDA;
  cudaFree(buf);
  if (res != TX_OK) return res;
  if (derr) return TX_ERR_DEVICE_TIMEOUT;
  if (iters) *iters = (int32_t)out[0];
  if (rel_res) *rel_res = out[1];
  return TX_OK;
}

extern "C" tx_status tx_bsr_pcg_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                        const double* vals, const double* b, double* x, double rel_tol,
                                        int32_t max_iter, int32_t* iters, double* rel_res, void* stream) {
  tx_status s = check_bsr_args(n, row_ptr, col_idx, vals, b, x, rel_tol, max_iter);
  if (s != TX_OK) return s;
  if (n > NOALLOC_MAX_ROWS) {
    set_last_error("tx_bsr_pcg_noalloc: more than 65536 block rows (use tx_bsr_pcg)");
    return TX_ERR_ARG;
  }
  if (n == 0) {
    if (iters) *iters = 0;
    if (rel_res) *rel_res = 0.0;
    return TX_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TX_ERR_CUDA;
  if (nsm > NOALLOC_MAX_CTAS) return TX_ERR_ARG;
  double* buf = nullptr;
  if (scratch_in_current_context(&buf) != cudaSuccess) return TX_ERR_CUDA;
  const size_t vec = (size_t)3 * n;
  BsrPcgArgs a;
  a.n = n;
  a.rp = row_ptr;
  a.ci = col_idx;
  a.va = vals;
  a.b = b;
  a.x = x;
  a.tol2 = rel_tol * rel_tol;
  a.maxit = max_iter;
  a.r = buf;
  a.z = a.r + vec;
  a.p = a.z + vec;
  a.q = a.p + vec;
  a.minv = a.q + vec;
  a.part = buf + 21 * (size_t)NOALLOC_MAX_ROWS;
  a.out = a.part + 2 * (size_t)NOALLOC_MAX_CTAS;
  a.bar = reinterpret_cast<unsigned*>(a.out + 2);
  a.err = reinterpret_cast<int*>(a.out + 3);
  int nctas = 0;
  double out[2] = {0.0, 0.0};
  int derr = 0;
  // the previous call's counters are still in the array: clear them before the launch
  if (cudaMemsetAsync(a.out, 0, 4 * sizeof(double), st) != cudaSuccess || launch_bsr_pcg(a, st, &nctas) != cudaSuccess ||
      cudaMemcpyAsync(out, a.out, sizeof(out), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&derr, a.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return TX_ERR_CUDA;
  if (derr) return TX_ERR_DEVICE_TIMEOUT;
  if (iters) *iters = (int32_t)out[0];
  if (rel_res) *rel_res = out[1];
  return TX_OK;
}

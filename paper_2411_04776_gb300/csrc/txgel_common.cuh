// Shared declarations of the GB300 gelpad IPC step library: device data layout, small
// fixed-size linear algebra, reductions and the bounded grid barrier.
//
// Data layout (all gels of a handle are concatenated; a single gel is a batch of one):
//   * vertex rows: each gel owns rows [v0, v0 + nv), v0 a multiple of 32 so every 32-row slice
//     (one warp) belongs to one gel; rows past nv up to the next multiple of 32 are inert
//     padding (fixed, zero mass).  Positions and all solver vectors are double4_32a (x, y, z, 0):
//     one 32-byte sector per vertex gather.
//   * Hessian: 3x3-block sparse, sliced ELL ("SELL-32") over the rows: slice s holds rows
//     [32 s, 32 s + 32) with width w_s = longest row; block k of lane l lives at position
//     slice_off[s] + 32 k + l; its 9 values are stored entry-major inside the slice column
//     (value e of lane l at 9 (slice_off[s] + 32 k) + 32 e + l) so a warp loads each entry
//     of 32 rows with one coalesced 256-byte access.  Padding entries point at the row itself
//     with zero values.
//   * per-tet scratch: the 10 upper 3x3 blocks of the 12x12 element Hessian and the 12-vector
//     gradient, gathered into the rows by fixed per-block contribution lists (deterministic,
//     no atomics).
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace txg {

constexpr int SLICE = 32;
// per-tet scratch: the 10 upper 3x3 blocks, each padded to a 16-byte multiple so the gather reads
// it with vector loads (FP64: 10 doubles per block, FP32: 12 floats), then the 12-entry gradient
constexpr int BLK64 = 10;      // doubles per block in the FP64 scratch
constexpr int BLK32 = 12;      // floats per block in the FP32 scratch
constexpr int GOFF = 100;      // gradient offset in the FP64 scratch
constexpr int TS = 112;        // per-tet FP64 scratch stride (10 x 10 blocks + 12 gradient), doubles
constexpr int TS32 = 120;      // per-tet FP32 block scratch stride (10 x 12), floats
constexpr int NTAB = 3;        // hash tables per gel: indenter tris, indenter verts, indenter edges
constexpr int PAIR_PT = 0;     // gel surface vertex   vs indenter triangle
constexpr int PAIR_TP = 1;     // indenter vertex      vs gel surface triangle
constexpr int PAIR_EE = 2;     // gel surface edge     vs indenter edge
// between two deformable bodies of one mesh (surface primitives of different connected components)
constexpr int PAIR_SPT = 3;    // surface vertex       vs surface triangle
constexpr int PAIR_SEE = 4;    // surface edge         vs surface edge
// distance kind of a pair type: 1 edge-edge (mollified), 0 point-triangle
__host__ __device__ constexpr int pair_kind(int type) { return (type == PAIR_EE || type == PAIR_SEE) ? 1 : 0; }
constexpr int SS_MAXC = 4;     // connected components of a mesh that take part in soft-soft contact
// streaming FP64 PCG coarse space: per-CTA partial sums of the set-up (21 entries of Z^T A Z, Z^T b,
// Z^T A p_prev) and, per iteration, of Z^T w in the first 6 slots
constexpr int CZ_N = 33;
constexpr int CZ_F = 49;       // per coarse group: E^-1 (36), Z^T b, Z^T A p_prev, ok flag
constexpr double ACCD_S = 0.1; // ACCD: the gap may shrink to this fraction per sweep

// phases of a gel inside a batch
enum Phase : int { PH_IDLE = 0, PH_BEGIN = 1, PH_NEWTON = 2, PH_START = 3, PH_SAVE = 4, PH_FINAL = 5, PH_EVAL = 6,
                   PH_PARK = 7, PH_FAIL = 8 };

struct GelInfo {  // per gel, read-only after create
  int v0, nv;     // rows
  int s0, ns;     // slices
  int t0, nt;     // tets
  int q0, nq;     // query primitives: [surface verts | surface tris | surface edges]
  int nsv, nst, nse;
  int sv0, st0, se0;
  int iv0, niv, it0, nit, ie0, nie;
  int hb0[NTAB], hnb[NTAB];  // hash bucket ranges (power-of-two sizes)
  int he0[NTAB], hcap[NTAB]; // hash entry ranges
  int pbase, pcap;           // candidate-pair segment
  int fixed_count;
  double mu, lam, kappa, dhat, cell, bbox_diag, newton_tol;
  double org[3];             // hash grid origin
  double mu_f, eps_v;        // IPC lagged friction: coefficient (0: frictionless), velocity threshold
  int top0, ntop;            // top-surface triangles (rest outward normal up) in Dev::top
  int ncomp;                 // connected components of the tet mesh (> 1: soft-soft contact)
  int ss;                    // its index in the soft-soft gel list (-1: one body)
  int cbody;                 // the largest body with no held vertex (-1: none): the streaming PCG's
  int pad5_;                 // coarse space is its six rigid motions about its rest centroid cctr
  double cctr[3];
};

struct GelCtl {  // per gel, written by the host before the launches of an iteration
  int phase;
  int pad_;
  double h;                  // current (sub)step length
  double tol_p;              // ||p||_inf tolerance = newton_tol * bbox_diag * h
  double eta2_near, eta2_far;  // squared PCG forcing terms near convergence / far from it
  double grav[3];
  double R[9], t[3];         // indenter pose at the end of the (sub)step
  double Rp[9], tp[3];       // indenter pose at its start
  // attachment-driven step (attached != 0): the Dirichlet (attached) vertices follow the sensor
  // case, at their rest positions carried by the case pose -- (Rc, tc) at the end of the
  // (sub)step, (Rcp, tcp) at its start
  int attached;
  int pad2_;
  double Rc[9], tc[3];
  double Rcp[9], tcp[3];
  double kappa;              // barrier stiffness of the step (the host's adaptive rule)
};

struct GelVar {  // per gel, written by the device
  double E_cur, E_try;
  double alpha, alpha0;
  double bb;                 // |b|^2 of the PCG right-hand side
  double gtp;                // g . p of the last Newton direction
  double eta2;               // squared forcing term of the next PCG solve
  double res2;               // |r|^2 / |b|^2 reached by the last PCG solve
  double pn_prev;            // ||p||_inf of the previous direction (0: none yet)
  double fc[3];              // contact force on the gel
  unsigned long long toi_bits;    // min ACCD time of impact (non-negative double bits)
  unsigned long long pnorm_bits;  // ||p||_inf of the last Newton direction
  unsigned long long dmin_bits;   // min pair distance
  int ls_state;              // 0 searching, 1 accepted, 2 failed
  int ls_total;              // halvings this step
  int converged;             // Newton converged at the last check
  int pcg_it;                // PCG iterations of the last solve
  int pcg_done;              // set inside the PCG kernel once the gel's solve converged
  int inner_done;            // mixed precision: FP32 inner solve of the current round converged
  int rounds;                // mixed precision: FP64 residual refinement rounds used
  int pair0, npair;          // candidate pair range
  int hent[NTAB];            // hash entries used
  int active_pairs;
  double ibox_lo[3], ibox_hi[3];  // indenter bounding box of the current hash build
  int flags;                 // 1 hash overflow, 2 ACCD cap, 4 inverted tet, 8 ACCD hit, 16 pattern miss
  int nfric;                 // friction records of the running (sub)step (slots of its pair segment)
  int ss_cut;                // soft-soft pairs whose cross-body blocks found no free slot (this substep)
};

// Per-gel record of the pooled streaming PCG (k_solve.cu): written by the gel's owner warp after
// a pool barrier, read by every CTA after the next one
struct PoolGel {
  double al, be;          // CG step and direction update of the current iteration
  double gprev, aprev;    // the previous iteration's gamma and alpha (owner only)
  double bb, th;          // |b|^2 of the right-hand side and the stopping threshold eta^2 |b|^2
  double rho;             // Galerkin start along the previous direction
  double rr, rr0, tol;    // mixed: |r|^2 (FP64 residual / FP32 inner), its round-start value, the inner target
  int act;                // in this solve
  int run;                // solve not finished (FP64: CG running; mixed: refinement rounds running)
  int inner;              // mixed: FP32 inner CG of the current round running
  int it;                 // CG iterations so far
};

struct PairBarrier;  // barrier setup of one contact pair (dev_pairwarp.cuh)

// Lagged friction data of one contact pair, taken at the start of the (sub)step (IPC, Li et al.
// 2020, Sec. 5): the pair (as in the candidate list), whether it was in contact then, the
// closest-point weights w (relative displacement of the closest points = sum_k w_k (P_k - Plag_k)),
// the orthonormal tangent basis T (two columns, row-major 3 x 2) and the lagged normal force lam.
struct FricRec {
  int4 pr;
  int active;
  int pad_;
  double w[4];
  double T[6];
  double lam;
  double Plag[12];
};

// Barrier block of a pair with one free gel point: its diagonal block position and kappa d2b/dx2
struct C1Rec {
  int bp;
  int pad_;
  double v[9];
};
constexpr int CH_STRIDE = 144;  // projected pair Hessian record: 12 x 12 values (row stride 3 ns)
constexpr int CH_BP = 17;       // and ns followed by the ns x ns block positions

// Everything the kernels touch, passed by value.
struct Dev {
  int n_gels;
  const GelInfo* gi;
  const GelCtl* gc;
  GelVar* gv;
  int niv_total;
  // rows
  int nrows;
  double4_32a *X, *x, *xn, *v, *xt, *p, *grad;
  double* mass;
  uint8_t* fixed;
  int* vgel;
  // tets
  int ntets;
  int4* tets;
  double* Dminv;  // 9 per tet
  double* vol;
  int* tgel;
  double* tscr;   // TS per tet
  float* tscr32;  // TS32 per tet (mixed precision Hessian)
  // sliced BSR
  int nslices;
  int* slice_off;  // nslices + 1 (block positions)
  int* colidx;     // per block position
  double* vals;    // 9 per block position (FP64)
  float* vals32;   // 9 per block position (mixed)
  int* bp_row;     // per block position: its row
  int* ctr_ptr;    // per block position + 1: contribution list range
  int* ctr;        // (tet << 4) | (4 a + b)
  int* diag_pos;   // per row: block position of the diagonal block
  double* Minv;    // 9 per row
  float* Minv32;
  // PCG
  double4_32a *r, *u, *w, *pp, *s;
  float4 *u32, *w32, *pp32, *s32, *r32, *x32;
  double* part;    // PCG: per-CTA partial sums exchanged inside a group, [2 sets][4][nctas]
  double* czpart;  // streaming FP64 PCG's coarse space: per-CTA partial sums [CZ_N][nctas]
  double* czfac;   // ... and per group (at its first CTA): [CZ_F] (E^-1, right-hand sides, flag)
  unsigned* bar;   // PCG: one barrier counter per group
  double* pslice;  // pooled PCG: per-slice partial sums [slice][4]
  PoolGel* pool;   // pooled PCG: per-gel records
  // surface primitives (global)
  int* sv;
  int4* st;
  int2* se;
  double* se_len2;
  int* q_gel;
  int* q_tp;       // (type << 28) | local primitive index within the gel's surface list
  // indenter
  double4_32a *iv_loc, *iv_cur, *iv_prev;
  int4* it;
  int2* ie;
  double* ie_len2;
  int* iv_gel;
  int* it_gel;
  int* ie_gel;
  int nit_total, nie_total;
  // bounding boxes of the indenter primitives [triangles | vertices | edges] at the pose of the
  // last hash build of their gel: (lo, hi) pairs, lo.w holds the packed lowest grid cell
  double4_32a* pbox;
  // hash
  int* hstart;     // bucket starts (global, per table segment nb + 1)
  int* hcount;     // bucket fill cursors
  int max_hnb;     // largest bucket count of any table
  int2* hent;      // entries (prim, packed cell)
  // candidate pairs
  int nq;
  int* qcount;     // nq + 1
  int* qoff;       // nq + 1 (exclusive scan)
  int* qnear;      // queries near the indenter (listed by the count pass), and their count
  int* qnear_n;
  int4* pairs;     // (type, gel prim, indenter prim, gel), per-gel segments [pbase, pbase + pcap)
  int* pslot_gel;  // gel of every pair slot
  int npslots;
  int* cwork;      // contact pairs with two or more free gel points (pair slots), and their count
  int* cwork_n;
  PairBarrier* crec;  // their barrier setup (the first crec_cap of them)
  int crec_cap;
  double* chv;     // the projected kappa-scaled Hessians of those crec_cap pairs (CH_STRIDE each)
  int* chbp;       // their ns and block positions (CH_BP each)
  C1Rec* c1rec;    // single-free-point barrier blocks (appended; one per pair slot at most)
  FricRec* fric;   // lagged friction records, one per pair slot at the (sub)step start (null: none)
  int4* top;       // top-surface triangles of every gel (rows a, b, c), the readout's surface
  // soft-soft contact (gels whose mesh has several connected components)
  int8_t* vcomp;   // per row: its connected component within its gel's mesh
  int n_ss;        // soft-soft gels, and the most surface primitives (queries) of one of them
  int ss_maxq;
  int* ss_gel;     // the soft-soft gels, and per soft-soft gel: component boxes (SS_MAXC x 6) ...
  double* ss_box;
  int* ss_cnt;     // ... and the counts of its listed vertices, triangles, edges (3 each)
  int* ss_list;    // listed primitives near another component (global query ids, the gel's query range)
  int* ss_claim;   // block positions whose column a cross-body block took (reset every Newton iteration)
  int* ss_nclaim;
  int ss_claim_cap;
  int* c1_n;
  double4_32a* cgrad;  // contact gradient per row: accumulated by the contact kernels, added by the gather
  int* err;
  unsigned wait_limit;  // polls a bounded device-side wait makes before it gives up (sets *err)
  unsigned wait_extra;  // fault-injection test hook: arrivals a group barrier waits for that never come (0)
};

// Partition of the slices of the gels being solved over the CTAs of the persistent PCG kernels
// (rebuilt when that set of gels changes).  The gels are split into independent groups: a gel
// with many slices forms a group alone, spread over several CTAs; runs of small gels are packed
// into a group of one CTA.  The CTAs of a group synchronise through a barrier counter of their
// own, so a group never waits for another one.
// Pooled streaming PCG launch: the gels [g0, g0 + ng) (those in the solve's phase take part)
struct PoolPlan {
  int g0, ng;
  int cap;  // room of a CTA's slice list (at least its share of the gels' slices)
};

struct PcgPlan {
  const int2* cta_rng;   // per CTA: its slices [x, y)
  const int* cta_grp;    // per CTA: its group
  const int4* grp;       // per group: (first CTA, CTA count, first gel, gel count)
  const int* slice_gel;  // per slice: its gel
  int max_slices;        // most slices any CTA owns
  int ngroups;
};

// Value layout of the sliced BSR.  The 32 block positions of one column k of a slice share 288
// consecutive values; element e (row-major 3x3) of the block at lane l = bp mod 32 sits at
//   FP64: e < 8: 64 (e / 2) + 2 l + e % 2 (pairs: one 16-byte load reads two), e = 8: 256 + l;
//   FP32: e < 8: 128 (e / 4) + 4 l + e % 4 (quads: one 16-byte load reads four), e = 8: 256 + l,
// so a lane reads its block with 5 (FP64) or 3 (FP32) loads instead of 9.
__host__ __device__ __forceinline__ size_t val_addr64(int bp, int e) {
  const int l = bp & 31;
  return (size_t)9 * (bp & ~31) + (e < 8 ? 64 * (e >> 1) + 2 * l + (e & 1) : 256 + l);
}
__host__ __device__ __forceinline__ size_t val_addr32(int bp, int e) {
  const int l = bp & 31;
  return (size_t)9 * (bp & ~31) + (e < 8 ? 128 * (e >> 2) + 4 * l + (e & 3) : 256 + l);
}

// one lane's block from its slice column image (column base b: 288 values, the layout above);
// returns the row-major elements
__device__ __forceinline__ void load_block64(const double* b, int lane, double e[9]) {
  const double2 p0 = *reinterpret_cast<const double2*>(b + 2 * lane);
  const double2 p1 = *reinterpret_cast<const double2*>(b + 64 + 2 * lane);
  const double2 p2 = *reinterpret_cast<const double2*>(b + 128 + 2 * lane);
  const double2 p3 = *reinterpret_cast<const double2*>(b + 192 + 2 * lane);
  e[0] = p0.x; e[1] = p0.y; e[2] = p1.x; e[3] = p1.y; e[4] = p2.x;
  e[5] = p2.y; e[6] = p3.x; e[7] = p3.y; e[8] = b[256 + lane];
}
__device__ __forceinline__ void load_block32(const float* b, int lane, float e[9]) {
  const float4 q0 = *reinterpret_cast<const float4*>(b + 4 * lane);
  const float4 q1 = *reinterpret_cast<const float4*>(b + 128 + 4 * lane);
  e[0] = q0.x; e[1] = q0.y; e[2] = q0.z; e[3] = q0.w;
  e[4] = q1.x; e[5] = q1.y; e[6] = q1.z; e[7] = q1.w; e[8] = b[256 + lane];
}

// host-side count of kernel launches (every launcher adds the kernels it enqueued)
void count_launch(int k);

// ------------------------------------------------------------------------------------------
// small helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long dbits(double v) {
  return static_cast<unsigned long long>(__double_as_longlong(v));
}
__device__ __forceinline__ double bitsd(unsigned long long b) {
  return __longlong_as_double(static_cast<long long>(b));
}
// min/max of non-negative doubles through their order-preserving bit patterns
__device__ __forceinline__ void atomic_min_pos(unsigned long long* a, double v) {
  atomicMin(a, dbits(v));
}
__device__ __forceinline__ void atomic_max_pos(unsigned long long* a, double v) {
  atomicMax(a, dbits(v));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Fixed-order block sum (deterministic): every thread gets the total.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sm) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sm[wid] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < NT / 32; ++k) t += sm[k];
  return t;
}

__device__ __forceinline__ void quat_to_R(const double q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double n = rsqrt(w * w + x * x + y * y + z * z);
  w *= n; x *= n; y *= n; z *= n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

__device__ __forceinline__ void ld3(const double4_32a& a, double r[3]) {
  r[0] = a.x; r[1] = a.y; r[2] = a.z;
}

// Bounded grid barrier for cooperative launches: a monotonic arrival counter; `epoch` counts the
// barriers passed so far.  A wait that exceeds the spin limit sets *err and returns, so a kernel
// can never hang the device.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned& epoch, int* err) {
  __syncthreads();
  bool ok = true;
  if (threadIdx.x == 0) {
    epoch += 1;
    const unsigned target = epoch * gridDim.x;
    __threadfence();
    atomicAdd(count, 1u);
    unsigned spins = 0;
    while (true) {
      unsigned cur;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(count) : "memory");
      if (cur >= target) break;
      if (++spins > (1u << 22)) {
        atomicExch(err, 1);
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  } else {
    epoch += 1;
  }
  __syncthreads();
  if (*((volatile int*)err) != 0) ok = false;
  return ok;
}

}  // namespace txg

// Contact kernels: indenter placement, spatial-hash broad phase, barrier assembly, ACCD.
//
// Broad phase.  Per gel, the indenter's primitives (triangles, vertices, edges: three tables)
// are inserted into a spatial hash (Teschner et al. 2003): every primitive goes into each cell
// of a uniform grid its bounding box overlaps, cells are hashed into a power-of-two bucket array
// (counting sort, then each bucket sorted by (primitive, cell) so the table is deterministic).
// The gel surface primitives query it: vertices -> indenter triangles, triangles -> indenter
// vertices, edges -> indenter edges.  A pair is a candidate when the two bounding boxes (each
// swept over the motion under test) come within dhat of each other along every axis; it is
// reported from exactly one cell (the lowest cell of the two boxes' common cell range), counted
// first, prefix-summed, then written, so the candidate list is ordered and identical run to run.
#include <algorithm>

#include "dev_elastic.cuh"
#include "dev_pairwarp.cuh"

namespace txg {

static inline int nblk(int n, int t) { return (n + t - 1) / t; }

constexpr int HMAXC = 1023;       // cell coordinates are clamped to [0, HMAXC]
constexpr int QUERY_CELL_LIMIT = 4096;
constexpr int BUILD_CELL_LIMIT = 512;  // a primitive spanning more cells turns the table brute-force

__device__ __forceinline__ int cell_of(double v, double org, double inv_cell) {
  double c = floor((v - org) * inv_cell);
  c = fmin(fmax(c, 0.0), (double)HMAXC);
  return (int)c;
}
__device__ __forceinline__ unsigned hash_cell(int ix, int iy, int iz) {
  return ((unsigned)ix * 73856093u) ^ ((unsigned)iy * 19349663u) ^ ((unsigned)iz * 83492791u);
}
__device__ __forceinline__ int pack_cell(int ix, int iy, int iz) { return ix | (iy << 10) | (iz << 20); }

struct Box {
  double lo[3], hi[3];
};
__device__ __forceinline__ void box_init(Box& b) {
  for (int c = 0; c < 3; ++c) {
    b.lo[c] = CUDART_INF;
    b.hi[c] = -CUDART_INF;
  }
}
__device__ __forceinline__ void box_add(Box& b, double x, double y, double z) {
  b.lo[0] = fmin(b.lo[0], x); b.hi[0] = fmax(b.hi[0], x);
  b.lo[1] = fmin(b.lo[1], y); b.hi[1] = fmax(b.hi[1], y);
  b.lo[2] = fmin(b.lo[2], z); b.hi[2] = fmax(b.hi[2], z);
}
__device__ __forceinline__ bool near_boxes(const Box& a, const Box& b, double pad) {
  for (int c = 0; c < 3; ++c)
    if (a.lo[c] - pad > b.hi[c] || b.lo[c] - pad > a.hi[c]) return false;
  return true;
}

// bounding box of indenter primitive k of table `tab` (global index), optionally swept
__device__ __forceinline__ Box ind_box(const Dev& d, int tab, int k, bool swept) {
  Box b;
  box_init(b);
  int ids[3], n;
  if (tab == 0) {
    const int4 t = d.it[k];
    ids[0] = t.x; ids[1] = t.y; ids[2] = t.z; n = 3;
  } else if (tab == 1) {
    ids[0] = k; n = 1;
  } else {
    const int2 e = d.ie[k];
    ids[0] = e.x; ids[1] = e.y; n = 2;
  }
  for (int m = 0; m < n; ++m) {
    const double4_32a q = d.iv_cur[ids[m]];
    box_add(b, q.x, q.y, q.z);
    if (swept) {
      const double4_32a r = d.iv_prev[ids[m]];
      box_add(b, r.x, r.y, r.z);
    }
  }
  return b;
}

// bounding box of gel surface primitive (type, global index), optionally swept by p
__device__ __forceinline__ Box gel_box(const Dev& d, int type, int k, bool swept) {
  Box b;
  box_init(b);
  int rows[3], n;
  if (type == PAIR_PT) {
    rows[0] = d.sv[k]; n = 1;
  } else if (type == PAIR_TP) {
    const int4 t = d.st[k];
    rows[0] = t.x; rows[1] = t.y; rows[2] = t.z; n = 3;
  } else {
    const int2 e = d.se[k];
    rows[0] = e.x; rows[1] = e.y; n = 2;
  }
  for (int m = 0; m < n; ++m) {
    const double4_32a x = d.x[rows[m]];
    box_add(b, x.x, x.y, x.z);
    if (swept) {
      const double4_32a p = d.p[rows[m]];
      box_add(b, x.x + p.x, x.y + p.y, x.z + p.z);
    }
  }
  return b;
}

// ---------------------------------------------------------------- indenter placement
__global__ void k_indenter_pose(Dev d, int phase) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.niv_total) return;
  const int g = d.iv_gel[k];
  if (d.gc[g].phase != phase) return;
  const GelCtl& c = d.gc[g];
  const double4_32a v = d.iv_loc[k];
  double4_32a a, b;
  a.x = c.R[0] * v.x + c.R[1] * v.y + c.R[2] * v.z + c.t[0];
  a.y = c.R[3] * v.x + c.R[4] * v.y + c.R[5] * v.z + c.t[1];
  a.z = c.R[6] * v.x + c.R[7] * v.y + c.R[8] * v.z + c.t[2];
  a.w = 0.0;
  b.x = c.Rp[0] * v.x + c.Rp[1] * v.y + c.Rp[2] * v.z + c.tp[0];
  b.y = c.Rp[3] * v.x + c.Rp[4] * v.y + c.Rp[5] * v.z + c.tp[1];
  b.z = c.Rp[6] * v.x + c.Rp[7] * v.y + c.Rp[8] * v.z + c.tp[2];
  b.w = 0.0;
  d.iv_cur[k] = a;
  d.iv_prev[k] = b;
}

// ---------------------------------------------------------------- indenter primitive boxes
__device__ __forceinline__ int pbox_base(const Dev& d, int tab) {
  return tab == 0 ? 0 : (tab == 1 ? d.nit_total : d.nit_total + d.niv_total);
}
__device__ __forceinline__ Box load_pbox(const Dev& d, int tab, int k, int* cell) {
  const int i = pbox_base(d, tab) + k;
  const double4_32a lo = d.pbox[2 * i], hi = d.pbox[2 * i + 1];
  *cell = (int)__double_as_longlong(lo.w);
  Box b;
  b.lo[0] = lo.x; b.lo[1] = lo.y; b.lo[2] = lo.z;
  b.hi[0] = hi.x; b.hi[1] = hi.y; b.hi[2] = hi.z;
  return b;
}

// one thread per indenter primitive of the gels in `phase`: its box (swept from the previous pose
// when asked) and lowest grid cell, read by the hash build and every query until the next build
__global__ void k_ind_boxes(Dev d, int phase, int swept) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nt = d.nit_total, nv = d.niv_total;
  if (i >= nt + nv + d.nie_total) return;
  const int tab = i < nt ? 0 : (i < nt + nv ? 1 : 2);
  const int k = i - (tab == 0 ? 0 : (tab == 1 ? nt : nt + nv));
  const int g = tab == 0 ? d.it_gel[k] : (tab == 1 ? d.iv_gel[k] : d.ie_gel[k]);
  if (d.gc[g].phase != phase) return;
  const GelInfo& G = d.gi[g];
  const Box b = ind_box(d, tab, k, swept != 0);
  const double ic = 1.0 / G.cell;
  const int c = pack_cell(cell_of(b.lo[0], G.org[0], ic), cell_of(b.lo[1], G.org[1], ic),
                          cell_of(b.lo[2], G.org[2], ic));
  d.pbox[2 * i] = make_double4_32a(b.lo[0], b.lo[1], b.lo[2], __longlong_as_double((long long)c));
  d.pbox[2 * i + 1] = make_double4_32a(b.hi[0], b.hi[1], b.hi[2], 0.0);
}

// ---------------------------------------------------------------- hash build (one CTA per table)
constexpr int HB_THREADS = 256;

__global__ void __launch_bounds__(HB_THREADS) k_hash_build(Dev d, int phase, int swept) {
  const int g = blockIdx.x / NTAB, tab = blockIdx.x % NTAB;
  if (d.gc[g].phase != phase) return;
  const GelInfo& G = d.gi[g];
  const int nb = G.hnb[tab], hb = G.hb0[tab], he = G.he0[tab], cap = G.hcap[tab];
  const int n = tab == 0 ? G.nit : (tab == 1 ? G.niv : G.nie);
  const int p0 = tab == 0 ? G.it0 : (tab == 1 ? G.iv0 : G.ie0);
  const double ic = 1.0 / G.cell;
  int* cnt = d.hcount + hb;
  int* start = d.hstart + hb;
  __shared__ int s_carry;
  __shared__ int s_brute;
  __shared__ int s_part[HB_THREADS];
  if (threadIdx.x == 0) s_brute = 0;
  for (int b = threadIdx.x; b <= nb; b += blockDim.x) cnt[b] = 0;
  __syncthreads();
  Box all;  // the indenter's bounding box (vertex table only)
  box_init(all);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    int c0;
    const Box bx = load_pbox(d, tab, p0 + k, &c0);
    for (int c = 0; c < 3; ++c) {
      all.lo[c] = fmin(all.lo[c], bx.lo[c]);
      all.hi[c] = fmax(all.hi[c], bx.hi[c]);
    }
    const int x0 = c0 & HMAXC, x1 = cell_of(bx.hi[0], G.org[0], ic);
    const int y0 = (c0 >> 10) & HMAXC, y1 = cell_of(bx.hi[1], G.org[1], ic);
    const int z0 = c0 >> 20, z1 = cell_of(bx.hi[2], G.org[2], ic);
    if ((x1 - x0 + 1) * (y1 - y0 + 1) * (z1 - z0 + 1) > BUILD_CELL_LIMIT) {
      s_brute = 1;
      continue;
    }
    for (int iz = z0; iz <= z1; ++iz)
      for (int iy = y0; iy <= y1; ++iy)
        for (int ix = x0; ix <= x1; ++ix) atomicAdd(&cnt[hash_cell(ix, iy, iz) & (nb - 1)], 1);
  }
  if (tab == 1) {  // min / max are exact: any reduction order gives the same box
    __shared__ double s_box[HB_THREADS / 32][6];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c = 0; c < 3; ++c) {
      all.lo[c] = warp_min(all.lo[c]);
      all.hi[c] = warp_max(all.hi[c]);
    }
    if (lane == 0)
      for (int c = 0; c < 3; ++c) {
        s_box[wid][c] = all.lo[c];
        s_box[wid][3 + c] = all.hi[c];
      }
    __syncthreads();
    if (threadIdx.x < 3) {
      const int c = threadIdx.x;
      double lo = s_box[0][c], hi = s_box[0][3 + c];
      for (int w = 1; w < HB_THREADS / 32; ++w) {
        lo = fmin(lo, s_box[w][c]);
        hi = fmax(hi, s_box[w][3 + c]);
      }
      d.gv[g].ibox_lo[c] = lo;
      d.gv[g].ibox_hi[c] = hi;
    }
  }
  __syncthreads();
  if (s_brute) {  // oversized primitive: every query of this table tests all primitives directly
    for (int b = threadIdx.x; b <= nb; b += blockDim.x) start[b] = 0;
    if (threadIdx.x == 0) d.gv[g].hent[tab] = -1;
    return;
  }
  // exclusive scan of the bucket counts: every thread scans a contiguous chunk serially, one
  // block-wide scan of the chunk totals
  const int per = (nb + HB_THREADS - 1) / HB_THREADS;
  const int b0 = min(nb, (int)threadIdx.x * per), b1 = min(nb, b0 + per);
  int own = 0;
  for (int b = b0; b < b1; ++b) own += cnt[b];
  s_part[threadIdx.x] = own;
  __syncthreads();
  for (int off = 1; off < HB_THREADS; off <<= 1) {
    const int t = threadIdx.x >= off ? s_part[threadIdx.x - off] : 0;
    __syncthreads();
    s_part[threadIdx.x] += t;
    __syncthreads();
  }
  int run = s_part[threadIdx.x] - own;
  for (int b = b0; b < b1; ++b) {
    const int c = cnt[b];
    start[b] = run;
    cnt[b] = run;  // fill cursor of the scatter below
    run += c;
  }
  if (threadIdx.x == HB_THREADS - 1) s_carry = s_part[HB_THREADS - 1];
  __syncthreads();
  const int total = s_carry;
  if (threadIdx.x == 0) {
    start[nb] = total;
    d.gv[g].hent[tab] = total;
    if (total > cap) atomicOr(&d.gv[g].flags, 1);
  }
  if (total > cap) {  // leave an empty table; the host grows the capacity and rebuilds
    __syncthreads();
    for (int b = threadIdx.x; b <= nb; b += blockDim.x) start[b] = 0;
    return;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    int c0;
    const Box bx = load_pbox(d, tab, p0 + k, &c0);
    const int x0 = c0 & HMAXC, x1 = cell_of(bx.hi[0], G.org[0], ic);
    const int y0 = (c0 >> 10) & HMAXC, y1 = cell_of(bx.hi[1], G.org[1], ic);
    const int z0 = c0 >> 20, z1 = cell_of(bx.hi[2], G.org[2], ic);
    for (int iz = z0; iz <= z1; ++iz)
      for (int iy = y0; iy <= y1; ++iy)
        for (int ix = x0; ix <= x1; ++ix) {
          const int pos = atomicAdd(&cnt[hash_cell(ix, iy, iz) & (nb - 1)], 1);
          d.hent[he + pos] = make_int2(p0 + k, pack_cell(ix, iy, iz));
        }
  }
}

// deterministic order inside every bucket (the scatter above fills them in arrival order): one
// thread per bucket, insertion sort by (primitive, cell); blockIdx.y = gel * NTAB + table
__global__ void k_hash_sort(Dev d, int phase) {
  const int g = blockIdx.y / NTAB, tab = blockIdx.y % NTAB;
  if (d.gc[g].phase != phase) return;
  const GelInfo& G = d.gi[g];
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= G.hnb[tab] || d.gv[g].hent[tab] < 0 || d.gv[g].hent[tab] > G.hcap[tab]) return;
  const int* start = d.hstart + G.hb0[tab];
  int2* e = d.hent + G.he0[tab];
  const int s = start[b], t = start[b + 1];
  for (int i = s + 1; i < t; ++i) {
    const int2 key = e[i];
    int j = i - 1;
    while (j >= s) {
      const int2 o = e[j];
      if (o.x < key.x || (o.x == key.x && o.y <= key.y)) break;
      e[j + 1] = o;
      --j;
    }
    e[j + 1] = key;
  }
}

// ---------------------------------------------------------------- hash query
// mode bit 0: write (else count); bit 1: gel boxes swept by p; bit 3: skip gels whose Newton
// iteration converged.  Counts of gels outside `phase` are left untouched: every gel only uses
// the offsets of its own queries relative to its first one.  The indenter boxes (swept or not)
// were stored by the last hash build of the gel.
//
// Two kernels: one thread per gel surface primitive drops those nowhere near the indenter's box
// (count 0) and lists the others; then, for a short list (a single gel: latency matters), one
// warp per listed primitive walks its cells, a lane per cell (a lane per indenter primitive when
// the box is too large for the hash or the table is brute force), and a warp scan of the lanes'
// counts places every candidate; for a long list (batches: throughput matters) one thread per
// listed primitive walks them serially.  Either way the order is the cell order (z, y, x) and the
// bucket order within a cell.

struct QueryCtx {
  int g, type, gk, tab;
  Box qb;
  double pad, ic;
  int lo[3], hi[3];
  long long ncell;
  bool brute;
};

__device__ __forceinline__ bool query_ctx(const Dev& d, int q, int phase, int mode, QueryCtx& c) {
  const bool gsw = (mode >> 1) & 1, skc = (mode >> 3) & 1;
  c.g = d.q_gel[q];
  if (d.gc[c.g].phase != phase) return false;
  if (skc && d.gv[c.g].converged) return false;
  const GelInfo& G = d.gi[c.g];
  const int tp = d.q_tp[q];
  c.type = tp >> 28;
  const int loc = tp & ((1 << 28) - 1);
  c.gk = (c.type == PAIR_PT ? G.sv0 : (c.type == PAIR_TP ? G.st0 : G.se0)) + loc;
  c.tab = c.type;
  c.qb = gel_box(d, c.type, c.gk, gsw);
  c.pad = G.dhat;
  c.ic = 1.0 / G.cell;
  for (int k = 0; k < 3; ++k) {
    c.lo[k] = cell_of(c.qb.lo[k] - c.pad, G.org[k], c.ic);
    c.hi[k] = cell_of(c.qb.hi[k] + c.pad, G.org[k], c.ic);
  }
  c.ncell = (long long)(c.hi[0] - c.lo[0] + 1) * (c.hi[1] - c.lo[1] + 1) * (c.hi[2] - c.lo[2] + 1);
  c.brute = c.ncell > QUERY_CELL_LIMIT || d.gv[c.g].hent[c.tab] < 0;
  return true;
}

__global__ void k_query_near(Dev d, int phase, int mode) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= d.nq) return;
  QueryCtx c;
  if (!query_ctx(d, q, phase, mode, c)) return;
  Box ib;
  for (int k = 0; k < 3; ++k) {
    ib.lo[k] = d.gv[c.g].ibox_lo[k];
    ib.hi[k] = d.gv[c.g].ibox_hi[k];
  }
  if (!near_boxes(c.qb, ib, c.pad)) {  // nowhere near the indenter
    d.qcount[q] = 0;
    return;
  }
  d.qnear[atomicAdd(d.qnear_n, 1)] = q;
}

// matches of indenter primitive entry `ent` found in cell (ix, iy, iz) of the query
__device__ __forceinline__ bool query_match(const Dev& d, const QueryCtx& c, int2 ent, int ix, int iy, int iz) {
  if (ent.y != pack_cell(ix, iy, iz)) return false;
  int c0;
  const Box pb = load_pbox(d, c.tab, ent.x, &c0);
  const int px = c0 & HMAXC, py = (c0 >> 10) & HMAXC, pz = c0 >> 20;
  if (ix != max(c.lo[0], px) || iy != max(c.lo[1], py) || iz != max(c.lo[2], pz)) return false;
  return near_boxes(c.qb, pb, c.pad);
}

// one thread per listed primitive: its cells and buckets walked serially (throughput mode, for
// lists much longer than the grid's warps)
__device__ void query_thread(const Dev& d, int q, int phase, int mode) {
  const bool write = mode & 1;
  QueryCtx c;
  query_ctx(d, q, phase, mode, c);
  const GelInfo& G = d.gi[c.g];
  const int base = write ? d.qoff[q] - d.qoff[G.q0] : 0;
  int count = 0;
  auto emit = [&](int P) {
    if (write && base + count < G.pcap) d.pairs[G.pbase + base + count] = make_int4(c.type, c.gk, P, c.g);
    ++count;
  };
  if (c.brute) {
    const int np = c.tab == 0 ? G.nit : (c.tab == 1 ? G.niv : G.nie);
    const int p0 = c.tab == 0 ? G.it0 : (c.tab == 1 ? G.iv0 : G.ie0);
    for (int k = 0; k < np; ++k) {
      int cc;
      const Box pb = load_pbox(d, c.tab, p0 + k, &cc);
      if (near_boxes(c.qb, pb, c.pad)) emit(p0 + k);
    }
  } else {
    const int nb = G.hnb[c.tab], hb = G.hb0[c.tab], he = G.he0[c.tab];
    for (int iz = c.lo[2]; iz <= c.hi[2]; ++iz)
      for (int iy = c.lo[1]; iy <= c.hi[1]; ++iy)
        for (int ix = c.lo[0]; ix <= c.hi[0]; ++ix) {
          const int bk = hash_cell(ix, iy, iz) & (nb - 1);
          const int s = d.hstart[hb + bk], e = d.hstart[hb + bk + 1];
          for (int m = s; m < e; ++m) {
            const int2 ent = d.hent[he + m];
            if (query_match(d, c, ent, ix, iy, iz)) emit(ent.x);
          }
        }
  }
  if (!write) d.qcount[q] = count;
}

__global__ void __launch_bounds__(128) k_query_list(Dev d, int phase, int mode) {
  const bool write = mode & 1;
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * (blockDim.x >> 5);
  const int n = *d.qnear_n;
  if (n > 4 * nw) {  // long list: a thread per primitive keeps every lane busy
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      query_thread(d, d.qnear[i], phase, mode);
    return;
  }
  for (int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < n; w += nw) {
    const int q = d.qnear[w];
    QueryCtx c;
    query_ctx(d, q, phase, mode, c);
    const GelInfo& G = d.gi[c.g];
    int base = write ? d.qoff[q] - d.qoff[G.q0] : 0;
    int total = 0;
    if (c.brute) {
      const int np = c.tab == 0 ? G.nit : (c.tab == 1 ? G.niv : G.nie);
      const int p0 = c.tab == 0 ? G.it0 : (c.tab == 1 ? G.iv0 : G.ie0);
      for (int k0 = 0; k0 < np; k0 += 32) {
        const int k = k0 + lane;
        bool hit = false;
        if (k < np) {
          int cc;
          const Box pb = load_pbox(d, c.tab, p0 + k, &cc);
          hit = near_boxes(c.qb, pb, c.pad);
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (write && hit) {
          const int pos = base + total + __popc(m & ((1u << lane) - 1u));
          if (pos < G.pcap) d.pairs[G.pbase + pos] = make_int4(c.type, c.gk, p0 + k, c.g);
        }
        total += __popc(m);
      }
    } else {
      const int nx = c.hi[0] - c.lo[0] + 1, ny = c.hi[1] - c.lo[1] + 1;
      const int nb = G.hnb[c.tab], hb = G.hb0[c.tab], he = G.he0[c.tab];
      // 32 cells at a time: a lane per cell reads its bucket's range; the bucket entries of the
      // 32 cells are then checked a lane per entry (owner cell found by a binary search over the
      // lanes' exclusive offsets), so no lane walks a bucket serially
      for (long long ci0 = 0; ci0 < c.ncell; ci0 += 32) {
        const long long ci = ci0 + lane;
        int cnt = 0, s = 0, ix = 0, iy = 0, iz = 0;
        if (ci < c.ncell) {
          ix = c.lo[0] + (int)(ci % nx);
          iy = c.lo[1] + (int)((ci / nx) % ny);
          iz = c.lo[2] + (int)(ci / ((long long)nx * ny));
          const int bk = hash_cell(ix, iy, iz) & (nb - 1);
          s = d.hstart[hb + bk];
          cnt = d.hstart[hb + bk + 1] - s;
        }
        int ex = cnt;  // inclusive, then exclusive warp scan of the entry counts
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, ex, o);
          if (lane >= o) ex += t;
        }
        const int T = __shfl_sync(0xffffffffu, ex, 31);
        ex -= cnt;
        for (int j0 = 0; j0 < T; j0 += 32) {
          const int j = j0 + lane;
          int L = 0;  // the last lane whose offset is <= j: it owns entry j (its count is > 0)
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int e2 = __shfl_sync(0xffffffffu, ex, L + step);
            if (e2 <= j) L += step;
          }
          const int sL = __shfl_sync(0xffffffffu, s, L), eL = __shfl_sync(0xffffffffu, ex, L);
          const int xL = __shfl_sync(0xffffffffu, ix, L), yL = __shfl_sync(0xffffffffu, iy, L);
          const int zL = __shfl_sync(0xffffffffu, iz, L);
          bool hit = false;
          int P = 0;
          if (j < T) {
            const int2 ent = d.hent[he + sL + (j - eL)];
            hit = query_match(d, c, ent, xL, yL, zL);
            P = ent.x;
          }
          const unsigned m = __ballot_sync(0xffffffffu, hit);
          if (write && hit) {
            const int pos = base + total + __popc(m & ((1u << lane) - 1u));
            if (pos < G.pcap) d.pairs[G.pbase + pos] = make_int4(c.type, c.gk, P, c.g);
          }
          total += __popc(m);
        }
      }
    }
    if (!write && lane == 0) d.qcount[q] = total;
  }
}

__global__ void k_pair_ranges(Dev d, int phase, int skip_conv) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= d.n_gels) return;
  if (d.gc[g].phase != phase) return;
  if (skip_conv && d.gv[g].converged) return;
  const GelInfo& G = d.gi[g];
  const int n = d.qoff[G.q0 + G.nq] - d.qoff[G.q0];
  d.gv[g].pair0 = G.pbase;
  d.gv[g].npair = n;
  if (n > G.pcap) atomicOr(&d.gv[g].flags, 32);
}

// ---------------------------------------------------------------- soft-soft candidates
// A gel whose mesh has several connected components (bodies) also pairs the surfaces of its
// different bodies: every surface vertex with every surface triangle of another body, and every
// two surface edges of different bodies (each unordered pair once), by the box rule of the
// indenter pairs (primitive boxes -- swept by p in Newton mode -- within d_hat on every axis).
// Three launches: the bodies' boxes (a CTA per soft-soft gel), the surface primitives near the box
// of another body (listed), then every listed pair tested by brute force and appended after the
// gel's indenter pairs.  mode bit 1: boxes swept by p; bit 3: skip gels whose Newton converged.
constexpr int SS_T = 256;

__device__ __forceinline__ bool ss_active(const Dev& d, int g, int phase, int mode) {
  return d.gc[g].phase == phase && !((mode & 8) && d.gv[g].converged);
}

__global__ void __launch_bounds__(SS_T) k_ss_boxes(Dev d, int phase, int mode) {
  __shared__ double sm[SS_T / 32][SS_MAXC * 6];
  const int j = blockIdx.x, g = d.ss_gel[j];
  if (!ss_active(d, g, phase, mode)) return;
  const GelInfo& G = d.gi[g];
  double bx[SS_MAXC * 6];  // per component: lo[3], then -hi[3] (all reduced by min)
#pragma unroll
  for (int e = 0; e < SS_MAXC * 6; ++e) bx[e] = CUDART_INF;
  for (int k = threadIdx.x; k < G.nsv; k += SS_T) {
    const int c = d.vcomp[d.sv[G.sv0 + k]];
    const Box b = gel_box(d, PAIR_PT, G.sv0 + k, (mode & 2) != 0);
#pragma unroll
    for (int q = 0; q < SS_MAXC; ++q)
      if (q == c)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          bx[6 * q + a] = fmin(bx[6 * q + a], b.lo[a]);
          bx[6 * q + 3 + a] = fmin(bx[6 * q + 3 + a], -b.hi[a]);
        }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int e = 0; e < SS_MAXC * 6; ++e) {
    double v = bx[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) sm[wid][e] = v;
  }
  __syncthreads();
  if (threadIdx.x < SS_MAXC * 6) {
    double v = CUDART_INF;
    for (int w = 0; w < SS_T / 32; ++w) v = fmin(v, sm[w][threadIdx.x]);
    const int a = threadIdx.x % 6;
    d.ss_box[(size_t)j * SS_MAXC * 6 + threadIdx.x] = a < 3 ? v : -v;
  }
  if (threadIdx.x < 3) d.ss_cnt[3 * j + threadIdx.x] = 0;
}

// type (PAIR_PT / PAIR_TP / PAIR_EE as the kind of surface primitive), global index, sub-list and
// first row of query q of gel G
__device__ __forceinline__ void ss_prim(const Dev& d, const GelInfo& G, int q, int& type, int& gk, int& t, int& r) {
  if (q < G.nsv) {
    type = PAIR_PT; gk = G.sv0 + q; t = 0; r = d.sv[gk];
  } else if (q < G.nsv + G.nst) {
    type = PAIR_TP; gk = G.st0 + q - G.nsv; t = 1; r = d.st[gk].x;
  } else {
    type = PAIR_EE; gk = G.se0 + q - G.nsv - G.nst; t = 2; r = d.se[gk].x;
  }
}

__global__ void __launch_bounds__(SS_T) k_ss_filter(Dev d, int phase, int mode) {
  const int j = blockIdx.y, g = d.ss_gel[j];
  if (!ss_active(d, g, phase, mode)) return;
  const GelInfo& G = d.gi[g];
  const double* cb = d.ss_box + (size_t)j * SS_MAXC * 6;
  const int nc = min(G.ncomp, SS_MAXC);
  for (int q = blockIdx.x * SS_T + threadIdx.x; q < G.nq; q += gridDim.x * SS_T) {
    int type, gk, t, r;
    ss_prim(d, G, q, type, gk, t, r);
    const int c = d.vcomp[r];
    const Box b = gel_box(d, type, gk, (mode & 2) != 0);
    bool near = false;
    for (int o = 0; o < nc; ++o) {
      if (o == c) continue;
      Box ob;
      for (int a = 0; a < 3; ++a) {
        ob.lo[a] = cb[6 * o + a];
        ob.hi[a] = cb[6 * o + 3 + a];
      }
      near = near || near_boxes(b, ob, G.dhat);
    }
    if (near) {
      const int base = t == 0 ? 0 : (t == 1 ? G.nsv : G.nsv + G.nst);
      d.ss_list[G.q0 + base + atomicAdd(&d.ss_cnt[3 * j + t], 1)] = gk;
    }
  }
}

__global__ void __launch_bounds__(SS_T) k_ss_pairs(Dev d, int phase, int mode) {
  const int j = blockIdx.y, g = d.ss_gel[j];
  if (!ss_active(d, g, phase, mode)) return;
  const GelInfo& G = d.gi[g];
  const bool sw = (mode & 2) != 0;
  const int nv = d.ss_cnt[3 * j], nt = d.ss_cnt[3 * j + 1], ne = d.ss_cnt[3 * j + 2];
  const int* lv = d.ss_list + G.q0;
  const int* lt = lv + G.nsv;
  const int* le = lt + G.nst;
  const long long n1 = (long long)nv * nt, n = n1 + (long long)ne * ne;
  for (long long w = (long long)blockIdx.x * SS_T + threadIdx.x; w < n; w += (long long)gridDim.x * SS_T) {
    int type, a, b, ra, rb;
    Box ba, bb;
    if (w < n1) {  // surface vertex vs surface triangle
      type = PAIR_SPT;
      a = lv[w / nt];
      b = lt[w % nt];
      ra = d.sv[a];
      rb = d.st[b].x;
      if (d.vcomp[ra] == d.vcomp[rb]) continue;
      ba = gel_box(d, PAIR_PT, a, sw);
      bb = gel_box(d, PAIR_TP, b, sw);
    } else {  // two surface edges, the first earlier in the list
      const long long u = w - n1;
      const int i = (int)(u / ne), k = (int)(u % ne);
      if (k <= i) continue;
      type = PAIR_SEE;
      a = le[i];
      b = le[k];
      ra = d.se[a].x;
      rb = d.se[b].x;
      if (d.vcomp[ra] == d.vcomp[rb]) continue;
      ba = gel_box(d, PAIR_EE, a, sw);
      bb = gel_box(d, PAIR_EE, b, sw);
    }
    if (!near_boxes(ba, bb, G.dhat)) continue;
    const int pos = atomicAdd(&d.gv[g].npair, 1);
    if (pos < G.pcap)
      d.pairs[G.pbase + pos] = make_int4(type, a, b, g);
    else
      atomicOr(&d.gv[g].flags, 32);  // the host grows the segment and redoes the search
  }
}

// the soft-soft candidates of the soft-soft gels in `phase`; returns the launches made
int launch_ss_pairs(const Dev& d, int phase, int mode, cudaStream_t st) {
  if (d.n_ss <= 0) return 0;
  k_ss_boxes<<<d.n_ss, SS_T, 0, st>>>(d, phase, mode);
  k_ss_filter<<<dim3(std::max(1, std::min(64, (d.ss_maxq + SS_T - 1) / SS_T)), d.n_ss), SS_T, 0, st>>>(d, phase, mode);
  k_ss_pairs<<<dim3(std::max(8, 592 / d.n_ss), d.n_ss), SS_T, 0, st>>>(d, phase, mode);
  count_launch(3);
  return 3;
}

// the pair in slot i, if its gel is in `phase` (and, optionally, not converged)
__device__ __forceinline__ bool pair_slot(const Dev& d, int i, int phase, bool skip_conv, int4& pr) {
  const int g = d.pslot_gel[i];
  if (d.gc[g].phase != phase) return false;
  if (skip_conv && d.gv[g].converged) return false;
  if (i - d.gi[g].pbase >= min(d.gv[g].npair, d.gi[g].pcap)) return false;
  pr = d.pairs[i];
  return true;
}

// ---------------------------------------------------------------- barrier assembly
__device__ __forceinline__ int find_block(const Dev& d, int row, int col) {
  const int s = row >> 5, lane = row & 31;
  const int o = d.slice_off[s], w = (d.slice_off[s + 1] - o) >> 5;
  for (int k = 0; k < w; ++k) {
    const int bp = o + 32 * k + lane;
    if (d.colidx[bp] == col) return bp;
  }
  return -1;
}

// Block (row, col) of a soft-soft pair between two bodies: not in the mesh pattern, so it takes a
// free slot of the row (a padding position: column = the row itself, past the diagonal, value 0
// after the gather) by a compare-and-swap of its column, listed for the reset before the next
// assembly.  Every claimer of a row walks its slots in the same order and takes the first free
// one, and a failed swap shows the column that won it, so a block gets one slot however many
// pairs claim it at once (a slot never becomes free again before the reset).  -1: no free slot.
__device__ __forceinline__ int claim_block(const Dev& d, int row, int col) {
  const int s = row >> 5, lane = row & 31;
  const int o = d.slice_off[s], w = (d.slice_off[s + 1] - o) >> 5, dg = d.diag_pos[row];
  for (int k = 0; k < w; ++k) {
    const int bp = o + 32 * k + lane;
    const int c = d.colidx[bp];
    if (c == col) return bp;
    if (c != row || bp == dg) continue;
    const int old = atomicCAS(&d.colidx[bp], row, col);
    if (old == col) return bp;  // another pair claimed this block here first
    if (old != row) continue;   // another block took the slot
    const int q = atomicAdd(d.ss_nclaim, 1);
    if (q < d.ss_claim_cap) {
      d.ss_claim[q] = bp;
      return bp;
    }
    return -1;  // not reached: the list holds every padding slot of the soft-soft gels
  }
  return -1;
}

// Reset of the claimed slots (one CTA; before the contact assembly of every Newton iteration)
__global__ void k_ss_reset(Dev d) {
  const int n = min(*d.ss_nclaim, d.ss_claim_cap);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int bp = d.ss_claim[k];
    d.colidx[bp] = d.bp_row[bp];
  }
  __syncthreads();
  if (threadIdx.x == 0) *d.ss_nclaim = 0;
}

void launch_ss_reset(const Dev& d, cudaStream_t st) {
  k_ss_reset<<<1, 512, 0, st>>>(d);
  count_launch(1);
}

// Contact assembly, part 1: one thread per candidate slot.  Active pairs (d < dhat) add their
// barrier gradient and the contact force; a pair whose value depends on a single gel point adds
// its projected block in closed form (the Hessian of b(d(P)) in the one free point is
// b'' u u^T + b' grad^2 d with u = grad d, grad^2 d PSD and orthogonal to u, b' < 0, so the
// projection keeps max(b'', 0) u u^T); pairs with two or three free gel points are listed for
// the warp kernel below.
template <bool MIXED>
__global__ void __launch_bounds__(128) k_contact_pairs(Dev d, int phase) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.npslots) return;
  int4 pr;
  if (!pair_slot(d, i, phase, false, pr)) return;
  const int g = pr.w;
  const GelInfo& G = d.gi[g];
  double P[4][3];
  int rows[4];
  pair_points(d, pr, 0.0, false, P, rows);
  PairBarrier pb;
  if (!pair_barrier_setup(pair_kind(pr.x), P, G.dhat, pair_eps_x(d, pr), pb)) return;
  atomicAdd(&d.gv[g].active_pairs, 1);
  const double kap = d.gc[g].kappa;  // the step's barrier stiffness (host-set, adaptive)
  int slots[4], ns = 0;
  for (int k = 0; k < 4; ++k)
    if (rows[k] >= 0 && (pb.involved >> k) & 1) slots[ns++] = k;
  const bool rigid = pr.x < PAIR_SPT;  // soft-soft forces are internal: not in the indenter force
  for (int a = 0; a < ns; ++a) {
    const int ra = rows[slots[a]];
    double gr[3];
    for (int c = 0; c < 3; ++c) {
      gr[c] = kap * pair_grad_entry(pb, 3 * slots[a] + c);
      if (rigid) atomicAdd(&d.gv[g].fc[c], -gr[c]);
    }
    if (d.fixed[ra]) continue;
    atomicAdd(&d.cgrad[ra].x, gr[0]);
    atomicAdd(&d.cgrad[ra].y, gr[1]);
    atomicAdd(&d.cgrad[ra].z, gr[2]);
  }
  if (ns == 1) {
    const int ra = rows[slots[0]];
    if (d.fixed[ra]) return;
    const double dd = sqrt(pb.dv.D), r = dd - G.dhat;
    const double bpp = -2.0 * log(dd / G.dhat) - 4.0 * r / dd + r * r / (dd * dd);
    double H3[9];
    single_point_block(bpp, pb.gDp + 3 * slots[0], H3);
    C1Rec& rec = d.c1rec[atomicAdd(d.c1_n, 1)];  // at most one per slot: never past npslots
    rec.bp = d.diag_pos[ra];
    for (int e = 0; e < 9; ++e) rec.v[e] = kap * H3[e];
  } else if (ns > 1) {
    const int pos = atomicAdd(d.cwork_n, 1);
    d.cwork[pos] = i;
    if (pos < d.crec_cap) d.crec[pos] = pb;  // the warp kernel starts from this setup
  }
}

// Contact assembly, part 2: one warp per listed pair.  Its lanes form the barrier Hessian block
// on the pair's free gel points (team_pair_block), project it to PSD and scale it by kappa.  (A
// CTA of four warps per pair measured no faster: the projection is bound by the latency of its
// Jacobi rounds, not by FP64 issue, and batches lose pairs in flight.)  Mode 0 (may run beside
// the elastic assembly): the first crec_cap listed pairs, starting from the setup part 1 stored;
// the result and its block positions go to the pair's record.  Mode 1 (after the gather wrote
// the matrix): the recorded blocks and the single-point blocks of part 1 are added to the gel's
// BSR; pairs beyond the record capacity are formed here (setup recomputed by one lane) and added
// directly.
constexpr int CW_WARPS = 4;

struct ContactWS {
  PairBarrier pb;
  ProjWS pj;
  double P[4][3];
  int rows[4], slots[4], fd[PW_MAXN], bp[16];
  int ns, g;
};

template <bool MIXED>
__device__ __forceinline__ void add_val(const Dev& d, int bp, int e, double v) {
  if (MIXED)
    atomicAdd(&d.vals32[val_addr32(bp, e)], (float)v);
  else
    atomicAdd(&d.vals[val_addr64(bp, e)], v);
}

template <bool MIXED>
__global__ void __launch_bounds__(32 * CW_WARPS) k_contact_hess(Dev d, int mode) {
  __shared__ ContactWS sws[CW_WARPS];
  ContactWS& w = sws[threadIdx.x >> 5];
  const Team<32> tm{(int)(threadIdx.x & 31), nullptr};
  const int wid = blockIdx.x * CW_WARPS + (threadIdx.x >> 5), nw = gridDim.x * CW_WARPS;
  const int n = *d.cwork_n;
  const int nrec = min(n, d.crec_cap);
  if (mode == 1) {
    // single-point blocks: a thread per record
    const int n1 = *d.c1_n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n1; k += gridDim.x * blockDim.x) {
      const C1Rec& r = d.c1rec[k];
      for (int e = 0; e < 9; ++e) add_val<MIXED>(d, r.bp, e, r.v[e]);
    }
    // recorded pair blocks: a warp per pair
    for (int k = wid; k < nrec; k += nw) {
      const int* bpk = d.chbp + (size_t)k * CH_BP;
      const int ns = bpk[0], nf = 3 * ns;
      const double* hv = d.chv + (size_t)k * CH_STRIDE;
      for (int e = tm.id; e < nf * nf; e += 32) {
        const int r = e / nf, c = e - r * nf;
        const int bp = bpk[1 + (r / 3) * ns + c / 3];
        if (bp >= 0) add_val<MIXED>(d, bp, 3 * (r % 3) + c % 3, hv[e]);
      }
    }
  }
  const int k0 = mode == 0 ? 0 : nrec, k1 = mode == 0 ? nrec : n;
  for (int k = k0 + wid; k < k1; k += nw) {
    const int i = d.cwork[k];
    if (k < d.crec_cap) {
      const double* src = reinterpret_cast<const double*>(d.crec + k);
      double* dst = reinterpret_cast<double*>(&w.pb);
      for (int q = tm.id; q < (int)(sizeof(PairBarrier) / sizeof(double)); q += 32) dst[q] = src[q];
    }
    if (tm.id == 0) {
      const int4 pr = d.pairs[i];
      const GelInfo& G = d.gi[pr.w];
      int rows[4];
      if (k >= d.crec_cap) {
        pair_points(d, pr, 0.0, false, w.P, rows);
        pair_barrier_setup(pair_kind(pr.x), w.P, G.dhat, pair_eps_x(d, pr), w.pb);
      } else {
        pair_rows(d, pr, rows);
      }
      int ns = 0;
      for (int q = 0; q < 4; ++q) {
        w.rows[q] = rows[q];
        if (rows[q] >= 0 && (w.pb.involved >> q) & 1) w.slots[ns++] = q;
      }
      for (int q = 0; q < 3 * ns; ++q) w.fd[q] = 3 * w.slots[q / 3] + q % 3;
      w.ns = ns;
      w.g = pr.w;
    }
    __syncwarp();
    const int ns = w.ns, nf = 3 * ns, m = nf + (nf & 1);
    team_pair_block(w.pb, w.fd, nf, m, w.pj.T, w.pj.H, tm);
    team_psd_project(w.pj, nf, tm);
    const int g = w.g;
    // a soft-soft pair's blocks between its two bodies claim free slots; if one finds none, all of
    // them are left out (the pair's block-diagonal part, its principal submatrices on each body,
    // is PSD on its own, so the matrix stays PSD and the direction a descent one)
    bool cross = false, miss = false;
    int bp = -1;
    if (tm.id < ns * ns) {
      const int a = tm.id / ns, c = tm.id - a * ns;
      const int ra = w.rows[w.slots[a]], rc = w.rows[w.slots[c]];
      if (!d.fixed[ra] && !d.fixed[rc]) {
        cross = d.gi[g].ncomp > 1 && d.vcomp[ra] != d.vcomp[rc];
        bp = cross ? claim_block(d, ra, rc) : find_block(d, ra, rc);
        if (bp < 0) {
          if (cross) miss = true;
          else atomicOr(&d.gv[g].flags, 16);
        }
      }
    }
    if (__any_sync(0xffffffffu, miss)) {
      if (cross) bp = -1;
      if (tm.id == 0) atomicAdd(&d.gv[g].ss_cut, 1);
    }
    if (tm.id < ns * ns) {
      w.bp[tm.id] = bp;
      if (mode == 0) d.chbp[(size_t)k * CH_BP + 1 + tm.id] = bp;
    }
    if (mode == 0 && tm.id == 0) d.chbp[(size_t)k * CH_BP] = ns;
    __syncwarp();
    const double kap = d.gc[g].kappa;
    for (int e = tm.id; e < nf * nf; e += 32) {
      const int r = e / nf, c = e - r * nf;
      const double v = kap * w.pj.H[r * m + c];
      if (mode == 0) {
        d.chv[(size_t)k * CH_STRIDE + e] = v;
      } else {
        const int bp = w.bp[(r / 3) * ns + c / 3];
        if (bp >= 0) add_val<MIXED>(d, bp, 3 * (r % 3) + c % 3, v);
      }
    }
    __syncwarp();  // w is reused by the warp's next pair
  }
}

// ---------------------------------------------------------------- lagged friction
// IPC's lagged friction (Li et al. 2020, Sec. 5; TacEx App. A notes that IPC models static and
// dynamic friction).  For a pair in contact at the start of the (sub)step,
//   D(x) = mu_f lam f0(|u|),   u = T^T sum_k w_k (P_k - Plag_k)  (tangential relative displacement),
// with the weights w, the tangent basis T and the normal force lam = kappa m |b'(d)| held at their
// values at the start, and the smoothed Coulomb law of IPC with e = eps_v h:
//   f0(y) = y for y >= e,   f0(y) = -y^3 / (3 e^2) + y^2 / e + e / 3 below.
// In u: grad f0 = phi u, Hessian = phi I + psi u u^T, with phi = f0'(y) / y and
// psi = (f0''(y) - phi) / y^2: for y >= e phi = 1 / y, psi = -1 / y^3; below, phi = 2 / e - y / e^2,
// psi = -1 / (e^2 y) (its u u^T term vanishes with y).  Its eigenvalues, phi across u and f0'' >= 0
// along it, are non-negative: D is convex in x and needs no projection.

// f0(y), phi, psi at |u| = y
__device__ __forceinline__ void coulomb_f0(double y, double e, double* f0, double* phi, double* psi) {
  if (y >= e) {
    *f0 = y;
    *phi = 1.0 / y;
    *psi = -1.0 / (y * y * y);
    return;
  }
  const double ie = 1.0 / e;
  *f0 = y * y * (ie - y * ie * ie / 3.0) + e / 3.0;
  *phi = ie * (2.0 - y * ie);
  *psi = y > 0.0 ? -ie * ie / y : 0.0;
}

// Lagged data of each candidate pair of a gel starting a (sub)step: gel at x_n (attached vertices
// already placed), indenter at its pose at the substep's start.  The records cover the gel's
// candidate list of that moment (the swept list of the placement check, a superset of the pairs
// within d_hat); pairs not in contact are marked inactive.
__global__ void __launch_bounds__(128) k_fric_setup(Dev d, int phase) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.npslots) return;
  const int g = d.pslot_gel[i];
  const GelInfo& G = d.gi[g];
  if (d.gc[g].phase != phase || !(G.mu_f > 0.0)) return;
  const int k = i - G.pbase, np = min(d.gv[g].npair, G.pcap);
  if (k == 0) d.gv[g].nfric = np;
  if (k >= np) return;
  FricRec& f = d.fric[i];
  const int4 pr = d.pairs[i];
  f.pr = pr;
  f.active = 0;
  if (pr.x >= PAIR_SPT) return;  // friction acts against the rigid indenter only
  double P[4][3];
  int rows[4];
  pair_points(d, pr, 0.0, true, P, rows);
  DType ty;
  const double D = pair_d2(pair_kind(pr.x), P, &ty);
  if (!(D > 0.0) || !(D < G.dhat * G.dhat)) return;
  double b, bD, bDD;
  barrier_D(D, G.dhat, &b, &bD, &bDD);
  double mol = 1.0;  // edge-edge mollifier at the lagged state scales the normal force
  if (pr.x == PAIR_EE) {
    double ea[3], eb[3], n[3];
    sub3(P[1], P[0], ea);
    sub3(P[3], P[2], eb);
    cross3(ea, eb, n);
    const double ex = pair_eps_x(d, pr), q = dot3(n, n) / ex;
    if (q < 1.0) mol = q * (2.0 - q);
  }
  f.lam = d.gc[g].kappa * mol * fabs(2.0 * sqrt(D) * bD);  // |b'(d)| = |2 d dB/dD|
  double w[4] = {0.0, 0.0, 0.0, 0.0}, nrm[3];
  const int* id = ty.i;
  if (ty.f == DF_PP) {
    w[id[0]] = 1.0;
    w[id[1]] = -1.0;
    sub3(P[id[0]], P[id[1]], nrm);
  } else if (ty.f == DF_PE) {
    double e[3], r[3];
    sub3(P[id[2]], P[id[1]], e);
    sub3(P[id[0]], P[id[1]], r);
    const double t = dot3(r, e) / dot3(e, e);
    w[id[0]] = 1.0;
    w[id[1]] = t - 1.0;
    w[id[2]] = -t;
    for (int c = 0; c < 3; ++c) nrm[c] = r[c] - t * e[c];
  } else if (ty.f == DF_PT) {  // the face's barycentric coordinates of the projected point
    double e1[3], e2[3], r[3];
    sub3(P[2], P[1], e1);
    sub3(P[3], P[1], e2);
    sub3(P[0], P[1], r);
    const double a = dot3(e1, e1), bb = dot3(e1, e2), c = dot3(e2, e2), p = dot3(e1, r), q = dot3(e2, r);
    const double den = a * c - bb * bb, l1 = (c * p - bb * q) / den, l2 = (a * q - bb * p) / den;
    w[0] = 1.0;
    w[1] = l1 + l2 - 1.0;
    w[2] = -l1;
    w[3] = -l2;
    cross3(e1, e2, nrm);
  } else {  // line-line: the closest points' parameters on both edges
    double u[3], v[3], r[3];
    sub3(P[1], P[0], u);
    sub3(P[3], P[2], v);
    sub3(P[0], P[2], r);
    const double a = dot3(u, u), bb = dot3(u, v), c = dot3(v, v), p = dot3(u, r), q = dot3(v, r);
    const double den = a * c - bb * bb, sa = (bb * q - c * p) / den, tb = (a * q - bb * p) / den;
    w[0] = 1.0 - sa;
    w[1] = sa;
    w[2] = tb - 1.0;
    w[3] = -tb;
    cross3(u, v, nrm);
  }
  const double nn = sqrt(dot3(nrm, nrm));
  for (int c = 0; c < 3; ++c) nrm[c] /= nn;
  // tangent basis: the coordinate axis least aligned with the normal, made orthogonal to it, and
  // normal x that
  int ax = 0;
  if (fabs(nrm[1]) < fabs(nrm[ax])) ax = 1;
  if (fabs(nrm[2]) < fabs(nrm[ax])) ax = 2;
  double t1[3] = {-nrm[ax] * nrm[0], -nrm[ax] * nrm[1], -nrm[ax] * nrm[2]}, t2[3];
  t1[ax] += 1.0;
  const double n1 = sqrt(dot3(t1, t1));
  for (int c = 0; c < 3; ++c) t1[c] /= n1;
  cross3(nrm, t1, t2);
  for (int c = 0; c < 3; ++c) {
    f.T[2 * c] = t1[c];
    f.T[2 * c + 1] = t2[c];
  }
  for (int q = 0; q < 4; ++q) {
    f.w[q] = w[q];
    for (int c = 0; c < 3; ++c) f.Plag[3 * q + c] = P[q][c];
  }
  f.active = 1;
}

// the friction record of slot i, if its gel is in `phase` and it was in contact at the start
__device__ __forceinline__ bool fric_slot(const Dev& d, int i, int phase, const FricRec*& f) {
  const int g = d.pslot_gel[i];
  if (d.gc[g].phase != phase || phase == PH_EVAL || !(d.gi[g].mu_f > 0.0)) return false;
  if (i - d.gi[g].pbase >= d.gv[g].nfric) return false;
  f = d.fric + i;
  return f->active != 0;
}

// u = T^T sum_k w_k (P_k - Plag_k) at the pair's points P (gel at x + alpha p, indenter at its
// current pose)
__device__ __forceinline__ void fric_u(const FricRec& f, const double P[4][3], double u[2]) {
  double dl[3] = {0.0, 0.0, 0.0};
  for (int q = 0; q < 4; ++q)
    for (int c = 0; c < 3; ++c) dl[c] = fma(f.w[q], P[q][c] - f.Plag[3 * q + c], dl[c]);
  u[0] = dl[0] * f.T[0] + dl[1] * f.T[2] + dl[2] * f.T[4];
  u[1] = dl[0] * f.T[1] + dl[1] * f.T[3] + dl[2] * f.T[5];
}

// friction energy of a record at x + alpha p
__device__ __forceinline__ double fric_energy(const Dev& d, const FricRec& f, int g, double alpha) {
  double P[4][3], u[2], f0, phi, psi;
  int rows[4];
  pair_points(d, f.pr, alpha, false, P, rows);
  fric_u(f, P, u);
  coulomb_f0(sqrt(u[0] * u[0] + u[1] * u[1]), d.gi[g].eps_v * d.gc[g].h, &f0, &phi, &psi);
  return d.gi[g].mu_f * f.lam * f0;
}

// Friction terms of the Newton iteration, one thread per record.  Mode 0 (with the contact
// gradient): dD/dP_k = mu_f lam w_k T (phi u) into the contact gradient of the free gel rows and
// the contact force.  Mode 1 (after the gather wrote the matrix): the blocks
// d2D/dP_k dP_l = mu_f lam w_k w_l T (phi I + psi u u^T) T^T between free gel rows.
template <bool MIXED>
__global__ void __launch_bounds__(128) k_fric(Dev d, int phase, int mode) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.npslots) return;
  const FricRec* fp;
  if (!fric_slot(d, i, phase, fp)) return;
  const FricRec& f = *fp;
  const int g = d.pslot_gel[i];
  double P[4][3], u[2], f0, phi, psi;
  int rows[4];
  pair_points(d, f.pr, 0.0, false, P, rows);
  fric_u(f, P, u);
  coulomb_f0(sqrt(u[0] * u[0] + u[1] * u[1]), d.gi[g].eps_v * d.gc[g].h, &f0, &phi, &psi);
  const double c = d.gi[g].mu_f * f.lam;
  if (mode == 0) {
    double gt[3];  // c T (phi u)
    for (int k = 0; k < 3; ++k) gt[k] = c * phi * (f.T[2 * k] * u[0] + f.T[2 * k + 1] * u[1]);
    for (int q = 0; q < 4; ++q) {
      const int r = rows[q];
      if (r < 0 || f.w[q] == 0.0) continue;
      const double gx = f.w[q] * gt[0], gy = f.w[q] * gt[1], gz = f.w[q] * gt[2];
      atomicAdd(&d.gv[g].fc[0], -gx);
      atomicAdd(&d.gv[g].fc[1], -gy);
      atomicAdd(&d.gv[g].fc[2], -gz);
      if (d.fixed[r]) continue;
      atomicAdd(&d.cgrad[r].x, gx);
      atomicAdd(&d.cgrad[r].y, gy);
      atomicAdd(&d.cgrad[r].z, gz);
    }
    return;
  }
  // H_delta = c T M T^T, M = phi I + psi u u^T (2 x 2)
  const double m00 = phi + psi * u[0] * u[0], m01 = psi * u[0] * u[1], m11 = phi + psi * u[1] * u[1];
  double H[9];
  for (int a = 0; a < 3; ++a) {
    const double ta0 = f.T[2 * a], ta1 = f.T[2 * a + 1];
    const double r0 = ta0 * m00 + ta1 * m01, r1 = ta0 * m01 + ta1 * m11;
    for (int b = 0; b < 3; ++b) H[3 * a + b] = c * (r0 * f.T[2 * b] + r1 * f.T[2 * b + 1]);
  }
  for (int qa = 0; qa < 4; ++qa) {
    const int ra = rows[qa];
    if (ra < 0 || f.w[qa] == 0.0 || d.fixed[ra]) continue;
    for (int qb = 0; qb < 4; ++qb) {
      const int rb = rows[qb];
      if (rb < 0 || f.w[qb] == 0.0 || d.fixed[rb]) continue;
      const int bp = find_block(d, ra, rb);
      if (bp < 0) {
        atomicOr(&d.gv[g].flags, 16);
        continue;
      }
      const double ww = f.w[qa] * f.w[qb];
      for (int e = 0; e < 9; ++e) add_val<MIXED>(d, bp, e, ww * H[e]);
    }
  }
}

// ---------------------------------------------------------------- ACCD and distances
// mode 0: Newton step (gel moves by p, indenter fixed at cur); mode 1: indenter sweep prev -> cur
// with the gel fixed at x.
__global__ void __launch_bounds__(128) k_accd(Dev d, int phase, int mode, int maxit) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.npslots) return;
  int4 pr;
  if (!pair_slot(d, i, phase, mode == 0, pr)) return;
  const int g = pr.w;
  double P[4][3], dP[4][3];
  int rows[4];
  pair_points(d, pr, 0.0, mode == 1, P, rows);
  if (mode == 0) {
    for (int k = 0; k < 4; ++k) {
      if (rows[k] >= 0) {
        const double4_32a p = d.p[rows[k]];
        dP[k][0] = p.x; dP[k][1] = p.y; dP[k][2] = p.z;
      } else {
        dP[k][0] = dP[k][1] = dP[k][2] = 0.0;
      }
    }
  } else {
    double Q[4][3];
    int r2[4];
    pair_points(d, pr, 0.0, false, Q, r2);
    for (int k = 0; k < 4; ++k)
      for (int c = 0; c < 3; ++c) dP[k][c] = Q[k][c] - P[k][c];
  }
  double toi = 1.0;
  const int r = accd_pair(pair_kind(pr.x), P, dP, ACCD_S, 1.0, maxit, &toi);
  if (r == 1) {
    atomic_min_pos(&d.gv[g].toi_bits, toi);
    atomicOr(&d.gv[g].flags, 8);
  } else if (r == 2) {
    atomicOr(&d.gv[g].flags, 2);
  }
}

// smallest pair distance at (x, indenter cur)
__global__ void k_min_dist(Dev d, int phase) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.npslots) return;
  int4 pr;
  if (!pair_slot(d, i, phase, false, pr)) return;
  const int g = pr.w;
  double P[4][3];
  int rows[4];
  pair_points(d, pr, 0.0, false, P, rows);
  DType ty;
  const double D = pair_d2(pair_kind(pr.x), P, &ty);
  atomic_min_pos(&d.gv[g].dmin_bits, sqrt(fmax(D, 0.0)));
  if (D < d.gi[g].dhat * d.gi[g].dhat) atomicAdd(&d.gv[g].active_pairs, 1);
}

// kappa b(d) of every candidate pair at x + alpha p (mode 1: line-search trial of the gels still
// searching, alpha = their trial step; otherwise alpha = 0), one thread per pair slot; the energy
// kernel sums a gel's slots in a fixed order
// ---------------------------------------------------------------- energy
// One launch per energy evaluation.  pieces: (gel, kind, begin, end); kind 0 tets [begin, end),
// 1 rows [begin, end), 2 pair slots (chunk begin of end chunks over the gel's candidate list).
// Every CTA sums its piece into part_e; the gel's last CTA to finish (a per-gel ticket) adds its
// pieces in order and applies the result.  mode 0: E_cur at x; 1: line-search trial at
// x + alpha p for gels still searching (accept, or halve alpha); 2: E_try at x.
constexpr int EN_T = 256;

__global__ void __launch_bounds__(EN_T) k_energy(Dev d, int phase, const int4* pieces, const int* gel_piece,
                                                 double* part_e, unsigned* ticket, int mode) {
  __shared__ double sm[EN_T / 32];
  __shared__ int last;
  const int4 pc = pieces[blockIdx.x];
  const int g = pc.x;
  if (d.gc[g].phase != phase) return;
  GelVar& v = d.gv[g];
  if (mode == 1 && (v.ls_state != 0 || v.converged)) return;
  const GelInfo& G = d.gi[g];
  const double alpha = mode == 1 ? v.alpha : 0.0;
  double acc = 0.0;
  if (pc.y == 0) {
    for (int t = pc.z + threadIdx.x; t < pc.w; t += EN_T) acc += tet_energy_at(d, t, alpha, G.mu, G.lam);
  } else if (pc.y == 1) {
    const double ih2 = 0.5 / (d.gc[g].h * d.gc[g].h);
    for (int r = pc.z + threadIdx.x; r < pc.w; r += EN_T) {
      const double4_32a x = d.x[r], xt = d.xt[r];
      double ex = x.x - xt.x, ey = x.y - xt.y, ez = x.z - xt.z;
      if (alpha != 0.0) {
        const double4_32a p = d.p[r];
        ex = x.x + alpha * p.x - xt.x;
        ey = x.y + alpha * p.y - xt.y;
        ez = x.z + alpha * p.z - xt.z;
      }
      acc += d.mass[r] * (ex * ex + ey * ey + ez * ez) * ih2;
    }
  } else if (pc.y == 2) {
    const int np = min(v.npair, G.pcap);
    for (int i = pc.z * EN_T + threadIdx.x; i < np; i += pc.w * EN_T) {
      const int4 pr = d.pairs[G.pbase + i];
      double P[4][3], dist;
      int rows[4];
      pair_points(d, pr, alpha, false, P, rows);
      acc += d.gc[g].kappa * pair_energy(pair_kind(pr.x), P, G.dhat, pair_eps_x(d, pr), &dist);
    }
  } else if (phase != PH_EVAL) {  // lagged friction records of the running (sub)step
    for (int i = pc.z * EN_T + threadIdx.x; i < v.nfric; i += pc.w * EN_T) {
      const FricRec& f = d.fric[G.pbase + i];
      if (f.active) acc += fric_energy(d, f, g, alpha);
    }
  }
  acc = block_sum<EN_T>(acc, sm);
  if (threadIdx.x == 0) {
    part_e[blockIdx.x] = acc;
    __threadfence();
    const unsigned n = (unsigned)(gel_piece[g + 1] - gel_piece[g]);
    last = atomicAdd(&ticket[g], 1u) == n - 1u;
  }
  __syncthreads();
  if (!last) return;
  // every piece of the gel is in part_e (each fenced before taking its ticket): a fixed-order
  // block sum of them, read past L1
  double E = 0.0;
  for (int k = gel_piece[g] + threadIdx.x; k < gel_piece[g + 1]; k += EN_T) E += __ldcg(part_e + k);
  E = block_sum<EN_T>(E, sm);
  if (threadIdx.x != 0) return;
  ticket[g] = 0u;
  if (mode == 0) {
    v.E_cur = E;
  } else if (mode == 2) {
    v.E_try = E;
  } else {
    v.E_try = E;
    if (E <= v.E_cur) {
      v.ls_state = 1;
      v.E_cur = E;
    } else {
      v.alpha *= 0.5;
      v.ls_total += 1;
      // no resolvable decrease: stationary to energy resolution (6) or failure (2)
      if (v.alpha < 1e-12 * v.alpha0) v.ls_state = (-v.gtp <= 1e-10 * fabs(v.E_cur)) ? 6 : 2;
    }
  }
}

void launch_energy(const Dev& d, int phase, const int4* pieces, int npieces, const int* gel_piece,
                   double* part_e, unsigned* ticket, int mode, cudaStream_t st) {
  if (npieces <= 0) return;
  k_energy<<<npieces, EN_T, 0, st>>>(d, phase, pieces, gel_piece, part_e, ticket, mode);
  count_launch(1);
}

// ---------------------------------------------------------------- unit-level entries
// unit-level entry: one warp per pair (the same team-parallel derivatives and projection as the
// assembly), full 12 x 12 Hessian with the free block projected
struct EvalWS {
  PairBarrier pb;
  ProjWS pj;
  double P[4][3];
  int act, nf;
  int fd[PW_MAXN], all[PW_MAXN];
};

__global__ void __launch_bounds__(128) k_eval_pairs(int n, const int* kind, const double* Pin, double dhat,
                                                    const double* eps_x, const int* free_mask, double* bo,
                                                    double* go, double* Ho, int* dtype) {
  __shared__ EvalWS sws[4];
  EvalWS& w = sws[threadIdx.x >> 5];
  const Team<32> tm{(int)(threadIdx.x & 31), nullptr};
  const int i = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (i >= n) return;  // whole warps
  if (tm.id == 0) {
    for (int k = 0; k < 4; ++k)
      for (int c = 0; c < 3; ++c) w.P[k][c] = Pin[12 * i + 3 * k + c];
    DType ty;
    w.act = pair_barrier_setup(kind[i], w.P, dhat, eps_x ? eps_x[i] : 0.0, w.pb, &ty) ? 1 : 0;
    if (dtype) {
      dtype[5 * i] = ty.f;
      for (int k = 0; k < 4; ++k) dtype[5 * i + 1 + k] = ty.i[k];
    }
    const int fm = free_mask ? free_mask[i] : 0;
    int nf = 0;
    for (int k = 0; k < 4; ++k)
      if (fm & (1 << k))
        for (int c = 0; c < 3; ++c) w.fd[nf++] = 3 * k + c;
    w.nf = nf;
    bo[i] = w.act ? w.pb.b : 0.0;
  }
  __syncwarp();
  const bool act = w.act != 0;
  if (go && tm.id < 12) go[12 * i + tm.id] = act ? pair_grad_entry(w.pb, tm.id) : 0.0;
  if (!act) {
    if (Ho)
      for (int e = tm.id; e < 144; e += 32) Ho[144 * (size_t)i + e] = 0.0;
    return;
  }
  if (Ho) {  // the whole 12 x 12 Hessian through the same team-parallel block code
    if (tm.id < 12) w.all[tm.id] = tm.id;
    __syncwarp();
    team_pair_block(w.pb, w.all, 12, 12, w.pj.T, w.pj.H, tm);
    for (int e = tm.id; e < 144; e += 32) Ho[144 * (size_t)i + e] = w.pj.H[e];
    __syncwarp();
  }
  const int nf = w.nf;
  if (nf == 0 || !Ho) return;
  const int m = nf + (nf & 1);
  team_pair_block(w.pb, w.fd, nf, m, w.pj.T, w.pj.H, tm);
  team_psd_project(w.pj, nf, tm);
  for (int e = tm.id; e < nf * nf; e += 32) {
    const int r = e / nf, c = e - r * nf;
    Ho[144 * (size_t)i + 12 * w.fd[r] + w.fd[c]] = w.pj.H[r * m + c];
  }
}

__global__ void k_eval_accd(int n, const int* kind, const double* Pin, const double* dPin, double s,
                            double tc, int maxit, double* toi, int* hit) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double P[4][3], dP[4][3];
  for (int k = 0; k < 4; ++k)
    for (int c = 0; c < 3; ++c) {
      P[k][c] = Pin[12 * i + 3 * k + c];
      dP[k][c] = dPin[12 * i + 3 * k + c];
    }
  double t = 1.0;
  hit[i] = accd_pair(kind[i], P, dP, s, tc, maxit, &t);
  toi[i] = t;
}

// ---------------------------------------------------------------- launchers

void launch_indenter_pose(const Dev& d, int phase, int n_ind_verts, cudaStream_t st) {
  if (n_ind_verts > 0) {
    k_indenter_pose<<<nblk(n_ind_verts, 128), 128, 0, st>>>(d, phase);
    count_launch(1);
  }
}
void launch_hash_build(const Dev& d, int phase, int swept, cudaStream_t st) {
  const int np = d.nit_total + d.niv_total + d.nie_total;
  if (np > 0) {
    k_ind_boxes<<<nblk(np, 128), 128, 0, st>>>(d, phase, swept);
    count_launch(1);
  }
  k_hash_build<<<d.n_gels * NTAB, HB_THREADS, 0, st>>>(d, phase, swept);
  count_launch(1);
  k_hash_sort<<<dim3(nblk(d.max_hnb, 128), d.n_gels * NTAB), 128, 0, st>>>(d, phase);
  count_launch(1);
}
void launch_query(const Dev& d, int phase, int mode, cudaStream_t st) {
  if (d.nq <= 0) return;
  if (!(mode & 1)) {  // the count pass lists the primitives near the indenter; the write pass reuses it
    cudaMemsetAsync(d.qnear_n, 0, sizeof(int), st);
    k_query_near<<<nblk(d.nq, 128), 128, 0, st>>>(d, phase, mode);
    count_launch(1);
  }
  k_query_list<<<std::min(nblk(d.nq, 4), 8 * 152), 128, 0, st>>>(d, phase, mode);
  count_launch(1);
}
void launch_pair_ranges(const Dev& d, int phase, int skip_conv, cudaStream_t st) {
  k_pair_ranges<<<nblk(d.n_gels, 128), 128, 0, st>>>(d, phase, skip_conv);
  count_launch(1);
}
size_t pair_record_doubles() { return sizeof(PairBarrier) / sizeof(double); }

// Contact assembly without the matrix: contact gradient into cgrad, single-point blocks and the
// first crec_cap projected pair Hessians into their records (independent of the elastic
// assembly and the gather, so it may run beside them)
void launch_contact_compute(const Dev& d, int phase, bool mixed, cudaStream_t st) {
  cudaMemsetAsync(d.cgrad, 0, sizeof(double4_32a) * (size_t)d.nrows, st);
  if (d.npslots <= 0) return;
  cudaMemsetAsync(d.cwork_n, 0, sizeof(int), st);
  cudaMemsetAsync(d.c1_n, 0, sizeof(int), st);
  const int nb = nblk(d.npslots, 128);
  const int nc = std::min(nblk(std::min(d.npslots, d.crec_cap), CW_WARPS), 8 * 152);
  if (mixed) {
    k_contact_pairs<true><<<nb, 128, 0, st>>>(d, phase);
    k_contact_hess<true><<<nc, 32 * CW_WARPS, 0, st>>>(d, 0);
  } else {
    k_contact_pairs<false><<<nb, 128, 0, st>>>(d, phase);
    k_contact_hess<false><<<nc, 32 * CW_WARPS, 0, st>>>(d, 0);
  }
  count_launch(2);
}
// ... and its blocks added to the matrix the gather wrote
void launch_contact_merge(const Dev& d, bool mixed, cudaStream_t st) {
  if (d.npslots <= 0) return;
  const int nc = std::min(nblk(d.npslots, CW_WARPS), 8 * 152);
  if (mixed)
    k_contact_hess<true><<<nc, 32 * CW_WARPS, 0, st>>>(d, 1);
  else
    k_contact_hess<false><<<nc, 32 * CW_WARPS, 0, st>>>(d, 1);
  count_launch(1);
}
void launch_fric_setup(const Dev& d, int phase, cudaStream_t st) {
  if (d.npslots <= 0 || !d.fric) return;
  k_fric_setup<<<nblk(d.npslots, 128), 128, 0, st>>>(d, phase);
  count_launch(1);
}
void launch_fric(const Dev& d, int phase, int mode, bool mixed, cudaStream_t st) {
  if (d.npslots <= 0 || !d.fric) return;
  if (mixed)
    k_fric<true><<<nblk(d.npslots, 128), 128, 0, st>>>(d, phase, mode);
  else
    k_fric<false><<<nblk(d.npslots, 128), 128, 0, st>>>(d, phase, mode);
  count_launch(1);
}
void launch_accd(const Dev& d, int phase, int mode, int maxit, cudaStream_t st) {
  if (d.npslots > 0) {
    k_accd<<<nblk(d.npslots, 128), 128, 0, st>>>(d, phase, mode, maxit);
    count_launch(1);
  }
}
void launch_min_dist(const Dev& d, int phase, cudaStream_t st) {
  if (d.npslots > 0) {
    k_min_dist<<<nblk(d.npslots, 128), 128, 0, st>>>(d, phase);
    count_launch(1);
  }
}
void launch_eval_pairs(int n, const int* kind, const double* P, double dhat, const double* eps_x,
                       const int* free_mask, double* b, double* g, double* H, int* dtype, cudaStream_t st) {
  if (n > 0) {
    k_eval_pairs<<<nblk(n, 4), 128, 0, st>>>(n, kind, P, dhat, eps_x, free_mask, b, g, H, dtype);
    count_launch(1);
  }
}
void launch_eval_accd(int n, const int* kind, const double* P, const double* dP, double s, double tc,
                      int maxit, double* toi, int* hit, cudaStream_t st) {
  if (n > 0) {
    k_eval_accd<<<nblk(n, 128), 128, 0, st>>>(n, kind, P, dP, s, tc, maxit, toi, hit);
    count_launch(1);
  }
}

}  // namespace txg

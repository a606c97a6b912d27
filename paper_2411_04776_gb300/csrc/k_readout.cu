// Gel-surface readout for the tactile simulation that consumes the physics state (TacEx, Sec.
// "Tactile Simulation": height maps of the gel surface feed the optical simulation, and markers
// tied to faces of the tet mesh follow the vertex positions of their facet, App. "Marker
// Simulation").  The top surface is the set of boundary triangles whose rest outward normal
// points up (+z).  Both readouts work on the current positions x of one gel:
//   * markers: a marker placed at a rest point (mx, my) of the top surface lies in a top triangle
//     of the rest mesh (its xy barycentric coordinates l, all >= -1e-12; the first such triangle
//     in the top list); it is carried to sum_k l_k x_k.  The search runs one thread per (marker,
//     top triangle) pair and keeps the smallest containing index with atomicMin; a thread per
//     marker then evaluates the position;
//   * height map: pixel (i, j) at (x0 + (i + 1/2) dx, y0 + (j + 1/2) dy) reads the largest z of
//     the deformed top triangles that cover it in the xy projection (barycentric coordinates
//     >= -1e-12), NaN where none does -- the top surface seen from above, rasterised by CUDA
//     without a graphics API.  One thread per top triangle visits the pixels of its xy bounding
//     box; the maximum is taken with 64-bit atomicMax on an order-preserving encoding of z.
#include <cuda_runtime.h>

#include "txgel_common.cuh"

namespace txg {

static inline int nblk_r(int n, int t) { return (n + t - 1) / t; }

// xy barycentric coordinates of (px, py) in triangle (a, b, c); false if it is degenerate
__device__ __forceinline__ bool bary_xy(const double4_32a a, const double4_32a b, const double4_32a c, double px,
                                        double py, double l[3]) {
  const double det = (b.x - a.x) * (c.y - a.y) - (c.x - a.x) * (b.y - a.y);
  if (det == 0.0) return false;
  l[1] = ((px - a.x) * (c.y - a.y) - (c.x - a.x) * (py - a.y)) / det;
  l[2] = ((b.x - a.x) * (py - a.y) - (px - a.x) * (b.y - a.y)) / det;
  l[0] = 1.0 - l[1] - l[2];
  return l[0] >= -1e-12 && l[1] >= -1e-12 && l[2] >= -1e-12;
}

// tri[i]: smallest index (within the gel's top list) of a top triangle containing marker i, or
// left at its initial value (INT_MAX: none)
__global__ void k_marker_find(Dev d, int g, int n, int ntop, const double* rest_xy, int* tri) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)n * (size_t)ntop) return;
  const int i = (int)(q / (size_t)ntop), k = (int)(q % (size_t)ntop);
  const int4 t = d.top[d.gi[g].top0 + k];
  double l[3];
  if (bary_xy(d.X[t.x], d.X[t.y], d.X[t.z], rest_xy[2 * i], rest_xy[2 * i + 1], l)) atomicMin(tri + i, k);
}

__global__ void k_markers(Dev d, int g, int n, const double* rest_xy, const int* tri, double* out, int* found) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const GelInfo& G = d.gi[g];
  const int k = tri[i];
  found[i] = 0;
  out[3 * i] = out[3 * i + 1] = out[3 * i + 2] = 0.0;
  if (k < 0 || k >= G.ntop) return;
  const int4 t = d.top[G.top0 + k];
  double l[3];
  bary_xy(d.X[t.x], d.X[t.y], d.X[t.z], rest_xy[2 * i], rest_xy[2 * i + 1], l);
  const double4_32a a = d.x[t.x], b = d.x[t.y], c = d.x[t.z];
  out[3 * i] = l[0] * a.x + l[1] * b.x + l[2] * c.x;
  out[3 * i + 1] = l[0] * a.y + l[1] * b.y + l[2] * c.y;
  out[3 * i + 2] = l[0] * a.z + l[1] * b.z + l[2] * c.z;
  found[i] = 1;
}

// order-preserving map of doubles to unsigned 64-bit (0 is below every encoded value: "none")
__device__ __forceinline__ unsigned long long z_key(double z) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(z));
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double z_of_key(unsigned long long k) {
  const unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double(static_cast<long long>(u));
}

__global__ void k_raster_top(Dev d, int g, int nx, int ny, double x0, double y0, double dx, double dy,
                             unsigned long long* img) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const GelInfo& G = d.gi[g];
  if (k >= G.ntop) return;
  const int4 t = d.top[G.top0 + k];
  const double4_32a a = d.x[t.x], b = d.x[t.y], c = d.x[t.z];
  const double lx = fmin(a.x, fmin(b.x, c.x)), hx = fmax(a.x, fmax(b.x, c.x));
  const double ly = fmin(a.y, fmin(b.y, c.y)), hy = fmax(a.y, fmax(b.y, c.y));
  // pixel centres x0 + (i + 1/2) dx inside [lx, hx] (one pixel of margin for the tolerance),
  // clamped to the image before the conversion to int
  const int i0 = (int)fmax(0.0, floor((lx - x0) / dx - 0.5) - 1.0);
  const int i1 = (int)fmin((double)(nx - 1), ceil((hx - x0) / dx - 0.5) + 1.0);
  const int j0 = (int)fmax(0.0, floor((ly - y0) / dy - 0.5) - 1.0);
  const int j1 = (int)fmin((double)(ny - 1), ceil((hy - y0) / dy - 0.5) + 1.0);
  for (int j = j0; j <= j1; ++j)
    for (int i = i0; i <= i1; ++i) {
      double l[3];
      if (!bary_xy(a, b, c, x0 + (i + 0.5) * dx, y0 + (j + 0.5) * dy, l)) continue;
      const double z = l[0] * a.z + l[1] * b.z + l[2] * c.z;
      atomicMax(img + (size_t)j * nx + i, z_key(z));
    }
}

__global__ void k_decode_heights(int n, const unsigned long long* img, double* out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const unsigned long long k = img[p];
  out[p] = k == 0ull ? CUDART_NAN : z_of_key(k);
}

// tri: n ints of device scratch; ntop: the gel's top triangles
void launch_markers(const Dev& d, int g, int n, int ntop, const double* rest_xy, int* tri, double* out, int* found,
                    cudaStream_t st) {
  if (n <= 0) return;
  cudaMemsetAsync(tri, 0x7f, sizeof(int) * (size_t)n, st);  // 0x7f7f7f7f: no triangle yet
  const size_t pairs = (size_t)n * (size_t)ntop;
  if (pairs > 0) {
    k_marker_find<<<(unsigned)((pairs + 255) / 256), 256, 0, st>>>(d, g, n, ntop, rest_xy, tri);
    count_launch(1);
  }
  k_markers<<<nblk_r(n, 128), 128, 0, st>>>(d, g, n, rest_xy, tri, out, found);
  count_launch(1);
}

// img: nx * ny zeroed 64-bit words; out: nx * ny doubles (device)
void launch_height_map(const Dev& d, int g, int ntop, int nx, int ny, double x0, double y0, double dx, double dy,
                       unsigned long long* img, double* out, cudaStream_t st) {
  if (ntop > 0) {
    k_raster_top<<<nblk_r(ntop, 128), 128, 0, st>>>(d, g, nx, ny, x0, y0, dx, dy, img);
    count_launch(1);
  }
  k_decode_heights<<<nblk_r(nx * ny, 256), 256, 0, st>>>(nx * ny, img, out);
  count_launch(1);
}

}  // namespace txg

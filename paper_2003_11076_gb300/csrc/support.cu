// Support points of the disparity prior (Sec. III-C "Disparity Prior"): a
// sparse grid of reference pixels matched along the epipolar lines over the
// full candidate range, points on dynamic objects removed with the
// segmentation prior, points of the other views that fall on the reference's
// occluded background added, one point per grid cell, and points without
// enough agreeing neighbours removed.
//
// Everything that decides whether and where a point exists is integer or
// double arithmetic (8-bit luminance, integer Sobel descriptors, integer SAD
// costs; target offsets, re-projected positions and disparity comparisons in
// double), so the result is exact, not approximate.
//
// Kernels (one run, all on the context's stream):
//   support_grad_kernel     8-bit luminance and integer Sobel of every camera
//   support_match_kernel    one thread per (source camera, grid cell): window
//                           static test, texture, costs over the candidates,
//                           arg-min and the uniqueness ratio
//   support_claim_kernel    reference points fill their cells; other views'
//                           points claim empty cells (first in camera, then
//                           raster order wins through atomicMin)
//   support_fill_kernel     the claimants that won write their cell
//   support_check_kernel    neighbourhood consistency
//   support_count_kernel /  the surviving points in cell raster order (per
//   support_compact_kernel  1024-cell chunk: count, then write after the
//                           earlier chunks' points)
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "lf_internal.h"

namespace lf {
namespace {

__device__ __forceinline__ int quant8(float x) {
  const float q = rintf(__fmul_rn(255.f, x));
  return static_cast<int>(fminf(fmaxf(q, 0.f), 255.f));
}

__device__ __forceinline__ int channel8(const uint8_t* row, int u, int c, int C, int dtype) {
  const int i = u * C + c;
  if (dtype == 0) return row[i];
  if (dtype == 1) return quant8(reinterpret_cast<const float*>(row)[i]);
  if (dtype == 2) return quant8(__half2float(reinterpret_cast<const __half*>(row)[i]));
  return quant8(__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(row)[i]));
}

__device__ __forceinline__ int luma8(const SupportArgs& a, int k, int v, int u) {
  const uint8_t* row = a.img + (static_cast<size_t>(k) * a.H + v) * a.img_pitch;
  if (a.C == 1) return channel8(row, u, 0, 1, a.dtype);
  const int r = channel8(row, u, 0, 3, a.dtype), g = channel8(row, u, 1, 3, a.dtype),
            b = channel8(row, u, 2, 3, a.dtype);
  return (77 * r + 150 * g + 29 * b + 128) >> 8;
}

__global__ void support_grad_kernel(const SupportArgs a) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= a.W) return;
  for (int row = blockIdx.y; row < a.K * a.H; row += gridDim.y) {
    const int k = row / a.H, v = row - k * a.H;
    const int vm = max(v - 1, 0), vp = min(v + 1, a.H - 1), um = max(u - 1, 0), up = min(u + 1, a.W - 1);
    const int y00 = luma8(a, k, vm, um), y01 = luma8(a, k, vm, u), y02 = luma8(a, k, vm, up);
    const int y10 = luma8(a, k, v, um), y12 = luma8(a, k, v, up);
    const int y20 = luma8(a, k, vp, um), y21 = luma8(a, k, vp, u), y22 = luma8(a, k, vp, up);
    const size_t o = static_cast<size_t>(row) * a.W + u;
    a.gx[o] = static_cast<int16_t>((y02 + 2 * y12 + y22) - (y00 + 2 * y10 + y20));
    a.gy[o] = static_cast<int16_t>((y20 + 2 * y21 + y22) - (y00 + 2 * y01 + y02));
  }
}

__device__ __forceinline__ int grad_at(const int16_t* m, const SupportArgs& a, int k, int v, int u) {
  v = min(max(v, 0), a.H - 1);
  u = min(max(u, 0), a.W - 1);
  return m[(static_cast<size_t>(k) * a.H + v) * a.W + u];
}

__device__ __forceinline__ bool window_static(const SupportArgs& a, int k, int u, int v) {
  bool ok = true;
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      const int y = min(max(v + dy, 0), a.H - 1), x = min(max(u + dx, 0), a.W - 1);
      const float P = reinterpret_cast<const float*>(reinterpret_cast<const uint8_t*>(a.P) +
                                                     (static_cast<size_t>(k) * a.H + y) * a.p_pitch)[x];
      ok = ok && (P < a.seg_threshold);
    }
  return ok;
}

// Thread (source si, cell): si indexes a.src (reference first).
__global__ void support_match_kernel(const SupportArgs a) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  const int si = blockIdx.y;
  if (cell >= a.nx * a.ny) return;
  const int ci = cell % a.nx, cj = cell / a.nx;
  const int u = a.grid * ci + a.grid / 2, v = a.grid * cj + a.grid / 2;
  int result = -1;
  const int s = a.src[si];
  const unsigned tmask = a.tmask[si];
  if (u <= a.W - 1 && v <= a.H - 1 && tmask != 0u && a.delta_c[si] > 0 && window_static(a, s, u, v)) {
    int ds[18];
    int tex = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int i = (dy + 1) * 3 + (dx + 1);
        ds[i] = grad_at(a.gx, a, s, v + dy, u + dx);
        ds[9 + i] = grad_at(a.gy, a, s, v + dy, u + dx);
        tex += abs(ds[i]) + abs(ds[9 + i]);
      }
    if (tex >= a.texture) {
      const int* off = a.offsets + static_cast<size_t>(si) * a.K * a.D;  // [K][D] target offsets of this source
      // pass 1: the arg-min (lowest j); pass 2: the best cost at least delta candidates away
      long long best_c = -1;
      int best = -1;
      for (int pass = 0; pass < 2; ++pass) {
        long long second = -1;
        for (int j = 0; j < a.D; ++j) {
          if (pass == 1 && abs(j - best) < a.delta_c[si]) continue;
          long long c = 0;
          bool ok = true;
          for (int t = 0; t < a.K && ok; ++t) {
            if (!(tmask >> t & 1u)) continue;
            const int x = u + off[t * a.D + j];
            if (x < 0 || x > a.W - 1) {
              ok = false;
              break;
            }
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
              for (int dx = -1; dx <= 1; ++dx) {
                const int i = (dy + 1) * 3 + (dx + 1);
                c += abs(ds[i] - grad_at(a.gx, a, t, v + dy, x + dx));
                c += abs(ds[9 + i] - grad_at(a.gy, a, t, v + dy, x + dx));
              }
          }
          if (!ok) continue;
          if (pass == 0) {
            if (best < 0 || c < best_c) { best_c = c; best = j; }
          } else if (second < 0 || c < second) {
            second = c;
          }
        }
        if (pass == 0 && best < 0) break;
        if (pass == 1 && second >= 0 && 100 * best_c < static_cast<long long>(a.ratio_pct) * second) result = best;
      }
    }
  }
  a.match[static_cast<size_t>(si) * a.nx * a.ny + cell] = result;
}

// Candidate disparity in double, rounded operation by operation (no fused
// multiply-add), as the host computes it.
__device__ __forceinline__ double cand_d(const SupportArgs& a, int j) {
  if (a.D == 1) return static_cast<double>(a.d_min);
  const double step = __ddiv_rn(__dsub_rn(static_cast<double>(a.d_max), static_cast<double>(a.d_min)),
                                static_cast<double>(a.D - 1));
  return __dadd_rn(static_cast<double>(a.d_min), __dmul_rn(static_cast<double>(j), step));
}

constexpr int kNoClaim = 0x7f7f7f7f;  // claim[] memset to 0x7f bytes

// Position of other-view point (si >= 1, cell) on the reference, or false.
__device__ __forceinline__ bool reproject(const SupportArgs& a, int si, int cell, int j, double* ur, int* target) {
  const int ci = cell % a.nx, cj = cell / a.nx;
  const int u = a.grid * ci + a.grid / 2, v = a.grid * cj + a.grid / 2;
  const double x = __dadd_rn(static_cast<double>(u), __dmul_rn(cand_d(a, j), static_cast<double>(a.b[a.src[si]])));
  if (x < 0.0 || x > static_cast<double>(a.W - 1)) return false;
  const int rr = static_cast<int>(floor(__dadd_rn(x, 0.5)));
  const float P = reinterpret_cast<const float*>(reinterpret_cast<const uint8_t*>(a.P) +
                                                 (static_cast<size_t>(a.ref) * a.H + v) * a.p_pitch)[rr];
  if (P < a.seg_threshold) return false;  // the reference sees this background itself
  *ur = x;
  *target = cj * a.nx + static_cast<int>(floor(__ddiv_rn(x, static_cast<double>(a.grid))));
  return true;
}

__global__ void support_claim_kernel(const SupportArgs a) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  const int si = blockIdx.y;
  const int ncell = a.nx * a.ny;
  if (cell >= ncell || si == 0) return;  // the reference's own points need no claim
  const int j = a.match[static_cast<size_t>(si) * ncell + cell];
  if (j < 0) return;
  double ur;
  int target;
  if (!reproject(a, si, cell, j, &ur, &target)) return;
  if (a.match[target] >= 0) return;  // the reference's own point holds the cell
  atomicMin(a.claim + target, (si - 1) * ncell + cell);
}

// Cell arrays before the consistency test: cell_j / cell_src / cell_u / cell_v.
__global__ void support_fill_kernel(const SupportArgs a) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  const int ncell = a.nx * a.ny;
  if (cell >= ncell) return;
  int j = a.match[cell], src = -1;
  double u = 0.0, v = 0.0;
  if (j >= 0) {
    src = a.ref;
    u = a.grid * (cell % a.nx) + a.grid / 2;
    v = a.grid * (cell / a.nx) + a.grid / 2;
  } else if (a.claim[cell] != kNoClaim) {
    const int key = a.claim[cell], si = key / ncell + 1, from = key % ncell;
    j = a.match[static_cast<size_t>(si) * ncell + from];
    int target;
    reproject(a, si, from, j, &u, &target);
    src = a.src[si];
    v = a.grid * (from / a.nx) + a.grid / 2;
  }
  a.pre_j[cell] = j;
  a.pre_src[cell] = src;
  a.pre_u[cell] = u;
  a.pre_v[cell] = v;
}

__global__ void support_check_kernel(const SupportArgs a) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= a.nx * a.ny) return;
  const int j = a.pre_j[cell];
  bool keep = false;
  if (j >= 0) {
    const int ci = cell % a.nx, cj = cell / a.nx;
    const double d = cand_d(a, j);
    int support = 0;
    for (int y = max(cj - a.window, 0); y <= min(cj + a.window, a.ny - 1); ++y)
      for (int x = max(ci - a.window, 0); x <= min(ci + a.window, a.nx - 1); ++x) {
        if (x == ci && y == cj) continue;
        const int o = a.pre_j[y * a.nx + x];
        if (o >= 0 && fabs(__dsub_rn(cand_d(a, o), d)) <= static_cast<double>(a.delta)) ++support;
      }
    keep = support >= a.min_support;
  }
  a.cell_j[cell] = keep ? j : -1;
  a.cell_src[cell] = keep ? a.pre_src[cell] : -1;
  a.cell_u[cell] = keep ? a.pre_u[cell] : 0.0;
  a.cell_v[cell] = keep ? a.pre_v[cell] : 0.0;
}

// The kept points in cell raster order as float (u, v, d) triples: every
// CTA counts the kept cells of its chunk of 1024 cells, then writes its
// points after the points of all earlier chunks.
__global__ void __launch_bounds__(1024) support_count_kernel(const SupportArgs a) {
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = __syncthreads_count(cell < a.nx * a.ny && a.cell_j[cell] >= 0);
  if (threadIdx.x == 0) a.chunk_count[blockIdx.x] = n;
}

__global__ void __launch_bounds__(1024) support_compact_kernel(const SupportArgs a) {
  __shared__ int s_warp[32];
  __shared__ int s_base;
  const int ncell = a.nx * a.ny;
  if (threadIdx.x == 0) {
    int base = 0;
    for (int b = 0; b < static_cast<int>(blockIdx.x); ++b) base += a.chunk_count[b];
    s_base = base;
    if (blockIdx.x == gridDim.x - 1) *a.n_points = base + a.chunk_count[blockIdx.x];
  }
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  const bool has = cell < ncell && a.cell_j[cell] >= 0;
  const unsigned ballot = __ballot_sync(0xffffffffu, has);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_warp[warp] = __popc(ballot);
  __syncthreads();
  int before = 0;
  for (int w = 0; w < warp; ++w) before += s_warp[w];
  const int rank = s_base + before + __popc(ballot & ((1u << lane) - 1u));
  if (has && rank < a.max_points) {
    // a fixed sub-pixel offset per cell (at most 0.01 px) keeps grid points
    // off common circles, so that their Delaunay triangulation is unique
    const int ci = cell % a.nx, cj = cell / a.nx;
    const double ju = __ddiv_rn(__dmul_rn(0.01, static_cast<double>((7 * ci + 13 * cj) % 17 + 1)), 18.0);
    const double jv = __ddiv_rn(__dmul_rn(0.01, static_cast<double>((11 * ci + 5 * cj) % 19 + 1)), 20.0);
    a.points[3 * rank] = static_cast<float>(__dadd_rn(a.cell_u[cell], ju));
    a.points[3 * rank + 1] = static_cast<float>(__dadd_rn(a.cell_v[cell], jv));
    a.points[3 * rank + 2] = static_cast<float>(cand_d(a, a.cell_j[cell]));
  }
}

}  // namespace

cudaError_t launch_support(const SupportArgs& a, cudaStream_t s) {
  const int ncell = a.nx * a.ny;
  cudaError_t e;
  support_grad_kernel<<<dim3((a.W + 127) / 128, std::min(a.K * a.H, 65535)), 128, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const dim3 cells((ncell + 127) / 128, a.n_src);
  support_match_kernel<<<cells, 128, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.claim, 0x7f, sizeof(int) * ncell, s)) != cudaSuccess) return e;  // 0x7f7f7f7f
  support_claim_kernel<<<cells, 128, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  support_fill_kernel<<<(ncell + 127) / 128, 128, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  support_check_kernel<<<(ncell + 127) / 128, 128, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int chunks = (ncell + 1023) / 1024;
  support_count_kernel<<<chunks, 1024, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  support_compact_kernel<<<chunks, 1024, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace lf

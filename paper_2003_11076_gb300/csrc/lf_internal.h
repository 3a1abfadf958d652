// Internal declarations shared by the host library and its kernels.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "lf.h"

namespace lf {

// A named NVTX range over a host scope (the library's entry points and their
// host phases), so that a profiler's timeline shows where the host time of a
// call goes; without a profiler attached the push and pop do nothing.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kMaxCams = 12;       // 2^K label vectors per E-step
constexpr int kMaxD = 1024;        // candidate disparities per sweep
constexpr int kPrecF32 = 0, kPrecF16 = 1, kPrecBF16 = 2;

// Device status word bits (written by kernels, read by the host after a sync).
constexpr unsigned kStatusTmaTimeout = 1u;
constexpr unsigned kStatusSmemMisaligned = 2u;
constexpr unsigned kStatusBoundsViolation = 4u;  // debug builds: a shared-memory index left its region

// One support-point triangle of the piecewise-planar prior: vertices (float
// input coordinates, counter-clockwise) and the plane through them,
// mu(u, v) = d_a + gu * (u - u_a) + gv * (v - v_a), with each coefficient
// (computed in double on the host) stored as an unevaluated float sum
// hi + lo, hi = float(x), lo = float(x - hi): about 48 significant bits,
// evaluated on the device in float32 double-float arithmetic (this GPU's
// float64 rate is a small fraction of its float32 rate).
struct PriorTri {
  float ua, va, ub, vb, uc, vc;
  float da_hi, da_lo, gu_hi, gu_lo, gv_hi, gv_lo;
};
// Split of a double into float hi + lo (host side).
inline void split_double(double x, float& hi, float& lo) {
  hi = static_cast<float>(x);
  lo = static_cast<float>(x - static_cast<double>(hi));
}

constexpr int kBinSize = 16;       // prior raster: triangles binned per 16x16 pixels

struct PriorArgs {
  int H, W, nbx, nby;
  const PriorTri* tris;
  const int* bin_start;            // [nbx * nby + 1]
  const int* bin_items;            // triangle indices, ascending per bin
  float* mu;                       // [H][W], NaN outside the triangulation
};

// Everything the fused sweep kernel needs besides the two tensor maps.
struct SweepArgs {
  int H, W, C, D, ref, dtype, bpp; // dtype 0 = uint8, 1 = float32, 2 = float16, 3 = bfloat16; bpp = bytes per pixel
  int TR, TW;                      // tile rows / columns; threads = TR * TW
  int L, R;                        // staged texel halo left / right of the tile
  int SW, SWp;                     // staged texels per row, padded to a multiple of 32
  int RW;                          // staged raw pixels per row (multiple of 16)
  int KP;                          // cameras padded to a multiple of 4 (table stride)
  int iters, early_exit, mseg;
  int prec;                        // staged maps: kPrecF32, kPrecF16 or kPrecBF16
  int dyn_only;                    // reconstruct only pixels with P_ref(dynamic) >= threshold
  float seg_threshold;             // that threshold (probability)
  const int* tile_list;            // non-null: blockIdx.x indexes this list of tile ids
  const int* n_tiles;              // its length (CTAs beyond it exit)
  float beta, gamma, inv2s2, log_thr, eps;
  const float* wtab;               // [D][KP] interpolation weight of camera k at d_j
  const int* otab;                 // [D][KP] floor(-d_j * b_k)
  const unsigned* chg;             // [D] bit k: otab[j][k] != otab[j-1][k] (j = 0: all)
  const float* dval;               // [D] d_j
  const float* mu;                 // [H][W] prior centre, NaN outside
  // fused prior (single-frame hard EM): non-null ptris means the kernel
  // computes the prior centre of its own pixels (the sweep while its TMA
  // copies are in flight, the dynamic-only tile classifier for the whole
  // frame) and writes it to mu_out instead of reading mu
  const PriorTri* ptris;
  const int* pbin_start;
  const int* pbin_items;
  int pnbx;
  float* mu_out;
  // fused refocus (same mode): non-null means the sweep kernel also writes
  // Eq. 2 for its pixels from the raw rows it staged, [H][W][C] float32
  // (the dynamic-only tile classifier reads the reference image from img)
  float* refocus_out;
  const uint8_t* img;              // [K][H] rows of img_pitch bytes
  size_t img_pitch;
  int omin[kMaxCams], omax[kMaxCams];  // per camera: min / max over j of otab[j][k]
  int32_t* d_idx;                  // [H][W]
  float* d_out;                    // [H][W] or null
  uint16_t* labels;                // [H][W] or null
  float* post;                     // [K][H][W] or null
  unsigned long long* counter;     // (pixel, candidate) objectives the M-steps evaluated
  unsigned long long* static_counter;  // static ray samples the M-steps evaluated (may be null)
  unsigned long long* sweeps;      // executed pixel-iterations (E-steps; may be null)
  unsigned* status;                // kStatus* bits
  unsigned long long timeout_ns;   // bounded-wait limit
  // exact candidate pruning (set_pruning): on/off, the rounding margin of
  // the segmentation bound, and d_j = d0 + j / inv_step
  int prune;
  float seg_margin, d0, inv_step;
};

// Candidate pruning of the sweep: the M-steps skip candidates whose upper
// bound (prior + largest segmentation term) is below an objective already
// computed, which leaves every arg-max unchanged.  It is switched off where
// the candidate spacing is too fine for the float32 index arithmetic of the
// interval (below 2^-12 of the largest |d|).  seg_margin covers the
// float32 rounding of the segmentation sums (at most K terms of magnitude
// <= max(1, |ln eps|) each, summed in at most 2K + 1 operations): 2^-14 (1 +
// K max(1, |ln eps|)), far above that rounding and far below the spread of the
// prior (log(1 + 1/gamma)).
// (SweepArgs and CalibArgs)
template <typename Args>
inline void set_pruning(Args& a, int on, int K, const float* dval, int D, float eps) {
  const double d0 = dval[0], d1 = dval[D - 1];
  const double step = D > 1 ? (d1 - d0) / (D - 1) : 0.0;
  const double scale = std::max(1.0, std::max(std::fabs(d0), std::fabs(d1)));
  a.prune = on && D > 1 && step >= scale * (1.0 / 4096.0);
  a.d0 = static_cast<float>(d0);
  a.inv_step = step > 0.0 ? static_cast<float>(1.0 / step) : 0.f;
  const double le = std::max(1.0, std::fabs(std::log(static_cast<double>(eps))));
  a.seg_margin = static_cast<float>((1.0 + K * le) / 16384.0);
}

// Per-frame arguments of the persistent sweep, in global memory (TMA
// descriptors must be 64-byte aligned; CUtensorMap's own alignment gives it).
struct FrameDesc {
  CUtensorMap img_map;
  CUtensorMap p_map;
  SweepArgs args;
};
static_assert(alignof(FrameDesc) >= 64 && sizeof(FrameDesc) % 64 == 0, "TMA descriptors need 64-byte alignment");

struct RefocusArgs {
  int H, W, C, K, ref, dtype, KP;
  size_t pitch;                    // bytes per image row
  const uint8_t* img;              // [K][H][pitch]
  const float* wtab;
  const int* otab;
  const int32_t* d_idx;
  const uint16_t* labels;
  float* out;                      // [H][W][C]
};

// Calibrated (non-rectified) array, Eq. 1 in generalized disparity space:
// camera k sees reference pixel (u, v) at disparity d at the dehomogenised
// cam[k] * (u, v, 1, d).  The descriptor maps of every camera are written to
// HBM once per run (fa, fb) and sampled bilinearly by the sweep.
struct CalibArgs {
  int K, H, W, C, D, ref, dtype, iters, early_exit, mseg, dyn_only;
  float seg_threshold, beta, gamma, inv2s2, log_thr, eps;
  float cam[kMaxCams][12];         // row-major 3x4 per camera
  const uint8_t* img;              // [K][H] rows of img_pitch bytes ([W][C] pixels)
  size_t img_pitch;
  const float* P;                  // [K][H] rows of p_pitch bytes, P(dynamic)
  size_t p_pitch;
  float4* fa;                      // [K][H][W] {Y, Sobel-x/8, Sobel-y/8, log max(1-P, eps)}
  float* fb;                       // [K][H][W] log max(P, eps)
  const float* dval;               // [D]
  const float* mu;                 // [H][W] prior centre, NaN outside
  int32_t* d_idx;                  // [H][W]
  float* d_out;                    // [H][W] or null
  uint16_t* labels;                // [H][W]
  float* post;                     // [K][H][W] or null
  float* refocus;                  // [H][W][C] or null
  unsigned long long* counter;     // (pixel, candidate) objectives the M-steps evaluated
  unsigned long long* sweeps;      // executed pixel-iterations (may be null)
  int prune;                       // exact candidate pruning (set_pruning; the
  float seg_margin, d0, inv_step;  // segmentation bound is 0: every log p <= 0)
};

// Support points of the disparity prior (rectified arrays).
struct SupportArgs {
  int K, H, W, C, dtype, ref, D;
  float d_min, d_max, seg_threshold;
  int grid, ratio_pct, texture, window, min_support;
  float delta;
  float b[kMaxCams];
  const uint8_t* img;              // [K][H] rows of img_pitch bytes
  size_t img_pitch;
  const float* P;                  // [K][H] rows of p_pitch bytes, P(dynamic)
  size_t p_pitch;
  int n_src;                       // sources: the reference, then every other camera in order
  int src[kMaxCams];
  unsigned tmask[kMaxCams];        // per source: the target cameras
  int delta_c[kMaxCams];           // per source: candidates spanning one pixel on the widest pair (0: none)
  const int* offsets;              // [n_src][K][D] target column offsets (double rounding on the host)
  int nx, ny;                      // cells
  int16_t* gx;                     // [K][H][W] integer Sobel responses
  int16_t* gy;
  int* match;                      // [n_src][ny*nx] accepted candidate or -1
  int* claim;                      // [ny*nx] first other-view claimant
  int* pre_j;                      // [ny*nx] before the consistency test
  int* pre_src;
  double* pre_u;
  double* pre_v;
  int* cell_j;                     // [ny*nx] final
  int* cell_src;
  double* cell_u;
  double* cell_v;
  float* points;                   // [max_points][3]
  int max_points;
  int* n_points;
  int* chunk_count;                // [ceil(ny*nx / 1024)] kept cells per chunk
};

struct MedianArgs {
  int H, W, C;
  const float* in;
  float* out;                      // null: frame has no refocus output
};

// Work item of the batched raster-order kernels: one row of one frame.
struct RowItem {
  int frame, row;
};

// Work item of the persistent sweep: tile (x, y) of frame `frame`.
struct TileItem {
  int frame, x, y, pad;
};

// Shared-memory bytes of the sweep kernel for a tile configuration.
size_t sweep_smem_bytes(int K, const SweepArgs& a);
// Largest CTA (tile rows x columns) the single-frame sweep kernel for K
// cameras is compiled for (its launcher rejects larger ones); the persistent
// kernel of uneven batches takes up to 256 threads at every K.
constexpr int sweep_max_threads(int K) { return K <= 8 ? 256 : 128; }
// The soft-EM state kept per tile pixel between iterations: P(ray static)
// per camera, then the K(K-1)/2 pair weights (one slot, unused, for a single
// camera); floats per pixel and shared-memory bytes per tile.
__host__ __device__ constexpr int soft_state_floats(int K) { return K + (K * (K - 1) / 2 > 0 ? K * (K - 1) / 2 : 1); }
__host__ __device__ inline size_t soft_state_bytes(int K, int pixels) {
  return static_cast<size_t>(pixels) * static_cast<size_t>(soft_state_floats(K)) * 4;
}

cudaError_t launch_prior_raster(const PriorArgs& a, cudaStream_t s);
// Dynamic-only mode: list the tiles holding a pixel with P_ref >= threshold
// (tile_list / *n_tiles, n_tiles zeroed by the caller) and write the outputs
// of the pixels of every other tile.
cudaError_t launch_tile_classify(int K, const SweepArgs& a, const float* seg_prior, size_t p_pitch,
                                 int* tile_list, int* n_tiles, cudaStream_t s);
cudaError_t launch_em_sweep(int K, const CUtensorMap& img_map, const CUtensorMap& p_map,
                            const SweepArgs& a, cudaStream_t s);
// Soft EM (mode 1, K <= 8) or joint MAP (mode 2) on float32 staged maps.
cudaError_t launch_em_variant(int K, int mode, const CUtensorMap& img_map, const CUtensorMap& p_map,
                              const SweepArgs& a, cudaStream_t s);
cudaError_t launch_refocus(const RefocusArgs& a, cudaStream_t s);
cudaError_t launch_support(const SupportArgs& a, cudaStream_t s);
// Calibrated array: descriptor maps, the per-pixel EM, the refocus.
cudaError_t launch_calib_features(const CalibArgs& a, cudaStream_t s);
cudaError_t launch_calib_sweep(const CalibArgs& a, cudaStream_t s);
cudaError_t launch_calib_refocus(const CalibArgs& a, cudaStream_t s);
cudaError_t launch_median3(const float* in, float* out, int H, int W, int C, cudaStream_t s);
cudaError_t launch_prior_raster_batched(const PriorArgs* frames, const RowItem* items, const int* n_items,
                                        int grid, cudaStream_t s);
cudaError_t launch_refocus_batched(const RefocusArgs* frames, const RowItem* items, const int* n_items, int grid,
                                   cudaStream_t s);
cudaError_t launch_median3_batched(const MedianArgs* frames, const RowItem* items, const int* n_items, int grid,
                                   cudaStream_t s);
// Persistent sweep over the items of one camera count; centred: every frame
// of the launch has its reference camera at index K / 2.
cudaError_t launch_em_sweep_persistent(int K, int prec, const FrameDesc* frames, const TileItem* items,
                                       const int* first_item, const int* n_items, unsigned* head, size_t smem,
                                       int grid, int threads, int centred, cudaStream_t s);
// Resident CTAs per SM of the persistent sweep for this shared-memory size.
int em_sweep_persistent_occupancy(int K, int prec, size_t smem, int threads, int centred);

// Validity of the model and run parameters every entry point shares: finite
// constants with sigma > 0, gamma >= 0, eps > 0, beta >= 0 and
// 0 < seg_threshold < 1; precision and em_mode among their enumerators; the
// two EM variants on float32 maps only.  False with *why set otherwise.
bool check_params(const lf_params& p, std::string* why);

// Host-side allocation-failure injection (lf_inject_alloc_failure): true
// when the library's allocation wrappers must report LF_ENOMEM for the
// allocation they are about to make (no allocation is attempted).
bool injected_alloc_failure();

// Sets the calling thread's message returned by lf_last_error.
void set_error_message(const std::string& msg);

// Host Delaunay triangulation (Bowyer-Watson with a symbolic point at infinity).
// pts: n points (x, y); writes counter-clockwise triangles into out (3 ints each).
int delaunay(const double* xy, int n, int* out_tris, int max_tris);

}  // namespace lf

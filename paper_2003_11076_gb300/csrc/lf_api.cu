// Host side of the C ABI declared in include/lf.h: validation, the per-(d, k)
// sampling tables, the host Delaunay and triangle bins of the prior, TMA
// descriptors, buffer ownership and kernel launches.  No compute happens on
// the host beyond the triangulation of the sparse support points.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <string>
#include <vector>

#include "em_sweep.cuh"
#include "lf.h"
#include "lf_internal.h"

namespace lf {
#define LF_DECL_SWEEP(t, k)                                                                                   \
  cudaError_t launch_em_sweep_##t##_k##k(const CUtensorMap&, const CUtensorMap&, const SweepArgs&, cudaStream_t); \
  cudaError_t launch_em_sweep_persistent_##t##_k##k(const FrameDesc*, const TileItem*, const int*, const int*, \
                                                    unsigned*, size_t, int, int, int, cudaStream_t);            \
  int em_sweep_persistent_occupancy_##t##_k##k(size_t, int, int);
#define LF_DECL_SWEEPS(t)                                                                                     \
  LF_DECL_SWEEP(t, 1) LF_DECL_SWEEP(t, 2) LF_DECL_SWEEP(t, 3) LF_DECL_SWEEP(t, 4) LF_DECL_SWEEP(t, 5)           \
  LF_DECL_SWEEP(t, 6) LF_DECL_SWEEP(t, 7) LF_DECL_SWEEP(t, 8) LF_DECL_SWEEP(t, 9) LF_DECL_SWEEP(t, 10)          \
  LF_DECL_SWEEP(t, 11) LF_DECL_SWEEP(t, 12)
LF_DECL_SWEEPS(f32)
LF_DECL_SWEEPS(f16)
LF_DECL_SWEEPS(bf16)
#define LF_DECL_CLASSIFY(k) \
  cudaError_t launch_tile_classify_k##k(const SweepArgs&, const float*, size_t, int*, int*, cudaStream_t);
LF_DECL_CLASSIFY(1) LF_DECL_CLASSIFY(2) LF_DECL_CLASSIFY(3) LF_DECL_CLASSIFY(4) LF_DECL_CLASSIFY(5)
LF_DECL_CLASSIFY(6) LF_DECL_CLASSIFY(7) LF_DECL_CLASSIFY(8) LF_DECL_CLASSIFY(9) LF_DECL_CLASSIFY(10)
LF_DECL_CLASSIFY(11) LF_DECL_CLASSIFY(12)
#undef LF_DECL_CLASSIFY
#undef LF_DECL_SWEEPS
#undef LF_DECL_SWEEP

#define LF_DECL_VARIANT(k) \
  cudaError_t launch_em_variant_k##k(int, const CUtensorMap&, const CUtensorMap&, const SweepArgs&, cudaStream_t);
LF_DECL_VARIANT(1) LF_DECL_VARIANT(2) LF_DECL_VARIANT(3) LF_DECL_VARIANT(4) LF_DECL_VARIANT(5)
LF_DECL_VARIANT(6) LF_DECL_VARIANT(7) LF_DECL_VARIANT(8) LF_DECL_VARIANT(9) LF_DECL_VARIANT(10)
LF_DECL_VARIANT(11) LF_DECL_VARIANT(12)
#undef LF_DECL_VARIANT

size_t sweep_smem_bytes(int K, const SweepArgs& a) { return dev::sweep_layout(K, a).total; }

cudaError_t launch_em_variant(int K, int mode, const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a,
                              cudaStream_t s) {
  typedef cudaError_t (*VariantLaunch)(int, const CUtensorMap&, const CUtensorMap&, const SweepArgs&, cudaStream_t);
  static const VariantLaunch table[kMaxCams] = {
      launch_em_variant_k1, launch_em_variant_k2, launch_em_variant_k3,  launch_em_variant_k4,
      launch_em_variant_k5, launch_em_variant_k6, launch_em_variant_k7,  launch_em_variant_k8,
      launch_em_variant_k9, launch_em_variant_k10, launch_em_variant_k11, launch_em_variant_k12};
  if (K < 1 || K > kMaxCams) return cudaErrorInvalidValue;
  return table[K - 1](mode, i, p, a, s);
}

typedef cudaError_t (*SweepLaunch)(const CUtensorMap&, const CUtensorMap&, const SweepArgs&, cudaStream_t);

cudaError_t launch_em_sweep(int K, const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a,
                            cudaStream_t s) {
#define LF_ROW(t)                                                                                           \
  {launch_em_sweep_##t##_k1, launch_em_sweep_##t##_k2,  launch_em_sweep_##t##_k3,  launch_em_sweep_##t##_k4, \
   launch_em_sweep_##t##_k5, launch_em_sweep_##t##_k6,  launch_em_sweep_##t##_k7,  launch_em_sweep_##t##_k8, \
   launch_em_sweep_##t##_k9, launch_em_sweep_##t##_k10, launch_em_sweep_##t##_k11, launch_em_sweep_##t##_k12}
  static const SweepLaunch table[3][kMaxCams] = {LF_ROW(f32), LF_ROW(f16), LF_ROW(bf16)};
#undef LF_ROW
  if (K < 1 || K > kMaxCams || a.prec < 0 || a.prec > 2) return cudaErrorInvalidValue;
  return table[a.prec][K - 1](i, p, a, s);
}

typedef cudaError_t (*PersistentLaunch)(const FrameDesc*, const TileItem*, const int*, const int*, unsigned*,
                                        size_t, int, int, int, cudaStream_t);
typedef int (*PersistentOcc)(size_t, int, int);

cudaError_t launch_em_sweep_persistent(int K, int prec, const FrameDesc* frames, const TileItem* items,
                                       const int* first_item, const int* n_items, unsigned* head, size_t smem,
                                       int grid, int threads, int centred, cudaStream_t s) {
#define LF_ROW(t)                                                                                   \
  {launch_em_sweep_persistent_##t##_k1, launch_em_sweep_persistent_##t##_k2,                         \
   launch_em_sweep_persistent_##t##_k3, launch_em_sweep_persistent_##t##_k4,                         \
   launch_em_sweep_persistent_##t##_k5, launch_em_sweep_persistent_##t##_k6,                         \
   launch_em_sweep_persistent_##t##_k7, launch_em_sweep_persistent_##t##_k8,                         \
   launch_em_sweep_persistent_##t##_k9, launch_em_sweep_persistent_##t##_k10,                        \
   launch_em_sweep_persistent_##t##_k11, launch_em_sweep_persistent_##t##_k12}
  static const PersistentLaunch table[3][kMaxCams] = {LF_ROW(f32), LF_ROW(f16), LF_ROW(bf16)};
#undef LF_ROW
  if (K < 1 || K > kMaxCams || prec < 0 || prec > 2) return cudaErrorInvalidValue;
  return table[prec][K - 1](frames, items, first_item, n_items, head, smem, grid, threads, centred, s);
}

cudaError_t launch_tile_classify(int K, const SweepArgs& a, const float* seg_prior, size_t p_pitch,
                                 int* tile_list, int* n_tiles, cudaStream_t s) {
  typedef cudaError_t (*Fn)(const SweepArgs&, const float*, size_t, int*, int*, cudaStream_t);
  static const Fn table[kMaxCams] = {launch_tile_classify_k1,  launch_tile_classify_k2,  launch_tile_classify_k3,
                                     launch_tile_classify_k4,  launch_tile_classify_k5,  launch_tile_classify_k6,
                                     launch_tile_classify_k7,  launch_tile_classify_k8,  launch_tile_classify_k9,
                                     launch_tile_classify_k10, launch_tile_classify_k11, launch_tile_classify_k12};
  if (K < 1 || K > kMaxCams) return cudaErrorInvalidValue;
  return table[K - 1](a, seg_prior, p_pitch, tile_list, n_tiles, s);
}

int em_sweep_persistent_occupancy(int K, int prec, size_t smem, int threads, int centred) {
#define LF_ROW(t)                                                                                       \
  {em_sweep_persistent_occupancy_##t##_k1, em_sweep_persistent_occupancy_##t##_k2,                       \
   em_sweep_persistent_occupancy_##t##_k3, em_sweep_persistent_occupancy_##t##_k4,                       \
   em_sweep_persistent_occupancy_##t##_k5, em_sweep_persistent_occupancy_##t##_k6,                       \
   em_sweep_persistent_occupancy_##t##_k7, em_sweep_persistent_occupancy_##t##_k8,                       \
   em_sweep_persistent_occupancy_##t##_k9, em_sweep_persistent_occupancy_##t##_k10,                      \
   em_sweep_persistent_occupancy_##t##_k11, em_sweep_persistent_occupancy_##t##_k12}
  static const PersistentOcc table[3][kMaxCams] = {LF_ROW(f32), LF_ROW(f16), LF_ROW(bf16)};
#undef LF_ROW
  if (K < 1 || K > kMaxCams || prec < 0 || prec > 2) return 0;
  return table[prec][K - 1](smem, threads, centred);
}
}  // namespace lf

using namespace lf;

namespace {

thread_local std::string g_err;

lf_status fail(lf_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

lf_status cuda_fail(cudaError_t e, const char* what) {
  return fail(LF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LF_CUDA(call, what)                         \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

template <class T>
lf_status grow(T** ptr, size_t* cap, size_t need, const char* what) {
  if (need <= *cap && *ptr) return LF_OK;
  if (*ptr) cudaFree(*ptr);
  *ptr = nullptr;
  *cap = 0;
  size_t n = std::max<size_t>(need, 1);
  if (injected_alloc_failure()) return fail(LF_ENOMEM, std::string(what) + ": out of device memory (injected)");
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), n * sizeof(T));
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return e == cudaErrorMemoryAllocation ? fail(LF_ENOMEM, std::string(what) + ": out of device memory")
                                          : cuda_fail(e, what);
  }
  *cap = n;
  return LF_OK;
}

constexpr unsigned long long kTimeoutNs = 2000000000ull;  // 2 s bounded device waits

}  // namespace

void lf::set_error_message(const std::string& msg) { g_err = msg; }

namespace {
std::atomic<long long> g_fail_after{-1};  // successful allocations left before the injected failure; < 0: off
}  // namespace

bool lf::injected_alloc_failure() {
  long long v = g_fail_after.load();
  while (v >= 0) {
    if (g_fail_after.compare_exchange_weak(v, v - 1)) return v == 0;  // the (after + 1)-th allocation fails
  }
  return false;
}

bool lf::check_params(const lf_params& p, std::string* why) {
  const char* msg = nullptr;
  if (!std::isfinite(p.beta) || !std::isfinite(p.gamma) || !std::isfinite(p.sigma) ||
      !std::isfinite(p.seg_threshold) || !std::isfinite(p.eps))
    msg = "invalid lf_params: non-finite constant";
  else if (p.sigma <= 0.f)
    msg = "invalid lf_params: sigma must be > 0";
  else if (1.0 / (2.0 * static_cast<double>(p.sigma) * p.sigma) >
           static_cast<double>(std::numeric_limits<float>::max()))
    msg = "invalid lf_params: sigma too small (the prior's 1 / (2 sigma^2) must be finite in float32)";
  else if (p.gamma < 0.f)
    msg = "invalid lf_params: gamma must be >= 0";
  else if (p.eps <= 0.f)
    msg = "invalid lf_params: eps must be > 0";
  else if (p.beta < 0.f)
    msg = "invalid lf_params: beta must be >= 0";
  else if (p.seg_threshold <= 0.f || p.seg_threshold >= 1.f)
    msg = "invalid lf_params: seg_threshold must be in (0, 1)";
  else if (p.precision != LF_PREC_F32 && p.precision != LF_PREC_F16 && p.precision != LF_PREC_BF16)
    msg = "precision must be LF_PREC_F32, LF_PREC_F16 or LF_PREC_BF16";
  else if (p.em_mode != LF_EM_HARD && p.em_mode != LF_EM_SOFT && p.em_mode != LF_EM_JOINT)
    msg = "em_mode must be LF_EM_HARD, LF_EM_SOFT or LF_EM_JOINT";
  else if (p.em_mode != LF_EM_HARD && p.precision != LF_PREC_F32)
    msg = "the soft-EM and joint-MAP modes stage float32 maps only (LF_PREC_F32)";
  if (msg && why) *why = msg;
  return msg == nullptr;
}

struct lf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int K = 0, H = 0, W = 0, D = 0, ref = 0;
  float d_min = 0.f, d_max = 0.f;
  std::vector<float> b;
  lf_params p{};
  // sampling tables (pixel independent): o = floor(-d_j b_k), w = -d_j b_k - o
  int KP = 4, L = 0, R = 0;
  std::vector<float> wtab, dval;
  std::vector<int> otab;
  std::vector<unsigned> chg;
  float* d_wtab = nullptr;
  int* d_otab = nullptr;
  unsigned* d_chg = nullptr;
  float* d_dval = nullptr;
  float* d_mu = nullptr;
  unsigned long long* d_counter = nullptr;
  unsigned* d_status = nullptr;
  // current inputs
  bool have_inputs = false;
  int C = 0, dtype = 0, bpp = 0;
  const uint8_t* img = nullptr;
  size_t img_pitch = 0;
  const float* P = nullptr;
  size_t p_pitch = 0;
  uint8_t* own_img = nullptr;
  size_t own_img_cap = 0;
  float* own_P = nullptr;
  size_t own_P_cap = 0;
  int* d_tiles = nullptr;        // dynamic-only: list of tiles to sweep, then its length
  size_t tiles_cap = 0;
  // support-point detection (lf_set_inputs with M = LF_DETECT_SUPPORT)
  lf_support_params sp{};
  std::vector<float> support_pts;  // the last detected points, (u, v, d) triples
  int16_t* d_sgrad = nullptr;      // gx then gy
  size_t sgrad_cap = 0;
  int* d_sint = nullptr;           // offsets, match, claim, pre_j, pre_src, cell_j, cell_src, count
  size_t sint_cap = 0;
  double* d_sdbl = nullptr;        // pre_u, pre_v, cell_u, cell_v
  size_t sdbl_cap = 0;
  float* d_spts = nullptr;
  size_t spts_cap = 0;
  cudaEvent_t sup_ev[2] = {nullptr, nullptr};
  double set_inputs_ms = 0.0;      // host time of lf_set_inputs since the last lf_get_stats
  int set_inputs_calls = 0;
  // calibrated array: camera matrices and the per-run descriptor maps
  bool calibrated = false;
  float cams[kMaxCams * 12] = {};
  float4* d_fa = nullptr;
  size_t fa_cap = 0;
  float* d_fb = nullptr;
  size_t fb_cap = 0;
  // prior
  std::vector<PriorTri> h_tris;
  std::vector<int> h_bins;  // [nbins + 1] starts, then items
  PriorTri* d_tris = nullptr;
  size_t tris_cap = 0;
  int* d_bins = nullptr;
  size_t bins_cap = 0;
  int nbx = 0, nby = 0;
  // staging for host outputs
  int32_t* o_didx = nullptr;
  float* o_d = nullptr;
  uint16_t* o_labels = nullptr;
  float* o_post = nullptr;
  float* o_ref = nullptr;
  float* o_tmp = nullptr;
  size_t o_didx_cap = 0, o_d_cap = 0, o_labels_cap = 0, o_post_cap = 0, o_ref_cap = 0, o_tmp_cap = 0;
  // TMA descriptors of the current inputs
  CUtensorMap img_map{}, p_map{};
  // tiles (force_TR > 0: shape set by lf_set_tile)
  int TR = 2, TW = 128, SW = 0, SWp = 0, RW = 0;
  int force_TR = 0, force_TW = 0;
  lf_stats stats{};
  // optional per-kernel timing: per run, events before prior, sweep, refocus,
  // median and after; summed by lf_get_stats
  bool timing = false;
  struct RunEvents {
    cudaEvent_t ev[5];
    bool used[5];
  };
  std::vector<RunEvents> events;
  size_t events_used = 0;
  uint64_t runs = 0;
};

namespace {

bool finite(float x) { return std::isfinite(x); }

// Pick the sweep tile: the first candidate whose staged rows fit one TMA box
// (256 eight-byte words per row) and whose shared memory allows at least two
// CTAs per SM, else at least one.  With a narrow disparity halo (L + R <= 32
// columns) 4 x 64 tiles come first (measured fastest on the 960x600
// five-camera frame, halo 26); wider halos favour wider tiles, which stage
// fewer redundant columns per pixel.
lf_status choose_tiles(lf_ctx* c) {
  static const int narrow[][2] = {{4, 64}, {2, 128}, {1, 128}, {2, 64}, {1, 64}, {2, 32}, {1, 32}};
  static const int wide[][2] = {{2, 128}, {1, 128}, {4, 64}, {2, 64}, {1, 64}, {2, 32}, {1, 32}};
  const auto& cand = c->L + c->R <= 32 ? narrow : wide;
  const int forced[1][2] = {{c->force_TR, c->force_TW}};
  int dev_smem = 0;
  cudaError_t e = cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  if (e != cudaSuccess || dev_smem <= 0) dev_smem = 227 * 1024;
  for (int pass = 0; pass < 2; ++pass) {
    const size_t limit = pass == 0 ? std::min<size_t>(dev_smem, 110 * 1024) : static_cast<size_t>(dev_smem);
    const int ncand = c->force_TR > 0 ? 1 : static_cast<int>(sizeof(cand) / sizeof(cand[0]));
    for (int ci = 0; ci < ncand; ++ci) {
      const int* t = c->force_TR > 0 ? forced[0] : cand[ci];
      if (t[0] * t[1] > sweep_max_threads(c->K)) continue;
      SweepArgs a{};
      a.TR = t[0];
      a.TW = t[1];
      a.SW = a.TW + c->L + c->R;
      a.SWp = (a.SW + 31) / 32 * 32;
      a.RW = (a.SW + 17 + 15) / 16 * 16;
      a.bpp = c->bpp;
      a.D = c->D;
      a.KP = c->KP;
      a.prec = c->p.precision;
      if (a.RW * a.bpp / 8 > 256 || a.RW / 2 > 256) continue;
      const size_t need = c->p.em_mode == LF_EM_SOFT ? dev::soft_state_offset(c->K, a) + soft_state_bytes(c->K, a.TR * a.TW)
                                                     : sweep_smem_bytes(c->K, a);
      if (need > limit) continue;
      c->TR = a.TR;
      c->TW = a.TW;
      c->SW = a.SW;
      c->SWp = a.SWp;
      c->RW = a.RW;
      return LF_OK;
    }
  }
  return fail(LF_EINVAL, c->force_TR > 0 ? "the tile set by lf_set_tile does not fit the staging limits"
                                         : "disparity halo too wide for the sweep kernel's shared-memory staging");
}

lf_status encode_maps(lf_ctx* c) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return fail(LF_ECUDA, "cuTensorMapEncodeTiled unavailable from the driver");
  {
    const cuuint64_t dims[3] = {static_cast<cuuint64_t>((static_cast<size_t>(c->W) * c->bpp + 7) / 8),
                                static_cast<cuuint64_t>(c->H), static_cast<cuuint64_t>(c->K)};
    const cuuint64_t strides[2] = {static_cast<cuuint64_t>(c->img_pitch),
                                   static_cast<cuuint64_t>(c->img_pitch * c->H)};
    const cuuint32_t box[3] = {static_cast<cuuint32_t>(c->RW * c->bpp / 8), static_cast<cuuint32_t>(c->TR + 2),
                               static_cast<cuuint32_t>(c->K)};
    const cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(&c->img_map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<uint8_t*>(c->img), dims, strides,
                     box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(LF_ECUDA, "cuTensorMapEncodeTiled(images) failed: " + std::to_string(r));
  }
  {
    const cuuint64_t dims[3] = {static_cast<cuuint64_t>((c->W + 1) / 2), static_cast<cuuint64_t>(c->H),
                                static_cast<cuuint64_t>(c->K)};
    const cuuint64_t strides[2] = {static_cast<cuuint64_t>(c->p_pitch), static_cast<cuuint64_t>(c->p_pitch * c->H)};
    const cuuint32_t box[3] = {static_cast<cuuint32_t>(c->RW / 2), static_cast<cuuint32_t>(c->TR),
                               static_cast<cuuint32_t>(c->K)};
    const cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(&c->p_map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<float*>(c->P), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(LF_ECUDA, "cuTensorMapEncodeTiled(seg_prior) failed: " + std::to_string(r));
  }
  return LF_OK;
}

// Host triangulation + plane coefficients + 16x16 bins of the prior.
void build_prior(lf_ctx* c, const float* pts, int M) {
  c->h_tris.clear();
  std::vector<double> xy(static_cast<size_t>(2) * M);
  for (int i = 0; i < M; ++i) {
    xy[2 * i] = pts[3 * i];
    xy[2 * i + 1] = pts[3 * i + 1];
  }
  std::vector<int> tris(static_cast<size_t>(6) * std::max(M, 1) + 6);
  int nt = M >= 3 ? lf::delaunay(xy.data(), M, tris.data(), static_cast<int>(tris.size() / 3)) : 0;
  if (nt > static_cast<int>(tris.size() / 3)) {
    tris.resize(static_cast<size_t>(3) * nt);
    nt = lf::delaunay(xy.data(), M, tris.data(), nt);
  }
  for (int t = 0; t < nt; ++t) {
    const int ia = tris[3 * t], ib = tris[3 * t + 1], ic = tris[3 * t + 2];
    PriorTri T;
    T.ua = pts[3 * ia]; T.va = pts[3 * ia + 1];
    T.ub = pts[3 * ib]; T.vb = pts[3 * ib + 1];
    T.uc = pts[3 * ic]; T.vc = pts[3 * ic + 1];
    const double da = pts[3 * ia + 2], db = pts[3 * ib + 2], dc = pts[3 * ic + 2];
    const double du1 = static_cast<double>(T.ub) - T.ua, dv1 = static_cast<double>(T.vb) - T.va;
    const double du2 = static_cast<double>(T.uc) - T.ua, dv2 = static_cast<double>(T.vc) - T.va;
    const double det = du1 * dv2 - du2 * dv1;
    if (det == 0.0) continue;
    split_double(da, T.da_hi, T.da_lo);
    split_double(((db - da) * dv2 - (dc - da) * dv1) / det, T.gu_hi, T.gu_lo);
    split_double((du1 * (dc - da) - du2 * (db - da)) / det, T.gv_hi, T.gv_lo);
    c->h_tris.push_back(T);
  }
  c->nbx = (c->W + kBinSize - 1) / kBinSize;
  c->nby = (c->H + kBinSize - 1) / kBinSize;
  const int nb = c->nbx * c->nby;
  std::vector<int> count(static_cast<size_t>(nb) + 1, 0);
  auto bbox = [&](const PriorTri& T, int& bx0, int& bx1, int& by0, int& by1) {
    const double u0 = std::ceil(std::min({T.ua, T.ub, T.uc})), u1 = std::floor(std::max({T.ua, T.ub, T.uc}));
    const double v0 = std::ceil(std::min({T.va, T.vb, T.vc})), v1 = std::floor(std::max({T.va, T.vb, T.vc}));
    const double uu0 = std::max(u0, 0.0), uu1 = std::min(u1, static_cast<double>(c->W - 1));
    const double vv0 = std::max(v0, 0.0), vv1 = std::min(v1, static_cast<double>(c->H - 1));
    if (uu1 < uu0 || vv1 < vv0) return false;
    bx0 = static_cast<int>(uu0) / kBinSize; bx1 = static_cast<int>(uu1) / kBinSize;
    by0 = static_cast<int>(vv0) / kBinSize; by1 = static_cast<int>(vv1) / kBinSize;
    return true;
  };
  for (const PriorTri& T : c->h_tris) {
    int bx0, bx1, by0, by1;
    if (!bbox(T, bx0, bx1, by0, by1)) continue;
    for (int by = by0; by <= by1; ++by)
      for (int bx = bx0; bx <= bx1; ++bx) count[by * c->nbx + bx + 1]++;
  }
  for (int i = 0; i < nb; ++i) count[i + 1] += count[i];
  c->h_bins.assign(static_cast<size_t>(nb) + 1 + count[nb], 0);
  std::copy(count.begin(), count.end(), c->h_bins.begin());
  std::vector<int> fill(count.begin(), count.end() - 1);
  for (size_t t = 0; t < c->h_tris.size(); ++t) {
    int bx0, bx1, by0, by1;
    if (!bbox(c->h_tris[t], bx0, bx1, by0, by1)) continue;
    for (int by = by0; by <= by1; ++by)
      for (int bx = bx0; bx <= bx1; ++bx) c->h_bins[nb + 1 + fill[by * c->nbx + bx]++] = static_cast<int>(t);
  }
}

lf_status copy_plane(lf_ctx* c, const void* src, size_t row_bytes, bool on_device, uint8_t** own,
                     size_t* own_cap, const uint8_t** use, size_t* pitch) {
  const size_t rows = static_cast<size_t>(c->K) * c->H;
  const bool aligned = (reinterpret_cast<uintptr_t>(src) % 16 == 0) && (row_bytes % 16 == 0);
  if (on_device && aligned) {  // borrow the caller's buffer
    *use = static_cast<const uint8_t*>(src);
    *pitch = row_bytes;
    return LF_OK;
  }
  const size_t p = (row_bytes + 15) / 16 * 16;
  lf_status s = grow(own, own_cap, rows * p, "input staging");
  if (s != LF_OK) return s;
  LF_CUDA(cudaMemcpy2DAsync(*own, p, src, row_bytes, row_bytes, rows,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream),
          "input copy");
  *use = *own;
  *pitch = p;
  return LF_OK;
}

}  // namespace

namespace {
// Self-test of the bounded wait the sweep kernels use on their TMA copies:
// thread 0 arms the CTA's mbarrier for `bytes` of transaction that no copy
// will deliver, every thread waits with the sweep's bounded wait, and the
// expiry is reported through the status word as in the sweep.  No copy is
// ever issued, so nothing is in flight when the CTA leaves.
__global__ void bounded_wait_selftest_kernel(unsigned* status, unsigned bytes, unsigned long long timeout_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    dev::mbar_init(&bar, 1);
    dev::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) dev::mbar_arrive_expect_tx(&bar, bytes);
  const bool ok = dev::mbar_wait_bounded(&bar, 0u, timeout_ns);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(status, kStatusTmaTimeout);
}
}  // namespace

extern "C" {

void lf_default_params(lf_params* p) {
  if (!p) return;
  p->beta = 200.f;
  p->gamma = 0.1f;
  p->sigma = 2.f;
  p->seg_threshold = 0.7f;
  p->eps = 1e-4f;
  p->mstep_seg_term = 1;
  p->median = 0;
  p->precision = LF_PREC_F32;
  p->early_exit = 1;
  p->dynamic_only = 0;
  p->em_mode = LF_EM_HARD;
  p->prune = 1;
}

const char* lf_last_error(const lf_ctx*) { return g_err.c_str(); }

int lf_triangulate(const float* points, int M, int32_t* tris, int max_tris) {
  if (M < 0 || (M > 0 && !points) || max_tris < 0 || (max_tris > 0 && !tris)) return -1;
  std::vector<double> xy(static_cast<size_t>(2) * M);
  for (int i = 0; i < M; ++i) {
    if (!std::isfinite(points[3 * i]) || !std::isfinite(points[3 * i + 1])) return -1;
    xy[2 * i] = points[3 * i];
    xy[2 * i + 1] = points[3 * i + 1];
  }
  return lf::delaunay(xy.data(), M, tris, max_tris);
}

}  // extern "C"

namespace {
// Both constructors: a rectified array (baselines) or a calibrated one
// (cameras, [K][3][4]; the sampling tables of the rectified sweep are then
// built for zero baselines and not used by the calibrated kernels).
lf_status create_ctx(lf_ctx** out, int n_cams, const float* baselines, const float* cameras, int H, int W,
                     float d_min, float d_max, int D, const lf_params* p) {
  g_err.clear();
  if (!out) return fail(LF_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_cams < 1 || n_cams > kMaxCams) return fail(LF_EINVAL, "n_cams must be in [1, 12]");
  if (!baselines && !cameras) return fail(LF_EINVAL, cameras ? "cameras is NULL" : "baselines is NULL");
  if (H < 3 || W < 3) return fail(LF_EINVAL, "H and W must be >= 3");
  if (D < 1 || D > kMaxD) return fail(LF_EINVAL, "D must be in [1, 1024]");
  if (!finite(d_min) || !finite(d_max) || d_max < d_min) return fail(LF_EINVAL, "need finite d_min <= d_max");
  int ref = -1;
  std::vector<float> zero_b;
  if (cameras) {
    for (int k = 0; k < n_cams; ++k) {
      bool identity = true;
      for (int i = 0; i < 12; ++i) {
        if (!finite(cameras[12 * k + i])) return fail(LF_EINVAL, "non-finite camera matrix entry");
        if (cameras[12 * k + i] != ((i == 0 || i == 5 || i == 10) ? 1.f : 0.f)) identity = false;
      }
      if (identity && ref < 0) ref = k;
      // the homogeneous coordinate is affine in (u, v, d): positive at the 8
      // corners of the pixel box x [d_min, d_max] means positive everywhere
      const float* M = cameras + 12 * k;
      for (int corner = 0; corner < 8; ++corner) {
        const double u = (corner & 1) ? W - 1 : 0, v = (corner & 2) ? H - 1 : 0, d = (corner & 4) ? d_max : d_min;
        if (!(static_cast<double>(M[8]) * u + static_cast<double>(M[9]) * v + M[10] + static_cast<double>(M[11]) * d >
              0.0))
          return fail(LF_EINVAL, "camera " + std::to_string(k) +
                                     ": a ray of the frame at a candidate disparity projects behind the camera");
      }
    }
    if (ref < 0) return fail(LF_EINVAL, "no camera matrix equals [I | 0] (reference camera)");
    if (static_cast<int64_t>(n_cams) * H * W + W + 1 > INT32_MAX)
      return fail(LF_EINVAL, "calibrated arrays: n_cams * H * W must stay below 2^31");
    zero_b.assign(n_cams, 0.f);
    baselines = zero_b.data();
  } else {
    for (int k = 0; k < n_cams; ++k) {
      if (!finite(baselines[k])) return fail(LF_EINVAL, "non-finite baseline");
      if (baselines[k] == 0.f && ref < 0) ref = k;
    }
    if (ref < 0) return fail(LF_EINVAL, "no baseline equals 0 (reference camera)");
  }
  lf_params prm;
  lf_default_params(&prm);
  if (p) prm = *p;
  std::string why;
  if (!check_params(prm, &why)) return fail(LF_EINVAL, why);
  if (prm.em_mode == LF_EM_SOFT && n_cams > 8) return fail(LF_EINVAL, "soft EM supports at most 8 cameras");
  if (cameras && (prm.em_mode != LF_EM_HARD || prm.precision != LF_PREC_F32))
    return fail(LF_EINVAL, "calibrated arrays run the hard EM on float32 maps (LF_EM_HARD, LF_PREC_F32)");

  lf_ctx* c = new (std::nothrow) lf_ctx();
  if (!c) return fail(LF_ENOMEM, "host allocation failed");
  lf_default_support_params(&c->sp);
  if (cameras) {
    c->calibrated = true;
    std::copy(cameras, cameras + 12 * n_cams, c->cams);
  }
  c->K = n_cams;
  c->H = H;
  c->W = W;
  c->D = D;
  c->ref = ref;
  c->d_min = d_min;
  c->d_max = d_max;
  c->b.assign(baselines, baselines + n_cams);
  c->p = prm;
  cudaGetDevice(&c->device);
  c->KP = (n_cams + 3) / 4 * 4;
  c->wtab.assign(static_cast<size_t>(D) * c->KP, 0.f);
  c->otab.assign(static_cast<size_t>(D) * c->KP, 0);
  c->chg.assign(static_cast<size_t>(D), 0u);
  c->dval.assign(static_cast<size_t>(D), 0.f);
  int omin = 0, omax = 0;
  for (int j = 0; j < D; ++j) {
    const double dj = D == 1 ? static_cast<double>(d_min)
                             : static_cast<double>(d_min) +
                                   j * ((static_cast<double>(d_max) - static_cast<double>(d_min)) / (D - 1));
    c->dval[j] = static_cast<float>(dj);
    unsigned m = 0;
    for (int k = 0; k < n_cams; ++k) {
      const double x = -dj * static_cast<double>(baselines[k]);
      const double o = std::floor(x);
      const int oi = static_cast<int>(o);
      c->otab[j * c->KP + k] = oi;
      c->wtab[j * c->KP + k] = static_cast<float>(x - o);
      if (j == 0 || c->otab[(j - 1) * c->KP + k] != oi) m |= 1u << k;
      omin = std::min(omin, oi);
      omax = std::max(omax, oi + 1);
    }
    c->chg[j] = m;
  }
  c->L = -omin;
  c->R = omax;
  lf_status s = LF_OK;
  size_t cap = 0;
  auto bail = [&](lf_status st) {
    lf_destroy(c);
    return st;
  };
  if ((s = grow(&c->d_wtab, &cap, c->wtab.size(), "tables")) != LF_OK) return bail(s);
  cap = 0;
  if ((s = grow(&c->d_otab, &cap, c->otab.size(), "tables")) != LF_OK) return bail(s);
  cap = 0;
  if ((s = grow(&c->d_chg, &cap, c->chg.size(), "tables")) != LF_OK) return bail(s);
  cap = 0;
  if ((s = grow(&c->d_dval, &cap, c->dval.size(), "tables")) != LF_OK) return bail(s);
  cap = 0;
  if ((s = grow(&c->d_mu, &cap, static_cast<size_t>(H) * W, "prior")) != LF_OK) return bail(s);
  cap = 0;
  if ((s = grow(&c->d_counter, &cap, 3, "counter")) != LF_OK) return bail(s);  // objectives, static samples, sweeps
  cap = 0;
  if ((s = grow(&c->d_status, &cap, 1, "status")) != LF_OK) return bail(s);
  cudaError_t e;
  if ((e = cudaMemset(c->d_counter, 0, 3 * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMemset(c->d_status, 0, sizeof(unsigned))) != cudaSuccess)
    return bail(cuda_fail(e, "counter init"));
  if ((e = cudaMemcpy(c->d_wtab, c->wtab.data(), c->wtab.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(c->d_otab, c->otab.data(), c->otab.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(c->d_chg, c->chg.data(), c->chg.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(c->d_dval, c->dval.data(), c->dval.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(cuda_fail(e, "table upload"));
  // the tile choice depends on the bytes per pixel of the inputs and is made
  // again in lf_set_inputs; reject now a halo that no input type can stage
  c->bpp = 1;
  if ((s = choose_tiles(c)) != LF_OK) return bail(s);
  c->bpp = 0;
  *out = c;
  return LF_OK;
}
// Support points of the current inputs into c->support_pts (Sec. III-C): the
// kernels of support.cu, then the points and their count back to the host.
lf_status detect_support(lf_ctx* c) {
  const int K = c->K, D = c->D, H = c->H, W = c->W;
  const lf_support_params& q = c->sp;
  SupportArgs a{};
  a.K = K; a.H = H; a.W = W; a.C = c->C; a.dtype = c->dtype; a.ref = c->ref; a.D = D;
  a.d_min = c->d_min; a.d_max = c->d_max; a.seg_threshold = c->p.seg_threshold;
  a.grid = q.grid; a.ratio_pct = q.ratio_pct; a.texture = q.texture; a.window = q.window;
  a.min_support = q.min_support; a.delta = q.delta;
  for (int k = 0; k < K; ++k) a.b[k] = c->b[k];
  a.img = c->img; a.img_pitch = c->img_pitch; a.P = c->P; a.p_pitch = c->p_pitch;
  a.nx = (W + q.grid - 1) / q.grid;
  a.ny = (H + q.grid - 1) / q.grid;
  const int ncell = a.nx * a.ny;
  // sources: the reference against every other camera, then each other camera
  // against every camera but itself and the reference
  unsigned others = 0;
  for (int t = 0; t < K; ++t)
    if (t != c->ref) others |= 1u << t;
  a.n_src = 0;
  a.src[a.n_src] = c->ref;
  a.tmask[a.n_src++] = others;
  for (int s = 0; s < K; ++s)
    if (s != c->ref) {
      a.src[a.n_src] = s;
      a.tmask[a.n_src++] = others & ~(1u << s);
    }
  // target offsets floor(-d_j (b_t - b_s) + 1/2) and the uniqueness spans, in double
  const double step = D > 1 ? (static_cast<double>(c->d_max) - static_cast<double>(c->d_min)) / (D - 1) : 0.0;
  std::vector<int> off(static_cast<size_t>(a.n_src) * K * D, 0);
  for (int si = 0; si < a.n_src; ++si) {
    const int s = a.src[si];
    double bmax = 0.0;
    for (int t = 0; t < K; ++t) {
      if (!(a.tmask[si] >> t & 1u)) continue;
      const double db = static_cast<double>(c->b[t]) - static_cast<double>(c->b[s]);
      bmax = std::max(bmax, std::fabs(db));
      for (int j = 0; j < D; ++j) {
        const double dj = D == 1 ? static_cast<double>(c->d_min)
                                 : static_cast<double>(c->d_min) + static_cast<double>(j) * step;
        off[(static_cast<size_t>(si) * K + t) * D + j] = static_cast<int>(std::floor(-dj * db + 0.5));
      }
    }
    a.delta_c[si] = (D >= 2 && step > 0.0 && bmax > 0.0) ? static_cast<int>(std::ceil(1.0 / (bmax * step))) : 0;
  }
  const size_t HWK = static_cast<size_t>(H) * W * K;
  const size_t n_chunks = (static_cast<size_t>(ncell) + 1023) / 1024;
  const size_t n_int =
      off.size() + static_cast<size_t>(a.n_src) * ncell + 5 * static_cast<size_t>(ncell) + 1 + n_chunks;
  lf_status s;
  if ((s = grow(&c->d_sgrad, &c->sgrad_cap, 2 * HWK, "support buffers")) != LF_OK) return s;
  if ((s = grow(&c->d_sint, &c->sint_cap, n_int, "support buffers")) != LF_OK) return s;
  if ((s = grow(&c->d_sdbl, &c->sdbl_cap, 4 * static_cast<size_t>(ncell), "support buffers")) != LF_OK) return s;
  if ((s = grow(&c->d_spts, &c->spts_cap, 3 * static_cast<size_t>(ncell), "support buffers")) != LF_OK) return s;
  a.gx = c->d_sgrad;
  a.gy = c->d_sgrad + HWK;
  int* ip = c->d_sint;
  a.offsets = ip; ip += off.size();
  a.match = ip; ip += static_cast<size_t>(a.n_src) * ncell;
  a.claim = ip; ip += ncell;
  a.pre_j = ip; ip += ncell;
  a.pre_src = ip; ip += ncell;
  a.cell_j = ip; ip += ncell;
  a.cell_src = ip; ip += ncell;
  a.n_points = ip;
  a.chunk_count = ip + 1;
  a.pre_u = c->d_sdbl;
  a.pre_v = c->d_sdbl + ncell;
  a.cell_u = c->d_sdbl + 2 * ncell;
  a.cell_v = c->d_sdbl + 3 * ncell;
  a.points = c->d_spts;
  a.max_points = ncell;
  LF_CUDA(cudaMemcpyAsync(const_cast<int*>(a.offsets), off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice,
                          c->stream),
          "support offsets upload");
  if (!c->sup_ev[0]) {
    LF_CUDA(cudaEventCreate(&c->sup_ev[0]), "event create");
    LF_CUDA(cudaEventCreate(&c->sup_ev[1]), "event create");
  }
  LF_CUDA(cudaEventRecord(c->sup_ev[0], c->stream), "event");
  LF_CUDA(launch_support(a, c->stream), "support-point kernels");
  LF_CUDA(cudaEventRecord(c->sup_ev[1], c->stream), "event");
  int n = 0;
  LF_CUDA(cudaMemcpyAsync(&n, a.n_points, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "support count");
  LF_CUDA(cudaStreamSynchronize(c->stream), "support points");
  LF_CUDA(cudaEventElapsedTime(&c->stats.ms_support, c->sup_ev[0], c->sup_ev[1]), "event time");
  c->support_pts.resize(static_cast<size_t>(3) * n);
  if (n > 0)
    LF_CUDA(cudaMemcpy(c->support_pts.data(), c->d_spts, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost),
            "support points");
  return LF_OK;
}
}  // namespace

extern "C" {

void lf_default_support_params(lf_support_params* q) {
  if (!q) return;
  q->grid = 5;
  q->ratio_pct = 85;
  q->texture = 120;
  q->window = 3;
  q->delta = 3.f;
  q->min_support = 2;
}

lf_status lf_set_support_params(lf_ctx* c, const lf_support_params* q) {
  g_err.clear();
  if (!c) return fail(LF_EINVAL, "ctx is NULL");
  lf_support_params v;
  lf_default_support_params(&v);
  if (q) v = *q;
  if (v.grid < 1 || v.grid > 64 || v.ratio_pct < 1 || v.ratio_pct > 100 || v.texture < 0 || v.window < 0 ||
      v.window > 32 || !(v.delta >= 0.f) || !std::isfinite(v.delta) || v.min_support < 0)
    return fail(LF_EINVAL, "invalid lf_support_params");
  c->sp = v;
  return LF_OK;
}

lf_status lf_get_support_points(const lf_ctx* c, float* points, int max_points, int* n_points) {
  g_err.clear();
  if (!c || !n_points) return fail(LF_EINVAL, "ctx and n_points must not be NULL");
  const int n = static_cast<int>(c->support_pts.size() / 3);
  *n_points = n;
  if (points && max_points > 0)
    std::copy(c->support_pts.begin(), c->support_pts.begin() + 3 * std::min(n, max_points), points);
  return LF_OK;
}

lf_status lf_create(lf_ctx** out, int n_cams, const float* baselines, int H, int W, float d_min, float d_max,
                    int D, const lf_params* p) {
  if (!baselines) {
    g_err.clear();
    if (out) *out = nullptr;
    return fail(LF_EINVAL, "baselines is NULL");
  }
  return create_ctx(out, n_cams, baselines, nullptr, H, W, d_min, d_max, D, p);
}

lf_status lf_create_calibrated(lf_ctx** out, int n_cams, const float* cameras, int H, int W, float d_min,
                               float d_max, int D, const lf_params* p) {
  if (!cameras) {
    g_err.clear();
    if (out) *out = nullptr;
    return fail(LF_EINVAL, "cameras is NULL");
  }
  return create_ctx(out, n_cams, nullptr, cameras, H, W, d_min, d_max, D, p);
}

lf_status lf_set_stream(lf_ctx* c, void* stream) {
  g_err.clear();
  if (!c) return fail(LF_EINVAL, "ctx is NULL");
  c->stream = static_cast<cudaStream_t>(stream);
  return LF_OK;
}

}  // extern "C"

namespace {
lf_status set_inputs_impl(lf_ctx* c, const void* images, int C, int dtype, const float* seg_prior,
                          const float* sparse_points, int M, int on_device);
}  // namespace

extern "C" {

lf_status lf_set_inputs(lf_ctx* c, const void* images, int C, int dtype, const float* seg_prior,
                        const float* sparse_points, int M, int on_device) {
  g_err.clear();
  if (!c) return fail(LF_EINVAL, "ctx is NULL");
  NvtxRange range("lf_set_inputs");
  const auto t0 = std::chrono::steady_clock::now();
  const lf_status st = set_inputs_impl(c, images, C, dtype, seg_prior, sparse_points, M, on_device);
  c->set_inputs_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  ++c->set_inputs_calls;
  return st;
}
}  // extern "C"

namespace {
lf_status set_inputs_impl(lf_ctx* c, const void* images, int C, int dtype, const float* seg_prior,
                          const float* sparse_points, int M, int on_device) {
  if (!images || !seg_prior) return fail(LF_EINVAL, "images and seg_prior must not be NULL");
  if (on_device < 0 || on_device > LF_HOST_ASYNC) return fail(LF_EINVAL, "on_device must be 0, 1 or LF_HOST_ASYNC");
  if (C != 1 && C != 3) return fail(LF_EINVAL, "C must be 1 or 3");
  if (dtype != LF_U8 && dtype != LF_F32 && dtype != LF_F16 && dtype != LF_BF16)
    return fail(LF_EINVAL, "dtype must be LF_U8, LF_F32, LF_F16 or LF_BF16");
  const bool detect = M == LF_DETECT_SUPPORT;
  if (detect && sparse_points) return fail(LF_EINVAL, "M = LF_DETECT_SUPPORT takes sparse_points = NULL");
  if (detect && c->calibrated) return fail(LF_EINVAL, "support-point detection needs a rectified array");
  if ((M < 0 && !detect) || (M > 0 && !sparse_points)) return fail(LF_EINVAL, "bad sparse points");
  for (int i = 0; i < 3 * M; ++i)
    if (!std::isfinite(sparse_points[i])) return fail(LF_EINVAL, "non-finite sparse point");
  c->have_inputs = false;
  c->C = C;
  c->dtype = dtype;
  c->bpp = C * (dtype == LF_U8 ? 1 : dtype == LF_F32 ? 4 : 2);
  lf_status s = copy_plane(c, images, static_cast<size_t>(c->W) * c->bpp, on_device == 1, &c->own_img,
                           &c->own_img_cap, &c->img, &c->img_pitch);
  if (s != LF_OK) return s;
  {
    const uint8_t* pp = nullptr;
    uint8_t* ownP = reinterpret_cast<uint8_t*>(c->own_P);
    s = copy_plane(c, seg_prior, static_cast<size_t>(c->W) * 4, on_device == 1, &ownP, &c->own_P_cap, &pp,
                   &c->p_pitch);
    c->own_P = reinterpret_cast<float*>(ownP);
    if (s != LF_OK) return s;
    c->P = reinterpret_cast<const float*>(pp);
  }
  if (detect) {  // Sec. III-C: support points from the inputs themselves (before any 16-bit conversion)
    NvtxRange range("support points");
    if ((s = detect_support(c)) != LF_OK) return s;
    sparse_points = c->support_pts.data();
    M = static_cast<int>(c->support_pts.size() / 3);
  }
  s = choose_tiles(c);
  if (s != LF_OK) return s;
  {
    NvtxRange range("prior: Delaunay and bins");
    build_prior(c, sparse_points, M);
  }
  if ((s = grow(&c->d_tris, &c->tris_cap, std::max<size_t>(c->h_tris.size(), 1), "prior")) != LF_OK) return s;
  if ((s = grow(&c->d_bins, &c->bins_cap, c->h_bins.size(), "prior")) != LF_OK) return s;
  if (!c->h_tris.empty())
    LF_CUDA(cudaMemcpyAsync(c->d_tris, c->h_tris.data(), c->h_tris.size() * sizeof(PriorTri),
                            cudaMemcpyHostToDevice, c->stream),
            "prior upload");
  LF_CUDA(cudaMemcpyAsync(c->d_bins, c->h_bins.data(), c->h_bins.size() * sizeof(int), cudaMemcpyHostToDevice,
                          c->stream),
          "prior upload");
  if ((s = encode_maps(c)) != LF_OK) return s;
  if (on_device == 0) LF_CUDA(cudaStreamSynchronize(c->stream), "input copy");
  c->have_inputs = true;
  return LF_OK;
}
}  // namespace

namespace {
// Statistics of a run and, for host outputs, the copies back (the call then
// waits for them).
lf_status finish_run(lf_ctx* c, int iters, int launched, bool dev, bool async_host, size_t HW, int32_t* disparity_idx,
                     float* disparity, uint16_t* labels, float* posteriors, float* refocused, const int32_t* didx,
                     const float* dout, const uint16_t* lab, const float* post, const float* refo) {
  ++c->runs;
  // joint MAP sweeps the candidates once, whatever the iteration count
  c->stats.nominal_ray_samples =
      static_cast<uint64_t>(HW) * c->K * c->D * (c->p.em_mode == LF_EM_JOINT ? 1 : iters);
  c->stats.halo_left = c->L;
  c->stats.halo_right = c->R;
  c->stats.tile_rows = c->calibrated ? 16 : c->TR;
  c->stats.tile_cols = c->calibrated ? 16 : c->TW;
  c->stats.kernels_launched = launched;
  if (dev) return LF_OK;
  const cudaMemcpyKind d2h = cudaMemcpyDeviceToHost;
  LF_CUDA(cudaMemcpyAsync(disparity_idx, didx, HW * 4, cudaMemcpyDeviceToHost, c->stream), "output copy");
  if (disparity) LF_CUDA(cudaMemcpyAsync(disparity, dout, HW * 4, cudaMemcpyDeviceToHost, c->stream), "output copy");
  if (labels) LF_CUDA(cudaMemcpyAsync(labels, lab, HW * 2, cudaMemcpyDeviceToHost, c->stream), "output copy");
  if (posteriors)
    LF_CUDA(cudaMemcpyAsync(posteriors, post, HW * 4 * c->K, cudaMemcpyDeviceToHost, c->stream), "output copy");
  if (refocused) LF_CUDA(cudaMemcpyAsync(refocused, refo, HW * 4 * c->C, d2h, c->stream), "output copy");
  if (async_host) return LF_OK;  // LF_HOST_ASYNC: lf_synchronize waits for the copies
  return lf_synchronize(c);
}
}  // namespace

extern "C" {

lf_status lf_run_em(lf_ctx* c, int iters, int32_t* disparity_idx, float* disparity, float* posteriors,
                    uint16_t* labels, float* refocused, int outputs_on_device) {
  g_err.clear();
  if (!c) return fail(LF_EINVAL, "ctx is NULL");
  NvtxRange range("lf_run_em");
  if (!c->have_inputs) return fail(LF_ESTATE, "lf_run_em called before lf_set_inputs");
  if (iters < 1 || iters > 255) return fail(LF_EINVAL, "iters must be in [1, 255]");
  if (!disparity_idx) return fail(LF_EINVAL, "disparity_idx must not be NULL");
  const size_t HW = static_cast<size_t>(c->H) * c->W;
  if (outputs_on_device < 0 || outputs_on_device > LF_HOST_ASYNC)
    return fail(LF_EINVAL, "outputs_on_device must be 0, 1 or LF_HOST_ASYNC");
  const bool dev = outputs_on_device == 1, async_host = outputs_on_device == LF_HOST_ASYNC;
  int32_t* didx = disparity_idx;
  float* dout = disparity;
  uint16_t* lab = labels;
  float* post = posteriors;
  float* refo = refocused;
  lf_status s;
  if (!dev) {
    if ((s = grow(&c->o_didx, &c->o_didx_cap, HW, "outputs")) != LF_OK) return s;
    didx = c->o_didx;
    if (disparity) {
      if ((s = grow(&c->o_d, &c->o_d_cap, HW, "outputs")) != LF_OK) return s;
      dout = c->o_d;
    }
    if (posteriors) {
      if ((s = grow(&c->o_post, &c->o_post_cap, HW * c->K, "outputs")) != LF_OK) return s;
      post = c->o_post;
    }
    if (refocused) {
      if ((s = grow(&c->o_ref, &c->o_ref_cap, HW * c->C, "outputs")) != LF_OK) return s;
      refo = c->o_ref;
    }
  }
  // the refocus needs the labels even when the caller does not want them
  if (!lab || !dev) {
    if ((s = grow(&c->o_labels, &c->o_labels_cap, HW, "outputs")) != LF_OK) return s;
    lab = c->o_labels;
  }
  float* refo_stage = refo;
  if (refo && c->p.median) {
    if ((s = grow(&c->o_tmp, &c->o_tmp_cap, HW * c->C, "outputs")) != LF_OK) return s;
    refo_stage = c->o_tmp;
  }
  int launched = 0;
  lf_ctx::RunEvents* re = nullptr;
  if (c->timing) {
    if (c->events_used == c->events.size()) {
      lf_ctx::RunEvents fresh{};
      for (cudaEvent_t& e : fresh.ev) LF_CUDA(cudaEventCreate(&e), "event create");
      c->events.push_back(fresh);
    }
    re = &c->events[c->events_used++];
    for (bool& u : re->used) u = false;
  }
  auto mark = [&](int i) -> cudaError_t {
    if (!re) return cudaSuccess;
    re->used[i] = true;
    return cudaEventRecord(re->ev[i], c->stream);
  };
  LF_CUDA(mark(0), "event");
  // The hard EM on a rectified array fuses the prior raster and the refocus
  // into its kernels: the sweep computes its pixels' prior centres while its
  // staging copies are in flight and writes Eq. 2 from the rows it staged (in
  // dynamic-only mode the tile classifier rasterises the prior).  The other
  // paths run prior, sweep and refocus kernels in order.
  const bool fused = !c->calibrated && c->p.em_mode == LF_EM_HARD;
  PriorArgs pa{c->H, c->W, c->nbx, c->nby, c->d_tris, c->d_bins, c->d_bins + (c->nbx * c->nby + 1), c->d_mu};
  if (!fused) {
    LF_CUDA(launch_prior_raster(pa, c->stream), "prior_raster launch");
    ++launched;
  }
  LF_CUDA(mark(1), "event");
  if (c->calibrated) {  // Eq. 1 with per-camera homographies: maps in HBM, gathered by the sweep
    const size_t KHW = HW * c->K + c->W + 1;  // + one zero row (and texel) past the end
    if ((s = grow(&c->d_fa, &c->fa_cap, KHW, "descriptor maps")) != LF_OK) return s;
    if ((s = grow(&c->d_fb, &c->fb_cap, KHW, "descriptor maps")) != LF_OK) return s;
    CalibArgs g{};
    g.K = c->K; g.H = c->H; g.W = c->W; g.C = c->C; g.D = c->D; g.ref = c->ref; g.dtype = c->dtype;
    g.iters = iters; g.early_exit = c->p.early_exit; g.mseg = c->p.mstep_seg_term;
    g.dyn_only = c->p.dynamic_only != 0;
    g.seg_threshold = c->p.seg_threshold; g.beta = c->p.beta; g.gamma = c->p.gamma;
    g.inv2s2 = static_cast<float>(1.0 / (2.0 * static_cast<double>(c->p.sigma) * c->p.sigma));
    g.log_thr = static_cast<float>(std::log(static_cast<double>(c->p.seg_threshold) / (1.0 - c->p.seg_threshold)));
    g.eps = c->p.eps;
    for (int k = 0; k < c->K; ++k)
      for (int i = 0; i < 12; ++i) g.cam[k][i] = c->cams[12 * k + i];
    g.img = c->img; g.img_pitch = c->img_pitch; g.P = c->P; g.p_pitch = c->p_pitch;
    g.fa = c->d_fa; g.fb = c->d_fb; g.dval = c->d_dval; g.mu = c->d_mu;
    g.d_idx = didx; g.d_out = dout; g.labels = lab; g.post = post; g.refocus = refo_stage;
    g.counter = c->d_counter;
    g.sweeps = c->d_counter + 2;
    set_pruning(g, c->p.prune, c->K, c->dval.data(), c->D, c->p.eps);
    LF_CUDA(launch_calib_features(g, c->stream), "calibrated features launch");
    LF_CUDA(launch_calib_sweep(g, c->stream), "calibrated sweep launch");
    launched += 2;
    LF_CUDA(mark(2), "event");
    if (refo) {
      LF_CUDA(launch_calib_refocus(g, c->stream), "calibrated refocus launch");
      ++launched;
      LF_CUDA(mark(3), "event");
      if (c->p.median) {
        LF_CUDA(launch_median3(refo_stage, refo, c->H, c->W, c->C, c->stream), "median launch");
        ++launched;
        LF_CUDA(mark(4), "event");
      }
    }
    return finish_run(c, iters, launched, dev, async_host, HW, disparity_idx, disparity, labels, posteriors, refocused,
                      didx, dout, lab, post, refo);
  }
  SweepArgs a{};
  a.H = c->H; a.W = c->W; a.C = c->C; a.D = c->D; a.ref = c->ref; a.dtype = c->dtype; a.bpp = c->bpp;
  a.TR = c->TR; a.TW = c->TW; a.L = c->L; a.R = c->R; a.SW = c->SW; a.SWp = c->SWp; a.RW = c->RW; a.KP = c->KP;
  a.iters = iters;
  a.early_exit = c->p.early_exit;
  a.mseg = c->p.mstep_seg_term;
  a.prec = c->p.precision;
  a.dyn_only = c->p.dynamic_only != 0;
  a.seg_threshold = c->p.seg_threshold;
  a.beta = c->p.beta;
  a.gamma = c->p.gamma;
  a.inv2s2 = static_cast<float>(1.0 / (2.0 * static_cast<double>(c->p.sigma) * c->p.sigma));
  a.log_thr = static_cast<float>(std::log(static_cast<double>(c->p.seg_threshold) / (1.0 - c->p.seg_threshold)));
  a.eps = c->p.eps;
  a.wtab = c->d_wtab; a.otab = c->d_otab; a.chg = c->d_chg; a.dval = c->d_dval; a.mu = c->d_mu;
  for (int k = 0; k < kMaxCams; ++k) {
    a.omin[k] = 0;
    a.omax[k] = 0;
  }
  for (int k = 0; k < c->K; ++k) {
    int lo = c->otab[k], hi = c->otab[k];
    for (int j = 0; j < c->D; ++j) {
      lo = std::min(lo, c->otab[j * c->KP + k]);
      hi = std::max(hi, c->otab[j * c->KP + k]);
    }
    a.omin[k] = lo;
    a.omax[k] = hi;
  }
  a.d_idx = didx; a.d_out = dout; a.labels = lab; a.post = post;
  a.counter = c->d_counter; a.static_counter = c->d_counter + 1; a.sweeps = c->d_counter + 2;
  a.status = c->d_status; a.timeout_ns = kTimeoutNs;
  set_pruning(a, c->p.prune, c->K, c->dval.data(), c->D, c->p.eps);
  if (fused) {
    a.refocus_out = refo_stage;
    a.img = c->img;
    a.img_pitch = c->img_pitch;
    if (!c->p.dynamic_only) {  // (in dynamic-only mode the classifier has written mu by then)
      a.ptris = pa.tris;
      a.pbin_start = pa.bin_start;
      a.pbin_items = pa.bin_items;
      a.pnbx = pa.nbx;
      a.mu_out = c->d_mu;
    }
  }
  if (a.dyn_only) {  // Sec. III-F: sweep only the tiles with dynamic reference pixels
    const int tiles = ((c->W + c->TW - 1) / c->TW) * ((c->H + c->TR - 1) / c->TR);
    if ((s = grow(&c->d_tiles, &c->tiles_cap, static_cast<size_t>(tiles) + 1, "tile list")) != LF_OK) return s;
    LF_CUDA(cudaMemsetAsync(c->d_tiles + tiles, 0, sizeof(int), c->stream), "memset");
    SweepArgs ca = a;  // the classifier also rasterises the prior when the refocus is fused
    if (fused) {
      ca.ptris = pa.tris;
      ca.pbin_start = pa.bin_start;
      ca.pbin_items = pa.bin_items;
      ca.pnbx = pa.nbx;
      ca.mu_out = c->d_mu;
    }
    LF_CUDA(launch_tile_classify(c->K, ca, c->P, c->p_pitch, c->d_tiles, c->d_tiles + tiles, c->stream),
            "tile_classify launch");
    ++launched;
    a.tile_list = c->d_tiles;
    a.n_tiles = c->d_tiles + tiles;
  }
  if (c->p.em_mode == LF_EM_HARD)
    LF_CUDA(launch_em_sweep(c->K, c->img_map, c->p_map, a, c->stream), "em_sweep launch");
  else
    LF_CUDA(launch_em_variant(c->K, c->p.em_mode, c->img_map, c->p_map, a, c->stream), "em_variant launch");
  ++launched;
  LF_CUDA(mark(2), "event");
  if (refo) {
    if (!fused) {
      RefocusArgs r{c->H, c->W, c->C, c->K, c->ref, c->dtype, c->KP, c->img_pitch, c->img, c->d_wtab, c->d_otab,
                    didx, lab, refo_stage};
      LF_CUDA(launch_refocus(r, c->stream), "refocus launch");
      ++launched;
    }
    LF_CUDA(mark(3), "event");
    if (c->p.median) {
      LF_CUDA(launch_median3(refo_stage, refo, c->H, c->W, c->C, c->stream), "median launch");
      ++launched;
      LF_CUDA(mark(4), "event");
    }
  }
  return finish_run(c, iters, launched, dev, async_host, HW, disparity_idx, disparity, labels, posteriors, refocused, didx, dout,
                    lab, post, refo);
}

void lf_inject_alloc_failure(int after) { g_fail_after.store(after < 0 ? -1 : after); }

lf_status lf_host_alloc(void** out, size_t bytes) {
  g_err.clear();
  if (!out) return fail(LF_EINVAL, "out is NULL");
  *out = nullptr;
  if (bytes == 0) return fail(LF_EINVAL, "bytes must be > 0");
  cudaError_t e = cudaMallocHost(out, bytes);
  if (e != cudaSuccess) {
    *out = nullptr;
    return e == cudaErrorMemoryAllocation ? fail(LF_ENOMEM, "page-locked host allocation failed")
                                          : cuda_fail(e, "cudaMallocHost");
  }
  return LF_OK;
}

void lf_host_free(void* p) {
  if (p) cudaFreeHost(p);
}

lf_status lf_synchronize(lf_ctx* c) {
  g_err.clear();
  if (!c) return fail(LF_EINVAL, "ctx is NULL");
  LF_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
  unsigned st = 0;
  LF_CUDA(cudaMemcpy(&st, c->d_status, sizeof(st), cudaMemcpyDeviceToHost), "status read");
  if (st) LF_CUDA(cudaMemset(c->d_status, 0, sizeof(st)), "status reset");
  if (st & kStatusTmaTimeout) return fail(LF_ETIMEOUT, "a bounded TMA wait in the sweep kernel expired");
  if (st & kStatusSmemMisaligned) return fail(LF_ECUDA, "sweep kernel: dynamic shared memory not 128-byte aligned");
  if (st & kStatusBoundsViolation)
    return fail(LF_ECUDA, "sweep kernel (debug build): a shared-memory index left its region");
  return LF_OK;
}

lf_status lf_get_prior(lf_ctx* c, float* mu, int on_device) {
  g_err.clear();
  if (!c || !mu) return fail(LF_EINVAL, "NULL argument");
  const size_t bytes = static_cast<size_t>(c->H) * c->W * 4;
  LF_CUDA(cudaMemcpyAsync(mu, c->d_mu, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          c->stream),
          "prior copy");
  if (!on_device) LF_CUDA(cudaStreamSynchronize(c->stream), "prior copy");
  return LF_OK;
}

lf_status lf_set_tile(lf_ctx* c, int tile_rows, int tile_cols) {
  g_err.clear();
  if (!c) return fail(LF_EINVAL, "ctx is NULL");
  if (tile_rows == 0 && tile_cols == 0) {
    c->force_TR = c->force_TW = 0;
  } else {
    if (tile_rows < 1 || tile_cols < 32 || tile_cols % 32 != 0 || tile_rows * tile_cols > sweep_max_threads(c->K))
      return fail(LF_EINVAL, c->K <= 8 ? "tile: columns a multiple of 32, rows * columns <= 256"
                                       : "tile: columns a multiple of 32, rows * columns <= 128 from nine cameras");
    c->force_TR = tile_rows;
    c->force_TW = tile_cols;
  }
  if (!c->have_inputs) return LF_OK;
  lf_status s = choose_tiles(c);
  if (s != LF_OK) {
    c->have_inputs = false;
    return s;
  }
  return encode_maps(c);
}

lf_status lf_selftest_bounded_wait(unsigned long long timeout_ns) {
  g_err.clear();
  if (timeout_ns == 0 || timeout_ns > 10000000000ull) return fail(LF_EINVAL, "timeout_ns must be in (0, 1e10]");
  unsigned* d_status = nullptr;
  cudaStream_t s = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&d_status), sizeof(unsigned));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) {
    bounded_wait_selftest_kernel<<<1, 64, 0, s>>>(d_status, 1024u, timeout_ns);
    e = cudaGetLastError();
  }
  unsigned st = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (s) cudaStreamDestroy(s);
  if (d_status) cudaFree(d_status);
  if (e != cudaSuccess) return fail(LF_ECUDA, std::string("bounded-wait self-test: ") + cudaGetErrorString(e));
  if (st & kStatusTmaTimeout) return fail(LF_ETIMEOUT, "bounded-wait self-test: the wait expired and was reported");
  return LF_OK;
}

lf_status lf_set_timing(lf_ctx* c, int enable) {
  g_err.clear();
  if (!c) return fail(LF_EINVAL, "ctx is NULL");
  c->timing = enable != 0;
  return LF_OK;
}

lf_status lf_get_stats(lf_ctx* c, lf_stats* out) {
  g_err.clear();
  if (!c || !out) return fail(LF_EINVAL, "NULL argument");
  LF_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
  unsigned long long n[3] = {0, 0, 0};
  LF_CUDA(cudaMemcpy(n, c->d_counter, sizeof(n), cudaMemcpyDeviceToHost), "counter read");
  LF_CUDA(cudaMemset(c->d_counter, 0, sizeof(n)), "counter reset");
  c->stats.runs = c->runs;
  c->stats.executed_ray_samples = static_cast<uint64_t>(n[0]) * c->K;
  c->stats.executed_static_ray_samples = static_cast<uint64_t>(n[1]);
  c->stats.executed_pixel_iterations = static_cast<uint64_t>(n[2]);
  float* ms[4] = {&c->stats.ms_prior, &c->stats.ms_sweep, &c->stats.ms_refocus, &c->stats.ms_median};
  for (int i = 0; i < 4; ++i) {
    double acc = 0.0;
    for (size_t r = 0; r < c->events_used; ++r) {
      const lf_ctx::RunEvents& e = c->events[r];
      if (!e.used[i] || !e.used[i + 1]) continue;
      float t = 0.f;
      LF_CUDA(cudaEventElapsedTime(&t, e.ev[i], e.ev[i + 1]), "event time");
      acc += t;
    }
    *ms[i] = c->events_used ? static_cast<float>(acc / c->events_used) : 0.f;
  }
  c->stats.ms_set_inputs = c->set_inputs_calls ? static_cast<float>(c->set_inputs_ms / c->set_inputs_calls) : 0.f;
  *out = c->stats;
  c->events_used = 0;
  c->runs = 0;
  c->set_inputs_ms = 0.0;
  c->set_inputs_calls = 0;
  return LF_OK;
}

void lf_destroy(lf_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  void* bufs[] = {c->d_wtab, c->d_otab, c->d_chg, c->d_dval, c->d_mu, c->d_counter, c->d_status,
                  c->own_img, c->own_P, c->d_tiles, c->d_tris, c->d_bins, c->o_didx, c->o_d, c->o_labels,
                  c->o_post, c->o_ref, c->o_tmp, c->d_fa, c->d_fb, c->d_sgrad, c->d_sint, c->d_sdbl,
                  c->d_spts};
  for (void* p : bufs)
    if (p) cudaFree(p);
  for (cudaEvent_t e : c->sup_ev)
    if (e) cudaEventDestroy(e);
  for (auto& re : c->events)
    for (cudaEvent_t e : re.ev)
      if (e) cudaEventDestroy(e);
  delete c;
}

}  // extern "C"

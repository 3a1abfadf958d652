// Uneven batches (C ABI lf_batch_*): frames of different sizes, camera
// counts, candidate counts and iteration counts run together.
//
// Per lf_batch_run the host prepares every frame in parallel threads (sampling
// tables, Delaunay triangulation and bins of the prior, tile shape) and
// uploads them into one device arena.  The device work is then one CUDA graph:
//   batched prior raster over (frame, row) items,
//   one persistent sweep launch per camera count present, each CTA pulling
//   (frame, tile) items of that camera count from a device-side queue,
//   batched refocus (and median) over (frame, row) items.
// (Fusing the prior and refocus into the persistent sweep, as the
// single-frame path does, measured slower on the uneven batch.)
// All kernels read their work lists and counts from device memory, so the
// captured graph stays valid while the batch contents change; it is captured
// again only when its shape changes (camera counts present, shared-memory
// sizes, precision, median flag, or a descriptor array had to grow).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "lf.h"
#include "lf_internal.h"

using namespace lf;

namespace {

lf_status fail(lf_status s, const std::string& m) {
  set_error_message(m);
  return s;
}

lf_status cuda_fail(cudaError_t e, const char* what) {
  return fail(LF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LF_CUDA(call, what)                            \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
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

bool encode(CUtensorMap* m, const void* base, size_t pitch, int W, int H, int K, size_t bpp, int box_px,
            int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>((static_cast<size_t>(W) * bpp + 7) / 8),
                              static_cast<cuuint64_t>(H), static_cast<cuuint64_t>(K)};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(pitch), static_cast<cuuint64_t>(pitch * H)};
  const cuuint32_t box[3] = {static_cast<cuuint32_t>(box_px * bpp / 8), static_cast<cuuint32_t>(box_rows),
                             static_cast<cuuint32_t>(K)};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Tile shapes of the persistent sweep: 256-thread shapes first (the ones the
// autotuner times), then 128- and 64-thread shapes for halos too wide for the
// larger tiles' shared memory.  One launch per (camera count, threads).
const int kTiles[][2] = {{2, 128}, {4, 64}, {1, 256}, {8, 32}, {1, 128}, {2, 64}, {4, 32}, {1, 64}, {2, 32}};
constexpr int kNumTiles = 9;
constexpr int kNumTuned = 4;  // shapes the autotuner times
constexpr int kThreadClasses = 3;
int thread_class(int tile) { return kTiles[tile][0] * kTiles[tile][1] == 256 ? 0 : kTiles[tile][0] * kTiles[tile][1] == 128 ? 1 : 2; }
constexpr int kThreadsOf[kThreadClasses] = {256, 128, 64};
constexpr int kGroups = kMaxCams * kThreadClasses;  // launch groups
int group_of(int K, int tile) { return (K - 1) * kThreadClasses + thread_class(tile); }

// Autotuner cache: frame signature -> index into kTiles (process wide).
// Signature: K, D, bytes per pixel, precision, halo in 8-px classes, width
// in 256-px classes.
typedef std::tuple<int, int, int, int, int, int> TileKey;
std::mutex g_tune_mutex;
std::map<TileKey, int> g_tune_cache;

struct Frame {
  // geometry and run
  int K = 0, H = 0, W = 0, D = 0, iters = 0, C = 0, dtype = 0, ref = 0, KP = 4, L = 0, R = 0;
  float d_min = 0.f, d_max = 0.f;
  std::vector<float> b, pts;
  // caller buffers
  const void* src_img = nullptr;
  const float* src_p = nullptr;
  int32_t* d_idx = nullptr;
  float* d_out = nullptr;
  float* post = nullptr;
  uint16_t* labels = nullptr;
  float* refocus = nullptr;
  // host-built per run
  std::vector<float> wtab, dval;
  std::vector<int> otab;
  std::vector<unsigned> chg;
  int omin[kMaxCams] = {0}, omax[kMaxCams] = {0};
  std::vector<PriorTri> tris;
  std::vector<int> bins;
  int nbx = 0, nby = 0;
  // staging decisions
  int bpp = 0, stage_dtype = 0;
  bool stage_img = false, stage_p = false;
  size_t img_pitch = 0, p_pitch = 0;
  // tile
  int tile = 0;
  bool untuned = false;
  TileKey key{};
  SweepArgs args{};
  size_t smem = 0;
  // arena offsets
  size_t o_w = 0, o_o = 0, o_chg = 0, o_dval = 0, o_tris = 0, o_bins = 0, o_mu = 0, o_img = 0, o_img32 = 0,
         o_p = 0, o_lab = 0, o_tmp = 0;
};

}  // namespace

struct lf_batch {
  lf_params p{};
  int autotune = 0;
  int device = 0, num_sms = 0, smem_optin = 0;
  cudaStream_t stream = nullptr, capture = nullptr;
  std::vector<Frame> frames;
  // device memory: one arena for variable-size per-frame data and
  // fixed-address descriptor arrays the graph refers to
  uint8_t* arena = nullptr;
  size_t arena_cap = 0;
  FrameDesc* d_frames = nullptr;
  PriorArgs* d_prior = nullptr;
  RefocusArgs* d_refocus = nullptr;
  MedianArgs* d_median = nullptr;
  size_t frames_cap = 0;
  TileItem* d_items = nullptr;
  size_t items_cap = 0;
  RowItem* d_rows = nullptr;
  size_t rows_cap = 0;
  int* d_counts = nullptr;  // [kGroups] items per launch group, [1] rows, [kGroups] first item
  unsigned long long* d_fcount = nullptr;  // per frame: (pixel, candidate) objectives evaluated
  unsigned* d_heads = nullptr;
  unsigned long long* d_counter = nullptr;
  unsigned* d_status = nullptr;
  // graph
  cudaGraphExec_t exec = nullptr;
  std::vector<long long> key;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // the persistent sweeps of different launch groups are captured as parallel
  // branches (so that one group's tail overlaps the others): branch streams
  // and the fork / join events between them
  static constexpr int kBranches = 4;
  cudaStream_t branch[kBranches] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kBranches] = {nullptr, nullptr, nullptr, nullptr};
  bool ran = false;
  uint64_t runs = 0, nominal = 0;
  int graph_captures = 0;
  int tuned = 0;
  size_t grp_smem[kGroups] = {0};  // shared memory of every group launched so far (only grows)
  bool grp_generic[kGroups] = {};  // a group has held a frame whose reference is not camera K / 2
};

namespace {

lf_status dev_grow(void** p, size_t* cap, size_t need, bool* moved = nullptr) {
  if (*p && need <= *cap) return LF_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  const size_t n = std::max<size_t>(need + need / 4, 256);
  if (injected_alloc_failure()) return fail(LF_ENOMEM, "batch: out of device memory (injected)");
  cudaError_t e = cudaMalloc(p, n);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? fail(LF_ENOMEM, "batch: out of device memory")
                                          : cuda_fail(e, "batch allocation");
  }
  *cap = n;
  if (moved) *moved = true;
  return LF_OK;
}

void choose_tile(Frame& f, const lf_params& p, int smem_optin);

// Host part of one frame: tables, prior triangles and bins, tile shape.
void prepare_frame(Frame& f, const lf_params& p, int smem_optin) {
  f.KP = (f.K + 3) / 4 * 4;
  f.wtab.assign(static_cast<size_t>(f.D) * f.KP, 0.f);
  f.otab.assign(static_cast<size_t>(f.D) * f.KP, 0);
  f.chg.assign(static_cast<size_t>(f.D), 0u);
  f.dval.assign(static_cast<size_t>(f.D), 0.f);
  int omin = 0, omax = 0;
  for (int k = 0; k < kMaxCams; ++k) f.omin[k] = f.omax[k] = 0;
  for (int j = 0; j < f.D; ++j) {
    const double dj = f.D == 1 ? static_cast<double>(f.d_min)
                               : static_cast<double>(f.d_min) +
                                     j * ((static_cast<double>(f.d_max) - static_cast<double>(f.d_min)) / (f.D - 1));
    f.dval[j] = static_cast<float>(dj);
    unsigned m = 0;
    for (int k = 0; k < f.K; ++k) {
      const double x = -dj * static_cast<double>(f.b[k]);
      const double o = std::floor(x);
      const int oi = static_cast<int>(o);
      f.otab[j * f.KP + k] = oi;
      f.wtab[j * f.KP + k] = static_cast<float>(x - o);
      if (j == 0 || f.otab[(j - 1) * f.KP + k] != oi) m |= 1u << k;
      if (j == 0 || oi < f.omin[k]) f.omin[k] = oi;
      if (j == 0 || oi > f.omax[k]) f.omax[k] = oi;
      omin = std::min(omin, oi);
      omax = std::max(omax, oi + 1);
    }
    f.chg[j] = m;
  }
  f.L = -omin;
  f.R = omax;
  // prior: Delaunay + plane coefficients + 16x16 bins
  const int M = static_cast<int>(f.pts.size() / 3);
  std::vector<double> xy(static_cast<size_t>(2) * M);
  for (int i = 0; i < M; ++i) {
    xy[2 * i] = f.pts[3 * i];
    xy[2 * i + 1] = f.pts[3 * i + 1];
  }
  std::vector<int> tri(static_cast<size_t>(6) * std::max(M, 1) + 6);
  int nt = M >= 3 ? delaunay(xy.data(), M, tri.data(), static_cast<int>(tri.size() / 3)) : 0;
  f.tris.clear();
  for (int t = 0; t < nt; ++t) {
    const int ia = tri[3 * t], ib = tri[3 * t + 1], ic = tri[3 * t + 2];
    PriorTri T;
    T.ua = f.pts[3 * ia]; T.va = f.pts[3 * ia + 1];
    T.ub = f.pts[3 * ib]; T.vb = f.pts[3 * ib + 1];
    T.uc = f.pts[3 * ic]; T.vc = f.pts[3 * ic + 1];
    const double da = f.pts[3 * ia + 2], db = f.pts[3 * ib + 2], dc = f.pts[3 * ic + 2];
    const double du1 = static_cast<double>(T.ub) - T.ua, dv1 = static_cast<double>(T.vb) - T.va;
    const double du2 = static_cast<double>(T.uc) - T.ua, dv2 = static_cast<double>(T.vc) - T.va;
    const double det = du1 * dv2 - du2 * dv1;
    if (det == 0.0) continue;
    split_double(da, T.da_hi, T.da_lo);
    split_double(((db - da) * dv2 - (dc - da) * dv1) / det, T.gu_hi, T.gu_lo);
    split_double((du1 * (dc - da) - du2 * (db - da)) / det, T.gv_hi, T.gv_lo);
    f.tris.push_back(T);
  }
  f.nbx = (f.W + kBinSize - 1) / kBinSize;
  f.nby = (f.H + kBinSize - 1) / kBinSize;
  const int nb = f.nbx * f.nby;
  std::vector<int> count(static_cast<size_t>(nb) + 1, 0);
  auto bbox = [&](const PriorTri& T, int& bx0, int& bx1, int& by0, int& by1) {
    const double u0 = std::max(std::ceil(static_cast<double>(std::min({T.ua, T.ub, T.uc}))), 0.0);
    const double u1 = std::min(std::floor(static_cast<double>(std::max({T.ua, T.ub, T.uc}))),
                               static_cast<double>(f.W - 1));
    const double v0 = std::max(std::ceil(static_cast<double>(std::min({T.va, T.vb, T.vc}))), 0.0);
    const double v1 = std::min(std::floor(static_cast<double>(std::max({T.va, T.vb, T.vc}))),
                               static_cast<double>(f.H - 1));
    if (u1 < u0 || v1 < v0) return false;
    bx0 = static_cast<int>(u0) / kBinSize; bx1 = static_cast<int>(u1) / kBinSize;
    by0 = static_cast<int>(v0) / kBinSize; by1 = static_cast<int>(v1) / kBinSize;
    return true;
  };
  for (const PriorTri& T : f.tris) {
    int bx0, bx1, by0, by1;
    if (!bbox(T, bx0, bx1, by0, by1)) continue;
    for (int by = by0; by <= by1; ++by)
      for (int bx = bx0; bx <= bx1; ++bx) count[by * f.nbx + bx + 1]++;
  }
  for (int i = 0; i < nb; ++i) count[i + 1] += count[i];
  f.bins.assign(static_cast<size_t>(nb) + 1 + count[nb], 0);
  std::copy(count.begin(), count.end(), f.bins.begin());
  std::vector<int> fill(count.begin(), count.end() - 1);
  for (size_t t = 0; t < f.tris.size(); ++t) {
    int bx0, bx1, by0, by1;
    if (!bbox(f.tris[t], bx0, bx1, by0, by1)) continue;
    for (int by = by0; by <= by1; ++by)
      for (int bx = bx0; bx <= bx1; ++bx) f.bins[nb + 1 + fill[by * f.nbx + bx]++] = static_cast<int>(t);
  }
  // input staging: TMA reads rows in place when they are 16-byte aligned
  const int in_bpp = f.C * (f.dtype == LF_U8 ? 1 : f.dtype == LF_F32 ? 4 : 2);
  // (the precision mode sets the storage of the staged maps; the images stay as given)
  f.stage_dtype = f.dtype;
  f.bpp = in_bpp;
  const size_t in_row = static_cast<size_t>(f.W) * in_bpp;
  f.stage_img = in_row % 16 != 0 || reinterpret_cast<uintptr_t>(f.src_img) % 16 != 0;
  f.img_pitch = f.stage_img ? align_up(static_cast<size_t>(f.W) * f.bpp, 16) : in_row;
  f.stage_p = (static_cast<size_t>(f.W) * 4) % 16 != 0 || reinterpret_cast<uintptr_t>(f.src_p) % 16 != 0;
  f.p_pitch = f.stage_p ? align_up(static_cast<size_t>(f.W) * 4, 16) : static_cast<size_t>(f.W) * 4;
  choose_tile(f, p, smem_optin);
}

// Tile: the tuned shape of the frame's signature if there is one, else the
// first shape that fits one TMA box per staged row and allows two CTAs per SM.
void choose_tile(Frame& f, const lf_params& p, int smem_optin) {
  SweepArgs a{};
  a.D = f.D;
  a.KP = f.KP;
  a.bpp = f.bpp;
  a.prec = p.precision;
  f.key = TileKey{f.K, f.D, f.bpp, p.precision, (f.L + f.R + 7) / 8, (f.W + 255) / 256};
  int tuned = -1;
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    auto it = g_tune_cache.find(f.key);
    if (it != g_tune_cache.end()) tuned = it->second;
  }
  f.untuned = tuned < 0;
  f.tile = -1;
  for (int pass = 0; pass < 3 && f.tile < 0; ++pass) {
    for (int t = 0; t < kNumTiles; ++t) {
      if (pass == 0 && t != tuned) continue;
      if (pass == 1 && t >= kNumTuned) continue;  // prefer 256-thread shapes with two CTAs per SM
      a.TR = kTiles[t][0];
      a.TW = kTiles[t][1];
      a.L = f.L;
      a.R = f.R;
      a.SW = a.TW + f.L + f.R;
      a.SWp = (a.SW + 31) / 32 * 32;
      a.RW = (a.SW + 17 + 15) / 16 * 16;
      if (a.RW * a.bpp / 8 > 256 || a.RW / 2 > 256) continue;
      const size_t sm = sweep_smem_bytes(f.K, a);
      if (sm > static_cast<size_t>(pass <= 1 ? std::min(smem_optin, 110 * 1024) : smem_optin)) continue;
      f.tile = t;
      f.smem = sm;
      break;
    }
  }
  f.args = a;
}

// Time every candidate tile shape of frame f through the single-frame path
// (same kernel arithmetic, one CTA per tile) and return the fastest, or -1.
int tune_frame(const Frame& f, const lf_params& p, cudaStream_t stream) {
  lf_ctx* c = nullptr;
  if (lf_create(&c, f.K, f.b.data(), f.H, f.W, f.d_min, f.d_max, f.D, &p) != LF_OK) return -1;
  lf_set_stream(c, stream);
  lf_set_timing(c, 1);
  int best = -1;
  float best_ms = 0.f;
  const int M = static_cast<int>(f.pts.size() / 3);
  if (lf_set_inputs(c, f.src_img, f.C, f.dtype, f.src_p, f.pts.data(), M, 1) == LF_OK) {
    for (int t = 0; t < kNumTuned; ++t) {
      if (lf_set_tile(c, kTiles[t][0], kTiles[t][1]) != LF_OK) continue;
      lf_stats st{};
      if (lf_run_em(c, f.iters, f.d_idx, nullptr, nullptr, nullptr, nullptr, 1) != LF_OK) break;
      lf_get_stats(c, &st);  // warm-up run; resets the counters
      bool ok = true;
      for (int r = 0; r < 2 && ok; ++r)
        ok = lf_run_em(c, f.iters, f.d_idx, nullptr, nullptr, nullptr, nullptr, 1) == LF_OK;
      if (!ok || lf_get_stats(c, &st) != LF_OK) break;
      if (best < 0 || st.ms_sweep < best_ms) {
        best = t;
        best_ms = st.ms_sweep;
      }
    }
  }
  lf_destroy(c);
  return best;
}

std::string sig_string(const Frame& f) {
  return std::to_string(f.K) + "x" + std::to_string(f.W) + "x" + std::to_string(f.H) + " D=" + std::to_string(f.D);
}

}  // namespace

extern "C" {

lf_status lf_batch_create(lf_batch** out, const lf_params* p, int autotune) {
  set_error_message("");
  if (!out) return fail(LF_EINVAL, "out is NULL");
  *out = nullptr;
  lf_params prm;
  lf_default_params(&prm);
  if (p) prm = *p;
  if (!std::isfinite(prm.beta) || !std::isfinite(prm.gamma) || !std::isfinite(prm.sigma) ||
      !std::isfinite(prm.seg_threshold) || !std::isfinite(prm.eps) || prm.sigma <= 0.f || prm.gamma < 0.f ||
      prm.eps <= 0.f || prm.seg_threshold <= 0.f || prm.seg_threshold >= 1.f || prm.beta < 0.f ||
      prm.precision < LF_PREC_F32 || prm.precision > LF_PREC_BF16)
    return fail(LF_EINVAL, "invalid lf_params");
  if (prm.em_mode != LF_EM_HARD) return fail(LF_EINVAL, "batches run the hard EM only (em_mode = LF_EM_HARD)");
  lf_batch* b = new (std::nothrow) lf_batch();
  if (!b) return fail(LF_ENOMEM, "host allocation failed");
  b->p = prm;
  b->autotune = autotune;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&b->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  for (cudaEvent_t& ev : b->ev)
    if (e == cudaSuccess) e = cudaEventCreate(&ev);
  for (int i = 0; i < lf_batch::kBranches; ++i) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->d_counts), sizeof(int) * (2 * kGroups + 1));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->d_heads), sizeof(unsigned) * kGroups);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->d_counter), sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->d_status), sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(unsigned));
  if (e != cudaSuccess) {
    lf_batch_destroy(b);
    return cuda_fail(e, "batch setup");
  }
  *out = b;
  return LF_OK;
}

lf_status lf_batch_set_stream(lf_batch* b, void* stream) {
  set_error_message("");
  if (!b) return fail(LF_EINVAL, "batch is NULL");
  b->stream = static_cast<cudaStream_t>(stream);
  return LF_OK;
}

lf_status lf_batch_add(lf_batch* b, int n_cams, const float* baselines, int H, int W, float d_min, float d_max,
                       int D, int iters, const void* images, int C, int dtype, const float* seg_prior,
                       const float* sparse_points, int M, int32_t* disparity_idx, float* disparity,
                       float* posteriors, uint16_t* labels, float* refocused, int* index) {
  set_error_message("");
  if (!b) return fail(LF_EINVAL, "batch is NULL");
  if (n_cams < 1 || n_cams > kMaxCams) return fail(LF_EINVAL, "n_cams must be in [1, 12]");
  if (!baselines || !images || !seg_prior || !disparity_idx)
    return fail(LF_EINVAL, "baselines, images, seg_prior and disparity_idx must not be NULL");
  if (H < 3 || W < 3) return fail(LF_EINVAL, "H and W must be >= 3");
  if (D < 1 || D > kMaxD) return fail(LF_EINVAL, "D must be in [1, 1024]");
  if (!std::isfinite(d_min) || !std::isfinite(d_max) || d_max < d_min) return fail(LF_EINVAL, "need d_min <= d_max");
  if (iters < 1 || iters > 255) return fail(LF_EINVAL, "iters must be in [1, 255]");
  if (C != 1 && C != 3) return fail(LF_EINVAL, "C must be 1 or 3");
  if (dtype < LF_U8 || dtype > LF_BF16) return fail(LF_EINVAL, "bad dtype");
  if (M < 0 || (M > 0 && !sparse_points)) return fail(LF_EINVAL, "bad sparse points");
  Frame f;
  f.ref = -1;
  for (int k = 0; k < n_cams; ++k) {
    if (!std::isfinite(baselines[k])) return fail(LF_EINVAL, "non-finite baseline");
    if (baselines[k] == 0.f && f.ref < 0) f.ref = k;
  }
  if (f.ref < 0) return fail(LF_EINVAL, "no baseline equals 0 (reference camera)");
  for (int i = 0; i < 3 * M; ++i)
    if (!std::isfinite(sparse_points[i])) return fail(LF_EINVAL, "non-finite sparse point");
  f.K = n_cams;
  f.H = H;
  f.W = W;
  f.D = D;
  f.iters = iters;
  f.C = C;
  f.dtype = dtype;
  f.d_min = d_min;
  f.d_max = d_max;
  f.b.assign(baselines, baselines + n_cams);
  f.pts.assign(sparse_points, sparse_points + 3 * M);
  f.src_img = images;
  f.src_p = seg_prior;
  f.d_idx = disparity_idx;
  f.d_out = disparity;
  f.post = posteriors;
  f.labels = labels;
  f.refocus = refocused;
  if (index) *index = static_cast<int>(b->frames.size());
  b->frames.push_back(std::move(f));
  return LF_OK;
}

lf_status lf_batch_clear(lf_batch* b) {
  set_error_message("");
  if (!b) return fail(LF_EINVAL, "batch is NULL");
  b->frames.clear();
  return LF_OK;
}

lf_status lf_batch_run(lf_batch* b) {
  set_error_message("");
  if (!b) return fail(LF_EINVAL, "batch is NULL");
  const int nf = static_cast<int>(b->frames.size());
  if (nf == 0) return fail(LF_ESTATE, "lf_batch_run on an empty batch");
  NvtxRange range("lf_batch_run");
  // 1. host preparation, frames in parallel
  {
    NvtxRange prep("batch: frame preparation");
    const int nt = std::max(1, std::min<int>(nf, static_cast<int>(std::thread::hardware_concurrency())));
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t)
      pool.emplace_back([b, t, nt, nf] {
        for (int i = t; i < nf; i += nt) prepare_frame(b->frames[i], b->p, b->smem_optin);
      });
    for (auto& th : pool) th.join();
  }
  if (b->autotune) {  // time the candidate tiles of signatures not seen before
    std::map<TileKey, int> done;
    for (Frame& f : b->frames) {
      // from nine cameras the single-frame kernel the tuner times takes no
      // 256-thread shapes: those frames keep the first shape that fits
      if (!f.untuned || kTiles[0][0] * kTiles[0][1] > sweep_max_threads(f.K)) continue;
      auto it = done.find(f.key);
      if (it == done.end()) {
        const int t = tune_frame(f, b->p, b->stream);
        it = done.emplace(f.key, t).first;
        if (t >= 0) {
          std::lock_guard<std::mutex> lk(g_tune_mutex);
          g_tune_cache[f.key] = t;
          ++b->tuned;
        }
      }
      choose_tile(f, b->p, b->smem_optin);
    }
    set_error_message("");
  }
  for (const Frame& f : b->frames)
    if (f.tile < 0) return fail(LF_EINVAL, "frame " + sig_string(f) + ": disparity halo too wide for staging");
  // 2. arena layout
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  size_t total_items = 0, total_rows = 0;
  // host-written region first (uploaded every run), then device-only buffers
  for (Frame& f : b->frames) {
    f.o_w = take(f.wtab.size() * 4);
    f.o_o = take(f.otab.size() * 4);
    f.o_chg = take(f.chg.size() * 4);
    f.o_dval = take(f.dval.size() * 4);
    f.o_tris = take(std::max<size_t>(f.tris.size(), 1) * sizeof(PriorTri));
    f.o_bins = take(f.bins.size() * 4);
  }
  const size_t host_bytes = o;
  for (Frame& f : b->frames) {
    const size_t HW = static_cast<size_t>(f.H) * f.W;
    f.o_mu = take(HW * 4);
    f.o_img = f.stage_img ? take(f.img_pitch * f.H * f.K) : 0;
    f.o_p = f.stage_p ? take(f.p_pitch * f.H * f.K) : 0;
    f.o_lab = f.labels ? 0 : take(HW * 2);
    f.o_tmp = (f.refocus && b->p.median) ? take(HW * f.C * 4) : 0;
    total_items += static_cast<size_t>((f.W + kTiles[f.tile][1] - 1) / kTiles[f.tile][1]) *
                   ((f.H + kTiles[f.tile][0] - 1) / kTiles[f.tile][0]);
    total_rows += f.H;
  }
  bool moved = false;
  lf_status s;
  if ((s = dev_grow(reinterpret_cast<void**>(&b->arena), &b->arena_cap, o, &moved)) != LF_OK) return s;
  if (b->frames_cap < static_cast<size_t>(nf)) {
    size_t cap = 0;
    const size_t n = std::max<size_t>(nf, 64);
    if (b->d_frames) cudaFree(b->d_frames);
    if (b->d_prior) cudaFree(b->d_prior);
    if (b->d_refocus) cudaFree(b->d_refocus);
    if (b->d_median) cudaFree(b->d_median);
    b->d_frames = nullptr;
    b->d_prior = nullptr;
    b->d_refocus = nullptr;
    b->d_median = nullptr;
    if ((s = dev_grow(reinterpret_cast<void**>(&b->d_frames), &cap, n * sizeof(FrameDesc))) != LF_OK) return s;
    cap = 0;
    if ((s = dev_grow(reinterpret_cast<void**>(&b->d_prior), &cap, n * sizeof(PriorArgs))) != LF_OK) return s;
    cap = 0;
    if ((s = dev_grow(reinterpret_cast<void**>(&b->d_refocus), &cap, n * sizeof(RefocusArgs))) != LF_OK) return s;
    cap = 0;
    if ((s = dev_grow(reinterpret_cast<void**>(&b->d_median), &cap, n * sizeof(MedianArgs))) != LF_OK) return s;
    if (b->d_fcount) cudaFree(b->d_fcount);
    b->d_fcount = nullptr;
    cap = 0;
    if ((s = dev_grow(reinterpret_cast<void**>(&b->d_fcount), &cap, n * sizeof(unsigned long long))) != LF_OK)
      return s;
    b->frames_cap = n;
    moved = true;
  }
  if ((s = dev_grow(reinterpret_cast<void**>(&b->d_items), &b->items_cap, total_items * sizeof(TileItem), &moved)) !=
      LF_OK)
    return s;
  if ((s = dev_grow(reinterpret_cast<void**>(&b->d_rows), &b->rows_cap, total_rows * sizeof(RowItem), &moved)) !=
      LF_OK)
    return s;
  // 3. host image of the arena's table/prior part, descriptors and work lists
  std::vector<uint8_t> host(host_bytes, 0);
  std::vector<FrameDesc> fd(nf);
  std::vector<PriorArgs> pa(nf);
  std::vector<RefocusArgs> ra(nf);
  std::vector<MedianArgs> ma(nf);
  std::vector<TileItem> items;
  items.reserve(total_items);
  std::vector<RowItem> rows;
  rows.reserve(total_rows);
  int counts[2 * kGroups + 1] = {0};
  uint8_t* A = b->arena;
  cudaStream_t st = b->stream;
  uint64_t nominal = 0;
  for (int g = 0; g < kGroups; ++g) {
    for (int i = 0; i < nf; ++i) {
      Frame& f = b->frames[i];
      if (group_of(f.K, f.tile) != g) continue;
      const int TR = kTiles[f.tile][0], TW = kTiles[f.tile][1];
      for (int y = 0; y < (f.H + TR - 1) / TR; ++y)
        for (int x = 0; x < (f.W + TW - 1) / TW; ++x) items.push_back(TileItem{i, x, y, 0});
      counts[g] += ((f.H + TR - 1) / TR) * ((f.W + TW - 1) / TW);
    }
  }
  for (int i = 0; i < nf; ++i) {
    Frame& f = b->frames[i];
    const size_t HW = static_cast<size_t>(f.H) * f.W;
    std::memcpy(&host[f.o_w], f.wtab.data(), f.wtab.size() * 4);
    std::memcpy(&host[f.o_o], f.otab.data(), f.otab.size() * 4);
    std::memcpy(&host[f.o_chg], f.chg.data(), f.chg.size() * 4);
    std::memcpy(&host[f.o_dval], f.dval.data(), f.dval.size() * 4);
    if (!f.tris.empty()) std::memcpy(&host[f.o_tris], f.tris.data(), f.tris.size() * sizeof(PriorTri));
    std::memcpy(&host[f.o_bins], f.bins.data(), f.bins.size() * 4);
    for (int y = 0; y < f.H; ++y) rows.push_back(RowItem{i, y});
    nominal += static_cast<uint64_t>(HW) * f.K * f.D * f.iters;
    // input staging (device to device, on the batch stream, before the graph)
    const uint8_t* img = static_cast<const uint8_t*>(f.src_img);
    const int in_bpp = f.C * (f.dtype == LF_U8 ? 1 : f.dtype == LF_F32 ? 4 : 2);
    const size_t in_row = static_cast<size_t>(f.W) * in_bpp;
    if (f.stage_img) {
      LF_CUDA(cudaMemcpy2DAsync(A + f.o_img, f.img_pitch, img, in_row, in_row, static_cast<size_t>(f.H) * f.K,
                                cudaMemcpyDeviceToDevice, st),
              "batch staging");
      img = A + f.o_img;
    }
    const float* P = f.src_p;
    if (f.stage_p) {
      LF_CUDA(cudaMemcpy2DAsync(A + f.o_p, f.p_pitch, f.src_p, static_cast<size_t>(f.W) * 4,
                                static_cast<size_t>(f.W) * 4, static_cast<size_t>(f.H) * f.K,
                                cudaMemcpyDeviceToDevice, st),
              "batch staging");
      P = reinterpret_cast<const float*>(A + f.o_p);
    }
    SweepArgs& a = f.args;
    a.H = f.H; a.W = f.W; a.C = f.C; a.ref = f.ref; a.dtype = f.stage_dtype;
    a.TR = kTiles[f.tile][0];
    a.TW = kTiles[f.tile][1];
    a.iters = f.iters;
    a.early_exit = b->p.early_exit;
    a.mseg = b->p.mstep_seg_term;
    a.prec = b->p.precision;
    a.dyn_only = b->p.dynamic_only != 0;
    a.seg_threshold = b->p.seg_threshold;
    a.beta = b->p.beta;
    a.gamma = b->p.gamma;
    a.inv2s2 = static_cast<float>(1.0 / (2.0 * static_cast<double>(b->p.sigma) * b->p.sigma));
    a.log_thr = static_cast<float>(std::log(static_cast<double>(b->p.seg_threshold) / (1.0 - b->p.seg_threshold)));
    a.eps = b->p.eps;
    a.wtab = reinterpret_cast<const float*>(A + f.o_w);
    a.otab = reinterpret_cast<const int*>(A + f.o_o);
    a.chg = reinterpret_cast<const unsigned*>(A + f.o_chg);
    a.dval = reinterpret_cast<const float*>(A + f.o_dval);
    a.mu = reinterpret_cast<const float*>(A + f.o_mu);
    for (int k = 0; k < kMaxCams; ++k) {
      a.omin[k] = f.omin[k];
      a.omax[k] = f.omax[k];
    }
    uint16_t* lab = f.labels ? f.labels : reinterpret_cast<uint16_t*>(A + f.o_lab);
    a.d_idx = f.d_idx;
    a.d_out = f.d_out;
    a.labels = lab;
    a.post = f.post;
    a.counter = b->d_fcount + i;
    set_pruning(a, b->p.prune, f.K, f.dval.data(), f.D, b->p.eps);
    a.status = b->d_status;
    a.timeout_ns = 2000000000ull;
    fd[i].args = a;
    if (!encode(&fd[i].img_map, img, f.img_pitch, f.W, f.H, f.K, f.bpp, a.RW, a.TR + 2) ||
        !encode(&fd[i].p_map, P, f.p_pitch, f.W, f.H, f.K, 4, a.RW, a.TR))
      return fail(LF_ECUDA, "cuTensorMapEncodeTiled failed for frame " + sig_string(f));
    pa[i] = PriorArgs{f.H, f.W, f.nbx, f.nby, reinterpret_cast<const PriorTri*>(A + f.o_tris),
                      reinterpret_cast<const int*>(A + f.o_bins),
                      reinterpret_cast<const int*>(A + f.o_bins) + (f.nbx * f.nby + 1),
                      reinterpret_cast<float*>(A + f.o_mu)};
    float* ref_out = f.refocus ? (b->p.median ? reinterpret_cast<float*>(A + f.o_tmp) : f.refocus) : nullptr;
    ra[i] = RefocusArgs{f.H, f.W, f.C, f.K, f.ref, f.stage_dtype, f.KP, f.img_pitch, img, a.wtab, a.otab,
                        f.d_idx, lab, ref_out};
    ma[i] = MedianArgs{f.H, f.W, f.C, ref_out, b->p.median ? f.refocus : nullptr};
  }
  counts[kGroups] = static_cast<int>(rows.size());
  for (int g = 1; g < kGroups; ++g) counts[kGroups + 1 + g] = counts[kGroups + g] + counts[g - 1];
  LF_CUDA(cudaMemcpyAsync(A, host.data(), host_bytes, cudaMemcpyHostToDevice, st), "batch upload");
  LF_CUDA(cudaMemcpyAsync(b->d_frames, fd.data(), nf * sizeof(FrameDesc), cudaMemcpyHostToDevice, st),
          "batch upload");
  LF_CUDA(cudaMemcpyAsync(b->d_prior, pa.data(), nf * sizeof(PriorArgs), cudaMemcpyHostToDevice, st),
          "batch upload");
  LF_CUDA(cudaMemcpyAsync(b->d_refocus, ra.data(), nf * sizeof(RefocusArgs), cudaMemcpyHostToDevice, st),
          "batch upload");
  LF_CUDA(cudaMemcpyAsync(b->d_median, ma.data(), nf * sizeof(MedianArgs), cudaMemcpyHostToDevice, st),
          "batch upload");
  LF_CUDA(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(TileItem), cudaMemcpyHostToDevice, st),
          "batch upload");
  LF_CUDA(cudaMemcpyAsync(b->d_rows, rows.data(), rows.size() * sizeof(RowItem), cudaMemcpyHostToDevice, st),
          "batch upload");
  LF_CUDA(cudaMemcpyAsync(b->d_counts, counts, sizeof(counts), cudaMemcpyHostToDevice, st), "batch upload");
  // 4. graph shape: every launch group seen so far, each with the largest
  // shared memory it has needed (groups stay and sizes only grow, so that
  // batches of other contents replay the same graph; a group without items
  // in this batch finds an empty queue)
  for (const Frame& f : b->frames) {
    const int g = group_of(f.K, f.tile);
    b->grp_smem[g] = std::max(b->grp_smem[g], f.smem);
    if (f.ref != f.K / 2) b->grp_generic[g] = true;  // sticky, like the sizes
  }
  const size_t* smem = b->grp_smem;
  std::vector<long long> key = {b->p.precision, b->p.median, reinterpret_cast<long long>(b->d_frames),
                                reinterpret_cast<long long>(b->d_items), reinterpret_cast<long long>(b->d_rows)};
  for (int g = 0; g < kGroups; ++g) key.push_back(static_cast<long long>(smem[g]) * 2 + (b->grp_generic[g] ? 1 : 0));
  if (!b->exec || key != b->key) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    const int rgrid = b->num_sms * 8;
    int grid[kGroups] = {0};  // resident CTAs of each persistent launch (queried before capturing)
    for (int g = 0; g < kGroups; ++g)
      if (smem[g])
        grid[g] = b->num_sms * std::max(1, em_sweep_persistent_occupancy(g / kThreadClasses + 1, b->p.precision,
                                                                         smem[g], kThreadsOf[g % kThreadClasses],
                                                                         b->grp_generic[g] ? 0 : 1));
    cudaStream_t c = b->capture;
    LF_CUDA(cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal), "graph capture");
    cudaError_t e = cudaSuccess;
    auto chk = [&e](cudaError_t x) {
      if (e == cudaSuccess) e = x;
    };
    chk(cudaEventRecordWithFlags(b->ev[0], c, cudaEventRecordExternal));
    chk(launch_prior_raster_batched(b->d_prior, b->d_rows, b->d_counts + kGroups, rgrid, c));
    chk(cudaMemsetAsync(b->d_heads, 0, sizeof(unsigned) * kGroups, c));
    chk(cudaMemsetAsync(b->d_fcount, 0, sizeof(unsigned long long) * b->frames_cap, c));
    chk(cudaEventRecordWithFlags(b->ev[1], c, cudaEventRecordExternal));
    chk(cudaEventRecord(b->fork, c));
    bool used[lf_batch::kBranches] = {false, false, false, false};
    int nb = 0;
    for (int g = 0; g < kGroups; ++g) {
      if (!smem[g]) continue;
      const int br = nb++ % lf_batch::kBranches;
      if (!used[br]) {
        chk(cudaStreamWaitEvent(b->branch[br], b->fork, 0));
        used[br] = true;
      }
      chk(launch_em_sweep_persistent(g / kThreadClasses + 1, b->p.precision, b->d_frames, b->d_items,
                                     b->d_counts + kGroups + 1 + g, b->d_counts + g, b->d_heads + g, smem[g],
                                     grid[g], kThreadsOf[g % kThreadClasses], b->grp_generic[g] ? 0 : 1,
                                     b->branch[br]));
    }
    for (int br = 0; br < lf_batch::kBranches; ++br) {
      if (!used[br]) continue;
      chk(cudaEventRecord(b->join[br], b->branch[br]));
      chk(cudaStreamWaitEvent(c, b->join[br], 0));
    }
    chk(cudaEventRecordWithFlags(b->ev[2], c, cudaEventRecordExternal));
    chk(launch_refocus_batched(b->d_refocus, b->d_rows, b->d_counts + kGroups, rgrid, c));
    chk(cudaEventRecordWithFlags(b->ev[3], c, cudaEventRecordExternal));
    if (b->p.median) chk(launch_median3_batched(b->d_median, b->d_rows, b->d_counts + kGroups, rgrid, c));
    chk(cudaEventRecordWithFlags(b->ev[4], c, cudaEventRecordExternal));
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->exec = nullptr;
      return cuda_fail(e, "batch graph");
    }
    b->key = key;
    ++b->graph_captures;
  }
  LF_CUDA(cudaGraphLaunch(b->exec, st), "batch graph launch");
  b->ran = true;
  ++b->runs;
  b->nominal = nominal;
  return LF_OK;
}

lf_status lf_batch_synchronize(lf_batch* b) {
  set_error_message("");
  if (!b) return fail(LF_EINVAL, "batch is NULL");
  LF_CUDA(cudaStreamSynchronize(b->stream), "synchronize");
  unsigned st = 0;
  LF_CUDA(cudaMemcpy(&st, b->d_status, sizeof(st), cudaMemcpyDeviceToHost), "status read");
  if (st) LF_CUDA(cudaMemset(b->d_status, 0, sizeof(st)), "status reset");
  if (st & kStatusTmaTimeout) return fail(LF_ETIMEOUT, "a bounded TMA wait in the sweep kernel expired");
  if (st & kStatusSmemMisaligned) return fail(LF_ECUDA, "sweep kernel: dynamic shared memory not 128-byte aligned");
  if (st & kStatusBoundsViolation)
    return fail(LF_ECUDA, "sweep kernel (debug build): a shared-memory index left its region");
  return LF_OK;
}

lf_status lf_batch_get_stats(lf_batch* b, lf_stats* out) {
  set_error_message("");
  if (!b || !out) return fail(LF_EINVAL, "NULL argument");
  lf_status s = lf_batch_synchronize(b);
  if (s != LF_OK) return s;
  lf_stats r{};
  r.runs = b->runs;
  r.nominal_ray_samples = b->nominal;
  if (b->ran) {
    std::vector<unsigned long long> n(b->frames.size());
    LF_CUDA(cudaMemcpy(n.data(), b->d_fcount, n.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost),
            "counter read");
    for (size_t i = 0; i < n.size(); ++i)
      r.executed_ray_samples += n[i] * static_cast<uint64_t>(b->frames[i].K);
    float* ms[4] = {&r.ms_prior, &r.ms_sweep, &r.ms_refocus, &r.ms_median};
    for (int i = 0; i < 4; ++i) LF_CUDA(cudaEventElapsedTime(ms[i], b->ev[i], b->ev[i + 1]), "event time");
    r.kernels_launched = 2 + b->p.median;
    for (size_t x : b->grp_smem) r.kernels_launched += x != 0;
    r.graph_captures = b->graph_captures;
    r.tuned_signatures = b->tuned;
  }
  b->runs = 0;
  *out = r;
  return LF_OK;
}

void lf_batch_destroy(lf_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  void* bufs[] = {b->arena, b->d_frames, b->d_prior, b->d_refocus, b->d_median, b->d_items, b->d_rows,
                  b->d_counts, b->d_heads, b->d_counter, b->d_status, b->d_fcount};
  for (void* p : bufs)
    if (p) cudaFree(p);
  for (cudaEvent_t e : b->ev)
    if (e) cudaEventDestroy(e);
  if (b->capture) cudaStreamDestroy(b->capture);
  for (int i = 0; i < lf_batch::kBranches; ++i) {
    if (b->branch[i]) cudaStreamDestroy(b->branch[i]);
    if (b->join[i]) cudaEventDestroy(b->join[i]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

}  // extern "C"

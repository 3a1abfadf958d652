// Allocation-free entry point: the fused EM sweep with its scratch memory in
// a fixed, file-scope device array instead of buffers the library allocates.
//
// Who needs this: callers that must not call cudaMalloc -- for example a host
// framework that owns all device memory through its own pool and forbids
// raw allocations, or a latency-critical loop that cannot afford the implicit
// device-wide synchronisation a cudaMalloc/cudaFree may cause.  They pass
// every input and output buffer themselves; the sweep's remaining scratch
// (the per-(candidate, camera) sampling tables, the executed-work counter and
// the status word) lives in g_lf_static_scratch below.  That array is part of
// the library image: every GPU that loads the library holds its
// kStaticScratchBytes until the process exits.
//
// The paper has no counterpart of this entry point; it is the same sweep as
// lf_run_em's (same kernel, same results) without the prior raster, the
// refocus and the library-owned buffers.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "lf.h"
#include "lf_internal.h"

namespace {

// Fixed capacity of the scratch array and the limits it implies.
constexpr size_t kStaticScratchBytes = 64 * 1024;
constexpr int kStaticMaxD = 256;
constexpr int kStaticMaxKP = 12;  // cameras padded to a multiple of 4

// Scratch layout (byte offsets), sized for kStaticMaxD x kStaticMaxKP.
constexpr size_t kOffW = 0;                                              // float [D][KP]
constexpr size_t kOffO = kOffW + sizeof(float) * kStaticMaxD * kStaticMaxKP;   // int   [D][KP]
constexpr size_t kOffChg = kOffO + sizeof(int) * kStaticMaxD * kStaticMaxKP;   // uint  [D]
constexpr size_t kOffDval = kOffChg + sizeof(unsigned) * kStaticMaxD;          // float [D]
constexpr size_t kOffCounter = kOffDval + sizeof(float) * kStaticMaxD;         // u64
constexpr size_t kOffStatus = kOffCounter + sizeof(unsigned long long);        // u32
constexpr size_t kStaticUsed = kOffStatus + sizeof(unsigned);
static_assert(kStaticUsed <= kStaticScratchBytes, "static scratch too small for its layout");

// The scratch itself.  In host code this name is only a host-side handle;
// the device address comes from cudaGetSymbolAddress, on every call.
static __device__ __align__(256) unsigned char g_lf_static_scratch[kStaticScratchBytes];

std::mutex g_static_mutex;                // serialises host staging and the GPU work
unsigned char g_host_stage[kOffCounter];  // host copy of the tables (pageable)

lf_status fail(lf_status s, const std::string& m) {
  lf::set_error_message(m);
  return s;
}

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

}  // namespace

extern "C" lf_status lf_run_em_static(int n_cams, const float* baselines, int H, int W, float d_min,
                                      float d_max, int D, const lf_params* p, int iters, const void* images,
                                      int C, int dtype, const float* seg_prior, const float* mu,
                                      int32_t* disparity_idx, float* disparity, float* posteriors,
                                      uint16_t* labels, void* stream) {
  using namespace lf;
  NvtxRange range("lf_run_em_static");
  set_error_message("");
  if (n_cams < 1 || n_cams > kMaxCams) return fail(LF_EINVAL, "n_cams must be in [1, 12]");
  if (!baselines || !images || !seg_prior || !mu || !disparity_idx)
    return fail(LF_EINVAL, "baselines, images, seg_prior, mu and disparity_idx must not be NULL");
  if (H < 3 || W < 3) return fail(LF_EINVAL, "H and W must be >= 3");
  if (D < 1 || D > kStaticMaxD)
    return fail(LF_EINVAL, "D must be in [1, 256]: the static scratch holds tables for at most 256 candidates");
  if (!std::isfinite(d_min) || !std::isfinite(d_max) || d_max < d_min) return fail(LF_EINVAL, "need d_min <= d_max");
  if (iters < 1 || iters > 255) return fail(LF_EINVAL, "iters must be in [1, 255]");
  if (C != 1 && C != 3) return fail(LF_EINVAL, "C must be 1 or 3");
  if (dtype != LF_U8 && dtype != LF_F32) return fail(LF_EINVAL, "dtype must be LF_U8 or LF_F32");
  int ref = -1;
  for (int k = 0; k < n_cams; ++k) {
    if (!std::isfinite(baselines[k])) return fail(LF_EINVAL, "non-finite baseline");
    if (baselines[k] == 0.f && ref < 0) ref = k;
  }
  if (ref < 0) return fail(LF_EINVAL, "no baseline equals 0 (reference camera)");
  lf_params prm;
  lf_default_params(&prm);
  if (p) prm = *p;
  std::string why;
  if (!check_params(prm, &why)) return fail(LF_EINVAL, why);  // the same checks as lf_create
  if (prm.precision != LF_PREC_F32) return fail(LF_EINVAL, "the allocation-free sweep stages float32 maps only (LF_PREC_F32)");
  if (prm.em_mode != LF_EM_HARD) return fail(LF_EINVAL, "the allocation-free sweep runs the hard EM only (LF_EM_HARD)");
  if (prm.dynamic_only) return fail(LF_EINVAL, "the allocation-free sweep reconstructs every pixel (dynamic_only = 0)");
  const size_t bpp = static_cast<size_t>(C) * (dtype == LF_U8 ? 1 : 4);
  // Without staging buffers the inputs are read in place by TMA: rows must
  // start on 16-byte boundaries.
  if ((static_cast<size_t>(W) * bpp) % 16 != 0 || (static_cast<size_t>(W) * 4) % 16 != 0 ||
      reinterpret_cast<uintptr_t>(images) % 16 != 0 || reinterpret_cast<uintptr_t>(seg_prior) % 16 != 0)
    return fail(LF_EINVAL, "images and seg_prior rows must be 16-byte aligned (W * bytes per pixel % 16 == 0)");

  std::lock_guard<std::mutex> lock(g_static_mutex);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(LF_ECUDA, "cudaGetDevice failed");
  // The array's device address, looked up on every call with the caller's
  // device current: cheap, allocates nothing, and never stale (a cached
  // address would outlive a cudaDeviceReset that reloads the module).
  void* addr = nullptr;
  e = cudaGetSymbolAddress(&addr, g_lf_static_scratch);
  if (e != cudaSuccess || !addr)
    return fail(LF_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  unsigned char* scratch = static_cast<unsigned char*>(addr);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // sampling tables, as lf_create builds them
  const int KP = (n_cams + 3) / 4 * 4;
  float* hw = reinterpret_cast<float*>(g_host_stage + kOffW);
  int* ho = reinterpret_cast<int*>(g_host_stage + kOffO);
  unsigned* hc = reinterpret_cast<unsigned*>(g_host_stage + kOffChg);
  float* hd = reinterpret_cast<float*>(g_host_stage + kOffDval);
  std::memset(g_host_stage, 0, sizeof(g_host_stage));
  int omin = 0, omax = 0;
  SweepArgs a{};
  for (int k = 0; k < kMaxCams; ++k) a.omin[k] = a.omax[k] = 0;
  for (int j = 0; j < D; ++j) {
    const double dj = D == 1 ? static_cast<double>(d_min)
                             : static_cast<double>(d_min) +
                                   j * ((static_cast<double>(d_max) - static_cast<double>(d_min)) / (D - 1));
    hd[j] = static_cast<float>(dj);
    unsigned m = 0;
    for (int k = 0; k < n_cams; ++k) {
      const double x = -dj * static_cast<double>(baselines[k]);
      const double o = std::floor(x);
      const int oi = static_cast<int>(o);
      ho[j * KP + k] = oi;
      hw[j * KP + k] = static_cast<float>(x - o);
      if (j == 0 || ho[(j - 1) * KP + k] != oi) m |= 1u << k;
      if (j == 0 || oi < a.omin[k]) a.omin[k] = oi;
      if (j == 0 || oi > a.omax[k]) a.omax[k] = oi;
      omin = oi < omin ? oi : omin;
      omax = oi + 1 > omax ? oi + 1 : omax;
    }
    hc[j] = m;
  }
  // tile shape: the widest whose staged rows fit one TMA box and whose
  // shared memory fits the device
  int dev_smem = 0;
  if (cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    dev_smem = 227 * 1024;
  static const int cand[][2] = {{2, 128}, {1, 128}, {4, 64}, {2, 64}, {1, 64}, {2, 32}, {1, 32}};
  bool found = false;
  for (auto& t : cand) {
    if (t[0] * t[1] > sweep_max_threads(n_cams)) continue;
    a.TR = t[0];
    a.TW = t[1];
    a.L = -omin;
    a.R = omax;
    a.SW = a.TW + a.L + a.R;
    a.SWp = (a.SW + 31) / 32 * 32;
    a.RW = (a.SW + 17 + 15) / 16 * 16;
    a.bpp = static_cast<int>(bpp);
    a.D = D;
    a.KP = KP;
    if (a.RW * a.bpp / 8 > 256 || a.RW / 2 > 256) continue;
    if (sweep_smem_bytes(n_cams, a) > static_cast<size_t>(dev_smem)) continue;
    found = true;
    break;
  }
  if (!found) return fail(LF_EINVAL, "disparity halo too wide for the sweep kernel's shared-memory staging");

  CUtensorMap img_map, p_map;
  if (!encode(&img_map, images, static_cast<size_t>(W) * bpp, W, H, n_cams, bpp, a.RW, a.TR + 2) ||
      !encode(&p_map, seg_prior, static_cast<size_t>(W) * 4, W, H, n_cams, 4, a.RW, a.TR))
    return fail(LF_ECUDA, "cuTensorMapEncodeTiled failed");

  // upload the tables and clear what must start at zero
  e = cudaMemcpyAsync(scratch, g_host_stage, kOffCounter, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(scratch + kOffCounter, 0, kStaticUsed - kOffCounter, s);
  if (e != cudaSuccess) return fail(LF_ECUDA, std::string("scratch upload: ") + cudaGetErrorString(e));

  a.H = H; a.W = W; a.C = C; a.ref = ref; a.dtype = dtype;
  a.iters = iters;
  a.early_exit = prm.early_exit;
  a.mseg = prm.mstep_seg_term;
  a.beta = prm.beta;
  a.gamma = prm.gamma;
  a.inv2s2 = static_cast<float>(1.0 / (2.0 * static_cast<double>(prm.sigma) * prm.sigma));
  a.log_thr = static_cast<float>(std::log(static_cast<double>(prm.seg_threshold) / (1.0 - prm.seg_threshold)));
  a.eps = prm.eps;
  a.wtab = reinterpret_cast<const float*>(scratch + kOffW);
  a.otab = reinterpret_cast<const int*>(scratch + kOffO);
  a.chg = reinterpret_cast<const unsigned*>(scratch + kOffChg);
  a.dval = reinterpret_cast<const float*>(scratch + kOffDval);
  a.mu = mu;
  a.d_idx = disparity_idx;
  a.d_out = disparity;
  a.labels = labels;
  a.post = posteriors;
  a.counter = reinterpret_cast<unsigned long long*>(scratch + kOffCounter);
  set_pruning(a, prm.prune, n_cams, hd, D, prm.eps);
  a.status = reinterpret_cast<unsigned*>(scratch + kOffStatus);
  a.timeout_ns = 2000000000ull;
  e = launch_em_sweep(n_cams, img_map, p_map, a, s);
  if (e != cudaSuccess) return fail(LF_ECUDA, std::string("em_sweep launch: ") + cudaGetErrorString(e));
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(LF_ECUDA, std::string("synchronize: ") + cudaGetErrorString(e));
  unsigned st = 0;
  e = cudaMemcpy(&st, scratch + kOffStatus, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(LF_ECUDA, std::string("status read: ") + cudaGetErrorString(e));
  if (st & kStatusTmaTimeout) return fail(LF_ETIMEOUT, "a bounded TMA wait in the sweep kernel expired");
  if (st & kStatusSmemMisaligned) return fail(LF_ECUDA, "sweep kernel: dynamic shared memory not 128-byte aligned");
  if (st & kStatusBoundsViolation)
    return fail(LF_ECUDA, "sweep kernel (debug build): a shared-memory index left its region");
  return LF_OK;
}

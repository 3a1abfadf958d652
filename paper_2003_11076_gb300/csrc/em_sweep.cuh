// Fused per-pixel EM sweep (Sec. III-B schedule; M-step Sec. III-C; E-step
// Sec. III-D; posteriors of the final labels), one CTA per tile of
// TR x TW reference pixels, one thread per pixel.
//
// Phases of one CTA:
//   1. TMA (cp.async.bulk.tensor) stages, for all K cameras at once, the raw
//      image rows v0-1 .. v0+TR (Sobel needs one row above and below) and the
//      P(dynamic) rows v0 .. v0+TR-1, over the tile's columns plus the
//      disparity halo, completing on one mbarrier (bounded wait).
//   2. Luminance, Sobel-x/8, Sobel-y/8, log(1-P) and log(P) per staged texel
//      are computed into shared memory with the image border replicated
//      (Sec. III-C descriptors).  Nothing of this is written to HBM.
//   3. Each thread runs the whole EM for its pixel.  The D x K cost volume is
//      never materialised: the M-step keeps, per camera, the two texels that
//      bracket the current sample in registers and reloads them only when the
//      integer part of u - d_j * b_k changes (the change mask is the same for
//      every pixel, so the reload branch is warp-uniform).  Each ray sample is
//      a linear interpolation (Sec. III-F non-integral disparities) and an
//      accumulation of the shifted sums of the static rays' descriptors.
//      Each M-step evaluates only the candidates whose upper bound (log prior
//      plus the largest segmentation term) reaches the objective of one
//      candidate already evaluated (exact: the arg-max is unchanged), and
//      the tile's pixels are sorted by that candidate interval so that a
//      warp's lanes sweep similar ranges.
//   4. The E-step enumerates all 2^K label vectors in increasing mask order
//      as a depth-first subset tree (each subset's sums built from its
//      parent, no subtraction), keeping the first maximum; from seven
//      cameras it skips blocks of vectors whose bound is below the
//      all-static vector's objective.
//   5. Posteriors: the same enumeration at the final disparity gives the
//      per-ray marginals of q(S) ~ exp J(d_T, S).
//
// Numerics: descriptors are shifted by the reference ray's descriptor before
// summation, so the variance sum(|g|^2) - |sum g|^2 / n is formed from small
// numbers; all accumulation is float32.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstdint>

#include "lf_internal.h"
#include "prior_pixel.cuh"

namespace lf {
namespace dev {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Spin on the mbarrier phase for at most limit_ns; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned phase,
                                                  unsigned long long limit_ns) {
  if (mbar_try_wait(bar, phase)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, phase)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Staged maps per camera and tile row (Sec. III-C descriptors and the
// segmentation prior of Sec. III-B), SWp texels each:
//   Y   luminance
//   X   Sobel-x / 8
//   Zs  Sobel-y / 8
//   ls  log p(static)  = log max(1 - P, eps)
//   ld  log p(dynamic) = log max(P, eps)
//   T   ld - ls, the first-iteration label test (static iff its
//       interpolated value is below log(thr / (1 - thr)))
// stored per precision mode as planes of register pairs, so that one load
// gives two values the packed float32x2 arithmetic uses together:
//   float32   (Y, X) float2 | (Zs, ld) float2 | ls float  | T float    24 B
//   float16   Y float | (X, Zs) half2  | (ld, ls) float2 | T float     20 B
//   bfloat16  Y float | (X, Zs) bf162  | (ld, ls) float2 | T float     20 B
// Only the Sobel responses (differences of neighbouring luminances: small
// numbers that keep their relative precision) are stored in 16 bits.  The
// luminance and the log segmentation maps stay float32: rounding the
// luminance to 16 bits moves the photometric variance, and rounding the log
// maps moves the segmentation term and the label test, by more than the
// arg-max margins the parity rule allows (16-bit luminance alone takes the
// disparity agreement of a float32 gray frame to 99.84 % in float16 and
// 98.8 % in bfloat16; bfloat16 log maps to 99.94 % on the 960 x 600 frame).
__host__ __device__ constexpr int texel_bytes(int prec) {
  return prec == kPrecF32 ? 24 : 20;
}

// First-iteration labels are decided on lerp(T) < log(thr / (1 - thr)).  A
// camera whose T texels over the pixel's whole sample range stay at least
// this far on one side of the threshold has the same label for every
// candidate (the interpolated value cannot leave [min, max] by more than a
// few units of float32 rounding, far below this margin).
constexpr float kThresholdMargin = 1e-4f;

// The hardware's base-2 exponential and logarithm (special-function unit,
// about 2^-22 relative error).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Debug builds (LF_DEBUG) check the indices into the shared-memory carve-up
// against their regions: an index outside [lo, hi] sets
// kStatusBoundsViolation in the run's status word (the call then reports
// LF_ECUDA) and is clamped into the region, so the access stays inside
// shared memory.  Release builds compile the check away.
__device__ __forceinline__ int chk(int i, int lo, int hi, unsigned* status) {
#ifdef LF_DEBUG
  if (i < lo || i > hi) {
    atomicOr(status, kStatusBoundsViolation);
    return i < lo ? lo : hi;
  }
#else
  (void)lo;
  (void)hi;
  (void)status;
#endif
  return i;
}

__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <typename TS>
struct Texels;

template <>
struct Texels<float> {
  static constexpr int kBytes = 24;
  // (Y, X) and (Zs, ld) of texel c of one camera row
  __device__ static __forceinline__ void quad(const uint8_t* R, int SWp, int c, float2& yx, float2& zd) {
    yx = reinterpret_cast<const float2*>(R)[c];
    zd = reinterpret_cast<const float2*>(R + 8 * SWp)[c];
  }
  __device__ static __forceinline__ float ls(const uint8_t* R, int SWp, int c) {
    return reinterpret_cast<const float*>(R + 16 * SWp)[c];
  }
  __device__ static __forceinline__ float t(const uint8_t* R, int SWp, int c) {
    return reinterpret_cast<const float*>(R + 20 * SWp)[c];
  }
  __device__ static __forceinline__ void store(uint8_t* R, int SWp, int c, float Y, float X, float Zs, float ls,
                                               float ld) {
    reinterpret_cast<float2*>(R)[c] = make_float2(Y, X);
    reinterpret_cast<float2*>(R + 8 * SWp)[c] = make_float2(Zs, ld);
    reinterpret_cast<float*>(R + 16 * SWp)[c] = ls;
    reinterpret_cast<float*>(R + 20 * SWp)[c] = ld - ls;
  }
};

template <>
struct Texels<__half> {
  static constexpr int kBytes = 20;
  __device__ static __forceinline__ void quad(const uint8_t* R, int SWp, int c, float2& yx, float2& zd) {
    const float2 xz = __half22float2(reinterpret_cast<const __half2*>(R + 4 * SWp)[c]);
    yx = make_float2(reinterpret_cast<const float*>(R)[c], xz.x);
    zd = make_float2(xz.y, reinterpret_cast<const float2*>(R + 8 * SWp)[c].x);
  }
  __device__ static __forceinline__ float ls(const uint8_t* R, int SWp, int c) {
    return reinterpret_cast<const float2*>(R + 8 * SWp)[c].y;
  }
  __device__ static __forceinline__ float t(const uint8_t* R, int SWp, int c) {
    return reinterpret_cast<const float*>(R + 16 * SWp)[c];
  }
  __device__ static __forceinline__ void store(uint8_t* R, int SWp, int c, float Y, float X, float Zs, float ls,
                                               float ld) {
    reinterpret_cast<float*>(R)[c] = Y;
    reinterpret_cast<__half2*>(R + 4 * SWp)[c] = __floats2half2_rn(X, Zs);
    reinterpret_cast<float2*>(R + 8 * SWp)[c] = make_float2(ld, ls);
    reinterpret_cast<float*>(R + 16 * SWp)[c] = ld - ls;
  }
};

template <>
struct Texels<__nv_bfloat16> {
  static constexpr int kBytes = 20;
  __device__ static __forceinline__ void quad(const uint8_t* R, int SWp, int c, float2& yx, float2& zd) {
    const float2 xz = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(R + 4 * SWp)[c]);
    yx = make_float2(reinterpret_cast<const float*>(R)[c], xz.x);
    zd = make_float2(xz.y, reinterpret_cast<const float2*>(R + 8 * SWp)[c].x);
  }
  __device__ static __forceinline__ float ls(const uint8_t* R, int SWp, int c) {
    return reinterpret_cast<const float2*>(R + 8 * SWp)[c].y;
  }
  __device__ static __forceinline__ float t(const uint8_t* R, int SWp, int c) {
    return reinterpret_cast<const float*>(R + 16 * SWp)[c];
  }
  __device__ static __forceinline__ void store(uint8_t* R, int SWp, int c, float Y, float X, float Zs, float ls,
                                               float ld) {
    reinterpret_cast<float*>(R)[c] = Y;
    reinterpret_cast<__nv_bfloat162*>(R + 4 * SWp)[c] = __floats2bfloat162_rn(X, Zs);
    reinterpret_cast<float2*>(R + 8 * SWp)[c] = make_float2(ld, ls);
    reinterpret_cast<float*>(R + 16 * SWp)[c] = ld - ls;
  }
};

static_assert(Texels<float>::kBytes == texel_bytes(kPrecF32) && Texels<__half>::kBytes == texel_bytes(kPrecF16) &&
                  Texels<__nv_bfloat16>::kBytes == texel_bytes(kPrecBF16),
              "staged texel sizes of host and device must agree");

__host__ __device__ inline size_t align_up(size_t x, size_t n) { return (x + n - 1) / n * n; }

// Shared-memory carve-up, identical on host (size) and device (offsets).
struct SmemLayout {
  size_t raw_img, raw_p, luma, feat, wtab, otab, chg, dval, rcp, mu, pix, wcnt, sortc, bar, total;
};

// Per-pixel EM state of one tile, kept in shared memory between iterations
// so that the unconverged pixels can be regrouped into dense warps.
struct PixelState {
  int16_t* list;    // pixel indices (tile order) to process in the current pass
  int16_t* list2;   // the next pass's (the two alternate)
  uint16_t* S;      // current labels
  uint16_t* S0;     // first-iteration labels when they do not depend on d
  int16_t* jb;      // current arg-max candidate
  float* emax;      // objective of the current labels at jb
  float* seg_ub;    // upper bound of the segmentation term (candidate pruning)
  int16_t* lo;      // candidates the next M-step evaluates: lo .. hi
  int16_t* hi;
  uint8_t* fixed0;  // S0 valid
  uint8_t* conv;    // reached its fixed point
};
constexpr int kPixelStateBytes = 24;
// The per-pixel state of a tile of P pixels at b (kPixelStateBytes * P bytes).
__device__ __forceinline__ PixelState pixel_state(uint8_t* b, int P) {
  PixelState ps;
  ps.emax = reinterpret_cast<float*>(b);
  ps.seg_ub = ps.emax + P;
  ps.S = reinterpret_cast<uint16_t*>(ps.seg_ub + P);
  ps.S0 = ps.S + P;
  ps.jb = reinterpret_cast<int16_t*>(ps.S0 + P);
  ps.list = ps.jb + P;
  ps.list2 = ps.list + P;
  ps.lo = ps.list2 + P;
  ps.hi = ps.lo + P;
  ps.fixed0 = reinterpret_cast<uint8_t*>(ps.hi + P);
  ps.conv = ps.fixed0 + P;
  return ps;
}
// Counters of the CTA's counting sort (sort_pixels): up to 64 keys per warp.
constexpr int kSortKeys = 64;

// Fixed head of the shared memory: the CTA's mbarrier, then (persistent
// kernel) the current frame's arguments, then the item index.  Everything
// after it depends on the frame.
constexpr size_t kSmemBar = 0;
constexpr size_t kSmemArgs = 16;
constexpr size_t kSmemItem = kSmemArgs + ((sizeof(SweepArgs) + 15) / 16) * 16;
constexpr size_t kSmemHead = ((kSmemItem + 16 + 127) / 128) * 128;

// float32 gray inputs: the staged raw rows already hold the luminance in the
// layout the descriptor maps read, so they are used in place.
__host__ __device__ inline bool luma_is_raw(const SweepArgs& a) { return a.dtype == 1 && a.C == 1; }

// The sampling tables in shared memory: per (candidate, camera) the
// interpolation weight and its square, (w, w^2) (float2), and the tap
// offset floor(-d_j b_k) (int).
__host__ __device__ inline SmemLayout sweep_layout(int K, const SweepArgs& a) {
  SmemLayout L{};
  size_t o = kSmemHead;
  L.raw_img = o;
  o = align_up(o + static_cast<size_t>(K) * (a.TR + 2) * a.RW * a.bpp, 128);
  L.raw_p = o;
  o = align_up(o + static_cast<size_t>(K) * a.TR * a.RW * 4, 128);
  L.luma = o;  // float32 gray inputs: the staged rows are the luminance (no region of its own)
  o = align_up(o + (luma_is_raw(a) ? 0 : static_cast<size_t>(K) * (a.TR + 2) * a.RW * 4), 16);
  L.feat = o;
  o = align_up(o + static_cast<size_t>(K) * a.TR * a.SWp * texel_bytes(a.prec), 16);
  L.wtab = o;
  o = align_up(o + static_cast<size_t>(a.D) * a.KP * 8, 16);
  L.otab = o;
  o = align_up(o + static_cast<size_t>(a.D) * a.KP * 4, 16);
  L.chg = o;
  o = align_up(o + static_cast<size_t>(a.D) * 4, 16);
  L.dval = o;
  o = align_up(o + static_cast<size_t>(a.D) * 4, 16);
  L.rcp = o;
  o = align_up(o + 16 * 4, 16);
  L.mu = o;  // fused prior: the tile's prior centres
  o = align_up(o + static_cast<size_t>(a.TR) * a.TW * 4, 16);
  L.pix = o;
  o = align_up(o + static_cast<size_t>(a.TR) * a.TW * kPixelStateBytes, 16);
  L.wcnt = o;  // 32 ints of per-warp scratch, then the tile's two statistics counters
  o = align_up(o + 34 * 4, 16);
  L.sortc = o;
  o = align_up(o + static_cast<size_t>(kSortKeys) * ((a.TR * a.TW + 31) / 32) * 2, 16);
  L.bar = kSmemBar;
  L.total = o;
  return L;
}

// The soft-EM variant keeps its per-pixel state after the sweep layout.
__host__ __device__ inline size_t soft_state_offset(int K, const SweepArgs& a) {
  return align_up(sweep_layout(K, a).total, 16);
}

__device__ __forceinline__ int floor16(int x) { return x >= 0 ? (x & ~15) : -((-x + 15) & ~15); }

// View of one CTA's staged maps for one thread's pixel.
template <typename TS>
struct Staged {
  const uint8_t* F;     // camera 0's maps, this thread's tile row
  int cam_stride;       // bytes between cameras
  int SWp;              // texels per map row
  int cbase;            // staged column of this pixel (offset 0)
  __device__ __forceinline__ const uint8_t* row(int k) const { return F + k * cam_stride; }
};

// (w, w^2) of cameras 0..K-1 at candidate j: entries come in pairs of cameras
// as float4 loads (the table's row stride KP is a multiple of 4).
template <int K>
__device__ __forceinline__ void load_weights(const float2* s_wq, int KP, int j, float2 (&w)[K]) {
  const float4* w4 = reinterpret_cast<const float4*>(s_wq + j * KP);
#pragma unroll
  for (int q = 0; q < (K + 1) / 2; ++q) {
    const float4 t = w4[q];
    w[2 * q] = make_float2(t.x, t.y);
    if (2 * q + 1 < K) w[(2 * q + 1) % K] = make_float2(t.z, t.w);
  }
}

// ---------------------------------------------------------------- M-step
// Both M-steps keep, per camera, the taps bracketing the current sample in
// registers and reload them only where the integer part of u - d_j b_k
// changes (the change mask s_chg[j] is the same for every pixel: the reload
// branch is warp-uniform).  Quantities that are used together are held as
// register pairs and combined with packed float32x2 operations; every lane
// of a packed operation is an IEEE float32 operation.  The log prior of
// candidate j + 1 (two dependent special-function operations) is evaluated
// while candidate j's sums are formed, off the loop's critical path.

// First M-step: arg-max over the D candidates of J(d_j, S_j) for one pixel
// (lowest j wins ties), where each ray's label S_j is thresholded at the
// ray's own sample (lerp(T) < log(thr / (1 - thr)) means static).  With
// e_k in {0, 1} the ray's label, g_k its shifted descriptor, the candidate's
// sums are
//   sum_k e_k g_k,   sum_k e_k |g_k|^2,   n = sum_k e_k,
//   seg = sum_k [e_k ls_k + (1 - e_k) ld_k] = sum_k ld_k - sum_k e_k T_k,
// formed without selects.  The loop body is straight-line code for the
// current candidate; the taps the next candidate needs are reloaded at its
// end (its change mask is read early, so the branch does not wait for it).
// REF >= 0: camera REF is the reference (known at compile time).  Its ray
// samples the pixel itself at every candidate (weight 0, shifted descriptor
// exactly 0), so only its label test and log prior are accumulated.
// Candidates j0 <= j < j1 (lowest j wins ties; *best_out = the maximum, may
// be NULL).  Every camera's taps are loaded at j0, so a range that starts
// mid-sweep computes each candidate's objective exactly as the whole sweep
// does.  In both M-steps the variance is clamped at 0 (it can come out a few
// units of rounding below 0 when the static rays agree), so that every
// objective is at most its prior and segmentation terms: the bound the
// candidate pruning (prune_range) rests on.
template <int K, typename TS, int REF>
__device__ __forceinline__ int m_step_init_range(const SweepArgs& a, const Staged<TS>& st, const float2* s_wq,
                                                 const int* s_o, const unsigned* s_chg, const float* s_d,
                                                 const float* s_rcp, float cy, float cx, float cz, float mu,
                                                 bool inside, int j0, int j1, float* best_out, unsigned* n_static) {
  using Tx = Texels<TS>;
  // per camera: p1 = (Y, X) at floor(x) minus the reference's, d1 the slope
  // to the next tap; p2 = (Zs minus the reference's, ld), d2; t0, dt the
  // label-test map
  float2 p1[K], d1[K], p2[K], d2[K];
  float t0[K], dt[K];
  const int SWp = st.SWp;
  const float2 ref1 = make_float2(-cy, -cx), ref2 = make_float2(-cz, 0.f);
  // outside the triangulation mu is NaN and the prior is uniform: the prior
  // is then evaluated at a finite centre and weighted by pin = 0
  const float lin = a.mseg ? 1.f : 0.f, pin = inside ? 1.f : 0.f, mu_in = inside ? mu : 0.f;
  const int js = j0 < j1 ? j0 : 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int c = chk(st.cbase + s_o[chk(js * a.KP + k, 0, a.D * a.KP - 1, a.status)], 0, a.SW - 2, a.status);
    const uint8_t* R = st.row(k);
    float2 yx0, zd0, yx1, zd1;
    Tx::quad(R, SWp, c, yx0, zd0);
    Tx::quad(R, SWp, c + 1, yx1, zd1);
    const float T0 = Tx::t(R, SWp, c), T1 = Tx::t(R, SWp, c + 1);
    p1[k] = fadd2(yx0, ref1);
    d1[k] = fsub2(yx1, yx0);
    p2[k] = fadd2(zd0, ref2);
    d2[k] = fsub2(zd1, zd0);
    t0[k] = T0;
    dt[k] = T1 - T0;
  }
  float best = -INFINITY, nsum = 0.f;  // nsum: static rays over the candidates (an exact integer)
  int jb = j0;
  // log prior in base-2 units (the objective takes it times ln 2 * pin):
  // log2(gamma + 2^(k2 t^2)) with k2 = -log2(e) / (2 sigma^2)
  const float k2 = -a.inv2s2 * 1.4426950408889634f, pin_ln2 = pin * 0.6931471805599453f;
  auto prior_at = [&](int j) {
    const float t = s_d[j] - mu_in;
    return lg2_approx(a.gamma + ex2_approx(t * t * k2));
  };
  float pr_next = prior_at(js);
  float2 w_next[K];
  load_weights<K>(s_wq, a.KP, js, w_next);
  for (int j = j0; j < j1; ++j) {
    float2 w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = w_next[k];
    const int jn = min(j + 1, j1 - 1);
    load_weights<K>(s_wq, a.KP, jn, w_next);  // the next candidate's weights, in flight during this one
    const unsigned chn = j + 1 < j1 ? s_chg[jn] : 0u;  // taps the next candidate reloads
    const float pr = pr_next;
    pr_next = prior_at(jn);  // the next candidate's prior, off this one's critical path
    float2 syx = make_float2(0.f, 0.f), szl = make_float2(0.f, 0.f), qq = make_float2(0.f, 0.f);
    float2 nt = make_float2(0.f, 0.f);  // (n, sum of e_k T_k)
    float qz = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (k == REF) {
        const float e = t0[k] < a.log_thr ? 1.f : 0.f;
        szl.y += p2[k].y;
        nt = ffma2(make_float2(e, e), make_float2(1.f, t0[k]), nt);
        continue;
      }
      const float2 ww = make_float2(w[k].x, w[k].x);
      const float2 g1 = ffma2(ww, d1[k], p1[k]);  // (gy, gx)
      const float2 g2 = ffma2(ww, d2[k], p2[k]);  // (gz, ld)
      const float tq = fmaf(w[k].x, dt[k], t0[k]);
      const float e = tq < a.log_thr ? 1.f : 0.f;
      const float2 ee = make_float2(e, e);
      const float2 h1 = fmul2(ee, g1);
      syx = fadd2(syx, h1);
      qq = ffma2(h1, g1, qq);
      const float2 h2 = fmul2(make_float2(e, 1.f), g2);  // (e gz, ld)
      szl = fadd2(szl, h2);
      qz = fmaf(h2.x, g2.x, qz);
      nt = ffma2(ee, make_float2(1.f, tq), nt);
    }
    const float rn = s_rcp[static_cast<int>(nt.x)];
    nsum += nt.x;
    const float q = qq.x + qq.y + qz;
    const float2 sq = fmul2(syx, syx);
    const float ss = fmaf(szl.x, szl.x, sq.x + sq.y);
    const float var = fmaxf(fmaf(-ss, rn, q) * rn, 0.f);
    const float J = fmaf(-a.beta, var, fmaf(pin_ln2, pr, lin * (szl.y - nt.y)));
    if (J > best) { best = J; jb = j; }
    if (chn) {  // same for every pixel: warp-uniform branch
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (!(chn & (1u << k))) continue;
        const int c = chk(st.cbase + s_o[chk(jn * a.KP + k, 0, a.D * a.KP - 1, a.status)], 0, a.SW - 2, a.status);
        const uint8_t* R = st.row(k);
        float2 yx0, zd0, yx1, zd1;
        Tx::quad(R, SWp, c, yx0, zd0);
        Tx::quad(R, SWp, c + 1, yx1, zd1);
        const float T0 = Tx::t(R, SWp, c), T1 = Tx::t(R, SWp, c + 1);
        p1[k] = fadd2(yx0, ref1);
        d1[k] = fsub2(yx1, yx0);
        p2[k] = fadd2(zd0, ref2);
        d2[k] = fsub2(zd1, zd0);
        t0[k] = T0;
        dt[k] = T1 - T0;
      }
    }
  }
  if (n_static) *n_static = static_cast<unsigned>(nsum);
  if (best_out) *best_out = best;
  return jb;
}

template <int K, typename TS, int REF>
__device__ __forceinline__ int m_step_init(const SweepArgs& a, const Staged<TS>& st, const float2* s_wq,
                                           const int* s_o, const unsigned* s_chg, const float* s_d,
                                           const float* s_rcp, float cy, float cx, float cz, float mu,
                                           bool inside, unsigned* n_static) {
  return m_step_init_range<K, TS, REF>(a, st, s_wq, s_o, s_chg, s_d, s_rcp, cy, cx, cz, mu, inside, 0, a.D, nullptr,
                                       n_static);
}

// Camera k's fixed-label terms from its taps at staged column c (the M-step
// with fixed labels S below): b1 = (m_Y, m_X), b2 = (m_Zs, m_L) with L the
// log prior of the ray's label; s1, s2 the slopes to the next tap; ac =
// (2 m.s, |s|^2) and q0 = |m|^2 over the descriptor (Y, X, Zs).
template <typename TS>
__device__ __forceinline__ void fixed_taps(const uint8_t* R, int SWp, int c, bool stat, float lin, float2 ref1,
                                           float2 ref2, float2& b1, float2& b2, float2& s1, float2& s2, float2& ac,
                                           float& q0) {
  using Tx = Texels<TS>;
  float2 yx0, zd0, yx1, zd1;
  Tx::quad(R, SWp, c, yx0, zd0);
  Tx::quad(R, SWp, c + 1, yx1, zd1);
  const float ls0 = Tx::ls(R, SWp, c), ls1 = Tx::ls(R, SWp, c + 1);
  zd0.y = stat ? ls0 : zd0.y;  // (Zs, log prior of the label)
  zd1.y = stat ? ls1 : zd1.y;
  const float sk = stat ? 1.f : 0.f;
  const float2 mk = make_float2(sk, sk), ml = make_float2(sk, lin);
  b1 = fmul2(fadd2(yx0, ref1), mk);
  s1 = fmul2(fsub2(yx1, yx0), mk);
  b2 = fmul2(fadd2(zd0, ref2), ml);
  s2 = fmul2(fsub2(zd1, zd0), ml);
  const float2 bs = fmul2(b1, s1), sq = fmul2(s1, s1), bb = fmul2(b1, b1);
  ac = make_float2(2.f * fmaf(b2.x, s2.x, bs.x + bs.y), fmaf(s2.x, s2.x, sq.x + sq.y));
  q0 = fmaf(b2.x, b2.x, bb.x + bb.y);
}

// M-step with fixed labels S: every iteration after the first, and the first
// when its labels do not depend on the candidate.  With g_k = m_k + w_jk s_k
// (m_k: camera k's tap at floor(x) shifted by the reference descriptor, s_k:
// the slope to the next tap; both zero for a dynamic ray) the static rays'
// sums are
//   sum_k g_k     = sum_k m_k     + sum_k w_jk s_k
//   sum_k |g_k|^2 = sum_k |m_k|^2 + sum_k (w_jk (2 m_k.s_k) + w_jk^2 |s_k|^2)
// and likewise for the log priors of the labels, so one candidate costs
// three packed fused multiply-adds per ray.  The base sums over k change only
// at candidates where some camera's tap moves; they are then summed afresh
// (no drift).  Candidates j0 <= j < j1 (lowest j wins ties; *best_out = the
// maximum).  Every camera's taps are loaded at j0, so a range that starts
// mid-sweep computes each candidate's objective exactly as the whole sweep
// does (a tap that has not moved since its last load holds the same texels).
// As in the first M-step, the loop body is straight-line code for the
// current candidate and the next candidate's reloads come at its end, and
// a reference camera known at compile time (REF >= 0) adds nothing per
// candidate (its slopes are multiplied by weight 0; its log prior is in the
// base sums).
template <int K, typename TS, int REF>
__device__ __forceinline__ int m_step_fixed_range(const SweepArgs& a, const Staged<TS>& st, const float2* s_wq,
                                                  const int* s_o, const unsigned* s_chg, const float* s_d,
                                                  const float* s_rcp, float cy, float cx, float cz, float mu,
                                                  bool inside, unsigned S, int j0, int j1, float* best_out) {
  float2 b1[K], b2[K], s1[K], s2[K], ac[K];
  float q0[K];
  const int SWp = st.SWp;
  const float rn = s_rcp[__popc(S)];
  const float2 ref1 = make_float2(-cy, -cx), ref2 = make_float2(-cz, 0.f);
  // outside the triangulation mu is NaN and the prior is uniform: the prior
  // is then evaluated at a finite centre and weighted by pin = 0
  const float lin = a.mseg ? 1.f : 0.f, pin = inside ? 1.f : 0.f, mu_in = inside ? mu : 0.f;
  const int js = j0 < j1 ? j0 : 0;
#pragma unroll
  for (int k = 0; k < K; ++k)
    fixed_taps<TS>(st.row(k), SWp, chk(st.cbase + s_o[js * a.KP + k], 0, a.SW - 2, a.status), (S >> k) & 1u, lin,
                   ref1, ref2, b1[k], b2[k],
                   s1[k], s2[k], ac[k], q0[k]);
  float2 B1 = b1[0], B2 = b2[0];
  float BQ = q0[0];
#pragma unroll
  for (int k = 1; k < K; ++k) {
    B1 = fadd2(B1, b1[k]);
    B2 = fadd2(B2, b2[k]);
    BQ += q0[k];
  }
  float best = -INFINITY;
  int jb = j0;
  // log prior in base-2 units (the objective takes it times ln 2 * pin):
  // log2(gamma + 2^(k2 t^2)) with k2 = -log2(e) / (2 sigma^2)
  const float k2 = -a.inv2s2 * 1.4426950408889634f, pin_ln2 = pin * 0.6931471805599453f;
  auto prior_at = [&](int j) {
    const float t = s_d[j] - mu_in;
    return lg2_approx(a.gamma + ex2_approx(t * t * k2));
  };
  float pr_next = prior_at(js);
  float2 w_next[K];
  load_weights<K>(s_wq, a.KP, js, w_next);
  for (int j = j0; j < j1; ++j) {
    float2 w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = w_next[k];
    const int jn = min(j + 1, j1 - 1);
    load_weights<K>(s_wq, a.KP, jn, w_next);  // the next candidate's weights, in flight during this one
    const unsigned chn = j + 1 < j1 ? s_chg[jn] : 0u;  // taps the next candidate reloads
    const float pr = pr_next;
    pr_next = prior_at(jn);  // the next candidate's prior, off this one's critical path
    float2 A1 = B1, A2 = B2, QQ = make_float2(BQ, 0.f);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (k == REF) continue;
      const float2 ww = make_float2(w[k].x, w[k].x);
      A1 = ffma2(ww, s1[k], A1);
      A2 = ffma2(ww, s2[k], A2);
      QQ = ffma2(w[k], ac[k], QQ);
    }
    const float q = QQ.x + QQ.y;
    const float2 sq = fmul2(A1, A1);
    const float ss = fmaf(A2.x, A2.x, sq.x + sq.y);
    const float var = fmaxf(fmaf(-ss, rn, q) * rn, 0.f);
    const float J = fmaf(-a.beta, var, fmaf(pin_ln2, pr, A2.y));
    if (J > best) { best = J; jb = j; }
    if (chn) {  // same for every pixel: warp-uniform branch
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (!(chn & (1u << k))) continue;
        fixed_taps<TS>(st.row(k), SWp,
                       chk(st.cbase + s_o[chk(jn * a.KP + k, 0, a.D * a.KP - 1, a.status)], 0, a.SW - 2, a.status),
                       (S >> k) & 1u, lin, ref1, ref2, b1[k],
                       b2[k], s1[k], s2[k], ac[k], q0[k]);
      }
      B1 = b1[0];
      B2 = b2[0];
      BQ = q0[0];
#pragma unroll
      for (int k = 1; k < K; ++k) {
        B1 = fadd2(B1, b1[k]);
        B2 = fadd2(B2, b2[k]);
        BQ += q0[k];
      }
    }
  }
  if (best_out) *best_out = best;
  return jb;
}

template <int K, typename TS, int REF>
__device__ __forceinline__ int m_step_fixed(const SweepArgs& a, const Staged<TS>& st, const float2* s_wq,
                                            const int* s_o, const unsigned* s_chg, const float* s_d,
                                            const float* s_rcp, float cy, float cx, float cz, float mu,
                                            bool inside, unsigned S) {
  return m_step_fixed_range<K, TS, REF>(a, st, s_wq, s_o, s_chg, s_d, s_rcp, cy, cx, cz, mu, inside, S, 0, a.D,
                                   nullptr);
}

// First-iteration labels of one pixel when they are the same for every
// candidate: bit k of *mask is camera k's label (static) and the return value
// says whether every camera's T texels stay clear of the threshold.  The same
// scan over each camera's sample range gives *seg_max = sum over cameras of
// the largest max(log p(static), log p(dynamic)) among the texels its rays
// interpolate, an upper bound (up to rounding) of the segmentation term of
// any label vector at any candidate; max(ls, ld) is formed as ls + max(T, 0)
// from the stored T = ld - ls.
template <int K, typename TS>
__device__ __forceinline__ bool constant_initial_labels(const SweepArgs& a, const Staged<TS>& st,
                                                        unsigned* mask, float* seg_max) {
  bool all = true;
  unsigned m = 0;
  float segsum = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint8_t* R = st.row(k);
    float lo = INFINITY, hi = -INFINITY, smax = -INFINITY;
    const int c_lo = chk(st.cbase + a.omin[k], 0, a.SW - 1, a.status);
    const int c_hi = chk(st.cbase + a.omax[k] + 1, 0, a.SW - 1, a.status);
    for (int c = c_lo; c <= c_hi; ++c) {
      const float z = Texels<TS>::t(R, st.SWp, c);
      lo = fminf(lo, z);
      hi = fmaxf(hi, z);
      smax = fmaxf(smax, Texels<TS>::ls(R, st.SWp, c) + fmaxf(z, 0.f));
    }
    if (hi < a.log_thr - kThresholdMargin) m |= 1u << k;
    else if (!(lo >= a.log_thr + kThresholdMargin)) all = false;
    segsum += smax;
  }
  *mask = m;
  *seg_max = segsum;
  return all;
}

// ------------------------------------------------------ candidate pruning
// With the variance clamped at 0 and beta >= 0, the objective of candidate j
// (either M-step) is at most  pin * prior(j) + seg(j)  (rounding is
// monotone), prior the log prior (evaluated in base 2 and scaled by ln 2) and
// seg(j) at most the pixel's seg_max.  Outside the triangulation (pin = 0)
// nothing is pruned.  Given J* = the objective of one candidate j*, computed by the same
// code the M-step runs, every candidate whose bound is below J* is beaten by
// j* and cannot be the arg-max (nor tie with it); the arg-max over the
// remaining candidates, lowest index on ties, is the arg-max over all D.
// The prior is unimodal in |d - mu|, so the candidates that remain form one
// interval around mu: with the prior in natural-log units, log(gamma +
// exp(-(d_j - mu)^2 / (2 sigma^2))) >= th  <=>  (d_j - mu)^2 <= -2 sigma^2
// log(e^th - gamma).  Slacks make the interval wider, never narrower, than
// the exact one: th is lowered by 1e-3 (the hardware exponential and
// logarithm err by about 1e-6 relative), J* by 2^-18 (1 + |J*|), the radius is
// widened by 0.1 % + 1e-3, the index range by one candidate on each side, and
// seg_max carries a margin for the rounding of the segmentation sums
// (a.seg_margin, set by the host).  j* itself is always kept.  Where th is
// below about -87, e^th would leave float32's normal range and its log would
// no longer be th, so nothing is pruned there (whatever the prior's
// exponential does with results below the normal range).
__device__ __forceinline__ int nearest_candidate(const SweepArgs& a, float mu) {
  const float f = fminf(fmaxf((mu - a.d0) * a.inv_step, 0.f), static_cast<float>(a.D - 1));
  return static_cast<int>(rintf(f));
}

// The interval in natural-log units (the objective's prior term is
// log(gamma + exp(-(d - mu)^2 / (2 sigma^2)))); d_j = d0 + j / inv_step.
__device__ __forceinline__ void prune_interval(float mu, float Js, float seg_ub, float gamma, float inv2s2, float d0,
                                               float inv_step, int D, int js, int& lo, int& hi) {
  lo = 0;
  hi = D - 1;
  if (!(fabsf(Js) <= 3.0e38f)) return;  // no finite objective to bound against
  const float th = Js - (1.f + fabsf(Js)) * 0x1p-18f - seg_ub - 1e-3f;
  // below about -87 exp(th) leaves float32's normal range and its log is no
  // longer th: keep every candidate there
  if (!(th >= -87.f)) return;
  const float A = expf(th) - gamma;
  if (!(A > 0.f && A < 1.f)) return;  // every candidate's prior reaches th (A >= 1 cannot happen)
  const float r = sqrtf(-logf(A) / inv2s2) * 1.001f + 1e-3f;
  const float flo = fmaxf((mu - r - d0) * inv_step, -2.f);
  const float fhi = fminf((mu + r - d0) * inv_step, static_cast<float>(D) + 1.f);
  lo = min(max(static_cast<int>(floorf(flo)) - 1, 0), js);
  hi = max(min(static_cast<int>(ceilf(fhi)) + 1, D - 1), js);
}

__device__ __forceinline__ void prune_range(const SweepArgs& a, float mu, float Js, float seg_ub, int js, int& lo,
                                            int& hi) {
  prune_interval(mu, Js, seg_ub, a.gamma, a.inv2s2, a.d0, a.inv_step, a.D, js, lo, hi);
}

// Stable counting sort of the tile pixels (thread tid = tile pixel) whose
// pred is set, by key in [0, NB): list[0 .. n) = their tile indices in (key,
// tid) order; returns n (the same in every thread).  s_cnt: NB x warps
// 16-bit counters, zero on entry and left zero on exit (each thread clears
// the counters it scanned once the list is written; the next call comes
// after another __syncthreads); s_tot: one int per warp.  Four
// __syncthreads.
__device__ __forceinline__ int sort_pixels(bool pred, int key, int NB, int16_t* list, uint16_t* s_cnt,
                                           int* s_tot) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int ncnt = NB * nw, per = (ncnt + blockDim.x - 1) / blockDim.x;
  const unsigned act = __ballot_sync(0xffffffffu, pred);
  int rank = 0;
  if (pred) {
    const unsigned peers = __match_any_sync(act, key);
    rank = __popc(peers & ((1u << lane) - 1u));
    if (rank == 0) s_cnt[key * nw + warp] = static_cast<uint16_t>(__popc(peers));
  }
  __syncthreads();
  // exclusive scan over the counters in (key, warp) order; thread tid owns
  // counters [tid * per, (tid + 1) * per)
  int loc = 0;
  for (int q = 0; q < per; ++q) {
    const int i = tid * per + q;
    if (i < ncnt) loc += s_cnt[i];
  }
  int incl = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_tot[warp] = incl;
  __syncthreads();
  int run = incl - loc, total = 0;
  for (int w = 0; w < nw; ++w) {
    const int t = s_tot[w];
    run += w < warp ? t : 0;
    total += t;
  }
  for (int q = 0; q < per; ++q) {
    const int i = tid * per + q;
    if (i < ncnt) {
      const int c = s_cnt[i];
      s_cnt[i] = static_cast<uint16_t>(run);
      run += c;
    }
  }
  __syncthreads();
  if (pred) list[s_cnt[key * nw + warp] + rank] = static_cast<int16_t>(tid);
  __syncthreads();
  for (int q = 0; q < per; ++q) {
    const int i = tid * per + q;
    if (i < ncnt) s_cnt[i] = 0;
  }
  return total;
}

// Sort keys of the bound intervals: pixels whose interval covers more than a
// quarter of the candidates come after the others, each class in 16 buckets
// of the interval's first candidate (NB = 32); in the first M-step the
// pixels whose labels do not depend on the candidate come first (NB = 64).
constexpr int kLoBuckets = 16;
static_assert(4 * kLoBuckets <= kSortKeys, "first-pass sort keys");
__device__ __forceinline__ int interval_key(int lo, int hi, int D) {
  const int wide = (hi - lo + 1) * 4 > D ? 1 : 0;
  return wide * kLoBuckets + (lo * kLoBuckets) / D;
}

// ---------------------------------------------------------------- E-step
struct Rays {
  // per camera: shifted descriptors, |g|^2, log p(static) - log p(dynamic)
  float gy[kMaxCams], gx[kMaxCams], gz[kMaxCams], qk[kMaxCams], ak[kMaxCams];
  float base;  // sum_k log p(dynamic)
};

template <int K, typename TS>
__device__ __forceinline__ void sample_rays(const SweepArgs& a, const Staged<TS>& st, const float2* s_wq,
                                            const int* s_o, int jt, float cy, float cx, float cz,
                                            Rays& r) {
  using Tx = Texels<TS>;
  const int SWp = st.SWp;
  const float2 ref1 = make_float2(-cy, -cx), ref2 = make_float2(-cz, 0.f);
  r.base = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int jk = chk(jt * a.KP + k, 0, a.D * a.KP - 1, a.status);
    const float w = s_wq[jk].x;
    const int c = chk(st.cbase + s_o[jk], 0, a.SW - 2, a.status);
    const uint8_t* R = st.row(k);
    float2 yx0, zd0, yx1, zd1;
    Tx::quad(R, SWp, c, yx0, zd0);
    Tx::quad(R, SWp, c + 1, yx1, zd1);
    const float S0 = Tx::ls(R, SWp, c), S1 = Tx::ls(R, SWp, c + 1);
    const float2 ww = make_float2(w, w);
    const float2 g1 = ffma2(ww, fsub2(yx1, yx0), fadd2(yx0, ref1));  // (gy, gx)
    const float2 g2 = ffma2(ww, fsub2(zd1, zd0), fadd2(zd0, ref2));  // (gz, ld)
    const float ls = fmaf(w, S1 - S0, S0);
    r.gy[k] = g1.x; r.gx[k] = g1.y; r.gz[k] = g2.x;
    r.qk[k] = fmaf(g2.x, g2.x, fmaf(g1.y, g1.y, g1.x * g1.x));
    r.ak[k] = ls - g2.y;
    r.base += g2.y;
  }
}

struct Acc {
  float sy, sx, sz, q, sa;
};

// Leaf evaluation shared by the arg-max and the posterior passes so that both
// see bit-identical objectives.  The variance is clamped at 0 (as in the
// M-steps), so a leaf's objective is at most base + its segmentation sum: the
// bound of the E-step's block pruning.
__device__ __forceinline__ float leaf_objective(const Acc& acc, float rn, float base, float beta) {
  const float ss = fmaf(acc.sz, acc.sz, fmaf(acc.sx, acc.sx, acc.sy * acc.sy));
  const float var = fmaxf(fmaf(-ss, rn, acc.q) * rn, 0.f);
  return fmaf(-beta, var, base + acc.sa);
}

template <int L>
struct EnumState {
  float best;        // arg-max pass: best objective so far
  unsigned bmask;    // arg-max pass: its mask
  float emax;        // posterior pass: the maximum objective
  float Z;           // posterior pass: partition sum of this high block
  float pl[L > 0 ? L : 1];  // posterior pass: mass on each low camera
};

// Depth-first over cameras k, k-1, ..., 0 of the low block; the "without
// camera k" subtree first so leaves come in increasing mask order.
// MODE 0: arg-max (first maximum kept); MODE 1: accumulate exp(J - Jmax).
template <int MODE, int L, int k, int N, unsigned MASK>
__device__ __forceinline__ void enum_low(const Rays& r, const Acc& acc, const float (&rnv)[L + 1],
                                         unsigned high, float beta, EnumState<L>& s) {
  if constexpr (k < 0) {
    const float E = leaf_objective(acc, rnv[N], r.base, beta);
    if constexpr (MODE == 0) {
      if (E > s.best) { s.best = E; s.bmask = high | MASK; }
    } else {
      const float e = ex2_approx((E - s.emax) * 1.4426950408889634f);  // exp(E - Emax) <= 1
      s.Z += e;
#pragma unroll
      for (int i = 0; i < L; ++i)
        if (MASK >> i & 1u) s.pl[i] += e;
    }
  } else {
    enum_low<MODE, L, k - 1, N, MASK>(r, acc, rnv, high, beta, s);
    const Acc a2{acc.sy + r.gy[k], acc.sx + r.gx[k], acc.sz + r.gz[k], acc.q + r.qk[k], acc.sa + r.ak[k]};
    enum_low<MODE, L, k - 1, N + 1, MASK | (1u << k)>(r, a2, rnv, high, beta, s);
  }
}

// Up to five cameras the subset tree runs on float32x2 pairs: lane .x holds
// the label vectors without camera 0, lane .y the same vector with camera 0,
// so each internal node adds camera k to both with one packed add per sum
// and each pair of leaves (masks m, m | 1) evaluates its two objectives with
// packed operations (each lane the scalar leaf's IEEE operations).  A
// vector's sums add camera 0 first, then the others from the highest down;
// the group form (enumerate_group) forms them in the same order, so both
// give the same bits.
constexpr int kPairEnumMaxCams = 5;

struct Acc2 {
  float2 sy, sx, sz, q, sa;
};

// the rays of cameras 1..K-1 duplicated into both lanes
template <int K>
struct DupRays {
  float2 gy[K], gx[K], gz[K], qk[K], ak[K];
};

template <int MODE, int K, int k, int N, unsigned MASK>
__device__ __forceinline__ void enum_pair(const DupRays<K>& dr, const Acc2& acc, const float2 (&rnp)[K],
                                          const float2 (&nrnp)[K], float2 nbeta, float2 base2, float2 nemax2,
                                          EnumState<K>& s) {
  if constexpr (k < 1) {
    const float2 ss = ffma2(acc.sz, acc.sz, ffma2(acc.sx, acc.sx, fmul2(acc.sy, acc.sy)));
    float2 var = fmul2(ffma2(ss, nrnp[N], acc.q), rnp[N]);
    var = make_float2(fmaxf(var.x, 0.f), fmaxf(var.y, 0.f));
    const float2 E = ffma2(nbeta, var, fadd2(base2, acc.sa));
    if constexpr (MODE == 0) {
      if (E.x > s.best) { s.best = E.x; s.bmask = MASK; }
      if (E.y > s.best) { s.best = E.y; s.bmask = MASK | 1u; }
    } else {
      const float2 t = fmul2(fadd2(E, nemax2), make_float2(1.4426950408889634f, 1.4426950408889634f));
      const float e0 = ex2_approx(t.x), e1 = ex2_approx(t.y);  // exp(E - Emax) <= 1
      s.Z += e0;
#pragma unroll
      for (int i = 1; i < K; ++i)
        if (MASK >> i & 1u) s.pl[i] += e0;
      s.Z += e1;
      s.pl[0] += e1;
#pragma unroll
      for (int i = 1; i < K; ++i)
        if (MASK >> i & 1u) s.pl[i] += e1;
    }
  } else {
    enum_pair<MODE, K, k - 1, N, MASK>(dr, acc, rnp, nrnp, nbeta, base2, nemax2, s);
    const Acc2 a2{fadd2(acc.sy, dr.gy[k]), fadd2(acc.sx, dr.gx[k]), fadd2(acc.sz, dr.gz[k]), fadd2(acc.q, dr.qk[k]),
                  fadd2(acc.sa, dr.ak[k])};
    enum_pair<MODE, K, k - 1, N + 1, MASK | (1u << k)>(dr, a2, rnp, nrnp, nbeta, base2, nemax2, s);
  }
}

template <int MODE, int K>
__device__ __forceinline__ void enumerate_pairs(const Rays& r, const float* s_rcp, float beta, float emax,
                                                unsigned& bmask, float& best, float* post) {
  DupRays<K> dr;
#pragma unroll
  for (int k = 1; k < K; ++k) {
    dr.gy[k] = make_float2(r.gy[k], r.gy[k]);
    dr.gx[k] = make_float2(r.gx[k], r.gx[k]);
    dr.gz[k] = make_float2(r.gz[k], r.gz[k]);
    dr.qk[k] = make_float2(r.qk[k], r.qk[k]);
    dr.ak[k] = make_float2(r.ak[k], r.ak[k]);
  }
  float2 rnp[K], nrnp[K];  // (1/n, 1/(n + 1)) of the leaf pairs with n cameras besides camera 0
#pragma unroll
  for (int n = 0; n < K; ++n) {
    rnp[n] = make_float2(s_rcp[n], s_rcp[n + 1]);
    nrnp[n] = make_float2(-rnp[n].x, -rnp[n].y);
  }
  EnumState<K> s;
  s.best = -INFINITY;
  s.bmask = 0;
  s.emax = emax;
  s.Z = 0.f;
#pragma unroll
  for (int i = 0; i < K; ++i) s.pl[i] = 0.f;
  const Acc2 root{make_float2(0.f, r.gy[0]), make_float2(0.f, r.gx[0]), make_float2(0.f, r.gz[0]),
                  make_float2(0.f, r.qk[0]), make_float2(0.f, r.ak[0])};
  enum_pair<MODE, K, K - 1, 0, 0u>(dr, root, rnp, nrnp, make_float2(-beta, -beta), make_float2(r.base, r.base),
                                   make_float2(-emax, -emax), s);
  if constexpr (MODE == 0) {
    bmask = s.bmask;
    best = s.best;
  } else {
    const float inv = 1.f / s.Z;
#pragma unroll
    for (int i = 0; i < K; ++i) post[i] = s.pl[i] * inv;
  }
}

// Block pruning of the E-step arg-max from seven cameras: the label vectors
// sharing high mask h (cameras >= L) form a block of 2^L leaves whose
// objectives are at most base + sa_h + sum_{k < L} max(a_k, 0) (the variance
// term is <= 0; sa_h the block's segmentation sum over its high cameras, a_k
// = log p(static) - log p(dynamic) of low camera k), plus a margin for the
// float32 rounding of the sums (at most L + 2 roundings of numbers of
// magnitude below 1 + |base| + |sa_h| + sum |a_k|; the margin is 2^-20 times
// that).  A block whose bound is below the objective of one leaf evaluated
// the same way -- the all-static vector, the usual winner -- holds neither the
// arg-max nor a tie with it, and is skipped.
template <int L>
struct BlockBound {
  float seed, pos, mag;
  template <int K>
  __device__ __forceinline__ void init(const Rays& r, const float* s_rcp, float beta) {
    constexpr int NH = K - L;
    // the all-static leaf, summed in the enumeration's order: high cameras
    // upwards, then the low subset tree from camera L - 1 down
    Acc acc{0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      acc.sy += r.gy[L + i]; acc.sx += r.gx[L + i]; acc.sz += r.gz[L + i];
      acc.q += r.qk[L + i]; acc.sa += r.ak[L + i];
    }
#pragma unroll
    for (int k = L - 1; k >= 0; --k) {
      acc.sy += r.gy[k]; acc.sx += r.gx[k]; acc.sz += r.gz[k];
      acc.q += r.qk[k]; acc.sa += r.ak[k];
    }
    seed = leaf_objective(acc, s_rcp[K], r.base, beta);
    pos = 0.f;
    mag = 1.f + fabsf(r.base);
#pragma unroll
    for (int k = 0; k < L; ++k) {
      pos += fmaxf(r.ak[k], 0.f);
      mag += fabsf(r.ak[k]);
    }
  }
  __device__ __forceinline__ bool skip(float base, float sa_h) const {
    const float ub = (base + sa_h + pos) + (mag + fabsf(sa_h)) * 0x1p-20f;
    return ub < seed;
  }
};

// Full enumeration: cameras >= L form a runtime loop over "high" masks (sums
// built from scratch), cameras < L the unrolled subset tree.
// prune: skip blocks by BlockBound (arg-max pass, from seven cameras).
template <int MODE, int K>
__device__ __forceinline__ void enumerate(const Rays& r, const float* s_rcp, float beta, float emax,
                                          unsigned& bmask, float& best, float* post, bool prune = false) {
  if constexpr (K <= kPairEnumMaxCams) {
    enumerate_pairs<MODE, K>(r, s_rcp, beta, emax, bmask, best, post);
    return;
  }
  constexpr int L = K < 6 ? K : 6;
  constexpr int NH = K - L;
  float ph[NH > 0 ? NH : 1];
#pragma unroll
  for (int i = 0; i < (NH > 0 ? NH : 1); ++i) ph[i] = 0.f;
  EnumState<L> s;
  s.best = -INFINITY;
  s.bmask = 0;
  s.emax = emax;
#pragma unroll
  for (int i = 0; i < (L > 0 ? L : 1); ++i) s.pl[i] = 0.f;
  float Ztot = 0.f;
  BlockBound<L> bb;
  if constexpr (MODE == 0 && NH > 0)
    if (prune) bb.template init<K>(r, s_rcp, beta);
  for (unsigned h = 0; h < (1u << NH); ++h) {
    Acc acc{0.f, 0.f, 0.f, 0.f, 0.f};
    int nh = 0;
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      if (h >> i & 1u) {
        acc.sy += r.gy[L + i]; acc.sx += r.gx[L + i]; acc.sz += r.gz[L + i];
        acc.q += r.qk[L + i]; acc.sa += r.ak[L + i];
        ++nh;
      }
    }
    if constexpr (MODE == 0 && NH > 0)
      if (prune && bb.skip(r.base, acc.sa)) continue;
    float rnv[L + 1];
#pragma unroll
    for (int i = 0; i <= L; ++i) rnv[i] = s_rcp[nh + i];
    s.Z = 0.f;
    enum_low<MODE, L, L - 1, 0, 0u>(r, acc, rnv, h << L, beta, s);
    if constexpr (MODE == 1) {
      Ztot += s.Z;
#pragma unroll
      for (int i = 0; i < NH; ++i)
        if (h >> i & 1u) ph[i] += s.Z;
    }
  }
  if constexpr (MODE == 0) {
    bmask = s.bmask;
    best = s.best;
  } else {
    const float inv = 1.f / Ztot;
#pragma unroll
    for (int i = 0; i < L; ++i) post[i] = s.pl[i] * inv;
#pragma unroll
    for (int i = 0; i < NH; ++i) post[L + i] = ph[i] * inv;
  }
}

// Cooperative forms for the last pixels of a tile still iterating (used by
// the calibrated sweep and the soft EM; the rectified sweep keeps one lane
// per pixel): a group of G lanes (G a power of two, up to the warp) takes
// one pixel, splits its candidates and then its label vectors, and reduces
// with the same tie rules as the one-thread sweep (lowest candidate,
// smallest mask), so the result is bit-identical.

// Larger objective, or on a tie the lower index, over the G lanes of each
// aligned group (every lane of the warp takes part).
__device__ __forceinline__ void group_argmax(float& best, unsigned& idx, int G) {
  for (int off = G >> 1; off > 0; off >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, off);
    const unsigned oi = __shfl_xor_sync(0xffffffffu, idx, off);
    if (ob > best || (ob == best && oi < idx)) {
      best = ob;
      idx = oi;
    }
  }
}

// Arg-max of the E-step by lane gl of a group of G.  Up to six cameras each
// lane takes masks gl, gl + G, ... and forms their sums from scratch in the
// subset tree's order (the low block from its highest camera down); from
// seven, each lane takes high masks gl, gl + G, ... of the tree's outer loop
// and runs its inner subset tree as is.  Either way the objectives equal the
// one-thread enumeration's bit for bit.
template <int K>
__device__ __forceinline__ void enumerate_group(const Rays& r, const float* s_rcp, float beta, int gl, int G,
                                                unsigned& bmask, float& best, bool prune = false) {
  constexpr int L = K < 6 ? K : 6;
  constexpr int NH = K - L;
  float b = -INFINITY;
  unsigned bm = gl == 0 ? 0u : 0xffffffffu;  // all objectives -inf: mask 0, as the one-thread form
  if constexpr (NH == 0) {
    for (unsigned m = gl; m < (1u << K); m += G) {
      Acc acc{0.f, 0.f, 0.f, 0.f, 0.f};
      // the order of the one-thread tree: up to five cameras (float32x2
      // pairs) camera 0 first, then the others from the highest down;
      // six cameras from the highest down
      constexpr bool pairs = K <= kPairEnumMaxCams;
      if (pairs && (m & 1u)) acc = Acc{r.gy[0], r.gx[0], r.gz[0], r.qk[0], r.ak[0]};
#pragma unroll
      for (int k = L - 1; k >= (pairs ? 1 : 0); --k)
        if (m >> k & 1u) {
          acc.sy += r.gy[k]; acc.sx += r.gx[k]; acc.sz += r.gz[k]; acc.q += r.qk[k]; acc.sa += r.ak[k];
        }
      const float E = leaf_objective(acc, s_rcp[__popc(m)], r.base, beta);
      if (E > b) { b = E; bm = m; }
    }
  } else {
    EnumState<L> s;
    s.best = -INFINITY;
    s.bmask = bm;
    s.emax = 0.f;
    BlockBound<L> bb;
    if (prune) bb.template init<K>(r, s_rcp, beta);
    for (unsigned h = gl; h < (1u << NH); h += G) {
      Acc acc{0.f, 0.f, 0.f, 0.f, 0.f};
      int nh = 0;
#pragma unroll
      for (int i = 0; i < NH; ++i) {
        if (h >> i & 1u) {
          acc.sy += r.gy[L + i]; acc.sx += r.gx[L + i]; acc.sz += r.gz[L + i];
          acc.q += r.qk[L + i]; acc.sa += r.ak[L + i];
          ++nh;
        }
      }
      if (prune && bb.skip(r.base, acc.sa)) continue;
      float rnv[L + 1];
#pragma unroll
      for (int i = 0; i <= L; ++i) rnv[i] = s_rcp[nh + i];
      enum_low<0, L, L - 1, 0, 0u>(r, acc, rnv, h << L, beta, s);
    }
    b = s.best;
    bm = s.bmask;
  }
  group_argmax(b, bm, G);
  bmask = bm;
  best = b;
}

// Element c of the pixel at p (an image of dtype a.dtype), unscaled.
__device__ __forceinline__ float pixel_element(const uint8_t* p, int c, int dtype) {
  if (dtype == 0) return static_cast<float>(p[c]);
  if (dtype == 1) return reinterpret_cast<const float*>(p)[c];
  if (dtype == 2) return __half2float(reinterpret_cast<const __half*>(p)[c]);
  return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[c]);
}

// Outputs of a reference pixel that the dynamic-only mode does not
// reconstruct: disparity from the prior centre mu (nearest candidate, lower
// on a tie; -1 / NaN outside the triangulation), no static ray, no
// posteriors (NaN).  The refocused value (the reference image) is written by
// the caller when the refocus is fused.
template <int K>
__device__ __forceinline__ void write_static_pixel(const SweepArgs& a, int u, int v, float mu) {
  const size_t pix = static_cast<size_t>(v) * a.W + u;
  int j = -1;
  if (!isnan(mu)) {
    j = 0;
    float bd = fabsf(a.dval[0] - mu);
    for (int i = 1; i < a.D; ++i) {
      const float dd = fabsf(a.dval[i] - mu);
      if (dd < bd) { bd = dd; j = i; }
    }
  }
  const float nan = __int_as_float(0x7fc00000);
  a.d_idx[pix] = j;
  if (a.d_out) a.d_out[pix] = j >= 0 ? a.dval[j] : nan;
  if (a.labels) a.labels[pix] = 0;
  if (a.post) {
    const size_t HW = static_cast<size_t>(a.H) * a.W;
#pragma unroll
    for (int k = 0; k < K; ++k) a.post[k * HW + pix] = nan;
  }
}

// Dynamic-only mode, before the sweep: one CTA per tile.  A tile with a
// reference pixel whose P(dynamic) reaches the threshold is appended to the
// list the sweep walks; the pixels of every other tile get their outputs here.
template <int K>
__global__ void tile_classify_kernel(const SweepArgs a, const float* seg_prior, size_t p_pitch, int* tile_list,
                                     int* n_tiles) {
  const int tiles_x = (a.W + a.TW - 1) / a.TW;
  const int tile = blockIdx.x, u0 = (tile % tiles_x) * a.TW, v0 = (tile / tiles_x) * a.TR;
  const int u = u0 + threadIdx.x % a.TW, v = v0 + threadIdx.x / a.TW;
  const bool valid = u < a.W && v < a.H;
  bool dyn = false;
  float mu = __int_as_float(0x7fc00000);
  if (valid) {
    const float* row = reinterpret_cast<const float*>(reinterpret_cast<const uint8_t*>(seg_prior) +
                                                      (static_cast<size_t>(a.ref) * a.H + v) * p_pitch);
    dyn = row[u] >= a.seg_threshold;
    const size_t pix = static_cast<size_t>(v) * a.W + u;
    if (a.ptris) {  // fused prior: this kernel rasterises it for the whole frame
      mu = prior::prior_pixel(a.ptris, a.pbin_start, a.pbin_items, a.pnbx, u, v);
      a.mu_out[pix] = mu;
    } else {
      mu = a.mu[pix];
    }
  }
  if (__syncthreads_or(dyn)) {
    if (threadIdx.x == 0) tile_list[atomicAdd(n_tiles, 1)] = tile;
  } else if (valid) {
    write_static_pixel<K>(a, u, v, mu);
    if (a.refocus_out) {  // fused refocus: a pixel with no static ray keeps the reference image
      const uint8_t* p = a.img + (static_cast<size_t>(a.ref) * a.H + v) * a.img_pitch + static_cast<size_t>(u) * a.bpp;
      const float scale = a.dtype == 0 ? (1.f / 255.f) : 1.f;
      for (int c = 0; c < a.C; ++c)
        a.refocus_out[(static_cast<size_t>(v) * a.W + u) * a.C + c] = pixel_element(p, c, a.dtype) * scale;
    }
  }
}

template <int K>
cudaError_t launch_tile_classify_k(const SweepArgs& a, const float* seg_prior, size_t p_pitch, int* tile_list,
                                   int* n_tiles, cudaStream_t s) {
  const int tiles = ((a.W + a.TW - 1) / a.TW) * ((a.H + a.TR - 1) / a.TR);
  tile_classify_kernel<K><<<tiles, a.TR * a.TW, 0, s>>>(a, seg_prior, p_pitch, tile_list, n_tiles);
  return cudaGetLastError();
}

// ------------------------------------------------------- tile bookkeeping
// Everything one thread needs to run the EM of pixel p of the tile.
template <typename TS>
struct PixelCtx {
  int u, v;
  bool valid, inside;
  float mu, cy, cx, cz;
  Staged<TS> st;
};

// s_mu: the tile's prior centres when the prior is fused, else NULL (read mu).
template <typename TS>
__device__ __forceinline__ PixelCtx<TS> load_pixel(const SweepArgs& a, const uint8_t* s_feat, int u0, int v0,
                                                   int cam_stride, int p, const float* s_mu = nullptr) {
  PixelCtx<TS> c;
  p = chk(p, 0, a.TR * a.TW - 1, a.status);
  const int r = p / a.TW, tx = p - r * a.TW;
  c.u = u0 + tx;
  c.v = v0 + r;
  c.valid = (c.u < a.W) && (c.v < a.H);
  c.mu = s_mu ? s_mu[p] : a.mu[static_cast<size_t>(min(c.v, a.H - 1)) * a.W + min(c.u, a.W - 1)];
  c.inside = !isnan(c.mu);
  c.st.F = s_feat + static_cast<size_t>(r) * a.SWp * texel_bytes(a.prec);
  c.st.cam_stride = cam_stride;
  c.st.SWp = a.SWp;
  c.st.cbase = tx + a.L;
  float2 yx, zd;
  Texels<TS>::quad(c.st.row(a.ref), a.SWp, c.st.cbase, yx, zd);
  c.cy = yx.x;
  c.cx = yx.y;
  c.cz = zd.x;
  return c;
}

// Stable CTA-wide compaction: the threads (tile pixel p = threadIdx.x) with
// pred set write p to list[base + rank]; returns how many did (every thread
// gets the same count).  Contains two __syncthreads.
__device__ __forceinline__ int compact_value(bool pred, int value, int16_t* list, int base, int* s_wcnt) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const unsigned b = __ballot_sync(0xffffffffu, pred);
  if (lane == 0) s_wcnt[warp] = __popc(b);
  __syncthreads();
  int off = 0, total = 0;
  for (int w = 0; w < nw; ++w) {
    const int c = s_wcnt[w];
    off += w < warp ? c : 0;
    total += c;
  }
  if (pred) list[base + off + __popc(b & ((1u << lane) - 1u))] = static_cast<int16_t>(value);
  __syncthreads();
  return total;
}
__device__ __forceinline__ int compact(bool pred, int16_t* list, int base, int* s_wcnt) {
  return compact_value(pred, static_cast<int>(threadIdx.x), list, base, s_wcnt);
}

// ---------------------------------------------------------------- kernel
// Launch shapes the sweep kernels are compiled for (minimum resident CTAs
// per SM requested from the register allocator).  Up to eight cameras: CTAs
// of at most 256 threads, two per SM (at most 128 registers).  From nine
// cameras the register taps and the wider E-step need more than 128
// registers: the single-frame kernel takes CTAs of at most 128 threads,
// three per SM (at most 168 registers, no spills) up to eleven cameras and
// two for twelve; the persistent kernel keeps 256-thread CTAs, one per SM,
// because its wide-halo frames are bound by shared memory, where a 128-thread
// CTA would leave half the warps.
template <int K>
constexpr int sweep_min_blocks() {
  return K <= 8 ? 2 : K <= 11 ? 3 : 2;
}
template <int K>
constexpr int persistent_min_blocks() {
  return K <= 8 ? 2 : 1;
}

// Luminance of an 8-bit RGB pixel on [0, 1] (BT.601 weights).
__device__ __forceinline__ float luma_u8(unsigned R, unsigned G, unsigned B) {
  return fmaf(0.114f, static_cast<float>(B), fmaf(0.587f, static_cast<float>(G), 0.299f * static_cast<float>(R))) *
         (1.f / 255.f);
}

// Fused prior of one tile (Sec. III-C "Disparity Prior"), one thread per
// tile pixel: the triangles of the 16 x 16 bins the tile covers are copied
// into shared memory first (three rounds of dependent global loads for the
// whole CTA instead of a chain per pixel), in bin order, so every pixel scans
// exactly the list it would scan in global memory.  scratch: shared memory
// that nothing uses until the staged maps are written (the map region).  A
// tile whose bins or
// triangles do not fit scans global memory instead (same result).  Writes
// mu_out and s_mu (NaN outside the triangulation); contains two
// __syncthreads.
constexpr int kTilePriorBins = 32;
__device__ __forceinline__ void tile_prior(const SweepArgs& a, int u0, int v0, uint8_t* scratch,
                                           size_t scratch_bytes, float* s_mu) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int bx0 = u0 / kBinSize, bx1 = min(u0 + a.TW - 1, a.W - 1) / kBinSize;
  const int by0 = v0 / kBinSize, by1 = min(v0 + a.TR - 1, a.H - 1) / kBinSize;
  const int nbx = bx1 - bx0 + 1, nb = nbx * (by1 - by0 + 1);
  int* s_off = reinterpret_cast<int*>(scratch);            // [kTilePriorBins + 1] first slot of each bin
  int* s_beg = s_off + kTilePriorBins + 1;                 // [kTilePriorBins] its first item in bin_items
  int* s_ok = s_beg + kTilePriorBins;                      // the staged lists are usable
  const size_t head = align_up((2 * kTilePriorBins + 2) * sizeof(int), 16);
  PriorTri* s_tri = reinterpret_cast<PriorTri*>(scratch + head);
  const int cap = scratch_bytes > head ? static_cast<int>((scratch_bytes - head) / sizeof(PriorTri)) : 0;
  if (tid < 32) {
    int cnt = 0, beg = 0;
    if (tid < nb && nb <= kTilePriorBins) {
      const int bin = (by0 + tid / nbx) * a.pnbx + bx0 + tid % nbx;
      beg = a.pbin_start[bin];
      cnt = a.pbin_start[bin + 1] - beg;
    }
    int incl = cnt;  // inclusive prefix over the bins
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (tid >= o) incl += y;
    }
    if (tid < nb && nb <= kTilePriorBins) {
      s_off[tid] = incl - cnt;
      s_beg[tid] = beg;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (tid == 0) {
      s_off[min(nb, kTilePriorBins)] = total;
      *s_ok = nb <= kTilePriorBins && total <= cap;
    }
  }
  __syncthreads();
  const bool ok = *s_ok != 0;
  if (ok) {
    const int total = s_off[nb];
    for (int i = tid; i < total; i += nthr) {
      int b = 0;
      while (b + 1 < nb && s_off[b + 1] <= i) ++b;
      const float4* src = reinterpret_cast<const float4*>(a.ptris + a.pbin_items[s_beg[b] + i - s_off[b]]);
      float4* dst = reinterpret_cast<float4*>(s_tri + i);
      static_assert(sizeof(PriorTri) == 48, "a triangle is three 16-byte words");
      dst[0] = src[0];
      dst[1] = src[1];
      dst[2] = src[2];
    }
  }
  __syncthreads();
  const int u = u0 + tid % a.TW, v = v0 + tid / a.TW;
  float m = __int_as_float(0x7fc00000);
  if (u < a.W && v < a.H) {
    if (ok) {
      const int b = chk((v / kBinSize - by0) * nbx + (u / kBinSize - bx0), 0, nb - 1, a.status);
      m = prior::prior_pixel_list(s_tri + s_off[b], s_off[b + 1] - s_off[b], u, v);
    } else {
      m = prior::prior_pixel(a.ptris, a.pbin_start, a.pbin_items, a.pnbx, u, v);
    }
    a.mu_out[static_cast<size_t>(v) * a.W + u] = m;
  }
  s_mu[tid] = m;
}

// Phases 1-2 for tile (tile_x, tile_y) of one frame: raw rows by TMA, then
// descriptors and log priors in shared memory.  The CTA's mbarrier
// (initialised by the caller) completes phase `phase` for this tile's copies.
// load_tables: the frame differs from the previous tile's (tables and
// constants must be staged again).  Returns false (same in every thread) when
// the staging wait timed out; ends with a __syncthreads either way.
template <int K, typename TS>
__device__ __forceinline__ bool stage_tile(const SweepArgs& a, const CUtensorMap* img_map,
                                           const CUtensorMap* p_map, int tile_x, int tile_y, uint8_t* smem,
                                           unsigned phase, bool load_tables, bool maps_in_global) {
  const SmemLayout Ly = sweep_layout(K, a);
  uint8_t* s_img = smem + Ly.raw_img;
  const float* s_p = reinterpret_cast<const float*>(smem + Ly.raw_p);
  float* s_luma = luma_is_raw(a) ? reinterpret_cast<float*>(s_img) : reinterpret_cast<float*>(smem + Ly.luma);
  uint8_t* s_feat = smem + Ly.feat;
  float2* s_wq = reinterpret_cast<float2*>(smem + Ly.wtab);
  int* s_o = reinterpret_cast<int*>(smem + Ly.otab);
  unsigned* s_chg = reinterpret_cast<unsigned*>(smem + Ly.chg);
  float* s_d = reinterpret_cast<float*>(smem + Ly.dval);
  float* s_rcp = reinterpret_cast<float*>(smem + Ly.rcp);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Ly.bar);

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int u0 = tile_x * a.TW, v0 = tile_y * a.TR;
  const int cs = floor16(u0 - a.L - 1);  // first staged raw column (16-px aligned)
  const int W = a.W, H = a.H, RW = a.RW, LR = a.TR + 2;

  // ---- 1. stage raw rows with TMA
  if (tid == 0) {
    if (maps_in_global) {  // descriptors written by copies since their last use
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(img_map) : "memory");
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(p_map) : "memory");
    }
    const unsigned bytes = static_cast<unsigned>(K * LR * RW * a.bpp + K * a.TR * RW * 4);
    mbar_arrive_expect_tx(bar, bytes);
    tma_load_3d(s_img, img_map, cs * a.bpp / 8, v0 - 1, 0, bar);
    tma_load_3d(smem + Ly.raw_p, p_map, cs / 2, v0, 0, bar);
  }
  if (load_tables) {
    for (int i = tid; i < a.D * a.KP; i += nthr) {
      const float w = a.wtab[i];
      s_wq[i] = make_float2(w, w * w);
      s_o[i] = a.otab[i];
    }
    for (int i = tid; i < a.D; i += nthr) {
      s_chg[i] = a.chg[i];
      s_d[i] = a.dval[i];
    }
    if (tid < 16) s_rcp[tid] = tid >= 2 ? 1.f / static_cast<float>(tid) : 0.f;
  }
  if (a.ptris)  // fused prior, computed while the copies are in flight
    tile_prior(a, u0, v0, smem + Ly.feat, Ly.wtab - Ly.feat, reinterpret_cast<float*>(smem + Ly.mu));
  const bool ok = mbar_wait_bounded(bar, phase, a.timeout_ns);
  if (__syncthreads_or(!ok)) {
    if (!ok) {
      atomicOr(a.status, kStatusTmaTimeout);
      mbar_wait_bounded(bar, phase, a.timeout_ns);  // let the copy land before the CTA moves on
    }
    __syncthreads();
    return false;
  }

  // ---- 2. descriptors and log priors (border replicated)
  // luminance of every staged raw pixel; four consecutive pixels per thread
  // for the common input types (same arithmetic per pixel as the general form)
  const int npx = K * LR * RW;  // a multiple of 16 (RW is)
  if (a.dtype == 0 && a.C == 3) {
    for (int q = tid; q < npx / 4; q += nthr) {
      const uint32_t* w = reinterpret_cast<const uint32_t*>(s_img + static_cast<size_t>(q) * 12);
      const uint32_t w0 = w[0], w1 = w[1], w2 = w[2];  // R0 G0 B0 R1 | G1 B1 R2 G2 | B2 R3 G3 B3
      reinterpret_cast<float4*>(s_luma)[q] =
          make_float4(luma_u8(w0 & 0xffu, (w0 >> 8) & 0xffu, (w0 >> 16) & 0xffu),
                      luma_u8(w0 >> 24, w1 & 0xffu, (w1 >> 8) & 0xffu),
                      luma_u8((w1 >> 16) & 0xffu, w1 >> 24, w2 & 0xffu),
                      luma_u8((w2 >> 8) & 0xffu, (w2 >> 16) & 0xffu, w2 >> 24));
    }
  } else if (a.dtype == 0 && a.C == 1) {
    for (int q = tid; q < npx / 4; q += nthr) {
      const uint32_t w = reinterpret_cast<const uint32_t*>(s_img)[q];
      const float sc = 1.f / 255.f;
      reinterpret_cast<float4*>(s_luma)[q] =
          make_float4(static_cast<float>(w & 0xffu) * sc, static_cast<float>((w >> 8) & 0xffu) * sc,
                      static_cast<float>((w >> 16) & 0xffu) * sc, static_cast<float>(w >> 24) * sc);
    }
  } else if (luma_is_raw(a)) {
    // nothing to do: s_luma is s_img
  } else {
    for (int i = tid; i < npx; i += nthr) {
      const uint8_t* px = s_img + static_cast<size_t>(i) * a.bpp;
      float y;
      if (a.dtype == 0) {
        y = a.C == 1 ? static_cast<float>(px[0]) * (1.f / 255.f) : luma_u8(px[0], px[1], px[2]);
      } else if (a.dtype == 1) {
        const float* f = reinterpret_cast<const float*>(px);
        y = a.C == 1 ? f[0] : fmaf(0.114f, f[2], fmaf(0.587f, f[1], 0.299f * f[0]));
      } else {
        float f[3];
        for (int ch = 0; ch < a.C; ++ch)
          f[ch] = a.dtype == 2 ? __half2float(reinterpret_cast<const __half*>(px)[ch])
                               : __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(px)[ch]);
        y = a.C == 1 ? f[0] : fmaf(0.114f, f[2], fmaf(0.587f, f[1], 0.299f * f[0]));
      }
      s_luma[i] = y;
    }
  }
  __syncthreads();
  const int cam_stride = a.TR * a.SWp * texel_bytes(a.prec);
  const int row_bytes = a.SWp * texel_bytes(a.prec);
  if (v0 >= 1 && v0 + a.TR <= H - 1) {
    // no row of the tile touches the top or bottom border: one thread per
    // staged column (k, c) walks its TR rows with a 3-row window of the
    // luminance (3 new values per output); same expressions as below
    for (int item = tid; item < K * a.SW; item += nthr) {
      const int k = item / a.SW, c = item - k * a.SW;
      const int Xc = min(max(u0 - a.L + c, 0), W - 1);
      const int cm = chk(max(Xc - 1, 0) - cs, 0, RW - 1, a.status), c0 = chk(Xc - cs, 0, RW - 1, a.status),
                cp = chk(min(Xc + 1, W - 1) - cs, 0, RW - 1, a.status);
      const float* Lk = s_luma + static_cast<size_t>(k) * LR * RW;
      const float* Pk = s_p + static_cast<size_t>(k) * a.TR * RW + c0;
      uint8_t* Fk = s_feat + static_cast<size_t>(k) * cam_stride;
      float m0 = Lk[cm], z0 = Lk[c0], p0 = Lk[cp];                 // staged row r (image row v0 + r - 1)
      float m1 = Lk[RW + cm], z1 = Lk[RW + c0], p1 = Lk[RW + cp];  // staged row r + 1
      for (int r = 0; r < a.TR; ++r) {
        const float* L2 = Lk + static_cast<size_t>(r + 2) * RW;
        const float m2 = L2[cm], z2 = L2[c0], p2 = L2[cp];
        const float gx = ((p0 + 2.f * p1) + p2) - ((m0 + 2.f * m1) + m2);
        const float gy = ((m2 + 2.f * z2) + p2) - ((m0 + 2.f * z0) + p0);
        const float P = Pk[static_cast<size_t>(r) * RW];
        const float ls = __logf(fmaxf(1.f - P, a.eps)), ld = __logf(fmaxf(P, a.eps));
        Texels<TS>::store(Fk + static_cast<size_t>(r) * row_bytes, a.SWp, c, z1, gx * 0.125f, gy * 0.125f, ls, ld);
        m0 = m1; z0 = z1; p0 = p1;
        m1 = m2; z1 = z2; p1 = p2;
      }
    }
  } else {
    // element (k, r, c) of the K x TR x SW staged maps, walked with a
    // mixed-radix counter (one step = nthr elements; no division in the loop)
    int c = tid % a.SW, r = (tid / a.SW) % a.TR, k = tid / (a.SW * a.TR);
    const int dc = nthr % a.SW, dr = (nthr / a.SW) % a.TR, dk = nthr / (a.SW * a.TR);
    for (; k < K; c += dc, r += dr, k += dk) {
      if (c >= a.SW) { c -= a.SW; ++r; }
      if (r >= a.TR) { r -= a.TR; ++k; }
      if (k >= K) break;
      const int Xc = min(max(u0 - a.L + c, 0), W - 1);
      const int V = min(v0 + r, H - 1);
      const int rm = chk(max(V - 1, 0) - (v0 - 1), 0, LR - 1, a.status), r0 = chk(V - (v0 - 1), 0, LR - 1, a.status),
                rp = chk(min(V + 1, H - 1) - (v0 - 1), 0, LR - 1, a.status);
      const int cm = chk(max(Xc - 1, 0) - cs, 0, RW - 1, a.status), c0 = chk(Xc - cs, 0, RW - 1, a.status),
                cp = chk(min(Xc + 1, W - 1) - cs, 0, RW - 1, a.status);
      const float* Lk = s_luma + static_cast<size_t>(k) * LR * RW;
      const float a00 = Lk[rm * RW + cm], a01 = Lk[rm * RW + c0], a02 = Lk[rm * RW + cp];
      const float a10 = Lk[r0 * RW + cm], a11 = Lk[r0 * RW + c0], a12 = Lk[r0 * RW + cp];
      const float a20 = Lk[rp * RW + cm], a21 = Lk[rp * RW + c0], a22 = Lk[rp * RW + cp];
      const float gx = ((a02 + 2.f * a12) + a22) - ((a00 + 2.f * a10) + a20);
      const float gy = ((a20 + 2.f * a21) + a22) - ((a00 + 2.f * a01) + a02);
      const float P = s_p[(static_cast<size_t>(k) * a.TR + (V - v0)) * RW + c0];
      uint8_t* F = s_feat + static_cast<size_t>(k) * cam_stride + static_cast<size_t>(r) * row_bytes;
      const float ls = __logf(fmaxf(1.f - P, a.eps)), ld = __logf(fmaxf(P, a.eps));
      Texels<TS>::store(F, a.SWp, c, a11, gx * 0.125f, gy * 0.125f, ls, ld);
    }
  }
  {  // the counting sort's counters start at zero (sort_pixels leaves them
     // so), and so do the tile's statistics counters
    uint32_t* z = reinterpret_cast<uint32_t*>(smem + Ly.sortc);
    const int nz = kSortKeys * (nthr >> 5) / 2;
    for (int i = tid; i < nz; i += nthr) z[i] = 0u;
    if (tid < 2) reinterpret_cast<unsigned*>(smem + Ly.wcnt)[32 + tid] = 0u;
  }
  __syncthreads();
  return true;
}

__device__ __forceinline__ float element_value(uint8_t x) { return static_cast<float>(x); }
__device__ __forceinline__ float element_value(float x) { return x; }
__device__ __forceinline__ float element_value(__half x) { return __half2float(x); }
__device__ __forceinline__ float element_value(__nv_bfloat16 x) { return __bfloat162float(x); }

// Eq. 2 for one pixel from the tile's staged raw rows (staged row `row` of
// every camera, first staged column cs): the mean of the static rays' samples
// at its final candidate jb (linear interpolation, column clamped), or the
// reference pixel when no ray is static; elements of type E, C = 1 or 3.
// Same operations in the same order as the standalone refocus kernel.
template <int K, typename E>
__device__ __forceinline__ void refocus_staged(const SweepArgs& a, const uint8_t* s_img, int row, int cs, int u, int jb,
                                               unsigned S, const int* s_o, const float2* s_wq, float* out) {
  const E* img = reinterpret_cast<const E*>(s_img);
  const int C = a.C, RW = a.RW, LR = a.TR + 2;
  const float scale = a.dtype == 0 ? (1.f / 255.f) : 1.f;
  if (S == 0u) {
    const E* px = img + (static_cast<size_t>(a.ref * LR + row) * RW + chk(u - cs, 0, RW - 1, a.status)) * C;
    out[0] = element_value(px[0]) * scale;
    if (C > 1) {
      out[1] = element_value(px[1]) * scale;
      out[2] = element_value(px[2]) * scale;
    }
    return;
  }
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
  int n = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (!(S >> k & 1u)) continue;
    ++n;
    const int o = s_o[jb * a.KP + k];
    const float w = s_wq[jb * a.KP + k].x;
    const int x0 = min(max(u + o, 0), a.W - 1), x1 = min(max(u + o + 1, 0), a.W - 1);
    const E* r = img + static_cast<size_t>(k * LR + row) * RW * C;
    const E* p0 = r + chk(x0 - cs, 0, RW - 1, a.status) * C;
    const E* p1 = r + chk(x1 - cs, 0, RW - 1, a.status) * C;
    {
      const float g0 = element_value(p0[0]), g1 = element_value(p1[0]);
      acc0 += fmaf(w, g1 - g0, g0) * scale;
    }
    if (C > 1) {
      const float g0 = element_value(p0[1]), g1 = element_value(p1[1]);
      acc1 += fmaf(w, g1 - g0, g0) * scale;
      const float h0 = element_value(p0[2]), h1 = element_value(p1[2]);
      acc2 += fmaf(w, h1 - h0, h0) * scale;
    }
  }
  const float inv = 1.f / static_cast<float>(n);
  out[0] = acc0 * inv;
  if (C > 1) {
    out[1] = acc1 * inv;
    out[2] = acc2 * inv;
  }
}

// One tile (tile_x, tile_y) of one frame: stage, run the EM, write the
// outputs.  Staging as in stage_tile.  Ends with a __syncthreads so that the
// next tile may reuse the shared memory.  Returns false (same in every
// thread) when the staging wait timed out.  REF: the reference camera's
// index when the caller guarantees it (a.ref == REF), else -1.
template <int K, typename TS, int REF>
__device__ __forceinline__ bool sweep_tile(const SweepArgs& a, const CUtensorMap* img_map,
                                           const CUtensorMap* p_map, int tile_x, int tile_y, uint8_t* smem,
                                           unsigned phase, bool load_tables, bool maps_in_global) {
  if (!stage_tile<K, TS>(a, img_map, p_map, tile_x, tile_y, smem, phase, load_tables, maps_in_global))
    return false;
  const SmemLayout Ly = sweep_layout(K, a);
  const float* s_p = reinterpret_cast<const float*>(smem + Ly.raw_p);
  const uint8_t* s_feat = smem + Ly.feat;
  const float2* s_wq = reinterpret_cast<const float2*>(smem + Ly.wtab);
  int* s_o = reinterpret_cast<int*>(smem + Ly.otab);
  unsigned* s_chg = reinterpret_cast<unsigned*>(smem + Ly.chg);
  float* s_d = reinterpret_cast<float*>(smem + Ly.dval);
  float* s_rcp = reinterpret_cast<float*>(smem + Ly.rcp);
  const int tid = threadIdx.x;
  const int u0 = tile_x * a.TW, v0 = tile_y * a.TR;
  const int cs = floor16(u0 - a.L - 1);
  const int W = a.W, H = a.H, RW = a.RW;
  const int cam_stride = a.TR * a.SWp * texel_bytes(a.prec);
  const float* s_mu = a.ptris ? reinterpret_cast<const float*>(smem + Ly.mu) : nullptr;

  // ---- 3-5. per-pixel EM.  Before the first M-step the tile's pixels are
  // sorted into warps by the interval of candidates their bound leaves (exact
  // candidate pruning, see prune_range); the later passes keep that order for
  // the pixels still iterating (exact per-pixel early exit).  A warp sweeps
  // the union of its pixels' intervals.  Each pixel's
  // first M-step uses the fixed-label form when its first-iteration labels do
  // not depend on the candidate, else the per-candidate form, whatever its
  // warp-mates use; those pixels are sorted first, so at most one warp mixes
  // the two forms.
  PixelState ps = pixel_state(smem + Ly.pix, a.TR * a.TW);
  int* s_wcnt = reinterpret_cast<int*>(smem + Ly.wcnt);
  uint16_t* s_sortc = reinterpret_cast<uint16_t*>(smem + Ly.sortc);
  const int warp = tid >> 5;
  const float lin = a.mseg ? 1.f : 0.f;

  bool my_valid = (u0 + tid % a.TW < W) && (v0 + tid / a.TW < H);
  if (a.dyn_only && my_valid) {  // Sec. III-F: only the reference pixels flagged dynamic
    const int r = tid / a.TW, u = u0 + tid % a.TW;
    const float Pref = s_p[(static_cast<size_t>(a.ref) * a.TR + r) * RW + (u - cs)];
    if (!(Pref >= a.seg_threshold)) {
      const size_t pix = static_cast<size_t>(v0 + r) * W + u;
      write_static_pixel<K>(a, u, v0 + r, s_mu ? s_mu[tid] : a.mu[pix]);
      if (a.refocus_out) {  // no static ray: the reference image, from the staged rows
        const uint8_t* p = smem + Ly.raw_img + ((static_cast<size_t>(a.ref) * (a.TR + 2) + r + 1) * RW + (u - cs)) * a.bpp;
        const float scale = a.dtype == 0 ? (1.f / 255.f) : 1.f;
        for (int c = 0; c < a.C; ++c) a.refocus_out[pix * a.C + c] = pixel_element(p, c, a.dtype) * scale;
      }
      my_valid = false;
    }
  }
  unsigned my_pairs = 0;   // (pixel, candidate) objectives this thread evaluated for the statistics
  unsigned my_static = 0;  // static ray samples among them
  int key = 0;
  {  // first-iteration labels, the segmentation bound and the first M-step's interval
    const PixelCtx<TS> me = load_pixel<TS>(a, s_feat, u0, v0, cam_stride, tid, s_mu);
    unsigned S0 = 0;
    float seg_max = 0.f;
    const bool f0 = me.valid && constant_initial_labels<K, TS>(a, me.st, &S0, &seg_max);
    const float seg_ub = fmaf(lin, seg_max, a.seg_margin);
    int lo = 0, hi = a.D - 1;
    if (a.prune && my_valid && me.inside) {
      const int js = nearest_candidate(a, me.mu);
      float Js;
      if (f0)
        m_step_fixed_range<K, TS, REF>(a, me.st, s_wq, s_o, s_chg, s_d, s_rcp, me.cy, me.cx, me.cz, me.mu, true, S0,
                                       js, js + 1, &Js);
      else
        m_step_init_range<K, TS, REF>(a, me.st, s_wq, s_o, s_chg, s_d, s_rcp, me.cy, me.cx, me.cz, me.mu, true, js,
                                      js + 1, &Js, nullptr);
      prune_range(a, me.mu, Js, seg_ub, js, lo, hi);
      ++my_pairs;
    }
    ps.fixed0[tid] = f0;
    ps.S0[tid] = static_cast<uint16_t>(S0);
    ps.conv[tid] = 0;
    ps.seg_ub[tid] = seg_ub;
    ps.lo[tid] = static_cast<int16_t>(lo);
    ps.hi[tid] = static_cast<int16_t>(hi);
    key = (f0 ? 0 : 2 * kLoBuckets) + interval_key(lo, hi, a.D);
  }
  const int nact = sort_pixels(my_valid, key, 4 * kLoBuckets, ps.list, s_sortc, s_wcnt);
  unsigned long long executed = static_cast<unsigned long long>(nact);

  // A later M-step's interval (fixed labels S of the last E-step), bounded by
  // the objective at the last arg-max jp; evaluated at the start of the pass
  // by every lane that takes part in the pixel's M-step.
  auto interval_at = [&](const PixelCtx<TS>& c, int p, unsigned S, int jp, int& lo, int& hi) {
    lo = 0;
    hi = a.D - 1;
    if (!(a.prune && c.inside)) return false;
    float Js;
    m_step_fixed_range<K, TS, REF>(a, c.st, s_wq, s_o, s_chg, s_d, s_rcp, c.cy, c.cx, c.cz, c.mu, true, S, jp, jp + 1,
                                   &Js);
    prune_range(a, c.mu, Js, ps.seg_ub[p], jp, lo, hi);
    return true;
  };

  // t = 1
  if (warp * 32 < nact) {
    const bool active = tid < nact;
    const int p = ps.list[active ? tid : nact - 1];
    const PixelCtx<TS> c = load_pixel<TS>(a, s_feat, u0, v0, cam_stride, p, s_mu);
    const bool f0 = ps.fixed0[p];
    const unsigned S0 = ps.S0[p];
    const int LO = __reduce_min_sync(0xffffffffu, ps.lo[p]), HI = __reduce_max_sync(0xffffffffu, ps.hi[p]);
    unsigned ns = __popc(S0) * static_cast<unsigned>(HI - LO + 1);
    const int jb = f0 ? m_step_fixed_range<K, TS, REF>(a, c.st, s_wq, s_o, s_chg, s_d, s_rcp, c.cy, c.cx, c.cz, c.mu,
                                                       c.inside, S0, LO, HI + 1, nullptr)
                      : m_step_init_range<K, TS, REF>(a, c.st, s_wq, s_o, s_chg, s_d, s_rcp, c.cy, c.cx, c.cz, c.mu,
                                                      c.inside, LO, HI + 1, nullptr, &ns);
    if (active) {
      my_pairs += static_cast<unsigned>(HI - LO + 1);
      my_static += ns;
    }
    Rays rays;
    sample_rays<K, TS>(a, c.st, s_wq, s_o, jb, c.cy, c.cx, c.cz, rays);
    unsigned S = 0;
    float emax = 0.f;
    enumerate<0, K>(rays, s_rcp, a.beta, 0.f, S, emax, nullptr, a.prune != 0);
    // the second M-step would repeat the first one exactly
    const bool conv = a.early_exit && f0 && S == S0;
    if (active) {
      ps.jb[p] = static_cast<int16_t>(jb);
      ps.S[p] = static_cast<uint16_t>(S);
      ps.emax[p] = emax;
      ps.conv[p] = conv;
    }
  }
  __syncthreads();
  // t >= 2: only the pixels not yet at their fixed point, in the first
  // pass's order (pixels of similar candidate intervals stay together
  // without sorting again)
  const int lane = tid & 31;
  int16_t* list = ps.list;
  int16_t* list_next = ps.list2;
  int n_prev = nact;
  for (int t = 2; t <= a.iters; ++t) {
    const int p_prev = tid < n_prev ? list[tid] : 0;
    const bool pend = tid < n_prev && !ps.conv[p_prev];
    const int n = compact_value(pend, p_prev, list_next, 0, s_wcnt);
    if (n == 0) break;
    int16_t* tmp = list;
    list = list_next;
    list_next = tmp;
    n_prev = n;
    executed += static_cast<unsigned long long>(n);
    // one lane per pixel, a warp sweeping its lanes' union (splitting the
    // last pixels over groups of lanes measured slower here: every lane of a
    // group reloads the taps, and the warps it keeps busy are the issue
    // slots the SM's other CTA would use)
    if (warp * 32 < n) {
      const bool active = tid < n;
      const int p = list[active ? tid : n - 1];
      const PixelCtx<TS> c = load_pixel<TS>(a, s_feat, u0, v0, cam_stride, p, s_mu);
      const unsigned Sp = ps.S[p];
      int plo, phi;
      if (interval_at(c, p, Sp, ps.jb[p], plo, phi) && active) ++my_pairs;
      const int LO = __reduce_min_sync(0xffffffffu, plo), HI = __reduce_max_sync(0xffffffffu, phi);
      const int jb = m_step_fixed_range<K, TS, REF>(a, c.st, s_wq, s_o, s_chg, s_d, s_rcp, c.cy, c.cx, c.cz, c.mu,
                                                    c.inside, Sp, LO, HI + 1, nullptr);
      if (active) {
        my_pairs += static_cast<unsigned>(HI - LO + 1);
        my_static += __popc(Sp) * static_cast<unsigned>(HI - LO + 1);
      }
      Rays rays;
      sample_rays<K, TS>(a, c.st, s_wq, s_o, jb, c.cy, c.cx, c.cz, rays);
      unsigned S = 0;
      float emax = 0.f;
      enumerate<0, K>(rays, s_rcp, a.beta, 0.f, S, emax, nullptr, a.prune != 0);
      const bool conv = a.early_exit && S == Sp;
      if (active) {
        ps.jb[p] = static_cast<int16_t>(jb);
        ps.S[p] = static_cast<uint16_t>(S);
        ps.emax[p] = emax;
        ps.conv[p] = conv;
      }
    }
    __syncthreads();
  }

  // posteriors and outputs, one thread per pixel
  if (my_valid) {
    const PixelCtx<TS> me = load_pixel<TS>(a, s_feat, u0, v0, cam_stride, tid, s_mu);
    const int jb = ps.jb[tid];
    const unsigned S = ps.S[tid];
    const size_t pix = static_cast<size_t>(me.v) * W + me.u;
    a.d_idx[pix] = jb;
    if (a.d_out) a.d_out[pix] = s_d[jb];
    if (a.labels) a.labels[pix] = static_cast<uint16_t>(S);
    if (a.post) {
      Rays rays;
      sample_rays<K, TS>(a, me.st, s_wq, s_o, jb, me.cy, me.cx, me.cz, rays);
      float post[K];
      unsigned dummy;
      float dummyf;
      enumerate<1, K>(rays, s_rcp, a.beta, ps.emax[tid], dummy, dummyf, post);
      const size_t HW = static_cast<size_t>(H) * W;
#pragma unroll
      for (int k = 0; k < K; ++k) a.post[k * HW + pix] = post[k];
    }
    if (a.refocus_out) {  // Eq. 2 from the staged raw rows (they hold every tap of every candidate)
      const int row = me.v - v0 + 1;  // staged rows start one above the tile
      float* out = a.refocus_out + pix * a.C;
      const uint8_t* s_img = smem + Ly.raw_img;
      if (a.dtype == 0)
        refocus_staged<K, uint8_t>(a, s_img, row, cs, me.u, jb, S, s_o, s_wq, out);
      else if (a.dtype == 1)
        refocus_staged<K, float>(a, s_img, row, cs, me.u, jb, S, s_o, s_wq, out);
      else if (a.dtype == 2)
        refocus_staged<K, __half>(a, s_img, row, cs, me.u, jb, S, s_o, s_wq, out);
      else
        refocus_staged<K, __nv_bfloat16>(a, s_img, row, cs, me.u, jb, S, s_o, s_wq, out);
    }
  }
  {  // statistics: warp sums into the tile's counters, one global atomic each per tile
    unsigned* s_stat = reinterpret_cast<unsigned*>(smem + Ly.wcnt) + 32;
    const unsigned wp = __reduce_add_sync(0xffffffffu, my_pairs);
    const unsigned ws = __reduce_add_sync(0xffffffffu, my_static);
    if (lane == 0) {
      atomicAdd_block(s_stat, wp);
      atomicAdd_block(s_stat + 1, ws);
    }
  }
  __syncthreads();
  if (tid == 0) {
    const unsigned* s_stat = reinterpret_cast<const unsigned*>(smem + Ly.wcnt) + 32;
    if (a.sweeps) atomicAdd(a.sweeps, executed);
    atomicAdd(a.counter, static_cast<unsigned long long>(s_stat[0]));
    if (a.static_counter) atomicAdd(a.static_counter, static_cast<unsigned long long>(s_stat[1]));
  }
  __syncthreads();
  return true;
}

// One CTA per tile of one frame.  REF: see sweep_tile.
template <int K, typename TS, int REF>
__global__ void __launch_bounds__(sweep_max_threads(K), sweep_min_blocks<K>()) em_sweep_kernel(const __grid_constant__ CUtensorMap img_map,
                                                       const __grid_constant__ CUtensorMap p_map,
                                                       const SweepArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  if ((smem_u32(smem) & 127u) != 0u) {  // TMA destinations must be 128-byte aligned
    if (threadIdx.x == 0) atomicOr(a.status, kStatusSmemMisaligned);
    return;
  }
#ifdef LF_DEBUG
  {  // the carve-up must fit the dynamic shared memory of the launch
    unsigned dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    if (sweep_layout(K, a).total > dyn) {
      if (threadIdx.x == 0) atomicOr(a.status, kStatusBoundsViolation);
      return;
    }
  }
#endif
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kSmemBar);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  int tx = blockIdx.x, ty = blockIdx.y;
  if (a.tile_list) {  // dynamic-only: this CTA's tile comes from the classified list
    if (static_cast<int>(blockIdx.x) >= *a.n_tiles) return;
    const int id = a.tile_list[blockIdx.x], tiles_x = (a.W + a.TW - 1) / a.TW;
    tx = id % tiles_x;
    ty = id / tiles_x;
  }
  sweep_tile<K, TS, REF>(a, &img_map, &p_map, tx, ty, smem, 0u, true, false);
}

// Persistent form for uneven batches: every CTA takes items from one queue
// (head counter in global memory) until it is empty; items of one frame are
// adjacent, so a CTA restages the frame's tables only when the frame changes.
// frames[] holds per-frame arguments and TMA descriptors in global memory.
template <int K, typename TS, int REF>
__global__ void __launch_bounds__(256, persistent_min_blocks<K>()) em_sweep_persistent(const FrameDesc* frames,
                                                                                const TileItem* items,
                                                                                const int* first_item,
                                                                                const int* n_items,
                                                                                unsigned* head) {
  extern __shared__ __align__(128) uint8_t smem[];
  SweepArgs* s_args = reinterpret_cast<SweepArgs*>(smem + kSmemArgs);
  int* s_item = reinterpret_cast<int*>(smem + kSmemItem);
  if ((smem_u32(smem) & 127u) != 0u) {
    if (threadIdx.x == 0) atomicOr(frames[0].args.status, kStatusSmemMisaligned);
    return;
  }
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kSmemBar);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int n = *n_items;
  items += *first_item;  // this camera count's items start here
  int cur = -1;
  unsigned phase = 0;
  for (;;) {
    if (threadIdx.x == 0) *s_item = static_cast<int>(atomicAdd(head, 1u));
    __syncthreads();
    const int it = *s_item;
    if (it >= n) break;
    const TileItem item = items[it];
    const bool fresh = item.frame != cur;
    if (fresh) {
      const int* src = reinterpret_cast<const int*>(&frames[item.frame].args);
      int* dst = reinterpret_cast<int*>(s_args);
      for (int i = threadIdx.x; i < static_cast<int>(sizeof(SweepArgs) / 4); i += blockDim.x) dst[i] = src[i];
      cur = item.frame;
      __syncthreads();
    }
    if (!sweep_tile<K, TS, REF>(*s_args, &frames[item.frame].img_map, &frames[item.frame].p_map, item.x, item.y,
                           smem, phase, fresh, true))
      break;  // a bounded wait expired: stop taking work (the status word says why)
    phase ^= 1u;
  }
}

// The reference camera sits in the middle of the array in every workload
// (centred baselines); that case runs the instantiation that knows it.
template <int K, typename TS, int REF>
cudaError_t launch_em_sweep_ref(const CUtensorMap& img_map, const CUtensorMap& p_map, const SweepArgs& a,
                                cudaStream_t s) {
  const size_t smem = sweep_layout(K, a).total;
  static int configured = -1;  // largest dynamic shared size set so far (per process)
  if (static_cast<int>(smem) > configured) {
    cudaError_t e = cudaFuncSetAttribute(em_sweep_kernel<K, TS, REF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    configured = static_cast<int>(smem);
  }
  if (a.TR * a.TW > sweep_max_threads(K)) return cudaErrorInvalidConfiguration;
  dim3 grid((a.W + a.TW - 1) / a.TW, (a.H + a.TR - 1) / a.TR);
  if (a.tile_list) grid = dim3(grid.x * grid.y, 1);  // one CTA per listed tile (at most all)
  em_sweep_kernel<K, TS, REF><<<grid, a.TR * a.TW, smem, s>>>(img_map, p_map, a);
  return cudaGetLastError();
}

template <int K, typename TS>
cudaError_t launch_em_sweep_k(const CUtensorMap& img_map, const CUtensorMap& p_map, const SweepArgs& a,
                              cudaStream_t s) {
  return a.ref == K / 2 ? launch_em_sweep_ref<K, TS, K / 2>(img_map, p_map, a, s)
                        : launch_em_sweep_ref<K, TS, -1>(img_map, p_map, a, s);
}

template <int K, typename TS, int REF>
int em_sweep_persistent_occupancy_ref(size_t smem, int threads) {
  cudaFuncSetAttribute(em_sweep_persistent<K, TS, REF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       static_cast<int>(smem));
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, em_sweep_persistent<K, TS, REF>, threads, smem) !=
      cudaSuccess)
    return 0;
  return blocks;
}

// centred: every frame of the launch has its reference camera in the middle
// of the array (index K / 2), which the instantiation that knows it uses.
template <int K, typename TS>
int em_sweep_persistent_occupancy_k(size_t smem, int threads, int centred) {
  return centred ? em_sweep_persistent_occupancy_ref<K, TS, K / 2>(smem, threads)
                 : em_sweep_persistent_occupancy_ref<K, TS, -1>(smem, threads);
}

template <int K, typename TS, int REF>
cudaError_t launch_em_sweep_persistent_ref(const FrameDesc* frames, const TileItem* items, const int* first_item,
                                           const int* n_items, unsigned* head, size_t smem, int grid, int threads,
                                           cudaStream_t s) {
  static int configured = -1;
  if (static_cast<int>(smem) > configured) {
    cudaError_t e = cudaFuncSetAttribute(em_sweep_persistent<K, TS, REF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    configured = static_cast<int>(smem);
  }
  em_sweep_persistent<K, TS, REF><<<grid, threads, smem, s>>>(frames, items, first_item, n_items, head);
  return cudaGetLastError();
}

template <int K, typename TS>
cudaError_t launch_em_sweep_persistent_k(const FrameDesc* frames, const TileItem* items, const int* first_item,
                                         const int* n_items, unsigned* head, size_t smem, int grid, int threads,
                                         int centred, cudaStream_t s) {
  return centred ? launch_em_sweep_persistent_ref<K, TS, K / 2>(frames, items, first_item, n_items, head, smem,
                                                                 grid, threads, s)
                 : launch_em_sweep_persistent_ref<K, TS, -1>(frames, items, first_item, n_items, head, smem, grid,
                                                              threads, s);
}

}  // namespace dev
}  // namespace lf

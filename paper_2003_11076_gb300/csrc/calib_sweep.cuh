// Per-pixel EM for a calibrated (non-rectified) camera array (Eq. 1 in
// generalized disparity space; the warping function W_k of Sec. III-C is the
// homography of the plane at disparity d).  The schedule and the objective
// are those of the rectified sweep (Sec. III-B..III-D): first M-step with
// per-candidate thresholded labels, then M-step / E-step alternation with an
// exact per-pixel early exit, posteriors of the final labels.
//
// What differs is the sampling.  A ray of reference pixel (u, v) at disparity
// d lands at (X / Z, Y / Z) with (X, Y, Z) = cam_k (u, v, 1, d); the kernel
// locates it by its offset from (u, v) (calib_geom.cuh), whose pixel-constant
// parts are computed once per pixel and pass.  The position moves along the epipolar line in both image directions, so the
// rectified kernel's row staging with a horizontal halo does not apply: the
// descriptor maps of all cameras are written to HBM once per run (20 bytes per
// camera pixel, L2-resident at the paper's frame size) and each ray sample is
// a bilinear gather of four float4 + four float texels through L1.
// Neighbouring pixels of a 16 x 16 block sample neighbouring texels, so the
// gathers of a warp share cache lines.
#pragma once

#include "calib_geom.cuh"
#include "em_sweep.cuh"

namespace lf {
namespace dev {

struct CalibRay {
  float2 g;  // (Y, Sobel-x / 8) of the ray minus the reference ray's
  float gz, ls, ld;
};

// One axis of a ray's bilinear footprint: the texel index i0 of the lower
// tap and the weight w of the upper one (i0 + 1), for the position
// p + off clamped to [0, n - 1].  Outside [0, n - 1) the clamped position is
// a border texel: w = 0, so the upper tap (still read, and finite: the maps
// carry one zero-filled row past their end) contributes 0 * finite = 0.
__device__ __forceinline__ int calib_lower_tap(float off, int p, int n, float& w) {
  const float f = floorf(off);
  const int fi = max(min(__float2int_rd(off), n), -n - 1);  // saturated far outside; p + fi cannot overflow
  const int c = p + fi;
  const bool in = static_cast<unsigned>(c) < static_cast<unsigned>(n - 1);
  w = in ? off - f : 0.f;
  return min(max(c, 0), n - 1);
}

// Bilinear sample of camera k's maps at the ray of pixel (u, v) at disparity
// d, both coordinates clamped to the image, with the descriptors shifted by
// the reference ray's.  The taps are (i0, j0), (i0 + 1, j0), (i0, j0 + 1),
// (i0 + 1, j0 + 1); the (Y, Sobel-x) and (Sobel-y, log(1 - P)) pairs are
// interpolated as float32x2 pairs (the same IEEE operations per lane as the
// scalar form).
__device__ __forceinline__ CalibRay calib_sample(const CalibArgs& a, int k, const CalibPix& cp, int u, int v,
                                                 float d, float2 cyx, float cz) {
  const float* M = a.cam[k];
  const float Z = fmaf(d, M[11], cp.az);
  const float X = fmaf(d, fmaf(-static_cast<float>(u), M[11], M[3]), cp.ax);
  const float Y = fmaf(d, fmaf(-static_cast<float>(v), M[11], M[7]), cp.ay);
  const float iz = 1.f / Z;
  float wx, wy;
  const int i0 = calib_lower_tap(X * iz, u, a.W, wx);
  const int j0 = calib_lower_tap(Y * iz, v, a.H, wy);
  const int o = (k * a.H + j0) * a.W + i0;  // < K H W: checked when the context is created
  const float4* f0 = a.fa + o;
  const float4* f1 = f0 + a.W;
  const float* b0 = a.fb + o;
  const float* b1 = b0 + a.W;
  const float4 p00 = __ldg(f0), p01 = __ldg(f0 + 1), p10 = __ldg(f1), p11 = __ldg(f1 + 1);
  const float q00 = __ldg(b0), q01 = __ldg(b0 + 1), q10 = __ldg(b1), q11 = __ldg(b1 + 1);
  const float2 wx2 = make_float2(wx, wx), wy2 = make_float2(wy, wy);
  auto bl2 = [&](float2 v00, float2 v01, float2 v10, float2 v11) {
    const float2 top = ffma2(wx2, fsub2(v01, v00), v00), bot = ffma2(wx2, fsub2(v11, v10), v10);
    return ffma2(wy2, fsub2(bot, top), top);
  };
  const float2 lo = bl2(make_float2(p00.x, p00.y), make_float2(p01.x, p01.y), make_float2(p10.x, p10.y),
                        make_float2(p11.x, p11.y));
  const float2 hi = bl2(make_float2(p00.z, p00.w), make_float2(p01.z, p01.w), make_float2(p10.z, p10.w),
                        make_float2(p11.z, p11.w));
  const float top = fmaf(wx, q01 - q00, q00), bot = fmaf(wx, q11 - q10, q10);
  CalibRay r;
  r.g = fsub2(lo, cyx);
  r.gz = hi.x - cz;
  r.ls = hi.y;
  r.ld = fmaf(wy, bot - top, top);
  return r;
}

// M-step over candidates j0 <= j < j1 (lowest index on ties; *best_out = the
// maximum).  INIT: labels thresholded at each ray's own sample (ld - ls <
// log(thr / (1 - thr)) means static); otherwise the fixed labels S.  Every
// candidate is evaluated from scratch, so a range computes the same
// objectives as the whole sweep.
template <int K, bool INIT>
__device__ __forceinline__ int calib_m_step(const CalibArgs& a, const CalibPix (&A)[K], int u, int v, float2 cyx,
                                            float cz, float mu, bool inside, unsigned S, int j0, int j1,
                                            float* best_out) {
  float best = -INFINITY;
  int jb = j0;
  auto prior_at = [&](int j) {
    const float t = __ldg(a.dval + j) - mu;
    return __logf(a.gamma + __expf(-(t * t) * a.inv2s2));
  };
  float pr_next = j0 < j1 ? prior_at(j0) : 0.f;
  for (int j = j0; j < j1; ++j) {
    const float pr = pr_next;
    pr_next = prior_at(min(j + 1, j1 - 1));  // the next candidate's prior, off this one's critical path
    const float d = __ldg(a.dval + j);
    float2 syx = make_float2(0.f, 0.f);
    float sz = 0.f, q = 0.f, seg = 0.f;
    int n = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (!INIT && !(S >> k & 1u)) {  // a dynamic ray contributes its log p(dynamic) only
        if (a.mseg) {
          const CalibRay r = calib_sample(a, k, A[k], u, v, d, cyx, cz);
          seg += r.ld;
        }
        continue;
      }
      const CalibRay r = calib_sample(a, k, A[k], u, v, d, cyx, cz);
      const bool stat = INIT ? (r.ld - r.ls < a.log_thr) : true;
      if (stat) {
        syx = fadd2(syx, r.g);
        sz += r.gz;
        q = fmaf(r.g.x, r.g.x, q); q = fmaf(r.g.y, r.g.y, q); q = fmaf(r.gz, r.gz, q);
        seg += r.ls;
        ++n;
      } else {
        seg += r.ld;
      }
    }
    const float rn = n >= 2 ? 1.f / static_cast<float>(n) : 0.f;
    const float ss = fmaf(sz, sz, fmaf(syx.y, syx.y, syx.x * syx.x));
    const float var = fmaxf(fmaf(-ss, rn, q) * rn, 0.f);  // >= 0: the bound of the candidate pruning
    float J = a.mseg ? seg : 0.f;
    if (inside) J += pr;
    J = fmaf(-a.beta, var, J);
    if (J > best) { best = J; jb = j; }
  }
  if (best_out) *best_out = best;
  return jb;
}

template <int K>
__device__ __forceinline__ void calib_rays(const CalibArgs& a, const CalibPix (&A)[K], int u, int v, int j,
                                           float2 cyx, float cz, Rays& r) {
  const float d = __ldg(a.dval + j);
  r.base = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const CalibRay s = calib_sample(a, k, A[k], u, v, d, cyx, cz);
    r.gy[k] = s.g.x; r.gx[k] = s.g.y; r.gz[k] = s.gz;
    r.qk[k] = fmaf(s.gz, s.gz, fmaf(s.g.y, s.g.y, s.g.x * s.g.x));
    r.ak[k] = s.ls - s.ld;
    r.base += s.ld;
  }
}

// One CTA per 16 x 16 block of reference pixels, one thread per pixel for
// the first iteration; afterwards only the pixels not yet at their fixed
// point, regrouped into dense warps before every pass (exact per-pixel early
// exit), and groups of 2 to 32 lanes per pixel once fewer are left than the
// CTA has threads (lanes split the candidates, then the label vectors; same
// tie rules, same bits).
template <int K>
__global__ void __launch_bounds__(256, K <= 5 ? 3 : 2) calib_sweep_kernel(const __grid_constant__ CalibArgs a) {
  __shared__ float s_rcp[16];  // 1/n for the E-step's subset sizes (0 for n < 2: Var = 0)
  __shared__ float s_emax[256];
  __shared__ int16_t s_jb[256], s_list[256], s_list2[256], s_lo[256], s_hi[256];
  __shared__ uint16_t s_S[256];
  __shared__ uint8_t s_conv[256];
  __shared__ int s_wcnt[8];
  __shared__ uint16_t s_sortc[2 * kLoBuckets * 8];  // counting sort (sort_pixels), zero between uses
  __shared__ unsigned s_stat;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  if (tid < 16) s_rcp[tid] = tid >= 2 ? 1.f / static_cast<float>(tid) : 0.f;
  for (int i = tid; i < 2 * kLoBuckets * 8; i += blockDim.x) s_sortc[i] = 0;
  if (tid == 0) s_stat = 0u;
  __syncthreads();
  const int bu = blockIdx.x * 16, bv = blockIdx.y * 16;
  const int u = bu + (tid & 15), v = bv + (tid >> 4);
  bool run = u < a.W && v < a.H;
  if (run && a.dyn_only) {  // Sec. III-F: only the reference pixels flagged dynamic
    const size_t pix = static_cast<size_t>(v) * a.W + u;
    const float Pref = reinterpret_cast<const float*>(reinterpret_cast<const uint8_t*>(a.P) +
                                                      (static_cast<size_t>(a.ref) * a.H + v) * a.p_pitch)[u];
    if (!(Pref >= a.seg_threshold)) {
      const float mu = a.mu[pix];
      int j = -1;
      if (!isnan(mu)) {  // the candidate nearest the prior centre, lower index on a tie
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
      a.labels[pix] = 0;
      if (a.post)
        for (int k = 0; k < K; ++k) a.post[k * static_cast<size_t>(a.H) * a.W + pix] = nan;
      run = false;
    }
  }
  // everything the EM of block pixel p needs, recomputed per pass
  struct Px {
    CalibPix A[K];
    int u, v;
    float2 cyx;
    float mu, cz;
    bool inside;
  };
  auto load = [&](int p) {
    Px x;
    const int pu = bu + (p & 15), pv = bv + (p >> 4);
    const size_t pix = static_cast<size_t>(pv) * a.W + pu;
#pragma unroll
    for (int k = 0; k < K; ++k) x.A[k] = calib_pixel(a.cam[k], static_cast<float>(pu), static_cast<float>(pv));
    x.u = pu;
    x.v = pv;
    x.mu = a.mu[pix];
    x.inside = !isnan(x.mu);
    const float4 fr = a.fa[static_cast<size_t>(a.ref) * a.H * a.W + pix];
    x.cyx = make_float2(fr.x, fr.y);
    x.cz = fr.z;
    return x;
  };
  // Exact candidate pruning (as in the rectified sweep, prune_interval): the
  // objective of a candidate is at most its log prior plus the segmentation
  // term, and every log p(static) / log p(dynamic) is <= 0, so the bound of
  // the segmentation term is 0 (plus a.seg_margin for rounding).  Before each
  // M-step a pixel's interval comes from the objective at one candidate (the
  // one nearest mu, then the last arg-max), evaluated by the same code.
  const float seg_ub = a.seg_margin;
  auto interval = [&](const Px& x, float Js, int js, int& lo, int& hi) {
    prune_interval(x.mu, Js, seg_ub, a.gamma, a.inv2s2, a.d0, a.inv_step, a.D, js, lo, hi);
  };
  unsigned my_pairs = 0;  // (pixel, candidate) objectives this thread evaluated
  unsigned long long executed = 0;
  // t = 1: the first M-step's interval, then the pixels sorted by it
  int key = 0;
  if (run) {
    int lo = 0, hi = a.D - 1;
    if (a.prune) {
      const Px x = load(tid);
      if (x.inside) {
        const int js = min(max(static_cast<int>(rintf((x.mu - a.d0) * a.inv_step)), 0), a.D - 1);
        float Js;
        calib_m_step<K, true>(a, x.A, x.u, x.v, x.cyx, x.cz, x.mu, true, 0u, js, js + 1, &Js);
        interval(x, Js, js, lo, hi);
        ++my_pairs;
      }
    }
    s_lo[tid] = static_cast<int16_t>(lo);
    s_hi[tid] = static_cast<int16_t>(hi);
    key = interval_key(lo, hi, a.D);
  }
  const int n1 = sort_pixels(run, key, 2 * kLoBuckets, s_list, s_sortc, s_wcnt);
  executed += static_cast<unsigned long long>(n1);
  // a later M-step's interval (labels S of the last E-step), bounded by the
  // objective at the last arg-max jp, evaluated at the start of the pass by
  // every lane that takes part in the pixel's M-step
  auto interval_at = [&](const Px& x, unsigned S, int jp, int& lo, int& hi) {
    lo = 0;
    hi = a.D - 1;
    if (!(a.prune && x.inside)) return false;
    float Js;
    calib_m_step<K, false>(a, x.A, x.u, x.v, x.cyx, x.cz, x.mu, true, S, jp, jp + 1, &Js);
    interval(x, Js, jp, lo, hi);
    return true;
  };
  s_conv[tid] = 0;
  if (warp * 32 < n1) {
    const bool active = tid < n1;
    const int p = s_list[active ? tid : n1 - 1];
    const Px x = load(p);
    const int LO = __reduce_min_sync(0xffffffffu, s_lo[p]), HI = __reduce_max_sync(0xffffffffu, s_hi[p]);
    const int jb = calib_m_step<K, true>(a, x.A, x.u, x.v, x.cyx, x.cz, x.mu, x.inside, 0u, LO, HI + 1, nullptr);
    if (active) my_pairs += static_cast<unsigned>(HI - LO + 1);
    Rays rays;
    calib_rays<K>(a, x.A, x.u, x.v, jb, x.cyx, x.cz, rays);
    unsigned S = 0;
    float emax = 0.f;
    enumerate<0, K>(rays, s_rcp, a.beta, 0.f, S, emax, nullptr, a.prune != 0);
    if (active) {
      s_jb[p] = static_cast<int16_t>(jb);
      s_S[p] = static_cast<uint16_t>(S);
      s_emax[p] = emax;
    }
  }
  __syncthreads();
  // later passes: the pixels still iterating, in the first pass's order
  int16_t* list = s_list;
  int16_t* list_next = s_list2;
  int n_prev = n1;
  for (int t = 2; t <= a.iters; ++t) {
    const int p_prev = tid < n_prev ? list[tid] : 0;
    const bool pend = tid < n_prev && !s_conv[p_prev];
    const int n = compact_value(pend, p_prev, list_next, 0, s_wcnt);
    if (n == 0) break;
    int16_t* tmp = list;
    list = list_next;
    list_next = tmp;
    n_prev = n;
    executed += static_cast<unsigned long long>(n);
    // lanes per pixel: the largest power of two that still fits every
    // remaining pixel into one round of the CTA's warps
    int G = 1;
    while (G < 32 && n * (G << 1) <= nwarps * 32) G <<= 1;
    if (G > 1) {
      const int gpw = 32 / G, gl = lane & (G - 1);
      const int slot = warp * gpw + lane / G;
      if (warp * gpw < n) {
        const bool act = slot < n;
        const int p = list[act ? slot : n - 1];  // idle groups repeat the last pixel
        const Px x = load(p);
        const unsigned Sp = s_S[p];
        int plo, phi;
        if (interval_at(x, Sp, s_jb[p], plo, phi) && act && gl == 0) ++my_pairs;
        const int per = (phi - plo + G) / G, j0 = min(plo + gl * per, phi + 1), j1 = min(j0 + per, phi + 1);
        float jbest;
        unsigned jb = static_cast<unsigned>(
            calib_m_step<K, false>(a, x.A, x.u, x.v, x.cyx, x.cz, x.mu, x.inside, Sp, j0, j1, &jbest));
        if (act) my_pairs += static_cast<unsigned>(j1 - j0);
        group_argmax(jbest, jb, G);
        Rays rays;
        calib_rays<K>(a, x.A, x.u, x.v, static_cast<int>(jb), x.cyx, x.cz, rays);
        unsigned S = 0;
        float emax = 0.f;
        enumerate_group<K>(rays, s_rcp, a.beta, gl, G, S, emax, a.prune != 0);
        const bool conv = a.early_exit && S == Sp;  // the next M-step would repeat this one exactly
        if (act && gl == 0) {
          s_jb[p] = static_cast<int16_t>(jb);
          s_S[p] = static_cast<uint16_t>(S);
          s_emax[p] = emax;
          s_conv[p] = conv;
        }
      }
    } else if (warp * 32 < n) {
      const bool active = tid < n;
      const int p = list[active ? tid : n - 1];
      const Px x = load(p);
      const unsigned Sp = s_S[p];
      int plo, phi;
      if (interval_at(x, Sp, s_jb[p], plo, phi) && active) ++my_pairs;
      const int LO = __reduce_min_sync(0xffffffffu, plo), HI = __reduce_max_sync(0xffffffffu, phi);
      const int jb = calib_m_step<K, false>(a, x.A, x.u, x.v, x.cyx, x.cz, x.mu, x.inside, Sp, LO, HI + 1, nullptr);
      if (active) my_pairs += static_cast<unsigned>(HI - LO + 1);
      Rays rays;
      calib_rays<K>(a, x.A, x.u, x.v, jb, x.cyx, x.cz, rays);
      unsigned S = 0;
      float emax = 0.f;
      enumerate<0, K>(rays, s_rcp, a.beta, 0.f, S, emax, nullptr, a.prune != 0);
      const bool conv = a.early_exit && S == Sp;
      if (active) {
        s_jb[p] = static_cast<int16_t>(jb);
        s_S[p] = static_cast<uint16_t>(S);
        s_emax[p] = emax;
        s_conv[p] = conv;
      }
    }
    __syncthreads();
  }
  // outputs, one thread per pixel
  if (run) {
    const size_t pix = static_cast<size_t>(v) * a.W + u;
    const int jb = s_jb[tid];
    const unsigned S = s_S[tid];
    a.d_idx[pix] = jb;
    if (a.d_out) a.d_out[pix] = a.dval[jb];
    a.labels[pix] = static_cast<uint16_t>(S);
    if (a.post) {
      const Px x = load(tid);
      Rays rays;
      calib_rays<K>(a, x.A, x.u, x.v, jb, x.cyx, x.cz, rays);
      float post[K];
      unsigned dummy;
      float dummyf;
      enumerate<1, K>(rays, s_rcp, a.beta, s_emax[tid], dummy, dummyf, post);
#pragma unroll
      for (int k = 0; k < K; ++k) a.post[k * static_cast<size_t>(a.H) * a.W + pix] = post[k];
    }
  }
  {  // statistics: one global atomic per block and counter
    const unsigned wp = __reduce_add_sync(0xffffffffu, my_pairs);
    if (lane == 0) atomicAdd_block(&s_stat, wp);
    __syncthreads();
    if (tid == 0) {
      atomicAdd(a.counter, static_cast<unsigned long long>(s_stat));
      if (a.sweeps) atomicAdd(a.sweeps, executed);
    }
  }
}

template <int K>
cudaError_t launch_calib_sweep_k(const CalibArgs& a, cudaStream_t s) {
  const dim3 grid((a.W + 15) / 16, (a.H + 15) / 16);
  calib_sweep_kernel<K><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dev
}  // namespace lf

// Variants of the per-pixel EM, on the same staged tile as the sweep kernel
// (Sec. III-B formulates EM over the hidden labels S; the paper runs it with
// hard assignments, Sec. III-C/III-D):
//
//   soft EM    the E-step keeps the whole posterior q(S) ~ exp J(d_t, S) over
//              the 2^K label vectors, and every M-step after the first
//              maximises the expected complete-data objective
//                Q(d) = sum_S q(S) J(d, S).
//              With Var_S = (1/|S|^2) sum_{k<l in S} |f_k - f_l|^2 this is
//                Q(d) = log p(d) + sum_k [pi_k ls_k + (1 - pi_k) ld_k]
//                       - beta * sum_{k<l} w_kl |f_k(d) - f_l(d)|^2
//              with pi_k = P(ray k static) and w_kl = sum_{S contains k,l}
//              q(S) / |S|^2, both taken from q once per iteration, so one
//              candidate costs K(K-1)/2 descriptor distances instead of 2^K
//              label vectors.  A pixel whose M-step returns the previous
//              candidate has reached its fixed point (q depends on d only).
//   joint MAP  (d, S) = arg-max of J(d, S) over every candidate and every
//              label vector (lowest candidate first, then smallest mask):
//              the E-step enumeration run at each of the D candidates.
//
// Both modes write the same outputs as the EM: candidate index and value,
// the labels at the final candidate (the arg-max over S), the per-ray
// marginals of q(S) at the final candidate, and in dynamic-only mode the
// stand-in outputs of the pixels it skips.
#pragma once

#include "em_sweep.cuh"

namespace lf {
namespace dev {

constexpr int kModeSoft = 1, kModeJoint = 2;
constexpr int kSoftMaxCams = 8;  // K(K-1)/2 pair weights live in registers

template <int K>
constexpr int kNumPairs = K * (K - 1) / 2 > 0 ? K * (K - 1) / 2 : 1;

// q(S) ~ exp J(d, S) at the candidate the rays were sampled at (emax = the
// maximum of J over S, without the prior, which q does not depend on).
// pi[k] = sum over S containing k of q(S); pw[pair (k, l)] = sum over S
// containing k and l of q(S) / |S|^2 (pairs in order (0,1), (0,2), ...,
// (1,2), ...).
template <int K>
__device__ __forceinline__ void soft_posterior(const Rays& r, const float* s_rcp, float beta, float emax,
                                               float (&pi)[K], float (&pw)[kNumPairs<K>]) {
#pragma unroll
  for (int k = 0; k < K; ++k) pi[k] = 0.f;
#pragma unroll
  for (int i = 0; i < kNumPairs<K>; ++i) pw[i] = 0.f;
  float Z = 0.f;
  for (unsigned m = 0; m < (1u << K); ++m) {
    Acc acc{0.f, 0.f, 0.f, 0.f, 0.f};
    int n = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (m >> k & 1u) {
        acc.sy += r.gy[k]; acc.sx += r.gx[k]; acc.sz += r.gz[k];
        acc.q += r.qk[k]; acc.sa += r.ak[k];
        ++n;
      }
    }
    const float rn = s_rcp[n];
    const float e = expf(leaf_objective(acc, rn, r.base, beta) - emax);
    Z += e;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (m >> k & 1u) pi[k] += e;
    const float c = e * rn * rn;
    int p = 0;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int l = k + 1; l < K; ++l) {
        if ((m >> k) & (m >> l) & 1u) pw[p] += c;
        ++p;
      }
  }
  const float inv = 1.f / Z;
#pragma unroll
  for (int k = 0; k < K; ++k) pi[k] *= inv;
#pragma unroll
  for (int i = 0; i < kNumPairs<K>; ++i) pw[i] *= inv;
}

// Soft-EM M-step: arg-max of Q(d_j) over candidates j0 <= j < j1 (lowest j
// on ties; *best_out = the maximum).  Each candidate is evaluated from
// scratch, so a range computes the same objectives as the whole sweep.
template <int K>
__device__ __forceinline__ int m_step_soft(const SweepArgs& a, const Staged<float>& st, const float2* s_wq,
                                           const int* s_o, const float* s_d, float cy, float cx, float cz,
                                           float mu, bool inside, const float* pi, const float* pw, int j0,
                                           int j1, float* best_out) {
  using Tx = Texels<float>;
  const int SWp = st.SWp;
  const float2 ref1 = make_float2(-cy, -cx), ref2 = make_float2(-cz, 0.f);
  float best = -INFINITY;
  int jb = j0;
  auto prior_at = [&](int j) {
    const float t = s_d[j] - mu;
    return __logf(a.gamma + __expf(-(t * t) * a.inv2s2));
  };
  float pr_next = j0 < j1 ? prior_at(j0) : 0.f;
  for (int j = j0; j < j1; ++j) {
    const float pr = pr_next;
    pr_next = prior_at(min(j + 1, j1 - 1));  // the next candidate's prior, off this one's critical path
    float gy[K], gx[K], gz[K];
    float seg = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float w = s_wq[j * a.KP + k].x;
      const int c = st.cbase + s_o[j * a.KP + k];
      const uint8_t* R = st.row(k);
      float2 yx0, zd0, yx1, zd1;
      Tx::quad(R, SWp, c, yx0, zd0);
      Tx::quad(R, SWp, c + 1, yx1, zd1);
      const float S0 = Tx::ls(R, SWp, c), S1 = Tx::ls(R, SWp, c + 1);
      const float2 ww = make_float2(w, w);
      const float2 g1 = ffma2(ww, fsub2(yx1, yx0), fadd2(yx0, ref1));  // (gy, gx)
      const float2 g2 = ffma2(ww, fsub2(zd1, zd0), fadd2(zd0, ref2));  // (gz, ld)
      gy[k] = g1.x;
      gx[k] = g1.y;
      gz[k] = g2.x;
      const float ls = fmaf(w, S1 - S0, S0), ld = g2.y;
      seg += fmaf(pi[k], ls - ld, ld);
    }
    float pv = 0.f;
    int p = 0;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int l = k + 1; l < K; ++l) {
        const float dy = gy[k] - gy[l], dx = gx[k] - gx[l], dz = gz[k] - gz[l];
        pv = fmaf(pw[p], fmaf(dz, dz, fmaf(dx, dx, dy * dy)), pv);
        ++p;
      }
    float J = a.mseg ? seg : 0.f;
    if (inside) J += pr;
    J = fmaf(-a.beta, pv, J);
    if (J > best) { best = J; jb = j; }
  }
  if (best_out) *best_out = best;
  return jb;
}

// Joint MAP over (d, S): the E-step's subset-tree arg-max at every candidate
// plus the candidate's prior.  Returns j; S and emax (J at (j, S) without the
// prior) through the references.
template <int K>
__device__ __forceinline__ int joint_map(const SweepArgs& a, const Staged<float>& st, const float2* s_wq,
                                         const int* s_o, const float* s_d, const float* s_rcp, float cy, float cx,
                                         float cz, float mu, bool inside, unsigned& S, float& emax) {
  float best = -INFINITY;
  int jb = 0;
  unsigned Sb = 0;
  float eb = 0.f;
  for (int j = 0; j < a.D; ++j) {
    Rays r;
    sample_rays<K, float>(a, st, s_wq, s_o, j, cy, cx, cz, r);
    unsigned m = 0;
    float e = 0.f;
    enumerate<0, K>(r, s_rcp, a.beta, 0.f, m, e, nullptr);
    float J = e;
    if (inside) {
      const float t = s_d[j] - mu;
      J += __logf(a.gamma + __expf(-(t * t) * a.inv2s2));
    }
    if (J > best) { best = J; jb = j; Sb = m; eb = e; }
  }
  S = Sb;
  emax = eb;
  return jb;
}

// Soft-EM state of one pixel between iterations, in shared memory after the
// sweep layout: pi[K] then the pair weights, per tile pixel.
template <int K>
constexpr int kSoftStateFloats = K + kNumPairs<K>;
static_assert(kSoftStateFloats<1> == soft_state_floats(1) && kSoftStateFloats<2> == soft_state_floats(2) &&
                  kSoftStateFloats<8> == soft_state_floats(8),
              "device and host sizes of the soft-EM state must agree");

// One tile.  Joint MAP: one thread per pixel (every pixel does the same
// work).  Soft EM: the first iteration one thread per pixel, then only the
// pixels not yet at their fixed point, regrouped into dense warps before
// every pass, and groups of 2 to 32 lanes per pixel once fewer are left than
// the CTA has threads (lanes split the candidates; same tie rule, same
// bits).
template <int K, int MODE>
__device__ __forceinline__ void variant_tile(const SweepArgs& a, const CUtensorMap* img_map,
                                             const CUtensorMap* p_map, int tile_x, int tile_y, uint8_t* smem) {
  if (!stage_tile<K, float>(a, img_map, p_map, tile_x, tile_y, smem, 0u, true, false)) return;
  const SmemLayout Ly = sweep_layout(K, a);
  const float* s_p = reinterpret_cast<const float*>(smem + Ly.raw_p);
  const uint8_t* s_feat = smem + Ly.feat;
  const float2* s_wq = reinterpret_cast<const float2*>(smem + Ly.wtab);
  const int* s_o = reinterpret_cast<const int*>(smem + Ly.otab);
  const unsigned* s_chg = reinterpret_cast<const unsigned*>(smem + Ly.chg);
  const float* s_d = reinterpret_cast<const float*>(smem + Ly.dval);
  const float* s_rcp = reinterpret_cast<const float*>(smem + Ly.rcp);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int u0 = tile_x * a.TW, v0 = tile_y * a.TR;
  const int cs = floor16(u0 - a.L - 1);
  const int cam_stride = a.TR * a.SWp * texel_bytes(a.prec);
  const size_t HW = static_cast<size_t>(a.H) * a.W;

  const PixelCtx<float> me = load_pixel<float>(a, s_feat, u0, v0, cam_stride, tid);
  bool run = me.valid;
  if (a.dyn_only && run) {  // Sec. III-F: only the reference pixels flagged dynamic
    const int r = tid / a.TW;
    const float Pref = s_p[(static_cast<size_t>(a.ref) * a.TR + r) * a.RW + (me.u - cs)];
    if (!(Pref >= a.seg_threshold)) {
      write_static_pixel<K>(a, me.u, me.v, me.mu);
      run = false;
    }
  }
  if constexpr (MODE == kModeJoint) {
    unsigned executed = 0;
    if (run) {
      unsigned S = 0;
      float emax = 0.f;
      const int jb = joint_map<K>(a, me.st, s_wq, s_o, s_d, s_rcp, me.cy, me.cx, me.cz, me.mu, me.inside, S, emax);
      executed = 1;
      const size_t pix = static_cast<size_t>(me.v) * a.W + me.u;
      a.d_idx[pix] = jb;
      if (a.d_out) a.d_out[pix] = s_d[jb];
      if (a.labels) a.labels[pix] = static_cast<uint16_t>(S);
      if (a.post) {
        Rays rays;
        sample_rays<K, float>(a, me.st, s_wq, s_o, jb, me.cy, me.cx, me.cz, rays);
        float post[K];
        unsigned dummy;
        float dummyf;
        enumerate<1, K>(rays, s_rcp, a.beta, emax, dummy, dummyf, post);
#pragma unroll
        for (int k = 0; k < K; ++k) a.post[k * HW + pix] = post[k];
      }
    }
    const unsigned warp_sum = __reduce_add_sync(0xffffffffu, executed);
    if (lane == 0 && warp_sum) atomicAdd(a.counter, static_cast<unsigned long long>(warp_sum) * a.D);
  } else {
    PixelState ps = pixel_state(smem + Ly.pix, a.TR * a.TW);
    int* s_wcnt = reinterpret_cast<int*>(smem + Ly.wcnt);
    float* s_soft = reinterpret_cast<float*>(smem + soft_state_offset(K, a));
    constexpr int NS = kSoftStateFloats<K>;
    static_assert(NS == soft_state_floats(K), "soft-EM state size");
    // E-step at candidate j (q(S) from the rays there) into pixel p's state
    auto e_step = [&](const PixelCtx<float>& c, int p, int j) {
      Rays rays;
      sample_rays<K, float>(a, c.st, s_wq, s_o, j, c.cy, c.cx, c.cz, rays);
      unsigned S = 0;
      float emax = 0.f;
      enumerate<0, K>(rays, s_rcp, a.beta, 0.f, S, emax, nullptr);
      float pi[K], pw[kNumPairs<K>];
      soft_posterior<K>(rays, s_rcp, a.beta, emax, pi, pw);
      float* st = s_soft + p * NS;
#pragma unroll
      for (int k = 0; k < K; ++k) st[k] = pi[k];
#pragma unroll
      for (int i = 0; i < kNumPairs<K>; ++i) st[K + i] = pw[i];
      ps.jb[p] = static_cast<int16_t>(j);
      ps.S[p] = static_cast<uint16_t>(S);
      ps.emax[p] = emax;
    };
    unsigned long long executed = 0;
    // t = 1: the EM's first M-step (labels thresholded per candidate)
    if (run) {
      unsigned S0 = 0, ns = 0;
      float seg_max;
      const bool f0 = constant_initial_labels<K, float>(a, me.st, &S0, &seg_max);
      const int jb = f0 ? m_step_fixed<K, float, -1>(a, me.st, s_wq, s_o, s_chg, s_d, s_rcp, me.cy, me.cx, me.cz, me.mu,
                                                 me.inside, S0)
                        : m_step_init<K, float, -1>(a, me.st, s_wq, s_o, s_chg, s_d, s_rcp, me.cy, me.cx, me.cz, me.mu,
                                                 me.inside, &ns);
      e_step(me, tid, jb);
    }
    ps.conv[tid] = 0;
    executed = static_cast<unsigned long long>(__syncthreads_count(run));
    for (int t = 2; t <= a.iters; ++t) {
      const int n = compact(run && !ps.conv[tid], ps.list, 0, s_wcnt);
      if (n == 0) break;
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
          const int p = ps.list[act ? slot : n - 1];  // idle groups repeat the last pixel
          const PixelCtx<float> c = load_pixel<float>(a, s_feat, u0, v0, cam_stride, p);
          const float* st = s_soft + p * NS;
          const int per = (a.D + G - 1) / G, j0 = min(gl * per, a.D), j1 = min(j0 + per, a.D);
          float jbest;
          unsigned jn = static_cast<unsigned>(m_step_soft<K>(a, c.st, s_wq, s_o, s_d, c.cy, c.cx, c.cz, c.mu,
                                                             c.inside, st, st + K, j0, j1, &jbest));
          group_argmax(jbest, jn, G);
          const bool conv = a.early_exit && static_cast<int>(jn) == ps.jb[p];  // q_t would equal q_{t-1}
          __syncwarp();
          // the E-step whenever some group of the warp goes on (every lane
          // takes part in its shuffles; the converged groups discard it)
          if (!__all_sync(0xffffffffu, conv)) {
            Rays rays;
            sample_rays<K, float>(a, c.st, s_wq, s_o, static_cast<int>(jn), c.cy, c.cx, c.cz, rays);
            unsigned S = 0;
            float emax = 0.f;
            enumerate_group<K>(rays, s_rcp, a.beta, gl, G, S, emax);
            float pi[K], pw[kNumPairs<K>];
            soft_posterior<K>(rays, s_rcp, a.beta, emax, pi, pw);
            __syncwarp();
            if (act && gl == 0 && !conv) {
              float* sto = s_soft + p * NS;
#pragma unroll
              for (int k = 0; k < K; ++k) sto[k] = pi[k];
#pragma unroll
              for (int q = 0; q < kNumPairs<K>; ++q) sto[K + q] = pw[q];
              ps.jb[p] = static_cast<int16_t>(jn);
              ps.S[p] = static_cast<uint16_t>(S);
              ps.emax[p] = emax;
            }
          }
          if (act && gl == 0 && conv) ps.conv[p] = 1;
        }
      } else if (tid < n) {
        const int p = ps.list[tid];
        const PixelCtx<float> c = load_pixel<float>(a, s_feat, u0, v0, cam_stride, p);
        const float* st = s_soft + p * NS;
        const int jn = m_step_soft<K>(a, c.st, s_wq, s_o, s_d, c.cy, c.cx, c.cz, c.mu, c.inside, st, st + K, 0,
                                      a.D, nullptr);
        if (a.early_exit && jn == ps.jb[p]) ps.conv[p] = 1;  // q_t would equal q_{t-1}: fixed point
        else e_step(c, p, jn);
      }
      __syncthreads();
    }
    if (run) {
      const size_t pix = static_cast<size_t>(me.v) * a.W + me.u;
      const int jb = ps.jb[tid];
      a.d_idx[pix] = jb;
      if (a.d_out) a.d_out[pix] = s_d[jb];
      if (a.labels) a.labels[pix] = ps.S[tid];
      if (a.post) {
        const float* st = s_soft + tid * NS;
#pragma unroll
        for (int k = 0; k < K; ++k) a.post[k * HW + pix] = st[k];
      }
    }
    if (tid == 0 && executed) atomicAdd(a.counter, executed * a.D);  // every candidate of every sweep
  }
}

// Two CTAs per SM (at most 128 registers) for soft EM up to seven cameras
// and joint MAP up to eight; one above.
template <int K, int MODE>
constexpr int variant_min_blocks() {
  return (MODE == kModeSoft && K <= 7) || (MODE == kModeJoint && K <= 8) ? 2 : 1;
}

template <int K, int MODE>
__global__ void __launch_bounds__(256, variant_min_blocks<K, MODE>()) em_variant_kernel(const __grid_constant__ CUtensorMap img_map,
                                                         const __grid_constant__ CUtensorMap p_map,
                                                         const SweepArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  if ((smem_u32(smem) & 127u) != 0u) {  // TMA destinations must be 128-byte aligned
    if (threadIdx.x == 0) atomicOr(a.status, kStatusSmemMisaligned);
    return;
  }
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
  variant_tile<K, MODE>(a, &img_map, &p_map, tx, ty, smem);
}

template <int K, int MODE>
cudaError_t launch_em_variant_k(const CUtensorMap& img_map, const CUtensorMap& p_map, const SweepArgs& a,
                                cudaStream_t s) {
  const size_t smem = MODE == kModeSoft ? soft_state_offset(K, a) + soft_state_bytes(K, a.TR * a.TW)
                                        : sweep_layout(K, a).total;
  static int configured = -1;  // largest dynamic shared size set so far (per process)
  if (static_cast<int>(smem) > configured) {
    cudaError_t e = cudaFuncSetAttribute(em_variant_kernel<K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    configured = static_cast<int>(smem);
  }
  dim3 grid((a.W + a.TW - 1) / a.TW, (a.H + a.TR - 1) / a.TR);
  if (a.tile_list) grid = dim3(grid.x * grid.y, 1);
  em_variant_kernel<K, MODE><<<grid, a.TR * a.TW, smem, s>>>(img_map, p_map, a);
  return cudaGetLastError();
}

}  // namespace dev
}  // namespace lf

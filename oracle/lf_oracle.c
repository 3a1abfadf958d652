/*
 * FP64 CPU oracle for the per-pixel EM of Kaveti, Katt & Singh, "Removing
 * Dynamic Objects for Static Scene Reconstruction using Light Fields"
 * (arXiv 2003.11076).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the CUDA path computes.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may build, load or call it; the
 * library never does.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * Every step follows the paper's definitions in the paper's order, in double
 * precision, with no blocking, fusion or reordering.  Where the paper is
 * silent, the reading taken is stated at the step:
 *
 *   features      f = [Y, Sobel-x/8, Sobel-y/8] of the luminance, 3x3 Sobel
 *                 with the border replicated (Sec. III-C "Pixel Likelihood")
 *   ray sampling  x_k = u - d * b_k on row v, column clamped to the image,
 *                 linear interpolation for non-integral shifts (Eq. 1 for a
 *                 rectified linear array; Sec. III-F non-integral disparities);
 *                 for a calibrated array, the homography of the plane at
 *                 generalized disparity d (a 3x4 matrix per camera, Eq. 1 and
 *                 the warping function of Sec. III-C), bilinear interpolation
 *                 with both coordinates clamped
 *   likelihood    -beta * Var_S(f): population variance over the static rays,
 *                 0 when at most one ray is static (Sec. III-C)
 *   prior         log(gamma + exp(-(d - mu)^2 / (2 sigma^2))) inside the
 *                 triangulation, 0 (uniform) outside (Sec. III-C "Disparity Prior")
 *   segmentation  sum_k S^k log(1 - P_k) + (1 - S^k) log(P_k) with P the
 *                 input probability that the ray is dynamic (Eq. e-step general)
 *   EM schedule   M-step first, with S thresholded at P >= 0.7 at each
 *                 candidate's own sample, then E-step, repeat (Sec. III-B
 *                 schedule, Sec. III-F threshold)
 *   variants      soft EM: after the first iteration the M-step maximises
 *                 sum_S q(S) J(d, S) with q the previous E-step's posterior
 *                 over all 2^K label vectors; joint MAP: the arg-max of
 *                 J(d, S) over every (d, S) pair (Sec. III-B, Sec. III-C)
 *   outputs       d, hard S, per-ray marginals of q(S) ~ exp J(d_T, S), and
 *                 the refocused image of Eq. 2 (Sec. III-E)
 *   median        3x3 per channel, border replicated (Sec. III-E)
 *
 * Parity status: every function here is pinned by the CPU test-suite against
 * closed forms, special cases, brute force or library routines.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double beta;          /* weight of the photometric variance */
    double gamma;         /* uniform floor of the disparity prior */
    double sigma;         /* width of the sampled Gaussian, disparity units */
    double seg_threshold; /* initial segmentation threshold on P(dynamic) (0.7) */
    double eps;           /* floor inside the log of the segmentation prior */
    int mstep_seg_term;   /* 1: M-step maximises the complete-data J */
    int em_mode;          /* 0: hard EM (the paper's), 1: soft EM, 2: joint MAP */
} orc_params;

/* ---------------------------------------------------------------- inputs */

/* Image value in [0,1] of camera k, row v, column u, channel c.
 * dtype 0 = uint8 (scaled by 1/255), 1 = float32. */
static double img_at(const void *images, int dtype, int H, int W, int C,
                     int k, int v, int u, int c)
{
    size_t idx = (((size_t)k * H + v) * W + u) * C + c;
    if (dtype == 0) return ((const uint8_t *)images)[idx] / 255.0;
    return (double)((const float *)images)[idx];
}

/* Luminance Y: gray images are used as is; RGB uses the BT.601 weights. */
static double luma_at(const void *images, int dtype, int H, int W, int C,
                      int k, int v, int u)
{
    if (C == 1) return img_at(images, dtype, H, W, C, k, v, u, 0);
    return 0.299 * img_at(images, dtype, H, W, C, k, v, u, 0)
         + 0.587 * img_at(images, dtype, H, W, C, k, v, u, 1)
         + 0.114 * img_at(images, dtype, H, W, C, k, v, u, 2);
}

static int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* Descriptor maps (Sec. III-C: "3x3 sobel filter responses").
 * feat is [K][3][H][W]: channel 0 = Y, 1 = Sobel-x / 8, 2 = Sobel-y / 8,
 * computed on Y with the border replicated. */
void orc_features(int K, int H, int W, int C, int dtype, const void *images, double *feat)
{
    double *Y = (double *)malloc(sizeof(double) * (size_t)H * W);
    for (int k = 0; k < K; ++k) {
        for (int v = 0; v < H; ++v)
            for (int u = 0; u < W; ++u)
                Y[(size_t)v * W + u] = luma_at(images, dtype, H, W, C, k, v, u);
        for (int v = 0; v < H; ++v) {
            for (int u = 0; u < W; ++u) {
                double n[3][3];
                for (int dv = -1; dv <= 1; ++dv)
                    for (int du = -1; du <= 1; ++du)
                        n[dv + 1][du + 1] = Y[(size_t)clampi(v + dv, 0, H - 1) * W + clampi(u + du, 0, W - 1)];
                /* Sobel kernels: x = [-1 0 1; -2 0 2; -1 0 1], y = its transpose */
                double gx = (n[0][2] + 2.0 * n[1][2] + n[2][2]) - (n[0][0] + 2.0 * n[1][0] + n[2][0]);
                double gy = (n[2][0] + 2.0 * n[2][1] + n[2][2]) - (n[0][0] + 2.0 * n[0][1] + n[0][2]);
                size_t base = (size_t)k * 3 * H * W + (size_t)v * W + u;
                feat[base] = n[1][1];
                feat[base + (size_t)H * W] = gx / 8.0;
                feat[base + 2 * (size_t)H * W] = gy / 8.0;
            }
        }
    }
    free(Y);
}

/* Log segmentation prior (Sec. III-B; the input P is the probability that the
 * pixel is dynamic, the Bodypix convention of Sec. III-F):
 * ls = log max(1 - P, eps) = log p(S = static), ld = log max(P, eps). */
void orc_log_seg(int K, int H, int W, const float *seg_prior, double eps, double *ls, double *ld)
{
    size_t n = (size_t)K * H * W;
    for (size_t i = 0; i < n; ++i) {
        double P = (double)seg_prior[i];
        ls[i] = log(fmax(1.0 - P, eps));
        ld[i] = log(fmax(P, eps));
    }
}

/* Linear interpolation along a row at continuous column x with the column
 * clamped to [0, W-1]: i0 = floor(x), i1 = min(i0 + 1, W - 1). */
static double sample_row(const double *row, int W, double x)
{
    if (x < 0.0) x = 0.0;
    if (x > (double)(W - 1)) x = (double)(W - 1);
    int i0 = (int)floor(x);
    int i1 = i0 + 1 < W ? i0 + 1 : W - 1;
    double w = x - (double)i0;
    return (1.0 - w) * row[i0] + w * row[i1];
}

/* ------------------------------------------------------------- the model */

/* Disparity prior, Sec. III-C "Disparity Prior" and the M-step energy:
 * log p(d | T, x_ref) = log(gamma + exp(-(d - mu)^2 / (2 sigma^2))) where mu is
 * the triangulation's interpolated disparity; uniform (0) outside it. */
static double log_prior(double d, double mu, int inside, const orc_params *p)
{
    if (!inside) return 0.0;
    double t = d - mu;
    return log(p->gamma + exp(-(t * t) / (2.0 * p->sigma * p->sigma)));
}

/* Population variance of the descriptors of the static rays (Sec. III-C
 * "Pixel Likelihood"): mean over S, then mean squared distance, summed over
 * the 3 descriptor channels; 0 when fewer than two rays are static. */
static double variance_static(int K, const double f[][3], unsigned S)
{
    int n = 0;
    double mean[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < K; ++k)
        if (S >> k & 1u) {
            ++n;
            for (int c = 0; c < 3; ++c) mean[c] += f[k][c];
        }
    if (n <= 1) return 0.0;
    for (int c = 0; c < 3; ++c) mean[c] /= n;
    double acc = 0.0;
    for (int k = 0; k < K; ++k)
        if (S >> k & 1u)
            for (int c = 0; c < 3; ++c) {
                double e = f[k][c] - mean[c];
                acc += e * e;
            }
    return acc / n;
}

/* log p(S | S_P) = sum_k S^k log p(static) + (1 - S^k) log p(dynamic). */
static double seg_term(int K, const double *ls, const double *ld, unsigned S)
{
    double acc = 0.0;
    for (int k = 0; k < K; ++k) acc += (S >> k & 1u) ? ls[k] : ld[k];
    return acc;
}

/* Complete-data objective J(d, S) = -beta Var_S + log p(d|T) + log p(S|S_P)
 * (Eqs. m-step 1 and m-step 2 with the likelihood of Sec. III-C). */
static double objective(int K, const double f[][3], const double *ls, const double *ld,
                        unsigned S, double lp, int with_seg, const orc_params *p)
{
    double J = -p->beta * variance_static(K, f, S) + lp;
    if (with_seg) J += seg_term(K, ls, ld, S);
    return J;
}

typedef struct {
    int K, H, W, C, dtype, D;
    const double *b;      /* [K] baselines (rectified linear array) */
    const double *P;      /* [K][3][4] camera matrices (calibrated array), or NULL */
    int ref;              /* reference camera */
    const double *dval;   /* [D] candidate disparities */
    const double *feat;   /* [K][3][H][W] */
    const double *ls, *ld;/* [K][H][W] */
    const void *images;
    const orc_params *p;
} orc_frame;

/* Where the ray of reference pixel (u, v) at disparity d meets camera k
 * (Eq. 1).  Calibrated array: the 3x4 matrix M_k maps (u, v, 1, d) to
 * homogeneous pixel coordinates of camera k -- in generalized disparity space
 * this is the homography of the plane at disparity d (the warping function
 * W_k of Sec. III-C).  Rectified linear array (no matrices): x = u - d b_k on
 * row v. */
static void ray_position(const orc_frame *F, int k, int u, int v, double d, double *x, double *y)
{
    if (!F->P) {
        *x = (double)u - d * F->b[k];
        *y = (double)v;
        return;
    }
    const double *M = F->P + 12 * (size_t)k;
    double X = M[0] * u + M[1] * v + M[2] + M[3] * d;
    double Y = M[4] * u + M[5] * v + M[6] + M[7] * d;
    double Z = M[8] * u + M[9] * v + M[10] + M[11] * d;
    *x = X / Z;
    *y = Y / Z;
}

/* Bilinear interpolation of an H x W map at (x, y) with each coordinate
 * clamped to the image: the two-dimensional form of sample_row. */
static double sample_2d(const double *map, int H, int W, double x, double y)
{
    if (x < 0.0) x = 0.0;
    if (x > (double)(W - 1)) x = (double)(W - 1);
    if (y < 0.0) y = 0.0;
    if (y > (double)(H - 1)) y = (double)(H - 1);
    int i0 = (int)floor(x), j0 = (int)floor(y);
    int i1 = i0 + 1 < W ? i0 + 1 : W - 1;
    int j1 = j0 + 1 < H ? j0 + 1 : H - 1;
    double wx = x - (double)i0, wy = y - (double)j0;
    double top = (1.0 - wx) * map[(size_t)j0 * W + i0] + wx * map[(size_t)j0 * W + i1];
    double bot = (1.0 - wx) * map[(size_t)j1 * W + i0] + wx * map[(size_t)j1 * W + i1];
    return (1.0 - wy) * top + wy * bot;
}

/* Sample the K rays of reference pixel (u, v) at disparity d (Eq. 1; see
 * ray_position). */
static void sample_rays(const orc_frame *F, int u, int v, double d,
                        double f[][3], double *ls, double *ld)
{
    size_t HW = (size_t)F->H * F->W;
    for (int k = 0; k < F->K; ++k) {
        double x, y;
        ray_position(F, k, u, v, d, &x, &y);
        if (!F->P) {
            for (int c = 0; c < 3; ++c)
                f[k][c] = sample_row(F->feat + (size_t)k * 3 * HW + (size_t)c * HW + (size_t)v * F->W, F->W, x);
            ls[k] = sample_row(F->ls + (size_t)k * HW + (size_t)v * F->W, F->W, x);
            ld[k] = sample_row(F->ld + (size_t)k * HW + (size_t)v * F->W, F->W, x);
        } else {
            for (int c = 0; c < 3; ++c)
                f[k][c] = sample_2d(F->feat + (size_t)k * 3 * HW + (size_t)c * HW, F->H, F->W, x, y);
            ls[k] = sample_2d(F->ls + (size_t)k * HW, F->H, F->W, x, y);
            ld[k] = sample_2d(F->ld + (size_t)k * HW, F->H, F->W, x, y);
        }
    }
}

#define ORC_MAXK 16

/* Posterior over the label vectors at one disparity (Sec. III-B: the E-step
 * of EM computes p(S | x, d)): q[S] = exp J(d, S) / sum_S' exp J(d, S') over
 * all 2^K vectors, with the rays already sampled at d.  Returns
 * log sum_S exp J(d, S) (the log marginal of the observations at d, up to a
 * constant) with the prior lp included. */
static double label_posterior(int K, const double f[][3], const double *ls, const double *ld,
                              double lp, const orc_params *p, double *q)
{
    double Jmax = -INFINITY;
    for (unsigned s = 0; s < (1u << K); ++s) {
        q[s] = objective(K, f, ls, ld, s, lp, 1, p);
        if (q[s] > Jmax) Jmax = q[s];
    }
    double Z = 0.0;
    for (unsigned s = 0; s < (1u << K); ++s) {
        q[s] = exp(q[s] - Jmax);
        Z += q[s];
    }
    for (unsigned s = 0; s < (1u << K); ++s) q[s] /= Z;
    return Jmax + log(Z);
}

/* One reference pixel through the whole EM (Sec. III-B schedule, M-step
 * first).  Writes outputs and per-iteration diagnostics. */
static void em_pixel(const orc_frame *F, int u, int v, double mu, int inside, int iters,
                     int32_t *d_idx, double *d_val, uint16_t *labels, double *post,
                     double *refocus, double *m_margin, double *e_margin, double *J_t,
                     double *init_margin)
{
    const orc_params *p = F->p;
    const int K = F->K, D = F->D, W = F->W, H = F->H;
    const size_t pix = (size_t)v * W + u, HW = (size_t)H * W;
    const double log_thr = log(p->seg_threshold / (1.0 - p->seg_threshold));
    double f[ORC_MAXK][3], ls[ORC_MAXK], ld[ORC_MAXK];
    unsigned S = 0;
    int jbest = 0;
    double imargin = INFINITY;
    /* soft EM: posterior over the label vectors from the previous E-step */
    double *q = p->em_mode == 1 ? (double *)malloc(sizeof(double) * ((size_t)1 << K)) : NULL;

    if (p->em_mode == 2) {
        /* ---- joint MAP: (d, S) = argmax over every candidate and every
         * label vector of J(d, S) (Sec. III-C considers all 2^K
         * configurations); lowest d index first, then smallest mask.  There
         * is nothing to iterate: every diagnostic slot holds the one result. */
        double Mbest = -INFINITY, Msecond = -INFINITY;
        unsigned Sbest = 0;
        for (int j = 0; j < D; ++j) {
            double d = F->dval[j];
            sample_rays(F, u, v, d, f, ls, ld);
            double lp = log_prior(d, mu, inside, p);
            double Mj = -INFINITY;
            unsigned Sj = 0;
            for (unsigned s = 0; s < (1u << K); ++s) {
                double J = objective(K, (const double(*)[3])f, ls, ld, s, lp, 1, p);
                if (J > Mj) { Mj = J; Sj = s; }
            }
            if (Mj > Mbest) { Msecond = Mbest; Mbest = Mj; jbest = j; Sbest = Sj; }
            else if (Mj > Msecond) Msecond = Mj;
        }
        S = Sbest;
        sample_rays(F, u, v, F->dval[jbest], f, ls, ld);
        double eb = -INFINITY, es = -INFINITY;
        for (unsigned s = 0; s < (1u << K); ++s) {
            double J = objective(K, (const double(*)[3])f, ls, ld, s, 0.0, 1, p);
            if (J > eb) { es = eb; eb = J; }
            else if (J > es) es = J;
        }
        for (int t = 1; t <= iters; ++t) {
            m_margin[(size_t)(t - 1) * HW + pix] = Mbest - Msecond;
            e_margin[(size_t)(t - 1) * HW + pix] = eb - es;
            J_t[(size_t)(t - 1) * HW + pix] = Mbest;
        }
        iters = 0;  /* skip the EM loop below */
    }

    for (int t = 1; t <= iters; ++t) {
        /* ---- M-step: d = argmax_d J(d, S), lowest index on ties */
        double best = -INFINITY, second = -INFINITY;
        int jb = 0;
        for (int j = 0; j < D; ++j) {
            double d = F->dval[j];
            sample_rays(F, u, v, d, f, ls, ld);
            unsigned Sj = S;
            if (t == 1) {
                /* first iteration: S^k static iff the prior at the ray's own
                 * sample is below the threshold (Sec. III-F):
                 * ld - ls < log(thr / (1 - thr)). */
                Sj = 0;
                for (int k = 0; k < K; ++k) {
                    double z = ld[k] - ls[k] - log_thr;
                    if (fabs(z) < imargin) imargin = fabs(z);
                    if (z < 0.0) Sj |= 1u << k;
                }
            }
            double J;
            if (p->em_mode == 1 && t > 1) {
                /* soft EM (Sec. III-B, Eq. m-step 1 as an expectation): the
                 * expected complete-data objective under the previous
                 * posterior, Q(d) = sum_S q(S) J(d, S) */
                J = 0.0;
                for (unsigned s = 0; s < (1u << K); ++s)
                    J += q[s] * objective(K, (const double(*)[3])f, ls, ld, s,
                                          log_prior(d, mu, inside, p), p->mstep_seg_term, p);
            } else {
                J = objective(K, (const double(*)[3])f, ls, ld, Sj,
                              log_prior(d, mu, inside, p), p->mstep_seg_term, p);
            }
            if (J > best) { second = best; best = J; jb = j; }
            else if (J > second) second = J;
        }
        jbest = jb;
        m_margin[(size_t)(t - 1) * HW + pix] = best - second;

        /* ---- E-step: S = argmax over all 2^K label vectors of J(d_t, S)
         * (Eq. e-step general, hard assignment), smallest mask on ties. */
        double d = F->dval[jbest];
        sample_rays(F, u, v, d, f, ls, ld);
        double eb = -INFINITY, es = -INFINITY;
        unsigned Sb = 0;
        for (unsigned s = 0; s < (1u << K); ++s) {
            double J = objective(K, (const double(*)[3])f, ls, ld, s, 0.0, 1, p);
            if (J > eb) { es = eb; eb = J; Sb = s; }
            else if (J > es) es = J;
        }
        S = Sb;
        e_margin[(size_t)(t - 1) * HW + pix] = eb - es;
        if (p->em_mode == 1)  /* soft EM: the posterior for the next M-step and
                               * the log marginal, which EM never decreases */
            J_t[(size_t)(t - 1) * HW + pix] =
                label_posterior(K, (const double(*)[3])f, ls, ld, log_prior(d, mu, inside, p), p, q);
        else
            J_t[(size_t)(t - 1) * HW + pix] = eb + log_prior(d, mu, inside, p);
    }
    init_margin[pix] = imargin;
    free(q);

    /* ---- outputs at (d_T, S_T) */
    double d = F->dval[jbest];
    d_idx[pix] = jbest;
    d_val[pix] = d;
    labels[pix] = (uint16_t)S;
    sample_rays(F, u, v, d, f, ls, ld);
    /* per-ray marginals of q(S) = exp J(d_T, S) / sum_S' exp J(d_T, S') */
    double Jmax = -INFINITY;
    for (unsigned s = 0; s < (1u << K); ++s) {
        double J = objective(K, (const double(*)[3])f, ls, ld, s, 0.0, 1, p);
        if (J > Jmax) Jmax = J;
    }
    double Z = 0.0, m[ORC_MAXK];
    for (int k = 0; k < K; ++k) m[k] = 0.0;
    for (unsigned s = 0; s < (1u << K); ++s) {
        double q = exp(objective(K, (const double(*)[3])f, ls, ld, s, 0.0, 1, p) - Jmax);
        Z += q;
        for (int k = 0; k < K; ++k)
            if (s >> k & 1u) m[k] += q;
    }
    for (int k = 0; k < K; ++k) post[(size_t)k * HW + pix] = m[k] / Z;

    /* refocused static image, Eq. 2; no static ray keeps the reference pixel */
    int n = 0;
    for (int k = 0; k < K; ++k) n += (S >> k) & 1u;
    const int ref = F->ref;
    for (int c = 0; c < F->C; ++c) {
        double acc = 0.0;
        if (n == 0) {
            acc = img_at(F->images, F->dtype, H, W, F->C, ref, v, u, c);
        } else {
            for (int k = 0; k < K; ++k) {
                if (!(S >> k & 1u)) continue;
                double x, y;
                ray_position(F, k, u, v, d, &x, &y);
                if (x < 0.0) x = 0.0;
                if (x > (double)(W - 1)) x = (double)(W - 1);
                int i0 = (int)floor(x);
                int i1 = i0 + 1 < W ? i0 + 1 : W - 1;
                double w = x - (double)i0;
                if (!F->P) {
                    acc += (1.0 - w) * img_at(F->images, F->dtype, H, W, F->C, k, v, i0, c)
                         + w * img_at(F->images, F->dtype, H, W, F->C, k, v, i1, c);
                } else {
                    if (y < 0.0) y = 0.0;
                    if (y > (double)(H - 1)) y = (double)(H - 1);
                    int j0 = (int)floor(y);
                    int j1 = j0 + 1 < H ? j0 + 1 : H - 1;
                    double wy = y - (double)j0;
                    double top = (1.0 - w) * img_at(F->images, F->dtype, H, W, F->C, k, j0, i0, c)
                               + w * img_at(F->images, F->dtype, H, W, F->C, k, j0, i1, c);
                    double bot = (1.0 - w) * img_at(F->images, F->dtype, H, W, F->C, k, j1, i0, c)
                               + w * img_at(F->images, F->dtype, H, W, F->C, k, j1, i1, c);
                    acc += (1.0 - wy) * top + wy * bot;
                }
            }
            acc /= (double)n;
        }
        refocus[pix * F->C + c] = acc;
    }
}

/*
 * Whole frame.  Rows [row_begin, row_end) are processed; outputs are full
 * frame-sized arrays (other rows untouched).  Layouts:
 *   images [K][H][W][C] (uint8 or float32), seg_prior [K][H][W] P(dynamic),
 *   mu/inside [H][W] from the triangulation prior, baselines [K] (one == 0),
 *   d_idx/d_val/labels [H][W], post [K][H][W], refocus [H][W][C],
 *   m_margin/e_margin/J_t [iters][H][W], init_margin [H][W].
 * Candidate disparities d_j = d_min + j (d_max - d_min) / (D - 1) (D = 1: d_min).
 * Returns 0, or -1 on invalid arguments.
 */
static int run_frame(int K, const float *baselines, const float *cameras, int H, int W, int C, int dtype,
                     const void *images, const float *seg_prior, const double *mu,
                     const uint8_t *inside, float d_min, float d_max, int D, int iters,
                     const orc_params *p, int row_begin, int row_end, int nthreads,
                     int32_t *d_idx, double *d_val, uint16_t *labels, double *post,
                     double *refocus, double *m_margin, double *e_margin, double *J_t,
                     double *init_margin)
{
    if (K < 1 || K > ORC_MAXK || H < 1 || W < 1 || D < 1 || iters < 1) return -1;
    if (p->em_mode < 0 || p->em_mode > 2) return -1;
    if (C != 1 && C != 3) return -1;
    double b[ORC_MAXK], P[ORC_MAXK * 12];
    int ref = -1;
    for (int k = 0; k < K; ++k) {
        if (cameras) {
            int identity = 1;
            for (int i = 0; i < 12; ++i) {
                P[12 * k + i] = (double)cameras[12 * k + i];
                double want = (i == 0 || i == 5 || i == 10) ? 1.0 : 0.0;
                if (P[12 * k + i] != want) identity = 0;
            }
            b[k] = 0.0;
            if (identity && ref < 0) ref = k;
        } else {
            b[k] = (double)baselines[k];
            if (b[k] == 0.0 && ref < 0) ref = k;
        }
    }
    if (ref < 0) return -1;
    size_t HW = (size_t)H * W;
    double *feat = (double *)malloc(sizeof(double) * 3 * K * HW);
    double *ls = (double *)malloc(sizeof(double) * K * HW);
    double *ld = (double *)malloc(sizeof(double) * K * HW);
    double *dval = (double *)malloc(sizeof(double) * D);
    for (int j = 0; j < D; ++j)
        dval[j] = D == 1 ? (double)d_min
                         : (double)d_min + (double)j * (((double)d_max - (double)d_min) / (double)(D - 1));
    orc_features(K, H, W, C, dtype, images, feat);
    orc_log_seg(K, H, W, seg_prior, p->eps, ls, ld);
    orc_frame F = {K, H, W, C, dtype, D, b, cameras ? P : NULL, ref, dval, feat, ls, ld, images, p};
    if (row_begin < 0) row_begin = 0;
    if (row_end > H) row_end = H;
#ifdef _OPENMP
    /* the thread count applies to this region only (rows are independent,
       so it never changes a result) */
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int v = row_begin; v < row_end; ++v)
        for (int u = 0; u < W; ++u)
            em_pixel(&F, u, v, mu[(size_t)v * W + u], inside[(size_t)v * W + u], iters,
                     d_idx, d_val, labels, post, refocus, m_margin, e_margin, J_t, init_margin);
    free(feat); free(ls); free(ld); free(dval);
    return 0;
}

/* Rectified linear array: baselines [K], one exactly 0 (the reference). */
int orc_run(int K, const float *baselines, int H, int W, int C, int dtype,
            const void *images, const float *seg_prior, const double *mu,
            const uint8_t *inside, float d_min, float d_max, int D, int iters,
            const orc_params *p, int row_begin, int row_end, int nthreads,
            int32_t *d_idx, double *d_val, uint16_t *labels, double *post,
            double *refocus, double *m_margin, double *e_margin, double *J_t,
            double *init_margin)
{
    return run_frame(K, baselines, NULL, H, W, C, dtype, images, seg_prior, mu, inside, d_min, d_max, D, iters,
                     p, row_begin, row_end, nthreads, d_idx, d_val, labels, post, refocus, m_margin, e_margin,
                     J_t, init_margin);
}

/* Calibrated array (Eq. 1): cameras [K][3][4] row-major, mapping the
 * reference pixel (u, v) at generalized disparity d, as (u, v, 1, d), to
 * homogeneous pixel coordinates of camera k; the reference camera is the
 * first whose matrix is exactly [I | 0].  Rays are sampled by bilinear
 * interpolation with both coordinates clamped to the image. */
int orc_run_general(int K, const float *cameras, int H, int W, int C, int dtype,
                    const void *images, const float *seg_prior, const double *mu,
                    const uint8_t *inside, float d_min, float d_max, int D, int iters,
                    const orc_params *p, int row_begin, int row_end, int nthreads,
                    int32_t *d_idx, double *d_val, uint16_t *labels, double *post,
                    double *refocus, double *m_margin, double *e_margin, double *J_t,
                    double *init_margin)
{
    if (!cameras) return -1;
    return run_frame(K, NULL, cameras, H, W, C, dtype, images, seg_prior, mu, inside, d_min, d_max, D, iters,
                     p, row_begin, row_end, nthreads, d_idx, d_val, labels, post, refocus, m_margin, e_margin,
                     J_t, init_margin);
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Objective of one label vector at one disparity, for tests:
 * J(d, S) with the rays of pixel (u, v) sampled at d. */
double orc_objective_at(int K, const float *baselines, int H, int W, int C, int dtype,
                        const void *images, const float *seg_prior, const orc_params *p,
                        int u, int v, double d, double mu, int inside, unsigned S, int with_seg)
{
    size_t HW = (size_t)H * W;
    double *feat = (double *)malloc(sizeof(double) * 3 * K * HW);
    double *ls = (double *)malloc(sizeof(double) * K * HW);
    double *ld = (double *)malloc(sizeof(double) * K * HW);
    double b[ORC_MAXK];
    for (int k = 0; k < K; ++k) b[k] = (double)baselines[k];
    orc_features(K, H, W, C, dtype, images, feat);
    orc_log_seg(K, H, W, seg_prior, p->eps, ls, ld);
    orc_frame F = {K, H, W, C, dtype, 1, b, NULL, 0, &d, feat, ls, ld, images, p};
    double f[ORC_MAXK][3], sls[ORC_MAXK], sld[ORC_MAXK];
    sample_rays(&F, u, v, d, f, sls, sld);
    double J = objective(K, (const double(*)[3])f, sls, sld, S, log_prior(d, mu, inside, p), with_seg, p);
    free(feat); free(ls); free(ld);
    return J;
}

/* 3x3 median per channel with the border replicated (Sec. III-E).
 * img/out are [H][W][C]; the median of 9 values is found by sorting. */
void orc_median3(int H, int W, int C, const double *img, double *out)
{
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u)
            for (int c = 0; c < C; ++c) {
                double a[9];
                int n = 0;
                for (int dv = -1; dv <= 1; ++dv)
                    for (int du = -1; du <= 1; ++du)
                        a[n++] = img[((size_t)clampi(v + dv, 0, H - 1) * W + clampi(u + du, 0, W - 1)) * C + c];
                for (int i = 1; i < 9; ++i) {
                    double x = a[i];
                    int j = i - 1;
                    while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
                    a[j + 1] = x;
                }
                out[((size_t)v * W + u) * C + c] = a[4];
            }
}

/* Exported for the tests: the clamp-to-edge linear sample of one row. */
double orc_sample(const double *row, int W, double x) { return sample_row(row, W, x); }

/*
 * FP64 / integer CPU oracle for the support points of the disparity prior
 * (Sec. III-C "Disparity Prior": sparse points matched along the epipolar
 * lines over the full disparity range, as in ELAS; points on dynamic objects
 * removed with the segmentation; points of other views that re-project onto
 * the reference's occluded background added; duplicates and inconsistent
 * points removed).
 *
 * TEST INFRASTRUCTURE ONLY, like lf_oracle.c: only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may build, load or call it.  It
 * shares no code with the CUDA path.
 *
 * The paper outlines these steps without their details; the reading taken
 * (every step below, in order):
 *
 *   luminance   8-bit integer: uint8 gray as is, uint8 RGB as
 *               (77 R + 150 G + 29 B + 128) >> 8; float inputs are first
 *               quantised per channel to rint(255 x) (float arithmetic),
 *               clamped to [0, 255]
 *   gradients   integer 3x3 Sobel responses Gx, Gy, border replicated
 *   descriptor  Gx and Gy over the 3x3 window around a pixel (18 integers,
 *               coordinates clamped)
 *   grid        candidate pixels (g i + g/2, g j + g/2); cell (i, j) is the
 *               g x g square of the reference image containing it
 *   matching    a source camera s against target cameras T: at candidate
 *               disparity d_j the target pixel is u + o_j(t) with
 *               o_j(t) = floor(-d_j (b_t - b_s) + 1/2) (double), cost =
 *               sum over t of the L1 distance of the descriptors; a candidate
 *               whose target centre leaves the image is not considered
 *   acceptance  texture (sum of |Gx| + |Gy| over the window) >= tau;
 *               j* = arg-min cost (lowest j); second = min cost over j with
 *               |j - j*| >= Delta, Delta = ceil(1 / (max_t |b_t - b_s| *
 *               step)) candidates (one pixel of shift on the widest pair);
 *               accept iff 100 cost(j*) < ratio * second
 *   static      a source pixel is static iff P < threshold at every pixel of
 *               its 3x3 window (coordinates clamped), the support the
 *               descriptor is drawn from
 *   reference   s = the reference camera, T = every other camera; the point
 *               must be static in the reference
 *   other views s = each other camera, T = every camera but s and the
 *               reference; static in s; re-projected to the reference at
 *               u_r = u + d_j* b_s (double), kept iff 0 <= u_r <= W - 1 and
 *               the reference pixel (floor(u_r + 1/2), v) is dynamic
 *               (P >= threshold): background the reference cannot see
 *   duplicates  one point per cell: the reference's own points first, then
 *               the other views in camera order, raster order within a view
 *   consistency a point is kept iff at least min_support other points within
 *               a Chebyshev radius of `window` cells have |d - d'| <= delta
 *   position    the point list (oracle.py) places each point at its cell
 *               position plus a fixed offset below 0.01 px per cell, so that
 *               points of the regular grid are not cocircular and the
 *               Delaunay triangulation of the prior is unique
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int grid;            /* grid step g (pixels) */
    int ratio_pct;       /* uniqueness ratio in percent */
    int texture;         /* minimum window texture */
    int window;          /* consistency radius in cells */
    double delta;        /* consistency tolerance (disparity units) */
    int min_support;     /* consistency: minimum number of agreeing neighbours */
    float seg_threshold; /* a pixel is dynamic iff P >= this */
} orc_support_params;

static int clampi_s(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* P(dynamic) < thr over the 3x3 window of camera k around (u, v). */
static int window_static(const float *seg_prior, int H, int W, int k, int u, int v, float thr)
{
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx)
            if (!(seg_prior[((size_t)k * H + clampi_s(v + dy, 0, H - 1)) * W + clampi_s(u + dx, 0, W - 1)] < thr))
                return 0;
    return 1;
}

static int quant8(float x)
{
    float q = rintf(255.0f * x);
    if (q < 0.0f) q = 0.0f;
    if (q > 255.0f) q = 255.0f;
    return (int)q;
}

/* 8-bit luminance of camera k at (u, v). */
static int luma8(const void *images, int dtype, int H, int W, int C, int k, int v, int u)
{
    size_t base = (((size_t)k * H + v) * W + u) * C;
    int r, g, b;
    if (dtype == 0) {
        const uint8_t *p = (const uint8_t *)images + base;
        if (C == 1) return p[0];
        r = p[0]; g = p[1]; b = p[2];
    } else {
        const float *p = (const float *)images + base;
        if (C == 1) return quant8(p[0]);
        r = quant8(p[0]); g = quant8(p[1]); b = quant8(p[2]);
    }
    return (77 * r + 150 * g + 29 * b + 128) >> 8;
}

typedef struct {
    int K, H, W;
    const int *gx, *gy;   /* [K][H][W] */
} grad_maps;

static int gx_at(const grad_maps *G, int k, int v, int u)
{
    return G->gx[((size_t)k * G->H + clampi_s(v, 0, G->H - 1)) * G->W + clampi_s(u, 0, G->W - 1)];
}

static int gy_at(const grad_maps *G, int k, int v, int u)
{
    return G->gy[((size_t)k * G->H + clampi_s(v, 0, G->H - 1)) * G->W + clampi_s(u, 0, G->W - 1)];
}

/* L1 distance of the 3x3-window descriptors of (s, u, v) and (t, x, v). */
static long descriptor_sad(const grad_maps *G, int s, int u, int t, int x, int v)
{
    long acc = 0;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            acc += labs((long)gx_at(G, s, v + dy, u + dx) - gx_at(G, t, v + dy, x + dx));
            acc += labs((long)gy_at(G, s, v + dy, u + dx) - gy_at(G, t, v + dy, x + dx));
        }
    return acc;
}

/* Match grid pixel (u, v) of camera s against the cameras flagged in tmask.
 * Returns j* or -1 when the point is not accepted. */
static int match_point(const grad_maps *G, const double *b, const double *dval, int D, double step,
                       int s, unsigned tmask, int u, int v, const orc_support_params *sp)
{
    const int W = G->W;
    long tex = 0;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx)
            tex += labs((long)gx_at(G, s, v + dy, u + dx)) + labs((long)gy_at(G, s, v + dy, u + dx));
    if (tex < sp->texture) return -1;
    double bmax = 0.0;
    for (int t = 0; t < G->K; ++t)
        if (tmask >> t & 1u) bmax = fmax(bmax, fabs(b[t] - b[s]));
    if (D < 2 || step <= 0.0 || bmax <= 0.0) return -1;
    int delta = (int)ceil(1.0 / (bmax * step));
    long *cost = (long *)malloc(sizeof(long) * D);
    int best = -1;
    for (int j = 0; j < D; ++j) {
        cost[j] = -1;  /* not considered */
        int ok = 1;
        long c = 0;
        for (int t = 0; t < G->K && ok; ++t) {
            if (!(tmask >> t & 1u)) continue;
            int o = (int)floor(-dval[j] * (b[t] - b[s]) + 0.5);
            int x = u + o;
            if (x < 0 || x > W - 1) { ok = 0; break; }
            c += descriptor_sad(G, s, u, t, x, v);
        }
        if (!ok) continue;
        cost[j] = c;
        if (best < 0 || c < cost[best]) best = j;
    }
    int result = -1;
    if (best >= 0) {
        long second = -1;
        for (int j = 0; j < D; ++j) {
            if (cost[j] < 0 || abs(j - best) < delta) continue;
            if (second < 0 || cost[j] < second) second = cost[j];
        }
        if (second >= 0 && 100 * cost[best] < (long)sp->ratio_pct * second) result = best;
    }
    free(cost);
    return result;
}

/*
 * Support points of one frame (rectified linear array, baselines [K] with one
 * 0).  Outputs per reference cell (ny x nx, nx = ceil(W / g), ny = ceil(H /
 * g)): cell_j = candidate index or -1 (no point), cell_src = source camera,
 * cell_u / cell_v = the point's reference coordinates (its disparity is
 * d_{cell_j}).  Returns the number of points, or -1 on invalid arguments.
 */
int orc_support_points(int K, const float *baselines, int H, int W, int C, int dtype, const void *images,
                       const float *seg_prior, float d_min, float d_max, int D, const orc_support_params *sp,
                       int32_t *cell_j, int32_t *cell_src, double *cell_u, double *cell_v)
{
    if (K < 1 || K > 16 || H < 1 || W < 1 || D < 1 || sp->grid < 1 || (C != 1 && C != 3)) return -1;
    const int g = sp->grid, h = g / 2;
    const int nx = (W + g - 1) / g, ny = (H + g - 1) / g;
    const size_t HW = (size_t)H * W;
    int ref = -1;
    double b[16];
    for (int k = 0; k < K; ++k) {
        b[k] = (double)baselines[k];
        if (b[k] == 0.0 && ref < 0) ref = k;
    }
    if (ref < 0) return -1;
    double *dval = (double *)malloc(sizeof(double) * D);
    for (int j = 0; j < D; ++j)
        dval[j] = D == 1 ? (double)d_min
                         : (double)d_min + (double)j * (((double)d_max - (double)d_min) / (double)(D - 1));
    const double step = D > 1 ? ((double)d_max - (double)d_min) / (double)(D - 1) : 0.0;

    /* luminance and Sobel responses */
    int *Y = (int *)malloc(sizeof(int) * K * HW);
    int *gx = (int *)malloc(sizeof(int) * K * HW);
    int *gy = (int *)malloc(sizeof(int) * K * HW);
    for (int k = 0; k < K; ++k)
        for (int v = 0; v < H; ++v)
            for (int u = 0; u < W; ++u) Y[((size_t)k * H + v) * W + u] = luma8(images, dtype, H, W, C, k, v, u);
    for (int k = 0; k < K; ++k)
        for (int v = 0; v < H; ++v)
            for (int u = 0; u < W; ++u) {
#define YY(dv, du) Y[((size_t)k * H + clampi_s(v + (dv), 0, H - 1)) * W + clampi_s(u + (du), 0, W - 1)]
                gx[((size_t)k * H + v) * W + u] = (YY(-1, 1) + 2 * YY(0, 1) + YY(1, 1)) - (YY(-1, -1) + 2 * YY(0, -1) + YY(1, -1));
                gy[((size_t)k * H + v) * W + u] = (YY(1, -1) + 2 * YY(1, 0) + YY(1, 1)) - (YY(-1, -1) + 2 * YY(-1, 0) + YY(-1, 1));
#undef YY
            }
    grad_maps G = {K, H, W, gx, gy};
    const float thr = sp->seg_threshold;

    for (int i = 0; i < nx * ny; ++i) {
        cell_j[i] = -1;
        cell_src[i] = -1;
        cell_u[i] = 0.0;
        cell_v[i] = 0.0;
    }
    /* the reference's own points */
    unsigned all_but_ref = 0;
    for (int t = 0; t < K; ++t)
        if (t != ref) all_but_ref |= 1u << t;
    for (int cj = 0; cj < ny; ++cj)
        for (int ci = 0; ci < nx; ++ci) {
            int u = g * ci + h, v = g * cj + h;
            if (u > W - 1 || v > H - 1) continue;
            if (!window_static(seg_prior, H, W, ref, u, v, thr)) continue;
            int j = match_point(&G, b, dval, D, step, ref, all_but_ref, u, v, sp);
            if (j < 0) continue;
            cell_j[cj * nx + ci] = j;
            cell_src[cj * nx + ci] = ref;
            cell_u[cj * nx + ci] = u;
            cell_v[cj * nx + ci] = v;
        }
    /* points of the other views on the reference's occluded background */
    for (int s = 0; s < K; ++s) {
        if (s == ref) continue;
        unsigned tmask = all_but_ref & ~(1u << s);
        if (!tmask) continue;
        for (int cj = 0; cj < ny; ++cj)
            for (int ci = 0; ci < nx; ++ci) {
                int u = g * ci + h, v = g * cj + h;
                if (u > W - 1 || v > H - 1) continue;
                if (!window_static(seg_prior, H, W, s, u, v, thr)) continue;
                int j = match_point(&G, b, dval, D, step, s, tmask, u, v, sp);
                if (j < 0) continue;
                double ur = (double)u + dval[j] * b[s];
                if (ur < 0.0 || ur > (double)(W - 1)) continue;
                int rr = (int)floor(ur + 0.5);
                if (seg_prior[(size_t)ref * HW + (size_t)v * W + rr] < thr) continue;
                int cell = cj * nx + (int)floor(ur / (double)g);
                if (cell_j[cell] >= 0) continue;
                cell_j[cell] = j;
                cell_src[cell] = s;
                cell_u[cell] = ur;
                cell_v[cell] = v;
            }
    }
    /* consistency with the neighbouring cells */
    int32_t *keep = (int32_t *)malloc(sizeof(int32_t) * nx * ny);
    for (int cj = 0; cj < ny; ++cj)
        for (int ci = 0; ci < nx; ++ci) {
            int c = cj * nx + ci;
            keep[c] = 0;
            if (cell_j[c] < 0) continue;
            int support = 0;
            for (int y = cj - sp->window; y <= cj + sp->window; ++y)
                for (int x = ci - sp->window; x <= ci + sp->window; ++x) {
                    if (x < 0 || y < 0 || x >= nx || y >= ny || (x == ci && y == cj)) continue;
                    int o = y * nx + x;
                    if (cell_j[o] >= 0 && fabs(dval[cell_j[o]] - dval[cell_j[c]]) <= sp->delta) ++support;
                }
            keep[c] = support >= sp->min_support;
        }
    int n = 0;
    for (int c = 0; c < nx * ny; ++c) {
        if (cell_j[c] >= 0 && !keep[c]) {
            cell_j[c] = -1;
            cell_src[c] = -1;
            cell_u[c] = 0.0;
            cell_v[c] = 0.0;
        }
        if (cell_j[c] >= 0) ++n;
    }
    free(keep); free(Y); free(gx); free(gy); free(dval);
    return n;
}

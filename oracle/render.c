/*
 * Oracle: masked alpha compositing of MaskGaussian (arXiv 2412.20522), FP64.
 *
 * TEST INFRASTRUCTURE ONLY -- never linked into the product library.
 *
 * What it computes, per pixel x (Sec. 3.1, Sec. 3.3, Appendix A):
 *   the Gaussians of the pixel's tile, front to back in depth order, each with
 *   alpha_i = min(0.99, o_i * exp(power_i)),
 *   power_i = -1/2 (x - p_i)^T Sigma_i^-1 (x - p_i),
 *   are blended by Eq. 3-4:
 *     c(x)    = sum_i M_i c_i alpha_i T_i (+ T_{N+1} c_bg, Appendix A)
 *     T_{i+1} = M_i (1 - alpha_i) T_i + (1 - M_i) T_i,   T_1 = 1.
 *   Only Gaussians intersecting the tile and with alpha above the 1/255 floor
 *   take part (Sec. 3.1: "alpha > 0"); blending stops before a Gaussian that
 *   would take T below 1e-4.  (The 1/255, 0.99 and 1e-4 constants come from
 *   the 3DGS rasteriser the paper modifies, Sec. 4.1.)
 *
 * The backward is Eq. 6 with the background term of Appendix A, in the
 * paper's notation: b_i is the colour rendered from the i-th Gaussian to the
 * last one (no background), b_i = M_i alpha_i c_i + (1 - M_i alpha_i) b_{i+1},
 *   dL/dM_i = alpha_i T_i g.(c_i - b_{i+1}) - alpha_i T_{N+1}/(1 - alpha_i M_i) g.c_bg
 * with g = dL/dc(x).  The alpha gradient follows the same structure:
 *   dL/dalpha_i = M_i T_i g.(c_i - b_{i+1}) - M_i T_{N+1}/(1 - alpha_i M_i) g.c_bg
 * (zero for a masked splat, Fig. 2 caption), then through the 0.99 clamp
 * (true derivative: zero when clamped) to o_i, the conic and the 2D mean.
 * T_i is taken from a forward prefix recomputed per pixel, not by division.
 *
 * Straddles: a decision whose FP64 operand lies within a relative band (eps
 * for the alpha floor and the power sign, eps_T for the termination test,
 * whose operand T accumulates the rounding of every blended splat) of its
 * threshold is flagged per pixel (bit 1: alpha floor, bit 2:
 * termination, bit 4: 0.99 clamp, bit 8: sign of power); an FP32 evaluation
 * may fall on the other side there.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ALPHA_MAX 0.99
#define ALPHA_MIN (1.0 / 255.0)
#define T_MIN 1e-4

typedef struct {
    int n;                 /* number of Gaussians */
    const double *mean2d;  /* [n][2] pixels */
    const double *conic;   /* [n][3] a, b, c of [[a, b], [b, c]] */
    const double *opacity; /* [n] */
    const double *rgb;     /* [n][3] */
    const double *mask;    /* [n] 0 or 1 */
} orc_splats;

typedef struct {
    int width, height, tile_w, tile_h;
    double bg[3];
    double eps;            /* straddle band (relative) of the alpha floor and the power sign */
    double eps_T;          /* straddle band (relative) of the termination test */
} orc_frame;

static void eval_fragment(const orc_splats *s, int g, double px, double py,
                          double *power, double *G, double *araw, double *alpha)
{
    double dx = px - s->mean2d[2 * g], dy = py - s->mean2d[2 * g + 1];
    const double *q = s->conic + 3 * g;
    *power = -0.5 * (q[0] * dx * dx + q[2] * dy * dy) - q[1] * dx * dy;
    *G = exp(*power);
    *araw = s->opacity[g] * *G;
    *alpha = *araw < ALPHA_MAX ? *araw : ALPHA_MAX;
}

static int near_rel(double v, double thr, double eps) { return fabs(v - thr) <= eps * thr; }

/* Composite one pixel over an explicit front-to-back list of Gaussians.
 * masked = 0 gives plain 3DGS (Eq. 1-2), masked = 1 gives Eq. 3-4. */
static void composite(const orc_splats *s, const orc_frame *f, const uint32_t *list,
                      int len, double px, double py, int masked,
                      double out[3], double *Tfin, int32_t *ncontrib, uint8_t *flag,
                      int64_t *frags)
{
    double T = 1.0, C[3] = {0.0, 0.0, 0.0};
    int32_t last = len;      /* positions processed: termination index or list length */
    uint8_t fl = 0;
    int64_t visited = 0;
    for (int j = 0; j < len; ++j) {
        int g = (int)list[j];
        double power, G, araw, alpha;
        ++visited;
        eval_fragment(s, g, px, py, &power, &G, &araw, &alpha);
        if (fabs(power) <= f->eps) fl |= 8;
        if (power > 0.0) continue;
        if (near_rel(alpha, ALPHA_MIN, f->eps)) fl |= 1;
        if (alpha < ALPHA_MIN) continue;
        if (near_rel(araw, ALPHA_MAX, f->eps)) fl |= 4;
        double testT;
        if (masked) {
            double M = s->mask[g];
            testT = T * (1.0 - M * alpha);
            if (near_rel(testT, T_MIN, f->eps_T)) fl |= 2;
            if (testT < T_MIN) { last = j; break; }
            for (int ch = 0; ch < 3; ++ch) C[ch] += ((M * alpha) * T) * s->rgb[3 * g + ch];
        } else {
            testT = T * (1.0 - alpha);
            if (near_rel(testT, T_MIN, f->eps_T)) fl |= 2;
            if (testT < T_MIN) { last = j; break; }
            for (int ch = 0; ch < 3; ++ch) C[ch] += (alpha * T) * s->rgb[3 * g + ch];
        }
        T = testT;
    }
    for (int ch = 0; ch < 3; ++ch) out[ch] = C[ch] + T * f->bg[ch];
    *Tfin = T;
    *ncontrib = last;
    *flag = fl;
    *frags += visited;
}

/* Tiled render: ``vals`` is the depth-sorted instance list, ``ranges`` [T][2]
 * gives each tile's [start, end) into it.  Outputs image [3][H][W], final T
 * [H][W], the number of list positions processed before blending stopped (the
 * index of the Gaussian that would have taken T below 1e-4, else the list
 * length) [H][W], straddle flags [H][W] and the number of evaluated
 * (pixel, Gaussian) pairs. */
int64_t orc_render_tiled(const orc_splats *s, const orc_frame *f, const uint32_t *vals,
                         const uint32_t *ranges, int masked, double *image,
                         double *final_T, int32_t *ncontrib, uint8_t *flags)
{
    int gx = (f->width + f->tile_w - 1) / f->tile_w;
    int gy = (f->height + f->tile_h - 1) / f->tile_h;
    int64_t frags = 0;
    const int64_t HW = (int64_t)f->width * f->height;
#pragma omp parallel for schedule(dynamic) reduction(+ : frags)
    for (int t = 0; t < gx * gy; ++t) {
        int tx = t % gx, ty = t / gx;
        uint32_t start = ranges[2 * t], end = ranges[2 * t + 1];
        for (int v = ty * f->tile_h; v < (ty + 1) * f->tile_h && v < f->height; ++v)
            for (int u = tx * f->tile_w; u < (tx + 1) * f->tile_w && u < f->width; ++u) {
                double out[3];
                int64_t p = (int64_t)v * f->width + u;
                composite(s, f, vals + start, (int)(end - start), u + 0.5, v + 0.5, masked,
                          out, &final_T[p], &ncontrib[p], &flags[p], &frags);
                for (int ch = 0; ch < 3; ++ch) image[ch * HW + p] = out[ch];
            }
    }
    return frags;
}

typedef struct { uint32_t depth_bits; uint32_t idx; } orc_key;

static int cmp_key(const void *a, const void *b)
{
    const orc_key *x = (const orc_key *)a, *y = (const orc_key *)b;
    if (x->depth_bits != y->depth_bits) return x->depth_bits < y->depth_bits ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

/* Brute force, no tile lists: for each pixel, every Gaussian whose tile
 * rectangle [x0,x1]x[y0,y1] (inclusive) contains the pixel's tile, ordered by
 * (depth bits, index). Must equal orc_render_tiled bit for bit. */
void orc_render_bruteforce(const orc_splats *s, const orc_frame *f, const int32_t *rect,
                           const uint32_t *depth_bits, int masked, double *image,
                           double *final_T, int32_t *ncontrib, uint8_t *flags)
{
    const int64_t HW = (int64_t)f->width * f->height;
#pragma omp parallel
    {
        orc_key *keys = (orc_key *)malloc(sizeof(orc_key) * (size_t)(s->n > 0 ? s->n : 1));
        uint32_t *list = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(s->n > 0 ? s->n : 1));
        int64_t frags = 0;
#pragma omp for schedule(dynamic)
        for (int64_t p = 0; p < HW; ++p) {
            int u = (int)(p % f->width), v = (int)(p / f->width);
            int tx = u / f->tile_w, ty = v / f->tile_h;
            int len = 0;
            for (int g = 0; g < s->n; ++g) {
                const int32_t *r = rect + 4 * g;
                if (r[0] <= tx && tx <= r[1] && r[2] <= ty && ty <= r[3]) {
                    keys[len].depth_bits = depth_bits[g];
                    keys[len].idx = (uint32_t)g;
                    ++len;
                }
            }
            qsort(keys, (size_t)len, sizeof(orc_key), cmp_key);
            for (int j = 0; j < len; ++j) list[j] = keys[j].idx;
            double out[3];
            composite(s, f, list, len, u + 0.5, v + 0.5, masked, out, &final_T[p],
                      &ncontrib[p], &flags[p], &frags);
            for (int ch = 0; ch < 3; ++ch) image[ch * HW + p] = out[ch];
        }
        free(keys);
        free(list);
    }
}

typedef struct {
    double *dmean2d;  /* [n][2] */
    double *dconic;   /* [n][3] */
    double *dopacity; /* [n] */
    double *drgb;     /* [n][3] */
    double *dmask;    /* [n] */
    double *dalpha;   /* [n]  (diagnostic: dL/dalpha before the clamp) */
} orc_grads;

static void atomic_add(double *p, double v)
{
#pragma omp atomic
    *p += v;
}

/* Backward of the tiled masked render for the upstream gradient dL/dimage
 * [3][H][W]; gradients ACCUMULATE into ``out``. */
void orc_render_backward(const orc_splats *s, const orc_frame *f, const uint32_t *vals,
                         const uint32_t *ranges, const double *dL_dimage, orc_grads *out)
{
    int gx = (f->width + f->tile_w - 1) / f->tile_w;
    int gy = (f->height + f->tile_h - 1) / f->tile_h;
    const int64_t HW = (int64_t)f->width * f->height;
#pragma omp parallel
    {
        int cap = 64;
        int *gi = (int *)malloc(sizeof(int) * cap);
        double *Ti = (double *)malloc(sizeof(double) * cap);
        double *Gi = (double *)malloc(sizeof(double) * cap);
        double *Ai = (double *)malloc(sizeof(double) * cap);
        double *Ri = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic)
        for (int t = 0; t < gx * gy; ++t) {
            int tx = t % gx, ty = t / gx;
            uint32_t start = ranges[2 * t], end = ranges[2 * t + 1];
            for (int v = ty * f->tile_h; v < (ty + 1) * f->tile_h && v < f->height; ++v)
                for (int u = tx * f->tile_w; u < (tx + 1) * f->tile_w && u < f->width; ++u) {
                    int64_t p = (int64_t)v * f->width + u;
                    double px = u + 0.5, py = v + 0.5;
                    double g[3] = {dL_dimage[p], dL_dimage[HW + p], dL_dimage[2 * HW + p]};
                    /* forward prefix: contributors and their T_i */
                    int n = 0;
                    double T = 1.0;
                    for (uint32_t k = start; k < end; ++k) {
                        int gg = (int)vals[k];
                        double power, G, araw, alpha;
                        eval_fragment(s, gg, px, py, &power, &G, &araw, &alpha);
                        if (power > 0.0 || alpha < ALPHA_MIN) continue;
                        double testT = T * (1.0 - s->mask[gg] * alpha);
                        if (testT < T_MIN) break;
                        if (n == cap) {
                            cap *= 2;
                            gi = (int *)realloc(gi, sizeof(int) * cap);
                            Ti = (double *)realloc(Ti, sizeof(double) * cap);
                            Gi = (double *)realloc(Gi, sizeof(double) * cap);
                            Ai = (double *)realloc(Ai, sizeof(double) * cap);
                            Ri = (double *)realloc(Ri, sizeof(double) * cap);
                        }
                        gi[n] = gg; Ti[n] = T; Gi[n] = G; Ai[n] = alpha; Ri[n] = araw;
                        ++n;
                        T = testT;
                    }
                    double TN1 = T;
                    double gbg = g[0] * f->bg[0] + g[1] * f->bg[1] + g[2] * f->bg[2];
                    double b[3] = {0.0, 0.0, 0.0};   /* b_{n+1} = 0 */
                    for (int i = n - 1; i >= 0; --i) {
                        int gg = gi[i];
                        double M = s->mask[gg], alpha = Ai[i], Tc = Ti[i];
                        const double *c = s->rgb + 3 * gg;
                        double gcb = g[0] * (c[0] - b[0]) + g[1] * (c[1] - b[1]) + g[2] * (c[2] - b[2]);
                        double bgterm = TN1 / (1.0 - alpha * M) * gbg;
                        double dM = alpha * Tc * gcb - alpha * bgterm;        /* Eq. 6 + App. A */
                        double dA = M * Tc * gcb - M * bgterm;
                        atomic_add(&out->dmask[gg], dM);
                        atomic_add(&out->dalpha[gg], dA);
                        for (int ch = 0; ch < 3; ++ch) {
                            atomic_add(&out->drgb[3 * gg + ch], M * alpha * Tc * g[ch]);
                            b[ch] = M * alpha * c[ch] + (1.0 - M * alpha) * b[ch];
                        }
                        if (Ri[i] < ALPHA_MAX) {          /* alpha = o G unclamped */
                            double o = s->opacity[gg];
                            atomic_add(&out->dopacity[gg], dA * Gi[i]);
                            double dpow = dA * o * Gi[i];
                            double dx = px - s->mean2d[2 * gg], dy = py - s->mean2d[2 * gg + 1];
                            const double *q = s->conic + 3 * gg;
                            atomic_add(&out->dconic[3 * gg + 0], dpow * (-0.5 * dx * dx));
                            atomic_add(&out->dconic[3 * gg + 1], dpow * (-dx * dy));
                            atomic_add(&out->dconic[3 * gg + 2], dpow * (-0.5 * dy * dy));
                            atomic_add(&out->dmean2d[2 * gg + 0], dpow * (q[0] * dx + q[1] * dy));
                            atomic_add(&out->dmean2d[2 * gg + 1], dpow * (q[2] * dy + q[1] * dx));
                        }
                    }
                }
        }
        free(gi); free(Ti); free(Gi); free(Ai); free(Ri);
    }
}

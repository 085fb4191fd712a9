/*
 * Oracle for the automatic spline detection of Section 3.3 -- TEST
 * INFRASTRUCTURE ONLY (the library never calls it).
 *
 * Steps, in the section's order:
 *   1. ring R: known pixels a fixed distance dR from the hole D_h;
 *   2. Canny edge detection on an annulus of known pixels around R: smoothing
 *      u_sigma = g_sigma * u, gradient, non-maximum suppression, two thresholds,
 *      hysteresis;
 *   3. for every ring pixel on an accepted edge, the structure tensor
 *      J_{sigma,rho} = g_rho * (grad u_sigma (x) grad u_sigma) (eq.
 *      structureTensor) at that pixel, its eigenpairs (lambda+, v+), (lambda-, v-),
 *      and a straight spline from the pixel along +-v- of length L, the sign
 *      chosen to point into D_h, with the coherence weight
 *      tanh((lambda+ - lambda-) / Lambda) of g_Gamma.
 * Plain loops over the whole image, one step at a time.  Every decision that
 * turns real numbers into a set (a threshold, a suppression, a sign, the ring)
 * uses FP32 values formed with correctly rounded operations only (+ - * / sqrt,
 * fused multiply-add where stated) and comparisons, no other contraction, so a
 * second implementation doing the same operations in the same order reaches
 * the same sets.
 *
 * Readings where the section is not specific:
 *  - distances are Chebyshev distances: d_hole to the nearest hole pixel
 *    (label 1), d_all to the nearest pixel that is not known (label 1 or 2); both
 *    capped at cap = dR + annulus + 1 (a larger distance reads as cap + 1);
 *  - ring R: known pixels with d_hole == dR and d_all == dR (no hole or
 *    bystander pixel nearer, so the tensor's windows stay clear of D_h u B_h);
 *    dR defaults to ceil(2 sigma) + ceil(2 rho) + 2, which keeps the (4 sigma +
 *    1)^2 and (4 rho + 1)^2 windows and the gradient stencil off D_h u B_h;
 *  - annulus: known pixels with |d_hole - dR| <= annulus (bystander pixels are
 *    "not the current object" and ignored);
 *  - the image is RGB: u_sigma per channel, gradient outer products summed over
 *    the channels in order R, G, B by fused multiply-add (the multichannel
 *    structure tensor);
 *  - g_s: truncated to radius r = ceil(2 s) (the (4 s + 1) window), taps
 *    exp(-i^2 / (2 s^2)) in FP64 rounded to FP32 and divided by their FP32 sum;
 *    applied separably, along rows then along columns, taps in order -r..r,
 *    each accumulated by a fused multiply-add (one rounding per tap),
 *    coordinates clamped to the image;
 *  - gradient: central differences (u(x+1) - u(x-1)) / 2, one-sided at the
 *    image border;
 *  - Canny: strength m2 = |grad u_sigma|^2 summed over channels (= trace of the
 *    unsmoothed tensor T); direction = major eigenvector of T quantised to 0,
 *    45, 90, 135 degrees by comparing d = Txx - Tyy with e = 2 Txy (|e| <= d:
 *    0; |e| <= -d: 90; else e > 0: 45, e < 0: 135); a pixel survives
 *    suppression when m2 >= m2 of both neighbours along that direction; strong
 *    when m2 > t_high^2, weak when m2 > t_low^2; weak pixels are kept when
 *    8-connected through kept annulus pixels to a strong one;
 *  - eigenvectors of [[a, b], [b, c]] without trigonometry: d = a - c, e = 2 b,
 *    r = sqrt(d^2 + e^2) = lambda+ - lambda-; v+ ~ (d + r, e) if d >= 0, else
 *    (e, r - d); (1, 0) when r == 0; normalised; v- = (-v+_y, v+_x);
 *  - sign: with P+- = base +- dR v- rounded to the nearest pixel and clamped to
 *    the image, the spline goes along -v- when d_hole(P-) < d_hole(P+), else
 *    along +v-;
 *  - weight: tanh((double)r / Lambda) rounded to FP32;
 *  - splines are listed in raster order of their base pixel.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    float sigma, rho;
    int32_t ring_dist; /* dR; <= 0: ceil(2 sigma) + ceil(2 rho) + 2 */
    int32_t annulus;
    float t_high, t_low;
    float length;
    float Lambda;
} det_params;

/* optional per-pixel outputs for the tests (any may be NULL) */
typedef struct {
    int32_t *d_hole;  /* [H][W] */
    int32_t *d_all;   /* [H][W] */
    uint8_t *edge_nms; /* [H][W] after suppression and thresholds: 0, 1 weak, 2 strong */
    uint8_t *edge;     /* [H][W] after hysteresis: 0 or 2 */
    float *us;         /* [H][W][3] u_sigma */
    float *T;          /* [H][W][3] Txx, Txy, Tyy */
    float *J;          /* [H][W][3] Jxx, Jxy, Jyy */
} det_debug;

static int iclamp(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

int oracle_gauss_taps(float s, float *w)
{
    int r = (int)ceil(2.0 * (double)s);
    float sum = 0.0f;
    for (int i = -r; i <= r; i++) {
        w[i + r] = (float)exp(-(double)(i * i) / (2.0 * (double)s * (double)s));
        sum = sum + w[i + r];
    }
    for (int i = 0; i <= 2 * r; i++) w[i] = w[i] / sum;
    return r;
}

/* separable blur of an [H][W][3] FP32 field, rows then columns, clamped */
static void blur3(int H, int W, const float *in, float *out, float s, float *tmp)
{
    float w[129];
    int r = oracle_gauss_taps(s, w);
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            for (int c = 0; c < 3; c++) {
                float a = 0.0f;
                for (int i = -r; i <= r; i++) a = fmaf(w[i + r], in[((size_t)y * W + iclamp(x + i, 0, W - 1)) * 3 + c], a);
                tmp[((size_t)y * W + x) * 3 + c] = a;
            }
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            for (int c = 0; c < 3; c++) {
                float a = 0.0f;
                for (int i = -r; i <= r; i++) a = fmaf(w[i + r], tmp[((size_t)iclamp(y + i, 0, H - 1) * W + x) * 3 + c], a);
                out[((size_t)y * W + x) * 3 + c] = a;
            }
}

/* Chebyshev distance to the nearest pixel whose label is in `set` (bit l for
 * label l), by brute force over the (2 cap + 1)^2 box; cap + 1 when none */
static void cheb_dist(int H, int W, const uint8_t *lab, unsigned set, int cap, int32_t *d)
{
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int best = cap + 1;
            for (int dy = -cap; dy <= cap; dy++)
                for (int dx = -cap; dx <= cap; dx++) {
                    int yy = y + dy, xx = x + dx;
                    if (yy < 0 || xx < 0 || yy >= H || xx >= W) continue;
                    if (!((set >> lab[(size_t)yy * W + xx]) & 1u)) continue;
                    int m = abs(dx) > abs(dy) ? abs(dx) : abs(dy);
                    if (m < best) best = m;
                }
            d[(size_t)y * W + x] = best;
        }
}

/* eigen-decomposition of [[a, b], [b, c]]: returns r = lambda+ - lambda-,
 * writes the unit minor eigenvector */
static float minor_eigvec(float a, float b, float c, float *mx, float *my)
{
    float d = a - c, e = 2.0f * b;
    float r = sqrtf(d * d + e * e);
    float px, py;
    if (d >= 0.0f) {
        px = d + r;
        py = e;
    } else {
        px = e;
        py = r - d;
    }
    if (px == 0.0f && py == 0.0f) {
        px = 1.0f;
        py = 0.0f;
    }
    float n = sqrtf(px * px + py * py);
    px = px / n;
    py = py / n;
    *mx = -py;
    *my = px;
    return r;
}

/* Returns the number of splines found (>= 0; only the first max_splines are
 * written) or -1 on bad arguments.  pts: [max_splines][4] = base x, base y,
 * end x, end y; weight: [max_splines]; base: [max_splines] pixel index. */
int oracle_detect_splines(int H, int W, const float *rgb, const uint8_t *lab, const det_params *P, int max_splines,
                          float *pts, float *weight, int32_t *base, det_debug *dbg)
{
    if (H <= 0 || W <= 0 || !(P->sigma > 0.0f) || !(P->rho > 0.0f) || P->annulus < 0 || max_splines < 0) return -1;
    if (P->sigma > 32.0f || P->rho > 32.0f) return -1;
    size_t N = (size_t)H * W;
    int dR = P->ring_dist > 0 ? P->ring_dist : (int)ceil(2.0 * P->sigma) + (int)ceil(2.0 * P->rho) + 2;
    int cap = dR + P->annulus + 1;
    int32_t *dh = (int32_t *)malloc(sizeof(int32_t) * N);
    int32_t *da = (int32_t *)malloc(sizeof(int32_t) * N);
    float *us = (float *)malloc(sizeof(float) * N * 3);
    float *tmp = (float *)malloc(sizeof(float) * N * 3);
    float *T = (float *)malloc(sizeof(float) * N * 3);
    float *J = (float *)malloc(sizeof(float) * N * 3);
    float *m2 = (float *)malloc(sizeof(float) * N);
    uint8_t *edge = (uint8_t *)calloc(N, 1);
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * N);

    /* 1. distances, ring and annulus */
    cheb_dist(H, W, lab, 1u << 1, cap, dh);
    cheb_dist(H, W, lab, (1u << 1) | (1u << 2), cap, da);

    /* 2. u_sigma, gradient, T = grad u_sigma (x) grad u_sigma summed over channels, m2 */
    blur3(H, W, rgb, us, P->sigma, tmp);
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int xl = x > 0 ? x - 1 : x, xr = x < W - 1 ? x + 1 : x;
            int yu = y > 0 ? y - 1 : y, yd = y < H - 1 ? y + 1 : y;
            float sx = (float)(xr - xl), sy = (float)(yd - yu);
            float jxx = 0.0f, jxy = 0.0f, jyy = 0.0f;
            for (int c = 0; c < 3; c++) {
                float gx = sx > 0.0f ? (us[((size_t)y * W + xr) * 3 + c] - us[((size_t)y * W + xl) * 3 + c]) / sx : 0.0f;
                float gy = sy > 0.0f ? (us[((size_t)yd * W + x) * 3 + c] - us[((size_t)yu * W + x) * 3 + c]) / sy : 0.0f;
                jxx = fmaf(gx, gx, jxx);
                jxy = fmaf(gx, gy, jxy);
                jyy = fmaf(gy, gy, jyy);
            }
            size_t p = (size_t)y * W + x;
            T[p * 3 + 0] = jxx;
            T[p * 3 + 1] = jxy;
            T[p * 3 + 2] = jyy;
            m2[p] = jxx + jyy;
        }
    /* J_{sigma,rho} = g_rho * T */
    blur3(H, W, T, J, P->rho, tmp);

    /* Canny on the annulus: suppression and thresholds */
    float th2 = P->t_high * P->t_high, tl2 = P->t_low * P->t_low;
    static const int ox[4] = {1, 1, 0, -1}, oy[4] = {0, 1, 1, 1};
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            size_t p = (size_t)y * W + x;
            if (lab[p] != 0 || dh[p] < dR - P->annulus || dh[p] > dR + P->annulus) continue;
            float d = T[p * 3 + 0] - T[p * 3 + 2], e = 2.0f * T[p * 3 + 1];
            int q;
            if (fabsf(e) <= d) q = 0;
            else if (fabsf(e) <= -d) q = 2;
            else q = e > 0.0f ? 1 : 3;
            int x1 = iclamp(x + ox[q], 0, W - 1), y1 = iclamp(y + oy[q], 0, H - 1);
            int x2 = iclamp(x - ox[q], 0, W - 1), y2 = iclamp(y - oy[q], 0, H - 1);
            float v = m2[p];
            if (!(v >= m2[(size_t)y1 * W + x1] && v >= m2[(size_t)y2 * W + x2])) continue;
            if (v > th2) edge[p] = 2;
            else if (v > tl2) edge[p] = 1;
        }
    if (dbg && dbg->edge_nms) memcpy(dbg->edge_nms, edge, N);
    /* hysteresis: depth-first from every strong pixel through weak ones */
    int top = 0;
    for (size_t p = 0; p < N; p++)
        if (edge[p] == 2) stack[top++] = (int32_t)p;
    while (top > 0) {
        int32_t p = stack[--top];
        int x = (int)(p % W), y = (int)(p / W);
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int xx = x + dx, yy = y + dy;
                if (xx < 0 || yy < 0 || xx >= W || yy >= H) continue;
                size_t q = (size_t)yy * W + xx;
                if (edge[q] == 1) {
                    edge[q] = 2;
                    stack[top++] = (int32_t)q;
                }
            }
    }
    for (size_t p = 0; p < N; p++)
        if (edge[p] == 1) edge[p] = 0;

    /* 3. one spline per ring pixel on an edge, raster order */
    int ns = 0;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            size_t p = (size_t)y * W + x;
            if (lab[p] != 0 || dh[p] != dR || da[p] != dR || edge[p] != 2) continue;
            if (ns < max_splines) {
                float vx, vy;
                float r = minor_eigvec(J[p * 3 + 0], J[p * 3 + 1], J[p * 3 + 2], &vx, &vy);
                float bx = (float)x, by = (float)y;
                float fdR = (float)dR;
                int xp = iclamp((int)floorf(bx + fdR * vx + 0.5f), 0, W - 1);
                int yp = iclamp((int)floorf(by + fdR * vy + 0.5f), 0, H - 1);
                int xm = iclamp((int)floorf(bx - fdR * vx + 0.5f), 0, W - 1);
                int ym = iclamp((int)floorf(by - fdR * vy + 0.5f), 0, H - 1);
                if (dh[(size_t)ym * W + xm] < dh[(size_t)yp * W + xp]) {
                    vx = -vx;
                    vy = -vy;
                }
                pts[4 * ns + 0] = bx;
                pts[4 * ns + 1] = by;
                pts[4 * ns + 2] = bx + P->length * vx;
                pts[4 * ns + 3] = by + P->length * vy;
                weight[ns] = (float)tanh((double)r / (double)P->Lambda);
                base[ns] = (int32_t)p;
            }
            ns++;
        }
    if (dbg) {
        if (dbg->d_hole) memcpy(dbg->d_hole, dh, sizeof(int32_t) * N);
        if (dbg->d_all) memcpy(dbg->d_all, da, sizeof(int32_t) * N);
        if (dbg->edge) memcpy(dbg->edge, edge, N);
        if (dbg->us) memcpy(dbg->us, us, sizeof(float) * N * 3);
        if (dbg->T) memcpy(dbg->T, T, sizeof(float) * N * 3);
        if (dbg->J) memcpy(dbg->J, J, sizeof(float) * N * 3);
    }
    free(dh); free(da); free(us); free(tmp); free(T); free(J); free(m2); free(edge); free(stack);
    return ns;
}

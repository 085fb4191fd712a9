/*
 * Plain CPU oracle for the Guidefill shell fill (Hocking, MacKenzie, Schoenlieb,
 * "Guidefill: GPU Accelerated, Artist Guided Geometric Inpainting for 3D
 * Conversion of Film", arxiv 1611.05319).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is called by the tests, by the smoke
 * check and by the benchmark's CPU-baseline leg; the product path never links
 * or calls it.  It shares no code with the CUDA library.
 *
 * Everything is single-threaded plain loops, FP64 for colours and weights.  The
 * only FP32 arithmetic is where the paper's geometry decides an integer (which
 * lattice pixels a rotated ghost sample touches, which spline segment is
 * nearest): there both sides must take the decision in the same precision, so
 * the offsets and candidate distances are formed from the FP32 inputs with
 * fixed FP32 expressions (compiled with -ffp-contract=off, no fast-math).
 *
 * Readings of the paper used here (where it is silent or garbled):
 *  R1 the origin y = x is excluded from the ball (its weight 1/0 is undefined
 *     and x is never readable; Section 3.3's kinking discussion);
 *  R2 the rotation uses the unit vector g/|g|; |g| enters only the weight;
 *     g = 0 gives the unrotated lattice ball (Section 4, definition of the
 *     half-ball sets);
 *  R3 a ghost sample is readable iff it lies in the image and every lattice
 *     pixel with non-zero bilinear weight is readable (the continuous sets
 *     D^(k), B carry a one-pixel open buffer, Notation and eq. bilinearDef);
 *  R4 FP32 offsets n*gh - m*gh_perp are snapped to the nearest integer when
 *     within tau (default 1e-5 px), so that "on a lattice line" is decided the
 *     same way on every machine;
 *  R5 onion order (smart order off) fills a front pixel iff it has at least one
 *     readable sample;
 *  R6 the fill colour uses the weights divided by their largest readable value
 *     (the common factor cancels in the normalised average; without it the
 *     exponentials underflow to 0/0 when only far-from-line samples are
 *     readable);
 *  R7 stall: if no front pixel is ready at step k while the front is not
 *     empty, every front pixel with a readable sample of the unrotated ball is
 *     filled at step k with g treated as 0 (isotropic weights 1/|y-x|);
 *  R8 hole pixels that never join the front (walled off) keep their colour,
 *     shell index -2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define LBL_KNOWN 0
#define LBL_HOLE 1
#define LBL_BYST 2

#define SH_KNOWN (-1)
#define SH_UNFILLED (-2)
#define SH_BYST (-3)

#define OF_GHOST 1u
#define OF_SMART 2u
#define OF_DATA 8u /* data term D(x) = |g(x)| of eq. ready2 (Section 3.5, possible extensions) */

#define MAX_SAMPLES 1024

typedef struct {
    int32_t shells;       /* K: number of steps that filled at least one pixel */
    int32_t stalls;       /* steps filled by the stall rule R7 */
    int64_t evaluations;  /* front pixels evaluated (sum over k of |front_k|) */
    int64_t filled;       /* hole pixels filled */
    int64_t unreachable;  /* hole pixels never filled */
    int64_t max_front;    /* max_k |front_k| */
    double min_margin;    /* min over smart-order decisions of |C - c| / c */
    int32_t data_switch;  /* eq. ready2: first step evaluated with eq. ready (-1: no data term) */
    int32_t pad;
} oracle_stats;

/* ---------------------------------------------------------------------- */
/* The discrete ball B_{eps,h}(0) minus the origin (Notation; eq. ctgf_limits
 * set form): lattice points (n, m) with n^2 + m^2 <= eps^2, listed with m
 * ascending, then n ascending. */
static int disc_points(double eps, int *ns, int *ms)
{
    int R = (int)ceil(eps);
    int cnt = 0;
    for (int m = -R; m <= R; m++)
        for (int n = -R; n <= R; n++) {
            if (n == 0 && m == 0) continue;
            if ((double)(n * n + m * m) <= eps * eps && cnt < MAX_SAMPLES) {
                ns[cnt] = n;
                ms[cnt] = m;
                cnt++;
            }
        }
    return cnt;
}

/* Readable at step k: inside Omega_h and in Omega_h \ (D^(k)_h u B_h)
 * (Section 2.1: known and not a bystander, or already filled before step k). */
static int readable(const uint8_t *lab, const int32_t *shell, int H, int W, int x, int y, int k)
{
    if (x < 0 || y < 0 || x >= W || y >= H) return 0;
    size_t p = (size_t)y * W + x;
    if (lab[p] == LBL_KNOWN) return 1;
    if (lab[p] == LBL_HOLE) return shell[p] >= 0 && shell[p] < k;
    return 0;
}

static float snap_coord(float o, float tau)
{
    float r = rintf(o);
    float d = o - r;
    return (fabsf(d) <= tau) ? r : o;
}

/* Unit guide direction in FP32 (R2). */
static void unit_dir(float gx, float gy, float *ch, float *sh)
{
    float s = gx * gx;
    s = s + gy * gy;
    float a = sqrtf(s);
    if (a > 0.0f) {
        *ch = gx / a;
        *sh = gy / a;
    } else {
        *ch = 1.0f;
        *sh = 0.0f;
    }
}

/* Position of sample (n, m) of the rotated ball around x: x + n*gh + m*gh_perp
 * with gh_perp = (-sh, ch) (Notation: B~ = R(B)); FP32, then snapped (R4). */
static void sample_offset(int n, int m, float ch, float sh, float tau, float *ox, float *oy)
{
    float fn = (float)n, fm = (float)m;
    float a = fn * ch;
    float b = fm * sh;
    float x = a - b;
    float c = fn * sh;
    float d = fm * ch;
    float y = c + d;
    *ox = snap_coord(x, tau);
    *oy = snap_coord(y, tau);
}

typedef struct {
    int n;
    int tx[4], ty[4];
    double lam[4];
} taps_t;

/* Lattice pixels with non-zero bilinear weight at (x + ox, y + oy) and those
 * weights (eq. bilinearDef: tensor-product hat functions). */
static void bilinear_taps(int x, int y, float ox, float oy, taps_t *t)
{
    float flx = floorf(ox), fly = floorf(oy);
    float frx = ox - flx, fry = oy - fly;
    int ix = x + (int)flx, iy = y + (int)fly;
    double fx = (double)frx, fy = (double)fry;
    t->n = 0;
    t->tx[t->n] = ix;
    t->ty[t->n] = iy;
    t->lam[t->n++] = (1.0 - fx) * (1.0 - fy);
    if (frx > 0.0f) {
        t->tx[t->n] = ix + 1;
        t->ty[t->n] = iy;
        t->lam[t->n++] = fx * (1.0 - fy);
    }
    if (fry > 0.0f) {
        t->tx[t->n] = ix;
        t->ty[t->n] = iy + 1;
        t->lam[t->n++] = (1.0 - fx) * fy;
    }
    if (frx > 0.0f && fry > 0.0f) {
        t->tx[t->n] = ix + 1;
        t->ty[t->n] = iy + 1;
        t->lam[t->n++] = fx * fy;
    }
}

typedef struct {
    int H, W, C;
    const double *u;
    const uint8_t *lab;
    const int32_t *shell;
    const float *guide;
    double eps, mu, c, coef; /* coef = mu^2 / (2 eps^2) */
    unsigned flags;
    float tau;
    int ns;
    int n_[MAX_SAMPLES], m_[MAX_SAMPLES];
} fillctx;

/* Exponent t of the weight (eq. weight): w = exp(-t) / |y - x| with
 * t = mu^2/(2 eps^2) (g_perp . (y - x))^2.  For the rotated ball
 * y - x = n gh + m gh_perp, so g_perp . (y - x) = |g| m exactly; for the
 * lattice ball (coherence transport) y - x = (n, m). */
static double weight_exponent(const fillctx *F, float gx, float gy, int n, int m, int isotropic)
{
    if (isotropic) return 0.0;
    if (F->flags & OF_GHOST) {
        double a2 = (double)gx * (double)gx + (double)gy * (double)gy;
        return F->coef * a2 * (double)(m * m);
    } else {
        double proj = -(double)gy * (double)n + (double)gx * (double)m;
        return F->coef * proj * proj;
    }
}

/* Evaluates front pixel (x, y) at step k (Algorithm 1, eqs. weight,
 * bilinearDef, confidence, ready).  Returns 1 if ready; then writes the new
 * colour into out[C].  *conf receives C(x) (smart order), *any_rd whether at
 * least one sample was readable. */
static int evaluate(const fillctx *F, int x, int y, int k, int isotropic, double *out, double *conf,
                    int *any_rd)
{
    size_t p = (size_t)y * F->W + x;
    float gx = F->guide[2 * p], gy = F->guide[2 * p + 1];
    float ch = 1.0f, sh = 0.0f;
    if (!isotropic && (F->flags & OF_GHOST)) unit_dir(gx, gy, &ch, &sh);

    double t_s[MAX_SAMPLES];
    unsigned char ok_s[MAX_SAMPLES];
    taps_t taps_s[MAX_SAMPLES];
    double S_all = 0.0, S_rd = 0.0, t_min = INFINITY;
    int nrd = 0;
    for (int s = 0; s < F->ns; s++) {
        int n = F->n_[s], m = F->m_[s];
        float ox, oy;
        if (!isotropic && (F->flags & OF_GHOST)) {
            sample_offset(n, m, ch, sh, F->tau, &ox, &oy);
        } else {
            ox = (float)n;
            oy = (float)m;
        }
        bilinear_taps(x, y, ox, oy, &taps_s[s]);
        int ok = 1;
        for (int j = 0; j < taps_s[s].n; j++)
            if (!readable(F->lab, F->shell, F->H, F->W, taps_s[s].tx[j], taps_s[s].ty[j], k)) ok = 0;
        ok_s[s] = (unsigned char)ok;
        double t = weight_exponent(F, gx, gy, n, m, isotropic);
        t_s[s] = t;
        double w = exp(-t) / sqrt((double)(n * n + m * m));
        S_all += w;
        if (ok) {
            S_rd += w;
            nrd++;
            if (t < t_min) t_min = t;
        }
    }
    *any_rd = nrd > 0;
    double C = S_rd / S_all;
    *conf = C;
    int ready;
    if (isotropic || !(F->flags & OF_SMART))
        ready = nrd > 0;
    else
        ready = C > F->c;
    if (!ready) return 0;

    /* normalised weighted average over the readable samples (Algorithm 1; R6) */
    double acc[16] = {0};
    double wsum = 0.0;
    for (int s = 0; s < F->ns; s++) {
        if (!ok_s[s]) continue;
        int n = F->n_[s], m = F->m_[s];
        double w = exp(-(t_s[s] - t_min)) / sqrt((double)(n * n + m * m));
        wsum += w;
        for (int j = 0; j < taps_s[s].n; j++) {
            size_t q = (size_t)taps_s[s].ty[j] * F->W + taps_s[s].tx[j];
            for (int ch2 = 0; ch2 < F->C; ch2++) acc[ch2] += w * taps_s[s].lam[j] * F->u[q * F->C + ch2];
        }
    }
    for (int ch2 = 0; ch2 < F->C; ch2++) out[ch2] = acc[ch2] / wsum;
    return 1;
}

/* Active boundary test (Notation, d_active D^(k)_h; Algorithm 1): a hole pixel
 * not yet filled with at least one readable 8-neighbour. */
static int in_front(const fillctx *F, int x, int y, int k)
{
    size_t p = (size_t)y * F->W + x;
    if (F->lab[p] != LBL_HOLE || F->shell[p] != SH_UNFILLED) return 0;
    for (int dy = -1; dy <= 1; dy++)
        for (int dx = -1; dx <= 1; dx++) {
            if (!dx && !dy) continue;
            if (readable(F->lab, F->shell, F->H, F->W, x + dx, y + dy, k)) return 1;
        }
    return 0;
}

/*
 * Algorithm 1 (shell-based geometric inpainting) with Guidefill's rotated
 * ghost-pixel ball, weights (eq. weight), bilinear extension (eq.
 * bilinearDef) and smart order (eqs. confidence, ready).  Each step k:
 *   front_k = active boundary of D^(k) (full rescan of the image);
 *   every front pixel is evaluated against D^(k) (same-step fills invisible);
 *   F = ready pixels; they are written; D^(k+1) = D^(k) \ F.
 * u      [H][W][C] FP64, updated in place at filled pixels
 * shell  [H][W] out: -1 known, -3 bystander, -2 hole never filled, k filled at step k
 * enter  [H][W] out (optional): first step at which the pixel joined the front, -1 never
 * stall_steps [max_shells] out (optional): 1 where step k was filled by the stall rule
 * Returns 0 on success, 1 if some hole pixels were never filled, -1 on bad arguments.
 */
int oracle_fill(int H, int W, int C, double *u, const uint8_t *lab, const float *guide, double eps,
                double mu, double c, unsigned flags, float tau, int max_shells, int32_t *shell,
                int32_t *enter, uint8_t *stall_steps, oracle_stats *st)
{
    if (H <= 0 || W <= 0 || C <= 0 || C > 16 || !(eps >= 1.0) || eps > 16.0) return -1;
    fillctx *F = (fillctx *)calloc(1, sizeof(fillctx));
    if (!F) return -1;
    F->H = H; F->W = W; F->C = C; F->u = u; F->lab = lab; F->shell = shell; F->guide = guide;
    F->eps = eps; F->mu = mu; F->c = c; F->flags = flags; F->tau = tau;
    F->coef = mu * mu / (2.0 * eps * eps);
    F->ns = disc_points(eps, F->n_, F->m_);

    size_t N = (size_t)H * W;
    int64_t holes = 0;
    for (size_t p = 0; p < N; p++) {
        shell[p] = lab[p] == LBL_KNOWN ? SH_KNOWN : lab[p] == LBL_HOLE ? SH_UNFILLED : SH_BYST;
        if (enter) enter[p] = -1;
        if (lab[p] == LBL_HOLE) holes++;
    }
    memset(st, 0, sizeof(*st));
    st->min_margin = 1e300;
    if (max_shells <= 0) max_shells = (int)(holes + 1);

    int32_t *front = (int32_t *)malloc(sizeof(int32_t) * (N > 0 ? N : 1));
    double *newc = (double *)malloc(sizeof(double) * (N > 0 ? N : 1) * C);
    uint8_t *rdy = (uint8_t *)malloc(N > 0 ? N : 1);
    uint8_t *rdy0 = (uint8_t *)malloc(N > 0 ? N : 1);
    int64_t filled = 0;
    /* eq. ready2 (Section 3.5, possible extensions): while phase 1 lasts, a front
     * pixel is ready only if also D(x) = |g(x)| > c2 = 0.  Phase 1 ends at the first
     * step at which no unfilled hole pixel has g != 0, or at which it would fill
     * nothing (that step is then evaluated with eq. ready); from then on eq. ready. */
    int phase1 = (flags & OF_DATA) != 0;
    st->data_switch = -1;
    int k;
    for (k = 0; k < max_shells; k++) {
        size_t nf = 0;
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x++)
                if (in_front(F, x, y, k)) front[nf++] = (int32_t)((size_t)y * W + x);
        if (nf == 0) break;
        if ((int64_t)nf > st->max_front) st->max_front = (int64_t)nf;
        st->evaluations += (int64_t)nf;
        if (phase1) {
            int64_t gleft = 0;
            for (size_t p = 0; p < N; p++)
                if (shell[p] == SH_UNFILLED && (guide[2 * p] != 0.0f || guide[2 * p + 1] != 0.0f)) gleft++;
            if (gleft == 0) {
                phase1 = 0;
                st->data_switch = k;
            }
        }
        size_t nready = 0;
        for (size_t i = 0; i < nf; i++) {
            int p = front[i];
            if (enter && enter[p] < 0) enter[p] = k;
            double conf;
            int any;
            rdy0[i] = (uint8_t)evaluate(F, p % W, p / W, k, 0, &newc[i * C], &conf, &any);
            if ((flags & OF_SMART) && c > 0) {
                double mg = fabs(conf - c) / c;
                if (mg < st->min_margin) st->min_margin = mg;
            }
            rdy[i] = rdy0[i];
            if (phase1 && guide[2 * (size_t)p] == 0.0f && guide[2 * (size_t)p + 1] == 0.0f) rdy[i] = 0;
            nready += rdy[i];
        }
        if (phase1 && nready == 0) {
            phase1 = 0;
            st->data_switch = k;
            for (size_t i = 0; i < nf; i++) {
                rdy[i] = rdy0[i];
                nready += rdy[i];
            }
        }
        int stall = 0;
        if (nready == 0) { /* R7 */
            stall = 1;
            for (size_t i = 0; i < nf; i++) {
                int p = front[i];
                double conf;
                int any;
                rdy[i] = (uint8_t)evaluate(F, p % W, p / W, k, 1, &newc[i * C], &conf, &any);
                nready += rdy[i];
            }
            if (nready == 0) break;
            st->stalls++;
        }
        if (stall_steps) stall_steps[k] = (uint8_t)stall;
        for (size_t i = 0; i < nf; i++) {
            if (!rdy[i]) continue;
            int p = front[i];
            for (int ch2 = 0; ch2 < C; ch2++) u[(size_t)p * C + ch2] = newc[i * C + ch2];
            shell[p] = k;
        }
        filled += (int64_t)nready;
    }
    st->shells = 0;
    for (size_t p = 0; p < N; p++)
        if (shell[p] >= 0 && shell[p] + 1 > st->shells) st->shells = shell[p] + 1;
    st->filled = filled;
    st->unreachable = holes - filled;
    free(front);
    free(newc);
    free(rdy);
    free(rdy0);
    free(F);
    return st->unreachable > 0 ? 1 : 0;
}

/* ---------------------------------------------------------------------- */
/*
 * Guide field from splines (Section 3.3): for each hole pixel x, the nearest
 * polyline segment over all splines; if its distance d <= 3 eta,
 * g(x) = t * exp(-d^2 / (2 eta^2)) with t the segment's unit tangent, else 0.
 * The nearest-segment choice and the 3-eta cut are decided in FP32 with a
 * fixed expression (ties: lowest global segment index); the returned value is
 * computed in FP64 for the chosen segment and rounded once to FP32.  The paper
 * fixes no rounding for this choice; the expression (with 1/|v|^2 formed once
 * per segment) was chosen to be the one the CUDA sampler evaluates, so that
 * both sides decide near-ties alike.  Where a decision is that close to a tie
 * (two segments within SEG_TIE_PX, or d within SEG_TIE_PX of 3 eta) both
 * choices are valid readings and the other choice's value is reported.
 * offsets[n+1], pts[P][2] as (x, y); guide [H][W][2] is written at hole
 * pixels only.  Zero-length segments are skipped.
 */
static float seg_dist2_f32(float px, float py, float ax, float ay, float bx, float by)
{
    float vx = bx - ax, vy = by - ay;
    float wx = px - ax, wy = py - ay;
    float l2 = vx * vx;
    l2 = l2 + vy * vy;
    float inv_l2 = 1.0f / l2; /* once per segment in the CUDA sampler */
    float dot = wx * vx;
    dot = dot + wy * vy;
    float t = dot * inv_l2;
    if (t < 0.0f) t = 0.0f;
    if (t > 1.0f) t = 1.0f;
    float qx = wx - t * vx;
    float qy = wy - t * vy;
    float d2 = qx * qx;
    d2 = d2 + qy * qy;
    return d2;
}

/* FP64 value of the guide field at pixel (x, y) from segment bi: t = ((x - a).v)
 * * (1/|v|^2) clamped to [0, 1], d^2 = |x - a - t v|^2, g = (v/|v|) *
 * exp(-(d^2 * (1/(2 eta^2)))) * w, rounded once to FP32 (Section 3.3:
 * g_Gamma e^(-d^2/(2 eta^2)) with |g_Gamma| = w the spline's coherence weight,
 * 1 when no weights are given).  *dist receives the FP64 distance d. */
static void seg_value(int n_splines, const int32_t *offsets, const float *pts, const float *weight, int bi,
                      int x, int y, double k2, float *gx, float *gy, double *dist)
{
    int sb = 0;
    while (sb + 1 < n_splines && offsets[sb + 1] <= bi) sb++;
    double w = weight ? (double)weight[sb] : 1.0;
    double ax = pts[2 * bi], ay = pts[2 * bi + 1];
    double bx = pts[2 * bi + 2], by = pts[2 * bi + 3];
    double vx = bx - ax, vy = by - ay;
    double len = sqrt(vx * vx + vy * vy);
    double inv_l2 = 1.0 / (len * len);
    double wx = (double)x - ax, wy = (double)y - ay;
    double t = (wx * vx + wy * vy) * inv_l2;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    double qx = wx - t * vx, qy = wy - t * vy;
    double d2 = qx * qx + qy * qy;
    double e = exp(-(d2 * k2));
    *gx = (float)(vx / len * e * w);
    *gy = (float)(vy / len * e * w);
    *dist = sqrt(d2);
}

/* Width of the band around a tie within which the nearest-segment choice and
 * the 3 eta cut are left to rounding: two segments whose FP64 distances differ
 * by less than this (in pixels), or a distance this close to 3 eta.  The FP32
 * distance expression errs by about 7 * 2^-24 * |v| px (|v| the segment
 * length), i.e. under 1e-4 px for segments up to 200 px. */
#define SEG_TIE_PX 1e-3

/*
 * alt [H][W][2] (optional): where the pixel's decision is within SEG_TIE_PX of
 * a tie, the value the other choice gives (the runner-up segment, or 0 / the
 * nearest segment's value across the 3 eta cut); elsewhere the same value as
 * guide.  Both are valid readings of "the nearest spline" there.
 * tie [H][W] (optional): 1 where alt holds the other choice.
 * min_gap (optional): the smallest decision gap (px) over the hole pixels that
 * are not ties (> SEG_TIE_PX by construction; +inf when there is none).
 * Returns the number of tie pixels, or -1 on bad arguments.
 */
int oracle_guidance(int H, int W, const uint8_t *lab, int n_splines, const int32_t *offsets,
                    const float *pts, float eta, const float *weight, float *guide, float *alt,
                    uint8_t *tie, double *min_gap)
{
    if (H <= 0 || W <= 0 || n_splines < 0 || !(eta > 0.0f)) return -1;
    float t3 = 3.0f * eta;
    float thr = t3 * t3;
    double k2 = 1.0 / (2.0 * (double)eta * (double)eta); /* 1/(2 eta^2) */
    double cut = 3.0 * (double)eta;
    int ties = 0;
    double mg = INFINITY;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            size_t p = (size_t)y * W + x;
            if (tie) tie[p] = 0;
            if (lab[p] != LBL_HOLE) continue;
            float px = (float)x, py = (float)y;
            float best = INFINITY, second = INFINITY;
            int bi = -1, si = -1;
            for (int s = 0; s < n_splines; s++)
                for (int i = offsets[s]; i + 1 < offsets[s + 1]; i++) {
                    float ax = pts[2 * i], ay = pts[2 * i + 1];
                    float bx = pts[2 * i + 2], by = pts[2 * i + 3];
                    float vx = bx - ax, vy = by - ay;
                    float l2 = vx * vx;
                    l2 = l2 + vy * vy;
                    if (!(l2 > 0.0f)) continue;
                    float d2 = seg_dist2_f32(px, py, ax, ay, bx, by);
                    if (d2 < best) {
                        second = best;
                        si = bi;
                        best = d2;
                        bi = i;
                    } else if (d2 < second) {
                        second = d2;
                        si = i;
                    }
                }
            float g0x = 0.0f, g0y = 0.0f, g1x = 0.0f, g1y = 0.0f;
            double d_best = INFINITY, d_second = INFINITY;
            if (bi >= 0) seg_value(n_splines, offsets, pts, weight, bi, x, y, k2, &g1x, &g1y, &d_best);
            const int inside = bi >= 0 && best <= thr;
            if (inside) {
                g0x = g1x;
                g0y = g1y;
            }
            guide[2 * p] = g0x;
            guide[2 * p + 1] = g0y;
            /* the decisions' gaps: runner-up segment, and the 3 eta cut */
            float ax_ = g0x, ay_ = g0y;
            double gap = INFINITY;
            int is_tie = 0;
            if (bi >= 0) {
                double gc = fabs(d_best - cut);
                if (gc < SEG_TIE_PX) {
                    is_tie = 1;
                    ax_ = inside ? 0.0f : g1x;
                    ay_ = inside ? 0.0f : g1y;
                } else if (gc < gap) {
                    gap = gc;
                }
            }
            if (inside && si >= 0) {
                float sx, sy;
                seg_value(n_splines, offsets, pts, weight, si, x, y, k2, &sx, &sy, &d_second);
                double gs = fabs(d_second - d_best);
                if (gs < SEG_TIE_PX) {
                    is_tie = 1;
                    ax_ = sx;
                    ay_ = sy;
                } else if (gs < gap) {
                    gap = gs;
                }
            }
            if (is_tie) ties++;
            else if (gap < mg) mg = gap;
            if (alt) {
                alt[2 * p] = ax_;
                alt[2 * p + 1] = ay_;
            }
            if (tie) tie[p] = (uint8_t)is_tie;
        }
    if (min_gap) *min_gap = mg;
    return ties;
}

/* ---------------------------------------------------------------------- */
/*
 * Algorithmic byte count of one fill under Algorithm 1's per-step semantics,
 * from the oracle's own sets (no reuse across steps):
 *   sum_k  |E_k| (8 B guide + 4 B front-list read)
 *        + |T_k| 4 B   distinct pixels whose state the E_k ready tests inspect
 *        + |U_k| 12 B  distinct pixels whose RGB the F_k fills read
 *        + |F_k| (12 B RGB + 4 B shell) writes
 *        + |front_{k+1}| 4 B front-list write
 * E_k = front_k pixels that joined the front at step k or have a pixel filled
 * at step k-1 within the ceil(eps) box (the only pixels whose ready test can
 * change).  Stall steps count their normal evaluation only.
 */
int64_t oracle_alg_bytes(int H, int W, const uint8_t *lab, const float *guide, double eps,
                         unsigned flags, float tau, const int32_t *shell, const int32_t *enter)
{
    size_t N = (size_t)H * W;
    int R = (int)ceil(eps);
    fillctx *F = (fillctx *)calloc(1, sizeof(fillctx));
    F->H = H; F->W = W; F->lab = lab; F->shell = shell; F->guide = guide; F->eps = eps;
    F->flags = flags; F->tau = tau;
    F->ns = disc_points(eps, F->n_, F->m_);
    int K = 0;
    for (size_t p = 0; p < N; p++)
        if (shell[p] >= 0 && shell[p] + 1 > K) K = shell[p] + 1;
    int32_t *stampT = (int32_t *)malloc(sizeof(int32_t) * N);
    int32_t *stampU = (int32_t *)malloc(sizeof(int32_t) * N);
    for (size_t p = 0; p < N; p++) stampT[p] = stampU[p] = -1;
    int64_t bytes = 0;
    for (int k = 0; k < K; k++) {
        int64_t nE = 0, nT = 0, nU = 0, nF = 0, nQ1 = 0;
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x++) {
                size_t p = (size_t)y * W + x;
                if (lab[p] != LBL_HOLE || enter[p] < 0) continue;
                int sh = shell[p];
                if (enter[p] <= k + 1 && (sh < 0 || sh >= k + 1)) nQ1++;
                if (!(enter[p] <= k && (sh < 0 || sh >= k))) continue;
                int wake = enter[p] == k;
                for (int dy = -R; dy <= R && !wake; dy++)
                    for (int dx = -R; dx <= R && !wake; dx++) {
                        int xx = x + dx, yy = y + dy;
                        if (xx < 0 || yy < 0 || xx >= W || yy >= H) continue;
                        if (shell[(size_t)yy * W + xx] == k - 1) wake = 1;
                    }
                if (!wake) continue;
                nE++;
                float gx = guide[2 * p], gy = guide[2 * p + 1];
                float ch = 1.0f, shh = 0.0f;
                if (flags & OF_GHOST) unit_dir(gx, gy, &ch, &shh);
                int filled_now = sh == k;
                if (filled_now) nF++;
                for (int s = 0; s < F->ns; s++) {
                    float ox, oy;
                    if (flags & OF_GHOST)
                        sample_offset(F->n_[s], F->m_[s], ch, shh, tau, &ox, &oy);
                    else {
                        ox = (float)F->n_[s];
                        oy = (float)F->m_[s];
                    }
                    taps_t t;
                    bilinear_taps(x, y, ox, oy, &t);
                    int ok = 1;
                    for (int j = 0; j < t.n; j++) {
                        if (t.tx[j] < 0 || t.ty[j] < 0 || t.tx[j] >= W || t.ty[j] >= H) {
                            ok = 0;
                            continue;
                        }
                        size_t q = (size_t)t.ty[j] * W + t.tx[j];
                        if (stampT[q] != k) {
                            stampT[q] = k;
                            nT++;
                        }
                        if (!readable(lab, shell, H, W, t.tx[j], t.ty[j], k)) ok = 0;
                    }
                    if (ok && filled_now)
                        for (int j = 0; j < t.n; j++) {
                            size_t q = (size_t)t.ty[j] * W + t.tx[j];
                            if (stampU[q] != k) {
                                stampU[q] = k;
                                nU++;
                            }
                        }
                }
            }
        /* pixels filled at step k that were not counted as evaluated (cannot
         * happen for an exact tracker; counted for completeness) */
        bytes += nE * 12 + nT * 4 + nU * 12 + nF * 16 + nQ1 * 4;
    }
    free(stampT);
    free(stampU);
    free(F);
    return bytes;
}

/*
 * Adjoint of the Guidefill fill for the CPU oracle -- TEST INFRASTRUCTURE ONLY
 * (called by tests and the benchmark's CPU leg, never by the product path).
 *
 * The fill is differentiated as a map of the known colours u0, the guidance
 * angle field phi (g = |g| (cos phi, sin phi), |g| held fixed) and mu, with the
 * step at which every pixel is filled, the stall steps and every ghost
 * sample's set of bilinear taps held fixed (they are piecewise constant in
 * phi and mu, so their derivative is zero almost everywhere).
 *
 * Frozen forward model, for each pixel x filled at step k (increasing k):
 *   samples s = (n, m) of the ball (origin excluded);
 *   position p_s = x + n gh + m gh_perp, gh = (cos phi, sin phi),
 *   gh_perp = (-sin phi, cos phi)                       (Notation: B~ = R(B))
 *   v_s = sum_t L_t(p_s) u(t) over the sample's taps t   (eq. bilinearDef)
 *   w_s = exp(-mu^2 |g|^2 m^2 / (2 eps^2)) / |(n, m)|    (eq. weight)
 *   u(x) = sum_{s readable} w_s v_s / sum_{s readable} w_s   (Algorithm 1)
 * A step filled by the stall rule uses the unrotated ball and weights 1/|(n,m)|.
 * The readable samples and the taps are those of the forward run (FP32
 * offsets from the FP32 guide, snapped, exactly as oracle_fill); the bilinear
 * weights L_t are evaluated at the FP64 position relative to that frozen cell
 * (along an axis with a single tap the position does not enter).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define LBL_KNOWN 0
#define LBL_HOLE 1
#define MAXS 1024

typedef struct {
    int ns;
    int n[MAXS], m[MAXS];
} disc_t;

static void make_disc(double eps, disc_t *D)
{
    int R = (int)ceil(eps);
    D->ns = 0;
    for (int m = -R; m <= R; m++)
        for (int n = -R; n <= R; n++) {
            if (n == 0 && m == 0) continue;
            if ((double)(n * n + m * m) <= eps * eps && D->ns < MAXS) {
                D->n[D->ns] = n;
                D->m[D->ns] = m;
                D->ns++;
            }
        }
}

static int readable_s(const uint8_t *lab, const int32_t *shell, int H, int W, int x, int y, int k)
{
    if (x < 0 || y < 0 || x >= W || y >= H) return 0;
    size_t p = (size_t)y * W + x;
    if (lab[p] == LBL_KNOWN) return 1;
    if (lab[p] == LBL_HOLE) return shell[p] >= 0 && shell[p] < k;
    return 0;
}

static float snapf(float o, float tau)
{
    float r = rintf(o);
    float d = o - r;
    return (fabsf(d) <= tau) ? r : o;
}

/* The forward's frozen cell of one sample: base lattice cell, which axes carry
 * two taps, readability. */
typedef struct {
    int ix, iy;      /* lattice cell corner (absolute) */
    int ax, ay;      /* axis active (two taps along it) */
    int ok;          /* readable at the pixel's step */
} cell_t;

static void frozen_cell(int x, int y, float gx, float gy, int n, int m, int iso, float tau, cell_t *c)
{
    float ch = 1.0f, sh = 0.0f;
    if (!iso) {
        float s = gx * gx;
        s = s + gy * gy;
        float a = sqrtf(s);
        if (a > 0.0f) {
            ch = gx / a;
            sh = gy / a;
        }
    }
    float fn = (float)n, fm = (float)m;
    float ox, oy;
    if (!iso) {
        float t1 = fn * ch, t2 = fm * sh, t3 = fn * sh, t4 = fm * ch;
        ox = snapf(t1 - t2, tau);
        oy = snapf(t3 + t4, tau);
    } else {
        ox = fn;
        oy = fm;
    }
    float flx = floorf(ox), fly = floorf(oy);
    c->ix = x + (int)flx;
    c->iy = y + (int)fly;
    c->ax = (ox - flx) > 0.0f;
    c->ay = (oy - fly) > 0.0f;
}

typedef struct {
    int H, W, C;
    const uint8_t *lab;
    const float *guide;
    const int32_t *shell;
    const uint8_t *stall;  /* [K] */
    int K;
    double eps, coef;      /* coef = 1 / (2 eps^2) (mu enters separately) */
    float tau;
    disc_t D;
} adjctx;

/* Per-sample data of pixel x at its step, for a given phi and mu. */
typedef struct {
    int ns;
    cell_t cell[MAXS];
    double px[MAXS], py[MAXS];     /* FP64 positions */
    double dpx[MAXS], dpy[MAXS];   /* d position / d phi */
    double w[MAXS];                /* normalised weights over readable samples */
    double lam[MAXS];              /* d ln w / d mu */
} pix_t;

static int pixel_samples(const adjctx *A, int x, int y, double phi, double mu, pix_t *P)
{
    size_t p = (size_t)y * A->W + x;
    int k = A->shell[p];
    int iso = A->stall[k] != 0;
    float gx = A->guide[2 * p], gy = A->guide[2 * p + 1];
    double a2 = (double)gx * (double)gx + (double)gy * (double)gy;
    double c = cos(phi), s = sin(phi);
    float g2 = gx * gx;
    g2 = g2 + gy * gy;
    const int dir = !iso && sqrtf(g2) > 0.0f; /* the forward rotates only where the FP32 |g| > 0 */
    if (!dir) {
        c = 1.0;
        s = 0.0;
    }
    double tmin = INFINITY;
    double t[MAXS];
    int any = 0;
    P->ns = A->D.ns;
    for (int i = 0; i < A->D.ns; i++) {
        int n = A->D.n[i], m = A->D.m[i];
        cell_t *ce = &P->cell[i];
        frozen_cell(x, y, gx, gy, n, m, iso, A->tau, ce);
        int ok = 1;
        int taps[4][2] = {{ce->ix, ce->iy}, {ce->ix + 1, ce->iy}, {ce->ix, ce->iy + 1}, {ce->ix + 1, ce->iy + 1}};
        int use[4] = {1, ce->ax, ce->ay, ce->ax && ce->ay};
        for (int j = 0; j < 4; j++)
            if (use[j] && !readable_s(A->lab, A->shell, A->H, A->W, taps[j][0], taps[j][1], k)) ok = 0;
        ce->ok = ok;
        P->px[i] = x + n * c - m * s;
        P->py[i] = y + n * s + m * c;
        P->dpx[i] = dir ? (-n * s - m * c) : 0.0;
        P->dpy[i] = dir ? (n * c - m * s) : 0.0;
        t[i] = iso ? 0.0 : mu * mu * a2 * (double)(m * m) * A->coef;
        P->lam[i] = iso ? 0.0 : -2.0 * mu * a2 * (double)(m * m) * A->coef;
        if (ok) {
            any = 1;
            if (t[i] < tmin) tmin = t[i];
        }
    }
    if (!any) return 0;
    double ws = 0.0;
    for (int i = 0; i < A->D.ns; i++) {
        int n = A->D.n[i], m = A->D.m[i];
        P->w[i] = P->cell[i].ok ? exp(-(t[i] - tmin)) / sqrt((double)(n * n + m * m)) : 0.0;
        ws += P->w[i];
    }
    for (int i = 0; i < A->D.ns; i++) P->w[i] /= ws;
    return 1;
}

/* Bilinear weights of the 4 cell corners at the FP64 position and their
 * derivatives along x and y (axes with a single tap: weight 1 / 0, derivative 0). */
static void hat(const cell_t *c, double px, double py, double L[4], double Lx[4], double Ly[4])
{
    double fx = c->ax ? px - c->ix : 0.0, fy = c->ay ? py - c->iy : 0.0;
    double wx[2] = {1.0 - fx, fx}, wy[2] = {1.0 - fy, fy};
    double dx[2] = {c->ax ? -1.0 : 0.0, c->ax ? 1.0 : 0.0}, dy[2] = {c->ay ? -1.0 : 0.0, c->ay ? 1.0 : 0.0};
    for (int b = 0; b < 2; b++)
        for (int a = 0; a < 2; a++) {
            int j = a + 2 * b;
            L[j] = wx[a] * wy[b];
            Lx[j] = dx[a] * wy[b];
            Ly[j] = wx[a] * dy[b];
        }
}

static int tap_used(const cell_t *c, int j)
{
    return j == 0 || (j == 1 && c->ax) || (j == 2 && c->ay) || (j == 3 && c->ax && c->ay);
}

static int32_t *order_by_shell(const int32_t *shell, size_t N, int K, int **start)
{
    int *cnt = (int *)calloc((size_t)K + 1, sizeof(int));
    for (size_t p = 0; p < N; p++)
        if (shell[p] >= 0 && shell[p] < K) cnt[shell[p] + 1]++;
    for (int k = 0; k < K; k++) cnt[k + 1] += cnt[k];
    int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (cnt[K] > 0 ? cnt[K] : 1));
    int *pos = (int *)malloc(sizeof(int) * ((size_t)K + 1));
    memcpy(pos, cnt, sizeof(int) * ((size_t)K + 1));
    for (size_t p = 0; p < N; p++)
        if (shell[p] >= 0 && shell[p] < K) ord[pos[shell[p]]++] = (int32_t)p;
    free(pos);
    *start = cnt;
    return ord;
}

/*
 * Frozen forward: u_out = fill with the schedule of (shell, stall) and the
 * taps of `guide`, at angle field phi (FP64, per pixel; NULL = angle of guide)
 * and mu.  u_in/u_out [H][W][C] FP64 (u_out may equal u_in).  Returns 0.
 */
int oracle_frozen_fill(int H, int W, int C, const double *u_in, const uint8_t *lab, const float *guide,
                       const double *phi, double eps, double mu, float tau, const int32_t *shell,
                       const uint8_t *stall, int K, double *u_out)
{
    adjctx A = {H, W, C, lab, guide, shell, stall, K, eps, 1.0 / (2.0 * eps * eps), tau};
    make_disc(eps, &A.D);
    size_t N = (size_t)H * W;
    if (u_out != u_in) memcpy(u_out, u_in, sizeof(double) * N * C);
    int *start;
    int32_t *ord = order_by_shell(shell, N, K, &start);
    pix_t *P = (pix_t *)malloc(sizeof(pix_t));
    for (int k = 0; k < K; k++)
        for (int i = start[k]; i < start[k + 1]; i++) {
            int p = ord[i], x = p % W, y = p / W;
            double ph = phi ? phi[p] : atan2((double)guide[2 * p + 1], (double)guide[2 * p]);
            if (!pixel_samples(&A, x, y, ph, mu, P)) continue;
            double acc[16] = {0};
            for (int s = 0; s < P->ns; s++) {
                if (!P->cell[s].ok) continue;
                double L[4], Lx[4], Ly[4];
                hat(&P->cell[s], P->px[s], P->py[s], L, Lx, Ly);
                for (int j = 0; j < 4; j++) {
                    if (!tap_used(&P->cell[s], j)) continue;
                    size_t q = (size_t)(P->cell[s].iy + (j >> 1)) * W + P->cell[s].ix + (j & 1);
                    for (int c = 0; c < C; c++) acc[c] += P->w[s] * L[j] * u_out[q * C + c];
                }
            }
            for (int c = 0; c < C; c++) u_out[(size_t)p * C + c] = acc[c];
        }
    free(P);
    free(ord);
    free(start);
    return 0;
}

/*
 * Reverse sweep (FP64) of the frozen forward at phi = angle of guide.
 * u_out: the forward's output image (values at every tap are final).
 * grad_out [H][W][C]: dL/du_out.  Outputs: grad_in [H][W][C] = dL/du_in (zero
 * at filled hole pixels), grad_phi [H][W] (zero where g = 0 or at stall-filled
 * pixels), *grad_mu.  Returns 0.
 */
int oracle_fill_backward(int H, int W, int C, const double *u_out, const uint8_t *lab, const float *guide,
                         double eps, double mu, float tau, const int32_t *shell, const uint8_t *stall, int K,
                         const double *grad_out, double *grad_in, double *grad_phi, double *grad_mu)
{
    adjctx A = {H, W, C, lab, guide, shell, stall, K, eps, 1.0 / (2.0 * eps * eps), tau};
    make_disc(eps, &A.D);
    size_t N = (size_t)H * W;
    memcpy(grad_in, grad_out, sizeof(double) * N * C);
    for (size_t p = 0; p < N; p++) grad_phi[p] = 0.0;
    double gmu = 0.0;
    int *start;
    int32_t *ord = order_by_shell(shell, N, K, &start);
    pix_t *P = (pix_t *)malloc(sizeof(pix_t));
    for (int k = K - 1; k >= 0; k--)
        for (int i = start[k]; i < start[k + 1]; i++) {
            int p = ord[i], x = p % W, y = p / W;
            double ub[16];
            for (int c = 0; c < C; c++) {
                ub[c] = grad_in[(size_t)p * C + c];
                grad_in[(size_t)p * C + c] = 0.0;  /* the input value of a filled pixel is never used */
            }
            double ph = atan2((double)guide[2 * p + 1], (double)guide[2 * p]);
            if (!pixel_samples(&A, x, y, ph, mu, P)) continue;
            /* v_s and dv_s/dphi */
            double lbar = 0.0;
            for (int s = 0; s < P->ns; s++) lbar += P->w[s] * P->lam[s];
            double dphi = 0.0, dmu = 0.0;
            for (int s = 0; s < P->ns; s++) {
                if (!P->cell[s].ok) continue;
                double L[4], Lx[4], Ly[4];
                hat(&P->cell[s], P->px[s], P->py[s], L, Lx, Ly);
                double vdot_u = 0.0, dvdot_u = 0.0;
                for (int j = 0; j < 4; j++) {
                    if (!tap_used(&P->cell[s], j)) continue;
                    size_t q = (size_t)(P->cell[s].iy + (j >> 1)) * W + P->cell[s].ix + (j & 1);
                    double dL = Lx[j] * P->dpx[s] + Ly[j] * P->dpy[s];
                    for (int c = 0; c < C; c++) {
                        vdot_u += L[j] * u_out[q * C + c] * ub[c];
                        dvdot_u += dL * u_out[q * C + c] * ub[c];
                        grad_in[q * C + c] += P->w[s] * L[j] * ub[c];
                    }
                }
                dphi += P->w[s] * dvdot_u;
                dmu += P->w[s] * (P->lam[s] - lbar) * vdot_u;
            }
            grad_phi[p] = dphi;
            gmu += dmu;
        }
    *grad_mu = gmu;
    free(P);
    free(ord);
    free(start);
    return 0;
}

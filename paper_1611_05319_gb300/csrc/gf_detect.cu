// Automatic spline detection (Guidefill, arxiv 1611.05319, Section 3.3) for sm_103a.
//
// A ring R of known pixels a distance dR from the hole; Canny edge detection
// on an annulus of known pixels around it; for every ring pixel on an accepted
// edge, the structure tensor J_{sigma,rho} (eq. structureTensor) there and a
// straight spline along its minor eigenvector v-, signed to point into the
// hole, weighted by tanh((lambda+ - lambda-)/Lambda) (g_Gamma).
//
// Seven launches over 32x32-pixel tiles of all frames of a request:
//   dist     Chebyshev distances to the hole and to any pixel not known (one
//            row pass and one column pass in shared memory); flags the tiles
//            that hold an annulus pixel;
//   tensor   on flagged tiles: the tile's input window (tile + rS + rR + 1 px)
//            staged in shared memory, u_sigma (rows, then columns), T = sum_c
//            grad u_sigma (x) grad u_sigma, the rho-blur of T along rows, then
//            per annulus pixel non-maximum suppression and the two thresholds,
//            and per ring pixel on an edge the column rho-blur (J), its
//            eigenvector, sign and weight;
//   union    union-find over the edge pixels (8-connected), lock-free hooking
//            of the larger root under the smaller one;
//   mark     roots of components holding a strong pixel;
//   accept   kept edge pixels; ring pixels among them as one 32-bit mask per
//            row segment of a tile;
//   scan     per frame, output positions in raster order (one CTA per frame);
//   write    the splines.
// Every value a decision depends on is formed with correctly rounded FP32
// operations in a fixed order (no contraction), so the sets and the end points
// do not depend on the machine.

#include "gf_detect.cuh"

namespace gf {

__device__ __forceinline__ int det_clamp(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ int det_frame_of(const int32_t *off, int n, int v)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&off[mid]) <= v) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void upload_detect_kernel(const __grid_constant__ DetectChunk c)
{
    for (int i = threadIdx.x; i < c.count; i += blockDim.x) {
        c.dst_frames[c.first + i] = c.frames[i];
        c.dst_to[c.first + i] = c.to[i];
    }
    if (threadIdx.x == 0 && c.last_chunk) c.dst_to[c.first + c.count] = c.to[c.count];
}

// ---------------------------------------------------------------------------
// distances

__global__ void __launch_bounds__(DET_THREADS) detect_dist_kernel(const __grid_constant__ DetectArgs a)
{
    extern __shared__ uint8_t dsm[];
    const int gt = blockIdx.x;
    const int f = det_frame_of(a.tile_offset, a.n_frames, gt);
    const DetectFrameDev &F = a.frames[f];
    const int t = gt - __ldg(&a.tile_offset[f]);
    const int x0 = (t % F.NBX) * DT, y0 = (t / F.NBX) * DT;
    const int cap = a.cap, L = DT + 2 * cap;
    const int far = cap + 1;
    uint8_t *lab = dsm;            // [L][L]: bit 0 hole, bit 1 not known (0 outside the image)
    uint8_t *rh = dsm + L * L;     // [L][DT] distance along the row to a hole pixel
    uint8_t *ra = rh + L * DT;     // [L][DT] distance along the row to a pixel not known
    if (t == 0 && threadIdx.x == 0) F.result[1] = 0;
    int any = 0;
    for (int i = threadIdx.x; i < L * L; i += blockDim.x) {
        const int Y = y0 - cap + i / L, X = x0 - cap + i % L;
        uint8_t v = 0;
        if (Y >= 0 && Y < F.H && X >= 0 && X < F.W) {
            const uint8_t l = __ldg(&F.labels[(size_t)Y * F.W + X]);
            v = (uint8_t)((l == 1 ? 1 : 0) | (l != 0 ? 2 : 0));
        }
        lab[i] = v;
        any |= v;
    }
    any = __syncthreads_or(any);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int X = x0 + lane;
    if (!any) {
        // nothing but known pixels within cap of the tile
        for (int r = warp; r < DT; r += DET_THREADS / 32) {
            const int Y = y0 + r;
            if (Y < F.H && X < F.W) F.dist[(size_t)Y * F.W + X] = make_uchar2((uint8_t)far, (uint8_t)far);
        }
        if (threadIdx.x == 0) F.active[t] = 0;
        return;
    }
    for (int i = threadIdx.x; i < L * DT; i += blockDim.x) {
        const uint8_t *row = lab + (i / DT) * L + cap + (i % DT);
        int dh = far, da = far;
        for (int d = 0; d <= cap; d++) {
            const uint8_t v = row[-d] | row[d];
            if (da == far && (v & 2)) da = d;
            if (v & 1) {
                dh = d;  // a hole pixel is not known, so da <= d is already set
                break;
            }
        }
        rh[i] = (uint8_t)dh;
        ra[i] = (uint8_t)da;
    }
    __syncthreads();
    int ann = 0;
    for (int r = warp; r < DT; r += DET_THREADS / 32) {
        const int Y = y0 + r;
        if (Y >= F.H || X >= F.W) continue;
        int bh = far, ba = far;
        for (int dy = -cap; dy <= cap; dy++) {
            const int ady = dy < 0 ? -dy : dy;
            const int k = (r + cap + dy) * DT + lane;
            bh = min(bh, max(ady, (int)rh[k]));
            ba = min(ba, max(ady, (int)ra[k]));
        }
        F.dist[(size_t)Y * F.W + X] = make_uchar2((uint8_t)bh, (uint8_t)ba);
        const bool known = lab[(r + cap) * L + cap + lane] == 0;
        const int dd = bh - a.dR;
        if (known && dd <= a.annulus && -dd <= a.annulus) ann = 1;
    }
    ann = __syncthreads_or(ann);
    if (threadIdx.x == 0) F.active[t] = (uint8_t)(ann ? 1 : 0);
}

// ---------------------------------------------------------------------------
// tensor, suppression, thresholds, ring candidates

// unit minor eigenvector of [[a, b], [b, c]]; returns r = lambda+ - lambda-
__device__ __forceinline__ float det_minor_eigvec(float a, float b, float c, float &mx, float &my)
{
    const float d = __fsub_rn(a, c), e = __fmul_rn(2.0f, b);
    const float r = __fsqrt_rn(__fadd_rn(__fmul_rn(d, d), __fmul_rn(e, e)));
    float px, py;
    if (d >= 0.0f) {
        px = __fadd_rn(d, r);
        py = e;
    } else {
        px = e;
        py = __fsub_rn(r, d);
    }
    if (px == 0.0f && py == 0.0f) {
        px = 1.0f;
        py = 0.0f;
    }
    const float n = __fsqrt_rn(__fadd_rn(__fmul_rn(px, px), __fmul_rn(py, py)));
    px = __fdiv_rn(px, n);
    py = __fdiv_rn(py, n);
    mx = -py;
    my = px;
    return r;
}

__global__ void __launch_bounds__(DET_THREADS) detect_tensor_kernel(const __grid_constant__ DetectArgs a)
{
    extern __shared__ float tsm[];
    const int gt = blockIdx.x;
    const int f = det_frame_of(a.tile_offset, a.n_frames, gt);
    const DetectFrameDev &F = a.frames[f];
    const int t = gt - __ldg(&a.tile_offset[f]);
    const int x0 = (t % F.NBX) * DT, y0 = (t / F.NBX) * DT;
    const int H = F.H, W = F.W;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (!__ldg(&F.active[t])) {
        for (int r = warp; r < DT; r += DET_THREADS / 32) {
            const int Y = y0 + r, X = x0 + lane;
            if (Y < H && X < W) F.edge[(size_t)Y * W + X] = 0;
        }
        return;
    }
    const int rS = a.rS, rR = a.rR;
    const int Rh = rS + rR + 1;
    const int LI = DT + 2 * Rh, LU = DT + 2 * (rR + 1), LT = DT + 2 * rR;
    const int PA = LI * LI;                                      // plane of buffer A
    const int PB = max(LI * LU, LT * LT);                        // plane of buffer B
    float *A = tsm;
    float *B = tsm + 3 * PA;
    float *M = B + 3 * PB;                                       // [DT + 2][DT + 2] m2
    const int ix0 = x0 - Rh, iy0 = y0 - Rh;                      // origin of the input window
    const int ux0 = x0 - rR - 1, uy0 = y0 - rR - 1;              // origin of u_sigma
    const int tx0 = x0 - rR, ty0 = y0 - rR;                      // origin of T

    // 1. input window (RGB), planar [3][LI][LI]; cells outside the image are never read
    for (int i = threadIdx.x; i < LI * LI; i += blockDim.x) {
        const int Y = iy0 + i / LI, X = ix0 + i % LI;
        if (Y >= 0 && Y < H && X >= 0 && X < W) {
            const float4 v = __ldg(&F.rgba[(size_t)Y * W + X]);
            A[i] = v.x;
            A[PA + i] = v.y;
            A[2 * PA + i] = v.z;
        }
    }
    __syncthreads();
    // 2. g_sigma along rows: B[c][r][j], image rows of the window, columns ux0 + j
    for (int i = threadIdx.x; i < LI * LU; i += blockDim.x) {
        const int r = i / LU, j = i % LU;
        const int Y = iy0 + r, X = ux0 + j;
        if (Y < 0 || Y >= H || X < 0 || X >= W) continue;
        float acc[3] = {0.0f, 0.0f, 0.0f};
        for (int k = -rS; k <= rS; k++) {
            const float w = a.wS[k + rS];
            const int xx = det_clamp(X + k, 0, W - 1) - ix0;
#pragma unroll
            for (int c = 0; c < 3; c++) acc[c] = __fadd_rn(acc[c], __fmul_rn(w, A[c * PA + r * LI + xx]));
        }
#pragma unroll
        for (int c = 0; c < 3; c++) B[c * PB + r * LU + j] = acc[c];
    }
    __syncthreads();
    // 3. g_sigma along columns: u_sigma into A as [3][LU][LU]
    for (int i = threadIdx.x; i < LU * LU; i += blockDim.x) {
        const int r = i / LU, j = i % LU;
        const int Y = uy0 + r, X = ux0 + j;
        if (Y < 0 || Y >= H || X < 0 || X >= W) continue;
        float acc[3] = {0.0f, 0.0f, 0.0f};
        for (int k = -rS; k <= rS; k++) {
            const float w = a.wS[k + rS];
            const int yy = det_clamp(Y + k, 0, H - 1) - iy0;
#pragma unroll
            for (int c = 0; c < 3; c++) acc[c] = __fadd_rn(acc[c], __fmul_rn(w, B[c * PB + yy * LU + j]));
        }
#pragma unroll
        for (int c = 0; c < 3; c++) A[c * PA + r * LU + j] = acc[c];
    }
    __syncthreads();
    // 4. gradient and T = sum_c grad (x) grad into B as [3][LT][LT]; m2 = Txx + Tyy on the tile +- 1
    for (int i = threadIdx.x; i < LT * LT; i += blockDim.x) {
        const int r = i / LT, j = i % LT;
        const int Y = ty0 + r, X = tx0 + j;
        if (Y < 0 || Y >= H || X < 0 || X >= W) continue;
        const int xl = X > 0 ? X - 1 : X, xr = X < W - 1 ? X + 1 : X;
        const int yu = Y > 0 ? Y - 1 : Y, yd = Y < H - 1 ? Y + 1 : Y;
        const float sx = (float)(xr - xl), sy = (float)(yd - yu);
        float jxx = 0.0f, jxy = 0.0f, jyy = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float *U = A + c * PA;
            const float gx = sx > 0.0f ? __fdiv_rn(__fsub_rn(U[(Y - uy0) * LU + xr - ux0], U[(Y - uy0) * LU + xl - ux0]), sx)
                                       : 0.0f;
            const float gy = sy > 0.0f ? __fdiv_rn(__fsub_rn(U[(yd - uy0) * LU + X - ux0], U[(yu - uy0) * LU + X - ux0]), sy)
                                       : 0.0f;
            jxx = __fadd_rn(jxx, __fmul_rn(gx, gx));
            jxy = __fadd_rn(jxy, __fmul_rn(gx, gy));
            jyy = __fadd_rn(jyy, __fmul_rn(gy, gy));
        }
        B[r * LT + j] = jxx;
        B[PB + r * LT + j] = jxy;
        B[2 * PB + r * LT + j] = jyy;
        const int my = Y - y0 + 1, mx = X - x0 + 1;
        if (my >= 0 && my < DT + 2 && mx >= 0 && mx < DT + 2) M[my * (DT + 2) + mx] = __fadd_rn(jxx, jyy);
    }
    __syncthreads();
    // 5. g_rho along rows of T for the tile's columns: A as [3][LT][DT]
    for (int i = threadIdx.x; i < LT * DT; i += blockDim.x) {
        const int r = i / DT, j = i % DT;
        const int Y = ty0 + r, X = x0 + j;
        if (Y < 0 || Y >= H || X >= W) continue;
        float acc[3] = {0.0f, 0.0f, 0.0f};
        for (int k = -rR; k <= rR; k++) {
            const float w = a.wR[k + rR];
            const int xx = det_clamp(X + k, 0, W - 1) - tx0;
#pragma unroll
            for (int c = 0; c < 3; c++) acc[c] = __fadd_rn(acc[c], __fmul_rn(w, B[c * PB + r * LT + xx]));
        }
#pragma unroll
        for (int c = 0; c < 3; c++) A[c * PA + r * DT + j] = acc[c];
    }
    __syncthreads();
    // 6. per pixel: suppression and thresholds on the annulus; ring candidates
    for (int rr = warp; rr < DT; rr += DET_THREADS / 32) {
        const int Y = y0 + rr, X = x0 + lane;
        if (Y >= H || X >= W) continue;
        const size_t p = (size_t)Y * W + X;
        const uchar2 dd = F.dist[p];
        const uint8_t l = __ldg(&F.labels[p]);
        uint8_t cls = 0;
        const int dev = (int)dd.x - a.dR;
        if (l == 0 && dev <= a.annulus && -dev <= a.annulus) {
            const int ti = (Y - ty0) * LT + (X - tx0);
            const float d = __fsub_rn(B[ti], B[2 * PB + ti]), e = __fmul_rn(2.0f, B[PB + ti]);
            int q;
            if (fabsf(e) <= d) q = 0;
            else if (fabsf(e) <= -d) q = 2;
            else q = e > 0.0f ? 1 : 3;
            // neighbour offsets along the direction: 0 -> (1, 0), 45 -> (1, 1), 90 -> (0, 1), 135 -> (-1, 1)
            const int ox = q < 2 ? 1 : (q == 2 ? 0 : -1), oy = q == 0 ? 0 : 1;
            const int x1 = det_clamp(X + ox, 0, W - 1), y1 = det_clamp(Y + oy, 0, H - 1);
            const int x2 = det_clamp(X - ox, 0, W - 1), y2 = det_clamp(Y - oy, 0, H - 1);
            const float v = M[(Y - y0 + 1) * (DT + 2) + (X - x0 + 1)];
            const float n1 = M[(y1 - y0 + 1) * (DT + 2) + (x1 - x0 + 1)];
            const float n2 = M[(y2 - y0 + 1) * (DT + 2) + (x2 - x0 + 1)];
            if (v >= n1 && v >= n2) {
                if (v > a.th2) cls = 2;
                else if (v > a.tl2) cls = 1;
            }
        }
        F.edge[p] = cls;
        if (!cls) continue;
        F.parent[p] = (int32_t)p;
        F.mark[p] = 0;
        if (dd.x != a.dR || dd.y != a.dR) continue;
        // ring pixel on an edge: J = g_rho along columns, at this pixel
        float J[3] = {0.0f, 0.0f, 0.0f};
        for (int k = -rR; k <= rR; k++) {
            const float w = a.wR[k + rR];
            const int yy = det_clamp(Y + k, 0, H - 1) - ty0;
#pragma unroll
            for (int c = 0; c < 3; c++) J[c] = __fadd_rn(J[c], __fmul_rn(w, A[c * PA + yy * DT + lane]));
        }
        float vx, vy;
        const float rl = det_minor_eigvec(J[0], J[1], J[2], vx, vy);
        const float bx = (float)X, by = (float)Y, fdR = (float)a.dR;
        const int xp = det_clamp((int)floorf(__fadd_rn(__fadd_rn(bx, __fmul_rn(fdR, vx)), 0.5f)), 0, W - 1);
        const int yp = det_clamp((int)floorf(__fadd_rn(__fadd_rn(by, __fmul_rn(fdR, vy)), 0.5f)), 0, H - 1);
        const int xm = det_clamp((int)floorf(__fadd_rn(__fsub_rn(bx, __fmul_rn(fdR, vx)), 0.5f)), 0, W - 1);
        const int ym = det_clamp((int)floorf(__fadd_rn(__fsub_rn(by, __fmul_rn(fdR, vy)), 0.5f)), 0, H - 1);
        if (F.dist[(size_t)ym * W + xm].x < F.dist[(size_t)yp * W + xp].x) {
            vx = -vx;
            vy = -vy;
        }
        const float wgt = (float)tanh(__ddiv_rn((double)rl, (double)a.Lambda));
        F.cand[p] = make_float4(__fadd_rn(bx, __fmul_rn(a.length, vx)), __fadd_rn(by, __fmul_rn(a.length, vy)), wgt, 0.0f);
    }
}

// ---------------------------------------------------------------------------
// hysteresis: union-find over the edge pixels

constexpr int UF_BUDGET = 1 << 20;  // find / hook steps per thread before giving up

// root of x with path halving; budget counts the steps taken
__device__ __forceinline__ int uf_find(volatile int32_t *par, int x, int &budget)
{
    int p = par[x];
    while (p != x) {
        const int g = par[p];
        if (g == p) return p;
        par[x] = g;  // g is an ancestor of x: the forest stays valid
        x = g;
        p = par[x];
        if (--budget <= 0) return x;
    }
    return x;
}

__device__ __forceinline__ void uf_unite(volatile int32_t *par, int a, int b, int &budget)
{
    while (budget > 0) {
        a = uf_find(par, a, budget);
        b = uf_find(par, b, budget);
        if (a == b) return;
        if (a < b) {
            const int s = a;
            a = b;
            b = s;
        }
        // hook the larger root under the smaller one: parents only ever decrease
        const int old = atomicCAS((int *)&par[a], a, b);
        if (old == a) return;
        a = old;
        budget--;
    }
}

__global__ void __launch_bounds__(DET_THREADS) detect_union_kernel(const __grid_constant__ DetectArgs a)
{
    const int gt = blockIdx.x;
    const int f = det_frame_of(a.tile_offset, a.n_frames, gt);
    const DetectFrameDev &F = a.frames[f];
    const int t = gt - __ldg(&a.tile_offset[f]);
    if (!__ldg(&F.active[t])) return;
    const int x0 = (t % F.NBX) * DT, y0 = (t / F.NBX) * DT;
    const int H = F.H, W = F.W;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int32_t *par = F.parent;
    int budget = UF_BUDGET;
    for (int rr = warp; rr < DT; rr += DET_THREADS / 32) {
        const int Y = y0 + rr, X = x0 + lane;
        if (Y >= H || X >= W) continue;
        const int p = Y * W + X;
        if (!__ldg(&F.edge[p])) continue;
        // the four neighbours before p in raster order (the others see p)
        if (X > 0 && __ldg(&F.edge[p - 1])) uf_unite(par, p, p - 1, budget);
        if (Y > 0) {
            if (X > 0 && __ldg(&F.edge[p - W - 1])) uf_unite(par, p, p - W - 1, budget);
            if (__ldg(&F.edge[p - W])) uf_unite(par, p, p - W, budget);
            if (X + 1 < W && __ldg(&F.edge[p - W + 1])) uf_unite(par, p, p - W + 1, budget);
        }
    }
    if (budget <= 0) atomicExch(&F.result[1], (int)GF_ERR_TIMEOUT);
}

__global__ void __launch_bounds__(DET_THREADS) detect_mark_kernel(const __grid_constant__ DetectArgs a)
{
    const int gt = blockIdx.x;
    const int f = det_frame_of(a.tile_offset, a.n_frames, gt);
    const DetectFrameDev &F = a.frames[f];
    const int t = gt - __ldg(&a.tile_offset[f]);
    if (!__ldg(&F.active[t])) return;
    const int x0 = (t % F.NBX) * DT, y0 = (t / F.NBX) * DT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int32_t *par = F.parent;
    int budget = UF_BUDGET;
    for (int rr = warp; rr < DT; rr += DET_THREADS / 32) {
        const int Y = y0 + rr, X = x0 + lane;
        if (Y >= F.H || X >= F.W) continue;
        const int p = Y * F.W + X;
        if (__ldg(&F.edge[p]) == 2) F.mark[uf_find(par, p, budget)] = 1;
    }
    if (budget <= 0) atomicExch(&F.result[1], (int)GF_ERR_TIMEOUT);
}

__global__ void __launch_bounds__(DET_THREADS) detect_accept_kernel(const __grid_constant__ DetectArgs a)
{
    const int gt = blockIdx.x;
    const int f = det_frame_of(a.tile_offset, a.n_frames, gt);
    const DetectFrameDev &F = a.frames[f];
    const int t = gt - __ldg(&a.tile_offset[f]);
    const int tx = t % F.NBX;
    const int x0 = tx * DT, y0 = (t / F.NBX) * DT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool act = __ldg(&F.active[t]) != 0;
    volatile int32_t *par = F.parent;
    int budget = UF_BUDGET;
    for (int rr = warp; rr < DT; rr += DET_THREADS / 32) {
        const int Y = y0 + rr, X = x0 + lane;
        if (Y >= F.H) break;  // warp-uniform
        bool kept = false, ring = false;
        if (act && X < F.W) {
            const int p = Y * F.W + X;
            if (__ldg(&F.edge[p])) {
                kept = __ldcg(&F.mark[uf_find(par, p, budget)]) != 0;
                const uchar2 dd = F.dist[p];
                ring = kept && dd.x == a.dR && dd.y == a.dR;
            }
        }
        const uint32_t m = __ballot_sync(0xffffffffu, ring);
        if (lane == 0) F.accm[(size_t)Y * F.NBX + tx] = m;
        if (F.edges_out && X < F.W) F.edges_out[(size_t)Y * F.W + X] = kept ? 1 : 0;
    }
    if (budget <= 0) atomicExch(&F.result[1], (int)GF_ERR_TIMEOUT);
}

// one CTA per frame: exclusive prefix of the accepted counts over the row
// segments in raster order; the count and the polyline offsets
__global__ void __launch_bounds__(DET_SCAN_THREADS) detect_scan_kernel(const __grid_constant__ DetectArgs a)
{
    __shared__ uint32_t wsum[DET_SCAN_THREADS / 32];
    __shared__ uint32_t total_s;
    const DetectFrameDev &F = a.frames[blockIdx.x];
    const int n = F.H * F.NBX;
    const int per = (n + DET_SCAN_THREADS - 1) / DET_SCAN_THREADS;
    const int i0 = min(n, threadIdx.x * per), i1 = min(n, i0 + per);
    uint32_t s = 0;
    for (int i = i0; i < i1; i++) s += __popc(F.accm[i]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = lane < DET_SCAN_THREADS / 32 ? wsum[lane] : 0u;
        uint32_t w = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        if (lane < DET_SCAN_THREADS / 32) wsum[lane] = w - v;  // exclusive
        if (lane == 31) total_s = w;
    }
    __syncthreads();
    uint32_t run = wsum[warp] + incl - s;
    for (int i = i0; i < i1; i++) {
        F.accpos[i] = run;
        run += __popc(F.accm[i]);
    }
    const uint32_t total = total_s;
    if (threadIdx.x == 0) F.result[0] = (int32_t)total;
    for (int k = threadIdx.x; k <= F.max_splines; k += DET_SCAN_THREADS)
        F.offsets[k] = 2 * (int32_t)min((uint32_t)k, total);
}

__global__ void __launch_bounds__(DET_THREADS) detect_write_kernel(const __grid_constant__ DetectArgs a)
{
    const int gt = blockIdx.x;
    const int f = det_frame_of(a.tile_offset, a.n_frames, gt);
    const DetectFrameDev &F = a.frames[f];
    const int t = gt - __ldg(&a.tile_offset[f]);
    if (!__ldg(&F.active[t])) return;
    const int tx = t % F.NBX;
    const int x0 = tx * DT, y0 = (t / F.NBX) * DT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int rr = warp; rr < DT; rr += DET_THREADS / 32) {
        const int Y = y0 + rr, X = x0 + lane;
        if (Y >= F.H) break;
        const size_t seg = (size_t)Y * F.NBX + tx;
        const uint32_t m = F.accm[seg];
        if (!((m >> lane) & 1u)) continue;
        const uint32_t pos = F.accpos[seg] + __popc(m & ((1u << lane) - 1u));
        if (pos >= (uint32_t)F.max_splines) continue;
        const int p = Y * F.W + X;
        const float4 c = F.cand[p];
        F.pts[2 * pos] = make_float2((float)X, (float)Y);
        F.pts[2 * pos + 1] = make_float2(c.x, c.y);
        F.weight[pos] = c.z;
        if (F.base) F.base[pos] = p;
    }
}

}  // namespace gf

// Automatic spline detection (Guidefill, arxiv 1611.05319, Section 3.3) for sm_103a.
//
// A ring R of known pixels a distance dR from the hole; Canny edge detection
// on an annulus of known pixels around it; for every ring pixel on an accepted
// edge, the structure tensor J_{sigma,rho} (eq. structureTensor) there and a
// straight spline along its minor eigenvector v-, signed to point into the
// hole, weighted by tanh((lambda+ - lambda-)/Lambda) (g_Gamma).
//
// Nine launches over the frames of a request (32x32-pixel tiles):
//   pack     the labels as bit masks (hole, not known), 32 pixels a word, and
//            a flag per tile holding a hole pixel;
//   classify one thread per tile: the tiles a hole pixel may be within reach
//            of go to a slow list;
//   dist     persistent over the slow tiles: Chebyshev distance to the hole
//            and the ring test by bit-parallel dilation of the masks in shared
//            memory; tiles holding an annulus pixel are flagged and go to an
//            active list (every later kernel reads only flagged tiles' data);
//   tensor   persistent CTAs over the active tiles: the tile's window (tile +
//            rS + rR + 1 px) staged in shared memory one colour at a time,
//            u_sigma (rows, then columns), T = sum_c grad u_sigma (x) grad
//            u_sigma; per annulus pixel non-maximum suppression and the two
//            thresholds; per ring pixel on an edge J = g_rho * T there (one
//            warp), its eigenvector, sign and weight;
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
        c.dst_wo[c.first + i] = c.wo[i];
    }
    if (threadIdx.x == 0 && c.last_chunk) {
        c.dst_to[c.first + c.count] = c.to[c.count];
        c.dst_wo[c.first + c.count] = c.wo[c.count];
    }
}

// bits c (0..3) of the result: byte c of r is 0xff
__device__ __forceinline__ uint32_t det_nib(uint32_t r)
{
    return ((r >> 7) & 1u) | ((r >> 14) & 2u) | ((r >> 21) & 4u) | ((r >> 28) & 8u);
}

// One thread per 32-pixel word of a row of every frame: the hole and not-known
// bits of the word's labels (two 16-byte loads where the row allows).
__global__ void __launch_bounds__(256) detect_pack_kernel(const __grid_constant__ DetectArgs a, int total_words)
{
    const int gw = blockIdx.x * blockDim.x + threadIdx.x;
    if (gw >= total_words) return;
    const int f = det_frame_of(a.word_offset, a.n_frames, gw);
    const DetectFrameDev &F = a.frames[f];
    const int wi = gw - __ldg(&a.word_offset[f]);
    const int Y = wi / F.NWF, k = wi - Y * F.NWF;
    const int X0 = 32 * k;
    const uint8_t *row = F.labels + (size_t)Y * F.W + X0;
    uint32_t hole = 0u, nk = 0u;
    if (X0 + 32 <= F.W && (reinterpret_cast<uintptr_t>(row) & 15u) == 0) {
        const uint4 q0 = __ldg(reinterpret_cast<const uint4 *>(row));
        const uint4 q1 = __ldg(reinterpret_cast<const uint4 *>(row) + 1);
        const uint32_t v[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
        for (int j = 0; j < 8; j++) {
            hole |= det_nib(__vcmpeq4(v[j], 0x01010101u)) << (4 * j);
            nk |= det_nib(__vcmpne4(v[j], 0u)) << (4 * j);
        }
    } else {
        for (int c = 0; c < 32 && X0 + c < F.W; c++) {
            const uint8_t l = __ldg(&row[c]);
            if (l == 1) hole |= 1u << c;
            if (l != 0) nk |= 1u << c;
        }
    }
    F.masks[wi] = make_uint2(hole, nk);
    if (hole) F.hole_t[(Y >> 5) * F.NBX + k] = 1;  // word k of a row is tile column k
}

// One thread per tile of every frame: the tile's distances are needed when a
// hole pixel may lie within cap of it, i.e. when a tile within ceil(cap / 32)
// tiles holds one (a superset of the distance kernel's window); such tiles go
// to the slow list.
__global__ void __launch_bounds__(256) detect_classify_kernel(const __grid_constant__ DetectArgs a)
{
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    if (gt >= a.total_tiles) return;
    const int f = det_frame_of(a.tile_offset, a.n_frames, gt);
    const DetectFrameDev &F = a.frames[f];
    const int t = gt - __ldg(&a.tile_offset[f]);
    if (t == 0) F.result[1] = 0;
    const int tx = t % F.NBX, ty = t / F.NBX, c = (a.cap + 31) >> 5;
    uint8_t slow = 0;
    for (int y = max(0, ty - c); y <= min(F.NBY - 1, ty + c) && !slow; y++)
        for (int x = max(0, tx - c); x <= min(F.NBX - 1, tx + c); x++)
            if (__ldcg(&F.hole_t[y * F.NBX + x])) {
                slow = 1;
                break;
            }
    F.slow_t[t] = slow;
    if (slow) a.slow_list[atomicAdd(a.slow_count, 1)] = gt;
}

// ---------------------------------------------------------------------------
// distances

// One step of Chebyshev dilation (3x3 box) of a window's row masks at the
// padded word index i (pitch NWP = NW + 2; the one-word rim around the window
// is zero, so the step needs no bounds).
__device__ __forceinline__ uint32_t det_dilate_word(const uint32_t *src, int i, int NWP)
{
    uint32_t acc = 0u;
#pragma unroll
    for (int dr = -1; dr <= 1; dr++) {
        const uint32_t *row = src + i + dr * NWP;
        const uint32_t m = row[0];
        acc |= m | (m << 1) | (row[-1] >> 31) | (m >> 1) | (row[1] << 31);
    }
    return acc;
}

// Persistent CTAs over the slow tiles.  The window (tile +- cap rows, whole mask
// words around tile +- cap columns) of the packed masks is staged in shared
// memory.  Without a hole pixel in it the tile is far from the hole.
// Otherwise the Chebyshev distance of a pixel to the hole is the first k at
// which the hole mask dilated k times by the 3x3 box covers it; the window's
// masks are dilated a step at a time (bit-parallel, 32 pixels a word), and the
// tile's pixels read their distance off as they get covered.  The same
// dilation of the not-known mask, at k = dR - 1, gives the ring test: no pixel
// that is not known within dR - 1.  Errors from the window's edge move inward
// one pixel a step and never reach the tile within cap steps.  Tiles holding an
// annulus pixel are flagged and appended to the active list.
__global__ void __launch_bounds__(DET_THREADS) detect_dist_kernel(const __grid_constant__ DetectArgs a)
{
    extern __shared__ uint32_t dsm[];
    const int nslow = __ldcg(a.slow_count);
    for (int it = blockIdx.x; it < nslow; it += gridDim.x) {
    const int gt = __ldcg(&a.slow_list[it]);
    const int f = det_frame_of(a.tile_offset, a.n_frames, gt);
    const DetectFrameDev &F = a.frames[f];
    const int t = gt - __ldg(&a.tile_offset[f]);
    const int tx = t % F.NBX;
    const int x0 = tx * DT, y0 = (t / F.NBX) * DT;
    const int cap = a.cap, L = DT + 2 * cap, NW = detect_window_words(cap);
    const int NWP = NW + 2, LWP = (L + 2) * NWP;          // padded window: a zero word and row all round
    const int far = cap + 1;
    const int wx0 = tx - (NW >> 1);                       // first mask word of the window
    const int qx = x0 - 32 * wx0;                         // bit position of the tile's column 0
    // [0, 2 LWP): hole masks dilated k times (double buffer); [2 LWP, 4 LWP): not-known
    // masks likewise; [4 LWP, 5 LWP): not-known masks as loaded
    uint32_t *nk0 = dsm + 4 * LWP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int any = 0;
    for (int i = threadIdx.x; i < LWP; i += DET_THREADS) {
        const int r = i / NWP - 1, k = i % NWP - 1;       // window row and word (-1 and L / NW: the rim)
        const int Y = y0 - cap + r, kw = wx0 + k;
        uint2 v = make_uint2(0u, 0u);
        if (r >= 0 && r < L && k >= 0 && k < NW && Y >= 0 && Y < F.H && kw >= 0 && kw < F.NWF)
            v = __ldg(&F.masks[(size_t)Y * F.NWF + kw]);
#pragma unroll
        for (int b = 0; b < 2; b++) {
            dsm[b * LWP + i] = v.x;
            dsm[(2 + b) * LWP + i] = v.y;
        }
        nk0[i] = v.y;
        any |= v.x != 0u;
    }
    any = __syncthreads_or(any);
    const int X = x0 + lane;
    const int q = qx + lane;
    const int qw = (q >> 5) + 1, qb = q & 31;             // padded word of the thread's column
    int ann = 0;
    if (any) {
        // the thread's pixels: tile rows warp + 8 j, column lane
        int d[DT / 8];
        bool nkcov[DT / 8];
#pragma unroll
        for (int j = 0; j < DT / 8; j++) {
            d[j] = far;
            nkcov[j] = true;
        }
        // the thread's interior words of the padded window, at most 8 (L NW <= 226 * 9)
        int own[8];
        int nown = 0;
#pragma unroll
        for (int m = 0; m < 8; m++) {
            const int i = threadIdx.x + DET_THREADS * m;
            own[m] = 0;
            if (i < L * NW) {
                const int r = i / NW, w = i - r * NW;
                own[m] = (r + 1) * NWP + w + 1;
                nown = m + 1;
            }
        }
        const int kn = a.dR - 1;  // dilation steps of the ring test
        int cur = 0;
        for (int k = 0;; k++) {
            const uint32_t *hc = dsm + cur * LWP, *nc = dsm + (2 + cur) * LWP;
            uint32_t *hn = dsm + (cur ^ 1) * LWP, *nn = dsm + (2 + (cur ^ 1)) * LWP;
            bool done = true;
#pragma unroll
            for (int j = 0; j < DT / 8; j++) {
                const int row = (warp + 8 * j + cap + 1) * NWP + qw;
                if (d[j] == far && ((hc[row] >> qb) & 1u)) d[j] = k;
                if (k == kn) nkcov[j] = (nc[row] >> qb) & 1u;
                done = done && d[j] != far;
            }
            if (k == cap) break;
            if (__syncthreads_and(done && k >= kn)) break;
            const bool do_nk = k < kn;
#pragma unroll
            for (int m = 0; m < 8; m++) {
                if (m >= nown) break;
                hn[own[m]] = det_dilate_word(hc, own[m], NWP);
                if (do_nk) nn[own[m]] = det_dilate_word(nc, own[m], NWP);
            }
            __syncthreads();
            cur ^= 1;
        }
#pragma unroll
        for (int j = 0; j < DT / 8; j++) {
            const int r = warp + 8 * j;
            const int Y = y0 + r;
            if (Y >= F.H || X >= F.W) continue;
            const bool known = !((nk0[(r + cap + 1) * NWP + qw] >> qb) & 1u);
            const uint8_t ring = (known && d[j] == a.dR && !nkcov[j]) ? 1 : 0;
            F.dist[(size_t)Y * F.W + X] = make_uchar2((uint8_t)d[j], ring);
            const int dd = d[j] - a.dR;
            if (known && dd <= a.annulus && -dd <= a.annulus) ann = 1;
        }
    } else {
        // no hole pixel within cap of the tile
        for (int r = warp; r < DT; r += DET_THREADS / 32) {
            const int Y = y0 + r;
            if (Y < F.H && X < F.W) F.dist[(size_t)Y * F.W + X] = make_uchar2((uint8_t)far, 0);
        }
    }
    ann = __syncthreads_or(ann);  // also: every read of the window is done before the next tile's loads
    if (ann && threadIdx.x == 0) {
        F.act_t[t] = 1;
        a.active_list[atomicAdd(a.active_count, 1)] = gt;
    }
    }
}

// Warp-per-tile form of the distance kernel for cap <= 31, where the window is
// at most 94 rows of 3 mask words: lane l holds window rows l, l + 32, l + 64 of
// both masks in registers, a dilation step takes the rows above and below from
// the neighbouring lanes by shuffles (rows past the window stay part of the
// domain: they start empty and hold no original bits, so every pixel still
// reads the OR of the original bits within its box), and the lane whose row is
// tile row y counts, in bit-sliced 6-bit counters, the steps at which each of
// its 32 pixels is not yet covered: that count is the distance (cap + 1 when
// never covered).  No block barriers; eight tiles per CTA at once.
constexpr int DW_SLOTS = 3;  // window rows per lane

__device__ __forceinline__ uint32_t det_sel3(int s, uint32_t a0, uint32_t a1, uint32_t a2)
{
    return s == 0 ? a0 : (s == 1 ? a1 : a2);
}

// one 3x3-box dilation step of a window held as m[slot][word] (row = lane + 32 slot)
__device__ __forceinline__ void det_dilate_warp(uint32_t (&m)[DW_SLOTS][3], int lane)
{
    uint32_t up[DW_SLOTS][3], dn[DW_SLOTS][3];
#pragma unroll
    for (int s = 0; s < DW_SLOTS; s++)
#pragma unroll
        for (int w = 0; w < 3; w++) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, m[s][w], 1);
            const uint32_t uw = __shfl_sync(0xffffffffu, s > 0 ? m[s > 0 ? s - 1 : 0][w] : 0u, 31);
            up[s][w] = lane == 0 ? (s > 0 ? uw : 0u) : u;
            const uint32_t d = __shfl_down_sync(0xffffffffu, m[s][w], 1);
            const uint32_t dw = __shfl_sync(0xffffffffu, s + 1 < DW_SLOTS ? m[s + 1 < DW_SLOTS ? s + 1 : s][w] : 0u, 0);
            dn[s][w] = lane == 31 ? (s + 1 < DW_SLOTS ? dw : 0u) : d;
        }
#pragma unroll
    for (int s = 0; s < DW_SLOTS; s++) {
        // the three rows' OR first (vertical step), then the horizontal step on it
        const uint32_t v0 = up[s][0] | m[s][0] | dn[s][0];
        const uint32_t v1 = up[s][1] | m[s][1] | dn[s][1];
        const uint32_t v2 = up[s][2] | m[s][2] | dn[s][2];
        m[s][0] = v0 | (v0 << 1) | (v0 >> 1) | (v1 << 31);
        m[s][1] = v1 | (v1 << 1) | (v1 >> 1) | (v0 >> 31) | (v2 << 31);
        m[s][2] = v2 | (v2 << 1) | (v2 >> 1) | (v1 >> 31);
    }
}

__global__ void __launch_bounds__(DET_THREADS) detect_dist_warp_kernel(const __grid_constant__ DetectArgs a)
{
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (DET_THREADS / 32);
    const int nslow = __ldcg(a.slow_count);
    const int cap = a.cap, L = DT + 2 * cap, far = cap + 1, kn = a.dR - 1;
    // tile row y of this lane: window row cap + y == lane (mod 32), in slot ts
    const int ty = (lane - cap) & 31, ts = (cap + ty) >> 5;
    for (int it = blockIdx.x * (DET_THREADS / 32) + (threadIdx.x >> 5); it < nslow; it += nwarps) {
        const int gt = __ldcg(&a.slow_list[it]);
        const int f = det_frame_of(a.tile_offset, a.n_frames, gt);
        const DetectFrameDev &F = a.frames[f];
        const int t = gt - __ldg(&a.tile_offset[f]);
        const int tx = t % F.NBX;
        const int x0 = tx * DT, y0 = (t / F.NBX) * DT;
        uint32_t h[DW_SLOTS][3], nk[DW_SLOTS][3];
        bool anyh = false;
#pragma unroll
        for (int s = 0; s < DW_SLOTS; s++) {
            const int r = lane + 32 * s, Y = y0 - cap + r;
#pragma unroll
            for (int w = 0; w < 3; w++) {
                const int k = tx - 1 + w;
                uint2 v = make_uint2(0u, 0u);
                if (r < L && Y >= 0 && Y < F.H && k >= 0 && k < F.NWF) v = __ldg(&F.masks[(size_t)Y * F.NWF + k]);
                h[s][w] = v.x;
                nk[s][w] = v.y;
                anyh = anyh || v.x != 0u;
            }
        }
        const uint32_t nk_orig = det_sel3(ts, nk[0][1], nk[1][1], nk[2][1]);
        uint32_t cnt[6] = {0u, 0u, 0u, 0u, 0u, 0u};
        uint32_t nkcov = 0xffffffffu;
        if (__any_sync(0xffffffffu, anyh)) {
            for (int k = 0;; k++) {
                const uint32_t cov = det_sel3(ts, h[0][1], h[1][1], h[2][1]);
                uint32_t carry = ~cov;  // pixels not covered at step k
#pragma unroll
                for (int b = 0; b < 6; b++) {
                    const uint32_t c2 = cnt[b] & carry;
                    cnt[b] ^= carry;
                    carry = c2;
                }
                if (k == kn) nkcov = det_sel3(ts, nk[0][1], nk[1][1], nk[2][1]);
                if (k == cap) break;
                if (__all_sync(0xffffffffu, cov == 0xffffffffu) && k >= kn) break;
                det_dilate_warp(h, lane);
                if (k < kn) det_dilate_warp(nk, lane);
            }
        } else {
#pragma unroll
            for (int b = 0; b < 6; b++) cnt[b] = ((far >> b) & 1) ? 0xffffffffu : 0u;
        }
        // the tile's rows, one at a time, from the lane holding each (coalesced writes)
        bool ann = false;
        for (int y = 0; y < DT; y++) {
            const int o = (cap + y) & 31;
            int d = 0;
#pragma unroll
            for (int b = 0; b < 6; b++) d |= (int)((__shfl_sync(0xffffffffu, cnt[b], o) >> lane) & 1u) << b;
            const uint32_t nkc = __shfl_sync(0xffffffffu, nkcov, o), nko = __shfl_sync(0xffffffffu, nk_orig, o);
            const int Y = y0 + y, X = x0 + lane;
            if (Y >= F.H || X >= F.W) continue;
            const bool known = !((nko >> lane) & 1u);
            const uint8_t ring = (known && d == a.dR && !((nkc >> lane) & 1u)) ? 1 : 0;
            F.dist[(size_t)Y * F.W + X] = make_uchar2((uint8_t)d, ring);
            const int dd = d - a.dR;
            if (known && dd <= a.annulus && -dd <= a.annulus) ann = true;
        }
        if (__any_sync(0xffffffffu, ann) && lane == 0) {
            F.act_t[t] = 1;
            a.active_list[atomicAdd(a.active_count, 1)] = gt;
        }
    }
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

// i / d for 0 <= i < 8192 and 32 <= d <= 82 (the window sides): with m =
// ceil(2^20 / d), i m < 2^32 and i (m d - 2^20) < 2^20, so the quotient is exact
struct DetDiv {
    uint32_t d, m;
    __device__ __forceinline__ explicit DetDiv(uint32_t d_) : d(d_), m(((1u << 20) + d_ - 1u) / d_) {}
    __device__ __forceinline__ uint32_t q(uint32_t i) const { return (i * m) >> 20; }
};

// distance to the hole at an image pixel: computed in slow tiles, cap + 1 elsewhere
__device__ __forceinline__ int det_dist_at(const DetectFrameDev &F, int X, int Y, int far)
{
    return __ldcg(&F.slow_t[(Y >> 5) * F.NBX + (X >> 5)]) ? (int)F.dist[(size_t)Y * F.W + X].x : far;
}

// edge class at an image pixel: written in active tiles, 0 elsewhere
__device__ __forceinline__ uint8_t det_edge_at(const DetectFrameDev &F, int X, int Y)
{
    return __ldcg(&F.act_t[(Y >> 5) * F.NBX + (X >> 5)]) ? F.edge[(size_t)Y * F.W + X] : 0;
}

__device__ __forceinline__ void det_cp_async4(float *dst, const float *src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void det_cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// T = sum over channels R, G, B of grad u_sigma (x) grad u_sigma at the image
// pixel (X, Y), from the three u_sigma planes U [3][LU][LU] with origin (ux0,
// uy0): central differences, one-sided at the image border (division by 2 as
// multiplication by 0.5, which is exact), products accumulated by fused
// multiply-add.
__device__ __forceinline__ void det_tensor_at(const float *U, int LU, int ux0, int uy0, int X, int Y, int W, int H,
                                              float &txx, float &txy, float &tyy)
{
    const int xl = X > 0 ? X - 1 : X, xr = X < W - 1 ? X + 1 : X;
    const int yu = Y > 0 ? Y - 1 : Y, yd = Y < H - 1 ? Y + 1 : Y;
    const float hx = xr - xl == 2 ? 0.5f : 1.0f, hy = yd - yu == 2 ? 0.5f : 1.0f;
    const int bc = (Y - uy0) * LU - ux0, bu = (yu - uy0) * LU - ux0, bd = (yd - uy0) * LU - ux0;
    const int PL = LU * LU;
    float jxx = 0.0f, jxy = 0.0f, jyy = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float *P = U + c * PL;
        const float gx = xr > xl ? __fmul_rn(__fsub_rn(P[bc + xr], P[bc + xl]), hx) : 0.0f;
        const float gy = yd > yu ? __fmul_rn(__fsub_rn(P[bd + X], P[bu + X]), hy) : 0.0f;
        jxx = __fmaf_rn(gx, gx, jxx);
        jxy = __fmaf_rn(gx, gy, jxy);
        jyy = __fmaf_rn(gy, gy, jyy);
    }
    txx = jxx;
    txy = jxy;
    tyy = jyy;
}

// Persistent CTAs over the active tiles.  Per tile, one colour channel at a
// time: the channel's plane of the window (tile +- rS + rR + 1), copied with
// cp.async from coordinates clamped to the image (so the blurs below read the
// border values the clamped definition reads, with no clamping per tap);
// g_sigma along rows, then along columns, each thread sliding a register
// window over a run of DSEG outputs (taps unrolled for the radius RS, one
// shared-memory load per output; odd row pitches keep the lanes, which walk
// consecutive rows, on distinct banks), into that channel's u_sigma plane.
// Then T and m2 = Txx + Tyy on the tile +- 1 only, suppression and thresholds
// per annulus pixel, and for the ring pixels on an edge (under one per tile on
// average) J = g_rho * T at that pixel by one warp: each lane the rho-blur along
// a row of the window with T formed on the fly, then the column sum in tap
// order.  Tap sums accumulate by fused multiply-add in tap order.
constexpr int DSEG = 8;
constexpr int DM = DT + 2;  // side of the tile +- 1

template <int RS>
__global__ void __launch_bounds__(DET_THREADS, 3) detect_tensor_kernel(const __grid_constant__ DetectArgs a)
{
    extern __shared__ float tsm[];
    __shared__ int cand_n;
    __shared__ short cand_s[DT * DT];
    constexpr int WIN = DSEG + 2 * RS;  // inputs of a run of DSEG outputs
    const int rR = a.rR;
    const int Rh = RS + rR + 1;
    const int LI = DT + 2 * Rh, LU = DT + 2 * (rR + 1);
    const int PI = LI | 1, PQ = LU | 1;   // odd pitches of the input and row-blurred planes
    const int NSEG = (LU + DSEG - 1) / DSEG;
    float *U = tsm;                                   // [3][LU][LU] u_sigma
    float *P = U + 3 * LU * LU;                       // [LI][PI] input plane of one channel
    float *Q = P + detect_plane_floats(LI, PI);       // [LI + DSEG - 1][PQ] rows blurred
    float *T3 = P;                                    // after the blurs: [3][DM][DM] T on the tile +- 1
    float *M = T3 + 3 * DM * DM;                      //                  [DM][DM] m2
    const DetDiv dI((uint32_t)LI), dU((uint32_t)LU);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float w[2 * RS + 1];
#pragma unroll
    for (int k = 0; k <= 2 * RS; k++) w[k] = a.wS[k];
    const int nact = __ldcg(a.active_count);
    for (int it = blockIdx.x; it < nact; it += gridDim.x) {
        const int gt = __ldcg(&a.active_list[it]);
        const int f = det_frame_of(a.tile_offset, a.n_frames, gt);
        const DetectFrameDev &F = a.frames[f];
        const int t = gt - __ldg(&a.tile_offset[f]);
        const int x0 = (t % F.NBX) * DT, y0 = (t / F.NBX) * DT;
        const int H = F.H, W = F.W;
        const int ix0 = x0 - Rh, iy0 = y0 - Rh;          // window origin
        const int ux0 = x0 - rR - 1, uy0 = y0 - rR - 1;  // u_sigma origin
        const float *img = reinterpret_cast<const float *>(F.rgba);
        // the thread's pixels (tile rows warp + 8 j, column lane): labels and distances, loaded early
        uchar2 dd[DT / 8];
        uint8_t lb[DT / 8];
#pragma unroll
        for (int j = 0; j < DT / 8; j++) {
            const int Y = y0 + warp + 8 * j, X = x0 + lane;
            dd[j] = make_uchar2(0, 0);
            lb[j] = 1;
            if (Y < H && X < W) {
                dd[j] = F.dist[(size_t)Y * W + X];
                lb[j] = __ldg(&F.labels[(size_t)Y * W + X]);
            }
        }
        for (int c = 0; c < 3; c++) {
            for (int r = warp; r < LI; r += DET_THREADS / 32) {
                const size_t rowb = (size_t)det_clamp(iy0 + r, 0, H - 1) * W;
                for (int j = lane; j < LI; j += 32)
                    det_cp_async4(P + r * PI + j, img + 4 * (rowb + det_clamp(ix0 + j, 0, W - 1)) + c);
            }
            det_cp_async_wait_all();
            __syncthreads();
            // rows: u_sigma column j reads window columns j .. j + 2 RS; lanes take
            // consecutive rows, each a run of DSEG columns
            for (uint32_t i = threadIdx.x; i < (uint32_t)(LI * NSEG); i += DET_THREADS) {
                const uint32_t sg = dI.q(i), r = i - sg * LI;
                const float *p = P + r * PI + sg * DSEG;
                float v[WIN];
#pragma unroll
                for (int k = 0; k < WIN; k++) v[k] = p[k];
                float *q = Q + r * PQ + sg * DSEG;
                const int nout = min(DSEG, LU - (int)(sg * DSEG));  // the last run stops at column LU
#pragma unroll
                for (int o = 0; o < DSEG; o++) {
                    float acc = 0.0f;
#pragma unroll
                    for (int k = 0; k <= 2 * RS; k++) acc = __fmaf_rn(w[k], v[o + k], acc);
                    if (o < nout) q[o] = acc;
                }
            }
            __syncthreads();
            // columns: u_sigma row r reads blurred rows r .. r + 2 RS; lanes take
            // consecutive columns, each a run of DSEG rows
            float *Uc = U + c * LU * LU;
            for (uint32_t i = threadIdx.x; i < (uint32_t)(LU * NSEG); i += DET_THREADS) {
                const uint32_t sg = dU.q(i), j = i - sg * LU;
                const float *q = Q + sg * DSEG * PQ + j;
                float v[WIN];
#pragma unroll
                for (int k = 0; k < WIN; k++) v[k] = q[k * PQ];
#pragma unroll
                for (int o = 0; o < DSEG; o++) {
                    const int r = sg * DSEG + o;
                    if (r >= LU) break;
                    float acc = 0.0f;
#pragma unroll
                    for (int k = 0; k <= 2 * RS; k++) acc = __fmaf_rn(w[k], v[o + k], acc);
                    Uc[r * LU + j] = acc;
                }
            }
            __syncthreads();  // P and Q are free for the next channel
        }
        // T and m2 on the tile and a one-pixel rim
        for (int i = threadIdx.x; i < DM * DM; i += DET_THREADS) {
            const int Y = y0 - 1 + i / DM, X = x0 - 1 + i % DM;
            if (Y < 0 || Y >= H || X < 0 || X >= W) continue;
            float txx, txy, tyy;
            det_tensor_at(U, LU, ux0, uy0, X, Y, W, H, txx, txy, tyy);
            T3[i] = txx;
            T3[DM * DM + i] = txy;
            T3[2 * DM * DM + i] = tyy;
            M[i] = __fadd_rn(txx, tyy);
        }
        if (threadIdx.x == 0) cand_n = 0;
        __syncthreads();
        // suppression and thresholds on the annulus
#pragma unroll
        for (int jj = 0; jj < DT / 8; jj++) {
            const int rr = warp + 8 * jj;
            const int Y = y0 + rr, X = x0 + lane;
            if (Y >= H || X >= W) continue;
            const size_t p = (size_t)Y * W + X;
            uint8_t cls = 0;
            const int dev = (int)dd[jj].x - a.dR;
            if (lb[jj] == 0 && dev <= a.annulus && -dev <= a.annulus) {
                const int ti = (rr + 1) * DM + lane + 1;
                const float d = __fsub_rn(T3[ti], T3[2 * DM * DM + ti]), e = __fmul_rn(2.0f, T3[DM * DM + ti]);
                int q;
                if (fabsf(e) <= d) q = 0;
                else if (fabsf(e) <= -d) q = 2;
                else q = e > 0.0f ? 1 : 3;
                // neighbours along the direction: 0 -> (1, 0), 45 -> (1, 1), 90 -> (0, 1), 135 -> (-1, 1)
                const int ox = q < 2 ? 1 : (q == 2 ? 0 : -1), oy = q == 0 ? 0 : 1;
                const int x1 = det_clamp(X + ox, 0, W - 1), y1 = det_clamp(Y + oy, 0, H - 1);
                const int x2 = det_clamp(X - ox, 0, W - 1), y2 = det_clamp(Y - oy, 0, H - 1);
                const float v = M[ti];
                const float n1 = M[(y1 - y0 + 1) * DM + (x1 - x0 + 1)];
                const float n2 = M[(y2 - y0 + 1) * DM + (x2 - x0 + 1)];
                if (v >= n1 && v >= n2) {
                    if (v > a.th2) cls = 2;
                    else if (v > a.tl2) cls = 1;
                }
            }
            F.edge[p] = cls;
            if (!cls) continue;
            F.parent[p] = (int32_t)p;
            F.mark[p] = 0;
            if (dd[jj].y) cand_s[atomicAdd(&cand_n, 1)] = (short)(rr * DT + lane);
        }
        __syncthreads();
        // J at the ring pixels on an edge, one warp each
        const int nc = cand_n;
        for (int ci = warp; ci < nc; ci += DET_THREADS / 32) {
            const int e = cand_s[ci];
            const int X = x0 + (e & (DT - 1)), Y = y0 + e / DT;
            float R[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int kk = lane + 32 * h;  // window row kk - rR
                if (kk > 2 * rR) continue;
                const int yy = det_clamp(Y + kk - rR, 0, H - 1);
                for (int k = 0; k <= 2 * rR; k++) {
                    const float wk = a.wR[k];
                    float tt[3];
                    det_tensor_at(U, LU, ux0, uy0, det_clamp(X + k - rR, 0, W - 1), yy, W, H, tt[0], tt[1], tt[2]);
#pragma unroll
                    for (int ch = 0; ch < 3; ch++) R[h][ch] = __fmaf_rn(wk, tt[ch], R[h][ch]);
                }
            }
            float J[3] = {0.0f, 0.0f, 0.0f};
            for (int kk = 0; kk <= 2 * rR; kk++) {
                const float wk = a.wR[kk];
                const bool hi = kk >= 32;
#pragma unroll
                for (int ch = 0; ch < 3; ch++) {
                    const float v = __shfl_sync(0xffffffffu, hi ? R[1][ch] : R[0][ch], kk & 31);
                    J[ch] = __fmaf_rn(wk, v, J[ch]);
                }
            }
            if (lane == 0) {
                float vx, vy;
                const float rl = det_minor_eigvec(J[0], J[1], J[2], vx, vy);
                const float bx = (float)X, by = (float)Y, fdR = (float)a.dR;
                const int xp = det_clamp((int)floorf(__fadd_rn(__fadd_rn(bx, __fmul_rn(fdR, vx)), 0.5f)), 0, W - 1);
                const int yp = det_clamp((int)floorf(__fadd_rn(__fadd_rn(by, __fmul_rn(fdR, vy)), 0.5f)), 0, H - 1);
                const int xm = det_clamp((int)floorf(__fadd_rn(__fsub_rn(bx, __fmul_rn(fdR, vx)), 0.5f)), 0, W - 1);
                const int ym = det_clamp((int)floorf(__fadd_rn(__fsub_rn(by, __fmul_rn(fdR, vy)), 0.5f)), 0, H - 1);
                if (det_dist_at(F, xm, ym, a.cap + 1) < det_dist_at(F, xp, yp, a.cap + 1)) {
                    vx = -vx;
                    vy = -vy;
                }
                const float wgt = (float)tanh(__ddiv_rn((double)rl, (double)a.Lambda));
                F.cand[(size_t)Y * W + X] = make_float4(__fadd_rn(bx, __fmul_rn(a.length, vx)),
                                                        __fadd_rn(by, __fmul_rn(a.length, vy)), wgt, 0.0f);
            }
        }
        __syncthreads();  // the next tile reuses shared memory
    }
}

const void *detect_tensor_entry(int rS)
{
    switch (rS) {
    case 1: return (const void *)detect_tensor_kernel<1>;
    case 2: return (const void *)detect_tensor_kernel<2>;
    case 3: return (const void *)detect_tensor_kernel<3>;
    case 4: return (const void *)detect_tensor_kernel<4>;
    case 5: return (const void *)detect_tensor_kernel<5>;
    case 6: return (const void *)detect_tensor_kernel<6>;
    case 7: return (const void *)detect_tensor_kernel<7>;
    case 8: return (const void *)detect_tensor_kernel<8>;
    default: return nullptr;
    }
}

cudaError_t launch_detect_tensor(int rS, unsigned grid, size_t smem, cudaStream_t st, const DetectArgs &a)
{
    switch (rS) {
    case 1: detect_tensor_kernel<1><<<grid, DET_THREADS, smem, st>>>(a); break;
    case 2: detect_tensor_kernel<2><<<grid, DET_THREADS, smem, st>>>(a); break;
    case 3: detect_tensor_kernel<3><<<grid, DET_THREADS, smem, st>>>(a); break;
    case 4: detect_tensor_kernel<4><<<grid, DET_THREADS, smem, st>>>(a); break;
    case 5: detect_tensor_kernel<5><<<grid, DET_THREADS, smem, st>>>(a); break;
    case 6: detect_tensor_kernel<6><<<grid, DET_THREADS, smem, st>>>(a); break;
    case 7: detect_tensor_kernel<7><<<grid, DET_THREADS, smem, st>>>(a); break;
    case 8: detect_tensor_kernel<8><<<grid, DET_THREADS, smem, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
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

// The later kernels run persistent CTAs over the active tiles (tile order does
// not change any result: the components of the union-find and every per-pixel
// output are the same whatever the order).
#define DET_FOR_ACTIVE_TILES(a)                                                   \
    const int nact_ = __ldcg((a).active_count);                                   \
    for (int it_ = blockIdx.x; it_ < nact_; it_ += gridDim.x)

struct DetTile {
    const DetectFrameDev *F;
    int tx, x0, y0;
};

__device__ __forceinline__ DetTile det_tile(const DetectArgs &a, int it)
{
    const int gt = __ldcg(&a.active_list[it]);
    const int f = det_frame_of(a.tile_offset, a.n_frames, gt);
    const DetectFrameDev *F = &a.frames[f];
    const int t = gt - __ldg(&a.tile_offset[f]);
    DetTile d;
    d.F = F;
    d.tx = t % F->NBX;
    d.x0 = d.tx * DT;
    d.y0 = (t / F->NBX) * DT;
    return d;
}

__global__ void __launch_bounds__(DET_THREADS) detect_union_kernel(const __grid_constant__ DetectArgs a)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int budget = UF_BUDGET;
    DET_FOR_ACTIVE_TILES(a)
    {
        const DetTile d = det_tile(a, it_);
        const DetectFrameDev &F = *d.F;
        const int H = F.H, W = F.W;
        volatile int32_t *par = F.parent;
        const int X = d.x0 + lane;
        uint8_t e[DT / 8];  // the thread's pixels (rows warp + 8 j), loaded together
#pragma unroll
        for (int j = 0; j < DT / 8; j++) {
            const int Y = d.y0 + warp + 8 * j;
            e[j] = (Y < H && X < W) ? __ldg(&F.edge[(size_t)Y * W + X]) : 0;
        }
#pragma unroll
        for (int j = 0; j < DT / 8; j++) {
            if (!e[j]) continue;
            const int Y = d.y0 + warp + 8 * j;
            const int p = Y * W + X;
            // the four neighbours before p in raster order (the others see p); inside the
            // tile they are read directly, across its border through the tile flags
            const bool in_l = X > d.x0, in_u = Y > d.y0, in_r = X + 1 < d.x0 + DT;
            if (X > 0 && (in_l ? __ldg(&F.edge[p - 1]) : det_edge_at(F, X - 1, Y))) uf_unite(par, p, p - 1, budget);
            if (Y > 0) {
                if (X > 0 && (in_l && in_u ? __ldg(&F.edge[p - W - 1]) : det_edge_at(F, X - 1, Y - 1)))
                    uf_unite(par, p, p - W - 1, budget);
                if (in_u ? __ldg(&F.edge[p - W]) : det_edge_at(F, X, Y - 1)) uf_unite(par, p, p - W, budget);
                if (X + 1 < W && (in_r && in_u ? __ldg(&F.edge[p - W + 1]) : det_edge_at(F, X + 1, Y - 1)))
                    uf_unite(par, p, p - W + 1, budget);
            }
        }
        if (budget <= 0) atomicExch(&F.result[1], (int)GF_ERR_TIMEOUT);
    }
}

__global__ void __launch_bounds__(DET_THREADS) detect_mark_kernel(const __grid_constant__ DetectArgs a)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int budget = UF_BUDGET;
    DET_FOR_ACTIVE_TILES(a)
    {
        const DetTile d = det_tile(a, it_);
        const DetectFrameDev &F = *d.F;
        volatile int32_t *par = F.parent;
        const int X = d.x0 + lane;
        uint8_t e[DT / 8];
#pragma unroll
        for (int j = 0; j < DT / 8; j++) {
            const int Y = d.y0 + warp + 8 * j;
            e[j] = (Y < F.H && X < F.W) ? __ldg(&F.edge[(size_t)Y * F.W + X]) : 0;
        }
#pragma unroll
        for (int j = 0; j < DT / 8; j++)
            if (e[j] == 2) F.mark[uf_find(par, (d.y0 + warp + 8 * j) * F.W + X, budget)] = 1;
        if (budget <= 0) atomicExch(&F.result[1], (int)GF_ERR_TIMEOUT);
    }
}

__global__ void __launch_bounds__(DET_THREADS) detect_accept_kernel(const __grid_constant__ DetectArgs a)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int budget = UF_BUDGET;
    DET_FOR_ACTIVE_TILES(a)
    {
        const DetTile d = det_tile(a, it_);
        const DetectFrameDev &F = *d.F;
        volatile int32_t *par = F.parent;
        const int X = d.x0 + lane;
        uint8_t e[DT / 8], ring[DT / 8];
#pragma unroll
        for (int j = 0; j < DT / 8; j++) {
            const int Y = d.y0 + warp + 8 * j;
            const bool in = Y < F.H && X < F.W;
            e[j] = in ? __ldg(&F.edge[(size_t)Y * F.W + X]) : 0;
            ring[j] = in ? F.dist[(size_t)Y * F.W + X].y : 0;
        }
#pragma unroll
        for (int j = 0; j < DT / 8; j++) {
            const int Y = d.y0 + warp + 8 * j;
            if (Y >= F.H) break;  // warp-uniform
            bool kept = false;
            if (e[j]) kept = __ldcg(&F.mark[uf_find(par, Y * F.W + X, budget)]) != 0;
            const uint32_t m = __ballot_sync(0xffffffffu, kept && ring[j]);
            if (lane == 0) F.accm[(size_t)Y * F.NBX + d.tx] = m;
            if (F.edges_out && X < F.W) F.edges_out[(size_t)Y * F.W + X] = kept ? 1 : 0;
        }
        if (budget <= 0) atomicExch(&F.result[1], (int)GF_ERR_TIMEOUT);
    }
}

// One CTA per frame: output positions in raster order, the exclusive prefix of
// the accepted counts over the frame's row segments [H][NBX].  Each warp takes a
// contiguous run of segments, 32 consecutive ones per step (coalesced): first
// the runs' totals, their prefix over the warps, then the positions.  Also the
// count and the polyline offsets.
__global__ void __launch_bounds__(DET_SCAN_THREADS) detect_scan_kernel(const __grid_constant__ DetectArgs a)
{
    constexpr int NWARP = DET_SCAN_THREADS / 32;
    __shared__ uint32_t wsum[NWARP];
    __shared__ uint32_t total_s;
    const DetectFrameDev &F = a.frames[blockIdx.x];
    const int n = F.H * F.NBX;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per = (((n + NWARP - 1) / NWARP) + 31) & ~31;
    const int s0 = min(n, warp * per), s1 = min(n, s0 + per);
    // the accepted ring pixels of row segment i (Y = i / NBX, tile column i % NBX); 0 outside
    // active tiles.  A warp's runs are read four steps of 32 at a time (independent loads).
    auto seg_count = [&](int i) -> uint32_t {
        if (i >= s1) return 0u;
        const int Y = i / F.NBX, tx = i - Y * F.NBX;
        const uint32_t m = __ldcg(&F.accm[i]);
        return __ldcg(&F.act_t[(Y >> 5) * F.NBX + tx]) ? (uint32_t)__popc(m) : 0u;
    };
    uint32_t tot = 0;
    for (int b = s0; b < s1; b += 128) {
        uint32_t c4[4];
#pragma unroll
        for (int u = 0; u < 4; u++) c4[u] = seg_count(b + 32 * u + lane);
#pragma unroll
        for (int u = 0; u < 4; u++) tot += __reduce_add_sync(0xffffffffu, c4[u]);
    }
    if (lane == 0) wsum[warp] = tot;
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = wsum[lane];
        uint32_t w = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        wsum[lane] = w - v;  // exclusive
        if (lane == 31) total_s = w;
    }
    __syncthreads();
    uint32_t run = wsum[warp];
    for (int b = s0; b < s1; b += 128) {
        uint32_t c4[4];
#pragma unroll
        for (int u = 0; u < 4; u++) c4[u] = seg_count(b + 32 * u + lane);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int i = b + 32 * u + lane;
            const uint32_t c = c4[u];
            uint32_t incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v2 = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v2;
            }
            if (i < s1) F.accpos[i] = run + incl - c;
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    const uint32_t total = total_s;
    if (threadIdx.x == 0) F.result[0] = (int32_t)total;
    for (int k = threadIdx.x; k <= F.max_splines; k += DET_SCAN_THREADS)
        F.offsets[k] = 2 * (int32_t)min((uint32_t)k, total);
}

__global__ void __launch_bounds__(DET_THREADS) detect_write_kernel(const __grid_constant__ DetectArgs a)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    DET_FOR_ACTIVE_TILES(a)
    {
        const DetTile d = det_tile(a, it_);
        const DetectFrameDev &F = *d.F;
        for (int rr = warp; rr < DT; rr += DET_THREADS / 32) {
            const int Y = d.y0 + rr, X = d.x0 + lane;
            if (Y >= F.H) break;
            const size_t seg = (size_t)Y * F.NBX + d.tx;
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
}

}  // namespace gf

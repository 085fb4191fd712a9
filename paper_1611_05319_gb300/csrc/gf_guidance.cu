// Guide field from splines (Guidefill, arxiv 1611.05319, Section 3.3) for sm_103a.
//
// g(x) = w_Gamma t_Gamma * exp(-d(x, Gamma)^2 / (2 eta^2)) for the nearest
// polyline segment Gamma when d <= 3 eta, else 0, at every hole pixel; w_Gamma =
// |g_Gamma| is the spline's weight (1 unless given, e.g. the coherence factor of
// detected splines).
//
// Two kernels per request:
//   bin_kernel    one thread per polyline point: the segment starting there is
//                 appended to every 32x32-pixel bin its bounding box, grown by
//                 3 eta + 1 px, overlaps (so no segment within 3 eta of a pixel
//                 is missed, FP32 rounding included);
//   guide_kernel  one CTA per bin: bins without hole pixels end after one
//                 load per row; otherwise the bin's segments are staged in
//                 shared memory and each hole pixel takes the nearest one.  A
//                 bin whose list overflowed scans all segments of its frame.
// The nearest-segment choice and the 3-eta cut use a fixed FP32 expression
// with no contraction (ties: lowest segment index), so the decision does not
// depend on the machine; the returned value is evaluated in FP64 for the
// chosen segment and rounded once to FP32.

#include "gf_detect.cuh"

namespace gf {

__global__ void upload_splines_kernel(const __grid_constant__ SplineChunk c)
{
    for (int i = threadIdx.x; i < c.count; i += blockDim.x) {
        c.dst_frames[c.first + i] = c.frames[i];
        c.dst_po[c.first + i] = c.po[i];
        c.dst_bo[c.first + i] = c.bo[i];
    }
    if (threadIdx.x == 0 && c.last_chunk) {
        c.dst_po[c.first + c.count] = c.po[c.count];
        c.dst_bo[c.first + c.count] = c.bo[c.count];
    }
}

__device__ __forceinline__ int find_frame(const int32_t *off, int n, int v)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(&off[mid]) <= v) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) bin_kernel(const __grid_constant__ GuideArgs a, int total_points)
{
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= total_points) return;
    int f = find_frame(a.point_offset, a.n_frames, gi);
    const SplineFrameDev &F = a.frames[f];
    int i = gi - __ldg(&a.point_offset[f]);
    // spline s with offsets[s] <= i < offsets[s+1]; the segment needs i+1 < offsets[s+1]
    int lo = 0, hi = F.n_splines;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(&F.offsets[mid]) <= i) lo = mid; else hi = mid;
    }
    if (F.n_splines <= 0 || i + 1 >= F.n_points || i < __ldg(&F.offsets[0]) || i + 1 >= __ldg(&F.offsets[lo + 1]))
        return;
    float2 A = __ldg(&F.pts[i]), B = __ldg(&F.pts[i + 1]);
    float vx = __fsub_rn(B.x, A.x), vy = __fsub_rn(B.y, A.y);
    float l2 = __fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy));
    if (!(l2 > 0.0f)) return;
    {
        // FP64 terms of this segment used by every pixel that picks it (same
        // expressions as a per-pixel evaluation, computed once)
        const double ax = A.x, ay = A.y;
        const double dvx = __dsub_rn((double)B.x, ax), dvy = __dsub_rn((double)B.y, ay);
        const double len = __dsqrt_rn(__dadd_rn(__dmul_rn(dvx, dvx), __dmul_rn(dvy, dvy)));
        double *s = F.seg64 + 8 * (size_t)i;
        s[0] = ax;
        s[1] = ay;
        s[2] = dvx;
        s[3] = dvy;
        s[4] = __ddiv_rn(1.0, __dmul_rn(len, len));
        s[5] = __ddiv_rn(dvx, len);
        s[6] = __ddiv_rn(dvy, len);
        s[7] = 1.0;  // the spline's weight, set by spline_weight_kernel when given
    }
    float grow = 3.0f * a.eta + 1.0f;
    float xmin = fminf(A.x, B.x) - grow, xmax = fmaxf(A.x, B.x) + grow;
    float ymin = fminf(A.y, B.y) - grow, ymax = fmaxf(A.y, B.y) + grow;
    int bx0 = max(0, (int)floorf(xmin / BIN)), bx1 = min(F.NBX - 1, (int)floorf(xmax / BIN));
    int by0 = max(0, (int)floorf(ymin / BIN)), by1 = min(F.NBY - 1, (int)floorf(ymax / BIN));
    for (int by = by0; by <= by1; by++)
        for (int bx = bx0; bx <= bx1; bx++) {
            int b = by * F.NBX + bx;
            int pos = atomicAdd(&F.bin_count[b], 1);
            if (pos < BIN_CAP) F.bin_list[(size_t)b * BIN_CAP + pos] = i;
        }
}

// Squared distance from p to the segment a + [0, 1] v with 1/|v|^2 given, in FP32
// with the oracle's expression (no contraction): t = ((p - a).v) * (1/|v|^2)
// clamped to [0, 1], |p - a - t v|^2.
__device__ __forceinline__ float seg_d2(float px, float py, float ax, float ay, float vx, float vy, float inv_l2)
{
    const float wx = __fsub_rn(px, ax), wy = __fsub_rn(py, ay);
    const float dot = __fadd_rn(__fmul_rn(wx, vx), __fmul_rn(wy, vy));
    float t = __fmul_rn(dot, inv_l2);
    if (t < 0.0f) t = 0.0f;
    if (t > 1.0f) t = 1.0f;
    const float qx = __fsub_rn(wx, __fmul_rn(t, vx));
    const float qy = __fsub_rn(wy, __fmul_rn(t, vy));
    return __fadd_rn(__fmul_rn(qx, qx), __fmul_rn(qy, qy));
}

// Hole bits of four labels: bit c is set iff byte c of w is 1 (a hole label).
__device__ __forceinline__ uint32_t hole4(uint32_t w)
{
    const uint32_t r = __vcmpeq4(w, 0x01010101u);  // 0xff in every byte equal to 1
    return ((r >> 7) & 1u) | ((r >> 14) & 2u) | ((r >> 21) & 4u) | ((r >> 28) & 8u);
}

struct BinSegs {
    float4 av[BIN_CAP];   // a.x, a.y, v.x, v.y
    float inv_l2[BIN_CAP];
    int id[BIN_CAP];      // global segment index (ties go to the lowest)
};

// Nearest segment of P hole pixels per thread (pixels q = tid + 256 j): the
// bin's segments form the outer loop, so each is read from shared memory once
// per thread.
template <int P>
__device__ __forceinline__ void nearest_in_bin(const BinSegs &sg, int nloc, const short *holes, int nh, int x0, int y0,
                                               float *best, int *bi)
{
    float px[P], py[P];
#pragma unroll
    for (int j = 0; j < P; j++) {
        const int q = threadIdx.x + 256 * j;
        const int e = q < nh ? holes[q] : 0;
        px[j] = (float)(x0 + (e & (BIN - 1)));
        py[j] = (float)(y0 + (e >> 5));
        best[j] = INFINITY;
        bi[j] = 0x7fffffff;
    }
    for (int s = 0; s < nloc; s++) {
        const float4 S = sg.av[s];
        const float il = sg.inv_l2[s];
        const int id = sg.id[s];
#pragma unroll
        for (int j = 0; j < P; j++) {
            const float d2 = seg_d2(px[j], py[j], S.x, S.y, S.z, S.w, il);
            if (d2 < best[j] || (d2 == best[j] && id < bi[j])) {
                best[j] = d2;
                bi[j] = id;
            }
        }
    }
}

// One CTA per 32x32-pixel bin.  Lanes 0-3 of each warp read one row of the bin's
// labels each (two 16-byte loads where the row is aligned and inside the frame)
// into a 32-bit hole mask; a bin without hole pixels ends there.  Otherwise the
// bin's segments are staged in shared memory with their reciprocal lengths, the
// hole pixels are compacted, and each thread takes the nearest segment of up to
// four of them.
__global__ void __launch_bounds__(256) guide_kernel(const __grid_constant__ GuideArgs a)
{
    __shared__ BinSegs sg;
    __shared__ short holes_s[BIN * BIN];
    __shared__ int wtot[8];
    const int gb = blockIdx.x;
    const int f = find_frame(a.bin_offset, a.n_frames, gb);
    const SplineFrameDev &F = a.frames[f];
    const int b = gb - __ldg(&a.bin_offset[f]);
    const int bx = b % F.NBX, by = b / F.NBX;
    const int x0 = bx * BIN, y0 = by * BIN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = warp * 4 + lane;  // the bin row of lanes 0-3
    uint32_t hm = 0u;
    if (lane < 4 && y0 + r < F.H) {
        const uint8_t *row = F.labels + (size_t)(y0 + r) * F.W + x0;
        if (x0 + BIN <= F.W && (reinterpret_cast<uintptr_t>(row) & 15u) == 0) {
            const uint4 q0 = __ldg(reinterpret_cast<const uint4 *>(row));
            const uint4 q1 = __ldg(reinterpret_cast<const uint4 *>(row) + 1);
            hm = hole4(q0.x) | (hole4(q0.y) << 4) | (hole4(q0.z) << 8) | (hole4(q0.w) << 12) | (hole4(q1.x) << 16) |
                 (hole4(q1.y) << 20) | (hole4(q1.z) << 24) | (hole4(q1.w) << 28);
        } else {
            for (int c = 0; c < BIN && x0 + c < F.W; c++)
                if (__ldg(&row[c]) == 1) hm |= 1u << c;
        }
    }
    if (!__syncthreads_or(hm != 0u)) return;  // CTA-uniform

    const int cnt = __ldcg(&F.bin_count[b]);
    const bool overflow = cnt > BIN_CAP;
    const int nloc = overflow ? 0 : cnt;
    for (int s = threadIdx.x; s < nloc; s += blockDim.x) {
        const int i = __ldcg(&F.bin_list[(size_t)b * BIN_CAP + s]);
        const float2 A = __ldg(&F.pts[i]), B = __ldg(&F.pts[i + 1]);
        const float vx = __fsub_rn(B.x, A.x), vy = __fsub_rn(B.y, A.y);
        const float l2 = __fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy));
        sg.av[s] = make_float4(A.x, A.y, vx, vy);
        sg.inv_l2[s] = __fdiv_rn(1.0f, l2);
        sg.id[s] = i;
    }
    // compact the hole pixels (row-major): row r's pixels follow rows 0..r-1
    const int c = __popc(hm);  // 0 on lanes >= 4
    int incl = c;
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 3) wtot[warp] = incl;
    __syncthreads();
    int base = 0, nh = 0;
#pragma unroll
    for (int w = 0; w < 8; w++) {
        const int v = wtot[w];
        if (w < warp) base += v;
        nh += v;
    }
    if (lane < 4) {
        int pos = base + incl - c;
        for (uint32_t m = hm; m; m &= m - 1u) holes_s[pos++] = (short)((r << 5) | (__ffs(m) - 1));
    }
    __syncthreads();

    float best[4];
    int bi[4];
    if (!overflow) {
        if (nh <= 256) nearest_in_bin<1>(sg, nloc, holes_s, nh, x0, y0, best, bi);
        else if (nh <= 512) nearest_in_bin<2>(sg, nloc, holes_s, nh, x0, y0, best, bi);
        else nearest_in_bin<4>(sg, nloc, holes_s, nh, x0, y0, best, bi);
    }
    const float t3 = 3.0f * a.eta;
    const float thr = __fmul_rn(t3, t3);
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int q = threadIdx.x + 256 * j;
        if (q >= nh) break;
        const int e = holes_s[q];
        const int x = x0 + (e & (BIN - 1)), y = y0 + (e >> 5);
        float bd = best[j];
        int bs = bi[j];
        if (overflow) {
            // the bin's list overflowed: every segment of the frame
            bd = INFINITY;
            bs = 0x7fffffff;
            const float px = (float)x, py = (float)y;
            for (int sp = 0; sp < F.n_splines; sp++) {
                const int i0 = max(0, __ldg(&F.offsets[sp])), i1 = min(F.n_points, __ldg(&F.offsets[sp + 1]));
                for (int i = i0; i + 1 < i1; i++) {
                    const float2 A = __ldg(&F.pts[i]), B = __ldg(&F.pts[i + 1]);
                    const float vx = __fsub_rn(B.x, A.x), vy = __fsub_rn(B.y, A.y);
                    const float l2 = __fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy));
                    if (!(l2 > 0.0f)) continue;
                    const float d2 = seg_d2(px, py, A.x, A.y, vx, vy, __fdiv_rn(1.0f, l2));
                    if (d2 < bd || (d2 == bd && i < bs)) {
                        bd = d2;
                        bs = i;
                    }
                }
            }
        }
        float2 out = make_float2(0.0f, 0.0f);
        if (bs != 0x7fffffff && bd <= thr) {
            // t = ((x - a).v) / |v|^2 clamped, d^2 = |x - a - t v|^2, g = (v/|v|) e^(-d^2/(2 eta^2)),
            // with the reciprocals 1/|v|^2 and 1/(2 eta^2) precomputed in FP64
            const double *s = F.seg64 + 8 * (size_t)bs;
            const double ax = __ldcg(&s[0]), ay = __ldcg(&s[1]), vx = __ldcg(&s[2]), vy = __ldcg(&s[3]);
            const double inv_l2 = __ldcg(&s[4]), tx = __ldcg(&s[5]), ty = __ldcg(&s[6]), sw = __ldcg(&s[7]);
            const double wx = __dsub_rn((double)x, ax), wy = __dsub_rn((double)y, ay);
            double t = __dmul_rn(__dadd_rn(__dmul_rn(wx, vx), __dmul_rn(wy, vy)), inv_l2);
            if (t < 0.0) t = 0.0;
            if (t > 1.0) t = 1.0;
            const double qx = __dsub_rn(wx, __dmul_rn(t, vx)), qy = __dsub_rn(wy, __dmul_rn(t, vy));
            const double d2 = __dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy));
            const double ev = exp(-__dmul_rn(d2, a.k2));
            out.x = (float)__dmul_rn(__dmul_rn(tx, ev), sw);
            out.y = (float)__dmul_rn(__dmul_rn(ty, ev), sw);
        }
        F.guide[(size_t)y * F.W + x] = out;
    }
}

// The weight of the spline holding each segment, for the frames of one chunk
// that have weights: one CTA per frame, after bin_kernel.
__global__ void __launch_bounds__(256) spline_weight_kernel(const __grid_constant__ GuideArgs a,
                                                            const __grid_constant__ WeightChunk c)
{
    const float *w = c.w[blockIdx.x];
    if (!w) return;
    const SplineFrameDev &F = a.frames[c.first + blockIdx.x];
    for (int i = threadIdx.x; i + 1 < F.n_points; i += blockDim.x) {
        int lo = 0, hi = F.n_splines;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(&F.offsets[mid]) <= i) lo = mid; else hi = mid;
        }
        if (F.n_splines <= 0 || i < __ldg(&F.offsets[0]) || i + 1 >= __ldg(&F.offsets[lo + 1])) continue;
        F.seg64[8 * (size_t)i + 7] = (double)__ldg(&w[lo]);
    }
}

// g = |g| (cos phi, sin phi) at hole pixels, evaluated in FP64 and rounded once
// (so a CPU evaluation in FP64 gives the same FP32 field).
__global__ void __launch_bounds__(256) angle_kernel(int64_t npx, const uint8_t *labels, const float *mag,
                                                    const float *phi, float2 *guide)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npx; p += (int64_t)gridDim.x * blockDim.x) {
        if (__ldg(&labels[p]) != 1) continue;
        double m = (double)__ldg(&mag[p]), a = (double)__ldg(&phi[p]);
        guide[p] = make_float2((float)__dmul_rn(m, cos(a)), (float)__dmul_rn(m, sin(a)));
    }
}

}  // namespace gf

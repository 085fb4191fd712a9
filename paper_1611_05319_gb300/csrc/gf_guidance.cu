// Guide field from splines (Guidefill, arxiv 1611.05319, Section 3.3) for sm_103a.
//
// g(x) = t_Gamma * exp(-d(x, Gamma)^2 / (2 eta^2)) for the nearest polyline
// segment Gamma when d <= 3 eta, else 0, at every hole pixel.
//
// Two kernels per request:
//   bin_kernel    one thread per polyline point: the segment starting there is
//                 appended to every 32x32-pixel bin its bounding box, grown by
//                 3 eta + 1 px, overlaps (so no segment within 3 eta of a pixel
//                 is missed, FP32 rounding included);
//   guide_kernel  one CTA per bin: the bin's segments are staged in shared
//                 memory, each hole pixel takes the nearest one.  A bin whose
//                 list overflowed scans all segments of its frame.
// The nearest-segment choice and the 3-eta cut use a fixed FP32 expression
// with no contraction (ties: lowest segment index), so the decision does not
// depend on the machine; the returned value is evaluated in FP64 for the
// chosen segment and rounded once to FP32.

#include "gf_internal.cuh"

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
        s[4] = __dmul_rn(len, len);
        s[5] = __ddiv_rn(dvx, len);
        s[6] = __ddiv_rn(dvy, len);
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

__device__ __forceinline__ float seg_d2(float px, float py, float ax, float ay, float bx, float by)
{
    float vx = __fsub_rn(bx, ax), vy = __fsub_rn(by, ay);
    float wx = __fsub_rn(px, ax), wy = __fsub_rn(py, ay);
    float l2 = __fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy));
    float dot = __fadd_rn(__fmul_rn(wx, vx), __fmul_rn(wy, vy));
    float t = __fdiv_rn(dot, l2);
    if (t < 0.0f) t = 0.0f;
    if (t > 1.0f) t = 1.0f;
    float qx = __fsub_rn(wx, __fmul_rn(t, vx));
    float qy = __fsub_rn(wy, __fmul_rn(t, vy));
    return __fadd_rn(__fmul_rn(qx, qx), __fmul_rn(qy, qy));
}

__global__ void __launch_bounds__(256) guide_kernel(const __grid_constant__ GuideArgs a)
{
    __shared__ float4 seg[BIN_CAP];
    __shared__ int segid[BIN_CAP];
    __shared__ short holes_s[BIN * BIN];
    __shared__ int nholes;
    const int gb = blockIdx.x;
    const int f = find_frame(a.bin_offset, a.n_frames, gb);
    const SplineFrameDev &F = a.frames[f];
    const int b = gb - __ldg(&a.bin_offset[f]);
    const int bx = b % F.NBX, by = b / F.NBX;
    if (threadIdx.x == 0) nholes = 0;
    const int cnt = __ldcg(&F.bin_count[b]);
    const bool overflow = cnt > BIN_CAP;
    const int nloc = overflow ? 0 : cnt;
    for (int s = threadIdx.x; s < nloc; s += blockDim.x) {
        int i = __ldcg(&F.bin_list[(size_t)b * BIN_CAP + s]);
        float2 A = __ldg(&F.pts[i]), B = __ldg(&F.pts[i + 1]);
        seg[s] = make_float4(A.x, A.y, B.x, B.y);
        segid[s] = i;
    }
    __syncthreads();
    // compact the bin's hole pixels so that the FP64 work below runs in full warps
    for (int e0 = 0; e0 < BIN * BIN; e0 += blockDim.x) {
        const int e = e0 + threadIdx.x;
        const int x = bx * BIN + (e & (BIN - 1)), y = by * BIN + (e >> 5);
        const bool h = x < F.W && y < F.H && __ldg(&F.labels[(size_t)y * F.W + x]) == 1;
        const unsigned m = __ballot_sync(0xffffffffu, h);
        int base = 0;
        if ((threadIdx.x & 31) == 0 && m) base = atomicAdd(&nholes, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (h) holes_s[base + __popc(m & ((1u << (threadIdx.x & 31)) - 1u))] = (short)e;
    }
    __syncthreads();
    const int nh = nholes;
    const float t3 = 3.0f * a.eta;
    const float thr = __fmul_rn(t3, t3);
    const double den = __dmul_rn(__dmul_rn(2.0, (double)a.eta), (double)a.eta);
    for (int q = threadIdx.x; q < nh; q += blockDim.x) {
        const int e = holes_s[q];
        const int x = bx * BIN + (e & (BIN - 1)), y = by * BIN + (e >> 5);
        const size_t p = (size_t)y * F.W + x;
        const float px = (float)x, py = (float)y;
        float best = INFINITY;
        int bi = 0x7fffffff;
        if (!overflow) {
            for (int s = 0; s < nloc; s++) {
                float4 S = seg[s];
                float d2 = seg_d2(px, py, S.x, S.y, S.z, S.w);
                int id = segid[s];
                if (d2 < best || (d2 == best && id < bi)) {
                    best = d2;
                    bi = id;
                }
            }
        } else {
            for (int sp = 0; sp < F.n_splines; sp++) {
                int i0 = max(0, __ldg(&F.offsets[sp])), i1 = min(F.n_points, __ldg(&F.offsets[sp + 1]));
                for (int i = i0; i + 1 < i1; i++) {
                    float2 A = __ldg(&F.pts[i]), B = __ldg(&F.pts[i + 1]);
                    float vx = __fsub_rn(B.x, A.x), vy = __fsub_rn(B.y, A.y);
                    if (!(__fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy)) > 0.0f)) continue;
                    float d2 = seg_d2(px, py, A.x, A.y, B.x, B.y);
                    if (d2 < best || (d2 == best && i < bi)) {
                        best = d2;
                        bi = i;
                    }
                }
            }
        }
        float2 out = make_float2(0.0f, 0.0f);
        if (bi != 0x7fffffff && best <= thr) {
            const double *s = F.seg64 + 8 * (size_t)bi;
            const double ax = __ldcg(&s[0]), ay = __ldcg(&s[1]), vx = __ldcg(&s[2]), vy = __ldcg(&s[3]);
            const double len2 = __ldcg(&s[4]), tx = __ldcg(&s[5]), ty = __ldcg(&s[6]);
            const double wx = __dsub_rn((double)x, ax), wy = __dsub_rn((double)y, ay);
            double t = __ddiv_rn(__dadd_rn(__dmul_rn(wx, vx), __dmul_rn(wy, vy)), len2);
            if (t < 0.0) t = 0.0;
            if (t > 1.0) t = 1.0;
            const double qx = __dsub_rn(wx, __dmul_rn(t, vx)), qy = __dsub_rn(wy, __dmul_rn(t, vy));
            const double d2 = __dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy));
            const double ev = exp(__ddiv_rn(-d2, den));
            out.x = (float)__dmul_rn(tx, ev);
            out.y = (float)__dmul_rn(ty, ev);
        }
        F.guide[p] = out;
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

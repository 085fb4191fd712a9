// Adjoint of the Guidefill fill (reverse sweep over the steps) for sm_103a.
//
// Differentiates the fill as a map of the known colours, the guidance angle
// field (|g| fixed) and mu, with the step of every pixel, the stall steps and
// every ghost sample's tap set held fixed (they are piecewise constant).  The
// forward's shell map reconstructs every D^(k) (readable at step k iff
// (uint)(s+1) < (uint)(k+1)), so no other forward state is stored.
//
// For a pixel x filled at step k with normalised weights wh_s over its
// readable samples and bilinear values v_s (Algorithm 1, eq. bilinearDef):
//   grad_in[t]  += wh_s * L_t * ubar(x)           for every tap t of sample s
//   grad_phi(x)  = ubar(x) . sum_s wh_s dv_s/dphi  (dp_s/dphi = n gh_perp - m gh)
//   grad_mu     += ubar(x) . sum_s wh_s (lam_s - lam_bar) v_s,
//                  lam_s = d ln w_s / d mu = -mu |g|^2 m^2 / eps^2  (eq. weight)
// Steps run K-1 .. 0; a pixel's ubar is final once every later step (the only
// readers of its value) has scattered into it.
//
// Kernels: adj_prep_kernel (per pixel: copy grad_out -> grad_in, clear
// grad_phi, histogram of shell indices, K), adj_scan_kernel (per frame: step
// offsets), adj_scatter_kernel (per pixel: pixel lists per step),
// adj_kernel (persistent: one cluster per frame, one cluster barrier per step).

#include <cooperative_groups.h>

#include "gf_internal.cuh"

namespace cg = cooperative_groups;

namespace gf {

constexpr unsigned AFULL = 0xffffffffu;

__device__ __forceinline__ int adj_find(const int32_t *off, int n, long long v)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if ((long long)__ldg(&off[mid]) <= v) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void adj_upload_kernel(const __grid_constant__ AdjChunk c)
{
    for (int i = threadIdx.x; i < c.count; i += blockDim.x) {
        c.dst_frames[c.first + i] = c.frames[i];
        c.dst_blk[c.first + i] = c.blk[i];
    }
    if (threadIdx.x == 0 && c.last_chunk) c.dst_blk[c.first + c.count] = c.blk[c.count];
}

// grid-stride over all pixels of all frames (pixel offsets in px_offset[n+1] as blocks of 1024)
__global__ void __launch_bounds__(256) adj_prep_kernel(const __grid_constant__ AdjArgs a)
{
    const long long total = (long long)__ldg(&a.blk_offset[a.n_frames]) * 1024;
    for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < total;
         gi += (long long)gridDim.x * blockDim.x) {
        int f = adj_find(a.blk_offset, a.n_frames, gi / 1024);
        const AdjFrameDev &F = a.frames[f];
        long long p = gi - (long long)__ldg(&a.blk_offset[f]) * 1024;
        long long np = (long long)F.H * F.W;
        if (p >= np) continue;
        if (F.grad_in != F.grad_out) F.grad_in[p] = __ldg(&F.grad_out[p]);
        F.grad_phi[p] = 0.0f;
        int s = __ldg(&F.shell[p]);
        if (s >= 0) {
            atomicAdd(&F.cnt[s], 1);
            atomicMax(F.K, s + 1);
        }
    }
}

// one CTA per frame: exclusive scan of cnt[0..K) into start[0..K], cursor = start
__global__ void __launch_bounds__(1024) adj_scan_kernel(const __grid_constant__ AdjArgs a)
{
    const AdjFrameDev &F = a.frames[blockIdx.x];
    const int K = __ldcg(F.K);
    __shared__ int carry;
    __shared__ int wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < K; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < K ? __ldcg(&F.cnt[i]) : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(AFULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            int s = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(AFULL, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        int excl = carry + (w > 0 ? wsum[w - 1] : 0) + x - v;
        if (i < K) {
            F.start[i] = excl;
            F.cnt[i] = excl;  // becomes the scatter cursor
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) F.start[K] = carry;
}

__global__ void __launch_bounds__(256) adj_scatter_kernel(const __grid_constant__ AdjArgs a)
{
    const long long total = (long long)__ldg(&a.blk_offset[a.n_frames]) * 1024;
    for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < total;
         gi += (long long)gridDim.x * blockDim.x) {
        int f = adj_find(a.blk_offset, a.n_frames, gi / 1024);
        const AdjFrameDev &F = a.frames[f];
        long long p = gi - (long long)__ldg(&a.blk_offset[f]) * 1024;
        if (p >= (long long)F.H * F.W) continue;
        int s = __ldg(&F.shell[p]);
        if (s >= 0) {
            int pos = atomicAdd(&F.cnt[s], 1);
            F.order[pos] = (int32_t)p;
        }
    }
}

__device__ __forceinline__ bool tap_readable(const AdjFrameDev &F, int x, int y, int k)
{
    if (x < 0 || y < 0 || x >= F.W || y >= F.H) return false;
    return readable_at(__ldg(&F.shell[(size_t)y * F.W + x]), k);
}

struct SampleGeo {
    int ix, iy;        // cell corner (absolute)
    float frx, fry;    // fractional offsets (0 along a single-tap axis)
    bool ok;
};

__device__ __forceinline__ SampleGeo sample_geo(const AdjArgs &a, const AdjFrameDev &F, int x, int y, float nf,
                                                float mf, float ch, float sh, bool rot, int k)
{
    float ox, oy;
    if (rot) {
        ox = __fsub_rn(__fmul_rn(nf, ch), __fmul_rn(mf, sh));
        oy = __fadd_rn(__fmul_rn(nf, sh), __fmul_rn(mf, ch));
        float r0 = rintf(ox);
        if (fabsf(__fsub_rn(ox, r0)) <= a.tau) ox = r0;
        r0 = rintf(oy);
        if (fabsf(__fsub_rn(oy, r0)) <= a.tau) oy = r0;
    } else {
        ox = nf;
        oy = mf;
    }
    const float flx = floorf(ox), fly = floorf(oy);
    SampleGeo g;
    g.frx = __fsub_rn(ox, flx);
    g.fry = __fsub_rn(oy, fly);
    g.ix = x + (int)flx;
    g.iy = y + (int)fly;
    bool ok = tap_readable(F, g.ix, g.iy, k);
    if (g.frx > 0.f) ok = ok && tap_readable(F, g.ix + 1, g.iy, k);
    if (g.fry > 0.f) {
        ok = ok && tap_readable(F, g.ix, g.iy + 1, k);
        if (g.frx > 0.f) ok = ok && tap_readable(F, g.ix + 1, g.iy + 1, k);
    }
    g.ok = ok;
    return g;
}

__device__ __forceinline__ float dot4(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }

__device__ __forceinline__ void red_add4(float4 *p, float4 v)
{
    atomicAdd(p, v);
}

// G lanes process pixel x of step k.
__device__ void adj_pixel(const AdjArgs &a, const AdjFrameDev &F, int p, int k, bool stall, bool act, int G,
                          int j, float &mu_acc)
{
    const int x = p % F.W, y = p / F.W;
    float4 ub = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 g = make_float2(0.f, 0.f);
    if (act) {
        ub = __ldcg(&F.grad_in[p]);
        if (!stall) g = __ldg(&F.guide[p]);
    }
    float ch = 1.f, sh = 0.f, beta = 0.f, a2 = 0.f;
    const bool rot = !stall;
    if (!stall) {
        a2 = __fadd_rn(__fmul_rn(g.x, g.x), __fmul_rn(g.y, g.y));
        float aa = __fsqrt_rn(a2);
        if (aa > 0.f) {
            ch = __fdiv_rn(g.x, aa);
            sh = __fdiv_rn(g.y, aa);
        }
        beta = a.coef32 * a2;
    }
    const bool has_dir = rot && __fsqrt_rn(a2) > 0.f;  // g = 0: unrotated ball, no angle dependence
    // pass 1: readable inverse distances per |m| group
    const int R = a.tab.R;
    float accg[MAX_R + 1];
#pragma unroll
    for (int gi = 0; gi <= MAX_R; gi++) accg[gi] = 0.f;
    if (act) {
#pragma unroll
        for (int gi = 0; gi <= MAX_R; gi++) {
            if (gi > R) break;
            for (int s = a.tab.m_start[gi] + j; s < a.tab.m_start[gi + 1]; s += G) {
                SampleGeo sg = sample_geo(a, F, x, y, a.tab.n_f[s], a.tab.m_f[s], ch, sh, rot, k);
                if (sg.ok) accg[gi] += a.tab.invd[s];
            }
        }
    }
#pragma unroll
    for (int gi = 0; gi <= MAX_R; gi++)
        for (int o = 1; o < G; o <<= 1) accg[gi] += __shfl_xor_sync(AFULL, accg[gi], o);
    int m0 = MAX_R + 1;
#pragma unroll
    for (int gi = MAX_R; gi >= 0; gi--)
        if (accg[gi] > 0.f) m0 = gi;
    float Wn = 0.f;
#pragma unroll
    for (int gi = 0; gi <= MAX_R; gi++)
        if (accg[gi] > 0.f) Wn += expf(-beta * (float)(gi * gi - m0 * m0)) * accg[gi];
    const float invW = Wn > 0.f ? 1.f / Wn : 0.f;
    // pass 2: scatter, angle and mu terms
    const float lam_scale = a.mu > 0.f ? -2.f * a.coef32 / a.mu * a2 : 0.f;  // lam_s = lam_scale * m^2
    float S1 = 0.f, S2 = 0.f, S3 = 0.f, S4 = 0.f;
    if (act && Wn > 0.f) {
        for (int gi = 0; gi <= R; gi++) {
            const float wg = expf(-beta * (float)(gi * gi - m0 * m0)) * invW;
            const float lam = lam_scale * (float)(gi * gi);
            for (int s = a.tab.m_start[gi] + j; s < a.tab.m_start[gi + 1]; s += G) {
                const float nf = a.tab.n_f[s], mf = a.tab.m_f[s];
                SampleGeo sg = sample_geo(a, F, x, y, nf, mf, ch, sh, rot, k);
                if (!sg.ok) continue;
                const float wh = wg * a.tab.invd[s];
                const size_t b = (size_t)sg.iy * F.W + sg.ix;
                const float fx = sg.frx, fy = sg.fry;
                const bool ax = fx > 0.f, ay = fy > 0.f;
                const float4 c00 = __ldg(&F.out[b]);
                const float4 c10 = ax ? __ldg(&F.out[b + 1]) : c00;
                const float4 c01 = ay ? __ldg(&F.out[b + F.W]) : c00;
                const float4 c11 = (ax && ay) ? __ldg(&F.out[b + F.W + 1]) : c00;
                const float wx0 = 1.f - fx, wx1 = fx, wy0 = 1.f - fy, wy1 = fy;
                // value v_s . ubar and its derivative along x and y
                const float d00 = dot4(c00, ub), d10 = dot4(c10, ub), d01 = dot4(c01, ub), d11 = dot4(c11, ub);
                float vu = wx0 * wy0 * d00;
                if (ax) vu += wx1 * wy0 * d10;
                if (ay) vu += wx0 * wy1 * d01;
                if (ax && ay) vu += wx1 * wy1 * d11;
                float gx_ = 0.f, gy_ = 0.f;
                if (ax) gx_ = wy0 * (d10 - d00) + (ay ? wy1 * (d11 - d01) : 0.f);
                if (ay) gy_ = wx0 * (d01 - d00) + (ax ? wx1 * (d11 - d10) : 0.f);
                if (has_dir) {
                    const float dpx = -nf * sh - mf * ch, dpy = nf * ch - mf * sh;
                    S4 += wh * (gx_ * dpx + gy_ * dpy);
                }
                S1 += wh * lam * vu;
                S2 += wh * lam;
                S3 += wh * vu;
                // scatter wh * L_t * ubar into the taps
                float l = wh * wx0 * wy0;
                red_add4(&F.grad_in[b], make_float4(l * ub.x, l * ub.y, l * ub.z, l * ub.w));
                if (ax) {
                    l = wh * wx1 * wy0;
                    red_add4(&F.grad_in[b + 1], make_float4(l * ub.x, l * ub.y, l * ub.z, l * ub.w));
                }
                if (ay) {
                    l = wh * wx0 * wy1;
                    red_add4(&F.grad_in[b + F.W], make_float4(l * ub.x, l * ub.y, l * ub.z, l * ub.w));
                    if (ax) {
                        l = wh * wx1 * wy1;
                        red_add4(&F.grad_in[b + F.W + 1], make_float4(l * ub.x, l * ub.y, l * ub.z, l * ub.w));
                    }
                }
            }
        }
    }
    for (int o = 1; o < G; o <<= 1) {
        S1 += __shfl_xor_sync(AFULL, S1, o);
        S2 += __shfl_xor_sync(AFULL, S2, o);
        S3 += __shfl_xor_sync(AFULL, S3, o);
        S4 += __shfl_xor_sync(AFULL, S4, o);
    }
    if (act && j == 0) {
        F.grad_phi[p] = has_dir ? S4 : 0.f;
        F.grad_in[p] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!stall) mu_acc += S1 - S2 * S3;
    }
}

__global__ void __launch_bounds__(CTA_THREADS, 1) adj_kernel(const __grid_constant__ AdjArgs a)
{
    __shared__ AdjFrameDev s_frame;
    cg::cluster_group cluster = cg::this_cluster();
    const int crank = (int)cluster.block_rank();
    const int csize = (int)cluster.num_blocks();
    const int cid = blockIdx.x / csize;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int gw = wid * csize + crank;
    const int nw = csize * WARPS_PER_CTA;
    int32_t *slot = a.cluster_frame + 2 * cid;
    for (int it = 0;; it++) {
        cluster.sync();
        if (crank == 0 && threadIdx.x == 0) slot[it & 1] = atomicAdd(a.frame_cursor, 1);
        cluster.sync();
        const int f = __ldcg(&slot[it & 1]);
        if (f >= a.n_frames) break;
        if (threadIdx.x == 0) s_frame = a.frames[f];
        __syncthreads();
        const AdjFrameDev &F = s_frame;
        const int K = __ldcg(F.K);
        float mu_acc = 0.f;
        for (int k = K - 1; k >= 0; k--) {
            const int b0 = __ldcg(&F.start[k]), b1 = __ldcg(&F.start[k + 1]);
            const int cnt = b1 - b0;
            const bool stall = F.stall ? ((__ldg(&F.stall[k >> 5]) >> (k & 31)) & 1u) != 0u : false;
            int G = 1;
            while (G < 8 && cnt * G * 2 <= 32 * nw) G <<= 1;
            const int per = 32 / G;
            const int j = lane & (G - 1), grp = lane / G;
            for (int base = gw * per; base < cnt; base += nw * per) {
                const int q = base + grp;
                const bool act = q < cnt;
                const int p = act ? __ldcg(&F.order[b0 + q]) : 0;
                adj_pixel(a, F, p, k, stall, act, G, j, mu_acc);
            }
            cluster.sync();
        }
        float wsum = mu_acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(AFULL, wsum, o);
        if (lane == 0 && wsum != 0.f) atomicAdd(&F.grad_mu[0], wsum);
        __syncthreads();
    }
}

}  // namespace gf

// Shell-by-shell transport fill (Guidefill, arxiv 1611.05319) for sm_103a.
//
// Kernels:
//   init_kernel   one pass over every frame: state word per pixel (out_shell),
//                 per 8x8 tile the bitmask of hole pixels (U) and of the initial
//                 active boundary (Qw = d_active D^(0)_h, Notation) from bit
//                 operations on the labels, per-frame hole count.
//   order_kernel  sorts frames by hole size (largest first) into the work queue
//                 (a split schedule gives its first frames to a second launch
//                 with larger clusters, running beside the first).
//   fill_kernel   persistent; one thread-block cluster runs one frame's whole
//                 shell loop (Algorithm 1) at a time, with one hardware cluster
//                 barrier per step, then takes the next frame from the queue.
//
// Front tracking.  Per step k the cluster processes a work list of tiles.  A
// tile is on the list of step k+1 iff a pixel was filled at step k within
// reach (ceil(eps)+1 pixels) of it; the tiles are claimed with atomicMax on a
// per-tile step word while list slots are reserved with one warp-aggregated
// atomicAdd (a warp-ballot stream compaction); lost claims leave skip markers.  Inside a tile only pixels within reach of a step-k fill
// are candidates: the only pixels whose ready test can change (new front
// pixels are 8-neighbours of fills, and a waiting pixel's test depends only on
// pixels of its ball).  Candidates get the exact active-boundary test from the
// state words, so the front sets equal a full rescan (Algorithm 1, last line).
// With GF_FLAG_RESCAN every step instead re-tests every unfilled pixel of the
// frame ("Guidefill without tracking", Section 3.6).
//
// State word s per pixel: -1 known, -2 unfilled hole, -3 bystander, k filled at
// step k.  Readable at step k (Omega_h \ (D^(k)_h u B_h), Section 2.1) iff
// (uint)(s+1) < (uint)(k+1).  Step-k fills write k, which no step-k test
// treats as readable, so fills are written in place (Algorithm 1 evaluates
// every front pixel against D^(k)).
//
// Mutable global data is read with plain (weak) loads.  Every value a step reads
// was written before the cluster barrier that began the step (whose wait has
// acquire semantics at cluster scope, so the loads observe those writes), or is
// being written during the step by another warp, in which case the old and the
// new value lead to the same decision: a state word becoming k is unreadable at
// step k like the -2 it replaces, and a neighbour's unfilled mask only filters
// claims.

#include <cooperative_groups.h>

#include "gf_internal.cuh"

namespace cg = cooperative_groups;

namespace gf {

constexpr unsigned FULL = 0xffffffffu;

// A plain load (weak, may be served by L1); see the note on mutable data above.
template <class T>
__device__ __forceinline__ T ld(const T *p)
{
    return *p;
}

// The sample table of the fill kernel in shared memory: (n, m, 1/|(n, m)|, |m|)
// in grouped order, padded to a multiple of 32 (one 16-byte load per sample; the
// lanes of a pixel read different entries, which the constant cache would
// serialise).
__shared__ float4 g_stab[MAX_SAMPLES];
// The same samples as mirror pairs {(n, m), (-n, -m)}: one entry per pair,
// (n, m, 1/|(n, m)|, |m| as int bits) with m < 0, or m = 0 and n < 0.
__shared__ float4 g_pair[MAX_SAMPLES / 2];

// ---------------------------------------------------------------------------
// init
// ---------------------------------------------------------------------------
// One warp per strip of 8 pixel rows x 32 tiles (256 columns); lane l owns tile
// column 32 s + l, i.e. 8 pixel columns, and holds the known and hole bits of its
// columns (plus one column each side) for the strip's rows and the row above and
// below.  The active boundary of D^(0)_h (hole pixels with a known 8-neighbour)
// is then a few bit operations per row, the state words are written as two
// 16-byte stores per row and lane, and each lane writes its tile's masks.
// INIT_WARPS strips per CTA.

__device__ __forceinline__ void init_label_row(const uint8_t *labels, int W, int H, int y, int x0, bool vec8,
                                               uint32_t &kn, uint32_t &ho)
{
    // labels of columns x0 .. x0+7 of row y (0xff outside the image) -> known and hole bits
    uint2 v = make_uint2(0xffffffffu, 0xffffffffu);
    if (y >= 0 && y < H && x0 < W) {
        const uint8_t *row = labels + (size_t)y * W;
        if (vec8) {
            v = __ldg(reinterpret_cast<const uint2 *>(row + x0));
        } else {
            uint32_t b[8];
#pragma unroll
            for (int c = 0; c < 8; c++) b[c] = (x0 + c < W) ? (uint32_t)__ldg(row + x0 + c) : 0xffu;
            v.x = b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
            v.y = b[4] | (b[5] << 8) | (b[6] << 16) | (b[7] << 24);
        }
    }
    // four labels at a time: __vseteq4 sets bit 8i of a word where byte i matches, and
    // the multiply gathers bits 0, 8, 16, 24 into bits 21..24 (the partial products
    // 2^(8i + 7j) are distinct, so nothing carries)
    auto bits4 = [](uint32_t x) { return ((x * 0x00204081u) >> 21) & 0xfu; };
    kn = bits4(__vseteq4(v.x, 0u)) | (bits4(__vseteq4(v.y, 0u)) << 4);
    ho = bits4(__vseteq4(v.x, 0x01010101u)) | (bits4(__vseteq4(v.y, 0x01010101u)) << 4);
}

__global__ void __launch_bounds__(32 * INIT_WARPS, 5) init_kernel(const __grid_constant__ InitArgs a)
{
    const int b = blockIdx.x;
    // frame f with cta_offset[f] <= b < cta_offset[f+1] (a division when every frame
    // takes the same number of CTAs)
    int lo = 0, first = 0;
    if (a.uniform_ctas > 0) {
        lo = b / a.uniform_ctas;
        first = lo * a.uniform_ctas;
    } else {
        int hi = a.n_frames;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (__ldg(&a.cta_offset[mid]) <= b) lo = mid; else hi = mid;
        }
        first = __ldg(&a.cta_offset[lo]);
    }
    const FrameDev &F = a.frames[lo];
    const int H = F.H, W = F.W, TW = F.TW, TH = F.TH;
    const int strips = (TW + 31) >> 5;
    const int unit = (b - first) * INIT_WARPS + (threadIdx.x >> 5);
    if (unit >= TH * strips) return;  // warp-uniform
    const int lane = threadIdx.x & 31;
    const int ty = unit / strips, sx = unit - ty * strips;
    const int tx = sx * 32 + lane;
    const bool tile_ok = tx < TW;
    const int x0 = tx * TILE, y0 = ty * TILE;
    const bool vec8 = (W & 7) == 0 && (reinterpret_cast<uintptr_t>(F.labels) & 7u) == 0;
    const bool vec16 = (W & 7) == 0 && (reinterpret_cast<uintptr_t>(F.shell) & 15u) == 0 &&
                       (!F.enter || (reinterpret_cast<uintptr_t>(F.enter) & 15u) == 0);

    // rows y0-1 .. y0+8: bit 0 = column x0-1, bits 1..8 = x0 .. x0+7, bit 9 = x0+8
    uint32_t kn[TILE + 2], ho[TILE + 2];
#pragma unroll
    for (int r = 0; r < TILE + 2; r++) {
        const int y = y0 - 1 + r;
        uint32_t k8 = 0, h8 = 0;
        if (tile_ok) init_label_row(F.labels, W, H, y, x0, vec8, k8, h8);
        // the neighbouring columns: from the adjacent lanes, or from memory at the strip's ends
        uint32_t kl = (__shfl_up_sync(FULL, k8, 1) >> 7) & 1u;
        uint32_t kr = __shfl_down_sync(FULL, k8, 1) & 1u;
        const bool rowin = y >= 0 && y < H;
        if (lane == 0) kl = (rowin && x0 > 0 && x0 - 1 < W) ? (uint32_t)(__ldg(&F.labels[(size_t)y * W + x0 - 1]) == 0) : 0u;
        if (lane == 31) kr = (rowin && x0 + 8 < W) ? (uint32_t)(__ldg(&F.labels[(size_t)y * W + x0 + 8]) == 0) : 0u;
        kn[r] = kl | (k8 << 1) | (kr << 9);
        ho[r] = h8 << 1;
    }
    // tile masks and state words of rows y0 .. y0+7
    unsigned long long U = 0ull, Q = 0ull;
#pragma unroll
    for (int r = 1; r <= TILE; r++) {
        uint32_t nb = kn[r - 1] | kn[r + 1];
        nb |= (nb << 1) | (nb >> 1) | (kn[r] << 1) | (kn[r] >> 1);
        const uint32_t f = ho[r] & nb;
        const uint32_t urow = (ho[r] >> 1) & 0xffu, qrow = (f >> 1) & 0xffu;
        U |= (unsigned long long)urow << (8 * (r - 1));
        Q |= (unsigned long long)qrow << (8 * (r - 1));
        const int y = y0 + r - 1;
        if (!tile_ok || y >= H) continue;
        // state word: -1 known, -2 hole, -3 anything else (bystander); outside the
        // image nothing is written
        const uint32_t known = (kn[r] >> 1) & 0xffu;
        int32_t sw[8], en[8];
#pragma unroll
        for (int c = 0; c < 8; c++) {
            // known and hole exclude each other
            static_assert(SH_KNOWN == SH_BYST + 2 && SH_UNFILLED == SH_BYST + 1, "state word values");
            sw[c] = SH_BYST + 2 * (int32_t)((known >> c) & 1u) + (int32_t)((urow >> c) & 1u);
            en[c] = ((qrow >> c) & 1u) ? 0 : -1;
        }
        const size_t o = (size_t)y * W + x0;
        if (vec16) {
            reinterpret_cast<int4 *>(F.shell + o)[0] = make_int4(sw[0], sw[1], sw[2], sw[3]);
            reinterpret_cast<int4 *>(F.shell + o)[1] = make_int4(sw[4], sw[5], sw[6], sw[7]);
            if (F.enter) {
                reinterpret_cast<int4 *>(F.enter + o)[0] = make_int4(en[0], en[1], en[2], en[3]);
                reinterpret_cast<int4 *>(F.enter + o)[1] = make_int4(en[4], en[5], en[6], en[7]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 8; c++) {
                if (x0 + c < W) {
                    F.shell[o + c] = sw[c];
                    if (F.enter) F.enter[o + c] = en[c];
                }
            }
        }
    }
    int gcount = 0;  // data term: hole pixels of this tile with g != 0
    if ((a.flags & GF_FLAG_DATA) && tile_ok) {
        for (unsigned long long m = U; m; m &= m - 1ull) {
            const int pix = __ffsll((long long)m) - 1;
            const float2 gv = __ldg(&F.guide[(size_t)(y0 + (pix >> 3)) * W + x0 + (pix & 7)]);
            gcount += (gv.x != 0.0f || gv.y != 0.0f) ? 1 : 0;
        }
    }
    const int t = ty * TW + tx;
    if (tile_ok) {
        F.U[t] = U;
        F.Qw[t] = Q;
        F.sched[t] = -1;
        // both fill records whole (mask 0, tag INT32_MIN): 16-byte stores leave no
        // partially written L2 sector to be read back from DRAM
        reinterpret_cast<int4 *>(&F.F[t])[0] = make_int4(0, 0, INT32_MIN, 0);
        reinterpret_cast<int4 *>(&F.F[F.ntiles + t])[0] = make_int4(0, 0, INT32_MIN, 0);
    }
    const int holes = __reduce_add_sync(FULL, __popcll(U));
    const int nq = __reduce_add_sync(FULL, __popcll(Q));
    gcount = __reduce_add_sync(FULL, gcount);
    // step-0 work list: warp-aggregated append of the tiles on the initial front
    const bool has_front = Q != 0ull;
    const unsigned bm = __ballot_sync(FULL, has_front);
    int b0 = 0;
    if (lane == 0) {
        if (holes) atomicAdd(F.holes, holes);
        if (gcount) atomicAdd(F.gleft, gcount);
        if (bm) {
            b0 = atomicAdd(&F.init_count[0], __popc(bm));
            atomicAdd(&F.init_count[1], nq);
        }
    }
    b0 = __shfl_sync(FULL, b0, 0);
    if (has_front) F.init_list[b0 + __popc(bm & ((1u << lane) - 1u))] = t;
}

__global__ void upload_frames_kernel(const __grid_constant__ FrameChunk c)
{
    for (int i = threadIdx.x; i < c.count; i += blockDim.x) {
        c.dst_frames[c.first + i] = c.frames[i];
        c.dst_cta[c.first + i] = c.cta[i];
    }
    if (threadIdx.x == 0 && c.last_chunk) c.dst_cta[c.first + c.count] = c.cta[c.count];
}

// Frames in decreasing hole size (ties: index), one thread per frame.
__global__ void order_kernel(const FrameDev *frames, int n, int32_t *order, int32_t *cursor)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int hi = ld(frames[i].holes);
        int rank = 0;
        for (int j = 0; j < n; j++) {
            int hj = ld(frames[j].holes);
            if (hj > hi || (hj == hi && j < i)) rank++;
        }
        order[rank] = i;
    }
    if (blockIdx.x == 0 && threadIdx.x < 2) cursor[threadIdx.x] = 0;
}

// ---------------------------------------------------------------------------
// fill
// ---------------------------------------------------------------------------
// NORMAL: a work-list tile, candidates near the last step's fills.  RESCAN:
// every unfilled pixel each step (no tracking).  STALL: the stall rule over the
// waiting front.  REVAL: every unfilled pixel once with eq. ready (the step at
// which the data term of eq. ready2 is switched off), with claims.
enum Mode { NORMAL = 0, RESCAN = 1, STALL = 2, REVAL = 3 };

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Pixels of the centre tile within Chebyshev distance `reach` of a set bit of
// the 3x3 neighbourhood masks; lane l < 9 holds the mask of neighbour
// (dx, dy) = (l%3 - 1, l/3 - 1).  reach <= 8.
__device__ __forceinline__ unsigned long long dilate_nbr(unsigned long long fm, int reach)
{
    const int lane = threadIdx.x & 31;
    const int gy = lane - 8;  // row in [-8, 16) of the 3-tile column
    const int tr = gy < 0 ? 0 : (gy < 8 ? 1 : 2);
    const int ry = (lane < 24) ? gy - (tr - 1) * 8 : 0;
    unsigned long long mL = __shfl_sync(FULL, fm, tr * 3 + 0);
    unsigned long long mC = __shfl_sync(FULL, fm, tr * 3 + 1);
    unsigned long long mR = __shfl_sync(FULL, fm, tr * 3 + 2);
    uint32_t row = 0;
    if (lane < 24)
        row = (uint32_t)((mL >> (8 * ry)) & 0xffu) | ((uint32_t)((mC >> (8 * ry)) & 0xffu) << 8) |
              ((uint32_t)((mR >> (8 * ry)) & 0xffu) << 16);
    // dilation by doubling: after a pass of step st <= c + 1 a set bit covers the
    // offsets 0 .. c + st (rows: shfl_up/down return the lane's own value at the
    // warp's ends, and lanes 24..31 hold no row)
    uint32_t h = row;
    for (int c = 0; c < reach;) {
        const int st = min(c + 1, reach - c);
        h |= (h << st) | (h >> st);
        c += st;
    }
    uint32_t v = (lane < 24) ? ((h >> 8) & 0xffu) : 0u;
    for (int c = 0; c < reach;) {
        const int st = min(c + 1, reach - c);
        v |= __shfl_up_sync(FULL, v, st) | __shfl_down_sync(FULL, v, st);
        c += st;
    }
    unsigned long long out = 0;
#pragma unroll
    for (int y = 0; y < 8; y++) out |= (unsigned long long)(__shfl_sync(FULL, v, 8 + y) & 0xffu) << (8 * y);
    return out;
}

// FP64 confidence of tile pixel `pix` in the canonical sample order with the
// oracle's expressions (eqs. weight, confidence); used only inside the FP32
// guard band.  The whole warp works on one pixel: every lane evaluates the
// weights of its share of the samples (FP64 runs at a small fraction of the
// FP32 rate on this part, so the exp/divide work is spread over 32 lanes),
// then the weights are added in the canonical order exactly as the oracle
// adds them.  Must be called by all 32 lanes.
template <int RW>
__device__ bool warp_ready_fp64(const FillParams &p, const WarpSmem<RW> *ws, int pix, bool ghost)
{
    constexpr int NSLOT = RW == 4 ? 1 : (RW == 5 ? 2 : 5);  // ceil(samples / 32) for ceil(eps) = 3, 4, 7
    const int lane = threadIdx.x & 31;
    const int px = pix & 7, py = pix >> 3;
    const float gx = ws->guide[pix].x, gy = ws->guide[pix].y;
    float ch = 1.0f, sh = 0.0f;
    if (ghost) {
        const float a2f = __fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy));
        const float a = __fsqrt_rn(a2f);
        if (a > 0.0f) {
            ch = __fdiv_rn(gx, a);
            sh = __fdiv_rn(gy, a);
        }
    }
    const double a2 = __dadd_rn(__dmul_rn((double)gx, (double)gx), __dmul_rn((double)gy, (double)gy));
    double w[NSLOT];
    int ok[NSLOT];
#pragma unroll
    for (int q = 0; q < NSLOT; q++) {
        const int s = q * 32 + lane;
        w[q] = 0.0;
        ok[q] = 0;
        if (s < p.tab.ns) {
            const int n = p.tab.cn[s], m = p.tab.cm[s];
            float ox, oy;
            if (ghost) {
                const float fn = (float)n, fm = (float)m;
                ox = __fsub_rn(__fmul_rn(fn, ch), __fmul_rn(fm, sh));
                oy = __fadd_rn(__fmul_rn(fn, sh), __fmul_rn(fm, ch));
                float r = rintf(ox);
                if (fabsf(__fsub_rn(ox, r)) <= p.tau) ox = r;
                r = rintf(oy);
                if (fabsf(__fsub_rn(oy, r)) <= p.tau) oy = r;
            } else {
                ox = (float)n;
                oy = (float)m;
            }
            const float flx = floorf(ox), fly = floorf(oy);
            const float frx = __fsub_rn(ox, flx), fry = __fsub_rn(oy, fly);
            const int ix = px + RW + (int)flx, iy = py + RW + (int)fly;
            const uint32_t need = frx > 0.0f ? 3u : 1u;
            bool rd = ((ws->rowmask[iy] >> ix) & need) == need;
            if (fry > 0.0f) rd = rd && (((ws->rowmask[iy + 1] >> ix) & need) == need);
            double t;
            if (ghost) {
                t = __dmul_rn(__dmul_rn(p.coef64, a2), (double)(m * m));
            } else {
                const double proj = __dadd_rn(__dmul_rn(-(double)gy, (double)n), __dmul_rn((double)gx, (double)m));
                t = __dmul_rn(__dmul_rn(p.coef64, proj), proj);
            }
            w[q] = __ddiv_rn(exp(-t), __dsqrt_rn((double)(n * n + m * m)));
            ok[q] = rd ? 1 : 0;
        }
    }
    double S_all = 0.0, S_rd = 0.0;
#pragma unroll
    for (int q = 0; q < NSLOT; q++) {
        for (int src = 0; src < 32; src++) {
            const double wv = __shfl_sync(FULL, w[q], src);
            const int okv = __shfl_sync(FULL, ok[q], src);
            if (q * 32 + src < p.tab.ns) {
                S_all = __dadd_rn(S_all, wv);
                if (okv) S_rd = __dadd_rn(S_rd, wv);
            }
        }
    }
    return __ddiv_rn(S_rd, S_all) > p.c64;
}

// The three work lists of a cluster (the list of step s in slot s % 3): the
// first DS_LIST entries of each in the shared memory of the cluster's first CTA
// (read and written by every CTA through distributed shared memory, a round trip
// within the GPC), the rest in global memory.
constexpr int DS_LIST = 2048;
struct Lists {
    int32_t *ds;    // [3][DS_LIST] in the first CTA's shared memory
    int32_t *glob;  // [3][list_cap]; entries from DS_LIST on
    int cap;        // list_cap
};
__device__ __forceinline__ void list_put(const Lists &L, int slot, int pos, int32_t v)
{
    if (pos < DS_LIST) L.ds[slot * DS_LIST + pos] = v;
    else L.glob[(size_t)slot * L.cap + pos] = v;
}
__device__ __forceinline__ int32_t list_get(const Lists &L, int slot, int pos)
{
    return pos < DS_LIST ? ld(&L.ds[slot * DS_LIST + pos]) : ld(&L.glob[(size_t)slot * L.cap + pos]);
}

struct WarpCounters {
    int filled, delta, evals, err, rechecks;
};

// Neighbour-tile claims of step k (tiles for the work list of step k+1).  A claim
// is an atomicMax of k+1 on the tile's step word; the claim that raises it wins.
// Two ways to turn claims into list entries:
//  * combined: list slots for every claim are reserved together with the claims
//    (one round trip); a lost claim leaves a skip marker (-1) in its slot;
//  * deferred: the warp reserves slots only for the claims it won, once their
//    atomics have returned (at its next tile), and writes the entries one tile
//    later, so the list holds no skip markers.  Used when a step's list is longer
//    than the cluster's warp count, where markers would be walked one by one.
// The struct carries the claims of a warp's last tiles between those points.
struct PendingClaims {
    unsigned m1;  // claims made, slots not yet reserved (warp-uniform lane mask)
    unsigned m2;  // slots reserved, entries not yet written (warp-uniform lane mask)
    int nt1, old1;  // per lane: claimed tile, previous step word
    int nt2, old2;  // per lane: entry tile; old2 >= k+1 turns it into a skip marker
    int base2;      // lane 0: first reserved slot
    int k;          // step of the pending claims
};

// Writes the reserved entries (their slot reservation has returned).
__device__ __forceinline__ void claims_write(const FillParams &p, const Lists &lists, PendingClaims &pc, WarpCounters &wc)
{
    if (pc.m2) {  // warp-uniform
        const int lane = threadIdx.x & 31;
        const int base = __shfl_sync(FULL, pc.base2, 0);
        if ((pc.m2 >> lane) & 1u) {
            const int pos = base + __popc(pc.m2 & ((1u << lane) - 1u));
            if (pos < p.list_cap) list_put(lists, (pc.k + 1) % 3, pos, pc.old2 < pc.k + 1 ? pc.nt2 : -1);
            else wc.err = 1;
        }
        pc.m2 = 0u;
    }
}

// Reserves slots for the won claims among the deferred ones (their claims have
// returned).  Stage 2 must be empty.
__device__ __forceinline__ void claims_reserve(GroupCtl *ctl, PendingClaims &pc)
{
    if (pc.m1) {  // warp-uniform
        const int lane = threadIdx.x & 31;
        const bool won = ((pc.m1 >> lane) & 1u) && pc.old1 < pc.k + 1;
        const unsigned wb = __ballot_sync(FULL, won);
        if (wb) {
            if (lane == 0) pc.base2 = atomicAdd(&ctl->list_count[(pc.k + 1) % 3], __popc(wb));
            pc.nt2 = pc.nt1;
            pc.old2 = INT32_MIN;
            pc.m2 = wb;
        }
        pc.m1 = 0u;
    }
}

// Everything pending is written (before the step's counter flush).
__device__ __forceinline__ void claims_drain(const FillParams &p, GroupCtl *ctl, const Lists &lists, PendingClaims &pc,
                                             WarpCounters &wc)
{
    claims_write(p, lists, pc, wc);
    claims_reserve(ctl, pc);
    claims_write(p, lists, pc, wc);
}

// Processes one tile at step k (one warp): candidates, exact front test, ready
// test and fill in one pass over each front pixel's samples, tile masks, claims
// of the neighbour tiles for step k+1.
template <int RW, int MODE>
__device__ void process_tile(const FillParams &p, const FrameDev &F, WarpSmem<RW> *ws, GroupCtl *ctl,
                             const Lists &lists, int t, int k, unsigned long long cand_in, WarpCounters &wc,
                             PendingClaims &pc, bool defer, bool phase1)
{
    constexpr int WS = WarpSmem<RW>::WS;
    const int lane = threadIdx.x & 31;
    const int W = F.W, H = F.H;
    // the previous tile's shared-memory reads and window copies are complete
    cp_async_wait_all();
    __syncwarp();
    const int tx = t % F.TW, ty = t / F.TW;
    const int x0 = tx * TILE, y0 = ty * TILE;
    const int R = p.tab.R;
    const bool ghost = (p.flags & GF_FLAG_GHOST) != 0;
    const bool smart = (p.flags & GF_FLAG_SMART) != 0;

    // Issue every load that depends only on the tile before using any of them:
    // tile masks, the neighbours' step-(k-1) fills and hole masks, the state
    // window, the guide vectors and (speculatively) the colour window.
    const unsigned long long U = ld(&F.U[t]);
    const unsigned long long Qold = ld(&F.Qw[t]);
    int ftag = INT32_MIN;
    unsigned long long fmsk = 0ull, unb = 0ull;
    const int ndx = lane % 3 - 1, ndy = lane / 3 - 1;
    const int nxt_x = tx + ndx, nxt_y = ty + ndy;
    const bool nvalid = lane < 9 && nxt_x >= 0 && nxt_y >= 0 && nxt_x < F.TW && nxt_y < F.TH;
    const int nt = nxt_y * F.TW + nxt_x;
    if (MODE != RESCAN && nvalid) {
        unb = ld(&F.U[nt]);
        if (MODE == NORMAL && k > 0) {
            const TileF *e = &F.F[(size_t)((k - 1) & 1) * F.ntiles + nt];
            ftag = ld(&e->tag);
            fmsk = ld(&e->mask);
        }
    }
    const int wx0 = x0 - RW, wy0 = y0 - RW;
    // State window.  With WS = 16 a lane holds 4 columns of 2 rows (lane = 4 row +
    // column group): one 16-byte load each when the row width is a multiple of 4 and
    // the state array is aligned (4 columns are then wholly inside or wholly outside
    // the frame), else 4 plain loads.  Other widths: one column per lane and row.
    constexpr bool Q4 = WS == 16;
    int32_t sv[Q4 ? 1 : WS];
    int4 sq[2];
    if (Q4) {
        const bool vec = (W & 3) == 0 && ((uintptr_t)F.shell & 15u) == 0;
#pragma unroll
        for (int i = 0; i < 2; i++) {
            const int gx = wx0 + 4 * (lane & 3), gy = wy0 + (lane >> 2) + 8 * i;
            const bool rin = gy >= 0 && gy < H;
            if (vec) {
                sq[i] = (rin && gx >= 0 && gx < W) ? ld(reinterpret_cast<const int4 *>(&F.shell[(size_t)gy * W + gx]))
                                                   : make_int4(SH_OUTSIDE, SH_OUTSIDE, SH_OUTSIDE, SH_OUTSIDE);
            } else {
                int e[4];
#pragma unroll
                for (int b = 0; b < 4; b++)
                    e[b] = (rin && gx + b >= 0 && gx + b < W) ? ld(&F.shell[(size_t)gy * W + gx + b]) : SH_OUTSIDE;
                sq[i] = make_int4(e[0], e[1], e[2], e[3]);
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < (Q4 ? 1 : WS); r++) {
            int gx = wx0 + lane, gy = wy0 + r;
            sv[r] = (lane < WS && gx >= 0 && gy >= 0 && gx < W && gy < H) ? ld(&F.shell[(size_t)gy * W + gx])
                                                                           : SH_OUTSIDE;
        }
    }
    float2 gv[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    if (MODE != STALL) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int pix = lane + 32 * h;
            const int gx = x0 + (pix & 7), gy = y0 + (pix >> 3);
            if (gx < W && gy < H) gv[h] = __ldg(&F.guide[(size_t)gy * W + gx]);
        }
    }
    if (WS == 16) {
        // lane = 16 (row parity) + column; the column test is the same for every row
        const int c = lane & 15, r0 = lane >> 4;
        const bool cin = (unsigned)(wx0 + c) < (unsigned)W;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int gy = wy0 + r0 + 2 * i;
            if (cin && (unsigned)gy < (unsigned)H)
                cp_async16(&ws->col[(r0 + 2 * i) * 16 + c], &F.rgba[(size_t)gy * W + wx0 + c]);
        }
    } else {
        for (int e = lane; e < WS * WS; e += 32) {
            int r = e / WS, c = e - r * WS;
            int gx = wx0 + c, gy = wy0 + r;
            if (gx >= 0 && gy >= 0 && gx < W && gy < H) cp_async16(&ws->col[e], &F.rgba[(size_t)gy * W + gx]);
        }
    }

    unsigned long long cand;
    if (MODE == NORMAL) {
        if (k > 0) {
            const unsigned long long fm = (ftag == k - 1) ? fmsk : 0ull;
            cand = U & dilate_nbr(fm, R + 1);
        } else {
            cand = U;
        }
    } else {
        cand = cand_in & U;
    }
    if (cand == 0) return;

    // ---- readable bits of the window by ballot; guide vectors of the candidates
    if (Q4) {
        // each lane's 4 readable bits at column 4 (lane & 3), OR-ed over the 4 lanes of a row
#pragma unroll
        for (int i = 0; i < 2; i++) {
            uint32_t v = (readable_at(sq[i].x, k) ? 1u : 0u) | (readable_at(sq[i].y, k) ? 2u : 0u) |
                         (readable_at(sq[i].z, k) ? 4u : 0u) | (readable_at(sq[i].w, k) ? 8u : 0u);
            v <<= 4 * (lane & 3);
            v |= __shfl_xor_sync(FULL, v, 1);
            v |= __shfl_xor_sync(FULL, v, 2);
            if ((lane & 3) == 0) ws->rowmask[(lane >> 2) + 8 * i] = v;
        }
    } else {
#pragma unroll
        for (int r = 0; r < (Q4 ? 1 : WS); r++) {
            unsigned b = __ballot_sync(FULL, readable_at(sv[r], k));
            if (lane == 0) ws->rowmask[r] = b;
        }
    }
    if (MODE != STALL) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int pix = lane + 32 * h;
            if ((cand >> pix) & 1ull) ws->guide[pix] = gv[h];
        }
    }
    if (lane == 0) {
        ws->ready = 0ull;
        ws->recheck = 0ull;
    }
    __syncwarp();

    // ---- exact active-boundary test of the candidates
    unsigned long long P;
    {
        bool f[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            int pix = lane + 32 * h;
            int px = pix & 7, py = pix >> 3;
            bool c = (cand >> pix) & 1ull;
            int wc_ = px + RW - 1, wr = py + RW;
            uint32_t nb = ((ws->rowmask[wr - 1] >> wc_) & 7u) | ((ws->rowmask[wr] >> wc_) & 5u) |
                          ((ws->rowmask[wr + 1] >> wc_) & 7u);
            f[h] = c && nb != 0u;
        }
        P = (unsigned long long)__ballot_sync(FULL, f[0]) | ((unsigned long long)__ballot_sync(FULL, f[1]) << 32);
        if (F.enter) {
            unsigned long long nf = P & ~Qold;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                int pix = lane + 32 * h;
                if ((nf >> pix) & 1ull)
                    F.enter[(size_t)(y0 + (pix >> 3)) * W + x0 + (pix & 7)] = k;
            }
        }
    }
    const int np = __popcll(P);
    wc.evals += np;
    // the front pixels in increasing order: pixel q of a pass is plist[q]
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int pix = lane + 32 * h;
        if ((P >> pix) & 1ull) ws->plist[__popcll(P & ((1ull << pix) - 1ull))] = (uint8_t)pix;
    }

    // ---- ready test (eqs. weight, confidence, ready) and the fill value in one
    //      pass over the samples, G lanes per front pixel.  Each lane keeps its
    //      colour sum relative to the smallest weight exponent it has read (the
    //      normalisation cancels in the average and keeps e^-t from underflowing);
    //      the G partial sums are brought to the group's smallest exponent when
    //      they are combined.
    if (np) {
        cp_async_wait_all();
        __syncwarp();
        const int G = np <= 4 ? 8 : (np <= 8 ? 4 : (np <= 16 ? 2 : 1));
        const int per = 32 / G;
        const int j = lane & (G - 1), grp = lane / G;
        const int ns = p.tab.ns;
        const int npair = ns >> 1;
        const bool rot = ghost && MODE != STALL;
        const bool iso = ghost || MODE == STALL;  // the exponent depends on |m| only
        const bool fast = MODE == STALL || (ghost && smart && p.c >= 1e-30f);
        for (int base = 0; base < np; base += per) {
            const int q = base + grp;
            const bool act = q < np;
            const int pix = act ? ws->plist[q] : 0;
            const int px = pix & 7, py = pix >> 3;
            float2 g = make_float2(0.f, 0.f);
            if (act && MODE != STALL) g = ws->guide[pix];
            float ch = 1.0f, sh = 0.0f, beta = 0.0f;
            if (MODE != STALL) {
                float a2 = __fadd_rn(__fmul_rn(g.x, g.x), __fmul_rn(g.y, g.y));
                if (ghost) {
                    float a = __fsqrt_rn(a2);
                    if (a > 0.0f) {
                        ch = __fdiv_rn(g.x, a);
                        sh = __fdiv_rn(g.y, a);
                    }
                    beta = p.coef32 * a2;
                }
            }
            float S_rd = 0.f, S_all = 0.f, tmin = INFINITY, wsum = 0.f;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            int cnt = 0;
            if (fast) {
                // group weights e^(-beta g^2), g = |m| = 0..R, shared by the pixel's G lanes
                __syncwarp();
                if (act)
                    for (int gg = j; gg <= R; gg += G) ws->eg[grp][gg] = expf(-(beta * (float)(gg * gg)));
                __syncwarp();
            }
            if (act && fast) {
                // Rotated ball under smart order, or the stall pass: the weights need no
                // normalisation (a ready pixel has S_rd > c S_all >= c times the m = 0
                // weights; stall weights are 1/|(n, m)|).  Branch-free, over mirror pairs
                // {(n, m), (-n, -m)}: negation is exact and commutes with every rounding of
                // the rotation and of the snap, so the second offset is the exact negative
                // of the first; the pair shares its rotation, snap, floor and weights, and
                // each tap of the second sample is the first's tap reflected through the
                // pixel, with the same bilinear weight.  Taps of zero weight and the taps of
                // unreadable samples are read from the window's zero entry (an unreadable
                // pixel's colour may be anything, and 0 * NaN is NaN).
                constexpr int ZI = WS * WS;
                const float *eg = ws->eg[grp];
                const int cx = px + RW, cy = py + RW;
#pragma unroll 1
                for (int q2 = j; q2 < npair; q2 += G) {
                    const float4 te = g_pair[q2];  // n, m, 1/|(n, m)|, |m|
                    const float nf = te.x, mf = te.y;
                    float ox, oy;
                    if (rot) {
                        ox = __fsub_rn(__fmul_rn(nf, ch), __fmul_rn(mf, sh));
                        oy = __fadd_rn(__fmul_rn(nf, sh), __fmul_rn(mf, ch));
                        float r0 = rintf(ox);
                        if (fabsf(__fsub_rn(ox, r0)) <= p.tau) ox = r0;
                        r0 = rintf(oy);
                        if (fabsf(__fsub_rn(oy, r0)) <= p.tau) oy = r0;
                    } else {
                        ox = nf;
                        oy = mf;
                    }
                    const float flx = floorf(ox), fly = floorf(oy);
                    const float frx = __fsub_rn(ox, flx), fry = __fsub_rn(oy, fly);
                    const int fx = (int)flx, fy = (int)fly;
                    const bool hx = frx > 0.0f, hy = fry > 0.0f;
                    const uint32_t need = hx ? 3u : 1u;
                    // first sample: columns ix (+1), rows iy (+1); second: columns jx (+1)
                    // and rows jy (-1), the reflections of the first's
                    const int ix = cx + fx, iy = cy + fy;
                    const int jx = cx - fx - (hx ? 1 : 0), jy = cy - fy;
                    const uint32_t a0m = ws->rowmask[iy], a1m = ws->rowmask[iy + 1];
                    const uint32_t b0m = ws->rowmask[jy], b1m = ws->rowmask[jy - 1];
                    const bool ok1 = (((a0m >> ix) & need) == need) && (!hy || (((a1m >> ix) & need) == need));
                    const bool ok2 = (((b0m >> jx) & need) == need) && (!hy || (((b1m >> jx) & need) == need));
                    const float w0 = eg[__float_as_int(te.w)] * te.z;
                    S_all += w0;
                    S_all += w0;
                    S_rd += ok1 ? w0 : 0.f;
                    S_rd += ok2 ? w0 : 0.f;
                    cnt += (ok1 ? 1 : 0) + (ok2 ? 1 : 0);
                    const float gx = 1.f - frx, gy = 1.f - fry;
                    const float l00 = w0 * (gx * gy), l10 = w0 * (frx * gy);
                    const float l01 = w0 * (gx * fry), l11 = w0 * (frx * fry);
                    const int A0 = iy * WS + ix, B0 = jy * WS + cx - fx;
                    const float4 a0 = ws->col[ok1 ? A0 : ZI];
                    const float4 a1 = ws->col[ok1 && hx ? A0 + 1 : ZI];
                    const float4 a2 = ws->col[ok1 && hy ? A0 + WS : ZI];
                    const float4 a3 = ws->col[ok1 && hx && hy ? A0 + WS + 1 : ZI];
                    const float4 b0 = ws->col[ok2 ? B0 : ZI];
                    const float4 b1 = ws->col[ok2 && hx ? B0 - 1 : ZI];
                    const float4 b2 = ws->col[ok2 && hy ? B0 - WS : ZI];
                    const float4 b3 = ws->col[ok2 && hx && hy ? B0 - WS - 1 : ZI];
                    acc.x = __fmaf_rn(l00, a0.x, acc.x); acc.y = __fmaf_rn(l00, a0.y, acc.y);
                    acc.z = __fmaf_rn(l00, a0.z, acc.z); acc.w = __fmaf_rn(l00, a0.w, acc.w);
                    acc.x = __fmaf_rn(l10, a1.x, acc.x); acc.y = __fmaf_rn(l10, a1.y, acc.y);
                    acc.z = __fmaf_rn(l10, a1.z, acc.z); acc.w = __fmaf_rn(l10, a1.w, acc.w);
                    acc.x = __fmaf_rn(l01, a2.x, acc.x); acc.y = __fmaf_rn(l01, a2.y, acc.y);
                    acc.z = __fmaf_rn(l01, a2.z, acc.z); acc.w = __fmaf_rn(l01, a2.w, acc.w);
                    acc.x = __fmaf_rn(l11, a3.x, acc.x); acc.y = __fmaf_rn(l11, a3.y, acc.y);
                    acc.z = __fmaf_rn(l11, a3.z, acc.z); acc.w = __fmaf_rn(l11, a3.w, acc.w);
                    acc.x = __fmaf_rn(l00, b0.x, acc.x); acc.y = __fmaf_rn(l00, b0.y, acc.y);
                    acc.z = __fmaf_rn(l00, b0.z, acc.z); acc.w = __fmaf_rn(l00, b0.w, acc.w);
                    acc.x = __fmaf_rn(l10, b1.x, acc.x); acc.y = __fmaf_rn(l10, b1.y, acc.y);
                    acc.z = __fmaf_rn(l10, b1.z, acc.z); acc.w = __fmaf_rn(l10, b1.w, acc.w);
                    acc.x = __fmaf_rn(l01, b2.x, acc.x); acc.y = __fmaf_rn(l01, b2.y, acc.y);
                    acc.z = __fmaf_rn(l01, b2.z, acc.z); acc.w = __fmaf_rn(l01, b2.w, acc.w);
                    acc.x = __fmaf_rn(l11, b3.x, acc.x); acc.y = __fmaf_rn(l11, b3.y, acc.y);
                    acc.z = __fmaf_rn(l11, b3.z, acc.z); acc.w = __fmaf_rn(l11, b3.w, acc.w);
                }
            } else if (act) {
#pragma unroll 2
                for (int s = j; s < ns; s += G) {
                    const float4 te = g_stab[s];
                    const float nf = te.x, mf = te.y, invd = te.z;
                    float ox, oy;
                    if (rot) {
                        ox = __fsub_rn(__fmul_rn(nf, ch), __fmul_rn(mf, sh));
                        oy = __fadd_rn(__fmul_rn(nf, sh), __fmul_rn(mf, ch));
                        float r0 = rintf(ox);
                        if (fabsf(__fsub_rn(ox, r0)) <= p.tau) ox = r0;
                        r0 = rintf(oy);
                        if (fabsf(__fsub_rn(oy, r0)) <= p.tau) oy = r0;
                    } else {
                        ox = nf;
                        oy = mf;
                    }
                    const float flx = floorf(ox), fly = floorf(oy);
                    const float frx = __fsub_rn(ox, flx), fry = __fsub_rn(oy, fly);
                    const int ix = px + RW + (int)flx, iy = py + RW + (int)fly;
                    const uint32_t need = frx > 0.0f ? 3u : 1u;
                    bool ok = ((ws->rowmask[iy] >> ix) & need) == need;
                    if (fry > 0.0f) ok = ok && (((ws->rowmask[iy + 1] >> ix) & need) == need);
                    float tt;
                    if (iso) {
                        tt = beta * (mf * mf);
                    } else {
                        const float proj = -g.y * nf + g.x * mf;  // lattice ball: g_perp . (n, m)
                        tt = p.coef32 * proj * proj;
                    }
                    const float w0 = expf(-tt) * invd;
                    S_all += w0;
                    if (ok) {
                        S_rd += w0;
                        cnt++;
                        if (tt < tmin) {
                            const float sc = expf(tt - tmin);  // 0 for the first readable sample
                            acc.x *= sc; acc.y *= sc; acc.z *= sc; acc.w *= sc;
                            wsum *= sc;
                            tmin = tt;
                        }
                        const float w = expf(tmin - tt) * invd;
                        const float4 *cb = &ws->col[iy * WS + ix];
                        const float4 v = cb[0];
                        const float l00 = (1.f - frx) * (1.f - fry);
                        float4 val = make_float4(l00 * v.x, l00 * v.y, l00 * v.z, l00 * v.w);
                        if (frx > 0.f) {
                            const float l = frx * (1.f - fry);
                            const float4 c1 = cb[1];
                            val.x += l * c1.x; val.y += l * c1.y; val.z += l * c1.z; val.w += l * c1.w;
                        }
                        if (fry > 0.f) {
                            const float l = (1.f - frx) * fry;
                            const float4 c2 = cb[WS];
                            val.x += l * c2.x; val.y += l * c2.y; val.z += l * c2.z; val.w += l * c2.w;
                            if (frx > 0.f) {
                                const float l3 = frx * fry;
                                const float4 c3 = cb[WS + 1];
                                val.x += l3 * c3.x; val.y += l3 * c3.y; val.z += l3 * c3.z; val.w += l3 * c3.w;
                            }
                        }
                        acc.x += w * val.x; acc.y += w * val.y; acc.z += w * val.z; acc.w += w * val.w;
                        wsum += w;
                    }
                }
            }
            // combine the G lanes of a pixel
            if (!fast) {
                float tg = tmin;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1)
                    if (o < G) tg = fminf(tg, __shfl_xor_sync(FULL, tg, o));
                const float sc = (tmin == INFINITY) ? 0.f : expf(tg - tmin);
                acc.x *= sc; acc.y *= sc; acc.z *= sc; acc.w *= sc;
                wsum *= sc;
            } else {
                wsum = S_rd;
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                if (o < G) {
                    S_rd += __shfl_xor_sync(FULL, S_rd, o);
                    S_all += __shfl_xor_sync(FULL, S_all, o);
                    cnt += __shfl_xor_sync(FULL, cnt, o);
                    acc.x += __shfl_xor_sync(FULL, acc.x, o);
                    acc.y += __shfl_xor_sync(FULL, acc.y, o);
                    acc.z += __shfl_xor_sync(FULL, acc.z, o);
                    acc.w += __shfl_xor_sync(FULL, acc.w, o);
                    wsum += __shfl_xor_sync(FULL, wsum, o);
                }
            }
            // Smart order: decided in FP32 outside a guard band around c, re-checked in
            // FP64 inside it.  Band: relative 1e-4 for the rotated ball, where the FP32
            // error of both sums is below ~1e-5 relative (the m = 0 terms are exact and
            // the error of each other term is bounded by t e^-t <= 1/e times a few ulp);
            // 1e-3 for the lattice ball, whose projection g_perp.(n, m) can cancel.
            bool ready = cnt > 0;
            bool recheck = false;
            if (MODE != STALL && smart) {
                const float d = S_rd - p.c * S_all;
                const float tol = (ghost ? 1e-4f : 1e-3f) * p.c * S_all;
                ready = d > tol;
                recheck = !(d > tol) && !(d < -tol);
            }
            if (phase1 && g.x == 0.0f && g.y == 0.0f) {
                // eq. ready2, first phase: the data term D(x) = |g(x)| must exceed c2 = 0
                ready = false;
                recheck = false;
            }
            if (act && j == 0 && cnt > 0 && (ready || recheck)) {
                atomicOr(recheck ? &ws->recheck : &ws->ready, 1ull << pix);
                const float inv = 1.0f / wsum;
                ws->colr[pix] = make_float4(acc.x * inv, acc.y * inv, acc.z * inv, acc.w * inv);
            }
        }
    }
    __syncwarp();
    // FP64 re-checks, one pixel at a time with the whole warp
    for (unsigned long long rc = ws->recheck; rc; rc &= rc - 1ull) {
        const int pix = __ffsll((long long)rc) - 1;
        const bool r64 = warp_ready_fp64<RW>(p, ws, pix, ghost);
        if (lane == 0 && r64) atomicOr(&ws->ready, 1ull << pix);
        wc.rechecks++;
    }
    __syncwarp();
    const unsigned long long Rm = ws->ready;
    const int nr = __popcll(Rm);
    if (phase1) {
        // guided pixels filled: the data term stays on while any is left
        bool gz[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int pix = lane + 32 * h;
            gz[h] = ((Rm >> pix) & 1ull) && (ws->guide[pix].x != 0.0f || ws->guide[pix].y != 0.0f);
        }
        const int ng = __popc(__ballot_sync(FULL, gz[0])) + __popc(__ballot_sync(FULL, gz[1]));
        if (lane == 0 && ng) atomicSub(F.gleft, ng);
    }

    // ---- the fills (state word k: not readable by any other test of step k)
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int pix = lane + 32 * h;
        if ((Rm >> pix) & 1ull) {
            const size_t o = (size_t)(y0 + (pix >> 3)) * W + x0 + (pix & 7);
            F.rgba[o] = ws->colr[pix];
            F.shell[o] = k;
        }
    }

    // ---- tile bookkeeping
    const unsigned long long Qnew = (Qold & ~cand) | (P & ~Rm);
    if (lane == 0) {
        if (Rm) {
            F.U[t] = U & ~Rm;
            TileF *e = &F.F[(size_t)(k & 1) * F.ntiles + t];
            e->mask = Rm;
            e->tag = k;
        }
        if (Qnew != Qold) F.Qw[t] = Qnew;
    }
    wc.filled += nr;
    wc.delta += __popcll(Qnew) - __popcll(Qold);

    // the previous tiles' claims and reservations have returned by now
    claims_write(p, lists, pc, wc);
    claims_reserve(ctl, pc);

    // ---- tiles for step k+1: the neighbours within reach of this step's fills
    //      that still hold unfilled pixels.  The list slots are reserved with one
    //      atomicAdd while the claims (atomicMax on the tile's step word) are in
    //      flight; a claim lost to another tile leaves a skip marker (-1).
    if (MODE != RESCAN && Rm) {
        const int reach = R + 1;
        // columns holding a fill: OR of the 8 row bytes; rows holding one: bit 8y of
        // the byte-wise OR, gathered into bit y by the multiply
        unsigned long long cb = Rm | (Rm >> 32);
        cb |= cb >> 16;
        cb |= cb >> 8;
        const uint32_t colocc = (uint32_t)(cb & 0xffu);
        unsigned long long rb = Rm | (Rm >> 4);
        rb |= rb >> 2;
        rb |= rb >> 1;
        const uint32_t rowocc = (uint32_t)(((rb & 0x0101010101010101ull) * 0x0102040810204080ull) >> 56);
        const uint32_t lowm = reach >= 8 ? 0xffu : ((1u << reach) - 1u);
        const bool nL = (colocc & lowm) != 0, nR = (colocc >> (8 - (reach >= 8 ? 8 : reach))) != 0;
        const bool nU = (rowocc & lowm) != 0, nD = (rowocc >> (8 - (reach >= 8 ? 8 : reach))) != 0;
        const unsigned long long left = (lane == 4) ? (U & ~Rm) : unb;
        const bool need = nvalid && (ndx == 0 || (ndx < 0 ? nL : nR)) && (ndy == 0 || (ndy < 0 ? nU : nD)) &&
                          left != 0ull;
        const unsigned bm = __ballot_sync(FULL, need);
        if (bm) {
            pc.k = k;
            if (defer) {
                pc.m1 = bm;
                pc.nt1 = nt;
                if (need) pc.old1 = atomicMax(&F.sched[nt], k + 1);
            } else {
                pc.m2 = bm;
                pc.nt2 = nt;
                if (lane == 0) pc.base2 = atomicAdd(&ctl->list_count[(k + 1) % 3], __popc(bm));
                if (need) pc.old2 = atomicMax(&F.sched[nt], k + 1);
            }
        }
    }
}

// Adds a warp's counters of step k to slot k%3.  With `clear_next`, lane 0 of
// the first warp of each CTA also clears the slot of step k+1 and the work-list
// count of step k+2: their last readers passed the barrier of step k-1 and
// their next writers start after the barrier of step k.
__device__ __forceinline__ void flush_counters(GroupCtl *ctl, const WarpCounters &wc, int k, bool stall,
                                               bool clear_next)
{
    const int lane = threadIdx.x & 31;
    const int s = k % 3;
    int f = wc.filled, d = wc.delta, e = wc.evals, er = wc.err, rc = wc.rechecks;
    // all lanes hold identical values except err (per lane)
    er = __reduce_or_sync(FULL, er);
    if (lane == 0) {
        if (f) atomicAdd(&ctl->filled[s], f);
        if (d) atomicAdd(&ctl->front_delta[s], d);
        if (e && !stall) atomicAdd(&ctl->evals[s], e);  // Sigma_k |front_k| counts the evaluation pass only
        if (er) atomicOr(&ctl->err[s], er);
        if (rc) atomicAdd(&ctl->rechecks, rc);
        if (clear_next) {
            const int s1 = (k + 1) % 3;
            ctl->cursor[s1] = 0;
            ctl->filled[s1] = 0;
            ctl->front_delta[s1] = 0;
            ctl->evals[s1] = 0;
            ctl->err[s1] = 0;
            ctl->list_count[(k + 2) % 3] = 0;
        }
    }
}

// Every warp of the cluster visits the frame's tiles (32 at a time); the mode
// selects the tile mask that makes a tile a member (U: rescan, re-evaluation;
// Qw: stall) and is passed on as the tile's candidates.
template <int RW, int MODE>
__device__ void sweep_tiles(const FillParams &p, const FrameDev &F, WarpSmem<RW> *ws, GroupCtl *ctl,
                            const Lists &lists, int k, int gw, int nw, WarpCounters &wc, PendingClaims &pc,
                            bool phase1 = false)
{
    const int lane = threadIdx.x & 31;
    for (int base = gw * 32; base < F.ntiles; base += nw * 32) {
        int t = base + lane;
        unsigned long long m = 0;
        if (t < F.ntiles) m = (MODE == RESCAN || MODE == REVAL) ? ld(&F.U[t]) : ld(&F.Qw[t]);
        unsigned bal = __ballot_sync(FULL, m != 0ull);
        while (bal) {
            int i = __ffs(bal) - 1;
            bal &= bal - 1;
            unsigned long long mi = __shfl_sync(FULL, m, i);
            process_tile<RW, MODE>(p, F, ws, ctl, lists, base + i, k, mi, wc, pc, false, phase1);
        }
    }
}

template <int RW>
__global__ void __launch_bounds__(fill_warps(RW) * 32, 1) fill_kernel(const __grid_constant__ FillParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ FrameDev s_frame;
    WarpSmem<RW> *ws = reinterpret_cast<WarpSmem<RW> *>(smem_raw) + (threadIdx.x >> 5);
    cg::cluster_group cluster = cg::this_cluster();
    const int crank = (int)cluster.block_rank();
    const int csize = (int)cluster.num_blocks();
    const int cid = blockIdx.x / csize;
    // the cluster's control block and the heads of its work lists live in the first
    // CTA's shared memory
    __shared__ GroupCtl s_ctl;
    __shared__ int32_t s_lists[3 * DS_LIST];
    GroupCtl *ctl = cluster.map_shared_rank(&s_ctl, 0);
    Lists lists;
    lists.ds = cluster.map_shared_rank(s_lists, 0);
    lists.glob = p.lists + (size_t)cid * 3 * p.list_cap;
    lists.cap = p.list_cap;
    const int gw = (threadIdx.x >> 5) * csize + crank;  // interleave CTAs
    const int nw = csize * fill_warps(RW);
    const bool leader = crank == 0 && threadIdx.x == 0;
    const bool rescan = (p.flags & GF_FLAG_RESCAN) != 0;
    for (int i = threadIdx.x; i < p.tab.nsp; i += blockDim.x) {
        g_stab[i] = make_float4(p.tab.n_f[i], p.tab.m_f[i], p.tab.invd[i], fabsf(p.tab.m_f[i]));
        // group |m| = g lists m = -g before m = +g (n ascending within each), and
        // n < 0 before n > 0 for g = 0: the first half of every group holds one
        // sample of each mirror pair, and every group before it has an even count
        if (i < p.tab.ns) {
            const int g = (int)fabsf(p.tab.m_f[i]);
            const int g0 = p.tab.m_start[g], half = (p.tab.m_start[g + 1] - g0) >> 1;
            if (i - g0 < half)
                g_pair[(g0 >> 1) + (i - g0)] =
                    make_float4(p.tab.n_f[i], p.tab.m_f[i], p.tab.invd[i], __int_as_float(g));
        }
    }
    if ((threadIdx.x & 31) == 0) ws->col[WarpSmem<RW>::WS * WarpSmem<RW>::WS] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();

    for (int it = 0;; it++) {
        cluster.sync();  // everyone is done with the previous frame's counters
        if (leader) {
            int f = atomicAdd(p.frame_cursor, 1);
            ctl->cur_frame[it & 1] = f;
            for (int i = 0; i < 3; i++) {
                ctl->list_count[i] = 0;
                ctl->cursor[i] = 0;
                ctl->filled[i] = 0;
                ctl->front_delta[i] = 0;
                ctl->evals[i] = 0;
                ctl->err[i] = 0;
            }
            ctl->rechecks = 0;
        }
        cluster.sync();
        const int f = ld(&ctl->cur_frame[it & 1]);
        if (f >= p.n_frames) break;
        if (threadIdx.x == 0) s_frame = p.frames[p.frame_order[p.order_first + f]];
        __syncthreads();
        const FrameDev &F = s_frame;

        long long n_front = ld(&F.init_count[1]);
        long long filled_tot = 0, evals_tot = 0, max_front = 0;
        int stalls = 0, status = GF_OK;
        int k = 0;
        const int max_shells = F.max_shells;
        // the length and the first item of the current step's work list are loaded
        // ahead, together with the previous step's counters
        int n_cur = ld(&F.init_count[0]);
        int t0_cur = gw < n_cur ? ld(&F.init_list[gw]) : -1;
        // eq. ready2 (GF_FLAG_DATA): phase 1 while hole pixels with g != 0 remain and
        // some front pixel is ready under the data term; `reval`: this step tests every
        // front pixel with eq. ready (the tracked front was built under phase 1)
        bool phase1 = (p.flags & GF_FLAG_DATA) != 0;
        int data_switch = -1;
        bool reval = false;
        if (phase1 && ld(F.gleft) == 0) {
            phase1 = false;
            data_switch = 0;
        }
        for (;;) {
            const int slot = k % 3;
            WarpCounters wc = {0, 0, 0, 0, 0};
            PendingClaims pc;
            pc.m1 = 0u;
            pc.m2 = 0u;
            if (rescan) {
                sweep_tiles<RW, RESCAN>(p, F, ws, ctl, lists, k, gw, nw, wc, pc, phase1);
            } else if (reval) {
                sweep_tiles<RW, REVAL>(p, F, ws, ctl, lists, k, gw, nw, wc, pc);
            } else {
                // step 0 takes the init kernel's list, later steps the lists built by the claims
                const int n = n_cur;

                // Item gw goes to warp gw; items beyond the warp count are handed out
                // by a per-step cursor (the next grab is in flight while a tile is
                // processed), so uneven tiles do not leave warps idle at the barrier.
                // Negative items are claims lost to another tile.
                const bool lane0 = (threadIdx.x & 31) == 0;
                const bool more = n > nw;
                int pre = 0;
                if (lane0 && more) pre = atomicAdd(&ctl->cursor[slot], 1);
                const int t0 = gw < n ? t0_cur : -1;
                if (t0 >= 0) process_tile<RW, NORMAL>(p, F, ws, ctl, lists, t0, k, 0ull, wc, pc, more, phase1);
                if (more) {
                    int nxt = nw + __shfl_sync(FULL, pre, 0);
                    while (nxt < n) {
                        const int t = k == 0 ? ld(&F.init_list[nxt]) : list_get(lists, slot, nxt);
                        if (lane0) pre = atomicAdd(&ctl->cursor[slot], 1);
                        if (t >= 0) process_tile<RW, NORMAL>(p, F, ws, ctl, lists, t, k, 0ull, wc, pc, more, phase1);
                        nxt = nw + __shfl_sync(FULL, pre, 0);
                    }
                }
            }
            claims_drain(p, ctl, lists, pc, wc);
            flush_counters(ctl, wc, k, false, threadIdx.x < 32);
            cluster.sync();
            // one round trip: this step's counters and the next step's list
            const int s3n = (k + 1) % 3;
            int filled = ld(&ctl->filled[slot]);
            int dlt = ld(&ctl->front_delta[slot]);
            const int ev = ld(&ctl->evals[slot]);
            const int er = ld(&ctl->err[slot]);
            int n_next = ld(&ctl->list_count[s3n]);
            int t0_next = gw < p.list_cap ? list_get(lists, s3n, gw) : -1;  // used only if gw < n_next
            const int gleft = phase1 ? ld(F.gleft) : -1;
            evals_tot += ev;
            if (er) {
                status = GF_ERR_INTERNAL;
                break;
            }
            long long front_k = n_front + dlt + filled;
            if (front_k > max_front) max_front = front_k;
            reval = false;
            if (phase1 && filled == 0) {
                // eq. ready2 fills nothing at this step: eq. ready from this step on,
                // and this step is evaluated again with it (every front pixel)
                phase1 = false;
                data_switch = k;
                WarpCounters wr = {0, 0, 0, 0, 0};
                sweep_tiles<RW, REVAL>(p, F, ws, ctl, lists, k, gw, nw, wr, pc);
                claims_drain(p, ctl, lists, pc, wr);
                flush_counters(ctl, wr, k, true, false);
                cluster.sync();
                filled = ld(&ctl->filled[slot]);
                dlt = ld(&ctl->front_delta[slot]);
                const int er1 = ld(&ctl->err[slot]);
                n_next = ld(&ctl->list_count[s3n]);
                t0_next = gw < p.list_cap ? list_get(lists, s3n, gw) : -1;
                if (er1) {
                    status = GF_ERR_INTERNAL;
                    break;
                }
                front_k = n_front + dlt + filled;
                if (front_k > max_front) max_front = front_k;
            } else if (phase1 && gleft == 0) {
                // every pixel with g != 0 is filled: eq. ready from the next step on
                phase1 = false;
                data_switch = k + 1;
                reval = true;
            }
            int fk = filled;
            if (filled == 0) {
                if (n_front + dlt == 0) break;  // Algorithm 1: D^(k) exhausted (or the rest unreachable)
                // stall rule: no front pixel is ready; fill the front isotropically.  The
                // stall pass adds to the same slot (its counters were zero after the
                // evaluation pass, except the front delta).
                WarpCounters ws2 = {0, 0, 0, 0, 0};
                sweep_tiles<RW, STALL>(p, F, ws, ctl, lists, k, gw, nw, ws2, pc);
                claims_drain(p, ctl, lists, pc, ws2);
                flush_counters(ctl, ws2, k, true, false);
                cluster.sync();
                const int sf = ld(&ctl->filled[slot]);
                const int dlt2 = ld(&ctl->front_delta[slot]);
                const int er2 = ld(&ctl->err[slot]);
                // the stall fills appended claims to the next step's list
                n_next = ld(&ctl->list_count[s3n]);
                t0_next = gw < p.list_cap ? list_get(lists, s3n, gw) : -1;
                if (er2) {
                    status = GF_ERR_INTERNAL;
                    break;
                }
                if (sf == 0) break;  // front pixels with no readable sample at all
                n_front += dlt2;
                stalls++;
                fk = sf;
                if (leader && F.stall_bits) atomicOr(&F.stall_bits[k >> 5], 1u << (k & 31));
            } else {
                n_front += dlt;
            }
            filled_tot += fk;
            n_cur = n_next;
            t0_cur = t0_next;
            k++;
            if (k >= max_shells) {
                status = GF_ERR_NO_PROGRESS;
                break;
            }
        }
        if (leader) {
            const int holes = ld(F.holes);
            gf_stats st;
            st.shells = k;
            st.stalls = stalls;
            st.filled = filled_tot;
            st.evaluations = evals_tot;
            st.max_front = max_front;
            st.holes = holes;
            st.rechecks = ld(&ctl->rechecks);
            st.data_switch = data_switch;
            st.reserved = 0;
            if (status == GF_OK && filled_tot < holes) status = GF_INCOMPLETE;
            st.status = status;
            *F.stats = st;
        }
        __syncthreads();
    }
    cp_async_wait_all();  // window copies of a last tile that had no candidates
    // no CTA leaves while another may still read its shared memory (the control
    // block and list heads of the first CTA)
    cluster.sync();
}

const void *fill_kernel_entry(int rw)
{
    if (rw == 4) return (const void *)fill_kernel<4>;
    if (rw == 5) return (const void *)fill_kernel<5>;
    return (const void *)fill_kernel<8>;
}

cudaError_t launch_fill(int rw, const cudaLaunchConfig_t &cfg, const FillParams &p)
{
    if (rw == 4) return cudaLaunchKernelEx(&cfg, fill_kernel<4>, p);
    if (rw == 5) return cudaLaunchKernelEx(&cfg, fill_kernel<5>, p);
    return cudaLaunchKernelEx(&cfg, fill_kernel<8>, p);
}

}  // namespace gf

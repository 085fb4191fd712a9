// Host side of the Guidefill C ABI (include/guidefill.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "gf_detect.cuh"


using namespace gf;

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct gf_ctx {
    int device = 0;
    int sm_count = 0;
    int last_cuda = 0;
    DevBuf arena;       // fill scratch
    DevBuf garena;      // guidance scratch
    DevBuf io;          // host-buffer path device copies
    void *hstage = nullptr;   // pinned staging of the host-buffer path's splines
    size_t hstage_bytes = 0;
    DevBuf aarena;      // adjoint scratch
    DevBuf darena;      // spline-detection scratch
    // cached graphs of the last batched fill: gexec = preparation (descriptor
    // upload, clears, init, frame order), gexec_fill = the persistent fill kernel
    cudaGraphExec_t gexec = nullptr;
    cudaGraphExec_t gexec_fill = nullptr;
    uint64_t gkey = 0;
    // launch configuration (0 = automatic)
    int cluster_size = 0;
    int n_clusters = 0;
    int use_graph = 1;
    int last_cluster_size = 0, last_n_clusters = 0;
    // split schedule (0 = none): the split_m frames with the largest holes go to a
    // second persistent launch of split_nc clusters of split_cs CTAs, beside the
    // launch that takes the other frames
    int split_m = 0, split_cs = 0, split_nc = 0;
    int last_split_m = 0, last_split_cs = 0, last_split_nc = 0;
    cudaStream_t aux = nullptr;                   // the second launch's stream
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    cudaEvent_t guide_ev = nullptr;               // guide field done (gf_fill_batched_splines)
    // host-buffer path: copy streams, the events of its chunk pipeline, and per
    // chunk a stream and scratch for its guide field and fill (chunks overlap)
    cudaStream_t copy_in = nullptr, copy_out = nullptr;
    std::vector<cudaEvent_t> pipe_ev;
    std::vector<cudaStream_t> pipe_st;
    std::vector<DevBuf> pipe_fill, pipe_guide;
    // autotuned launch shapes keyed by (n frames, H, W, eps, flags)
    struct Tuned {
        uint64_t key;
        int cluster_size, n_clusters;
        int split_m, split_cs, split_nc;
        float ms;
    };
    std::vector<Tuned> tuned;
};

static uint64_t tune_key(int n, const gf_frame *frames, const gf_params *p)
{
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < n; i++) {
        const uint64_t hw = ((uint64_t)(uint32_t)frames[i].H << 32) | (uint32_t)frames[i].W;
        for (int b = 0; b < 8; b++) {
            h ^= (hw >> (8 * b)) & 0xff;
            h *= 1099511628211ull;
        }
    }
    const uint32_t v[3] = {(uint32_t)n, p->flags, (uint32_t)std::ceil((double)p->eps)};
    const unsigned char *c = (const unsigned char *)v;
    for (size_t i = 0; i < sizeof(v); i++) {
        h ^= c[i];
        h *= 1099511628211ull;
    }
    return h;
}

static gf_status cuda_fail(gf_ctx *ctx, cudaError_t e)
{
    if (ctx) ctx->last_cuda = (int)e;
    return e == cudaErrorMemoryAllocation ? GF_ERR_OOM : GF_ERR_CUDA;
}
#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_); \
    } while (0)

static void drop_graphs(gf_ctx *ctx, cudaStream_t stream)
{
    if (stream) cudaStreamSynchronize(stream);
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->gexec_fill) cudaGraphExecDestroy(ctx->gexec_fill);
    ctx->gexec = nullptr;
    ctx->gexec_fill = nullptr;
    ctx->gkey = 0;
}

// Puts back the context's launch settings (cluster size, cluster count, split
// schedule) when a call that overrides them for its own launches returns, on
// every path including the early returns of CK.
struct LaunchSettingsGuard {
    gf_ctx *ctx;
    int cs, nc, sm, scs, snc;
    explicit LaunchSettingsGuard(gf_ctx *c)
        : ctx(c), cs(c->cluster_size), nc(c->n_clusters), sm(c->split_m), scs(c->split_cs), snc(c->split_nc)
    {
    }
    ~LaunchSettingsGuard()
    {
        ctx->cluster_size = cs;
        ctx->n_clusters = nc;
        ctx->split_m = sm;
        ctx->split_cs = scs;
        ctx->split_nc = snc;
    }
    LaunchSettingsGuard(const LaunchSettingsGuard &) = delete;
    LaunchSettingsGuard &operator=(const LaunchSettingsGuard &) = delete;
};

// Two timing events destroyed on every return path.
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    EventPair() = default;
    ~EventPair()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    EventPair(const EventPair &) = delete;
    EventPair &operator=(const EventPair &) = delete;
};

static gf_status ensure(gf_ctx *ctx, DevBuf &b, size_t bytes)
{
    if (b.bytes >= bytes) return GF_OK;
    if (b.ptr) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(ctx, e);
        cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
        drop_graphs(ctx, nullptr);
    }
    size_t nb = std::max(bytes, (size_t)1 << 20);
    nb = (nb + ((size_t)1 << 20) - 1) & ~(((size_t)1 << 20) - 1);
    cudaError_t e = cudaMalloc(&b.ptr, nb);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    b.bytes = nb;
    return GF_OK;
}

static inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

namespace gf {
void build_tab(float eps, SampleTab &tab);
}
void gf::build_tab(float eps, SampleTab &tab)
{
    memset(&tab, 0, sizeof(tab));
    const double e = (double)eps;
    const int R = (int)std::ceil(e);
    std::vector<int> cn, cm;
    for (int m = -R; m <= R; m++)
        for (int n = -R; n <= R; n++) {
            if (n == 0 && m == 0) continue;
            if ((double)(n * n + m * m) <= e * e) {
                cn.push_back(n);
                cm.push_back(m);
            }
        }
    tab.ns = (int)cn.size();
    tab.nsp = (tab.ns + 31) / 32 * 32;  // padding entries stay (0, 0) with 1/|.| = 0 (memset above)
    tab.R = R;
    for (int s = 0; s < tab.ns; s++) {
        tab.cn[s] = (int8_t)cn[s];
        tab.cm[s] = (int8_t)cm[s];
    }
    int pos = 0;
    for (int g = 0; g <= R; g++) {
        tab.m_start[g] = pos;
        float D = 0.f;
        for (int s = 0; s < tab.ns; s++) {
            if (std::abs(cm[s]) != g) continue;
            float inv = (float)(1.0 / std::sqrt((double)(cn[s] * cn[s] + cm[s] * cm[s])));
            tab.n_f[pos] = (float)cn[s];
            tab.m_f[pos] = (float)cm[s];
            tab.invd[pos] = inv;
            D += inv;
            pos++;
        }
        tab.Dm[g] = D;
    }
    for (int g = R + 1; g <= MAX_R + 1; g++) tab.m_start[g] = pos;
}

static uint64_t fnv(uint64_t h, const void *p, size_t n)
{
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < n; i++) {
        h ^= c[i];
        h *= 1099511628211ull;
    }
    return h;
}

static int rw_for(float eps)
{
    int R = (int)std::ceil((double)eps);
    return R <= 3 ? 4 : (R == 4 ? 5 : 8);
}

static size_t warp_smem(int rw)
{
    return rw == 4 ? sizeof(WarpSmem<4>) : (rw == 5 ? sizeof(WarpSmem<5>) : sizeof(WarpSmem<8>));
}

static const void *fill_kernel_ptr(int rw) { return fill_kernel_entry(rw); }

static gf_status check_params(const gf_params *p)
{
    if (!p) return GF_ERR_ARG;
    if (!(p->eps >= 1.0f && p->eps <= 7.0f)) return GF_ERR_ARG;
    if (!(p->mu >= 0.0f) || !std::isfinite(p->mu)) return GF_ERR_ARG;
    if (p->flags & ~(GF_FLAG_GHOST | GF_FLAG_SMART | GF_FLAG_RESCAN | GF_FLAG_DATA)) return GF_ERR_ARG;
    if ((p->flags & GF_FLAG_SMART) && !(p->c >= 1e-6f && p->c < 1.0f)) return GF_ERR_ARG;
    if (!(p->snap_tau >= 0.0f && p->snap_tau < 0.01f)) return GF_ERR_ARG;
    if (p->max_shells < 0) return GF_ERR_ARG;
    return GF_OK;
}

static gf_status check_frame(const gf_frame *f)
{
    if (!f) return GF_ERR_ARG;
    if (f->H <= 0 || f->W <= 0) return GF_ERR_ARG;
    if ((int64_t)f->H * f->W > ((int64_t)1 << 31) - 64) return GF_ERR_ARG;
    if (!f->rgba || !f->labels || !f->guide || !f->out_rgba || !f->out_shell) return GF_ERR_ARG;
    if (((uintptr_t)f->rgba & 15) || ((uintptr_t)f->out_rgba & 15)) return GF_ERR_ARG;
    if (((uintptr_t)f->guide & 7) || ((uintptr_t)f->out_shell & 3)) return GF_ERR_ARG;
    if (f->out_enter && ((uintptr_t)f->out_enter & 3)) return GF_ERR_ARG;
    if (f->out_stall && ((uintptr_t)f->out_stall & 3)) return GF_ERR_ARG;
    return GF_OK;
}

extern "C" {

const char *gf_status_string(int s)
{
    switch (s) {
    case GF_OK: return "ok";
    case GF_INCOMPLETE: return "incomplete: some hole pixels could not be reached";
    case GF_ERR_ARG: return "invalid argument";
    case GF_ERR_CUDA: return "CUDA error";
    case GF_ERR_TIMEOUT: return "device wait timed out";
    case GF_ERR_NO_PROGRESS: return "shell loop reached max_shells";
    case GF_ERR_OOM: return "out of device memory";
    case GF_ERR_UNSUPPORTED: return "unsupported device";
    case GF_ERR_INTERNAL: return "internal consistency check failed";
    case GF_ERR_TOO_LARGE: return "frame larger than the fixed scratch of gf_fill_noalloc (max 4096 x 4096 px, 4194304 px)";
    default: return "unknown status";
    }
}

int gf_last_cuda_error(const gf_ctx *ctx) { return ctx ? ctx->last_cuda : 0; }

gf_status gf_create(gf_ctx **out, int device)
{
    if (!out) return GF_ERR_ARG;
    *out = nullptr;
    gf_ctx *ctx = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return GF_ERR_CUDA;
    if (device < 0 || device >= ndev) return GF_ERR_ARG;
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) return GF_ERR_CUDA;
    if (!(prop.major == 10 && prop.minor == 3)) return GF_ERR_UNSUPPORTED;
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return GF_ERR_CUDA;
    ctx = new gf_ctx();
    ctx->device = device;
    ctx->sm_count = prop.multiProcessorCount;
    e = cudaFuncSetAttribute((const void *)adj_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
        ctx->last_cuda = (int)e;
        delete ctx;
        return GF_ERR_CUDA;
    }
    for (int rw : {4, 5, 8}) {
        const void *k = fill_kernel_ptr(rw);
        size_t smem = warp_smem(rw) * fill_warps(rw);
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) {
            ctx->last_cuda = (int)e;
            delete ctx;
            return GF_ERR_CUDA;
        }
    }
    e = cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        // highest priority: the host-buffer gather on this stream takes SMs ahead of
        // the guide kernel's large grid beside it
        int lo = 0, hi = 0;
        e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->copy_in, cudaStreamNonBlocking, hi);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->copy_out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->guide_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        ctx->last_cuda = (int)e;
        gf_destroy(ctx);
        return GF_ERR_CUDA;
    }
    *out = ctx;
    return GF_OK;
}

void gf_destroy(gf_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    if (ctx->copy_in) cudaStreamDestroy(ctx->copy_in);
    if (ctx->hstage) cudaFreeHost(ctx->hstage);
    if (ctx->copy_out) cudaStreamDestroy(ctx->copy_out);
    for (cudaEvent_t ev : ctx->pipe_ev) cudaEventDestroy(ev);
    for (cudaStream_t s : ctx->pipe_st) cudaStreamDestroy(s);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
    if (ctx->guide_ev) cudaEventDestroy(ctx->guide_ev);
    cudaDeviceSynchronize();
    drop_graphs(ctx, nullptr);
    if (ctx->arena.ptr) cudaFree(ctx->arena.ptr);
    if (ctx->garena.ptr) cudaFree(ctx->garena.ptr);
    if (ctx->io.ptr) cudaFree(ctx->io.ptr);
    if (ctx->aarena.ptr) cudaFree(ctx->aarena.ptr);
    if (ctx->darena.ptr) cudaFree(ctx->darena.ptr);
    for (DevBuf &b : ctx->pipe_fill)
        if (b.ptr) cudaFree(b.ptr);
    for (DevBuf &b : ctx->pipe_guide)
        if (b.ptr) cudaFree(b.ptr);
    delete ctx;
}

/* Launch shape of the persistent fill (0 = automatic).  Used by the autotuner
 * and by tests that check results do not depend on the launch shape. */
gf_status gf_set_launch_config(gf_ctx *ctx, int cluster_size, int n_clusters, int use_graph)
{
    if (!ctx) return GF_ERR_ARG;
    if (cluster_size != 0 && cluster_size != 1 && cluster_size != 2 && cluster_size != 4 &&
        cluster_size != 8 && cluster_size != 16)
        return GF_ERR_ARG;
    if (n_clusters < 0) return GF_ERR_ARG;
    ctx->cluster_size = cluster_size;
    ctx->n_clusters = n_clusters;
    ctx->use_graph = use_graph ? 1 : 0;
    return GF_OK;
}

/* Launch shape used by the last fill call. */
gf_status gf_get_last_launch(const gf_ctx *ctx, int *cluster_size, int *n_clusters)
{
    if (!ctx || !cluster_size || !n_clusters) return GF_ERR_ARG;
    *cluster_size = ctx->last_cluster_size;
    *n_clusters = ctx->last_n_clusters;
    return GF_OK;
}

gf_status gf_set_split(gf_ctx *ctx, int split_m, int cluster_size, int n_clusters)
{
    if (!ctx || split_m < 0 || n_clusters < 0) return GF_ERR_ARG;
    if (split_m > 0 && cluster_size != 1 && cluster_size != 2 && cluster_size != 4 && cluster_size != 8 &&
        cluster_size != 16)
        return GF_ERR_ARG;
    ctx->split_m = split_m;
    ctx->split_cs = split_m > 0 ? cluster_size : 0;
    ctx->split_nc = split_m > 0 ? n_clusters : 0;
    return GF_OK;
}

gf_status gf_get_last_split(const gf_ctx *ctx, int *split_m, int *cluster_size, int *n_clusters)
{
    if (!ctx || !split_m || !cluster_size || !n_clusters) return GF_ERR_ARG;
    *split_m = ctx->last_split_m;
    *cluster_size = ctx->last_split_cs;
    *n_clusters = ctx->last_split_nc;
    return GF_OK;
}

/* Maximum number of co-resident clusters of the given size for eps. */
int gf_max_active_clusters(gf_ctx *ctx, float eps, int cluster_size)
{
    if (!ctx) return -1;
    int rw = rw_for(eps);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster_size * 64);
    cfg.blockDim = dim3(32 * fill_warps(rw));
    cfg.dynamicSmemBytes = warp_smem(rw) * fill_warps(rw);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster_size;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&n, fill_kernel_ptr(rw), &cfg);
    if (e != cudaSuccess) {
        ctx->last_cuda = (int)e;
        cudaGetLastError();
        return 0;
    }
    return n;
}

static gf_status enqueue_fill(gf_ctx *ctx, int n, const gf_frame *frames, const gf_params *prm,
                              gf_stats *dev_stats, cudaStream_t stream, cudaEvent_t ev0 = nullptr,
                              cudaEvent_t ev1 = nullptr, bool allow_graph = true, DevBuf *scratch = nullptr,
                              cudaEvent_t wait_before_fill = nullptr)
{
    DevBuf &arena = scratch ? *scratch : ctx->arena;
    // ---- layout of the scratch arena
    std::vector<size_t> off_U(n), off_Q(n), off_F(n), off_S(n), off_L(n);
    std::vector<int> ntiles(n);
    size_t pos = 0;
    int list_cap = 1;
    for (int i = 0; i < n; i++) {
        int TW = (frames[i].W + 7) / 8, TH = (frames[i].H + 7) / 8;
        ntiles[i] = TW * TH;
        list_cap = std::max(list_cap, 9 * ntiles[i]);  // a tile with fills reserves up to 9 slots
        off_U[i] = pos; pos = align_up(pos + 8 * (size_t)ntiles[i], 256);
        off_Q[i] = pos; pos = align_up(pos + 8 * (size_t)ntiles[i], 256);
        off_F[i] = pos; pos = align_up(pos + sizeof(TileF) * 2 * (size_t)ntiles[i], 256);
        off_S[i] = pos; pos = align_up(pos + 4 * (size_t)ntiles[i], 256);
        off_L[i] = pos; pos = align_up(pos + 4 * (size_t)ntiles[i], 256);
    }
    const size_t off_holes = pos; pos = align_up(pos + 4 * (size_t)n, 256);
    const size_t off_gleft = pos; pos = align_up(pos + 4 * (size_t)n, 256);
    const size_t off_icnt = pos; pos = align_up(pos + 8 * (size_t)n, 256);
    const size_t off_desc = pos; pos = align_up(pos + sizeof(FrameDev) * (size_t)n, 256);
    const size_t off_order = pos; pos = align_up(pos + 4 * (size_t)n, 256);
    const size_t off_cursor = pos; pos = align_up(pos + 8, 256);  // queue heads of the two launches
    const size_t off_ctaoff = pos; pos = align_up(pos + 4 * (size_t)(n + 1), 256);

    // ---- launch shape
    const int rw = rw_for(prm->eps);
    int cs = ctx->cluster_size;
    int tuned_nc = 0;
    int sm = ctx->split_m, scs = ctx->split_cs, snc = ctx->split_nc;
    if (cs == 0) {
        const uint64_t tk = tune_key(n, frames, prm);
        for (const auto &t : ctx->tuned)
            if (t.key == tk) {
                cs = t.cluster_size;
                tuned_nc = t.n_clusters;
                if (sm == 0) {
                    sm = t.split_m;
                    scs = t.split_cs;
                    snc = t.split_nc;
                }
            }
    }
    if (cs == 0) cs = (n == 1) ? 16 : 4;  // before any autotuning: 16 CTAs for one frame, 4 per frame of a batch
    int maxc = gf_max_active_clusters(ctx, prm->eps, cs);
    while (maxc <= 0 && cs > 1) {
        cs /= 2;
        maxc = gf_max_active_clusters(ctx, prm->eps, cs);
    }
    if (maxc <= 0) return GF_ERR_UNSUPPORTED;
    int nc = ctx->n_clusters > 0 ? std::min(ctx->n_clusters, maxc) : (tuned_nc > 0 ? std::min(tuned_nc, maxc) : maxc);
    // split schedule: the second launch takes snc clusters of scs CTAs (one CTA per
    // SM) for the sm largest holes; the first launch keeps the SMs left over
    bool split = sm > 0 && sm < n && scs > 0 && snc > 0;
    if (split) {
        const int maxa = gf_max_active_clusters(ctx, prm->eps, scs);
        snc = std::min(std::min(snc, sm), maxa);
        const int spare = snc > 0 ? (ctx->sm_count - snc * scs) / cs : 0;
        if (snc <= 0 || spare < 1) split = false;
        else nc = std::min(nc, spare);
    }
    if (!split) sm = scs = snc = 0;
    nc = std::max(1, std::min(nc, n - sm));
    ctx->last_cluster_size = cs;
    ctx->last_n_clusters = nc;
    ctx->last_split_m = sm;
    ctx->last_split_cs = scs;
    ctx->last_split_nc = snc;
    const int ncall = nc + snc;  // control blocks and work lists of both launches

    const size_t off_lists = pos; pos = align_up(pos + 4 * (size_t)3 * list_cap * ncall, 256);
    gf_status st = ensure(ctx, arena, pos);
    if (st != GF_OK) return st;
    char *A = (char *)arena.ptr;

    // ---- frame descriptors (uploaded by value through kernel parameters)
    std::vector<FrameDev> hdv(n);
    std::vector<int32_t> hctav(n + 1);
    FrameDev *hd = hdv.data();
    int32_t *hcta = hctav.data();
    int64_t ctas = 0;
    for (int i = 0; i < n; i++) {
        const gf_frame &f = frames[i];
        FrameDev d;
        memset(&d, 0, sizeof(d));
        d.H = f.H;
        d.W = f.W;
        d.TW = (f.W + 7) / 8;
        d.TH = (f.H + 7) / 8;
        d.ntiles = ntiles[i];
        const int64_t full = (int64_t)f.H * f.W + 1;
        int64_t cap = prm->max_shells > 0 ? std::min<int64_t>(prm->max_shells, full) : full;
        d.max_shells = (int32_t)std::min<int64_t>(cap, INT32_MAX - 2);
        d.rgba = (float4 *)f.out_rgba;
        d.labels = f.labels;
        d.guide = (const float2 *)f.guide;
        d.shell = f.out_shell;
        d.enter = f.out_enter;
        d.stall_bits = f.out_stall;
        d.stats = dev_stats + i;
        d.U = (unsigned long long *)(A + off_U[i]);
        d.Qw = (unsigned long long *)(A + off_Q[i]);
        d.F = (TileF *)(A + off_F[i]);
        d.sched = (int32_t *)(A + off_S[i]);
        d.holes = (int32_t *)(A + off_holes) + i;
        d.gleft = (int32_t *)(A + off_gleft) + i;
        d.init_list = (int32_t *)(A + off_L[i]);
        d.init_count = (int32_t *)(A + off_icnt) + 2 * i;
        hd[i] = d;
        hcta[i] = (int32_t)ctas;
        ctas += (int64_t)init_ctas(d.TH, f.W);
    }
    hcta[n] = (int32_t)ctas;
    if (ctas >= INT32_MAX) return GF_ERR_ARG;

    FillParams fp;
    memset(&fp, 0, sizeof(fp));
    fp.eps = prm->eps;
    fp.mu = prm->mu;
    fp.c = prm->c;
    fp.tau = prm->snap_tau;
    fp.coef32 = (prm->mu * prm->mu) / (2.0f * prm->eps * prm->eps);
    fp.coef64 = (double)prm->mu * (double)prm->mu / (2.0 * (double)prm->eps * (double)prm->eps);
    fp.c64 = (double)prm->c;
    fp.flags = prm->flags;
    fp.n_frames = n - sm;  // the first launch: frame_order[sm ..)
    fp.order_first = sm;
    fp.list_cap = list_cap;
    fp.frames = (FrameDev *)(A + off_desc);
    fp.frame_order = (int32_t *)(A + off_order);
    fp.frame_cursor = (int32_t *)(A + off_cursor);
    fp.lists = (int32_t *)(A + off_lists);
    build_tab(prm->eps, fp.tab);
    FillParams fpa = fp;  // the second launch: frame_order[0 .. sm)
    fpa.n_frames = sm;
    fpa.order_first = 0;
    fpa.frame_cursor = fp.frame_cursor + 1;
    fpa.lists = fp.lists + (size_t)nc * 3 * list_cap;

    // graph key: everything the enqueued work depends on
    uint64_t key = 1469598103934665603ull;
    key = fnv(key, hd, sizeof(FrameDev) * (size_t)n);
    key = fnv(key, prm, sizeof(*prm));
    key = fnv(key, &cs, sizeof(cs));
    key = fnv(key, &nc, sizeof(nc));
    key = fnv(key, &sm, sizeof(sm));
    key = fnv(key, &scs, sizeof(scs));
    key = fnv(key, &snc, sizeof(snc));
    key = fnv(key, &n, sizeof(n));
    for (int i = 0; i < n; i++) key = fnv(key, &frames[i].rgba, sizeof(void *));
    key = fnv(key, &arena.ptr, sizeof(void *));

    const bool graph = allow_graph && ctx->use_graph && stream != nullptr;
    if (graph && ctx->gexec && ctx->gexec_fill && ctx->gkey == key) {
        CK(cudaGraphLaunch(ctx->gexec, stream));
        if (wait_before_fill) CK(cudaStreamWaitEvent(stream, wait_before_fill, 0));
        if (ev0) CK(cudaEventRecord(ev0, stream));
        CK(cudaGraphLaunch(ctx->gexec_fill, stream));
        if (ev1) CK(cudaEventRecord(ev1, stream));
        return GF_OK;
    }
    if (graph && (ctx->gexec || ctx->gexec_fill)) drop_graphs(ctx, stream);

    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nc * cs));
    cfg.blockDim = dim3(32 * fill_warps(rw));
    cfg.dynamicSmemBytes = warp_smem(rw) * fill_warps(rw);
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;

    // ---- phase 1: descriptors, clears, init, frame order
    if (graph) CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    do {
        for (int c0 = 0; c0 < n && !e; c0 += DESC_CHUNK) {
            static thread_local FrameChunk ch;  // large: keep off the stack
            ch.dst_frames = (FrameDev *)(A + off_desc);
            ch.dst_cta = (int32_t *)(A + off_ctaoff);
            ch.first = c0;
            ch.count = std::min(DESC_CHUNK, n - c0);
            ch.last_chunk = (c0 + ch.count == n) ? 1 : 0;
            for (int i = 0; i < ch.count; i++) {
                ch.frames[i] = hd[c0 + i];
                ch.cta[i] = hcta[c0 + i];
            }
            ch.cta[ch.count] = hcta[c0 + ch.count];
            upload_frames_kernel<<<1, 128, 0, stream>>>(ch);
            e = cudaGetLastError();
        }
        if (e) break;
        e = cudaMemsetAsync(A + off_holes, 0, 4 * (size_t)n, stream);
        if (!e) e = cudaMemsetAsync(A + off_gleft, 0, 4 * (size_t)n, stream);
        if (e) break;
        e = cudaMemsetAsync(A + off_icnt, 0, 8 * (size_t)n, stream);
        if (e) break;
        for (int i = 0; i < n && !e; i++) {
            const gf_frame &f = frames[i];
            if (f.out_rgba != f.rgba)
                e = cudaMemcpyAsync(f.out_rgba, f.rgba, (size_t)f.H * f.W * 16, cudaMemcpyDeviceToDevice, stream);
            if (!e && f.out_stall)
                e = cudaMemsetAsync(f.out_stall, 0, 4 * (((size_t)f.H * f.W + 1 + 31) / 32), stream);
        }
        if (e) break;
        InitArgs ia;
        ia.frames = fp.frames;
        ia.cta_offset = (const int32_t *)(A + off_ctaoff);
        ia.n_frames = n;
        ia.flags = prm->flags;
        ia.uniform_ctas = hcta[1] - hcta[0];
        for (int i = 1; i < n; i++)
            if (hcta[i + 1] - hcta[i] != ia.uniform_ctas) ia.uniform_ctas = 0;
        init_kernel<<<(unsigned)ctas, 32 * INIT_WARPS, 0, stream>>>(ia);
        e = cudaGetLastError();
        if (e) break;
        order_kernel<<<1, 256, 0, stream>>>(fp.frames, n, fp.frame_order, fp.frame_cursor);
        e = cudaGetLastError();
    } while (0);
    cudaGraph_t g1 = nullptr;
    if (graph) {
        cudaError_t e2 = cudaStreamEndCapture(stream, &g1);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) {
        if (g1) cudaGraphDestroy(g1);
        return cuda_fail(ctx, e);
    }
    // phase 2: the persistent fill, or with a split schedule the two persistent
    // launches side by side (the second on the context's own stream, forked from
    // and joined back into `stream`; neither waits for the other)
    auto launch_phase2 = [&]() -> cudaError_t {
        if (!split) return launch_fill(rw, cfg, fp);
        cudaError_t r = cudaEventRecord(ctx->fork_ev, stream);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(ctx->aux, ctx->fork_ev, 0);
        cudaLaunchConfig_t cfga = cfg;
        cudaLaunchAttribute ata[1] = {at[0]};
        ata[0].val.clusterDim.x = scs;
        cfga.attrs = ata;
        cfga.gridDim = dim3((unsigned)(snc * scs));
        cfga.stream = ctx->aux;
        if (r == cudaSuccess) r = launch_fill(rw, cfga, fpa);
        if (r == cudaSuccess) r = launch_fill(rw, cfg, fp);
        if (r == cudaSuccess) r = cudaEventRecord(ctx->join_ev, ctx->aux);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(stream, ctx->join_ev, 0);
        return r;
    };
    if (!graph) {
        // ---- phase 2 directly
        if (wait_before_fill) CK(cudaStreamWaitEvent(stream, wait_before_fill, 0));
        if (ev0) CK(cudaEventRecord(ev0, stream));
        CK(launch_phase2());
        if (ev1) CK(cudaEventRecord(ev1, stream));
        return GF_OK;
    }
    // ---- phase 2 captured separately so that timing events can sit between the two graphs
    cudaGraph_t g2 = nullptr;
    e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        e = launch_phase2();
        cudaError_t e2 = cudaStreamEndCapture(stream, &g2);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->gexec, g1, 0);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->gexec_fill, g2, 0);
    if (g1) cudaGraphDestroy(g1);
    if (g2) cudaGraphDestroy(g2);
    if (e != cudaSuccess) {
        drop_graphs(ctx, nullptr);
        return cuda_fail(ctx, e);
    }
    ctx->gkey = key;
    CK(cudaGraphLaunch(ctx->gexec, stream));
    if (wait_before_fill) CK(cudaStreamWaitEvent(stream, wait_before_fill, 0));
    if (ev0) CK(cudaEventRecord(ev0, stream));
    CK(cudaGraphLaunch(ctx->gexec_fill, stream));
    if (ev1) CK(cudaEventRecord(ev1, stream));
    return GF_OK;
}

gf_status gf_fill_batched_ex(gf_ctx *ctx, int n, const gf_frame *frames, const gf_params *params,
                             gf_stats *dev_stats, void *stream, void *event_fill_start, void *event_fill_end)
{
    if (!ctx || n <= 0 || !frames || !dev_stats) return GF_ERR_ARG;
    gf_status s = check_params(params);
    if (s != GF_OK) return s;
    for (int i = 0; i < n; i++) {
        s = check_frame(&frames[i]);
        if (s != GF_OK) return s;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    return enqueue_fill(ctx, n, frames, params, dev_stats, (cudaStream_t)stream, (cudaEvent_t)event_fill_start,
                        (cudaEvent_t)event_fill_end);
}

gf_status gf_fill_batched(gf_ctx *ctx, int n, const gf_frame *frames, const gf_params *params,
                          gf_stats *dev_stats, void *stream)
{
    return gf_fill_batched_ex(ctx, n, frames, params, dev_stats, stream, nullptr, nullptr);
}

/* Times the batched fill of these frames under candidate launch shapes and keeps
 * the fastest for later calls on frames of the same sizes and parameters:
 * uniform schedules (cluster sizes 1..16, as many clusters as fit), then split
 * schedules (the m = 1..8, 10, 12, 14, 16, 20, 24 largest holes on m, 3m/4 or m/2
 * clusters of 8 or 16 CTAs beside the best uniform launch, then the split sizes and
 * cluster counts within 2 of the best split).  The frames are filled (in place if
 * out_rgba == rgba) by every trial.  Synchronises stream. */
gf_status gf_autotune(gf_ctx *ctx, int n, const gf_frame *frames, const gf_params *params, gf_stats *dev_stats,
                      void *stream, int trials, int *best_cluster_size, float *best_ms)
{
    if (!ctx || n <= 0 || !frames || !dev_stats) return GF_ERR_ARG;
    gf_status s = check_params(params);
    if (s != GF_OK) return s;
    for (int i = 0; i < n; i++) {
        s = check_frame(&frames[i]);
        if (s != GF_OK) return s;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    cudaStream_t st = (cudaStream_t)stream;
    if (trials <= 0) trials = 3;
    LaunchSettingsGuard keep(ctx);
    EventPair ev;
    CK(cudaEventCreate(&ev.a));
    CK(cudaEventCreate(&ev.b));
    const cudaEvent_t e0 = ev.a, e1 = ev.b;
    // mean fill-kernel time of one schedule over `trials` runs (after a capture run)
    auto measure = [&](float *avg) -> gf_status {
        gf_status r = enqueue_fill(ctx, n, frames, params, dev_stats, st);  // warm-up / capture
        float tot = 0.f;
        for (int t = 0; t < trials && r == GF_OK; t++) {
            r = enqueue_fill(ctx, n, frames, params, dev_stats, st, e0, e1);
            if (r != GF_OK) break;
            cudaError_t ee = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (ee == cudaSuccess) ee = cudaEventElapsedTime(&ms, e0, e1);
            if (ee != cudaSuccess) r = cuda_fail(ctx, ee);
            tot += ms;
        }
        *avg = tot / trials;
        return r;
    };
    // uniform schedules: one cluster size for every frame
    int best_cs = 0, best_nc = 0, best_sm = 0, best_scs = 0, best_snc = 0;
    float best = 1e30f;
    ctx->split_m = ctx->split_cs = ctx->split_nc = 0;
    for (int cs : {1, 2, 4, 8, 16}) {
        if (gf_max_active_clusters(ctx, params->eps, cs) <= 0) continue;
        ctx->cluster_size = cs;
        ctx->n_clusters = 0;
        float avg = 0.f;
        s = measure(&avg);
        if (s != GF_OK) break;
        if (avg < best) {
            best = avg;
            best_cs = cs;
            best_nc = ctx->last_n_clusters;
        }
    }
    // split schedules: the frames with the largest holes (whose shell chains are
    // usually the longest) on a few larger clusters, the rest on the best uniform
    // cluster size with the SMs left over.  The batch time is not smooth in the
    // split (the dynamic queue of each launch decides when the long frames start),
    // so a coarse grid is followed by the neighbours of its best point.
    if (s == GF_OK && best_cs > 0 && n > 1) {
        ctx->cluster_size = best_cs;
        ctx->n_clusters = 0;
        auto trial = [&](int m, int scs, int snc) {
            if (s != GF_OK || m < 1 || m >= n || snc < 1 || snc > m || scs <= best_cs) return;
            if (snc * scs > ctx->sm_count - best_cs) return;
            ctx->split_m = m;
            ctx->split_cs = scs;
            ctx->split_nc = snc;
            float avg = 0.f;
            s = measure(&avg);
            if (s != GF_OK) return;
            if (ctx->last_split_m == m && avg < best) {
                best = avg;
                best_nc = ctx->last_n_clusters;
                best_sm = m;
                best_scs = scs;
                best_snc = ctx->last_split_nc;
            }
        };
        for (int m : {1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16, 20, 24}) {
            for (int scs : {8, 16}) {
                const int cands[3] = {m, (3 * m + 3) / 4, (m + 1) / 2};
                for (int ci = 0; ci < 3; ci++) {
                    if (ci > 0 && cands[ci] == cands[ci - 1]) continue;
                    trial(m, scs, cands[ci]);
                }
            }
        }
        if (best_sm > 0) {
            const int m0 = best_sm, scs0 = best_scs, snc0 = best_snc;
            for (int dm = -2; dm <= 2; dm++)
                for (int dc = -2; dc <= 2; dc++)
                    if (dm != 0 || dc != 0) trial(m0 + dm, scs0, snc0 + dc);
        }
    }
    if (s != GF_OK) return s;
    if (best_cs == 0) return GF_ERR_UNSUPPORTED;
    const uint64_t tk = tune_key(n, frames, params);
    bool found = false;
    for (auto &t : ctx->tuned)
        if (t.key == tk) {
            t.cluster_size = best_cs;
            t.n_clusters = best_nc;
            t.split_m = best_sm;
            t.split_cs = best_scs;
            t.split_nc = best_snc;
            t.ms = best;
            found = true;
        }
    if (!found) ctx->tuned.push_back({tk, best_cs, best_nc, best_sm, best_scs, best_snc, best});
    if (best_cluster_size) *best_cluster_size = best_cs;
    if (best_ms) *best_ms = best;
    return GF_OK;
}

gf_status gf_fill(gf_ctx *ctx, const gf_frame *frame, const gf_params *params, gf_stats *dev_stats,
                  void *stream)
{
    return gf_fill_batched(ctx, 1, frame, params, dev_stats, stream);
}

static gf_status guidance_impl(gf_ctx *ctx, DevBuf &garena, int n, const gf_spline_frame *frames, float eta,
                               void *stream);

gf_status gf_guidance_batched(gf_ctx *ctx, int n, const gf_spline_frame *frames, float eta, void *stream)
{
    if (!ctx) return GF_ERR_ARG;
    return guidance_impl(ctx, ctx->garena, n, frames, eta, stream);
}

static gf_status guidance_impl(gf_ctx *ctx, DevBuf &garena, int n, const gf_spline_frame *frames, float eta,
                               void *stream)
{
    if (!ctx || n <= 0 || !frames || !(eta > 0.0f) || !std::isfinite(eta)) return GF_ERR_ARG;
    for (int i = 0; i < n; i++) {
        const gf_spline_frame &f = frames[i];
        if (f.H <= 0 || f.W <= 0 || !f.labels || !f.guide || f.n_splines < 0 || f.n_points < 0) return GF_ERR_ARG;
        if ((int64_t)f.H * f.W > ((int64_t)1 << 31) - 64) return GF_ERR_ARG;
        if (f.n_splines > 0 && (!f.offsets || !f.pts)) return GF_ERR_ARG;
        if (((uintptr_t)f.guide & 7) || (f.pts && ((uintptr_t)f.pts & 7))) return GF_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<size_t> off_cnt(n), off_list(n), off_seg(n);
    size_t pos = 0;
    int64_t tot_pts = 0, tot_bins = 0;
    for (int i = 0; i < n; i++) {
        int NBX = (frames[i].W + BIN - 1) / BIN, NBY = (frames[i].H + BIN - 1) / BIN;
        off_cnt[i] = pos; pos = align_up(pos + 4 * (size_t)NBX * NBY, 256);
        off_list[i] = pos; pos = align_up(pos + 4 * (size_t)NBX * NBY * BIN_CAP, 256);
        off_seg[i] = pos; pos = align_up(pos + 64 * (size_t)std::max(frames[i].n_points, 1), 256);
        tot_pts += frames[i].n_points;
        tot_bins += (int64_t)NBX * NBY;
    }
    if (tot_pts >= INT32_MAX || tot_bins >= INT32_MAX) return GF_ERR_ARG;
    const size_t off_desc = pos; pos = align_up(pos + sizeof(SplineFrameDev) * (size_t)n, 256);
    const size_t off_po = pos; pos = align_up(pos + 4 * (size_t)(n + 1), 256);
    const size_t off_bo = pos; pos = align_up(pos + 4 * (size_t)(n + 1), 256);
    gf_status s = ensure(ctx, garena, pos);
    if (s != GF_OK) return s;
    char *A = (char *)garena.ptr;
    std::vector<SplineFrameDev> hdv(n);
    std::vector<int32_t> hpov(n + 1), hbov(n + 1);
    SplineFrameDev *hd = hdv.data();
    int32_t *hpo = hpov.data();
    int32_t *hbo = hbov.data();
    int64_t pp = 0, bb = 0;
    for (int i = 0; i < n; i++) {
        const gf_spline_frame &f = frames[i];
        SplineFrameDev d;
        d.H = f.H; d.W = f.W;
        d.NBX = (f.W + BIN - 1) / BIN; d.NBY = (f.H + BIN - 1) / BIN;
        d.n_splines = f.n_splines; d.n_points = f.n_points;
        d.labels = f.labels; d.offsets = f.offsets; d.pts = (const float2 *)f.pts;
        d.guide = (float2 *)f.guide;
        d.bin_count = (int32_t *)(A + off_cnt[i]);
        d.bin_list = (int32_t *)(A + off_list[i]);
        d.seg64 = (double *)(A + off_seg[i]);
        hd[i] = d;
        hpo[i] = (int32_t)pp; hbo[i] = (int32_t)bb;
        pp += f.n_points;
        bb += (int64_t)d.NBX * d.NBY;
    }
    hpo[n] = (int32_t)pp; hbo[n] = (int32_t)bb;
    // counts must be zero; lists need no clearing
    for (int i = 0; i < n; i++) {
        size_t nbins = (size_t)hd[i].NBX * hd[i].NBY;
        CK(cudaMemsetAsync(A + off_cnt[i], 0, 4 * nbins, st));
    }
    for (int c0 = 0; c0 < n; c0 += DESC_CHUNK) {
        static thread_local SplineChunk ch;
        ch.dst_frames = (SplineFrameDev *)(A + off_desc);
        ch.dst_po = (int32_t *)(A + off_po);
        ch.dst_bo = (int32_t *)(A + off_bo);
        ch.first = c0;
        ch.count = std::min(DESC_CHUNK, n - c0);
        ch.last_chunk = (c0 + ch.count == n) ? 1 : 0;
        for (int i = 0; i < ch.count; i++) {
            ch.frames[i] = hd[c0 + i];
            ch.po[i] = hpo[c0 + i];
            ch.bo[i] = hbo[c0 + i];
        }
        ch.po[ch.count] = hpo[c0 + ch.count];
        ch.bo[ch.count] = hbo[c0 + ch.count];
        upload_splines_kernel<<<1, 128, 0, st>>>(ch);
        CK(cudaGetLastError());
    }
    GuideArgs ga;
    ga.frames = (const SplineFrameDev *)(A + off_desc);
    ga.point_offset = (const int32_t *)(A + off_po);
    ga.bin_offset = (const int32_t *)(A + off_bo);
    ga.n_frames = n;
    ga.total_bins = (int32_t)bb;
    ga.eta = eta;
    ga.k2 = 1.0 / (2.0 * (double)eta * (double)eta);
    if (pp > 0) {
        bin_kernel<<<(unsigned)((pp + 255) / 256), 256, 0, st>>>(ga, (int)pp);
        CK(cudaGetLastError());
        for (int c0 = 0; c0 < n; c0 += DESC_CHUNK) {
            WeightChunk wc;
            wc.first = c0;
            wc.count = std::min(DESC_CHUNK, n - c0);
            bool any = false;
            for (int i = 0; i < wc.count; i++) {
                wc.w[i] = frames[c0 + i].n_points > 1 ? frames[c0 + i].weight : nullptr;
                any = any || wc.w[i];
            }
            if (!any) continue;
            spline_weight_kernel<<<(unsigned)wc.count, 256, 0, st>>>(ga, wc);
            CK(cudaGetLastError());
        }
    }
    guide_kernel<<<(unsigned)bb, 256, 0, st>>>(ga);
    CK(cudaGetLastError());
    return GF_OK;
}

gf_status gf_guidance_from_splines(gf_ctx *ctx, int H, int W, const uint8_t *labels, int n_splines,
                                   const int32_t *offsets, int n_points, const float *pts, float eta,
                                   float *guide, void *stream)
{
    gf_spline_frame f;
    f.H = H; f.W = W; f.labels = labels; f.n_splines = n_splines; f.n_points = n_points;
    f.weight = nullptr;
    f.offsets = offsets; f.pts = pts; f.guide = guide;
    return gf_guidance_batched(ctx, 1, &f, eta, stream);
}

// Normalised taps of g_s (radius ceil(2 s)): exp(-i^2/(2 s^2)) in FP64 rounded
// to FP32, divided by their FP32 sum (Section 3.3's (4 s + 1) windows).
static int gauss_taps(float s, float *w)
{
    const int r = (int)std::ceil(2.0 * (double)s);
    float sum = 0.0f;
    for (int i = -r; i <= r; i++) {
        w[i + r] = (float)std::exp(-(double)(i * i) / (2.0 * (double)s * (double)s));
        sum = sum + w[i + r];
    }
    for (int i = 0; i <= 2 * r; i++) w[i] = w[i] / sum;
    return r;
}

gf_status gf_detect_splines_batched(gf_ctx *ctx, int n, const gf_detect_frame *frames, const gf_detect_params *prm,
                                    void *stream)
{
    if (!ctx || n <= 0 || !frames || !prm) return GF_ERR_ARG;
    const gf_detect_params P = *prm;
    if (!(P.sigma > 0.0f && P.sigma <= 4.0f) || !(P.rho > 0.0f && P.rho <= 8.0f)) return GF_ERR_ARG;
    if (!(P.t_high >= 0.0f) || !(P.t_low >= 0.0f) || !std::isfinite(P.t_high) || !std::isfinite(P.t_low))
        return GF_ERR_ARG;
    if (!(P.length > 0.0f) || !std::isfinite(P.length) || !(P.Lambda > 0.0f) || !std::isfinite(P.Lambda))
        return GF_ERR_ARG;
    const int rS = (int)std::ceil(2.0 * (double)P.sigma), rR = (int)std::ceil(2.0 * (double)P.rho);
    const int dR = P.ring_dist > 0 ? P.ring_dist : rS + rR + 2;
    if (P.ring_dist < 0 || P.annulus < 0 || P.annulus > 16 || P.annulus >= dR || dR + P.annulus > 96)
        return GF_ERR_ARG;
    for (int i = 0; i < n; i++) {
        const gf_detect_frame &f = frames[i];
        if (f.H <= 0 || f.W <= 0 || !f.rgba || !f.labels || !f.result || !f.offsets || f.max_splines < 0)
            return GF_ERR_ARG;
        if ((int64_t)f.H * f.W > ((int64_t)1 << 31) - 64) return GF_ERR_ARG;
        if (f.max_splines > 0 && (!f.pts || !f.weight)) return GF_ERR_ARG;
        if (((uintptr_t)f.rgba & 15) || (f.pts && ((uintptr_t)f.pts & 7)) || ((uintptr_t)f.result & 3) ||
            ((uintptr_t)f.offsets & 3) || (f.weight && ((uintptr_t)f.weight & 3)) || (f.base && ((uintptr_t)f.base & 3)))
            return GF_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    cudaStream_t st = (cudaStream_t)stream;
    // scratch per frame: distances, tile flags, edge classes, union-find, candidates, row-segment masks
    std::vector<DetectFrameDev> hd(n);
    std::vector<int32_t> hto(n + 1);
    std::vector<size_t> o_mask(n), o_dist(n), o_edge(n), o_par(n), o_mark(n), o_cand(n), o_accm(n), o_accp(n);
    std::vector<int32_t> hwo(n + 1);
    int64_t words = 0;
    size_t pos = 0;
    int64_t tiles = 0;
    for (int i = 0; i < n; i++) {
        const size_t np = (size_t)frames[i].H * frames[i].W;
        const int NBX = (frames[i].W + DT - 1) / DT, NBY = (frames[i].H + DT - 1) / DT;
        const int NWF = (frames[i].W + 31) / 32;
        o_mask[i] = pos; pos = align_up(pos + 8 * (size_t)frames[i].H * NWF, 256);
        o_dist[i] = pos; pos = align_up(pos + 2 * np, 256);
        o_edge[i] = pos; pos = align_up(pos + np, 256);
        o_par[i] = pos; pos = align_up(pos + 4 * np, 256);
        o_mark[i] = pos; pos = align_up(pos + 4 * np, 256);
        o_cand[i] = pos; pos = align_up(pos + 16 * np, 256);
        o_accm[i] = pos; pos = align_up(pos + 4 * (size_t)frames[i].H * NBX, 256);
        o_accp[i] = pos; pos = align_up(pos + 4 * (size_t)frames[i].H * NBX, 256);
        hto[i] = (int32_t)tiles;
        tiles += (int64_t)NBX * NBY;
        hwo[i] = (int32_t)words;
        words += (int64_t)frames[i].H * NWF;
    }
    hto[n] = (int32_t)tiles;
    hwo[n] = (int32_t)words;
    if (tiles >= INT32_MAX || words >= INT32_MAX) return GF_ERR_ARG;
    const size_t o_desc = pos; pos = align_up(pos + sizeof(DetectFrameDev) * (size_t)n, 256);
    const size_t o_to = pos; pos = align_up(pos + 4 * (size_t)(n + 1), 256);
    const size_t o_wo = pos; pos = align_up(pos + 4 * (size_t)(n + 1), 256);
    const size_t o_list = pos; pos = align_up(pos + 4 * (size_t)tiles, 256);
    const size_t o_slist = pos; pos = align_up(pos + 4 * (size_t)tiles, 256);
    const size_t o_cnt = pos; pos = align_up(pos + 8, 256);                 // active, slow counts
    const size_t o_flags = pos; pos = align_up(pos + 2 * (size_t)tiles, 256);  // hole_t, act_t (cleared)
    const size_t o_slow = pos; pos = align_up(pos + (size_t)tiles, 256);       // slow_t
    gf_status s = ensure(ctx, ctx->darena, pos);
    if (s != GF_OK) return s;
    char *A = (char *)ctx->darena.ptr;
    for (int i = 0; i < n; i++) {
        const gf_detect_frame &f = frames[i];
        DetectFrameDev d;
        d.H = f.H; d.W = f.W;
        d.NBX = (f.W + DT - 1) / DT; d.NBY = (f.H + DT - 1) / DT;
        d.rgba = (const float4 *)f.rgba; d.labels = f.labels;
        d.masks = (uint2 *)(A + o_mask[i]);
        d.hole_t = (uint8_t *)(A + o_flags) + hto[i];
        d.act_t = (uint8_t *)(A + o_flags) + tiles + hto[i];
        d.slow_t = (uint8_t *)(A + o_slow) + hto[i];
        d.NWF = (f.W + 31) / 32;
        d.dist = (uchar2 *)(A + o_dist[i]);
        d.edge = (uint8_t *)(A + o_edge[i]);
        d.parent = (int32_t *)(A + o_par[i]);
        d.mark = (int32_t *)(A + o_mark[i]);
        d.cand = (float4 *)(A + o_cand[i]);
        d.accm = (uint32_t *)(A + o_accm[i]);
        d.accpos = (uint32_t *)(A + o_accp[i]);
        d.pts = (float2 *)f.pts; d.weight = f.weight; d.offsets = f.offsets; d.base = f.base;
        d.edges_out = f.edges; d.result = f.result;
        d.max_splines = f.max_splines;
        hd[i] = d;
    }
    for (int c0 = 0; c0 < n; c0 += DET_CHUNK) {
        static thread_local DetectChunk ch;
        ch.dst_frames = (DetectFrameDev *)(A + o_desc);
        ch.dst_to = (int32_t *)(A + o_to);
        ch.dst_wo = (int32_t *)(A + o_wo);
        ch.first = c0;
        ch.count = std::min(DET_CHUNK, n - c0);
        ch.last_chunk = (c0 + ch.count == n) ? 1 : 0;
        for (int i = 0; i < ch.count; i++) {
            ch.frames[i] = hd[c0 + i];
            ch.to[i] = hto[c0 + i];
            ch.wo[i] = hwo[c0 + i];
        }
        ch.to[ch.count] = hto[c0 + ch.count];
        ch.wo[ch.count] = hwo[c0 + ch.count];
        upload_detect_kernel<<<1, 64, 0, st>>>(ch);
        CK(cudaGetLastError());
    }
    DetectArgs da;
    da.frames = (const DetectFrameDev *)(A + o_desc);
    da.tile_offset = (const int32_t *)(A + o_to);
    da.active_list = (int32_t *)(A + o_list);
    da.active_count = (int32_t *)(A + o_cnt);
    da.slow_list = (int32_t *)(A + o_slist);
    da.slow_count = (int32_t *)(A + o_cnt) + 1;
    da.word_offset = (const int32_t *)(A + o_wo);
    da.n_frames = n;
    da.total_tiles = (int32_t)tiles;
    da.rS = rS; da.rR = rR; da.dR = dR; da.annulus = P.annulus; da.cap = dR + P.annulus + 1;
    da.th2 = P.t_high * P.t_high;
    da.tl2 = P.t_low * P.t_low;
    da.length = P.length;
    da.Lambda = P.Lambda;
    std::memset(da.wS, 0, sizeof(da.wS));
    std::memset(da.wR, 0, sizeof(da.wR));
    gauss_taps(P.sigma, da.wS);
    gauss_taps(P.rho, da.wR);
    const size_t sm_dist = detect_dist_smem(da.cap), sm_tensor = detect_tensor_smem(rS, rR);
    const void *tensor = detect_tensor_entry(rS);
    if (!tensor) return GF_ERR_ARG;
    CK(cudaFuncSetAttribute(detect_dist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_dist));
    CK(cudaFuncSetAttribute(tensor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_tensor));
    // persistent grids over the active tiles: as many CTAs as fit on the SMs at once
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tensor, DET_THREADS, sm_tensor));
    const unsigned g_tensor = (unsigned)std::min<int64_t>(tiles, (int64_t)std::max(per_sm, 1) * ctx->sm_count);
    const unsigned g_list = (unsigned)std::min<int64_t>(tiles, 8 * (int64_t)ctx->sm_count);
    int per_sm_dist = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_dist, detect_dist_kernel, DET_THREADS, sm_dist));
    const unsigned g_dist = (unsigned)std::min<int64_t>(tiles, (int64_t)std::max(per_sm_dist, 1) * ctx->sm_count);
    CK(cudaMemsetAsync(A + o_cnt, 0, 8, st));
    CK(cudaMemsetAsync(A + o_flags, 0, 2 * (size_t)tiles, st));
    for (int i = 0; i < n; i++)
        if (frames[i].edges) CK(cudaMemsetAsync(frames[i].edges, 0, (size_t)frames[i].H * frames[i].W, st));
    detect_pack_kernel<<<(unsigned)((words + 255) / 256), 256, 0, st>>>(da, (int)words);
    CK(cudaGetLastError());
    detect_classify_kernel<<<(unsigned)((tiles + 255) / 256), 256, 0, st>>>(da);
    CK(cudaGetLastError());
    if (da.cap <= DET_WARP_DIST_MAX_CAP) {
        int per_sm_w = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_w, detect_dist_warp_kernel, DET_THREADS, 0));
        const unsigned g_w = (unsigned)std::min<int64_t>((tiles + 7) / 8, (int64_t)std::max(per_sm_w, 1) * ctx->sm_count);
        detect_dist_warp_kernel<<<g_w, DET_THREADS, 0, st>>>(da);
    } else {
        detect_dist_kernel<<<g_dist, DET_THREADS, sm_dist, st>>>(da);
    }
    CK(cudaGetLastError());
    CK(launch_detect_tensor(rS, g_tensor, sm_tensor, st, da));
    detect_union_kernel<<<g_list, DET_THREADS, 0, st>>>(da);
    CK(cudaGetLastError());
    detect_mark_kernel<<<g_list, DET_THREADS, 0, st>>>(da);
    CK(cudaGetLastError());
    detect_accept_kernel<<<g_list, DET_THREADS, 0, st>>>(da);
    CK(cudaGetLastError());
    detect_scan_kernel<<<(unsigned)n, DET_SCAN_THREADS, 0, st>>>(da);
    CK(cudaGetLastError());
    detect_write_kernel<<<g_list, DET_THREADS, 0, st>>>(da);
    CK(cudaGetLastError());
    return GF_OK;
}

gf_status gf_detect_splines(gf_ctx *ctx, const gf_detect_frame *frame, const gf_detect_params *params, void *stream)
{
    return gf_detect_splines_batched(ctx, 1, frame, params, stream);
}

gf_status gf_fill_batched_splines(gf_ctx *ctx, int n, const gf_frame *frames, const gf_spline_frame *splines, float eta,
                                  const gf_params *params, gf_stats *dev_stats, void *stream, void *event_fill_start,
                                  void *event_fill_end)
{
    if (!ctx || n <= 0 || !frames || !splines || !dev_stats) return GF_ERR_ARG;
    gf_status s = check_params(params);
    if (s != GF_OK) return s;
    for (int i = 0; i < n; i++) {
        s = check_frame(&frames[i]);
        if (s != GF_OK) return s;
        const gf_spline_frame &g = splines[i];
        if (g.H != frames[i].H || g.W != frames[i].W || g.labels != frames[i].labels || g.guide != frames[i].guide)
            return GF_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    cudaStream_t st = (cudaStream_t)stream;
    if (params->flags & GF_FLAG_DATA) {
        // the init pass counts guided hole pixels: the guide field comes first
        s = gf_guidance_batched(ctx, n, splines, eta, stream);
        if (s != GF_OK) return s;
        return enqueue_fill(ctx, n, frames, params, dev_stats, st, (cudaEvent_t)event_fill_start,
                            (cudaEvent_t)event_fill_end);
    }
    // the guide field on the context's second stream, beside the fill's preparation
    // (descriptors, init pass, frame order), which does not read it; the fill kernel
    // waits for both
    CK(cudaEventRecord(ctx->fork_ev, st));
    CK(cudaStreamWaitEvent(ctx->aux, ctx->fork_ev, 0));
    s = gf_guidance_batched(ctx, n, splines, eta, ctx->aux);
    if (s != GF_OK) {
        cudaStreamSynchronize(ctx->aux);
        return s;
    }
    CK(cudaEventRecord(ctx->guide_ev, ctx->aux));
    s = enqueue_fill(ctx, n, frames, params, dev_stats, st, (cudaEvent_t)event_fill_start, (cudaEvent_t)event_fill_end,
                     true, nullptr, ctx->guide_ev);
    if (s != GF_OK) {
        CK(cudaStreamWaitEvent(st, ctx->guide_ev, 0));  // leave nothing of this call unjoined
        return s;
    }
    return GF_OK;
}

gf_status gf_guide_from_angle(gf_ctx *ctx, int H, int W, const uint8_t *labels, const float *mag, const float *phi,
                              float *guide, void *stream)
{
    if (!ctx || H <= 0 || W <= 0 || !labels || !mag || !phi || !guide) return GF_ERR_ARG;
    if ((int64_t)H * W > ((int64_t)1 << 31) - 64 || ((uintptr_t)guide & 7)) return GF_ERR_ARG;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    int64_t np = (int64_t)H * W;
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>((np + 255) / 256, (int64_t)ctx->sm_count * 16));
    angle_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(np, labels, mag, phi, (float2 *)guide);
    CK(cudaGetLastError());
    return GF_OK;
}

gf_status gf_fill_backward(gf_ctx *ctx, int n, const gf_adjoint_frame *frames, const gf_params *prm, void *stream)
{
    if (!ctx || n <= 0 || !frames) return GF_ERR_ARG;
    gf_status s = check_params(prm);
    if (s != GF_OK) return s;
    if (!(prm->flags & GF_FLAG_GHOST)) return GF_ERR_UNSUPPORTED;
    for (int i = 0; i < n; i++) {
        const gf_adjoint_frame &f = frames[i];
        if (f.H <= 0 || f.W <= 0 || (int64_t)f.H * f.W > ((int64_t)1 << 31) - 64) return GF_ERR_ARG;
        if (!f.out_rgba || !f.guide || !f.shell || !f.grad_out || !f.grad_in || !f.grad_phi || !f.grad_mu)
            return GF_ERR_ARG;
        if (((uintptr_t)f.out_rgba & 15) || ((uintptr_t)f.grad_out & 15) || ((uintptr_t)f.grad_in & 15) ||
            ((uintptr_t)f.guide & 7) || ((uintptr_t)f.shell & 3) || ((uintptr_t)f.grad_phi & 3) ||
            ((uintptr_t)f.grad_mu & 3) || (f.stall && ((uintptr_t)f.stall & 3)))
            return GF_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<size_t> o_cnt(n), o_start(n), o_order(n);
    size_t pos = 0;
    std::vector<int32_t> blk(n + 1);
    int64_t nb = 0;
    for (int i = 0; i < n; i++) {
        size_t np = (size_t)frames[i].H * frames[i].W;
        o_cnt[i] = pos; pos = align_up(pos + 4 * (np + 1), 256);
        o_start[i] = pos; pos = align_up(pos + 4 * (np + 2), 256);
        o_order[i] = pos; pos = align_up(pos + 4 * np, 256);
        blk[i] = (int32_t)nb;
        nb += (int64_t)((np + 1023) / 1024);
    }
    blk[n] = (int32_t)nb;
    if (nb >= INT32_MAX / 2) return GF_ERR_ARG;
    const size_t o_K = pos; pos = align_up(pos + 4 * (size_t)n, 256);
    const size_t o_desc = pos; pos = align_up(pos + sizeof(AdjFrameDev) * (size_t)n, 256);
    const size_t o_blk = pos; pos = align_up(pos + 4 * (size_t)(n + 1), 256);
    const size_t o_cur = pos; pos = align_up(pos + 4, 256);
    // launch shape: clusters of up to 8 CTAs, one frame per cluster at a time
    int cs = 8;
    while (cs > 1 && cs * n > ctx->sm_count) cs >>= 1;
    int maxc = 0;
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs * 64);
        cfg.blockDim = dim3(CTA_THREADS);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        while (cs >= 1) {
            at[0].val.clusterDim.x = cs;
            cfg.gridDim = dim3(cs * 64);
            if (cudaOccupancyMaxActiveClusters(&maxc, (const void *)adj_kernel, &cfg) == cudaSuccess && maxc > 0) break;
            cudaGetLastError();
            cs >>= 1;
        }
    }
    if (maxc <= 0) return GF_ERR_UNSUPPORTED;
    const int nc = std::max(1, std::min(maxc, n));
    const size_t o_cf = pos; pos = align_up(pos + 8 * (size_t)nc, 256);
    s = ensure(ctx, ctx->aarena, pos);
    if (s != GF_OK) return s;
    char *A = (char *)ctx->aarena.ptr;

    AdjArgs aa;
    memset(&aa, 0, sizeof(aa));
    aa.frames = (const AdjFrameDev *)(A + o_desc);
    aa.blk_offset = (const int32_t *)(A + o_blk);
    aa.n_frames = n;
    aa.mu = prm->mu;
    aa.coef32 = (prm->mu * prm->mu) / (2.0f * prm->eps * prm->eps);
    aa.tau = prm->snap_tau;
    aa.frame_cursor = (int32_t *)(A + o_cur);
    aa.cluster_frame = (int32_t *)(A + o_cf);
    build_tab(prm->eps, aa.tab);

    for (int c0 = 0; c0 < n; c0 += DESC_CHUNK) {
        static thread_local AdjChunk ch;
        ch.dst_frames = (AdjFrameDev *)(A + o_desc);
        ch.dst_blk = (int32_t *)(A + o_blk);
        ch.first = c0;
        ch.count = std::min(DESC_CHUNK, n - c0);
        ch.last_chunk = (c0 + ch.count == n) ? 1 : 0;
        for (int i = 0; i < ch.count; i++) {
            const gf_adjoint_frame &f = frames[c0 + i];
            AdjFrameDev d;
            d.H = f.H; d.W = f.W;
            d.out = (const float4 *)f.out_rgba;
            d.guide = (const float2 *)f.guide;
            d.shell = f.shell;
            d.stall = f.stall;
            d.grad_out = (const float4 *)f.grad_out;
            d.grad_in = (float4 *)f.grad_in;
            d.grad_phi = f.grad_phi;
            d.grad_mu = f.grad_mu;
            d.cnt = (int32_t *)(A + o_cnt[c0 + i]);
            d.start = (int32_t *)(A + o_start[c0 + i]);
            d.order = (int32_t *)(A + o_order[c0 + i]);
            d.K = (int32_t *)(A + o_K) + (c0 + i);
            ch.frames[i] = d;
            ch.blk[i] = blk[c0 + i];
        }
        ch.blk[ch.count] = blk[c0 + ch.count];
        adj_upload_kernel<<<1, 128, 0, st>>>(ch);
        CK(cudaGetLastError());
    }
    for (int i = 0; i < n; i++) {
        size_t np = (size_t)frames[i].H * frames[i].W;
        CK(cudaMemsetAsync(A + o_cnt[i], 0, 4 * (np + 1), st));
        CK(cudaMemsetAsync(frames[i].grad_mu, 0, 4, st));
    }
    CK(cudaMemsetAsync(A + o_K, 0, 4 * (size_t)n, st));
    CK(cudaMemsetAsync(A + o_cur, 0, 4, st));
    const int grid = std::max(1, std::min<int>((int)std::min<int64_t>(nb * 4, INT32_MAX), ctx->sm_count * 8));
    adj_prep_kernel<<<grid, 256, 0, st>>>(aa);
    CK(cudaGetLastError());
    adj_scan_kernel<<<n, 1024, 0, st>>>(aa);
    CK(cudaGetLastError());
    adj_scatter_kernel<<<grid, 256, 0, st>>>(aa);
    CK(cudaGetLastError());
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nc * cs));
    cfg.blockDim = dim3(CTA_THREADS);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, adj_kernel, aa));
    return GF_OK;
}

}  // extern "C"

// The in-place host-buffer fill on device-accessible host memory: the labels
// (copied in by the pass that finds the hole tiles, straight from the caller's
// buffer where the device can address it) and polylines in; the colours of the
// tiles within one tile of a hole tile and, for caller-given guide fields, the
// guide of the hole tiles read from the caller's buffers, beside the guide fields
// from the polylines and the fill's preparation; the batched fill in the
// context's launch shape (autotuned or set); then the hole pixels' colours and
// shell values written into the caller's buffers (gf_hostio.cu).
static gf_status fill_host_in_place(gf_ctx *ctx, int n, const int32_t *H, const int32_t *W,
                                    const uint8_t *const *host_labels, const int32_t *const *host_offsets,
                                    const float *const *host_pts, const int32_t *n_splines, const int32_t *n_points,
                                    float eta, int32_t *const *host_out_shell, const gf_params *params,
                                    gf_stats *host_stats, cudaStream_t st, char *A, const std::vector<size_t> &o_rgba,
                                    const std::vector<size_t> &o_lab, const std::vector<size_t> &o_g,
                                    const std::vector<size_t> &o_sh, const std::vector<size_t> &o_off,
                                    const std::vector<size_t> &o_pts, const std::vector<size_t> &o_th, size_t o_st,
                                    const std::vector<char> &from_splines, const std::vector<float4 *> &dev_host_rgba,
                                    const std::vector<const float2 *> &dev_host_guide, size_t o_spl, size_t spl_bytes)
{
    std::vector<gf_frame> fr(n);
    std::vector<gf_spline_frame> sf;
    std::vector<int32_t *> dev_host_shell(n, nullptr);
    std::vector<const uint8_t *> dev_host_labels(n, nullptr);
    // the splines of every frame: packed into the context's pinned staging buffer
    // (the previous call synchronised its stream before returning) and sent with
    // one copy, instead of two copies from pageable memory per frame
    if (spl_bytes > 0) {
        if (ctx->hstage_bytes < spl_bytes) {
            if (ctx->hstage) cudaFreeHost(ctx->hstage);
            ctx->hstage = nullptr;
            ctx->hstage_bytes = 0;
            CK(cudaHostAlloc(&ctx->hstage, spl_bytes, cudaHostAllocDefault));
            ctx->hstage_bytes = spl_bytes;
        }
        char *hs = (char *)ctx->hstage;
        for (int i = 0; i < n; i++) {
            if (!from_splines[i] || n_splines[i] <= 0) continue;
            memcpy(hs + (o_off[i] - o_spl), host_offsets[i], 4 * (size_t)(n_splines[i] + 1));
            memcpy(hs + (o_pts[i] - o_spl), host_pts[i], 8 * (size_t)n_points[i]);
        }
        CK(cudaMemcpyAsync(A + o_spl, hs, spl_bytes, cudaMemcpyHostToDevice, st));
    }
    for (int i = 0; i < n; i++) {
        const size_t np = (size_t)H[i] * W[i];
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, host_labels[i]) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer)
            dev_host_labels[i] = (const uint8_t *)pa.devicePointer;
        else {
            cudaGetLastError();
            CK(cudaMemcpyAsync(A + o_lab[i], host_labels[i], np, cudaMemcpyHostToDevice, st));
        }
        gf_frame &f = fr[i];
        f.H = H[i];
        f.W = W[i];
        f.rgba = (const float *)(A + o_rgba[i]);
        f.labels = (const uint8_t *)(A + o_lab[i]);
        f.guide = (const float *)(A + o_g[i]);
        f.out_rgba = (float *)(A + o_rgba[i]);
        f.out_shell = (int32_t *)(A + o_sh[i]);
        f.out_enter = nullptr;
        f.out_stall = nullptr;
        if (from_splines[i]) {
            gf_spline_frame g;
            g.H = H[i];
            g.W = W[i];
            g.labels = f.labels;
            g.n_splines = n_splines[i];
            g.n_points = n_points[i];
            g.offsets = (const int32_t *)(A + o_off[i]);
            g.pts = (const float *)(A + o_pts[i]);
            g.guide = (float *)(A + o_g[i]);
            g.weight = nullptr;
            sf.push_back(g);
        }
        if (cudaPointerGetAttributes(&pa, host_out_shell[i]) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer)
            dev_host_shell[i] = (int32_t *)pa.devicePointer;
        else
            cudaGetLastError();
    }
    // the frames' host-side descriptors, in launches of up to HOSTIO_MAX frames
    bool all_shell = true;
    for (int i = 0; i < n; i++) all_shell = all_shell && dev_host_shell[i];
    auto hostio = [&](int which, cudaStream_t sk) -> cudaError_t {
        for (int b = 0; b < n; b += HOSTIO_MAX) {
            HostIOArgs ha;
            memset(&ha, 0, sizeof(ha));
            int max_strips = 1;
            for (int i = b; i < std::min(n, b + HOSTIO_MAX); i++) {
                HostIOFrame &hf = ha.f[ha.n++];
                hf.H = H[i];
                hf.W = W[i];
                hf.TW = (W[i] + 7) / 8;
                hf.TH = (H[i] + 7) / 8;
                hf.labels = (uint8_t *)(A + o_lab[i]);
                hf.host_labels = dev_host_labels[i];
                hf.host_rgba = dev_host_rgba[i];
                hf.dev_rgba = (float4 *)(A + o_rgba[i]);
                hf.host_guide = dev_host_guide[i];
                hf.dev_guide = (float2 *)(A + o_g[i]);
                hf.tile_hole = (uint8_t *)(A + o_th[i]);
                hf.dev_shell = (const int32_t *)(A + o_sh[i]);
                hf.host_shell = all_shell ? dev_host_shell[i] : nullptr;
                max_strips = std::max(max_strips, hf.TH * ((hf.TW + 31) / 32));
            }
            const dim3 grid((unsigned)((max_strips + 7) / 8), (unsigned)ha.n);
            if (which == 0) hostio_holes_kernel<<<grid, 256, 0, sk>>>(ha);
            // the gather: a third of the SMs (about as fast as the guide kernel it shares
            // them with, measured on the 64 x 1080p batch: 32, 48, 64, 96 CTAs gave
            // 8.2, 8.0, 8.1, 8.2 ms per call)
            else if (which == 1) hostio_gather_kernel<<<std::max(1, ctx->sm_count / 3), 256, 0, sk>>>(ha);
            else hostio_write_back_kernel<<<grid, 256, 0, sk>>>(ha);
            cudaError_t e2 = cudaGetLastError();
            if (e2 != cudaSuccess) return e2;
        }
        return cudaSuccess;
    };
    // the hole tiles (and the labels, where the device reads them from the host)
    CK(hostio(0, st));
    gf_stats *dst = (gf_stats *)(A + o_st);
    while ((int)ctx->pipe_ev.size() < 3) {
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        ctx->pipe_ev.push_back(ev);
    }
    // the shell maps are copied on the copy stream once the init pass has written
    // them (every entry but the hole pixels' is then final), beside the fill
    cudaEvent_t ev_init = all_shell ? ctx->pipe_ev[0] : nullptr;
    gf_status s = GF_OK;
    if (!(params->flags & GF_FLAG_DATA)) {
        // beside the fill's preparation (descriptors, init pass, frame order): the
        // guide fields on the context's second stream and the colours near the holes
        // on its copy-in stream (the gather is bound by the host link, the guide
        // kernel by the SMs); the second stream then waits for the gather, so that
        // guide_ev covers both
        CK(cudaEventRecord(ctx->fork_ev, st));
        CK(cudaStreamWaitEvent(ctx->aux, ctx->fork_ev, 0));
        CK(cudaStreamWaitEvent(ctx->copy_in, ctx->fork_ev, 0));
        cudaError_t eg = hostio(1, ctx->copy_in);
        if (eg == cudaSuccess) eg = cudaEventRecord(ctx->pipe_ev[2], ctx->copy_in);
        if (eg == cudaSuccess && !sf.empty()) s = guidance_impl(ctx, ctx->garena, (int)sf.size(), sf.data(), eta, ctx->aux);
        if (s != GF_OK || eg != cudaSuccess) {
            cudaStreamSynchronize(ctx->copy_in);
            cudaStreamSynchronize(ctx->aux);
            return s != GF_OK ? s : cuda_fail(ctx, eg);
        }
        CK(cudaStreamWaitEvent(ctx->aux, ctx->pipe_ev[2], 0));
        CK(cudaEventRecord(ctx->guide_ev, ctx->aux));
        s = enqueue_fill(ctx, n, fr.data(), params, dst, st, ev_init, nullptr, true, nullptr, ctx->guide_ev);
        if (s != GF_OK) {
            CK(cudaStreamWaitEvent(st, ctx->guide_ev, 0));
            cudaStreamSynchronize(st);
            return s;
        }
    } else {
        // the init pass counts guided hole pixels: the guide fields come first
        if (!sf.empty()) {
            s = guidance_impl(ctx, ctx->garena, (int)sf.size(), sf.data(), eta, st);
            if (s != GF_OK) return s;
        }
        CK(hostio(1, st));
        s = enqueue_fill(ctx, n, fr.data(), params, dst, st, ev_init, nullptr, true, nullptr, nullptr);
        if (s != GF_OK) {
            cudaStreamSynchronize(st);
            return s;
        }
    }
    if (all_shell) {
        CK(cudaStreamWaitEvent(ctx->copy_out, ev_init, 0));
        for (int i = 0; i < n; i++)
            CK(cudaMemcpyAsync(host_out_shell[i], A + o_sh[i], 4 * (size_t)H[i] * W[i], cudaMemcpyDeviceToHost,
                               ctx->copy_out));
        CK(cudaEventRecord(ctx->pipe_ev[1], ctx->copy_out));
        CK(cudaStreamWaitEvent(st, ctx->pipe_ev[1], 0));
    }
    // the hole pixels' colours (and, after the bulk copy, their shell values)
    CK(hostio(2, st));
    if (!all_shell)
        for (int i = 0; i < n; i++)
            CK(cudaMemcpyAsync(host_out_shell[i], A + o_sh[i], 4 * (size_t)H[i] * W[i], cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(host_stats, dst, sizeof(gf_stats) * (size_t)n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return GF_OK;
}

extern "C" {

gf_status gf_fill_batched_host(gf_ctx *ctx, int n, const int32_t *H, const int32_t *W,
                               const float *const *host_rgba, const uint8_t *const *host_labels,
                               const float *const *host_guide, const int32_t *n_splines,
                               const int32_t *const *host_offsets, const int32_t *n_points,
                               const float *const *host_pts, float eta, float *const *host_out_rgba,
                               int32_t *const *host_out_shell, const gf_params *params,
                               gf_stats *host_stats, void *stream)
{
    if (!ctx || n <= 0 || !H || !W || !host_rgba || !host_labels || !host_out_rgba || !host_out_shell ||
        !host_stats)
        return GF_ERR_ARG;
    gf_status s = check_params(params);
    if (s != GF_OK) return s;
    std::vector<size_t> o_rgba(n), o_lab(n), o_g(n), o_sh(n), o_off(n), o_pts(n), o_th(n);
    std::vector<char> from_splines(n, 0);
    // In place (out_rgba == rgba) on host memory the device can address: only the
    // colours near the holes come in and only the hole pixels' colours go out
    // (fill_host_in_place); otherwise whole frames are copied both ways.
    bool sparse = true;
    std::vector<float4 *> dev_host_rgba(n, nullptr);
    std::vector<const float2 *> dev_host_guide(n, nullptr);
    size_t pos = 0;
    for (int i = 0; i < n; i++) {
        if (H[i] <= 0 || W[i] <= 0 || !host_rgba[i] || !host_labels[i] || !host_out_rgba[i] || !host_out_shell[i])
            return GF_ERR_ARG;
        if ((int64_t)H[i] * W[i] > ((int64_t)1 << 31) - 64) return GF_ERR_ARG;
        from_splines[i] = (!host_guide || !host_guide[i]) ? 1 : 0;
        if (from_splines[i]) {
            if (!n_splines || !n_points || !host_offsets || !host_pts || n_splines[i] < 0 || n_points[i] < 0)
                return GF_ERR_ARG;
            if (n_splines[i] > 0 && (!host_offsets[i] || !host_pts[i])) return GF_ERR_ARG;
            if (!(eta > 0.0f) || !std::isfinite(eta)) return GF_ERR_ARG;
        }
        size_t np = (size_t)H[i] * W[i];
        o_rgba[i] = pos; pos = align_up(pos + 16 * np, 256);
        o_lab[i] = pos; pos = align_up(pos + np, 256);
        o_g[i] = pos; pos = align_up(pos + 8 * np, 256);
        o_sh[i] = pos; pos = align_up(pos + 4 * np, 256);
        o_th[i] = pos; pos = align_up(pos + (size_t)((W[i] + 7) / 8) * ((H[i] + 7) / 8), 256);
    }
    // every frame's spline offsets and points in one block (one copy from a pinned
    // staging buffer on the in-place path)
    const size_t o_spl = pos;
    for (int i = 0; i < n; i++) {
        o_off[i] = pos; pos = align_up(pos + (from_splines[i] ? 4 * (size_t)(n_splines[i] + 1) : 0), 16);
        o_pts[i] = pos; pos = align_up(pos + (from_splines[i] ? 8 * (size_t)n_points[i] : 0), 16);
    }
    const size_t spl_bytes = pos - o_spl;
    pos = align_up(pos, 256);
    for (int i = 0; i < n && sparse; i++) {
        if (host_out_rgba[i] != host_rgba[i]) {
            sparse = false;
            break;
        }
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, host_rgba[i]) != cudaSuccess || pa.type != cudaMemoryTypeHost ||
            !pa.devicePointer) {
            cudaGetLastError();
            sparse = false;
            break;
        }
        dev_host_rgba[i] = (float4 *)pa.devicePointer;
        if (!from_splines[i]) {
            if (cudaPointerGetAttributes(&pa, host_guide[i]) != cudaSuccess || pa.type != cudaMemoryTypeHost ||
                !pa.devicePointer) {
                cudaGetLastError();
                sparse = false;
                break;
            }
            dev_host_guide[i] = (const float2 *)pa.devicePointer;
        }
    }
    const size_t o_st = pos; pos = align_up(pos + sizeof(gf_stats) * (size_t)n, 256);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    s = ensure(ctx, ctx->io, pos);
    if (s != GF_OK) return s;
    char *A = (char *)ctx->io.ptr;
    cudaStream_t st = (cudaStream_t)stream;
    if (sparse) return fill_host_in_place(ctx, n, H, W, host_labels, host_offsets, host_pts, n_splines, n_points,
                                          eta, host_out_shell, params, host_stats, st, A, o_rgba, o_lab, o_g, o_sh,
                                          o_off, o_pts, o_th, o_st, from_splines, dev_host_rgba, dev_host_guide,
                                          o_spl, spl_bytes);
    // Chunk pipeline: the frames' inputs are copied in on one stream; each chunk's
    // guide field, fill and output copies run on a stream of their own (with
    // scratch of their own) as soon as its inputs have landed, so chunks whose
    // frames have long shell chains overlap the next chunks instead of delaying
    // them.  `copy_out` only joins the chunks' streams before `stream` continues.
    const int nchunk = std::min(n, 16);
    // frames are dealt to the chunks round-robin (position q of the pipeline order
    // holds frame perm[q])
    std::vector<int> perm;
    perm.reserve(n);
    for (int c = 0; c < nchunk; c++)
        for (int i = c; i < n; i += nchunk) perm.push_back(i);
    while ((int)ctx->pipe_ev.size() < 2 * nchunk + 2) {
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        ctx->pipe_ev.push_back(ev);
    }
    while ((int)ctx->pipe_st.size() < nchunk) {
        cudaStream_t ps;
        CK(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking));
        ctx->pipe_st.push_back(ps);
    }
    if ((int)ctx->pipe_fill.size() < nchunk) ctx->pipe_fill.resize(nchunk);
    if ((int)ctx->pipe_guide.size() < nchunk) ctx->pipe_guide.resize(nchunk);
    cudaEvent_t ev_start = ctx->pipe_ev[0], ev_out_done = ctx->pipe_ev[1];
    CK(cudaEventRecord(ev_start, st));  // inputs may be written by work already on `stream`
    CK(cudaStreamWaitEvent(ctx->copy_in, ev_start, 0));
    CK(cudaStreamWaitEvent(ctx->copy_out, ev_start, 0));
    std::vector<gf_frame> fr(n);  // in pipeline order
    std::vector<gf_spline_frame> sf(n);
    for (int q = 0; q < n; q++) {
        const int i = perm[q];
        gf_frame &f = fr[q];
        f.H = H[i]; f.W = W[i];
        f.rgba = (const float *)(A + o_rgba[i]);
        f.labels = (const uint8_t *)(A + o_lab[i]);
        f.guide = (const float *)(A + o_g[i]);
        f.out_rgba = (float *)(A + o_rgba[i]);
        f.out_shell = (int32_t *)(A + o_sh[i]);
        f.out_enter = nullptr;
        f.out_stall = nullptr;
        gf_spline_frame &g = sf[q];
        g.H = H[i]; g.W = W[i];
        g.labels = (const uint8_t *)(A + o_lab[i]);
        g.n_splines = from_splines[i] ? n_splines[i] : 0;
        g.n_points = from_splines[i] ? n_points[i] : 0;
        g.offsets = (const int32_t *)(A + o_off[i]);
        g.pts = (const float *)(A + o_pts[i]);
        g.guide = (float *)(A + o_g[i]);
    }
    for (int c = 0; c < nchunk; c++) {
        const int q0 = n * c / nchunk, q1 = n * (c + 1) / nchunk;
        for (int q = q0; q < q1; q++) {
            const int i = perm[q];
            size_t np = (size_t)H[i] * W[i];
            CK(cudaMemcpyAsync(A + o_rgba[i], host_rgba[i], 16 * np, cudaMemcpyHostToDevice, ctx->copy_in));
            CK(cudaMemcpyAsync(A + o_lab[i], host_labels[i], np, cudaMemcpyHostToDevice, ctx->copy_in));
            if (!from_splines[i]) {
                CK(cudaMemcpyAsync(A + o_g[i], host_guide[i], 8 * np, cudaMemcpyHostToDevice, ctx->copy_in));
            } else if (n_splines[i] > 0) {
                CK(cudaMemcpyAsync(A + o_off[i], host_offsets[i], 4 * (size_t)(n_splines[i] + 1),
                                   cudaMemcpyHostToDevice, ctx->copy_in));
                CK(cudaMemcpyAsync(A + o_pts[i], host_pts[i], 8 * (size_t)n_points[i], cudaMemcpyHostToDevice,
                                   ctx->copy_in));
            }
        }
        CK(cudaEventRecord(ctx->pipe_ev[2 + 2 * c], ctx->copy_in));
    }
    // Unless a launch shape was set, a chunk's frames get the largest cluster size at
    // which every one of them has its own cluster and two chunks fit on the SMs at
    // once (16 CTAs for 4 frames on 152 SMs).  No split schedule: its second stream
    // and events belong to the context.
    LaunchSettingsGuard keep(ctx);
    ctx->split_m = ctx->split_cs = ctx->split_nc = 0;
    gf_status fs = GF_OK;
    for (int c = 0; c < nchunk && fs == GF_OK; c++) {
        const int q0 = n * c / nchunk, q1 = n * (c + 1) / nchunk;
        cudaStream_t cs_st = ctx->pipe_st[c];
        CK(cudaStreamWaitEvent(cs_st, ctx->pipe_ev[2 + 2 * c], 0));
        std::vector<gf_spline_frame> sfc;
        for (int q = q0; q < q1; q++)
            if (from_splines[perm[q]]) sfc.push_back(sf[q]);
        if (!sfc.empty()) {
            fs = guidance_impl(ctx, ctx->pipe_guide[c], (int)sfc.size(), sfc.data(), eta, cs_st);
            if (fs != GF_OK) break;
        }
        if (keep.cs == 0) {
            int cs = 16;
            while (cs > 1 && 2 * cs * (q1 - q0) > ctx->sm_count) cs >>= 1;
            ctx->cluster_size = cs;
            ctx->n_clusters = 0;
        }
        fs = enqueue_fill(ctx, q1 - q0, fr.data() + q0, params, (gf_stats *)(A + o_st) + q0, cs_st, nullptr, nullptr,
                          false, &ctx->pipe_fill[c]);
        ctx->cluster_size = keep.cs;
        ctx->n_clusters = keep.nc;
        if (fs != GF_OK) break;
        // the chunk's outputs leave on its own stream, so a chunk with a long shell
        // chain holds back no other chunk's copies
        for (int q = q0; q < q1; q++) {
            const int i = perm[q];
            size_t np = (size_t)H[i] * W[i];
            CK(cudaMemcpyAsync(host_out_rgba[i], A + o_rgba[i], 16 * np, cudaMemcpyDeviceToHost, cs_st));
            CK(cudaMemcpyAsync(host_out_shell[i], A + o_sh[i], 4 * np, cudaMemcpyDeviceToHost, cs_st));
        }
        CK(cudaEventRecord(ctx->pipe_ev[3 + 2 * c], cs_st));
        CK(cudaStreamWaitEvent(ctx->copy_out, ctx->pipe_ev[3 + 2 * c], 0));
    }
    CK(cudaEventRecord(ev_out_done, ctx->copy_out));
    CK(cudaStreamWaitEvent(st, ev_out_done, 0));
    if (fs != GF_OK) {
        cudaStreamSynchronize(ctx->copy_in);
        cudaStreamSynchronize(ctx->copy_out);
        for (int c = 0; c < nchunk; c++) cudaStreamSynchronize(ctx->pipe_st[c]);
        cudaStreamSynchronize(st);
        return fs;
    }
    std::vector<gf_stats> st_q(n);
    CK(cudaMemcpyAsync(st_q.data(), A + o_st, sizeof(gf_stats) * (size_t)n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int q = 0; q < n; q++) host_stats[perm[q]] = st_q[q];
    return GF_OK;
}

}  // extern "C"

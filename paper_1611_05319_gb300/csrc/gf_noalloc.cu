// gf_fill_noalloc: the fill of one frame with no device allocation.
//
// Some callers cannot call cudaMalloc: hosts that own every byte of device
// memory (a frame server or engine that sizes its pools at start-up) and hand
// libraries none, and real-time loops that must not allocate, or risk an
// allocation failure, once they run.  This entry point runs the same kernels
// as gf_fill, but the library's scratch lives in a fixed file-scope __device__
// array instead of memory from cudaMalloc.
//
// Limits: frames up to 4096 x 4096 px and 4,194,304 px in total; larger frames
// are rejected with GF_ERR_TOO_LARGE before anything is launched.  The array
// is about 11 MB and every GPU that loads the library holds it until the
// process exits.  All calls share the one array: it keeps the contents of the
// last call (everything that must start at zero is cleared by each call), and
// calls that overlap on the GPU (different streams, or different host threads,
// without ordering between them) race on it.
//
// The first call on each device looks up the array's device address and sets
// the kernels' shared-memory and cluster attributes; make that first call
// before starting any stream capture.  The address is kept for the rest of the
// process: after a cudaDeviceReset of that device, do not call this entry point
// again.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "gf_internal.cuh"

using namespace gf;

namespace gf {
void build_tab(float eps, SampleTab &tab);
}

namespace {

constexpr int NOALLOC_MAX_SIDE = 4096;
constexpr int64_t NOALLOC_MAX_PIXELS = (int64_t)1 << 22;
// ceil(W/8) * ceil(H/8) <= W*H/64 + (W+H)/8 + 1 <= 65536 + 1024 + 1 under both limits
constexpr int64_t NOALLOC_MAX_TILES = 66561;

constexpr size_t up256(size_t v) { return (v + 255) / 256 * 256; }

struct Layout {
    size_t U, Q, F, S, L, holes, gleft, icnt, desc, order, cursor, ctaoff, lists, total;
};

// scratch layout of one frame with T tiles, filled by one cluster
constexpr Layout layout(int64_t T)
{
    Layout l{};
    size_t p = 0;
    l.U = p; p = up256(p + 8 * (size_t)T);
    l.Q = p; p = up256(p + 8 * (size_t)T);
    l.F = p; p = up256(p + sizeof(TileF) * 2 * (size_t)T);
    l.S = p; p = up256(p + 4 * (size_t)T);
    l.L = p; p = up256(p + 4 * (size_t)T);
    l.holes = p; p = up256(p + 4);
    l.gleft = p; p = up256(p + 4);
    l.icnt = p; p = up256(p + 8);
    l.desc = p; p = up256(p + sizeof(FrameDev));
    l.order = p; p = up256(p + 4);
    l.cursor = p; p = up256(p + 8);  // two queue heads (order_kernel clears both)
    l.ctaoff = p; p = up256(p + 8);
    l.lists = p; p = up256(p + 4 * 3 * 9 * (size_t)T);  // three work lists of 9 slots per tile
    l.total = p;
    return l;
}

constexpr size_t NOALLOC_SCRATCH_BYTES = layout(NOALLOC_MAX_TILES).total;

}  // namespace

// The scratch.  In host code this name is a host-side stand-in, not a device
// address; the device address comes from cudaGetSymbolAddress (per device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[MAX_DEVICES] = {};
int g_cluster[MAX_DEVICES][3] = {};  // largest schedulable cluster size per window radius 4, 5, 8

int rw_of(float eps)
{
    const int R = (int)std::ceil((double)eps);
    return R <= 3 ? 4 : (R == 4 ? 5 : 8);
}

size_t smem_of(int rw)
{
    return fill_warps(rw) * (rw == 4 ? sizeof(WarpSmem<4>) : (rw == 5 ? sizeof(WarpSmem<5>) : sizeof(WarpSmem<8>)));
}

// Once per device, with that device current: the scratch's device address and
// the kernel attributes.  Returns the cuda error of the first failing call.
cudaError_t setup_device(int dev)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_addr[dev]) return cudaSuccess;
    // an error left pending by the caller's own earlier work is reported, not
    // cleared by the probes below
    cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) return pending;
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    const int rws[3] = {4, 5, 8};
    for (int i = 0; i < 3; i++) {
        const void *k = fill_kernel_entry(rws[i]);
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_of(rws[i]));
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        int best = 0;
        for (int cs = 16; cs >= 1 && best == 0; cs >>= 1) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(cs);
            cfg.blockDim = dim3(32 * fill_warps(rws[i]));
            cfg.dynamicSmemBytes = smem_of(rws[i]);
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = cs;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) cudaGetLastError();
            else if (n > 0) best = cs;
        }
        if (best == 0) return cudaErrorInvalidConfiguration;
        g_cluster[dev][i] = best;
    }
    g_scratch_addr[dev] = ptr;
    return cudaSuccess;
}

}  // namespace

extern "C" gf_status gf_fill_noalloc(const gf_frame *f, const gf_params *p, gf_stats *dev_stats, void *stream)
{
    // ---- arguments (as gf_fill), then the size limit of the fixed scratch
    if (!f || !p || !dev_stats) return GF_ERR_ARG;
    if (!(p->eps >= 1.0f && p->eps <= 7.0f) || !(p->mu >= 0.0f) || !std::isfinite(p->mu)) return GF_ERR_ARG;
    if (p->flags & ~(GF_FLAG_GHOST | GF_FLAG_SMART | GF_FLAG_RESCAN | GF_FLAG_DATA)) return GF_ERR_ARG;
    if ((p->flags & GF_FLAG_SMART) && !(p->c >= 1e-6f && p->c < 1.0f)) return GF_ERR_ARG;
    if (!(p->snap_tau >= 0.0f && p->snap_tau < 0.01f) || p->max_shells < 0) return GF_ERR_ARG;
    if (f->H <= 0 || f->W <= 0) return GF_ERR_ARG;
    if (!f->rgba || !f->labels || !f->guide || !f->out_rgba || !f->out_shell) return GF_ERR_ARG;
    if (((uintptr_t)f->rgba & 15) || ((uintptr_t)f->out_rgba & 15) || ((uintptr_t)f->guide & 7) ||
        ((uintptr_t)f->out_shell & 3) || (f->out_enter && ((uintptr_t)f->out_enter & 3)) ||
        (f->out_stall && ((uintptr_t)f->out_stall & 3)) || ((uintptr_t)dev_stats & 7))
        return GF_ERR_ARG;
    if (f->H > NOALLOC_MAX_SIDE || f->W > NOALLOC_MAX_SIDE || (int64_t)f->H * f->W > NOALLOC_MAX_PIXELS)
        return GF_ERR_TOO_LARGE;
    const int TW = (f->W + 7) / 8, TH = (f->H + 7) / 8;
    const int64_t T = (int64_t)TW * TH;
    if (T > NOALLOC_MAX_TILES) return GF_ERR_TOO_LARGE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return GF_ERR_CUDA;
    if (setup_device(dev) != cudaSuccess) return GF_ERR_CUDA;
    char *A = (char *)g_scratch_addr[dev];
    const Layout l = layout(T);
    cudaStream_t st = (cudaStream_t)stream;
    const int rw = rw_of(p->eps);
    const int cs = g_cluster[dev][rw == 4 ? 0 : (rw == 5 ? 1 : 2)];

    // ---- descriptor (by value through kernel parameters)
    FrameDev d;
    memset(&d, 0, sizeof(d));
    d.H = f->H;
    d.W = f->W;
    d.TW = TW;
    d.TH = TH;
    d.ntiles = (int32_t)T;
    const int64_t full = (int64_t)f->H * f->W + 1;
    d.max_shells = (int32_t)(p->max_shells > 0 ? std::min<int64_t>(p->max_shells, full) : full);
    d.rgba = (float4 *)f->out_rgba;
    d.labels = f->labels;
    d.guide = (const float2 *)f->guide;
    d.shell = f->out_shell;
    d.enter = f->out_enter;
    d.stall_bits = f->out_stall;
    d.stats = dev_stats;
    d.U = (unsigned long long *)(A + l.U);
    d.Qw = (unsigned long long *)(A + l.Q);
    d.F = (TileF *)(A + l.F);
    d.sched = (int32_t *)(A + l.S);
    d.holes = (int32_t *)(A + l.holes);
    d.gleft = (int32_t *)(A + l.gleft);
    d.init_list = (int32_t *)(A + l.L);
    d.init_count = (int32_t *)(A + l.icnt);
    static thread_local FrameChunk ch;
    ch.dst_frames = (FrameDev *)(A + l.desc);
    ch.dst_cta = (int32_t *)(A + l.ctaoff);
    ch.first = 0;
    ch.count = 1;
    ch.last_chunk = 1;
    ch.frames[0] = d;
    ch.cta[0] = 0;
    ch.cta[1] = init_ctas(TH, f->W);

    FillParams fp;
    memset(&fp, 0, sizeof(fp));
    fp.eps = p->eps;
    fp.mu = p->mu;
    fp.c = p->c;
    fp.tau = p->snap_tau;
    fp.coef32 = (p->mu * p->mu) / (2.0f * p->eps * p->eps);
    fp.coef64 = (double)p->mu * (double)p->mu / (2.0 * (double)p->eps * (double)p->eps);
    fp.c64 = (double)p->c;
    fp.flags = p->flags;
    fp.n_frames = 1;
    fp.list_cap = (int32_t)(9 * T);
    fp.frames = (FrameDev *)(A + l.desc);
    fp.frame_order = (int32_t *)(A + l.order);
    fp.frame_cursor = (int32_t *)(A + l.cursor);
    fp.lists = (int32_t *)(A + l.lists);
    build_tab(p->eps, fp.tab);

    // ---- clear what must start at zero (the array keeps the last call's contents)
    if (cudaMemsetAsync(A + l.holes, 0, 4, st) != cudaSuccess) return GF_ERR_CUDA;
    if (cudaMemsetAsync(A + l.gleft, 0, 4, st) != cudaSuccess) return GF_ERR_CUDA;
    if (cudaMemsetAsync(A + l.icnt, 0, 8, st) != cudaSuccess) return GF_ERR_CUDA;
    if (f->out_stall && cudaMemsetAsync(f->out_stall, 0, 4 * (((size_t)f->H * f->W + 1 + 31) / 32), st) != cudaSuccess)
        return GF_ERR_CUDA;
    if (f->out_rgba != f->rgba &&
        cudaMemcpyAsync(f->out_rgba, f->rgba, (size_t)f->H * f->W * 16, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return GF_ERR_CUDA;

    // ---- the kernels of gf_fill
    upload_frames_kernel<<<1, 128, 0, st>>>(ch);
    InitArgs ia;
    ia.frames = fp.frames;
    ia.cta_offset = (const int32_t *)(A + l.ctaoff);
    ia.n_frames = 1;
    ia.uniform_ctas = 0;
    ia.flags = p->flags;
    init_kernel<<<(unsigned)ch.cta[1], 32 * INIT_WARPS, 0, st>>>(ia);
    order_kernel<<<1, 256, 0, st>>>(fp.frames, 1, fp.frame_order, fp.frame_cursor);
    if (cudaGetLastError() != cudaSuccess) return GF_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cs);
    cfg.blockDim = dim3(32 * fill_warps(rw));
    cfg.dynamicSmemBytes = smem_of(rw);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (launch_fill(rw, cfg, fp) != cudaSuccess) return GF_ERR_CUDA;
    return GF_OK;
}

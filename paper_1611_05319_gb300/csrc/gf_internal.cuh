// Internal device-side structures of the Guidefill library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/guidefill.h"

namespace gf {

constexpr int TILE = 8;              // 8x8 pixel tiles; one 64-bit mask per tile
constexpr int MAX_SAMPLES = 224;     // lattice points with n^2+m^2 <= 64, minus the origin
constexpr int MAX_R = 8;             // ceil(eps) <= 8
constexpr int WARPS_PER_CTA = 16;
constexpr int CTA_THREADS = WARPS_PER_CTA * 32;
// Warps per CTA of the fill kernel: 16, or 12 for the 24x24 window (eps > 4),
// whose state-window loads need more than the 128 registers a thread gets at
// 16 warps.
__host__ __device__ constexpr int fill_warps(int rw) { return rw == 8 ? 12 : 16; }
// init kernel: CTAs of a frame (INIT_WARPS warps, one strip of 8 rows x 256 columns each)
constexpr int INIT_WARPS = 8;
__host__ __device__ inline int init_ctas(int TH, int W) {
    const int strips = ((W + 7) / 8 + 31) / 32;
    return (TH * strips + INIT_WARPS - 1) / INIT_WARPS;
}

// Per-pixel state word (out_shell): readable at step k  <=>  (uint)(s+1) < (uint)(k+1)
constexpr int32_t SH_KNOWN = -1;
constexpr int32_t SH_UNFILLED = -2;
constexpr int32_t SH_BYST = -3;
constexpr int32_t SH_OUTSIDE = -4;   // only inside staged windows

__host__ __device__ inline bool readable_at(int32_t s, int32_t k) {
    return (uint32_t)(s + 1) < (uint32_t)(k + 1);
}

// Sample table of the eps-ball (origin excluded).  The fast path walks the
// samples grouped by |m| (the weight of a rotated sample depends on m only);
// the FP64 re-check walks them in canonical order (m ascending, n ascending).
struct SampleTab {
    int ns;                      // number of samples
    int nsp;                     // ns rounded up to a multiple of 32; entries ns.. are (0, 0) with weight 0
    int R;                       // ceil(eps)
    int m_start[MAX_R + 2];      // group |m| = g occupies [m_start[g], m_start[g+1])
    float Dm[MAX_R + 1];         // sum of 1/|(n,m)| over group g
    float n_f[MAX_SAMPLES];      // grouped order
    float m_f[MAX_SAMPLES];
    float invd[MAX_SAMPLES];     // 1 / sqrt(n^2 + m^2)
    int8_t cn[MAX_SAMPLES];      // canonical order
    int8_t cm[MAX_SAMPLES];
};

// Per-warp shared memory of the fill kernel: the staged (8 + 2 RW)^2 window
// around one 8x8 tile.
template <int RW>
struct WarpSmem {
    static constexpr int WS = TILE + 2 * RW;
    float4 col[WS * WS + 1];     // colour window (cp.async); the extra last entry stays zero
    float2 guide[64];            // guide vectors of the tile's candidate pixels
    uint32_t rowmask[WS];        // readable bits of the window rows
    float4 colr[64];             // fill value of each ready (or re-checked) pixel
    float eg[32][MAX_R + 1];     // per pixel slot of a pass: e^(-beta g^2) for g = |m| = 0..R
    unsigned long long ready;
    unsigned long long recheck;   // pixels whose ready test is re-done in FP64
    uint8_t plist[64];           // the tile's front pixels in increasing order
};

struct TileF {                    // fills of one tile at one step
    unsigned long long mask;
    int32_t tag;                  // step index the mask belongs to
    int32_t pad;
};

// One frame as seen by the kernels.
struct FrameDev {
    int32_t H, W, TW, TH, ntiles;
    int32_t max_shells;
    float4 *rgba;                 // working image (out_rgba)
    const uint8_t *labels;
    const float2 *guide;
    int32_t *shell;
    int32_t *enter;               // optional
    uint32_t *stall_bits;         // optional
    gf_stats *stats;
    // scratch (library-owned)
    unsigned long long *U;        // unfilled hole pixels per tile
    unsigned long long *Qw;       // front pixels (active boundary, unfilled) per tile
    TileF *F;                     // [2][ntiles]
    int32_t *sched;               // last step the tile was scheduled for
    int32_t *holes;               // |D_h| (written by the init kernel)
    int32_t *init_list;           // tiles holding part of d_active D^(0)_h (written by the init kernel)
    int32_t *init_count;          // [0] tiles on init_list, [1] |d_active D^(0)_h|
    int32_t *gleft;               // GF_FLAG_DATA: unfilled hole pixels with g != 0 (init kernel, then fills)
};

// Per-cluster control block (in the shared memory of the cluster's first CTA,
// used by every CTA through distributed shared memory).  Counters are indexed by
// the step that writes them (mod 3) so that no counter is reset while another
// CTA of the cluster may still read it.
struct GroupCtl {
    // Per-step counters live in slot s%3 for step s.  During step s the slot of
    // step s+1 (and the work-list count of step s+2) is cleared, so a slot is
    // never cleared while a warp of the cluster may still read it.
    int32_t list_count[3];        // work list consumed by step s lives in slot s%3
    int32_t cursor[3];            // hand-out cursor of the items of step s beyond the warp count
    int32_t filled[3];            // fills of step s (evaluation pass, then stall pass if any)
    int32_t front_delta[3];       // net change of the front size during step s
    int32_t evals[3];             // front pixels evaluated at step s (evaluation pass only)
    int32_t err[3];
    int32_t rechecks;             // FP64 re-checks of the current frame (statistics only)
    int32_t cur_frame[2];
    int32_t pad[3];
};

struct FillParams {
    float eps, mu, c, tau;
    float coef32;                 // mu^2 / (2 eps^2), FP32
    double coef64;                // mu^2 / (2 eps^2), FP64 (same expression as the host)
    double c64;
    uint32_t flags;
    int32_t n_frames;             // frames of this launch: frame_order[order_first .. order_first + n_frames)
    int32_t list_cap;             // capacity of each work list (max ntiles)
    int32_t order_first;
    FrameDev *frames;
    int32_t *frame_order;         // all frames of the request, largest hole first (device)
    int32_t *frame_cursor;        // this launch's work queue head
    int32_t *lists;               // [n_clusters][3][list_cap]
    SampleTab tab;
};

// init kernel arguments: CTA b belongs to frame f with cta_offset[f] <= b < cta_offset[f+1]
struct InitArgs {
    const FrameDev *frames;
    const int32_t *cta_offset;
    int32_t n_frames;
    uint32_t flags;
    int32_t uniform_ctas;         // CTAs of every frame when all frames take the same number, else 0
};

// guide-field sampler
constexpr int BIN = 32;       // bins of 32x32 pixels
constexpr int BIN_CAP = 256;  // segments listed per bin before falling back to a full scan

struct SplineFrameDev {
    int32_t H, W, NBX, NBY;
    int32_t n_splines, n_points;
    const uint8_t *labels;
    const int32_t *offsets;
    const float2 *pts;
    float2 *guide;
    int32_t *bin_count;  // [NBX*NBY]
    int32_t *bin_list;   // [NBX*NBY*BIN_CAP]
    double *seg64;       // [n_points][8]: per segment start a, v = b - a, 1/(|v|*|v|), v/|v| (FP64)
};

struct GuideArgs {
    const SplineFrameDev *frames;
    const int32_t *point_offset;  // [n+1] first global point of each frame
    const int32_t *bin_offset;    // [n+1] first global bin of each frame
    int32_t n_frames;
    int32_t total_bins;
    float eta;
    double k2;                    // 1 / (2 eta^2) in FP64
};

constexpr int DESC_CHUNK = 128;  // frame descriptors per upload kernel

// adjoint
struct AdjFrameDev {
    int32_t H, W;
    const float4 *out;        // forward output image
    const float2 *guide;
    const int32_t *shell;
    const uint32_t *stall;    // optional stall bitmap
    const float4 *grad_out;
    float4 *grad_in;
    float *grad_phi;
    float *grad_mu;           // one float per frame
    int32_t *cnt;             // [H*W+1]: histogram, then scatter cursor
    int32_t *start;           // [H*W+2]
    int32_t *order;           // [H*W]
    int32_t *K;
};

struct AdjArgs {
    const AdjFrameDev *frames;
    const int32_t *blk_offset;    // [n+1] first 1024-pixel block of each frame
    int32_t n_frames;
    float mu, coef32, tau;
    int32_t *frame_cursor;
    int32_t *cluster_frame;       // [2 * clusters]
    SampleTab tab;
};

struct AdjChunk {
    AdjFrameDev *dst_frames;
    int32_t *dst_blk;
    int32_t first, count, last_chunk, pad;
    AdjFrameDev frames[DESC_CHUNK];
    int32_t blk[DESC_CHUNK + 1];
};

__global__ void adj_upload_kernel(const __grid_constant__ AdjChunk c);
__global__ void adj_prep_kernel(const __grid_constant__ AdjArgs a);
__global__ void adj_scan_kernel(const __grid_constant__ AdjArgs a);
__global__ void adj_scatter_kernel(const __grid_constant__ AdjArgs a);
__global__ void adj_kernel(const __grid_constant__ AdjArgs a);

// Descriptor upload by value through kernel parameters: no host staging buffer
// whose lifetime would have to outlast an asynchronous copy or a graph replay.
struct FrameChunk {
    FrameDev *dst_frames;
    int32_t *dst_cta;
    int32_t first, count, last_chunk, pad;
    FrameDev frames[DESC_CHUNK];
    int32_t cta[DESC_CHUNK + 1];
};
struct SplineChunk {
    SplineFrameDev *dst_frames;
    int32_t *dst_po, *dst_bo;
    int32_t first, count, last_chunk, pad;
    SplineFrameDev frames[DESC_CHUNK];
    int32_t po[DESC_CHUNK + 1];
    int32_t bo[DESC_CHUNK + 1];
};
__global__ void upload_frames_kernel(const __grid_constant__ FrameChunk c);
__global__ void upload_splines_kernel(const __grid_constant__ SplineChunk c);

// Host-side inputs of the in-place host-buffer fill (gf_hostio.cu).
struct HostIOFrame {
    int32_t H, W, TW, TH;
    uint8_t *labels;              // device
    const uint8_t *host_labels;   // caller's host labels (device-accessible) to copy in, or nullptr
    float4 *host_rgba;            // caller's host colours (device-accessible) to gather near holes, or nullptr
    float4 *dev_rgba;             // device working image
    const float2 *host_guide;     // caller's host guide field (device-accessible), or nullptr
    float2 *dev_guide;
    uint8_t *tile_hole;           // device scratch [TW * TH]
    const int32_t *dev_shell;     // device shell map (hostio_write_back_kernel)
    int32_t *host_shell;          // caller's host shell map (device-accessible), or nullptr
};
constexpr int HOSTIO_MAX = 16;    // frames per launch
struct HostIOArgs {
    int32_t n, pad;
    HostIOFrame f[HOSTIO_MAX];
};
__global__ void hostio_holes_kernel(const __grid_constant__ HostIOArgs a);
__global__ void hostio_gather_kernel(const __grid_constant__ HostIOArgs a);
__global__ void hostio_write_back_kernel(const __grid_constant__ HostIOArgs a);

// Host-side entry points of the templated fill kernel (defined beside it).
const void *fill_kernel_entry(int rw);
cudaError_t launch_fill(int rw, const cudaLaunchConfig_t &cfg, const FillParams &p);
__global__ void init_kernel(const __grid_constant__ InitArgs a);
// sorts the frames by hole size (largest first) into `order`; clears the two
// work-queue heads cursor[0..1]
__global__ void order_kernel(const FrameDev *frames, int n, int32_t *order, int32_t *cursor);
__global__ void angle_kernel(int64_t npx, const uint8_t *labels, const float *mag, const float *phi,
                             float2 *guide);
__global__ void bin_kernel(const __grid_constant__ GuideArgs a, int total_points);
__global__ void guide_kernel(const __grid_constant__ GuideArgs a);

}  // namespace gf
